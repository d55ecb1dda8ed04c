// noalloc.cu -- a bucket-offset build that allocates no device memory.
//
// Why this exists: the regular entry points draw their scratch from the
// context's workspace, which grows with cudaMalloc on first use.  Some callers
// cannot call cudaMalloc (or cudaFree) at the point where they need the
// offsets: code that runs while a stream is being captured into a CUDA graph,
// code inside a memory budget that forbids new allocations after start-up,
// or a real-time loop where a blocking allocation is not acceptable.  For them
// idl_bucket_offsets_noalloc keeps its scratch in a file-scope __device__
// array of fixed size, reserved when the library is loaded.
//
// The scratch (the per-bucket scatter cursor, the list of oversized buckets and
// its count) is shared by every call in the process on that device and keeps
// the last call's contents: each call clears what must start at zero, so calls
// that overlap on the GPU (two streams at once, or two threads) race on it.
#include <cuda_runtime.h>

#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace idl {

// The kernels of the regular bucket-offset build (draws.cu).
__global__ void bucket_hist_kernel(const int32_t* __restrict__ h, int64_t I, int64_t L, int32_t* __restrict__ cnt,
                                   int* status);
__global__ void bucket_scan_kernel(const int32_t* cnt, int64_t L, int32_t* __restrict__ ptr, int32_t* cursor);
__global__ void bucket_scatter_kernel(const int32_t* __restrict__ h, int64_t I, int64_t L,
                                      int32_t* __restrict__ cursor, int32_t* __restrict__ row_list);
__global__ void bucket_sort_warp_kernel(const int32_t* __restrict__ ptr, int64_t L, int32_t* __restrict__ row_list,
                                        int32_t* __restrict__ big, int32_t* __restrict__ nbig);
__global__ void bucket_sort_block_kernel(const int32_t* __restrict__ ptr, int32_t* __restrict__ row_list,
                                         const int32_t* __restrict__ big, const int32_t* __restrict__ nbig,
                                         const int32_t* __restrict__ h, int64_t I);

namespace {

constexpr int64_t kMaxBuckets = IDL_NOALLOC_MAX_BUCKETS;
// layout (int32 words): cursor[kMaxBuckets + 1] | big[kMaxBuckets + 1] | nbig | pad
constexpr int64_t kWords = 2 * (kMaxBuckets + 1) + 4;

__device__ __align__(256) int32_t g_noalloc_scratch[kWords];

struct DeviceScratch {
  int32_t* base = nullptr;  // device address of g_noalloc_scratch on that device
  int num_sms = 0;
  bool ready = false;
};
constexpr int kMaxDevices = 64;
DeviceScratch g_dev[kMaxDevices];
std::mutex g_mu;

// Once per device, with that device current: look up the array's device
// address (the host-side name is only a stand-in) and the SM count.
int setup_current_device(DeviceScratch** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    (void)cudaGetLastError();
    return IDL_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  DeviceScratch& d = g_dev[dev];
  if (!d.ready) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
      (void)cudaGetLastError();
      return IDL_ECUDA;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
      (void)cudaGetLastError();
      return IDL_ECUDA;
    }
    d.base = (int32_t*)p;
    d.num_sms = sms;
    d.ready = true;
  }
  *out = &d;
  return IDL_OK;
}

}  // namespace
}  // namespace idl

using namespace idl;

extern "C" int idl_bucket_offsets_noalloc(void* stream, const int32_t* h, int64_t I, int64_t L, int32_t* bucket_ptr,
                                          int32_t* row_list) {
  if (I < 0 || I > 0x7fffffffLL || L < 1 || !bucket_ptr || (I > 0 && (!h || !row_list))) return IDL_EINVAL;
  if (L > kMaxBuckets) return IDL_ELIMIT;
  DeviceScratch* d = nullptr;
  int rc = setup_current_device(&d);
  if (rc != IDL_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  int32_t* cursor = d->base;
  int32_t* big = d->base + (kMaxBuckets + 1);
  int32_t* nbig = big + (kMaxBuckets + 1);
  // the counters and the oversized-bucket count must start at zero on every call
  if (cudaMemsetAsync(cursor, 0, sizeof(int32_t) * (size_t)L, st) != cudaSuccess ||
      cudaMemsetAsync(nbig, 0, sizeof(int32_t), st) != cudaSuccess) {
    (void)cudaGetLastError();
    return IDL_ECUDA;
  }
  {
    const int threads = 512;
    int64_t blocks = cdiv(I, threads * 8);
    if (blocks > 4 * d->num_sms) blocks = 4 * d->num_sms;
    if (blocks < 1) blocks = 1;
    const size_t sm = L <= 12288 ? sizeof(int32_t) * (size_t)L : 0;
    // no status word: out-of-range entries of h show as bucket_ptr[L] < I
    bucket_hist_kernel<<<(unsigned)blocks, threads, sm, st>>>(h, I, L, cursor, nullptr), count_launch();
  }
  bucket_scan_kernel<<<1, 1024, 0, st>>>(cursor, L, bucket_ptr, cursor), count_launch();
  if (I > 0) bucket_scatter_kernel<<<(unsigned)cdiv(I, 256), 256, 0, st>>>(h, I, L, cursor, row_list), count_launch();
  const int warps = 8;
  bucket_sort_warp_kernel<<<(unsigned)cdiv(L, warps), warps * 32, sizeof(int32_t) * warps * 1024, st>>>(
      bucket_ptr, L, row_list, big, nbig), count_launch();
  bucket_sort_block_kernel<<<64, 512, sizeof(int32_t) * 12288, st>>>(bucket_ptr, row_list, big, nbig, h, I),
      count_launch();
  if (cudaGetLastError() != cudaSuccess) return IDL_ECUDA;
  return IDL_OK;
}
