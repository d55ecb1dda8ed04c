#!/usr/bin/env python
"""Throughput of the CountSketch interpolative decomposition on one GB300.

One step = one full ID through the C ABI (id_matrix_csr / id_matrix /
id_cp_tensor): draws, bucket offsets, the sketch, the Gaussian stage, the
pivoted QR, the FP64 T solve and the FP64 residual -- every stage of the hot
path, on a seeded synthetic workload shaped like the paper's experiments.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload sparse|dense64|mixed|cp]

Prints one JSON line (rank 0).  Under torchrun every rank solves its own
problem instance (independent draws) with no collective on the data path;
value = solves of all ranks / max-over-ranks time ("weak" scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "ID solves/sec and sketch HBM GB/s at rel err<=1e-3, learned vs plain, 1 GB300"
FALLBACK_HBM_GBS = 6800.0

WORKLOADS = {
    "sparse": dict(
        desc="sparse matrix ID, fp32: CSR A 1,000,000 x 10,000, density 1e-3 uniform positions N(0,1) values, "
             "plus a rank-50 dense term of scale 10 on 1% of rows; k=50, CountSketch m1=3600 (modified), "
             "Gaussian m2=60 (FP32-accurate), T in FP64",
        I=1_000_000, R=10_000, k=50, m1=3600, m2=60, dtype="f32", precision="FP32", seed=20190131),
    "sparse_small": dict(
        desc="sparse matrix ID, fp32, profiling case: CSR A 200,000 x 10,000 built like the sparse workload "
             "(density 1e-3 plus the rank-50 term on 1% of rows); k=50, m1=3600, m2=60",
        I=200_000, R=10_000, k=50, m1=3600, m2=60, dtype="f32", precision="FP32", seed=20190134),
    "dense64": dict(
        desc="plain matrix ID, fp64: dense A 4000 x 2000 = U diag(0.8^i) V^T + 1e-8 N(0,1); k=20, m1=900, m2=30",
        I=4000, R=2000, k=20, m1=900, m2=30, dtype="f64", precision="FP64", seed=20190130),
    "mixed": dict(
        desc="large dense matrix ID, mixed precision: A 131072 x 4096 fp32 rank 100 + 1e-4 relative noise; k=100, "
             "m1=14400, Gaussian m2=120 in BF16X3 (bf16 tensor cores, FP32 accumulate), T in FP64",
        I=131072, R=4096, k=100, m1=14400, m2=120, dtype="f32", precision="BF16X3", seed=20190132),
    "cp": dict(
        desc="CP tensor ID: 3-way 1000^3 CP tensor, R=1000 N(0,1) unit-norm factors, lambda_r=0.9^r; k=50, "
             "TensorSketch L=8192 per mode, Gaussian m2=60, T in FP64",
        dims=(1000, 1000, 1000), R=1000, k=50, m1=8192, m2=60, dtype="f32", precision="FP32", seed=20190133),
    "batched": dict(
        desc="batched: 256 dense FP32 matrices (rows log-uniform 2048-65536, cols log-uniform 256-2048, rank r in "
             "8..64, sigma_i = d^i with d in [0.7, 0.95], 1e-6 relative noise; k=r, m2=k+10, m1=min(m2^2, rows/2)) "
             "plus 64 four-way CP tensors (dims 200, R=5000, N(0,1) unit-norm factors, lambda_r=10^(-6(r-1)/K) for "
             "r<=K then 1e-6, K cycling 16/32/48/64; L=8192, m2=K+10); one batch call per step",
        n_dense=256, n_cp=64, R=0, k=0, m1=0, m2=0, dtype="f32", precision="BF16X3", seed=20190134),
}


# ----------------------------------------------------------------------------- helpers
def max_over_ranks(x: float, dist, device: str) -> float:
    """The maximum of x over all ranks (x itself without a process group)."""
    if not dist:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_seed(w: dict, rank: int) -> int:
    """Each rank solves its own instance: independent draws per rank."""
    return w["seed"] + 1000 * rank


def job_value(ws: int, steps: int, solves_per_step: int, seconds: float) -> float:
    """Whole-job throughput: the solves of all ranks over the slowest rank's time."""
    return ws * steps * solves_per_step / seconds


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": FALLBACK_HBM_GBS}, "fallback"


def recorded_traffic(kernel: str, workload: str, sources):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary, if none of
    the kernel's source files changed since the counters were taken (else None).
    The summary's source_sha256 is the SHA-256 of the files' bytes concatenated in
    the order given."""
    path = os.path.join(ROOT, "profiles", f"traffic_{kernel}_{workload}.txt")
    if not os.path.exists(path):
        return None
    kv = {}
    for line in open(path):
        if ":" in line and not line.startswith("#"):
            a, b = line.split(":", 1)
            kv[a.strip()] = b.strip()
    if isinstance(sources, str):
        sources = [sources]
    h = hashlib.sha256()
    for src in sources:
        h.update(open(os.path.join(ROOT, "paper_1901_10559_gb300", "csrc", src), "rb").read())
    if kv.get("source_sha256") != h.hexdigest():
        return None
    try:
        return float(kv["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def fp32_peak_tflops(sms: int, mhz: float) -> float:
    """FP32 ALU peak: SMs x 128 FP32 lanes x 2 flop per FMA x SM clock."""
    return sms * 128 * 2 * mhz * 1e6 / 1e12


def ts_flops(R: int, N: int, L: int) -> float:
    """Algorithmic FLOP of one TensorSketch of R columns: ceil(R/2) column pairs, N + 1
    complex length-L FFTs per pair, 5 L log2 L each (the usual FFT count)."""
    return ((R + 1) // 2) * (N + 1) * 5.0 * L * np.log2(L)


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


# ----------------------------------------------------------------------------- workloads
def make_inputs(name: str, rank: int = 0):
    import synth
    w = WORKLOADS[name]
    if name == "batched":
        dense, cps = make_batch(w["seed"], rank, w["n_dense"], w["n_cp"])
        return {"dense": dense, "cps": cps}
    if name in ("sparse", "sparse_small"):
        c = synth.sparse_plus_lowrank_csr(w["I"], w["R"], 1e-3, rank=50, scale=10.0, dense_frac=0.01, seed=w["seed"])
        return {"csr": c}
    if name == "dense64":
        return {"A": synth.lowrank_dense(w["I"], w["R"], 0.8, 1e-8, seed=w["seed"], dtype=np.float64)}
    if name == "mixed":
        return {"A": synth.gaussian_lowrank_dense(w["I"], w["R"], 100, 1e-4, seed=w["seed"])}
    facs, lam = synth.cp_factors(w["dims"], w["R"], seed=w["seed"])
    return {"factors": facs, "lam": lam}


def sketch_bytes(name: str, inp) -> float:
    """Algorithmic bytes of one launch of the sketch kernel (reads once, writes once)."""
    w = WORKLOADS[name]
    if name in ("sparse", "sparse_small"):
        c = inp["csr"]
        I, R = c.shape
        return (8.0 * c.nnz                       # colidx int32 + vals fp32
                + 8.0 * (I + 1)                   # rowptr int64
                + 4.0 * I + 1.0 * I               # row list int32, signs int8
                + 4.0 * (w["m1"] + 1)             # bucket pointers
                + 4.0 * w["m1"] * R)              # Y1 fp32 written
    if name in ("dense64", "mixed"):
        es = 8 if w["dtype"] == "f64" else 4
        I, R = w["I"], w["R"]
        return es * I * R + 5.0 * I + 4.0 * (w["m1"] + 1) + es * w["m1"] * R
    if name == "batched":      # the dense items' sketch (one launch over all of them)
        tot = 0.0
        for pr in inp["dense"]:
            I, R = pr["A"].shape
            tot += 4.0 * I * R + 5.0 * I + 4.0 * (pr["m1"] + 1) + 4.0 * pr["m1"] * R
        return tot
    R = w["R"]
    return 4.0 * sum(w["dims"]) * R + 5.0 * sum(w["dims"]) + 4.0 * w["m1"] * R


# ----------------------------------------------------------------------------- batched workload
def make_batch(seed, rank=0, n_dense=256, n_cp=64):
    """Seeded synthetic batch, generated on the GPU (16 GB of dense matrices)."""
    import torch
    import synth
    g = torch.Generator(device="cuda").manual_seed(seed + 7 * rank)
    dense = []
    for spec in synth.batch_matrix_specs(n_dense, seed):
        I, R, r, d = spec["I"], spec["R"], spec["rank"], spec["decay"]
        U = torch.randn(I, r, device="cuda", generator=g) / np.sqrt(I)
        V = torch.randn(R, r, device="cuda", generator=g) / np.sqrt(R)
        sig = torch.tensor([d ** (i + 1) for i in range(r)], device="cuda", dtype=torch.float32)
        A = (U * sig) @ V.T
        A += (1e-6 * d / np.sqrt(max(I, R))) * torch.randn(I, R, device="cuda", generator=g)
        m2 = r + 10
        dense.append(dict(A=A.contiguous(), K=r, m1=min(m2 * m2, I // 2), m2=m2, seed=spec["seed"]))
    cps = []
    for b in range(n_cp):
        K = (16, 32, 48, 64)[b % 4]
        R = 5000
        facs = []
        for _ in range(4):
            F = torch.randn(R, 200, device="cuda", generator=g)
            facs.append((F / F.norm(dim=1, keepdim=True)).contiguous())
        lam = torch.from_numpy(synth.batch_cp_lambda(R, K)).cuda()
        cps.append(dict(facs=facs, lam=lam, K=K, L=8192, m2=K + 10, seed=seed * 10 + b))
    return dense, cps


def copy_floor_ms(host_tensors, reps: int = 2) -> float:
    """Milliseconds to copy these pinned host tensors to the device with plain copies,
    one after another into a reused device buffer: the host link's floor under the
    end-to-end number (untimed for the metric itself)."""
    import torch
    srcs = [t.contiguous().view(torch.uint8).reshape(-1) for t in host_tensors]
    dst = torch.empty(max(x.numel() for x in srcs), dtype=torch.uint8, device="cuda")
    for x in srcs:
        dst[:x.numel()].copy_(x, non_blocking=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        for x in srcs:
            dst[:x.numel()].copy_(x, non_blocking=True)
    torch.cuda.synchronize()
    return (time.perf_counter() - t0) / reps * 1e3


def precision_code(idl, name):
    """IDL_PREC_* of a precision mode's name."""
    return {"FP64": idl.PREC_FP64, "FP32": idl.PREC_FP32, "BF16X3": idl.PREC_BF16X3, "BF16": idl.PREC_BF16,
            "TF32X3": idl.PREC_TF32X3}[name]


def batch_items(idl, dense, cps, prec, learned=0):
    import torch
    items, outs = [], []
    for pr in dense:
        K, R = pr["K"], pr["A"].shape[1]
        J = torch.empty(K, dtype=torch.int32, device="cuda")
        T = torch.empty(K * (R - K), dtype=torch.float64, device="cuda")
        p = idl.make_params(pr["m1"], pr["m2"], seed=pr["seed"], modified=True, precision=prec, learned=learned)
        items.append(idl.dense_item(pr["A"], K, p, J, T))
        outs.append((J, T, None))
    for pr in cps:
        K, R = pr["K"], pr["facs"][0].shape[0]
        J = torch.empty(K, dtype=torch.int32, device="cuda")
        T = torch.empty(K * (R - K), dtype=torch.float64, device="cuda")
        lh = torch.empty(K, dtype=torch.float64, device="cuda")
        p = idl.make_params(pr["L"], pr["m2"], seed=pr["seed"], modified=False, precision=prec, learned=learned)
        items.append(idl.cp_item(pr["facs"], pr["lam"], K, p, J, T, lh))
        outs.append((J, T, lh))
    return items, outs


# ----------------------------------------------------------------------------- our arm
def run_ours(args, ws, rank, local):
    import torch
    import paper_1901_10559_gb300 as idl
    from paper_1901_10559_gb300 import build as b
    b.build()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    name = args.workload
    w = WORKLOADS[name]
    inp = make_inputs(name, rank)
    ctx = idl.Context(local)
    # repeated pipeline calls with the same arguments replay as CUDA graphs (the warm-up
    # steps run the eager call and the capture; the batch call has its own graph)
    idl.idl_set_graphs(ctx, True)
    prec = precision_code(idl, w["precision"])
    seed = rank_seed(w, rank)                         # independent draws per rank
    p = idl.make_params(w["m1"], w["m2"], seed=seed, modified=(name != "cp"), precision=prec, residual=1)
    K = max(1, w["k"])
    R = max(2, w["R"])
    J = torch.empty(K, dtype=torch.int32, device="cuda")
    T = torch.empty(K * (R - K), dtype=torch.float64, device="cuda")
    lh = torch.empty(K, dtype=torch.float64, device="cuda")

    if name in ("sparse", "sparse_small"):
        c = inp["csr"]
        d_rp, d_ci, d_v = (torch.from_numpy(c.rowptr).cuda(), torch.from_numpy(c.colidx).cuda(),
                           torch.from_numpy(c.vals).cuda())
        h_rp, h_ci, h_v = (torch.from_numpy(c.rowptr).pin_memory(), torch.from_numpy(c.colidx).pin_memory(),
                           torch.from_numpy(c.vals).pin_memory())
        in_bytes = c.rowptr.nbytes + c.colidx.nbytes + c.vals.nbytes
        host_inputs = [h_rp, h_ci, h_v]

        def step(J, T, lh, host_in=False):
            if host_in:
                idl.id_matrix_csr(ctx, h_rp, h_ci, h_v, c.shape, K, p, J, T)
            else:
                idl.id_matrix_csr(ctx, d_rp, d_ci, d_v, c.shape, K, p, J, T)
    elif name in ("dense64", "mixed"):
        A = inp["A"]
        d_A = torch.from_numpy(A).cuda()
        h_A = torch.from_numpy(A).pin_memory()
        in_bytes = A.nbytes
        host_inputs = [h_A]

        def step(J, T, lh, host_in=False):
            idl.id_matrix(ctx, h_A if host_in else d_A, K, p, J, T)
    else:
        facs, lam = inp["factors"], inp["lam"]
        d_f = [torch.from_numpy(np.ascontiguousarray(F.T)).cuda() for F in facs]
        h_f = [torch.from_numpy(np.ascontiguousarray(F.T)).pin_memory() for F in facs]
        d_lam = torch.from_numpy(lam).cuda()
        h_lam = torch.from_numpy(lam).pin_memory()
        in_bytes = sum(F.nbytes for F in facs) + lam.nbytes
        host_inputs = h_f + [h_lam]

        def step(J, T, lh, host_in=False):
            if host_in:     # host factors and s-values: the call stages them itself
                idl.id_cp_tensor(ctx, h_f, h_lam, K, p, J, T, lh)
            else:
                idl.id_cp_tensor(ctx, d_f, d_lam, K, p, J, T, lh)

    # the same step with the QR stage's learned column proposal (shipped MLP weights)
    idl.idl_load_weights(ctx, idl.PROPOSAL_WEIGHTS)
    p_l = idl.make_params(w["m1"], w["m2"], seed=seed, modified=(name != "cp"), precision=prec, residual=1,
                          learned=idl.PROPOSAL_MLP)
    if name in ("sparse", "sparse_small"):
        def step_learned():
            idl.id_matrix_csr(ctx, d_rp, d_ci, d_v, c.shape, K, p_l, J, T)
    elif name in ("dense64", "mixed"):
        def step_learned():
            if w["dtype"] == "f32":
                idl.id_matrix(ctx, d_A, K, p_l, J, T)
    else:
        def step_learned():
            idl.id_cp_tensor(ctx, d_f, d_lam, K, p_l, J, T, lh)

    for _ in range(args.warmup):
        step(J, T, lh)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    n0 = idl.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(args.steps):
        step(J, T, lh)
    e1.record()
    torch.cuda.synchronize()
    n1 = idl.launch_count()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    # stage breakdown from a separate, untimed pass with per-stage events (eager calls:
    # profiling turns graph replay off)
    ctx.profile(True)
    for _ in range(min(args.steps, 50)):
        step(J, T, lh)
    torch.cuda.synchronize()
    prof = ctx.profile_read()
    ctx.profile(False)
    ms = max_over_ranks(ms, dist, "cuda")
    if dist:
        dist.barrier()
    ms_per_step = ms / args.steps
    solves_per_step = 1
    value = job_value(ws, args.steps, solves_per_step, ms / 1e3)

    # learned vs plain: the same workload with the column proposal in the QR stage (fallbacks count
    # with their full time); untimed runs first (graph capture / tuning for a new batch shape)
    lvp = None
    if w["dtype"] == "f32":
        for _ in range(max(3, args.warmup)):
            step_learned()
        torch.cuda.synchronize()
        nl = max(1, min(args.steps, args.learned_steps))
        e0.record()
        for _ in range(nl):
            step_learned()
        e1.record()
        torch.cuda.synchronize()
        ms_l = e0.elapsed_time(e1)
        info = idl.Info()
        if name in ("sparse", "sparse_small"):
            idl.id_matrix_csr(ctx, d_rp, d_ci, d_v, c.shape, K, p_l, J, T, info=info)
        elif name == "mixed":
            idl.id_matrix(ctx, d_A, K, p_l, J, T, info=info)
        else:
            idl.id_cp_tensor(ctx, d_f, d_lam, K, p_l, J, T, lh, info=info)
        cert = 1.0 if info.proposal == 1 else 0.0
        ms_l = max_over_ranks(ms_l, dist, "cuda")
        v_l = job_value(ws, nl, solves_per_step, ms_l / 1e3)
        lvp = {"proposal": "mlp (shipped weights), top-2K candidates, certificate, plain QR on rejection",
               "value_learned": round(v_l, 3), "value_plain": round(value, 3), "ratio": round(v_l / value, 4),
               "certified_fraction": round(cert, 4), "steps": nl, "unit": "solves/s"}
        for _ in range(2):
            step(J, T, lh)        # restore the plain path's outputs for the accuracy check below
        torch.cuda.synchronize()

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    hJ = torch.empty(K, dtype=torch.int32).pin_memory()
    hT = torch.empty(K * (R - K), dtype=torch.float64).pin_memory()
    hl = torch.empty(K, dtype=torch.float64).pin_memory()
    for _ in range(2):
        step(hJ, hT, hl, host_in=True)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        step(hJ, hT, hl, host_in=True)
        if name == "cp":
            torch.cuda.synchronize()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, dist, "cuda")
    e2e_val = job_value(ws, e2e_steps, solves_per_step, e2e_s)
    d2h = 4 * K + 8 * K * (R - K) + (8 * K if name == "cp" else 0)
    floor_ms = copy_floor_ms(host_inputs)

    if rank != 0:
        ctx.close()
        if dist:
            dist.destroy_process_group()
        return None

    # roofline of the dominant kernel (the sketch), timed live with events on the library's stream
    peaks, peak_kind = measured_peaks()
    sk_ms, sk_n = prof["sketch"]
    sk_avg_s = (sk_ms / sk_n) / 1e3 if sk_n else float("nan")
    abytes = sketch_bytes(name, inp)
    achieved = abytes / sk_avg_s / 1e9
    kernel, src = {"sparse": ("cs_csr_kernel", "countsketch.cu"), "sparse_small": ("cs_csr_kernel", "countsketch.cu"),
                   "dense64": ("cs_dense_kernel", "countsketch.cu"),
                   "mixed": ("cs_dense_kernel", "countsketch.cu"),
                   "cp": ("tensorsketch8k_kernel", ["tsketch8k_dev.cuh", "tensorsketch.cu"])}[name]
    roof = {"bound": "hbm", "kernel": kernel, "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"],
            "unit": "GB/s", "frac": round(achieved / peaks["hbm_gbs"], 4),
            "traffic": recorded_traffic(kernel, name, src), "algorithmic_bytes": abytes,
            "avg_launch_us": round(sk_avg_s * 1e6, 2), "peak_source": f"{peak_kind} MEASURED_PEAKS.json hbm_gbs"
            if peak_kind == "measured" else "fallback 6.8 TB/s"}
    if name == "cp":           # the TensorSketch is arithmetic, not a stream: its roof is the FP32 pipe
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        mhz = peaks.get("sm_max_mhz", 2070.0)
        pk = fp32_peak_tflops(sms, mhz)
        fl = ts_flops(w["R"], len(w["dims"]), w["m1"])
        a = fl / sk_avg_s / 1e12
        roof = {"bound": "alu", "kernel": kernel, "achieved": round(a, 2), "peak": round(pk, 2), "unit": "TFLOP/s",
                "frac": round(a / pk, 4), "traffic": recorded_traffic(kernel, name, src), "algorithmic_flop": fl,
                "avg_launch_us": round(sk_avg_s * 1e6, 2),
                "peak_source": f"derived: {sms} SMs x 128 FP32 lanes x 2 flop (FMA) x {mhz:.0f} MHz"}
    stages = {k: round(v[0] / v[1] * 1e3, 2) if v[1] else None for k, v in prof.items()}

    # accuracy of this step's result (untimed): the oracle's error evaluation of the GPU's J, T
    from oracle import errors as oer
    Jg = J.cpu().numpy()
    Tg = T.cpu().numpy().reshape(K, R - K)
    if name in ("sparse", "sparse_small"):
        c = inp["csr"]
        rel_err = oer.matrix_id_error(csr=(c.rowptr, c.colidx, c.vals, c.shape), J=Jg, T=Tg, iters=20)
    elif name in ("dense64", "mixed"):
        rel_err = oer.matrix_id_error(inp["A"], J=Jg, T=Tg, exact=(name == "dense64"), iters=20)
    else:
        rel_err = oer.tensor_id_error(inp["factors"], inp["lam"], Jg, lh.cpu().numpy())

    out = {
        "metric": METRIC, "value": round(value, 3), "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if w["dtype"] == "f64" else "f32", "data": "synthetic",
        "config": {"workload": w["desc"], "precision": w["precision"],
                   "l2": "no flush: inputs larger than L2 (129 MB)" if abytes > 2e8 else
                         "inputs smaller than L2; steps run back to back (L2-warm)",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "1 GPU",
                   "launch": "timed steps replay the pipeline as a CUDA graph (idl_set_graphs); stage and "
                             "kernel times (roofline, stage_us) from per-stage CUDA events in an eager pass of "
                             "the same steps right after the timed region"},
        "rel_err": rel_err,
        "sketch_gbs": round(achieved, 1),
        "stage_us": stages,
        "roofline": roof,
        "e2e": {"value": round(e2e_val, 3), "unit": "solves/s", "h2d_bytes_per_step": int(in_bytes),
                "d2h_bytes_per_step": int(d2h), "steps": e2e_steps,
                "h2d_copy_floor_ms": round(floor_ms, 2), "link_gbs": round(in_bytes / floor_ms / 1e6, 1),
                "floor_note": "plain copies of the same pinned inputs, untimed for the metric: the host "
                              "link's limit under the end-to-end number"},
        "gpu_launches": int(n1 - n0),
        "clocks": clk,
        "learned_vs_plain": lvp,
    }
    if ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(name, inp, budget_s=args.cpu_budget)
    ctx.close()
    if dist:
        dist.destroy_process_group()
    return out


# ----------------------------------------------------------------------------- batched workload (the default)
BATCH_KERNELS = {   # stage group -> (kernel, source files, bound)
    "sketch_cp": ("b_sketch_cp8k_kernel", ["tsketch8k_dev.cuh", "batch.cu"], "alu"),
    "sketch_dense": ("b_sketch_dense_kernel", ["sketch_dev.cuh", "batch.cu"], "hbm"),
    "gaussian": ("b_gemm_kernel", ["gemm_dev.cuh", "batch.cu"], "hbm"),
}


def host_batch_items(idl, dense, cps, prec):
    """The batch with every array in pinned host memory (inputs copied from the
    device ones, outputs allocated): the end-to-end leg hands these to
    idl_batch_run, which stages them itself."""
    import torch
    items, outs, keep = [], [], []
    in_b = out_b = 0
    for pr in dense:
        A = pr["A"].cpu().pin_memory()
        K, R = pr["K"], A.shape[1]
        J = torch.empty(K, dtype=torch.int32).pin_memory()
        T = torch.empty(K * (R - K), dtype=torch.float64).pin_memory()
        p = idl.make_params(pr["m1"], pr["m2"], seed=pr["seed"], modified=True, precision=prec)
        items.append(idl.dense_item(A, K, p, J, T))
        outs.append((J, T, None))
        keep.append(A)
        in_b += A.numel() * 4
        out_b += J.numel() * 4 + T.numel() * 8
    for pr in cps:
        fs = [f.cpu().pin_memory() for f in pr["facs"]]
        lam = pr["lam"].cpu().pin_memory()
        K, R = pr["K"], fs[0].shape[0]
        J = torch.empty(K, dtype=torch.int32).pin_memory()
        T = torch.empty(K * (R - K), dtype=torch.float64).pin_memory()
        lh = torch.empty(K, dtype=torch.float64).pin_memory()
        p = idl.make_params(pr["L"], pr["m2"], seed=pr["seed"], modified=False, precision=prec)
        items.append(idl.cp_item(fs, lam, K, p, J, T, lh))
        outs.append((J, T, lh))
        keep.append((fs, lam))
        in_b += sum(f.numel() * 4 for f in fs) + lam.numel() * 8
        out_b += J.numel() * 4 + T.numel() * 8 + lh.numel() * 8
    return items, outs, keep, in_b, out_b


def batch_work(dense, cps):
    """Algorithmic work of the batch's three main kernels: dense-sketch bytes,
    TensorSketch FLOP, Gaussian-stage FLOP (the method's 2 m2 m1 R per item)."""
    by = 0.0
    for pr in dense:
        I, R = pr["A"].shape
        by += 4.0 * I * R + 5.0 * I + 4.0 * (pr["m1"] + 1) + 4.0 * pr["m1"] * R
    fl_ts = sum(ts_flops(pr["facs"][0].shape[0], len(pr["facs"]), pr["L"]) for pr in cps)
    fl_g = sum(2.0 * pr["m2"] * pr["m1"] * pr["A"].shape[1] for pr in dense)
    fl_g += sum(2.0 * pr["m2"] * pr["L"] * pr["facs"][0].shape[0] for pr in cps)
    return by, fl_ts, fl_g


def batch_gauss_bytes(dense, cps):
    """Algorithmic bytes of the batch's Gaussian stage: Y1 read (FP32), Omega read
    (FP64, by the plane builders), Y2 written (FP32)."""
    b = 0.0
    for pr in dense:
        R = pr["A"].shape[1]
        b += 4.0 * pr["m1"] * R + 8.0 * pr["m2"] * pr["m1"] + 4.0 * pr["m2"] * R
    for pr in cps:
        R = pr["facs"][0].shape[0]
        b += 4.0 * pr["L"] * R + 8.0 * pr["m2"] * pr["L"] + 4.0 * pr["m2"] * R
    return b


def batch_rooflines(stage_ms, dense, cps, sms):
    """Roofline entries of the batch's main kernels from their event-timed stage
    times (ms per launch group) and the measured / derived peaks."""
    peaks, kind = measured_peaks()
    tag = "of measured" if kind == "measured" else "of fallback"
    mhz = peaks.get("sm_max_mhz", 2070.0)
    by, fl_ts, fl_g = batch_work(dense, cps)
    out = {}
    t = stage_ms["sketch_cp"] / 1e3
    if t > 0 and fl_ts > 0:
        pk = fp32_peak_tflops(sms, mhz)
        a = fl_ts / t / 1e12
        out["sketch_cp"] = {"bound": "alu", "achieved": round(a, 2), "peak": round(pk, 2), "unit": "TFLOP/s",
                            "frac": round(a / pk, 4), "algorithmic_flop": fl_ts, "avg_launch_us": round(t * 1e6, 1),
                            "peak_source": f"derived: {sms} SMs x 128 FP32 lanes x 2 flop (FMA) x {mhz:.0f} MHz"}
    t = stage_ms["sketch_dense"] / 1e3
    if t > 0 and by > 0:
        pk = peaks["hbm_gbs"]
        a = by / t / 1e9
        out["sketch_dense"] = {"bound": "hbm", "achieved": round(a, 1), "peak": pk, "unit": "GB/s",
                               "frac": round(a / pk, 4), "algorithmic_bytes": by, "avg_launch_us": round(t * 1e6, 1),
                               "peak_source": f"{tag} MEASURED_PEAKS.json hbm_gbs" if kind == "measured"
                               else "fallback 6.8 TB/s"}
    t = stage_ms["gaussian"] / 1e3
    if t > 0 and fl_g > 0:
        # 2 m2 FLOP per 4-byte Y1 value (about 100 for m2 ~ 50) is below the bf16 ridge
        # (sustained TFLOP/s / HBM GB/s ~ 250 FLOP/byte): the stage's roof is the Y1 read
        gb = batch_gauss_bytes(dense, cps)
        pk = peaks["hbm_gbs"]
        a = gb / t / 1e9
        out["gaussian"] = {"bound": "hbm", "achieved": round(a, 1), "peak": pk, "unit": "GB/s",
                           "frac": round(a / pk, 4), "algorithmic_bytes": gb, "avg_launch_us": round(t * 1e6, 1),
                           "peak_source": f"{tag} MEASURED_PEAKS.json hbm_gbs" if kind == "measured"
                           else "fallback 6.8 TB/s",
                           "tensor": {"achieved_tflops": round(fl_g / t / 1e12, 2), "algorithmic_flop": fl_g,
                                      "note": "the method's 2 m2 m1 R FLOP per item; each precision mode "
                                              "issues 1, 3 or 6 bf16 (or 3 tf32) products of it"},
                           "launches": "planes + tensor-core product + split-K reduction"}
    for k, v in out.items():
        kern, srcs, _ = BATCH_KERNELS[k]
        v["kernel"] = kern
        v["traffic"] = recorded_traffic(kern, "batched", srcs)
    return out


def run_batched(args, ws, rank, local):
    """One step = one idl_batch_run over 256 dense matrices and 64 CP tensors."""
    import torch
    import paper_1901_10559_gb300 as idl
    from paper_1901_10559_gb300 import build as b
    b.build()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    w = WORKLOADS["batched"]
    inp = make_inputs("batched", rank)
    dense, cps = inp["dense"], inp["cps"]
    ctx = idl.Context(local)
    prec = precision_code(idl, w["precision"])
    items, bouts = batch_items(idl, dense, cps, prec)
    arr = idl.batch_array(items)
    n_items = len(items)

    for _ in range(args.warmup):                 # the first call tunes the shape and captures its graph
        idl.idl_batch_run(ctx, arr)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    n0 = idl.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(args.steps):
        idl.idl_batch_run(ctx, arr)
    e1.record()
    torch.cuda.synchronize()
    n1 = idl.launch_count()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    assert ctx.sync() == idl.IDL_OK
    ms = max_over_ranks(ms, dist, "cuda")
    value = job_value(ws, args.steps, n_items, ms / 1e3)

    # per-stage times: event-timed eager runs of the same batch right after the timed region
    reps = 3
    stage_ms = {k: 0.0 for k in idl.BATCH_STAGES}
    for _ in range(reps):
        for k, v in idl.batch_stage_ms(ctx, items).items():
            stage_ms[k] += v / reps

    # learned vs plain: the same batch with the MLP column proposal in the QR stage
    idl.idl_load_weights(ctx, idl.PROPOSAL_WEIGHTS)
    items_l, bouts_l = batch_items(idl, dense, cps, prec, learned=idl.PROPOSAL_MLP)
    arr_l = idl.batch_array(items_l)
    for _ in range(max(3, args.warmup)):
        idl.idl_batch_run(ctx, arr_l)
    torch.cuda.synchronize()
    nl = max(1, min(args.steps, args.learned_steps))
    e0.record()
    for _ in range(nl):
        idl.idl_batch_run(ctx, arr_l)
    e1.record()
    torch.cuda.synchronize()
    ms_l = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
    nfb = idl.idl_batch_fallbacks(ctx)
    v_l = job_value(ws, nl, n_items, ms_l / 1e3)
    same_j = all(torch.equal(a[0], b[0]) for a, b in zip(bouts, bouts_l))
    lvp = {"proposal": "mlp (shipped weights), top-2K candidates, certificate, plain QR on rejection",
           "value_learned": round(v_l, 3), "value_plain": round(value, 3), "ratio": round(v_l / value, 4),
           "certified_fraction": round((n_items - nfb) / n_items, 4), "steps": nl, "unit": "solves/s",
           "same_pivots_as_plain": bool(same_j)}
    idl.idl_batch_run(ctx, arr)                  # the plain outputs again for the accuracy check
    torch.cuda.synchronize()

    # end to end through the C ABI with pinned host buffers: idl_batch_run stages the
    # inputs (copies overlapped with the kernels that do not need them yet) and
    # copies the outputs back before it returns
    h_items, h_outs, h_keep, in_bytes, out_bytes = host_batch_items(idl, dense, cps, prec)
    h_arr = idl.batch_array(h_items)
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    h_tensors = []
    for k in h_keep:
        h_tensors += (list(k[0]) + [k[1]]) if isinstance(k, tuple) else [k]
    for _ in range(2):
        idl.idl_batch_run(ctx, h_arr)
    floor_before = copy_floor_ms(h_tensors)      # the shared host link drifts: bracket the timed loop
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        idl.idl_batch_run(ctx, h_arr)
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    e2e_val = job_value(ws, e2e_steps, n_items, e2e_s)
    floor_ms = copy_floor_ms(h_tensors)
    e2e_same = all(torch.equal(a[0].cpu(), b[0]) for a, b in zip(bouts, h_outs))

    if rank != 0:
        ctx.close()
        if dist:
            dist.destroy_process_group()
        return None

    sms = torch.cuda.get_device_properties(local).multi_processor_count
    roofs = batch_rooflines(stage_ms, dense, cps, sms)
    dom = max(roofs, key=lambda k: stage_ms[k]) if roofs else None
    roof = dict(roofs[dom]) if dom else None

    # accuracy of this step's result (untimed): the oracle's error evaluation of the GPU's
    # J, T on a seeded sample of items (the ID error is relative to the spectral / Frobenius norm)
    from oracle import errors as oer
    rng = np.random.default_rng(w["seed"])
    errs = []
    for q in sorted(rng.choice(len(dense), size=6, replace=False)):
        pr = dense[q]
        Kq, Rq = pr["K"], pr["A"].shape[1]
        errs.append(oer.matrix_id_error(pr["A"].cpu().numpy(), J=bouts[q][0].cpu().numpy(),
                                        T=bouts[q][1].cpu().numpy().reshape(Kq, Rq - Kq), exact=False, iters=20))
    for q in sorted(rng.choice(len(cps), size=2, replace=False)):
        pr = cps[q]
        o = bouts[len(dense) + q]
        facs = [f.cpu().numpy().T.astype(np.float64) for f in pr["facs"]]
        errs.append(oer.tensor_id_error(facs, pr["lam"].cpu().numpy(), o[0].cpu().numpy(), o[2].cpu().numpy()))

    vs_gauss = compare_gaussian_id(idl, ctx, dense, cps, prec)

    out = {
        "metric": METRIC, "value": round(value, 3), "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w["desc"], "precision": f"{w['precision']} Gaussian stage, FP32 sketches, FP64 T",
                   "items_per_step": n_items,
                   "l2": "no flush: inputs larger than L2 (16 GB of dense matrices, 1 GB of CP factors per step)",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "1 GPU",
                   "launch": "one idl_batch_run per step, replayed as one CUDA graph; stage times from "
                             "event-timed eager runs of the same batch right after the timed region"},
        "rel_err": max(errs),
        "rel_err_items": "max over 6 dense items (spectral norm) and 2 CP items (Frobenius norm, exact)",
        "stage_us": {k: round(v * 1e3, 1) for k, v in stage_ms.items()},
        "roofline": roof,
        "rooflines": roofs,
        "e2e": {"value": round(e2e_val, 3), "unit": "solves/s", "h2d_bytes_per_step": int(in_bytes),
                "d2h_bytes_per_step": int(out_bytes), "steps": e2e_steps, "pivots_match_device_run": bool(e2e_same),
                "h2d_copy_floor_ms": [round(floor_before, 2), round(floor_ms, 2)],
                "link_gbs": [round(in_bytes / floor_before / 1e6, 1), round(in_bytes / floor_ms / 1e6, 1)],
                "floor_note": "plain copies of the same pinned inputs right before and right after the timed "
                              "loop (untimed for the metric): the host link's limit under the end-to-end "
                              "number; the link is shared and drifts",
                "how": "idl_batch_run with pinned host arrays: the call copies inputs in and outputs out"},
        "gpu_launches": int(n1 - n0),
        "clocks": clk,
        "learned_vs_plain": lvp,
        "vs_gaussian_id": vs_gauss,
    }
    if ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline_batched(dense, cps, bouts, budget_s=args.cpu_budget)
    ctx.close()
    if dist:
        dist.destroy_process_group()
    return out


def compare_gaussian_id(idl, ctx, dense, cps, prec, reps=5):
    """The paper's comparison on GB300: the CountSketch / TensorSketch pipelines against
    Gaussian ID (Sec. 1.2.1; Khatri-Rao Gaussian sketch of Eq. G-matrix for CP tensors)
    on the same items, one call at a time, CUDA-event timed; both sketch to the
    item's m2 = K + 10 rows before the same QR stage and T solve."""
    import torch
    from oracle import errors as oer
    rng = np.random.default_rng(11)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    res = {}
    t_cs = t_g = 0.0
    err = {"countsketch": [], "gaussian": []}
    for q in sorted(rng.choice(len(dense), size=4, replace=False)):
        pr = dense[q]
        K, R = pr["K"], pr["A"].shape[1]
        J = torch.empty(K, dtype=torch.int32, device="cuda")
        T = torch.empty(K * (R - K), dtype=torch.float64, device="cuda")
        pc = idl.make_params(pr["m1"], pr["m2"], seed=pr["seed"], modified=True, precision=prec)
        pg = idl.make_params(0, pr["m2"], seed=pr["seed"], modified=False, precision=prec)
        t_cs += timed(lambda: idl.id_matrix(ctx, pr["A"], K, pc, J, T))
        err["countsketch"].append(oer.matrix_id_error(pr["A"].cpu().numpy(), J=J.cpu().numpy(),
                                                      T=T.cpu().numpy().reshape(K, R - K), exact=False, iters=20))
        t_g += timed(lambda: idl.id_matrix_gaussian(ctx, pr["A"], K, pg, J, T))
        err["gaussian"].append(oer.matrix_id_error(pr["A"].cpu().numpy(), J=J.cpu().numpy(),
                                                   T=T.cpu().numpy().reshape(K, R - K), exact=False, iters=20))
    res["dense"] = {"items": 4, "countsketch_ms": round(t_cs, 3), "gaussian_ms": round(t_g, 3),
                    "speedup": round(t_g / t_cs, 3), "max_rel_err_countsketch": max(err["countsketch"]),
                    "max_rel_err_gaussian": max(err["gaussian"])}
    t_cs = t_g = 0.0
    err = {"countsketch": [], "gaussian": []}
    for q in sorted(rng.choice(len(cps), size=2, replace=False)):
        pr = cps[q]
        K, R = pr["K"], pr["facs"][0].shape[0]
        J = torch.empty(K, dtype=torch.int32, device="cuda")
        T = torch.empty(K * (R - K), dtype=torch.float64, device="cuda")
        lh = torch.empty(K, dtype=torch.float64, device="cuda")
        pc = idl.make_params(pr["L"], pr["m2"], seed=pr["seed"], modified=False, precision=prec)
        pg = idl.make_params(0, pr["m2"], seed=pr["seed"], modified=False, precision=prec)
        facs = [f.cpu().numpy().T.astype(np.float64) for f in pr["facs"]]
        lam = pr["lam"].cpu().numpy()
        t_cs += timed(lambda: idl.id_cp_tensor(ctx, pr["facs"], pr["lam"], K, pc, J, T, lh))
        err["countsketch"].append(oer.tensor_id_error(facs, lam, J.cpu().numpy(), lh.cpu().numpy()))
        t_g += timed(lambda: idl.id_cp_tensor_gaussian(ctx, pr["facs"], pr["lam"], K, pg, J, T, lh))
        err["gaussian"].append(oer.tensor_id_error(facs, lam, J.cpu().numpy(), lh.cpu().numpy()))
    res["cp"] = {"items": 2, "tensorsketch_ms": round(t_cs, 3), "gaussian_ms": round(t_g, 3),
                 "speedup": round(t_g / t_cs, 3), "max_rel_err_tensorsketch": max(err["countsketch"]),
                 "max_rel_err_gaussian": max(err["gaussian"])}
    res["paper_context"] = ("the paper (4-core Xeon, Matlab) reports CountSketch ID about 18x faster than "
                            "Gaussian ID on a 1e6 x 1e4 sparse matrix and about 35x on SuiteSparse specular "
                            "(Sec. 6.1, Table 3), TensorSketch ID about 14x faster than Gaussian tensor ID on a "
                            "sparse 5-way CP tensor (Sec. 6.2); here dense items of the batched workload")
    return res


def _oracle_dense(A, K, m1, m2, seed):
    from oracle import idmethods as oid
    from oracle.gaussian import FP32
    return oid.id_matrix(A, k=K, m1=m1, m2=m2, seed=seed, modified=True, precision=FP32)


def _oracle_cp(facs, lam, K, L, m2, seed):
    from oracle import idmethods as oid
    from oracle.gaussian import FP32
    return oid.id_cp_tensor(facs, lam, k=K, L=L, m2=m2, seed=seed, precision=FP32)


def batch_estimate(t_dense, t_cp, n_dense=256, n_cp=64):
    """Oracle time of a whole batch from per-item samples of each kind (stratified)."""
    return n_dense * statistics.mean(t_dense) + n_cp * statistics.mean(t_cp)


def cpu_baseline_batched(dense, cps, bouts, budget_s=20.0):
    """The oracle on a seeded, stratified sample of the step's own items: one CP
    tensor, then dense matrices until the budget is spent (at least two); the
    batch's time is estimated as 256 x mean(dense) + 64 x mean(CP)."""
    rng = np.random.default_rng(7)
    t_cp, t_dense = [], []
    q = int(rng.integers(len(cps)))
    pr = cps[q]
    facs = [f.cpu().numpy().T.copy() for f in pr["facs"]]
    t0 = time.perf_counter()
    _oracle_cp(facs, pr["lam"].cpu().numpy(), pr["K"], pr["L"], pr["m2"], pr["seed"])
    t_cp.append(time.perf_counter() - t0)
    start = time.perf_counter()
    for q in rng.permutation(len(dense)):
        pr = dense[q]
        A = pr["A"].cpu().numpy()
        t0 = time.perf_counter()
        _oracle_dense(A, pr["K"], pr["m1"], pr["m2"], pr["seed"])
        t_dense.append(time.perf_counter() - t0)
        if len(t_dense) >= 2 and time.perf_counter() - start > budget_s:
            break
    T = batch_estimate(t_dense, t_cp, len(dense), len(cps))
    return {"value": round((len(dense) + len(cps)) / T, 5), "unit": "solves/s", "cores": os.cpu_count(),
            "kind": "oracle",
            "sample": f"stratified seeded sample of this step's items: {len(t_cp)} CP tensor "
                      f"({statistics.mean(t_cp):.2f} s) and {len(t_dense)} dense matrices (mean "
                      f"{statistics.mean(t_dense):.2f} s); batch time estimated as 256 x mean(dense) + 64 x mean(CP) "
                      f"= {T:.0f} s; numpy/BLAS default threading"}


# ----------------------------------------------------------------------------- oracle (CPU) arm
def oracle_solve(name, inp, seed):
    from oracle import idmethods as oid
    from oracle.gaussian import FP32, FP64
    w = WORKLOADS[name]
    prec = FP64 if w["precision"] == "FP64" else FP32
    if name in ("sparse", "sparse_small"):
        c = inp["csr"]
        return oid.id_matrix(csr=(c.rowptr, c.colidx, c.vals, c.shape), k=w["k"], m1=w["m1"], m2=w["m2"], seed=seed,
                             modified=True, precision=prec)
    if name in ("dense64", "mixed"):
        return oid.id_matrix(inp["A"], k=w["k"], m1=w["m1"], m2=w["m2"], seed=seed, modified=True, precision=prec)
    return oid.id_cp_tensor(inp["factors"], inp["lam"], k=w["k"], L=w["m1"], m2=w["m2"], seed=seed, precision=prec)


def sample_of(name, inp):
    """A bounded sample of the workload for the oracle and its fraction of the full work."""
    if name == "mixed":     # 131072 x 4096: the first 16384 rows (1/8 of the sketch's O(nnz) work)
        A = inp["A"][:16384]
        return {"A": A}, A.shape[0] / inp["A"].shape[0], "rows 0..16383 of A (1/8 of the rows); value scaled by 1/8"
    return inp, 1.0, "one full solve of the same workload"


def cpu_baseline(name, inp, budget_s=20.0):
    smp, frac, desc = sample_of(name, inp)
    times = []
    t_start = time.perf_counter()
    while True:
        t0 = time.perf_counter()
        oracle_solve(name, smp, WORKLOADS[name]["seed"])
        times.append(time.perf_counter() - t0)
        if time.perf_counter() - t_start > budget_s or len(times) >= 3:
            break
    t = statistics.median(times)
    return {"value": round(frac / t, 5), "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{desc}; median of {len(times)} run(s), {t:.2f} s each; numpy/BLAS default threading"}


def bounded_sample(name, inp, per_step_s):
    """The workload restricted to its first rows so that one oracle solve takes
    about per_step_s (never fewer rows than 4 m1).  Returns (sample, fraction of
    the rows, description)."""
    if name not in ("sparse", "sparse_small", "mixed"):
        return sample_of(name, inp)
    w = WORKLOADS[name]
    I = w["I"]
    full, frac0, desc0 = sample_of(name, inp)
    if name == "mixed":
        I = int(frac0 * I)
    # cost model t(n) = a + b n from two small calibration solves (untimed)
    pts = []
    for n in (max(4 * w["m1"], I // 50), max(8 * w["m1"], I // 10)):
        sub = _rows(name, full, n)
        t0 = time.perf_counter()
        oracle_solve(name, sub, w["seed"])
        pts.append((n, time.perf_counter() - t0))
    (n1, t1), (n2, t2) = pts
    b = max((t2 - t1) / max(n2 - n1, 1), 1e-12)
    a = max(t1 - b * n1, 0.0)
    n = int(min(I, max(4 * w["m1"], (per_step_s - a) / b)))
    frac = frac0 * n / I
    desc = (f"rows 0..{n - 1} of the workload ({100 * frac:.2f}% of its rows, all columns, same k, m1, m2); "
            f"value scaled by that row fraction (the O(nnz) sketch share; the oracle's fixed "
            f"Gaussian-stage and QR cost, ~{a:.2f} s per solve, is then counted once per sampled solve)")
    return _rows(name, full, n), frac, desc


def _rows(name, inp, n):
    if name == "mixed":
        return {"A": inp["A"][:n]}
    import synth
    c = inp["csr"]
    e = int(c.rowptr[n])
    return {"csr": synth.CSR(c.rowptr[:n + 1].copy(), c.colidx[:e], c.vals[:e], (n, c.shape[1]))}


def run_reference(args, ws, rank):
    name = args.workload
    if rank != 0:
        return None
    inp = make_inputs(name)
    per_step = min(30.0, 150.0 / max(1, args.steps + args.warmup))
    smp, frac, desc = bounded_sample(name, inp, per_step)
    for _ in range(args.warmup):
        oracle_solve(name, smp, WORKLOADS[name]["seed"])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_solve(name, smp, WORKLOADS[name]["seed"])
    dt = time.perf_counter() - t0
    value = frac * args.steps / dt
    w = WORKLOADS[name]
    return {"impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": "solves/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3 / frac, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": w["desc"], "precision": "FP64 oracle"},
            "cpu_baseline": {"value": round(value, 5), "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": desc + "; numpy/BLAS default threading"},
            "e2e": {"value": round(value, 5), "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_reference_batched(args, ws, rank):
    """The oracle on the batched workload: each timed step solves one item of the
    recipe (generated on the host with numpy: same recipe, other draws than the
    GPU arm's torch generator), a CP tensor on every fifth step and a dense
    matrix otherwise, from seeded permutations; the batch's time is estimated
    as 256 x mean(dense) + 64 x mean(CP).  Warm-up steps solve the smallest
    dense item."""
    import synth
    if rank != 0:
        return None
    w = WORKLOADS["batched"]
    seed = w["seed"]
    specs = synth.batch_matrix_specs(w["n_dense"], seed)
    rng = np.random.default_rng(seed)
    pd, pc = rng.permutation(len(specs)), rng.permutation(w["n_cp"])

    def dense_job(q):
        sp = specs[q]
        A = synth.batch_dense_item(sp, sp["seed"])
        m2 = sp["rank"] + 10
        return lambda: _oracle_dense(A, sp["rank"], min(m2 * m2, sp["I"] // 2), m2, sp["seed"])

    def cp_job(b):
        facs, lam, K = synth.batch_cp_item(b, seed * 10 + b)
        return lambda: _oracle_cp(facs, lam, K, 8192, K + 10, seed * 10 + b)

    small = min(range(len(specs)), key=lambda q: specs[q]["I"] * specs[q]["R"])
    for _ in range(args.warmup):
        dense_job(small)()
    t_dense, t_cp = [], []
    for st in range(args.steps):
        job = cp_job(int(pc[(st // 5) % len(pc)])) if st % 5 == 0 else dense_job(int(pd[st % len(pd)]))
        t0 = time.perf_counter()
        job()
        (t_cp if st % 5 == 0 else t_dense).append(time.perf_counter() - t0)
    if not t_dense:                              # one step: time one dense item as well
        job = dense_job(int(pd[0]))
        t0 = time.perf_counter()
        job()
        t_dense.append(time.perf_counter() - t0)
    T = batch_estimate(t_dense, t_cp, w["n_dense"], w["n_cp"])
    value = (w["n_dense"] + w["n_cp"]) / T
    desc = (f"one item per step ({len(t_cp)} CP tensors, mean {statistics.mean(t_cp):.2f} s; {len(t_dense)} dense "
            f"matrices, mean {statistics.mean(t_dense):.2f} s); batch of 256 + 64 estimated at {T:.0f} s; "
            f"numpy/BLAS default threading")
    return {"impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": "solves/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(T * 1e3, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w["desc"], "precision": "FP64 oracle", "items_per_step": 320},
            "cpu_baseline": {"value": round(value, 5), "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": round(value, 5), "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_batch_probe(args, spec):
    """``batch:n_dense,n_cp``: the first n_dense dense matrices and n_cp CP tensors of
    the batched workload's recipe as one batch; after --warmup calls (the first tunes
    the shape), --steps event-timed un-graphed runs.  Prints the mean milliseconds of
    each stage group -- a small case of the batch kernels for profilers."""
    import torch
    import paper_1901_10559_gb300 as idl
    from paper_1901_10559_gb300 import build as b
    b.build()
    n_dense, n_cp = (int(x) for x in spec.split(","))
    w = WORKLOADS["batched"]
    dense, cps = make_batch(w["seed"], 0, n_dense, n_cp)
    ctx = idl.Context(0)
    items, _ = batch_items(idl, dense, cps, precision_code(idl, args.precision or w["precision"]))
    arr = idl.batch_array(items)
    for _ in range(args.warmup):
        idl.idl_batch_run(ctx, arr)
    torch.cuda.synchronize()
    tot = {k: 0.0 for k in idl.BATCH_STAGES}
    for _ in range(args.steps):
        for k, v in idl.batch_stage_ms(ctx, items).items():
            tot[k] += v / args.steps
    if ctx.sync() != idl.IDL_OK:
        raise SystemExit("probe: device status not OK")
    gb = sum(4.0 * pr["A"].shape[0] * pr["A"].shape[1] for pr in dense) / 1e9
    return {"probe": args.probe, "precision": args.precision or w["precision"],
            "stage_ms": {k: round(v, 4) for k, v in tot.items()}, "dense_A_gb": round(gb, 3),
            "dense_sketch_tbs": round(gb / tot["sketch_dense"], 2) if tot["sketch_dense"] > 0 else None}


def run_probe(args):
    """One stage call timed alone (CUDA events, after warm-up) on seeded synthetic
    input: ``gaussian:<cm|rm>:m2,m1,R`` (Omega Y1 with column- or row-major FP32 Y1
    of N(0,1) values, the mode of --precision, default BF16X3), or the batch stages
    of a smaller batch (``batch:n_dense,n_cp``, run_batch_probe).  Prints one JSON
    line with the average microseconds per call and the Y1 read rate."""
    import torch
    import paper_1901_10559_gb300 as idl
    if args.probe.startswith("batch:"):
        return run_batch_probe(args, args.probe.split(":", 1)[1])
    kind, layout, dims = args.probe.split(":")
    if kind != "gaussian" or layout not in ("cm", "rm"):
        raise SystemExit("probe: gaussian:<cm|rm>:m2,m1,R")
    m2, m1, R = (int(x) for x in dims.split(","))
    prec_name = args.precision or "BF16X3"
    prec = precision_code(idl, prec_name)
    ctx = idl.Context(0)
    Om = torch.empty(m2 * m1, dtype=torch.float64, device="cuda")
    idl.idl_draw_gaussian(ctx, 3, m2, m1, Om)
    g = torch.Generator(device="cuda").manual_seed(20190130)
    Y1 = torch.randn(R * m1, dtype=torch.float32, device="cuda", generator=g)
    Y2 = torch.empty(R * m2, dtype=torch.float32, device="cuda")
    if layout == "cm":
        call = lambda: idl.idl_gaussian_stage_colmajor(ctx, Om, m2, m1, Y1, R, m1, prec, Y2, m2)
    else:
        call = lambda: idl.idl_gaussian_stage(ctx, Om, m2, m1, Y1, R, R, idl.IDL_F32, prec, Y2, m2)
    for _ in range(args.warmup):
        call()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        call()
    e1.record()
    torch.cuda.synchronize()
    if ctx.sync() != idl.IDL_OK:
        raise SystemExit("probe: device status not OK")
    us = e0.elapsed_time(e1) * 1e3 / args.steps
    return {"probe": args.probe, "precision": prec_name, "us_per_call": round(us, 2),
            "y1_read_gbs": round(4.0 * m1 * R / us / 1e3, 1),
            "note": "Omega planes + tensor-core product + split-K reduction per call; L2 not flushed "
                    "(Y1 larger than L2 when 4 m1 R > 129 MB)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=None)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="batched")
    ap.add_argument("--e2e-steps", type=int, default=30)
    ap.add_argument("--learned-steps", type=int, default=300)
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--probe", default=None, help="time one stage call alone, e.g. gaussian:cm:74,8192,5000")
    ap.add_argument("--precision", choices=["FP32", "BF16X3", "BF16", "TF32X3"], default=None,
                    help="Gaussian-stage mode of an FP32 workload (default: the workload's own)")
    args = ap.parse_args()
    if args.probe:
        args.steps = args.steps or 20
        args.warmup = args.warmup or 3
        print(json.dumps(run_probe(args)), flush=True)
        return
    batched = args.workload == "batched"
    if args.steps is None:
        args.steps = 3 if args.impl == "reference" else (50 if batched else 2000)
    if args.warmup is None:
        args.warmup = 3 if args.impl == "reference" else (5 if batched else 20)
    if batched:
        args.e2e_steps = min(args.e2e_steps, 5)
    if args.precision is not None:
        if WORKLOADS[args.workload]["precision"] == "FP64":
            ap.error("the FP64 workload has FP64 data: no other Gaussian-stage mode")
        WORKLOADS[args.workload]["precision"] = args.precision
    ws, rank, local = dist_env()
    if args.impl == "reference":
        out = run_reference_batched(args, ws, rank) if batched else run_reference(args, ws, rank)
    else:
        out = run_batched(args, ws, rank, local) if batched else run_ours(args, ws, rank, local)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
