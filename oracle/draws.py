"""Random maps of the sketching operators, from the counter-based draws spec.

TEST INFRASTRUCTURE (see ``oracle/__init__``).

The paper draws (Sec. 1.3):
  * h : [I] -> [L], each h(i) iid uniform, and D = diag(d_ii), d_ii = +-1
    with probability 1/2 -- the CountSketch S = Phi D;
  * the modified map h~ = f o pi of Remark 2 / Sec. 7.2: pi a uniform random
    permutation of [I], f(i) = i for i < L and an iid uniform x_i otherwise,
    so every one of the L buckets receives at least one row;
  * per-mode maps h_n, s_n of TensorSketch (Sec. 1.3);
  * a Gaussian matrix Omega with iid N(0,1) entries (Sec. 1.2.1).

Both this oracle and the CUDA library derive these from one published
counter-based generator, each in its own code:

  u(seed, tag, i) = SplitMix64 output number i (0-based) of the stream whose
                    state starts at base(seed, tag) = mix64(seed XOR tag*C_TAG),
                  = mix64(base + (i+1) * GAMMA)
  mix64           = the SplitMix64 finaliser (Steele, Lea & Flood 2014;
                    Vigna's splitmix64.c)
  bounded(u, L)   = floor(u * L / 2**64)  (multiply-shift, Lemire 2019)
  sign(u)         = +1 if the top bit of u is 0, else -1

Indices are 0-based here (the paper is 1-based), so H = (sum_n h_n) mod L.
"""
from __future__ import annotations

import numpy as np

MASK64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15
MIX_C1 = 0xBF58476D1CE4E5B9
MIX_C2 = 0x94D049BB133111EB
C_TAG = 0xD1B54A32D192ED03

# stream tags
TAG_BUCKET = 1       # h(i), and x_i of the modified map
TAG_SIGN = 2         # d_ii
TAG_PERM = 3         # round keys of the permutation pi
TAG_GAUSS = 4        # Omega
TAG_MODE_BUCKET = 16  # + n : h_n of TensorSketch
TAG_MODE_SIGN = 32    # + n : s_n of TensorSketch
TAG_GAUSS_ID = 5      # the L x I Gaussian sketch of Gaussian matrix ID (Sec. 1.2.1)
TAG_GAUSS_MODE = 48   # + n : the per-mode Gaussian matrices of Eq. G-matrix
TAG_ERR_START = 6     # start vectors of the power-method error estimate (Sec. 6)
FEISTEL_ROUNDS = 4

_U64 = np.uint64


# ---------------------------------------------------------------- scalar forms
def mix64_int(z: int) -> int:
    """SplitMix64 finaliser on a Python int (exact 64-bit arithmetic)."""
    z &= MASK64
    z ^= z >> 30
    z = (z * MIX_C1) & MASK64
    z ^= z >> 27
    z = (z * MIX_C2) & MASK64
    z ^= z >> 31
    return z


def base_int(seed: int, tag: int) -> int:
    return mix64_int((seed & MASK64) ^ ((tag * C_TAG) & MASK64))


def u_int(seed: int, tag: int, i: int) -> int:
    return mix64_int(base_int(seed, tag) + (i + 1) * GAMMA)


def bounded_int(u: int, L: int) -> int:
    return (u * L) >> 64


# ---------------------------------------------------------------- array forms
def mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser, elementwise on uint64 (wrapping arithmetic)."""
    z = np.asarray(z, dtype=_U64).copy()
    with np.errstate(over="ignore"):
        z ^= z >> _U64(30)
        z *= _U64(MIX_C1)
        z ^= z >> _U64(27)
        z *= _U64(MIX_C2)
        z ^= z >> _U64(31)
    return z


def stream(seed: int, tag: int, idx: np.ndarray) -> np.ndarray:
    """u(seed, tag, i) for every i in ``idx``."""
    b = _U64(base_int(seed, tag))
    idx = np.asarray(idx, dtype=_U64)
    with np.errstate(over="ignore"):
        ctr = b + (idx + _U64(1)) * _U64(GAMMA)
    return mix64(ctr)


def bounded(u: np.ndarray, L: int) -> np.ndarray:
    """floor(u * L / 2**64) for L < 2**32, exact (no 128-bit type in numpy):
    u*L = uh*L*2^32 + ul*L, so the high word is (uh*L + (ul*L >> 32)) >> 32."""
    assert 0 < L < (1 << 32)
    u = np.asarray(u, dtype=_U64)
    uh = u >> _U64(32)
    ul = u & _U64(0xFFFFFFFF)
    Lu = _U64(L)
    with np.errstate(over="ignore"):
        t = uh * Lu + ((ul * Lu) >> _U64(32))
    return (t >> _U64(32)).astype(np.int64)


def sign(u: np.ndarray) -> np.ndarray:
    return np.where((np.asarray(u, dtype=_U64) >> _U64(63)) == 0, 1, -1).astype(np.int8)


# ---------------------------------------------------------------- permutation
def feistel_width(I: int) -> int:
    """Even bit width w >= 2 with 2**w >= I."""
    w = max(1, int(I - 1).bit_length())
    if w % 2:
        w += 1
    return max(w, 2)


def permutation(seed: int, I: int, idx: np.ndarray | None = None) -> np.ndarray:
    """pi(i) for i in idx (default all of [I]): a keyed balanced Feistel
    network on w-bit integers (4 rounds, round function mix64(key_r XOR x)
    truncated to w/2 bits; Luby & Rackoff 1988) restricted to [I] by cycle
    walking (Black & Rogaway 2002): re-apply until the value lands in [I].
    Being a bijection of [2**w] restricted by cycle walking, it is a bijection
    of [I]."""
    w = feistel_width(I)
    half = w // 2
    mask = _U64((1 << half) - 1)
    keys = [_U64(u_int(seed, TAG_PERM, r)) for r in range(FEISTEL_ROUNDS)]

    def enc(x):
        left = x >> _U64(half)
        right = x & mask
        for k in keys:
            f = mix64(k ^ right) & mask
            left, right = right, left ^ f
        return (left << _U64(half)) | right

    if idx is None:
        idx = np.arange(I)
    y = enc(np.asarray(idx, dtype=_U64))
    out_of_range = y >= _U64(I)
    while np.any(out_of_range):
        y[out_of_range] = enc(y[out_of_range])
        out_of_range = y >= _U64(I)
    return y.astype(np.int64)


# ---------------------------------------------------------------- the maps
def countsketch_maps(seed: int, I: int, L: int, modified: bool):
    """(h, s) of a CountSketch S in R^{L x I} (Sec. 1.3).

    plain:    h(i) = bounded(u(seed, BUCKET, i), L)
    modified: h~(i) = pi(i) if pi(i) < L else bounded(u(seed, BUCKET, i), L)
              (Remark 2 / Sec. 7.2; f(pi(i)) with the iid x indexed by the
              row, which has the same joint law as x indexed by pi(i))
    s(i) = sign(u(seed, SIGN, i)).
    Returns h int64 in [0, L) and s int8 in {-1, +1}.
    """
    idx = np.arange(I)
    x = bounded(stream(seed, TAG_BUCKET, idx), L)
    if modified:
        if not L < I:
            raise ValueError("modified CountSketch needs L < I (Remark 2)")
        p = permutation(seed, I)
        h = np.where(p < L, p, x)
    else:
        h = x
    s = sign(stream(seed, TAG_SIGN, idx))
    return h.astype(np.int64), s


def tensorsketch_maps(seed: int, dims, L: int):
    """Per-mode (h_n, s_n) of TensorSketch (Sec. 1.3): plain iid maps."""
    hs, ss = [], []
    for n, In in enumerate(dims):
        idx = np.arange(In)
        hs.append(bounded(stream(seed, TAG_MODE_BUCKET + n, idx), L))
        ss.append(sign(stream(seed, TAG_MODE_SIGN + n, idx)))
    return hs, ss


def gaussian_matrix(seed: int, m2: int, m1: int, tag: int = TAG_GAUSS) -> np.ndarray:
    """Omega in R^{m2 x m1}, iid N(0,1) by the Box-Muller transform (Box &
    Muller 1958), row-major flat index q = j*m1 + b, pair p = q // 2:
      U1 = ((u(seed, tag, 2p) >> 11) + 1) * 2**-53   in (0, 1]
      U2 =  (u(seed, tag, 2p+1) >> 11)     * 2**-53   in [0, 1)
      rho = sqrt(-2 ln U1);  z_q = rho cos(2 pi U2) for even q, rho sin(2 pi U2) for odd q.
    tag = GAUSS for the Gaussian stage; GAUSS_ID and GAUSS_MODE + n for the
    Gaussian ID comparators.  Returned in float64."""
    n = m2 * m1
    q = np.arange(n)
    p = q // 2
    a = stream(seed, tag, 2 * p)
    c = stream(seed, tag, 2 * p + 1)
    U1 = ((a >> _U64(11)).astype(np.float64) + 1.0) * 2.0 ** -53
    U2 = (c >> _U64(11)).astype(np.float64) * 2.0 ** -53
    rho = np.sqrt(-2.0 * np.log(U1))
    ang = (2.0 * np.pi) * U2
    z = np.where(q % 2 == 0, rho * np.cos(ang), rho * np.sin(ang))
    return z.reshape(m2, m1)
