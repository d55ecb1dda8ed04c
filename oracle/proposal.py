"""Learned column proposal for the pivoted QR stage: column features, the
scoring MLP (forward, backward, Adam step), the candidate set and the
certificate, in float64.

TEST INFRASTRUCTURE (see ``oracle/__init__``).

The paper has no learned component.  The QR stage of Algorithm 1 picks K
pivots greedily by remaining column norm; this module states what the
library's proposal path computes so that every device stage has a plain
definition to be compared with:

Features of column c of the sketch Y (m x R), with n_c = ||y_c||^2,
nmax = max_c n_c, G = Y Y^T and lambda_q = rho_q tr(G) / m, rho = (1e-1, 1e-2, 1e-3):
  f0 = max(log(n_c / nmax), -64) / 16        (-4 for a zero column)
  f1 = sqrt(n_c / nmax)
  f2, f3, f4 = y_c^T (G + lambda_q I)^{-1} y_c  (ridge leverage scores, in [0, 1))
  f5 = max_i |y_ic| / sqrt(n_c)               (0 for a zero column)
  f6 = K / R,   f7 = m / R
A zero sketch (tr G = 0) has f2 = f3 = f4 = 0 and f0 = -4, f1 = 0 everywhere.

MLP (width 128): z1 = relu(W1 f + b1), z2 = relu(W2 z1 + b2), s = w3 . z2 + b3.
With ``bf16=True`` the operands the device multiplies in bfloat16 are rounded
first: f, W1, W2, w3 and z1 (round to nearest even); biases and all sums stay
exact here (float64).  Gradients treat the rounding as the identity.

Loss over examples (f_b, y_b), y in {0, 1} (1: column is a pivot of the plain
method), with positive weight w:
  L = (1/B) sum_b [ w y_b softplus(-s_b) + (1 - y_b) softplus(s_b) ].

Candidates: the C = min(2K, R) highest scores, ties to the smaller column
index, returned in ascending index order.

Certificate: run the K-step pivoted QR on the candidate columns only, giving
pivots j_0..j_{K-1}, orthonormal q_0..q_{K-1} and pivot norms |r_tt|.  For
every column o outside the candidate set let rho_o(t)^2 = ||y_o||^2 -
sum_{s<t} (q_s^T y_o)^2, its remaining norm after t steps.  If
rho_o(t) < |r_tt| for every such o and every t < K, the pivoted QR of all R
columns takes the same pivots in the same order (by induction on t: the
remaining norms of the candidates are the same in both runs, and no outside
column reaches the step's maximum).  Otherwise the proposal is rejected and
the plain QR runs.

Parity: features, MLP forward/backward and the certificate are pinned in
``tests/test_oracle_proposal.py`` (closed forms, finite differences, brute
force against the full pivoted QR).  The candidate set a trained model
produces is not unique in any useful sense ("parity unpinned" for the exact
candidate set); only the resulting ID is gated.
"""
from __future__ import annotations

import numpy as np

from .cpqr import cpqr
from .gaussian import round_bf16

NF = 8
HID = 128
RIDGE = (1e-1, 1e-2, 1e-3)
# flat parameter layout shared by the tests and the C ABI: row-major W1 (HID x NF),
# b1, row-major W2 (HID x HID), b2, w3, b3
SHAPES = (("W1", (HID, NF)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)), ("w3", (HID,)), ("b3", (1,)))
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def features(Y: np.ndarray, K: int) -> np.ndarray:
    """(R, NF) float64 feature matrix of the columns of Y (m x R)."""
    Y = np.asarray(Y, dtype=np.float64)
    m, R = Y.shape
    n = np.sum(Y * Y, axis=0)
    nmax = n.max()
    F = np.zeros((R, NF))
    F[:, 0] = -4.0
    F[:, 6] = K / R
    F[:, 7] = m / R
    if nmax == 0.0:
        return F
    with np.errstate(divide="ignore"):
        F[:, 0] = np.maximum(np.log(n / nmax), -64.0) / 16.0
    F[:, 1] = np.sqrt(n / nmax)
    G = Y @ Y.T
    tr = np.trace(G)
    for q, rho in enumerate(RIDGE):
        M = G + (rho * tr / m) * np.eye(m)
        X = np.linalg.solve(M, Y)
        F[:, 2 + q] = np.sum(Y * X, axis=0)
    amax = np.max(np.abs(Y), axis=0)
    nz = n > 0
    F[nz, 5] = amax[nz] / np.sqrt(n[nz])
    return F


def norm_scores(Y: np.ndarray) -> np.ndarray:
    """The norm-heuristic ablation's scores: the columns' 2-norms."""
    return np.sqrt(np.sum(np.asarray(Y, dtype=np.float64) ** 2, axis=0))


def labels(J, R: int) -> np.ndarray:
    """1 for the plain method's pivots, 0 elsewhere."""
    y = np.zeros(R)
    y[np.asarray(J)] = 1.0
    return y


# --------------------------------------------------------------------------- parameters
def unflatten(theta: np.ndarray) -> dict:
    theta = np.asarray(theta, dtype=np.float64)
    if theta.size != NPARAM:
        raise ValueError("expected %d parameters" % NPARAM)
    P, o = {}, 0
    for name, shape in SHAPES:
        sz = int(np.prod(shape))
        P[name] = theta[o:o + sz].reshape(shape).copy()
        o += sz
    return P


def flatten(P: dict) -> np.ndarray:
    return np.concatenate([np.asarray(P[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def init_params(seed: int) -> dict:
    """He-style random weights (test input; the library has its own initialiser)."""
    rng = np.random.default_rng(seed)
    P = dict(W1=rng.standard_normal((HID, NF)) * np.sqrt(2.0 / NF), b1=0.1 * rng.standard_normal(HID),
             W2=rng.standard_normal((HID, HID)) * np.sqrt(2.0 / HID), b2=0.1 * rng.standard_normal(HID),
             w3=rng.standard_normal(HID) * np.sqrt(1.0 / HID), b3=np.zeros(1))
    # float32-representable, as the device keeps its master weights in float32
    return {k: v.astype(np.float32).astype(np.float64) for k, v in P.items()}


def _operands(P: dict, F: np.ndarray, bf16: bool):
    if not bf16:
        return np.asarray(F, dtype=np.float64), P["W1"], P["W2"], P["w3"]
    rb = lambda a: round_bf16(np.asarray(a, dtype=np.float64).astype(np.float32)).astype(np.float64)
    return rb(F), rb(P["W1"]), rb(P["W2"]), rb(P["w3"])


def forward(P: dict, F: np.ndarray, bf16: bool = False):
    """Scores s (B,) and the activations the backward pass needs."""
    Fo, W1, W2, w3 = _operands(P, F, bf16)
    a1 = Fo @ W1.T + P["b1"]
    z1 = np.maximum(a1, 0.0)
    if bf16:
        z1 = round_bf16(z1.astype(np.float32)).astype(np.float64)
    a2 = z1 @ W2.T + P["b2"]
    z2 = np.maximum(a2, 0.0)
    s = z2 @ w3 + P["b3"][0]
    return s, dict(F=Fo, a1=a1, z1=z1, a2=a2, z2=z2, W2=W2, w3=w3)


def softplus(x):
    return np.logaddexp(0.0, x)


def loss(P: dict, F: np.ndarray, y: np.ndarray, pos_weight: float = 1.0, bf16: bool = False) -> float:
    s, _ = forward(P, F, bf16)
    return float(np.mean(pos_weight * y * softplus(-s) + (1.0 - y) * softplus(s)))


def backward(P: dict, F: np.ndarray, y: np.ndarray, pos_weight: float = 1.0, bf16: bool = False) -> dict:
    """Gradients of ``loss`` with respect to every parameter, by the chain rule."""
    s, c = forward(P, F, bf16)
    B = F.shape[0]
    sig = 1.0 / (1.0 + np.exp(-s))
    # d/ds of w y softplus(-s) + (1 - y) softplus(s), divided by B
    ds = (pos_weight * y * (sig - 1.0) + (1.0 - y) * sig) / B
    g = {"w3": c["z2"].T @ ds, "b3": np.array([ds.sum()])}
    da2 = np.outer(ds, c["w3"]) * (c["a2"] > 0)
    g["W2"] = da2.T @ c["z1"]
    g["b2"] = da2.sum(axis=0)
    da1 = (da2 @ c["W2"]) * (c["a1"] > 0)
    g["W1"] = da1.T @ c["F"]
    g["b1"] = da1.sum(axis=0)
    return g


def adam_step(theta, grad, m, v, t: int, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """One Adam update (Kingma & Ba, 2015) of flat parameters; t counts from 1.
    Returns the new (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


# --------------------------------------------------------------------------- candidates and certificate
def candidates(scores: np.ndarray, C: int) -> np.ndarray:
    """Indices of the C highest scores, ties to the smaller index, ascending."""
    scores = np.asarray(scores)
    order = np.lexsort((np.arange(len(scores)), -scores))
    return np.sort(order[:C])


def certificate(Y: np.ndarray, cand: np.ndarray, K: int):
    """(ok, J): the pivots of the QR restricted to the candidates (original
    indices, pivot order) and whether every outside column stays strictly
    below each step's pivot norm."""
    Y = np.asarray(Y, dtype=np.float64)
    m, R = Y.shape
    cand = np.asarray(cand)
    f = cpqr(Y[:, cand], K)
    J = cand[f["perm"][:K]]
    outside = np.setdiff1d(np.arange(R), cand)
    if outside.size == 0:
        return True, J
    Q, _ = np.linalg.qr(Y[:, J])                 # q_0..q_{K-1} span the pivots in order
    r2 = (Q.T @ Y[:, outside]) ** 2              # K x |outside|
    n = np.sum(Y[:, outside] ** 2, axis=0)
    rho2 = n[None, :] - np.vstack([np.zeros((1, outside.size)), np.cumsum(r2, axis=0)[:-1]])
    rho = np.sqrt(np.maximum(rho2, 0.0))
    ok = bool(np.all(rho < f["norms"][:, None]))
    return ok, J
