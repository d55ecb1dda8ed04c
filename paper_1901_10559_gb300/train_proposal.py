"""Trains the QR stage's column-proposal MLP and writes its weight file.

    python -m paper_1901_10559_gb300.train_proposal [--out FILE] [--seed S] ...

Training examples are the columns of Gaussian-stage sketches Y2 of synthetic
problems shaped like the batched workload: dense low-rank matrices (rows
log-uniform in [2048, 65536], columns log-uniform in [256, 2048], rank
r ~ U{8..64}, singular values d^i with d ~ U[0.7, 0.95], K = r, m2 = K + 10,
m1 = min(m2^2, rows/2)) and 4-way CP tensors (I_n = 200, R = 5000, unit-norm
N(0,1) factor columns, lambda_r = 10^(-6 r / K) for r < K and 1e-6 beyond,
K in {16, 32, 48, 64}, TensorSketch length 8192, m2 = K + 10).  Each sketch
is formed by the library's own stage kernels; its label vector marks the K
pivots of the plain pivoted QR (idl_proposal_labels).  Training runs the
library's MLP kernels (idl_train_proposal, Adam).  Every step runs on the
GPU; torch only generates the problems and holds the buffers.

``evaluate`` reports, on held-out problems, how often the learned proposal
and the norm-heuristic proposal are certified (the QR stage then skips the
full pivoted QR) and the QR stage's device time with each.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

import paper_1901_10559_gb300 as idl

DEFAULT_WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "proposal_weights.bin")


def problem_specs(seed: int, n_dense: int, n_cp: int):
    """Seeded problem shapes (the batched workload's recipe)."""
    rng = np.random.default_rng(seed)
    specs = []
    for b in range(n_dense):
        I = int(round(math.exp(rng.uniform(math.log(2048), math.log(65536)))))
        R = int(round(math.exp(rng.uniform(math.log(256), math.log(2048)))))
        r = int(rng.integers(8, 65))
        d = float(rng.uniform(0.7, 0.95))
        specs.append(dict(kind="dense", I=I, R=R, K=r, decay=d, m2=r + 10, m1=min((r + 10) ** 2, I // 2),
                          seed=int(seed * 7919 + b)))
    for b in range(n_cp):
        K = (16, 32, 48, 64)[b % 4]
        specs.append(dict(kind="cp", dims=(200, 200, 200, 200), R=5000, K=K, L=8192, m2=K + 10,
                          seed=int(seed * 7919 + 5000 + b)))
    return specs


def sketch(ctx, spec):
    """Y2 (R columns of m2 floats, device) of one problem, through the library's stages."""
    import torch
    g = torch.Generator(device="cuda").manual_seed(spec["seed"])
    m2 = spec["m2"]
    if spec["kind"] == "dense":
        I, R, r, d = spec["I"], spec["R"], spec["K"], spec["decay"]
        U = torch.randn(I, r, device="cuda", generator=g) / math.sqrt(I)
        V = torch.randn(R, r, device="cuda", generator=g) / math.sqrt(R)
        sig = torch.tensor([d ** (i + 1) for i in range(r)], device="cuda", dtype=torch.float32)
        A = ((U * sig) @ V.T).contiguous()
        A += (1e-6 * d / math.sqrt(max(I, R))) * torch.randn(I, R, device="cuda", generator=g)
        m1 = spec["m1"]
        h = torch.empty(I, dtype=torch.int32, device="cuda")
        s = torch.empty(I, dtype=torch.int8, device="cuda")
        idl.idl_draw_countsketch(ctx, spec["seed"], I, m1, True, h, s)
        ptr = torch.empty(m1 + 1, dtype=torch.int32, device="cuda")
        rows = torch.empty(I, dtype=torch.int32, device="cuda")
        idl.idl_bucket_offsets(ctx, h, I, m1, ptr, rows)
        ldy1 = (R + 31) // 32 * 32
        Y1 = torch.empty(m1 * ldy1, dtype=torch.float32, device="cuda")
        idl.idl_countsketch_dense(ctx, A, I, R, R, idl.IDL_F32, h, s, ptr, rows, m1, Y1, ldy1)
        del A, U, V
    else:
        R, L, K = spec["R"], spec["L"], spec["K"]
        facs = []
        for _ in spec["dims"]:
            F = torch.randn(R, spec["dims"][0], device="cuda", generator=g)
            facs.append((F / F.norm(dim=1, keepdim=True)).contiguous())
        r = torch.arange(R, device="cuda", dtype=torch.float64)
        lam = torch.where(r < K, 10.0 ** (-6.0 * r / K), torch.full_like(r, 1e-6))
        hs, ss = [], []
        for n, In in enumerate(spec["dims"]):
            h = torch.empty(In, dtype=torch.int32, device="cuda")
            s = torch.empty(In, dtype=torch.int8, device="cuda")
            idl.idl_draw_mode(ctx, spec["seed"], n, In, L, h, s)
            hs.append(h)
            ss.append(s)
        m1 = L
        ldy1 = (R + 31) // 32 * 32
        Y1 = torch.empty(m1 * ldy1, dtype=torch.float32, device="cuda")
        idl.idl_tensorsketch(ctx, facs, list(spec["dims"]), lam, hs, ss, L, Y1, ldy1)
    Om = torch.empty(m2 * m1, dtype=torch.float64, device="cuda")
    idl.idl_draw_gaussian(ctx, spec["seed"], m2, m1, Om)
    Y2 = torch.empty(spec["R"] * m2, dtype=torch.float32, device="cuda")
    idl.idl_gaussian_stage(ctx, Om, m2, m1, Y1, spec["R"], ldy1, idl.IDL_F32, idl.PREC_FP32, Y2, m2)
    return Y2


def collect(ctx, specs):
    """Features and plain-QR labels of every column of every problem (device tensors)."""
    import torch
    Fs, ys = [], []
    for sp in specs:
        Y2 = sketch(ctx, sp)
        R = sp["R"]
        F = torch.empty(R * 8, dtype=torch.float32, device="cuda")
        y = torch.empty(R, dtype=torch.float32, device="cuda")
        idl.idl_proposal_labels(ctx, Y2, sp["m2"], R, sp["m2"], sp["K"], F, y)
        Fs.append(F.view(R, 8))
        ys.append(y)
    return torch.cat(Fs).contiguous(), torch.cat(ys).contiguous()


def evaluate(ctx, specs, factors=(2, 4), reps=5):
    """Per problem kind: certified fraction of the learned and the norm-heuristic
    proposal for each candidate factor, whether J equals the plain QR's, and the
    QR stage's device time (mean of ``reps`` back-to-back calls) of each path."""
    import torch
    res = {}
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for sp in specs:
        r = res.setdefault(sp["kind"], {"problems": 0, "plain_us": 0.0})
        r["problems"] += 1
        Y2 = sketch(ctx, sp)
        m, R, K = sp["m2"], sp["R"], sp["K"]
        copies = [Y2.clone() for _ in range(reps)]
        Jp = torch.empty(K, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        ev0.record()
        for Yp in copies:
            idl.idl_cpqr(ctx, Yp, m, R, m, idl.IDL_F32, K, Jp)
        ev1.record()
        torch.cuda.synchronize()
        r["plain_us"] += 1e3 * ev0.elapsed_time(ev1) / reps
        Yf = torch.empty_like(Y2)
        J = torch.empty(K, dtype=torch.int32, device="cuda")
        for mode, name in ((idl.PROPOSAL_MLP, "mlp"), (idl.PROPOSAL_NORM, "norm")):
            for c in factors:
                key = "%s_c%d" % (name, c)
                ev0.record()
                for _ in range(reps):
                    idl.idl_cpqr_proposal(ctx, Y2, Yf, m, R, m, K, mode, J, cand_factor=c, sync=False)
                ev1.record()
                torch.cuda.synchronize()
                r[key + "_us"] = r.get(key + "_us", 0.0) + 1e3 * ev0.elapsed_time(ev1) / reps
                st = idl.idl_cpqr_proposal(ctx, Y2, Yf, m, R, m, K, mode, J, cand_factor=c)
                r[key + "_certified"] = r.get(key + "_certified", 0) + int(st == 1)
                r[key + "_same_J"] = r.get(key + "_same_J", 0) + int(torch.equal(J, Jp))
    for r in res.values():
        for k in list(r):
            if k.endswith("_us"):
                r[k] /= r["problems"]
    return res


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--out", default=DEFAULT_WEIGHTS)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--n-dense", type=int, default=256)
    ap.add_argument("--n-cp", type=int, default=64)
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--batch", type=int, default=4096)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--pos-weight", type=float, default=0.0, help="0: the negative / positive ratio")
    ap.add_argument("--eval-dense", type=int, default=48)
    ap.add_argument("--eval-cp", type=int, default=16)
    ap.add_argument("--report", default="")
    a = ap.parse_args(argv)
    import torch
    from paper_1901_10559_gb300 import build
    build.build()
    torch.cuda.init()
    ctx = idl.Context(0)
    t0 = time.time()
    F, y = collect(ctx, problem_specs(a.seed, a.n_dense, a.n_cp))
    n = int(y.numel())
    npos = float(y.sum().item())
    pw = a.pos_weight if a.pos_weight > 0 else (n - npos) / max(npos, 1.0)
    t1 = time.time()
    idl.idl_mlp_init(ctx, a.seed)
    losses = idl.idl_train_proposal(ctx, F, y, n, epochs=a.epochs, batch=a.batch, lr=a.lr, pos_weight=pw,
                                    seed=a.seed)
    t2 = time.time()
    idl.idl_save_weights(ctx, a.out)
    ev = evaluate(ctx, problem_specs(a.seed + 1000, a.eval_dense, a.eval_cp))
    rep = dict(examples=n, positives=int(npos), pos_weight=pw, epochs=a.epochs, batch=a.batch, lr=a.lr,
               loss_first=losses[0], loss_last=losses[-1], collect_s=t1 - t0, train_s=t2 - t1, eval=ev)
    print(json.dumps(rep))
    if a.report:
        with open(a.report, "w") as f:
            json.dump(rep, f, indent=1)
    ctx.close()


if __name__ == "__main__":
    main()
