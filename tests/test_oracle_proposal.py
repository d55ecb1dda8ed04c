"""Pins of the oracle's learned-proposal functions (features, MLP gradients,
Adam step, candidates, certificate) -- CPU only."""
import numpy as np
import pytest

from oracle import cpqr
from oracle import proposal as pr
from oracle.gaussian import round_bf16


def _rand_Y(seed, m, R):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((m, R)) * rng.uniform(0.2, 3.0, R)[None, :]


# --------------------------------------------------------------------------- features
def test_leverage_of_orthogonal_columns_closed_form():
    """Y = Q diag(d) with orthonormal Q: y_c^T (G + lam I)^{-1} y_c = d_c^2 / (d_c^2 + lam)."""
    rng = np.random.default_rng(1)
    m, R = 12, 7
    Q, _ = np.linalg.qr(rng.standard_normal((m, R)))
    d = rng.uniform(0.1, 4.0, R)
    Y = Q * d[None, :]
    F = pr.features(Y, 3)
    tr = np.sum(d ** 2)
    for q, rho in enumerate(pr.RIDGE):
        lam = rho * tr / m
        assert np.allclose(F[:, 2 + q], d ** 2 / (d ** 2 + lam), rtol=1e-12, atol=0)


def test_leverage_sum_matches_singular_values():
    """sum_c y_c^T (G + lam I)^{-1} y_c = sum_i s_i^2 / (s_i^2 + lam), s = singular values of Y."""
    Y = _rand_Y(2, 20, 90)
    F = pr.features(Y, 5)
    s = np.linalg.svd(Y, compute_uv=False)
    tr = np.sum(s ** 2)
    for q, rho in enumerate(pr.RIDGE):
        lam = rho * tr / Y.shape[0]
        assert abs(F[:, 2 + q].sum() - np.sum(s ** 2 / (s ** 2 + lam))) <= 1e-10 * F.shape[0]


def test_norm_features_by_hand():
    Y = np.array([[3.0, 0.0, 1.0], [4.0, 0.0, -1.0]])          # norms^2 25, 0, 2
    F = pr.features(Y, 1)
    assert np.allclose(F[:, 0], [0.0, -4.0, np.log(2 / 25) / 16])
    assert np.allclose(F[:, 1], [1.0, 0.0, np.sqrt(2 / 25)])
    assert np.allclose(F[:, 5], [4 / 5, 0.0, 1 / np.sqrt(2)])
    assert np.allclose(F[:, 6], 1 / 3) and np.allclose(F[:, 7], 2 / 3)
    assert F[1, 2] == 0.0 and F[1, 3] == 0.0 and F[1, 4] == 0.0


def test_features_zero_sketch_and_invariances():
    Z = np.zeros((5, 9))
    F = pr.features(Z, 2)
    assert np.all(F[:, 0] == -4.0) and np.all(F[:, 1:6] == 0.0)
    Y = _rand_Y(3, 10, 30)
    F = pr.features(Y, 4)
    assert np.allclose(pr.features(7.5 * Y, 4), F, atol=1e-12)      # scale invariant
    perm = np.random.default_rng(4).permutation(30)
    assert np.allclose(pr.features(Y[:, perm], 4), F[perm], atol=1e-12)  # permutation equivariant
    rot, _ = np.linalg.qr(np.random.default_rng(5).standard_normal((10, 10)))
    assert np.allclose(pr.features(rot @ Y, 4)[:, [0, 1, 2, 3, 4, 6, 7]], F[:, [0, 1, 2, 3, 4, 6, 7]], atol=1e-10)


# --------------------------------------------------------------------------- MLP
def test_forward_by_hand():
    """Selection weights make every layer computable by hand."""
    P = {k: np.zeros(s) for k, s in pr.SHAPES}
    P["W1"][0, 0] = 1.0      # z1_0 = relu(f0)
    P["W1"][1, 1] = -2.0     # z1_1 = relu(-2 f1 + 0.5)
    P["b1"][1] = 0.5
    P["W2"][0, 0] = 3.0      # z2_0 = relu(3 z1_0 - z1_1)
    P["W2"][0, 1] = -1.0
    P["b2"][2] = 0.25        # z2_2 = 0.25
    P["w3"][0] = 2.0
    P["w3"][2] = 4.0
    P["b3"][0] = -1.0
    F = np.zeros((2, pr.NF))
    F[0, 0], F[0, 1] = 0.5, 0.1      # z1 = (0.5, 0.3) -> z2_0 = 1.2 -> s = 2.4 + 1 - 1
    F[1, 0], F[1, 1] = -1.0, 0.0     # z1 = (0, 0.5)   -> z2_0 = 0   -> s = 0 + 1 - 1
    s, _ = pr.forward(P, F)
    assert np.allclose(s, [2.4, 0.0])


@pytest.mark.parametrize("pos_weight", [1.0, 7.0])
def test_backward_matches_central_differences(pos_weight):
    rng = np.random.default_rng(6)
    P = pr.init_params(7)
    F = rng.standard_normal((24, pr.NF))
    y = (rng.uniform(size=24) < 0.3).astype(float)
    g = pr.flatten(pr.backward(P, F, y, pos_weight))
    theta = pr.flatten(P)
    idx = rng.choice(pr.NPARAM, 300, replace=False)
    idx = np.concatenate([idx, [pr.NPARAM - 1, 0, 1024, 1024 + 128]])     # b3, W1, b1, W2 corners
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (pr.loss(pr.unflatten(tp), F, y, pos_weight) - pr.loss(pr.unflatten(tm), F, y, pos_weight)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1e-3, abs(g[i])) + 1e-10, (i, fd, g[i])


def test_bf16_forward_rounds_operands():
    """bf16 mode equals the exact forward on bf16-representable data and weights."""
    rng = np.random.default_rng(8)
    P = pr.init_params(9)
    for k in ("W1", "W2", "w3"):
        P[k] = round_bf16(P[k].astype(np.float32)).astype(np.float64)
    F = round_bf16(rng.standard_normal((10, pr.NF)).astype(np.float32)).astype(np.float64)
    s16, c16 = pr.forward(P, F, bf16=True)
    assert np.all(round_bf16(c16["z1"].astype(np.float32)) == c16["z1"])
    P2 = dict(P)
    s64, c64 = pr.forward(P2, F)
    assert np.allclose(c16["a1"], c64["a1"], rtol=0, atol=0)
    assert np.allclose(s16, s64, rtol=2e-2, atol=2e-2)


def test_adam_first_step_closed_form():
    """From zero moments the first Adam step is lr * g / (|g| + eps)."""
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    th, m, v = pr.adam_step(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, lr=0.01)
    assert np.allclose(th, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_param_layout_roundtrip():
    P = pr.init_params(10)
    theta = pr.flatten(P)
    assert theta.size == pr.NPARAM == 128 * 8 + 128 + 128 * 128 + 128 + 128 + 1
    Q = pr.unflatten(theta)
    assert all(np.array_equal(P[k], Q[k]) for k in P)


# --------------------------------------------------------------------------- candidates / certificate
def test_candidates_ties_smaller_index():
    s = np.array([1.0, 3.0, 3.0, 2.0, 3.0, 0.5])
    assert list(pr.candidates(s, 2)) == [1, 2]
    assert list(pr.candidates(s, 4)) == [1, 2, 3, 4]
    assert list(pr.candidates(s, 6)) == list(range(6))


def test_certificate_implies_plain_pivots_brute_force():
    """Whenever the certificate holds, the pivots equal those of the pivoted QR
    of all columns; and with every column a candidate it always holds."""
    rng = np.random.default_rng(11)
    held = 0
    for trial in range(200):
        m, R, K = int(rng.integers(4, 10)), int(rng.integers(8, 30)), 0
        K = int(rng.integers(1, min(m, R // 2) + 1))
        Y = rng.standard_normal((m, R)) * rng.uniform(0.1, 3.0, R)[None, :]
        C = min(2 * K, R)
        scores = pr.norm_scores(Y) + rng.uniform(0, 1.5, R)     # a noisy proposal
        cand = pr.candidates(scores, C)
        ok, J = pr.certificate(Y, cand, K)
        plain = cpqr.cpqr(Y, K)["perm"][:K]
        if ok:
            held += 1
            assert np.array_equal(J, plain), trial
        ok_all, J_all = pr.certificate(Y, np.arange(R), K)
        assert ok_all and np.array_equal(J_all, plain)
    assert 20 < held < 200            # both outcomes occur


def test_certificate_rejects_a_missed_pivot():
    """A dominant column left out of the candidates fails the certificate at step 0."""
    rng = np.random.default_rng(12)
    Y = rng.standard_normal((6, 12))
    Y[:, 5] *= 50.0
    cand = np.array([0, 1, 2, 3])
    ok, _ = pr.certificate(Y, cand, 2)
    assert not ok
    assert pr.certificate(Y, np.array([0, 1, 2, 5]), 1)[0] == (np.argmax(pr.norm_scores(Y)) == 5)
