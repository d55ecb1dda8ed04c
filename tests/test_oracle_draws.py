"""Pins of the oracle's draws (Sec. 1.3, Remark 2, Sec. 7.2) -- CPU only."""
import os

import numpy as np
import pytest
from scipy import stats

from oracle import draws
from oracle.countsketch import explicit_S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "splitmix64.txt")


def _golden():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        parts = line.split()
        rows.append((int(parts[0], 0), [int(p, 0) for p in parts[1:]]))
    return rows


def test_splitmix64_published_vectors():
    # the raw sequence mix64(x0 + (i+1) gamma) must reproduce the published outputs
    for x0, outs in _golden():
        got = [draws.mix64_int(x0 + (i + 1) * draws.GAMMA) for i in range(len(outs))]
        assert got == outs
        # array form of the same counter-based stream
        arr = draws.mix64(np.array([(x0 + (i + 1) * draws.GAMMA) & draws.MASK64
                                    for i in range(len(outs))], dtype=np.uint64))
        assert [int(v) for v in arr] == outs


def test_stream_is_counter_based_splitmix():
    seed, tag = 20190130, draws.TAG_SIGN
    b = draws.base_int(seed, tag)
    idx = np.array([0, 1, 2, 1000, 123456789])
    got = draws.stream(seed, tag, idx)
    want = [draws.mix64_int(b + (int(i) + 1) * draws.GAMMA) for i in idx]
    assert [int(v) for v in got] == want


def test_bounded_exact_against_bigint():
    rng = np.random.default_rng(0)
    us = list(rng.integers(0, 2**63, size=200, dtype=np.uint64) * np.uint64(2) + np.uint64(1))
    us += [np.uint64(0), np.uint64(2**64 - 1), np.uint64(2**63), np.uint64(2**32 - 1)]
    for L in [1, 2, 3, 900, 3600, 14400, 65535, 2**31 + 11, 2**32 - 1]:
        arr = np.array(us, dtype=np.uint64)
        got = draws.bounded(arr, L)
        want = [(int(u) * L) >> 64 for u in us]
        assert [int(v) for v in got] == want
        assert got.min() >= 0 and got.max() < L


def test_bounded_uniform_and_sign_balanced():
    L, n = 97, 200_000
    h = draws.bounded(draws.stream(5, draws.TAG_BUCKET, np.arange(n)), L)
    counts = np.bincount(h, minlength=L)
    chi2 = ((counts - n / L) ** 2 / (n / L)).sum()
    assert stats.chi2.sf(chi2, L - 1) > 1e-4
    s = draws.sign(draws.stream(5, draws.TAG_SIGN, np.arange(n)))
    assert set(np.unique(s)) == {-1, 1}
    assert abs(s.astype(np.int64).sum()) < 5 * np.sqrt(n)


@pytest.mark.parametrize("I", [1, 2, 3, 4, 5, 7, 16, 17, 100, 1000, 4096, 4097, 65537])
def test_permutation_is_bijection(I):
    p = draws.permutation(11, I)
    assert np.array_equal(np.sort(p), np.arange(I))


def test_permutation_spreads_uniformly():
    # position of element 0 under many keyed permutations of [13] is ~uniform
    I, n = 13, 6000
    pos = np.array([draws.permutation(seed, I, np.array([0]))[0] for seed in range(n)])
    counts = np.bincount(pos, minlength=I)
    chi2 = ((counts - n / I) ** 2 / (n / I)).sum()
    assert stats.chi2.sf(chi2, I - 1) > 1e-4


@pytest.mark.parametrize("I,L", [(50, 10), (4000, 900), (1000, 999), (131072, 14400)])
def test_modified_map_invariants(I, L):
    h, s = draws.countsketch_maps(3, I, L, modified=True)
    counts = np.bincount(h, minlength=L)
    assert len(counts) == L and counts.min() >= 1          # every bucket non-empty (Remark 2)
    assert h.min() >= 0 and h.max() < L
    # multiset = [0..L-1] plus I-L further draws: removing one of each bucket leaves I-L
    assert counts.sum() - L == I - L
    if I <= 4000:
        S = explicit_S(h, s, L)
        assert np.sum(S ** 2) == I                         # ||S||_F^2 = I (Lemma 4)
        assert np.linalg.matrix_rank(S) == L              # full rank (Remark 2)


def test_modified_map_needs_L_below_I():
    with pytest.raises(ValueError):
        draws.countsketch_maps(1, 10, 10, modified=True)


def test_collision_rates():
    """P(h(i) = h(i')) for i != i': 1/L for plain h (Sec. 7.1); 1/L - (L-1)/(I(I-1))
    for the modified map (Sec. 7.2).  Monte Carlo over seeds, within 5 sigma."""
    I, L, trials = 12, 8, 20000
    hits_p = hits_m = 0
    for seed in range(trials):
        hp, _ = draws.countsketch_maps(seed, I, L, modified=False)
        hm, _ = draws.countsketch_maps(seed, I, L, modified=True)
        hits_p += hp[0] == hp[1]
        hits_m += hm[0] == hm[1]
    for hits, p in [(hits_p, 1 / L), (hits_m, 1 / L - (L - 1) / (I * (I - 1)))]:
        sd = np.sqrt(p * (1 - p) / trials)
        assert abs(hits / trials - p) < 5 * sd, (hits / trials, p)


def test_gaussian_matrix_is_standard_normal():
    Om = draws.gaussian_matrix(9, 101, 999)     # odd m1: pairs straddle rows
    z = Om.ravel()
    assert abs(z.mean()) < 5 / np.sqrt(z.size)
    assert abs(z.var() - 1) < 5 * np.sqrt(2 / z.size)
    assert stats.kstest(z, "norm").pvalue > 1e-4
    # the two members of a Box-Muller pair are uncorrelated
    pairs = z[: (z.size // 2) * 2].reshape(-1, 2)
    assert abs(np.corrcoef(pairs[:, 0], pairs[:, 1])[0, 1]) < 5 / np.sqrt(len(pairs))


def test_gaussian_matrix_flat_indexing():
    # Omega(m2, m1) is a prefix-consistent reshape of one flat stream
    a = draws.gaussian_matrix(4, 3, 7).ravel()
    b = draws.gaussian_matrix(4, 7, 3).ravel()
    assert np.array_equal(a, b)


def test_tensor_maps_independent_per_mode():
    hs, ss = draws.tensorsketch_maps(2, [50, 50, 50], 64)
    assert not np.array_equal(hs[0], hs[1]) and not np.array_equal(ss[1], ss[2])
    for h in hs:
        assert h.min() >= 0 and h.max() < 64
