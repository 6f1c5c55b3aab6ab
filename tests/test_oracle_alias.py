"""Pins of the oracle's alias sampler (Sec. Methodology, "The Alias Method"):
a hand-built table, exact preservation of the integer masses of the inverse-CDF
thresholds (so both samplers draw from one quantised distribution), the
column/position boundaries of a draw, special cases, and chi-square of draws
through the full step draw."""
import math

import numpy as np
import pytest
from scipy import stats

import oracle
from test_oracle_pins import tiny_hist, vacuum_world
from workloads import gen


def masses(T, ncell):
    """Integer masses m_c = T_c - T_{c-1} of one threshold row (T_{N-1} = 2^32)."""
    t = np.concatenate([[0], np.asarray(T, dtype=np.uint64).astype(object), [1 << 32]])
    return np.array([int(t[c + 1]) - int(t[c]) for c in range(ncell)], dtype=object)


def counts_from_table(prob, alias):
    """Number of 32-bit draws w0 that pick each cell, read off the table: column j
    holds 2^(32-n) draws; the first ceil(Prob_j / 2^n) of them (r = w0 << n below
    Prob_j) take cell j, the rest take Alias_j."""
    N = len(prob)
    n = N.bit_length() - 1
    C = 1 << (32 - n)
    cnt = [0] * N
    for j in range(N):
        own = min(-(-int(prob[j]) // (1 << n)), C)
        cnt[j] += own
        cnt[int(alias[j])] += C - own
    return np.array(cnt, dtype=object)


def test_alias_hand_built_table():
    # weights 1, 1, 1, 5 (of 8): masses 2^29, 2^29, 2^29, 5 * 2^29; column capacity 2^30.
    # Cells 0..2 are small and cell 3 large; popping 2, 1, 0 in turn, each column
    # keeps half of its capacity (Prob = 2^29 * 4 = 2^31) and takes the rest from 3,
    # which ends with exactly 2^30 and fills its own column.
    T = oracle.build_thresholds(np.array([[1.0, 1.0], [1.0, 5.0]]))
    assert T.tolist() == [1 << 29, 1 << 30, 3 << 29]
    prob, alias = oracle.build_alias(T, 4)
    assert prob.tolist() == [1 << 31, 1 << 31, 1 << 31, 0xFFFFFFFF]
    assert alias.tolist() == [3, 3, 3, 3]


@pytest.mark.parametrize("shape,seed", [((2, 4), 1), ((4, 4), 2), ((8, 8), 3), ((16, 4), 4)])
def test_alias_preserves_integer_masses_exactly(shape, seed):
    rng = np.random.default_rng(seed)
    w = rng.integers(0, 50, size=shape).astype(np.float64)
    w.ravel()[rng.integers(0, w.size)] += 1.0          # at least one non-empty cell
    w.ravel()[-1] = 0.0                                # trailing empty cell
    T = oracle.build_thresholds(w)
    N = w.size
    prob, alias = oracle.build_alias(T, N)
    m = masses(T, N)
    assert sum(m) == 1 << 32
    cnt = counts_from_table(prob, alias)
    assert (cnt == m).all(), (cnt.tolist(), m.tolist())
    # zero-mass cells are never chosen: no draw reaches them through any column
    assert all(cnt[c] == 0 for c in range(N) if m[c] == 0)


def test_alias_preserves_masses_on_generated_histograms():
    h = gen.histogram_set(["iron", "air"], n_pbin=3, nf=128, ntheta=64, n_samples=20000, cache=False)
    T = oracle.build_thresholds(h["weights"])
    ncell = 128 * 64
    prob, alias = oracle.build_alias(T, ncell)
    for mat in range(2):
        for i in range(3):
            m = masses(T[mat, i], ncell)
            cnt = counts_from_table(prob[mat, i], alias[mat, i])
            assert (cnt == m).all()


def test_alias_draw_boundaries():
    rng = np.random.default_rng(7)
    w = rng.integers(1, 40, size=(4, 4)).astype(np.float64)
    T = oracle.build_thresholds(w)
    prob, alias = oracle.build_alias(T, 16)
    n, C = 4, 1 << 28
    partial = [j for j in range(16) if prob[j] != 0xFFFFFFFF]
    assert partial
    for j in partial:
        q = int(prob[j]) >> n                          # own share of column j in draws
        assert int(prob[j]) == q << n
        base = j * C
        if q > 0:
            assert oracle.sample_alias(prob, alias, base) == j
            assert oracle.sample_alias(prob, alias, base + q - 1) == j
        assert oracle.sample_alias(prob, alias, base + q) == alias[j]
        assert oracle.sample_alias(prob, alias, base + C - 1) == alias[j]
    for j in range(16):
        if prob[j] == 0xFFFFFFFF:
            assert oracle.sample_alias(prob, alias, j * C + C - 1) == j


def test_alias_uniform_and_single_cell():
    T = oracle.build_thresholds(np.ones((8, 4)))
    prob, alias = oracle.build_alias(T, 32)
    assert (prob == 0xFFFFFFFF).all() and alias.tolist() == list(range(32))
    rng = np.random.default_rng(3)
    for w0 in rng.integers(0, 1 << 32, size=200, dtype=np.uint64):
        assert oracle.sample_alias(prob, alias, int(w0)) == int(w0) >> 27
    w = np.zeros((8, 4))
    w[5, 2] = 3.0
    T = oracle.build_thresholds(w)
    prob, alias = oracle.build_alias(T, 32)
    for w0 in rng.integers(0, 1 << 32, size=200, dtype=np.uint64):
        assert oracle.sample_alias(prob, alias, int(w0)) == 5 * 4 + 2


def test_alias_rejects_non_power_of_two():
    T = oracle.build_thresholds(np.ones((3, 4)))
    with pytest.raises(ValueError):
        oracle.build_alias(T, 12)


def test_alias_chi_square_through_the_step_draw():
    rng = np.random.default_rng(5)
    w = rng.integers(0, 30, size=(8, 4)).astype(np.float64)
    w[0, 0] = 0.0
    w[3, :] = 0.0
    hist = dict(tiny_hist(w, n_pbin=1, f_max=0.2, theta_max=0.04), sampler="alias")
    world = vacuum_world(hist=hist, world_mat=1)
    world_icdf = vacuum_world(hist=tiny_hist(w, n_pbin=1, f_max=0.2, theta_max=0.04), world_mat=1)
    n = 60000
    counts = np.zeros(w.size)
    differ = 0
    for k in range(n):
        (_, _, _, cell), _ = oracle.draw(world, [0, 0, 0], [0, 0, 10.0], k, 17, 99)
        counts[cell] += 1
        if k < 2000:
            (_, _, _, c2), _ = oracle.draw(world_icdf, [0, 0, 0], [0, 0, 10.0], k, 17, 99)
            differ += c2 != cell
    prob = w.ravel() / w.sum()
    nz = prob > 0
    assert counts[~nz].sum() == 0
    chi2 = ((counts[nz] - n * prob[nz]) ** 2 / (n * prob[nz])).sum()
    assert stats.chi2.sf(chi2, nz.sum() - 1) > 1e-3
    assert differ > 100          # a different draw -> cell map from the inverse CDF


def test_alias_transport_matches_inverse_cdf_in_distribution():
    wl = gen.workload("block1e4", n=3000, hist_samples=20000)
    h_alias = dict(wl.hist, sampler="alias")
    a = oracle.transport(oracle.OracleWorld(wl.geometry, wl.field, h_alias), wl.muons, wl.step_len, wl.max_steps,
                         wl.seed)
    b = oracle.transport(oracle.world_of(wl), wl.muons, wl.step_len, wl.max_steps, wl.seed)
    Pa = np.sqrt(a["px"] ** 2 + a["py"] ** 2 + a["pz"] ** 2)
    Pb = np.sqrt(b["px"] ** 2 + b["py"] ** 2 + b["pz"] ** 2)
    assert not np.array_equal(Pa, Pb)
    for u, v in ((Pa, Pb), (a["x"], b["x"]), (a["y"], b["y"])):
        assert stats.ks_2samp(u, v).pvalue > 0.01
