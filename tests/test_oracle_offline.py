"""Pins of the oracle's offline phase (Sec. Building histograms, Appendix A):
the parametric physics sampler against the independent numpy fixture of the
same model, the pilot estimator of Appendix A against a direct Monte Carlo, the
bounded-variation edge recursion against its defining properties, and the
binary-search momentum bin against numpy."""
import numpy as np
import pytest
from scipy import stats

import oracle
from workloads import gen
from workloads.gen import _highland, _hist_one


def test_highland_width_matches_the_fixture():
    for name in ("iron", "air", "concrete", "lead"):
        X0 = gen.MATERIALS[name]["X0"]
        for p in (1.0, 10.0, 350.0):
            assert abs(oracle.highland(p, 2.0, X0) - float(_highland(np.array([p]), 2.0, X0)[0])) < 1e-15


@pytest.mark.parametrize("name,p_a,p_b", [("iron", 10.0, 11.0), ("concrete", 2.0, 2.2), ("air", 50.0, 55.0)])
def test_sampler_histograms_match_the_numpy_fixture(name, p_a, p_b):
    """Same model, independent code and random streams: two-sample chi-square
    of the f and theta marginals."""
    mat = gen.MATERIALS[name]
    n, nf, nt = 200000, 32, 16
    c_or, tmax = oracle.build_histograms([mat], [p_a, p_b], nf, nt, 0.02 if name != "air" else 2e-4, 0.02, n, 11)
    rng = np.random.default_rng(5)
    c_np, tmax_np = _hist_one(rng, mat, p_a, p_b, 2.0, 0.02 if name != "air" else 2e-4, nf, nt, n)
    assert abs(tmax[0, 0] - tmax_np) < 1e-15
    for axis in (1, 0):
        a, b = c_or[0, 0].sum(axis=axis), c_np.sum(axis=axis)
        keep = (a + b) > 20
        tab = np.stack([a[keep], b[keep]])
        chi2, pval, _, _ = stats.chi2_contingency(tab)
        assert pval > 1e-3, (name, axis, pval)


def test_pilot_estimator_matches_a_direct_monte_carlo():
    mat = gen.MATERIALS["iron"]
    probes = np.array([1.5, 12.0, 200.0])
    K = 50000
    phi = oracle.pilot_phi(mat, probes, K, 0.02, 7)
    rng = np.random.default_rng(3)
    for j, p in enumerate(probes):
        # the fixture's sampler at fixed p (p_a = p_b), the estimator written out
        vals = []
        f, th = _samples_fixture(rng, mat, p, 40000)
        fz = np.minimum(f, 1.0)
        fz = fz + (1.0 - fz) * 2.0 * np.sin(0.5 * th) ** 2
        lv = np.log(fz)
        sigma = lv.std() * np.sqrt(1 / 40000 + 1 / K)
        assert abs(phi[j] - lv.mean()) < 5 * sigma, (p, phi[j], lv.mean(), sigma)
    assert phi[0] > phi[1] > phi[2]            # relative loss falls with momentum


def _samples_fixture(rng, mat, p, n):
    """f and theta of the numpy fixture's model at fixed p (its histogram code, unbinned)."""
    pm = np.full(n, p * 1e3)
    E = np.sqrt(pm * pm + gen._MMU ** 2)
    beta2 = (pm / E) ** 2
    bg = pm / gen._MMU
    rho, ZA, I = mat["rho"], mat["ZA"], mat["I"]
    xi = 0.5 * gen._K * ZA * rho * 2.0 / beta2
    hw = 28.816e-6 * np.sqrt(rho * ZA)
    delta = np.maximum(0.0, 2.0 * np.log(bg) + 2.0 * np.log(hw / I) - 1.0)
    dmp = xi * (np.log(2.0 * gen._ME * bg * bg / I) + np.log(xi / I) + 0.2 - beta2 - delta)
    z = rng.standard_normal(n)
    dE = np.maximum(dmp + xi * -np.log(np.maximum(z * z, 1e-300)), 0.0)
    f = dE / pm
    v0 = 1e-3
    p_rad = min(1.0, mat["b"] * rho * 2.0 / (np.log(1 / v0) / (1 / v0 - 1)))
    rad = rng.random(n) < p_rad
    v = 1.0 / (1.0 / v0 - rng.random(n) * (1.0 / v0 - 1.0))
    f = f + np.where(rad, v, 0.0)
    th0 = _highland(np.full(n, p), 2.0, mat["X0"])
    single = rng.random(n) < 0.01
    th = np.where(single, 2 * th0 / np.sqrt(1 - rng.random(n)), th0 * np.sqrt(-2 * np.log(1 - rng.random(n))))
    return f, th


def _check_bv(probes, phi, eps, edges):
    idx = [int(np.searchsorted(probes, e)) for e in edges]
    assert edges[0] == probes[0] and edges[-1] == probes[-1]
    assert all(probes[i] == e for i, e in zip(idx, edges))
    for a, b in zip(idx[:-1], idx[1:]):
        assert b > a
        var = np.abs(phi[a:b + 1] - phi[a]).max()
        if b > a + 1:
            assert var <= eps                 # the bin's variation stays within eps
        if b < len(probes) - 1:               # and one more probe would exceed it
            assert np.abs(phi[a:b + 2] - phi[a]).max() > eps


def test_bv_edges_defining_properties():
    rng = np.random.default_rng(2)
    for trial in range(20):
        n = int(rng.integers(5, 300))
        probes = np.sort(rng.uniform(1, 400, n))
        phi = np.cumsum(rng.normal(0, 0.05, n)) + rng.normal(0, 0.01, n)
        eps = float(rng.uniform(0.01, 0.3))
        _check_bv(probes, phi, eps, oracle.bv_edges(probes, phi, eps))


def test_bv_edges_hand_example():
    probes = np.array([1.0, 2.0, 3.0, 4.0, 5.0, 6.0])
    phi = np.array([0.0, 0.1, 0.15, 0.5, 0.55, 2.0])
    # from 1: 2, 3 stay within 0.2, 4 does not -> edge 3; from 3: 4 (0.35) exceeds but is taken
    # (one probe at least); from 4: 5 within, 6 not -> edge 5; then 6
    assert oracle.bv_edges(probes, phi, 0.2).tolist() == [1.0, 3.0, 4.0, 5.0, 6.0]
    assert oracle.bv_edges(probes, phi, 10.0).tolist() == [1.0, 6.0]


def test_momentum_bin_over_edges():
    rng = np.random.default_rng(8)
    edges = np.sort(np.concatenate([[1.0, 400.0], rng.uniform(1.0, 400.0, 40)]))
    for P in np.concatenate([rng.uniform(0.5, 500.0, 3000), edges]):
        i = oracle.momentum_bin_edges(P, edges)
        expect = min(max(int(np.searchsorted(edges, P, side="right")) - 1, 0), len(edges) - 2)
        assert i == expect, (P, i, expect)
    # explicit log10 edges give the implicit log bins
    log_edges = gen.pbin_edges(1.0, 400.0, 64)
    for P in rng.uniform(0.5, 500.0, 2000):
        assert oracle.momentum_bin_edges(P, log_edges) == oracle.momentum_bin(P, 1.0, 400.0, 64)
