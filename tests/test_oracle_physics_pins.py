"""Pins of the oracle's offline physics model (Sec. "Building histograms",
Appendix A) against what mathematics and published constants fix, with no
reference to the numpy fixture in workloads/:

- Highland's width at x = X0 is 13.6 MeV / (beta c p), and its log term
  vanishes at x = X0 and cancels the width at x / X0 = exp(-1/0.038);
- the Landau width xi in the beta -> 1 limit equals 2 pi N_A r_e^2 m_e c^2
  (Z/A) rho x, from CODATA constants (not the oracle's rounded K);
- on the density-effect plateau the most probable loss obeys
  Delta_mp / xi = ln(2 m_e c^2 xi / (hbar omega_p)^2) + 1.2 - beta^2, with the
  plasma energy of iron as the PDG prints it;
- the ionisation loss is Moyal-distributed about Delta_mp with scale xi;
- the radiative tail is taken with the probability that makes the mean
  fractional loss b rho x (the definition of b), and has a v^-2 shape;
- the angle is a Highland-width Rayleigh variate, with a 1 % single-scatter
  tail whose density falls as theta^-3;
- histograms of a one-momentum bin hold the exact cell probabilities of those
  distributions (chi-square goodness of fit);
- Appendix A's pilot estimate equals the expectation of log(-dPz/P) under the
  model, computed by quadrature, within its statistical error.

Every sample here comes from or_physics_sample (fed chosen uniforms) or from
the oracle's own Philox-driven histogram and pilot loops."""
import math

import numpy as np
import pytest
import scipy.constants as sc
from scipy import stats

import oracle
from conftest import read_golden

MMU = sc.physical_constants["muon mass energy equivalent in MeV"][0]
ME = sc.physical_constants["electron mass energy equivalent in MeV"][0]
RE_CM = 100.0 * sc.physical_constants["classical electron radius"][0]
X_CM = 2.0                       # the 2 cm step of every workload


def _iron(b=0.0):
    g = {k[0]: float(v[0]) for k, v in read_golden("pdg_iron.txt")}
    mat = dict(rho=g["density_g_cm3"], ZA=g["Z_over_A"], I=g["mean_excitation_eV"] * 1e-6,
               X0=g["radiation_length_cm"], b=b)
    return mat, g["plasma_energy_eV"] * 1e-6


def _beta2(p_gev):
    pm = p_gev * 1e3
    return pm * pm / (pm * pm + MMU * MMU)


def _u(n=1, **fixed):
    """Rows of eight uniforms: u1, u2 (normal), u3, u4 (radiative), u5, u6, u7
    (angle) set so that no tail is taken unless asked; 'fixed' overrides."""
    U = np.tile(np.array([0.5, math.exp(-0.5), 0.0, 1.0 - 1e-12, 0.5, 1.0 - 1e-12, 0.5, math.exp(-0.5)]), (n, 1))
    for k, v in fixed.items():
        U[:, int(k[1:])] = v
    return U


def _xi_dmp(mat, p):
    """xi and Delta_mp read off the sampler: z = 1 gives the loss Delta_mp
    exactly (-ln z^2 = 0), z^2 = 1/e gives Delta_mp + xi."""
    pm = p * 1e3
    f0, _ = oracle.physics_samples(mat, p, X_CM, _u(u1=math.exp(-0.5)))
    f1, _ = oracle.physics_samples(mat, p, X_CM, _u(u1=math.exp(-0.5 * math.exp(-1.0))))
    return (f1[0] - f0[0]) * pm, f0[0] * pm


def test_highland_closed_forms():
    mat, _ = _iron()
    for p in (0.2, 1.0, 10.0, 1e3, 1e6):
        beta = math.sqrt(_beta2(p))
        # x = X0: sqrt(x/X0) = 1 and the log term vanishes
        assert oracle.highland(p, mat["X0"], mat["X0"]) * beta * p * 1e3 == pytest.approx(13.6, rel=1e-13)
    assert oracle.highland(1e6, 7.0, 7.0) == pytest.approx(13.6e-9, rel=1e-10)   # beta -> 1
    # the log correction cancels the width where 1 + 0.038 ln(x/X0) = 0
    assert abs(oracle.highland(5.0, mat["X0"] * math.exp(-1.0 / 0.038), mat["X0"])) < 1e-16


def test_landau_width_from_codata():
    mat, _ = _iron()
    xi_inf = 2.0 * math.pi * sc.N_A * RE_CM ** 2 * ME * mat["ZA"] * mat["rho"] * X_CM   # MeV
    xi, _ = _xi_dmp(mat, 1e5)
    assert xi == pytest.approx(xi_inf, rel=2e-6)      # PDG's K = 0.307075 is CODATA's rounded
    for p in (0.3, 1.0, 5.0):                         # xi grows as 1 / beta^2
        xi_p, _ = _xi_dmp(mat, p)
        assert xi_p * _beta2(p) == pytest.approx(xi, rel=1e-9)


def test_most_probable_loss_on_the_density_plateau():
    """With the density correction delta = 2 ln(beta gamma) + 2 ln(hbar omega_p / I) - 1,
    Delta_mp / xi = ln(2 m_e c^2 beta^2 gamma^2 / I) + ln(xi / I) + 0.2 - beta^2 - delta
    loses its dependence on I and on beta gamma."""
    mat, hw = _iron()
    for p in (50.0, 300.0, 1e4):
        xi, dmp = _xi_dmp(mat, p)
        expect = math.log(2.0 * ME * xi / hw ** 2) + 1.2 - _beta2(p)
        assert dmp / xi == pytest.approx(expect, abs=5e-5), p


def test_ionisation_loss_is_moyal():
    mat, _ = _iron()
    rng = np.random.default_rng(11)
    n = 20000
    p = 20.0
    xi, dmp = _xi_dmp(mat, p)
    U = _u(n, u1=rng.uniform(1e-12, 1.0, n), u2=rng.uniform(0.0, 1.0, n))
    f, _ = oracle.physics_samples(mat, p, X_CM, U)
    lam = (f * p * 1e3 - dmp) / xi
    assert stats.kstest(lam, stats.moyal.cdf).pvalue > 1e-3
    # the mode sits at Delta_mp: the densest 0.2-wide window of lambda is centred near 0
    h, e = np.histogram(lam, bins=np.arange(-3.0, 6.0, 0.2))
    mode = 0.5 * (e[np.argmax(h)] + e[np.argmax(h) + 1])
    assert abs(mode) <= 0.4


def test_radiative_tail_rate_mean_and_shape():
    p_rad_target = 0.3
    v0 = 1e-3
    mean_v = math.log(1.0 / v0) / (1.0 / v0 - 1.0)     # mean of the v^-2 density on [v0, 1)
    mat, _ = _iron()
    mat["b"] = p_rad_target * mean_v / (mat["rho"] * X_CM)
    rng = np.random.default_rng(12)
    n = 40000
    p = 30.0
    U = _u(n, u3=rng.uniform(0.0, 1.0, n), u4=rng.uniform(0.0, 1.0, n))
    f, _ = oracle.physics_samples(mat, p, X_CM, U)
    f_none, _ = oracle.physics_samples(mat, p, X_CM, _u(1))
    dv = f - f_none[0]
    rad = dv > 0.5 * v0
    assert stats.binomtest(int(rad.sum()), n, p_rad_target).pvalue > 1e-3
    assert np.all(np.abs(dv[~rad]) < 1e-15)
    # mean fractional radiative loss over the mass thickness rho x is b rho x
    se = dv.std() / math.sqrt(n)
    assert abs(dv.mean() - mat["b"] * mat["rho"] * X_CM) < 5.0 * se
    cdf = lambda v: np.clip((1.0 / v0 - 1.0 / np.maximum(v, v0)) / (1.0 / v0 - 1.0), 0.0, 1.0)
    assert stats.kstest(dv[rad], cdf).pvalue > 1e-3


def test_scattering_rayleigh_core_and_single_scatter_tail():
    mat, _ = _iron()
    p = 8.0
    th0 = oracle.highland(p, X_CM, mat["X0"])
    rng = np.random.default_rng(13)
    n = 20000
    # branch: u6 -> 1 makes a tail angle 2 theta0, u7 = e^-1/2 a core angle theta0
    _, th = oracle.physics_samples(mat, p, X_CM, _u(n, u5=rng.uniform(0.0, 1.0, n), u6=1.0))
    tail = th > 1.5 * th0
    assert np.all(np.isclose(th[tail], 2.0 * th0)) and np.all(np.isclose(th[~tail], th0))
    assert stats.binomtest(int(tail.sum()), n, 0.01).pvalue > 1e-3
    # core: theta / theta0 Rayleigh (a 2-D Gaussian of projected width theta0)
    _, th = oracle.physics_samples(mat, p, X_CM, _u(n, u7=rng.uniform(1e-12, 1.0, n)))
    assert stats.kstest(th / th0, stats.rayleigh.cdf).pvalue > 1e-3
    # tail: P(theta > t theta0) = (2/t)^2 for t >= 2, a theta^-3 density
    _, th = oracle.physics_samples(mat, p, X_CM, _u(n, u5=0.0, u6=rng.uniform(1e-12, 1.0, n)))
    assert stats.kstest(th / th0, stats.pareto(b=2.0, scale=2.0).cdf).pvalue > 1e-3


def _gof(counts, probs):
    keep = probs * counts.sum() > 5.0
    obs = np.append(counts[keep], counts[~keep].sum())
    exp = np.append(probs[keep], probs[~keep].sum()) * counts.sum()
    if exp[-1] == 0.0:
        obs, exp = obs[:-1], exp[:-1]
    return stats.chisquare(obs, exp).pvalue


def test_histogram_of_one_momentum_holds_the_exact_cell_probabilities():
    """A bin of zero width (p_a = p_b) makes every sample's momentum p, so the
    theta marginal is the Rayleigh + tail mixture at theta0(p), binned on
    [0, 5 theta0) with the overflow in the last cell, and (no radiative tail)
    the f marginal is the Moyal law of (f p - Delta_mp) / xi binned on [0, f_max)."""
    mat, _ = _iron(b=0.0)
    p = 12.0
    nf, nt, n = 40, 40, 400000
    xi, dmp = _xi_dmp(mat, p)
    f_max = 4.0 * dmp / (p * 1e3)
    counts, tmax = oracle.build_histograms([mat], [p, p], nf, nt, f_max, 0.02, n, 21)
    H = counts[0, 0]
    assert H.sum() == n
    th0 = oracle.highland(p, X_CM, mat["X0"])
    assert tmax[0, 0] == pytest.approx(5.0 * th0, rel=1e-15)
    t = np.linspace(0.0, 5.0, nt + 1)
    F = 0.99 * stats.rayleigh.cdf(t) + 0.01 * stats.pareto(b=2.0, scale=2.0).cdf(t)
    pt = np.diff(F)
    pt[-1] += 1.0 - F[-1]
    assert _gof(H.sum(axis=0), pt) > 1e-3
    fe = np.linspace(0.0, f_max, nf + 1)
    G = stats.moyal.cdf((fe * p * 1e3 - dmp) / xi)
    G[0] = 0.0                       # a loss floored at 0 lands in the first cell
    pf = np.diff(G)
    pf[-1] += 1.0 - G[-1]
    assert _gof(H.sum(axis=1), pf) > 1e-3


def test_pilot_estimate_equals_the_model_expectation():
    """Appendix A's pilot value at a momentum is the mean of log(-dPz/P) with
    -dPz/P = 1 - (1 - f) cos(theta).  With no radiative tail, f = (Delta_mp + xi
    lambda) / p with lambda Moyal and theta = theta0 r with r Rayleigh (99 %) or
    the 2 / sqrt(U) tail (1 %); the expectation is computed by midpoint
    quadrature in probability space and compared within the estimate's
    statistical error."""
    mat, _ = _iron(b=0.0)
    probes = np.array([2.0, 20.0, 200.0])
    K = 200000
    phi = oracle.pilot_phi(mat, probes, K, 0.02, 5)
    m = 2000
    q = (np.arange(m) + 0.5) / m
    lam = stats.moyal.ppf(q)
    r_core = stats.rayleigh.ppf(q)
    r_tail = stats.pareto(b=2.0, scale=2.0).ppf(q)
    for j, p in enumerate(probes):
        xi, dmp = _xi_dmp(mat, p)
        th0 = oracle.highland(p, X_CM, mat["X0"])
        f = np.minimum(np.maximum(dmp + xi * lam, 0.0) / (p * 1e3), 1.0)[:, None]

        def g(r):
            return np.log(f + (1.0 - f) * 2.0 * np.sin(0.5 * th0 * r[None, :]) ** 2)
        e1 = 0.99 * g(r_core).mean() + 0.01 * g(r_tail).mean()
        e2 = 0.99 * (g(r_core) ** 2).mean() + 0.01 * (g(r_tail) ** 2).mean()
        se = math.sqrt(max(e2 - e1 * e1, 0.0) / K)
        assert abs(phi[j] - e1) < 5.0 * se + 2e-3 * abs(e1) / m ** 0.5, (p, phi[j], e1, se)
    assert phi[0] > phi[1] > phi[2]


def test_pilot_estimate_is_the_mean_log_of_the_longitudinal_loss():
    """Sample by sample: the pilot loop draws the uniforms (w >> 8 + 1/2) 2^-24 of
    Philox4x32-10 (key = seed, counters (s, probe, 0x0FF1, 0 | 1)) and averages
    log(-dPz/P) with -dPz/P = 1 - (1 - f) cos(theta), f capped at 1.  A material
    with a strong radiative tail at low momentum makes f and theta both large,
    so every factor of that expression shows."""
    mat, _ = _iron()
    mat["b"] = 0.5 * math.log(1e3) / (1e3 - 1.0) / (mat["rho"] * X_CM)    # half the samples radiate
    probes = np.array([0.6, 3.0])
    K, seed = 3000, 77
    phi = oracle.pilot_phi(mat, probes, K, 0.02, seed)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for j, p in enumerate(probes):
        U = np.empty((K, 8))
        for s in range(K):
            for half in range(2):
                w = oracle.philox4x32_10([s, j, 0x0FF1, half], key)
                U[s, 4 * half:4 * half + 4] = ((w >> 8).astype(np.float64) + 0.5) * 2.0 ** -24
        f, th = oracle.physics_samples(mat, p, X_CM, U)
        f = np.minimum(f, 1.0)
        assert f.max() > 0.2 and th.max() > 0.02
        assert phi[j] == pytest.approx(np.mean(np.log(1.0 - (1.0 - f) * np.cos(th))), rel=1e-9)
