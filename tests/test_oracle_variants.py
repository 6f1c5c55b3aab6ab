"""Pins of the oracle's paper variants of the step: the nearest-node field
(Sec. Simulation item 3) against a brute-force nearest node, the log-scaled
(-dPz/P, dPt/P) histogram axes with Algorithm 1's additive dp (Sec. Building
histograms, Algorithm 1) against the angle form and closed forms, and the
adjoint through both against forward-mode dual numbers."""
import math

import numpy as np
import pytest
from scipy import stats

import oracle
from test_oracle_pins import tiny_hist, vacuum_world
from workloads import gen


def _random_map(rng, dims=(7, 5, 9), origin=(-1.0, -0.5, 2.0), spacing=(0.3, 0.25, 0.4)):
    B = rng.standard_normal((dims[2], dims[1], dims[0], 3)).astype(np.float32)
    return dict(kind="map_nearest", dims=list(dims), origin=list(origin), spacing=list(spacing), B=B)


def test_nearest_field_against_brute_force():
    rng = np.random.default_rng(3)
    fld = _random_map(rng)
    w = vacuum_world(field=fld)
    nodes = [fld["origin"][a] + fld["spacing"][a] * np.arange(fld["dims"][a]) for a in range(3)]
    lo = [fld["origin"][a] - 0.5 * fld["spacing"][a] for a in range(3)]
    hi = [nodes[a][-1] + 0.5 * fld["spacing"][a] for a in range(3)]
    n_in = 0
    for _ in range(3000):
        r = np.array([rng.uniform(lo[a] - 0.4, hi[a] + 0.4) for a in range(3)])
        inside = all(lo[a] <= r[a] < hi[a] for a in range(3))
        if inside:
            i = [int(np.argmin(np.abs(nodes[a] - r[a]))) for a in range(3)]
            expect = fld["B"][i[2], i[1], i[0]].astype(np.float64)
            n_in += 1
        else:
            expect = np.zeros(3)
        np.testing.assert_array_equal(w.field(r), expect)
    assert n_in > 1000
    # node values at the nodes
    for i, j, k in [(0, 0, 0), (6, 4, 8), (3, 2, 5)]:
        r = [nodes[0][i], nodes[1][j], nodes[2][k]]
        np.testing.assert_array_equal(w.field(r), fld["B"][k, j, i].astype(np.float64))


def test_additive_dp_equals_the_angle_form_and_closed_forms():
    rng = np.random.default_rng(11)
    for _ in range(300):
        p = rng.standard_normal(3) * rng.uniform(1, 100)
        f = 10 ** rng.uniform(-9, -0.5)
        t = 10 ** rng.uniform(-8, -0.5)
        phi = rng.uniform(0, 2 * math.pi)
        cz, ct = oracle.dp_coeffs("log", f, t)
        assert (cz, ct) == (-f, t)
        out = oracle.scatter_c(p, cz, ct, phi)
        # the same map in the angle form: |p_new| = P sqrt((1-f)^2 + t^2) at angle atan2(t, 1-f)
        r = math.hypot(1.0 - f, t)
        ref = oracle.scatter(p, 1.0 - r, math.atan2(t, 1.0 - f), phi)
        np.testing.assert_allclose(out, ref, rtol=0, atol=1e-12 * np.linalg.norm(p))
        P = np.linalg.norm(p)
        assert abs(np.linalg.norm(out) - P * r) <= 1e-12 * P
        ang = math.atan2(np.linalg.norm(np.cross(p, out)), float(np.dot(p, out)))
        assert abs(ang - math.atan2(t, 1.0 - f)) <= 1e-9
    # linear axes: the coefficients of the angle form
    cz, ct = oracle.dp_coeffs("linear", 0.1, 0.3)
    assert abs(cz - (0.9 * math.cos(0.3) - 1.0)) < 1e-15 and abs(ct - 0.9 * math.sin(0.3)) < 1e-15


def _log_hist(w, f_rng=(1e-6, 1e-1), t_rng=(1e-5, 1e-1)):
    nf, nt = w.shape
    return dict(n_mat=1, n_pbin=1, p_lo=1.0, p_hi=100.0, nf=nf, ntheta=nt, weights=w[None, None],
                f_min=np.full((1, 1), f_rng[0]), f_max=np.full((1, 1), f_rng[1]),
                theta_min=np.full((1, 1), t_rng[0]), theta_max=np.full((1, 1), t_rng[1]), axes="log")


def test_log_axes_draw_chi_square_and_log_uniform_jitter():
    rng = np.random.default_rng(4)
    w = rng.integers(0, 20, size=(8, 4)).astype(np.float64)
    w[2, :] = 0.0
    world = vacuum_world(hist=_log_hist(w), world_mat=1)
    n = 40000
    counts = np.zeros(w.size)
    ju, jv = np.zeros(n), np.zeros(n)
    for k in range(n):
        (_, _, _, cell), (f, t, phi) = oracle.draw(world, [0, 0, 0], [0, 0, 10.0], k, 5, 3)
        counts[cell] += 1
        a, b = divmod(cell, 4)
        ju[k] = math.log(f / 1e-6) / math.log(1e-1 / 1e-6) * 8 - a
        jv[k] = math.log(t / 1e-5) / math.log(1e-1 / 1e-5) * 4 - b
    prob = w.ravel() / w.sum()
    nz = prob > 0
    assert counts[~nz].sum() == 0
    chi2 = ((counts[nz] - n * prob[nz]) ** 2 / (n * prob[nz])).sum()
    assert stats.chi2.sf(chi2, nz.sum() - 1) > 1e-3
    assert ju.min() > -1e-9 and ju.max() < 1 + 1e-9 and jv.min() > -1e-9 and jv.max() < 1 + 1e-9
    assert stats.kstest(ju, "uniform").pvalue > 1e-3 and stats.kstest(jv, "uniform").pvalue > 1e-3


def test_log_axes_step_applies_the_additive_dp():
    w = np.zeros((4, 2))
    w[1, 1] = 1.0
    hist = _log_hist(w, f_rng=(1e-4, 1e-0), t_rng=(1e-3, 1e-1))
    world = vacuum_world(hist=hist, world_mat=1)
    p0 = np.array([0.3, -0.2, 20.0])
    out = oracle.trace(world, [0, 0, 0], p0, 1, 1, 0.02, 9, 0)
    (_, _, _, cell), (f, t, phi) = oracle.draw(world, [0, 0, 0], p0, 0, 0, 9)
    assert cell == 1 * 2 + 1
    P = np.linalg.norm(p0)
    # the step's momentum after scattering is Algorithm 1's p + Rot([P t cos phi, P t sin phi, -P f])
    p1 = oracle.scatter_c(p0, -f, t, phi)
    assert out["n"] == 1
    np.testing.assert_allclose(out["p_scat"][0], p1, rtol=0, atol=1e-12 * P)
    assert abs(np.linalg.norm(p1) - P * math.hypot(1 - f, t)) < 1e-12 * P


@pytest.mark.parametrize("variant", ["log_axes", "nearest_field"])
def test_adjoint_of_variants_matches_dual_numbers(variant):
    if variant == "log_axes":
        wl = gen.workload("shield1e6", n=80, hist_samples=20000, field="box", axes="log")
    else:
        wl = gen.workload("shield1e6", n=80, hist_samples=20000)
        wl.field = dict(gen.field_map_shield1e6(nx=60, ny=60, nz=180), kind="map_nearest")
    rng = np.random.default_rng(5)
    alpha = 1.0 + 0.2 * rng.standard_normal((6, 3))
    world = oracle.world_of(wl, alpha)
    fin = oracle.transport(world, wl.muons, wl.step_len, wl.max_steps, wl.seed)
    _, g = oracle.acceptance_loss(fin)
    adj = oracle.adjoint(world, wl.muons, wl.step_len, wl.max_steps, wl.seed, g)
    dual = np.zeros(18)
    for m in range(wl.n):
        r = [wl.muons[k][m] for k in ("x", "y", "z")]
        p = [wl.muons[k][m] for k in ("px", "py", "pz")]
        out, tan, ns = oracle.transport_tangent(world, r, p, int(wl.muons["q"][m]), wl.max_steps, wl.step_len,
                                                wl.seed, m)
        assert ns == fin["steps"][m]
        np.testing.assert_allclose(out, [fin[k][m] for k in ("x", "y", "z", "px", "py", "pz")], rtol=0, atol=1e-12)
        dual += g[:, m] @ tan
    scale = np.abs(dual).max()
    assert scale > 0
    np.testing.assert_allclose(adj.ravel(), dual, rtol=1e-9, atol=1e-12 * scale)


def _linear_field_map(b0=1.25, b1=0.75, per_stage=True):
    """A node map of B = (b1 z / 8, b0 + b1 z, 0), trilinear reproduces it exactly;
    dyadic nodes and coefficients make the float32 node values exact."""
    nx, ny, nz = 3, 3, 33
    z = -0.5 + 0.125 * np.arange(nz)
    B = np.zeros((nz, ny, nx, 3), np.float32)
    B[..., 0] = (0.125 * b1 * z)[:, None, None]
    B[..., 1] = (b0 + b1 * z)[:, None, None]
    return dict(kind="map", dims=[nx, ny, nz], origin=[-5.0, -5.0, -0.5], spacing=[5.0, 5.0, 0.125],
                B=np.ascontiguousarray(B), per_stage=per_stage)


def _ode_reference(r0, p0, q, L, b0=1.25, b1=0.75):
    from scipy.integrate import solve_ivp
    P0 = np.linalg.norm(p0)

    def rhs(s, y):
        r, p = y[:3], y[3:]
        Bv = np.array([0.125 * b1 * r[2], b0 + b1 * r[2], 0.0])
        return np.concatenate([p / P0, 0.299792458 * q * np.cross(p, Bv) / P0])
    sol = solve_ivp(rhs, (0.0, L), np.concatenate([r0, p0]), method="DOP853", rtol=1e-13, atol=1e-15)
    return sol.y[:, -1]


def _run(field, d, n_steps, r0, p0, q):
    geo = dict(kind="boxes", boxes=[], world_material=0, x_max=100.0, y_max=100.0, z_max=1e6, p_min=0.1)
    w = oracle.OracleWorld(geo, field, tiny_hist())
    mu = {k: np.array([v], np.float32) for k, v in zip(("x", "y", "z", "px", "py", "pz"), list(r0) + list(p0))}
    mu.update(q=np.array([q], np.int8), steps=np.zeros(1, np.int32), status=np.zeros(1, np.uint8))
    out = oracle.transport(w, mu, d, n_steps, 1)
    return np.array([out[k][0] for k in ("x", "y", "z", "px", "py", "pz")])


def test_per_stage_field_equals_fixed_field_in_a_uniform_map():
    fld_u = _linear_field_map(b1=0.0, per_stage=True)
    fld_f = dict(fld_u, per_stage=False)
    r0, p0 = np.array([0.1, -0.2, 0.0]), np.array([0.3, 0.1, 2.0])
    a = _run(fld_u, 0.02, 50, r0, p0, -1)
    b = _run(fld_f, 0.02, 50, r0, p0, -1)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-13)


def test_per_stage_field_is_fourth_order_in_a_varying_field():
    r0, p0, q, L = np.array([0.125, -0.25, 0.0]), np.array([0.25, 0.125, 2.0]), -1, 2.0   # exact in float32
    ref = _ode_reference(r0, p0, q, L)
    err = {}
    for per_stage in (True, False):
        fld = _linear_field_map(per_stage=per_stage)
        err[per_stage] = [np.abs(_run(fld, L / n, n, r0, p0, q) - ref).max() for n in (40, 80, 160)]
    e = err[True]
    assert 10.0 < e[0] / e[1] < 24.0 and 10.0 < e[1] / e[2] < 24.0, e       # ~16: fourth order
    f = err[False]
    assert 1.6 < f[0] / f[1] < 2.6 and 1.6 < f[1] / f[2] < 2.6, f           # ~2: the held field is first order
    assert e[0] < 1e-3 * f[0]
