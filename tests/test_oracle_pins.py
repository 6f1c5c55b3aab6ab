"""Pins of the FP64 oracle against facts fixed outside it: published known-answer
vectors, the paper's worked binning example, closed forms (straight lines,
helices), invariants of the rotation, exact integer thresholds on tiny
histograms, brute force over lattices, and chi-square against the histogram.
"""
import math
from fractions import Fraction

import numpy as np
import pytest
from scipy import stats

import oracle
from conftest import read_golden
from workloads import gen

KAPPA = 0.299792458


def vacuum_world(field=None, x_max=100.0, y_max=100.0, z_max=1e6, p_min=0.5, boxes=(), world_mat=0,
                 hist=None, alpha=None):
    geo = dict(kind="boxes", boxes=list(boxes), world_material=world_mat, x_max=x_max, y_max=y_max,
               z_max=z_max, p_min=p_min)
    if hist is None:
        hist = tiny_hist()
    return oracle.OracleWorld(geo, field or dict(kind="none"), hist, alpha)


def tiny_hist(weights=None, n_pbin=4, p_lo=1.0, p_hi=100.0, f_max=0.1, theta_max=0.01):
    if weights is None:
        weights = np.array([[3.0, 1.0], [0.0, 2.0]])
    w = np.asarray(weights, dtype=np.float64)
    nf, nt = w.shape
    W = np.broadcast_to(w, (1, n_pbin, nf, nt)).copy()
    return dict(n_mat=1, n_pbin=n_pbin, p_lo=p_lo, p_hi=p_hi, nf=nf, ntheta=nt, weights=W,
                f_max=np.full((1, n_pbin), f_max), theta_max=np.full((1, n_pbin), theta_max))


# --------------------------------------------------------------------------
# S3: Philox4x32-10
# --------------------------------------------------------------------------
def test_philox_known_answers():
    rows = read_golden("philox4x32_10_kat.txt")
    assert len(rows) == 3
    for lhs, rhs in rows:
        v = [int(t, 16) for t in lhs]
        out = oracle.philox4x32_10(v[:4], v[4:6])
        assert [int(t, 16) for t in rhs] == [int(x) for x in out]


def test_uniform_from_top_24_bits():
    assert oracle.uniform(0) == 0.0
    assert oracle.uniform(255) == 0.0
    assert oracle.uniform(256) == 2.0 ** -24
    assert oracle.uniform(0xFFFFFFFF) == 1.0 - 2.0 ** -24


# --------------------------------------------------------------------------
# S4: thresholds and inverse-CDF cell choice
# --------------------------------------------------------------------------
def test_thresholds_tiny_exact():
    # weights 1,0 / 2,1 -> CDF 1/4, 1/4, 3/4 -> T = 2^30, 2^30, 3*2^30
    T = oracle.build_thresholds(np.array([[1.0, 0.0], [2.0, 1.0]]))
    assert [int(t) for t in T] == [2 ** 30, 2 ** 30, 3 * 2 ** 30]
    cases = {0: 0, 2 ** 30 - 1: 0, 2 ** 30: 2, 3 * 2 ** 30 - 1: 2, 3 * 2 ** 30: 3, 2 ** 32 - 1: 3}
    for w0, cell in cases.items():
        assert oracle.sample_cell(T, w0) == cell
    # the empty cell 1 is never chosen at any band boundary
    for w0 in (2 ** 30 - 1, 2 ** 30, 2 ** 30 + 1):
        assert oracle.sample_cell(T, w0) != 1


def test_thresholds_trailing_empty_cells():
    T = oracle.build_thresholds(np.array([[1.0, 1.0], [0.0, 0.0]]))
    assert [int(t) for t in T] == [2 ** 31, 2 ** 32, 2 ** 32]
    assert oracle.sample_cell(T, 2 ** 32 - 1) == 1
    assert oracle.sample_cell(T, 2 ** 31 - 1) == 0
    assert oracle.sample_cell(T, 2 ** 31) == 1


def test_thresholds_reject_bad_weights():
    for bad in ([[1.0, -1.0], [1.0, 1.0]], [[1.0, np.nan], [1.0, 1.0]], [[0.0, 0.0], [0.0, 0.0]],
                [[1.0, np.inf], [1.0, 1.0]]):
        with pytest.raises(ValueError):
            oracle.build_thresholds(np.array(bad))


def test_threshold_band_masses_match_weights():
    rng = np.random.default_rng(3)
    w = rng.integers(0, 50, size=(6, 5)).astype(np.float64)
    w[2, :] = 0.0
    T = [int(t) for t in oracle.build_thresholds(w)]
    flat = w.ravel()
    tot = Fraction(int(flat.sum()))
    edges = [0] + T + [2 ** 32]
    for c in range(len(flat)):
        exact_hi = Fraction(int(flat[: c + 1].sum())) / tot * 2 ** 32
        if c < len(flat) - 1:
            assert abs(edges[c + 1] - exact_hi) < 1   # floor of the exact CDF, to rounding
        width = edges[c + 1] - edges[c]
        assert abs(Fraction(width, 2 ** 32) - Fraction(int(flat[c])) / tot) <= Fraction(2, 2 ** 32)
        if width > 0:
            assert oracle.sample_cell(np.array(T, np.uint64), edges[c]) == c
            assert oracle.sample_cell(np.array(T, np.uint64), edges[c + 1] - 1) == c


def test_sampler_chi_square_and_jitter():
    rng = np.random.default_rng(5)
    w = rng.integers(0, 30, size=(8, 4)).astype(np.float64)
    w[0, 0] = 0.0
    w[3, :] = 0.0
    hist = tiny_hist(w, n_pbin=1, f_max=0.2, theta_max=0.04)
    world = vacuum_world(hist=hist, world_mat=1)
    n = 60000
    counts = np.zeros(w.size)
    fs = np.zeros(n)
    ths = np.zeros(n)
    phis = np.zeros(n)
    cells = np.zeros(n, np.int64)
    for k in range(n):
        (mat, box, pbin, cell), (f, th, phi) = oracle.draw(world, [0, 0, 0], [0, 0, 10.0], k, 17, 99)
        assert mat == 1 and box == -1 and pbin == 0
        counts[cell] += 1
        fs[k], ths[k], phis[k], cells[k] = f, th, phi, cell
    prob = w.ravel() / w.sum()
    nz = prob > 0
    assert counts[~nz].sum() == 0
    chi2 = ((counts[nz] - n * prob[nz]) ** 2 / (n * prob[nz])).sum()
    pval = stats.chi2.sf(chi2, nz.sum() - 1)
    assert pval > 1e-3, (chi2, pval)
    # jitter stays inside the chosen cell and is uniform there
    a, b = cells // 4, cells % 4
    fu = fs / 0.2 * 8 - a
    tu = ths / 0.04 * 4 - b
    assert fu.min() >= -1e-12 and fu.max() < 1 + 1e-12
    assert tu.min() >= -1e-12 and tu.max() < 1 + 1e-12
    assert abs(fu.mean() - 0.5) < 0.01 and abs(tu.mean() - 0.5) < 0.01
    assert stats.kstest(fu, "uniform").pvalue > 1e-3
    assert stats.kstest(phis / (2 * math.pi), "uniform").pvalue > 1e-3


# --------------------------------------------------------------------------
# S2: momentum bins
# --------------------------------------------------------------------------
def test_momentum_bin_paper_example():
    rows = read_golden("momentum_bin_example.txt")
    for lhs, rhs in rows:
        n, lo, hi = int(lhs[0]), float(lhs[1]), float(lhs[2])
        P, expect = float(rhs[0]), int(rhs[1])
        assert oracle.momentum_bin(P, lo, hi, n) == expect


def test_momentum_bin_edges_and_clamp():
    n, lo, hi = 64, 1.0, 400.0
    edges = gen.pbin_edges(lo, hi, n)
    for k in range(1, n):
        assert oracle.momentum_bin(edges[k] * (1 + 1e-12), lo, hi, n) == k
        assert oracle.momentum_bin(edges[k] * (1 - 1e-12), lo, hi, n) == k - 1
    assert oracle.momentum_bin(0.5, lo, hi, n) == 0
    assert oracle.momentum_bin(399.999, lo, hi, n) == n - 1
    assert oracle.momentum_bin(1e4, lo, hi, n) == n - 1
    assert oracle.momentum_bin(float("nan"), lo, hi, n) == 0


# --------------------------------------------------------------------------
# S1: material lookup
# --------------------------------------------------------------------------
def _first_box_numpy(geo, pts):
    mat = np.full(len(pts), geo["world_material"])
    box = np.full(len(pts), -1)
    done = np.zeros(len(pts), bool)
    for b, bx in enumerate(geo["boxes"]):
        lo, hi = np.array(bx["lo"]), np.array(bx["hi"])
        inside = np.all((pts >= lo) & (pts < hi), axis=1) & ~done
        mat[inside] = bx["material"]
        box[inside] = b
        done |= inside
    return mat, box


def test_material_boxes_lattice():
    geo = gen.geometry_shield1e6()
    # overlapping extra box after the others: list order decides
    geo["boxes"].append(dict(lo=[-1.0, -1.0, 3.0], hi=[1.0, 1.0, 5.0], material=3, block_id=-1, B=[0, 0, 0]))
    world = oracle.OracleWorld(geo, dict(kind="none"), tiny_hist())
    xs = np.array([-3.0, -1.0, -0.6, -0.3, 0.0, 0.6, 0.59999999, 1.0, 2.9])
    zs = np.array([-0.1, 0.0, 2.0, 3.99999, 4.0, 4.5, 4.2, 26.5, 26.4999, 27.0, 28.9, 29.0, 29.5])
    pts = np.array([[x, y, z] for x in xs for y in xs[::2] for z in zs])
    mat_np, box_np = _first_box_numpy(geo, pts)
    for p, m, b in zip(pts, mat_np, box_np):
        assert world.material(p) == (m, b)


def test_material_voxels_vs_numpy_indexing():
    rng = np.random.default_rng(11)
    vox = rng.integers(0, 4, size=(7, 5, 6)).astype(np.uint8)   # [nz][ny][nx]
    geo = dict(kind="voxels", voxels=vox, origin=[-1.5, -1.25, 0.0], spacing=[0.5, 0.5, 0.25],
               world_material=2, x_max=9, y_max=9, z_max=9, p_min=0.5)
    hist = tiny_hist()
    hist = dict(hist, n_mat=3, weights=np.repeat(hist["weights"], 3, 0), f_max=np.repeat(hist["f_max"], 3, 0),
                theta_max=np.repeat(hist["theta_max"], 3, 0))
    world = oracle.OracleWorld(geo, dict(kind="none"), hist)
    pts = rng.uniform([-2, -2, -0.5], [2, 2, 2.25], size=(3000, 3))
    pts[:50, 0] = -1.5 + 0.5 * rng.integers(0, 6, 50)      # exact voxel faces
    for p in pts:
        ijk = np.floor((p - np.array([-1.5, -1.25, 0.0])) / np.array([0.5, 0.5, 0.25])).astype(int)
        if np.all(ijk >= 0) and np.all(ijk < [6, 5, 7]):
            expect = int(vox[ijk[2], ijk[1], ijk[0]])
        else:
            expect = 2
        assert world.material(p)[0] == expect


# --------------------------------------------------------------------------
# S6: field lookup
# --------------------------------------------------------------------------
def _map_field(B, origin, spacing):
    nz, ny, nx, _ = B.shape
    return dict(kind="map", dims=[nx, ny, nz], origin=origin, spacing=spacing, B=B)


def test_trilinear_reproduces_affine_fields():
    nx, ny, nz = 5, 4, 6
    origin, spacing = [-1.0, 0.5, 2.0], [0.5, 0.25, 0.5]
    A = np.array([[1.0, -2.0, 0.5], [0.25, 3.0, -1.0], [2.0, 0.0, 1.5]])
    b = np.array([0.5, -1.0, 0.25])
    ii, jj, kk = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    pos = np.stack([origin[0] + ii * spacing[0], origin[1] + jj * spacing[1], origin[2] + kk * spacing[2]], -1)
    vals = pos @ A.T + b                                   # exact in float32 (dyadic)
    B = np.transpose(vals, (2, 1, 0, 3)).astype(np.float32)
    assert np.array_equal(B.astype(np.float64), np.transpose(vals, (2, 1, 0, 3)))
    world = vacuum_world(field=_map_field(B, origin, spacing))
    rng = np.random.default_rng(1)
    hi = np.array(origin) + (np.array([nx, ny, nz]) - 1) * np.array(spacing)
    for r in rng.uniform(origin, hi, size=(500, 3)):
        np.testing.assert_allclose(world.field(r), A @ r + b, rtol=0, atol=1e-12)
    # nodes return node values; the far corner is inside; just outside is zero
    np.testing.assert_allclose(world.field(hi), A @ hi + b, atol=1e-12)
    np.testing.assert_array_equal(world.field(hi + [1e-9, 0, 0]), 0.0)
    np.testing.assert_array_equal(world.field(np.array(origin) - [0, 1e-9, 0]), 0.0)


def test_field_nodes_random_map():
    rng = np.random.default_rng(2)
    B = rng.normal(size=(4, 3, 5, 3)).astype(np.float32)
    origin, spacing = [0.0, 0.0, 0.0], [0.1, 0.2, 0.3]
    world = vacuum_world(field=_map_field(B, origin, spacing))
    for k in range(4):
        for j in range(3):
            for i in range(5):
                r = np.array([i * 0.1, j * 0.2, k * 0.3])
                np.testing.assert_allclose(world.field(r), B[k, j, i], rtol=1e-9, atol=1e-9)


def test_box_field_and_block_scale():
    geo = gen.geometry_shield1e6()
    alpha = np.arange(1, 19, dtype=np.float64).reshape(6, 3) / 10.0
    world = oracle.OracleWorld(geo, dict(kind="box"), tiny_hist(), alpha)
    for k in range(6):
        r = np.array([0.1, -0.2, 4.5 * k + 1.0])
        m, b = world.material(r)
        assert (m, b) == (1, k)
        B = world.field(r, b)
        np.testing.assert_allclose(B, alpha[k] * np.array(geo["boxes"][k]["B"]), rtol=1e-15)
    r = np.array([0.0, 0.0, 28.0])       # concrete: no block id, no field
    m, b = world.material(r)
    assert (m, b) == (3, 6)
    np.testing.assert_array_equal(world.field(r, b), 0.0)


# --------------------------------------------------------------------------
# S5: rotation (Eq. 3)
# --------------------------------------------------------------------------
def _rot_columns(p):
    P = np.linalg.norm(p)
    ex = oracle.scatter(p, 0.0, math.pi / 2, 0.0) / P
    ey = oracle.scatter(p, 0.0, math.pi / 2, math.pi / 2) / P
    ez = oracle.scatter(p, 0.0, 0.0, 0.0) / P
    return np.stack([ex, ey, ez], 1)


def test_rotation_is_proper_and_maps_z_to_direction():
    rng = np.random.default_rng(4)
    for _ in range(200):
        p = rng.normal(size=3) * rng.uniform(0.5, 300)
        R = _rot_columns(p)
        np.testing.assert_allclose(R.T @ R, np.eye(3), atol=1e-12)
        assert abs(np.linalg.det(R) - 1.0) < 1e-12
        np.testing.assert_allclose(R[:, 2], p / np.linalg.norm(p), atol=1e-14)


def test_scatter_invariants():
    rng = np.random.default_rng(6)
    for _ in range(300):
        p = rng.normal(size=3) * rng.uniform(0.5, 300)
        f = rng.uniform(0, 0.2)
        th = rng.uniform(0, 0.3)
        ph1, ph2 = rng.uniform(0, 2 * math.pi, 2)
        q1 = oracle.scatter(p, f, th, ph1)
        q2 = oracle.scatter(p, f, th, ph2)
        P = np.linalg.norm(p)
        assert abs(np.linalg.norm(q1) - (1 - f) * P) <= 1e-12 * P
        cosang = q1 @ p / (np.linalg.norm(q1) * P)
        assert abs(math.acos(min(1.0, cosang)) - th) < 1e-7
        # azimuths differ by ph2 - ph1 around p
        u = p / P
        t1 = q1 - (q1 @ u) * u
        t2 = q2 - (q2 @ u) * u
        if th > 1e-3:
            cosd = t1 @ t2 / (np.linalg.norm(t1) * np.linalg.norm(t2))
            assert abs(cosd - math.cos(ph2 - ph1)) < 1e-9


def test_scatter_along_axes():
    P, f, th, ph = 7.0, 0.05, 0.2, 1.1
    s = P * (1 - f)
    exp_up = s * np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
    np.testing.assert_allclose(oracle.scatter([0, 0, P], f, th, ph), exp_up, atol=1e-13)
    exp_dn = exp_up * np.array([1, -1, -1])
    np.testing.assert_allclose(oracle.scatter([0, 0, -P], f, th, ph), exp_dn, atol=1e-13)
    # f = 0, theta = 0 leaves p unchanged
    p = np.array([0.3, -1.2, 5.0])
    np.testing.assert_allclose(oracle.scatter(p, 0.0, 0.0, 2.0), p, atol=1e-14)


# --------------------------------------------------------------------------
# S7: RK4 in a fixed field
# --------------------------------------------------------------------------
def test_rk4_straight_line_without_field():
    r = np.array([0.1, -0.2, 0.3])
    p = np.array([1.0, 2.0, 20.0])
    u = p / np.linalg.norm(p)
    r0 = r.copy()
    for n in range(1, 301):
        r, p = oracle.rk4(r, p, [0, 0, 0], 1, 0.02)
    np.testing.assert_allclose(r, r0 + 300 * 0.02 * u, atol=1e-12)
    np.testing.assert_allclose(p, [1.0, 2.0, 20.0], atol=0)


@pytest.mark.parametrize("q", [1, -1])
def test_rk4_helix_closed_form(q):
    Bz, pt, pz, d, n = 1.5, 2.0, 7.0, 0.02, 1000
    P = math.hypot(pt, pz)
    r = np.array([0.0, 0.0, 0.0])
    p = np.array([pt, 0.0, pz])
    for _ in range(n):
        r, p = oracle.rk4(r, p, [0, 0, Bz], q, d)
    s = n * d
    w = KAPPA * q * Bz / P
    x = (pt / P) * math.sin(w * s) / w
    y = (pt / P) * (math.cos(w * s) - 1.0) / w
    np.testing.assert_allclose(r, [x, y, s * pz / P], atol=1e-9)
    np.testing.assert_allclose(p, [pt * math.cos(w * s), -pt * math.sin(w * s), pz], atol=1e-9)
    # the projected track is a circle of radius p_T / (kappa |q| B) about (0, -(p_T/P)/w)
    R = pt / (KAPPA * Bz)
    yc = -(pt / P) / w
    assert abs(math.hypot(r[0], r[1] - yc) - R) < 1e-9


@pytest.mark.parametrize("q", [1, -1])
def test_rk4_equals_taylor_polynomial_of_the_generator(q):
    """With B and P0 held, dp/ds = A p is linear (A v = kappa q (v x B) / P0), so one
    classical RK4 step is the degree-4 Taylor polynomial of exp(dA): p1 = T4(dA) p and
    r1 = r + (d/P0) (I + dA/2 + (dA)^2/6 + (dA)^3/24) p.  Written here with 3x3
    matrices, independently of the oracle's stage form (a wrong stage weight, sign or
    operand order there fails it)."""
    rng = np.random.default_rng(11)
    for _ in range(20):
        r = rng.normal(size=3)
        p = rng.normal(size=3) * np.array([1.0, 1.0, 8.0])
        B = rng.normal(size=3) * 1.7
        d = 0.02 * rng.uniform(0.5, 50.0)
        P0 = np.linalg.norm(p)
        Bx = np.array([[0.0, B[2], -B[1]], [-B[2], 0.0, B[0]], [B[1], -B[0], 0.0]])   # v -> v x B
        M = d * KAPPA * q / P0 * Bx
        I = np.eye(3)
        M2 = M @ M
        M3 = M2 @ M
        p1 = (I + M + M2 / 2 + M3 / 6 + M3 @ M / 24) @ p
        r1 = r + d / P0 * ((I + M / 2 + M2 / 6 + M3 / 24) @ p)
        ro, po = oracle.rk4(r, p, B, q, d)
        np.testing.assert_allclose(po, p1, rtol=0, atol=1e-13 * P0)
        np.testing.assert_allclose(ro, r1, rtol=0, atol=1e-13 * (1.0 + np.abs(r).max() + d))


def test_rk4_momentum_magnitude_conserved():
    rng = np.random.default_rng(8)
    r = np.zeros(3)
    p = np.array([0.5, -0.3, 3.0])
    P0 = np.linalg.norm(p)
    B = rng.normal(size=3) * 1.7
    for _ in range(2000):
        r, p = oracle.rk4(r, p, B, -1, 0.02)
    assert abs(np.linalg.norm(p) / P0 - 1.0) < 1e-9


# --------------------------------------------------------------------------
# S0 + whole loop: hand-built single-muon cases hit each status exactly
# --------------------------------------------------------------------------
def _one(world, r, p, q=1, max_steps=1000, steps=0, status=0, d=0.02, seed=7):
    mu = dict(x=np.array([r[0]]), y=np.array([r[1]]), z=np.array([r[2]]), px=np.array([p[0]]),
              py=np.array([p[1]]), pz=np.array([p[2]]), q=np.array([q], np.int8),
              steps=np.array([steps], np.int32), status=np.array([status], np.uint8))
    return oracle.transport(world, mu, d, max_steps, seed, n_threads=1)


def test_status_exit_z():
    out = _one(vacuum_world(z_max=1.01), [0, 0, 0], [0, 0, 10.0])
    assert out["status"][0] == oracle.EXIT_Z and out["steps"][0] == 51
    assert abs(out["z"][0] - 1.02) < 1e-12


def test_status_exit_xy_both_signs():
    out = _one(vacuum_world(x_max=0.51), [0, 0, 0], [10.0, 0, 0])
    assert out["status"][0] == oracle.EXIT_XY and out["steps"][0] == 26
    out = _one(vacuum_world(y_max=0.51), [0, 0, 0], [0, -10.0, 0])
    assert out["status"][0] == oracle.EXIT_XY and out["steps"][0] == 26


def test_status_stopped_max_steps_terminal_and_invalid():
    w = vacuum_world()
    out = _one(w, [0, 0, 0], [0, 0, 0.4])
    assert out["status"][0] == oracle.STOPPED and out["steps"][0] == 0
    out = _one(w, [0, 0, 0], [0, 0, 10.0], max_steps=37)
    assert out["status"][0] == oracle.MAX_STEPS and out["steps"][0] == 37
    for st in (oracle.STOPPED, oracle.EXIT_Z, oracle.EXIT_XY, oracle.INVALID):
        out = _one(w, [0, 0, 0], [0, 0, 10.0], status=st, steps=3)
        assert out["status"][0] == st and out["steps"][0] == 3 and out["z"][0] == 0.0
    out = _one(w, [0, float("nan"), 0], [0, 0, 10.0])
    assert out["status"][0] == oracle.INVALID and out["steps"][0] == 0


def test_stopping_in_dense_loss():
    # a histogram whose only cell is f in [0.1, 0.2): P falls below 0.5 GeV from 10 GeV
    # within ceil(log(0.05)/log(0.9)) = 29 steps and no later than ceil(log(.05)/log(.8)) = 14
    hist = tiny_hist(np.array([[0.0], [1.0]]), n_pbin=1, f_max=0.2, theta_max=1e-3)
    w = vacuum_world(hist=hist, world_mat=1)
    out = _one(w, [0, 0, 0], [0, 0, 10.0])
    assert out["status"][0] == oracle.STOPPED
    assert 14 <= out["steps"][0] <= 29


def test_resume_subset_and_threads_are_invariant():
    wl = gen.workload("block1e4", n=300, hist_samples=20000)
    world = oracle.world_of(wl)
    full = oracle.transport(world, wl.muons, wl.step_len, wl.max_steps, wl.seed, n_threads=4)
    one = oracle.transport(world, wl.muons, wl.step_len, wl.max_steps, wl.seed, n_threads=1)
    part = oracle.transport(world, wl.muons, wl.step_len, 80, wl.seed, n_threads=3)
    part_mu = {k: part[k] for k in ("x", "y", "z", "px", "py", "pz", "q", "steps", "status")}
    rest = oracle.transport(world, part_mu, wl.step_len, wl.max_steps, wl.seed, n_threads=2)
    idx = np.array([5, 6, 7, 100, 299, 2])
    sub = oracle.transport(world, wl.muons, wl.step_len, wl.max_steps, wl.seed, index=idx)
    for k in ("x", "y", "z", "px", "py", "pz", "steps", "status"):
        np.testing.assert_array_equal(full[k], one[k])
        np.testing.assert_array_equal(full[k], rest[k])
        np.testing.assert_array_equal(full[k][idx], sub[k])
    assert set(np.unique(full["status"])) <= {oracle.STOPPED, oracle.EXIT_Z, oracle.EXIT_XY, oracle.MAX_STEPS}
    # the iron block is 2 m long: most muons leave through the z = 3 m plane
    assert (full["status"] == oracle.EXIT_Z).mean() > 0.5
