"""Pins of the oracle's convex-polyhedron geometry (Sec. Simulation item 1,
Eq. 2): a solid with equal axis-aligned ends is a box; tapered and sheared
solids against scipy's Delaunay point location on the interpolated slice;
closed sides, half-open z; invariance under a quarter turn and a shift; first
containing solid wins."""
import numpy as np
import pytest
from scipy.spatial import Delaunay

import oracle
from workloads import gen


def world(solids, world_mat=2):
    geo = dict(kind="polyhedra", solids=solids, world_material=world_mat, x_max=50.0, y_max=50.0, z_max=100.0,
               p_min=0.5)
    return oracle.OracleWorld(geo, dict(kind="none"), _hist3())


def _hist3():
    w = np.ones((3, 1, 2, 2))
    return dict(n_mat=3, n_pbin=1, p_lo=1.0, p_hi=100.0, nf=2, ntheta=2, weights=w, f_max=np.full((3, 1), 0.1),
                theta_max=np.full((3, 1), 0.01))


def rect(x0, x1, y0, y1):
    return [(x0, y0), (x1, y0), (x1, y1), (x0, y1)]


def test_solid_with_equal_rectangular_ends_is_a_box():
    s = gen.solid(1.0, 3.0, rect(-0.5, 0.7, -0.3, 0.4), rect(-0.5, 0.7, -0.3, 0.4), 1)
    w = world([s])
    box_geo = dict(kind="boxes", boxes=[dict(lo=[-0.5, -0.3, 1.0], hi=[0.7, 0.4, 3.0], material=1)],
                   world_material=2, x_max=50.0, y_max=50.0, z_max=100.0, p_min=0.5)
    wb = oracle.OracleWorld(box_geo, dict(kind="none"), _hist3())
    xs = np.linspace(-1.0, 1.2, 23)
    ys = np.linspace(-0.8, 0.9, 18)
    zs = np.array([0.5, 1.0, 1.7, 2.999, 3.0, 3.5])
    n_in = 0
    for x in xs:
        for y in ys:
            for z in zs:
                m, b = w.material([x, y, z])
                mb, bb = wb.material([x, y, z])
                on_hi_face = (x == 0.7 or y == 0.4) and 1.0 <= z < 3.0 and -0.5 <= x <= 0.7 and -0.3 <= y <= 0.4
                if on_hi_face:
                    assert m == 1          # sides are closed, the box's upper faces are open
                else:
                    assert (m, b) == (mb, bb), (x, y, z)
                n_in += m == 1
    assert n_in > 100


def _slice(s, z):
    t = (z - s["z0"]) / (s["z1"] - s["z0"])
    return np.array(s["bottom"]) + t * (np.array(s["top"]) - np.array(s["bottom"]))


@pytest.mark.parametrize("k", range(6))
def test_tapered_solids_against_delaunay_point_location(k):
    geo = gen.geometry_tapered()
    s = geo["solids"][k]
    w = world([s])
    rng = np.random.default_rng(k)
    pts = np.column_stack([rng.uniform(-1.0, 1.0, 4000), rng.uniform(-0.8, 0.8, 4000),
                           rng.uniform(s["z0"] - 0.3, s["z1"] + 0.3, 4000)])
    agree = 0
    for p in pts:
        m, _ = w.material(p)
        inside_z = s["z0"] <= p[2] < s["z1"]
        expect = inside_z and Delaunay(_slice(s, p[2])).find_simplex(p[:2]) >= 0
        assert (m == 1) == expect, p
        agree += expect
    assert agree > 300


def test_quarter_turn_and_shift_invariance():
    rng = np.random.default_rng(9)
    s = gen.geometry_tapered()["solids"][2]
    rot = lambda v: (-v[1] + 0.3, v[0] - 1.1)      # +90 degrees about z, then a shift (keeps the orientation)
    s2 = gen.solid(s["z0"], s["z1"], [rot(v) for v in s["bottom"]], [rot(v) for v in s["top"]], 1)
    w1, w2 = world([s]), world([s2])
    for _ in range(3000):
        p = np.array([rng.uniform(-1, 1), rng.uniform(-1, 1), rng.uniform(s["z0"] - 0.2, s["z1"] + 0.2)])
        q = np.array([*rot(p[:2]), p[2]])
        assert w1.material(p)[0] == w2.material(q)[0]


def test_first_containing_solid_wins_and_edges_are_inside():
    a = gen.solid(0.0, 2.0, rect(-1, 1, -1, 1), rect(-0.5, 0.5, -0.5, 0.5), 1)
    b = gen.solid(1.0, 3.0, rect(-2, 2, -2, 2), rect(-2, 2, -2, 2), 3)
    w = world([a, b])
    assert w.material([0, 0, 1.5]) == (1, 0)
    assert w.material([0.9, 0, 1.5]) == (3, 1)      # outside a's slice (half-width 0.625), inside b
    assert w.material([0.625, 0, 1.5]) == (1, 0)    # on a's edge: inside
    assert w.material([0, 0, 2.0]) == (3, 1)        # z = z1 of a is outside a
    assert w.material([0, 0, 3.0]) == (2, -1)
    assert w.material([1.0, 1.0, 0.0]) == (1, 0)    # a corner at z0


def test_tapered_geometry_transport_runs_and_differs_from_boxes():
    wl = gen.workload("tapered1e6", n=400, hist_samples=20000)
    out = oracle.transport(oracle.world_of(wl), wl.muons, wl.step_len, wl.max_steps, wl.seed)
    wb = gen.workload("shield1e6", n=400, hist_samples=20000)
    ob = oracle.transport(oracle.world_of(wb), wb.muons, wb.step_len, wb.max_steps, wb.seed)
    assert (out["steps"] > 0).all()
    assert not np.array_equal(out["x"], ob["x"])
