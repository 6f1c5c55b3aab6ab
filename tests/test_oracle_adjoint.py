"""Pins of the FP64 oracle's reverse-mode adjoint of the transport with respect
to per-block field scales alpha: forward-mode dual numbers (exact to FP64),
central finite differences with common random numbers, and closed forms of
the acceptance loss."""
import math

import numpy as np
import pytest

import oracle
from workloads import gen


def _world_and_muons(n, field_kind, seed=5):
    wl = gen.workload("shield1e6", n=n, hist_samples=20000, field="box" if field_kind == "box" else None)
    if field_kind == "smallmap":
        wl.field = gen.field_map_shield1e6(nx=60, ny=60, nz=180)
    rng = np.random.default_rng(seed)
    alpha = 1.0 + 0.2 * rng.standard_normal((6, 3))
    return wl, alpha


def _final(world, wl):
    return oracle.transport(world, wl.muons, wl.step_len, wl.max_steps, wl.seed)


@pytest.mark.parametrize("field_kind", ["box", "smallmap"])
def test_adjoint_matches_dual_numbers(field_kind):
    wl, alpha = _world_and_muons(120, field_kind)
    world = oracle.world_of(wl, alpha)
    fin = _final(world, wl)
    L, g = oracle.acceptance_loss(fin)
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


def test_adjoint_matches_central_differences():
    wl, alpha = _world_and_muons(300, "smallmap", seed=8)
    world = oracle.world_of(wl, alpha)
    fin = _final(world, wl)
    _, g = oracle.acceptance_loss(fin)
    adj = oracle.adjoint(world, wl.muons, wl.step_len, wl.max_steps, wl.seed, g).ravel()
    h = 1e-7
    fd = np.zeros(18)
    for j in range(18):
        ap, am = alpha.copy().ravel(), alpha.copy().ravel()
        ap[j] += h
        am[j] -= h
        Lp, _ = oracle.acceptance_loss(_final(oracle.world_of(wl, ap.reshape(6, 3)), wl))
        Lm, _ = oracle.acceptance_loss(_final(oracle.world_of(wl, am.reshape(6, 3)), wl))
        fd[j] = (Lp - Lm) / (2 * h)
    scale = np.abs(adj).max()
    np.testing.assert_allclose(adj, fd, rtol=1e-4, atol=1e-4 * scale)


def test_acceptance_loss_closed_forms():
    fin = dict(x=np.array([0.0, 0.3, 0.0, 0.0, 0.0]), y=np.array([0.0, -0.2, 0.0, 0.0, 0.0]),
               z=np.array([29.0, 10.0, 5.0, 5.0, 5.0]), px=np.array([0.0, 0.1, 0.0, 0.0, 1.0]),
               py=np.array([0.0, 0.0, 0.0, 0.0, 0.0]), pz=np.array([10.0, 20.0, 10.0, -1.0, 0.0]),
               status=np.array([4, 3, 1, 4, 4], np.uint8))
    L, g = oracle.acceptance_loss(fin)
    sig = lambda t: 1.0 / (1.0 + math.exp(-t))
    l0 = sig(50.0) ** 2
    xe = 0.3 + 20.0 * 0.1 / 20.0
    l1 = sig((0.5 - xe) / 0.01) * sig((0.5 - 0.2) / 0.01)
    assert abs(L - (l0 + l1) / 5) < 1e-15
    # stopped, backward and transverse muons contribute nothing
    assert np.all(g[:, 2:] == 0.0)
    # gradient of muon 1 against the closed-form derivative along x
    s1 = sig((0.5 - xe) / 0.01)
    dxe = -s1 * (1 - s1) * sig(30.0) / 0.01 / 5
    assert abs(g[0, 1] - dxe) < 1e-12 * abs(dxe)
    assert abs(g[3, 1] - dxe * 20.0 / 20.0) < 1e-12 * abs(dxe)
