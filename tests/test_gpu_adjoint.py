"""GPU parity of the differentiable form: the checkpointing forward, the
acceptance-loss kernel and the hand-written adjoint (dL/dalpha of per-magnet
field scales) against the FP64 oracle adjoint and central finite differences
with common random numbers."""
import numpy as np
import pytest

import oracle
from helpers import gpu_transport
from workloads import gen

pytestmark = pytest.mark.gpu

ALPHA_SEED = 5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2512_10520_gb300 as mt
    mt.load_library()


def _alpha(seed=ALPHA_SEED):
    rng = np.random.default_rng(seed)
    return (1.0 + 0.2 * rng.standard_normal((6, 3))).astype(np.float32)


def _gpu_grad(wl, alpha, K=32, want_initial=False):
    """(loss, dL/dalpha, final state, dL/dinitial) from the GPU: ckpt forward, loss kernel, adjoint."""
    import torch
    import paper_2512_10520_gb300 as mt
    with mt.World.from_workload(wl) as world:
        dev = mt.muons_to_device(wl.muons)
        a = torch.as_tensor(alpha, dtype=torch.float32).cuda().contiguous()
        n = wl.n
        ckpt = torch.empty(mt.mt_ckpt_bytes(n, wl.max_steps, K), dtype=torch.uint8, device="cuda")
        mt.mt_transport_ckpt(world.handle, dev, wl.step_len, wl.max_steps, wl.seed, a, K, ckpt)
        loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        g = torch.empty((6, n), dtype=torch.float32, device="cuda")
        mt.mt_acceptance_loss(dev, loss, g)
        da = torch.empty_like(a)
        gi = torch.empty((6, n), dtype=torch.float32, device="cuda") if want_initial else None
        mt.mt_adjoint_ckpt(world.handle, n, wl.step_len, wl.max_steps, wl.seed, a, K, ckpt, g, da, gi)
        torch.cuda.synchronize()
        return (float(loss.item()), da.cpu().numpy().astype(np.float64), mt.muons_to_host(dev),
                None if gi is None else gi.cpu().numpy())


def test_checkpointing_forward_equals_transport():
    wl = gen.workload("shield1e6", n=5000)
    alpha = _alpha()
    ref = gpu_transport(wl, alpha=alpha)
    _, _, fin, _ = _gpu_grad(wl, alpha)
    for k in ("x", "y", "z", "px", "py", "pz", "steps", "status"):
        np.testing.assert_array_equal(ref[k], fin[k])


def test_loss_kernel_matches_oracle_loss():
    wl = gen.workload("shield1e6", n=20000)
    alpha = _alpha()
    L, _, fin, _ = _gpu_grad(wl, alpha)
    Lo, go = oracle.acceptance_loss({k: np.asarray(v, np.float64) for k, v in fin.items()})
    assert abs(L - Lo) <= 1e-6 * max(abs(Lo), 1e-12), (L, Lo)
    import torch
    import paper_2512_10520_gb300 as mt
    dev = mt.muons_to_device(fin)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    g = torch.empty((6, wl.n), dtype=torch.float32, device="cuda")
    mt.mt_acceptance_loss(dev, loss, g)
    g = g.cpu().numpy()
    scale = np.abs(go).max()
    assert scale > 0
    np.testing.assert_allclose(g, go, rtol=1e-3, atol=1e-4 * scale)


@pytest.mark.parametrize("field", ["map", "box"])
def test_adjoint_matches_fp64_oracle_adjoint(field):
    wl = gen.workload("shield1e6", n=10000, field="box" if field == "box" else None)
    alpha = _alpha()
    _, g_gpu, _, _ = _gpu_grad(wl, alpha)
    world = oracle.world_of(wl, alpha.astype(np.float64))
    fin = oracle.transport(world, wl.muons, wl.step_len, wl.max_steps, wl.seed)
    _, go = oracle.acceptance_loss(fin)
    g_ora = oracle.adjoint(world, wl.muons, wl.step_len, wl.max_steps, wl.seed, go)
    rel = np.linalg.norm(g_gpu - g_ora) / np.linalg.norm(g_ora)
    assert rel <= 1e-3, (rel, g_gpu.ravel().tolist(), g_ora.ravel().tolist())


def _per_muon_loss(f, z_plane=30.0, half=0.5, edge=0.01):
    """Per-muon acceptance term (used only to sort muons into smooth and jumping)."""
    x, y, z, px, py, pz = (np.asarray(f[k], np.float64) for k in ("x", "y", "z", "px", "py", "pz"))
    ok = (f["status"] != 1) & (f["status"] != 5) & (pz > 0)
    safe = np.where(ok, pz, 1.0)
    xe = x + (z_plane - z) * px / safe
    ye = y + (z_plane - z) * py / safe
    sig = lambda t: 0.5 * (1.0 + np.tanh(0.5 * t))
    return np.where(ok, sig((half - np.abs(xe)) / edge) * sig((half - np.abs(ye)) / edge), 0.0)


def test_adjoint_against_central_differences():
    """Central differences with common random numbers on 1e4 muons, h = 2e-4
    relative (at h = 1e-3 the 1 cm sigmoid edge of the loss already gives the
    central difference a ~1 % truncation error).  A step of h moves tracks by
    up to a millimetre; some muons then change a discrete
    choice (a box face, a momentum bin, a stop or exit step) and their term jumps
    (muon 3633 of this set goes from 1.0 to 0.0 across +-h and alone outweighs
    the whole sum).  The pathwise gradient holds those choices fixed by
    construction, so the two are compared on the muons that kept every discrete
    choice: the field never changes |p| and, with the same materials and bins,
    the common random numbers give the same losses, so such a muon keeps its step
    count, status and final |p| (to rounding) for every alpha +- h.  The adjoint
    is run with dL/dfinal of the other muons set to zero."""
    import torch
    import paper_2512_10520_gb300 as mt
    wl = gen.workload("shield1e6", n=10000)
    alpha = _alpha().astype(np.float32)
    h = 2e-4
    n = wl.n
    with mt.World.from_workload(wl) as world:
        def run(a):
            dev = mt.muons_to_device(wl.muons)
            world.transport(dev, wl.step_len, wl.max_steps, wl.seed,
                            alpha=torch.as_tensor(a, dtype=torch.float32).cuda().contiguous())
            torch.cuda.synchronize()
            return mt.muons_to_host(dev)

        f0 = run(alpha)
        P = lambda f: np.sqrt(f["px"].astype(np.float64) ** 2 + f["py"] ** 2 + f["pz"] ** 2)
        P0 = P(f0)
        d = np.zeros((18, n))
        smooth = np.ones(n, bool)
        for j in range(18):
            ap, am = alpha.ravel().copy(), alpha.ravel().copy()
            ap[j] = np.float32(ap[j] * (1 + h))
            am[j] = np.float32(am[j] * (1 - h))
            fp, fm = run(ap.reshape(6, 3)), run(am.reshape(6, 3))
            for f in (fp, fm):
                smooth &= (f["steps"] == f0["steps"]) & (f["status"] == f0["status"])
                smooth &= np.abs(P(f) - P0) <= 1e-5 * P0
            d[j] = (_per_muon_loss(fp) - _per_muon_loss(fm)) / (float(ap[j]) - float(am[j])) / n
        fd = d[:, smooth].sum(1)
        # adjoint restricted to the smooth muons
        dev = mt.muons_to_device(wl.muons)
        a = torch.as_tensor(alpha).cuda().contiguous()
        ckpt = torch.empty(mt.mt_ckpt_bytes(n, wl.max_steps, 32), dtype=torch.uint8, device="cuda")
        mt.mt_transport_ckpt(world.handle, dev, wl.step_len, wl.max_steps, wl.seed, a, 32, ckpt)
        g = torch.empty((6, n), dtype=torch.float32, device="cuda")
        mt.mt_acceptance_loss(dev, torch.zeros(1, dtype=torch.float64, device="cuda"), g)
        g *= torch.as_tensor(smooth, device="cuda").to(torch.float32)
        da = torch.empty_like(a)
        mt.mt_adjoint_ckpt(world.handle, n, wl.step_len, wl.max_steps, wl.seed, a, 32, ckpt, g, da)
        torch.cuda.synchronize()
    adj = da.cpu().numpy().astype(np.float64).ravel()
    rel = np.linalg.norm(adj - fd) / np.linalg.norm(fd)
    print("smooth muons", smooth.sum(), "of", n, "FD rel", rel, "full-population FD",
          d.sum(1).tolist(), "smooth FD", fd.tolist(), "adjoint", adj.tolist())
    assert smooth.mean() > 0.5
    assert rel < 1e-2, (rel, adj.tolist(), fd.tolist())


def test_autograd_function_and_one_call_adjoint():
    import torch
    import paper_2512_10520_gb300 as mt
    wl = gen.workload("shield1e6", n=4000)
    alpha = _alpha()
    _, g_ref, _, _ = _gpu_grad(wl, alpha)
    with mt.World.from_workload(wl) as world:
        a = torch.as_tensor(alpha).cuda().requires_grad_(True)
        fin = mt.transport_differentiable(world, mt.muons_to_device(wl.muons), a, wl.step_len, wl.max_steps, wl.seed)
        L = mt.acceptance_loss(fin)
        L.backward()
        np.testing.assert_allclose(a.grad.cpu().numpy(), g_ref, rtol=1e-5, atol=1e-7 * np.abs(g_ref).max())
        # the one-call form from the initial state
        dev0 = mt.muons_to_device(wl.muons)
        g6 = torch.empty((6, wl.n), dtype=torch.float32, device="cuda")
        dev = mt.muons_to_device(wl.muons)
        world.transport(dev, wl.step_len, wl.max_steps, wl.seed, alpha=a.detach().contiguous())
        mt.mt_acceptance_loss(dev, torch.zeros(1, dtype=torch.float64, device="cuda"), g6)
        da = torch.empty_like(a.detach())
        mt.mt_transport_adjoint(world.handle, dev0, wl.step_len, wl.max_steps, wl.seed, a.detach().contiguous(), g6,
                                da, 32)
        torch.cuda.synchronize()
        np.testing.assert_allclose(da.cpu().numpy(), g_ref, rtol=1e-5, atol=1e-7 * np.abs(g_ref).max())
        # the initial state is left unchanged
        np.testing.assert_array_equal(dev0["x"].cpu().numpy(), wl.muons["x"])


def test_initial_state_gradient_matches_finite_differences():
    """dL/d(initial px) of single muons against central differences on the GPU."""
    import torch
    import paper_2512_10520_gb300 as mt
    wl = gen.workload("shield1e6", n=4000)
    alpha = _alpha()
    _, _, fin, gi = _gpu_grad(wl, alpha, want_initial=True)
    # muons with a sizeable gradient, i.e. ending near the acceptance edge
    mag = np.abs(gi[3])
    cand = np.argsort(-mag)[:6]
    with mt.World.from_workload(wl) as world:
        a = torch.as_tensor(alpha).cuda().contiguous()
        loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        for m in cand:
            vals = []
            for sgn in (+1, -1):
                mu = {k: v.copy() for k, v in wl.muons.items()}
                mu["px"][m] = np.float32(mu["px"][m] + sgn * 1e-3)
                dev = mt.muons_to_device(mu)
                world.transport(dev, wl.step_len, wl.max_steps, wl.seed, alpha=a)
                mt.mt_acceptance_loss(dev, loss)
                vals.append(float(loss.item()))
            dpx = float(np.float32(wl.muons["px"][m] + 1e-3)) - float(np.float32(wl.muons["px"][m] - 1e-3))
            fd = (vals[0] - vals[1]) / dpx
            assert abs(fd - gi[3][m]) <= 0.05 * abs(gi[3][m]) + 1e-9, (m, fd, gi[3][m])


def _gpu_grad_tape(wl, alpha, K=32, want_initial=False):
    """(loss, dL/dalpha, final state, dL/dinitial) with the full-tape forward and backward."""
    import torch
    import paper_2512_10520_gb300 as mt
    with mt.World.from_workload(wl) as world:
        dev = mt.muons_to_device(wl.muons)
        a = torch.as_tensor(alpha, dtype=torch.float32).cuda().contiguous()
        n = wl.n
        tape = torch.empty(mt.mt_tape_bytes(n, wl.max_steps, K), dtype=torch.uint8, device="cuda")
        mt.mt_transport_tape(world.handle, dev, wl.step_len, wl.max_steps, wl.seed, a, K, tape)
        loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        g = torch.empty((6, n), dtype=torch.float32, device="cuda")
        mt.mt_acceptance_loss(dev, loss, g)
        da = torch.empty_like(a)
        gi = torch.empty((6, n), dtype=torch.float32, device="cuda") if want_initial else None
        mt.mt_adjoint_tape(world.handle, n, wl.step_len, wl.max_steps, a, K, tape, g, da, gi)
        torch.cuda.synchronize()
        return (float(loss.item()), da.cpu().numpy().astype(np.float64), mt.muons_to_host(dev),
                None if gi is None else gi.cpu().numpy())


@pytest.mark.parametrize("field,K", [("map", 32), ("box", 32), ("map", 7), ("map", 64)])
def test_tape_form_equals_checkpoint_form(field, K):
    """The full-tape forward gives the plain transport's results bit for bit, and
    its backward the checkpoint form's gradients (the same recorded quantities
    and reverse arithmetic; only the order of the dL/dalpha atomics differs)."""
    wl = gen.workload("shield1e6", n=6000, field="box" if field == "box" else None)
    alpha = _alpha()
    ref = gpu_transport(wl, alpha=alpha)
    _, g_ck, _, gi_ck = _gpu_grad(wl, alpha, K=K, want_initial=True)
    _, g_tp, fin, gi_tp = _gpu_grad_tape(wl, alpha, K=K, want_initial=True)
    for k in ("x", "y", "z", "px", "py", "pz", "steps", "status"):
        np.testing.assert_array_equal(ref[k], fin[k])
    np.testing.assert_allclose(g_tp, g_ck, rtol=1e-5, atol=1e-6 * np.abs(g_ck).max())
    np.testing.assert_allclose(gi_tp, gi_ck, rtol=1e-5, atol=1e-6 * np.abs(gi_ck).max())


def test_tape_adjoint_matches_fp64_oracle_adjoint():
    wl = gen.workload("shield1e6", n=10000)
    alpha = _alpha()
    _, g_gpu, _, _ = _gpu_grad_tape(wl, alpha)
    world = oracle.world_of(wl, alpha.astype(np.float64))
    fin = oracle.transport(world, wl.muons, wl.step_len, wl.max_steps, wl.seed)
    _, go = oracle.acceptance_loss(fin)
    g_ora = oracle.adjoint(world, wl.muons, wl.step_len, wl.max_steps, wl.seed, go)
    rel = np.linalg.norm(g_gpu - g_ora) / np.linalg.norm(g_ora)
    assert rel <= 1e-3, (rel, g_gpu.ravel().tolist(), g_ora.ravel().tolist())


def test_tape_buffer_checks_and_autograd_mode():
    import torch
    import paper_2512_10520_gb300 as mt
    wl = gen.workload("shield1e6", n=3000)
    alpha = _alpha()
    with mt.World.from_workload(wl) as world:
        dev = mt.muons_to_device(wl.muons)
        a = torch.as_tensor(alpha).cuda().contiguous()
        need = mt.mt_tape_bytes(wl.n, wl.max_steps, 32)
        assert need >= 40 * wl.n * wl.max_steps
        small = torch.empty(need - 256, dtype=torch.uint8, device="cuda")
        with pytest.raises(mt.MtError):
            mt.mt_transport_tape(world.handle, dev, wl.step_len, wl.max_steps, wl.seed, a, 32, small)
        with pytest.raises(mt.MtError):
            mt.mt_transport_tape(world.handle, dev, wl.step_len, wl.max_steps, wl.seed, a, 65,
                                 torch.empty(need, dtype=torch.uint8, device="cuda"))
        grads = []
        for tape in (True, False):
            x = torch.as_tensor(alpha).cuda().requires_grad_(True)
            fin = mt.transport_differentiable(world, mt.muons_to_device(wl.muons), x, wl.step_len, wl.max_steps,
                                              wl.seed, tape=tape)
            mt.acceptance_loss(fin).backward()
            grads.append(x.grad.cpu().numpy())
        np.testing.assert_allclose(grads[0], grads[1], rtol=1e-5, atol=1e-7 * np.abs(grads[1]).max())


def test_zero_cotangents_are_skipped_exactly():
    """The backward is linear in dL/d(final state), and a muon whose six components
    are zero is neither recomputed nor reversed.  Check: with half the muons' rows
    zeroed, dL/d(initial state) of those muons is exactly zero, and dL/dalpha is
    additive over a split of the muons (each part skipping the other) and equals
    the full-tape form's (whose reverse pass skips zero adjoints the same way)."""
    import torch
    import paper_2512_10520_gb300 as mt
    wl = gen.workload("shield1e6", n=6000)
    n, K = wl.n, 32
    a = torch.as_tensor(_alpha(), dtype=torch.float32).cuda().contiguous()
    rng = np.random.default_rng(9)
    g_full = torch.as_tensor(rng.standard_normal((6, n)).astype(np.float32) * 1e-3).cuda()
    part = torch.as_tensor(rng.random(n) < 0.5).cuda()
    gA = (g_full * part).contiguous()
    gB = (g_full * ~part).contiguous()
    out = {}
    with mt.World.from_workload(wl) as world:
        ckpt = torch.empty(mt.mt_ckpt_bytes(n, wl.max_steps, K), dtype=torch.uint8, device="cuda")
        dev = mt.muons_to_device(wl.muons)
        mt.mt_transport_ckpt(world.handle, dev, wl.step_len, wl.max_steps, wl.seed, a, K, ckpt)
        for name, g in (("full", g_full.contiguous()), ("A", gA), ("B", gB)):
            da = torch.empty_like(a)
            gi = torch.empty((6, n), dtype=torch.float32, device="cuda")
            mt.mt_adjoint_ckpt(world.handle, n, wl.step_len, wl.max_steps, wl.seed, a, K, ckpt, g, da, gi)
            out[name] = (da.cpu().numpy().astype(np.float64), gi.cpu().numpy())
        tape = torch.empty(mt.mt_tape_bytes(n, wl.max_steps, K), dtype=torch.uint8, device="cuda")
        dev2 = mt.muons_to_device(wl.muons)
        mt.mt_transport_tape(world.handle, dev2, wl.step_len, wl.max_steps, wl.seed, a, K, tape)
        dt = torch.empty_like(a)
        mt.mt_adjoint_tape(world.handle, n, wl.step_len, wl.max_steps, a, K, tape, gA, dt)
        torch.cuda.synchronize()
    pm = part.cpu().numpy()
    assert np.all(out["A"][1][:, ~pm] == 0.0) and np.all(out["B"][1][:, pm] == 0.0)
    np.testing.assert_array_equal(out["A"][1][:, pm], out["full"][1][:, pm])
    gsum = out["A"][0] + out["B"][0]
    assert np.linalg.norm(gsum - out["full"][0]) <= 1e-5 * np.linalg.norm(out["full"][0])
    tp = dt.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(tp - out["A"][0]) <= 1e-5 * np.linalg.norm(out["A"][0])


def test_two_muon_groups_in_the_differentiable_forms():
    """From 2^19 muons the checkpoint and full-tape forms run as two groups of half
    the muons on two streams, each with its own checkpoints (or tape) and scratch.
    The forward's final states equal the static grid's bit for bit; each half's
    dL/d(initial state) equals a separate one-group call on that half alone (its
    muons' ids offset as in the whole) bit for bit, in both forms; dL/dalpha, a
    sum in another order, to 1e-5."""
    import torch
    import paper_2512_10520_gb300 as mt
    wl = gen.workload("shield1e6", n=(1 << 19) + 5)
    n, K = wl.n, 32
    n0 = n // 2
    a = torch.as_tensor(_alpha(), dtype=torch.float32).cuda().contiguous()

    def run(world, lo, hi, g_all, tape):
        mu = {k: v[lo:hi].copy() for k, v in wl.muons.items()}
        m = hi - lo
        dev = mt.muons_to_device(mu)
        da = torch.empty_like(a)
        gi = torch.empty((6, m), dtype=torch.float32, device="cuda")
        g = g_all[:, lo:hi].contiguous()
        if tape:
            buf = torch.empty(mt.mt_tape_bytes(m, wl.max_steps, K), dtype=torch.uint8, device="cuda")
            mt.mt_transport_tape(world.handle, dev, wl.step_len, wl.max_steps, wl.seed, a, K, buf, id_offset=lo)
            mt.mt_adjoint_tape(world.handle, m, wl.step_len, wl.max_steps, a, K, buf, g, da, gi)
        else:
            buf = torch.empty(mt.mt_ckpt_bytes(m, wl.max_steps, K), dtype=torch.uint8, device="cuda")
            mt.mt_transport_ckpt(world.handle, dev, wl.step_len, wl.max_steps, wl.seed, a, K, buf, id_offset=lo)
            mt.mt_adjoint_ckpt(world.handle, m, wl.step_len, wl.max_steps, wl.seed, a, K, buf, g, da, gi,
                               id_offset=lo)
        torch.cuda.synchronize()
        del buf
        return dev, da.cpu().numpy().astype(np.float64), gi.cpu().numpy()

    with mt.World.from_workload(wl) as world:
        ref = mt.muons_to_device(wl.muons)
        world.transport(ref, wl.step_len, wl.max_steps, wl.seed, alpha=a, mode=mt.MT_LAUNCH_STATIC)
        loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        g = torch.empty((6, n), dtype=torch.float32, device="cuda")
        mt.mt_acceptance_loss(ref, loss, g)
        torch.cuda.synchronize()
        assert int((g != 0).any(0).sum().item()) > 1000
        for tape in (False, True):
            dev, da, gi = run(world, 0, n, g, tape)
            for k in ("x", "y", "z", "px", "py", "pz", "steps", "status"):
                assert torch.equal(ref[k], dev[k]), (tape, k)
            _, da0, gi0 = run(world, 0, n0, g, tape)
            _, da1, gi1 = run(world, n0, n, g, tape)
            np.testing.assert_array_equal(gi[:, :n0], gi0, err_msg=f"tape={tape}, first half")
            np.testing.assert_array_equal(gi[:, n0:], gi1, err_msg=f"tape={tape}, second half")
            assert np.linalg.norm(da - (da0 + da1)) <= 1e-5 * np.linalg.norm(da), tape
