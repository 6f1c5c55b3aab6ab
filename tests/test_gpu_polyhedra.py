"""GPU parity of the convex-polyhedron geometry (Sec. Simulation item 1, Eq. 2;
MT_GEOM_POLYHEDRA) against the FP64 oracle: tapered magnets with the field map
and with per-solid fields, solids with rectangular ends against the box
geometry (identical results), launch-shape and batch invariance, and the
adjoint through solids."""
import numpy as np
import pytest

import oracle
from helpers import assert_parity, compare, gpu_transport
from workloads import gen

pytestmark = pytest.mark.gpu
FIELDS = ("x", "y", "z", "px", "py", "pz", "steps", "status")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2512_10520_gb300 as mt
    mt.load_library()


@pytest.mark.parametrize("field", ["map", "box"])
def test_tapered_magnets_parity(field):
    wl = gen.workload("tapered1e6", n=50000 if field == "map" else 20000, field="box" if field == "box" else None)
    ora = oracle.transport(oracle.world_of(wl), wl.muons, wl.step_len, wl.max_steps, wl.seed)
    gpu = gpu_transport(wl)
    assert_parity(gpu, ora)
    ok, err = compare(gpu, ora)
    assert np.median(err["pos_err"]) < 1e-5


def _as_solids(geo):
    solids = []
    for b in geo["boxes"]:
        (x0, y0, z0), (x1, y1, z1) = b["lo"], b["hi"]
        q = [(x0, y0), (x1, y0), (x1, y1), (x0, y1)]
        solids.append(gen.solid(z0, z1, q, q, b["material"], b.get("block_id", -1), b.get("B", (0, 0, 0))))
    return dict(geo, kind="polyhedra", solids=solids, boxes=None)


@pytest.mark.parametrize("field", ["map", "box"])
def test_rectangular_solids_equal_boxes(field):
    wl = gen.workload("shield1e6", n=5000, field="box" if field == "box" else None)
    ref = gpu_transport(wl)
    wl.geometry = _as_solids(wl.geometry)
    out = gpu_transport(wl)
    for k in FIELDS:
        np.testing.assert_array_equal(ref[k], out[k], err_msg=k)


def test_launch_shapes_and_batch_are_bit_identical():
    import paper_2512_10520_gb300 as mt
    wl = gen.workload("tapered1e6", n=3000)
    outs = [gpu_transport(wl)]
    with mt.World.from_workload(wl) as world:
        for mode in (mt.MT_LAUNCH_STATIC, mt.MT_LAUNCH_PERSISTENT):
            dev = mt.muons_to_device(wl.muons)
            world.transport(dev, wl.step_len, wl.max_steps, wl.seed, mode=mode)
            outs.append(mt.muons_to_host(dev))
    with mt.Batch(wl.hist, 2) as b:
        b.set_instance(0, wl.geometry, wl.field)
        b.set_instance(1, wl.geometry, wl.field)
        devs = [mt.muons_to_device(wl.muons), mt.muons_to_device({k: v[:10] for k, v in wl.muons.items()})]
        b.transport(devs, wl.step_len, wl.max_steps, wl.seed, instances=[0, 0])
        outs.append(mt.muons_to_host(devs[0]))
        small = mt.muons_to_host(devs[1])
    for o in outs[1:]:
        for k in FIELDS:
            np.testing.assert_array_equal(outs[0][k], o[k], err_msg=k)
    for k in FIELDS:
        np.testing.assert_array_equal(outs[0][k][:10], small[k], err_msg=k)


def test_adjoint_through_solids_matches_fp64_oracle_adjoint():
    import torch
    import paper_2512_10520_gb300 as mt
    wl = gen.workload("tapered1e6", n=6000, field="box")
    rng = np.random.default_rng(5)
    alpha = (1.0 + 0.2 * rng.standard_normal((6, 3))).astype(np.float32)
    with mt.World.from_workload(wl) as world:
        dev = mt.muons_to_device(wl.muons)
        a = torch.as_tensor(alpha).cuda().contiguous()
        tape = torch.empty(mt.mt_tape_bytes(wl.n, wl.max_steps, 32), dtype=torch.uint8, device="cuda")
        mt.mt_transport_tape(world.handle, dev, wl.step_len, wl.max_steps, wl.seed, a, 32, tape)
        g = torch.empty((6, wl.n), dtype=torch.float32, device="cuda")
        mt.mt_acceptance_loss(dev, torch.zeros(1, dtype=torch.float64, device="cuda"), g)
        da = torch.empty_like(a)
        mt.mt_adjoint_tape(world.handle, wl.n, wl.step_len, wl.max_steps, a, 32, tape, g, da)
        torch.cuda.synchronize()
    ow = oracle.world_of(wl, alpha.astype(np.float64))
    fin = oracle.transport(ow, wl.muons, wl.step_len, wl.max_steps, wl.seed)
    _, go = oracle.acceptance_loss(fin)
    g_ora = oracle.adjoint(ow, wl.muons, wl.step_len, wl.max_steps, wl.seed, go)
    g_gpu = da.cpu().numpy().astype(np.float64)
    rel = np.linalg.norm(g_gpu - g_ora) / np.linalg.norm(g_ora)
    assert rel <= 1e-3, (rel, g_gpu.ravel().tolist(), g_ora.ravel().tolist())
