"""Every combination the dispatchers route: geometry (boxes, voxels, solids) x
field (none, per-volume, trilinear map, nearest node, per-stage map) with the
sampler, histogram axes and momentum bins varied alongside, each against the
FP64 oracle on a small case and across the three launch shapes."""
import numpy as np
import pytest

import oracle
from helpers import assert_parity, gpu_transport
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


def _voxelise(geo, dims=(60, 60, 300), half=3.0, zmax=30.0):
    nx, ny, nz = dims
    sx, sy, sz = 2 * half / nx, 2 * half / ny, zmax / nz
    xc = -half + (np.arange(nx) + 0.5) * sx
    yc = -half + (np.arange(ny) + 0.5) * sy
    zc = (np.arange(nz) + 0.5) * sz
    vox = np.full((nz, ny, nx), geo["world_material"], np.uint8)
    for b in reversed(geo["boxes"]):
        (x0, y0, z0), (x1, y1, z1) = b["lo"], b["hi"]
        m = ((zc >= z0) & (zc < z1))[:, None, None] & ((yc >= y0) & (yc < y1))[None, :, None] & \
            ((xc >= x0) & (xc < x1))[None, None, :]
        vox[m] = b["material"]
    return dict(kind="voxels", voxels=vox, origin=[-half, -half, 0.0], spacing=[sx, sy, sz],
                world_material=geo["world_material"], x_max=geo["x_max"], y_max=geo["y_max"], z_max=geo["z_max"],
                p_min=geo["p_min"])


CASES = [
    # geometry, field, sampler, axes, explicit edges
    ("boxes", "none", "icdf", "linear", False),
    ("boxes", "nearest", "alias", "log", True),
    ("boxes", "per_stage", "icdf", "linear", True),
    ("voxels", "map", "alias", "linear", False),
    ("voxels", "nearest", "icdf", "log", False),
    ("voxels", "per_stage", "alias", "linear", False),
    ("voxels", "none", "icdf", "linear", True),
    ("solids", "box", "alias", "log", False),
    ("solids", "nearest", "icdf", "linear", True),
    ("solids", "per_stage", "icdf", "log", False),
    ("solids", "none", "alias", "linear", False),
]


@pytest.mark.parametrize("geom,field,sampler,axes,edges", CASES)
def test_combination(geom, field, sampler, axes, edges):
    import paper_2512_10520_gb300 as mt
    wl = gen.workload("tapered1e6" if geom == "solids" else "shield1e6", n=20000, hist_samples=50000,
                      field={"box": "box", "nearest": "nearest"}.get(field), axes=axes)
    if geom == "voxels":
        wl.geometry = _voxelise(gen.geometry_shield1e6())
    if field == "none":
        wl.field = dict(kind="none")
    if field == "per_stage":
        wl.field = dict(wl.field, per_stage=True)
    hist = dict(wl.hist, sampler=sampler)
    if edges:
        e = gen.pbin_edges(hist["p_lo"], hist["p_hi"], hist["n_pbin"])
        e[1:-1] *= np.exp(0.3 * np.sin(np.arange(1, hist["n_pbin"])))      # uneven bins
        e = np.sort(e)
        hist["p_edges"] = e
    wl.hist = hist
    ora = oracle.transport(oracle.world_of(wl), wl.muons, wl.step_len, wl.max_steps, wl.seed)
    gpu = gpu_transport(wl)
    assert_parity(gpu, ora)
    with mt.World.from_workload(wl) as world:
        for mode in (mt.MT_LAUNCH_STATIC, mt.MT_LAUNCH_PERSISTENT):
            dev = mt.muons_to_device(wl.muons)
            world.transport(dev, wl.step_len, wl.max_steps, wl.seed, mode=mode)
            out = mt.muons_to_host(dev)
            for k in FIELDS:
                np.testing.assert_array_equal(gpu[k], out[k], err_msg=f"{mode} {k}")
