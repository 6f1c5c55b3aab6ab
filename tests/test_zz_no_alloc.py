"""mt_transport_noalloc: the transport for callers that cannot allocate device
memory (a framework that already owns the GPU's memory pool, a latency-critical
path, a fixed memory budget).  It runs the same compacting kernels as
mt_transport with its scratch list in a fixed device array that every call
reuses, so its results must equal mt_transport's bit for bit, call after call,
up to the array's capacity; and a call must leave the device's free memory as
it found it.  This file is collected last so that a failure here leaves every
other test run."""
import numpy as np
import pytest
from scipy import stats

import oracle
from helpers import PASS_FRAC, compare, describe

pytestmark = pytest.mark.gpu
FIELDS = ("x", "y", "z", "px", "py", "pz", "steps", "status")


@pytest.fixture(scope="module")
def mt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_10520_gb300 import _build
    _build.build()
    import paper_2512_10520_gb300 as mt
    mt.load_library()
    return mt


@pytest.fixture(scope="module")
def wl():
    from workloads import gen
    return gen.workload("shield1e6", n=100000)


def _part(muons, lo, hi):
    return {k: v[lo:hi].copy() for k, v in muons.items()}


def test_noalloc_equals_transport_bit_for_bit_on_consecutive_calls(mt, wl):
    """Three calls in a row of different sizes, the middle one at the array's
    capacity: each must equal mt_transport on the same muons exactly, so no
    call sees what the one before it left in the shared array."""
    import torch
    cap = mt.MT_NOALLOC_MAX_MUONS
    spans = [(0, 20000), (20000, 20000 + cap), (20000 + cap, 20000 + cap + 777)]
    with mt.World.from_workload(wl) as world:
        for call, (lo, hi) in enumerate(spans):
            mu = _part(wl.muons, lo, hi)
            ref = mt.muons_to_device(mu)
            mt.mt_transport(world.handle, ref, wl.step_len, wl.max_steps, wl.seed, id_offset=lo)
            out = mt.muons_to_device(mu)
            mt.mt_transport_noalloc(world.handle, out, wl.step_len, wl.max_steps, wl.seed, id_offset=lo)
            torch.cuda.synchronize()
            a, b = mt.muons_to_host(ref), mt.muons_to_host(out)
            for k in FIELDS:
                np.testing.assert_array_equal(b[k], a[k], err_msg=f"call {call} ({hi - lo} muons), field {k}")
            assert (b["steps"] > 0).all()


def test_noalloc_leaves_free_device_memory_unchanged(mt, wl):
    """Two calls on a fresh handle, measured from before the first: the array
    and the kernels were made resident by mt_create, so the device's free
    memory does not move."""
    import torch
    with mt.World.from_workload(wl) as world:
        devs = [mt.muons_to_device(_part(wl.muons, 0, 30000)) for _ in range(2)]
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        for d in devs:
            mt.mt_transport_noalloc(world.handle, d, wl.step_len, wl.max_steps, wl.seed)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0, f"free device memory moved by {free0 - free1} bytes"
        for k in FIELDS:
            np.testing.assert_array_equal(devs[0][k].cpu().numpy(), devs[1][k].cpu().numpy())


def test_noalloc_matches_the_fp64_oracle(mt, wl):
    import torch
    mu = _part(wl.muons, 0, 20000)
    with mt.World.from_workload(wl) as world:
        dev = mt.muons_to_device(mu)
        mt.mt_transport_noalloc(world.handle, dev, wl.step_len, wl.max_steps, wl.seed)
        torch.cuda.synchronize()
        gpu = mt.muons_to_host(dev)
    ora = oracle.transport(oracle.world_of(wl), mu, wl.step_len, wl.max_steps, wl.seed)
    ok, err = compare(gpu, ora)
    assert ok.mean() >= PASS_FRAC, describe(ok, err)
    P = lambda f: np.sqrt(np.asarray(f["px"], np.float64) ** 2 + f["py"] ** 2 + f["pz"] ** 2)
    for a, b in ((gpu["x"], ora["x"]), (gpu["y"], ora["y"]), (P(gpu), P(ora))):
        assert stats.ks_2samp(a, b).pvalue > 0.01


def test_noalloc_rejects_oversized_batches(mt):
    from workloads import gen
    n = mt.MT_NOALLOC_MAX_MUONS + 1
    w = gen.workload("block1e4", n=n, hist_samples=20000)
    with mt.World.from_workload(w) as world:
        dev = mt.muons_to_device(w.muons)
        with pytest.raises(mt.MtError) as e:
            mt.mt_transport_noalloc(world.handle, dev, w.step_len, w.max_steps, w.seed)
        assert "at most 65536 muons" in str(e.value)
