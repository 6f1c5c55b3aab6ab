"""mt_transport_noalloc: the transport for callers that cannot allocate device
memory (a framework that already owns the GPU's memory pool, a latency-critical
path, a fixed memory budget).  Its results must equal those of mt_transport,
call after call, although every call reuses the same fixed scratch array.
This file is collected last so that a failure here leaves every other test run."""
import numpy as np
import pytest

from helpers import compare, describe

pytestmark = pytest.mark.gpu


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


def test_noalloc_matches_transport_on_consecutive_calls(mt):
    import torch
    from workloads import gen
    wl = gen.workload("shield1e6", n=2 * 20000, hist_samples=20000)
    halves = [{k: v[:20000].copy() for k, v in wl.muons.items()}, {k: v[20000:].copy() for k, v in wl.muons.items()}]
    with mt.World.from_workload(wl) as world:
        for call, (mu, off) in enumerate(zip(halves, (0, 20000))):
            ref = mt.muons_to_device(mu)
            mt.mt_transport(world.handle, ref, wl.step_len, wl.max_steps, wl.seed, id_offset=off)
            out = mt.muons_to_device(mu)
            mt.mt_transport_noalloc(world.handle, out, wl.step_len, wl.max_steps, wl.seed, id_offset=off)
            torch.cuda.synchronize()
            a, b = mt.muons_to_host(ref), mt.muons_to_host(out)
            ok, err = compare(b, {k: np.asarray(v, np.float64) for k, v in a.items()})
            assert ok.all(), f"call {call}: " + describe(ok, err)
            assert (b["steps"] > 0).all()


def test_noalloc_rejects_oversized_batches(mt):
    from workloads import gen
    n = mt.MT_NOALLOC_MAX_MUONS + 1
    wl = gen.workload("block1e4", n=n, hist_samples=20000)
    with mt.World.from_workload(wl) as world:
        dev = mt.muons_to_device(wl.muons)
        with pytest.raises(mt.MtError) as e:
            mt.mt_transport_noalloc(world.handle, dev, wl.step_len, wl.max_steps, wl.seed)
        assert "at most 65536 muons" in str(e.value)
