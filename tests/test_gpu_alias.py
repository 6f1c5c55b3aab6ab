"""GPU parity of the alias sampler (Sec. Methodology, "The Alias Method";
mt_hist_desc.sampler = MT_SAMPLER_ALIAS) against the FP64 oracle running the
same alias tables: the draw -> cell map is integer-exact on both sides, so
results agree per muon at the plain transport's tolerances, and in
distribution with the inverse-CDF sampler (same quantised distribution,
different draws)."""
import numpy as np
import pytest
from scipy import stats

import oracle
from helpers import assert_parity, compare, gpu_transport
from workloads import gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2512_10520_gb300 as mt
    mt.load_library()


def _alias(wl):
    wl.hist = dict(wl.hist, sampler="alias")
    return wl


def test_alias_block1e4_full_parity():
    wl = _alias(gen.workload("block1e4"))
    ora = oracle.transport(oracle.world_of(wl), wl.muons, wl.step_len, wl.max_steps, wl.seed)
    gpu = gpu_transport(wl)
    assert_parity(gpu, ora)


def test_alias_shield1e6_parity_and_distribution():
    wl = _alias(gen.workload("shield1e6", n=50000))
    ora = oracle.transport(oracle.world_of(wl), wl.muons, wl.step_len, wl.max_steps, wl.seed)
    gpu = gpu_transport(wl)
    assert_parity(gpu, ora)
    ok, err = compare(gpu, ora)
    assert np.median(err["pos_err"]) < 1e-5
    icdf = gpu_transport(gen.workload("shield1e6", n=50000))
    P = lambda f: np.sqrt(np.asarray(f["px"], np.float64) ** 2 + f["py"] ** 2 + f["pz"] ** 2)
    assert not np.array_equal(P(gpu), P(icdf))
    assert stats.ks_2samp(P(gpu), P(icdf)).pvalue > 0.01


def test_alias_launch_shapes_and_batch_are_bit_identical():
    import paper_2512_10520_gb300 as mt
    wl = _alias(gen.workload("shield1e6", n=3000))
    outs = [gpu_transport(wl)]
    with mt.World.from_workload(wl) as world:
        for mode in (mt.MT_LAUNCH_STATIC, mt.MT_LAUNCH_PERSISTENT):
            dev = mt.muons_to_device(wl.muons)
            world.transport(dev, wl.step_len, wl.max_steps, wl.seed, mode=mode)
            outs.append(mt.muons_to_host(dev))
    with mt.Batch(wl.hist, 1) as b:
        b.set_instance(0, wl.geometry, wl.field)
        dev = mt.muons_to_device(wl.muons)
        b.transport([dev], wl.step_len, wl.max_steps, wl.seed, instances=[0])
        outs.append(mt.muons_to_host(dev))
    for o in outs[1:]:
        for k in ("x", "y", "z", "px", "py", "pz", "steps", "status"):
            np.testing.assert_array_equal(outs[0][k], o[k])
