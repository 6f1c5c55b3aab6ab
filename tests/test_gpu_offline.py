"""GPU offline phase (Sec. Building histograms, Appendix A) against the FP64
oracle: histograms from the parametric sampler (the same Philox streams and
FP64 arithmetic, so the counts agree cell by cell), the pilot estimator, and
the transport over bounded-variation momentum bins found by binary search."""
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


def test_histograms_match_the_oracle_cell_by_cell():
    import torch
    import paper_2512_10520_gb300 as mt
    mats = [gen.MATERIALS[m] for m in ("iron", "air", "concrete")]
    edges = gen.pbin_edges(1.0, 400.0, 6)
    n = 50000
    w = torch.empty((3, 6, 64, 32), dtype=torch.float64, device="cuda")
    tmax = mt.mt_build_histograms(mats, edges, 64, 32, 0.05, 0.02, n, 99, w)
    torch.cuda.synchronize()
    c_or, t_or = oracle.build_histograms(mats, edges, 64, 32, 0.05, 0.02, n, 99)
    np.testing.assert_allclose(tmax, t_or, rtol=1e-14, atol=0)
    got = w.cpu().numpy()
    assert got.sum() == 3 * 6 * n
    # identical draws and FP64 arithmetic: a sample can change cell only when
    # CUDA's and the C library's transcendentals differ in the last bit on a cell edge
    moved = np.abs(got - c_or).sum() / 2
    assert moved <= 2, moved


def test_pilot_estimator_matches_the_oracle():
    import paper_2512_10520_gb300 as mt
    probes = np.geomspace(1.0, 400.0, 37)
    for name in ("iron", "air"):
        phi = mt.mt_pilot_phi(gen.MATERIALS[name], probes, 20000, 0.02, 3)
        ref = oracle.pilot_phi(gen.MATERIALS[name], probes, 20000, 0.02, 3)
        np.testing.assert_allclose(phi, ref, rtol=1e-10, atol=0)


def test_bounded_variation_bins_through_the_transport():
    import paper_2512_10520_gb300 as mt
    edges, probes, phi = mt.bounded_variation_edges("iron", 1.0, 400.0, 0.08, n_probe=512, K=20000)
    assert 20 < len(edges) - 1 <= 256, len(edges)
    np.testing.assert_array_equal(edges, oracle.bv_edges(probes, phi, 0.08))
    hist = mt.build_histogram_set(["iron", "air", "concrete"], edges=edges, n_samples=100000)
    wl = gen.workload("shield1e6", n=20000)
    wl.hist = hist
    ora = oracle.transport(oracle.world_of(wl), wl.muons, wl.step_len, wl.max_steps, wl.seed)
    gpu = gpu_transport(wl)
    assert_parity(gpu, ora)


def test_explicit_log_edges_equal_the_implicit_log_bins():
    wl = gen.workload("shield1e6", n=5000)
    ref = gpu_transport(wl)
    wl.hist = dict(wl.hist, p_edges=gen.pbin_edges(wl.hist["p_lo"], wl.hist["p_hi"], wl.hist["n_pbin"]))
    out = gpu_transport(wl)
    for k in FIELDS:
        np.testing.assert_array_equal(ref[k], out[k], err_msg=k)
