"""GPU check of the momentum-bin decision (Sec. Momentum binning) at the densest
binnings the library takes and on the bin edges themselves.

The step settles a bin from its FP32 estimate unless the estimate lies within a
host-bounded error of a bin face; there, and for |p|^2 near an edge, the squared
edges held as hi + lo pairs decide.  Here every bin's histogram has a single cell,
cell (i mod nf, 0), so a wrong bin changes the sampled momentum loss by 1/nf of
f_max.  Each muon takes exactly one step from the same state on the GPU and in the
FP64 oracle (one iron block, uniform field), which leaves no room for trajectory
divergence: every muon must agree."""
import numpy as np
import pytest

import oracle
from helpers import compare, describe
from workloads import gen

pytestmark = pytest.mark.gpu

NF, NT = 8, 4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2512_10520_gb300 as mt
    mt.load_library()


def _hist(n_pbin, p_lo, p_hi):
    W = np.zeros((2, n_pbin, NF, NT))
    for i in range(n_pbin):
        W[:, i, i % NF, 0] = 1.0
    return dict(n_mat=2, n_pbin=n_pbin, p_lo=p_lo, p_hi=p_hi, nf=NF, ntheta=NT, weights=W,
                f_max=np.full((2, n_pbin), 0.2), theta_max=np.full((2, n_pbin), 1e-3))


def _muons(n_pbin, p_lo, p_hi, n, rng):
    """Log-uniform momenta around [p_lo, p_hi] along z (|p| = p_z exactly), with and
    without transverse momentum, plus every edge as a float32 and its two float32
    neighbours; all inside the iron block."""
    p = np.exp(rng.uniform(np.log(max(0.6, 0.9 * p_lo)), np.log(1.1 * p_hi), n))
    e32 = gen.pbin_edges(p_lo, p_hi, n_pbin).astype(np.float32)
    pe = np.concatenate([e32, np.nextafter(e32, np.float32(0.0)), np.nextafter(e32, np.float32(np.inf))])
    p = np.concatenate([p, pe.astype(np.float64)])
    m = len(p)
    pt = np.where(np.arange(m) % 2 == 0, 0.0, 0.05 * p)
    phi = rng.uniform(0.0, 2.0 * np.pi, m)
    px, py = pt * np.cos(phi), pt * np.sin(phi)
    pz = np.where(pt == 0.0, p, np.sqrt(np.maximum(p * p - pt * pt, 0.0)))
    x, y = rng.uniform(-0.3, 0.3, m), rng.uniform(-0.3, 0.3, m)
    q = np.where(rng.random(m) < 0.5, -1, 1)
    return gen._soa(x, y, np.full(m, 1.0), px, py, pz, q)


@pytest.mark.parametrize("n_pbin,p_lo,p_hi", [(64, 1.0, 400.0), (256, 1.0, 400.0), (256, 10.0, 11.0)])
def test_one_step_bins_match_the_oracle(n_pbin, p_lo, p_hi):
    import torch
    import paper_2512_10520_gb300 as mt
    rng = np.random.default_rng(n_pbin + int(p_lo))
    hist = _hist(n_pbin, p_lo, p_hi)
    geo, fld = gen.geometry_block1e4(), dict(kind="box")
    mu = _muons(n_pbin, p_lo, p_hi, 20000, rng)
    with mt.World(geo, fld, hist) as w:
        dev = mt.muons_to_device(mu)
        w.transport(dev, 0.02, 1, 99)
        torch.cuda.synchronize()
        got = mt.muons_to_host(dev)
    ora = oracle.transport(oracle.OracleWorld(geo, fld, hist), mu, 0.02, 1, 99)
    ok, err = compare(got, ora)
    assert ok.all(), describe(ok, err)
    # the loss really depends on the bin: muons of adjacent bins lost different fractions
    P0 = np.sqrt(mu["px"].astype(np.float64) ** 2 + mu["py"] ** 2 + mu["pz"].astype(np.float64) ** 2)
    P1 = np.sqrt(ora["px"] ** 2 + ora["py"] ** 2 + ora["pz"] ** 2)
    assert np.unique(np.floor((1.0 - P1 / P0) / (0.2 / NF))).size == NF
