"""CPU checks of the C-ABI library: it builds for sm_103a, loads without a GPU,
exports every function include/mt.h declares, and rejects bad arguments on the
host before touching the device."""
import ctypes as C

import numpy as np
import pytest

import paper_2512_10520_gb300 as mt
from paper_2512_10520_gb300 import _binding as B
from paper_2512_10520_gb300 import _build


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return mt.load_library()


def test_exports_every_declared_symbol(lib):
    names = mt.declared_symbols()
    assert {"mt_create", "mt_transport", "mt_destroy", "mt_last_error"} <= set(names)
    for name in names:
        assert hasattr(lib, name), name


def test_abi_version(lib):
    assert mt.mt_abi_version() == 1


def _descs(weights=None):
    from workloads import gen
    h = gen.histogram_set(["iron"], n_pbin=2, nf=4, ntheta=4, n_samples=1000, cache=False)
    if weights is not None:
        h["weights"] = weights
    geo = gen.geometry_block1e4()
    geo["boxes"][0]["material"] = 1
    geo["world_material"] = 0
    return geo, dict(kind="box"), h


def test_create_rejects_bad_tables_on_host(lib):
    geo, fld, h = _descs()
    w = h["weights"].copy()
    w[0, 1, 2, 3] = -1.0
    with pytest.raises(mt.MtError) as e:
        mt.mt_create(geo, fld, dict(h, weights=w))
    assert e.value.status == B.MT_ERR_TABLE
    w = h["weights"].copy()
    w[0, 0] = 0.0
    with pytest.raises(mt.MtError) as e:
        mt.mt_create(geo, fld, dict(h, weights=w))
    assert e.value.status == B.MT_ERR_TABLE and "no positive" in mt.mt_last_error()


def test_create_rejects_bad_descriptors_on_host(lib):
    geo, fld, h = _descs()
    bad = dict(geo, world_material=7)
    with pytest.raises(mt.MtError) as e:
        mt.mt_create(bad, fld, h)
    assert e.value.status == B.MT_ERR_INVALID_ARG
    with pytest.raises(mt.MtError):
        mt.mt_create(geo, fld, dict(h, p_lo=5.0, p_hi=1.0))
    with pytest.raises(mt.MtError):
        mt.mt_create(dict(geo, kind="boxes", boxes=geo["boxes"] * 40), fld, h)
    out = C.c_void_p()
    assert lib.mt_create(None, None, None, C.byref(out)) == B.MT_ERR_INVALID_ARG
    assert out.value is None


def test_transport_rejects_bad_arguments_on_host(lib):
    s = B.mt_muon_soa()
    assert lib.mt_transport(None, C.byref(s), 10, 0.02, 10, 1, None) == B.MT_ERR_INVALID_ARG
    assert "null handle" in mt.mt_last_error()
    mt.mt_destroy(None)


def test_declared_symbols_parser_sees_comments_removed():
    names = mt.declared_symbols()
    assert all(n.startswith("mt_") for n in names)
    assert "mt_status" not in names and "mt_box" not in names


def test_batch_host_errors(lib):
    """The batch entry points reject bad arguments on the host, before any device work."""
    _, _, h = _descs()
    with pytest.raises(mt.MtError) as e:
        mt.mt_batch_create(h, 0)
    assert e.value.status == B.MT_ERR_INVALID_ARG
    w = h["weights"].copy()
    w[0, 1, 2, 3] = -1.0
    with pytest.raises(mt.MtError) as e:
        mt.mt_batch_create(dict(h, weights=w), 4)
    assert e.value.status == B.MT_ERR_TABLE
    assert lib.mt_batch_workspace_bytes(None, None) == -1
    assert lib.mt_batch_device_bytes(None) == 0
    lib.mt_batch_destroy(None)
    n = (C.c_int64 * 1)(5)
    st = lib.mt_transport_batched(None, None, n, 0.02, 10, 1, None, None)
    assert st == B.MT_ERR_INVALID_ARG and "null batch" in mt.mt_last_error()
    st = lib.mt_batch_autotune(None, None, n, 0.02, 10, 1, 0, None, None)
    assert st == B.MT_ERR_INVALID_ARG


def test_alias_sampler_needs_power_of_two_cells(lib):
    from workloads import gen
    h = gen.histogram_set(["iron"], n_pbin=2, nf=6, ntheta=4, n_samples=1000, cache=False)
    geo = gen.geometry_block1e4()
    geo["boxes"][0]["material"] = 1
    geo["world_material"] = 0
    with pytest.raises(mt.MtError) as e:
        mt.mt_create(geo, dict(kind="box"), dict(h, sampler="alias"))
    assert e.value.status == B.MT_ERR_INVALID_ARG and "power" in mt.mt_last_error()
    with pytest.raises(KeyError):
        mt.mt_create(geo, dict(kind="box"), dict(h, sampler="walker"))


def test_polyhedra_descriptor_checks_on_host(lib):
    from workloads import gen
    h = gen.histogram_set(["iron", "air", "concrete"], n_pbin=2, nf=4, ntheta=4, n_samples=1000, cache=False)
    geo = gen.geometry_tapered()
    bad = dict(geo, solids=[dict(geo["solids"][0], bottom=geo["solids"][0]["bottom"][::-1])])   # clockwise
    with pytest.raises(mt.MtError) as e:
        mt.mt_create(bad, dict(kind="box"), h)
    assert e.value.status == B.MT_ERR_INVALID_ARG and "solid 0" in mt.mt_last_error()
    s0 = geo["solids"][0]
    bowtie = dict(s0, top=[s0["top"][0], s0["top"][2], s0["top"][1], s0["top"][3]])            # not convex
    with pytest.raises(mt.MtError):
        mt.mt_create(dict(geo, solids=[bowtie]), dict(kind="box"), h)
    with pytest.raises(mt.MtError):
        mt.mt_create(dict(geo, solids=[dict(s0, z1=s0["z0"])]), dict(kind="box"), h)
    assert ctypes_size_ok()


def ctypes_size_ok():
    # the descriptor the binding builds has the C layout of include/mt.h (8-byte aligned tail)
    return C.sizeof(B.mt_polyhedron) == 8 * (2 + 8 + 8) + 8 + 24 and C.sizeof(B.mt_geometry_desc) % 8 == 0


def test_bv_edges_host_recursion_matches_the_oracle(lib):
    """mt_bv_edges is host code: same edges as the oracle's recursion."""
    import oracle
    rng = np.random.default_rng(4)
    for _ in range(30):
        n = int(rng.integers(3, 400))
        probes = np.sort(rng.uniform(1, 400, n))
        probes = probes[np.concatenate([[True], np.diff(probes) > 0])]
        phi = np.cumsum(rng.normal(0, 0.05, len(probes)))
        eps = float(rng.uniform(0.01, 0.3))
        np.testing.assert_array_equal(mt.mt_bv_edges(probes, phi, eps), oracle.bv_edges(probes, phi, eps))
    with pytest.raises(mt.MtError):
        mt.mt_bv_edges([1.0, 1.0, 2.0], [0.0, 0.0, 0.0], 0.1)


def test_offline_and_edges_host_checks(lib):
    from workloads import gen
    h = gen.histogram_set(["iron"], n_pbin=2, nf=4, ntheta=4, n_samples=1000, cache=False)
    geo, fld, _ = _descs()
    bad = dict(h, p_edges=np.array([1.0, 0.5, 400.0]))
    with pytest.raises(mt.MtError) as e:
        mt.mt_create(geo, fld, bad)
    assert "p_edges" in mt.mt_last_error()
    bad = dict(h, p_edges=np.array([2.0, 20.0, 400.0]))          # must start at p_lo
    with pytest.raises(mt.MtError):
        mt.mt_create(geo, fld, bad)
    st = lib.mt_pilot_phi(None, None, 0, 0, 0.02, 1, None, None)
    assert st == B.MT_ERR_INVALID_ARG
    st = lib.mt_build_histograms(None, 1, 1, None, 4, 4, 0.2, 0.02, 10, 1, None, None, None)
    assert st == B.MT_ERR_INVALID_ARG


def test_compact_workspace_layout(lib):
    """mt_transport_workspace_bytes: one group below 2^19 muons (256 B of
    counters, two 64-byte live entries per muon, the spatial order's two
    16384-word arrays, rounded up to 256 B); from 2^19 muons two groups of
    n // 2 and n - n // 2 muons, each laid out the same way."""
    def group(n):
        b = 256 + 2 * 64 * max(n, 1) + 2 * 16384 * 4
        return (b + 255) // 256 * 256
    for n in (0, 1, 777, 65536, (1 << 19) - 1):
        assert mt.mt_transport_workspace_bytes(n) == group(n), n
    for n in (1 << 19, (1 << 19) + 3, 10**6, (1 << 31) - 1):
        assert mt.mt_transport_workspace_bytes(n) == group(n // 2) + group(n - n // 2), n
    # the no-allocation entry point's fixed array holds one group at its capacity
    assert mt.mt_transport_workspace_bytes(mt.MT_NOALLOC_MAX_MUONS) == group(mt.MT_NOALLOC_MAX_MUONS)
