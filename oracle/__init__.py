"""FP64 CPU oracle for the histogram-sampling muon transport (Algorithm 1).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA path: the C source ``oracle.c`` is compiled on its own with gcc
and loaded here through ctypes.  Inputs come from the ``workloads`` generators
(or from the tests directly); nothing here ever reads a result of the CUDA path.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

ALIVE, STOPPED, EXIT_Z, EXIT_XY, MAX_STEPS, INVALID = range(6)


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` (plain gcc, no fast-math, no FP contraction)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fno-fast-math", "-Wall", "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class World(C.Structure):
    _fields_ = [
        ("geom_kind", C.c_int32), ("n_box", C.c_int32),
        ("box_lo", C.c_void_p), ("box_hi", C.c_void_p), ("box_mat", C.c_void_p),
        ("box_block", C.c_void_p), ("box_B", C.c_void_p), ("poly_z", C.c_void_p), ("poly_xy", C.c_void_p),
        ("world_mat", C.c_int32),
        ("vox_dims", C.c_int32 * 3), ("vox_origin", C.c_double * 3), ("vox_spacing", C.c_double * 3),
        ("vox", C.c_void_p),
        ("x_max", C.c_double), ("y_max", C.c_double), ("z_max", C.c_double), ("p_min", C.c_double),
        ("field_kind", C.c_int32), ("fdims", C.c_int32 * 3), ("forigin", C.c_double * 3),
        ("fspacing", C.c_double * 3), ("Bmap", C.c_void_p), ("field_per_stage", C.c_int32), ("alpha", C.c_void_p),
        ("n_block", C.c_int32),
        ("n_mat", C.c_int32), ("n_pbin", C.c_int32), ("nf", C.c_int32), ("ntheta", C.c_int32),
        ("p_lo", C.c_double), ("p_hi", C.c_double), ("p_edges", C.c_void_p),
        ("f_max", C.c_void_p), ("theta_max", C.c_void_p), ("T", C.c_void_p),
        ("axes", C.c_int32), ("f_min", C.c_void_p), ("theta_min", C.c_void_p),
        ("sampler", C.c_int32), ("alias_prob", C.c_void_p), ("alias_idx", C.c_void_p),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P = C.c_void_p
            L.or_philox4x32_10.argtypes = [P, P, P]
            L.or_philox4x32_10.restype = None
            L.or_uniform.argtypes = [C.c_uint32]
            L.or_uniform.restype = C.c_double
            L.or_build_thresholds.argtypes = [C.c_int64, C.c_int32, P, P]
            L.or_build_thresholds.restype = C.c_int
            L.or_sample_cell.argtypes = [P, C.c_int32, C.c_uint32]
            L.or_sample_cell.restype = C.c_int32
            L.or_build_alias.argtypes = [C.c_int64, C.c_int32, P, P, P]
            L.or_build_alias.restype = C.c_int
            L.or_sample_alias.argtypes = [P, P, C.c_int32, C.c_uint32]
            L.or_sample_alias.restype = C.c_int32
            L.or_momentum_bin.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int32]
            L.or_momentum_bin.restype = C.c_int32
            L.or_momentum_bin_edges.argtypes = [C.c_double, P, C.c_int32]
            L.or_momentum_bin_edges.restype = C.c_int32
            L.or_highland.argtypes = [C.c_double, C.c_double, C.c_double]
            L.or_highland.restype = C.c_double
            L.or_physics_sample.argtypes = [P, C.c_double, C.c_double, P, P, P]
            L.or_physics_sample.restype = None
            L.or_build_histograms.argtypes = [P, C.c_int32, C.c_int32, P, C.c_int32, C.c_int32, C.c_double,
                                              C.c_double, C.c_int64, C.c_uint64, P, P]
            L.or_build_histograms.restype = C.c_int
            L.or_pilot_phi.argtypes = [P, P, C.c_int32, C.c_int64, C.c_double, C.c_uint64, P]
            L.or_pilot_phi.restype = C.c_int
            L.or_bv_edges.argtypes = [P, P, C.c_int32, C.c_double, P, C.c_int32]
            L.or_bv_edges.restype = C.c_int32
            L.or_material.argtypes = [P, P, P]
            L.or_material.restype = C.c_int32
            L.or_in_solid.argtypes = [P, C.c_int32, P]
            L.or_in_solid.restype = C.c_int
            L.or_field.argtypes = [P, P, C.c_int32, P]
            L.or_field.restype = None
            L.or_scatter.argtypes = [P, C.c_double, C.c_double, C.c_double, P]
            L.or_scatter.restype = None
            L.or_scatter_c.argtypes = [P, C.c_double, C.c_double, C.c_double, P]
            L.or_scatter_c.restype = None
            L.or_dp_coeffs.argtypes = [C.c_int32, C.c_double, C.c_double, P, P]
            L.or_dp_coeffs.restype = None
            L.or_rk4.argtypes = [P, P, P, C.c_int32, C.c_double]
            L.or_rk4.restype = None
            L.or_transport.argtypes = [P, C.c_int64] + [P] * 9 + [C.c_int64, C.c_int32, C.c_double,
                                                               C.c_int32, C.c_uint64, C.c_int32]
            L.or_transport.restype = C.c_int
            L.or_trace.argtypes = [P, P, P, C.c_int32, C.c_int32, C.c_uint64, C.c_int32, C.c_double,
                                   C.c_int32, C.c_uint64, P, P, P]
            L.or_trace.restype = C.c_int32
            L.or_draw.argtypes = [P, P, P, C.c_int32, C.c_uint64, C.c_int32, C.c_uint64, P, P]
            L.or_draw.restype = C.c_int32
            L.or_acceptance_loss.argtypes = [C.c_int64] + [P] * 7 + [C.c_double] * 3 + [P]
            L.or_acceptance_loss.restype = C.c_double
            L.or_adjoint.argtypes = [P, C.c_int64] + [P] * 9 + [C.c_int64, C.c_int32, C.c_double, C.c_int32,
                                                             C.c_uint64, P, P, C.c_int32]
            L.or_adjoint.restype = C.c_int
            L.or_transport_tangent.argtypes = [P, P, P, C.c_int32, C.c_int32, C.c_uint64, C.c_int32, C.c_double,
                                               C.c_int32, C.c_uint64, P, P]
            L.or_transport_tangent.restype = C.c_int32
            _lib = L
    return _lib


def _p(a: np.ndarray) -> int:
    return a.ctypes.data


# --------------------------------------------------------------------------
# primitives
# --------------------------------------------------------------------------
def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib().or_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def uniform(w: int) -> float:
    return lib().or_uniform(int(w))


def build_thresholds(weights: np.ndarray) -> np.ndarray:
    """weights [..., nf, ntheta] -> uint64 thresholds [..., nf*ntheta-1]."""
    w = np.ascontiguousarray(weights, dtype=np.float64)
    ncell = w.shape[-1] * w.shape[-2]
    lead = w.shape[:-2]
    n_hist = int(np.prod(lead)) if lead else 1
    T = np.zeros(lead + (ncell - 1,), np.uint64)
    rc = lib().or_build_thresholds(n_hist, ncell, _p(w), _p(T))
    if rc != 0:
        raise ValueError(f"or_build_thresholds failed ({rc})")
    return T


def sample_cell(T_row: np.ndarray, w0: int) -> int:
    T = np.ascontiguousarray(T_row, dtype=np.uint64)
    return lib().or_sample_cell(_p(T), T.shape[-1] + 1, int(w0))


def build_alias(T: np.ndarray, ncell: int):
    """uint64 thresholds [..., ncell-1] -> alias tables (prob uint32 [..., ncell], alias int32 [..., ncell])."""
    T = np.ascontiguousarray(T, dtype=np.uint64)
    lead = T.shape[:-1]
    n_hist = int(np.prod(lead)) if lead else 1
    prob = np.zeros(lead + (ncell,), np.uint32)
    alias = np.zeros(lead + (ncell,), np.int32)
    rc = lib().or_build_alias(n_hist, int(ncell), _p(T), _p(prob), _p(alias))
    if rc != 0:
        raise ValueError(f"or_build_alias failed ({rc})")
    return prob, alias


def sample_alias(prob_row: np.ndarray, alias_row: np.ndarray, w0: int) -> int:
    P = np.ascontiguousarray(prob_row, dtype=np.uint32)
    A = np.ascontiguousarray(alias_row, dtype=np.int32)
    return lib().or_sample_alias(_p(P), _p(A), P.shape[-1], int(w0))


def momentum_bin(P: float, p_lo: float, p_hi: float, n_pbin: int) -> int:
    return lib().or_momentum_bin(float(P), float(p_lo), float(p_hi), int(n_pbin))


def scatter(p, f, theta, phi) -> np.ndarray:
    pp = np.ascontiguousarray(p, dtype=np.float64)
    out = np.zeros(3)
    lib().or_scatter(_p(pp), float(f), float(theta), float(phi), _p(out))
    return out


def scatter_c(p, cz, ct, phi) -> np.ndarray:
    """p + Rot([P ct cos phi, P ct sin phi, P cz]) (Algorithm 1's dp with dz = P cz, dt = P ct; Eq. 3)."""
    pp = np.ascontiguousarray(p, dtype=np.float64)
    out = np.zeros(3)
    lib().or_scatter_c(_p(pp), float(cz), float(ct), float(phi), _p(out))
    return out


def dp_coeffs(axes: str, f: float, theta_or_t: float):
    cz = C.c_double()
    ct = C.c_double()
    lib().or_dp_coeffs(1 if axes == "log" else 0, float(f), float(theta_or_t), C.byref(cz), C.byref(ct))
    return cz.value, ct.value


def rk4(r, p, B, q, d):
    rr = np.array(r, dtype=np.float64)
    pp = np.array(p, dtype=np.float64)
    BB = np.ascontiguousarray(B, dtype=np.float64)
    lib().or_rk4(_p(rr), _p(pp), _p(BB), int(q), float(d))
    return rr, pp


# --------------------------------------------------------------------------
# world
# --------------------------------------------------------------------------
class OracleWorld:
    """Owns the arrays behind an ``or_world`` built from workload dicts."""

    def __init__(self, geometry: dict, field: dict, hist: dict, alpha: Optional[np.ndarray] = None):
        w = World()
        keep = []

        def arr(a, dt):
            a = np.ascontiguousarray(a, dtype=dt)
            keep.append(a)
            return a

        if geometry["kind"] == "boxes":
            boxes = geometry["boxes"]
            w.geom_kind = 0
            w.n_box = len(boxes)
            if boxes:
                w.box_lo = _p(arr([b["lo"] for b in boxes], np.float64))
                w.box_hi = _p(arr([b["hi"] for b in boxes], np.float64))
                w.box_mat = _p(arr([b["material"] for b in boxes], np.int32))
                w.box_block = _p(arr([b.get("block_id", -1) for b in boxes], np.int32))
                w.box_B = _p(arr([b.get("B", [0, 0, 0]) for b in boxes], np.float64))
        elif geometry["kind"] == "polyhedra":
            solids = geometry["solids"]
            w.geom_kind = 2
            w.n_box = len(solids)
            if solids:
                w.poly_z = _p(arr([[s_["z0"], s_["z1"]] for s_ in solids], np.float64))
                w.poly_xy = _p(arr([[s_["bottom"], s_["top"]] for s_ in solids], np.float64))
                w.box_mat = _p(arr([s_["material"] for s_ in solids], np.int32))
                w.box_block = _p(arr([s_.get("block_id", -1) for s_ in solids], np.int32))
                w.box_B = _p(arr([s_.get("B", [0, 0, 0]) for s_ in solids], np.float64))
        elif geometry["kind"] == "voxels":
            w.geom_kind = 1
            w.n_box = 0
            vox = arr(geometry["voxels"], np.uint8)
            nz, ny, nx = vox.shape
            w.vox_dims[:] = [nx, ny, nz]
            w.vox_origin[:] = list(map(float, geometry["origin"]))
            w.vox_spacing[:] = list(map(float, geometry["spacing"]))
            w.vox = _p(vox)
        else:
            raise ValueError(geometry["kind"])
        w.world_mat = int(geometry["world_material"])
        w.x_max, w.y_max, w.z_max = float(geometry["x_max"]), float(geometry["y_max"]), float(geometry["z_max"])
        w.p_min = float(geometry["p_min"])

        fk = field["kind"]
        if fk == "none":
            w.field_kind = 0
        elif fk == "box":
            w.field_kind = 1
        elif fk in ("map", "map_nearest"):
            w.field_kind = 2 if fk == "map" else 3
            B = arr(field["B"], np.float32)
            w.fdims[:] = list(map(int, field["dims"]))
            w.forigin[:] = list(map(float, field["origin"]))
            w.fspacing[:] = list(map(float, field["spacing"]))
            w.Bmap = _p(B)
            w.field_per_stage = int(bool(field.get("per_stage", False)))
        else:
            raise ValueError(fk)
        if alpha is not None:
            a = arr(alpha, np.float64).reshape(-1, 3)
            w.alpha = _p(a)
            w.n_block = a.shape[0]

        w.n_mat, w.n_pbin = int(hist["n_mat"]), int(hist["n_pbin"])
        w.nf, w.ntheta = int(hist["nf"]), int(hist["ntheta"])
        w.p_lo, w.p_hi = float(hist["p_lo"]), float(hist["p_hi"])
        if hist.get("p_edges") is not None:
            w.p_edges = _p(arr(hist["p_edges"], np.float64))
        w.f_max = _p(arr(hist["f_max"], np.float64))
        w.theta_max = _p(arr(hist["theta_max"], np.float64))
        axes = hist.get("axes", "linear")
        if axes == "log":
            w.axes = 1
            w.f_min = _p(arr(hist["f_min"], np.float64))
            w.theta_min = _p(arr(hist["theta_min"], np.float64))
        elif axes != "linear":
            raise ValueError(axes)
        self.T = arr(build_thresholds(hist["weights"]), np.uint64)
        w.T = _p(self.T)
        if hist.get("sampler", "icdf") == "alias":
            prob, alias = build_alias(self.T, w.nf * w.ntheta)
            w.sampler = 1
            w.alias_prob = _p(arr(prob, np.uint32))
            w.alias_idx = _p(arr(alias, np.int32))
        elif hist.get("sampler", "icdf") != "icdf":
            raise ValueError(hist["sampler"])
        self.w = w
        self._keep = keep

    @property
    def ptr(self) -> int:
        return C.addressof(self.w)

    def material(self, r):
        rr = np.ascontiguousarray(r, dtype=np.float64)
        box = np.zeros(1, np.int32)
        m = lib().or_material(self.ptr, _p(rr), _p(box))
        return m, int(box[0])

    def field(self, r, box: int = -1) -> np.ndarray:
        rr = np.ascontiguousarray(r, dtype=np.float64)
        B = np.zeros(3)
        lib().or_field(self.ptr, _p(rr), int(box), _p(B))
        return B


def draw(world: OracleWorld, r, p, k: int, mid: int, seed: int, instance: int = 0):
    """One step's draw at state (r, p): ((mat, box, pbin, cell), (f, theta, phi))."""
    rr = np.ascontiguousarray(r, dtype=np.float64)
    pp = np.ascontiguousarray(p, dtype=np.float64)
    ib = np.zeros(4, np.int32)
    db = np.zeros(3, np.float64)
    lib().or_draw(world.ptr, _p(rr), _p(pp), int(k), int(mid), int(instance), int(seed), _p(ib), _p(db))
    return tuple(int(v) for v in ib), tuple(float(v) for v in db)


def world_of(wl, alpha=None) -> OracleWorld:
    return OracleWorld(wl.geometry, wl.field, wl.hist, alpha)


def transport(world: OracleWorld, muons: dict, step_len: float, max_steps: int, seed: int,
              id_offset: int = 0, instance: int = 0, n_threads: Optional[int] = None,
              index: Optional[np.ndarray] = None) -> dict:
    """Run Algorithm 1 in FP64 on a copy of ``muons`` (float32 SoA dict).

    ``index`` selects a subset of muons; muon ids stay id_offset + original index, so a
    subset reproduces exactly what a full run gives for those muons.
    """
    sel = np.arange(len(muons["x"])) if index is None else np.asarray(index, dtype=np.int64)
    out = {k: np.ascontiguousarray(np.asarray(muons[k])[sel], dtype=np.float64)
           for k in ("x", "y", "z", "px", "py", "pz")}
    q = np.ascontiguousarray(np.asarray(muons["q"])[sel], dtype=np.int8)
    steps = np.ascontiguousarray(np.asarray(muons["steps"])[sel], dtype=np.int32)
    status = np.ascontiguousarray(np.asarray(muons["status"])[sel], dtype=np.uint8)
    nt = n_threads or os.cpu_count() or 1
    L = lib()
    if index is None:
        rc = L.or_transport(world.ptr, len(sel), *(_p(out[k]) for k in ("x", "y", "z", "px", "py", "pz")),
                            _p(q), _p(steps), _p(status), int(id_offset), int(instance), float(step_len),
                            int(max_steps), int(seed), int(nt))
        if rc != 0:
            raise RuntimeError("or_transport failed")
    else:
        # ids are not contiguous: run each contiguous run of indices with its own offset
        order = np.argsort(sel, kind="stable")
        s_sorted = sel[order]
        tmp = {k: out[k][order].copy() for k in out}
        q_s, st_s, stat_s = q[order].copy(), steps[order].copy(), status[order].copy()
        start = 0
        n = len(s_sorted)
        runs = []
        while start < n:
            end = start + 1
            while end < n and s_sorted[end] == s_sorted[end - 1] + 1:
                end += 1
            runs.append((start, end))
            start = end
        def run(ab):
            a, b = ab
            views = [tmp[k][a:b] for k in ("x", "y", "z", "px", "py", "pz")]
            return L.or_transport(world.ptr, b - a, *(_p(v) for v in views), _p(q_s[a:b]), _p(st_s[a:b]),
                                  _p(stat_s[a:b]), int(id_offset + s_sorted[a]), int(instance),
                                  float(step_len), int(max_steps), int(seed), int(min(nt, b - a)))

        # runs are independent muons: short runs go to a pool of host threads (the
        # C call releases the GIL), long runs thread inside the oracle
        short = [r for r in runs if r[1] - r[0] < nt]
        rcs = [run(r) for r in runs if r[1] - r[0] >= nt]
        if short:
            import concurrent.futures
            with concurrent.futures.ThreadPoolExecutor(max_workers=nt) as ex:
                rcs += list(ex.map(run, short))
        if any(rc != 0 for rc in rcs):
            raise RuntimeError("or_transport failed")
        inv = np.empty_like(order)
        inv[order] = np.arange(n)
        for k in out:
            out[k] = tmp[k][inv]
        steps, status = st_s[inv], stat_s[inv]
    out["q"] = q
    out["steps"] = steps
    out["status"] = status
    return out


def trace(world: OracleWorld, r, p, q: int, max_steps: int, step_len: float, seed: int, mid: int = 0,
          instance: int = 0, steps0: int = 0) -> dict:
    """Per-step record of one muon: draws (mat, box, pbin, cell, f, theta, phi), r before the
    step, p after scattering and B used.  Returns the final state too."""
    rr = np.array(r, dtype=np.float64)
    pp = np.array(p, dtype=np.float64)
    ib = np.zeros((max_steps, 4), np.int32)
    db = np.zeros((max_steps, 9), np.float64)
    fb = np.zeros((max_steps, 3), np.float64)
    s = lib().or_trace(world.ptr, _p(rr), _p(pp), int(q), int(steps0), int(mid), int(instance),
                       float(step_len), int(max_steps), int(seed), _p(ib), _p(db), _p(fb))
    return dict(n=s, mat=ib[:s, 0], box=ib[:s, 1], pbin=ib[:s, 2], cell=ib[:s, 3], f=fb[:s, 0],
                theta=fb[:s, 1], phi=fb[:s, 2], r=db[:s, :3], p_scat=db[:s, 3:6], B=db[:s, 6:9],
                r_final=rr, p_final=pp)


# --------------------------------------------------------------------------
# differentiable form
# --------------------------------------------------------------------------
N_TANGENT = 18


def acceptance_loss(final: dict, z_plane: float = 30.0, half: float = 0.5, width: float = 0.01):
    """Mean acceptance loss of a final state and dL/d(x, y, z, px, py, pz) as a [6, n] array."""
    cols = [np.ascontiguousarray(final[k], dtype=np.float64) for k in ("x", "y", "z", "px", "py", "pz")]
    st = np.ascontiguousarray(final["status"], dtype=np.uint8)
    n = len(cols[0])
    g = np.zeros((6, n))
    L = lib().or_acceptance_loss(n, *(_p(c) for c in cols), _p(st), float(z_plane), float(half), float(width),
                                 _p(g))
    return L, g


def adjoint(world: OracleWorld, muons: dict, step_len: float, max_steps: int, seed: int, g: np.ndarray,
            id_offset: int = 0, instance: int = 0, n_threads: Optional[int] = None) -> np.ndarray:
    """dL/dalpha [n_block, 3] from the INITIAL muons and dL/d(final state) g [6, n] (FP64 reverse mode)."""
    if not world.w.alpha:
        raise ValueError("the oracle world needs alpha for the adjoint")
    cols = [np.ascontiguousarray(muons[k], dtype=np.float64) for k in ("x", "y", "z", "px", "py", "pz")]
    q = np.ascontiguousarray(muons["q"], dtype=np.int8)
    steps = np.ascontiguousarray(muons["steps"], dtype=np.int32)
    status = np.ascontiguousarray(muons["status"], dtype=np.uint8)
    gg = np.ascontiguousarray(g, dtype=np.float64)
    out = np.zeros(3 * world.w.n_block)
    rc = lib().or_adjoint(world.ptr, len(cols[0]), *(_p(c) for c in cols), _p(q), _p(steps), _p(status),
                          int(id_offset), int(instance), float(step_len), int(max_steps), int(seed), _p(gg),
                          _p(out), int(n_threads or os.cpu_count() or 1))
    if rc != 0:
        raise RuntimeError("or_adjoint failed")
    return out.reshape(-1, 3)


def transport_tangent(world: OracleWorld, r, p, q: int, max_steps: int, step_len: float, seed: int, mid: int,
                      instance: int = 0, steps0: int = 0):
    """Final (x,y,z,px,py,pz) of one muon and d(final)/d(alpha) [6, 18] by forward-mode dual numbers."""
    rr = np.ascontiguousarray(r, dtype=np.float64)
    pp = np.ascontiguousarray(p, dtype=np.float64)
    out = np.zeros(6)
    tan = np.zeros((6, N_TANGENT))
    ns = lib().or_transport_tangent(world.ptr, _p(rr), _p(pp), int(q), int(steps0), int(mid), int(instance),
                                    float(step_len), int(max_steps), int(seed), _p(out), _p(tan))
    return out, tan, ns


# --------------------------------------------------------------------------
# offline phase: parametric physics sampler, histograms, pilot estimator, binning
# --------------------------------------------------------------------------
def _material_array(materials):
    """Materials as a packed (rho, Z/A, I [MeV], X0 [cm], b) float64 array (dicts as in workloads.MATERIALS)."""
    return np.ascontiguousarray([[m["rho"], m["ZA"], m["I"], m["X0"], m["b"]] for m in materials], np.float64)


def momentum_bin_edges(P: float, edges) -> int:
    e = np.ascontiguousarray(edges, dtype=np.float64)
    return lib().or_momentum_bin_edges(float(P), _p(e), len(e) - 1)


def highland(p: float, x_cm: float, X0: float) -> float:
    return lib().or_highland(float(p), float(x_cm), float(X0))


def physics_sample(material: dict, p: float, x_cm: float, u):
    m = _material_array([material])
    uu = np.ascontiguousarray(u, dtype=np.float64)
    f = C.c_double()
    th = C.c_double()
    lib().or_physics_sample(_p(m), float(p), float(x_cm), _p(uu), C.byref(f), C.byref(th))
    return f.value, th.value


def physics_samples(material: dict, p: float, x_cm: float, U: np.ndarray):
    """(f, theta) arrays of or_physics_sample for each row of U (rows of eight uniforms)."""
    m = _material_array([material])
    U = np.ascontiguousarray(U, dtype=np.float64)
    f = np.zeros(len(U))
    th = np.zeros(len(U))
    fn = lib().or_physics_sample
    pm, fb, tb = _p(m), f.ctypes.data, th.ctypes.data
    for i in range(len(U)):
        fn(pm, float(p), float(x_cm), U[i].ctypes.data, fb + 8 * i, tb + 8 * i)
    return f, th


def build_histograms(materials, edges, nf: int, ntheta: int, f_max: float, step_len: float, n_samples: int,
                     seed: int):
    """(counts [n_mat][n_pbin][nf][ntheta], theta_max [n_mat][n_pbin]) from the parametric sampler."""
    m = _material_array(materials)
    e = np.ascontiguousarray(edges, dtype=np.float64)
    n_pbin = len(e) - 1
    counts = np.zeros((len(materials), n_pbin, nf, ntheta))
    tmax = np.zeros((len(materials), n_pbin))
    lib().or_build_histograms(_p(m), len(materials), n_pbin, _p(e), nf, ntheta, float(f_max), step_len * 100.0,
                              int(n_samples), int(seed), _p(counts), _p(tmax))
    return counts, tmax


def pilot_phi(material: dict, probes, K: int, step_len: float, seed: int) -> np.ndarray:
    m = _material_array([material])
    pr = np.ascontiguousarray(probes, dtype=np.float64)
    phi = np.zeros(len(pr))
    lib().or_pilot_phi(_p(m), _p(pr), len(pr), int(K), step_len * 100.0, int(seed), _p(phi))
    return phi


def bv_edges(probes, phi, eps: float) -> np.ndarray:
    pr = np.ascontiguousarray(probes, dtype=np.float64)
    ph = np.ascontiguousarray(phi, dtype=np.float64)
    out = np.zeros(len(pr))
    n = lib().or_bv_edges(_p(pr), _p(ph), len(pr), float(eps), _p(out), len(pr))
    if n < 0:
        raise ValueError("or_bv_edges failed")
    return out[:n].copy()
