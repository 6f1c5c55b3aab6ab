"""ctypes binding of libmt.so (include/mt.h): argument marshalling only.

Every step of the transport runs in the library's CUDA kernels; this module only
turns Python/numpy descriptors into the C structs of mt.h and torch device
tensors into raw pointers.  It raises if libmt.so has not been built: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import re
import threading
from typing import Dict, Optional

import numpy as np

from . import _build

MT_OK, MT_ERR_INVALID_ARG, MT_ERR_CUDA, MT_ERR_OOM, MT_ERR_TIMEOUT, MT_ERR_TABLE, MT_ERR_DEVICE = range(7)
MT_ALIVE, MT_STOPPED, MT_EXIT_Z, MT_EXIT_XY, MT_MAX_STEPS, MT_INVALID = range(6)
MT_GEOM_BOXES, MT_GEOM_VOXELS, MT_GEOM_POLYHEDRA = 0, 1, 2
MT_FIELD_NONE, MT_FIELD_BOX, MT_FIELD_MAP, MT_FIELD_MAP_NEAREST = 0, 1, 2, 3
STATUS_NAMES = {0: "MT_OK", 1: "MT_ERR_INVALID_ARG", 2: "MT_ERR_CUDA", 3: "MT_ERR_OOM", 4: "MT_ERR_TIMEOUT",
                5: "MT_ERR_TABLE", 6: "MT_ERR_DEVICE"}


class MtError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class mt_box(C.Structure):
    _fields_ = [("lo", C.c_double * 3), ("hi", C.c_double * 3), ("material", C.c_int32),
                ("block_id", C.c_int32), ("B", C.c_double * 3)]


class mt_polyhedron(C.Structure):
    _fields_ = [("z0", C.c_double), ("z1", C.c_double), ("bottom", (C.c_double * 2) * 4),
                ("top", (C.c_double * 2) * 4), ("material", C.c_int32), ("block_id", C.c_int32),
                ("B", C.c_double * 3)]


class mt_geometry_desc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n_boxes", C.c_int32), ("boxes", C.POINTER(mt_box)),
                ("world_material", C.c_int32), ("vox_dims", C.c_int32 * 3), ("vox_origin", C.c_double * 3),
                ("vox_spacing", C.c_double * 3), ("voxels", C.c_void_p), ("x_max", C.c_double),
                ("y_max", C.c_double), ("z_max", C.c_double), ("p_min", C.c_double),
                ("polys", C.POINTER(mt_polyhedron)), ("n_polys", C.c_int32), ("reserved", C.c_int32)]


class mt_field_desc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("dims", C.c_int32 * 3), ("origin", C.c_double * 3),
                ("spacing", C.c_double * 3), ("B", C.c_void_p), ("per_stage", C.c_int32), ("reserved", C.c_int32)]


class mt_hist_desc(C.Structure):
    _fields_ = [("n_mat", C.c_int32), ("n_pbin", C.c_int32), ("p_lo", C.c_double), ("p_hi", C.c_double),
                ("nf", C.c_int32), ("ntheta", C.c_int32), ("weights", C.c_void_p), ("f_max", C.c_void_p),
                ("theta_max", C.c_void_p), ("sampler", C.c_int32), ("axes", C.c_int32), ("f_min", C.c_void_p),
                ("theta_min", C.c_void_p), ("p_edges", C.c_void_p)]


class mt_material(C.Structure):
    _fields_ = [("rho", C.c_double), ("z_over_a", C.c_double), ("I_mev", C.c_double), ("X0_cm", C.c_double),
                ("b_rad", C.c_double)]


MT_SAMPLER_ICDF, MT_SAMPLER_ALIAS = 0, 1
SAMPLERS = {"icdf": MT_SAMPLER_ICDF, "alias": MT_SAMPLER_ALIAS}
MT_AXES_LINEAR, MT_AXES_LOG = 0, 1
AXES = {"linear": MT_AXES_LINEAR, "log": MT_AXES_LOG}


class mt_launch_cfg(C.Structure):
    _fields_ = [("mode", C.c_int32), ("blocks_per_sm", C.c_int32), ("steps_per_pass", C.c_int32),
                ("order", C.c_int32), ("workspace", C.c_void_p), ("workspace_bytes", C.c_int64)]


MT_LAUNCH_AUTO, MT_LAUNCH_STATIC, MT_LAUNCH_PERSISTENT, MT_LAUNCH_COMPACT = 0, 1, 2, 3
MT_ORDER_AUTO, MT_ORDER_ALWAYS, MT_ORDER_NEVER = 0, 1, 2


MT_BATCH_STAGE_SHARED, MT_BATCH_STAGE_GLOBAL = 1, 2


class mt_batch_cfg(C.Structure):
    _fields_ = [("block", C.c_int32), ("steps_per_pass", C.c_int32), ("use_graph", C.c_int32),
                ("staging", C.c_int32), ("order", C.c_int32), ("reserved", C.c_int32), ("workspace", C.c_void_p),
                ("workspace_bytes", C.c_int64)]


class mt_muon_soa(C.Structure):
    _fields_ = [("x", C.c_void_p), ("y", C.c_void_p), ("z", C.c_void_p), ("px", C.c_void_p),
                ("py", C.c_void_p), ("pz", C.c_void_p), ("q", C.c_void_p), ("steps", C.c_void_p),
                ("status", C.c_void_p), ("id_offset", C.c_int64), ("instance", C.c_int32),
                ("reserved", C.c_int32)]


_lib = None
_lock = threading.Lock()

_P = C.c_void_p
_SIGNATURES = {
    "mt_abi_version": ([], C.c_int32),
    "mt_last_error": ([], C.c_char_p),
    "mt_create": ([C.POINTER(mt_geometry_desc), C.POINTER(mt_field_desc), C.POINTER(mt_hist_desc),
                   C.POINTER(_P)], C.c_int),
    "mt_destroy": ([_P], None),
    "mt_device_bytes": ([_P], C.c_int64),
    "mt_transport": ([_P, C.POINTER(mt_muon_soa), C.c_int64, C.c_float, C.c_int32, C.c_uint64, _P], C.c_int),
    "mt_transport_scaled": ([_P, C.POINTER(mt_muon_soa), C.c_int64, C.c_float, C.c_int32, C.c_uint64, _P,
                             C.c_int32, _P], C.c_int),
    "mt_transport_cfg": ([_P, C.POINTER(mt_muon_soa), C.c_int64, C.c_float, C.c_int32, C.c_uint64, _P,
                          C.c_int32, C.POINTER(mt_launch_cfg), _P], C.c_int),
    "mt_transport_workspace_bytes": ([C.c_int64], C.c_int64),
    "mt_transport_launches": ([_P, C.c_int64, C.c_float, C.c_int32, C.POINTER(mt_launch_cfg)], C.c_int64),
    "mt_transport_noalloc": ([_P, C.POINTER(mt_muon_soa), C.c_int64, C.c_float, C.c_int32, C.c_uint64, _P],
                             C.c_int),
    "mt_ckpt_bytes": ([C.c_int64, C.c_int32, C.c_int32], C.c_int64),
    "mt_transport_ckpt": ([_P, C.POINTER(mt_muon_soa), C.c_int64, C.c_float, C.c_int32, C.c_uint64, _P, C.c_int32,
                           C.c_int32, _P, C.c_int64, _P], C.c_int),
    "mt_adjoint_ckpt": ([_P, C.c_int64, C.c_float, C.c_int32, C.c_uint64, _P, C.c_int32, C.c_int32, _P, C.c_int64,
                         C.c_int64, C.c_int32, _P, _P, _P, _P], C.c_int),
    "mt_transport_adjoint": ([_P, C.POINTER(mt_muon_soa), C.c_int64, C.c_float, C.c_int32, C.c_uint64, _P,
                              C.c_int32, _P, _P, C.c_int32, _P], C.c_int),
    "mt_acceptance_loss": ([C.POINTER(mt_muon_soa), C.c_int64, C.c_double, C.c_double, C.c_double, _P, _P, _P],
                           C.c_int),
    "mt_tape_bytes": ([C.c_int64, C.c_int32, C.c_int32], C.c_int64),
    "mt_transport_tape": ([_P, C.POINTER(mt_muon_soa), C.c_int64, C.c_float, C.c_int32, C.c_uint64, _P, C.c_int32,
                           C.c_int32, _P, C.c_int64, _P], C.c_int),
    "mt_adjoint_tape": ([_P, C.c_int64, C.c_float, C.c_int32, _P, C.c_int32, C.c_int32, _P, C.c_int64, _P, _P, _P,
                         _P], C.c_int),
    "mt_build_histograms": ([C.POINTER(mt_material), C.c_int32, C.c_int32, _P, C.c_int32, C.c_int32, C.c_double,
                             C.c_double, C.c_int64, C.c_uint64, _P, _P, _P], C.c_int),
    "mt_pilot_phi": ([C.POINTER(mt_material), _P, C.c_int32, C.c_int64, C.c_double, C.c_uint64, _P, _P], C.c_int),
    "mt_bv_edges": ([_P, _P, C.c_int32, C.c_double, _P, C.c_int32], C.c_int32),
    "mt_batch_create": ([C.POINTER(mt_hist_desc), C.c_int32, C.POINTER(_P)], C.c_int),
    "mt_batch_set_instance": ([_P, C.c_int32, C.POINTER(mt_geometry_desc), C.POINTER(mt_field_desc)], C.c_int),
    "mt_batch_destroy": ([_P], None),
    "mt_batch_device_bytes": ([_P], C.c_int64),
    "mt_batch_workspace_bytes": ([_P, C.POINTER(C.c_int64)], C.c_int64),
    "mt_transport_batched": ([_P, C.POINTER(mt_muon_soa), C.POINTER(C.c_int64), C.c_float, C.c_int32, C.c_uint64,
                              C.POINTER(mt_batch_cfg), _P], C.c_int),
    "mt_batch_autotune": ([_P, C.POINTER(mt_muon_soa), C.POINTER(C.c_int64), C.c_float, C.c_int32, C.c_uint64,
                           C.c_int64, C.POINTER(mt_batch_cfg), _P], C.c_int),
}

MT_NOALLOC_MAX_MUONS = 65536


def library_path() -> str:
    return _build.LIB_PATH


def load_library():
    """Load libmt.so; raises if it has not been built (call __graft_entry__.build())."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if not os.path.exists(path):
                raise ImportError(f"libmt.so not built at {path}: run `python -c 'import __graft_entry__ as g; "
                                  f"g.build()'` first (there is no CPU fallback)")
            L = C.CDLL(path)
            for name, (args, res) in _SIGNATURES.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = res
            _lib = L
    return _lib


def declared_symbols(header: Optional[str] = None):
    """Names of the functions declared in include/mt.h."""
    header = header or os.path.join(_build.INCLUDE, "mt.h")
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mt_[a-z_0-9]+)\s*\(", text)))


def _check(status: int, where: str):
    if status != MT_OK:
        msg = load_library().mt_last_error().decode(errors="replace")
        raise MtError(status, where, msg)


def mt_abi_version() -> int:
    return load_library().mt_abi_version()


def mt_last_error() -> str:
    return load_library().mt_last_error().decode(errors="replace")


# --------------------------------------------------------------------------
# descriptors from workload dicts
# --------------------------------------------------------------------------
class _Descs:
    """C descriptors plus the numpy arrays they point into (kept alive here)."""

    def __init__(self, geometry: Optional[dict], field: Optional[dict], hist: Optional[dict]):
        keep = []
        self.g = self.f = self.h = None

        def arr(a, dt):
            a = np.ascontiguousarray(a, dtype=dt)
            keep.append(a)
            return a

        if geometry is not None:
            self.g = self._geometry(geometry, arr, keep)
        if field is not None:
            self.f = self._field(field, arr)
        if hist is not None:
            self.h = self._hist(hist, arr)
        self._keep = keep

    @staticmethod
    def _geometry(geometry, arr, keep):
        g = mt_geometry_desc()
        if geometry["kind"] == "boxes":
            boxes = geometry["boxes"]
            g.kind = MT_GEOM_BOXES
            g.n_boxes = len(boxes)
            arr_t = mt_box * max(1, len(boxes))
            barr = arr_t()
            for i, b in enumerate(boxes):
                barr[i].lo[:] = list(map(float, b["lo"]))
                barr[i].hi[:] = list(map(float, b["hi"]))
                barr[i].material = int(b["material"])
                barr[i].block_id = int(b.get("block_id", -1))
                barr[i].B[:] = list(map(float, b.get("B", [0.0, 0.0, 0.0])))
            keep.append(barr)
            g.boxes = C.cast(barr, C.POINTER(mt_box))
        elif geometry["kind"] == "polyhedra":
            solids = geometry["solids"]
            g.kind = MT_GEOM_POLYHEDRA
            g.n_polys = len(solids)
            parr = (mt_polyhedron * max(1, len(solids)))()
            for i, sd in enumerate(solids):
                parr[i].z0, parr[i].z1 = float(sd["z0"]), float(sd["z1"])
                for v in range(4):
                    parr[i].bottom[v][:] = list(map(float, sd["bottom"][v]))
                    parr[i].top[v][:] = list(map(float, sd["top"][v]))
                parr[i].material = int(sd["material"])
                parr[i].block_id = int(sd.get("block_id", -1))
                parr[i].B[:] = list(map(float, sd.get("B", [0.0, 0.0, 0.0])))
            keep.append(parr)
            g.polys = C.cast(parr, C.POINTER(mt_polyhedron))
        elif geometry["kind"] == "voxels":
            vox = arr(geometry["voxels"], np.uint8)
            nz, ny, nx = vox.shape
            g.kind = MT_GEOM_VOXELS
            g.vox_dims[:] = [nx, ny, nz]
            g.vox_origin[:] = list(map(float, geometry["origin"]))
            g.vox_spacing[:] = list(map(float, geometry["spacing"]))
            g.voxels = vox.ctypes.data
        else:
            raise ValueError(geometry["kind"])
        g.world_material = int(geometry["world_material"])
        g.x_max, g.y_max, g.z_max = (float(geometry[k]) for k in ("x_max", "y_max", "z_max"))
        g.p_min = float(geometry["p_min"])
        return g

    @staticmethod
    def _field(field, arr):
        f = mt_field_desc()
        kind = field["kind"]
        f.kind = {"none": MT_FIELD_NONE, "box": MT_FIELD_BOX, "map": MT_FIELD_MAP,
                  "map_nearest": MT_FIELD_MAP_NEAREST}[kind]
        if kind in ("map", "map_nearest"):
            B = arr(field["B"], np.float32)
            f.dims[:] = list(map(int, field["dims"]))
            f.origin[:] = list(map(float, field["origin"]))
            f.spacing[:] = list(map(float, field["spacing"]))
            f.B = B.ctypes.data
        f.per_stage = int(bool(field.get("per_stage", False)))
        return f

    @staticmethod
    def _hist(hist, arr):
        h = mt_hist_desc()
        h.n_mat, h.n_pbin = int(hist["n_mat"]), int(hist["n_pbin"])
        h.p_lo, h.p_hi = float(hist["p_lo"]), float(hist["p_hi"])
        h.nf, h.ntheta = int(hist["nf"]), int(hist["ntheta"])
        h.weights = arr(hist["weights"], np.float64).ctypes.data
        h.f_max = arr(hist["f_max"], np.float64).ctypes.data
        h.theta_max = arr(hist["theta_max"], np.float64).ctypes.data
        h.sampler = SAMPLERS[hist.get("sampler", "icdf")]
        h.axes = AXES[hist.get("axes", "linear")]
        if hist.get("p_edges") is not None:
            h.p_edges = arr(hist["p_edges"], np.float64).ctypes.data
        if h.axes == MT_AXES_LOG:
            h.f_min = arr(hist["f_min"], np.float64).ctypes.data
            h.theta_min = arr(hist["theta_min"], np.float64).ctypes.data
        return h


def mt_create(geometry: dict, field: dict, hist: dict) -> int:
    """Build a device-resident world on the current CUDA device; returns the handle (int)."""
    L = load_library()
    d = _Descs(geometry, field, hist)
    out = C.c_void_p()
    _check(L.mt_create(C.byref(d.g), C.byref(d.f), C.byref(d.h), C.byref(out)), "mt_create")
    return out.value


def mt_destroy(handle: Optional[int]) -> None:
    if handle:
        load_library().mt_destroy(C.c_void_p(handle))


def mt_device_bytes(handle: int) -> int:
    return load_library().mt_device_bytes(C.c_void_p(handle))


SOA_FIELDS = ("x", "y", "z", "px", "py", "pz", "q", "steps", "status")
SOA_DTYPES = dict(x="float32", y="float32", z="float32", px="float32", py="float32", pz="float32", q="int8",
                  steps="int32", status="uint8")


def soa_struct(muons: Dict, id_offset: int = 0, instance: int = 0) -> mt_muon_soa:
    """mt_muon_soa over torch CUDA tensors (contiguous, dtypes of mt.h)."""
    s = mt_muon_soa()
    for k in SOA_FIELDS:
        t = muons[k]
        if str(t.dtype).replace("torch.", "") != SOA_DTYPES[k]:
            raise TypeError(f"muon field {k}: dtype {t.dtype}, want {SOA_DTYPES[k]}")
        if not t.is_cuda or not t.is_contiguous():
            raise ValueError(f"muon field {k} must be a contiguous CUDA tensor")
        setattr(s, k, t.data_ptr())
    s.id_offset = int(id_offset)
    s.instance = int(instance)
    return s


def _stream_ptr(stream) -> int:
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return int(getattr(stream, "cuda_stream", stream))


def mt_transport(handle: int, muons: Dict, step_len: float, max_steps: int, seed: int, id_offset: int = 0,
                 instance: int = 0, stream=None, n: Optional[int] = None) -> None:
    """Transport the muons (dict of CUDA tensors, updated in place) on `stream`."""
    s = soa_struct(muons, id_offset, instance)
    n = int(muons["x"].numel()) if n is None else int(n)
    _check(load_library().mt_transport(C.c_void_p(handle), C.byref(s), n, float(step_len), int(max_steps),
                                       int(seed) & 0xFFFFFFFFFFFFFFFF, C.c_void_p(_stream_ptr(stream))),
           "mt_transport")


def mt_transport_scaled(handle: int, muons: Dict, step_len: float, max_steps: int, seed: int, alpha,
                        id_offset: int = 0, instance: int = 0, stream=None) -> None:
    """mt_transport with per-block field scales alpha (CUDA float32 tensor [n_block, 3] or None)."""
    s = soa_struct(muons, id_offset, instance)
    n = int(muons["x"].numel())
    if alpha is not None:
        if not alpha.is_cuda or str(alpha.dtype) != "torch.float32" or not alpha.is_contiguous():
            raise TypeError("alpha must be a contiguous float32 CUDA tensor")
        a_ptr, nb = alpha.data_ptr(), alpha.numel() // 3
    else:
        a_ptr, nb = None, 0
    _check(load_library().mt_transport_scaled(C.c_void_p(handle), C.byref(s), n, float(step_len), int(max_steps),
                                              int(seed) & 0xFFFFFFFFFFFFFFFF, C.c_void_p(a_ptr), int(nb),
                                              C.c_void_p(_stream_ptr(stream))), "mt_transport_scaled")


def mt_transport_workspace_bytes(n: int) -> int:
    return load_library().mt_transport_workspace_bytes(int(n))


def mt_transport_launches(handle: int, n: int, step_len: float, max_steps: int, mode: int = MT_LAUNCH_AUTO,
                          steps_per_pass: int = 0, order: int = MT_ORDER_AUTO) -> int:
    """Kernel launches of one mt_transport_cfg call with these arguments (-1: invalid)."""
    cfg = mt_launch_cfg(int(mode), 0, int(steps_per_pass), int(order), None, 0)
    return int(load_library().mt_transport_launches(C.c_void_p(handle), int(n), float(step_len), int(max_steps),
                                                    C.byref(cfg)))


def mt_transport_cfg(handle: int, muons: Dict, step_len: float, max_steps: int, seed: int, alpha=None,
                     mode: int = MT_LAUNCH_AUTO, blocks_per_sm: int = 0, id_offset: int = 0, instance: int = 0,
                     stream=None, steps_per_pass: int = 0, workspace=None, order: int = MT_ORDER_AUTO) -> None:
    """mt_transport with field scales (or None) and an explicit launch shape."""
    s = soa_struct(muons, id_offset, instance)
    n = int(muons["x"].numel())
    if alpha is not None:
        if not alpha.is_cuda or str(alpha.dtype) != "torch.float32" or not alpha.is_contiguous():
            raise TypeError("alpha must be a contiguous float32 CUDA tensor")
        a_ptr, nb = alpha.data_ptr(), alpha.numel() // 3
    else:
        a_ptr, nb = None, 0
    ws_ptr, ws_bytes = (None, 0) if workspace is None else (workspace.data_ptr(),
                                                           workspace.numel() * workspace.element_size())
    cfg = mt_launch_cfg(int(mode), int(blocks_per_sm), int(steps_per_pass), int(order), ws_ptr, int(ws_bytes))
    _check(load_library().mt_transport_cfg(C.c_void_p(handle), C.byref(s), n, float(step_len), int(max_steps),
                                           int(seed) & 0xFFFFFFFFFFFFFFFF, C.c_void_p(a_ptr), int(nb), C.byref(cfg),
                                           C.c_void_p(_stream_ptr(stream))), "mt_transport_cfg")


def mt_transport_noalloc(handle: int, muons: Dict, step_len: float, max_steps: int, seed: int, id_offset: int = 0,
                         instance: int = 0, stream=None) -> None:
    """mt_transport without any device allocation (scratch in the library's fixed device array;
    at most MT_NOALLOC_MAX_MUONS muons per call; calls on one device must not overlap)."""
    s = soa_struct(muons, id_offset, instance)
    n = int(muons["x"].numel())
    _check(load_library().mt_transport_noalloc(C.c_void_p(handle), C.byref(s), n, float(step_len), int(max_steps),
                                               int(seed) & 0xFFFFFFFFFFFFFFFF, C.c_void_p(_stream_ptr(stream))),
           "mt_transport_noalloc")


# --------------------------------------------------------------------------
# differentiable form
# --------------------------------------------------------------------------
def _alpha_ptr(alpha):
    if alpha is None:
        return None, 0
    if not alpha.is_cuda or str(alpha.dtype) != "torch.float32" or not alpha.is_contiguous():
        raise TypeError("alpha must be a contiguous float32 CUDA tensor [n_block, 3]")
    return alpha.data_ptr(), alpha.numel() // 3


def _f32_dev(t, what):
    if t is None:
        return None
    if not t.is_cuda or str(t.dtype) != "torch.float32" or not t.is_contiguous():
        raise TypeError(f"{what} must be a contiguous float32 CUDA tensor")
    return t.data_ptr()


def mt_ckpt_bytes(n: int, max_steps: int, ckpt_every: int) -> int:
    return load_library().mt_ckpt_bytes(int(n), int(max_steps), int(ckpt_every))


def mt_transport_ckpt(handle: int, muons: Dict, step_len: float, max_steps: int, seed: int, alpha, ckpt_every: int,
                      ckpt, id_offset: int = 0, instance: int = 0, stream=None) -> None:
    """Checkpointing forward: transport in place, keeping every K-step live list in `ckpt` (uint8 CUDA tensor)."""
    s = soa_struct(muons, id_offset, instance)
    a_ptr, nb = _alpha_ptr(alpha)
    _check(load_library().mt_transport_ckpt(C.c_void_p(handle), C.byref(s), int(muons["x"].numel()), float(step_len),
                                            int(max_steps), int(seed) & 0xFFFFFFFFFFFFFFFF, C.c_void_p(a_ptr),
                                            int(nb), int(ckpt_every), C.c_void_p(ckpt.data_ptr()),
                                            int(ckpt.numel() * ckpt.element_size()),
                                            C.c_void_p(_stream_ptr(stream))), "mt_transport_ckpt")


def mt_adjoint_ckpt(handle: int, n: int, step_len: float, max_steps: int, seed: int, alpha, ckpt_every: int, ckpt,
                    dL_dfinal, dL_dalpha, dL_dinitial=None, id_offset: int = 0, instance: int = 0,
                    stream=None) -> None:
    """Backward from the checkpoints: dL/dalpha (and optionally dL/d initial state) from dL/d final state [6, n]."""
    a_ptr, nb = _alpha_ptr(alpha)
    _check(load_library().mt_adjoint_ckpt(C.c_void_p(handle), int(n), float(step_len), int(max_steps),
                                          int(seed) & 0xFFFFFFFFFFFFFFFF, C.c_void_p(a_ptr), int(nb),
                                          int(ckpt_every), C.c_void_p(ckpt.data_ptr()),
                                          int(ckpt.numel() * ckpt.element_size()), int(id_offset), int(instance),
                                          C.c_void_p(_f32_dev(dL_dfinal, "dL_dfinal")),
                                          C.c_void_p(_f32_dev(dL_dinitial, "dL_dinitial")),
                                          C.c_void_p(_f32_dev(dL_dalpha, "dL_dalpha")),
                                          C.c_void_p(_stream_ptr(stream))), "mt_adjoint_ckpt")


def mt_transport_adjoint(handle: int, muons0: Dict, step_len: float, max_steps: int, seed: int, alpha, dL_dfinal,
                         dL_dalpha, ckpt_every: int = 32, id_offset: int = 0, instance: int = 0, stream=None) -> None:
    """dL/dalpha from the INITIAL muons (left unchanged) and dL/d final state, in one call."""
    s = soa_struct(muons0, id_offset, instance)
    a_ptr, nb = _alpha_ptr(alpha)
    _check(load_library().mt_transport_adjoint(C.c_void_p(handle), C.byref(s), int(muons0["x"].numel()),
                                               float(step_len), int(max_steps), int(seed) & 0xFFFFFFFFFFFFFFFF,
                                               C.c_void_p(a_ptr), int(nb), C.c_void_p(_f32_dev(dL_dfinal, "dL_dfinal")),
                                               C.c_void_p(_f32_dev(dL_dalpha, "dL_dalpha")), int(ckpt_every),
                                               C.c_void_p(_stream_ptr(stream))), "mt_transport_adjoint")


def mt_tape_bytes(n: int, max_steps: int, steps_per_pass: int) -> int:
    return load_library().mt_tape_bytes(int(n), int(max_steps), int(steps_per_pass))


def mt_transport_tape(handle: int, muons: Dict, step_len: float, max_steps: int, seed: int, alpha,
                      steps_per_pass: int, tape, id_offset: int = 0, instance: int = 0, stream=None) -> None:
    """Forward recording every step into `tape` (uint8 CUDA tensor of mt_tape_bytes bytes)."""
    s = soa_struct(muons, id_offset, instance)
    a_ptr, nb = _alpha_ptr(alpha)
    _check(load_library().mt_transport_tape(C.c_void_p(handle), C.byref(s), int(muons["x"].numel()), float(step_len),
                                            int(max_steps), int(seed) & 0xFFFFFFFFFFFFFFFF, C.c_void_p(a_ptr),
                                            int(nb), int(steps_per_pass), C.c_void_p(tape.data_ptr()),
                                            int(tape.numel() * tape.element_size()),
                                            C.c_void_p(_stream_ptr(stream))), "mt_transport_tape")


def mt_adjoint_tape(handle: int, n: int, step_len: float, max_steps: int, alpha, steps_per_pass: int, tape,
                    dL_dfinal, dL_dalpha, dL_dinitial=None, stream=None) -> None:
    """Backward from the tape of one mt_transport_tape call."""
    a_ptr, nb = _alpha_ptr(alpha)
    _check(load_library().mt_adjoint_tape(C.c_void_p(handle), int(n), float(step_len), int(max_steps),
                                          C.c_void_p(a_ptr), int(nb), int(steps_per_pass), C.c_void_p(tape.data_ptr()),
                                          int(tape.numel() * tape.element_size()),
                                          C.c_void_p(_f32_dev(dL_dfinal, "dL_dfinal")),
                                          C.c_void_p(_f32_dev(dL_dinitial, "dL_dinitial")),
                                          C.c_void_p(_f32_dev(dL_dalpha, "dL_dalpha")),
                                          C.c_void_p(_stream_ptr(stream))), "mt_adjoint_tape")


def mt_acceptance_loss(muons: Dict, loss, dL_dfinal=None, z_plane: float = 30.0, half_width: float = 0.5,
                       edge: float = 0.01, stream=None) -> None:
    """Acceptance loss of final states into `loss` (float64 CUDA tensor [1]); dL/d final state into dL_dfinal."""
    s = mt_muon_soa()
    for k in ("x", "y", "z", "px", "py", "pz", "status"):
        setattr(s, k, muons[k].data_ptr())
    if not loss.is_cuda or str(loss.dtype) != "torch.float64":
        raise TypeError("loss must be a float64 CUDA tensor")
    _check(load_library().mt_acceptance_loss(C.byref(s), int(muons["x"].numel()), float(z_plane), float(half_width),
                                             float(edge), C.c_void_p(loss.data_ptr()),
                                             C.c_void_p(_f32_dev(dL_dfinal, "dL_dfinal")),
                                             C.c_void_p(_stream_ptr(stream))), "mt_acceptance_loss")


# --------------------------------------------------------------------------
# batched form
# --------------------------------------------------------------------------
def mt_batch_create(hist: dict, n_inst: int) -> int:
    """A batch of n_inst worlds sharing the histogram set `hist`; returns the batch pointer (int)."""
    L = load_library()
    d = _Descs(None, None, hist)
    out = C.c_void_p()
    _check(L.mt_batch_create(C.byref(d.h), int(n_inst), C.byref(out)), "mt_batch_create")
    return out.value


def mt_batch_set_instance(batch: int, i: int, geometry: dict, field: dict) -> None:
    d = _Descs(geometry, field, None)
    _check(load_library().mt_batch_set_instance(C.c_void_p(batch), int(i), C.byref(d.g), C.byref(d.f)),
           "mt_batch_set_instance")


def mt_batch_destroy(batch: Optional[int]) -> None:
    if batch:
        load_library().mt_batch_destroy(C.c_void_p(batch))


def mt_batch_device_bytes(batch: int) -> int:
    return load_library().mt_batch_device_bytes(C.c_void_p(batch))


def _counts(counts):
    a = (C.c_int64 * max(1, len(counts)))()
    for i, c in enumerate(counts):
        a[i] = int(c)
    return a


def mt_batch_workspace_bytes(batch: int, counts) -> int:
    return load_library().mt_batch_workspace_bytes(C.c_void_p(batch), _counts(counts))


def _soas(muons_list, id_offsets, instances):
    arr = (mt_muon_soa * max(1, len(muons_list)))()
    n = []
    for i, m in enumerate(muons_list):
        arr[i] = soa_struct(m, 0 if id_offsets is None else id_offsets[i], i if instances is None else instances[i])
        n.append(int(m["x"].numel()))
    return arr, _counts(n)


def mt_transport_batched(batch: int, muons_list, step_len: float, max_steps: int, seed: int, block: int = 0,
                         steps_per_pass: int = 0, use_graph: bool = False, workspace=None, id_offsets=None,
                         instances=None, stream=None, staging: int = 0, order: int = MT_ORDER_AUTO) -> None:
    """Transport instance i's muons (dict of CUDA tensors, in place) in world i, for every i.
    Muon ids are id_offsets[i] + m (default 0) and the Philox instance word is instances[i] (default i).
    staging: MT_BATCH_STAGE_SHARED or MT_BATCH_STAGE_GLOBAL (0: the tuned one, else shared).
    order: spatial order of the live lists (MT_ORDER_AUTO, _ALWAYS or _NEVER; results do not change)."""
    soas, n = _soas(muons_list, id_offsets, instances)
    ws_ptr, ws_bytes = (None, 0) if workspace is None else (workspace.data_ptr(),
                                                           workspace.numel() * workspace.element_size())
    cfg = mt_batch_cfg(int(block), int(steps_per_pass), int(bool(use_graph)), int(staging), int(order), 0, ws_ptr,
                       int(ws_bytes))
    _check(load_library().mt_transport_batched(C.c_void_p(batch), soas, n, float(step_len), int(max_steps),
                                               int(seed) & 0xFFFFFFFFFFFFFFFF, C.byref(cfg),
                                               C.c_void_p(_stream_ptr(stream))), "mt_transport_batched")


def mt_batch_autotune(batch: int, muons_list, step_len: float, max_steps: int, seed: int,
                      sample_per_instance: int = 4096, id_offsets=None, instances=None, stream=None):
    """Time the launch shapes on a sample of every instance's muons (left unchanged); returns
    (block, steps_per_pass, staging), which the batch also keeps as its defaults."""
    soas, n = _soas(muons_list, id_offsets, instances)
    best = mt_batch_cfg()
    _check(load_library().mt_batch_autotune(C.c_void_p(batch), soas, n, float(step_len), int(max_steps),
                                            int(seed) & 0xFFFFFFFFFFFFFFFF, int(sample_per_instance),
                                            C.byref(best), C.c_void_p(_stream_ptr(stream))), "mt_batch_autotune")
    return int(best.block), int(best.steps_per_pass), int(best.staging)


# --------------------------------------------------------------------------
# offline phase
# --------------------------------------------------------------------------
def _materials(materials):
    arr = (mt_material * len(materials))()
    for i, m in enumerate(materials):
        arr[i] = mt_material(float(m["rho"]), float(m["ZA"]), float(m["I"]), float(m["X0"]), float(m["b"]))
    return arr


def mt_build_histograms(materials, edges, nf: int, ntheta: int, f_max: float, step_len: float, n_samples: int,
                        seed: int, weights, stream=None):
    """Histograms of the parametric sampler into `weights` (float64 CUDA tensor [n_mat][n_pbin][nf][ntheta]);
    returns theta_max [n_mat][n_pbin] (numpy)."""
    e = np.ascontiguousarray(edges, dtype=np.float64)
    n_pbin = len(e) - 1
    if not weights.is_cuda or str(weights.dtype) != "torch.float64" or not weights.is_contiguous() or \
            weights.numel() != len(materials) * n_pbin * nf * ntheta:
        raise TypeError("weights must be a contiguous float64 CUDA tensor [n_mat][n_pbin][nf][ntheta]")
    tmax = np.zeros((len(materials), n_pbin))
    _check(load_library().mt_build_histograms(_materials(materials), len(materials), n_pbin, e.ctypes.data, int(nf),
                                              int(ntheta), float(f_max), float(step_len), int(n_samples),
                                              int(seed) & 0xFFFFFFFFFFFFFFFF, C.c_void_p(weights.data_ptr()),
                                              tmax.ctypes.data, C.c_void_p(_stream_ptr(stream))),
           "mt_build_histograms")
    return tmax


def mt_pilot_phi(material, probes, K: int, step_len: float, seed: int, stream=None) -> np.ndarray:
    pr = np.ascontiguousarray(probes, dtype=np.float64)
    phi = np.zeros(len(pr))
    _check(load_library().mt_pilot_phi(_materials([material]), pr.ctypes.data, len(pr), int(K), float(step_len),
                                       int(seed) & 0xFFFFFFFFFFFFFFFF, phi.ctypes.data,
                                       C.c_void_p(_stream_ptr(stream))), "mt_pilot_phi")
    return phi


def mt_bv_edges(probes, phi, eps: float) -> np.ndarray:
    pr = np.ascontiguousarray(probes, dtype=np.float64)
    ph = np.ascontiguousarray(phi, dtype=np.float64)
    out = np.zeros(len(pr))
    n = load_library().mt_bv_edges(pr.ctypes.data, ph.ctypes.data, len(pr), float(eps), out.ctypes.data, len(pr))
    if n < 0:
        raise MtError(MT_ERR_INVALID_ARG, "mt_bv_edges", mt_last_error())
    return out[:n].copy()
