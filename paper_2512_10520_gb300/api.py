"""Owning wrappers around the binding: a World (one mt_handle) and SoA transfers."""
from __future__ import annotations

import hashlib
import json
import os
import threading
from typing import Dict, Optional

import numpy as np

from . import _binding as B

# autotune results, one JSON file keyed by (workload fingerprint, GPU name)
_TUNE_CACHE = os.environ.get("MT_AUTOTUNE_CACHE",
                             os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "_build",
                                          "autotune.json"))
_tune_lock = threading.Lock()


def source_digest() -> str:
    """Hash of the library's sources, headers and target architecture: a tuned
    launch shape cached for one build is not reused by another."""
    from . import _build
    h = hashlib.sha1(" ".join(_build.ARCH).encode())
    files = sorted(os.path.join(_build.CSRC, f) for f in os.listdir(_build.CSRC) if f.endswith((".cu", ".cuh", ".h")))
    files += sorted(os.path.join(_build.INCLUDE, f) for f in os.listdir(_build.INCLUDE) if f.endswith(".h"))
    for f in files:
        h.update(os.path.basename(f).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _fingerprint(h, obj) -> None:
    """Feed a descriptor dict (numbers, strings, arrays) into hash h: scalars and
    shapes exactly, large arrays through a strided sample plus their sums."""
    if isinstance(obj, dict):
        for k in sorted(obj):
            h.update(str(k).encode())
            _fingerprint(h, obj[k])
    elif isinstance(obj, (list, tuple)):
        for v in obj:
            _fingerprint(h, v)
    elif isinstance(obj, np.ndarray):
        a = np.ascontiguousarray(obj)
        h.update(f"{a.dtype}{a.shape}".encode())
        flat = a.reshape(-1)
        step = max(1, flat.size // 4096)
        h.update(np.ascontiguousarray(flat[::step]).tobytes())
        if a.dtype.kind in "fiu" and flat.size:
            h.update(np.float64(flat.sum(dtype=np.float64)).tobytes())
    else:
        h.update(repr(obj).encode())


class World:
    """A device-resident world (geometry, field map, sampling tables) = one mt_handle."""

    def __init__(self, geometry: dict, field: dict, hist: dict):
        self.handle = B.mt_create(geometry, field, hist)

    @classmethod
    def from_workload(cls, wl) -> "World":
        return cls(wl.geometry, wl.field, wl.hist)

    @property
    def device_bytes(self) -> int:
        return B.mt_device_bytes(self.handle)

    def transport(self, muons: Dict, step_len: float, max_steps: int, seed: int, id_offset: int = 0,
                  instance: int = 0, alpha=None, stream=None, mode: Optional[int] = None,
                  blocks_per_sm: int = 0, steps_per_pass: int = 0, workspace=None, order: int = 0) -> None:
        if mode is not None or blocks_per_sm or steps_per_pass or workspace is not None or order:
            B.mt_transport_cfg(self.handle, muons, step_len, max_steps, seed, alpha, mode or 0, blocks_per_sm,
                               id_offset, instance, stream, steps_per_pass, workspace, order)
        elif alpha is None:
            B.mt_transport(self.handle, muons, step_len, max_steps, seed, id_offset, instance, stream)
        else:
            B.mt_transport_scaled(self.handle, muons, step_len, max_steps, seed, alpha, id_offset, instance,
                                  stream)

    def close(self) -> None:
        if getattr(self, "handle", None):
            B.mt_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many worlds sharing one histogram set (one mt_batch), transported together."""

    def __init__(self, hist: dict, n_inst: int):
        self.handle = B.mt_batch_create(hist, n_inst)
        self.n_inst = int(n_inst)
        self._tables = hashlib.sha1()
        _fingerprint(self._tables, hist)
        self._worlds = [b""] * self.n_inst
        self.tuned = None

    def set_instance(self, i: int, geometry: dict, field: dict) -> None:
        B.mt_batch_set_instance(self.handle, i, geometry, field)
        h = hashlib.sha1()
        _fingerprint(h, geometry)
        _fingerprint(h, field)
        self._worlds[i] = h.digest()

    @property
    def device_bytes(self) -> int:
        return B.mt_batch_device_bytes(self.handle)

    def workspace_bytes(self, counts) -> int:
        return B.mt_batch_workspace_bytes(self.handle, counts)

    def transport(self, muons_list, step_len: float, max_steps: int, seed: int, **kw) -> None:
        if self.tuned is not None:
            for k, v in zip(("block", "steps_per_pass", "staging"), self.tuned):
                if not kw.get(k):
                    kw[k] = v
        B.mt_transport_batched(self.handle, muons_list, step_len, max_steps, seed, **kw)

    def autotune(self, muons_list, step_len: float, max_steps: int, seed: int, sample_per_instance: int = 4096,
                 cache: bool = True, **kw):
        """(block, steps_per_pass, staging) fastest on a sample of every instance
        (mt_batch_autotune); later transports use it unless told otherwise.  With
        cache, the result is kept in a JSON file keyed by a fingerprint of the
        worlds, tables, muon counts, run arguments and library sources and by the
        GPU's name, and a later call with the same key reuses it without timing
        anything."""
        key = None
        if cache:
            import torch
            h = hashlib.sha1(self._tables.digest())
            for w in self._worlds:
                h.update(w)
            counts = [int(m["x"].numel()) if hasattr(m["x"], "numel") else len(m["x"]) for m in muons_list]
            h.update(json.dumps([counts, float(step_len), int(max_steps), int(seed), int(sample_per_instance),
                                 B.mt_abi_version(), source_digest()]).encode())
            key = f"{h.hexdigest()[:24]}|{torch.cuda.get_device_name()}"
            with _tune_lock:
                try:
                    with open(_TUNE_CACHE) as fh:
                        hit = json.load(fh).get(key)
                except (OSError, ValueError):
                    hit = None
            if hit:
                self.tuned = tuple(int(v) for v in hit)
                return self.tuned
        self.tuned = B.mt_batch_autotune(self.handle, muons_list, step_len, max_steps, seed, sample_per_instance,
                                         **kw)
        if key is not None:
            with _tune_lock:
                try:
                    with open(_TUNE_CACHE) as fh:
                        table = json.load(fh)
                except (OSError, ValueError):
                    table = {}
                table[key] = list(self.tuned)
                os.makedirs(os.path.dirname(_TUNE_CACHE), exist_ok=True)
                tmp = f"{_TUNE_CACHE}.tmp{os.getpid()}"
                with open(tmp, "w") as fh:
                    json.dump(table, fh, indent=1, sort_keys=True)
                os.replace(tmp, _TUNE_CACHE)
        return self.tuned

    def close(self) -> None:
        if getattr(self, "handle", None):
            B.mt_batch_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def build_histogram_set(materials, p_lo: float = 1.0, p_hi: float = 400.0, n_pbin: int = 64, edges=None,
                        nf: int = 128, ntheta: int = 64, f_max: float = 0.2, step_len: float = 0.02,
                        n_samples: int = 10**6, seed: int = 42, material_table=None, stream=None) -> dict:
    """A histogram set (the dict mt_create takes) built on the GPU by the parametric
    sampler (mt_build_histograms): log10 bins on [p_lo, p_hi], or the given edges
    (e.g. bounded-variation edges), which the transport then searches."""
    import torch
    if material_table is None:
        from workloads import MATERIALS as material_table
    mats = [material_table[m] if isinstance(m, str) else m for m in materials]
    if edges is None:
        k = np.arange(n_pbin + 1, dtype=np.float64)
        e = p_lo * (p_hi / p_lo) ** (k / n_pbin)
        custom = None
    else:
        e = np.ascontiguousarray(edges, dtype=np.float64)
        n_pbin, p_lo, p_hi = len(e) - 1, float(e[0]), float(e[-1])
        custom = e
    w = torch.empty((len(mats), n_pbin, nf, ntheta), dtype=torch.float64, device="cuda")
    tmax = B.mt_build_histograms(mats, e, nf, ntheta, f_max, step_len, n_samples, seed, w, stream)
    out = dict(n_mat=len(mats), n_pbin=n_pbin, p_lo=float(p_lo), p_hi=float(p_hi), nf=nf, ntheta=ntheta,
               weights=w.cpu().numpy(), f_max=np.full((len(mats), n_pbin), float(f_max)), theta_max=tmax)
    if custom is not None:
        out["p_edges"] = custom
    return out


def bounded_variation_edges(material, p_lo: float, p_hi: float, eps: float, n_probe: int = 1024,
                            K: int = 100000, step_len: float = 0.02, seed: int = 7, material_table=None):
    """Appendix A: pilot estimator on n_probe log-spaced probes (mt_pilot_phi),
    then the bounded-variation edges with tolerance eps (mt_bv_edges)."""
    if material_table is None:
        from workloads import MATERIALS as material_table
    m = material_table[material] if isinstance(material, str) else material
    probes = np.geomspace(p_lo, p_hi, n_probe)
    phi = B.mt_pilot_phi(m, probes, K, step_len, seed)
    return B.mt_bv_edges(probes, phi, eps), probes, phi


def muons_to_device(soa: Dict[str, np.ndarray], device="cuda", pin: bool = False) -> Dict:
    """Copy a numpy SoA (fields of mt_muon_soa) to CUDA tensors."""
    import torch
    out = {}
    for k in B.SOA_FIELDS:
        t = torch.from_numpy(np.ascontiguousarray(soa[k], dtype=B.SOA_DTYPES[k]))
        out[k] = t.to(device, non_blocking=pin)
    return out


def muons_to_host(dev: Dict) -> Dict[str, np.ndarray]:
    return {k: dev[k].cpu().numpy() for k in B.SOA_FIELDS}


def empty_like_soa(n: int, device="cuda", pinned: bool = False) -> Dict:
    import torch
    out = {}
    for k in B.SOA_FIELDS:
        dt = getattr(torch, B.SOA_DTYPES[k])
        if device == "cpu":
            out[k] = torch.empty(n, dtype=dt, pin_memory=pinned)
        else:
            out[k] = torch.empty(n, dtype=dt, device=device)
    return out
