"""Owning wrappers around the binding: a World (one mt_handle) and SoA transfers."""
from __future__ import annotations

from typing import Dict, Optional

import numpy as np

from . import _binding as B


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
                  blocks_per_sm: int = 0, steps_per_pass: int = 0, workspace=None) -> None:
        if mode is not None or blocks_per_sm or steps_per_pass or workspace is not None:
            B.mt_transport_cfg(self.handle, muons, step_len, max_steps, seed, alpha, mode or 0, blocks_per_sm,
                               id_offset, instance, stream, steps_per_pass, workspace)
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

    def set_instance(self, i: int, geometry: dict, field: dict) -> None:
        B.mt_batch_set_instance(self.handle, i, geometry, field)

    @property
    def device_bytes(self) -> int:
        return B.mt_batch_device_bytes(self.handle)

    def workspace_bytes(self, counts) -> int:
        return B.mt_batch_workspace_bytes(self.handle, counts)

    def transport(self, muons_list, step_len: float, max_steps: int, seed: int, **kw) -> None:
        B.mt_transport_batched(self.handle, muons_list, step_len, max_steps, seed, **kw)

    def autotune(self, muons_list, step_len: float, max_steps: int, seed: int, sample_per_instance: int = 4096,
                 **kw):
        return B.mt_batch_autotune(self.handle, muons_list, step_len, max_steps, seed, sample_per_instance, **kw)

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
