"""torch.autograd wrappers of the differentiable form.  Every forward and
backward computation runs in libmt's kernels (checkpointing transport, acceptance
loss, hand-written adjoint); these classes only hand tensors to the C ABI."""
from __future__ import annotations

from typing import Dict, Optional

from . import _binding as B

_FIELDS = ("x", "y", "z", "px", "py", "pz")


class MuonTransportFn:
    """Final (x, y, z, px, py, pz, steps, status) of a muon batch as a differentiable
    function of the per-block field scales alpha [n_block, 3] (pathwise gradient,
    draws held fixed).  Use through ``transport_differentiable``."""

    @staticmethod
    def _make():
        import torch

        class _Fn(torch.autograd.Function):
            @staticmethod
            def forward(ctx, alpha, world, muons, step_len, max_steps, seed, ckpt_every, id_offset, instance, tape):
                n = int(muons["x"].numel())
                work = {k: v.clone() for k, v in muons.items()}
                a = alpha.detach().contiguous()
                if tape == "auto":
                    free, _ = torch.cuda.mem_get_info(alpha.device)
                    tape = B.mt_tape_bytes(n, max_steps, ckpt_every) <= free // 2
                if tape:
                    buf = torch.empty(max(1, B.mt_tape_bytes(n, max_steps, ckpt_every)), dtype=torch.uint8,
                                      device=alpha.device)
                    B.mt_transport_tape(world.handle, work, step_len, max_steps, seed, a, ckpt_every, buf, id_offset,
                                        instance)
                else:
                    buf = torch.empty(max(1, B.mt_ckpt_bytes(n, max_steps, ckpt_every)), dtype=torch.uint8,
                                      device=alpha.device)
                    B.mt_transport_ckpt(world.handle, work, step_len, max_steps, seed, a, ckpt_every, buf, id_offset,
                                        instance)
                ctx.save_for_backward(a)
                ctx.ckpt = buf
                ctx.tape = bool(tape)
                ctx.world = world
                ctx.args = (n, step_len, max_steps, seed, ckpt_every, id_offset, instance)
                ctx.mark_non_differentiable(work["steps"], work["status"])
                return tuple(work[k] for k in _FIELDS) + (work["steps"], work["status"])

            @staticmethod
            def backward(ctx, gx, gy, gz, gpx, gpy, gpz, _gs, _gst):
                (a,) = ctx.saved_tensors
                n, step_len, max_steps, seed, ckpt_every, id_offset, instance = ctx.args
                grads = [g if g is not None else torch.zeros(n, dtype=torch.float32, device=a.device)
                         for g in (gx, gy, gz, gpx, gpy, gpz)]
                g6 = torch.stack([g.float() for g in grads]).contiguous()
                dalpha = torch.empty_like(a)
                if ctx.tape:
                    B.mt_adjoint_tape(ctx.world.handle, n, step_len, max_steps, a, ckpt_every, ctx.ckpt, g6, dalpha)
                else:
                    B.mt_adjoint_ckpt(ctx.world.handle, n, step_len, max_steps, seed, a, ckpt_every, ctx.ckpt, g6,
                                      dalpha, id_offset=id_offset, instance=instance)
                return dalpha, None, None, None, None, None, None, None, None, None

        return _Fn

    _fn = None

    @classmethod
    def apply(cls, *args):
        if cls._fn is None:
            cls._fn = cls._make()
        return cls._fn.apply(*args)


class AcceptanceLossFn:
    """Mean acceptance loss of final states (sigmoid window at z = 30 m) with its
    gradient computed by the same kernel."""

    @staticmethod
    def _make():
        import torch

        class _Fn(torch.autograd.Function):
            @staticmethod
            def forward(ctx, x, y, z, px, py, pz, status, z_plane, half_width, edge):
                n = int(x.numel())
                loss = torch.zeros(1, dtype=torch.float64, device=x.device)
                g = torch.empty((6, n), dtype=torch.float32, device=x.device)
                B.mt_acceptance_loss(dict(x=x, y=y, z=z, px=px, py=py, pz=pz, status=status), loss, g, z_plane,
                                     half_width, edge)
                ctx.save_for_backward(g)
                return loss[0]

            @staticmethod
            def backward(ctx, gl):
                (g,) = ctx.saved_tensors
                s = gl.to(torch.float32)
                return (g[0] * s, g[1] * s, g[2] * s, g[3] * s, g[4] * s, g[5] * s, None, None, None, None)

        return _Fn

    _fn = None

    @classmethod
    def apply(cls, *args):
        if cls._fn is None:
            cls._fn = cls._make()
        return cls._fn.apply(*args)


def transport_differentiable(world, muons: Dict, alpha, step_len: float, max_steps: int, seed: int,
                             ckpt_every: int = 32, id_offset: int = 0, instance: int = 0, tape=False) -> Dict:
    """Differentiable transport: returns the final state dict; x..pz carry grad to alpha.

    tape: False (default) keeps a checkpoint every ckpt_every steps, and the
    backward recomputes each segment for the muons whose cotangent is not zero
    only; True records every step of every muon in the forward (56 B per
    muon-step of device memory) and the backward only walks the record; "auto"
    takes the tape when it needs at most half of the free device memory.  With
    the acceptance loss, whose cotangent is zero for most muons of a shield, the
    checkpoint form is the faster (10^6 muons on a GB300: forward + backward 1.5x
    the plain transport, against 2.0x with the tape); with a cotangent on every
    muon the tape form is (2.8x, against 4.0x)."""
    out = MuonTransportFn.apply(alpha, world, muons, step_len, max_steps, seed, ckpt_every, id_offset, instance,
                                tape)
    return dict(zip(_FIELDS + ("steps", "status"), out))


def acceptance_loss(final: Dict, z_plane: float = 30.0, half_width: float = 0.5, edge: float = 0.01):
    return AcceptanceLossFn.apply(final["x"], final["y"], final["z"], final["px"], final["py"], final["pz"],
                                  final["status"], z_plane, half_width, edge)
