"""Benchmark: muon-steps/s of the histogram-sampling muon transport on one GB300.

A "step" of this benchmark is one full transport of one batch: 1e6 muons of the
p^-2.7 spectrum through the six-magnet shield and concrete wall (trilinear
200x200x600 FP32 field map, 3 materials x 64 log bins x 128x64 histograms,
2 cm steps, at most 1500 steps per muon), i.e. every muon runs Algorithm 1
until it stops, exits or uses its 1500 steps.  The throughput is
muon-steps/s = (sum of steps taken by all muons) / time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mine|reference]

Prints one JSON line (rank 0).  Under torchrun each rank transports its own 1e6
muons (ids offset by rank, no collective on the data path: weak scaling) and the
time is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "muon-steps/s on 1 GB300: plain, batched, fwd+adjoint; % of memory roofline"
UNIT = "muon-steps/s"
BYTES_PER_STEP = 112          # algorithmic bytes per muon-step (8 field corners x 12 B + 16 B sampler)
WORKLOAD = ("shield1e6: 1e6 muons (p^-2.7 on 10-350 GeV, p_T ~ Exp(1 GeV)), 6 iron magnet blocks "
            "+/-1.7 T + 2 m concrete wall, trilinear 200x200x600 FP32 field map, 3 materials x 64 log10 "
            "p-bins x 128x64 (f, theta) histograms, d = 2 cm, max 1500 steps")


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# the sources of the plain transport's kernels (compact_init, compact_pass, sort_scan,
# sort_scatter), of the world's device layout (api.cu) and their build flags
_TRANSPORT_SOURCES = ("paper_2512_10520_gb300/csrc/step.cuh", "paper_2512_10520_gb300/csrc/compact.cuh",
                      "paper_2512_10520_gb300/csrc/compact.cu", "paper_2512_10520_gb300/csrc/transport.cu",
                      "paper_2512_10520_gb300/csrc/mt_internal.cuh", "paper_2512_10520_gb300/csrc/api.cu",
                      "include/mt.h", "paper_2512_10520_gb300/_build.py")


def _csrc_hash() -> str:
    """Hash of the plain transport's kernel sources: the committed DRAM traffic is
    used only while it matches."""
    h = hashlib.sha1()
    for f in _TRANSPORT_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(f.encode())
            h.update(fh.read())
    return h.hexdigest()[:12]


def _profile_entry(kernel: str) -> dict:
    """The committed ncu figures of a kernel (profiles/traffic.json), if they were
    taken on this source; else an empty dict."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            t = json.load(fh)
        e = t.get(kernel)
        if e and e.get("csrc_hash") == _csrc_hash():
            return e
    except Exception:
        pass
    return {}


def _traffic(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, if it matches this source."""
    return _profile_entry(kernel).get("dram_bytes_per_launch")


def issue_roofline(kernel: str, muon_steps_per_s: float, sm_mhz, sms: int):
    """Instruction-issue ("alu") view of a transport kernel: warp instructions per
    muon-step (from the committed ncu capture of this source) times the measured
    muon-steps/s, against the issue peak of 4 warp instructions per cycle per SM
    (one per SM sub-partition) x the SMs the device reports x the SM clock
    sampled during the timed region."""
    e = _profile_entry(kernel)
    wips = e.get("warp_inst_per_step")
    if not wips or not sm_mhz or not sms:
        return {"bound": "alu", "achieved": None, "peak": None, "unit": "warp-instructions/s", "frac": None,
                "warp_inst_per_step": wips, "sms": sms, "sm_mhz": sm_mhz,
                "note": "no ncu capture of this source" if not wips else "no clock sample"}
    achieved = wips * muon_steps_per_s
    peak = sms * 4 * sm_mhz * 1e6
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "warp-instructions/s",
            "frac": achieved / peak, "warp_inst_per_step": wips, "sms": sms, "sm_mhz": sm_mhz,
            "source": e.get("summary")}


class ClockSampler:
    """nvidia-smi clock/throttle sampling while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.rows = []
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def summary(self):
        rows = getattr(self, "rows", [])
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max((num(r[3]) or 0.0) for r in rows)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _barrier_max(value: float, ws: int, device=None) -> float:
    if ws == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _barrier_sum(value: float, ws: int, device=None) -> float:
    if ws == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def cpu_oracle_run(wl, n_sample: int, threads: int):
    """Time the FP64 oracle on the first n_sample muons (ids 0..n_sample-1)."""
    import oracle
    world = oracle.world_of(wl)
    mu = {k: v[:n_sample] for k, v in wl.muons.items()}
    t0 = time.perf_counter()
    out = oracle.transport(world, mu, wl.step_len, wl.max_steps, wl.seed, n_threads=threads)
    dt = time.perf_counter() - t0
    return float(out["steps"].sum()), dt


def time_adjoint_form(mt, world, wl, init, work, stream, id_offset, reps=3, K=32, tape=True):
    """fwd+adjoint form (diff1e6: shield1e6 geometry, 18 field scales, checkpoints every K
    steps): checkpointing forward + acceptance loss + adjoint, each timed with CUDA events."""
    import torch
    n = wl.n
    alpha = torch.ones((6, 3), dtype=torch.float32, device=init["x"].device)
    ckpt = torch.empty(mt.mt_ckpt_bytes(n, wl.max_steps, K), dtype=torch.uint8, device=init["x"].device)
    loss = torch.zeros(1, dtype=torch.float64, device=init["x"].device)
    g = torch.empty((6, n), dtype=torch.float32, device=init["x"].device)
    da = torch.empty_like(alpha)
    times = []
    with torch.cuda.stream(stream):
        for r in range(reps + 1):
            for k in work:
                work[k].copy_(init[k], non_blocking=True)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            ev[0].record(stream)
            mt.mt_transport_ckpt(world.handle, work, wl.step_len, wl.max_steps, wl.seed, alpha, K, ckpt,
                                 id_offset=id_offset, stream=stream)
            ev[1].record(stream)
            mt.mt_acceptance_loss(work, loss, g, stream=stream)
            ev[2].record(stream)
            mt.mt_adjoint_ckpt(world.handle, n, wl.step_len, wl.max_steps, wl.seed, alpha, K, ckpt, g, da,
                               id_offset=id_offset, stream=stream)
            ev[3].record(stream)
            torch.cuda.synchronize()
            if r:
                times.append([ev[i].elapsed_time(ev[i + 1]) / 1e3 for i in range(3)])
    t = np.mean(np.array(times), axis=0)
    steps = float(work["steps"].sum().item())
    da_ck = da.clone()
    del ckpt
    out = dict(t_forward_ckpt_ms=1e3 * t[0], t_loss_ms=1e3 * t[1], t_adjoint_ms=1e3 * t[2], muon_steps=steps,
               loss=float(loss.item()), ckpt_every=K, dL_dalpha_norm=float(da.norm().item()),
               passes=int((wl.max_steps + K - 1) // K))
    # full-tape variant: the forward records every step, the backward does not recompute
    free, _ = torch.cuda.mem_get_info(init["x"].device)
    tb = mt.mt_tape_bytes(n, wl.max_steps, K)
    if tape and tb <= free - (8 << 30):
        buf = torch.empty(tb, dtype=torch.uint8, device=init["x"].device)
        times = []
        with torch.cuda.stream(stream):
            for r in range(reps + 1):
                for k in work:
                    work[k].copy_(init[k], non_blocking=True)
                ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
                ev[0].record(stream)
                mt.mt_transport_tape(world.handle, work, wl.step_len, wl.max_steps, wl.seed, alpha, K, buf,
                                     id_offset=id_offset, stream=stream)
                ev[1].record(stream)
                mt.mt_acceptance_loss(work, loss, g, stream=stream)
                ev[2].record(stream)
                mt.mt_adjoint_tape(world.handle, n, wl.step_len, wl.max_steps, alpha, K, buf, g, da, stream=stream)
                ev[3].record(stream)
                torch.cuda.synchronize()
                if r:
                    times.append([ev[i].elapsed_time(ev[i + 1]) / 1e3 for i in range(3)])
        t = np.mean(np.array(times), axis=0)
        out["tape"] = dict(t_forward_tape_ms=1e3 * t[0], t_loss_ms=1e3 * t[1], t_adjoint_ms=1e3 * t[2],
                           tape_bytes=tb, tape_bytes_used=int(56 * steps),
                           dL_dalpha_rel_diff_vs_ckpt=float((da - da_ck).norm().item() / max(da_ck.norm().item(),
                                                                                              1e-30)))
        del buf
    return out


def time_alias_form(mt, wl, init, work, stream, id_offset, reps=3):
    """The plain transport of the same workload with the alias sampler
    (Sec. Methodology, "The Alias Method") in place of the inverse CDF."""
    import torch
    times = []
    with mt.World(wl.geometry, wl.field, dict(wl.hist, sampler="alias")) as world, torch.cuda.stream(stream):
        for r in range(reps + 1):
            for k in work:
                work[k].copy_(init[k], non_blocking=True)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            world.transport(work, wl.step_len, wl.max_steps, wl.seed, id_offset=id_offset, stream=stream)
            b.record(stream)
            torch.cuda.synchronize()
            if r:
                times.append(a.elapsed_time(b) / 1e3)
        t = float(np.mean(times))
        steps = float(work["steps"].sum().item())
    return dict(value=steps / t, unit=UNIT, kernel_ms=1e3 * t, muon_steps=steps,
                roofline_frac=BYTES_PER_STEP * steps / t / 1e9 / _peaks()[0]["hbm_gbs"])


def _time_world(mt, wl, geometry, dev, stream, reps, id_offset):
    import torch
    from paper_2512_10520_gb300.api import empty_like_soa
    init = mt.muons_to_device(wl.muons, device=dev)
    work = empty_like_soa(wl.n, device=dev)
    times = []
    with mt.World(geometry, wl.field, wl.hist) as world, torch.cuda.stream(stream):
        for r in range(reps + 1):
            for k in work:
                work[k].copy_(init[k], non_blocking=True)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            world.transport(work, wl.step_len, wl.max_steps, wl.seed, id_offset=id_offset, stream=stream)
            b.record(stream)
            torch.cuda.synchronize()
            if r:
                times.append(a.elapsed_time(b) / 1e3)
        return float(np.mean(times)), float(work["steps"].sum().item())


def time_block1e4_form(mt, dev, stream, reps=20, big=1_000_000, id_offset=0):
    """block1e4: 1e4 muons (log-uniform 5-300 GeV) through one 1x1x2 m iron block
    in air with a uniform 1.7 T field inside the block (analytic, no map),
    2 materials x 64 bins x 128x64 tables, 200 steps.  The call as specified
    (1e4 muons, about a fifth of one wave of the GPU) is timed, and the same
    configuration with 1e6 muons (distinct ids), which fills the GPU.  CUDA
    events on the launching stream."""
    import torch
    from paper_2512_10520_gb300.api import empty_like_soa
    from workloads import gen
    out = {}
    for key, n, r in (("as_specified", None, reps), ("muons_1e6", big, 5)):
        wl = gen.workload("block1e4", n=n)
        init = mt.muons_to_device(wl.muons, device=dev)
        work = empty_like_soa(wl.n, device=dev)
        times = []
        with mt.World.from_workload(wl) as world, torch.cuda.stream(stream):
            for i in range(r + 2):
                for k in work:
                    work[k].copy_(init[k], non_blocking=True)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                world.transport(work, wl.step_len, wl.max_steps, wl.seed, id_offset=id_offset, stream=stream)
                b.record(stream)
                torch.cuda.synchronize()
                if i >= 2:
                    times.append(a.elapsed_time(b) / 1e3)
            t = float(np.median(times))
            steps = float(work["steps"].sum().item())
            launches = mt.mt_transport_launches(world.handle, wl.n, wl.step_len, wl.max_steps)
        out[key] = dict(muons=wl.n, value=steps / t, unit=UNIT, kernel_ms=1e3 * t, muon_steps=steps,
                        muons_per_s=wl.n / t, launches_per_call=launches)
    out["value"] = out["as_specified"]["value"]
    out["unit"] = UNIT
    return out


def boxes_as_solids(geo):
    """The same boxes as polyhedron solids with equal rectangular ends."""
    from workloads import gen
    solids = []
    for b in geo["boxes"]:
        (x0, y0, z0), (x1, y1, z1) = b["lo"], b["hi"]
        q = [(x0, y0), (x1, y0), (x1, y1), (x0, y1)]
        solids.append(gen.solid(z0, z1, q, q, b["material"], b.get("block_id", -1), b.get("B", (0, 0, 0))))
    return dict(geo, kind="polyhedra", solids=solids, boxes=None)


def time_polyhedra_form(mt, dev, stream, n=None, reps=3, id_offset=0):
    """tapered1e6: shield1e6 with tapered magnets as convex solids (Sec. Simulation
    item 1, Eq. 2), same field map and spectrum.  Also timed: shield1e6's own
    boxes given as solids with rectangular ends (same results as the boxes, so
    the difference to the plain form is the cost of the solid lookup alone)."""
    from workloads import gen
    wl = gen.workload("tapered1e6", n=n)
    t, steps = _time_world(mt, wl, wl.geometry, dev, stream, reps, id_offset)
    w1 = gen.workload("shield1e6", n=n)
    t1, steps1 = _time_world(mt, w1, boxes_as_solids(w1.geometry), dev, stream, reps, id_offset)
    return dict(value=steps / t, unit=UNIT, kernel_ms=1e3 * t, muon_steps=steps,
                roofline_frac=BYTES_PER_STEP * steps / t / 1e9 / _peaks()[0]["hbm_gbs"],
                shield1e6_as_solids=dict(value=steps1 / t1, kernel_ms=1e3 * t1, muon_steps=steps1))


def time_offline_form(mt, stream, cpu=True):
    """Offline phase on the GPU (Sec. Building histograms, Appendix A): shield1e6's
    histogram set (3 materials x 64 bins x 128x64 cells, 1e6 samples each) from
    the parametric sampler, and the Appendix A pilot (1024 probes x 1e5 samples)
    with its bounded-variation edges; CUDA events.  CPU: the numpy fixture of
    the same model on one material x 4 bins (4e6 samples), scaled per sample."""
    import torch
    from workloads import gen
    mats = [gen.MATERIALS[m] for m in ("iron", "air", "concrete")]
    edges = gen.pbin_edges(1.0, 400.0, 64)
    w = torch.empty((3, 64, 128, 64), dtype=torch.float64, device="cuda")
    mt.mt_build_histograms(mats, edges, 128, 64, 0.2, 0.02, 10**5, 42, w, stream)      # warm-up
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    mt.mt_build_histograms(mats, edges, 128, 64, 0.2, 0.02, 10**6, 42, w, stream)
    b.record(stream)
    torch.cuda.synchronize()
    t_hist = a.elapsed_time(b) / 1e3
    n_samples = 3 * 64 * 10**6
    probes = np.geomspace(1.0, 400.0, 1024)
    t0 = time.perf_counter()
    phi = mt.mt_pilot_phi(mats[0], probes, 10**5, 0.02, 7, stream)
    t_pilot = time.perf_counter() - t0
    e = mt.mt_bv_edges(probes, phi, 0.05)
    out = dict(value=n_samples / t_hist, unit="samples/s", histograms_ms=1e3 * t_hist, samples=n_samples,
               pilot_ms=1e3 * t_pilot, pilot_samples=1024 * 10**5, bv_bins_iron_eps_0p05=len(e) - 1)
    if cpu:
        rng = np.random.default_rng(1)
        t0 = time.perf_counter()
        for i in range(4):
            gen._hist_one(rng, mats[0], edges[i], edges[i + 1], 2.0, 0.2, 128, 64, 10**6)
        dt = time.perf_counter() - t0
        out["cpu_fixture"] = dict(value=4e6 / dt, unit="samples/s", sample="numpy fixture, iron, 4 bins x 1e6",
                                  cores=1)
    return out


def time_batched_form(mt, stream, dev, n_inst=256, reps=3, rank=0, separate=True, block=0, spp=0):
    """Batched form (worlds256): n_inst worlds, each its own 64x64x512 voxel geometry
    and 100x100x300 field map, one shared histogram set, instance sizes log-uniform
    in [1e3, 1e6].  One mt_transport_batched call (autotuned launch shape, CUDA
    graph) is timed with CUDA events; the same instances as one mt_transport call
    each, in n_inst separate worlds, are timed beside it."""
    import torch
    from paper_2512_10520_gb300.api import empty_like_soa
    from workloads import gen
    hist = gen.batched_hist()
    b = mt.Batch(hist, n_inst)
    inits, insts = [], []
    for i, inst in enumerate(gen.batched_instances(n_inst)):
        b.set_instance(i, inst["geometry"], inst["field"])
        inits.append(mt.muons_to_device(inst["muons"], device=dev))
        insts.append(inst if separate else None)
    counts = [int(t["x"].numel()) for t in inits]
    ids = list(np.cumsum([0] + counts[:-1]) + rank * sum(counts))
    works = [empty_like_soa(c, device=dev) for c in counts]

    def reset():
        for w, s0 in zip(works, inits):
            for k in w:
                w[k].copy_(s0[k], non_blocking=True)

    args = (gen.BATCH_STEP_LEN, gen.BATCH_MAX_STEPS, gen.BATCH_SEED)
    out = dict(instances=n_inst, muons=sum(counts), min_instance=min(counts), max_instance=max(counts))
    with torch.cuda.stream(stream):
        reset()
        if block and spp:
            blk, S, stg = block, spp, 0
        else:
            blk, S, stg = b.autotune(works, *args, sample_per_instance=16384, id_offsets=ids, stream=stream,
                                     cache=False)
        times = []
        for r in range(reps + 1):
            reset()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.transport(works, *args, use_graph=True, id_offsets=ids, stream=stream, block=blk, steps_per_pass=S,
                        staging=stg)
            e1.record(stream)
            torch.cuda.synchronize()
            if r:
                times.append(e0.elapsed_time(e1))
        steps = float(sum(int(w["steps"].sum().item()) for w in works))
        ref_status = [w["status"].clone() for w in works[:8]]
        t = float(np.mean(times)) / 1e3
        out.update(value=steps / t, unit=UNIT, batched_ms=1e3 * t, muon_steps=steps, block=blk, steps_per_pass=S,
                   staging={0: "default", 1: "shared", 2: "global"}[stg],
                   graph=True, device_bytes=b.device_bytes)
        # the plain kernel on the same kind of world: the largest instances (each
        # enough muons to fill the GPU) through one mt_transport call each
        big = sorted(range(n_inst), key=lambda i: -counts[i])[:max(1, min(16, n_inst // 16))]
        if separate:
            bw = [(i, mt.World(insts[i]["geometry"], insts[i]["field"], hist)) for i in big]
            ptimes, psteps = [], 0.0
            for r in range(2):
                reset()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for i, w in bw:
                    w.transport(works[i], *args, id_offset=int(ids[i]), instance=i, stream=stream)
                e1.record(stream)
                torch.cuda.synchronize()
                if r:
                    ptimes.append(e0.elapsed_time(e1))
                    psteps = float(sum(int(works[i]["steps"].sum().item()) for i, _ in bw))
            for _, w in bw:
                w.close()
            tp = float(np.mean(ptimes)) / 1e3
            out.update(plain_largest=dict(instances=len(big), muons=sum(counts[i] for i in big),
                                          value=psteps / tp, ms=1e3 * tp, muon_steps=psteps),
                       vs_plain_same_worlds=(steps / t) / (psteps / tp))
        if separate:
            worlds = [mt.World(inst["geometry"], inst["field"], hist) for inst in insts]
            times = []
            for r in range(2):
                reset()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for i, w in enumerate(worlds):
                    w.transport(works[i], *args, id_offset=int(ids[i]), instance=i, stream=stream)
                e1.record(stream)
                torch.cuda.synchronize()
                if r:
                    times.append(e0.elapsed_time(e1))
            same = all(torch.equal(a, w["status"]) for a, w in zip(ref_status, works[:8]))
            for w in worlds:
                w.close()
            ts = float(np.mean(times)) / 1e3
            out.update(separate_calls_ms=1e3 * ts, separate_value=steps / ts, speedup_vs_separate=ts / t,
                       separate_equal_status_first8=bool(same))
    b.close()
    return out


def time_shield1e8_form(mt, dev, n_total=None, chunk=None, rank=0, cpu_sample=2000):
    """Throughput at scale (shield1e8): 1e8 muons of shield1e6's spectrum in 16M-muon chunks
    through the shield1e6 geometry with a 400x400x1200 map and 4 materials x 128 bins x
    256x128 tables.  Three timings, CUDA events:
      plain     -- all chunks resident in HBM, one mt_transport call per chunk, one stream;
      batched   -- the same muons as one instance of a batch: one mt_transport_batched call
                   (persistent work-queue kernel, CUDA graph);
      streamed  -- pinned host chunks, double-buffered on two streams: H2D copy,
                   mt_transport and D2H copy of chunk c overlap those of chunk c +- 1.
    The FP64 oracle is timed on the first cpu_sample muons on the host cores."""
    import torch
    from paper_2512_10520_gb300.api import empty_like_soa
    from workloads import gen
    n_total = n_total or gen.SHIELD1E8_MUONS
    chunk = min(chunk or gen.SHIELD1E8_CHUNK, n_total)
    wl = gen.workload("shield1e8", n=1)
    bounds = list(range(0, n_total, chunk)) + [n_total]
    spans = list(zip(bounds[:-1], bounds[1:]))
    base_id = rank * n_total
    host_in = empty_like_soa(n_total, device="cpu", pinned=True)
    for c, (lo, hi) in enumerate(spans):
        mu = gen.muons_shield1e8_chunk(c, hi - lo)
        for k in host_in:
            host_in[k][lo:hi].copy_(torch.from_numpy(np.ascontiguousarray(mu[k], dtype=mt._binding.SOA_DTYPES[k])))
    host_out = empty_like_soa(n_total, device="cpu", pinned=True)
    init = {k: v.to(dev) for k, v in host_in.items()}
    work = empty_like_soa(n_total, device=dev)
    args = (wl.step_len, wl.max_steps, wl.seed)
    st0 = torch.cuda.Stream(device=dev)
    out = dict(muons=n_total, chunk=chunk, chunks=len(spans), max_steps=wl.max_steps)

    def reset():
        for k in work:
            work[k].copy_(init[k], non_blocking=True)

    with mt.World.from_workload(wl) as world, torch.cuda.stream(st0):
        out["world_device_bytes"] = world.device_bytes
        # warm-up on the first chunk
        reset()
        sub = {k: v[spans[0][0]:spans[0][1]] for k, v in work.items()}
        world.transport(sub, *args, id_offset=base_id, stream=st0)
        reset()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st0)
        for lo, hi in spans:
            sub = {k: v[lo:hi] for k, v in work.items()}
            world.transport(sub, *args, id_offset=base_id + lo, stream=st0)
        e1.record(st0)
        torch.cuda.synchronize()
        t_plain = e0.elapsed_time(e1) / 1e3
        steps = float(work["steps"].sum().item())
        ref_steps = work["steps"].clone()
        out.update(muon_steps=steps, plain_value=steps / t_plain, plain_ms=1e3 * t_plain,
                   muons_per_s=n_total / t_plain)
        # streamed: pinned host -> device -> host, two streams
        streams = [st0, torch.cuda.Stream(device=dev)]
        bufs = [empty_like_soa(chunk, device=dev) for _ in range(2)]
        torch.cuda.synchronize()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(st0)
        streams[1].wait_event(s0)
        for c, (lo, hi) in enumerate(spans):
            s = streams[c % 2]
            b = {k: v[:hi - lo] for k, v in bufs[c % 2].items()}
            with torch.cuda.stream(s):
                for k in b:
                    b[k].copy_(host_in[k][lo:hi], non_blocking=True)
                world.transport(b, *args, id_offset=base_id + lo, stream=s)
                for k in b:
                    host_out[k][lo:hi].copy_(b[k], non_blocking=True)
        ev = torch.cuda.Event()
        ev.record(streams[1])
        st0.wait_event(ev)
        s1.record(st0)
        torch.cuda.synchronize()
        t_stream = s0.elapsed_time(s1) / 1e3
        out.update(streamed_value=steps / t_stream, streamed_ms=1e3 * t_stream,
                   streamed_h2d_bytes=sum(t.numel() * t.element_size() for t in host_in.values()),
                   streamed_d2h_bytes=sum(t.numel() * t.element_size() for t in host_out.values()),
                   streamed_equal_steps=bool(torch.equal(host_out["steps"], ref_steps.cpu())))
        del bufs
    # batched-persistent: one instance holding all n_total muons
    b = mt.Batch(wl.hist, 1)
    b.set_instance(0, wl.geometry, wl.field)
    with torch.cuda.stream(st0):
        reset()
        b.transport([{k: v[:chunk] for k, v in work.items()}], *args, id_offsets=[base_id], instances=[0],
                    use_graph=False, stream=st0)   # warm-up
        reset()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st0)
        b.transport([work], *args, id_offsets=[base_id], instances=[0], use_graph=True, stream=st0)
        e1.record(st0)
        torch.cuda.synchronize()
        t_b = e0.elapsed_time(e1) / 1e3
        out.update(batched_value=steps / t_b, batched_ms=1e3 * t_b,
                   batched_equal_steps=bool(torch.equal(work["steps"], ref_steps)))
    b.close()
    if cpu_sample and rank == 0:
        import oracle
        mu = {k: host_in[k][:cpu_sample].numpy() for k in host_in}
        ow = oracle.world_of(wl)
        t0 = time.perf_counter()
        o = oracle.transport(ow, mu, *args, id_offset=base_id, n_threads=os.cpu_count() or 1)
        dt = time.perf_counter() - t0
        out["cpu_oracle"] = {"value": float(o["steps"].sum()) / dt, "unit": UNIT, "cores": os.cpu_count(),
                             "sample": f"first {cpu_sample} muons of shield1e8"}
    out["value"] = out["plain_value"]
    out["unit"] = UNIT
    return out


def forms_summary(value: float, kernel_s: float, forms: dict) -> dict:
    """The headline figure of every form, short enough to end the JSON line."""
    def r(x, nd=4):
        return None if x is None else float(f"{x:.{nd}g}")
    out = {"plain": {"value": r(value), "ms": r(1e3 * kernel_s)}}
    if "fwd_adjoint" in forms:
        f = forms["fwd_adjoint"]
        out["fwd_adjoint_ckpt"] = {"value": r(f["value"]), "total_over_forward": r(f["total_over_forward"]),
                                   "fwd_ms": r(f["t_forward_ckpt_ms"]), "adj_ms": r(f["t_adjoint_ms"])}
        if "tape" in f:
            t = f["tape"]
            out["fwd_adjoint_tape"] = {"value": r(t["value"]), "total_over_forward": r(t["total_over_forward"])}
    for k in ("alias", "polyhedra", "nearest_field", "log_axes", "per_stage_field"):
        if k in forms:
            out[k] = {"value": r(forms[k]["value"]),
                      "vs_plain": r(forms[k]["value"] / value)}
    if "batched" in forms:
        b = forms["batched"]
        out["batched"] = {"value": r(b["value"]), "vs_plain": r(b["value"] / value),
                          "vs_plain_same_worlds": r(b.get("vs_plain_same_worlds")), "block": b.get("block"),
                          "steps_per_pass": b.get("steps_per_pass"), "staging": b.get("staging")}
    if "shield1e8" in forms:
        b = forms["shield1e8"]
        out["shield1e8"] = {k: r(b.get(k + "_value")) for k in ("plain", "batched", "streamed")}
    if "block1e4" in forms:
        b = forms["block1e4"]
        out["block1e4"] = {"value": r(b["as_specified"]["value"]), "value_1e6_muons": r(b["muons_1e6"]["value"]),
                           "issue_frac": r((b["as_specified"].get("issue") or {}).get("frac")),
                           "issue_frac_1e6_muons": r((b["muons_1e6"].get("issue") or {}).get("frac"))}
    if "offline" in forms:
        out["offline_samples_per_s"] = r(forms["offline"]["value"])
    return out


def run_reference(args):
    ws, rank, local = _dist()
    if rank != 0:
        return 0
    from workloads import gen
    wl = gen.workload("shield1e6")
    threads = os.cpu_count() or 1
    n_sample = args.cpu_sample
    for _ in range(args.warmup):
        cpu_oracle_run(wl, max(256, n_sample // 8), threads)
    steps_tot, t_tot = 0.0, 0.0
    for _ in range(args.steps):
        s, dt = cpu_oracle_run(wl, n_sample, threads)
        steps_tot += s
        t_tot += dt
    value = steps_tot / t_tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample_muons": n_sample, "parallelism": "host threads"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"first {n_sample} muons of shield1e6 per step (FP64 C oracle, "
                                   f"{threads} POSIX threads)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line))
    return 0


def run_mine(args):
    import torch
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    import __graft_entry__
    __graft_entry__.build()
    import paper_2512_10520_gb300 as mt
    from paper_2512_10520_gb300.api import empty_like_soa
    from workloads import gen

    if args.shield1e8_only:
        with ClockSampler(local) as clk:
            res = time_shield1e8_form(mt, dev, n_total=args.shield1e8_muons, rank=rank, cpu_sample=0 if args.no_cpu else 2000)
        if rank == 0:
            print(json.dumps({"form": "shield1e8", "clocks": clk.summary(), **res}))
        return 0
    if args.only == "block1e4":
        with ClockSampler(local) as clk:
            res = time_block1e4_form(mt, dev, torch.cuda.Stream(device=dev), id_offset=rank * 1_000_000)
        clocks = clk.summary()
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        for key, kern in (("as_specified", "transport_block1e4"), ("muons_1e6", "transport_block1e4_1e6")):
            f = res[key]
            f["issue"] = issue_roofline(kern, f["muon_steps"] / (f["kernel_ms"] / 1e3), clocks.get("sm_mhz"), sms)
        if rank == 0:
            print(json.dumps({"form": "block1e4", "clocks": clocks, **res}))
        return 0
    if args.only == "polyhedra":
        with ClockSampler(local) as clk:
            res = time_polyhedra_form(mt, dev, torch.cuda.Stream(device=dev), n=args.muons, id_offset=rank * (args.muons or 0))
        if rank == 0:
            print(json.dumps({"form": "polyhedra", "clocks": clk.summary(), **res}))
        return 0
    if args.batch_only:
        with ClockSampler(local) as clk:
            res = time_batched_form(mt, torch.cuda.Stream(device=dev), dev, n_inst=args.batch_instances,
                                    rank=rank, separate=not args.no_separate, block=args.batch_block,
                                    spp=args.batch_spp)
        if rank == 0:
            print(json.dumps({"form": "batched", "clocks": clk.summary(), **res}))
        return 0
    wl = gen.workload("shield1e6", n=args.muons)
    n = wl.n
    if args.adjoint_only:
        world = mt.World.from_workload(wl)
        init = mt.muons_to_device(wl.muons, device=dev)
        work = empty_like_soa(n, device=dev)
        stream = torch.cuda.Stream(device=dev)
        with ClockSampler(local) as clk:
            adj = time_adjoint_form(mt, world, wl, init, work, stream, rank * n, K=args.ckpt_every,
                                    tape=not args.no_tape)
        world.close()
        if rank == 0:
            print(json.dumps({"form": "fwd_adjoint", "muons": n, "clocks": clk.summary(), **adj}))
        return 0
    id_offset = rank * n
    stream = torch.cuda.Stream(device=dev)
    world = mt.World.from_workload(wl)
    init = mt.muons_to_device(wl.muons, device=dev)
    work = empty_like_soa(n, device=dev)

    def reset():
        for k in work:
            work[k].copy_(init[k], non_blocking=True)

    ev_k = []
    launch = {}
    if args.mode != "auto" or args.blocks_per_sm or args.steps_per_pass or args.order != "auto":
        launch = dict(mode={"auto": mt.MT_LAUNCH_AUTO, "static": mt.MT_LAUNCH_STATIC,
                            "persistent": mt.MT_LAUNCH_PERSISTENT, "compact": mt.MT_LAUNCH_COMPACT}[args.mode],
                      blocks_per_sm=args.blocks_per_sm, steps_per_pass=args.steps_per_pass,
                      order={"auto": mt.MT_ORDER_AUTO, "always": mt.MT_ORDER_ALWAYS,
                             "never": mt.MT_ORDER_NEVER}[args.order])

    def one_step(timed: bool):
        reset()
        if timed:
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            world.transport(work, wl.step_len, wl.max_steps, wl.seed, id_offset=id_offset, stream=stream, **launch)
            b.record(stream)
            ev_k.append((a, b))
        else:
            world.transport(work, wl.step_len, wl.max_steps, wl.seed, id_offset=id_offset, stream=stream, **launch)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            one_step(False)
        torch.cuda.synchronize()
        steps_per_batch = float(work["steps"].sum().item())
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clk:
            start.record(stream)
            for _ in range(args.steps):
                one_step(True)
            stop.record(stream)
            torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
    elapsed = start.elapsed_time(stop) / 1e3
    elapsed = _barrier_max(elapsed, ws, dev)
    kernel_s = float(np.mean([a.elapsed_time(b) for a, b in ev_k])) / 1e3
    # kernels of this library per transport call, as the library plans them
    launches_per_call = mt.mt_transport_launches(world.handle, n, wl.step_len, wl.max_steps,
                                                 **{k: v for k, v in launch.items() if k != "blocks_per_sm"})
    total_steps = _barrier_sum(steps_per_batch * args.steps, ws, dev)
    value = total_steps / elapsed

    # e2e: pinned host buffers -> device -> mt_transport -> host, every step
    host_in = {k: torch.from_numpy(np.ascontiguousarray(wl.muons[k])).pin_memory() for k in mt._binding.SOA_FIELDS}
    host_out = empty_like_soa(n, device="cpu", pinned=True)
    h2d = sum(t.numel() * t.element_size() for t in host_in.values())
    d2h = sum(t.numel() * t.element_size() for t in host_out.values())
    e2e_steps = 0 if args.no_e2e else max(3, args.steps // 2)
    with torch.cuda.stream(stream):
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(e2e_steps):
            for k in work:
                work[k].copy_(host_in[k], non_blocking=True)
            world.transport(work, wl.step_len, wl.max_steps, wl.seed, id_offset=id_offset, stream=stream, **launch)
            for k in work:
                host_out[k].copy_(work[k], non_blocking=True)
        b.record(stream)
        torch.cuda.synchronize()
    e2e_t = _barrier_max(a.elapsed_time(b) / 1e3, ws, dev)
    e2e_value = (_barrier_sum(float(host_out["steps"].sum().item()) * e2e_steps, ws, dev) / e2e_t
                 if e2e_steps else None)

    forms = {}
    if not args.no_forms:
        adj = time_adjoint_form(mt, world, wl, init, work, stream, id_offset, K=args.ckpt_every)
        t_all = (adj["t_forward_ckpt_ms"] + adj["t_loss_ms"] + adj["t_adjoint_ms"]) / 1e3
        forms["fwd_adjoint"] = dict(
            value=_barrier_sum(adj["muon_steps"], ws, dev) / _barrier_max(t_all, ws, dev), unit=UNIT,
            workload="diff1e6: shield1e6 geometry and map, 18 field scales alpha = 1, 1e6 muons, 1500 steps, "
                     "checkpoints every 32 steps, acceptance loss at z = 30 m",
            adjoint_over_forward=adj["t_adjoint_ms"] / (kernel_s * 1e3),
            total_over_forward=t_all / kernel_s, **adj)
        if "tape" in adj:
            tp = adj["tape"]
            t_tape = (tp["t_forward_tape_ms"] + tp["t_loss_ms"] + tp["t_adjoint_ms"]) / 1e3
            tp.update(value=_barrier_sum(adj["muon_steps"], ws, dev) / _barrier_max(t_tape, ws, dev), unit=UNIT,
                      adjoint_over_forward=tp["t_adjoint_ms"] / (kernel_s * 1e3),
                      total_over_forward=t_tape / kernel_s)
        forms["plain"] = dict(value=value, unit=UNIT, kernel_ms=kernel_s * 1e3)
        al = time_alias_form(mt, wl, init, work, stream, id_offset)
        al["value"] = _barrier_sum(al["muon_steps"], ws, dev) / _barrier_max(al["kernel_ms"] / 1e3, ws, dev)
        al["workload"] = "shield1e6 with the alias sampler (8 B column per draw) instead of the inverse CDF"
        al["vs_inverse_cdf"] = al["value"] / value
        forms["alias"] = al
        ph = time_polyhedra_form(mt, dev, stream, n=args.muons, id_offset=id_offset)
        ph["value"] = _barrier_sum(ph["muon_steps"], ws, dev) / _barrier_max(ph["kernel_ms"] / 1e3, ws, dev)
        ph["workload"] = ("tapered1e6: shield1e6 with the six magnets as tapered convex solids (trapezoid sections "
                          "narrowing along z), spatial-hash pruning, 200x200x600 map")
        ph["vs_boxes"] = ph["value"] / value
        forms["polyhedra"] = ph
        forms["offline"] = time_offline_form(mt, stream, cpu=not args.no_cpu)
        b4 = time_block1e4_form(mt, dev, stream, id_offset=id_offset)
        for key in ("as_specified", "muons_1e6"):
            b4[key]["value"] = (_barrier_sum(b4[key]["muon_steps"], ws, dev)
                                / _barrier_max(b4[key]["kernel_ms"] / 1e3, ws, dev))
        b4["value"] = b4["as_specified"]["value"]
        b4["workload"] = ("block1e4: 1e4 muons (log-uniform 5-300 GeV) through one 1x1x2 m iron block in air, "
                          "uniform 1.7 T inside the block (no map), 2 materials x 64 bins x 128x64, 200 steps")
        forms["block1e4"] = b4
        for name, kw, desc in (("nearest_field", dict(field="nearest"),
                                "shield1e6 with the map read at the nearest node (the paper's lookup, 1 gather)"),
                               ("log_axes", dict(axes="log"),
                                "shield1e6 with histograms on log-scaled (-dPz/P, dPt/P) axes, additive dp"),
                               ("per_stage_field", dict(),
                                "shield1e6 with the map read at every RK4 stage (4 trilinear lookups per step)")):
            wv = gen.workload("shield1e6", n=args.muons, **kw)
            if name == "per_stage_field":
                wv.field = dict(wv.field, per_stage=True)
            tv, sv = _time_world(mt, wv, wv.geometry, dev, stream, 3, id_offset)
            forms[name] = dict(value=_barrier_sum(sv, ws, dev) / _barrier_max(tv, ws, dev), unit=UNIT,
                               kernel_ms=1e3 * tv, muon_steps=sv, vs_plain=(sv / tv) / value, workload=desc)
        bt = time_batched_form(mt, stream, dev, n_inst=args.batch_instances, rank=rank,
                               separate=not args.no_separate)
        bt["value"] = _barrier_sum(bt["muon_steps"], ws, dev) / _barrier_max(bt["batched_ms"] / 1e3, ws, dev)
        bt["workload"] = (f"worlds256: {bt['instances']} worlds (64x64x512 voxels, 100x100x300 map each), shared "
                          f"iron/air/concrete tables, {bt['muons']} muons, log-uniform sizes, 2000 steps")
        forms["batched"] = bt
        if not args.no_shield1e8:
            big = time_shield1e8_form(mt, dev, n_total=args.shield1e8_muons, rank=rank, cpu_sample=0 if args.no_cpu else 2000)
            peaks_, _ = _peaks()
            for key in ("plain", "batched", "streamed"):
                big[key + "_value"] = (_barrier_sum(big["muon_steps"], ws, dev)
                                      / _barrier_max(big[key + "_ms"] / 1e3, ws, dev))
            big["value"] = big["plain_value"]
            big["roofline_frac_plain"] = BYTES_PER_STEP * big["plain_value"] / ws / 1e9 / peaks_["hbm_gbs"]
            big["workload"] = ("shield1e8: 1e8 muons of shield1e6's spectrum in 16M chunks, shield1e6 geometry, "
                              "400x400x1200 map, 4 materials x 128 bins x 256x128 tables")
            forms["shield1e8"] = big
    peaks, peak_kind = _peaks()
    achieved_gbs = BYTES_PER_STEP * steps_per_batch / kernel_s / 1e9
    roof = {"bound": "hbm", "achieved": achieved_gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved_gbs / peaks["hbm_gbs"],
            # the committed figure is for the default launch on the full 1e6-muon call
            "traffic": (_traffic("transport") if args.mode == "auto" and not args.steps_per_pass
                        and not args.blocks_per_sm and args.muons is None else None),
            "peak_kind": peak_kind, "bytes_per_step": BYTES_PER_STEP,
            "kernel_ms": kernel_s * 1e3,
            "timed_unit": "one mt_transport call (all of its kernels), CUDA events on the launching stream"}
    clocks = clk.summary()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    roof["issue"] = issue_roofline("transport", steps_per_batch / kernel_s, clocks.get("sm_mhz"), sms)
    if "block1e4" in forms:
        for key, kern in (("as_specified", "transport_block1e4"), ("muons_1e6", "transport_block1e4_1e6")):
            f = forms["block1e4"][key]
            f["issue"] = issue_roofline(kern, f["muon_steps"] / (f["kernel_ms"] / 1e3), clocks.get("sm_mhz"), sms)
        forms["block1e4"]["roofline"] = dict(forms["block1e4"]["as_specified"]["issue"],
                                             note="no field map: bound by instruction issue, not bytes")
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        threads = os.cpu_count() or 1
        s, dt = cpu_oracle_run(wl, args.cpu_sample, threads)
        cpu = {"value": s / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"first {args.cpu_sample} muons of shield1e6 (FP64 C oracle, {threads} POSIX threads)"}
    world.close()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "form": "plain", "launch": args.mode, "order": args.order,
                       "blocks_per_sm": args.blocks_per_sm, "muons_per_gpu": n, "max_steps": wl.max_steps,
                       "muon_steps_per_batch_per_gpu": steps_per_batch, "muons_per_s": n * ws * args.steps / elapsed,
                       "l2": "inputs larger than L2 (field map 764 MB in HBM vs 129 MB L2); no flush",
                       "parallelism": f"replicas x{ws}"},
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": args.steps * launches_per_call,
            "clocks": clocks,
            "forms": forms,
            "forms_summary": forms_summary(value, kernel_s, forms),
        }
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--cpu-sample", type=int, default=20000)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the fwd+adjoint and batched forms")
    ap.add_argument("--ckpt-every", type=int, default=32, help="checkpoint interval of the fwd+adjoint form")
    ap.add_argument("--muons", type=int, default=None, help="muons per GPU (default: the workload's 1e6)")
    ap.add_argument("--mode", default="auto", choices=["auto", "static", "persistent", "compact"])
    ap.add_argument("--blocks-per-sm", type=int, default=0)
    ap.add_argument("--steps-per-pass", type=int, default=0)
    ap.add_argument("--order", default="auto", choices=["auto", "always", "never"],
                    help="spatial order of the live list between passes (compacting transport with a field map)")
    ap.add_argument("--batch-instances", type=int, default=256, help="worlds in the batched form")
    ap.add_argument("--batch-only", action="store_true", help="run only the batched form (one JSON line)")
    ap.add_argument("--no-shield1e8", action="store_true", help="skip the shield1e8 (1e8 muons) form")
    ap.add_argument("--shield1e8-only", action="store_true", help="run only the shield1e8 form (one JSON line)")
    ap.add_argument("--shield1e8-muons", type=int, default=None, help="muons of the shield1e8 form (default 1e8)")
    ap.add_argument("--batch-block", type=int, default=0, help="batched form: block size (with --batch-spp: no autotune)")
    ap.add_argument("--batch-spp", type=int, default=0, help="batched form: steps per pass")
    ap.add_argument("--adjoint-only", action="store_true", help="run only the fwd+adjoint forms (one JSON line)")
    ap.add_argument("--no-tape", action="store_true", help="fwd+adjoint form: skip the full-tape variant")
    ap.add_argument("--only", default=None, choices=["polyhedra", "block1e4"], help="run only this form (one JSON line)")
    ap.add_argument("--no-separate", action="store_true",
                    help="batched form: skip timing one mt_transport call per instance")
    args = ap.parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    return run_mine(args)


if __name__ == "__main__":
    sys.exit(main())
