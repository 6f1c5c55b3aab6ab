"""Shared test helpers: run the CUDA path on a numpy SoA, compare with the oracle."""
import numpy as np

POS_TOL = 1e-4      # m, per-muon final position
MOM_TOL = 1e-5      # relative, per-muon final momentum
PASS_FRAC = 0.999   # fraction of muons that must match (rare FP32 decision flips allowed)


def gpu_transport(wl, muons=None, alpha=None, max_steps=None, id_offset=None, world=None, chunks=None):
    """Run mt_transport through the C ABI; returns host numpy SoA."""
    import torch
    import paper_2512_10520_gb300 as mt
    muons = wl.muons if muons is None else muons
    own = world is None
    if own:
        world = mt.World.from_workload(wl)
    try:
        dev = mt.muons_to_device(muons)
        a = None if alpha is None else torch.as_tensor(np.asarray(alpha, np.float32)).cuda().contiguous()
        ms = wl.max_steps if max_steps is None else max_steps
        off = wl.id_offset if id_offset is None else id_offset
        if chunks is None:
            world.transport(dev, wl.step_len, ms, wl.seed, id_offset=off, instance=wl.instance, alpha=a)
        else:
            n = len(muons["x"])
            bounds = np.linspace(0, n, chunks + 1).astype(int)
            for lo, hi in zip(bounds[:-1], bounds[1:]):
                sub = {k: v[lo:hi] for k, v in dev.items()}
                world.transport(sub, wl.step_len, ms, wl.seed, id_offset=off + int(lo), instance=wl.instance,
                                alpha=a)
        torch.cuda.synchronize()
        return mt.muons_to_host(dev)
    finally:
        if own:
            world.close()


def compare(gpu, ora, idx=None):
    """Per-muon agreement mask and the error arrays."""
    if idx is not None:
        gpu = {k: np.asarray(v)[idx] for k, v in gpu.items()}
    pg = np.stack([gpu["x"], gpu["y"], gpu["z"]], 1).astype(np.float64)
    po = np.stack([ora["x"], ora["y"], ora["z"]], 1)
    mg = np.stack([gpu["px"], gpu["py"], gpu["pz"]], 1).astype(np.float64)
    mo = np.stack([ora["px"], ora["py"], ora["pz"]], 1)
    pos_err = np.abs(pg - po).max(1)
    mom_err = np.linalg.norm(mg - mo, axis=1) / np.maximum(np.linalg.norm(mo, axis=1), 1e-30)
    same_steps = gpu["steps"] == ora["steps"]
    same_status = gpu["status"] == ora["status"]
    ok = (pos_err <= POS_TOL) & (mom_err <= MOM_TOL) & same_steps & same_status
    both_invalid = (np.asarray(gpu["status"]) == 5) & (np.asarray(ora["status"]) == 5)
    ok |= both_invalid & same_steps
    return ok, dict(pos_err=pos_err, mom_err=mom_err, same_steps=same_steps, same_status=same_status)


def describe(ok, err):
    bad = np.flatnonzero(~ok)
    return (f"pass {ok.mean():.5f} ({(~ok).sum()} of {len(ok)} fail); max pos err {err['pos_err'].max():.3g} m, "
            f"max mom err {err['mom_err'].max():.3g}; median pos err {np.median(err['pos_err']):.3g}; "
            f"steps mismatches {(~err['same_steps']).sum()}, status mismatches {(~err['same_status']).sum()}; "
            f"first failures {bad[:8].tolist()}")


KS_MIN_P = 0.01     # two-sample KS on final x, y, |p| (distribution agreement)


def ks_pvalues(gpu, ora):
    """Two-sample KS p-values of final x, y and |p|, GPU against oracle."""
    from scipy import stats

    def P(f):
        return np.sqrt(np.asarray(f["px"], np.float64) ** 2 + np.asarray(f["py"], np.float64) ** 2
                       + np.asarray(f["pz"], np.float64) ** 2)
    return {"x": stats.ks_2samp(np.asarray(gpu["x"], np.float64), np.asarray(ora["x"], np.float64)).pvalue,
            "y": stats.ks_2samp(np.asarray(gpu["y"], np.float64), np.asarray(ora["y"], np.float64)).pvalue,
            "|p|": stats.ks_2samp(P(gpu), P(ora)).pvalue}


def assert_parity(gpu, ora, idx=None, frac=PASS_FRAC):
    """The acceptance bar of the GPU path against the FP64 oracle: at least `frac` of
    muons within (POS_TOL, MOM_TOL) with identical steps and status, and KS p >
    KS_MIN_P on final x, y and |p|.  Returns the per-muon mask."""
    ok, err = compare(gpu, ora, idx)
    assert ok.mean() >= frac, describe(ok, err)
    g = gpu if idx is None else {k: np.asarray(v)[idx] for k, v in gpu.items()}
    ks = ks_pvalues(g, ora)
    assert min(ks.values()) > KS_MIN_P, (ks, describe(ok, err))
    return ok
