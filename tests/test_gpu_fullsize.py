"""Parity at the benchmark's full sizes, in the launch configurations bench.py
times, on sampled outputs the FP64 oracle computes muon by muon:
- the batched form over all 256 worlds (37.6 M muons);
- the differentiable form on 1e6 muons: the adjoint is linear in dL/dfinal, so
  the gradient restricted to a muon sample is compared with the oracle's
  adjoint of those muons alone;
- one 16 M-muon chunk of the 1e8-muon stream with the 400x400x1200 map."""
import numpy as np
import pytest

import oracle
from helpers import assert_parity, compare, describe
from workloads import gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2512_10520_gb300 as mt
    mt.load_library()


def test_worlds256_full_batch_sampled_parity():
    import torch
    import paper_2512_10520_gb300 as mt
    hist = gen.batched_hist()
    n_inst = 256
    check = list(range(0, n_inst, 8))          # 32 instances, up to 625 sampled muons each
    kept = {}
    with mt.Batch(hist, n_inst) as b:
        devs = []
        for i, inst in enumerate(gen.batched_instances(n_inst)):
            b.set_instance(i, inst["geometry"], inst["field"])
            devs.append(mt.muons_to_device(inst["muons"]))
            if i in check:
                kept[i] = inst
        blk, S, stg = b.autotune(devs, gen.BATCH_STEP_LEN, gen.BATCH_MAX_STEPS, gen.BATCH_SEED,
                                 sample_per_instance=2048)
        b.transport(devs, gen.BATCH_STEP_LEN, gen.BATCH_MAX_STEPS, gen.BATCH_SEED, use_graph=True)
        torch.cuda.synchronize()
        assert sum(int(d["x"].numel()) for d in devs) > 3e7
        rng = np.random.default_rng(1)
        gots, oras = [], []
        for i in check:
            inst = kept[i]
            n = inst["n"]
            idx = np.sort(rng.choice(n, size=min(n, 625), replace=False))
            got = {k: v.cpu().numpy()[idx] for k, v in devs[i].items()}
            ora = oracle.transport(oracle.OracleWorld(inst["geometry"], inst["field"], hist), inst["muons"],
                                   gen.BATCH_STEP_LEN, gen.BATCH_MAX_STEPS, gen.BATCH_SEED, instance=i, index=idx)
            ok, err = compare(got, ora)
            # per instance a gross-error guard (a wrong world or id mapping fails most
            # muons); the 99.9 % bar is statistical and applies to the pooled sample
            assert ok.mean() >= 0.99, (i, describe(ok, err))
            gots.append(got)
            oras.append(ora)
        cat = lambda L: {k: np.concatenate([d[k] for d in L]) for k in L[0]}
        pooled_g, pooled_o = cat(gots), cat(oras)
        assert len(pooled_g["x"]) >= 10_000
        assert_parity(pooled_g, pooled_o)


def test_diff1e6_full_size_adjoint_sampled():
    import torch
    import paper_2512_10520_gb300 as mt
    wl = gen.workload("shield1e6")
    n = wl.n
    assert n == 1_000_000
    rng = np.random.default_rng(5)
    alpha = (1.0 + 0.2 * rng.standard_normal((6, 3))).astype(np.float32)
    sample = np.sort(rng.choice(n, size=400, replace=False))
    with mt.World.from_workload(wl) as world:
        a = torch.as_tensor(alpha).cuda().contiguous()
        ref = mt.muons_to_device(wl.muons)
        # the checkpointing forward reorders its saved lists at this size; the reference does not
        world.transport(ref, wl.step_len, wl.max_steps, wl.seed, alpha=a, mode=mt.MT_LAUNCH_COMPACT,
                        order=mt.MT_ORDER_NEVER)
        dev = mt.muons_to_device(wl.muons)
        ck = torch.empty(mt.mt_ckpt_bytes(n, wl.max_steps, 32), dtype=torch.uint8, device="cuda")
        mt.mt_transport_ckpt(world.handle, dev, wl.step_len, wl.max_steps, wl.seed, a, 32, ck)
        for k in ("x", "y", "z", "px", "py", "pz", "steps", "status"):
            assert torch.equal(ref[k], dev[k]), k
        loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        g = torch.empty((6, n), dtype=torch.float32, device="cuda")
        mt.mt_acceptance_loss(dev, loss, g)
        mask = torch.zeros(n, dtype=torch.float32, device="cuda")
        mask[torch.as_tensor(sample, device="cuda")] = 1.0
        gs = (g * mask).contiguous()
        da = torch.empty_like(a)
        mt.mt_adjoint_ckpt(world.handle, n, wl.step_len, wl.max_steps, wl.seed, a, 32, ck, gs, da)
        del ck
        tape = torch.empty(mt.mt_tape_bytes(n, wl.max_steps, 32), dtype=torch.uint8, device="cuda")
        dev2 = mt.muons_to_device(wl.muons)
        mt.mt_transport_tape(world.handle, dev2, wl.step_len, wl.max_steps, wl.seed, a, 32, tape)
        db = torch.empty_like(a)
        mt.mt_adjoint_tape(world.handle, n, wl.step_len, wl.max_steps, a, 32, tape, gs, db)
        torch.cuda.synchronize()
        g_s = g.cpu().numpy()[:, sample].astype(np.float64)
    ow = oracle.world_of(wl, alpha.astype(np.float64))
    # each sampled muon with its own id (id_offset = its index)
    g_ora = np.zeros((6, 3))
    for j, m in enumerate(sample):
        one = {k: v[m:m + 1] for k, v in wl.muons.items()}
        g_ora += oracle.adjoint(ow, one, wl.step_len, wl.max_steps, wl.seed, g_s[:, j:j + 1], id_offset=int(m))
    for got in (da, db):
        gg = got.cpu().numpy().astype(np.float64)
        rel = np.linalg.norm(gg - g_ora) / np.linalg.norm(g_ora)
        assert rel <= 1e-3, (rel, gg.ravel().tolist(), g_ora.ravel().tolist())


def test_shield1e8_chunk_sampled_parity():
    import torch
    import paper_2512_10520_gb300 as mt
    wl = gen.workload("shield1e8", n=1)
    mu = gen.muons_shield1e8_chunk(0, gen.SHIELD1E8_CHUNK)
    with mt.World.from_workload(wl) as world:
        dev = mt.muons_to_device(mu)
        world.transport(dev, wl.step_len, wl.max_steps, wl.seed, id_offset=0)
        torch.cuda.synchronize()
        rng = np.random.default_rng(2)
        idx = np.sort(rng.choice(gen.SHIELD1E8_CHUNK, size=20_000, replace=False))
        got = {k: v.cpu().numpy()[idx] for k, v in dev.items()}
    ora = oracle.transport(oracle.world_of(wl), mu, wl.step_len, wl.max_steps, wl.seed, index=idx)
    assert_parity(got, ora)
