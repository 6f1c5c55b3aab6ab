"""The multi-process path on CPU (gloo, world size 2): the bench's max/sum
reductions over ranks, and sharding by global muon id.  Ranks transport disjoint
id ranges with no collective on the data path; because every Philox counter
holds the global id, the shards together reproduce one single-process run
bit for bit (here with the FP64 oracle standing in for the per-rank transport)."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, n_total, out_dir):
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    import oracle
    from workloads import gen
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        assert bench._dist() == (ws, rank, rank)
        # reductions used for the timed region and the step counts
        assert bench._barrier_max(float(rank + 1), ws) == float(ws)
        assert bench._barrier_sum(float(rank + 1), ws) == float(ws * (ws + 1) // 2)
        # shard: rank r takes ids [r*m, (r+1)*m)
        wl = gen.workload("block1e4", n=n_total, hist_samples=20000)
        m = n_total // ws
        sub = {k: v[rank * m:(rank + 1) * m] for k, v in wl.muons.items()}
        out = oracle.transport(oracle.world_of(wl), sub, wl.step_len, wl.max_steps, wl.seed, id_offset=rank * m,
                               n_threads=2)
        steps = bench._barrier_sum(float(out["steps"].sum()), ws)
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), steps_total=steps, **out)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_by_muon_id(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as tmp
    import oracle
    from workloads import gen
    ws, n_total = 2, 256
    tmp.start_processes(_rank_main, args=(ws, _free_port(), n_total, str(tmp_path)), nprocs=ws, join=True,
                        start_method="spawn")
    wl = gen.workload("block1e4", n=n_total, hist_samples=20000)
    ref = oracle.transport(oracle.world_of(wl), wl.muons, wl.step_len, wl.max_steps, wl.seed, n_threads=2)
    parts = [np.load(tmp_path / f"rank{r}.npz") for r in range(ws)]
    for k in ("x", "y", "z", "px", "py", "pz", "steps", "status"):
        np.testing.assert_array_equal(np.concatenate([p[k] for p in parts]), ref[k], err_msg=k)
    assert all(float(p["steps_total"]) == float(ref["steps"].sum()) for p in parts)
