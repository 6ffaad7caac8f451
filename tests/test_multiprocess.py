"""Multi-process paths on CPU with the gloo backend (world size 2).

1. Target-leaf sharding: rank r of N computes the targets of schedule
   entries r, r+N, ... (psr_opts.shard_count / shard_index); here each rank
   evaluates its shard with the FP64 oracle, the shards are summed with an
   all-reduce, and the result must equal the unsharded oracle.
2. The benchmark's job timing: the slowest rank's time, reduced over ranks.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _workload():
    import synth
    rng = np.random.default_rng(21)
    pos, _ = synth.nfw_clustered(3000, 50.0, 0.6, 4, rng)
    r_s, r_c = synth.box_params(50.0, 16)
    return pos, rng.uniform(0.5, 1.5, 3000), 50.0, r_s, r_c


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import oracle
        import paper_2107_14008_gb300 as psr
        pos, mass, L, r_s, r_c = _workload()
        lv = psr.Leaves.build(pos, mass, L, r_s, r_c, max_leaf=16)
        perm = lv.perm
        mine = perm[lv.shard_targets(world, rank)]  # original indices of my targets
        acc = torch.zeros((pos.shape[0], 3), dtype=torch.float64)
        a, _, _ = oracle.forces(pos, mass, L, r_s, r_c, targets=mine, threads=2)
        acc[torch.from_numpy(mine)] = torch.from_numpy(a)
        owner = torch.zeros(pos.shape[0], dtype=torch.int64)
        owner[torch.from_numpy(mine)] = 1
        dist.all_reduce(acc)
        dist.all_reduce(owner)
        t = bench.max_over_ranks(10.0 + rank, dist, "cpu")
        if rank == 0:
            full, _, _ = oracle.forces(pos, mass, L, r_s, r_c, threads=2)
            q.put({"owner_ok": bool(torch.all(owner == 1)),
                   "err": float(np.max(np.abs(acc.numpy() - full))),
                   "scale": float(np.max(np.abs(full))), "tmax": t})
    finally:
        dist.destroy_process_group()


def test_sharded_targets_all_reduce_to_the_full_result():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert res["owner_ok"]  # every target computed by exactly one rank
    assert res["err"] <= 1e-14 * res["scale"]
    assert res["tmax"] == 11.0


def test_shards_are_balanced_and_disjoint():
    import paper_2107_14008_gb300 as psr
    pos, mass, L, r_s, r_c = _workload()
    lv = psr.Leaves.build(pos, mass, L, r_s, r_c, max_leaf=16)
    A = lv.host_arrays()
    leaf, rp, pairs, items = A["leaf"], A["rowptr"], A["pairs"], A["items"]
    src = np.array([leaf[(pairs[rp[i]:rp[i + 1]] >> 5).astype(np.int64), 1].sum()
                    for i in range(leaf.shape[0])])
    cost = src * leaf[:, 1]
    for world in (2, 3, 4):
        parts = [lv.shard_targets(world, r) for r in range(world)]
        allt = np.concatenate(parts)
        assert np.array_equal(np.sort(allt), np.arange(lv.n))
        loads = np.array([cost[items[r::world]].sum() for r in range(world)])
        assert loads.max() <= 1.1 * loads.mean()
