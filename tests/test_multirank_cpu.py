"""The multi-rank host path on CPU: two gloo ranks split the parameter sets
of an ensemble (`shard.split_sets`), each draws and integrates its own sets
with the oracle (the counter-based sampler draws set s the same on every
rank), and the gathered per-set results equal a single-process run of all
sets; the max over ranks of the timed region is the largest rank's value.
No GPU: this covers the sharding and exchange logic that bench.py uses with
NCCL on one GPU per rank."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N_SETS, N_ICS, SEED = 7, 4, 2000


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_path):
    sys.path.insert(0, ROOT)
    import oracle as O
    from paper_2503_18356_gb300 import shard, workloads as W
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        topo = W.toggle_switch()
        net = O.Network(*topo.edges())
        s0, n = shard.split_sets(N_SETS, rank, world)
        p = O.sample_params(net, SEED, n, set0=s0)
        ic = O.sample_ics(topo.n_nodes, SEED, N_ICS)
        o = O.run_sets(net, p, ic)
        states = shard.gather_rows(o["states"])
        status = shard.gather_rows(o["status"])
        nu = shard.gather_rows(o["n_unique"].astype(np.int64))
        G = shard.gather_rows(p.G)
        mx = shard.max_over_ranks(10.0 + rank)
        if rank == 0:
            np.savez(out_path, states=states, status=status, n_unique=nu, G=G, mx=mx)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_match_one_process(tmp_path):
    import oracle as O
    from paper_2503_18356_gb300 import shard, workloads as W
    out = str(tmp_path / "ranks.npz")
    mp.spawn(_rank, args=(2, _free_port(), out), nprocs=2, join=True)
    r = np.load(out)
    topo = W.toggle_switch()
    net = O.Network(*topo.edges())
    p = O.sample_params(net, SEED, N_SETS)
    o = O.run_sets(net, p, O.sample_ics(topo.n_nodes, SEED, N_ICS))
    assert r["G"].shape[0] == N_SETS
    assert np.array_equal(r["G"], p.G)                 # shards drew exactly the sets of the full run
    assert np.array_equal(r["states"], o["states"])
    assert np.array_equal(r["status"], o["status"])
    assert np.array_equal(r["n_unique"], o["n_unique"].astype(np.int64))
    assert float(r["mx"]) == 11.0


@pytest.mark.parametrize("n,world", [(7, 2), (1, 2), (10, 4), (0, 3), (100, 8)])
def test_split_sets_covers_every_set_once(n, world):
    from paper_2503_18356_gb300 import shard
    ranges = [shard.split_sets(n, r, world) for r in range(world)]
    covered = [s for first, cnt in ranges for s in range(first, first + cnt)]
    assert covered == list(range(n))
    counts = [c for _, c in ranges]
    assert max(counts) - min(counts) <= 1
    assert shard.rank_sets(50, 3) == (150, 50)
