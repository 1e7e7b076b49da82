"""The multi-GPU path on the CPU: two gloo ranks, each advancing its own
shard of particles with global ids rank*N + i (as bench.py does under
torchrun), then one integer all-reduce (sum) of histograms and counters.
The reduced result must equal a single process over all particles, bit for
bit -- the random streams are keyed by global particle id, so sharding
changes nothing.  The per-rank work is the CPU oracle (no GPU here); the
sharding, id offsets and reduction are what is under test."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as tmp

from paper_2512_02175_gb300 import workloads as W

N_PER_RANK, STEPS, DT, M, BINS, SEED = 1500, 150, 2e-3, 8, 8, 21


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _shard(rank):
    from oracle import oracle as O
    d = W.random_mixed(5)
    e, x = W.uniform_on_edges(d, 2 * N_PER_RANK, 3)
    lo, hi = rank * N_PER_RANK, (rank + 1) * N_PER_RANK
    g = O.Graph.from_desc(d)
    st = O.State(e[lo:hi], x[lo:hi], np.arange(lo, hi, dtype=np.uint32))
    cnt = O.Counters(g)
    O.simulate(g, st, cnt, seed=SEED, instance=0, dt=DT, steps=STEPS, M=M)
    hist = O.histogram(g, st, BINS)
    return np.concatenate([hist, cnt.exits, cnt.absorbed, cnt.truncations,
                           cnt.particle_steps.astype(np.uint64)])


def _rank_main(rank, world, port, out_path):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local = torch.from_numpy(_shard(rank).astype(np.int64))
    dist.all_reduce(local, op=dist.ReduceOp.SUM)
    if rank == 0:
        np.save(out_path, local.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_shards_equal_one_process(tmp_path, oracle):
    out = str(tmp_path / "reduced.npy")
    tmp.spawn(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True)
    reduced = np.load(out)
    # one process over all 2N particles
    from oracle import oracle as O
    d = W.random_mixed(5)
    e, x = W.uniform_on_edges(d, 2 * N_PER_RANK, 3)
    g = O.Graph.from_desc(d)
    st = O.State(e, x)
    cnt = O.Counters(g)
    O.simulate(g, st, cnt, seed=SEED, instance=0, dt=DT, steps=STEPS, M=M)
    whole = np.concatenate([O.histogram(g, st, BINS), cnt.exits, cnt.absorbed,
                            cnt.truncations, cnt.particle_steps.astype(np.uint64)])
    assert np.array_equal(reduced, whole.astype(np.int64))
    assert 0 < whole[-1] <= 2 * N_PER_RANK * STEPS
