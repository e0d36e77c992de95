"""Multi-process (gloo, world size 2) checks of the N > 1 paths, on CPU.

- bench.py's replica timing: barrier, and the max over ranks of the per-rank time.
- Sharding by tuples: because sketches are linear (Section 2.2), per-rank partial
  sketches of disjoint tuple shards, summed with an int64 all-reduce, equal the sketch
  of the whole stream (the oracle computes both).
"""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    import oracle as O
    import synth
    dist.init_process_group("gloo")
    try:
        bench.barrier(world)
        t = bench.max_over_ranks(world, float(rank + 1) * 1.5)
        w = synth.chain3(n=3000, m=64, d=3, seed=11)
        q = O.canonical_query(w.num_join_attrs, w.edges)
        co = O.draw_coefficients(w.hash_seed, w.d, q.n_comp, len(q.edges))
        cols = w.relations[1].cols.numpy()
        n = cols.shape[1]
        lo, hi = rank * n // world, (rank + 1) * n // world
        part = O.sketch_relation(q, co, 1, cols[:, lo:hi], None, w.m)
        tot = torch.from_numpy(part.copy())
        dist.all_reduce(tot, op=dist.ReduceOp.SUM)
        full = O.sketch_relation(q, co, 1, cols, None, w.m)
        ok = bool(np.array_equal(tot.numpy(), full))
        with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
            f.write(f"{t} {int(ok)}\n")
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo(tmp_path):
    world = 2
    port = _free_port()
    mp.start_processes(_worker, args=(world, port, str(tmp_path)), nprocs=world, join=True, start_method="spawn")
    for r in range(world):
        t, ok = open(tmp_path / f"r{r}.txt").read().split()
        assert float(t) == 3.0          # max over ranks of 1.5 and 3.0
        assert ok == "1"
