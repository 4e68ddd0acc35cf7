"""Multi-rank host logic on CPU (gloo, world size 2).

* bench.py's rank helpers: rendezvous on 127.0.0.1, barrier, max over ranks.
* The sharded lattice plan: dimers partitioned across ranks (longest-first
  greedy on cost), each rank accumulates its per-monomer halves, and one
  all-reduce of N_mon x 2 + 2 values gives the same lattice result as the
  unsharded accumulation.  The per-dimer terms here come from the FP64 oracle
  (the GPU part of a rank is the single-GPU library, tested elsewhere).
"""
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


def _env(rank, port):
    os.environ.update({"WORLD_SIZE": "2", "RANK": str(rank), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})


def _bench_helpers_worker(rank, port, q):
    try:
        sys.path.insert(0, ROOT)
        _env(rank, port)
        import torch.distributed as dist
        import bench
        ws, r, local = bench.dist_init()
        bench.barrier(ws)
        m = bench.max_over_ranks(ws, 1.5 + r)
        dist.destroy_process_group()
        q.put((rank, ws, r, m))
    except Exception as e:  # pragma: no cover - reported through the queue
        q.put((rank, "error", repr(e), None))


def _shard_worker(rank, port, q):
    try:
        sys.path.insert(0, ROOT)
        _env(rank, port)
        import torch
        import torch.distributed as dist
        import oracle
        import synth
        dist.init_process_group("gloo")
        w = synth.workload("lattice-2x2x2")
        # longest-first greedy partition on cost (all equal here: round robin)
        cost = [w.nao[X] ** 2 * w.nao[Y] ** 2 for X, Y in w.pairs]
        order = sorted(range(w.n_dimers), key=lambda d: -cost[d])
        load = [0, 0]
        mine = []
        for d in order:
            k = 0 if load[0] <= load[1] else 1
            load[k] += cost[d]
            if k == rank:
                mine.append(d)
        mine.sort()
        items = []
        for d in mine:
            X, Y = w.pairs[d]
            mX, mY = w.monomer(X), w.monomer(Y)
            A, K = w.blocks(d)
            items.append((A, K, mX.C, mX.eps, mY.C, mY.eps, 5, 5))
        E = oracle.dimers_parallel(items)
        mon, tot = oracle.accumulate(E, [w.pairs[d][0] for d in mine], [w.pairs[d][1] for d in mine],
                                     w.n_monomers)
        vec = torch.from_numpy(np.concatenate([mon.ravel(), tot]))
        dist.all_reduce(vec)                      # the one exchange step
        dist.destroy_process_group()
        q.put((rank, vec.numpy(), sorted(mine)))
    except Exception as e:  # pragma: no cover
        q.put((rank, "error", repr(e)))


def _run2(target):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=target, args=(r, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = [q.get(timeout=240) for _ in ps]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    return sorted(out, key=lambda t: t[0])


def test_bench_rank_helpers_gloo():
    pytest.importorskip("torch")
    out = _run2(_bench_helpers_worker)
    for rank, ws, r, m in out:
        assert ws == 2 and r == rank, out
        assert m == 2.5


def test_sharded_lattice_reduction_matches_unsharded():
    pytest.importorskip("torch")
    import oracle
    import synth
    out = _run2(_shard_worker)
    assert all(len(o) == 3 for o in out), out
    (_, v0, m0), (_, v1, m1) = out
    assert np.array_equal(v0, v1)
    assert sorted(m0 + m1) == list(range(28)) and not set(m0) & set(m1)
    w = synth.workload("lattice-2x2x2")
    items = []
    for d in range(w.n_dimers):
        X, Y = w.pairs[d]
        mX, mY = w.monomer(X), w.monomer(Y)
        A, K = w.blocks(d)
        items.append((A, K, mX.C, mX.eps, mY.C, mY.eps, 5, 5))
    E = oracle.dimers_parallel(items)
    mon, tot = oracle.accumulate(E, [p[0] for p in w.pairs], [p[1] for p in w.pairs], w.n_monomers)
    ref = np.concatenate([mon.ravel(), tot])
    assert np.allclose(v0, ref, rtol=1e-13, atol=1e-18)
