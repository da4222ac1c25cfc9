"""Multi-process host logic of the benchmark on CPU (gloo, world size 2).

Exact kNN splits by queries: each rank answers its own query shard against the
same reference set, with no exchange step; only the timing takes a maximum
over ranks.  These tests run that logic with two CPU processes."""
import hashlib
import os
import socket
import sys
from types import SimpleNamespace

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _digest(a):
    return int.from_bytes(hashlib.sha256(np.ascontiguousarray(a).tobytes()).digest()[:7], "little")


def _worker(rank, world, port, errq):
    try:
        sys.path.insert(0, ROOT)
        sys.path.insert(0, os.path.join(ROOT, "tests"))
        os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        dist.init_process_group("gloo", rank=rank, world_size=world)
        import bench
        import oracle

        args = SimpleNamespace(n_ref=3000, n_query=257, leaf=16)
        W = bench.shard_workload(args, rank)
        h = torch.tensor([_digest(W.ref), _digest(W.query)], dtype=torch.int64)
        hs = [torch.zeros_like(h) for _ in range(world)]
        dist.all_gather(hs, h)
        assert all(int(x[0]) == int(hs[0][0]) for x in hs), "reference sets differ"
        assert len({int(x[1]) for x in hs}) == world, "query shards repeat"

        # each shard's answers are those of the whole query set: no exchange
        idx, dd = oracle.knn_brute(W.ref, W.query, W.k)
        ti, td, _ = oracle.knn_dualtree(W.ref, W.query, W.k, W.leaf_size)
        assert np.array_equal(idx, ti) and np.array_equal(dd, td)
        out = torch.from_numpy(idx.astype(np.int64))
        outs = [torch.zeros_like(out) for _ in range(world)]
        dist.all_gather(outs, out)
        qs = [bench.shard_workload(args, r).query for r in range(world)]
        whole, _ = oracle.knn_brute(W.ref, np.concatenate(qs), W.k)
        assert np.array_equal(np.concatenate([o.numpy() for o in outs]), whole)

        # timing: the slowest rank sets the job's time
        ms = 10.0 + 5.0 * rank
        mx = bench.max_over_ranks(ms, world, "cpu")
        assert mx == 10.0 + 5.0 * (world - 1)
        assert bench.job_rate(world, 257, mx) == pytest.approx(world * 257 / (mx / 1e3))
        dist.barrier()
        dist.destroy_process_group()
    except BaseException as e:  # noqa: BLE001
        errq.put(f"rank {rank}: {type(e).__name__}: {e}")
        raise


def test_query_shards_gloo_world2():
    ctx = mp.get_context("spawn")
    errq = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, errq)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    alive = [p for p in procs if p.is_alive()]
    for p in alive:
        p.kill()
        p.join()
    errs = []
    while not errq.empty():
        errs.append(errq.get())
    assert not alive, "a rank did not finish"
    assert not errs, errs
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]


def test_single_rank_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.job_rate(1, 1000, 500.0) == pytest.approx(2000.0)
    a = bench.shard_workload(SimpleNamespace(n_ref=100, n_query=10, leaf=8), 0)
    b = bench.shard_workload(SimpleNamespace(n_ref=100, n_query=10, leaf=8), 1)
    assert np.array_equal(a.ref, b.ref) and not np.array_equal(a.query, b.query)
    assert a.leaf_size == 8
