"""The multi-rank path of bench.py on CPU: two gloo ranks (127.0.0.1), replicas with
disjoint guesses, the maximum time over ranks, the whole-job value, and the reference arm
leaving every rank but 0 idle.  No GPU and no collective on the data path."""
import os
import socket
import types

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank), PCF_BENCH_BACKEND="gloo")
    import bench
    dist, r, w = bench._dist()
    mx = bench.reduce_max(dist, 10.0 + r, "cpu")          # rank-dependent step times
    value = bench.aggregate_value(8, w, 5, mx * 1e-3)
    out = None
    if r != 0:  # the reference arm: ranks other than 0 return at once, with no output
        args = types.SimpleNamespace(gpus=w, steps=1, warmup=0)
        out = bench.run_reference(args)
    dist.barrier()
    dist.destroy_process_group()
    q.put((r, w, mx, bench.rank_seeds(r), value, out))


def test_two_ranks_reduce_and_shard():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1] and all(r[1] == 2 for r in res)
    assert all(r[2] == 11.0 for r in res)                       # the slowest rank's time
    assert sorted(res[0][3] + res[1][3]) == list(range(16))     # disjoint guesses, all covered
    assert all(abs(r[4] - 8 * 2 * 5 / 11e-3) < 1e-9 for r in res)
    assert res[1][5] is None


def test_single_rank_has_no_process_group():
    import bench
    dist, r, w = bench._dist()
    assert dist is None and (r, w) == (0, 1)
    assert bench.reduce_max(None, 3.5, "cpu") == 3.5
