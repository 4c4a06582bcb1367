"""The replica path of bench.py on CPU: two gloo ranks get disjoint marker blocks, meet at
barriers and agree on the max over ranks of their elapsed times (no GPU, no data collective)."""
import multiprocessing as mp
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench

    dist, r, w = bench._dist()
    bench._barrier(dist)
    t = bench._max_over_ranks(dist, 10.0 * (r + 1))
    q.put((r, w, bench.rank_blocks(r, w, 4), t))
    bench._barrier(dist)
    dist.destroy_process_group()


def test_two_replicas_shard_blocks_and_reduce_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, b0, t0), (r1, w1, b1, t1) = out
    assert (r0, r1, w0, w1) == (0, 1, 2, 2)
    assert not set(b0) & set(b1) and sorted(b0 + b1) == list(range(8))
    assert t0 == t1 == 20.0
