"""The multi-process path of bench.py on CPU: two gloo ranks (127.0.0.1) run the replica
aggregation that bench.py uses under torchrun. The job's step time is the slowest rank's and
the job's throughput counts the units of every rank; the reference arm runs on rank 0 only."""
import multiprocessing as mp
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    w, r, _ = bench.dist_info()
    dist = bench.dist_init(w, "gloo")
    ms_local = 2.0 + 3.0 * r  # rank 1 is the slower replica
    ms, units_per_s = bench.aggregate_replicas(ms_local, 1000.0, w, "cpu")
    bench.barrier(w)
    q.put((r, ms, units_per_s))
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_bench():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, ms, units_per_s in out:
        assert ms == 5.0                          # max over ranks
        assert abs(units_per_s - 2 * 1000.0 / 5e-3) < 1e-6  # both ranks' units / job time


def test_single_process_aggregation_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    ms, ups = bench.aggregate_replicas(4.0, 100.0, 1, "cpu")
    assert ms == 4.0 and abs(ups - 100.0 / 4e-3) < 1e-9
