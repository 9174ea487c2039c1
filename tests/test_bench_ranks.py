"""bench.py's multi-replica path on CPU: two gloo ranks agree on the slowest
rank's time and report the whole job's throughput (weak scaling, no collective on
the data path)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    local_ms = [100.0 + 50.0 * rank, 7.0 - rank]        # rank 1 is slower on the first value
    got = bench.max_over_ranks(local_ms, dist, "cpu")
    value = bench.job_throughput(980, 10, world, got[0] / 1000.0)
    out.put((rank, got, value, bench.workload(12, 2 + rank).name))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, value, name in res:
        assert got == [150.0, 7.0]                       # the max over ranks, on every rank
        assert value == pytest.approx(2 * 980 * 10 / 0.150)
    assert res[0][3] != res[1][3]                        # each rank runs its own seeded replica


def test_single_rank_is_identity():
    import bench

    assert bench.max_over_ranks([3.0, 4.0]) == [3.0, 4.0]
    assert bench.job_throughput(10, 2, 1, 0.5) == 40.0


def test_kernel_hash_ignores_comments_only():
    """The recorded-traffic key changes with the code the compiler sees, not with
    comments or layout; strings that look like comments are code."""
    import bench

    a = "int f(int x) { // doubles\n  return 2 * x; /* twice */ }\nconst char *u = \"a//b\";\n"
    b = "int f(int x) {\n\n   return 2 * x;   }\nconst char *u = \"a//b\";  // note\n"
    c = "int f(int x) { return 3 * x; }\nconst char *u = \"a//b\";\n"
    d = "int f(int x) { return 2 * x; }\nconst char *u = \"a/*b*/\";\n"
    assert bench.code_only(a) == bench.code_only(b)
    assert bench.code_only(a) != bench.code_only(c)
    assert "/*b*/" in bench.code_only(d)
