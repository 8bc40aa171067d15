"""The multi-rank path of the benchmark on CPU ranks (gloo, world size 2):
barriers, the max-over-ranks duration, the whole-job rate, and a rank that
fails before the timed region (the other rank learns of it from the
monitored barrier instead of waiting forever)."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, mode, q):
    sys.path.insert(0, ROOT)
    import datetime
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=30))
    try:
        if mode == "ok":
            bench.ranks_barrier(world, timeout_s=20)
            t = bench.max_over_ranks(1.0 + rank, world)
            v = bench.aggregate_rate(100.0, 3, world, t)
            bench.ranks_barrier(world, timeout_s=20)
            q.put((rank, "ok", t, v))
        else:
            if rank == 1:
                q.put((rank, "raised", None, None))
                raise SystemExit(0)      # leaves without joining the barrier
            try:
                bench.ranks_barrier(world, timeout_s=3)
                q.put((rank, "passed", None, None))
            except Exception as ex:      # the monitored barrier names the missing rank
                q.put((rank, "error", str(ex)[:200], None))
    finally:
        try:
            dist.destroy_process_group()
        except Exception:
            pass


def _run(mode):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, mode, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        if p.is_alive():
            p.kill()
    return sorted(out)


def test_two_cpu_ranks_reduce_to_the_slowest_rank():
    out = _run("ok")
    assert [o[1] for o in out] == ["ok", "ok"]
    for _, _, t, v in out:
        assert t == 2.0                       # max over ranks
        assert v == pytest.approx(100.0 * 3 * 2 / 2.0)


def test_a_rank_that_leaves_is_reported_not_waited_for():
    out = _run("fail")
    assert out[1][1] == "raised"
    assert out[0][1] == "error"


def test_hv_count_of_a_solve():
    """H·v calls a solve runs, as the benchmark counts them: the recurrence,
    the second run of it after the kept head of the basis (none with a stored
    basis), and the FP64 refinement."""
    import bench
    base = {"iters": 150, "ritz_terms": 120}
    assert bench.hv_count(dict(base, stored_basis=True, basis_head=0)) == 151
    assert bench.hv_count(dict(base, stored_basis=False, basis_head=0)) == 150 + 119 + 1
    assert bench.hv_count(dict(base, stored_basis=False, basis_head=16)) == 150 + 104 + 1
    assert bench.hv_count(dict(base, stored_basis=False, basis_head=120)) == 151
    assert bench.hv_count(dict(base, stored_basis=False)) == 150 + 119 + 1
