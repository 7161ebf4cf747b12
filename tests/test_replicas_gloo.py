"""Multi-GPU host logic on CPU: the benchmark runs one independent replica of
the workload per rank (the method has no exchange step between systems), and
reports the slowest rank's time against the atom-steps of all ranks.  Two
gloo ranks on CPU check that aggregation, and that a rank which fails before
the collective ends the others' wait with an error instead of a hang.
"""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, units, out, fail_rank):
    import datetime

    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=20))
    try:
        if rank == fail_rank:
            raise RuntimeError("planted failure before the collective")
        dist.barrier()
        t, u = bench.aggregate_ranks(times[rank], units[rank], world, "cpu")
        out.put((rank, t, u))
    except Exception as e:  # reported to the parent, never a hang
        out.put((rank, "error", type(e).__name__))
    finally:
        try:
            dist.destroy_process_group()
        except Exception:
            pass


def _run(world, times, units, fail_rank=-1):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, times, units, q, fail_rank))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    alive = [p for p in procs if p.is_alive()]
    for p in alive:
        p.kill()
    assert not alive, "a rank hung"
    res = {}
    while not q.empty():
        r = q.get()
        res[r[0]] = r[1:]
    return res


def test_replica_aggregation_two_ranks():
    res = _run(2, times=[1.25, 2.5], units=[98304 * 30, 98304 * 30])
    assert set(res) == {0, 1}
    for r in (0, 1):
        t, u = res[r]
        assert t == 2.5                      # slowest rank
        assert u == 2 * 98304 * 30           # whole-job units


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_ranks(0.75, 1000, 1, "cpu") == (0.75, 1000.0)


@pytest.mark.timeout(180)
def test_failed_rank_does_not_hang_the_other():
    res = _run(2, times=[1.0, 1.0], units=[1, 1], fail_rank=1)
    assert res[1] == ("error", "RuntimeError")
    # rank 0's barrier ends with an error once its peer is gone
    assert res[0][0] == "error"
