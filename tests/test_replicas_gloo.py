"""The N > 1 bench path on CPU: two gloo ranks run the host logic of the
replicas (independent index streams, max-over-ranks timing, whole-job value),
and a rank that leaves before the timing reduction is detected by the other
through the process group's timeout.  No GPU is involved."""
import datetime
import multiprocessing as mp
import os
import socket
import sys

import pytest

pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _worker(rank, ws, port, q, leave_early):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws,
                            timeout=datetime.timedelta(seconds=5))
    dist.barrier()
    if leave_early and rank == 1:
        q.put((rank, "left"))
        return  # leaves between steps, before the timing reduction
    ms_local = 10.0 + 2.5 * rank
    try:
        ms = bench.job_ms(ms_local, ws, "cpu")
    except Exception as e:  # the peer never joins the reduction
        q.put((rank, "error", type(e).__name__))
        return
    q.put((rank, "ok", ms, bench.job_value(ws, 4096 * 64, ms), bench.replica_seed(0, rank),
           [bench.batch_seed(rank, p) for p in range(3)]))
    dist.destroy_process_group()


def _run(leave_early):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q, leave_early)) for r in range(2)]
    for p in ps:
        p.start()
    out = {}
    try:
        for _ in range(2):
            item = q.get(timeout=90)
            out[item[0]] = item[1:]
    finally:
        for p in ps:
            p.join(timeout=30)
            if p.is_alive():  # only the processes this test started
                p.terminate()
                p.join(timeout=10)
    return out, [p.exitcode for p in ps]


def test_two_replicas_time_and_value():
    out, codes = _run(leave_early=False)
    assert codes == [0, 0]
    (s0, ms0, v0, seed0, bs0), (s1, ms1, v1, seed1, bs1) = out[0], out[1]
    assert s0 == s1 == "ok"
    assert ms0 == ms1 == 12.5  # the slowest rank's time, on every rank
    assert v0 == pytest.approx(2 * 4096 * 64 / 0.0125)
    assert seed0 != seed1  # independent index streams
    assert not set(bs0) & set(bs1)


def test_rank_leaving_is_detected():
    out, codes = _run(leave_early=True)
    assert out[1] == ("left",)
    assert out[0][0] == "error"  # rank 0's reduction fails within the timeout
