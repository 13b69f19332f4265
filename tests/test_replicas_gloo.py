"""The multi-GPU form is replicas only (independent chains, no collective on
the data path).  Its host logic runs here as two gloo ranks on the CPU: the
slowest rank's time sets the whole-job throughput, and the reference arm
prints from rank 0 alone."""
import contextlib
import io
import multiprocessing as mp
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=ws)
    import bench
    # rank r timed 100 + 50 r ms for 40 gradient evaluations
    max_ms, value = bench.replica_aggregate(100.0 + 50.0 * rank, 40, ws)
    out = io.StringIO()
    if rank != 0:
        class A:   # the reference arm returns at once on ranks other than 0
            steps, warmup, eps, gpus = 1, 0, 0.025, ws
        with contextlib.redirect_stdout(out):
            bench.reference_arm(A)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, max_ms, value, out.getvalue()))


def test_two_gloo_replicas_report_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, max_ms, value, printed in res:
        assert max_ms == 150.0
        assert abs(value - 2 * 40 / 0.150) < 1e-9
        assert printed == ""
