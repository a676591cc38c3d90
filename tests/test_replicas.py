"""bench.py's multi-GPU mode runs independent replicas (the path has no data
exchange): the whole-job throughput is ranks x solves / the slowest rank's
time.  The host logic runs here as two gloo ranks on the CPU."""
import importlib.util
import os
import socket

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as tdist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    local_ms = 100.0 + 50.0 * rank              # rank 1 is the slower replica
    value, total = mod.replica_throughput(local_ms, 10, world, "cpu")
    out.put((rank, value, total))
    tdist.barrier()
    tdist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, total in res:
        assert total == 150.0
        assert abs(value - 2 * 10 / 0.150) < 1e-9


def test_single_replica_needs_no_process_group():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    value, total = mod.replica_throughput(200.0, 20, 1, "cpu")
    assert total == 200.0 and value == 100.0
