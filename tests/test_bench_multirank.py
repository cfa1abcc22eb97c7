"""The N > 1 path of bench.py on CPU: two gloo ranks, each with its own step time, must both
obtain the max over ranks and the whole-job throughput (replicas, no data-path collective)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t_max, value = bench.whole_job(1000, 100.0 + 50.0 * rank, world, dist, "cpu")
    q.put((rank, t_max, value))
    dist.barrier()
    dist.destroy_process_group()


def test_whole_job_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t_max, value in out:
        assert t_max == 150.0
        assert abs(value - 2 * 1000 / 0.150) < 1e-9


def test_whole_job_single_rank():
    import bench
    assert bench.whole_job(500, 250.0, 1) == (250.0, 2000.0)


def test_kernel_source_map_resolves_and_traffic_is_current():
    """Every timed kernel name that bench.py maps to CUDA source text resolves to functions that
    exist, and every recorded ncu traffic figure belongs to the current text of its kernel."""
    import bench
    for name in bench.KERNEL_SOURCES:
        assert bench.kernel_digest(name) is not None, name
    for (name, _workload), rec in bench.NCU_TRAFFIC.items():
        assert rec["digest"] == bench.kernel_digest(name), name
        assert name in bench.stored_bytes_names()
