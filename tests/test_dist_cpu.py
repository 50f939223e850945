"""The multi-process paths of bench.py on CPU with the gloo backend (world size 2): the job's
time is the maximum over ranks, and the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    worst = bench.max_over_ranks(10.0 + 3.0 * rank)
    cfg = bench.workload_config(512, False, world)
    # the reference arm: every rank but 0 returns at once, before reading its arguments
    out = bench.run_reference(None) if rank != 0 else None
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, worst, cfg["parallelism"], out))


def test_bench_max_over_ranks_and_reference_rank_rule_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [13.0, 13.0]
    assert all(r[2] == "replicas x2" for r in res)
    assert res[1][3] is None


def test_max_over_ranks_without_a_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(4.5) == 4.5


def test_cpulist_parsing():
    """The sysfs cpulist format that places the end-to-end host buffers on the GPU's node."""
    sys.path.insert(0, ROOT)
    import bench

    assert bench.parse_cpulist("0-3,8,10-11\n") == {0, 1, 2, 3, 8, 10, 11}
    assert bench.parse_cpulist("5") == {5}
    assert bench.parse_cpulist("") == set()


def test_roofline_kernels_have_a_traffic_figure():
    """bench.py fills `traffic` from its table of ncu DRAM bytes per cell by kernel name: every
    kernel its roofline lines name has a figure there, scaled by the cell count."""
    sys.path.insert(0, ROOT)
    import re

    import bench

    src = open(os.path.join(ROOT, "bench.py")).read()
    names = re.findall(r'_traffic\("([A-Za-z0-9_]+)"', src)
    assert names, "no roofline kernel named"
    for k in names:
        per_launch = bench._traffic(k, 1000)
        assert per_launch is not None, k
        assert 1000 <= per_launch <= 1000 * 200, (k, per_launch)  # 1 to 200 bytes per cell
    assert bench._traffic("no_such_kernel", 1000) is None
