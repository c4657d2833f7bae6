"""The multi-GPU path is replicas only (one matrix does not shard; section
"Multi-GPU" of the design): each rank factors its own copy and the bench
reports all ranks' work over the slowest rank's time. This checks that host
logic with two gloo ranks on the CPU (no GPU, no collective on the data path)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t_local = [1.5, 2.5][rank]  # the slower rank defines the job time
        t_max = bench.max_over_ranks(t_local, world)
        rate = bench.whole_job_rate(world, 4, 1.6e12, t_max)
        out.put((rank, t_max, rate))
    finally:
        dist.destroy_process_group()


def test_two_rank_max_time_and_weak_scaling_rate():
    mp = pytest.importorskip("torch.multiprocessing")
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t_max, rate in res:
        assert t_max == 2.5
        assert rate == pytest.approx(2 * 4 * 1.6e12 / 2.5)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    sys.path.insert(0, ROOT)
    import bench

    class A:
        steps, warmup, gpus = 1, 0, 2
    bench.run_reference(A(), 2, 1)  # rank 1: no work, no output
    assert capsys.readouterr().out == ""


def test_oracle_throughput_on_all_host_cores():
    """The bench's all-cores CPU baseline: one copy of the single-thread oracle
    sample per host core, run as separate processes; the aggregate is every
    copy's flops over the overlapped wall time (positive, and not above cores
    x a single copy's rate beyond timing noise)."""
    sys.path.insert(0, ROOT)
    import bench
    value, cores = bench.oracle_sample_all_cores(1)
    assert isinstance(cores, int) and cores >= 1
    assert value is not None and value > 0
    dt, flops = bench.oracle_sample(1)
    single = flops / dt / 1e12
    assert value <= cores * single * 1.5


def test_reference_arm_loads_nothing_of_the_cuda_library():
    """The CPU-oracle arm counts its flops with the closed form: in a fresh
    interpreter, a sample run imports no module of the CUDA package but the
    input generators and maps no library of it."""
    import json
    import subprocess
    code = ("import json, sys; sys.path.insert(0, sys.argv[1]); import bench; bench.oracle_sample(1); "
            "maps = open('/proc/self/maps').read(); "
            "print(json.dumps({'mods': sorted(m for m in sys.modules if m.startswith('paper_2504_19171_gb300')), "
            "'libstiles': 'libstiles' in maps}))")
    out = subprocess.run([sys.executable, "-c", code, ROOT], capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    r = json.loads(out.stdout.strip().splitlines()[-1])
    assert r["mods"] == ["paper_2504_19171_gb300", "paper_2504_19171_gb300.workloads"]
    assert r["libstiles"] is False
