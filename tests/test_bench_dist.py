"""Host-side checks of bench.py's multi-GPU contract with world_size-2 gloo
process groups on the CPU: the job time is the max over ranks, and the
reference arm runs on rank 0 only (N GPUs run independent replicas)."""
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


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    out[rank] = bench.reduce_max(10.0 * (rank + 1), world, device="cpu")
    r, w, _ = bench.dist_env()
    assert (r, w) == (rank, world)
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_max_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert dict(out) == {0: 20.0, 1: 20.0}


def test_reference_arm_is_rank0_only(capsys):
    sys.path.insert(0, ROOT)
    import bench

    class A:
        n, steps, warmup, cpu_iters, gpus = 4, 1, 0, 2, 2
    bench.run_reference(A(), rank=1, world=2)      # other ranks exit without work
    assert capsys.readouterr().out == ""


def test_workload_bytes_formulas():
    sys.path.insert(0, ROOT)
    import bench
    w = bench.workload_bytes(8_000_000, 23_880_000)
    assert w["amul64"] == 16 * 23_880_000 + 24 * 8_000_000          # 574.08 MB
    assert w["it64"] == 152 * 8_000_000 + 48 * 23_880_000
    assert w["it32"] == 76 * 8_000_000 + 36 * 23_880_000


def test_cpulist_parsing():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.parse_cpulist("0-3,8,10-11\n") == {0, 1, 2, 3, 8, 10, 11}
    assert bench.parse_cpulist("5") == {5}
    assert bench.parse_cpulist("") == set()


def test_traffic_record_scaling(monkeypatch):
    """The roofline traffic record scales from the captured case by the
    algorithmic bytes, and is withheld once the solver source has changed."""
    import hashlib
    sys.path.insert(0, ROOT)
    import bench
    with open(os.path.join(ROOT, "paper_2512_22215_gb300", "csrc", "solve.cu"), "rb") as fh:
        sha = hashlib.sha1(fh.read()).hexdigest()
    rec = {"solve_cu_sha1": sha, "n": 128, "bytes": 10 ** 11, "inner": 500, "outer": 4}
    monkeypatch.setattr(bench, "TRAFFIC", rec)
    n, nf = 128 ** 3, 3 * 127 * 128 * 128
    assert bench.traffic_bytes(n, nf, 500, 4) == 10 ** 11                      # the captured case itself
    w = bench.workload_bytes(8_000_000, 23_880_000)
    wc = bench.workload_bytes(n, nf)
    want = 10 ** 11 * (795 * w["it32"] + 5 * w["resid64"]) / (500 * wc["it32"] + 5 * wc["resid64"])
    assert abs(bench.traffic_bytes(8_000_000, 23_880_000, 795, 4) - want) <= 1
    monkeypatch.setattr(bench, "TRAFFIC", dict(rec, solve_cu_sha1="0" * 40))
    assert bench.traffic_bytes(n, nf, 500, 4) is None
