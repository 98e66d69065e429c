"""The replicas path of bench.py on the CPU (no GPU): under torchrun each rank
steps its own instance, and the line reports the slowest rank's time (max over
ranks) and the particle-steps of all ranks (sum).  Two gloo ranks exercise the
same combination; the reference arm runs on rank 0 alone."""
import argparse
import socket

import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, secs, pushed, q):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        q.put((rank,) + bench.combine_ranks(secs[rank], pushed[rank], dist, "cpu"))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_report_the_slowest_time_and_the_summed_steps():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    secs, pushed = [0.5, 0.8], [100, 250]
    procs = [ctx.Process(target=_rank, args=(r, 2, port, secs, pushed, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        got = sorted(q.get(timeout=120) for _ in procs)
    finally:
        for p in procs:
            p.join(60)
            if p.is_alive():
                p.kill()
    assert [p.exitcode for p in procs] == [0, 0]
    assert got == [(0, 0.8, 350.0), (1, 0.8, 350.0)]


def test_one_rank_keeps_its_own_figures():
    assert bench.combine_ranks(0.25, 7, None, "cpu") == (0.25, 7.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    bench.run_reference(argparse.Namespace(workload="sphere16", steps=1, warmup=0))
    assert capsys.readouterr().out == ""
