"""The N > 1 path of bench.py on CPU: two gloo ranks agree on the max-over-ranks time and the
whole-job rate, and the reference arm runs on rank 0 alone; and its command line."""

import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [0.21, 0.25][rank]  # replica times in ms
    slowest = bench.max_over_ranks(ms, dist, torch.device("cpu"))
    out[rank] = (slowest, bench.job_rate(world, slowest))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time_and_the_job_rate():
    world, port = 2, _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        got = dict(out)
    assert got[0] == got[1]
    slowest, rate = got[0]
    assert slowest == pytest.approx(0.25)
    assert rate == pytest.approx(2 * 1e3 / 0.25)  # both replicas' steps over the slowest time


def test_single_process_needs_no_group():
    import bench
    assert bench.max_over_ranks(0.3, None, None) == 0.3
    assert bench.job_rate(1, 0.5, units_per_step=8) == pytest.approx(16000.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = bench.argparse.Namespace(steps=1, warmup=0, candidate=-1)
    assert bench.run_reference(args) is None


def test_command_line_help_and_workload_names(monkeypatch, capsys):
    import bench
    monkeypatch.setattr(sys, "argv", ["bench.py", "--help"])
    with pytest.raises(SystemExit) as e:
        bench.parse()
    assert e.value.code == 0
    text = capsys.readouterr().out
    for name in ("target", "masked-step", "full-frame", "forward-2k", "keyframes", "large", "global", "adding",
                 "state", "sh"):
        assert name in text
    monkeypatch.setattr(sys, "argv", ["bench.py", "--workload", "full-frame", "--steps", "3", "--warmup", "3"])
    args = bench.parse()
    assert (args.workload, args.steps, args.warmup, args.gpus, args.impl) == ("full-frame", 3, 3, 1, "ours")
