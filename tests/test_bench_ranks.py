"""The bench's multi-rank logic on CPU (gloo, world size 2): the barrier and
the maximum over ranks that every timed number goes through, and the
reference arm's rule that only rank 0 runs and prints under torchrun."""
import importlib.util
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port):
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        ctx = _bench().Ctx(world, rank, torch.device("cpu"))
        ctx.barrier()
        # each rank's time differs; every rank reports the slowest
        assert ctx.max_over_ranks(1.0 + rank * 0.5) == 1.0 + (world - 1) * 0.5
        assert ctx.max_over_ranks(3.0 - rank) == 3.0
        ctx.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_barrier_gloo():
    import torch.multiprocessing as mp
    mp.spawn(_rank_main, args=(2, _free_port()), nprocs=2, join=True)


def test_single_rank_context_needs_no_process_group():
    import torch
    ctx = _bench().Ctx(1, 0, torch.device("cpu"))
    ctx.barrier()
    assert ctx.max_over_ranks(2.5) == 2.5


@pytest.mark.parametrize("rank", ["1", "3"])
def test_reference_arm_other_ranks_exit_without_work(rank):
    env = dict(os.environ, RANK=rank, WORLD_SIZE="4", LOCAL_RANK=rank, MASTER_ADDR="127.0.0.1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "4"],
                       capture_output=True, text=True, timeout=120, env=env, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_log_appends_the_json_line(tmp_path):
    """--log appends the printed JSON line to a JSONL file (reference arm,
    small oracle sample, CPU)."""
    import json
    log = tmp_path / "runs.jsonl"
    env = dict(os.environ, RANK="0", WORLD_SIZE="1")
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1", "--warmup", "0",
           "--sample", "300", "--log", str(log)]
    log.write_text('{"earlier": "run"}\n')
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=300, env=env, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = log.read_text().splitlines()
    assert len(lines) == 2 and json.loads(lines[0]) == {"earlier": "run"}     # appended, not overwritten
    rec = json.loads(lines[1])
    assert rec["impl"] == "reference" and rec["unit"] == "GB/s" and rec["value"] > 0
    assert json.loads(r.stdout.strip().splitlines()[-1]) == rec
