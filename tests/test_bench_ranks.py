"""CPU checks of bench.py's host logic: the max-over-ranks reduction of the
step time across replica ranks (world size 2 over gloo), and the oracle arm
(`--impl reference`), which prints one JSON line on rank 0 and nothing on the
other ranks, and the all-cores oracle leg."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        got = bench.max_over_ranks(1.5 + 2.0 * rank, dist, "cpu")
        alone = bench.max_over_ranks(1.5 + 2.0 * rank, None, "cpu")
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump({"max": got, "alone": alone}, f)
    finally:
        dist.destroy_process_group()


def test_step_time_is_the_slowest_rank(tmp_path):
    import torch.multiprocessing as mp

    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    for r in range(world):
        got = json.load(open(tmp_path / f"rank{r}.json"))
        assert got["max"] == 3.5
        assert got["alone"] == 1.5 + 2.0 * r


def _run_reference(rank, world):
    env = dict(os.environ, RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    return subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1"],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_other_ranks_exit_without_work():
    r = _run_reference(1, 2)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_reference_arm_prints_the_contract_line():
    r = _run_reference(0, 1)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["steps"] == 1 and d["warmup"] == 1 and d["higher_is_better"] is True
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["unit"] == d["unit"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    # the unknowns per step and the step time give the value
    assert d["value"] == pytest.approx(d["config"]["angular_unknowns"] / (d["ms_per_step"] * 1e-3), rel=1e-12)


def test_oracle_on_every_core_sums_independent_copies():
    """The all-cores oracle leg runs one single-threaded copy of the sample per
    core and adds their rates; each copy's rate is that of the one-core leg's
    kind (a tiny 2x2 sample here)."""
    sys.path.insert(0, ROOT)
    import bench

    one = bench.oracle_rate(0.05, 2)
    both = bench.run_oracle_all_cores(0.05, 2, cores=2)
    assert "error" not in both, both
    assert both["cores"] == 2 and both["kind"] == "oracle" and both["unit"] == one["unit"]
    assert both["value"] > 0 and isinstance(both["cpu"], str)


def test_network_flop_count_matches_the_layer_list():
    """The learned-guess roofline's numerator: 2 x the multiply-adds of every layer of the oracle's layer
    list over real channels (the stride-2 layer and the one after it on the half-resolution grid), at both
    sets of widths."""
    import bench
    from oracle import cnn
    for nx, n_out, c1, c2 in ((128, 9, 64, 384), (64, 9, 24, 32), (16, 4, 16, 48)):
        macs = 0
        for i, (ci, co, k, _) in enumerate(cnn.layer_specs(n_out, c1, c2)):
            side = nx // 2 if i in (1, 2) else nx
            macs += co * ci * k * k * side * side
        assert bench.network_flops(nx, n_out, c1, c2) == 2.0 * macs
    assert abs(bench.network_flops(128, 9, 64, 384) - 22.42e9) < 0.01e9
