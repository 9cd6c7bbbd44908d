"""The bench's multi-rank host logic on CPU with the gloo backend (world size 2): each rank
searches its own stack (weak scaling, no collective on the data path), the timed region's
duration is the maximum over ranks, every rank agrees on the step count, and under torchrun the
reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = bench.dist_env()
    got = {"env": (r, w, lr),
           "ms_max": bench.max_over_ranks(10.0 + 5.0 * rank, world, "cpu"),
           "steps": bench.max_over_ranks(3 + rank, world, "cpu"),
           "seed": bench.rank_seed(5, rank)}
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, got))


def test_max_over_ranks_and_rank_seeds_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(world):
        assert res[r]["env"] == (r, world, r)
        assert res[r]["ms_max"] == 15.0          # the slowest rank's time, on every rank
        assert res[r]["steps"] == 4.0
    assert res[0]["seed"] != res[1]["seed"]       # independent stacks


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.5, 1, "cpu") == 7.5
    assert bench.rank_seed(5, 0) == 5


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        workload = "decam"
        warmup = 1
        steps = 1
        cpu_seconds = 0.1
        gpus = 2

    bench.run_reference(A())   # returns at once: no oracle work, nothing printed
    assert capsys.readouterr().out == ""


def test_reference_arm_prints_one_contract_line(monkeypatch, capsys):
    """Rank 0 of the reference arm times the oracle and prints one JSON line with the keys the
    bench contract names (here on the tiny stack, a fraction of a second of CPU work)."""
    import json
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.delenv("RANK", raising=False)
    monkeypatch.delenv("WORLD_SIZE", raising=False)

    class A:
        workload = "tiny"
        warmup = 1
        steps = 2
        cpu_seconds = 0.05
        gpus = 1

    bench.run_reference(A())
    lines = capsys.readouterr().out.strip().splitlines()
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["unit"] == "TE/s" and d["value"] > 0
    assert (d["steps"], d["warmup"], d["n_gpus"]) == (2, 1, 1)
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"] == d["e2e"]["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"].startswith("tiny") and "fit in L2" in d["config"]["l2"]
    assert "larger than L2" in bench.workload_config("decam")["l2"]


def test_clock_summary_of_nvidia_smi_rows():
    """The clocks block of the bench line: median SM clock under load, the max clock, and every
    throttle reason seen active in any sample (rows that do not parse are skipped)."""
    sys.path.insert(0, ROOT)
    import bench
    rows = [
        "0, 2032, 2032, 613.62, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2032, [N/A], 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2010, 2032, 700.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "[N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A]",
        "garbage",
    ]
    s = bench.summarize_clock_rows(rows)
    assert s["sm_mhz"] == 2010.0 and s["sm_max_mhz"] == 2032.0
    assert s["power_w_max"] == 700.5 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    hot = rows[0].replace("Not Active, Not Active, Not Active, Not Active",
                          "Active, Not Active, Active, Not Active")
    assert bench.summarize_clock_rows([hot])["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    assert bench.summarize_clock_rows([])["reasons"] == ["no samples"]


def test_refine_recovery_matching():
    """The refine line's recovery figure: for each mover, the highest-L candidate whose track is
    within 2.5 px of the true one at the first and at the last epoch, else -1."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    times = np.array([0.0, 0.5, 2.0])
    movers = dict(x0=np.array([10.0, 50.0]), y0=np.array([20.0, 60.0]),
                  vx=np.array([100.0, -40.0]), vy=np.array([5.0, 0.0]))
    params = np.array([
        [10.5, 20.0, 100.0, 5.0],     # mover 0, L 8
        [11.0, 21.0, 100.5, 5.0],     # mover 0, L 9: within 2.5 px at both ends -> chosen
        [10.0, 20.0, 102.0, 5.0],     # starts on mover 0 but 4 px off at the last epoch
        [50.0, 60.0, -40.0, 0.0],     # mover 1, but L is NaN (refine stopped): not eligible
    ], np.float32)
    lh = np.array([8.0, 9.0, 30.0, np.nan], np.float32)
    got = bench._match_movers(params, lh, movers, times)
    assert got.tolist() == [1, -1]


def test_measured_peaks_and_fallback(tmp_path, monkeypatch):
    """The roofline denominators come from MEASURED_PEAKS.json when present, else from the stated
    fallback (6.4 TB/s HBM, 1.8 PFLOP/s bf16), labelled as such."""
    import json
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    peaks, src = bench.measured_peaks()
    assert src == "fallback" and peaks["hbm_gbs"] == 6400.0 and peaks["bf16_tflops"] == 1800.0
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6505.9,
                                                              "sm_max_mhz": 2032.0}))
    peaks, src = bench.measured_peaks()
    assert src == "measured" and peaks["hbm_gbs"] == 6505.9


def test_bench_launches_its_own_ranks_dry_run():
    """`python bench.py --gpus 2` outside torchrun starts two ranks itself (torch.distributed.run
    on this node); in --dry-run mode they join a gloo group on CPU, take the slowest rank's time
    and rank 0 alone prints one line for the whole job, each rank with its own stack seed."""
    import json
    import subprocess
    env = dict(os.environ)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK", "MASTER_ADDR", "MASTER_PORT"):
        env.pop(k, None)
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--gpus", "2",
                          "--steps", "2", "--warmup", "3", "--dry-run"], capture_output=True,
                         text=True, timeout=300, env=env, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, out.stdout
    d = json.loads(lines[0])
    assert d["dry_run"] and d["n_gpus"] == 2 and d["scaling"] == "weak" and d["steps"] == 2
    seeds = d["config"]["seeds"]
    assert len(seeds) == 2 and seeds[0] != seeds[1]
    te = 26 * 2046 * 4094 * 32768
    assert abs(d["value"] - 2 * te * 2 / (d["ms_per_step"] * 2 / 1e3)) <= 1e-6 * d["value"]


def test_bench_rejects_a_rank_count_other_than_gpus():
    import subprocess
    env = dict(os.environ, WORLD_SIZE="2", RANK="0", LOCAL_RANK="0")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--gpus", "4",
                          "--dry-run"], capture_output=True, text=True, timeout=120, env=env,
                         cwd=ROOT)
    assert out.returncode != 0 and "ranks were started" in out.stderr
