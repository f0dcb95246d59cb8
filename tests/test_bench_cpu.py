"""bench.py on the CPU: the reference arm's JSON line (the FP64 oracle timed on
the host cores), the arithmetic behind the reported numbers, and the GPU arm
failing loudly where no GPU exists (no CPU fallback)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _run(*args, timeout=300):
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=timeout)


def test_reference_arm_prints_one_contract_line():
    r = _run("--impl", "reference", "--workload", "tiny", "--steps", "2", "--warmup", "1", "--cpu-seconds", "1")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    out = json.loads(lines[0])
    assert out["impl"] == "reference" and out["metric"] == bench.METRIC and out["unit"] == bench.UNIT
    assert out["steps"] == 2 and out["warmup"] == 1 and out["n_gpus"] == 1
    assert out["higher_is_better"] is True and out["value"] > 0 and out["ms_per_step"] > 0
    cb = out["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == out["value"] and cb["cores"] >= 1 and cb["sample"]
    assert out["e2e"] == {"value": out["value"], "unit": out["unit"], "h2d_bytes_per_step": 0,
                          "d2h_bytes_per_step": 0}
    assert out["config"]["patches"] == 988 and out["config"]["candidates"] == 200


def test_reference_arm_other_ranks_print_nothing():
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="", RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "tiny",
                        "--steps", "1", "--warmup", "0"], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_gpu_arm_fails_loudly_without_a_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    r = _run("--workload", "tiny", "--steps", "1", "--warmup", "0", "--no-cpu-baseline", "--no-e2e")
    assert r.returncode != 0
    assert not [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]


def test_job_value_counts_every_rank_over_the_slowest_step():
    assert bench.job_value(2_000 * 102_030, 1, 97.2) == pytest.approx(2_000 * 102_030 / 0.0972 / 1e9)
    assert bench.job_value(10, 4, 1.0) == pytest.approx(4 * 10 / 1e-3 / 1e9)
    assert bench.max_over_ranks(3.5) == 3.5


def test_rank_seeds_give_rank_zero_the_reference_room():
    assert bench.rank_seeds("ward", 0) == (1, 2)
    assert bench.rank_seeds("tiny", 0) == (0, 2)
    assert bench.rank_seeds("ward", 3) == (3001, 3002)


def test_kernel_hash_ignores_comments_and_whitespace():
    a = "int f(int x) {\n  return x + 1; // one\n}\n"
    b = "/* doc\n block */ int  f(int x)\n{ return x + 1;\n}\n"
    assert bench._code_only(a) == bench._code_only(b)
    assert bench._code_only(a) != bench._code_only(a.replace("+ 1", "+ 2"))
    assert len(bench.kernel_hash()) == 16


def test_measured_traffic_scales_and_goes_stale(tmp_path):
    cur = bench.kernel_hash()
    per_pair = tmp_path / "per_pair.txt"
    per_pair.write_text(f"header line\nkernel_source_hash: {cur}\ndram_bytes_per_pair: 4.5\n")
    assert bench.measured_traffic(1000, str(per_pair)) == pytest.approx(4500.0)
    per_launch = tmp_path / "per_launch.txt"
    per_launch.write_text(f"kernel_source_hash: {cur}\ndram_bytes_per_launch: 1.25e9\npairs_per_launch: 1000\n")
    assert bench.measured_traffic(1000, str(per_launch)) == pytest.approx(1.25e9)
    assert bench.measured_traffic(999, str(per_launch)) is None      # another launch size: not scalable
    both = tmp_path / "both.txt"
    both.write_text(f"kernel_source_hash: {cur}\ndram_bytes_per_launch: 1.25e9\npairs_per_launch: 1000\n"
                    "dram_bytes_per_pair: 4.5\n")
    assert bench.measured_traffic(1000, str(both)) == pytest.approx(1.25e9)
    assert bench.measured_traffic(2000, str(both)) == pytest.approx(9000.0)
    stale = tmp_path / "stale.txt"
    stale.write_text("kernel_source_hash: 0000000000000000\ndram_bytes_per_pair: 4.5\n")
    assert bench.measured_traffic(1000, str(stale)) is None
    assert bench.measured_traffic(1000, str(tmp_path / "missing.txt")) is None



def test_room_waves_fit_the_pool():
    """Whole rooms are grouped into waves in order; a wave's buffers never
    exceed the pool unless a single room does (it then forms its own wave)."""
    rooms = [{"n": n} for n in (5, 3, 4, 9, 1, 2, 12)]
    waves = bench._waves(rooms, lambda R: R["n"], 8)
    assert [r for w in waves for r in w] == list(range(len(rooms)))
    assert waves == [[0, 1], [2], [3], [4, 5], [6]]
    for w in waves:
        assert sum(rooms[r]["n"] for r in w) <= 8 or len(w) == 1


def test_rooms_block_is_bounded():
    """The rooms-per-second block of the default line runs a fixed number of
    timed steps whatever --steps says, on a stated number of rooms."""
    assert bench.BL_STEPS == 3 and bench.BL_QUALITY_JOBS >= 1
    saved = sys.argv
    try:
        sys.argv = ["bench.py", "--steps", "20"]
        a = bench.parse()
    finally:
        sys.argv = saved
    assert a.bl_rooms == 16 and a.steps == 20
