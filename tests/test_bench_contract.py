"""The benchmark's reference arm (the FP64 oracle timed on the host cores)
keeps the one-line JSON contract: the same metric, unit and config keys as
the GPU arm, the oracle's cpu_baseline block, and an e2e block; under a
multi-rank launch only rank 0 prints.  CPU only."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra, *args):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, "bench.py", "--impl", "reference", *args], cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_contract_line():
    r = _run({}, "--workload", "tree15_32", "--steps", "1", "--warmup", "3", "--count", "1")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["unit"] == "solves/s" and d["higher_is_better"] is True
    assert d["warmup"] >= 3 and d["steps"] == 1 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    other = d["cpu_baseline"]["other_oracle_solvers"]
    assert other["jacobi_cg"]["relres"] <= 1e-8 and other["jacobi_cg"]["iterations"] > 0
    assert other["sparse_direct"]["s_per_solve"] > 0
    assert d["e2e"] == {"value": d["value"], "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"].startswith("tree15_32") and d["config"]["prec_order"] == "upper"
    assert d["config"]["jacobi_smoothing"]["sweeps_before_and_after"] == 0 and d["config"]["inner_fgmres_steps"] == 0


def test_reference_arm_other_ranks_exit_quietly():
    r = _run({"RANK": "1", "WORLD_SIZE": "2"}, "--steps", "1", "--warmup", "3", "--count", "1")
    assert r.returncode == 0
    assert not [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]


def test_default_workload_is_the_mixed_batch():
    """Without flags the benchmark runs the mixed 256-instance batch in the
    block order that solves it fastest, and each workload names its order."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.WORKLOAD == "batch256_mixed" and bench.DEFAULT_COUNT["batch256_mixed"] == 256
    assert set(bench.DEFAULT_ORDER) == set(bench.WORKLOAD_TEXT)
    assert bench.DEFAULT_ORDER["batch256_mixed"] == "lower" and bench.DEFAULT_ORDER["tree15_32"] == "upper"
    picked = bench._reference_sample("batch256_mixed", 256)
    assert sorted({w["N"] for _, w in picked}) == [32, 48, 64] and len(picked) == 9
