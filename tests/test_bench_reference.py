"""The benchmark's reference arm (the oracle timed on the host cores), run on the CPU at R-MAT
scale 14: its JSON line must follow from its own printed numbers -- the timed samples are time
actually spent, and the extrapolated solve time is the sample's time per block SpMM times the
block count of the oracle's own full solve of that graph (tests/golden/oracle_solves.json)."""
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(tmp_path, extra_env=None, steps=2):
    env = dict(os.environ)
    env.pop("RANK", None)
    env.pop("WORLD_SIZE", None)
    env.update(extra_env or {})
    t0 = time.perf_counter()
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--scale", "14", "--steps", str(steps), "--warmup", "0", "--no-config1",
                        "--outdir", str(tmp_path)],
                       capture_output=True, text=True, env=env, cwd=ROOT, timeout=600)
    return p, time.perf_counter() - t0


def test_reference_line_follows_from_its_numbers(tmp_path):
    p, wall = _run(tmp_path)
    assert p.returncode == 0, p.stderr
    lines = [l for l in p.stdout.splitlines() if l.strip()]
    assert len(lines) == 1                                   # one JSON line
    r = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in r, key
    assert r["impl"] == "reference" and r["unit"] == "solves/s" and r["higher_is_better"]
    assert r["steps"] == 2 and r["n_gpus"] == 1
    # timed steps are time actually spent inside this process
    assert r["steps"] * r["ms_per_step"] / 1000.0 <= wall
    # the sample: two Krylov-Schur cycles -- 8 expansion blocks, then 3 after keeping k = 20
    # Ritz vectors -- and the final residual's 2 blocks (nev 8 / b 4)
    s = r["sample"]
    assert s["block_spmms_per_step"] == 13
    assert abs(s["s_per_block_spmm"] * s["block_spmms_per_step"] - s["ms_per_step"] / 1000.0) \
        <= 1e-9 * s["ms_per_step"]
    # the extrapolation uses the oracle's own full solve of this graph, not a constant
    golden = json.load(open(os.path.join(ROOT, "tests", "golden", "oracle_solves.json")))["rmat14"]
    x = r["extrapolation"]
    assert x["full_solve_block_spmms"] == golden["spmm_blocks"] == 151
    assert abs(x["s_per_solve"] - s["s_per_block_spmm"] * 151) <= 1e-12 * x["s_per_solve"]
    assert abs(r["value"] * x["s_per_solve"] - 1.0) <= 1e-12
    # the cpu_baseline and e2e objects repeat the line's own value; no device copies
    assert r["cpu_baseline"]["value"] == r["value"] and r["cpu_baseline"]["kind"] == "oracle"
    assert r["cpu_baseline"]["cores"] >= 1
    assert r["e2e"] == {"value": r["value"], "unit": "solves/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert r["vs_baseline"] is None


def test_reference_other_ranks_exit_without_work(tmp_path):
    p, _ = _run(tmp_path, {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}, steps=1)
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""
