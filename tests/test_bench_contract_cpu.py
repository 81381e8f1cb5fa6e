"""The bench's reference arm (the oracle on the host cores) prints one JSON line
with the fields of the bench contract (CPU; no GPU needed)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 1
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["config"]["workload"] and d["config"]["name"] == "ground"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_warmup_below_three_is_refused():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "2"], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode != 0


def test_walk_profile_key_ignores_comments_only():
    """The key of the captured walk-kernel figures (bench._src_sha) hashes the
    sources' code: comments and layout do not change it, code and string
    literals (inline PTX) do."""
    sys.path.insert(0, ROOT)
    import bench
    base = 'asm("add.rn.f32 %0, %1, %2;" : "=f"(r));  // one add\nint x = 1; /* c */\n'
    same = '/* a note */ asm("add.rn.f32 %0, %1, %2;"   :  "=f"(r));\n\nint x = 1;\n'
    code = 'asm("add.rn.f32 %0, %1, %2;" : "=f"(r));\nint x = 2;\n'
    ptx = 'asm("sub.rn.f32 %0, %1, %2;" : "=f"(r));\nint x = 1;\n'
    t = bench._code_tokens
    assert t(base) == t(same)
    assert t(base) != t(code) and t(base) != t(ptx)
    assert t('char c = \'/\'; // x\n') == "char c = '/';"
