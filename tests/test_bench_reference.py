"""The bench's reference arm (the FP64 oracle timed on the host cores) runs
without a GPU and prints one JSON line with the keys its consumers read."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_its_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_counter_digest_follows_code_not_comments():
    """The digest that ties recorded ncu counters to the kernel source ignores
    comments and whitespace, keeps string literals, and changes with code."""
    sys.path.insert(0, ROOT)
    import bench
    base = 'int f(int a) { return a + 1; }  // one\n/* two */ const char* s = "x // y /* z */";\n'
    same = '/* moved */ int  f(int a)\n{\n    return a + 1;   // other words\n}\nconst char* s = "x // y /* z */";'
    assert bench._code_only(base) == bench._code_only(same)
    assert bench._code_only(base) != bench._code_only(base.replace("a + 1", "a + 2"))
    assert bench._code_only(base) != bench._code_only(base.replace('"x // y', '"x / y'))
    assert "//" in bench._code_only(base) and "one" not in bench._code_only(base)
    assert len(bench.source_digest()) == 16
