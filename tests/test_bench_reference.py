"""The benchmark's reference arm times the FP64 oracle on the host cores and
needs no GPU: its JSON line carries the keys of the benchmark line, with the
copy counts of a host-only run."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

KEYS = ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
        "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline",
        "e2e")


def test_reference_arm_prints_one_contract_line():
    run = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                          "--warmup", "3"], cwd=ROOT, capture_output=True, text=True,
                         timeout=900)
    assert run.returncode == 0, run.stderr[-2000:]
    lines = [x for x in run.stdout.splitlines() if x.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for k in KEYS:
        assert k in line, k
    assert line["impl"] == "reference"
    assert line["value"] > 0 and line["steps"] == 1 and line["warmup"] == 3
    assert line["higher_is_better"] is True and line["dtype"] == "f64"
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"],
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_kernel_hash_follows_code_not_comments():
    # the committed DRAM figures are tied to the kernel code by a hash that
    # leaves comments out: a comment edit keeps them, a code edit voids them
    sys.path.insert(0, ROOT)
    import bench

    code = 'int f(int x) {  // twice x\n    /* a "block" comment */\n    return 2 * x;\n}\n'
    assert bench._code_only(code) == "int f(int x) {\n    return 2 * x;\n}"
    assert bench._code_only(code.replace("twice", "double")) == bench._code_only(code)
    assert bench._code_only(code.replace("2 * x", "3 * x")) != bench._code_only(code)
    # a comment marker inside a string literal is code
    assert bench._code_only('const char* s = "a // b";') == 'const char* s = "a // b";'
    prof = bench._dram_profile()
    assert prof is not None and len(prof["kernel_sha"]) == 16
