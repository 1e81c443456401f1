"""The benchmark's reference arm (the FP64 oracle on the host cores) runs without a GPU and prints one JSON
line with the contract's keys.  CPU only."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    # the 32^3 workload keeps this CPU test short; the default (64^3) takes the same code path
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "1", "--workload", "batch32"], cwd=ROOT, capture_output=True, text=True,
                         timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert "workload" in d["config"]


def test_default_workload_is_the_precision_form():
    """Without flags the bench measures the largest single-GPU configuration: 4096 x 64^3, l <= 32, marching
    4-8-16-32, 32 starts, with the FP64 re-score of the best starts."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2509_01180_gb300 import synth
    assert bench.HEADLINE == "precision64"
    N, Lmax, _, _, _, _, stages, steps, S, B = synth.CONFIGS[bench.HEADLINE]
    assert (N, Lmax, stages, steps, S, B) == (64, 32, [4, 8, 16, 32], 30, 32, 4096)
    # flop accounting: one evaluation at band L costs 30 flop per orbit-step and 46 per orbit
    assert bench.orbit_steps(32) == 12529 and bench.eval_flops(4) == 30 * 55 + 46 * 25


def test_source_hash_ignores_comments_only():
    """The stored ascent traffic figure is keyed on the alignment source without comments: a comment or
    blank-line edit keeps the key, a code edit changes it (the bench then reports no traffic)."""
    sys.path.insert(0, ROOT)
    import bench
    code = "int f(int x) {\n  return x + 1;  // one more\n}\n"
    assert bench.source_sha(code) == bench.source_sha("/* doc */\nint f(int x) {\n\n  return x + 1;\n}\n")
    assert bench.source_sha(code) != bench.source_sha(code.replace("x + 1", "x + 2"))
