"""The benchmark's reference arm (the oracle on the host cores) and its JSON line: every
key the line must carry, with the oracle's matvec counted by the planner's flops.  Runs
on the CPU only (the reference arm never touches the GPU)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["unit"] == "GFLOP/s" and d["value"] > 0
    assert d["steps"] == 1 and d["warmup"] == 0 and d["n_gpus"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "GFLOP/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert "workload" in d["config"] and "sample" in d["config"]


def _bench():
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench
    return bench


class _Ctx:
    """Stands in for a context: records the sites and directions the walker steps."""

    def __init__(self):
        self.steps, self.hints = [], []

    def set_next_site(self, s):
        self.hints.append(s)

    def sweep_step(self, site, direction, D):
        self.steps.append((site, direction))
        return 0.0, 0.0, 1, True


def test_walker_sweeps_the_window_both_ways():
    """The timed steps' sweep window: each step's site is the neighbour of the last one in
    the current direction, the sweep turns at both ends (the same site twice, as a
    macro-iteration does, Sec. 4.2), and every step announces the next one's site."""
    bench = _bench()
    lo, hi = bench.window(13)
    assert (lo, hi) == (8, 17)
    w, ctx = bench.Walker(lo, hi), _Ctx()
    for _ in range(2 * (hi - lo + 1) + 3):
        w.step(ctx, 100)
    right = [(s, 1) for s in range(lo, hi + 1)]
    left = [(s, -1) for s in range(hi, lo - 1, -1)]
    expect = (right + left + right)[:len(ctx.steps)]
    assert ctx.steps == expect
    assert ctx.hints == [s for s, _ in ctx.steps[1:]] + [w.site]


def test_recorded_traffic_belongs_to_the_current_kernel():
    """roofline.traffic comes from NCU_TRAFFIC only for the kernel code it was measured on:
    the recorded entry's key is the current code hash (comments and blank space left out,
    so a comment edit keeps it and a code edit turns the figure into null)."""
    bench = _bench()
    h = bench.kernel_source_hash()
    assert any(k[1] == h for k in bench.NCU_TRAFFIC), (h, list(bench.NCU_TRAFFIC))
    path = os.path.join(ROOT, "paper_1312_2415_gb300", "csrc", "kernels_tc.cu")
    src = open(path).read()
    import hashlib
    import re
    def code_hash(text):
        code = re.sub(r"\s+", " ", re.sub(r"//[^\n]*", "", text))
        return hashlib.sha256(code.encode()).hexdigest()[:16]
    assert code_hash(src) == h
    assert code_hash(src + "\n// a comment\n") == h
    assert code_hash(src + "\nint x;\n") != h
