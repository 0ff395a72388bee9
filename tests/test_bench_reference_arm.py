"""bench.py's reference arm (the FP64 oracle on the host cores) on the small 20^3
workload: the JSON line carries the keys the measurement contract names, and a
rank other than 0 exits without work.  CPU only."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CMD = [sys.executable, "bench.py", "--impl", "reference", "--workload", "g20_w2_n64_m10", "--steps", "1",
       "--warmup", "1", "--cpu-cols", "8"]


def _run(env_extra):
    env = dict(os.environ)
    env.update(env_extra)
    return subprocess.run(CMD, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_json_line():
    p = _run({"RANK": "0"})
    assert p.returncode == 0, p.stderr[-2000:]
    line = json.loads(p.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["unit"] == "GFLOP/s" and line["higher_is_better"] is True
    assert line["value"] > 0 and line["ms_per_step"] > 0
    assert line["config"]["workload"] == "g20_w2_n64_m10"
    assert line["config"]["N"] == 8000 and line["config"]["m"] == 10
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "GFLOP/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_do_no_work():
    p = _run({"RANK": "1"})
    assert p.returncode == 0, p.stderr[-2000:]
    assert p.stdout.strip() == ""


def test_bench_uses_only_exported_binding_names():
    """Every P.<name> that bench.py calls exists in the package (a host check that
    catches a missing export before a GPU run)."""
    import re
    import paper_2110_15853_gb300 as P
    src = open(os.path.join(ROOT, "bench.py")).read()
    names = set(re.findall(r"\bP\.([A-Za-z_]+)", src))
    assert names and not [n for n in names if not hasattr(P, n)]


def test_flop_model_counts():
    """The algorithmic FLOP counts behind `value` and the closure rate, counted again
    product by product: one step 2 nnz n + 5 N n (3 N n for the first); CholQR2 with the
    last pass's X_F folded away: two symmetric Grams (N n^2 each), one triangular
    product (N n^2), the n^3 fold products (P R2^-1 and R2^-1 Q, n^3 each; the upper
    triangle of R2^-T T, n^3 / 3), H X_F (2 nnz n), the symmetric projection (N n^2) and
    the rotation (2 N n^2); the Ozaki schedules' slice products per element and state."""
    sys.path.insert(0, ROOT)
    import bench
    nnz, N, n = 171879616, 262144, 6000
    assert bench.filter_flops(nnz, N, n, 1) == 2 * nnz * n + 3 * N * n
    assert bench.filter_flops(nnz, N, n, 30) == 30 * 2 * nnz * n + 3 * N * n + 29 * 5 * N * n
    gram, tri, proj, rot = N * n * n, N * n * n, N * n * n, 2 * N * n * n
    fold = n ** 3 + n ** 3 + n ** 3 / 3
    assert abs(bench.closure_flops(nnz, N, n, 2) - (2 * gram + tri + fold + 2 * nnz * n + proj + rot)) < 1e-6 * gram
    assert abs(bench.closure_flops(nnz, N, n, 1) - (gram + tri + 2 * nnz * n + proj + rot)) < 1e-6 * gram
    s = bench.ozaki_schedules(30)
    assert s["ozaki"] == ["ozaki"] * 30
    assert s["ozaki40_prefix"] == ["ozaki40"] * 26 + ["ozaki"] * 4
    assert bench.slice_products(s["ozaki"]) == 30 * 28
    assert bench.slice_products(s["ozaki40_prefix"]) == 26 * 15 + 4 * 28
