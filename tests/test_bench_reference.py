"""The CPU-side parts of bench.py: the reference arm (the FP64 oracle timed on
the host cores) prints the one JSON line of the benchmark contract, and the
helpers behind the reported exact-solution errors agree with the oracle's
metrics.  Runs on a CPU with a short time budget."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "3", "--warmup", "1", "--ref-seconds", "1"],
                       capture_output=True, text=True, timeout=300, cwd=ROOT,
                       env=dict(os.environ, WORLD_SIZE="1", RANK="0"))
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["steps"] == 3 and d["warmup"] == 3 and d["value"] > 0  # W is raised to >= 3
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert "3 steps after 3 warm-up" in cb["sample"]
    # the line describes the sub-batch it timed: steps x ms_per_step is the timed
    # region and value is sub-batch points per second
    assert d["config"]["batch"] == cb["sub_batch"] <= d["config"]["workload_batch"]
    assert abs(d["steps"] * d["ms_per_step"] / 1e3 - cb["timed_s"]) <= 1e-9 * cb["timed_s"]
    assert abs(d["value"] - d["steps"] * cb["sub_batch"] / cb["timed_s"]) <= 1e-9 * d["value"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_bench_accuracy_helpers_agree_with_the_oracle_metrics():
    """bench.py reports exact-solution errors with its own numpy helpers; they
    give the oracle's L-inf and RMS over the interior nodes for both
    manufactured pairs."""
    import numpy as np

    import bench
    from oracle import pyoracle as O

    rng = np.random.default_rng(3)
    for sol, exact in ((O.SOL_BENCH, bench.sphere_exact), (O.SOL_SEC41, bench.sec41_exact)):
        pr = O.make_problem(geometry=O.GEOM_SPHERE, solution=sol)
        for n in (8, 16):
            g = -1.0 + np.arange(n + 1) * (2.0 / n)
            Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
            x = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
            u = exact(x) + rng.normal(scale=1e-3, size=len(x))
            linf, rms = bench.node_errors(u, n, exact)
            linf_o, rms_o = O.grid_error(pr, n, u)
            assert abs(linf - linf_o) <= 1e-15 and abs(rms - rms_o) <= 1e-15


def test_bench_trilinear_interpolation_reproduces_multilinear_functions():
    """bench.py's trilinear interpolation of node values (the grid method's
    value between nodes in the gain comparison) is exact for any function
    that is linear in each coordinate, including at the cube's faces."""
    import numpy as np

    import bench

    def f(x, y, z):
        return 0.3 - 1.2 * x + 0.7 * y + 2.0 * z + 0.5 * x * y - 0.25 * y * z + 1.5 * x * y * z

    n = 12
    g = -1.0 + np.arange(n + 1) * (2.0 / n)
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    u = f(X, Y, Z).reshape(-1)
    rng = np.random.default_rng(6)
    pts = np.concatenate([rng.uniform(-1, 1, size=(500, 3)), [[1.0, 1.0, 1.0], [-1.0, 0.2, 1.0]]])
    got = bench.trilinear(u, n, pts)
    assert np.max(np.abs(got - f(pts[:, 0], pts[:, 1], pts[:, 2]))) <= 1e-13
