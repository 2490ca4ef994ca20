"""The benchmark's reference arm on CPU: `bench.py --impl reference` times
the oracle on a bounded sample and prints one JSON line with the keys of the
benchmark contract (no GPU needed)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run(
        [sys.executable, "bench.py", "--impl", "reference", "--steps", "3", "--warmup", "3",
         "--grid", "16", "--ppc", "8", "--cpu-sample", "4096"],
        cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config"):
        assert k in d, k
    assert d["value"] > 0 and d["steps"] == 3 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["higher_is_better"] is True and d["unit"] == "particle-steps/s"
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_all_core_oracle_driver_reproduces_the_oracle_step():
    """The all-core CPU baseline drives the oracle's own functions over
    particle chunks; its state after two steps equals po.run's."""
    import numpy as np

    sys.path.insert(0, ROOT)
    import bench
    import pic_inputs as pi
    from oracle import pic_oracle as po

    w = pi.penning(n=8, n_particles=3000, L=20.0, seed=9)
    val, secs, (x, v) = bench.time_oracle_parallel(w, 2, 2, return_state=True)
    assert val > 0 and secs > 0
    xo, vo, _ = po.run(w.x, w.v, po.Grid(w.n, w.L),
                       po.Params(dt=w.dt, q_over_m=w.q_over_m, Q=w.Q, B=w.B, wz2=w.wz2), 2)
    assert np.max(np.abs(x - xo)) < 1e-12 and np.max(np.abs(v - vo)) < 1e-12


def test_cpu_configuration_figures_report_both_oracle_timings():
    """The per-configuration CPU baseline times the oracle single-threaded and
    over a process pool on each configuration it is given."""
    sys.path.insert(0, ROOT)
    import bench

    tiny = [("landau 8^3 x 2", lambda pi: pi.landau(n=8, ppc=2, seed=5), 1),
            ("penning 8^3, 1000 particles",
             lambda pi: pi.penning(n=8, n_particles=1000, L=20.0, seed=6), 1)]
    out = bench.cpu_config_figures(2, tiny)
    assert [e["config"] for e in out] == [c[0] for c in tiny]
    for e in out:
        assert e["steps"] == 1 and e["single"] > 0 and e["all_cores"] > 0
