"""Writes the stored oracle histories used by the GPU physics tests.

Every value comes from the FP64 oracle (oracle/pic_oracle.py) run on the
seeded generators of pic_inputs.py; nothing here calls the CUDA path.

  landau_32x32x32_ppc64_history.json
      Weak Landau damping (Section 4.1, Eq. landau_f: alpha = 0.05, k = 0.5,
      L = 4 pi, dt = 0.05) on a 32^3 grid with 64 particles per cell
      (2,097,152 particles, pic_inputs.landau seed 1001), 200 steps: the
      (1,0,0) mode of E_x and W_x per step.  About 10 minutes.
  landau_lattice_1d_history.json
      The same physics on a quiet 1D phase-space lattice (128 cells, 128 x 2048
      particles, 200 steps): the noise-free reference for the damping rate
      fitted at scale.
  bump_on_tail_quiet_1d_history.json
      Bump-on-tail (Section 4.2 family; 0.9 N(0,1) + 0.1 N(4, 0.3^2)) on
      L = 20 pi seeded at k = 0.3 (mode 3) with alpha = 1e-3, on a quiet 1D
      lattice with the resolution of the 64^3 benchmark grid (64 cells,
      256 x 512 particles, 400 steps).  About a minute.

  two_stream_quiet_1d_history.json
      The symmetric two-stream instability (Section 4.2, Eq. twostream_f:
      beams at v_z = -pi/2 and +pi/2, spread 0.1, k = 0.5) seeded with
      alpha = 1e-3 on a quiet 1D lattice (32 cells, 64 x 512 particles,
      400 steps).
  strong_landau_16_history.json
      Strong Landau damping (Section 4.1 with alpha = 0.5; Section 5.3) on a
      16^3 grid with 16 particles per cell (65,536 particles), 200 steps.

    python tests/golden/make_physics_goldens.py [name ...]
"""
import json
import math
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import pic_inputs as pi  # noqa: E402
from oracle import pic_oracle as po  # noqa: E402


def _run(w, n_steps):
    g = po.Grid(w.n, w.L)
    p = po.Params(dt=w.dt, Q=w.Q, q_over_m=w.q_over_m)
    _, _, hist = po.run(w.x, w.v, g, p, n_steps, mode=w.mode, mode_comp=w.mode_comp)
    return {"t_field": [d["t_field"] for d in hist],
            "mode": [[d["mode"].real, d["mode"].imag] for d in hist],
            "Wx": [d["Wx"] for d in hist], "Wz": [d["Wz"] for d in hist],
            "Q": [d["Q"] for d in hist]}


def landau_32():
    w = pi.landau(n=32, ppc=64, seed=1001)
    return {"workload": "pic_inputs.landau(n=32, ppc=64, seed=1001)", "n_steps": 200,
            **_run(w, 200)}


def landau_lattice():
    w = pi.landau_lattice_1d(nx=128, mx=128, mv=2048, alpha=0.05, k=0.5, n_steps=200)
    return {"workload": "pic_inputs.landau_lattice_1d(nx=128, mx=128, mv=2048, alpha=0.05)",
            "n_steps": 200, **_run(w, 200)}


def bump_on_tail_quiet():
    w = bump_on_tail_quiet_1d()
    return {"workload": "pic_inputs.bump_on_tail_quiet(n=(64,1,1), L=20 pi, axis=0, m=3, "
                        "alpha=1e-3, ms=256, mv=512)", "n_steps": 400, **_run(w, 400)}


def bump_on_tail_quiet_1d():
    """The input of bump_on_tail_quiet_1d_history.json (also run by the GPU test)."""
    return pi.bump_on_tail_quiet(n=(64, 1, 1), L=20.0 * math.pi, axis=0, m=3, alpha=1e-3,
                                 ms=256, mv=512)


def two_stream_quiet_1d():
    """The input of two_stream_quiet_1d_history.json (also run by the GPU test)."""
    return pi.bump_on_tail_quiet(n=(32, 1, 1), L=4.0 * math.pi, axis=0, m=1, alpha=1e-3, ms=64,
                                 mv=512, eps=0.5, v_beam=0.5 * math.pi, sigma_beam=0.1,
                                 sigma_bulk=0.1, u_bulk=-0.5 * math.pi)


def two_stream_quiet():
    w = two_stream_quiet_1d()
    return {"workload": "pic_inputs.bump_on_tail_quiet(n=(32,1,1), L=4 pi, axis=0, m=1, alpha=1e-3, "
                        "ms=64, mv=512, eps=0.5, v_beam=pi/2, sigma_beam=0.1, sigma_bulk=0.1, "
                        "u_bulk=-pi/2)", "n_steps": 400, **_run(w, 400)}


def strong_landau_16():
    w = pi.landau(n=16, ppc=16, alpha=0.5, seed=1007)
    return {"workload": "pic_inputs.landau(n=16, ppc=16, alpha=0.5, seed=1007)", "n_steps": 200,
            **_run(w, 200)}


TABLE = {
    "landau_32x32x32_ppc64_history.json": landau_32,
    "landau_lattice_1d_history.json": landau_lattice,
    "bump_on_tail_quiet_1d_history.json": bump_on_tail_quiet,
    "two_stream_quiet_1d_history.json": two_stream_quiet,
    "strong_landau_16_history.json": strong_landau_16,
}

if __name__ == "__main__":
    names = sys.argv[1:] or list(TABLE)
    for name in names:
        t0 = time.time()
        out = TABLE[name]()
        with open(os.path.join(HERE, name), "w") as f:
            json.dump(out, f)
        print(f"{name}: {time.time() - t0:.1f} s", flush=True)
