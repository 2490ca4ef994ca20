"""Writes the stored oracle gradients of the 200-step bump-on-tail adjoint test.

Every value comes from the FP64 oracle (oracle/pic_oracle.py) run on the
seeded generators of pic_inputs.py; nothing here calls the CUDA path.

  bump_on_tail_16_adjoint_200.json
      The bump-on-tail adjoint workload's settings (velocities 0.9 N(0,1) +
      0.1 N(4, 0.3^2) along z, N(0,1) across, density 1 + 0.05 cos(k z),
      dt = 0.05, 200 steps, objective W_z of the field of the last step) on a
      grid the oracle reverses in about a minute: 16^3 cells with 16
      particles per cell (65,536 particles), k = 0.4, so the cell size
      (L / 16 = 0.98) is that of the 64^3 workload.  Stored: J; dJ/dalpha
      from the oracle's discrete adjoint (through the input sampler's
      Jacobian) and from central differences of J over re-sampled inputs
      (alpha +- 1e-6, fixed uniforms); dJ/dx0 and dJ/dv0 of 512 particles
      drawn with a fixed seed, with the largest |component| of each over all
      particles.  About three minutes.

    python tests/golden/make_adjoint_goldens.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import pic_inputs as pi  # noqa: E402
from oracle import pic_oracle as po  # noqa: E402

SETUP = dict(n=16, ppc=16, seed=1013, alpha=0.05, k=0.4)
N_STEPS = 200
WEIGHTS = (0.0, 0.0, 1.0)
EPS_ALPHA = 1e-6
N_SAMPLE = 512


def main():
    t0 = time.time()
    w = pi.bump_on_tail(**SETUP)
    g = po.Grid(w.n, w.L)
    p = po.Params(dt=w.dt, Q=w.Q, q_over_m=w.q_over_m)
    J, gx, gv = po.run_with_gradient(w.x, w.v, g, p, N_STEPS, WEIGHTS)
    dxa = po.cosine_sample_dalpha(w.x[:, 2], SETUP["alpha"], SETUP["k"])
    dJ_da_adj = float(np.sum(gx[:, 2] * dxa))
    Js = []
    for s in (+1.0, -1.0):
        ws = pi.bump_on_tail(**dict(SETUP, alpha=SETUP["alpha"] + s * EPS_ALPHA))
        Js.append(po.run_with_gradient(ws.x, ws.v, g, p, N_STEPS, WEIGHTS)[0])
    dJ_da_fd = (Js[0] - Js[1]) / (2.0 * EPS_ALPHA)
    idx = np.sort(np.random.default_rng(77).choice(w.n_particles, N_SAMPLE, replace=False))
    out = {
        "setup": dict(SETUP, dt=w.dt, n_steps=N_STEPS, weights=list(WEIGHTS),
                      n_particles=w.n_particles),
        "J": J,
        "dJ_dalpha_adjoint": dJ_da_adj,
        "dJ_dalpha_central_difference": dJ_da_fd,
        "eps_alpha": EPS_ALPHA,
        "sample": idx.tolist(),
        "gx": gx[idx].tolist(),
        "gv": gv[idx].tolist(),
        "max_abs_gx": float(np.max(np.abs(gx))),
        "max_abs_gv": float(np.max(np.abs(gv))),
    }
    with open(os.path.join(HERE, "bump_on_tail_16_adjoint_200.json"), "w") as f:
        json.dump(out, f)
    print(f"J = {J:.12g}, dJ/dalpha adjoint {dJ_da_adj:.10g}, central difference "
          f"{dJ_da_fd:.10g} ({time.time() - t0:.0f} s)")


if __name__ == "__main__":
    main()
