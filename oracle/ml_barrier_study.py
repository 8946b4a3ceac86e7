"""Does the multi-lattice reading of the modified Shan-Chen model form a
barrier film?  (Sec. 3.1: each bubble on its own lattice, coupled through
the fluid; with eta_m = 1 the paper reports a film that does not rupture.)

Part of the FP64 oracle (test infrastructure): runs the two-disk case of the
configs (D2Q9 128^2, disks r = 20 with a 4-cell liquid gap, tau 1, G -5,
liquid 2.0, the fluid's vapour 0.15 inside the disks, no noise) on the
oracle's multi-lattice step with the barrier never switched off, and reports
the step at which the liquid film between the disks is gone (the fluid
density at the midpoint of the centre line below 1.0), next to the
single-component model.  Usage: python -m oracle.ml_barrier_study [steps]
"""
from __future__ import annotations

import sys
import time

import numpy as np

import oracle as O

N, R, GAP, TAU, G = 128, 20.0, 4.0, 1.0, -5.0


def rupture_step(nl, Gm, rho_gas, steps, every=50):
    c1, c2 = N / 2 - R - GAP / 2, N / 2 + R + GAP / 2
    b = np.array([[c1, N / 2, 0, R], [c2, N / 2, 0, R]])
    if nl == 1:
        f = O.init(O.D2Q9, N, N, 1, b, 2.0, 0.15, 2.0, 0.0, 0)[0][None]
    else:
        f = O.ml_init(O.D2Q9, N, N, 1, b, 2.0, 0.15, rho_gas, 2.0, 0.0, 0)
    t = 0
    while t < steps:
        f = O.ml_run(O.D2Q9, f, every, TAU, Gm)
        t += every
        rho = O.ml_moments(O.D2Q9, f)[0]
        if not np.isfinite(rho).all():
            return t, "non-finite"
        if rho[0, 0, N // 2, N // 2] < 1.0:
            return t, "film gone"
    return t, "film holds"


def main():
    steps = int(sys.argv[1]) if len(sys.argv) > 1 else 5000
    rows = [("single-component Shan-Chen (the hot path)", 1, np.array([[G]]), 0.0)]
    for gx in (0.5, 1.0, 2.0):
        for gb in (0.0, 2.0, 5.0, 20.0):
            for rg in (0.05, 0.15):
                rows.append((f"G_x {gx}, G_b {gb}, gas {rg}", 3, O.ml_coupling(3, G, gx, gb), rg))
    print(f"two disks r = {R:g}, gap {GAP:g}, {N}^2, tau {TAU:g}, G {G:g}, {steps} steps max")
    for name, nl, Gm, rg in rows:
        t0 = time.perf_counter()
        step, what = rupture_step(nl, Gm, rg, steps)
        print(f"{name:45s} {what:11s} at step {step:5d}  ({time.perf_counter() - t0:.0f} s)",
              flush=True)


if __name__ == "__main__":
    main()
