"""Seeded synthetic workloads (parameters only, no arithmetic of the method).

The paper reports no grid sizes or run lengths; these recipes stand in for
its two-bubble runs (Sec. 4, Fig. 2), its bubble-size sweep (Fig. 3) and its
foam runs.  Each recipe lists the lattice, the physical parameters, how the
bubbles are placed (explicit centres, or random nucleation sites drawn with
the library's / the oracle's SplitMix64 sampler from the given seed), the
blowing-agent rates and the reference density of the offset storage (the
liquid density, where most cells sit).  Both the CUDA path and the CPU oracle read these
dictionaries; neither imports the other.
"""
from __future__ import annotations

# two gas disks r = 20 separated by a 4-cell liquid gap on 128^2 (D2Q9, FP64)
TWO_DISKS_128 = dict(
    name="d2q9_two_disks_128", lattice="D2Q9", nx=128, ny=128, nz=1, tau=1.0, G=-5.0,
    rho0=1.0, storage="f64", rho_l=2.0, rho_g=0.15, width=2.0, noise=1e-3, seed=0,
    bubbles=[[42.0, 64.0, 0.0, 20.0], [86.0, 64.0, 0.0, 20.0]], steps=5000,
    gap_line=(0, 64, 0, 0, 128), threshold=1.0)

# 64 nucleation sites, spheres r = 3, injection 1e-4/step, budget 50 (D3Q19)
FOAM_128 = dict(
    name="d3q19_foam_128", lattice="D3Q19", nx=128, ny=128, nz=128, tau=1.0, G=-5.0,
    rho0=1.0, storage="f32", rho_l=2.0, rho_g=0.15, width=2.0, noise=1e-3, seed=1,
    sites=dict(n=64, r_min=3.0, r_max=3.0, min_spacing=12.0, min_gap=0.0),
    rate=1e-4, budget=50.0, steps=20000, diag_every=100, threshold=1.0, rho_ref=2.0)

# 1000 bubbles r ~ U(4, 12) on 512^3, tau 0.8.  The liquid starts at 1.80,
# not at the nominal 2.0: in a closed periodic box a bubble of radius R holds
# only while the liquid sits below the flat-interface coexistence density
# (1.93 at G = -5) by about 2 sigma / R, since no reservoir absorbs what the
# Laplace pressure pushes into the liquid.  With 1.9 % of the volume in gas,
# the FP64 oracle dissolves these bubbles within 100 steps at 2.0 and at 1.93
# and keeps them over 800 steps at 1.80 (64^3, the same recipe).  The offset
# storage's reference density is that liquid density.
FOAM_512 = dict(
    name="d3q19_foam_512", lattice="D3Q19", nx=512, ny=512, nz=512, tau=0.8, G=-5.0,
    rho0=1.0, storage="f32", rho_l=1.8, rho_g=0.15, width=2.0, noise=1e-3, seed=2,
    sites=dict(n=1000, r_min=4.0, r_max=12.0, min_spacing=0.0, min_gap=4.0),
    rate=0.0, budget=0.0, steps=2000, rho_ref=1.8, threshold=1.0)

# full foam, 4096 sites, FP16-offset storage (768^3); the per-cell rounding
# residual keeps the blowing agent's sub-quantum deposits (mass_residual)
FOAM_768 = dict(
    name="d3q19_foam_768", lattice="D3Q19", nx=768, ny=768, nz=768, tau=0.9, G=-5.0,
    rho0=1.0, storage="f16", rho_l=2.0, rho_g=0.15, width=2.0, noise=1e-3, seed=4,
    sites=dict(n=4096, r_min=3.0, r_max=3.0, min_spacing=12.0, min_gap=0.0),
    rate=5e-5, budget=(20.0, 80.0), steps=50000, diag_every=100, rho_ref=2.0, threshold=1.0,
    mass_residual=True)

# 256 independent two-bubble D2Q9 domains (FP32): side log-uniform 64..512
# (rounded to multiples of 8), gap U(2, 10), radius U(8, min(60, (L - 2 gap)/4
# - 2)) so that the gap around the periodic wrap is no smaller, tau U(0.6,
# 1.0), G = -5; run until the rupture criterion fires or 20000 steps
ENSEMBLE_256 = dict(
    name="d2q9_ensemble_256", n=256, side=(64, 512), gap=(2.0, 10.0), radius=(8.0, 60.0),
    tau=(0.6, 1.0), G=-5.0, rho0=1.0, rho_ref=2.0, rho_l=2.0, rho_g=0.15, width=2.0,
    noise=1e-3, seed=3, steps=20000, diag_every=20, eps_arm=1e-3, h_max=8.0)

# nine bubble sizes (Sec. 4, Fig. 3: simulations for 9 bubble sizes), two
# D2Q9 disks of radius R_b at a 4-cell liquid gap on a periodic square of
# side 4 R_b + 24 rounded up to a multiple of 8; run in the multi-lattice
# model (fluid + one gas lattice per bubble, gas 0.05 inside each bubble,
# fluid-gas coupling G_x, barrier G_b) and in the single-component model,
# until the rupture criterion fires or the film is gone
ML_SWEEP_9 = dict(
    name="d2q9_ml_sweep_9", radii=(8.0, 11.0, 14.0, 17.0, 20.0, 24.0, 28.0, 33.0, 38.0),
    gap=4.0, tau=1.0, G=-5.0, G_x=1.0, G_b=2.0, rho0=1.0, rho_l=2.0, rho_v=0.15, rho_gas=0.05,
    width=2.0, noise=1e-4, seed=9, steps=20000, diag_every=20, eps_arm=1e-3, h_max=8.0)

WORKLOADS = {w["name"]: w for w in (TWO_DISKS_128, FOAM_128, FOAM_512, FOAM_768, ENSEMBLE_256,
                                    ML_SWEEP_9)}


def ml_sweep_domains(recipe=ML_SWEEP_9):
    """The domains of the nine-size sweep: dicts with side L, the two disks
    (x, y, 0, R) on the middle row and the probe line from centre to
    centre."""
    import math
    out = []
    for R in recipe["radii"]:
        L = int(math.ceil((4 * R + 24) / 8.0)) * 8
        c1 = L / 2 - R - recipe["gap"] / 2
        c2 = L / 2 + R + recipe["gap"] / 2
        x0 = int(math.floor(c1))
        out.append(dict(L=L, R=R, bubbles=[(c1, L / 2, 0.0, R), (c2, L / 2, 0.0, R)],
                        line=(x0, L // 2, 0, 0, int(math.ceil(c2)) - x0 + 1)))
    return out


def ensemble_domains(recipe=ENSEMBLE_256, n=None, side=None):
    """Draw the domain list of an ensemble recipe (numpy generator seeded with
    recipe['seed']): dicts with the fields of lbm_domain.  Two gas disks of
    radius R sit on the middle row at a surface-to-surface distance `gap`;
    the film probe line runs from one centre to the other."""
    import numpy as np
    rng = np.random.default_rng(recipe["seed"])
    n = recipe["n"] if n is None else n
    lo, hi = recipe["side"] if side is None else side
    out = []
    for k in range(n):
        L = int(round(np.exp(rng.uniform(np.log(lo), np.log(hi))) / 8.0)) * 8
        gap = float(rng.uniform(*recipe["gap"]))
        rmax = min(recipe["radius"][1], (L - 2 * gap) / 4 - 2)
        R = float(rng.uniform(recipe["radius"][0], max(recipe["radius"][0], rmax)))
        tau = float(rng.uniform(*recipe["tau"]))
        yc = L // 2
        c1 = L / 2 - R - gap / 2
        c2 = L / 2 + R + gap / 2
        x0 = int(np.floor(c1))
        out.append(dict(
            nx=L, ny=L, tau=tau, G=recipe["G"], rho0=recipe["rho0"], rho_ref=recipe["rho_ref"],
            rho_l=recipe["rho_l"], rho_g=recipe["rho_g"], width=recipe["width"],
            noise_amp=recipe["noise"], seed=recipe["seed"] * 100003 + k,
            bubbles=[(c1, float(yc), 0.0, R), (c2, float(yc), 0.0, R)],
            line=(x0, yc, 0, 0, int(np.ceil(c2)) - x0 + 1),
            rho_mid=0.5 * (recipe["rho_l"] + recipe["rho_g"]), R=R, gap=gap))
    return out
