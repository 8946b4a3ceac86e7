"""CPU checks of two exactness arguments the CUDA path relies on.

Both kernels decide in FP32 first and fall back to FP64 where FP32 cannot
decide, so that every decision is the one the FP64 arithmetic of the method
takes.  These tests check the arguments with float32 models of the rules
(numpy rounds every float32 operation), on random inputs:

* the film probe's density test rho < mid: the FP32 sum of the eighteen
  terms w_i rho_ref and g_i lies within 20 u sum|terms| of the FP64 sum
  (u = 2^-24), so a band of 4e-6 sum|terms| around mid is wide enough;
* the seeding kernel's brick rule: with c the brick's centre, h its
  half-diagonal and d_c the smallest FP32 signed distance from c to a
  bubble, every bubble that a cell of the brick re-evaluates in FP64 (those
  within 1e-3 of the cell's FP32 minimum) has
  d_c(b) - (d_c + 2h) <= 0.05 + 1e-6 (|d_c(b)| + r_b + |d_c + 2h|).
"""
import numpy as np

F32 = np.float32
W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def test_fp32_density_band_covers_the_fp64_sum():
    rng = np.random.default_rng(11)
    n = 200_000
    rho_ref = rng.choice([1.0, 2.0, 2.7], n)
    # offsets g_i of liquid, gas and interface cells, and some large ones
    scale = rng.choice([1e-3, 0.1, 1.0, 30.0], n)
    g = (rng.normal(0, 1, (n, 9)) * scale[:, None]).astype(F32)
    wr64 = W9[None, :] * rho_ref[:, None]
    rho64 = np.zeros(n)
    for i in range(9):  # the FP64 accessor: sum of (w_i rho_ref + g_i) in order
        rho64 = rho64 + (wr64[:, i] + g[:, i].astype(np.float64))
    t = W9.astype(F32)[None, :] * rho_ref.astype(F32)[:, None]  # rounded products
    r = np.zeros(n, F32)
    s = np.zeros(n, F32)
    for i in range(9):
        r = (r + (t[:, i] + g[:, i])).astype(F32)
        s = (s + (np.abs(t[:, i]) + np.abs(g[:, i]))).astype(F32)
    err = np.abs(r.astype(np.float64) - rho64)
    bound = 20 * 2.0 ** -24 * s.astype(np.float64)
    assert (err <= bound).all(), float((err / bound).max())
    # the band the kernel uses is wider than the bound, so outside it the
    # FP32 sign of rho - mid is the FP64 sign
    assert (4e-6 * s.astype(np.float64) >= 3 * bound).all()


def _mi(d, n):
    d = np.fmod(d, n).astype(F32)
    d = np.where(d < 0, (d + n).astype(F32), d)
    return np.where(d > F32(0.5) * n, (d - n).astype(F32), d).astype(F32)


def _dist(p, B, n):
    dx = _mi(F32(p[0]) - B[:, 0], n[0])
    dy = _mi(F32(p[1]) - B[:, 1], n[1])
    dz = _mi(F32(p[2]) - B[:, 2], n[2])
    return (np.sqrt((dx * dx + dy * dy + dz * dz).astype(F32)) - B[:, 3]).astype(F32)


def test_seeding_brick_candidates_hold_every_reevaluated_bubble():
    rng = np.random.default_rng(5)
    for trial in range(8):
        d3 = trial % 2 == 0
        if d3:
            (NX, NY, NZ), (bx, by, bz) = rng.integers(9, 30, 3), (8, 8, 8)
        else:
            (NX, NZ), NY, (bx, by, bz) = rng.integers(17, 60, 2), 1, (16, 1, 16)
        nb = int(rng.integers(2, 150))
        B = np.stack([rng.uniform(0, NX, nb), rng.uniform(0, NY, nb) if NY > 1 else np.zeros(nb),
                      rng.uniform(0, NZ, nb), rng.uniform(0.5, 9, nb)], 1)
        if trial % 4 == 1:  # half-integer centres and equal radii: exact ties
            B[:, :3] = np.round(B[:, :3] * 2) / 2
            B[:, 3] = 3.0
        Bf = B.astype(F32)
        n = (F32(NX), F32(NY), F32(NZ))
        for z0 in range(0, NZ, bz):
            for y0 in range(0, NY, by):
                for x0 in range(0, NX, bx):
                    ex, ey, ez = min(bx, NX - x0), min(by, NY - y0), min(bz, NZ - z0)
                    c = (F32(x0) + F32(0.5) * F32(ex - 1), F32(y0) + F32(0.5) * F32(ey - 1),
                         F32(z0) + F32(0.5) * F32(ez - 1))
                    h = F32(0.5) * np.sqrt(F32((ex - 1) ** 2 + (ey - 1) ** 2 + (ez - 1) ** 2))
                    dc = _dist(c, Bf, n)
                    t0 = F32(dc.min() + F32(2) * h)
                    keep = (dc - t0) <= F32(0.05) + F32(1e-6) * (np.abs(dc) + np.abs(Bf[:, 3]) +
                                                               abs(t0))
                    for z in range(z0, z0 + ez):
                        for y in range(y0, y0 + ey):
                            for x in range(x0, x0 + ex):
                                d = _dist((x, y, z), Bf, n)
                                need = d <= d.min() + F32(1e-3)
                                assert not (need & ~keep).any(), (trial, x, y, z)
