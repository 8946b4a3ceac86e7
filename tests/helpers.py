"""Shared helpers of the test-suite: build the library, run both sides."""
import numpy as np

import oracle as O

LAT = {"D2Q9": O.D2Q9, "D3Q19": O.D3Q19}


def lbm_mod():
    from paper_1708_01608_gb300 import build_lib
    build_lib.build()
    from paper_1708_01608_gb300 import lbm
    return lbm


def rel_err(a, b):
    """max |a - b| / max |b|"""
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300))


def site_cells(lat_name, bubbles, nx, ny, nz):
    """Linear cell of each bubble centre rounded to the nearest cell."""
    b = np.asarray(bubbles, dtype=float).reshape(-1, 4)
    x = np.floor(b[:, 0] + 0.5).astype(np.int64) % nx
    y = np.floor(b[:, 1] + 0.5).astype(np.int64) % ny
    z = np.floor(b[:, 2] + 0.5).astype(np.int64) % nz
    return x + nx * (y + ny * z)


def _bf16(x32):
    """float32 -> bfloat16 (round to nearest, ties to even) -> float32."""
    u = np.ascontiguousarray(x32, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def as_stored(lat_name, f, storage, rho_ref):
    """The populations a lattice of this storage holds after write_f(f), as
    FP64: offset storages keep g = f - w rho_ref rounded to FP32 (then to
    FP16 / BF16), FP64 keeps f.  Used to hand the oracle and the GPU the same
    seeded input."""
    f = np.asarray(f, dtype=np.float64)
    if storage == "f64":
        return f.copy()
    _, w = O.velocities(LAT[lat_name])
    wr = (w * rho_ref).reshape((-1,) + (1,) * (f.ndim - 1))
    g = (f - wr).astype(np.float32)
    if storage == "f16":
        g = g.astype(np.float16).astype(np.float32)
    elif storage == "bf16":
        g = _bf16(g)
    return wr + g.astype(np.float64)


def oracle_init(lat_name, nx, ny, nz, bubbles, rho_l, rho_g, width, noise, seed):
    """Seeded initial populations (FP64) from the oracle's initialiser."""
    b = np.asarray(bubbles, dtype=float).reshape(-1, 4)
    f, _ = O.init(LAT[lat_name], nx, ny, nz, b, rho_l, rho_g, width, noise, seed)
    return f
