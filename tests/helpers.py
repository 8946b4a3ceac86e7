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
