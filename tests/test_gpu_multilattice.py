"""GPU parity of the multi-lattice Shan-Chen model (Sec. 3.1, Fig. 1: each
bubble and the fluid on their own lattices, coupled through interaction
forces, eta_m merging a pair's lattices) against the FP64 oracle's
orc_ml_step: FP64 within 1e-12 and FP32 within 1e-5 of max|f|, element by
element, from the same seeded state, with the blowing agent on and a merge
in the middle of the run; the on-device rupture criterion fires at the same
step as the oracle's loop with the same h_c."""
import numpy as np
import pytest

import oracle as O
from helpers import LAT, lbm_mod, rel_err

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}


@pytest.fixture(scope="module")
def lbm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return lbm_mod()


def _bubbles(lat, nx, ny, nz):
    if lat == "D2Q9":
        return np.array([[nx * 0.3, ny * 0.5, 0, 6.0], [nx * 0.68, ny * 0.47, 0, 5.0]])
    return np.array([[nx * 0.3, ny * 0.5, nz * 0.5, 4.0], [nx * 0.7, ny * 0.45, nz * 0.4, 3.5]])


@pytest.mark.parametrize("lat,ext,storage,gx,gb", [
    ("D2Q9", (48, 32, 1), "f64", 1.0, 2.0),
    ("D2Q9", (48, 32, 1), "f32", 1.0, 2.0),
    ("D2Q9", (37, 21, 1), "f64", 0.5, 0.0),
    ("D3Q19", (24, 16, 12), "f64", 1.0, 2.0),
    ("D3Q19", (24, 16, 12), "f32", 2.0, 5.0),
    ("D3Q19", (13, 7, 9), "f64", 1.0, 1.0)])
def test_ml_step_parity_with_injection_and_merge(lbm, lat, ext, storage, gx, gb):
    nx, ny, nz = ext
    b = _bubbles(lat, nx, ny, nz)
    M = lbm.MultiLattice(lat, nx, ny, nz, nl=3, tau=0.9, G=-5.0, G_x=gx, G_b=gb, storage=storage)
    M.seed(b, 2.0, 0.15, 0.1, 2.0, 1e-3, 7)           # registers the two sites
    f0 = O.ml_init(LAT[lat], nx, ny, nz, b, 2.0, 0.15, 0.1, 2.0, 1e-3, 7)
    # the library's own seeding gives the oracle's initial state (rounded to
    # the storage)
    if storage == "f32":
        f0 = f0.astype(np.float32).astype(np.float64)
    assert rel_err(M.read_f(), f0) < 1e-15
    Gm = O.ml_coupling(3, -5.0, gx, gb)
    assert np.array_equal(M.coupling(), Gm)
    rate, budget = np.array([2e-3, 1e-3]), np.array([0.05, 0.03])
    M.inject(rate, budget)
    cells = []
    for x, y, z, _ in b:
        X, Y, Z = (int(np.floor(v + 0.5)) for v in (x, y, z))
        cells.append(X % nx + nx * ((Y % ny) + ny * (Z % nz)))
    ob = budget.copy()
    M.step(40)
    fo = O.ml_run(LAT[lat], f0, 40, 0.9, Gm, sites=cells, site_lattice=[1, 2], rate=rate,
                  budget=ob)
    assert rel_err(M.read_f(), fo) < TOL[storage]
    # eta_m = 0 for the pair: the lattices merge and the barrier goes
    M.merge(1, 2)
    fo, Gm2 = O.ml_merge(fo, Gm, 1, 2)
    assert np.array_equal(M.coupling(), Gm2)
    M.step(30)
    fo = O.ml_run(LAT[lat], fo, 30, 0.9, Gm2, sites=cells, site_lattice=[1, 2], rate=rate,
                  budget=ob)
    fg = M.read_f()
    assert rel_err(fg, fo) < TOL[storage], rel_err(fg, fo)
    assert np.abs(M.read_budgets() - ob).max() < 1e-15
    rho, p = M.fields()
    ro = O.ml_moments(LAT[lat], fo)[0]
    assert rel_err(rho, ro) < TOL[storage]
    assert rel_err(p, O.ml_pressure(ro, Gm2)) < 10 * TOL[storage]
    M.close()


def test_ml_single_lattice_equals_the_hot_path(lbm):
    """nl = 1 on the GPU follows the single-component step of lbm_step (the
    FP64 two-pass kernels) to 1e-13."""
    nx, ny = 40, 28
    b = np.array([[12.0, 14.0, 0, 6.0], [29.0, 13.0, 0, 5.0]])
    f0 = O.init(O.D2Q9, nx, ny, 1, b, 2.0, 0.15, 2.0, 1e-3, 3)[0]
    M = lbm.MultiLattice("D2Q9", nx, ny, 1, nl=1, tau=0.8, G=-5.0)
    M.seed(np.zeros((0, 4)), 2.0, 0.15, 0.0, 2.0, 0.0, 3)
    M.write_f(f0[None])
    M.step(100)
    L = lbm.Lattice("D2Q9", nx, ny, 1, tau=0.8, G=-5.0, storage="f64", kernel="two_pass")
    L.seed_bubbles(b, 2.0, 0.15, 2.0, 1e-3, 3)
    L.write_f(f0)
    L.step(100)
    assert rel_err(M.read_f()[0], L.read("f")) < 1e-13
    M.close()
    L.close()


def test_ml_rupture_criterion_matches_the_oracle_loop(lbm):
    """Two disks in the multi-lattice model (FP64): the on-device criterion
    fires at the oracle loop's step with the same interpolated h_c, and the
    merge leaves the same lattices (or both report the film gone first)."""
    n, R, gap = 96, 14.0, 4.0
    c1, c2 = n / 2 - R - gap / 2, n / 2 + R + gap / 2
    b = np.array([[c1, n / 2, 0, R], [c2, n / 2, 0, R]])
    line = (int(np.floor(c1)), n // 2, 0, 0, int(np.ceil(c2)) - int(np.floor(c1)) + 1)
    M = lbm.MultiLattice("D2Q9", n, n, 1, nl=3, tau=1.0, G=-5.0, G_x=1.0, G_b=2.0)
    M.seed(b, 2.0, 0.15, 0.05, 2.0, 0.0, 1)
    f0 = M.read_f()
    r = M.run_until_rupture(line, 1.075, 1e-3, 20, 3000, h_max=8.0)
    o = O.ml_run_until_rupture(O.D2Q9, f0, 1.0, O.ml_coupling(3, -5.0, 1.0, 2.0), line[:3],
                               0, line[4], 1.075, 1e-3, 3000, 20, h_max=8.0)
    assert (r["fired"], r["merged"], r["steps"]) == (o["fired"], o["merged"], o["step"])
    if r["fired"]:
        assert abs(r["h_c"] - o["h_c"]) < 1e-9
        assert rel_err(M.read_f(), o["f"]) < 1e-12
    M.close()
