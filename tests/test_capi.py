"""CPU checks of the C ABI: the library loads, exports every function that
include/lbm.h declares, validates its arguments without touching a GPU, and
its host-side site sampler agrees bit for bit with the oracle's."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle as O
from helpers import lbm_mod

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lbm():
    return lbm_mod()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "lbm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", text)))


def test_header_symbols_exported(lbm):
    names = declared_functions()
    assert len(names) >= 18
    lib = C.CDLL(lbm.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(lbm.EXPORTS)


def test_header_constants_match_binding(lbm):
    """Every integer constant of include/lbm.h (enum members and #defines)
    that the Python binding mirrors under the same name, without the LBM_
    prefix, has the same value there."""
    text = open(os.path.join(ROOT, "include", "lbm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    consts = dict(re.findall(r"#define\s+LBM_([A-Z0-9_]+)\s+(-?\d+)\b", text))
    consts.update(re.findall(r"\bLBM_([A-Z0-9_]+)\s*=\s*(-?\d+)", text))
    mirrored = {k: int(v) for k, v in consts.items() if hasattr(lbm, k)}
    assert len(mirrored) >= 25, sorted(mirrored)
    for k, v in mirrored.items():
        assert getattr(lbm, k) == v, k


def test_version(lbm):
    assert "sm_103a" in lbm.version()


@pytest.mark.parametrize("kw", [
    dict(lattice="D2Q9", nz=2), dict(nx=0), dict(tau=0.5), dict(tau=float("nan")),
    dict(rho0=0.0), dict(storage=7), dict(kernel=9), dict(lattice=5),
    # size limits: an extent above 2^20; padded cells (x rounded up to 8) at 2^31
    dict(nx=2**20 + 8, ny=1, nz=1), dict(nx=1024, ny=1024, nz=2048),
    dict(nx=1020, ny=1024, nz=2048)])
def test_create_rejects_bad_config_without_gpu(lbm, kw):
    args = dict(lattice="D3Q19", nx=8, ny=8, nz=8, torch_memory=False)
    args.update(kw)
    with pytest.raises(lbm.LBMError) as e:
        lbm.Lattice(**args)
    assert e.value.status == lbm.EINVAL


def test_null_arguments(lbm):
    L = lbm.lib()
    assert L.lbm_create(None, None) == lbm.EINVAL
    assert L.lbm_step(None, 1) == lbm.EINVAL
    assert L.lbm_sync(None) == lbm.EINVAL
    assert L.lbm_step_count(None) == -1
    L.lbm_destroy(None)
    assert "NULL" in L.lbm_last_error().decode()


def test_null_arguments_of_diagnostics_and_modes(lbm):
    """The film pair census, the one-call interval, the injection mode and
    the ensemble's calls reject a missing context before any device work."""
    L = lbm.lib()
    census = lbm.FilmCensus()
    n = C.c_int64(0)
    assert L.lbm_film_pairs(None, 12, 1e-3, C.byref(census), None, 0, C.byref(n)) == lbm.EINVAL
    rep = lbm.IntervalReport()
    assert L.lbm_diagnostic_interval(None, 12, 1e-3, None, None, 0, None, None, 0, None, 0,
                                     C.byref(rep)) == lbm.EINVAL
    assert L.lbm_set_injection_mode(None, 1) == lbm.EINVAL
    assert L.lbm_film_cells(None, 12, 1e-3, C.byref(census), None, 0) == lbm.EINVAL
    assert L.lbm_bubble_sizes(None, None, None, 0, None, None, 0) == lbm.EINVAL
    assert L.lbm_ensemble_run(None, 10, None) == lbm.EINVAL


@pytest.mark.parametrize("args", [
    (128, 128, 128, 64, 3.0, 3.0, 12.0, 0.0, 1),
    (64, 64, 64, 30, 4.0, 12.0, 0.0, 4.0, 2),
    (512, 512, 1, 40, 8.0, 20.0, 0.0, 3.0, 7),
])
def test_site_sampler_matches_oracle(lbm, args):
    s = lbm.sample_sites(*args)
    got, so = O.sample_sites(*args)
    assert got == args[3] and (s == so).all()


def test_site_sampler_reports_overfull(lbm):
    with pytest.raises(lbm.LBMError) as e:
        lbm.sample_sites(16, 16, 1, 50, 3.0, 3.0, 8.0, 0.0, 1, max_tries=10000)
    assert e.value.status == lbm.ESTATE


def test_fig3_fit_recovers_exact_forms():
    """Rows generated exactly from the two functional forms of Fig. 3 give
    back their coefficients (R^2 = 1)."""
    from paper_1708_01608_gb300.sweep import fit_fig3
    R_b = np.array([8.0, 11.0, 15.0, 21.0, 30.0, 42.0, 60.0])
    R_d = 2.088 * np.log(R_b) + 0.114
    h_c = 0.002 * R_d ** 2 - 0.003 * R_d + 0.035
    f = fit_fig3(R_b, R_d, h_c)
    q, l = f["h_c_vs_R_d"], f["R_d_vs_ln_R_b"]
    assert (q["a"], q["b"], q["c"]) == pytest.approx((0.002, -0.003, 0.035), abs=1e-9)
    assert (l["alpha"], l["beta"]) == pytest.approx((2.088, 0.114), abs=1e-9)
    assert q["r2"] == pytest.approx(1.0) and l["r2"] == pytest.approx(1.0)
    assert f["corr_h_c_R_d"] > 0.99 and f["n"] == 7
    with pytest.raises(ValueError):
        fit_fig3(R_b[:2], R_d[:2], h_c[:2])


def test_static_step_rejects_without_gpu(lbm):
    """lbm_step_static_f32 bounds nx*ny*nz by its 2,097,152-cell scratch
    array without forming an overflowing product (2^21 per axis passes
    every per-axis bound, and (2^21)^3 = 2^63 overflows int64), rejects
    non-finite parameters and aliased buffers, and launches nothing."""
    L = lbm.lib()
    p, q = C.c_void_p(1 << 20), C.c_void_p(1 << 21)
    big = 2 ** 21
    for ext in [(big, big, big), (big, big, 1), (256, 128, 128), (big + 1, 1, 1),
                (2, big, 2), (1, 1, big + 1)]:
        assert L.lbm_step_static_f32(1, *ext, 0.9, -5.0, 1.0, p, q, None) == lbm.EINVAL, ext
        assert "2097152" in L.lbm_last_error().decode()
    inf, nan = float("inf"), float("nan")
    for tau, G, rho0 in [(inf, -5.0, 1.0), (0.9, inf, 1.0), (0.9, nan, 1.0), (0.9, -5.0, inf),
                         (0.5, -5.0, 1.0), (0.9, -5.0, 0.0)]:
        assert L.lbm_step_static_f32(1, 16, 16, 16, tau, G, rho0, p, q, None) == lbm.EINVAL
    assert L.lbm_step_static_f32(1, 16, 16, 16, 0.9, -5.0, 1.0, p, p, None) == lbm.EINVAL
    assert L.lbm_step_static_f32(0, 16, 16, 2, 0.9, -5.0, 1.0, p, q, None) == lbm.EINVAL
    assert L.lbm_step_static_f32(2, 16, 16, 16, 0.9, -5.0, 1.0, p, q, None) == lbm.EINVAL


@pytest.mark.gpu
@pytest.mark.parametrize("lat,ext,n,r,spacing,seed", [
    ("D3Q19", (128, 128, 128), 64, 3.0, 12.0, 1),
    ("D2Q9", (96, 64, 1), 5, 6.0, 20.0, 9)])
def test_seed_bubbles_draws_sites_like_the_oracle(lbm, lat, ext, n, r, spacing, seed):
    """lbm_seed_bubbles with no bubble list draws n nuclei from the seed:
    the drawn sites equal the oracle's sampler bit for bit, and the seeded
    state equals the one seeded from that explicit list."""
    import torch
    assert torch.cuda.is_available()
    nx, ny, nz = ext
    A = lbm.Lattice(lat, nx, ny, nz, storage="f64", nucleus_radius=r)
    A.seed_bubbles(None, 2.0, 0.15, 2.0, 1e-3, seed, n=n, min_spacing=spacing)
    got, want = O.sample_sites(nx, ny, nz, n, r, r, spacing, 0.0, seed)
    assert got == n
    assert (A.sites() == want).all()
    B = lbm.Lattice(lat, nx, ny, nz, storage="f64")
    B.seed_bubbles(want, 2.0, 0.15, 2.0, 1e-3, seed)
    assert (A.read("rho") == B.read("rho")).all()
    with pytest.raises(lbm.LBMError) as e:  # more nuclei than the spacing allows
        A.seed_bubbles(None, 2.0, 0.15, 2.0, 0.0, seed, n=10 ** 4, min_spacing=40.0)
    assert e.value.status == lbm.ESTATE
    A.close()
    B.close()


@pytest.mark.gpu
def test_fp64_rate_is_measured(lbm):
    """The measured FP64 FMA rate is positive and within an order of
    magnitude of what the unit counts give (2 DFMA per SM and cycle)."""
    import torch
    assert torch.cuda.is_available()
    r = lbm.fp64_rate(2000)
    props = torch.cuda.get_device_properties(0)
    derived = 2 * props.multi_processor_count * 2 * 2.07e9 / 1e12
    assert 0.1 * derived < r < 10 * derived, (r, derived)
