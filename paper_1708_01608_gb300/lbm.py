"""Python binding of the C ABI in ``include/lbm.h`` (ctypes; argument
marshalling only).

Every step of the method runs in the CUDA kernels of ``libsclbm.so``; this
module converts numpy arrays and Python values into the C structures and
raises :class:`LBMError` on any non-OK status.  PyTorch, when present, only
provides device memory (its caching allocator, through the allocator
callbacks of the config) and the current CUDA stream.

There is no CPU fallback: if the library has not been built the import of
this module fails.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsclbm.so")

# enums (include/lbm.h)
OK, EINVAL, ENOMEM, ECUDA, ESTATE, ENUMERIC, ETIMEOUT = range(7)
D2Q9, D3Q19 = 0, 1
F64, F32, F16_OFFSET, BF16_OFFSET = 0, 1, 2, 3
RHO, PSI, P, U, F, LAPP = range(6)
KERNEL_AUTO, KERNEL_FUSED, KERNEL_TWO_PASS = 0, 1, 2
DEBUG_WITHHOLD_TMA = 1
DEBUG_CONVERT_BEFORE_FMA = 2
DEBUG_SMALL_FILM_QUEUE = 4
# lbm_ensemble_set_launch modes
ENS_AUTO, ENS_GRAPH, ENS_DEBUG_WITHHOLD_FLAG, ENS_PERSISTENT, ENS_TEMPORAL = 0, 1, 2, 3, 4

STORAGE = {"f64": F64, "f32": F32, "f16": F16_OFFSET, "bf16": BF16_OFFSET}
LATTICE = {"D2Q9": D2Q9, "D3Q19": D3Q19}
KERNEL = {"auto": KERNEL_AUTO, "fused": KERNEL_FUSED, "two_pass": KERNEL_TWO_PASS}
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ESTATE", 5: "ENUMERIC",
                6: "ETIMEOUT"}

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class Config(C.Structure):
    _fields_ = [
        ("lattice", C.c_int32), ("storage", C.c_int32),
        ("nx", C.c_int64), ("ny", C.c_int64), ("nz", C.c_int64),
        ("tau", C.c_double), ("G", C.c_double), ("rho0", C.c_double),
        ("rho_ref", C.c_double), ("gas_threshold", C.c_double),
        ("kernel", C.c_int32), ("tile", C.c_int32),
        ("stream", C.c_void_p),
        ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_user", C.c_void_p),
        ("debug_flags", C.c_int32), ("nucleus_radius", C.c_double),
        ("mass_residual", C.c_int32),
    ]


class Bubble(C.Structure):
    _fields_ = [("x", C.c_double), ("y", C.c_double), ("z", C.c_double), ("r", C.c_double)]


class Film(C.Structure):
    _fields_ = [("found", C.c_int32), ("x1", C.c_double), ("x2", C.c_double), ("h", C.c_double),
                ("d2p_mid", C.c_double), ("r_d", C.c_double)]


class Rupture(C.Structure):
    _fields_ = [("fired", C.c_int32), ("merged", C.c_int32), ("steps", C.c_int64),
                ("h_c", C.c_double), ("h_probe", C.c_double), ("r_d", C.c_double)]


class FilmCensus(C.Structure):
    _fields_ = [("film", C.c_int64), ("midpoints", C.c_int64), ("armed", C.c_int64),
                ("fired", C.c_int64)]


class IntervalReport(C.Structure):
    _fields_ = [("totals", C.c_double * 4), ("ncomp", C.c_int64), ("merge_events", C.c_int64),
                ("film", FilmCensus), ("nfired", C.c_int64), ("nsizes", C.c_int64)]


# lbm_film_cell as a numpy record
FILM_CELL = np.dtype([("cell", np.int64), ("axis", np.int32), ("label_minus", np.int32),
                      ("label_plus", np.int32), ("thickness", np.int32), ("d2p", np.float64)],
                     align=True)
# lbm_film_pair
FILM_PAIR = np.dtype([("label_a", np.int32), ("label_b", np.int32), ("axis", np.int32),
                      ("h_min", np.int32), ("lines", np.int64), ("midpoints", np.int64),
                      ("fired", np.int64), ("r_d", np.float64), ("h_c", np.float64)], align=True)


class Domain(C.Structure):
    _fields_ = [("nx", C.c_int64), ("ny", C.c_int64), ("tau", C.c_double), ("G", C.c_double),
                ("rho0", C.c_double), ("rho_ref", C.c_double), ("rho_l", C.c_double),
                ("rho_g", C.c_double), ("width", C.c_double), ("noise_amp", C.c_double),
                ("seed", C.c_uint64), ("nbubbles", C.c_int32), ("bubbles", Bubble * 4),
                ("line", C.c_int64 * 5), ("rho_mid", C.c_double)]


class MLConfig(C.Structure):
    _fields_ = [("lattice", C.c_int32), ("storage", C.c_int32), ("nx", C.c_int64),
                ("ny", C.c_int64), ("nz", C.c_int64), ("nl", C.c_int32), ("tau", C.c_double),
                ("rho0", C.c_double), ("G", C.c_double), ("G_x", C.c_double),
                ("G_b", C.c_double), ("stream", C.c_void_p), ("alloc", ALLOC_FN),
                ("free", FREE_FN), ("alloc_user", C.c_void_p)]


class LBMError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build the CUDA library first "
            "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = C.CDLL(LIB_PATH)
    P_ = C.c_void_p
    i32, i64, u64, d, sz = C.c_int32, C.c_int64, C.c_uint64, C.c_double, C.c_size_t
    sig = {
        "lbm_config_default": (None, [C.POINTER(Config)]),
        "lbm_create": (i32, [C.POINTER(Config), C.POINTER(P_)]),
        "lbm_destroy": (None, [P_]),
        "lbm_sample_sites": (i32, [i64, i64, i64, i32, d, d, d, d, u64, i64, P_, C.POINTER(i32)]),
        "lbm_seed_bubbles": (i32, [P_, P_, i32, d, d, d, d, d, u64]),
        "lbm_read_sites": (i32, [P_, P_, i32]),
        "lbm_inject": (i32, [P_, P_, P_, i32]),
        "lbm_read_budgets": (i32, [P_, P_, i32]),
        "lbm_step": (i32, [P_, i64]),
        "lbm_step_count": (i64, [P_]),
        "lbm_autotune": (i32, [P_, i32, C.POINTER(i32), C.POINTER(d)]),
        "lbm_plan_info": (i32, [P_, P_]),
        "lbm_sync": (i32, [P_]),
        "lbm_pressure_laplacian": (i32, [P_, P_, i64, P_]),
        "lbm_label_gas": (i32, [P_, P_, C.POINTER(i64)]),
        "lbm_diagnose": (i32, [P_, P_, P_, C.POINTER(i64)]),
        "lbm_film_probe": (i32, [P_, P_, d, C.POINTER(Film)]),
        "lbm_run_until_rupture": (i32, [P_, P_, d, d, d, i64, i64, C.POINTER(Rupture)]),
        "lbm_site_labels": (i32, [P_, P_, i32, C.POINTER(i64)]),
        "lbm_bubble_sizes": (i32, [P_, P_, P_, i64, C.POINTER(i64), P_, i32]),
        "lbm_film_cells": (i32, [P_, i32, d, C.POINTER(FilmCensus), P_, i64]),
        "lbm_film_pairs": (i32, [P_, i32, d, C.POINTER(FilmCensus), P_, i64, C.POINTER(i64)]),
        "lbm_set_injection_mode": (i32, [P_, i32]),
        "lbm_diagnostic_interval": (i32, [P_, i32, d, P_, P_, i64, P_, P_, i64, P_, i32,
                                          C.POINTER(IntervalReport)]),
        "lbm_totals": (i32, [P_, P_]),
        "lbm_read": (i32, [P_, i32, P_, sz]),
        "lbm_write_f": (i32, [P_, P_, sz]),
        "lbm_step_static_f32": (i32, [i32, i64, i64, i64, d, d, d, P_, P_, P_]),
        "lbm_ensemble_create": (i32, [P_, i32, d, d, i32, ALLOC_FN, FREE_FN, P_, C.POINTER(P_)]),
        "lbm_ensemble_destroy": (None, [P_]),
        "lbm_ensemble_run": (i32, [P_, i64, C.POINTER(i64)]),
        "lbm_ensemble_results": (i32, [P_, P_, i32]),
        "lbm_ensemble_stats": (i32, [P_, P_]),
        "lbm_ensemble_read_f": (i32, [P_, i32, P_, sz]),
        "lbm_ensemble_set_launch": (i32, [P_, i32]),
        "lbm_fp64_rate": (i32, [i32, C.POINTER(d)]),
        "lbm_ml_config_default": (None, [C.POINTER(MLConfig)]),
        "lbm_ml_create": (i32, [C.POINTER(MLConfig), C.POINTER(P_)]),
        "lbm_ml_destroy": (None, [P_]),
        "lbm_ml_coupling": (i32, [P_, P_]),
        "lbm_ml_seed": (i32, [P_, P_, d, d, d, d, d, u64]),
        "lbm_ml_write_f": (i32, [P_, P_, sz]),
        "lbm_ml_read_f": (i32, [P_, P_, sz]),
        "lbm_ml_inject": (i32, [P_, P_, P_, i32]),
        "lbm_ml_read_budgets": (i32, [P_, P_, i32]),
        "lbm_ml_step": (i32, [P_, i64]),
        "lbm_ml_step_count": (i64, [P_]),
        "lbm_ml_merge": (i32, [P_, i32, i32]),
        "lbm_ml_fields": (i32, [P_, P_, P_]),
        "lbm_ml_run_until_rupture": (i32, [P_, P_, d, d, d, i64, i64, i32, i32,
                                           C.POINTER(Rupture)]),
        "lbm_last_error": (C.c_char_p, []),
        "lbm_version": (C.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()

# every symbol the header declares (checked by the CPU tests)
EXPORTS = ("lbm_config_default", "lbm_create", "lbm_destroy", "lbm_sample_sites",
           "lbm_seed_bubbles", "lbm_read_sites", "lbm_inject", "lbm_set_injection_mode", "lbm_read_budgets",
           "lbm_step", "lbm_step_count",
           "lbm_autotune", "lbm_plan_info",
           "lbm_sync", "lbm_pressure_laplacian", "lbm_label_gas", "lbm_diagnose", "lbm_film_probe",
           "lbm_run_until_rupture",
           "lbm_site_labels", "lbm_bubble_sizes", "lbm_film_cells", "lbm_film_pairs",
           "lbm_diagnostic_interval",
           "lbm_totals", "lbm_read", "lbm_write_f", "lbm_step_static_f32", "lbm_fp64_rate",
           "lbm_last_error", "lbm_ml_config_default", "lbm_ml_create", "lbm_ml_destroy",
           "lbm_ml_coupling", "lbm_ml_seed", "lbm_ml_write_f", "lbm_ml_read_f", "lbm_ml_inject",
           "lbm_ml_read_budgets", "lbm_ml_step", "lbm_ml_step_count", "lbm_ml_merge",
           "lbm_ml_fields", "lbm_ml_run_until_rupture",
           "lbm_version", "lbm_ensemble_create", "lbm_ensemble_destroy", "lbm_ensemble_run",
           "lbm_ensemble_results", "lbm_ensemble_stats", "lbm_ensemble_read_f",
           "lbm_ensemble_set_launch")


def lib():
    return _lib


def _check(st: int):
    if st != OK:
        raise LBMError(st, _lib.lbm_last_error().decode())


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def version() -> str:
    return _lib.lbm_version().decode()


def sample_sites(nx, ny, nz, n, r_min, r_max, min_spacing=0.0, min_gap=0.0, seed=0,
                 max_tries=10_000_000):
    """Random nucleation sites (host sampler of the library): (n, 4) x, y, z, r."""
    out = (Bubble * max(n, 1))()
    got = C.c_int32(0)
    _check(_lib.lbm_sample_sites(nx, ny, nz, n, r_min, r_max, min_spacing, min_gap,
                                 seed & (2**64 - 1), max_tries, C.cast(out, C.c_void_p),
                                 C.byref(got)))
    return np.array([[b.x, b.y, b.z, b.r] for b in out[:n]], dtype=np.float64).reshape(-1, 4)


class _TorchMemory:
    """Allocator callbacks backed by torch's CUDA caching allocator."""

    def __init__(self):
        import torch
        self.torch = torch

        def alloc(nbytes, stream, user):
            try:
                return int(torch.cuda.caching_allocator_alloc(int(nbytes), stream=stream or 0))
            except Exception:  # reported to C as a NULL pointer -> ENOMEM
                return None

        def free(ptr, nbytes, stream, user):
            try:
                torch.cuda.caching_allocator_delete(ptr)
            except Exception:
                pass

        self.alloc = ALLOC_FN(alloc)
        self.free = FREE_FN(free)


class Lattice:
    """One periodic Shan-Chen lattice on the current CUDA device."""

    def __init__(self, lattice="D3Q19", nx=64, ny=64, nz=1, tau=1.0, G=-5.0, rho0=1.0,
                 storage="f32", rho_ref=1.0, gas_threshold=1.0, kernel="auto", tile=0,
                 stream: Optional[int] = None, torch_memory: bool = True, debug_flags: int = 0,
                 nucleus_radius: float = 3.0, mass_residual: bool = False):
        cfg = Config()
        _lib.lbm_config_default(C.byref(cfg))
        cfg.lattice = LATTICE[lattice] if isinstance(lattice, str) else int(lattice)
        cfg.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
        cfg.nx, cfg.ny, cfg.nz = int(nx), int(ny), int(nz)
        cfg.tau, cfg.G, cfg.rho0 = float(tau), float(G), float(rho0)
        cfg.rho_ref, cfg.gas_threshold = float(rho_ref), float(gas_threshold)
        cfg.kernel = KERNEL[kernel] if isinstance(kernel, str) else int(kernel)
        cfg.tile = int(tile)
        cfg.debug_flags = int(debug_flags)
        cfg.nucleus_radius = float(nucleus_radius)
        cfg.mass_residual = 1 if mass_residual else 0
        self._mem = None
        if torch_memory:
            try:
                import torch
                if torch.cuda.is_available():
                    self._mem = _TorchMemory()
                    if stream is None:
                        stream = torch.cuda.current_stream().cuda_stream
            except ImportError:
                self._mem = None
        if self._mem is not None:
            cfg.alloc, cfg.free = self._mem.alloc, self._mem.free
        cfg.stream = stream or None
        self.cfg = cfg
        self._census_buf = (np.empty(4096, np.int64), np.empty(4096, np.int64))
        self._film_buf = np.empty(0, dtype=FILM_CELL)
        self.q = 9 if cfg.lattice == D2Q9 else 19
        self.shape = (cfg.nz, cfg.ny, cfg.nx)
        self.n = cfg.nx * cfg.ny * cfg.nz
        self.nsites = 0
        h = C.c_void_p()
        _check(_lib.lbm_create(C.byref(cfg), C.byref(h)))
        self._h = h

    # -- lifetime
    def close(self):
        if getattr(self, "_h", None):
            _lib.lbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    # -- set-up
    def seed_bubbles(self, bubbles, rho_l, rho_g, width=2.0, noise_amp=0.0, seed=0, n=0,
                     min_spacing=0.0):
        """Initial state (lbm_seed_bubbles).  bubbles: (n, 4) rows x, y, z, r;
        None with n > 0 draws n nuclei of the configured nucleus radius from
        the seed, at least min_spacing apart (read them with sites())."""
        if bubbles is None and n > 0:
            self.nsites = int(n)
            _check(_lib.lbm_seed_bubbles(self._h, None, int(n), rho_l, rho_g, width, noise_amp,
                                         float(min_spacing), seed & (2**64 - 1)))
            return
        b = np.ascontiguousarray(np.zeros((0, 4)) if bubbles is None else bubbles,
                                 dtype=np.float64).reshape(-1, 4)
        self.nsites = len(b)
        _check(_lib.lbm_seed_bubbles(self._h, _ptr(b) if len(b) else None, len(b), rho_l, rho_g,
                                     width, noise_amp, float(min_spacing), seed & (2**64 - 1)))

    def sites(self):
        """The seeded bubbles (given or drawn) as (n, 4) rows x, y, z, r."""
        out = (Bubble * max(self.nsites, 1))()
        _check(_lib.lbm_read_sites(self._h, C.cast(out, C.c_void_p), self.nsites))
        return np.array([[b.x, b.y, b.z, b.r] for b in out[:self.nsites]],
                        dtype=np.float64).reshape(-1, 4)

    def inject(self, rate, budget):
        r = np.ascontiguousarray(rate, dtype=np.float64).reshape(-1)
        b = np.ascontiguousarray(budget, dtype=np.float64).reshape(-1)
        _check(_lib.lbm_inject(self._h, _ptr(r) if len(r) else None,
                               _ptr(b) if len(b) else None, len(r)))
        self._ninj = len(r)

    def set_injection_mode(self, mode):
        """"site" (the site cell, default) or "bubble" (spread over the site's
        bubble after every step; lbm_set_injection_mode)."""
        _check(_lib.lbm_set_injection_mode(self._h, {"site": 0, "bubble": 1}[mode]))

    def read_budgets(self):
        out = np.empty(getattr(self, "_ninj", 0))
        _check(_lib.lbm_read_budgets(self._h, _ptr(out), len(out)))
        return out

    def write_f(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        assert f.size == self.q * self.n
        _check(_lib.lbm_write_f(self._h, _ptr(f), f.nbytes))

    # -- time stepping
    def step(self, n=1):
        _check(_lib.lbm_step(self._h, int(n)))

    def sync(self):
        _check(_lib.lbm_sync(self._h))

    def autotune(self, steps=10):
        """Time every fitting fused tile on the current state (restored
        afterwards) and keep the fastest: (tile id, ms per step)."""
        t = C.c_int32(0)
        ms = C.c_double(0)
        _check(_lib.lbm_autotune(self._h, int(steps), C.byref(t), C.byref(ms)))
        return int(t.value), float(ms.value)

    def plan(self):
        """(kernel, tile id, tile x, tile y, z chunks, CTAs per step)."""
        out = np.zeros(6, dtype=np.int32)
        _check(_lib.lbm_plan_info(self._h, _ptr(out)))
        return tuple(int(v) for v in out)

    @property
    def steps(self):
        return int(_lib.lbm_step_count(self._h))

    # -- diagnostics
    def read(self, field):
        field = {"rho": RHO, "psi": PSI, "p": P, "u": U, "f": F, "lapp": LAPP}.get(field, field)
        comps = {U: 3, F: self.q}.get(field, 1)
        out = np.empty((comps,) + self.shape) if comps > 1 else np.empty(self.shape)
        _check(_lib.lbm_read(self._h, int(field), _ptr(out), out.nbytes))
        return out

    def pressure_laplacian(self, line=None):
        """Full periodic Laplacian of p (line None) or the second difference
        along line = (x, y, z, axis, length)."""
        if line is None:
            out = np.empty(self.shape)
            _check(_lib.lbm_pressure_laplacian(self._h, _ptr(out), out.size, None))
            return out
        ln = np.ascontiguousarray(line, dtype=np.int64)
        out = np.empty(int(ln[4]))
        _check(_lib.lbm_pressure_laplacian(self._h, _ptr(out), out.size, _ptr(ln)))
        return out

    def label_gas(self, want_labels=True):
        """(labels int32 shaped like the lattice or None, number of components)."""
        lab = np.empty(self.shape, dtype=np.int32) if want_labels else None
        nc = C.c_int64(0)
        _check(_lib.lbm_label_gas(self._h, _ptr(lab) if want_labels else None, C.byref(nc)))
        return lab, int(nc.value)

    def film_probe(self, line, rho_mid):
        """Film between two bubbles along line = (x, y, z, axis, len):
        dict(found, x1, x2, h, d2p_mid, r_d)."""
        ln = np.ascontiguousarray(line, dtype=np.int64)
        out = Film()
        _check(_lib.lbm_film_probe(self._h, _ptr(ln), float(rho_mid), C.byref(out)))
        return dict(found=bool(out.found), x1=out.x1, x2=out.x2, h=out.h, d2p_mid=out.d2p_mid,
                    r_d=out.r_d)

    def run_until_rupture(self, line, rho_mid, eps_arm, diag_every, max_steps, h_max=8.0):
        """Rupture criterion (lbm_run_until_rupture): dict(fired, merged, steps,
        h_c, h_probe, r_d); h_c is the interpolated zero crossing of d2p."""
        ln = np.ascontiguousarray(line, dtype=np.int64)
        out = Rupture()
        _check(_lib.lbm_run_until_rupture(self._h, _ptr(ln), float(rho_mid), float(eps_arm),
                                          float(h_max), int(diag_every), int(max_steps),
                                          C.byref(out)))
        return dict(fired=bool(out.fired), merged=bool(out.merged), steps=int(out.steps),
                    h_c=out.h_c, h_probe=out.h_probe, r_d=out.r_d)

    def diagnose(self, want_labels=False):
        """One diagnostic interval: (totals[4], labels or None, components)."""
        tot = np.zeros(4)
        lab = np.empty(self.shape, dtype=np.int32) if want_labels else None
        nc = C.c_int64(0)
        _check(_lib.lbm_diagnose(self._h, _ptr(tot), _ptr(lab) if want_labels else None,
                                 C.byref(nc)))
        return tot, lab, int(nc.value)

    def site_labels(self):
        out = np.empty(self.nsites, dtype=np.int32)
        ev = C.c_int64(0)
        _check(_lib.lbm_site_labels(self._h, _ptr(out) if self.nsites else None, self.nsites,
                                    C.byref(ev)))
        return out, int(ev.value)

    def bubble_sizes(self, nbins=32, cap=1 << 20):
        """Label the gas and measure its components (lbm_bubble_sizes):
        (roots, sizes) in increasing root order and the log2 size histogram."""
        # The output arrays are kept between calls (large allocations are
        # costly at every diagnostic interval) and grown, with the call
        # repeated, when the lattice has more components than they hold.
        hist = np.zeros(max(nbins, 1), dtype=np.int64)
        nc = C.c_int64(0)
        while True:
            buf = self._census_buf
            room = min(int(cap), len(buf[0]))
            _check(_lib.lbm_bubble_sizes(self._h, _ptr(buf[0]), _ptr(buf[1]), room, C.byref(nc),
                                         _ptr(hist), int(nbins)))
            n = int(nc.value)
            if n <= room or room >= cap:
                break
            grow = min(int(cap), 2 * n)
            self._census_buf = (np.empty(grow, np.int64), np.empty(grow, np.int64))
        n = min(n, room)
        return buf[0][:n].copy(), buf[1][:n].copy(), hist[:nbins]

    def film_cells(self, h_max=12, eps_arm=1e-3, cap=1 << 16):
        """The film test at every lattice point (lbm_film_cells): (counts
        dict, fired records as a FILM_CELL array in (cell, axis) order)."""
        out = FilmCensus()
        if len(self._film_buf) < max(cap, 1):  # kept between calls, as for the census
            self._film_buf = np.empty(max(cap, 1), dtype=FILM_CELL)
        rec = self._film_buf
        _check(_lib.lbm_film_cells(self._h, int(h_max), float(eps_arm), C.byref(out), _ptr(rec),
                                   int(cap)))
        return (dict(film=out.film, midpoints=out.midpoints, armed=out.armed, fired=out.fired),
                rec[:min(out.fired, cap)].copy())

    def diagnostic_interval(self, h_max=12, eps_arm=1e-3, fired_cap=4096, nbins=32,
                            want_labels=False):
        """Totals, labels, site labels, the film test and the bubble census of
        the current state in one call (lbm_diagnostic_interval): dict with
        totals, ncomp, merge_events, film (counts), fired (FILM_CELL records),
        roots, sizes, hist, and labels (shape of the lattice) if asked."""
        lab = np.empty(self.shape, dtype=np.int32) if want_labels else None
        if len(self._film_buf) < max(fired_cap, 1):
            self._film_buf = np.empty(max(fired_cap, 1), dtype=FILM_CELL)
        roots, sizes = self._census_buf
        hist = np.zeros(max(nbins, 1), dtype=np.int64)
        rep = IntervalReport()
        _check(_lib.lbm_diagnostic_interval(self._h, int(h_max), float(eps_arm),
                                            _ptr(lab) if want_labels else None,
                                            _ptr(self._film_buf), int(fired_cap), _ptr(roots),
                                            _ptr(sizes), len(roots), _ptr(hist), int(nbins),
                                            C.byref(rep)))
        n = int(rep.ncomp)
        if n > len(roots):
            # more components than the kept arrays hold: the census alone,
            # again on the same labels (the film test is not repeated)
            roots, sizes, _ = self.bubble_sizes(nbins, cap=n)
        else:
            roots, sizes = roots[:n].copy(), sizes[:n].copy()
        f = rep.film
        return dict(totals=np.array(rep.totals[:]), ncomp=n, merge_events=int(rep.merge_events),
                    film=dict(film=f.film, midpoints=f.midpoints, armed=f.armed, fired=f.fired),
                    fired=self._film_buf[:int(rep.nfired)].copy(), roots=roots, sizes=sizes,
                    hist=hist[:nbins], labels=lab)

    def film_pairs(self, h_max=12, eps_arm=1e-3, cap=1 << 14):
        """The film test reported per pair of bubbles (lbm_film_pairs):
        (counts dict, FILM_PAIR array in (label_a, label_b) order)."""
        out = FilmCensus()
        pairs = np.empty(max(cap, 1), dtype=FILM_PAIR)
        n = C.c_int64(0)
        _check(_lib.lbm_film_pairs(self._h, int(h_max), float(eps_arm), C.byref(out), _ptr(pairs),
                                   int(cap), C.byref(n)))
        return (dict(film=out.film, midpoints=out.midpoints, armed=out.armed, fired=out.fired),
                pairs[:min(int(n.value), cap)].copy())

    def totals(self):
        out = np.zeros(4)
        _check(_lib.lbm_totals(self._h, _ptr(out)))
        return out


def step_static_f32(lattice, nx, ny, nz, tau, G, rho0, f_in_ptr, f_out_ptr, stream=None):
    """One allocation-free step on caller-owned device buffers (see
    lbm_step_static_f32 in include/lbm.h): pointers are device addresses."""
    lat = LATTICE[lattice] if isinstance(lattice, str) else int(lattice)
    _check(_lib.lbm_step_static_f32(lat, nx, ny, nz, tau, G, rho0, C.c_void_p(f_in_ptr),
                                    C.c_void_p(f_out_ptr), C.c_void_p(stream) if stream else None))


def fp64_rate(iters=20000):
    """Measured FP64 FMA rate of the current device in TFLOP/s (lbm_fp64_rate)."""
    out = C.c_double(0)
    _check(_lib.lbm_fp64_rate(int(iters), C.byref(out)))
    return float(out.value)


class MultiLattice:
    """The multi-lattice Shan-Chen model (lbm_ml_* in include/lbm.h): the
    fluid on lattice 0 and the gas of bubble k on lattice k, coupled by the
    multicomponent force with the eta_m-switched barrier between bubbles."""

    def __init__(self, lattice="D2Q9", nx=128, ny=128, nz=1, nl=3, tau=1.0, rho0=1.0, G=-5.0,
                 G_x=1.0, G_b=0.0, storage="f64", torch_memory=True):
        cfg = MLConfig()
        _lib.lbm_ml_config_default(C.byref(cfg))
        cfg.lattice = LATTICE[lattice] if isinstance(lattice, str) else int(lattice)
        cfg.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
        cfg.nx, cfg.ny, cfg.nz, cfg.nl = int(nx), int(ny), int(nz), int(nl)
        cfg.tau, cfg.rho0, cfg.G, cfg.G_x, cfg.G_b = (float(tau), float(rho0), float(G),
                                                      float(G_x), float(G_b))
        self._mem = None
        if torch_memory:
            try:
                import torch
                if torch.cuda.is_available():
                    self._mem = _TorchMemory()
                    cfg.alloc, cfg.free = self._mem.alloc, self._mem.free
                    cfg.stream = torch.cuda.current_stream().cuda_stream or None
            except ImportError:
                pass
        self.q = 9 if cfg.lattice == D2Q9 else 19
        self.nl = cfg.nl
        self.shape = (cfg.nz, cfg.ny, cfg.nx)
        self.n = cfg.nx * cfg.ny * cfg.nz
        h = C.c_void_p()
        _check(_lib.lbm_ml_create(C.byref(cfg), C.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            _lib.lbm_ml_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def coupling(self):
        out = np.zeros((self.nl, self.nl))
        _check(_lib.lbm_ml_coupling(self._h, _ptr(out)))
        return out

    def seed(self, bubbles, rho_l, rho_v, rho_gas, width=2.0, noise_amp=0.0, seed=0):
        b = np.ascontiguousarray(bubbles, dtype=np.float64).reshape(-1, 4)
        assert len(b) == self.nl - 1
        _check(_lib.lbm_ml_seed(self._h, _ptr(b) if len(b) else None, rho_l, rho_v, rho_gas,
                                width, noise_amp, seed & (2**64 - 1)))

    def write_f(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        assert f.size == self.nl * self.q * self.n
        _check(_lib.lbm_ml_write_f(self._h, _ptr(f), f.nbytes))

    def read_f(self):
        out = np.empty((self.nl, self.q) + self.shape)
        _check(_lib.lbm_ml_read_f(self._h, _ptr(out), out.nbytes))
        return out

    def inject(self, rate, budget):
        r = np.ascontiguousarray(rate, dtype=np.float64).reshape(-1)
        b = np.ascontiguousarray(budget, dtype=np.float64).reshape(-1)
        _check(_lib.lbm_ml_inject(self._h, _ptr(r) if len(r) else None,
                                  _ptr(b) if len(b) else None, len(r)))
        self._ninj = len(r)

    def read_budgets(self):
        out = np.empty(getattr(self, "_ninj", 0))
        _check(_lib.lbm_ml_read_budgets(self._h, _ptr(out), len(out)))
        return out

    def step(self, n=1):
        _check(_lib.lbm_ml_step(self._h, int(n)))

    @property
    def steps(self):
        return int(_lib.lbm_ml_step_count(self._h))

    def merge(self, k, l):
        _check(_lib.lbm_ml_merge(self._h, int(k), int(l)))

    def fields(self):
        """(rho of every lattice (nl, nz, ny, nx), coupled pressure (nz, ny, nx))."""
        rho = np.empty((self.nl,) + self.shape)
        p = np.empty(self.shape)
        _check(_lib.lbm_ml_fields(self._h, _ptr(rho), _ptr(p)))
        return rho, p

    def run_until_rupture(self, line, rho_mid, eps_arm, diag_every, max_steps, h_max=8.0,
                          pair=(1, 2)):
        ln = np.ascontiguousarray(line, dtype=np.int64)
        out = Rupture()
        _check(_lib.lbm_ml_run_until_rupture(self._h, _ptr(ln), float(rho_mid), float(eps_arm),
                                             float(h_max), int(diag_every), int(max_steps),
                                             int(pair[0]), int(pair[1]), C.byref(out)))
        return dict(fired=bool(out.fired), merged=bool(out.merged), steps=int(out.steps),
                    h_c=out.h_c, h_probe=out.h_probe, r_d=out.r_d)


class Ensemble:
    """Batched two-bubble D2Q9 domains with the on-device rupture criterion
    (lbm_ensemble_* in include/lbm.h).  domains: list of dicts with the
    lbm_domain fields (bubbles as (x, y, 0, r) rows, line as 5 ints)."""

    def __init__(self, domains, eps_arm=1e-3, diag_every=20, torch_memory=True, h_max=8.0):
        n = len(domains)
        arr = (Domain * n)()
        for k, dm in enumerate(domains):
            a = arr[k]
            for f in ("nx", "ny", "seed", "nbubbles"):
                setattr(a, f, int(dm[f]) if f != "nbubbles" else len(dm["bubbles"]))
            a.nbubbles = len(dm["bubbles"])
            for f in ("tau", "G", "rho0", "rho_ref", "rho_l", "rho_g", "width", "noise_amp",
                      "rho_mid"):
                setattr(a, f, float(dm[f]))
            for j, bb in enumerate(dm["bubbles"]):
                a.bubbles[j] = Bubble(*[float(v) for v in bb])
            for j, v in enumerate(dm["line"]):
                a.line[j] = int(v)
        self._mem = None
        alloc, free = ALLOC_FN(), FREE_FN()
        if torch_memory:
            try:
                import torch
                if torch.cuda.is_available():
                    self._mem = _TorchMemory()
                    alloc, free = self._mem.alloc, self._mem.free
            except ImportError:
                pass
        self.n = n
        self.shapes = [(int(dm["ny"]), int(dm["nx"])) for dm in domains]
        h = C.c_void_p()
        _check(_lib.lbm_ensemble_create(C.cast(arr, C.c_void_p), n, float(eps_arm), float(h_max),
                                        int(diag_every), alloc, free, None, C.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            _lib.lbm_ensemble_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, max_steps):
        done = C.c_int64(0)
        _check(_lib.lbm_ensemble_run(self._h, int(max_steps), C.byref(done)))
        return int(done.value)

    def results(self):
        out = (Rupture * self.n)()
        _check(_lib.lbm_ensemble_results(self._h, C.cast(out, C.c_void_p), self.n))
        return [dict(fired=bool(r.fired), merged=bool(r.merged), steps=int(r.steps), h_c=r.h_c,
                     h_probe=r.h_probe, r_d=r.r_d) for r in out]

    def stats(self):
        out = np.zeros(4)
        _check(_lib.lbm_ensemble_stats(self._h, _ptr(out)))
        return dict(steps=int(out[0]), updates=out[1], active=int(out[2]), launches=int(out[3]))

    def set_launch(self, mode):
        """ENS_AUTO, ENS_GRAPH, ENS_TEMPORAL, ENS_PERSISTENT or the test
        hook ENS_DEBUG_WITHHOLD_FLAG (lbm_ensemble_set_launch)."""
        _check(_lib.lbm_ensemble_set_launch(self._h, int(mode)))

    def read_f(self, d):
        ny, nx = self.shapes[d]
        out = np.empty((9, 1, ny, nx))
        _check(_lib.lbm_ensemble_read_f(self._h, int(d), _ptr(out), out.nbytes))
        return out
