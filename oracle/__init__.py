"""FP64 CPU oracle for the Shan-Chen bubble-merging LBM (arXiv 1708.01608).

TEST INFRASTRUCTURE ONLY: the plain, slow statement of what the GPU path
computes.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import it; the library package never does.  It shares
no code with the CUDA path.

The arithmetic lives in ``sc_oracle.c`` (plain C, double precision); this
module only marshals numpy arrays.  Population arrays have shape
``(Q, nz, ny, nx)`` in the post-streaming form ``f_i(x, t)``; velocity order
as in ``velocities()``.

Functions whose result is not pinned by a closed form, invariant or brute
force are marked "parity unpinned" in their docstrings.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "sc_oracle.c")
LIB = os.path.join(HERE, "_build", "libsc_oracle.so")

D2Q9, D3Q19 = 0, 1


# A prebuilt variant of the library (the mutation tests load deliberately
# broken copies of sc_oracle.c through this variable).
_LIB_OVERRIDE = os.environ.get("SC_ORACLE_LIB")

GCC_FLAGS = ["-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11", "-ffp-contract=off"]


def build(force: bool = False) -> str:
    """Compile sc_oracle.c into _build/libsc_oracle.so (gcc, OpenMP)."""
    if _LIB_OVERRIDE:
        return _LIB_OVERRIDE
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        os.makedirs(os.path.dirname(LIB), exist_ok=True)
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *GCC_FLAGS, "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


_lib = None


def _L():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        d, i64, i32, u64 = C.c_double, C.c_int64, C.c_int32, C.c_uint64
        P = C.c_void_p
        _lib.orc_q.argtypes = [C.c_int]
        _lib.orc_velocities.argtypes = [C.c_int, P, P]
        _lib.orc_splitmix64.argtypes = [u64, u64]
        _lib.orc_splitmix64.restype = u64
        _lib.orc_eos.argtypes = [i64, P, d, d, P, P]
        _lib.orc_moments.argtypes = [C.c_int, i64, i64, i64, P, P, P, P, P]
        _lib.orc_force.argtypes = [C.c_int, i64, i64, i64, P, d, P, P, P]
        _lib.orc_step.argtypes = [C.c_int, i64, i64, i64, d, d, d, P, P, i32, P, P, P]
        _lib.orc_run.argtypes = [C.c_int, i64, i64, i64, d, d, d, P, i64, i32, P, P, P]
        _lib.orc_step_cells.argtypes = [C.c_int, i64, i64, i64, d, d, d, P, i64, P, P]
        _lib.orc_init.argtypes = [C.c_int, i64, i64, i64, i32, P, d, d, d, d, u64, P, P]
        _lib.orc_sample_sites.argtypes = [i64, i64, i64, i32, d, d, d, d, u64, i64, P]
        _lib.orc_sample_sites.restype = i32
        _lib.orc_laplacian.argtypes = [C.c_int, i64, i64, i64, P, P]
        _lib.orc_line_d2.argtypes = [i64, i64, i64, P, i64, i64, i64, C.c_int, i64, P]
        _lib.orc_label_gas.argtypes = [C.c_int, i64, i64, i64, P, d, P]
        _lib.orc_label_gas.restype = i64
        _lib.orc_totals.argtypes = [C.c_int, i64, i64, i64, P, P]
        _lib.orc_film_probe.argtypes = [C.c_int, i64, i64, i64, P, P, i64, i64, i64, C.c_int, i64,
                                        d, P]
        _lib.orc_bubble_sizes.argtypes = [i64, P, i64, P, P]
        _lib.orc_bubble_sizes.restype = i64
        _lib.orc_size_histogram.argtypes = [i64, P, C.c_int, P]
        _lib.orc_film_cells.argtypes = [C.c_int, i64, i64, i64, P, P, C.c_int, d, P, P, i64, P, P]
        _lib.orc_film_midpoints.argtypes = [C.c_int, i64, i64, i64, P, P, C.c_int, d, P, P, i64,
                                            P, P]
        _lib.orc_ml_run.argtypes = [C.c_int, i64, i64, i64, i32, d, P, d, P, i64, i32, P, P, P, P]
        _lib.orc_ml_force.argtypes = [C.c_int, i64, i64, i64, i32, P, P, P, P, P]
        _lib.orc_ml_pressure.argtypes = [i64, i32, P, P, d, P]
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def q_of(lat: int) -> int:
    return 9 if lat == D2Q9 else 19


def velocities(lat: int):
    """(c, w): c int array (Q, 3), w float64 (Q,) in the oracle's order."""
    q = q_of(lat)
    c = np.zeros((q, 3), dtype=np.int32)
    w = np.zeros(q, dtype=np.float64)
    _L().orc_velocities(lat, _p(c), _p(w))
    return c, w


def splitmix64(key: int, k: int) -> int:
    """k-th output of a SplitMix64 generator seeded with key."""
    return int(_L().orc_splitmix64(key & (2**64 - 1), k))


def _shape(f):
    q, nz, ny, nx = f.shape
    return q, nx, ny, nz


def eos(rho, G, rho0=1.0):
    """(psi, p): psi = rho0 (1 - exp(-rho/rho0)), p = rho/3 + G/6 psi^2 (Sec. 3.1)."""
    rho = _f64(rho)
    psi = np.empty_like(rho)
    p = np.empty_like(rho)
    _L().orc_eos(rho.size, _p(rho), G, rho0, _p(psi), _p(p))
    return psi, p


def moments(lat, f):
    """(rho, jx, jy, jz), each shaped (nz, ny, nx)."""
    f = _f64(f)
    q, nx, ny, nz = _shape(f)
    out = [np.empty((nz, ny, nx)) for _ in range(4)]
    _L().orc_moments(lat, nx, ny, nz, _p(f), *[_p(o) for o in out])
    return tuple(out)


def force(lat, psi, G):
    """Shan-Chen force (Fx, Fy, Fz) for a psi field shaped (nz, ny, nx)."""
    psi = _f64(psi)
    nz, ny, nx = psi.shape
    out = [np.empty_like(psi) for _ in range(3)]
    _L().orc_force(lat, nx, ny, nz, _p(psi), G, *[_p(o) for o in out])
    return tuple(out)


def run(lat, f, nsteps, tau, G, rho0=1.0, sites=None, rate=None, budget=None):
    """Advance f (copied) by nsteps.  sites: linear cell indices; budget is
    updated in place when given.  Returns the new f."""
    f = _f64(f).copy()
    q, nx, ny, nz = _shape(f)
    n = 0 if sites is None else len(sites)
    sc = np.ascontiguousarray(sites, dtype=np.int64) if n else None
    rt = _f64(rate) if n else None
    if n:
        assert budget is not None and budget.dtype == np.float64 and budget.flags.c_contiguous
    _L().orc_run(lat, nx, ny, nz, tau, G, rho0, _p(f), int(nsteps), n, _p(sc), _p(rt),
                 _p(budget) if n else None)
    return f


def step_cells(lat, f, cells, tau, G, rho0=1.0):
    """f_i(x, t+1) at the listed linear cells computed one by one: (ncells, Q)."""
    f = _f64(f)
    q, nx, ny, nz = _shape(f)
    cells = np.ascontiguousarray(cells, dtype=np.int64)
    out = np.empty((len(cells), q))
    _L().orc_step_cells(lat, nx, ny, nz, tau, G, rho0, _p(f), len(cells), _p(cells), _p(out))
    return out


def init(lat, nx, ny, nz, bubbles, rho_l, rho_g, width, noise_amp, seed):
    """Initial populations f_eq(rho, 0) for tanh gas bubbles in liquid plus
    SplitMix64 noise.  bubbles: (n, 4) array of x, y, z, r.  Returns (f, rho)."""
    q = q_of(lat)
    b = _f64(np.zeros((0, 4)) if bubbles is None else bubbles).reshape(-1, 4)
    f = np.empty((q, nz, ny, nx))
    rho = np.empty((nz, ny, nx))
    _L().orc_init(lat, nx, ny, nz, len(b), _p(b), rho_l, rho_g, width, noise_amp,
                  seed & (2**64 - 1), _p(f), _p(rho))
    return f, rho


def sample_sites(nx, ny, nz, n, r_min, r_max, min_spacing, min_gap, seed, max_tries=10**7):
    """Random nucleation sites by rejection sampling (Sec. 3): (got, (n, 4))."""
    out = np.zeros((max(n, 1), 4))
    got = _L().orc_sample_sites(nx, ny, nz, n, r_min, r_max, min_spacing, min_gap,
                                seed & (2**64 - 1), max_tries, _p(out))
    return got, out[:n]


def laplacian(lat, p):
    """5-point (2-D) / 7-point (3-D) periodic Laplacian of a field (nz, ny, nx)."""
    p = _f64(p)
    nz, ny, nx = p.shape
    out = np.empty_like(p)
    _L().orc_laplacian(lat, nx, ny, nz, _p(p), _p(out))
    return out


def line_d2(p, start, axis, length):
    """p(x+e) - 2p(x) + p(x-e) at `length` cells from start=(x, y, z) along axis."""
    p = _f64(p)
    nz, ny, nx = p.shape
    out = np.empty(length)
    _L().orc_line_d2(nx, ny, nz, _p(p), int(start[0]), int(start[1]), int(start[2]),
                     int(axis), int(length), _p(out))
    return out


def label_gas(lat, rho, thr):
    """Face-connected periodic components of rho < thr; labels = min linear
    index of the component, -1 for liquid.  Returns (labels int32, ncomp)."""
    rho = _f64(rho)
    nz, ny, nx = rho.shape
    lab = np.empty(rho.shape, dtype=np.int32)
    n = _L().orc_label_gas(lat, nx, ny, nz, _p(rho), thr, _p(lab))
    return lab, int(n)


def totals(lat, f):
    """FP64 (M, Jx, Jy, Jz) summed cell by cell in velocity order."""
    f = _f64(f)
    q, nx, ny, nz = _shape(f)
    out = np.zeros(4)
    _L().orc_totals(lat, nx, ny, nz, _p(f), _p(out))
    return out


def film_probe(lat, rho, p, start, axis, length, rho_mid):
    """Film between two bubbles along a line from inside bubble A (Sec. 3.1,
    Sec. 4): dict(found, x1, x2, h, d2p_mid, r_d); see sc_oracle.c."""
    rho = _f64(rho)
    p = _f64(p)
    nz, ny, nx = rho.shape
    out = np.zeros(6)
    _L().orc_film_probe(lat, nx, ny, nz, _p(rho), _p(p), int(start[0]), int(start[1]),
                        int(start[2]), int(axis), int(length), float(rho_mid), _p(out))
    return dict(found=bool(out[0]), x1=out[1], x2=out[2], h=out[3], d2p_mid=out[4], r_d=out[5])


def bubble_sizes(labels):
    """(roots, sizes) of the gas components of a label field (label_gas), in
    increasing order of the root label (Sec. 4 bubble census)."""
    lab = np.ascontiguousarray(labels, dtype=np.int32)
    n = _L().orc_bubble_sizes(lab.size, _p(lab), 0, None, None)
    roots = np.zeros(max(n, 1), dtype=np.int64)
    sizes = np.zeros(max(n, 1), dtype=np.int64)
    _L().orc_bubble_sizes(lab.size, _p(lab), n, _p(roots), _p(sizes))
    return roots[:n], sizes[:n]


def size_histogram(sizes, nbins):
    """Counts of sizes s with 2^b <= s < 2^(b+1), b = 0..nbins-1 (the last bin
    open-ended)."""
    sz = np.ascontiguousarray(sizes, dtype=np.int64)
    hist = np.zeros(nbins, dtype=np.int64)
    _L().orc_size_histogram(len(sz), _p(sz), nbins, _p(hist))
    return hist


def film_cells(lat, labels, p, h_max, eps_arm, state, cap=1 << 16):
    """The per-lattice-point film test of Sec. 4 (see sc_oracle.c): updates
    the uint8 arming state (shape of the lattice) in place and returns
    (counts dict(film, midpoints, armed, fired), fired records (k, 5) int64
    = cell, axis, label on the -axis side, label on the +axis side,
    thickness; their d2 values)."""
    lab = np.ascontiguousarray(labels, dtype=np.int32)
    p = _f64(p)
    nz, ny, nx = lab.shape
    assert state.dtype == np.uint8 and state.shape == lab.shape and state.flags.c_contiguous
    counts = np.zeros(4, dtype=np.int64)
    rec = np.zeros((cap, 5), dtype=np.int64)
    d2 = np.zeros(cap)
    _L().orc_film_cells(lat, nx, ny, nz, _p(lab), _p(p), int(h_max), float(eps_arm), _p(state),
                        _p(counts), cap, _p(rec), _p(d2))
    nf = int(min(counts[3], cap))
    return (dict(film=int(counts[0]), midpoints=int(counts[1]), armed=int(counts[2]),
                 fired=int(counts[3])), rec[:nf], d2[:nf])


def run_spread(lat, f, steps, tau, G, sites, rate, budget, relabel_every, threshold=1.0):
    """Blowing agent spread over each site's bubble (a reading of Sec. 3:
    gas is added to each bubble every step until the agent is used up).
    Every ``relabel_every`` steps (from the first) the gas is labelled and
    each site takes the label of its cell.  Each step is the plain step of
    ``run`` without injection, followed by the deposits: for every bubble
    holding sites, its sites in increasing order take dm = min(rate, budget)
    from their budgets (``budget`` is updated in place) and the total D is
    spread evenly over the bubble's n cells, each population f_i of each of
    its cells gaining w_i D / n; a site whose cell is liquid adds w_i dm to
    its cell.  ``sites`` are linear cell indices.  Returns the populations."""
    f = _f64(f)
    _, w = velocities(lat)
    Q = len(w)
    sites = np.asarray(sites, dtype=np.int64)
    for t in range(steps):
        if t % relabel_every == 0:
            lab, _ = label_gas(lat, moments(lat, f)[0], threshold)
            lab_flat = lab.ravel()
            site_lab = lab_flat[sites]
            sizes = {}
            for root, size in zip(*bubble_sizes(lab)):
                sizes[int(root)] = int(size)
        f = run(lat, f, 1, tau, G)
        flat = f.reshape(Q, -1)
        groups = {}
        for s in range(len(sites)):
            key = int(site_lab[s]) if site_lab[s] >= 0 else -1 - int(sites[s])
            groups.setdefault(key, []).append(s)
        for key, members in groups.items():
            total = 0.0
            for s in members:
                d = min(rate[s], budget[s])
                budget[s] -= d
                total += d
            if key >= 0:
                per_cell = total / sizes[key]
                cells = np.nonzero(lab_flat == key)[0]
                for i in range(Q):
                    flat[i, cells] += w[i] * per_cell
            else:
                for i in range(Q):
                    flat[i, -1 - key] += w[i] * total
    return f


def film_midpoints(lat, labels, p, h_max, eps_arm, state, cap=1 << 20):
    """The film test of film_cells (the same arming update of ``state``)
    returning every film midpoint: (counts dict as film_cells, records (k, 6)
    int64 = cell, axis, label on the -axis side, label on the +axis side,
    thickness, fired flag, in increasing (cell, axis) order)."""
    lab = np.ascontiguousarray(labels, dtype=np.int32)
    p = _f64(p)
    nz, ny, nx = lab.shape
    assert state.dtype == np.uint8 and state.shape == lab.shape and state.flags.c_contiguous
    counts = np.zeros(5, dtype=np.int64)
    rec = np.zeros((cap, 6), dtype=np.int64)
    _L().orc_film_midpoints(lat, nx, ny, nz, _p(lab), _p(p), int(h_max), float(eps_arm),
                            _p(state), _p(counts), cap, _p(rec), None)
    n = int(min(counts[4], cap))
    return (dict(film=int(counts[0]), midpoints=int(counts[1]), armed=int(counts[2]),
                 fired=int(counts[3])), rec[:n])


def film_pairs(lat, shape, mids):
    """Per bubble pair census of the film test in a foam (Sec. 4: the
    criterion at each lattice point; Fig. 3's film disc radius R_d and
    critical thickness h_c per pair of bubbles).  ``mids`` are the midpoint
    records of film_midpoints on a lattice of ``shape`` = (nz, ny, nx).
    For each unordered pair of labels meeting in a film, and each axis: the
    lattice lines along the axis that hold a midpoint of the pair (a film of
    even thickness has two midpoints on one line), the midpoints, the
    thinnest run.  The pair's film lies across the axis with the most lines
    (the lower axis on a tie); the lines are its disc's area in cells, so
    R_d = sqrt(lines / pi) in 3-D and lines / 2 in 2-D (a film segment).
    h_c = mean thickness of the pair's fired midpoints (any axis), 0 when none
    fired.  Returns rows (label_a < label_b, axis, lines, midpoints, h_min,
    r_d, fired, h_c) in increasing (label_a, label_b) order."""
    nz, ny, nx = shape
    dims = 2 if lat == D2Q9 else 3
    groups = {}
    for cell, a, lm, lp, t, fired in np.asarray(mids, dtype=np.int64).reshape(-1, 6).tolist():
        x, y, z = cell % nx, (cell // nx) % ny, cell // (nx * ny)
        line = (y, z) if a == 0 else ((x, z) if a == 1 else (x, y))
        g = groups.setdefault((min(lm, lp), max(lm, lp)),
                              dict(lines=[set() for _ in range(dims)], mid=[0] * dims,
                                   hmin=[None] * dims, fired=0, tsum=0))
        g["lines"][a].add(line)
        g["mid"][a] += 1
        g["hmin"][a] = t if g["hmin"][a] is None else min(g["hmin"][a], t)
        if fired:
            g["fired"] += 1
            g["tsum"] += t
    rows = []
    for (la, lb) in sorted(groups):
        g = groups[(la, lb)]
        a = max(range(dims), key=lambda q: (len(g["lines"][q]), -q))
        n = len(g["lines"][a])
        r_d = float(np.sqrt(n / np.pi)) if dims == 3 else n / 2.0
        h_c = g["tsum"] / g["fired"] if g["fired"] else 0.0
        rows.append((la, lb, a, n, g["mid"][a], g["hmin"][a], r_d, g["fired"], h_c))
    return rows


def criterion_step(state, probe, eps_arm, h_max):
    """One probe of the rupture criterion of Sec. 3.1 / Sec. 4.  state is
    None at the start; probe = dict(found, h, d2p_mid, r_d) as film_probe.
    The criterion concerns a thin film (h <= h_max): it is armed once the
    film-midpoint d2p/dn2 has been below -eps_arm, disarmed whenever the film
    is thicker than h_max, and fires at the first probe of a thin film where
    d2p/dn2 >= 0.  A probe that finds no film is a merge before the
    criterion.  On firing, h_c is the thickness at the zero of d2p/dn2 on
    the straight line through the last two probes' (h, d2p) points (the
    previous probe had d2p < 0: otherwise the criterion would have fired or
    been disarmed there); h_probe and r_d are the firing probe's.
    Returns (state, outcome) with outcome None while the run goes on."""
    armed, last = (False, None) if state is None else state
    if not probe["found"]:
        return (armed, last), dict(fired=False, merged=True, h_c=0.0, h_probe=0.0, r_d=0.0)
    h, d = probe["h"], probe["d2p_mid"]
    if h > h_max:
        armed = False
    elif d < -eps_arm:
        armed = True
    elif armed and d >= 0.0:
        h0, d0 = last
        h_c = h0 + (h - h0) * (-d0 / (d - d0))
        return (armed, last), dict(fired=True, merged=False, h_c=h_c, h_probe=h,
                                   r_d=probe["r_d"])
    return (armed, (h, d)), None


def run_until_rupture(lat, f, tau, G, start, axis, length, rho_mid, eps_arm, max_steps,
                      diag_every, rho0=1.0, h_max=8.0):
    """The rupture criterion as a plain loop: advance f by diag_every steps,
    probe the film (film_probe on the FP64 density and pressure) and apply
    criterion_step, until it fires, the film is gone or max_steps.
    Returns dict(fired, merged, step, h_c, h_probe, r_d, f)."""
    state = None
    t = 0
    while t < max_steps:
        f = run(lat, f, diag_every, tau, G, rho0)
        t += diag_every
        rho = moments(lat, f)[0]
        _, p = eos(rho, G, rho0)
        pr = film_probe(lat, rho, p, start, axis, length, rho_mid)
        state, out = criterion_step(state, pr, eps_arm, h_max)
        if out is not None:
            return dict(step=t, f=f, **out)
    return dict(fired=False, merged=False, step=t, h_c=0.0, h_probe=0.0, r_d=0.0, f=f)


# ---- multi-lattice Shan-Chen (Sec. 3.1, Fig. 1) -----------------------------

def ml_coupling(nl, G, G_x, G_b, eta=None):
    """Coupling matrix of the multi-lattice model: lattice 0 = the fluid
    (self-attraction G), lattices 1..nl-1 = one gas lattice per bubble
    (fluid-gas coupling G_x, no self-coupling) and, between two different
    bubbles k and l, the barrier eta_m(k, l) G_b (eta: nl x nl array of 0/1,
    default all 1)."""
    Gm = np.zeros((nl, nl))
    Gm[0, 0] = G
    Gm[0, 1:] = G_x
    Gm[1:, 0] = G_x
    for k in range(1, nl):
        for l in range(1, nl):
            if k != l:
                Gm[k, l] = G_b * (1.0 if eta is None else float(eta[k][l]))
    return Gm


def ml_run(lat, f, nsteps, tau, Gm, rho0=1.0, sites=None, site_lattice=None, rate=None,
           budget=None):
    """Advance the lattices f (nl, Q, nz, ny, nx), copied, by nsteps of the
    multi-lattice step (orc_ml_step).  sites: linear cells; site_lattice:
    the lattice each site deposits into; budget is updated in place."""
    f = _f64(f).copy()
    nl, q, nz, ny, nx = f.shape
    Gm = _f64(Gm)
    assert Gm.shape == (nl, nl)
    n = 0 if sites is None else len(sites)
    sc = np.ascontiguousarray(sites, dtype=np.int64) if n else None
    sl = np.ascontiguousarray(site_lattice, dtype=np.int32) if n else None
    rt = _f64(rate) if n else None
    if n:
        assert budget is not None and budget.dtype == np.float64 and budget.flags.c_contiguous
    _L().orc_ml_run(lat, nx, ny, nz, nl, tau, _p(Gm), rho0, _p(f), int(nsteps), n, _p(sc),
                    _p(sl), _p(rt), _p(budget) if n else None)
    return f


def ml_force(lat, psi, Gm):
    """Multicomponent Shan-Chen force (Fx, Fy, Fz), each (nl, nz, ny, nx),
    from psi fields (nl, nz, ny, nx) and the coupling matrix."""
    psi = _f64(psi)
    nl, nz, ny, nx = psi.shape
    out = [np.empty_like(psi) for _ in range(3)]
    _L().orc_ml_force(lat, nx, ny, nz, nl, _p(psi), _p(_f64(Gm)), *[_p(o) for o in out])
    return tuple(out)


def ml_moments(lat, f):
    """(rho, jx, jy, jz) of every lattice, each (nl, nz, ny, nx)."""
    f = _f64(f)
    out = [moments(lat, f[s]) for s in range(f.shape[0])]
    return tuple(np.stack([o[m] for o in out]) for m in range(4))


def ml_pressure(rho, Gm, rho0=1.0):
    """Pressure of the coupled lattices, rho (nl, ...) -> p (...):
    p = rho_total/3 + 1/6 sum_s sum_t Gm[s][t] psi_s psi_t."""
    rho = _f64(rho)
    nl = rho.shape[0]
    p = np.empty(rho.shape[1:])
    _L().orc_ml_pressure(p.size, nl, _p(rho), _p(_f64(Gm)), rho0, _p(p))
    return p


def ml_init(lat, nx, ny, nz, bubbles, rho_l, rho_v, rho_gas, width, noise_amp, seed):
    """Initial lattices (nl = 1 + bubbles, Q, nz, ny, nx): the fluid as
    init() (liquid rho_l, its vapour rho_v inside the bubbles, noise), and
    bubble k's gas on lattice k: rho_gas inside bubble k with the same tanh
    profile, zero far outside it; every lattice at rest, f = w rho."""
    b = _f64(bubbles).reshape(-1, 4)
    f0, _ = init(lat, nx, ny, nz, b, rho_l, rho_v, width, noise_amp, seed)
    out = [f0]
    for k in range(len(b)):
        fk, _ = init(lat, nx, ny, nz, b[k:k + 1], 0.0, rho_gas, width, 0.0, seed)
        out.append(fk)
    return np.stack(out)


def ml_merge(f, Gm, k, l):
    """eta_m(k, l) = 0: bubble l's lattice is merged into bubble k's (Fig. 1
    steps 8-9, merging lattices): f_k += f_l, f_l = 0, and the pair's
    barrier coupling is removed.  Returns new (f, Gm)."""
    f = _f64(f).copy()
    Gm = _f64(Gm).copy()
    f[k] = f[k] + f[l]
    f[l] = 0.0
    Gm[k, l] = Gm[l, k] = 0.0
    return f, Gm


def ml_run_until_rupture(lat, f, tau, Gm, start, axis, length, rho_mid, eps_arm, max_steps,
                         diag_every, pair=(1, 2), rho0=1.0, h_max=8.0):
    """The rupture criterion on the multi-lattice model, as a plain loop:
    advance diag_every steps, probe the film on the fluid lattice's density
    with the coupled pressure (ml_pressure), apply criterion_step; when it
    fires, eta_m of the pair becomes 0 and the pair's lattices merge
    (ml_merge), and the run stops.  Returns dict(fired, merged, step, h_c,
    h_probe, r_d, f, Gm)."""
    state = None
    t = 0
    while t < max_steps:
        f = ml_run(lat, f, diag_every, tau, Gm, rho0)
        t += diag_every
        rho = ml_moments(lat, f)[0]
        p = ml_pressure(rho, Gm, rho0)
        pr = film_probe(lat, rho[0], p, start, axis, length, rho_mid)
        state, out = criterion_step(state, pr, eps_arm, h_max)
        if out is not None:
            if out["fired"]:
                f, Gm = ml_merge(f, Gm, pair[0], pair[1])
            return dict(step=t, f=f, Gm=Gm, **out)
    return dict(fired=False, merged=False, step=t, h_c=0.0, h_probe=0.0, r_d=0.0, f=f, Gm=Gm)
