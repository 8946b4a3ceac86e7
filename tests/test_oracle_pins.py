"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: each test checks a closed form,
an invariant, a special case that reduces to textbook lattice Boltzmann, a
published test vector, or a brute-force computation on a tiny input, chosen so
that a dropped term, a wrong sign, index or weight in the oracle fails one of
them.  CPU only.
"""
import math

import networkx as nx
import os

import numpy as np
import pytest
from scipy import integrate, optimize

import oracle as O

LATS = [O.D2Q9, O.D3Q19]


def textbook_feq(lat, rho, u):
    """Second-order Maxwell-Boltzmann equilibrium on a lattice with cs^2 = 1/3."""
    c, w = O.velocities(lat)
    cu = np.tensordot(c.astype(float), u, axes=([1], [0]))  # (Q, ...)
    uu = (u * u).sum(0)
    return w.reshape((-1,) + (1,) * rho.ndim) * rho * (1 + 3 * cu + 4.5 * cu**2 - 1.5 * uu)


# ---------------------------------------------------------------- tables / RNG

@pytest.mark.parametrize("lat", LATS)
def test_velocity_set_isotropy(lat):
    """Weights reproduce the lattice moments of a Maxwellian with cs^2 = 1/3 up
    to fourth order (this fixes every weight and every velocity)."""
    c, w = O.velocities(lat)
    c = c.astype(float)
    d = 2 if lat == O.D2Q9 else 3
    assert len(w) == (9 if lat == O.D2Q9 else 19)
    assert abs(w.sum() - 1) < 1e-15
    assert np.abs((w[:, None] * c).sum(0)).max() < 1e-15
    m2 = np.einsum("i,ia,ib->ab", w, c, c)
    assert np.allclose(m2[:d, :d], np.eye(d) / 3, atol=1e-15)
    m4 = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)[:d, :d, :d, :d]
    I = np.eye(d)
    iso = (np.einsum("ab,cd->abcd", I, I) + np.einsum("ac,bd->abcd", I, I)
           + np.einsum("ad,bc->abcd", I, I)) / 9
    assert np.allclose(m4, iso, atol=1e-15)
    # odd moments vanish
    assert np.abs(np.einsum("i,ia,ib,ic->abc", w, c, c, c)).max() < 1e-15
    # every velocity appears with its opposite, all distinct
    s = {tuple(v) for v in c.astype(int)}
    assert len(s) == len(w) and all(tuple(-np.array(v)) in s for v in s)


def test_splitmix64_published_vector():
    """SplitMix64 seeded with 1234567: the published first outputs
    (tests/golden/splitmix64_seed1234567.txt, with its citation)."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                        "splitmix64_seed1234567.txt")
    with open(path) as fh:
        want = [int(line) for line in fh if line.strip() and not line.startswith("#")]
    assert len(want) == 5
    assert [O.splitmix64(1234567, k) for k in range(len(want))] == want


# ---------------------------------------------------------------- EOS / psi

def test_eos_critical_point_closed_form():
    """p = rho/3 + G/6 psi^2 with psi = 1 - exp(-rho): dp/drho = d2p/drho2 = 0
    at G = -4, rho = ln 2 (psi psi' has its maximum 1/4 there)."""
    h = 1e-4
    r = np.array([math.log(2) - h, math.log(2), math.log(2) + h])
    _, p = O.eos(r, -4.0)
    assert abs((p[2] - p[0]) / (2 * h)) < 1e-7
    assert abs((p[2] - 2 * p[1] + p[0]) / h**2) < 1e-5
    psi, _ = O.eos(np.array([0.0, 1.0, 50.0]), 0.0)
    assert psi[0] == 0.0 and abs(psi[1] - (1 - math.exp(-1))) < 1e-16 and abs(psi[2] - 1) < 1e-15
    psi2, _ = O.eos(np.array([2.0]), 0.0, rho0=2.0)
    assert abs(psi2[0] - 2 * (1 - math.exp(-1))) < 1e-15


# ---------------------------------------------------------------- force

@pytest.mark.parametrize("lat", LATS)
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_force_on_cosine_psi(lat, axis):
    """For psi = a + b cos(k s) varying along one axis the weighted stencil
    reduces to F_s = -G psi (1/6)(psi(s+1) - psi(s-1)) = (G/3) b sin k sin(ks) psi,
    zero in the other axes."""
    if lat == O.D2Q9 and axis == 2:
        pytest.skip("no z axis in 2-D")
    n = 16
    shape = [1, n, n] if lat == O.D2Q9 else [n, n, n]  # (nz, ny, nx)
    G, a, b = -5.0, 0.6, 0.1
    k = 2 * math.pi * 3 / n
    s = np.arange(n, dtype=float)
    prof = a + b * np.cos(k * s)
    psi = np.empty(shape)
    idx = [slice(None)] * 3
    target_dim = 2 - axis  # array dims are (z, y, x)
    view = [1, 1, 1]
    view[target_dim] = n
    psi[...] = prof.reshape(view)
    F = O.force(lat, psi, G)
    expect = (G / 3) * b * math.sin(k) * np.sin(k * s).reshape(view) * psi
    for ax in range(3):
        if ax == axis:
            assert np.abs(F[ax] - expect).max() < 1e-15
        else:
            assert np.abs(F[ax]).max() < 1e-16


@pytest.mark.parametrize("lat", LATS)
def test_uniform_psi_gives_zero_force(lat):
    shape = (1, 8, 8) if lat == O.D2Q9 else (6, 5, 4)
    F = O.force(lat, np.full(shape, 0.7), -5.0)
    assert all(np.abs(f).max() == 0.0 for f in F)


# ---------------------------------------------------------------- collision / streaming

@pytest.mark.parametrize("lat", LATS)
@pytest.mark.parametrize("G", [0.0, -5.0])
def test_uniform_moving_equilibrium_is_fixed_point(lat, G):
    """A uniform f_eq(rho, u) is invariant: streaming moves identical values and
    the (zero) force leaves the equilibrium unchanged."""
    shape = (1, 6, 7) if lat == O.D2Q9 else (4, 5, 6)
    rho = np.full(shape, 1.3)
    u = np.zeros((3,) + shape)
    u[0], u[1] = 0.05, -0.03
    if lat == O.D3Q19:
        u[2] = 0.02
    f0 = textbook_feq(lat, rho, u)
    f1 = O.run(lat, f0, 3, 0.7, G)
    assert np.abs(f1 - f0).max() < 1e-15


@pytest.mark.parametrize("lat", LATS)
def test_streaming_direction(lat):
    """With tau huge the collision barely changes f: a marker added to
    population i at cell x0 shows up at x0 + c_i after one step."""
    c, w = O.velocities(lat)
    shape = (1, 5, 6) if lat == O.D2Q9 else (5, 6, 7)
    nz, ny, nx_ = shape
    x0 = (2, 3, 1 if lat == O.D3Q19 else 0)
    for i in range(len(w)):
        f = textbook_feq(lat, np.ones(shape), np.zeros((3,) + shape))
        f[i, x0[2], x0[1], x0[0]] += 1e-3
        g = O.run(lat, f, 1, 1e12, 0.0)
        d = g - textbook_feq(lat, np.ones(shape), np.zeros((3,) + shape))
        j = ((x0[0] + c[i, 0]) % nx_, (x0[1] + c[i, 1]) % ny, (x0[2] + c[i, 2]) % nz)
        assert abs(d[i, j[2], j[1], j[0]] - 1e-3) < 1e-12
        d[i, j[2], j[1], j[0]] = 0
        assert np.abs(d).max() < 1e-12


@pytest.mark.parametrize("lat", LATS)
def test_collision_adds_exactly_F_momentum(lat):
    """Velocity-shift forcing: post-collision momentum at x is j(x) + F(x) and
    post-collision mass is rho(x), for any tau (gathered from f(t+1) at x + c_i)."""
    c, w = O.velocities(lat)
    shape = (1, 12, 10) if lat == O.D2Q9 else (6, 7, 8)
    nz, ny, nx_ = shape
    bub = np.array([[4.0, 5.0, 2.0 if lat == O.D3Q19 else 0.0, 3.0]])
    f0, _ = O.init(lat, nx_, ny, nz, bub, 2.0, 0.15, 2.0, 1e-2, 7)
    f0 = O.run(lat, f0, 5, 0.8, -5.0)  # develop non-equilibrium parts and velocity
    tau, G = 0.73, -5.0
    rho, jx, jy, jz = O.moments(lat, f0)
    psi, _ = O.eos(rho, G)
    F = O.force(lat, psi, G)
    f1 = O.run(lat, f0, 1, tau, G)
    fs = np.empty_like(f1)
    for i in range(len(w)):
        fs[i] = np.roll(f1[i], shift=(-c[i, 2], -c[i, 1], -c[i, 0]), axis=(0, 1, 2))
    assert np.abs(fs.sum(0) - rho).max() < 1e-13
    for a, (j, Fa) in enumerate(zip((jx, jy, jz), F)):
        mom = np.tensordot(c[:, a].astype(float), fs, axes=(0, 0))
        assert np.abs(mom - (j + Fa)).max() < 1e-13


def test_shear_wave_viscosity():
    """G = 0: a shear wave u_y = A sin(kx) decays as exp(-nu k^2 t) with
    nu = cs^2 (tau - 1/2) (BGK lattice viscosity)."""
    for lat in LATS:
        n, tau, A = 64, 0.8, 1e-4
        shape = (1, 2, n) if lat == O.D2Q9 else (2, 2, n)
        k = 2 * math.pi / n
        x = np.arange(n)
        u = np.zeros((3,) + shape)
        u[1] = A * np.sin(k * x)
        f = textbook_feq(lat, np.ones(shape), u)
        T = 400
        g = O.run(lat, f, T, tau, 0.0)
        rho, jx, jy, jz = O.moments(lat, g)
        amp = 2.0 / n * ((jy / rho)[0, 0] * np.sin(k * x)).sum()
        rate = -math.log(amp / A) / T
        nu = (tau - 0.5) / 3
        assert abs(rate / (nu * k * k) - 1) < 5e-3, (lat, rate, nu * k * k)


# ---------------------------------------------------------------- conservation

@pytest.mark.parametrize("lat", LATS)
def test_mass_and_momentum_conserved_without_injection(lat):
    shape = (1, 24, 24) if lat == O.D2Q9 else (10, 12, 14)
    nz, ny, nx_ = shape
    bub = np.array([[6.0, 7.0, 4.0 if lat == O.D3Q19 else 0.0, 4.0],
                    [15.0, 14.0, 5.0 if lat == O.D3Q19 else 0.0, 3.0]])
    f0, _ = O.init(lat, nx_, ny, nz, bub, 2.0, 0.15, 2.0, 1e-3, 3)
    t0 = O.totals(lat, f0)
    f1 = O.run(lat, f0, 60, 0.9, -5.0)
    t1 = O.totals(lat, f1)
    assert abs(t1[0] - t0[0]) / t0[0] < 1e-13
    assert np.abs(t1[1:]).max() / t0[0] < 1e-13


def test_injection_ledger_and_placement():
    """Virtual blowing agent: the mass gained equals sum_s min(r_s t, B_s) and
    is deposited at the site after collision (so it streams to x_s + c_i)
    with zero momentum; budgets never go negative."""
    lat = O.D2Q9
    c, w = O.velocities(lat)
    n = 16
    f0 = textbook_feq(lat, np.ones((1, n, n)), np.zeros((3, 1, n, n)))
    sites = np.array([3 + n * 4, 11 + n * 12], dtype=np.int64)
    rate = np.array([1e-4, 3e-4])
    budget = np.array([0.01, 5e-3])
    # one step at tau = 1, G = 0 from rest: rho(x_s + c_i) = 1 + w_i r_s
    b1 = budget.copy()
    f1 = O.run(lat, f0, 1, 1.0, 0.0, sites=sites, rate=rate, budget=b1)
    rho1 = O.moments(lat, f1)[0][0]
    expect = np.ones((n, n))
    for s, r in zip(sites, rate):
        x, y = s % n, s // n
        for i in range(9):
            expect[(y + c[i, 1]) % n, (x + c[i, 0]) % n] += w[i] * r
    assert np.abs(rho1 - expect).max() < 1e-15
    assert np.allclose(b1, budget - rate, rtol=0, atol=1e-18)
    # ledger over 120 steps with G = -5 (site 2 exhausts after ~17 steps)
    b = budget.copy()
    t0 = O.totals(lat, f0)
    T = 120
    g = O.run(lat, f0, T, 0.9, -5.0, sites=sites, rate=rate, budget=b)
    t1 = O.totals(lat, g)
    added = sum(min(r * T, B) for r, B in zip(rate, budget))
    assert abs((t1[0] - t0[0]) - added) < 1e-13 * t0[0]
    assert np.abs(t1[1:]).max() < 1e-12
    assert (b >= 0).all() and b[1] == 0.0


# ---------------------------------------------------------------- phase behaviour

def _run_cosine(G, steps=400):
    n = 64
    k = 2 * math.pi / n
    rho = math.log(2) + 1e-3 * np.cos(k * np.arange(n)).reshape(1, 1, n)
    f = textbook_feq(O.D2Q9, rho, np.zeros((3, 1, 1, n)))
    g = O.run(O.D2Q9, f, steps, 1.0, G)
    r = O.moments(O.D2Q9, g)[0][0, 0]
    return r.max() - r.min()


def test_phase_separation_only_below_critical_G():
    """Uniform rho = ln 2 with a long-wave perturbation is unstable only when
    dp/drho < 0, i.e. G < -4 for psi = 1 - exp(-rho)."""
    assert _run_cosine(-4.8) > 2e-2      # grew by > 10x
    assert _run_cosine(-3.2) < 2e-3      # did not grow


def _coexistence_integral(G, eps):
    """Mechanical-stability coexistence (Shan & Chen 1994 form):
    p(rho_g) = p(rho_l) = p0 and int (p0 - p) psi'/psi^(1+eps) drho = 0."""
    psi = lambda r: 1 - np.exp(-r)
    dpsi = lambda r: np.exp(-r)
    p = lambda r: r / 3 + G / 6 * psi(r) ** 2

    def eqs(v):
        rg, rl = v
        p0 = p(rl)
        I = integrate.quad(lambda r: (p0 - p(r)) * dpsi(r) / psi(r) ** (1 + eps), rg, rl,
                           epsabs=1e-13, epsrel=1e-12)[0]
        return [p(rg) - p(rl), I]

    return optimize.fsolve(eqs, [0.15, 1.9], xtol=1e-13)


def test_flat_interface_coexistence():
    """A flat interface relaxes to bulk densities with equal EOS pressure
    (momentum balance across the interface for the pairwise force) close to
    the Shan-Chen mechanical-stability prediction."""
    n = 64
    pg, pl = _coexistence_integral(-5.0, 1.0)
    bub = np.array([[0.0, 0.0, 0.0, 16.0]])
    f, _ = O.init(O.D2Q9, n, 1, 1, bub, pl, pg, 4.0, 0.0, 0)
    g = O.run(O.D2Q9, f, 20000, 1.0, -5.0)
    rho = O.moments(O.D2Q9, g)[0][0, 0]
    rg, rl = rho[0], rho[n // 2]
    _, p = O.eos(np.array([rg, rl]), -5.0)
    assert abs(p[0] - p[1]) < 1e-9
    assert abs(rl / pl - 1) < 0.03 and abs(rg / pg - 1) < 0.03, (rg, rl, pg, pl)


def test_laplace_law():
    """Liquid drops of radius R in gas: p_in - p_out = sigma / R (2-D Laplace
    law): linear in 1/R with a vanishing intercept."""
    n = 64
    dp, Rm = [], []
    for R in (8.0, 10.0, 12.0, 14.0, 16.0):
        drop = np.array([[n / 2, n / 2, 0.0, R]])
        # inside the disk takes the second density: a liquid drop in gas
        f, _ = O.init(O.D2Q9, n, n, 1, drop, 0.1555, 1.9315, 2.0, 0.0, 0)
        g = O.run(O.D2Q9, f, 3000, 1.0, -5.0)
        rho = O.moments(O.D2Q9, g)[0][0]
        _, p = O.eos(rho, -5.0)
        rin, rout = rho[n // 2, n // 2], rho[0, 0]
        dp.append(p[n // 2, n // 2] - p[0, 0])
        # equivalent radius from the excess liquid mass
        Rm.append(math.sqrt(((rho - rout) / (rin - rout)).sum() / math.pi))
    dp, Rm = np.array(dp), np.array(Rm)
    A = np.vstack([1 / Rm, np.ones_like(Rm)]).T
    (sigma, b), res, *_ = np.linalg.lstsq(A, dp, rcond=None)
    r2 = 1 - res[0] / ((dp - dp.mean()) ** 2).sum()
    assert sigma > 0 and r2 > 0.999 and abs(b) < 0.05 * dp[0], (sigma, b, r2)


# ---------------------------------------------------------------- diagnostics

@pytest.mark.parametrize("lat", LATS)
def test_laplacian_eigenvalues(lat):
    shape = (1, 12, 10) if lat == O.D2Q9 else (6, 12, 10)
    nz, ny, nx_ = shape
    ks = (2, 3, 1)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx_), indexing="ij")
    ax = 2 * math.pi * ks[0] / nx_
    ay = 2 * math.pi * ks[1] / ny
    az = 2 * math.pi * ks[2] / nz if lat == O.D3Q19 else 0.0
    p = np.cos(ax * x) * np.cos(ay * y) * np.cos(az * z)
    lam = 2 * (math.cos(ax) - 1) + 2 * (math.cos(ay) - 1)
    if lat == O.D3Q19:
        lam += 2 * (math.cos(az) - 1)
    assert np.abs(O.laplacian(lat, p) - lam * p).max() < 1e-13
    d2 = O.line_d2(p, (0, 5, min(3, nz - 1)), 0, nx_)
    assert np.abs(d2 - 2 * (math.cos(ax) - 1) * p[min(3, nz - 1), 5, :]).max() < 1e-14
    d2y = O.line_d2(p, (4, 0, 0), 1, ny + 3)  # wraps around
    yy = np.arange(ny + 3) % ny
    assert np.abs(d2y - 2 * (math.cos(ay) - 1) * p[0, yy, 4]).max() < 1e-14


def _labels_networkx(mask):
    nz, ny, nx_ = mask.shape
    g = nx.Graph()
    dims = [(0, 0, 1), (0, 1, 0)] + ([(1, 0, 0)] if nz > 1 else [])
    for z, y, x in zip(*np.nonzero(mask)):
        k = x + nx_ * (y + ny * z)
        g.add_node(k)
        for dz, dy, dx in dims:
            zz, yy, xx = (z + dz) % nz, (y + dy) % ny, (x + dx) % nx_
            if mask[zz, yy, xx]:
                g.add_edge(k, xx + nx_ * (yy + ny * zz))
    lab = -np.ones(mask.size, dtype=np.int64)
    comps = list(nx.connected_components(g))
    for comp in comps:
        m = min(comp)
        for k in comp:
            lab[k] = m
    return lab.reshape(mask.shape), len(comps)


@pytest.mark.parametrize("seed", range(6))
def test_labels_match_graph_components(seed):
    rng = np.random.default_rng(seed)
    lat = O.D2Q9 if seed % 2 == 0 else O.D3Q19
    shape = (1, 9, 11) if lat == O.D2Q9 else (5, 6, 7)
    rho = rng.uniform(0.0, 2.0, size=shape)
    lab, n = O.label_gas(lat, rho, 0.9)
    ref, nref = _labels_networkx(rho < 0.9)
    assert n == nref and (lab == ref).all()


def test_labels_wraparound_and_threshold_edge():
    rho = np.full((1, 6, 8), 2.0)
    rho[0, 2, 0] = rho[0, 2, 7] = 0.5    # joined through the x wrap
    rho[0, 0, 3] = rho[0, 5, 3] = 0.5    # joined through the y wrap
    rho[0, 4, 5] = 1.0                   # exactly at threshold: liquid
    lab, n = O.label_gas(O.D2Q9, rho, 1.0)
    assert n == 2
    assert lab[0, 2, 0] == lab[0, 2, 7] == 16
    assert lab[0, 0, 3] == lab[0, 5, 3] == 3
    assert lab[0, 4, 5] == -1


# ---------------------------------------------------------------- initial state, sites

def test_init_profile_closed_form():
    n = 16
    bub = np.array([[3.0, 4.0, 0.0, 5.0]])
    f, rho = O.init(O.D2Q9, n, n, 1, bub, 2.0, 0.15, 2.0, 0.0, 0)
    mid = 0.5 * (2.0 + 0.15)
    assert abs(rho[0, 4, 8] - mid) < 1e-15     # d = r
    assert abs(rho[0, 4, 14] - mid) < 1e-15    # d = r through the wrap
    assert abs(rho[0, 4, 3] - (0.15 + 0.5 * 1.85 * (1 + math.tanh(-5.0)))) < 1e-15
    c, w = O.velocities(O.D2Q9)
    assert np.abs(f - w[:, None, None, None] * rho).max() == 0
    f2, rho2 = O.init(O.D2Q9, n, n, 1, None, 2.0, 0.15, 2.0, 1e-3, 5)
    noise = rho2 - 2.0
    assert np.abs(noise).max() <= 1e-3 and abs(noise.mean()) < 2e-4 and noise.std() > 4e-4


def test_sites_spacing_and_determinism():
    got, s = O.sample_sites(128, 128, 128, 64, 3.0, 3.0, 12.0, 0.0, 1)
    assert got == 64
    assert (s[:, :3] >= 0).all() and (s[:, :3] < 128).all() and (s[:, :3] == np.floor(s[:, :3])).all()
    d = s[:, None, :3] - s[None, :, :3]
    d = (d + 64) % 128 - 64
    dist = np.sqrt((d ** 2).sum(-1)) + np.eye(64) * 1e9
    assert dist.min() >= 12.0
    got2, s2 = O.sample_sites(128, 128, 128, 64, 3.0, 3.0, 12.0, 0.0, 1)
    assert (s2 == s).all()
    got3, s3 = O.sample_sites(64, 64, 64, 30, 4.0, 12.0, 0.0, 4.0, 2)
    assert got3 == 30 and (s3[:, 3] >= 4).all() and (s3[:, 3] < 12).all()
    d = s3[:, None, :3] - s3[None, :, :3]
    d = (d + 32) % 64 - 32
    dist = np.sqrt((d ** 2).sum(-1))
    need = s3[:, None, 3] + s3[None, :, 3] + 4.0
    off = ~np.eye(30, dtype=bool)
    assert (dist[off] >= need[off]).all()


def test_step_cells_matches_full_step():
    """The one-cell-at-a-time update (used on lattices too large for a full
    oracle run) agrees with the full step."""
    lat = O.D3Q19
    nz, ny, nx_ = 7, 6, 9
    bub = np.array([[4.0, 3.0, 3.0, 2.5]])
    f0, _ = O.init(lat, nx_, ny, nz, bub, 2.0, 0.15, 2.0, 1e-3, 4)
    f0 = O.run(lat, f0, 3, 0.8, -5.0)
    f1 = O.run(lat, f0, 1, 0.8, -5.0)
    cells = np.array([0, 5, 17, 100, nx_ * ny * nz - 1])
    out = O.step_cells(lat, f0, cells, 0.8, -5.0)
    ref = f1.reshape(19, -1)[:, cells].T
    assert np.abs(out - ref).max() < 1e-15


# ---------------------------------------------------------------- film probe

def test_film_probe_constructed_slab_and_parabola():
    """Two gas blocks separated by a liquid slab whose width is exact under
    linear interpolation; p a parabola with known second difference; the
    film disc of a slab that widens beyond |dy| = J has R_d = (2J + 1)/2."""
    nx, ny = 40, 30
    rho = np.full((1, ny, nx), 2.0)
    rg, rl, mid = 0.2, 2.0, 1.1
    J = 4
    for y in range(ny):
        dy = abs(y - 15)
        gap = 6 if dy <= J else 12          # liquid cells between the blocks
        a_end = 20 - gap // 2               # gas block A: x in [5, a_end)
        rho[0, y, 5:a_end] = rg
        rho[0, y, a_end + gap:35] = rg
    p = 0.05 * (np.arange(nx) - 17.25) ** 2 * np.ones((1, ny, 1))
    r = O.film_probe(O.D2Q9, rho, p, (8, 15, 0), 0, 25, mid)
    # crossings: between gas cell a_end-1 and liquid a_end at fraction 0.5
    a_end = 17
    assert r["found"]
    assert abs(r["x1"] - (a_end - 1 - 8 + 0.5)) < 1e-12
    assert abs(r["h"] - 6.0) < 1e-12
    assert abs(r["d2p_mid"] - 0.1) < 1e-12          # 2 * 0.05
    assert r["r_d"] == (2 * J + 1) / 2
    # no film once the blocks touch
    rho2 = rho.copy()
    rho2[0, 15, :] = rg
    r2 = O.film_probe(O.D2Q9, rho2, p, (8, 15, 0), 0, 25, mid)
    assert not r2["found"]


def test_film_probe_disc_radius_of_a_wedge():
    """A film whose liquid run widens by one cell per row away from the
    centre row: rows with run <= h + 2 form the disc, so R_d = 5/2."""
    nx, ny = 48, 30
    rho = np.full((1, ny, nx), 2.0)
    rg, mid = 0.2, 1.1
    for y in range(ny):
        gap = 6 + abs(y - 15)
        a_end = 24 - gap // 2
        rho[0, y, 4:a_end] = rg
        rho[0, y, a_end + gap:44] = rg
    p = np.zeros((1, ny, nx))
    r = O.film_probe(O.D2Q9, rho, p, (8, 15, 0), 0, 30, mid)
    assert r["found"] and abs(r["h"] - 6.0) < 1e-12
    assert r["r_d"] == 2.5


def test_film_probe_midpoint_tie_averages():
    nx = 32
    rho = np.full((1, 1, nx), 2.0)
    rho[0, 0, :10] = 0.2
    rho[0, 0, 15:] = 0.2                   # liquid cells 10..14, crossings 9.5 and 14.5
    p = np.zeros((1, 1, nx))
    p[0, 0, 12] = 1.0                      # d2(12) = -2, d2(11) = d2(13) = 1
    r = O.film_probe(O.D2Q9, rho, p, (0, 0, 0), 0, 30, 1.1)
    assert abs(r["x1"] - 9.5) < 1e-12 and abs(r["x2"] - 14.5) < 1e-12
    assert r["d2p_mid"] == -2.0            # midpoint 12.0: nearest cell
    p2 = np.zeros((1, 1, nx))
    rho[0, 0, 14] = 0.2                    # liquid 10..13: midpoint 11.5 -> tie
    p2[0, 0, 11] = 1.0
    r2 = O.film_probe(O.D2Q9, rho, p2, (0, 0, 0), 0, 30, 1.1)
    assert abs(r2["d2p_mid"] - 0.5 * (-2.0 + 1.0)) < 1e-15


def _run_criterion(probes, eps_arm=1e-3, h_max=8.0):
    state = None
    for k, pr in enumerate(probes):
        state, out = O.criterion_step(state, pr, eps_arm, h_max)
        if out is not None:
            return k, out
    return None, None


def _pr(h, d, r_d=4.5, found=True):
    return dict(found=found, h=h, d2p_mid=d, r_d=r_d)


def test_criterion_zero_crossing_of_a_linear_film():
    """A film thinning at a constant rate with d2p/dn2 = a (h* - h): the
    interpolated zero crossing is h* exactly (to rounding), whatever the
    probe spacing; h_probe is the first probe past it."""
    for dh in (0.05, 0.13, 0.4):
        hs = 6.0 - dh * np.arange(int(5.0 / dh))
        probes = [_pr(h, 0.02 * (2.37 - h)) for h in hs]
        k, out = _run_criterion(probes)
        assert out["fired"] and not out["merged"]
        assert hs[k] <= 2.37 < hs[k - 1]
        assert abs(out["h_c"] - 2.37) < 1e-12 and out["h_probe"] == hs[k]


def test_criterion_arming_disarming_and_merge():
    # never below -eps_arm: never armed, never fires
    k, out = _run_criterion([_pr(5.0, -5e-4), _pr(4.0, 1e-3), _pr(3.0, 2e-3)])
    assert out is None
    # armed, then the film thickens past h_max: disarmed, a later d >= 0 does not fire
    k, out = _run_criterion([_pr(6.0, -2e-3), _pr(9.0, 0.0), _pr(7.0, 1e-3)])
    assert out is None
    # armed by a thin film, fires at the first d >= 0; d = 0 exactly counts
    k, out = _run_criterion([_pr(12.0, 1.0), _pr(6.0, -2e-3), _pr(5.0, -1e-3), _pr(4.0, 0.0)])
    assert k == 3 and out["fired"] and out["h_c"] == 4.0
    # a probe without film ends the run as a merge, armed or not
    k, out = _run_criterion([_pr(6.0, -2e-3), _pr(0.0, 0.0, found=False)])
    assert k == 1 and out["merged"] and not out["fired"]
    # a film thicker than h_max with d >= 0 after arming does not fire
    k, out = _run_criterion([_pr(7.9, -2e-3), _pr(8.1, 5e-3), _pr(7.0, -5e-4), _pr(6.0, 1e-3)])
    assert out is None


# ---------------------------------------------------------------- bubble census

@pytest.mark.parametrize("shape,lat", [((1, 12, 17), "D2Q9"), ((6, 7, 9), "D3Q19")])
def test_bubble_sizes_match_graph_components(shape, lat):
    """Component sizes against networkx on random masks (periodic, face
    connectivity), keyed by the smallest cell index of each component."""
    nx_ = pytest.importorskip("networkx")
    rng = np.random.default_rng(7)
    nz, ny, nx = shape
    for trial in range(4):
        rho = np.where(rng.random(shape) < 0.45, 0.3, 1.7)
        lab, n = O.label_gas(O.D2Q9 if lat == "D2Q9" else O.D3Q19, rho, 1.0)
        roots, sizes = O.bubble_sizes(lab)
        g = nx_.Graph()
        gas = np.argwhere(rho.reshape(-1) < 1.0).reshape(-1)
        g.add_nodes_from(gas.tolist())
        for k in gas:
            x, y, z = k % nx, (k // nx) % ny, k // (nx * ny)
            for dx, dy, dz in ((1, 0, 0), (0, 1, 0), (0, 0, 1)):
                if lat == "D2Q9" and dz:
                    continue
                m = (x + dx) % nx + nx * (((y + dy) % ny) + ny * ((z + dz) % nz))
                if rho.reshape(-1)[m] < 1.0:
                    g.add_edge(int(k), int(m))
        comps = sorted((min(c), len(c)) for c in nx_.connected_components(g))
        assert n == len(comps) == len(roots)
        assert [int(r) for r in roots] == [c[0] for c in comps]
        assert [int(s) for s in sizes] == [c[1] for c in comps]
        assert sizes.sum() == (rho < 1.0).sum()


def test_size_histogram_bins():
    sizes = [1, 2, 3, 4, 7, 8, 15, 16, 1000, 1]
    assert list(O.size_histogram(sizes, 4)) == [2, 2, 2, 4]
    assert list(O.size_histogram(sizes, 12)) == [2, 2, 2, 2, 1, 0, 0, 0, 0, 1, 0, 0]
    assert list(O.size_histogram([], 3)) == [0, 0, 0]


# ------------------------------------------------------- film at every lattice point

def _slab_labels(nx, ny, a_lo, a_hi, t, gap_gas=None):
    """Two gas blocks across all rows: A = [a_lo, a_hi), B = [a_hi + t, a_hi + t +
    (a_hi - a_lo)); labels as label_gas gives them."""
    rho = np.full((1, ny, nx), 2.0)
    rho[0, :, a_lo:a_hi] = 0.2
    rho[0, :, a_hi + t:a_hi + t + (a_hi - a_lo)] = 0.2
    lab, n = O.label_gas(O.D2Q9, rho, 1.0)
    return lab, n


@pytest.mark.parametrize("t", [3, 4, 12])
def test_film_cells_slab_arm_then_fire(t):
    """A liquid slab of t cells between two bubbles (x axis): t film cells per
    row, 1 (odd t) or 2 (even t) midpoints per row; a pressure with d2 < 0
    arms every midpoint, one with d2 >= 0 then fires every one, with the
    bubbles' labels on the two sides and the thickness t."""
    nx, ny, h_max = 48, 5, 12
    lab, n = _slab_labels(nx, ny, 4, 12, t)
    assert n == 2
    xs = np.arange(nx, dtype=float)[None, None, :] * np.ones((1, ny, 1))
    state = np.zeros(lab.shape, dtype=np.uint8)
    mids = 1 if t % 2 else 2
    c1, r1, d21 = O.film_cells(O.D2Q9, lab, -0.01 * xs ** 2, h_max, 1e-3, state)
    assert c1 == dict(film=t * ny, midpoints=mids * ny, armed=mids * ny, fired=0)
    c2, r2, d22 = O.film_cells(O.D2Q9, lab, 0.01 * xs ** 2, h_max, 1e-3, state)
    assert c2 == dict(film=t * ny, midpoints=mids * ny, armed=0, fired=mids * ny)
    a_root, b_root = 4, 12 + t
    xm = [12 + (t - 1) // 2] if t % 2 else [12 + t // 2 - 1, 12 + t // 2]
    want = sorted(x + nx * y for y in range(ny) for x in xm)
    assert list(r2[:, 0]) == want
    assert (r2[:, 1] == 0).all() and (r2[:, 2] == a_root).all() and (r2[:, 3] == b_root).all()
    assert (r2[:, 4] == t).all() and np.allclose(d22, 0.02)
    # a third call: nothing is armed any more
    c3, _, _ = O.film_cells(O.D2Q9, lab, 0.01 * xs ** 2, h_max, 1e-3, state)
    assert c3["fired"] == 0 and c3["armed"] == 0


def test_film_cells_rules():
    nx, ny = 48, 4
    xs = np.arange(nx, dtype=float)[None, None, :] * np.ones((1, ny, 1))
    p_arm, p_fire = -0.01 * xs ** 2, 0.01 * xs ** 2
    # thicker than h_max: no film
    lab, _ = _slab_labels(nx, ny, 4, 12, 9)
    st = np.zeros(lab.shape, dtype=np.uint8)
    c, _, _ = O.film_cells(O.D2Q9, lab, p_arm, 8, 1e-3, st)
    assert c["film"] == 0 and c["midpoints"] == 0
    # one bubble seen on both sides through the periodic wrap: no film
    rho = np.full((1, ny, 12), 2.0)
    rho[0, :, 0:6] = 0.2
    lab1, n1 = O.label_gas(O.D2Q9, rho, 1.0)
    assert n1 == 1
    c, _, _ = O.film_cells(O.D2Q9, lab1, np.zeros_like(rho), 12, 1e-3,
                           np.zeros(lab1.shape, dtype=np.uint8))
    assert c["film"] == 0
    # armed, then the film thickens beyond h_max: disarmed, no fire afterwards
    lab4, _ = _slab_labels(nx, ny, 4, 12, 4)
    st = np.zeros(lab4.shape, dtype=np.uint8)
    O.film_cells(O.D2Q9, lab4, p_arm, 12, 1e-3, st)
    assert st.any()
    lab10, _ = _slab_labels(nx, ny, 4, 12, 10)
    c, _, _ = O.film_cells(O.D2Q9, lab10, p_fire, 8, 1e-3, st)
    assert c["film"] == 0 and c["armed"] == 0 and not st.any()
    c, _, _ = O.film_cells(O.D2Q9, lab4, p_fire, 12, 1e-3, st)
    assert c["fired"] == 0
    # |d2| below eps_arm neither arms nor fires
    st = np.zeros(lab4.shape, dtype=np.uint8)
    c, _, _ = O.film_cells(O.D2Q9, lab4, -1e-4 * xs ** 2, 12, 1e-3, st)
    assert c["armed"] == 0


def test_film_cells_3d_along_z():
    """Two gas slabs stacked in z with a 5-cell liquid layer: the film runs
    along z only; midpoints on the middle plane."""
    nx, ny, nz = 6, 5, 30
    rho = np.full((nz, ny, nx), 2.0)
    rho[2:8] = 0.2
    rho[13:19] = 0.2
    lab, n = O.label_gas(O.D3Q19, rho, 1.0)
    assert n == 2
    zs = np.arange(nz, dtype=float)[:, None, None] * np.ones((1, ny, nx))
    st = np.zeros(lab.shape, dtype=np.uint8)
    c, _, _ = O.film_cells(O.D3Q19, lab, -0.01 * zs ** 2, 12, 1e-3, st)
    assert c["film"] == 5 * nx * ny and c["midpoints"] == nx * ny and c["armed"] == nx * ny
    assert (st[10] == 4).all() and st.sum() == 4 * nx * ny
    c, r, _ = O.film_cells(O.D3Q19, lab, 0.01 * zs ** 2, 12, 1e-3, st)
    assert c["fired"] == nx * ny and (r[:, 1] == 2).all() and (r[:, 0] // (nx * ny) == 10).all()


# ------------------------------------------------------- film pairs (per pair)
def test_film_pairs_disc_between_two_gas_cylinders():
    """Two gas cylinders of radius 4 stacked in z with a 5-cell liquid layer
    between them: the film is the disc of (x, y) lines inside the cylinders,
    across z only, thinnest run 5; R_d = sqrt(lines / pi).  Armed, then
    fired on every line with h_c = 5."""
    nx, ny, nz = 16, 16, 30
    xx, yy = np.meshgrid(np.arange(nx), np.arange(ny))
    disc = (xx - 7.5) ** 2 + (yy - 7.5) ** 2 <= 16.0
    lines = int(disc.sum())
    rho = np.full((nz, ny, nx), 2.0)
    rho[2:8][:, disc] = 0.2
    rho[13:19][:, disc] = 0.2
    lab, n = O.label_gas(O.D3Q19, rho, 1.0)
    assert n == 2
    zs = np.arange(nz, dtype=float)[:, None, None] * np.ones((1, ny, nx))
    st = np.zeros(lab.shape, dtype=np.uint8)
    c, mids = O.film_midpoints(O.D3Q19, lab, -0.01 * zs ** 2, 12, 1e-3, st)
    assert c["midpoints"] == lines == len(mids)
    rows = O.film_pairs(O.D3Q19, lab.shape, mids)
    la, lb = sorted({int(v) for v in lab.ravel() if v >= 0})
    assert len(rows) == 1
    assert rows[0][:6] == (la, lb, 2, lines, lines, 5)
    assert rows[0][6] == pytest.approx(np.sqrt(lines / np.pi)) and rows[0][7:] == (0, 0.0)
    c2, mids2 = O.film_midpoints(O.D3Q19, lab, 0.01 * zs ** 2, 12, 1e-3, st)
    rows2 = O.film_pairs(O.D3Q19, lab.shape, mids2)
    assert c2["fired"] == lines and rows2[0][7] == lines and rows2[0][8] == 5.0


@pytest.mark.parametrize("t", [3, 4])
def test_film_pairs_2d_slab_counts_lines_not_midpoints(t):
    """A 2-D slab film across every row: an even thickness has two midpoints
    per row, but the film segment still has one line per row: lines = ny,
    R_d = ny / 2, midpoints = ny or 2 ny."""
    nx, ny = 48, 6
    lab, n = _slab_labels(nx, ny, 4, 12, t)
    st = np.zeros(lab.shape, dtype=np.uint8)
    c, mids = O.film_midpoints(O.D2Q9, lab, np.zeros(lab.shape), 12, 1e-3, st)
    rows = O.film_pairs(O.D2Q9, lab.shape, mids)
    per_row = 1 if t % 2 else 2
    assert rows == [(4, 12 + t, 0, ny, per_row * ny, t, ny / 2.0, 0, 0.0)]
    assert c["midpoints"] == per_row * ny


def test_film_pairs_three_bubbles_two_films():
    """Gas blocks A | B | C along x: a 3-cell film A-B over rows 0..9 and a
    5-cell film B-C over rows 0..3 (C is 4 rows tall): two pairs, each with
    its own lines and thickness, in increasing label order; the midpoint
    totals add up to the census."""
    nx, ny = 60, 16
    rho = np.full((1, ny, nx), 2.0)
    rho[0, 0:10, 4:12] = 0.2      # A
    rho[0, 0:10, 15:25] = 0.2     # B (3 liquid cells after A)
    rho[0, 0:4, 30:38] = 0.2      # C (5 liquid cells after B)
    lab, n = O.label_gas(O.D2Q9, rho, 1.0)
    assert n == 3
    st = np.zeros(lab.shape, dtype=np.uint8)
    c, mids = O.film_midpoints(O.D2Q9, lab, np.zeros(lab.shape), 12, 1e-3, st)
    rows = O.film_pairs(O.D2Q9, lab.shape, mids)
    A, B, Cc = 4, 15, 30
    assert [r[:6] for r in rows] == [(A, B, 0, 10, 10, 3), (B, Cc, 0, 4, 4, 5)]
    assert sum(r[4] for r in rows) == c["midpoints"] == len(mids)


def test_film_pairs_h_min_is_the_thinnest_line():
    """Gas blocks A and B over rows 0..9 with a film along x whose thickness
    alternates 3 (even rows) and 5 (odd rows): one film line per row,
    h_min = 3 (not the thickest run, 5); R_d = 10 / 2."""
    nx, ny = 40, 30
    rho = np.full((1, ny, nx), 2.0)
    rho[0, 0:10, 4:12] = 0.2                       # A
    for y in range(10):
        rho[0, y, 12 + (3 if y % 2 == 0 else 5):25] = 0.2   # B, a comb on its left side
    lab, n = O.label_gas(O.D2Q9, rho, 1.0)
    assert n == 2
    st = np.zeros(lab.shape, dtype=np.uint8)
    c, mids = O.film_midpoints(O.D2Q9, lab, np.zeros(lab.shape), 12, 1e-3, st)
    rows = O.film_pairs(O.D2Q9, lab.shape, mids)
    assert rows == [(4, 15, 0, 10, 10, 3, 5.0, 0, 0.0)]


def test_film_pairs_axis_with_most_lines_not_most_midpoints():
    """Gas block A (x 0..9, rows 0..9) and an L-shaped B: an arm right of A
    over rows 0..2 leaves an even 4-cell film along x (3 lines, 6
    midpoints); an arm above A over columns 6..9 leaves an odd 3-cell film
    along y (4 lines, 4 midpoints); a connector far to the right joins the
    arms (none of B's other runs comes within 12 cells of A).  The film
    lies across the axis with the most lines, y:
    (A, B, axis 1, 4 lines, 4 midpoints, h_min 3, R_d 2)."""
    nx, ny = 48, 30
    rho = np.full((1, ny, nx), 2.0)
    rho[0, 0:10, 0:10] = 0.2      # A
    rho[0, 0:3, 14:31] = 0.2      # B: arm right of A (liquid x 10..13)
    rho[0, 0:17, 26:31] = 0.2     # B: connector
    rho[0, 13:17, 6:31] = 0.2     # B: arm above A (liquid rows 10..12 over x 6..9)
    lab, n = O.label_gas(O.D2Q9, rho, 1.0)
    assert n == 2
    st = np.zeros(lab.shape, dtype=np.uint8)
    c, mids = O.film_midpoints(O.D2Q9, lab, np.zeros(lab.shape), 12, 1e-3, st)
    by_axis = [int((np.asarray(mids)[:, 1] == a).sum()) for a in (0, 1)]
    assert by_axis == [6, 4]
    rows = O.film_pairs(O.D2Q9, lab.shape, mids)
    assert rows == [(0, 14, 1, 4, 4, 3, 2.0, 0, 0.0)]


# ---------------------------------------------- injection spread over a bubble
def _disk_state(nx=48, ny=40, r=8.0, seed=3):
    f, rho = O.init(O.D2Q9, nx, ny, 1, np.array([[20.0, 20.0, 0.0, r]]), 2.0, 0.15, 2.0, 1e-3,
                    seed)
    return f, rho


def test_spread_injection_deposit_is_uniform_over_the_bubble():
    """One step with two sites in the disk and one in the liquid, against
    the same step without injection: every cell of the disk (as labelled at
    the start) gains w_i (dm1 + dm2) / n on each population, the liquid site
    cell gains w_i dm3, nothing else changes; budgets drop by the dm taken
    (the second disk site's budget runs out)."""
    f, rho = _disk_state()
    nx = 48
    lab, n = O.label_gas(O.D2Q9, rho, 1.0)
    assert n == 1
    root = int(lab.ravel()[20 + nx * 20])
    ncell = int((lab == root).sum())
    sites = np.array([20 + nx * 20, 22 + nx * 21, 40 + nx * 5])
    rate = np.array([1e-3, 2e-3, 5e-4])
    budget = np.array([1.0, 1.5e-3, 1.0])
    g = O.run_spread(O.D2Q9, f, 1, 1.0, -5.0, sites, rate, budget, 1)
    h = O.run(O.D2Q9, f, 1, 1.0, -5.0)
    _, w = O.velocities(O.D2Q9)
    diff = (g - h).reshape(9, -1)
    D = 1e-3 + 1.5e-3
    in_bub = lab.ravel() == root
    assert np.allclose(diff[:, in_bub], w[:, None] * D / ncell, rtol=0, atol=1e-15)
    assert np.allclose(diff[:, 40 + nx * 5], w * 5e-4, rtol=0, atol=1e-15)
    other = ~in_bub
    other[40 + nx * 5] = False
    assert np.abs(diff[:, other]).max() == 0.0
    assert np.allclose(budget, [1.0 - 1e-3, 0.0, 1.0 - 5e-4], rtol=0, atol=1e-15)
    # zero momentum (sum_i c_i w_i = 0), up to the rounding of g - h (|f| ~ 0.2)
    c, _ = O.velocities(O.D2Q9)
    assert np.abs(c.T @ diff).max() < 1e-16


def test_spread_injection_mass_ledger_with_relabelling():
    """Over 30 steps relabelled every 10 (G = -5 dynamics conserve mass), the
    total mass grows by exactly the agent taken."""
    f, _ = _disk_state()
    sites = np.array([20 + 48 * 20, 3 + 48 * 3])
    rate = np.array([1e-3, 2e-4])
    budget = np.array([0.02, 1.0])
    m0 = O.totals(O.D2Q9, f)[0]
    g = O.run_spread(O.D2Q9, f, 30, 1.0, -5.0, sites, rate, budget, 10)
    taken = (0.02 - budget[0]) + (1.0 - budget[1])
    assert taken == pytest.approx(0.02 + 30 * 2e-4, abs=1e-15)
    # FP64 totals of a mass ~3800 carry ~1e-11 of rounding; a lost or doubled
    # deposit would be off by >= 2e-4
    assert O.totals(O.D2Q9, g)[0] - m0 == pytest.approx(taken, abs=1e-9)


# ------------------------------------------------- hand-expanded 4x4 D2Q9 step

# D2Q9 as printed in the lattice Boltzmann textbooks (rest, E, N, W, S, NE,
# NW, SW, SE), written out here rather than read from the oracle
HAND_C = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]


def _hand_step(f, tau, G, exp, one, sites=()):
    """One Shan-Chen step on a 4x4 periodic grid, every operation written out
    in the number type of ``one`` (Fraction: exact; Decimal: 50 digits).
    f[i][y][x] are the populations that have arrived at (x, y); ``exp`` is
    the exponential of that number type (unused when G = 0).  Order of
    Sec. 3.1: moments, psi of every cell, the force from the neighbours'
    psi, the velocity shift u = (j + tau F)/rho, the equilibrium, BGK, the
    blowing-agent deposit w_i dm at a site cell, streaming to x + c_i."""
    n = 4
    w = [one * 4 / 9] + [one / 9] * 4 + [one / 36] * 4
    rho = [[sum(f[i][y][x] for i in range(9)) for x in range(n)] for y in range(n)]
    jx = [[sum(f[i][y][x] * HAND_C[i][0] for i in range(9)) for x in range(n)] for y in range(n)]
    jy = [[sum(f[i][y][x] * HAND_C[i][1] for i in range(9)) for x in range(n)] for y in range(n)]
    psi = [[(one - exp(-rho[y][x])) if G != 0 else one for x in range(n)] for y in range(n)]
    fs = [[[None] * n for _ in range(n)] for _ in range(9)]
    for y in range(n):
        for x in range(n):
            sx = sum(w[i] * psi[(y + HAND_C[i][1]) % n][(x + HAND_C[i][0]) % n] * HAND_C[i][0]
                     for i in range(1, 9))
            sy = sum(w[i] * psi[(y + HAND_C[i][1]) % n][(x + HAND_C[i][0]) % n] * HAND_C[i][1]
                     for i in range(1, 9))
            Fx, Fy = -G * psi[y][x] * sx, -G * psi[y][x] * sy
            ux = (jx[y][x] + tau * Fx) / rho[y][x]
            uy = (jy[y][x] + tau * Fy) / rho[y][x]
            for i in range(9):
                cu = HAND_C[i][0] * ux + HAND_C[i][1] * uy
                feq = w[i] * rho[y][x] * (1 + 3 * cu + cu * cu * 9 / 2 - (ux * ux + uy * uy) * 3 / 2)
                fs[i][y][x] = f[i][y][x] - (f[i][y][x] - feq) / tau
    for (sxy, dm) in sites:
        for i in range(9):
            fs[i][sxy[1]][sxy[0]] += w[i] * dm
    out = [[[None] * n for _ in range(n)] for _ in range(9)]
    for i in range(9):
        for y in range(n):
            for x in range(n):
                out[i][(y + HAND_C[i][1]) % n][(x + HAND_C[i][0]) % n] = fs[i][y][x]
    return out


def _hand_start():
    """Seeded 4x4 start (float64), far from equilibrium: densities 0.2..2.2,
    every population perturbed."""
    rng = np.random.default_rng(44)
    rho = rng.uniform(0.2, 2.2, (4, 4))
    _, w = O.velocities(O.D2Q9)
    f = w[:, None, None] * rho[None] * (1 + rng.uniform(-0.3, 0.3, (9, 4, 4)))
    return f


@pytest.mark.parametrize("G", [0.0, -5.0])
def test_hand_expanded_single_step_4x4(G):
    """One D2Q9 step on a 4x4 periodic grid written out by hand: G = 0 in
    exact rational arithmetic (with one blowing-agent site), G = -5 with
    psi = 1 - exp(-rho) and everything after it in 50-digit decimal
    arithmetic.  The oracle's FP64 step matches to 1e-15 of the largest
    population (a few ulp), which pins its velocity table and order,
    streaming direction, force sign and neighbour, velocity shift,
    equilibrium, relaxation and deposit placement at once."""
    from decimal import Decimal, localcontext
    from fractions import Fraction
    c, _ = O.velocities(O.D2Q9)
    assert [tuple(v[:2]) for v in c.tolist()] == HAND_C   # the convention both use
    f0 = _hand_start()
    tau = 0.8
    if G == 0.0:
        site, dm = (1, 2), 1.0 / 64
        exact = _hand_step([[[Fraction(float(v)) for v in row] for row in f0[i]] for i in range(9)],
                           Fraction(tau), Fraction(0), None, Fraction(1),
                           sites=[(site, Fraction(dm))])
        want = np.array([[[float(v) for v in row] for row in exact[i]] for i in range(9)])
        budget = np.array([1.0])
        got = O.run(O.D2Q9, f0[:, None], 1, tau, G, sites=np.array([site[0] + 4 * site[1]]),
                    rate=np.array([dm]), budget=budget)[:, 0]
        assert budget[0] == 1.0 - dm
    else:
        with localcontext() as ctx:
            ctx.prec = 50
            D = lambda v: Decimal(float(v))  # noqa: E731  exact binary value
            exact = _hand_step([[[D(v) for v in row] for row in f0[i]] for i in range(9)],
                               Decimal(tau), Decimal(G), lambda v: v.exp(), Decimal(1))
            want = np.array([[[float(v) for v in row] for row in exact[i]] for i in range(9)])
        got = O.run(O.D2Q9, f0[:, None], 1, tau, G)[:, 0]
        # the force is not small here: the step differs from the G = 0 one
        base = O.run(O.D2Q9, f0[:, None], 1, tau, 0.0)[:, 0]
        assert np.abs(base - want).max() > 1e-3
    assert np.abs(got - want).max() <= 1e-15 * np.abs(want).max()


# ------------------------------------- multi-lattice Shan-Chen (Sec. 3.1, Fig. 1)

def _ml_state(lat, nx, ny, nz, seed=5):
    """Three lattices (fluid + two bubbles' gas), seeded, away from rest."""
    rng = np.random.default_rng(seed)
    b = np.array([[nx * 0.3, ny * 0.5, nz * 0.5 if nz > 1 else 0, 3.0],
                  [nx * 0.7, ny * 0.45, nz * 0.5 if nz > 1 else 0, 3.5]])
    f = O.ml_init(lat, nx, ny, nz, b, 2.0, 0.15, 0.3, 2.0, 1e-3, seed)
    return f * (1 + 0.05 * rng.uniform(-1, 1, f.shape))


@pytest.mark.parametrize("lat", LATS)
def test_ml_single_lattice_is_the_single_component_step(lat):
    """One lattice with coupling G is the single-component step of Sec. 3.1
    (u = (j + tau F)/rho there, j/rho + tau (psi/rho)(-G S) here: equal up
    to rounding)."""
    nx, ny, nz = (16, 12, 1) if lat == O.D2Q9 else (10, 8, 6)
    f = _ml_state(lat, nx, ny, nz)[0]
    a = O.run(lat, f, 25, 0.85, -5.0)
    b = O.ml_run(lat, f[None], 25, 0.85, np.array([[-5.0]]))[0]
    assert np.abs(a - b).max() <= 1e-14 * np.abs(a).max()


@pytest.mark.parametrize("lat", LATS)
def test_ml_uncoupled_lattices_sum_to_one_ideal_fluid(lat):
    """With every coupling zero the lattices share the common velocity
    u' = sum j / sum rho, and f_eq is linear in rho at fixed u: the sum of
    the lattices evolves exactly as one lattice (G = 0) started from the
    summed populations.  A per-lattice velocity j_s / rho_s, or a mass-free
    weighting, breaks this."""
    nx, ny, nz = (16, 12, 1) if lat == O.D2Q9 else (10, 8, 6)
    f = _ml_state(lat, nx, ny, nz)
    nl = f.shape[0]
    a = O.ml_run(lat, f, 30, 0.7, np.zeros((nl, nl))).sum(0)
    b = O.run(lat, f.sum(0), 30, 0.7, 0.0)
    assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max()
    # the lattices themselves differ from an even split (each keeps its mass)
    rho = O.ml_moments(lat, O.ml_run(lat, f, 30, 0.7, np.zeros((nl, nl))))[0]
    rho0 = O.ml_moments(lat, f)[0]
    assert np.allclose(rho.sum(axis=(1, 2, 3)), rho0.sum(axis=(1, 2, 3)), rtol=1e-13, atol=0)


@pytest.mark.parametrize("lat,axis", [(O.D2Q9, 0), (O.D2Q9, 1), (O.D3Q19, 2)])
def test_ml_force_on_cosines_with_an_asymmetric_coupling(lat, axis):
    """psi_t = 1 + a_t cos(2 pi x/L) along one axis on each lattice: the
    lattice sum sum_i w_i psi_t(x + c_i) c_i is -(1/3) a_t sin(2 pi x/L)
    sin(2 pi/L) along the axis (the weights' second moment is 1/3 for every
    shift pattern along one axis), so F_s = -psi_s sum_t Gm[s][t] (that),
    closed form; an asymmetric Gm catches a transposed coupling."""
    L = 12
    shape = {0: (1, 1, L), 1: (1, L, 1), 2: (L, 1, 1)}[axis]
    if lat == O.D2Q9:
        shape = {0: (1, 1, L), 1: (1, L, 1)}[axis]
    nz, ny, nx = shape
    x = np.arange(L)
    amp = np.array([0.3, 0.1, 0.2])
    psi = np.stack([(1 + a * np.cos(2 * np.pi * x / L)).reshape(shape) for a in amp])
    Gm = np.array([[-5.0, 0.7, 1.1], [0.4, 0.0, 2.0], [1.5, 3.0, 0.0]])
    F = O.ml_force(lat, psi, Gm)
    S = (-(1.0 / 3.0) * amp[:, None] * np.sin(2 * np.pi * x / L) * np.sin(2 * np.pi / L))
    want = -psi.reshape(3, L) * (Gm @ S)
    got = F[axis].reshape(3, L)
    assert np.abs(got - want).max() < 1e-14
    for a in range(3):
        if a != axis and not (lat == O.D2Q9 and a == 2):
            assert np.abs(F[a]).max() < 1e-15


@pytest.mark.parametrize("lat", LATS)
def test_ml_mass_per_lattice_momentum_and_ledger(lat):
    """Without injection every lattice keeps its mass; with a symmetric
    coupling matrix the pair forces cancel over the periodic lattice, so the
    total momentum sum_s sum_x (j_s + F_s/2) stays at its start value; the
    blowing agent adds its dm to its own lattice only (Sec. 3)."""
    nx, ny, nz = (20, 16, 1) if lat == O.D2Q9 else (10, 8, 8)
    f = _ml_state(lat, nx, ny, nz)
    Gm = O.ml_coupling(3, -5.0, 0.9, 1.7)
    assert np.array_equal(Gm, Gm.T)

    def momentum(f):
        rho, jx, jy, jz = O.ml_moments(lat, f)
        psi, _ = O.eos(rho, 0.0)
        F = O.ml_force(lat, psi, Gm)
        return np.array([(j + F_ / 2).sum() for j, F_ in zip((jx, jy, jz), F)])

    m0 = O.ml_moments(lat, f)[0].sum(axis=(1, 2, 3))
    p0 = momentum(f)
    g = O.ml_run(lat, f, 40, 0.9, Gm)
    assert np.allclose(O.ml_moments(lat, g)[0].sum(axis=(1, 2, 3)), m0, rtol=1e-13, atol=0)
    assert np.abs(momentum(g) - p0).max() < 1e-12
    sites = np.array([3 + nx * 4, 7 + nx * 5])
    budget = np.array([0.03, 0.01])
    g = O.ml_run(lat, f, 40, 0.9, Gm, sites=sites, site_lattice=[1, 2],
                 rate=np.array([1e-3, 4e-4]), budget=budget)
    gain = O.ml_moments(lat, g)[0].sum(axis=(1, 2, 3)) - m0
    assert budget[0] == 0.0 and budget[1] == 0.0           # 30 and 25 steps of the agent
    assert np.allclose(gain, [0.0, 0.03, 0.01], rtol=0, atol=1e-14 * m0.max())


def test_ml_uniform_rest_state_is_a_fixed_point_and_empty_lattices_stay_finite():
    """Uniform lattices at rest: every force is zero and f_eq(rho, 0) = f,
    so nothing changes beyond the rounding of the density sums; a lattice that is empty everywhere (a merged
    bubble's) stays empty and finite (psi/rho is taken as its limit 1)."""
    nx, ny = 8, 6
    _, w = O.velocities(O.D2Q9)
    f = np.stack([w[:, None, None, None] * r * np.ones((1, ny, nx)) for r in (1.9, 0.2, 0.0)])
    g = O.ml_run(O.D2Q9, f, 10, 0.8, O.ml_coupling(3, -5.0, 1.0, 2.0))
    assert np.abs(g - f).max() <= 4e-16     # the density sums round in the last bit
    assert np.array_equal(g[2], f[2]) and np.isfinite(g).all()


def test_ml_pressure_reduces_to_the_eos_and_expands_the_coupling():
    """One lattice: p = rho/3 + G/6 psi^2 (Sec. 3.1).  Three lattices: the
    double sum over the coupling matrix written out."""
    rng = np.random.default_rng(2)
    rho = rng.uniform(0.0, 2.0, (3, 5))
    p1 = O.ml_pressure(rho[:1], np.array([[-5.0]]))
    assert np.allclose(p1, O.eos(rho[0], -5.0)[1], rtol=1e-15, atol=1e-15)
    Gm = np.array([[-5.0, 0.7, 0.7], [0.7, 0.0, 1.3], [0.7, 1.3, 0.0]])
    psi = 1 - np.exp(-rho)
    want = rho.sum(0) / 3 + (-5.0 * psi[0] ** 2 + 2 * 0.7 * psi[0] * (psi[1] + psi[2])
                             + 2 * 1.3 * psi[1] * psi[2]) / 6
    assert np.allclose(O.ml_pressure(rho, Gm), want, rtol=1e-14, atol=1e-15)


def test_ml_merge_conserves_and_removes_the_barrier():
    """eta_m = 0 merges lattice l into k: the pair's mass and momentum are
    kept on lattice k, lattice l is empty, and their coupling is zero."""
    f = _ml_state(O.D2Q9, 16, 12, 1)
    Gm = O.ml_coupling(3, -5.0, 1.0, 2.0)
    g, Gm2 = O.ml_merge(f, Gm, 1, 2)
    rf, jxf, jyf, _ = O.ml_moments(O.D2Q9, f)
    rg, jxg, jyg, _ = O.ml_moments(O.D2Q9, g)
    assert np.array_equal(g[2], np.zeros_like(g[2]))
    assert np.allclose(rg[1], rf[1] + rf[2], rtol=1e-15, atol=0)
    assert np.allclose(jxg[1], jxf[1] + jxf[2], rtol=1e-15, atol=1e-17)
    assert Gm2[1, 2] == Gm2[2, 1] == 0.0 and Gm2[0, 1] == Gm[0, 1]
