"""Planted mistakes in the oracle must fail its pins.

Each mutation below is a plausible slip in sc_oracle.c (a coefficient, a
sign, an index, a weight, the tau factor, the streaming direction, the
injection, the minimum image, the RNG, the site spacing, the film probe)
or in the oracle's Python layer (the spread injection, the per-pair film
census, the rupture criterion).  The test builds a mutated copy in a
temporary directory and runs tests/test_oracle_pins.py against it; every
mutant must fail at least one pin.  The unmutated copy must pass.
Mutations live only in the temporary copies: the oracle's source is never
written.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTATIONS = [
    # equilibrium and collision (Sec. 3.1)
    ("4.5 * cu * cu", "4.0 * cu * cu"),
    ("1.5 * uu", "1.0 * uu"),
    ("(jx[k] + tau * Fx[k])", "(jx[k] + Fx[k])"),
    ("fi - (fi - feq(lat, i, rho[k], ux, uy, uz)) / tau",
     "fi - (fi - feq(lat, i, rho[k], ux, uy, uz)) * tau"),
    # Shan-Chen force and EOS
    ("Fx[k] = -G * psi[k] * sx;", "Fx[k] = G * psi[k] * sx;"),
    ("double s = lat_w(lat, i) * psi[nb(x, y, z, ci[0], ci[1], ci[2], nx, ny, nz)];",
     "double s = lat_w(lat, i) * psi[nb(x, y, z, ci[0], ci[0], ci[2], nx, ny, nz)];"),
    ("return rho0 * (1.0 - exp(-rho / rho0));", "return rho0 * (1.0 - exp(-rho));"),
    ("G / 6.0 * s * s", "G / 6.0 * s"),
    # velocity set, weights, streaming
    ("1.0 / 18, 1.0 / 18, 1.0 / 18,\n    1.0 / 36", "1.0 / 18, 1.0 / 18, 1.0 / 17,\n    1.0 / 36"),
    ("{1, 0, -1}, {-1, 0, 1}", "{1, 0, -1}, {-1, 1, 1}"),
    ("f[(int64_t)i * N + nb(x, y, z, c[0], c[1], c[2], nx, ny, nz)] =",
     "f[(int64_t)i * N + nb(x, y, z, -c[0], -c[1], -c[2], nx, ny, nz)] ="),
    # injection (Sec. 3)
    ("fs[(int64_t)i * N + site_cell[s]] += lat_w(lat, i) * dm;",
     "fs[(int64_t)i * N + site_cell[s]] += dm / q;"),
    ("double dm = rate[s] < budget[s] ? rate[s] : budget[s];", "double dm = rate[s];"),
    # initial state, minimum image, RNG, nucleation sites
    ("rho = rho_g + 0.5 * (rho_l - rho_g) * (1.0 + tanh(2.0 * s / width));",
     "rho = rho_g + 0.5 * (rho_l - rho_g) * (1.0 + tanh(s / width));"),
    ("if (d > 0.5 * n) d -= n;", ""),
    ("z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;", "z = (z ^ (z >> 28)) * 0x94D049BB133111EBULL;"),
    ("double need = r + out[4 * a + 3] + min_gap;", "double need = r + min_gap;"),
    # pressure second difference and Laplacian
    ("s += p[nb(x, y, z, e[0], e[1], e[2], nx, ny, nz)] - 2.0 * p[k] +",
     "s += p[nb(x, y, z, e[0], e[0], e[2], nx, ny, nz)] - 2.0 * p[k] +"),
    ("for (int sg = -1; sg <= 1; sg += 2) {", "for (int sg = 1; sg <= 1; sg += 2) {"),
    # multi-lattice model (Sec. 3.1, Fig. 1): the coupling matrix transposed,
    # the common velocity of one lattice only, the shifted velocity without
    # tau, the gas injected into the fluid, the coupled pressure's matrix
    # entry, the streaming of the bubble lattices
    ("double v = Gm[s * nl + t] * lat_w(lat, i) *", "double v = Gm[t * nl + s] * lat_w(lat, i) *"),
    ("      rt += rho[s * N + k];\n", "      rt = rho[s * N + k];\n"),
    ("        ux += tau * Fx[s * N + k] / r;", "        ux += Fx[s * N + k] / r;"),
    ("      fs[((int64_t)site_lattice[m] * q + i) * N + site_cell[m]] += lat_w(lat, i) * dm;",
     "      fs[((int64_t)i) * N + site_cell[m]] += lat_w(lat, i) * dm;"),
    ("        e += Gm[s * nl + t] * psi_of(rho[s * N + k], rho0) * psi_of(rho[t * N + k], rho0);",
     "        e += Gm[s * nl + s] * psi_of(rho[s * N + k], rho0) * psi_of(rho[t * N + k], rho0);"),
    ("            f[((int64_t)s * q + i) * N + nb(x, y, z, c[0], c[1], c[2], nx, ny, nz)] =",
     "            f[((int64_t)s * q + i) * N + nb(x, y, z, c[0], c[1], -c[2], nx, ny, nz)] ="),
    # film probe (crossings, midpoint tie, disc radius)
    ("x1 = (double)(m - 1) + lerp_cross(ra, rb, mid);", "x1 = (double)m + lerp_cross(ra, rb, mid);"),
    ("d2 = 0.5 * (dd[0] + dd[1]);", "d2 = dd[1];"),
    ("int64_t cc = xm - fl < 0.5 ? c : c + 1;", "int64_t cc = xm - fl < 0.5 ? c + 1 : c;"),
    ("if (t < 0 || t > h + 2.0) break;", "if (t < 0 || t > h + 3.0) break;"),
    # bubble census and the film test at every lattice point
    ("if (label[k] >= 0) count[label[k]] += 1;", "if (label[k] > 0) count[label[k]] += 1;"),
    ("while (b + 1 < nbins && ((int64_t)1 << (b + 1)) <= sizes[q]) ++b;",
     "while (b + 1 < nbins && ((int64_t)1 << (b + 1)) < sizes[q]) ++b;"),
    ("film = Lp >= 0 && Lm >= 0 && Lp != Lm && dp + dm - 1 <= h_max;",
     "film = Lp >= 0 && Lm >= 0 && dp + dm - 1 <= h_max;"),
    ("film = Lp >= 0 && Lm >= 0 && Lp != Lm && dp + dm - 1 <= h_max;",
     "film = Lp >= 0 && Lm >= 0 && Lp != Lm && dp + dm <= h_max;"),
    ("mid = film && (dp - dm <= 1 && dm - dp <= 1);", "mid = film && (dp - dm <= 1);"),
    ("} else if ((state[k] & bit) && d2 >= 0.0) {", "} else if (d2 >= 0.0) {"),
]

# the same for the oracle's Python layer (oracle/__init__.py): the blowing
# agent spread over a bubble, the per-pair film census, the rupture criterion
PY_MUTATIONS = [
    ("per_cell = total / sizes[key]", "per_cell = total"),
    ("flat[i, cells] += w[i] * per_cell", "flat[i, cells] += per_cell / Q"),
    ("                d = min(rate[s], budget[s])\n", "                d = rate[s]\n"),
    ("flat[i, -1 - key] += w[i] * total", "flat[i, -1 - key] += w[i] * total / Q"),
    ("r_d = float(np.sqrt(n / np.pi)) if dims == 3 else n / 2.0",
     "r_d = float(np.sqrt(n / np.pi)) if dims == 3 else float(n)"),
    ("r_d = float(np.sqrt(n / np.pi)) if dims == 3 else n / 2.0",
     "r_d = float(np.sqrt(n)) if dims == 3 else n / 2.0"),
    ("key=lambda q: (len(g[\"lines\"][q]), -q))", "key=lambda q: (g[\"mid\"][q], -q))"),
    ("h_c = g[\"tsum\"] / g[\"fired\"] if g[\"fired\"] else 0.0",
     "h_c = g[\"tsum\"] if g[\"fired\"] else 0.0"),
    ("else min(g[\"hmin\"][a], t)", "else max(g[\"hmin\"][a], t)"),
    ("h_c = h0 + (h - h0) * (-d0 / (d - d0))", "h_c = h"),
    ("    if h > h_max:\n        armed = False\n", "    if h > h_max:\n        pass\n"),
    ("    elif d < -eps_arm:\n", "    elif d < 0.0:\n"),
    # multi-lattice model (Sec. 3.1, Fig. 1): the pair's lattices not summed
    # on a merge, the fluid-gas coupling on one side only, a bubble's gas
    # laid on the fluid's profile
    ("    f[k] = f[k] + f[l]\n", "    f[k] = f[k]\n"),
    ("    Gm[1:, 0] = G_x\n", "    Gm[1:, 0] = 0.0\n"),
    ("        fk, _ = init(lat, nx, ny, nz, b[k:k + 1], 0.0, rho_gas, width, 0.0, seed)",
     "        fk, _ = init(lat, nx, ny, nz, b, 0.0, rho_gas, width, 0.0, seed)"),
]


def _compile(tmp, name, text):
    d = os.path.join(tmp, name)
    os.makedirs(d)
    src = os.path.join(d, "sc_oracle.c")
    with open(src, "w") as fh:
        fh.write(text)
    lib = os.path.join(d, "libsc_oracle.so")
    subprocess.check_call(["gcc", *O.GCC_FLAGS, "-o", lib, src, "-lm"])
    return lib


def _pins(lib):
    env = dict(os.environ, SC_ORACLE_LIB=lib, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests",
                        "test_oracle_pins.py"), "-x", "-q", "-p", "no:cacheprovider"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    return r.returncode, r.stdout[-400:]


def _py_tree(tmp, name, text):
    """A copy of the oracle package with a mutated __init__.py beside a copy of
    the pins (their conftest puts the copy's root first on sys.path)."""
    d = os.path.join(tmp, name)
    os.makedirs(os.path.join(d, "oracle"))
    with open(os.path.join(d, "oracle", "__init__.py"), "w") as fh:
        fh.write(text)
    shutil.copy(O.SRC, os.path.join(d, "oracle", "sc_oracle.c"))
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), os.path.join(d, "tests", "golden"))
    for f in ("conftest.py", "test_oracle_pins.py"):
        shutil.copy(os.path.join(ROOT, "tests", f), os.path.join(d, "tests", f))
    return d


def _py_pins(args):
    root, lib = args
    env = dict(os.environ, SC_ORACLE_LIB=lib, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(root, "tests",
                        "test_oracle_pins.py"), "-x", "-q", "-p", "no:cacheprovider"],
                       cwd=root, env=env, capture_output=True, text=True, timeout=900)
    return r.returncode, r.stdout[-400:]


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc needed")
def test_planted_mistakes_in_the_python_layer_fail_the_pins(tmp_path):
    init = os.path.join(os.path.dirname(O.SRC), "__init__.py")
    with open(init) as fh:
        orig = fh.read()
    with open(O.SRC) as fh:
        lib = _compile(str(tmp_path), "lib", fh.read())
    jobs = {"unmutated": (_py_tree(str(tmp_path), "unmutated", orig), lib)}
    for k, (a, b) in enumerate(PY_MUTATIONS):
        assert orig.count(a) == 1, a
        jobs[f"p{k:02d}: {a[:60]}"] = (_py_tree(str(tmp_path), f"p{k:02d}", orig.replace(a, b)),
                                       lib)
    with cf.ThreadPoolExecutor(max_workers=max(2, min(8, os.cpu_count() or 2))) as ex:
        res = dict(zip(jobs, ex.map(_py_pins, jobs.values())))
    rc, out = res.pop("unmutated")
    assert rc == 0, out
    survivors = [name for name, (rc, _) in res.items() if rc == 0]
    assert not survivors, survivors


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc needed")
def test_planted_mistakes_fail_the_pins(tmp_path):
    with open(O.SRC) as fh:
        orig = fh.read()
    jobs = {"unmutated": _compile(str(tmp_path), "unmutated", orig)}
    for k, (a, b) in enumerate(MUTATIONS):
        assert orig.count(a) >= 1, a
        jobs[f"m{k:02d}: {a[:60]}"] = _compile(str(tmp_path), f"m{k:02d}", orig.replace(a, b, 1))
    with cf.ThreadPoolExecutor(max_workers=max(2, min(8, os.cpu_count() or 2))) as ex:
        res = dict(zip(jobs, ex.map(_pins, jobs.values())))
    rc, out = res.pop("unmutated")
    assert rc == 0, out
    survivors = [name for name, (rc, _) in res.items() if rc == 0]
    assert not survivors, survivors
