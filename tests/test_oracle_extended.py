"""Pins for the oracle's k_z, Bloch, CPML and Lorentz paths.

P8  z-invariant PEC/vacuum: (1/pi) int dk_z F(k_z) over hybrid (d/dz -> i k_z)
    simulations equals the single k_z = 0 TE+TM run with the z-invariant kernel of
    Appendix A.2 (Sec. III B); the two lattice estimates converge to each other
    at O(Delta^2);
P9  Bloch-periodic systems (Sec. III D): the N_k-point average over the Brillouin
    zone equals one k = 0 run on the N_k-fold supercell, exactly (complete bases);
CPML (Sec. III B): a PML-terminated cell reproduces the response of a much
    larger closed cell until that cell's wall echoes return;
Lorentz (Eq. (9) continued onto the contour): at sigma = 0 a plane wave in a
    uniform medium oscillates at the two polariton roots of
    w^2 eps(w) = k^2 (to O(dt^2)), and with sigma > 0 the force on a dispersive
    slab is sigma independent (Sec. II), which fixes the ADE damping to sigma.
"""
import math

import numpy as np
import pytest
from scipy.optimize import brentq, curve_fit

import oracle
import workloads as W


def _zinv_vs_kz(res, nk=12, kmax=16.0):
    p = W.plates_box_2d(res, 1.0, lines=("inner", "outer"), polarization="TE+TM", t_max=20.0, g_variant="zinv")
    fz = oracle.force(p)
    q = dict(p, g_variant="plain", polarization="full")
    u, w = np.polynomial.legendre.leggauss(nk)
    q["k_points"] = [{"k": [0, 0, kmax * (1 + ui) / 2], "weight": wi * kmax / 2 / math.pi} for ui, wi in zip(u, w)]
    return oracle.force(q) / fz - 1.0


def test_p8_kz_integral_equals_zinv_kernel():
    r8 = _zinv_vs_kz(8)
    r16 = _zinv_vs_kz(16)
    assert abs(r16) < 0.03
    assert 3.0 < r8 / r16 < 6.5          # O(Delta^2) convergence of the difference


def _grating(ncells_x, nx, res, kpts):
    p = W._base(2, (ncells_x, 24, 1), res, 300)
    p["bc"] = ["periodic", "pec", "pec"]
    L = ncells_x / res
    objs = []
    for c in range(ncells_x // nx):
        x0 = c * nx / res
        objs.append({"shape": "box", "lo": [x0 + 0.25, 1.0, 0], "hi": [x0 + 0.75, 1.5, 0],
                     "kind": "dielectric", "eps": 4.0, "mu": 1.0})
    objs.append({"shape": "box", "lo": [0, 2.25, 0], "hi": [L, 2.5, 0], "kind": "pec"})
    p["objects"] = objs
    p["faces"] = [{"axis": 1, "sign": -1, "pos": 0.75, "lo": [0, 0.75, 0], "hi": [L, 0.75, 0]},
                  {"axis": 1, "sign": 1, "pos": 1.75, "lo": [0, 1.75, 0], "hi": [L, 1.75, 0]}]
    p["n_harm"] = ncells_x
    p["polarization"] = "TE+TM"
    p["force_axis"] = 1
    p["k_points"] = kpts
    return p


def test_p9_bloch_average_equals_supercell():
    res, nx, nk = 8.0, 8, 3
    L = nx / res
    cell = _grating(nx, nx, res, [{"k": [2 * math.pi * m / (nk * L), 0, 0], "weight": 1.0 / nk} for m in range(nk)])
    sup = _grating(nx * nk, nx, res, [{"k": [0, 0, 0], "weight": 1.0 / nk}])
    fc, pc, _ = oracle.force(cell, return_parts=True)
    fs = oracle.force(sup)
    assert abs(fc - fs) < 1e-11 * sum(abs(x) for x in pc)


def _pml_prob(n, pml):
    res = 10.0
    p = W._base(2, (n, n, 1), res, 400)
    c = n / res / 2
    p["bc"] = ["pml", "pml", "pec"] if pml else ["pec", "pec", "pec"]
    p["pml_cells"] = [pml, pml, 0]
    p["objects"] = [{"shape": "box", "lo": [c - 0.3, c - 0.8, 0], "hi": [c - 0.1, c + 0.8, 0],
                     "kind": "dielectric", "eps": 3.0, "mu": 1.0}]
    p["faces"] = W.box_faces([c, c - 0.5], [c + 0.5, c + 0.5], 2)
    p["n_harm"] = 3
    p["polarization"] = "TE+TM"
    p["force_axis"] = 0
    return p


def test_cpml_mimics_open_space():
    small, closed, big = _pml_prob(60, 10), _pml_prob(60, 0), _pml_prob(260, 0)
    sims = oracle.enumerate_sims(small)[::4]
    assert len(sims) >= 8
    for sm in sims:
        a, c, b = (oracle.run_sim(q, sm) for q in (small, closed, big))
        s = np.max(np.abs(b))          # 400 steps: the large cell's echoes have not returned yet
        e_pml = np.max(np.abs(a - b)) / s
        e_closed = np.max(np.abs(c - b)) / s
        assert e_pml < 2e-3
        assert e_closed > 20 * e_pml


def _lorentz_wave(cour, res=16.0, nx=32, ny=2, eps_inf=1.0, de=3.0, w0=3.0):
    p = W._base(2, (nx, ny, 1), res, int(round(40 / (cour / res))), sigma=0.0, courant=cour)
    p["bc"] = ["periodic", "periodic", "pec"]
    p["objects"] = [{"shape": "box", "lo": [-1, -1, 0], "hi": [10, 10, 0], "kind": "lorentz",
                     "eps_inf": eps_inf, "delta_eps": de, "omega0": w0}]
    st = oracle.grid_setup(p)
    d = 1 / res
    k = 2 * math.pi / (nx * d)
    src, meas = {}, {}
    for j in range(ny):
        for i in range(nx):
            v = math.cos(k * i * d)
            src[(2, j * nx + i)] = v
            meas[(2, j * nx + i)] = v / (nx * ny / 2)
    s = oracle.run_vectors(p, st, False, src, meas, pol="TM").real
    t = cour / res * np.arange(1, len(s) + 1)
    kl = 2 / d * math.sin(k * d / 2)               # lattice wavenumber of the mode
    f = lambda w: w * w * (eps_inf + de * w0 * w0 / (w0 * w0 - w * w)) - kl * kl
    roots = (brentq(f, 1e-6, w0 - 1e-9), brentq(f, w0 * math.sqrt(1 + de / eps_inf) + 1e-9, 100))
    fit = lambda t, a, b, w1, w2: a * np.cos(w1 * t) + b * np.cos(w2 * t)
    popt, _ = curve_fit(fit, t, s, p0=[0.5, 0.5, *roots])
    assert np.max(np.abs(s - fit(t, *popt))) < 1e-10      # exactly two undamped modes
    return np.array(popt[2:]), np.array(roots)


def test_lorentz_polariton_dispersion():
    w05, roots = _lorentz_wave(0.5)
    w025, _ = _lorentz_wave(0.25)
    e05, e025 = np.abs(w05 / roots - 1), np.abs(w025 / roots - 1)
    assert np.all(e025 < e05)
    assert np.allclose(e05 / e025, 4.0, rtol=0.1)          # O(dt^2)
    ext = (4 * w025 - w05) / 3
    assert np.allclose(ext, roots, rtol=1e-5)


def test_lorentz_sigma_independence():
    def prob(s, cour):
        p = W.plates_box_2d(12, 1.0, lines=("inner", "outer"), polarization="TE+TM",
                            t_max=(40.0 if s < 1 else 25.0), sigma=s, courant=cour)
        p["objects"] = [p["objects"][0], {"shape": "box", "lo": [0.0, 1.25, 0], "hi": [1.0, 1.5, 0],
                                          "kind": "lorentz", "eps_inf": 1.5, "delta_eps": 3.0, "omega0": 2.0}]
        return p
    out = {c: [oracle.force(prob(s, c)) for s in (0.5, 1.0, 2.0)] for c in (0.5, 0.25)}
    spread = {c: np.ptp(v) / np.mean(v) for c, v in out.items()}
    assert spread[0.5] / spread[0.25] == pytest.approx(4.0, rel=0.3)
    ext = [(4 * b - a) / 3 for a, b in zip(out[0.5], out[0.25])]
    assert np.ptp(ext) / np.mean(ext) < 5e-5
