"""Pins for sums of undamped Lorentz poles (the silica model of Sec. III D; one pole is the
silicon model of Eq. (9)), continued onto the contour omega^2 -> xi^2 + i sigma xi.

* At sigma = 0 a plane wave in a uniform two-pole medium oscillates at exactly three
  undamped frequencies, which converge at O(dt^2) to the three roots of
  w^2 eps(w) = k^2 with eps = eps_inf + sum_j de_j w_j^2 / (w_j^2 - w^2).
* Splitting one pole into two or three poles at the same frequency whose strengths add
  up leaves every field unchanged (the polarisations obey one linear equation): the
  force agrees to rounding.
* A pole far above the frequencies that carry the force acts as its static strength:
  the force tends to that of the dielectric eps_inf + de like (omega / omega_j)^2.
* With sigma > 0 the force on a three-pole slab does not depend on sigma (Sec. II) up to
  O(dt^2): the damping of every pole's equation is the contour's sigma.
"""
import math

import numpy as np
import pytest
from scipy.optimize import brentq, curve_fit

import oracle
import workloads as W


def _uniform_wave(cour, poles, eps_inf=1.5, res=16.0, nx=32):
    p = W._base(2, (nx, 2, 1), res, int(round(40 / (cour / res))), sigma=0.0, courant=cour)
    p["bc"] = ["periodic", "periodic", "pec"]
    p["objects"] = [{"shape": "box", "lo": [-1, -1, 0], "hi": [10, 10, 0], "kind": "lorentz",
                     "eps_inf": eps_inf, "delta_eps": [a for a, _ in poles], "omega0": [b for _, b in poles]}]
    st = oracle.grid_setup(p)
    d = 1 / res
    k = 2 * math.pi / (nx * d)
    src, meas = {}, {}
    for j in range(2):
        for i in range(nx):
            v = math.cos(k * i * d)
            src[(2, j * nx + i)] = v
            meas[(2, j * nx + i)] = v / nx
    s = oracle.run_vectors(p, st, False, src, meas, pol="TM").real
    t = cour / res * np.arange(1, len(s) + 1)
    kl = 2 / d * math.sin(k * d / 2)                 # lattice wavenumber of the mode
    eps = lambda w: eps_inf + sum(de * w0 * w0 / (w0 * w0 - w * w) for de, w0 in poles)
    f = lambda w: w * w * eps(w) - kl * kl
    w1, w2 = sorted(w0 for _, w0 in poles)
    roots = (brentq(f, 1e-6, w1 - 1e-9), brentq(f, w1 + 1e-9, w2 - 1e-9), brentq(f, w2 + 1e-9, 200.0))
    fit = lambda t, a, b, c, x1, x2, x3: a * np.cos(x1 * t) + b * np.cos(x2 * t) + c * np.cos(x3 * t)
    popt, _ = curve_fit(fit, t, s, p0=[0.3, 0.3, 0.3, *roots])
    assert np.max(np.abs(s - fit(t, *popt))) < 1e-11      # exactly three undamped modes
    assert np.all(np.abs(popt[:3]) > 0.05)                 # each of them excited
    return np.array(popt[3:]), np.array(roots)


def test_two_pole_polariton_dispersion():
    poles = ((2.0, 2.0), (1.5, 5.0))
    w05, roots = _uniform_wave(0.5, poles)
    w025, _ = _uniform_wave(0.25, poles)
    e05, e025 = np.abs(w05 / roots - 1), np.abs(w025 / roots - 1)
    assert np.all(e025 < e05)
    assert np.allclose(e05 / e025, 4.0, rtol=0.02)          # O(dt^2)
    assert np.allclose((4 * w025 - w05) / 3, roots, rtol=1e-5)


def _slab(mat, sigma=1.0, cour=0.5, res=12):
    p = W.plates_box_2d(res, 1.0, lines=("inner", "outer"), polarization="TE+TM",
                        t_max=(40.0 if sigma < 1 else 25.0), sigma=sigma, courant=cour)
    p["objects"] = [p["objects"][0], dict(shape="box", lo=[0.0, 1.25, 0], hi=[1.0, 1.5, 0], **mat)]
    return p


def test_pole_split_is_exact():
    one = oracle.force(_slab({"kind": "lorentz", "eps_inf": 1.5, "delta_eps": 3.0, "omega0": 2.0}))
    two = oracle.force(_slab({"kind": "lorentz", "eps_inf": 1.5, "delta_eps": [1.0, 2.0], "omega0": [2.0, 2.0]}))
    three = oracle.force(_slab({"kind": "lorentz", "eps_inf": 1.5, "delta_eps": [1.0, 1.5, 0.5],
                                "omega0": [2.0, 2.0, 2.0]}))
    assert abs(one) > 0.05
    assert two == pytest.approx(one, rel=1e-12)
    assert three == pytest.approx(one, rel=1e-12)
    # a pole of zero strength is no pole; a second pole that is not split changes the force
    zero = oracle.force(_slab({"kind": "lorentz", "eps_inf": 1.5, "delta_eps": [3.0, 0.0], "omega0": [2.0, 9.0]}))
    assert zero == pytest.approx(one, rel=1e-12)
    other = oracle.force(_slab({"kind": "lorentz", "eps_inf": 1.5, "delta_eps": [1.0, 2.0], "omega0": [2.0, 3.0]}))
    assert abs(other / one - 1) > 1e-3


def test_high_pole_tends_to_static_strength():
    stat = oracle.force(_slab({"kind": "dielectric", "eps": 2.5, "mu": 1.0}))
    dev = {}
    for w3 in (15.0, 30.0):
        f = oracle.force(_slab({"kind": "lorentz", "eps_inf": 1.5, "delta_eps": [1.0], "omega0": [w3]}))
        dev[w3] = f / stat - 1
    assert abs(dev[30.0]) < 5e-3
    assert 3.0 < dev[15.0] / dev[30.0] < 4.5                 # ~ (omega / omega_j)^2


def test_three_pole_sigma_independence():
    # silica's strengths, frequencies raised so that the slab settles within t = 25..40
    mat = {"kind": "lorentz", "eps_inf": 1.0, "delta_eps": [0.829, 0.095, 1.098], "omega0": [1.5, 2.5, 12.0]}
    out = {c: [oracle.force(_slab(mat, s, c)) for s in (0.5, 1.0, 2.0)] for c in (0.5, 0.25)}
    spread = {c: np.ptp(v) / abs(np.mean(v)) for c, v in out.items()}
    assert spread[0.5] > 1e-4                                 # the lattice error depends on sigma ...
    assert spread[0.5] / spread[0.25] == pytest.approx(4.0, rel=0.3)   # ... at O(dt^2)
    ext = [(4 * b - a) / 3 for a, b in zip(out[0.5], out[0.25])]
    assert np.ptp(ext) / abs(np.mean(ext)) < 5e-5


def test_pole_lists_are_validated():
    with pytest.raises(ValueError):
        oracle.lorentz_poles({"delta_eps": [1.0, 2.0], "omega0": [1.0]})
    with pytest.raises(ValueError):
        oracle.lorentz_poles({"delta_eps": [1.0] * 4, "omega0": [1.0] * 4})
    assert oracle.lorentz_poles({"delta_eps": 2.0, "omega0": 3.0}) == [(2.0, 3.0)]
    assert oracle.MAX_POLES == 3


def test_material_models_of_the_paper():
    # the constants the paper prints (tests/golden/paper_values.txt)
    from conftest import PAPER_VALUES as G
    si, sio2 = W.silicon(), W.silica()
    c = W.C_UM_PER_S
    eps_si = lambda w: si["eps_inf"] + si["delta_eps"] * si["omega0"] ** 2 / (si["omega0"] ** 2 - w * w)
    assert eps_si(0.0) == pytest.approx(G["silicon_eps_f"])              # static: eps_f
    assert eps_si(1e9) == pytest.approx(G["silicon_eps_0"], abs=1e-9)   # high frequency: eps_0
    assert si["omega0"] * c == pytest.approx(G["silicon_omega0_rad_s"])
    eps_s = lambda w: sio2["eps_inf"] + sum(C * w0 * w0 / (w0 * w0 - w * w)
                                           for C, w0 in zip(sio2["delta_eps"], sio2["omega0"]))
    Cs = [G["silica_C1"], G["silica_C2"], G["silica_C3"]]
    assert np.allclose(sio2["delta_eps"], Cs, rtol=0, atol=0)
    assert eps_s(0.0) == pytest.approx(1 + sum(Cs))
    assert np.allclose(np.array(sio2["omega0"]) * c,
                       [G["silica_omega1_rad_s"], G["silica_omega2_rad_s"], G["silica_omega3_rad_s"]])
    # on the imaginary axis both are real, above 1 and falling
    xi = np.array([0.1, 1.0, 10.0])
    e = np.array([eps_s(1j * x).real for x in xi])
    assert np.all(e > 1.0) and np.all(np.diff(e) < 0)
