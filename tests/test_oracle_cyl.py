"""Pins of the oracle's cylindrical (r, z) lattice with fields ~ exp(i m phi) (Sec. III C and the
appendix on cylindrical coordinates).

C1  discrete energy: with sigma = 0 the energy sum_s w_s (eps |E_s|^2 + mu H^{n-1/2}.H^{n+1/2}),
    site weights w_s = r_s (Delta/8 on the axis), is conserved to rounding for m = 0, 1, 2 --
    the discrete curl is self-adjoint in the r-weighted product, axis treatment included;
C2  the lowest TM and TE frequencies of a PEC tube converge as Delta^2 to j_{m,1}/R and
    j'_{m,1}/R (Bessel zeros, computed here by scipy), m = 0, 1, 2;
C3  a PEC disk in a closed PEC tube: the force per m, after Richardson extrapolation, equals
    the exact sum over the tube's TM_{mn} and TE_{mn} waveguide modes of the 1D massive-mode
    plate pressure difference between the two cavities;
C4  complete cosine basis == point-source basis (the force does not depend on the basis);
C5  a disk midway between the caps feels no force (mirror symmetry).
"""
import math

import numpy as np
import pytest
from scipy.special import jn_zeros, jnp_zeros

import oracle
from workloads import _base, cylinder_piston
from test_oracle_physics import _massive_1d


def _tube(nr, nz, res, bc_z="periodic", objects=()):
    p = _base(2, (nr, nz, 1), float(res), 10, sigma=0.0)
    p["coords"] = "cylindrical"
    p["bc"] = ["pec", bc_z, "pec"]
    p["polarization"] = "full"
    p["objects"] = list(objects)
    return p


def _weights(st, problem):
    """Site weights (r_s, Delta/8 on the axis) for every component of E and H."""
    nr = problem["n"][0]
    i = np.arange(st.N) % nr
    wE = [np.array([oracle.cyl_site_weight(problem, oracle.E_OFF[c][0], k) for k in i]) for c in range(3)]
    wH = [np.array([oracle.cyl_site_weight(problem, oracle.H_OFF[c][0], k) for k in i]) for c in range(3)]
    return wE, wH


def _energy(st, wE, wH, E, Hm, Hp):
    w = 0.0
    for c in range(3):
        m = st.ce[c] != 0
        w += np.sum(wE[c][m] * np.abs(E[c][m]) ** 2 / st.ce[c][m])
        m = st.ch[c] != 0
        w += np.sum(wH[c][m] * (np.conj(Hm[c][m]) * Hp[c][m]).real / st.ch[c][m])
    return 0.5 * w


@pytest.mark.parametrize("m", [0, 1, 2])
def test_c1_energy_conservation(m):
    rng = np.random.default_rng(11 + m)
    objs = [{"shape": "box", "lo": [0.3, 0.2, 0], "hi": [0.5, 0.5, 0], "kind": "dielectric", "eps": 2.5, "mu": 1.5},
            {"shape": "box", "lo": [0.0, 0.8, 0], "hi": [0.4, 0.9, 0], "kind": "pec"},
            {"shape": "box", "lo": [0.6, 1.0, 0], "hi": [0.8, 1.2, 0], "kind": "pmc"}]
    p = _tube(10, 12, 8.0, "periodic", objs)
    p["courant"] = 0.9 * 2 / math.sqrt(max(9, 8 + 4 * m * m))
    kvec = (0.0, 1.3, 0.0)
    st = oracle.grid_setup(p, kvec, m)
    N = st.N
    E0 = rng.normal(size=(3, N)) + 1j * rng.normal(size=(3, N))
    H0 = rng.normal(size=(3, N)) + 1j * rng.normal(size=(3, N))
    for c in range(3):
        E0[c][st.ce[c] == 0] = 0
        H0[c][st.ch[c] == 0] = 0
    wE, wH = _weights(st, p)
    Ea, Ha, _ = oracle.evolve(p, E0, H0, 3, kvec, st)
    _, Ha1, _ = oracle.evolve(p, E0, H0, 4, kvec, st)
    Eb, Hb, _ = oracle.evolve(p, E0, H0, 600, kvec, st)
    _, Hb1, _ = oracle.evolve(p, E0, H0, 601, kvec, st)
    Wa = _energy(st, wE, wH, Ea, Ha, Ha1)
    Wb = _energy(st, wE, wH, Eb, Hb, Hb1)
    assert Wa > 0
    assert abs(Wb - Wa) <= 1e-11 * Wa


def _lowest(res, m, block, R=1.0):
    """Lowest non-zero eigenfrequency of the spatial operator curl_H curl_E on the TM (E_z) or TE
    (E_r, E_phi) unknowns of a z-invariant PEC tube, read off one leapfrog step of the oracle:
    E^1 = E^0 - (dt^2/2) curl_H curl_E E^0."""
    nr = int(round(R * res))
    p = _tube(nr, 1, res)
    st = oracle.grid_setup(p, (0.0, 0.0, 0.0), m)
    N, dt = st.N, st.dt
    comps = [1] if block == "TM" else [0, 2]
    cols = [(c, i) for c in comps for i in range(N) if st.ce[c][i] != 0]
    A = np.zeros((len(cols), len(cols)), dtype=complex)
    for q, (c, i) in enumerate(cols):
        E0 = np.zeros((3, N), complex)
        E0[c][i] = 1.0
        E1, _, _ = oracle.evolve(p, E0, np.zeros((3, N), complex), 1, (0.0, 0.0, 0.0), st)
        v = 2.0 * (E0 - E1) / dt**2
        A[:, q] = [v[cc][ii] for cc, ii in cols]
    ev = np.linalg.eigvals(A).real
    return math.sqrt(np.min(ev[ev > 1e-6]))


@pytest.mark.parametrize("m", [0, 1, 2])
@pytest.mark.parametrize("block", ["TM", "TE"])
def test_c2_tube_modes_bessel_zeros(m, block):
    exact = (jn_zeros(m, 1) if block == "TM" else jnp_zeros(m, 1))[0]
    w16, w32, w64 = (_lowest(r, m, block) for r in (16, 32, 64))
    e32, e64 = w32 - exact, w64 - exact
    assert abs(e32 / e64) == pytest.approx(4.0, rel=0.05)         # second order
    assert (4 * w64 - w32) / 3 == pytest.approx(exact, rel=2e-6)   # Richardson


def _tube_pressure(a, m, R, nzeros=40):
    """Exact force on a PEC plate from a closed cavity of length a in a PEC tube of radius R,
    the e^{i m phi} sector: minus the 1D massive-mode pressure summed over the TM_{mn}
    (k = j_{m,n}/R) and TE_{mn} (k = j'_{m,n}/R) waveguide modes."""
    return -sum(_massive_1d(a, z / R) for z in list(jn_zeros(m, nzeros)) + list(jnp_zeros(m, nzeros)))


@pytest.mark.parametrize("m,tol", [(0, 3e-3), (1, 2e-3), (2, 1.5e-2)])
def test_c3_cylinder_piston_mode_sum(m, tol):
    R, below, above = 0.5, 0.5, 1.0
    exact = _tube_pressure(below, m, R) - _tube_pressure(above, m, R)
    f20, f40 = (oracle.force(cylinder_piston(r, [m], radius=R, below=below, above=above)) for r in (20, 40))
    # the single-m problems carry weight 2 for m > 0; compare per +m sector
    if m > 0:
        f20, f40 = f20 / 2, f40 / 2
    assert (f20 - exact) / (f40 - exact) == pytest.approx(4.0, rel=0.1)
    ext = (4 * f40 - f20) / 3
    assert ext == pytest.approx(exact, rel=tol)
    assert ext < 0          # the disk is pulled toward the nearer cap below it


def test_c4_complete_cosine_basis_equals_point_basis():
    p = cylinder_piston(12, [0, 1], t_max=6.0)
    f_cos = oracle.force(p)
    f_pt = oracle.force(dict(p, basis="point"))
    assert f_cos == pytest.approx(f_pt, rel=1e-11, abs=1e-14)


def test_c5_mirror_symmetric_disk_feels_no_force():
    # lengths on grid planes (resolution 10): the lattice is symmetric about the disk's middle
    p = cylinder_piston(10, [0, 1, 2], thickness=0.2, below=0.6, above=0.6, t_max=8.0)
    F, parts, _ = oracle.force(p, return_parts=True)
    assert abs(F) <= 1e-11 * np.sum(np.abs(parts))
