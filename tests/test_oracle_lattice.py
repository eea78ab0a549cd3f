"""Lattice pins for the oracle's Yee leapfrog (Sec. III A; Eq. (1) needs the
response at t_n = n Delta_t).

P1  discrete eigenmodes of a PEC cavity oscillate at the exact Yee dispersion
    (2/dt)^2 sin^2(w dt/2) = sum_a (2/Delta)^2 sin^2(k_a Delta/2);
P2  with sigma = 0 the discrete energy  eps E^n.E^n + mu H^{n-1/2}.H^{n+1/2}
    is conserved to round-off (PEC walls, PEC/PMC objects, dielectrics, Bloch wrap);
P3  with sigma > 0 a single mode follows the two-variable recurrence of the
    semi-implicit conductive update;
P10 a PEC geometry's electric sims equal the dual PMC geometry's magnetic sims;
and the real-field build equals the complex build where both apply.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import casimir_oracle as oc
from workloads import _base, box_faces


def _box(nx, ny, nz, res, dims, sigma=0.0, bc=("pec", "pec", "pec"), objects=()):
    p = _base(dims, (nx, ny, nz), res, 10, sigma=sigma)
    p["bc"] = list(bc)
    p["objects"] = list(objects)
    return p


def _site_grid(p, off):
    nx, ny, nz = p["n"]
    d = 1.0 / p["resolution"]
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return (i + off[0]) * d, (j + off[1]) * d, (k + off[2]) * d


def _omega(dt, d, ks):
    s = sum((2 / d) ** 2 * math.sin(k * d / 2) ** 2 for k in ks)
    return 2 / dt * math.asin(dt / 2 * math.sqrt(s))


@pytest.mark.parametrize("m,n", [(1, 1), (3, 2), (7, 5)])
def test_p1_tm_cavity_mode_dispersion(m, n):
    nx, ny, res = 24, 16, 8.0
    p = _box(nx, ny, 1, res, 2)
    d = 1 / res
    dt = p["courant"] * d
    kx, ky = m * math.pi / (nx * d), n * math.pi / (ny * d)
    x, y, _ = _site_grid(p, oc.E_OFF[2])
    E0 = np.zeros((3, nx * ny), complex)
    E0[2] = (np.sin(kx * x) * np.sin(ky * y)).ravel()
    T = 3000
    E, _, _ = oracle.evolve(p, E0, np.zeros_like(E0), T)
    w = _omega(dt, d, (kx, ky))
    assert np.max(np.abs(E[2] - math.cos(w * T * dt) * E0[2])) < 1e-11
    assert np.max(np.abs(E[:2])) == 0.0


def test_p1_te_cavity_mode_dispersion():
    nx, ny, res = 20, 12, 8.0
    p = _box(nx, ny, 1, res, 2)
    d = 1 / res
    dt = p["courant"] * d
    kx, ky = 3 * math.pi / (nx * d), 2 * math.pi / (ny * d)
    sx, sy = math.sin(kx * d / 2), math.sin(ky * d / 2)
    E0 = np.zeros((3, nx * ny), complex)
    x, y, _ = _site_grid(p, oc.E_OFF[0])
    E0[0] = (-sy * np.cos(kx * x) * np.sin(ky * y)).ravel()      # E = curl(H_z z) of H_z = cos cos
    x, y, _ = _site_grid(p, oc.E_OFF[1])
    E0[1] = (sx * np.sin(kx * x) * np.cos(ky * y)).ravel()
    T = 2000
    E, _, _ = oracle.evolve(p, E0, np.zeros_like(E0), T)
    c = math.cos(_omega(dt, d, (kx, ky)) * T * dt)
    assert np.max(np.abs(E[:2] - c * E0[:2])) < 1e-11


def test_p1_3d_cavity_mode_dispersion():
    nx, ny, nz, res = 10, 8, 6, 4.0
    p = _box(nx, ny, nz, res, 3)
    d = 1 / res
    dt = p["courant"] * d
    ks = [2 * math.pi / (nx * d), 1 * math.pi / (ny * d), 3 * math.pi / (nz * d)]
    s = [math.sin(k * d / 2) for k in ks]
    A = [1.0, 0.5, -(s[0] + 0.5 * s[1]) / s[2]]   # discrete divergence-free
    E0 = np.zeros((3, nx * ny * nz), complex)
    for c in range(3):
        x = _site_grid(p, oc.E_OFF[c])
        f = A[c] * np.ones_like(x[0])
        for a in range(3):
            f = f * (np.cos(ks[a] * x[a]) if a == c else np.sin(ks[a] * x[a]))
        E0[c] = f.ravel()
    T = 400
    E, _, _ = oracle.evolve(p, E0, np.zeros_like(E0), T)
    c = math.cos(_omega(dt, d, ks) * T * dt)
    assert np.max(np.abs(E - c * E0)) < 1e-11


def test_p1_bloch_plane_wave():
    # periodic box with Bloch phases: a travelling wave exp(i k.x) keeps its shape
    nx, ny, res = 16, 12, 8.0
    p = _box(nx, ny, 1, res, 2, bc=("periodic", "periodic", "pec"))
    d = 1 / res
    dt = p["courant"] * d
    kx, ky = 2 * math.pi * (2 + 0.3) / (nx * d), 2 * math.pi * (1 + 0.45) / (ny * d)
    x, y, _ = _site_grid(p, oc.E_OFF[2])
    E0 = np.zeros((3, nx * ny), complex)
    E0[2] = np.exp(1j * (kx * x + ky * y)).ravel()
    T = 500
    E, _, _ = oracle.evolve(p, E0, np.zeros_like(E0), T, kvec=(kx, ky, 0.0))
    c = math.cos(_omega(dt, d, (kx, ky)) * T * dt)
    assert np.max(np.abs(E[2] - c * E0[2])) < 1e-11


def _energy(setup, E, Hm, Hp):
    w = 0.0
    for c in range(3):
        m = setup.ce[c] != 0
        w += np.sum(np.abs(E[c][m]) ** 2 / setup.ce[c][m])
        m = setup.ch[c] != 0
        w += np.sum((np.conj(Hm[c][m]) * Hp[c][m]).real / setup.ch[c][m])
    return 0.5 * w


@pytest.mark.parametrize("dims,bc,kvec", [
    (2, ("pec", "pec", "pec"), (0, 0, 0)),
    (2, ("periodic", "pec", "pec"), (1.7, 0, 0)),
    (2, ("periodic", "periodic", "pec"), (0.9, 2.1, 0.7)),   # also d/dz -> i kz
    (3, ("pec", "periodic", "pec"), (0, 1.3, 0)),
])
def test_p2_energy_conservation(dims, bc, kvec):
    rng = np.random.default_rng(7)
    n = (12, 10, 1) if dims == 2 else (8, 7, 6)
    objs = [
        {"shape": "box", "lo": [0.5, 0.5, 0.5], "hi": [0.9, 1.0, 0.9], "kind": "pec"},
        {"shape": "box", "lo": [0.2, 0.1, 0.1], "hi": [0.45, 0.6, 0.5], "kind": "dielectric", "eps": 3.0, "mu": 1.5},
        {"shape": "box", "lo": [1.0, 0.2, 0.3], "hi": [1.3, 0.5, 0.6], "kind": "pmc"},
    ]
    p = _box(*n, 8.0, dims, bc=bc, objects=objs)
    st = oracle.grid_setup(p, kvec)
    N = st.N
    E0 = rng.normal(size=(3, N)) + 1j * rng.normal(size=(3, N))
    H0 = rng.normal(size=(3, N)) + 1j * rng.normal(size=(3, N))
    for c in range(3):
        E0[c][st.ce[c] == 0] = 0
        H0[c][st.ch[c] == 0] = 0
    if dims == 2 and kvec[2] == 0:
        pass
    Ea, Ha, _ = oracle.evolve(p, E0, H0, 3, kvec, st)
    _, Ha1, _ = oracle.evolve(p, E0, H0, 4, kvec, st)
    Eb, Hb, _ = oracle.evolve(p, E0, H0, 700, kvec, st)
    _, Hb1, _ = oracle.evolve(p, E0, H0, 701, kvec, st)
    Wa = _energy(st, Ea, Ha, Ha1)
    Wb = _energy(st, Eb, Hb, Hb1)
    assert Wa > 0
    assert abs(Wb - Wa) < 1e-11 * Wa


@pytest.mark.parametrize("sigma", [0.3, 1.0, 4.0])
def test_p3_conductive_mode_recurrence(sigma):
    nx, ny, res = 16, 12, 8.0
    p = _box(nx, ny, 1, res, 2, sigma=sigma)
    d = 1 / res
    dt = p["courant"] * d
    kx, ky = 2 * math.pi / (nx * d), 3 * math.pi / (ny * d)
    x, y, _ = _site_grid(p, oc.E_OFF[2])
    E0 = np.zeros((3, nx * ny), complex)
    E0[2] = (np.sin(kx * x) * np.sin(ky * y)).ravel()
    lam = math.sqrt(sum((2 / d) ** 2 * math.sin(k * d / 2) ** 2 for k in (kx, ky)))
    a = (1 - sigma * dt / 2) / (1 + sigma * dt / 2)
    b = dt / (1 + sigma * dt / 2)
    xs, ys = 1.0, 0.0
    T = 600
    for n in range(1, T + 1):
        ys -= (dt / 2 if n == 1 else dt) * lam * xs   # B update (no sigma on B in electric sims)
        xs = a * xs + b * lam * ys                     # D update with sigma
    E, _, _ = oracle.evolve(p, E0, np.zeros_like(E0), T)
    assert np.max(np.abs(E[2] - xs * E0[2])) < 1e-12 + 1e-9 * abs(xs)


def _shift(p, s):
    q = {**p}
    q["objects"] = []
    for o in p["objects"]:
        o = dict(o)
        if o["kind"] == "pec":
            o["kind"] = "pmc"
        o["lo"] = [v + s for v in o["lo"]]
        o["hi"] = [v + s for v in o["hi"]]
        q["objects"].append(o)
    q["faces"] = []
    for f in p["faces"]:
        f = dict(f)
        f["pos"] = f["pos"] + s
        f["lo"] = [v + s for v in f["lo"]]
        f["hi"] = [v + s for v in f["hi"]]
        q["faces"].append(f)
    return q


def test_p10_pec_pmc_duality():
    res = 8.0
    p = _base(2, (32, 24, 1), res, 400, sigma=1.0)
    p["bc"] = ["periodic", "periodic", "pec"]
    p["objects"] = [{"shape": "box", "lo": [1.0, 1.0, 0.0], "hi": [1.75, 1.5, 0.0], "kind": "pec"}]
    p["faces"] = box_faces([0.875, 0.875], [1.875, 1.625], 2)
    p["n_harm"] = 3
    p["polarization"] = "TE+TM"
    p["force_axis"] = 0
    q = _shift(p, 0.5 / res)
    sims_p = oracle.enumerate_sims(p)
    pairs = {("TM", "J", 2): ("TE", "K", 2), ("TM", "K", 0): ("TE", "J", 0), ("TM", "K", 1): ("TE", "J", 1)}
    checked = 0
    for sm in sims_p:
        key = (sm["pol"], sm["kind"], sm["comp"])
        if key not in pairs:
            continue
        pol, kind, comp = pairs[key]
        dual = dict(sm, pol=pol, kind=kind, comp=comp)
        a = oracle.run_sim(p, sm)
        b = oracle.run_sim(q, dual)
        assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(a))
        checked += 1
    assert checked >= 10


def test_real_and_complex_builds_agree():
    from workloads import piston_small
    p = piston_small(n_steps=300)
    sims = oracle.enumerate_sims(p)[:6]
    st = oracle.grid_setup(p)
    assert st.real
    for sm in sims:
        a = oracle.run_sim(p, sm, st)
        st.real = False
        b = oracle.run_sim(p, sm, st)
        st.real = True
        assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(a))
