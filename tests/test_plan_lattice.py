"""The planner's rasterisation (step a0: materials, PEC/PMC masks, closed walls, cylindrical
axis masks, Lorentz eps_inf) against the oracle's own lattice, site by site, bit for bit.

casimir_plan_site_coefs returns, for one field array of a host-only plan, the coefficient the
step kernels read at every site (1/eps or 1/mu, 0 where masked); the oracle's lattice set-up
holds the same coefficients for its leapfrog.  The TE family of two-dimensional runs sits on
the lattice shifted by half a cell, so its arrays are compared after the integer shift between
the two site positions (periodic in the canonical cell).  casimir_plan_sim_entries and
casimir_plan_site_poles extend the same check to every simulation's source and measurement
entries (steps a2, a8) and to the per-site Lorentz pole tables.
"""
import numpy as np
import pytest

import oracle
import paper_0906_5170_gb300 as pk
import workloads as W


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_0906_5170_gb300 import build as pkbuild
    pkbuild.build()                  # the host planner of the C ABI (incremental)


def _mask_problem():
    p = W.piston_small(n_steps=50, precision="fp64", g_variant="plain")
    m = np.zeros((10, 10), np.uint8)
    m[:, :5] = 1
    m[:5, 5:] = 1
    r = (np.random.default_rng(3).random((10, 7)) < 0.4).astype(np.uint8)
    p["objects"] = [p["objects"][0], W.grid_object(m, [3.5, 0.5], [4.5, 1.5], kind="pec"),
                    W.grid_object(r, [2.6, 0.75], [3.3, 1.24], kind="dielectric", eps=2.5, mu=1.0)]
    return p


def _pmc_problem():
    p = W.piston_small(n_steps=50, precision="fp64")
    p["objects"].append({"shape": "box", "lo": [0.0, 0.0, 0], "hi": [0.3, 2.0, 0], "kind": "pmc"})
    p["objects"].append({"shape": "sphere", "center": [3.0, 1.0, 0], "radius": 0.3, "kind": "dielectric",
                         "eps": 4.0, "mu": 2.0})
    return p


PROBLEMS = {
    "piston_te_tm": lambda: W.piston_small(n_steps=50),
    "pmc_and_disk": _pmc_problem,
    "voxel_masks": _mask_problem,
    "plates_filled": lambda: W.plates_box_2d(10, 1.0, polarization="TE+TM", n_steps=50, fill_eps=2.0),
    "waveguides_kz": lambda: W.config3_waveguides(0.5, resolution=8, n_cells=48, pml_units=0.75, n_harm=2,
                                                  n_steps=50, k_points=[{"k": [0, 0, 1.3], "weight": 1.0}]),
    "grating_silica": lambda: W.grating_silica(0.5, nk_x=2, nk_z=1, n_harm=2, t_max=1.0),
    "sphere_3d": lambda: W.config4_sphere_notch(0.55, n_cells=24, pml_cells=4, resolution=16),
    "cylinder": lambda: W.cylinder_piston(12, (0, 1, 2)),
}


@pytest.mark.parametrize("name", sorted(PROBLEMS))
def test_site_coefficients_match_the_oracle(name):
    p = PROBLEMS[name]()
    plan = pk.Plan(p)
    nx, ny, nz = p["n"]
    checked = 0
    for k, kp in enumerate(p["k_points"]):
        st = oracle.grid_setup(p, kp["k"], kp.get("m", 0))
        for field, offs, ref in ((0, oracle.E_OFF, st.ce), (1, oracle.H_OFF, st.ch)):
            for c in range(3):
                try:
                    got, off = plan.site_coefs(k, field, c)
                except pk.CasimirError:
                    continue                      # this polarisation has no such array
                want = np.asarray(ref[c]).reshape(nz, ny, nx).transpose(2, 1, 0)
                shift = [off[a] - offs[c][a] for a in range(3)]
                for a in range(p["dims"]):
                    assert shift[a] == round(shift[a]), (name, field, c, off)
                    want = np.roll(want, -int(round(shift[a])), axis=a)
                assert np.array_equal(got, want), (name, k, field, c, np.argwhere(got != want)[:5])
                checked += 1
    assert checked >= (6 if p["polarization"] in ("TE+TM", "full") else 3) * len(p["k_points"])


def test_site_coefficients_reject_absent_arrays():
    plan = pk.Plan(W.plates_box_2d(10, 1.0, polarization="TM", n_steps=50))
    with pytest.raises(pk.CasimirError):
        plan.site_coefs(0, 1, 2)                  # no H_z in a TM run
    with pytest.raises(pk.CasimirError):
        plan.site_coefs(1, 0, 2)                  # one k-point only
    got, off = plan.site_coefs(0, 0, 2)
    assert off == (0.0, 0.0, 0.5) and got.shape == (10, 20, 1)


def _shift(plan, field, c, dims):
    """Integer site shift of the planner's array against the standard Yee site of (field, c)."""
    _, off = plan.site_coefs(0, field, c)
    std = (oracle.H_OFF if field else oracle.E_OFF)[c]
    return [int(round(off[a] - std[a])) if a < dims else 0 for a in range(3)]


@pytest.mark.parametrize("name", sorted(PROBLEMS))
def test_sources_and_measurements_match_the_oracle(name):
    # steps a2 and a8: the impulse source (stored as E = D/eps or H = B/mu, masked) and the
    # stress-tensor measurement functional of every simulation, entry by entry
    from oracle.casimir_oracle import _sim_vectors
    p = PROBLEMS[name]()
    plan = pk.Plan(p)
    nx, ny, nz = p["n"]
    dims = p["dims"]
    sims = oracle.enumerate_sims(p)
    setups = [oracle.grid_setup(p, kp["k"], kp.get("m", 0)) for kp in p["k_points"]]
    te = p["polarization"] == "TE+TM"
    step = max(1, len(sims) // 40)
    for s in range(0, len(sims), step):
        sim = sims[s]
        st = setups[sim["k"]]
        src_o, meas_o = _sim_vectors(p, st, sim)

        def to_oracle(field, c, idx):
            sh = _shift(plan, field, c, dims)
            i, j, k = idx % nx, (idx // nx) % ny, idx // (nx * ny)
            return (((k + sh[2]) % nz) * ny + (j + sh[1]) % ny) * nx + (i + sh[0]) % nx

        def sign(field, c):
            return -1.0 if te and sim["pol"] == "TE" and field == 0 else 1.0

        field = 1 if sim["kind"] == "K" else 0
        c = sim["comp"]
        coef = (st.ch if field else st.ce)[c]
        comp, idx, val = plan.sim_entries(s, 0)
        assert np.all(comp == 3 * field + c)
        got = {to_oracle(field, c, int(q)): v * sign(field, c) for q, v in zip(idx, val)}
        want = {q: v * coef[q] for q, v in src_o.items()}
        assert set(got) == set(want), (name, s)
        scale = max(abs(v) for v in want.values())
        assert max(abs(got[q] - want[q]) for q in want) <= 1e-13 * scale, (name, s)

        comp, idx, val = plan.sim_entries(s, 1)
        got = {}
        for cc, q, v in zip(comp, idx, val):
            fq, cq = divmod(int(cc), 3)
            assert fq == field
            got[(cq, to_oracle(fq, cq, int(q)))] = v * sign(fq, cq)
        assert set(got) == set(meas_o), (name, s)
        scale = max(abs(v) for v in meas_o.values())
        assert max(abs(got[q] - meas_o[q]) for q in meas_o) <= 1e-13 * scale, (name, s)


def _poles_problem():
    # a three-pole slab written with an empty first pole, a one-pole block inside it, a PEC
    # box cutting both, CPML around: packing, overrides and masks of the pole tables
    p = W.config3_waveguides(0.5, resolution=8, n_cells=48, pml_units=0.75, n_harm=2, n_steps=50,
                             k_points=[{"k": [0, 0, 0.7], "weight": 1.0}])
    p["objects"] = [
        {"shape": "box", "lo": [1.0, 1.0, 0], "hi": [5.0, 3.0, 0], "kind": "lorentz", "eps_inf": 1.5,
         "delta_eps": [0.0, 0.8, 1.1, ], "omega0": [2.0, 1.5, 3.0]},
        {"shape": "box", "lo": [2.0, 1.5, 0], "hi": [3.0, 2.5, 0], "kind": "lorentz", "eps_inf": 2.0,
         "delta_eps": 3.0, "omega0": 2.5},
        {"shape": "box", "lo": [3.5, 1.25, 0], "hi": [4.0, 2.75, 0], "kind": "pec"},
    ]
    return p


@pytest.mark.parametrize("name", ["waveguides_kz", "grating_silica", "poles"])
def test_site_poles_match_the_oracle(name):
    # the (delta_eps, omega0) pairs present at every E site, as sets (the planner packs the
    # present poles first; the oracle keeps each pole at the index it was given)
    p = _poles_problem() if name == "poles" else PROBLEMS[name]()
    plan = pk.Plan(p)
    nx, ny, nz = p["n"]
    for k, kp in enumerate(p["k_points"]):
        st = oracle.grid_setup(p, kp["k"], kp.get("m", 0))
        for c in range(3):
            got = np.stack([np.stack(plan.site_poles(k, c, q), -1) for q in range(oracle.MAX_POLES)], -2)
            want = np.zeros_like(got)
            for q in range(len(st.lde[c])):
                de = np.asarray(st.lde[c][q]).reshape(nz, ny, nx).transpose(2, 1, 0)
                w0 = np.asarray(st.lw0[c][q]).reshape(nz, ny, nx).transpose(2, 1, 0)
                want[..., q, 0] = de
                want[..., q, 1] = np.where(de != 0.0, w0, 0.0)
            key = lambda a: np.sort(a[..., 0] + 1j * a[..., 1], axis=-1)
            assert np.array_equal(key(got), key(want)), (name, k, c)
            assert np.any(got[..., 0] != 0.0)
    if name == "poles":
        de0, _ = plan.site_poles(0, 2, 0)
        assert np.count_nonzero(np.unique(de0)) == 2           # 0.8 (packed first) and 3.0


@pytest.mark.parametrize("name", ["waveguides_kz", "grating_silica", "sphere_3d"])
def test_pml_profiles_match_the_oracle(name):
    # step a5: the CPML coefficients of every PML axis, integer and half-integer sites
    from oracle.casimir_oracle import _pml_profile
    p = PROBLEMS[name]()
    plan = pk.Plan(p)
    dt = p["courant"] / p["resolution"]
    axes = [a for a in range(p["dims"]) if p["bc"][a] == "pml"]
    assert axes
    for a in axes:
        for half in (0, 1):
            got = plan.pml(a, half)
            want = _pml_profile(p["n"][a], p["pml_cells"][a], p["resolution"], dt, half)
            # b and 1/kappa to rounding; c = s/(s k + k^2 a) (b - 1) inherits the rounding of b
            # (the two sides' exp may differ by an ulp) amplified by the cancellation in b - 1
            assert np.allclose(got[0], want[0], rtol=1e-15, atol=0), (name, a, half)
            assert np.array_equal(got[2], want[2]), (name, a, half)
            bm1 = np.where(want[0] != 1.0, want[0] - 1.0, 1.0)
            tol = 1e-14 * np.abs(want[1]) + 4e-16 * np.abs(want[1] / bm1)
            assert np.all(np.abs(got[1] - want[1]) <= tol), (name, a, half)
            assert np.any(got[1] != 0) and np.all(got[0] <= 1)
    for a in [a for a in range(3) if a not in axes] + [3]:
        with pytest.raises(pk.CasimirError):
            plan.pml(a, 0)                        # not a PML axis (or no axis at all)
