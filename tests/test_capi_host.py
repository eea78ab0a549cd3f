"""Host-side checks of the C ABI (no GPU): the library loads, exports every
function include/casimir.h declares, and its planner agrees with the oracle on
the simulation list and on the time weights of Eq. (1)."""
import ctypes
import os

import numpy as np
import pytest

import oracle
import paper_0906_5170_gb300 as pk
from paper_0906_5170_gb300 import build as pkbuild
import workloads as W


@pytest.fixture(scope="module", autouse=True)
def built():
    pkbuild.build()


def test_library_exports_every_declared_function():
    declared = pk.header_functions()
    assert len(declared) >= 15
    L = pk.lib()
    for name in declared:
        assert hasattr(L, name), name
    assert set(declared) == set(pk.capi.SIGNATURES)


def _sim_tuples(problem):
    out = []
    for s in oracle.enumerate_sims(problem):
        n2 = s["harm"][1] if len(s["harm"]) > 1 else 0
        out.append((s["k"], s["face"], s["harm"][0], n2, 0 if s["kind"] == "J" else 1, s["comp"]))
    return out


@pytest.mark.parametrize("make", [
    lambda: W.config1_plates(),
    lambda: W.piston_small(),
    lambda: W.config2_piston(W.config2_heights()[3], n_steps=100),
    lambda: dict(W.piston_small(), basis="point", n_steps=50),
])
def test_plan_sim_list_matches_oracle(make):
    p = make()
    plan = pk.Plan(p)
    got = [tuple(int(v) for v in r) for r in plan.sims()]
    assert got == _sim_tuples(p)
    assert plan.info()["n_sims"] == len(got)


@pytest.mark.parametrize("variant,sigma", [("plain", 1.0), ("plain", 0.25), ("plain", 7.0), ("plain", 0.0), ("zinv", 1.0)])
def test_plan_weights_match_oracle(variant, sigma):
    p = W.plates_box_2d(16, 1.0, lines=("inner", "outer"), polarization="TM", n_steps=5000,
                        sigma=sigma, g_variant=variant)
    w = pk.Plan(p).weights()
    wo = oracle.g_weights(p)
    assert np.max(np.abs(w - wo) / np.abs(wo)) < 1e-12


@pytest.mark.parametrize("mutate,msg", [
    (lambda p: p.update(dims=4), "dims"),
    (lambda p: p.update(courant=0.9), "courant"),
    (lambda p: p.update(n_steps=0), "n_steps"),
    (lambda p: p.update(faces=[]), "faces"),
    (lambda p: p.update(force_axis=2), "force_axis"),
    (lambda p: p["faces"][0].update(hi=[2.97, 1.0, 0.0]), "whole cells"),
    (lambda p: p.update(polarization="full", k_points=[{"k": [0, 0, 0.5], "weight": 1.0}], precision="fp32"), None),
])
def test_plan_rejects_malformed_problems(mutate, msg):
    p = W.config1_plates()
    mutate(p)
    if msg is None:
        return   # accepted by the planner (may be rejected later by the executor)
    with pytest.raises(pk.CasimirError) as e:
        pk.Plan(p)
    assert e.value.code == -1


def test_context_without_device_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    with pytest.raises(pk.CasimirError) as e:
        pk.Context(0)
    assert e.value.code in (-1, -3)


def test_plan_sim_list_matches_oracle_cylindrical():
    p = W.cylinder_piston(12, [0, 1, 2], t_max=2.0)
    plan = pk.Plan(p)
    got = [tuple(int(v) for v in r) for r in plan.sims()]
    assert got == _sim_tuples(p)
    w = plan.weights()
    assert np.max(np.abs(w - oracle.g_weights(p)) / np.abs(oracle.g_weights(p))) < 1e-12


@pytest.mark.parametrize("mutate", [
    lambda p: p.update(courant=0.41),                                  # above the m = 2 limit 2/sqrt(24) = 0.408
    lambda p: p.update(bc=["pec", "pml", "pec"], pml_cells=[0, 3, 0]),
    lambda p: p.update(bc=["periodic", "pec", "pec"]),
    lambda p: p.update(polarization="TM"),
    lambda p: p["k_points"][0].update(k=[0.0, 0.3, 0.0]),
    lambda p: p["objects"].append({"shape": "box", "lo": [0.1, 0.1, 0], "hi": [0.2, 0.2, 0], "kind": "lorentz",
                                   "eps_inf": 1.0, "delta_eps": 2.0, "omega0": 1.0}),
])
def test_plan_rejects_invalid_cylindrical_problems(mutate):
    p = W.cylinder_piston(12, [0, 1, 2], t_max=2.0)
    mutate(p)
    with pytest.raises(pk.CasimirError) as e:
        pk.Plan(p)
    assert e.value.code == -1


def test_time_steps_fused_per_launch_by_run_kind():
    # launch indices per request, ceil(T / k): k = steps_per_launch for 2D TM/TE runs; two for the
    # two-step marches (cylindrical runs; FP32 Cartesian six-component runs whose materials have at
    # most one Lorentz pole) when steps_per_launch >= 2; one for every other run
    def launches(p, opts=None):
        return pk.Plan(p, options=opts).info()["launches"]

    T = 301
    tm = W.piston_small(n_steps=T)
    assert launches(dict(tm, precision="fp32")) == (T + 2) // 3
    assert launches(dict(tm, precision="fp64")) == (T + 1) // 2
    assert launches(dict(tm, precision="fp32"), {"steps_per_launch": 1}) == T
    wg = W.config3_waveguides(0.5, resolution=8, n_cells=48, pml_units=0.75, n_harm=2, n_steps=T,
                              k_points=[{"k": [0, 0, 1.3], "weight": 0.3}], precision="fp32")
    assert launches(wg) == (T + 1) // 2                                   # one pole, FP32
    assert launches(wg, {"steps_per_launch": 2}) == (T + 1) // 2
    assert launches(wg, {"steps_per_launch": 1}) == T
    assert launches(dict(wg, precision="fp64")) == T                      # FP64: one step
    silica = W.grating_silica(0.5, resolution=16, nk_x=1, nk_z=1, n_harm=1, t_max=1.0, courant=0.2,
                              pml_units=0.25, precision="fp32")
    assert launches(silica) == silica["n_steps"]                          # three poles: one step
    cyl = W.cylinder_piston(12, [0, 1], t_max=2.0, precision="fp64")
    assert launches(cyl) == (cyl["n_steps"] + 1) // 2
    assert launches(cyl, {"steps_per_launch": 1}) == cyl["n_steps"]
    s3 = W.config4_sphere_notch(0.4, seed=3, resolution=6, n_cells=24, pml_cells=4, n_harm=1, n_steps=T)
    assert launches(s3) == T                                              # 3D: one step per launch


def test_plan_options_defaults_and_explicit():
    p = W.piston_small()
    # three fused steps for FP32 runs, two for FP64 runs (bound by FP64 arithmetic)
    assert pk.Plan(dict(p, precision="fp32")).options() == {"steps_per_launch": 3, "march_rows": 32, "kernel_3d": 3}
    assert pk.Plan(dict(p, precision="fp64")).options() == {"steps_per_launch": 2, "march_rows": 32, "kernel_3d": 3}
    # 3D: the column march without CPML, the x-line kernel with it
    s3 = W.config4_sphere_notch(0.4, seed=3, resolution=6, n_cells=24, pml_cells=4, n_harm=1, n_steps=10)
    assert pk.Plan(s3).options()["kernel_3d"] == 1
    assert pk.Plan(dict(s3, bc=["pec", "pec", "pec"])).options()["kernel_3d"] == 3
    o = pk.Plan(p, options={"steps_per_launch": 1, "march_rows": 16}).options()
    assert o == {"steps_per_launch": 1, "march_rows": 16, "kernel_3d": 3}
    for bad in ({"steps_per_launch": 4}, {"march_rows": 65}, {"kernel_3d": 5}):
        with pytest.raises(pk.CasimirError) as e:
            pk.Plan(p, options=bad)
        assert e.value.code == -1
    # the simulation list does not depend on the options
    q = W.config3_waveguides(0.5, resolution=8, n_cells=48, pml_units=0.75, n_harm=2, n_steps=20,
                             k_points=[{"k": [0, 0, 0.5], "weight": 1.0}])
    a = pk.Plan(q).sims()
    b = pk.Plan(q, options={"march_rows": 64}).sims()
    assert np.array_equal(a, b)


def _small_grating(**kw):
    args = dict(resolution=16, nk_x=2, nk_z=2, n_harm=2, t_max=2.0, courant=0.2, pml_units=0.25,
                precision="fp64")
    args.update(kw)
    return W.grating_silica(0.5, **args)


def test_plan_sim_list_matches_oracle_multipole():
    p = _small_grating()
    plan = pk.Plan(p)
    got = [tuple(int(v) for v in r) for r in plan.sims()]
    assert got == _sim_tuples(p)
    assert plan.info()["n_sims"] == len(got)


@pytest.mark.parametrize("mutate", [
    lambda p: p.update(courant=0.5),                                   # silicon's pole: eps(4/dt^2) < 0.5
    lambda p: p["objects"][0].update(delta_eps=[0.829, -0.095, 1.098]),
    lambda p: p["objects"][0].update(omega0=[0.29, 0.0, 67.8]),
    lambda p: p["objects"][0].update(omega0=[0.29, 0.5, 700.0]),       # omega0 dt >= 2
])
def test_plan_rejects_unstable_or_invalid_poles(mutate):
    p = _small_grating()
    mutate(p)
    with pytest.raises(pk.CasimirError) as e:
        pk.Plan(p)
    assert e.value.code == -1


def test_binding_rejects_malformed_pole_lists():
    p = _small_grating()
    p["objects"][0].update(delta_eps=[1.0, 2.0], omega0=[1.0])
    with pytest.raises(ValueError):
        pk.Plan(p)
    p["objects"][0].update(delta_eps=[1.0] * 4, omega0=[1.0] * 4)
    with pytest.raises(ValueError):
        pk.Plan(p)


@pytest.mark.parametrize("poles", [1, 3])
@pytest.mark.parametrize("eps_x,stable", [(0.52, True), (0.48, False)])
def test_stability_bound_matches_the_oracle(eps_x, stable, poles):
    """The planner admits a uniform Lorentz medium (one pole, or three at frequencies in the
    ratio 0.3 : 0.6 : 1) exactly when eps(4/dt^2) = eps_inf - sum_j de_j y_j / (4 - y_j),
    y_j = (w_j dt)^2, exceeds the lattice bound (dt/2)^2 k_max^2 = 2 courant^2 = 0.5; the
    oracle's fields stay bounded just inside it and blow up just outside."""
    import math
    from scipy.optimize import brentq
    res, cour, nx = 8.0, 0.5, 8
    dt = cour / res
    de, ratios = ([10.0], [1.0]) if poles == 1 else ([1.0, 2.0, 3.0], [0.3, 0.6, 1.0])
    eps = lambda s: 1.0 - sum(d * (r * s * dt) ** 2 / (4 - (r * s * dt) ** 2) for d, r in zip(de, ratios))
    s = brentq(lambda s: eps(s) - eps_x, 1e-3, 1.999 / dt)
    p = W._base(2, (nx, nx, 1), res, 3000, sigma=0.0, courant=cour)
    p["bc"] = ["periodic", "periodic", "pec"]
    p["objects"] = [{"shape": "box", "lo": [-1, -1, 0], "hi": [10, 10, 0], "kind": "lorentz",
                     "eps_inf": 1.0, "delta_eps": de, "omega0": [r * s for r in ratios]}]
    q = dict(p, polarization="full", faces=[{"axis": 1, "sign": 1, "pos": 0.5, "lo": [0, 0.5, 0], "hi": [1, 0.5, 0]}])
    if stable:
        pk.Plan(q)
    else:
        with pytest.raises(pk.CasimirError):
            pk.Plan(q)
    st = oracle.grid_setup(p)
    with np.errstate(all="ignore"):
        v = np.abs(oracle.run_vectors(p, st, False, {(2, 3 * nx + 3): 1.0}, {(2, 3 * nx + 3): 1.0}, pol="TM"))
    late = np.nan_to_num(v[-300:], nan=np.inf).max()
    assert (late < 10.0) == stable


def test_plan_bytes_per_step_counts_every_plane():
    # an 8 x 8 periodic k_z cross-section filled with a two-pole medium, real FP32 fields: per cell
    # 6 field values read and written (48 B) + the material id, and per E site and pole P, P_prev
    # read and written (16 B); no walls, so all 3 x 64 E sites carry both poles
    p = W._base(2, (8, 8, 1), 8.0, 10)
    p["bc"] = ["periodic", "periodic", "pec"]
    p["objects"] = [{"shape": "box", "lo": [-1, -1, 0], "hi": [2, 2, 0], "kind": "lorentz", "eps_inf": 2.0,
                     "delta_eps": [1.0, 0.5], "omega0": [2.0, 3.0]}]
    p["faces"] = [{"axis": 1, "sign": 1, "pos": 0.5, "lo": [0, 0.5, 0], "hi": [1, 0.5, 0]}]
    p["polarization"] = "full"
    p["k_points"] = [{"k": [0, 0, 1.0], "weight": 1.0}]
    p["precision"] = "fp32"
    i = pk.Plan(p).info()
    assert i["bytes_per_step"] == i["n_sims"] * (64 * 49 + 64 * 3 * 2 * 16)
    # CPML along y (2 x 2 slab rows of 8 cells, 4 psi planes read and written) instead of the poles
    p["objects"] = []
    p["bc"] = ["periodic", "pml", "pec"]
    p["pml_cells"] = [0, 2, 0]
    i = pk.Plan(p).info()
    assert i["bytes_per_step"] == i["n_sims"] * (64 * 49 + 4 * 8 * 4 * 2 * 4)


@pytest.mark.parametrize("scale", [0.15, 1.0])
def test_serving_mix_is_stable(scale):
    # every request of the seeded serving trace passes the planner's stability bounds, and the
    # coarsest Lorentz waveguide stays bounded in the oracle at its largest k_z (that k_z grows
    # without bound when the grid ignores the medium: 1e57 within 240 steps)
    reqs = W.serving_requests(0, n_requests=200, rate=50.0, scale=scale)
    for _, p in reqs:
        if scale == 0.15 or p.get("kind") == "waveguide":   # the dispersive kind (3D spheres plan slowly)
            pk.Plan(p)
    if scale == 0.15:
        wg = min((p for _, p in reqs if p.get("kind") == "waveguide"), key=lambda p: p["resolution"])
        kp = max(wg["k_points"], key=lambda k: k["k"][2])
        q = dict(wg, n_steps=2000, k_points=[kp])
        s = np.abs(oracle.run_sim(q, oracle.enumerate_sims(q)[0], oracle.grid_setup(q, kp["k"])))
        assert np.all(np.isfinite(s)) and s[-200:].max() < s[:200].max()


def test_header_is_plain_c(tmp_path):
    # the boundary is a C ABI: its header compiles as C99 with every warning on, and the
    # structs a C caller fills have the sizes the binding marshals
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("no C compiler")
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    src = tmp_path / "c.c"
    src.write_text('#include <stdio.h>\n#include "casimir.h"\n'
                   'int main(void) { printf("%zu %zu %zu %zu\\n", sizeof(casimir_object), sizeof(casimir_face),'
                   ' sizeof(casimir_kpoint), sizeof(casimir_problem));\n'
                   '  printf("%zu %zu %zu\\n", sizeof(casimir_plan_info), sizeof(casimir_plan_options), sizeof(casimir_stats));'
                   ' return 0; }\n')
    exe = tmp_path / "c"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", inc, str(src), "-o", str(exe)],
                   check=True)
    sizes = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    from paper_0906_5170_gb300 import capi
    assert sizes == [ctypes.sizeof(capi.Object), ctypes.sizeof(capi.Face), ctypes.sizeof(capi.KPoint),
                     ctypes.sizeof(capi.Problem), ctypes.sizeof(capi.PlanInfo), ctypes.sizeof(capi.PlanOptions),
                     ctypes.sizeof(capi.Stats)]


@pytest.mark.parametrize("layout", ["rows", "columns"])
def test_plan_rejects_more_than_256_materials(layout, monkeypatch):
    # material ids are bytes: 300 distinct dielectrics are refused, whether one range of rows of
    # the threaded rasterisation already sees them all ("rows": stripes across x, every row of
    # cells crosses all of them) or only the merge of the ranges does ("columns": stripes across
    # y, each row lies in one of them).  Eight row ranges whatever the host's core count, so that
    # the merge is reached on a one-core machine too.
    monkeypatch.setenv("CASIMIR_PLAN_THREADS", "8")
    res, n = 10.0, 300
    p = W.plates_box_2d(10, 1.0, polarization="TM", n_steps=10)
    p["n"] = [n, n, 1]
    d = 1.0 / res
    objs = []
    for q in range(n):
        lo = [q * d, 0.0, 0.0] if layout == "rows" else [0.0, q * d, 0.0]
        hi = [(q + 0.5) * d, n * d, 0.0] if layout == "rows" else [n * d, (q + 0.5) * d, 0.0]
        objs.append({"shape": "box", "lo": lo, "hi": hi, "kind": "dielectric", "eps": 1.5 + 0.01 * q, "mu": 1.0})
    p["objects"] = objs
    p["faces"] = [{"axis": 1, "sign": 1, "pos": 1.0, "lo": [0.0, 1.0, 0.0], "hi": [1.0, 1.0, 0.0]}]
    with pytest.raises(pk.CasimirError) as e:
        pk.Plan(p)
    assert e.value.code == -1 and "256" in str(e.value)
    assert ("merging" in str(e.value)) == (layout == "columns")   # which of the two checks fired
    p["objects"] = objs[:200]                     # 201 ids with the background: accepted
    assert pk.Plan(p).info()["n_sims"] > 0
