"""GPU parity of the two-step march of Cartesian six-component runs (two leapfrog steps per
launch: k_z cross-sections with real fields, Bloch cells with complex fields, CPML, one
undamped Lorentz pole per material at most) against the FP64 oracle and against the one-step
march on the same problem.

FP32 fields with FP64 accumulation, so the bounds of tests/parity_bounds.py apply: each
simulation within 2e-5 of the largest contribution, the force within 1e-4 of itself (plus the
rounding floor of its FP64 sum where the contributions cancel).  The one-
step march (steps_per_launch 1) performs the same per-cell arithmetic in the same order, so the
two executions agree to FP32 rounding; they are held to the same bound against each other.
Odd step counts end on a launch that holds one step; run lengths of 1, 2 and 3 steps cover the
centred start of the sources and of the Lorentz recurrence inside a fused launch."""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from parity_bounds import assert_parity, fp64_force_floor

pytestmark = pytest.mark.gpu

ONE = {"steps_per_launch": 1}
TWO = {"steps_per_launch": 2}


@pytest.fixture(scope="module")
def pk():
    from paper_0906_5170_gb300 import build
    build.build()
    import paper_0906_5170_gb300 as pkg
    return pkg


@pytest.fixture(scope="module")
def ctx(pk):
    c = pk.Context(0)
    yield c
    c.close()


_CACHE = {}


def _oracle(p, key):
    if key not in _CACHE:
        F, parts, _ = oracle.force(p, return_parts=True)
        _CACHE[key] = (F, np.array(parts))
    return _CACHE[key]


def _run(ctx, p, opts):
    """One synchronous run; st["steps_launched"] = launch indices the run took (ceil(T / k) for
    k steps per launch)."""
    ctx.kernel_stats(reset=True)
    F, per, st = ctx.plan(p, options=opts).run(per_sim=True)
    st = dict(st, steps_launched=ctx.kernel_stats(reset=True)[1])
    return F[p["force_axis"]], np.asarray(per), st


def _check_two_step(ctx, p, key, opts=TWO):
    """The two-step march against the oracle and against the one-step march; returns the launch
    indices each run took."""
    T = p["n_steps"]
    F2, per2, st2 = _run(ctx, p, opts)
    F1, per1, st1 = _run(ctx, p, dict(opts, steps_per_launch=1))
    Fo, parts = _oracle(p, key)
    assert_parity(per2, F2, parts, Fo, T, False, str(key) + " two-step")
    assert_parity(per1, F1, parts, Fo, T, False, str(key) + " one-step")
    scale = np.max(np.abs(per1))
    err = np.max(np.abs(per2 - per1))
    assert err <= 2e-5 * scale, f"{key}: two-step vs one-step per-sim error {err:.3e} > 2e-5 * {scale:.3e}"
    assert abs(F2 - F1) <= 1e-4 * abs(F1) + fp64_force_floor(per1, T), f"{key}: two-step {F2!r} vs one-step {F1!r}"
    return st2["steps_launched"], st1["steps_launched"]


def _waveguides(n_steps, kz_list=(0.0, 1.3, 4.0)):
    # two Lorentz waveguides (one pole), CPML all round, real fields with d/dz -> k_z; 48 x 48 cells
    # make one full strip of 28 columns and a ragged one of 20
    return W.config3_waveguides(0.5, resolution=8, n_cells=48, pml_units=0.75, n_harm=3, n_steps=n_steps,
                                k_points=[{"k": [0, 0, k], "weight": 0.3} for k in kz_list], precision="fp32")


def _bloch(n_steps):
    # complex fields: Bloch phase along periodic x and k_z; CPML along y; a dielectric bar and a
    # Lorentz slab (one pole) next to the CPML; stress lines on both sides of the bar
    p = W._base(2, (16, 24, 1), 8.0, n_steps)
    p["bc"] = ["periodic", "pml", "pec"]
    p["pml_cells"] = [0, 4, 0]
    p["objects"] = [{"shape": "box", "lo": [0.5, 1.0, 0], "hi": [1.5, 1.5, 0], "kind": "dielectric", "eps": 4.0, "mu": 1.0},
                    {"shape": "box", "lo": [0.0, 1.9, 0], "hi": [2.0, 2.0, 0], "kind": "lorentz",
                     "eps_inf": 1.0, "delta_eps": 3.0, "omega0": 2.0}]
    p["faces"] = [{"axis": 1, "sign": -1, "pos": 0.75, "lo": [0, 0.75, 0], "hi": [2.0, 0.75, 0]},
                  {"axis": 1, "sign": 1, "pos": 1.75, "lo": [0, 1.75, 0], "hi": [2.0, 1.75, 0]}]
    p["n_harm"] = 4
    p["polarization"] = "full"
    p["force_axis"] = 1
    p["k_points"] = [{"k": [2 * math.pi * m / (3 * 2.0), 0, 0.7 * m], "weight": 1 / 3} for m in range(3)]
    p["precision"] = "fp32"
    return p


@pytest.mark.parametrize("n_steps", [300, 301])
def test_waveguides_kz_cpml_one_pole(ctx, n_steps):
    l2, l1 = _check_two_step(ctx, _waveguides(n_steps), ("wg", n_steps))
    assert l1 == n_steps and l2 == (n_steps + 1) // 2


@pytest.mark.parametrize("n_steps", [240, 241])
def test_bloch_complex_cpml_one_pole(ctx, n_steps):
    l2, l1 = _check_two_step(ctx, _bloch(n_steps), ("bloch", n_steps))
    assert l2 == (n_steps + 1) // 2 and l1 == n_steps


@pytest.mark.parametrize("n_steps", [1, 2, 3])
def test_short_runs(ctx, n_steps):
    # the halved first step and the Lorentz start from rest inside a fused launch; one-step runs
    # take a launch with step A alone
    _check_two_step(ctx, _bloch(n_steps), ("bloch_short", n_steps))
    _check_two_step(ctx, _waveguides(n_steps, (1.3,)), ("wg_short", n_steps))


@pytest.mark.parametrize("rows", [16, 64])
def test_tile_heights(ctx, rows):
    # tiles of 16 rows (several row bands, ragged last band) and of 64 (one band taller than the grid)
    _check_two_step(ctx, _waveguides(200, (0.0, 2.5)), ("wg_rows", rows), dict(TWO, march_rows=rows))


def test_grating_membrane_serving_cell(ctx):
    # the grooved membrane of the serving mix at a quarter of its size: 32 x 128 cells, 16 Bloch
    # k_x points (complex fields), CPML along y, dielectric only
    rng = np.random.default_rng(11)
    p = W._serving_grating(0.25, rng)
    p["n_steps"] = 400
    p["k_points"] = p["k_points"][::4]
    _check_two_step(ctx, p, "grating_serving")


def _tiny(nx, ny, kind):
    res = 10.0
    p = W._base(2, (nx, ny, 1), res, 240)
    Lx, Ly = nx / res, ny / res
    if ny >= 8:
        p["bc"] = ["periodic", "pec", "pec"]
        p["objects"] = [{"shape": "box", "lo": [0.0, 2.5, 0], "hi": [Lx, 2.5, 0], "kind": "pec"},
                        {"shape": "box", "lo": [0.0, 0.5, 0], "hi": [Lx, 1.0, 0], "kind": "dielectric", "eps": 2.5, "mu": 1.0}]
        p["faces"] = [{"axis": 1, "sign": -1, "pos": 1.9, "lo": [0.0, 1.9, 0], "hi": [Lx, 1.9, 0]}]
        p["force_axis"] = 1
        ax = 0
    else:
        p["bc"] = ["pec", "periodic", "pec"]
        p["objects"] = [{"shape": "box", "lo": [0.6 * Lx, 0.0, 0], "hi": [0.8 * Lx, Ly, 0], "kind": "dielectric", "eps": 3.0, "mu": 1.0}]
        x = round(0.3 * nx) / res
        p["faces"] = [{"axis": 0, "sign": 1, "pos": x, "lo": [x, 0.0, 0], "hi": [x, Ly, 0]}]
        p["force_axis"] = 0
        ax = 1
    p["n_harm"] = min(3, max(1, (nx if p["force_axis"] == 1 else ny)))
    p["polarization"] = "full"
    p["precision"] = "fp32"
    if kind == "kz":
        p["k_points"] = [{"k": [0.0, 0.0, kz], "weight": 0.5} for kz in (0.0, 1.7)]
    else:
        L = p["n"][ax] / res
        p["k_points"] = []
        for m in range(2):
            k = [0.0, 0.0, 0.9]
            k[ax] = 2 * math.pi * (m + 0.5) / (2 * L)
            p["k_points"].append({"k": k, "weight": 0.5})
    return p


@pytest.mark.parametrize("nx,ny,kind", [(7, 40, "kz"), (40, 1, "bloch"), (3, 2, "kz"), (6, 33, "bloch"), (29, 30, "bloch")])
def test_tiny_and_narrow_grids(ctx, nx, ny, kind):
    # grids narrower than the strip's halo (the wrapped lanes repeat columns), one or two rows
    # high, and one column wider than a strip (a second strip of one column)
    _check_two_step(ctx, _tiny(nx, ny, kind), ("tiny", nx, ny, kind))


def test_three_poles_and_fp64_keep_one_step(ctx):
    # a material with three poles (silica), or FP64 fields, take the one-step march whatever the option
    p = W.grating_silica(0.5, resolution=16, nk_x=2, nk_z=2, n_harm=2, t_max=3.0, courant=0.2, pml_units=0.25,
                         precision="fp32")
    _, _, st = _run(ctx, p, TWO)
    assert st["steps_launched"] == p["n_steps"]
    q = _waveguides(60, (1.3,))
    q["precision"] = "fp64"
    _, _, st = _run(ctx, q, TWO)
    assert st["steps_launched"] == q["n_steps"]


def test_mixed_batch_of_one_and_two_step_runs(ctx, pk):
    # two-step Cartesian runs share the batch with one-step and three-step runs; the forces equal
    # those of each problem alone
    probs = [(_waveguides(301, (1.3,)), TWO), (_bloch(240), ONE), (W.piston_small(h=0.7, n_steps=300, precision="fp32"), None),
             (_bloch(241), TWO)]
    alone = [_run(ctx, p, o)[0] for p, o in probs]
    plans = [ctx.plan(p, options=o) for p, o in probs]
    tickets = [pl.submit(tag=i) for i, pl in enumerate(plans)]
    for i, t in enumerate(tickets):
        F = t.force(-1)[0][probs[i][0]["force_axis"]]
        assert np.isclose(F, alone[i], rtol=1e-9, atol=0), (i, F, alone[i])
