"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle,
simulation by simulation and for the force, on seeded synthetic geometries.

Tolerances (tests/parity_bounds.py): FP64 mode 1e-10 relative per simulation, and
for the force 1e-10 relative plus the FP64 rounding floor of a cancelling sum; FP32
fields with FP64 accumulation: the force within 1e-4 of itself (plus the same floor of
its FP64 sum), each simulation within 2e-5 of the largest contribution."""
import numpy as np
import pytest

import oracle
import workloads as W
from parity_bounds import assert_parity, fp64_force_floor

pytestmark = pytest.mark.gpu


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


_ORACLE_CACHE = {}


def _oracle(p, key):
    if key not in _ORACLE_CACHE:
        F, parts, _ = oracle.force(p, return_parts=True)
        _ORACLE_CACHE[key] = (F, np.array(parts))
    return _ORACLE_CACHE[key]


def _check(ctx, p, key, fp64, options=None):
    F, per, st = ctx.plan(p, options=options).run(per_sim=True)
    Fo, parts = _oracle(p, key)
    fa = p["force_axis"]
    assert_parity(per, F[fa], parts, Fo, p["n_steps"], fp64, str(key))
    assert st["kernel_launches"] > 0
    return F[fa], Fo, per, parts


def test_config1_plates_fp64_full(ctx):
    p = W.config1_plates()           # the full-size configuration: 60 x 40, 8 harmonics, 4000 steps
    _check(ctx, p, "c1", True)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_piston_te_tm(ctx, prec):
    p = W.piston_small(n_steps=800, precision=prec)
    _check(ctx, p, ("piston", prec), prec == "fp64")


def test_piston_fp32_force_relative(ctx):
    # the force itself (after cancellation) to 1e-4 relative on a closed contour
    p = W.piston_small(n_steps=1200, precision="fp32", n_harm=8)
    Fg, Fo, _, _ = _check(ctx, p, "pist32f", False)
    assert abs(Fg - Fo) <= 1e-4 * abs(Fo)


def test_ragged_multi_tile_grid(ctx):
    # several tiles in both directions with ragged tails (nx = 83, ny = 45)
    p = W._base(2, (83, 45, 1), 10.0, 500)
    p["objects"] = [{"shape": "box", "lo": [3.0, 1.0, 0], "hi": [4.5, 2.9, 0], "kind": "pec"},
                    {"shape": "box", "lo": [5.5, 0.5, 0], "hi": [6.0, 3.5, 0], "kind": "dielectric", "eps": 3.0, "mu": 1.0}]
    p["faces"] = W.box_faces([2.8, 0.8], [4.8, 3.3], 2)
    p["n_harm"] = 5
    p["polarization"] = "TE+TM"
    p["force_axis"] = 0
    p["precision"] = "fp64"
    _check(ctx, p, "ragged", True)


def test_pmc_sidewalls_and_point_basis(ctx):
    p = W.piston_small(n_steps=400, precision="fp64")
    L = p["n"][1] / p["resolution"]
    p["objects"] = p["objects"] + [
        {"shape": "box", "lo": [0.0, 0.0, 0.0], "hi": [6.0, 0.05, 0.0], "kind": "pmc"},
        {"shape": "box", "lo": [0.0, L - 0.05, 0.0], "hi": [6.0, L, 0.0], "kind": "pmc"}]
    _check(ctx, p, "pmc", True)
    q = dict(p, basis="point", n_steps=200)
    _check(ctx, q, "point", True)


def test_periodic_axis(ctx):
    p = W.piston_small(n_steps=400, precision="fp64")
    p["bc"] = ["periodic", "pec", "pec"]
    _check(ctx, p, "periodic", True)


def test_results_identical_alone_and_in_a_mix(ctx, pk):
    probs = [W.piston_small(h=0.5, n_steps=600), W.config1_plates(),
             W.piston_small(h=1.0, n_steps=300, precision="fp32"), W.piston_small(h=0.7, n_steps=900)]
    for p in probs:
        if p.get("precision") != "fp64":
            p["precision"] = "fp32"
    probs[1] = dict(probs[1], precision="fp32")
    alone = [ctx.plan(p).run()[0] for p in probs]
    plans = [ctx.plan(p) for p in probs]
    tickets = []
    for i, pl in enumerate(plans):
        tickets.append(pl.submit(tag=i))
    res = [t.force(-1) for t in tickets]
    for a, (F, err, st) in zip(alone, res):
        assert np.allclose(F, a, rtol=1e-12, atol=0)


def test_staggered_arrivals_join_running_batch(ctx, pk):
    import time
    p1 = W.config1_plates()
    p1["precision"] = "fp32"
    p2 = W.piston_small(n_steps=3000, precision="fp32")
    a1 = ctx.plan(p1).run()[0]
    a2 = ctx.plan(p2).run()[0]
    pl2 = ctx.plan(p2)
    pl1 = ctx.plan(p1)
    t2 = pl2.submit()
    time.sleep(0.02)
    t1 = pl1.submit()           # arrives while the first request runs
    F1 = t1.force(-1)[0]
    F2 = t2.force(-1)[0]
    assert np.allclose(F1, a1, rtol=1e-12, atol=0)
    assert np.allclose(F2, a2, rtol=1e-12, atol=0)


def test_watchdog_and_cancel_leave_context_usable(ctx, pk):
    p = W.config2_piston(W.config2_heights()[0], n_harm=4, n_steps=20000)
    ctx.set_watchdog(50.0)
    t = ctx.plan(p).submit()
    with pytest.raises(pk.CasimirError) as e:
        t.force(-1)
    assert e.value.code == -5
    ctx.set_watchdog(0.0)
    t = ctx.plan(p).submit()
    t.cancel()
    with pytest.raises(pk.CasimirError) as e:
        t.force(-1)
    assert e.value.code == -6
    q = W.piston_small(n_steps=300, precision="fp64")
    _check(ctx, q, "after", True)


def test_plan_teardown_overlapping_graph_capture(ctx, pk):
    """Destroying a plan from the caller's thread (its tables are freed after a synchronisation of
    the context stream) while the worker admits the next request and captures its first chunk
    graph on that stream: the capture and the request are unaffected; a cancelled request ends
    cancelled, never failed."""
    p = W.piston_small(n_steps=120)
    ref = ctx.plan(p).run()[0]
    prev = ctx.plan(p)
    prev.run()                                  # its tables are on the device
    for it in range(12):
        pl = ctx.plan(p)
        t = pl.submit()
        if it % 2:
            t.cancel()
        prev.close()                            # overlaps the worker's admission and capture
        prev = pl
        try:
            F = t.force(-1)[0]
        except pk.CasimirError as e:
            assert it % 2 and e.code == -6, (it, e)
            continue
        assert F == pytest.approx(ref, rel=1e-9, abs=0)
    prev.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_voxel_mask_objects(ctx, prec):
    """Arbitrary geometry as voxel masks: an L-shaped PEC block (voxels on the Yee lattice) and a
    seeded random dielectric pattern of 0.07-wide voxels in the gap (sites anywhere in a voxel,
    some on voxel faces); the planner's mask rasterisation against the oracle's."""
    p = W.piston_small(n_steps=400, precision=prec, g_variant="plain")   # plain g: any medium
    m = np.zeros((10, 10), np.uint8)
    m[:, :5] = 1
    m[:5, 5:] = 1
    r = (np.random.default_rng(3).random((10, 7)) < 0.4).astype(np.uint8)
    p["objects"] = [p["objects"][0], W.grid_object(m, [3.5, 0.5], [4.5, 1.5], kind="pec"),
                    W.grid_object(r, [2.6, 0.75], [3.3, 1.24], kind="dielectric", eps=2.5, mu=1.0)]
    _check(ctx, p, ("mask", prec), prec == "fp64")


def test_budget_rejects_oversized_plan(pk):
    c = pk.Context(0, hbm_budget_bytes=1 << 20)
    with pytest.raises(pk.CasimirError) as e:
        c.plan(W.config2_piston(W.config2_heights()[7], n_steps=100))
    assert e.value.code == -2
    c.close()


# ---- six-component kernel: k_z cross-sections, Bloch cells, 3D; CPML; Lorentz ----------

def _waveguides_small(prec, kz_list=(0.0, 1.3, 4.0)):
    p = W.config3_waveguides(0.5, resolution=8, n_cells=48, pml_units=0.75, n_harm=3, n_steps=300,
                             k_points=[{"k": [0, 0, k], "weight": 0.3} for k in kz_list], precision=prec)
    return p


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_full_kz_pml_lorentz(ctx, prec):
    p = _waveguides_small(prec)
    _check(ctx, p, ("wg", prec), prec == "fp64")


def test_full_bloch_complex(ctx):
    import math
    p = W._base(2, (16, 24, 1), 8.0, 300)
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
    p["precision"] = "fp64"
    _check(ctx, p, "bloch", True)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_full_3d_sphere_notch(ctx, prec):
    p = W.config4_sphere_notch(0.4, seed=3, resolution=6, n_cells=24, pml_cells=4, n_harm=2, n_steps=120,
                               precision=prec, substrate_top=1.0)
    _check(ctx, p, ("3d", prec), prec == "fp64")


def _box3d_ragged(pml):
    """A 3D cell of 37 x 19 x 45 cells: several column tiles with ragged edges along x and y and
    two chunks of planes along z; a dielectric sphere over a PEC slab, a cubic stress surface
    around the sphere, J and K sources (force along z); with CPML on x and z when pml."""
    res = 8.0
    p = W._base(3, (37, 19, 45), res, 60)
    p["objects"] = [{"shape": "box", "lo": [0.0, 0.0, 0.0], "hi": [37 / res, 19 / res, 1.0], "kind": "pec"},
                    {"shape": "sphere", "center": [2.3, 1.2, 3.0], "radius": 0.6, "kind": "dielectric",
                     "eps": 3.0, "mu": 1.0}]
    p["faces"] = W.box_faces([1.5, 0.375, 2.25], [3.125, 2.0, 3.875], 3)
    p["n_harm"] = 2
    p["polarization"] = "full"
    p["force_axis"] = 2
    if pml:
        p["bc"] = ["pml", "pec", "pml"]
        p["pml_cells"] = [4, 0, 4]
    return p


@pytest.mark.parametrize("pml", [False, True])
def test_column_march_ragged_tiles_and_plane_chunks(ctx, pml):
    # the fused 3D column march (kernel_3d 3) against the oracle, and against the x-line kernel
    p = _box3d_ragged(pml)
    _check(ctx, p, ("col3", pml), True, {"kernel_3d": 3})
    _, per3, _ = ctx.plan(p, options={"kernel_3d": 3}).run(per_sim=True)
    _, per1, _ = ctx.plan(p, options={"kernel_3d": 1}).run(per_sim=True)
    assert np.allclose(per3, per1, rtol=1e-10, atol=1e-14 * np.sum(np.abs(per1)))


def test_mixed_2d_and_full_requests_share_the_batch(ctx):
    probs = [W.piston_small(n_steps=400, precision="fp32"), _waveguides_small("fp32", (0.5,)),
             W.piston_small(h=0.8, n_steps=250, precision="fp64"), _waveguides_small("fp64", (2.0,))]
    alone = [ctx.plan(p).run()[0] for p in probs]
    plans = [ctx.plan(p) for p in probs]
    tickets = [pl.submit(tag=i) for i, pl in enumerate(plans)]
    for a, t in zip(alone, tickets):
        F, err, st = t.force(-1)
        assert np.allclose(F, a, rtol=1e-12, atol=0)


@pytest.mark.parametrize("which", ["2d", "full"])
def test_plain_path_matches_batched(ctx, which):
    p = W.piston_small(n_steps=300, precision="fp64") if which == "2d" else _waveguides_small("fp64", (0.0, 2.5))
    Fb, pb, _ = ctx.plan(p).run(per_sim=True)
    Fp, pp, st = ctx.plan(p).run(per_sim=True, plain=True)
    assert np.allclose(pp, pb, rtol=1e-9, atol=1e-13 * np.sum(np.abs(pb)))
    assert st["kernel_launches"] > p["n_steps"]


def test_waves_do_not_change_results(ctx):
    probs = [W.piston_small(n_steps=300, precision="fp32"), _waveguides_small("fp32", (0.0, 2.0))]
    whole = []
    for p in probs:
        ctx.set_wave_bytes(0)                    # every simulation of the request at once
        whole.append(ctx.plan(p).run(per_sim=True))
        ctx.set_wave_bytes(200_000)             # a few simulations per wave
        _, waves, _ = ctx.plan(p).run(per_sim=True)
        assert np.allclose(waves, whole[-1][1], rtol=1e-12, atol=1e-15 * np.sum(np.abs(whole[-1][1])))
    # both requests in flight together, in small waves
    plans = [ctx.plan(p) for p in probs]
    tickets = [pl.submit() for pl in plans]
    for t, (F0, _, _) in zip(tickets, whole):
        F, _, _ = t.force(-1)
        assert np.allclose(F, F0, rtol=1e-12, atol=0)
    ctx.set_wave_bytes(0)


# ---- three time steps per launch (2D TM/TE) ----------------------------------------------

K3 = {"steps_per_launch": 3}


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n_steps", [300, 301, 302])
def test_three_steps_per_launch_piston(ctx, prec, n_steps):
    # J and K sources (sigma on u and on v), and runs whose last launch holds 3, 1 or 2 steps
    p = W.piston_small(n_steps=n_steps, precision=prec)
    _check(ctx, p, ("piston", prec, n_steps), prec == "fp64", K3)


@pytest.mark.parametrize("n_steps", [1, 2, 4])
def test_three_steps_per_launch_short_runs(ctx, n_steps):
    # the first launch itself holds fewer than three steps (the half step at n = 1 included)
    p = W.piston_small(n_steps=n_steps, precision="fp64")
    _check(ctx, p, ("piston_short", n_steps), True, K3)


def test_three_steps_per_launch_ragged_periodic_pmc(ctx):
    p = W._base(2, (83, 45, 1), 10.0, 500)
    p["objects"] = [{"shape": "box", "lo": [3.0, 1.0, 0], "hi": [4.5, 2.9, 0], "kind": "pec"},
                    {"shape": "box", "lo": [5.5, 0.5, 0], "hi": [6.0, 3.5, 0], "kind": "dielectric", "eps": 3.0, "mu": 1.0}]
    p["faces"] = W.box_faces([2.8, 0.8], [4.8, 3.3], 2)
    p["n_harm"] = 5
    p["polarization"] = "TE+TM"
    p["force_axis"] = 0
    p["precision"] = "fp64"
    _check(ctx, p, "ragged", True, K3)
    q = W.piston_small(n_steps=400, precision="fp64")
    q["bc"] = ["periodic", "pec", "pec"]
    _check(ctx, q, "periodic", True, K3)
    r = W.piston_small(n_steps=400, precision="fp64")
    L = r["n"][1] / r["resolution"]
    r["objects"] = r["objects"] + [
        {"shape": "box", "lo": [0.0, 0.0, 0.0], "hi": [6.0, 0.05, 0.0], "kind": "pmc"},
        {"shape": "box", "lo": [0.0, L - 0.05, 0.0], "hi": [6.0, L, 0.0], "kind": "pmc"}]
    _check(ctx, r, "pmc", True, K3)


@pytest.mark.parametrize("nx,ny", [(7, 40), (40, 1), (3, 2), (26, 3), (27, 64)])
def test_three_steps_per_launch_tiny_grids(ctx, nx, ny):
    p = _tiny_2d(nx, ny, "TE+TM")
    _check(ctx, p, ("tiny2d", nx, ny), True, K3)


def test_three_steps_per_launch_in_a_mixed_batch(ctx):
    # plans of 1, 2 and 3 steps per launch run side by side in one batch, each as alone
    probs = [(W.piston_small(h=0.5, n_steps=301), {"steps_per_launch": 3}),
             (W.piston_small(h=0.7, n_steps=300), {"steps_per_launch": 2}),
             (W.piston_small(h=0.9, n_steps=299, precision="fp32"), {"steps_per_launch": 3}),
             (W.piston_small(h=0.6, n_steps=200), {"steps_per_launch": 1})]
    alone = [ctx.plan(p, options=o).run()[0] for p, o in probs]
    plans = [ctx.plan(p, options=o) for p, o in probs]
    tickets = [pl.submit(tag=i) for i, pl in enumerate(plans)]
    for a, t in zip(alone, tickets):
        F, err, st = t.force(-1)
        assert np.allclose(F, a, rtol=1e-12, atol=0)


# ---- degenerate grids: narrower than a warp strip, a single row ---------------------------

def _tiny_2d(nx, ny, pol):
    res = 10.0
    p = W._base(2, (nx, ny, 1), res, 240)
    Lx, Ly = nx / res, ny / res
    if ny >= 8:      # periodic x, a PEC plate across the cell, an open line below it
        p["bc"] = ["periodic", "pec", "pec"]
        p["objects"] = [{"shape": "box", "lo": [0.0, 2.5, 0], "hi": [Lx, 2.5, 0], "kind": "pec"},
                        {"shape": "box", "lo": [0.0, 0.5, 0], "hi": [Lx, 1.0, 0], "kind": "dielectric", "eps": 2.5, "mu": 1.0}]
        p["faces"] = [{"axis": 1, "sign": -1, "pos": 1.9, "lo": [0.0, 1.9, 0], "hi": [Lx, 1.9, 0]}]
        p["force_axis"] = 1
    else:            # periodic y (one or two rows), a dielectric slab across x, a line normal to x
        p["bc"] = ["pec", "periodic", "pec"]
        p["objects"] = [{"shape": "box", "lo": [0.6 * Lx, 0.0, 0], "hi": [0.8 * Lx, Ly, 0], "kind": "dielectric", "eps": 3.0, "mu": 1.0}]
        x = round(0.3 * nx) / res
        p["faces"] = [{"axis": 0, "sign": 1, "pos": x, "lo": [x, 0.0, 0], "hi": [x, Ly, 0]}]
        p["force_axis"] = 0
    p["n_harm"] = min(3, max(1, (nx if p["force_axis"] == 1 else ny)))
    p["polarization"] = pol
    return p


@pytest.mark.parametrize("nx,ny", [(7, 40), (40, 1), (3, 2)])
def test_tiny_grids_2d(ctx, nx, ny):
    # the two-step kernel (batched path) and the one-step kernel (plain path) on grids
    # narrower than a warp strip or only one or two rows high
    p = _tiny_2d(nx, ny, "TE+TM")
    _check(ctx, p, ("tiny2d", nx, ny), True)
    Fb, pb, _ = ctx.plan(p).run(per_sim=True)
    Fp, pp, _ = ctx.plan(p).run(per_sim=True, plain=True)
    assert np.allclose(pp, pb, rtol=1e-9, atol=1e-13 * np.sum(np.abs(pb)))


@pytest.mark.parametrize("nx,ny,kind", [(7, 40, "kz"), (40, 1, "bloch"), (3, 2, "kz"), (6, 33, "bloch")])
def test_tiny_grids_six_component(ctx, nx, ny, kind):
    import math
    p = _tiny_2d(nx, ny, "full")
    if kind == "kz":          # real fields, d/dz -> k_z
        p["k_points"] = [{"k": [0.0, 0.0, kz], "weight": 0.5} for kz in (0.0, 1.7)]
    else:                     # complex fields: Bloch phase along the periodic axis, and k_z
        ax = 0 if p["bc"][0] == "periodic" else 1
        L = p["n"][ax] / p["resolution"]
        p["k_points"] = []
        for m in range(2):
            k = [0.0, 0.0, 0.9]
            k[ax] = 2 * math.pi * (m + 0.5) / (2 * L)
            p["k_points"].append({"k": k, "weight": 0.5})
    _check(ctx, p, ("tiny6", nx, ny, kind), True)
    Fb, pb, _ = ctx.plan(p).run(per_sim=True)
    Fp, pp, _ = ctx.plan(p).run(per_sim=True, plain=True)
    assert np.allclose(pp, pb, rtol=1e-9, atol=1e-13 * np.sum(np.abs(pb)))


def test_plain_path_march_kernel_in_subprocess():
    # the plain path runs large two-dimensional six-component runs through the march kernel and
    # small ones through the two-phase kernel; force the march kernel here and compare with the
    # batched results of the same plan
    import os, subprocess, sys, json
    code = r'''
import json, sys
import numpy as np
sys.path.insert(0, ".")
import workloads as W
import paper_0906_5170_gb300 as pk
p = W.config3_waveguides(0.5, resolution=8, n_cells=48, pml_units=0.75, n_harm=3, n_steps=300,
                         k_points=[{"k": [0, 0, k], "weight": 0.3} for k in (0.0, 2.5)], precision="fp64")
ctx = pk.Context(0)
_, pb, _ = ctx.plan(p).run(per_sim=True)
_, pp, st = ctx.plan(p).run(per_sim=True, plain=True)
print(json.dumps({"ok": bool(np.allclose(pp, pb, rtol=1e-9, atol=1e-13 * np.sum(np.abs(pb)))),
                  "launches": st["kernel_launches"]}))
ctx.close()
'''
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, CASIMIR_PLAIN_MARCH_TILES="0")
    out = subprocess.run([sys.executable, "-c", code], cwd=root, env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    res = json.loads(out.stdout.strip().splitlines()[-1])
    assert res["ok"]


def test_complete_cosine_basis_equals_point_basis_on_gpu(ctx):
    # completeness of the face basis (Sec. III A, Eq. 7): with every harmonic of every face the
    # cosine-basis force equals the point-source force, on the GPU path alone (no oracle)
    p = W.piston_small(n_steps=400, precision="fp64")
    F_cos, per_cos, _ = ctx.plan(dict(p, n_harm=100000)).run(per_sim=True)
    F_pt, per_pt, _ = ctx.plan(dict(p, basis="point")).run(per_sim=True)
    fa = p["force_axis"]
    bound = 1e-10 * abs(F_pt[fa]) + fp64_force_floor(np.concatenate([per_cos, per_pt]), p["n_steps"])
    assert abs(F_cos[fa] - F_pt[fa]) <= bound
    # a truncated cosine basis differs, and the difference shrinks with the harmonic count
    errs = [abs(ctx.plan(dict(p, n_harm=k)).run()[0][fa] - F_pt[fa]) for k in (2, 4, 8)]
    assert errs[0] > errs[1] > errs[2] > bound


def test_complete_cosine_basis_equals_point_basis_3d(ctx):
    # the same completeness in 3D (x-line kernel): every face of the cubic surface carries
    # a 2D cosine series over its pixels; complete, it spans the same space as the pixels
    p = W.config4_sphere_notch(0.4, seed=3, resolution=6, n_cells=24, pml_cells=4, n_harm=1, n_steps=60,
                               precision="fp64", substrate_top=1.0)
    F_cos, per_cos, _ = ctx.plan(dict(p, n_harm=100000)).run(per_sim=True)
    F_pt, per_pt, _ = ctx.plan(dict(p, basis="point")).run(per_sim=True)
    assert len(per_pt) == len(per_cos) > 1000
    fa = p["force_axis"]
    assert abs(F_cos[fa] - F_pt[fa]) <= 1e-10 * abs(F_pt[fa]) + fp64_force_floor(
        np.concatenate([per_cos, per_pt]), p["n_steps"])
    # and sampled point-basis simulations against the oracle
    sims = oracle.enumerate_sims(dict(p, basis="point"))
    w = oracle.g_weights(p)
    q = dict(p, basis="point")
    st = oracle.grid_setup(q, q["k_points"][0]["k"])
    for i in (0, len(sims) // 2, len(sims) - 1):
        r = float(np.sum(w * oracle.run_sim(q, sims[i], st).real)) * q["k_points"][0]["weight"]
        assert abs(per_pt[i] - r) <= 1e-10 * abs(r)


# ---- cylindrical (r, z) runs with exp(i m phi) fields (Sec. III C) -------------------------

@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_cylindrical_piston(ctx, prec):
    p = W.cylinder_piston(12, [0, 1, 2, 3], t_max=6.0, precision=prec)
    _check(ctx, p, ("cyl", prec), prec == "fp64")


def test_cylindrical_multi_strip_ragged(ctx):
    # 40 radial cells: two warp strips (30 + 10) and two row bands along z
    p = W.cylinder_piston(40, [0, 2], radius=1.0, below=0.4, above=0.7, t_max=1.5, n_harm=6)
    _check(ctx, p, "cyl_wide", True)


@pytest.mark.parametrize("steps", [1, 2])
@pytest.mark.parametrize("n_extra", [0, 1])
def test_cylindrical_steps_per_launch(ctx, steps, n_extra):
    # one and two steps per launch against the oracle, runs of even and odd length (the last
    # two-step launch then holds one step), J and K sources, m = 0 .. 2
    p = W.cylinder_piston(12, [0, 1, 2], t_max=4.0, precision="fp64")
    p["n_steps"] = p["n_steps"] + n_extra
    _check(ctx, p, ("cyl_steps", n_extra), True, {"steps_per_launch": steps})


@pytest.mark.parametrize("rows", [16, 64])
def test_cylindrical_two_steps_ragged_tiles(ctx, rows):
    # 40 radial cells: two 28-column strips (28 + 12), row bands of 16 or 64 along z
    p = W.cylinder_piston(40, [0, 2], radius=1.0, below=0.4, above=0.7, t_max=1.5, n_harm=6)
    _check(ctx, p, ("cyl_wide", rows), True, {"steps_per_launch": 2, "march_rows": rows})


def test_batch_mixing_fusion_depths(ctx):
    # a two-step cylindrical plan, three-step and two-step 2D plans and a one-step six-component
    # plan in one batch: each simulation derives its steps from the shared launch counter and
    # its plan's depth; every force equals the plan's force alone
    probs = [W.cylinder_piston(12, [0, 1], t_max=3.0, precision="fp32"),
             W.piston_small(h=0.6, n_steps=301, precision="fp32"),
             W.piston_small(h=0.8, n_steps=300, precision="fp64"),
             W.config3_waveguides(0.5, resolution=8, n_cells=48, pml_units=0.75, n_harm=2, n_steps=150,
                                  k_points=[{"k": [0, 0, 1.0], "weight": 0.5}], precision="fp32")]
    alone = [ctx.plan(p).run()[0] for p in probs]
    plans = [ctx.plan(p) for p in probs]
    assert [pl.options()["steps_per_launch"] for pl in plans][:3] == [3, 3, 2]
    tickets = [pl.submit(tag=i) for i, pl in enumerate(plans)]
    for a, t in zip(alone, tickets):
        F, err, st = t.force(-1)
        assert np.allclose(F, a, rtol=1e-12, atol=0)


def test_cylindrical_plain_path_and_mixed_batch(ctx):
    p = W.cylinder_piston(10, [0, 1], t_max=4.0, precision="fp64")
    Fb, pb, _ = ctx.plan(p).run(per_sim=True)
    Fp, pp, _ = ctx.plan(p).run(per_sim=True, plain=True)
    assert np.allclose(pp, pb, rtol=1e-9, atol=1e-13 * np.sum(np.abs(pb)))
    q = W.piston_small(n_steps=300, precision="fp64")
    Fq = ctx.plan(q).run()[0]
    t1, t2 = ctx.plan(p).submit(), ctx.plan(q).submit()
    assert np.allclose(t1.force(-1)[0], Fb, rtol=1e-12, atol=0)
    assert np.allclose(t2.force(-1)[0], Fq, rtol=1e-12, atol=0)


# ---- execution options and the autotuner ---------------------------------------------------

def test_execution_options_do_not_change_results(ctx):
    cases = [
        (W.piston_small(n_steps=300, precision="fp64"), [{"steps_per_launch": 1}, {"steps_per_launch": 2}, {"steps_per_launch": 3}]),
        (_waveguides_small("fp64", (0.0, 1.3)), [{"march_rows": 16}, {"march_rows": 32}, {"march_rows": 64}]),
        (W.config4_sphere_notch(0.4, seed=3, resolution=6, n_cells=24, pml_cells=4, n_harm=1, n_steps=60,
                                precision="fp64", substrate_top=1.0), [{"kernel_3d": 3}, {"kernel_3d": 1}, {"kernel_3d": 2}]),
        (W.cylinder_piston(12, [0, 1, 2], t_max=4.0), [{"march_rows": 16}, {"march_rows": 64}]),
    ]
    for p, opts in cases:
        res = []
        for o in opts:
            pl = ctx.plan(p, options=o)
            assert all(pl.options()[k] == v for k, v in o.items())
            res.append(pl.run(per_sim=True)[1])
        scale = np.sum(np.abs(res[0]))
        for r in res[1:]:
            assert np.allclose(r, res[0], rtol=1e-10, atol=1e-14 * scale)


def test_autotune_picks_caches_and_keeps_results(pk, ctx):
    c = pk.Context(0)
    try:
        c.set_autotune(True)
        p = W.piston_small(n_steps=300, precision="fp64")
        pl = c.plan(p)
        o = pl.options()
        assert o["steps_per_launch"] in (1, 2, 3)
        # a problem of the same class reuses the choice
        assert c.plan(W.piston_small(h=0.55, n_steps=300, precision="fp64")).options() == o
        F, per, _ = pl.run(per_sim=True)
        _, ref, _ = ctx.plan(p).run(per_sim=True)
        assert np.allclose(per, ref, rtol=1e-10, atol=1e-14 * np.sum(np.abs(ref)))
        # six-component class: one of the candidate tile heights
        q = _waveguides_small("fp32", (0.0, 1.3))
        assert c.plan(q).options()["march_rows"] in (16, 32, 64)
        # the trials leave the user's kernel statistics alone
        c.kernel_stats(reset=True)
        c.plan(W.cylinder_piston(10, [0, 1], t_max=2.0))
        assert c.kernel_stats()[0] == 0.0
    finally:
        c.close()
