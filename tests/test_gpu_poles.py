"""GPU parity for sums of undamped Lorentz poles (the silicon and silica models of
Sec. III D): every kernel that carries the auxiliary equations (the two-dimensional march,
the two-phase one-thread-per-cell kernel, the three-dimensional x-line kernel, the plain
path) against the FP64 oracle, simulation by simulation.

Tolerances as in the other parity tests (tests/parity_bounds.py): FP64 1e-10 relative per
simulation and for the force (plus the rounding floor of a cancelling sum); FP32 fields with
FP64 accumulation 2e-5 of the largest simulation per simulation and 1e-4 of the force itself
(plus the rounding floor of its FP64 sum)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
import workloads as W
from parity_bounds import assert_parity

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


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


def _compare(per, F, p, key, fp64):
    Fo, parts = _oracle(p, key)
    fa = p["force_axis"]
    assert_parity(per, F[fa], parts, Fo, p["n_steps"], fp64, str(key))


def small_grating(prec="fp64", **kw):
    """The silicon-waveguide grating over silicon/silica at resolution 16 (courant 0.2 keeps
    silicon's pole stable), 2 k_x x 2 k_z points (complex fields), 2 harmonics."""
    args = dict(resolution=16, nk_x=2, nk_z=2, n_harm=2, t_max=3.0, courant=0.2, pml_units=0.25, precision=prec)
    args.update(kw)
    return W.grating_silica(0.5, **args)


def poles_grating(prec="fp64", de=(2.0, 1.0, 3.0), w0=(3.0, 8.0, 20.0), **kw):
    """small_grating with the waveguide itself a three-pole medium whose poles lie among the
    field's frequencies, so that every pole carries weight in the force."""
    p = small_grating(prec, **kw)
    o = p["objects"][2]
    p["objects"][2] = {"shape": "box", "lo": o["lo"], "hi": o["hi"], "kind": "lorentz", "eps_inf": 1.5,
                       "delta_eps": list(de), "omega0": list(w0)}
    return p


def sphere_three_pole(prec="fp64"):
    """The 3D sphere over the notched substrate with a three-pole sphere (silica's strengths,
    frequencies scaled into the lattice's stable range at resolution 6)."""
    p = W.config4_sphere_notch(0.4, seed=3, resolution=6, n_cells=24, pml_cells=4, n_harm=1, n_steps=100,
                               precision=prec, substrate_top=1.0)
    sph = p["objects"][-1]
    p["objects"][-1] = {"shape": "sphere", "center": sph["center"], "radius": sph["radius"], "kind": "lorentz",
                        "eps_inf": 1.0, "delta_eps": [0.829, 0.095, 1.098], "omega0": [1.5, 2.5, 6.0]}
    return p


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("which", ["silicon_silica", "three_pole_waveguide"])
def test_grating_march(ctx, prec, which):
    p = small_grating(prec) if which == "silicon_silica" else poles_grating(prec)
    F, per, st = ctx.plan(p).run(per_sim=True)
    _compare(per, F, p, (which, prec), prec == "fp64")
    assert st["kernel_launches"] > 0


def test_every_pole_carries_weight(ctx):
    # the comparison is sensitive to each pole: dropping one moves every result well above the tolerance
    _, a, _ = ctx.plan(poles_grating()).run(per_sim=True)
    for de, w0 in (((2.0, 3.0), (3.0, 20.0)), ((2.0, 1.0), (3.0, 8.0))):
        _, b, _ = ctx.plan(poles_grating(de=de, w0=w0)).run(per_sim=True)
        assert np.max(np.abs(a - b)) > 1e-4 * np.max(np.abs(a))


def test_grating_tile_heights(ctx):
    p = poles_grating("fp64", t_max=2.0)
    res = [ctx.plan(p, options={"march_rows": r}).run(per_sim=True)[1] for r in (16, 32, 64)]
    for r in res[1:]:
        assert np.allclose(r, res[0], rtol=1e-10, atol=1e-14 * np.sum(np.abs(res[0])))


def test_grating_plain_path(ctx):
    p = poles_grating("fp64", t_max=2.0)
    _, pb, _ = ctx.plan(p).run(per_sim=True)
    _, pp, st = ctx.plan(p).run(per_sim=True, plain=True)
    assert np.allclose(pp, pb, rtol=1e-9, atol=1e-13 * np.sum(np.abs(pb)))
    assert st["kernel_launches"] > p["n_steps"]


def test_grating_silica_two_phase_kernel_in_subprocess():
    # with the march kernel switched off the two-dimensional runs take the one-thread-per-cell
    # two-phase kernel; compare it with the oracle in a fresh process
    code = r'''
import json, sys
import numpy as np
sys.path.insert(0, ".")
sys.path.insert(0, "tests")
from test_gpu_poles import poles_grating
import paper_0906_5170_gb300 as pk
p = poles_grating("fp64", t_max=2.0)
ctx = pk.Context(0)
F, per, st = ctx.plan(p).run(per_sim=True)
print(json.dumps({"per": per.tolist(), "F": list(F)}))
ctx.close()
'''
    env = dict(os.environ, CASIMIR_MARCH6="0")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert out.returncode == 0, out.stderr[-2000:]
    res = json.loads(out.stdout.strip().splitlines()[-1])
    p = poles_grating("fp64", t_max=2.0)
    _compare(np.array(res["per"]), res["F"], p, "poles_t2", True)


@pytest.mark.parametrize("kernel_3d", [3, 1, 2])
def test_sphere_three_pole_3d(ctx, kernel_3d):
    p = sphere_three_pole("fp64")
    F, per, _ = ctx.plan(p, options={"kernel_3d": kernel_3d}).run(per_sim=True)
    _compare(per, F, p, "sphere3p", True)


def test_sphere_three_pole_3d_fp32(ctx):
    p = sphere_three_pole("fp32")
    F, per, _ = ctx.plan(p).run(per_sim=True)
    _compare(per, F, p, "sphere3p32", False)


def bloch_slab_3d(prec="fp64"):
    """A 3D cell periodic in x and y with Bloch phases (complex fields), CPML along z, a
    three-pole slab under a dielectric block; force along z on the block."""
    import math
    p = W._base(3, (12, 10, 24), 8.0, 80)
    p["bc"] = ["periodic", "periodic", "pml"]
    p["pml_cells"] = [0, 0, 4]
    p["objects"] = [
        {"shape": "box", "lo": [-1, -1, 0.0], "hi": [3, 3, 1.0], "kind": "lorentz", "eps_inf": 1.2,
         "delta_eps": [0.8, 0.4, 1.1], "omega0": [2.0, 4.0, 7.0]},
        {"shape": "box", "lo": [0.5, 0.375, 1.5], "hi": [1.0, 0.875, 2.0], "kind": "dielectric", "eps": 3.0, "mu": 1.0},
    ]
    lo, hi = [0.375, 0.25, 1.375], [1.125, 1.0, 2.125]
    p["faces"] = W.box_faces(lo, hi, 3)
    p["n_harm"] = 1
    p["polarization"] = "full"
    p["k_points"] = [{"k": [2 * math.pi / 1.5 * 0.25, 2 * math.pi / 1.25 * 0.5, 0.0], "weight": 1.0}]
    p["force_axis"] = 2
    p["precision"] = prec
    return p


@pytest.mark.parametrize("kernel_3d", [3, 1, 2])
def test_bloch_three_pole_3d_complex(ctx, kernel_3d):
    p = bloch_slab_3d("fp64")
    F, per, _ = ctx.plan(p, options={"kernel_3d": kernel_3d}).run(per_sim=True)
    _compare(per, F, p, "bloch3d", True)
