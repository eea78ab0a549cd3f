"""Full-size parity: the configurations at their full grid sizes, run the way the
benchmark runs them (several plans in flight together, executed in waves), with
sampled simulations recomputed one by one by the FP64 oracle.

  * 2D piston sweep: 400 x 80 and 400 x 280 grids, 40 harmonics, TE + TM, 20000 steps;
  * waveguides: 256 x 256 with 1-unit CPML, Lorentz pole, 4 of the 32 k_z points, 3840 steps;
  * rotationally symmetric two-block piston: 60 x 400 (r, z), m, n in {0, 1, 2}, 10314 steps;
  * silicon/silica grating (one- and three-pole Lorentz media, complex fields): 40 x 160 at
    resolution 40, 4 k_x x 8 k_z, 8 harmonics, 3200 steps, the three gaps of the benchmark;
  * sphere over an indented substrate: 160^3 with 12-cell CPML, one harmonic per face,
    a shortened run of 100 steps (the oracle's cost per full-length 3D simulation is
    about ten minutes).
Tolerance: FP32 fields, per simulation 2e-5 of that simulation's magnitude scale."""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_0906_5170_gb300 import build
    build.build()
    import paper_0906_5170_gb300 as pk
    c = pk.Context(0)
    yield c
    c.close()


def _run_together(ctx, probs):
    plans = [ctx.plan(p) for p in probs]
    tickets = [pl.submit(tag=i) for i, pl in enumerate(plans)]
    out = [t.force(-1) for t in tickets]
    per = [pl.run(per_sim=True)[1] for pl in plans]     # the same plans once more, synchronously
    for (F, _, _), pp in zip(out, per):
        assert abs(F[0] + F[1] + F[2] - pp.sum()) <= 1e-9 * np.sum(np.abs(pp))
    return per


def _oracle_sims(p, picks):
    sims = oracle.enumerate_sims(p)
    w = oracle.g_weights(p)
    setup = oracle.grid_setup(p, p["k_points"][sims[picks[0]]["k"]]["k"]) if len(p["k_points"]) == 1 else None

    def one(i):
        s = sims[i]
        st = setup or oracle.grid_setup(p, p["k_points"][s["k"]]["k"])
        return float(np.sum(w * oracle.run_sim(p, s, st).real)) * p["k_points"][s["k"]]["weight"]
    with ThreadPoolExecutor(max_workers=len(picks)) as ex:
        return list(ex.map(one, picks))


def test_piston_sweep_full_size(ctx):
    hs = W.config2_heights()
    probs = [W.config2_piston(hs[0]), W.config2_piston(hs[-1])]
    per = _run_together(ctx, probs)
    for p, pp in zip(probs, per):
        n = len(pp)
        picks = [0, n // 3 + 1, n - 1]
        ref = _oracle_sims(p, picks)
        for i, r in zip(picks, ref):
            assert abs(pp[i] - r) <= 2e-5 * max(abs(r), 1e-3 * np.max(np.abs(pp))), (i, pp[i], r)


def test_waveguides_full_size(ctx):
    kp = W.config3_kz_points(0.5, medium=W.waveguide_material())
    p = W.config3_waveguides(0.5, k_points=[kp[i] for i in (0, 7, 15, 22)])
    per = _run_together(ctx, [p])[0]
    n = len(per)
    picks = [1, n // 2, n - 2]
    ref = _oracle_sims(p, picks)
    for i, r in zip(picks, ref):
        assert abs(per[i] - r) <= 2e-5 * max(abs(r), 1e-3 * np.max(np.abs(per))), (i, per[i], r)


def test_sphere_notch_full_grid(ctx):
    p = W.config4_sphere_notch(0.55, seed=1, n_harm=1, n_steps=100)
    per = _run_together(ctx, [p])[0]
    picks = [0, len(per) - 1]
    ref = _oracle_sims(p, picks)
    for i, r in zip(picks, ref):
        assert abs(per[i] - r) <= 2e-5 * max(abs(r), 1e-3 * np.max(np.abs(per))), (i, per[i], r)


def test_cylinder_blocks_full_size(ctx):
    # the rotationally symmetric two-block piston at its benchmark size: 60 x 400 (r, z) at
    # resolution 40, m, n in {0, 1, 2}, 10314 steps; one sampled simulation per m and the last one
    p = W.cylinder_blocks(1.0)
    per = _run_together(ctx, [p])[0]
    sims = oracle.enumerate_sims(p)
    w = oracle.g_weights(p)
    picks = sorted({next(i for i, s in enumerate(sims) if s["k"] == k) for k in range(len(p["k_points"]))} | {len(sims) - 1})

    def one(i):
        s = sims[i]
        return float(np.sum(w * oracle.run_sim(p, s).real)) * p["k_points"][s["k"]]["weight"]
    with ThreadPoolExecutor(max_workers=len(picks)) as ex:
        ref = list(ex.map(one, picks))
    for i, r in zip(picks, ref):
        assert abs(per[i] - r) <= 2e-5 * max(abs(r), 1e-3 * np.max(np.abs(per))), (i, per[i], r)


def test_grating_silica_full_size(ctx):
    # the three gaps the benchmark runs together; sampled simulations of different k-points,
    # sources and harmonics per gap
    probs = [W.grating_silica(g, nk_x=4) for g in (0.25, 0.5, 1.0)]
    per = _run_together(ctx, probs)
    for p, pp in zip(probs, per):
        n = len(pp)
        picks = [5, n // 2 + 7, n - 3]
        ref = _oracle_sims(p, picks)
        for i, r in zip(picks, ref):
            assert abs(pp[i] - r) <= 2e-5 * max(abs(r), 1e-3 * np.max(np.abs(pp))), (i, pp[i], r)
