"""End-to-end physics pins for the oracle (method of Sec. II, Eq. (1)).

P4  complete cosine basis == point-source basis (Sec. II: the result does not
    depend on the complete orthonormal basis chosen);
P5  sigma independence (Sec. II: the force converges to the same value for every sigma);
P6  parallel PEC plates: the two-dimensional (k_z = 0) Casimir pressure and, with
    the z-invariant kernel of Appendix A.2, the three-dimensional pressure
    (the text quotes pi^2/(240 d^4) for perfect-metal plates), after O(Delta^2)
    Richardson extrapolation; the analytic sums are evaluated here independently;
P7  a uniform dielectric filling scales the force by 1/sqrt(eps) (Minkowski eps weight);
P11 an empty closed contour carries no force (-> 0 as Delta^2);
P14 mirror symmetry: no lateral force; block A feels minus the force on block B.
"""
import math

import numpy as np
import pytest
from scipy.integrate import quad

import oracle
from workloads import plates_box_2d, piston_small, box_faces, _base

ZETA3 = 1.2020569031595942


def _massive_1d(a, k):
    """(1/pi) int_0^inf dxi q/(e^{2aq}-1), q = sqrt(xi^2 + k^2): one 1D mode's pressure magnitude."""
    if k == 0.0:
        return math.pi / (24 * a * a)
    f = lambda x: (lambda q: q * math.exp(-2 * a * q) / (-math.expm1(-2 * a * q)))(math.hypot(x, k))
    return quad(f, 0, np.inf, epsabs=1e-17, epsrel=1e-12, limit=200)[0] / math.pi


def pressure_2d(a, width, pol):
    """2D-world pressure between PEC plates a apart with PEC sidewalls `width` apart:
    TM = Dirichlet sidewall modes m >= 1, TE = Neumann m >= 0."""
    tot, m = 0.0, (1 if pol == "TM" else 0)
    while True:
        v = _massive_1d(a, m * math.pi / width)
        tot += v
        if m > 0 and v < 1e-18:
            break
        m += 1
    return -tot / width


def pressure_3d(a, width, pol):
    """Same plates in a z-invariant PEC tube: per sidewall mode, the (xi, k_z) integral
    in polar form gives (1/2pi) int_{k_m}^inf q^2/(e^{2aq}-1) dq."""
    tot, m = 0.0, (1 if pol == "TM" else 0)
    while True:
        k = m * math.pi / width
        if k == 0.0:
            v = 2 * ZETA3 / (2 * a) ** 3 / (2 * math.pi)
        else:
            v = quad(lambda q: q * q * math.exp(-2 * a * q) / (-math.expm1(-2 * a * q)), k, np.inf,
                     epsabs=1e-17, epsrel=1e-12, limit=200)[0] / (2 * math.pi)
        tot += v
        if m > 0 and v < 1e-18:
            break
        m += 1
    return -tot / width


def test_analytic_plate_sums_limits():
    # wide sidewalls recover the infinite-plate values the paper prints (tests/golden/paper_values.txt):
    # zeta(3)/(8 pi a^3) per polarisation in the two-dimensional world (the PFA normalisation of the
    # double-block figure) and pi^2/(240 a^4) for TE + TM in three dimensions
    from conftest import PAPER_VALUES as G
    assert G["pfa_2d_pressure"] == pytest.approx(ZETA3 / (8 * math.pi), rel=1e-15)
    assert G["plate_pressure_3d"] == pytest.approx(math.pi ** 2 / 240, rel=1e-15)
    for pol in ("TM", "TE"):
        assert pressure_2d(1.0, 400.0, pol) == pytest.approx(-G["pfa_2d_pressure"], rel=5e-3)
        assert pressure_3d(1.0, 400.0, pol) == pytest.approx(-G["plate_pressure_3d"] / 2, rel=5e-3)


def _upper_plate_force(res, pol, g_variant="plain", **kw):
    p = plates_box_2d(res, 1.0, lines=("inner", "outer"), polarization=pol, t_max=25.0, g_variant=g_variant, **kw)
    return oracle.force(p)


@pytest.mark.parametrize("pol", ["TM", "TE"])
def test_p6_plates_2d_pressure(pol):
    # upper plate (y = 1.5): cavity of 1 below, 0.5 above; closed contour through the PEC sidewalls
    exact = 1.0 * (pressure_2d(1.0, 1.0, pol) - pressure_2d(0.5, 1.0, pol))
    f16, f24, f32 = (_upper_plate_force(r, pol) for r in (16, 24, 32))
    # second-order convergence
    e16, e24, e32 = f16 - exact, f24 - exact, f32 - exact
    assert e24 / e32 == pytest.approx((32 / 24) ** 2, rel=0.08)
    ext = (32**2 * f32 - 24**2 * f24) / (32**2 - 24**2)
    assert ext == pytest.approx(exact, rel=2e-3)
    # sign: the plate is pulled toward the closer wall above it
    assert ext > 0


@pytest.mark.parametrize("pol", ["TM", "TE"])
def test_p6_plates_3d_pressure_zinv(pol):
    exact = 1.0 * (pressure_3d(1.0, 1.0, pol) - pressure_3d(0.5, 1.0, pol))
    f24, f32 = (_upper_plate_force(r, pol, "zinv") for r in (24, 32))
    ext = (32**2 * f32 - 24**2 * f24) / (32**2 - 24**2)
    assert ext == pytest.approx(exact, rel=1e-2)


def test_p7_uniform_dielectric_scales_force():
    f = {}
    for eps in (1.0, 2.0):
        a, b = (_upper_plate_force(r, "TE", fill_eps=eps) for r in (24, 32))
        f[eps] = (32**2 * b - 24**2 * a) / (32**2 - 24**2)
    assert f[2.0] / f[1.0] == pytest.approx(1 / math.sqrt(2), rel=3e-3)


def test_p5_sigma_independence():
    out = {}
    for c in (0.5, 0.25):
        out[c] = []
        for s in (0.5, 1.0, 2.0):
            p = plates_box_2d(16, 1.0, lines=("inner", "outer"), polarization="TM",
                              t_max=60.0 if s < 1 else 30.0, sigma=s, courant=c)
            out[c].append(oracle.force(p))
    spread = {c: np.ptp(v) / np.mean(v) for c, v in out.items()}
    # the dependence on sigma is a time-step error: it falls as Delta_t^2 ...
    assert spread[0.5] / spread[0.25] == pytest.approx(4.0, rel=0.3)
    # ... and the Delta_t -> 0 extrapolations agree across sigma
    ext = [(4 * b - a) / 3 for a, b in zip(out[0.5], out[0.25])]
    assert np.ptp(ext) / np.mean(ext) < 2e-5


def test_p4_cosine_basis_equals_point_basis():
    p = piston_small(n_steps=400, polarization="TE+TM")
    d = 1.0 / p["resolution"]
    counts = [int(round((f["hi"][1 - f["axis"]] - f["lo"][1 - f["axis"]]) / d)) for f in p["faces"]]
    p["n_harm"] = max(counts)               # complete on every face
    fc, parts_c, sims_c = oracle.force(p, return_parts=True)
    q = dict(p, basis="point")
    fp, parts_p, sims_p = oracle.force(q, return_parts=True)
    scale = sum(abs(x) for x in parts_c)
    assert abs(fc - fp) < 1e-12 * scale
    # face by face, source component by component
    for fi in range(4):
        for kind in ("J", "K"):
            a = math.fsum(x for x, s in zip(parts_c, sims_c) if s["face"] == fi and s["kind"] == kind)
            b = math.fsum(x for x, s in zip(parts_p, sims_p) if s["face"] == fi and s["kind"] == kind)
            assert abs(a - b) < 1e-12 * scale


def test_p11_empty_contour_carries_no_force():
    vals = {}
    for res in (8, 16):
        p = _base(2, (int(3 * res), int(2.5 * res), 1), float(res), int(30 / (0.5 / res)))
        p["faces"] = box_faces([0.75, 0.75], [1.75, 1.5], 2)
        p["n_harm"] = res
        p["polarization"] = "TE+TM"
        p["force_axis"] = 0
        vals[res] = oracle.force(p)
        blk = dict(p, objects=[{"shape": "box", "lo": [1.0, 1.0, 0], "hi": [1.5, 1.25, 0], "kind": "pec"}])
        vals[("blk", res)] = oracle.force(blk)
    assert vals[8] / vals[16] == pytest.approx(4.0, rel=0.1)
    assert abs(vals[16]) < 5e-3 * abs(vals[("blk", 16)])


def test_p14_mirror_symmetry():
    p = piston_small(n_steps=500)              # blocks symmetric about x = 3
    fb, parts, _ = oracle.force(p, return_parts=True)
    scale = sum(abs(x) for x in parts)
    d = 1.0 / p["resolution"]
    pa = dict(p, faces=box_faces([1.5 - d, 0.5 - d], [2.5 + d, 1.5 + d], 2))
    fa = oracle.force(pa)
    assert fb < 0 < fa                          # the blocks attract
    assert abs(fa + fb) < 1e-10 * scale
    # a single centred block: no lateral force at all
    pc = dict(p, objects=[{"shape": "box", "lo": [2.5, 0.5, 0], "hi": [3.5, 1.5, 0], "kind": "pec"}],
              faces=box_faces([2.5 - d, 0.5 - d], [3.5 + d, 1.5 + d], 2))
    f0, parts0, _ = oracle.force(pc, return_parts=True)
    assert abs(f0) < 1e-11 * sum(abs(x) for x in parts0)


def test_p13_harmonic_contributions_fall_as_n_to_the_minus_4():
    # Sec. III A: on a rectangular contour the fields, seen as functions along a face, have
    # nonzero slopes at the corners while every cosine has zero slope there, so their cosine
    # coefficients fall as n^-2 and each harmonic's force contribution as n^-4.  Contour 0.25
    # away from the right block of a 2D TM piston (away from the block's own edge fields), 45
    # pixels per face at resolution 30; contributions summed over faces and sources per n; the
    # log-log slope over n = 8..24 (below half the face's pixel count, where the lattice takes
    # over), for even and odd n separately (the mirror symmetry about the block's mid-plane
    # splits them) and together.
    res = 30
    p = piston_small(0.5, resolution=res, n_harm=1000, n_steps=int(20 / (0.5 / res)),
                     polarization="TM", precision="fp64")
    p["faces"] = box_faces([3.25, 0.25], [4.75, 1.75], 2)
    F, parts, sims = oracle.force(p, return_parts=True)
    c = {}
    for v, s in zip(parts, sims):
        c[s["harm"][0]] = c.get(s["harm"][0], 0.0) + v
    n = np.array(sorted(c))
    v = np.array([c[k] for k in n])
    assert len(n) == 45
    assert F < 0 and abs(v[0]) > 0.5 * abs(F)          # attraction; n = 0 carries most of it
    tail = (n >= 8) & (n <= 24)
    assert np.all(v[tail] > 0)                          # one sign over the fitted range
    for sel in (tail & (n % 2 == 0), tail & (n % 2 == 1), tail):
        slope = np.polyfit(np.log(n[sel]), np.log(v[sel]), 1)[0]
        assert -4.5 < slope < -3.5, slope
