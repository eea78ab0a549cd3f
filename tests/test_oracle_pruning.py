"""Pin of the oracle's simulation pruning (step a8 of the method, Sec. II, Eqs. (3)-(6)).

The oracle runs only the simulations whose source component can enter the stress
functional of a face: on a face with normal axis a, for force component i, every source
component when a == i and only c == a otherwise.  Here the oracle runs every simulation,
unpruned, on a closed two-dimensional contour (TE and TM) and on a closed three-dimensional
box, records every field component at the face pixels, and forms the force from the full
Maxwell stress tensor instead: with C_pq(t) the p component of the field radiated by a
q-directed harmonic source (projected on the same harmonic),

    F_i = sum_j n_j [C_ij - 1/2 delta_ij sum_k C_kk],

contracted with the face normal as a 3 x 3 matrix.  Every simulation the pruning drops
contributes exactly 0 to this sum, the kept ones equal the oracle's own per-simulation
contributions, and the total equals oracle.force.
"""
import itertools

import numpy as np
import pytest

import oracle
from oracle import casimir_oracle as co
import workloads as W


def _component_series(p, setup, sim, q):
    """G_q(n) = sum_k dA w_S f(x_k) F_q(x_k, t_n): the q component of the field of `sim`
    interpolated to the face pixels and projected on the sim's harmonic."""
    face = p["faces"][sim["face"]]
    _, _, centres, dA = co.face_pixels(p, face)
    f = co.harmonic(p, face, sim["harm"])
    magnetic = sim["kind"] == "K"
    offs = co.H_OFF if magnetic else co.E_OFF
    eps, mu, _, _, _, _ = co._materials(p, [centres[:, 0], centres[:, 1], centres[:, 2]])
    wS = mu if magnetic else eps
    meas = {}
    for k in range(centres.shape[0]):
        for idx, w in co.interp_weights(p, setup, centres[k], offs[q]):
            meas[(q, idx)] = meas.get((q, idx), 0.0) + dA * wS[k] * f[k] * w
    src, _ = co._sim_vectors(p, setup, sim)
    src = {(sim["comp"], idx): v for idx, v in src.items()}
    return co.run_vectors(p, setup, magnetic, src, meas, pol=sim["pol"])


def _stress_contribution(p, setup, sim, w):
    """sum_n w_n Re sum_j n_j T_ij(n) for the column of C that `sim` fills (source along c)."""
    i = p["force_axis"]
    face = p["faces"][sim["face"]]
    nvec = np.zeros(3)
    nvec[face["axis"]] = float(face["sign"])
    c = sim["comp"]
    T = p["n_steps"]
    C = np.zeros((T, 3, 3), dtype=np.complex128)
    for q in range(3):
        C[:, q, c] = _component_series(p, setup, sim, q)
    trace = np.einsum("tkk->t", C)
    stress = C - 0.5 * trace[:, None, None] * np.eye(3)[None]
    s = np.einsum("tj,j->t", stress[:, i, :], nvec)
    return float(np.sum(w * s.real)) * p["k_points"][sim["k"]]["weight"]


def _all_sims(p):
    sims = []
    for ki, _ in enumerate(p["k_points"]):
        for fi, face in enumerate(p["faces"]):
            for nvec in co.harmonic_list(p, face):
                for pol, kind, c in co._families(p):
                    sims.append({"k": ki, "face": fi, "harm": nvec, "pol": pol, "kind": kind, "comp": c})
    return sims


def _key(s):
    return (s["k"], s["face"], tuple(s["harm"]), s["pol"], s["kind"], s["comp"])


def _problems():
    two_d = W.piston_small(n_steps=120, n_harm=3, precision="fp64")            # closed 2D contour, TE + TM
    three_d = W.config4_sphere_notch(0.4, seed=3, resolution=6, n_cells=24, pml_cells=4, n_harm=1,
                                     n_steps=40, precision="fp64", substrate_top=1.0)   # closed 3D box
    tilted = dict(three_d, force_axis=0)                                         # a lateral component
    return [("2d", two_d), ("3d_z", three_d), ("3d_x", tilted)]


@pytest.mark.parametrize("name,p", _problems(), ids=lambda v: v if isinstance(v, str) else "")
def test_pruned_simulations_contribute_exactly_zero(name, p):
    w = oracle.g_weights(p)
    setups = [oracle.grid_setup(p, kp["k"]) for kp in p["k_points"]]
    kept = {_key(s) for s in oracle.enumerate_sims(p)}
    full = _all_sims(p)
    assert len(full) > len(kept)                    # the pruning does drop simulations here
    F, parts, sims = oracle.force(p, return_parts=True)
    by_key = dict(zip((_key(s) for s in sims), parts))
    total = []
    for s in full:
        c = _stress_contribution(p, setups[s["k"]], s, w)
        if _key(s) in kept:
            ref = by_key[_key(s)]
            assert abs(c - ref) <= 1e-12 * abs(ref) + 1e-15 * max(abs(x) for x in parts), (name, s, c, ref)
        else:
            assert c == 0.0, (name, s, c)
        total.append(c)
    scale = float(np.sum(np.abs(parts)))
    assert abs(sum(total) - F) <= 1e-12 * abs(F) + 1e-14 * scale
