"""Pins for voxel-mask objects (arbitrary geometry given as a grid of filled voxels).

A mask is the union of its closed filled voxels, so a mask whose voxels tile a box is that
box, and a mask of two boxes is their union: the oracle's forces agree bit for bit with the
box objects', at several voxel sizes and with empty padding voxels, in 2D and 3D.  The
C ABI's planner takes the same masks (its rasterisation is parity-checked on the GPU) and
rejects malformed ones.
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


def _box_mask(box, vox, pad, dims):
    n = [int(round((box["hi"][a] - box["lo"][a]) / vox)) + 2 * pad for a in range(dims)]
    m = np.zeros(n, np.uint8)
    m[tuple(slice(pad, k - pad) for k in n)] = 1
    lo = [box["lo"][a] - pad * vox for a in range(dims)]
    hi = [box["hi"][a] + pad * vox for a in range(dims)]
    return W.grid_object(m, lo, hi, kind=box["kind"], **{k: box[k] for k in ("eps", "mu") if k in box})


@pytest.mark.parametrize("vox,pad", [(0.1, 0), (0.2, 0), (0.1, 3), (0.05, 2)])
def test_mask_of_a_box_is_the_box(vox, pad):
    p = W.piston_small(n_steps=300, precision="fp64")
    q = dict(p, objects=[p["objects"][0], _box_mask(p["objects"][1], vox, pad, 2)])
    F0 = oracle.force(p)
    assert abs(F0) > 1e-3
    assert oracle.force(q) == F0


def test_mask_of_two_boxes_is_their_union():
    # an L-shaped PEC block: as two boxes and as one 10 x 10 mask
    p = W.piston_small(n_steps=300, precision="fp64")
    mat = {"kind": "pec"}
    two = dict(p, objects=[p["objects"][0],
                           dict(shape="box", lo=[3.5, 0.5, 0.0], hi=[4.5, 1.0, 0.0], **mat),
                           dict(shape="box", lo=[3.5, 1.0, 0.0], hi=[4.0, 1.5, 0.0], **mat)])
    m = np.zeros((10, 10), np.uint8)
    m[:, :5] = 1
    m[:5, 5:] = 1
    one = dict(p, objects=[p["objects"][0], W.grid_object(m, [3.5, 0.5], [4.5, 1.5], **mat)])
    F = oracle.force(two)
    assert abs(F) > 1e-4
    assert oracle.force(one) == F
    # the L mirrored along x (its notch now faces the other block) is a different body; mirrored
    # along y it is the same body up to the geometry's own mirror symmetry, so the same force
    mx = dict(one, objects=[p["objects"][0], W.grid_object(m[::-1, :], [3.5, 0.5], [4.5, 1.5], **mat)])
    my = dict(one, objects=[p["objects"][0], W.grid_object(m[:, ::-1], [3.5, 0.5], [4.5, 1.5], **mat)])
    assert oracle.force(my) == pytest.approx(F, rel=1e-12)
    assert abs(oracle.force(mx) / F - 1) > 1e-3


def test_mask_of_a_box_is_the_box_3d():
    # the substrate of the sphere-over-notch geometry as a 3D mask of 0.1-wide voxels
    p = W.config4_sphere_notch(0.55, n_cells=32, pml_cells=6, resolution=20)
    p["n_harm"], p["n_steps"], p["precision"] = 1, 60, "fp64"
    sub = p["objects"][0]
    q = dict(p, objects=[_box_mask(sub, 0.1, 1, 3)] + p["objects"][1:])
    sims = oracle.enumerate_sims(p)[:6]
    assert oracle.force(q, sims=sims) == oracle.force(p, sims=sims)


def test_planner_takes_masks_and_rejects_malformed_ones():
    p = W.piston_small(n_steps=300, precision="fp64")
    q = dict(p, objects=[p["objects"][0], _box_mask(p["objects"][1], 0.1, 2, 2)])
    assert pk.Plan(q).info() == pk.Plan(p).info()
    bad_3d = _box_mask(p["objects"][1], 0.1, 0, 2)
    bad_3d["mask"] = np.ones((10, 10, 2), np.uint8)            # two z layers in a 2D problem
    flat = _box_mask(p["objects"][1], 0.1, 0, 2)
    flat["hi"] = [flat["lo"][0], flat["hi"][1], 0.0]             # zero extent along x
    for obj in (bad_3d, flat):
        with pytest.raises(pk.CasimirError) as e:
            pk.Plan(dict(p, objects=[p["objects"][0], obj]))
        assert e.value.code == -1
