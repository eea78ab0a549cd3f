"""Seeded, synthetic problem descriptions for the time-domain Casimir method.

This module only *describes* geometries (grid sizes, objects, boundary kinds,
stress contours, harmonic counts, k-points).  It holds none of the method's
arithmetic: no field update, no basis, no g(t), no rasterisation.  Both the
CPU oracle and the CUDA path consume the same plain dictionaries.

Problem dictionary (all lengths in units of the geometry's length scale a,
c = eps0 = mu0 = hbar = 1; the computational cell spans [0, n_a / resolution]
along each axis a):

    dims          2 or 3
    n             [nx, ny, nz] cells (nz == 1 when dims == 2)
    resolution    cells per unit length (Delta = 1 / resolution)
    courant       S_c, Delta_t = S_c * Delta
    n_steps       number of time steps T
    sigma         uniform conductivity of the complex-frequency contour
    background    {"eps": .., "mu": ..}
    objects       list of {"shape": "box"|"sphere", "lo","hi" | "center","radius",
                  "kind": "pec"|"pmc"|"dielectric"|"lorentz", "eps", "mu",
                  "eps_inf", "delta_eps", "omega0"}; later objects win.  A Lorentz
                  object's delta_eps / omega0 are numbers (one undamped pole) or
                  equal-length lists of up to three (a sum of poles)
    bc            per axis "pec" | "pml" | "periodic"
    pml_cells     per axis CPML thickness in cells (for "pml" axes)
    faces         stress-surface faces {"axis", "sign", "pos", "lo", "hi"}
    n_harm        cosine harmonics per tangential axis of every face
    polarization  "TM" | "TE" | "TE+TM" (two-dimensional, k_z = 0) or
                  "full" (all six source components)
    k_points      [{"k": [kx, ky, kz], "weight": w}]
    force_axis    0, 1 or 2
    g_variant     "plain" | "zinv"
    precision     "fp64" | "fp32"
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "box_faces", "plates_box_2d", "config1_plates", "config2_piston",
    "config2_heights", "config3_waveguides", "config3_gaps", "config3_kz_points",
    "config4_sphere_notch", "serving_requests", "piston_small",
    "silicon", "silica", "grating_silica", "cylinder_piston", "cylinder_blocks",
]


def box_faces(lo, hi, dims):
    """The closed axis-aligned contour around the box [lo, hi] as outward faces."""
    faces = []
    for a in range(dims):
        for sign, pos in ((-1, lo[a]), (+1, hi[a])):
            flo = list(lo) + [0.0] * (3 - len(lo))
            fhi = list(hi) + [0.0] * (3 - len(hi))
            flo[a] = fhi[a] = pos
            faces.append({"axis": a, "sign": sign, "pos": float(pos),
                          "lo": [float(v) for v in flo], "hi": [float(v) for v in fhi]})
    return faces


def grid_object(mask, lo, hi, **material):
    """An arbitrary shape as a voxel mask over the box [lo, hi]: mask[i, j] (2D) or mask[i, j, k]
    (3D), non-zero where the voxel belongs to the object; `material` as for any object
    (kind="pec", or kind="dielectric", eps=..., and so on)."""
    lo = [float(v) for v in lo] + [0.0] * (3 - len(lo))
    hi = [float(v) for v in hi] + [0.0] * (3 - len(hi))
    return dict(shape="grid", lo=lo, hi=hi, mask=np.asarray(mask, dtype=np.uint8), **material)


def _base(dims, n, resolution, n_steps, sigma=1.0, courant=0.5):
    return {
        "dims": dims, "n": list(n), "resolution": float(resolution),
        "courant": float(courant), "n_steps": int(n_steps), "sigma": float(sigma),
        "background": {"eps": 1.0, "mu": 1.0}, "objects": [],
        "bc": ["pec", "pec", "pec"], "pml_cells": [0, 0, 0], "faces": [],
        "n_harm": 1, "polarization": "TM",
        "k_points": [{"k": [0.0, 0.0, 0.0], "weight": 1.0}],
        "force_axis": 0, "g_variant": "plain", "precision": "fp64",
    }


def plates_box_2d(resolution, width, *, lines=("inner",), n_harm=None, polarization="TM",
                  n_steps=None, t_max=None, sigma=1.0, g_variant="plain",
                  courant=0.5, fill_eps=1.0):
    """Two thin PEC plates at y = 0.5 and y = 1.5 inside a width x 2 PEC box.

    The inner cavity (separation 1) and the upper outer cavity (separation 0.5)
    each get a wall-to-wall stress line through their middle (y = 1.0 and
    y = 1.75).  With both lines, oriented away from the upper plate, the
    contour is closed through the PEC sidewalls around that plate.
    """
    nx = int(round(width * resolution))
    ny = int(round(2 * resolution))
    if n_steps is None:
        t_max = 100.0 if t_max is None else t_max
        n_steps = int(round(t_max / (courant / resolution)))
    p = _base(2, (nx, ny, 1), resolution, n_steps, sigma=sigma, courant=courant)
    p["background"] = {"eps": float(fill_eps), "mu": 1.0}
    p["objects"] = [
        {"shape": "box", "lo": [0.0, 0.5, 0.0], "hi": [float(width), 0.5, 0.0], "kind": "pec"},
        {"shape": "box", "lo": [0.0, 1.5, 0.0], "hi": [float(width), 1.5, 0.0], "kind": "pec"},
    ]
    faces = []
    for which in lines:
        if which == "inner":        # below the upper plate: outward normal -y
            faces.append({"axis": 1, "sign": -1, "pos": 1.0, "lo": [0.0, 1.0, 0.0],
                          "hi": [float(width), 1.0, 0.0]})
        elif which == "inner_up":   # the same line with normal +y (open line)
            faces.append({"axis": 1, "sign": +1, "pos": 1.0, "lo": [0.0, 1.0, 0.0],
                          "hi": [float(width), 1.0, 0.0]})
        elif which == "outer":      # above the upper plate: outward normal +y
            faces.append({"axis": 1, "sign": +1, "pos": 1.75, "lo": [0.0, 1.75, 0.0],
                          "hi": [float(width), 1.75, 0.0]})
        else:
            raise ValueError(which)
    p["faces"] = faces
    p["n_harm"] = int(nx if n_harm is None else n_harm)
    p["polarization"] = polarization
    p["force_axis"] = 1
    p["g_variant"] = g_variant
    return p


def config1_plates():
    """2D k_z = 0 TM plates: 3 x 2 PEC box, plates at y = 0.5 and 1.5, resolution 20,
    open midway line y = 1 with cosine harmonics n = 0..7, Courant 0.5, 4000 steps, FP64."""
    p = plates_box_2d(20, 3.0, lines=("inner_up",), n_harm=8, polarization="TM", n_steps=4000)
    p["precision"] = "fp64"
    return p


def config2_heights():
    """Sidewall half-gaps h: 8 evenly spaced values in [0.5, 3], snapped to 1/40."""
    return [round(40.0 * (0.5 + j * 2.5 / 7.0)) / 40.0 for j in range(8)]


def config2_piston(h, *, resolution=40, n_harm=40, n_steps=20000, polarization="TE+TM",
                   precision="fp32", g_variant="zinv"):
    """Two 1 x 1 PEC blocks (gap 1 along x) between PEC sidewalls at y = +-(1/2 + h).

    Cell: x in [0, 10] (PEC ends at x = +-5 about the centre), y in [0, 1 + 2h].
    Stress contour: the rectangle one pixel outside the right block; force along x.
    """
    d = 1.0 / resolution
    nx = int(round(10 * resolution))
    ny = int(round((1 + 2 * h) * resolution))
    p = _base(2, (nx, ny, 1), resolution, n_steps)
    yc = 0.5 + h
    p["objects"] = [
        {"shape": "box", "lo": [3.5, yc - 0.5, 0.0], "hi": [4.5, yc + 0.5, 0.0], "kind": "pec"},
        {"shape": "box", "lo": [5.5, yc - 0.5, 0.0], "hi": [6.5, yc + 0.5, 0.0], "kind": "pec"},
    ]
    p["faces"] = box_faces([5.5 - d, yc - 0.5 - d], [6.5 + d, yc + 0.5 + d], 2)
    p["n_harm"] = n_harm
    p["polarization"] = polarization
    p["force_axis"] = 0
    p["g_variant"] = g_variant
    p["precision"] = precision
    return p


def piston_small(h=0.5, *, resolution=10, n_harm=6, n_steps=600, polarization="TE+TM",
                 precision="fp32", g_variant="zinv", block_offset=0.0):
    """A coarse version of the piston geometry (parity-test size)."""
    d = 1.0 / resolution
    nx = int(round(6 * resolution))
    ny = int(round((1 + 2 * h) * resolution))
    p = _base(2, (nx, ny, 1), resolution, n_steps)
    yc = 0.5 + h
    p["objects"] = [
        {"shape": "box", "lo": [1.5 + block_offset, yc - 0.5, 0.0], "hi": [2.5 + block_offset, yc + 0.5, 0.0], "kind": "pec"},
        {"shape": "box", "lo": [3.5, yc - 0.5, 0.0], "hi": [4.5, yc + 0.5, 0.0], "kind": "pec"},
    ]
    p["faces"] = box_faces([3.5 - d, yc - 0.5 - d], [4.5 + d, yc + 0.5 + d], 2)
    p["n_harm"] = n_harm
    p["polarization"] = polarization
    p["force_axis"] = 0
    p["g_variant"] = g_variant
    p["precision"] = precision
    return p


def config3_gaps():
    """Waveguide gaps 0.3 .. 1.0 in steps of 0.1, snapped to 1/16 (two cells at resolution 32)."""
    return [round(16.0 * (0.3 + 0.1 * j)) / 16.0 for j in range(8)]


def waveguide_material():
    """The waveguides' single undamped Lorentz pole (eps_inf 1, delta_eps 10.7, omega_0 3)."""
    return {"kind": "lorentz", "eps_inf": 1.0, "delta_eps": 10.7, "omega0": 3.0}


def config3_kz_points(gap, n=32, resolution=32, courant=0.5, medium=None):
    """n Gauss-Legendre nodes for the k_z integral on [0, K].

    K = min(12/gap, 0.8 k_max): the integrand decays like exp(-2 gap k_z), and k_max is
    the largest k_z the time step resolves, (dt/2)^2 (8/Delta^2 + k_max^2) = min(1, eps_X),
    where eps_X is the Lorentz `medium`'s permittivity at Omega^2 = 4/dt^2 (a lattice mode
    above it grows without bound) and 1 without one.
    The weight includes the Jacobian K/2 and the 1/pi of the k_z measure.
    """
    d = 1.0 / resolution
    dt = courant * d
    eps_x = 1.0
    if medium is not None and medium.get("kind") == "lorentz":
        des, ws = medium["delta_eps"], medium["omega0"]
        des, ws = ([des], [ws]) if np.isscalar(des) else (des, ws)
        eps_x = medium["eps_inf"] - sum(de * (w * dt) ** 2 / (4.0 - (w * dt) ** 2) for de, w in zip(des, ws))
    kmax = math.sqrt(max(0.0, (2.0 / dt) ** 2 * min(1.0, eps_x) - 8.0 / d**2))
    K = min(12.0 / gap, 0.8 * kmax)
    u, w = np.polynomial.legendre.leggauss(n)
    return [{"k": [0.0, 0.0, float(K * (1 + ui) / 2)], "weight": float(wi * K / 2 / math.pi)}
            for ui, wi in zip(u, w)]


def config3_waveguides(gap, *, resolution=32, n_cells=256, pml_units=1.0, n_harm=30,
                       n_steps=3840, k_points=None, precision="fp32"):
    """Two suspended single-Lorentz-pole waveguides (1 wide along x, 0.5 tall) in vacuum,
    CPML on all four sides; force along x on the right waveguide."""
    d = 1.0 / resolution
    L = n_cells * d
    p = _base(2, (n_cells, n_cells, 1), resolution, n_steps)
    xc, yc = L / 2, L / 2
    mat = waveguide_material()
    p["objects"] = [
        dict(shape="box", lo=[xc - gap / 2 - 1.0, yc - 0.25, 0.0], hi=[xc - gap / 2, yc + 0.25, 0.0], **mat),
        dict(shape="box", lo=[xc + gap / 2, yc - 0.25, 0.0], hi=[xc + gap / 2 + 1.0, yc + 0.25, 0.0], **mat),
    ]
    p["bc"] = ["pml", "pml", "pec"]
    pc = int(round(pml_units * resolution))
    p["pml_cells"] = [pc, pc, 0]
    p["faces"] = box_faces([xc + gap / 2 - d, yc - 0.25 - d], [xc + gap / 2 + 1.0 + d, yc + 0.25 + d], 2)
    p["n_harm"] = n_harm
    p["polarization"] = "full"
    p["k_points"] = (config3_kz_points(gap, resolution=resolution, medium=mat) if k_points is None
                     else k_points)
    p["force_axis"] = 0
    p["g_variant"] = "plain"
    p["precision"] = precision
    return p


def config4_sphere_notch(height, *, seed=0, resolution=40, n_cells=160, pml_cells=12,
                         n_harm=6, n_steps=3200, precision="fp32", substrate_top=1.0):
    """Dielectric sphere (r = 0.5, eps 2.1) above an indented PEC substrate in a fluid
    (eps 1.8): a flat PEC plane with a 1.0-wide, 0.5-deep square notch whose centre is
    offset laterally by a seeded dx in [0, 0.2]; cubic stress surface around the sphere,
    force along z."""
    rng = np.random.default_rng(seed)
    dx_off = float(rng.uniform(0.0, 0.2))
    d = 1.0 / resolution
    L = n_cells * d
    p = _base(3, (n_cells, n_cells, n_cells), resolution, n_steps)
    p["background"] = {"eps": 1.8, "mu": 1.0}
    cx = cy = L / 2
    zs = substrate_top
    r = 0.5
    cz = zs + height + r
    nx0 = cx + dx_off
    p["objects"] = [
        {"shape": "box", "lo": [0.0, 0.0, 0.0], "hi": [L, L, zs], "kind": "pec"},
        {"shape": "box", "lo": [nx0 - 0.5, cy - 0.5, zs - 0.5], "hi": [nx0 + 0.5, cy + 0.5, zs + 1e-9],
         "kind": "dielectric", "eps": 1.8, "mu": 1.0},
        {"shape": "sphere", "center": [cx, cy, cz], "radius": r, "kind": "dielectric", "eps": 2.1, "mu": 1.0},
    ]
    p["bc"] = ["pml", "pml", "pml"]
    p["pml_cells"] = [pml_cells] * 3
    h = r + 2 * d
    lo = [round((cx - h) * resolution) * d, round((cy - h) * resolution) * d, round((cz - h) * resolution) * d]
    hi = [lo[0] + 2 * h, lo[1] + 2 * h, lo[2] + 2 * h]
    p["faces"] = box_faces(lo, hi, 3)
    p["n_harm"] = n_harm
    p["polarization"] = "full"
    p["force_axis"] = 2
    p["g_variant"] = "plain"
    p["precision"] = precision
    p["meta"] = {"dx": dx_off}
    return p


def serving_requests(seed, n_requests=200, rate=50.0, *, scale=1.0):
    """Poisson arrivals (mean `rate` per second) of force requests drawn from `seed`.

    Mix: 60% 2D piston / waveguide grids (side 64..512, 10..60 harmonics), 30% periodic
    grooved-membrane cells 128 x 512 with 16 Bloch k_x points, 10% 3D sphere-substrate
    grids (side 64..128).  `scale` < 1 shrinks every grid side (for tests).
    Returns a list of (arrival_time_s, problem_dict).
    """
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for _ in range(n_requests):
        t += float(rng.exponential(1.0 / rate))
        u = float(rng.uniform())
        if u < 0.6:
            side = int(rng.integers(64, 513))
            side = max(16, int(round(side * scale)) // 4 * 4)
            nh = int(rng.integers(10, 61))
            if rng.uniform() < 0.5:
                prob = _serving_piston(side, nh, rng)
            else:
                prob = _serving_waveguide(side, nh, rng)
        elif u < 0.9:
            prob = _serving_grating(scale, rng)
        else:
            side = int(rng.integers(64, 129))
            side = max(16, int(round(side * scale)) // 4 * 4)
            prob = _serving_sphere(side, rng)
        out.append((t, prob))
    return out


def _serving_piston(side, n_harm, rng):
    res = side / 8.0
    d = 1.0 / res
    p = _base(2, (side, side, 1), res, int(round(40.0 / (0.5 * d))))
    h = float(rng.uniform(0.5, 2.5))
    yc = 4.0
    p["objects"] = [
        {"shape": "box", "lo": [0.0, yc - 0.5 - h, 0.0], "hi": [8.0, yc - 0.5 - h, 0.0], "kind": "pec"},
        {"shape": "box", "lo": [0.0, yc + 0.5 + h, 0.0], "hi": [8.0, yc + 0.5 + h, 0.0], "kind": "pec"},
        {"shape": "box", "lo": [2.5, yc - 0.5, 0.0], "hi": [3.5, yc + 0.5, 0.0], "kind": "pec"},
        {"shape": "box", "lo": [4.5, yc - 0.5, 0.0], "hi": [5.5, yc + 0.5, 0.0], "kind": "pec"},
    ]
    lo = [round((4.5) * res - 1) * d, round((yc - 0.5) * res - 1) * d]
    hi = [round((5.5) * res + 1) * d, round((yc + 0.5) * res + 1) * d]
    p["faces"] = box_faces(lo, hi, 2)
    nmax = int(round((hi[1] - lo[1]) * res))
    p["n_harm"] = int(min(n_harm, nmax))
    p["polarization"] = "TE+TM"
    p["force_axis"] = 0
    p["g_variant"] = "zinv"
    p["precision"] = "fp32"
    p["kind"] = "piston"
    return p


def _serving_waveguide(side, n_harm, rng):
    """Two Lorentz waveguides in a CPML-terminated cell of 8 units, 4 k_z points
    (side rounded to a multiple of 16 so that the guides fall on whole cells)."""
    side = max(32, side // 16 * 16)
    res = side / 8.0
    gap = float(rng.uniform(0.3, 1.0))
    kp = config3_kz_points(gap, n=4, resolution=res, medium=waveguide_material())
    p = config3_waveguides(round(gap * res / 2) * 2 / res, resolution=res, n_cells=side, pml_units=1.0,
                           n_harm=int(min(n_harm, 12)), n_steps=int(round(30.0 / (0.5 / res))), k_points=kp)
    p["kind"] = "waveguide"
    return p


def _serving_grating(scale, rng):
    nx = max(16, int(round(128 * scale)) // 4 * 4)
    ny = max(32, int(round(512 * scale)) // 4 * 4)
    res = nx / 1.0                     # period 1 along x
    d = 1.0 / res
    Ly = ny * d
    p = _base(2, (nx, ny, 1), res, int(round(30.0 / (0.5 * d))))
    pc = max(4, ny // 16)
    p["bc"] = ["periodic", "pml", "pec"]
    p["pml_cells"] = [0, pc, 0]
    gap = float(rng.uniform(0.3, 1.0))
    yb = Ly / 2 - gap / 2
    # membrane below the gap with grooves of depth 0.5 and period 1 (half-period teeth)
    p["objects"] = [
        {"shape": "box", "lo": [0.0, yb - 1.0, 0.0], "hi": [1.0, yb - 0.5, 0.0], "kind": "dielectric", "eps": 11.7, "mu": 1.0},
        {"shape": "box", "lo": [0.25, yb - 0.5, 0.0], "hi": [0.75, yb, 0.0], "kind": "dielectric", "eps": 11.7, "mu": 1.0},
        {"shape": "box", "lo": [0.0, Ly / 2 + gap / 2, 0.0], "hi": [1.0, Ly / 2 + gap / 2 + 0.5, 0.0], "kind": "dielectric", "eps": 11.7, "mu": 1.0},
    ]
    ytop = round((Ly / 2 + gap / 2 + 0.5) * res + 1) * d
    ybot = round((Ly / 2 + gap / 2) * res - 1) * d
    p["faces"] = [
        {"axis": 1, "sign": -1, "pos": ybot, "lo": [0.0, ybot, 0.0], "hi": [1.0, ybot, 0.0]},
        {"axis": 1, "sign": +1, "pos": ytop, "lo": [0.0, ytop, 0.0], "hi": [1.0, ytop, 0.0]},
    ]
    p["n_harm"] = int(min(8, nx))
    p["polarization"] = "full"
    nk = 16
    p["k_points"] = [{"k": [2 * math.pi * m / nk, 0.0, 0.0], "weight": 1.0 / nk} for m in range(nk)]
    p["force_axis"] = 1
    p["g_variant"] = "plain"
    p["precision"] = "fp32"
    p["kind"] = "grating"
    return p


def _serving_sphere(side, rng):
    res = side / 4.0
    p = config4_sphere_notch(float(rng.uniform(0.3, 0.8)), seed=int(rng.integers(0, 2**31)),
                             resolution=res, n_cells=side, pml_cells=max(4, int(round(0.3 * res))),
                             n_harm=2, n_steps=int(round(30.0 / (0.5 / res))))
    p["kind"] = "sphere"
    return p


def cylinder_piston(resolution, m_list, *, radius=0.5, thickness=0.1, below=0.5, above=1.0, t_max=25.0,
                    n_harm=1000, sigma=1.0, precision="fp64", basis="cosine", courant=None):
    """Rotationally symmetric piston (Sec. III C): a PEC disk of the given thickness inside a PEC
    tube of radius `radius` closed by PEC end caps, `below` above the lower cap and `above` below
    the upper one; the (r, z) cross-section with fields ~ exp(i m phi), one k-point per m with
    weight 1 for m = 0 and 2 for m > 0 (the +m and -m terms).  The closed contour is two disks
    through the tube wall, one in the middle of each cavity; force along z.  The Courant number
    defaults to 0.95 of the leapfrog limit of the largest m (the i m / r terms next to the axis)."""
    d = 1.0 / resolution
    m_max = max(abs(int(m)) for m in m_list)
    if courant is None:
        courant = 0.95 * 2.0 / math.sqrt(max(9.0, 8.0 + 4.0 * m_max * m_max))
    L = below + thickness + above
    nr, nz = int(round(radius * resolution)), int(round(L * resolution))
    p = _base(2, (nr, nz, 1), resolution, int(round(t_max / (courant * d))), sigma=sigma, courant=courant)
    p["coords"] = "cylindrical"
    p["bc"] = ["pec", "pec", "pec"]
    p["polarization"] = "full"
    p["objects"] = [{"shape": "box", "lo": [0.0, below, 0.0], "hi": [radius, below + thickness, 0.0], "kind": "pec"}]
    z1 = round(0.5 * below * resolution) * d
    z2 = round((below + thickness + 0.5 * above) * resolution) * d
    p["faces"] = [{"axis": 1, "sign": -1, "pos": z1, "lo": [0.0, z1, 0.0], "hi": [radius, z1, 0.0]},
                  {"axis": 1, "sign": 1, "pos": z2, "lo": [0.0, z2, 0.0], "hi": [radius, z2, 0.0]}]
    p["n_harm"] = n_harm
    p["basis"] = basis
    p["force_axis"] = 1
    p["k_points"] = [{"k": [0.0, 0.0, 0.0], "m": int(m), "weight": 1.0 if int(m) == 0 else 2.0} for m in m_list]
    p["precision"] = precision
    p["kind"] = "cylinder"
    return p


def cylinder_blocks(h, *, resolution=40, m_list=(0, 1, 2), n_harm=3, t_max=100.0, sidewall="pec",
                    precision="fp32", sigma=1.0):
    """The piston of the two-block configuration rotated about its axis (Sec. III C): two PEC disks
    of radius 1/2 and thickness 1, gap 1 along z, inside a tube of radius 1/2 + h (PEC, or PMC
    with `sidewall="pmc"`: a one-cell PMC lining inside the PEC wall), PEC end caps 10 apart.
    Contour: the surface of revolution one pixel outside the upper disk (two disks and a
    cylinder); force along z, summed over m in m_list (weight 1 for m = 0, 2 otherwise) with
    n_harm cosine harmonics per face."""
    d = 1.0 / resolution
    R = 0.5 + h
    m_max = max(m_list)
    courant = 0.95 * 2.0 / math.sqrt(max(9.0, 8.0 + 4.0 * m_max * m_max))
    nr, nz = int(round(R * resolution)), int(round(10 * resolution))
    p = _base(2, (nr, nz, 1), resolution, int(round(t_max / (courant * d))), sigma=sigma, courant=courant)
    p["coords"] = "cylindrical"
    p["bc"] = ["pec", "pec", "pec"]
    p["polarization"] = "full"
    p["objects"] = [
        {"shape": "box", "lo": [0.0, 3.5, 0.0], "hi": [0.5, 4.5, 0.0], "kind": "pec"},
        {"shape": "box", "lo": [0.0, 5.5, 0.0], "hi": [0.5, 6.5, 0.0], "kind": "pec"},
    ]
    if sidewall == "pmc":
        p["objects"].append({"shape": "box", "lo": [R - d, 0.0, 0.0], "hi": [R, 10.0, 0.0], "kind": "pmc"})
    z0, z1, r1 = 5.5 - d, 6.5 + d, 0.5 + d
    p["faces"] = [{"axis": 1, "sign": -1, "pos": z0, "lo": [0.0, z0, 0.0], "hi": [r1, z0, 0.0]},
                  {"axis": 1, "sign": 1, "pos": z1, "lo": [0.0, z1, 0.0], "hi": [r1, z1, 0.0]},
                  {"axis": 0, "sign": 1, "pos": r1, "lo": [r1, z0, 0.0], "hi": [r1, z1, 0.0]}]
    p["n_harm"] = n_harm
    p["force_axis"] = 1
    p["k_points"] = [{"k": [0.0, 0.0, 0.0], "m": int(m), "weight": 1.0 if int(m) == 0 else 2.0} for m in m_list]
    p["precision"] = precision
    p["kind"] = "cylinder"
    return p


# ---------------------------------------------------------------------------
# Dispersive materials of Sec. III D in units of a = 1 um: omega [rad/s] * a / c
# ---------------------------------------------------------------------------

C_UM_PER_S = 2.99792458e14      # the speed of light in um / s


def silicon():
    """Silicon, one undamped pole: eps(0) = 11.87, eps(inf) = 1.035, omega_0 = 6.6e15 rad/s
    (the printed formula's leading term read as eps(inf), so that eps(0) is silicon's 11.87)."""
    return {"kind": "lorentz", "eps_inf": 1.035, "delta_eps": 11.87 - 1.035, "omega0": 6.6e15 / C_UM_PER_S}


def silica():
    """Silica, three undamped poles: eps = 1 + sum_j C_j w_j^2 / (w_j^2 - w^2),
    C = (0.829, 0.095, 1.098), w = (0.867, 1.508, 203.4) x 1e14 rad/s."""
    return {"kind": "lorentz", "eps_inf": 1.0, "delta_eps": [0.829, 0.095, 1.098],
            "omega0": [w * 1e14 / C_UM_PER_S for w in (0.867, 1.508, 203.4)]}


def grating_silica(gap, *, resolution=40, nk_x=8, nk_z=8, n_harm=8, t_max=40.0, courant=0.5,
                   kz_max=None, pml_units=0.5, precision="fp32"):
    """A periodic array of silicon waveguides (period 1 along x, 0.5 wide, 0.5 tall, invariant
    along z) a distance `gap` above a substrate of a 0.25 silicon film on 1.0 of silica, CPML
    above and below (Sec. III D).  Force along y on one waveguide per unit length: the
    Brillouin-zone average over nk_x Bloch k_x in [0, pi] (the +-k_x pairs folded) times
    (1/pi) int_0^K dk_z by nk_z-point Gauss-Legendre, K = min(12/gap, kz_max); the stress
    surface is two full-period lines one pixel below and above the waveguide."""
    d = 1.0 / resolution
    nx = int(round(resolution))
    pc = int(round(pml_units * resolution))
    y_silica = pc * d
    y_film = y_silica + round(1.0 * resolution) * d
    y_top = y_film + round(0.25 * resolution) * d          # substrate surface
    y_wg = y_top + round(gap * resolution) * d               # waveguide bottom
    y_wg_top = y_wg + round(0.5 * resolution) * d
    ny = int(round((y_wg_top + 0.75) * resolution)) + pc
    dt = courant * d
    n_steps = int(round(t_max / dt))
    p = _base(2, (nx, ny, 1), resolution, n_steps, courant=courant)
    p["bc"] = ["periodic", "pml", "pec"]
    p["pml_cells"] = [0, pc, 0]
    p["objects"] = [
        dict(shape="box", lo=[-1.0, -1.0, 0.0], hi=[2.0, y_film, 0.0], **silica()),
        dict(shape="box", lo=[-1.0, y_film, 0.0], hi=[2.0, y_top, 0.0], **silicon()),
        dict(shape="box", lo=[0.25, y_wg, 0.0], hi=[0.75, y_wg_top, 0.0], **silicon()),
    ]
    ylo, yhi = y_wg - d, y_wg_top + d
    p["faces"] = [
        {"axis": 1, "sign": -1, "pos": ylo, "lo": [0.0, ylo, 0.0], "hi": [1.0, ylo, 0.0]},
        {"axis": 1, "sign": +1, "pos": yhi, "lo": [0.0, yhi, 0.0], "hi": [1.0, yhi, 0.0]},
    ]
    p["n_harm"] = int(min(n_harm, nx))
    p["polarization"] = "full"
    # k_x: midpoints of [0, pi] (each stands for +-k_x); k_z: Gauss-Legendre on [0, K]
    K = 12.0 / gap if kz_max is None else min(12.0 / gap, kz_max)
    u, w = np.polynomial.legendre.leggauss(nk_z)
    kxs = [math.pi * (i + 0.5) / nk_x for i in range(nk_x)]
    p["k_points"] = [{"k": [kx, 0.0, float(K * (1 + ui) / 2)], "weight": float(wi * K / 2 / math.pi / nk_x)}
                     for kx in kxs for ui, wi in zip(u, w)]
    p["force_axis"] = 1
    p["g_variant"] = "plain"
    p["precision"] = precision
    return p
