"""FP64 CPU oracle for the time-domain Casimir method (arXiv:0906.5170).

TEST INFRASTRUCTURE ONLY -- see the package docstring.  Nothing here is used
by the product path.

The method, in the order the paper gives it (Sec. II and Sec. III):
  1. define the geometry and the stress surface S (Sec. II; Fig. 2);
  2. choose a harmonic basis {f_n} on S: a cosine series on each face of a
     rectangular S (Sec. III, Eq. (7));
  3. for every harmonic n and source direction, run an FDTD simulation with
     the current J = delta(t) f_n on S in a medium of uniform conductivity
     sigma (Sec. II) and record the surface functional Gamma_{ij;n}(t);
  4. integrate against Im g(-t) (Eq. (1); Appendix A) and sum over n, source
     directions, polarisations and k-points (Sec. III B, III D).

Readings where the paper is silent or ambiguous (each listed with its reason
in the design notes of the repository):
  * f_0 = sqrt(1/L) (orthonormal DCT-II on pixel centres (k+1/2) Delta);
  * sources are spread onto the Yee sites by the adjoint of the (bi/tri)linear
    interpolation used for measurement ("suitably averaged currents", Sec. III A);
  * sigma sits on D for electric (J) sources, on B for magnetic (K) sources;
  * the impulse sets the flux at t = 0+; the leapfrog starts with a half step
    so that sample n is the response at t_n = n Delta_t; rectangle rule n >= 1;
  * the Minkowski stress carries eps (mu) at the surface;
  * prefactor: F_i = 2 * Im int_0^inf dt g(-t) [Gamma^E_i + Gamma^H_i] with the
    paper's g(-t) = (1/2pi) int_0^inf g(xi) e^{i xi t} d xi;
  * z-invariant PEC/vacuum variant: g_zinv(xi) = (-i omega(xi)/2) g(xi), i.e. half
    of the printed closed form of Appendix A.2 (the factor i omega/2 the text
    states); pinned by the three-dimensional plate pressure.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBS = {}
_LIB_LOCK = threading.Lock()

# ---------------------------------------------------------------------------
# C core
# ---------------------------------------------------------------------------

DP = ctypes.POINTER(ctypes.c_double)
IP = ctypes.POINTER(ctypes.c_int)
MAX_POLES = 3      # undamped Lorentz poles per material (the silica model of Sec. III D has three)


class _OgGrid(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int * 3), ("twod", ctypes.c_int),
        ("eact", ctypes.c_int * 3), ("hact", ctypes.c_int * 3), ("kz", ctypes.c_double),
        ("dx", ctypes.c_double), ("dt", ctypes.c_double), ("sigma", ctypes.c_double),
        ("bloch_re", ctypes.c_double * 3), ("bloch_im", ctypes.c_double * 3),
        ("ce", DP * 3), ("ch", DP * 3), ("npole", ctypes.c_int),
        ("lde", (DP * 3) * MAX_POLES), ("lw0", (DP * 3) * MAX_POLES),
        ("pb", (DP * 2) * 3), ("pc", (DP * 2) * 3), ("pk", (DP * 2) * 3),
        ("cyl", ctypes.c_int), ("mphi", ctypes.c_double),
    ]


class _OgSim(ctypes.Structure):
    _fields_ = [
        ("magnetic", ctypes.c_int), ("nsteps", ctypes.c_int), ("nsrc", ctypes.c_int),
        ("src_comp", IP), ("src_idx", IP), ("src_re", DP), ("src_im", DP),
        ("nset", ctypes.c_int), ("set_ptr", IP), ("m_comp", IP), ("m_idx", IP),
        ("m_re", DP), ("m_im", DP),
    ]


def build_library(force_rebuild: bool = False, real: bool = False) -> str:
    """Compile yee_oracle.c with the system C compiler (plain gcc, no GPU).
    real=True builds the real-field variant (same source, -DORACLE_REAL)."""
    src = os.path.join(_HERE, "yee_oracle.c")
    outdir = os.path.join(_HERE, "_build")
    out = os.path.join(outdir, "liboracle_real.so" if real else "liboracle.so")
    if force_rebuild or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        os.makedirs(outdir, exist_ok=True)
        tmp = out + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O3", "-std=c99", "-fcx-limited-range", "-fPIC", "-shared", "-o", tmp, src, "-lm"]
        if real:
            cmd.insert(1, "-DORACLE_REAL")
        subprocess.check_call(cmd)
        os.replace(tmp, out)
    return out


def build_all(force_rebuild: bool = False):
    return [build_library(force_rebuild, False), build_library(force_rebuild, True)]


def _lib(real=False):
    with _LIB_LOCK:
        if real not in _LIBS:
            lib = ctypes.CDLL(build_library(real=real))
            lib.oracle_run.argtypes = [ctypes.POINTER(_OgGrid), ctypes.POINTER(_OgSim), DP, DP]
            lib.oracle_run.restype = ctypes.c_int
            lib.oracle_evolve.argtypes = [ctypes.POINTER(_OgGrid), ctypes.c_int, DP, DP, DP, DP, DP, DP]
            lib.oracle_evolve.restype = ctypes.c_int
            _LIBS[real] = lib
    return _LIBS[real]


def _dp(a):
    return a.ctypes.data_as(DP)


def _ip(a):
    return a.ctypes.data_as(IP)


# ---------------------------------------------------------------------------
# Appendix A: Im g(-t)
# ---------------------------------------------------------------------------

ZINV_FACTOR = 0.5   # g_zinv(xi) = (-i omega(xi) / 2) g(xi): text of Appendix A.2


def img_minus_t(t, sigma, variant="plain"):
    """Im g(-t) for t > 0 (Appendix A).

    plain: g(xi) = -i xi (1 + i sigma/xi)(1 + i sigma/2xi) / sqrt(1 + i sigma/xi)
    (Appendix A, first equation) transformed with g(-t) = (1/2pi) int_0^inf
    g(xi) e^{i xi t} d xi.  Rotating the integration path onto xi = i eta
    (the branch points 0 and -i sigma lie off the upper half plane) gives
        Im g(-t) = (1/2pi) int_0^inf sqrt(1 + sigma/eta) (eta + sigma/2) e^{-eta t} d eta,
    and eta = sigma u^2 gives (sigma^2/pi) int_0^inf e^{-sigma t u^2} sqrt(1+u^2) (u^2 + 1/2) du,
    evaluated here with u = sinh(w) by the trapezoid rule in w (double-exponential decay).
    For sigma = 0 it is 1/(2 pi t^2), the transform of g_1 (Appendix A, Eq. for g_1(-t)).

    zinv: the z-invariant PEC/vacuum variant (Appendix A.2): ZINV_FACTOR times
    (1/2pi)(2/t^3 + 3 sigma/(2 t^2) + sigma^2/(2 t)).
    """
    t = np.asarray(t, dtype=np.float64)
    if variant == "zinv":
        return ZINV_FACTOR * (2.0 / t**3 + 1.5 * sigma / t**2 + 0.5 * sigma**2 / t) / (2.0 * math.pi)
    if variant != "plain":
        raise ValueError(variant)
    if sigma == 0.0:
        return 1.0 / (2.0 * math.pi * t**2)
    s = sigma * t
    out = np.empty_like(t)
    for idx, sv in np.ndenumerate(s):
        # the integrand's width in w shrinks like 1/sqrt(sigma t): keep >= 5 nodes across it
        h = min(1.0 / 64.0, 0.2 / math.sqrt(sv))
        wmax = math.asinh(math.sqrt(45.0 / sv)) + 0.5
        w = np.arange(0.0, wmax + h, h)
        u = np.sinh(w)
        c = np.cosh(w)
        f = np.exp(-sv * u * u) * c * c * (u * u + 0.5)
        val = h * (np.sum(f) - 0.5 * f[0])
        out[idx] = sigma**2 / math.pi * val
    return out


def g_weights(problem):
    """w_n = 2 Delta_t Im g(-n Delta_t), n = 1..T (Eq. (1), rectangle rule)."""
    dt = problem["courant"] / problem["resolution"]
    T = problem["n_steps"]
    t = dt * np.arange(1, T + 1, dtype=np.float64)
    return 2.0 * dt * img_minus_t(t, problem["sigma"], problem.get("g_variant", "plain"))


# ---------------------------------------------------------------------------
# Geometry on the Yee lattice
# ---------------------------------------------------------------------------

E_OFF = ((0.5, 0.0, 0.0), (0.0, 0.5, 0.0), (0.0, 0.0, 0.5))
H_OFF = ((0.0, 0.5, 0.5), (0.5, 0.0, 0.5), (0.5, 0.5, 0.0))
_TOL = 1e-6


def _site_coords(problem, off):
    nx, ny, nz = problem["n"]
    d = 1.0 / problem["resolution"]
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return [((i + off[0]) * d).ravel(), ((j + off[1]) * d).ravel(), ((k + off[2]) * d).ravel()]


def _inside(obj, pts, dims, d):
    tol = _TOL * d
    if obj["shape"] == "box":
        m = np.ones(pts[0].shape, dtype=bool)
        for a in range(dims):
            m &= (pts[a] >= obj["lo"][a] - tol) & (pts[a] <= obj["hi"][a] + tol)
        return m
    if obj["shape"] == "sphere":
        r2 = np.zeros(pts[0].shape)
        for a in range(dims):
            r2 += (pts[a] - obj["center"][a]) ** 2
        return r2 <= (obj["radius"] + tol) ** 2
    if obj["shape"] == "grid":
        # voxel (i, j, k) of mask[i, j(, k)] is the closed box lo + [i, i+1] h along each axis,
        # h = (hi - lo) / (voxels along that axis); the object is the union of the filled ones.
        # A point is in it when a filled voxel lies within the tolerance of it.
        mask = np.asarray(obj["mask"]) != 0
        if mask.ndim == 2:
            mask = mask[:, :, None]
        inbox = np.ones(pts[0].shape, dtype=bool)
        near = []                                   # per axis: the voxel indices within tol
        for a in range(3):
            if a >= dims:
                near.append([np.zeros(pts[0].shape, dtype=int)])
                continue
            lo, hi, n = obj["lo"][a], obj["hi"][a], mask.shape[a]
            inbox &= (pts[a] >= lo - tol) & (pts[a] <= hi + tol)
            h = (hi - lo) / n
            u = (pts[a] - lo) / h
            near.append([np.clip(np.floor(u - tol / h), 0, n - 1).astype(int),
                         np.clip(np.floor(u + tol / h), 0, n - 1).astype(int)])
        out = np.zeros(pts[0].shape, dtype=bool)
        for i in near[0]:
            for j in near[1]:
                for k in near[2]:
                    out |= mask[i, j, k]
        return out & inbox
    raise ValueError(obj["shape"])


def lorentz_poles(obj):
    """The (delta_eps_j, omega_j) of a Lorentz object: `delta_eps` and `omega0` are numbers (one
    pole, Eq. (9) without damping) or equal-length sequences (a sum of poles, as in the silica
    model of Sec. III D).  Poles with delta_eps_j = 0 contribute nothing."""
    de, w0 = obj["delta_eps"], obj["omega0"]
    de = [float(de)] if np.isscalar(de) else [float(x) for x in de]
    w0 = [float(w0)] if np.isscalar(w0) else [float(x) for x in w0]
    if len(de) != len(w0) or not 1 <= len(de) <= MAX_POLES:
        raise ValueError("lorentz: delta_eps and omega0 need 1..%d entries each" % MAX_POLES)
    return list(zip(de, w0))


def _materials(problem, pts):
    """Material at each point: (eps, mu, pec, pmc, delta_eps[pole], omega0[pole]); later objects win."""
    dims = problem["dims"]
    d = 1.0 / problem["resolution"]
    M = pts[0].shape[0]
    eps = np.full(M, float(problem["background"]["eps"]))
    mu = np.full(M, float(problem["background"]["mu"]))
    pec = np.zeros(M, dtype=bool)
    pmc = np.zeros(M, dtype=bool)
    lde = np.zeros((MAX_POLES, M))
    lw0 = np.zeros((MAX_POLES, M))
    for obj in problem["objects"]:
        m = _inside(obj, pts, dims, d)
        kind = obj["kind"]
        pec[m] = kind == "pec"
        pmc[m] = kind == "pmc"
        lde[:, m] = 0.0
        lw0[:, m] = 0.0
        if kind == "dielectric":
            eps[m] = obj.get("eps", 1.0)
            mu[m] = obj.get("mu", 1.0)
        elif kind == "lorentz":
            eps[m] = obj.get("eps_inf", 1.0)
            mu[m] = 1.0
            for j, (de, w0) in enumerate(lorentz_poles(obj)):
                lde[j, m] = de
                lw0[j, m] = w0
    return eps, mu, pec, pmc, lde, lw0


def _pml_profile(n, cells, res, dt, half):
    """CPML b, c, 1/kappa (polynomial grading m = 3, R0 = 1e-8, kappa_max = 1,
    alpha linear from 0.05 at the inner interface to 0 at the wall)."""
    d = 1.0 / res
    pos = (np.arange(n) + (0.5 if half else 0.0)) * d
    L = n * d
    w = cells * d
    rho = np.maximum((w - pos) / w, (pos - (L - w)) / w)
    rho = np.clip(rho, 0.0, 1.0)
    smax = -(3 + 1) * math.log(1e-8) / (2.0 * w)
    sig = smax * rho**3
    kap = 1.0 + (1.0 - 1.0) * rho**3
    alpha = 0.05 * (1.0 - rho)
    b = np.exp(-(sig / kap + alpha) * dt)
    c = np.where(sig > 0, sig / np.where(sig > 0, sig * kap + kap * kap * alpha, 1.0) * (b - 1.0), 0.0)
    return b, c, 1.0 / kap


def is_cyl(problem):
    """Cylindrical (r, z) cross-section with fields ~ exp(i m phi) (Sec. III C)."""
    return problem.get("coords", "cartesian") == "cylindrical"


def cyl_site_weight(problem, off_r, i):
    """Volume weight of a cylindrical Yee site (the ring volume over 2 pi Delta^2, in units of
    length): its radius r = (i + off_r) Delta, and Delta/8 on the axis (the disk of radius
    Delta/2 around it) -- the weights that make the discrete curl self-adjoint."""
    d = 1.0 / problem["resolution"]
    r = (i + off_r) * d
    return r if r > 0.5 * _TOL * d else d / 8.0


class _Setup:
    """Per-(problem, k-point) lattice arrays kept alive for the C core."""

    def __init__(self, problem, kvec, m=0):
        self.problem = problem
        dims = problem["dims"]
        nx, ny, nz = problem["n"]
        if dims == 2 and nz != 1:
            raise ValueError("two-dimensional problems have nz == 1")
        cyl = is_cyl(problem)
        if cyl and (dims != 2 or problem["bc"][0] != "pec" or "pml" in problem["bc"]):
            raise ValueError("cylindrical problems are (r, z) cross-sections with a PEC wall at r = R, no PML")
        res = problem["resolution"]
        d = 1.0 / res
        dt = problem["courant"] * d
        self.N = nx * ny * nz
        self.keep = []
        g = _OgGrid()
        g.n[0], g.n[1], g.n[2] = nx, ny, nz
        g.twod = 1 if dims == 2 else 0
        for c in range(3):
            g.eact[c] = g.hact[c] = 1
        g.kz = float(kvec[2]) if dims == 2 and not cyl else 0.0
        g.dx, g.dt, g.sigma = d, dt, float(problem["sigma"])
        g.cyl = 1 if cyl else 0
        g.mphi = float(m) if cyl else 0.0
        self.cyl, self.m = cyl, (int(m) if cyl else 0)
        self.bloch = []
        for a in range(3):
            ph = 1.0 + 0.0j
            if a < dims and problem["bc"][a] == "periodic":
                ph = complex(np.exp(1j * kvec[a] * problem["n"][a] * d))
            self.bloch.append(ph)
            g.bloch_re[a], g.bloch_im[a] = ph.real, ph.imag
        self.ce, self.ch, lde_all, lw0_all = [], [], [], []
        for c in range(3):
            pts = _site_coords(problem, E_OFF[c])
            eps, mu, pec, pmc, lde, lw0 = _materials(problem, pts)
            wall = np.zeros(self.N, dtype=bool)
            for a in range(dims):
                if cyl and a == 0:
                    continue        # r = 0 is the axis, not a wall (the wall r = R lies beyond the grid)
                if problem["bc"][a] in ("pec", "pml") and E_OFF[c][a] == 0.0:
                    wall |= np.abs(pts[a]) < _TOL * d
            if cyl:
                axis = np.abs(pts[0]) < _TOL * d
                if c == 2 or (c == 1 and m != 0):
                    wall |= axis      # E_phi(0) carries no weight; E_z ~ r^|m| vanishes there for m != 0
            ce = np.where(pec | wall, 0.0, 1.0 / eps)
            self.ce.append(np.ascontiguousarray(ce))
            lde_all.append([np.ascontiguousarray(np.where(pec | wall, 0.0, lde[j])) for j in range(MAX_POLES)])
            lw0_all.append([np.ascontiguousarray(lw0[j]) for j in range(MAX_POLES)])
            pts = _site_coords(problem, H_OFF[c])
            eps, mu, pec, pmc, lde, lw0 = _materials(problem, pts)
            if cyl and c == 0:
                pmc = pmc | (np.abs(pts[0]) < _TOL * d)   # H_r(0) carries no weight
            self.ch.append(np.ascontiguousarray(np.where(pmc, 0.0, 1.0 / mu)))
        for c in range(3):
            g.ce[c] = _dp(self.ce[c])
            g.ch[c] = _dp(self.ch[c])
        used = [j for j in range(MAX_POLES) if any(np.any(lde_all[c][j] != 0.0) for c in range(3))]
        if used:
            g.npole = max(used) + 1
            self.lde, self.lw0 = lde_all, lw0_all
            for j in range(g.npole):
                for c in range(3):
                    g.lde[j][c] = _dp(self.lde[c][j])
                    g.lw0[j][c] = _dp(self.lw0[c][j])
        self.pml = {}
        for a in range(dims):
            if problem["bc"][a] == "pml":
                for half in (0, 1):
                    b, cc, ik = _pml_profile(problem["n"][a], problem["pml_cells"][a], res, dt, half)
                    self.pml[(a, half)] = (b, cc, ik)
                    g.pb[a][half] = _dp(b)
                    g.pc[a][half] = _dp(cc)
                    g.pk[a][half] = _dp(ik)
        self.grid = g
        self.real = (g.kz == 0.0) and all(abs(ph.imag) == 0.0 for ph in self.bloch) and self.m == 0
        self.dt = dt
        self.d = d
        self.kvec = kvec


# ---------------------------------------------------------------------------
# Sec. III: faces, pixels, cosine harmonics, interpolation onto the Yee grid
# ---------------------------------------------------------------------------

def face_pixels(problem, face):
    """Pixel centres on a face: (k + 1/2) Delta from the face's low corner along each
    tangential axis; returns (tangential axes, counts, centres (M x 3), pixel area)."""
    dims = problem["dims"]
    d = 1.0 / problem["resolution"]
    a = face["axis"]
    tang = [b for b in range(dims) if b != a]
    counts = [int(round((face["hi"][b] - face["lo"][b]) / d)) for b in tang]
    grids = np.meshgrid(*[np.arange(c) for c in counts], indexing="ij")
    centres = np.zeros((int(np.prod(counts)), 3))
    centres[:, a] = face["pos"]
    for t, b in enumerate(tang):
        centres[:, b] = face["lo"][b] + (grids[t].ravel() + 0.5) * d
    return tang, counts, centres, d ** (dims - 1)


def harmonic(problem, face, nvec):
    """f_n on the pixels of a face (Eq. (7)): sqrt(2/L) cos(n pi x / L), with f_0 = sqrt(1/L);
    in three dimensions the product over the two tangential axes.

    With problem["basis"] == "point" the basis is instead the point-source basis of
    Sec. II (one pixel per function, f = 1/sqrt(dA) on pixel nvec[0], zero elsewhere)."""
    d = 1.0 / problem["resolution"]
    tang, counts, centres, dA = face_pixels(problem, face)
    if problem.get("basis", "cosine") == "point":
        f = np.zeros(centres.shape[0])
        f[nvec[0]] = 1.0 / math.sqrt(dA)
        return f
    f = np.ones(centres.shape[0])
    for t, b in enumerate(tang):
        L = counts[t] * d
        x = centres[:, b] - face["lo"][b]
        n = nvec[t]
        f *= math.sqrt(1.0 / L) if n == 0 else math.sqrt(2.0 / L) * np.cos(n * math.pi * x / L)
    return f


def interp_weights(problem, setup, point, off):
    """(Bi/tri)linear interpolation weights from the Yee sites with offset `off` to `point`.
    Returns a list of (flat index, complex weight); wrapped sites carry the Bloch factor."""
    dims = problem["dims"]
    d = 1.0 / problem["resolution"]
    per_axis = []
    for a in range(3):
        if a >= dims:
            per_axis.append([(0, 1.0 + 0j)])
            continue
        u = point[a] / d - off[a]
        i0 = math.floor(u)
        t = u - i0
        if t < 1e-9:
            t = 0.0
        elif t > 1.0 - 1e-9:
            i0 += 1
            t = 0.0
        ent = [(i0, 1.0 - t)] + ([(i0 + 1, t)] if t > 0.0 else [])
        n = problem["n"][a]
        out = []
        for i, w in ent:
            q = i // n
            if a == 0 and is_cyl(problem):
                if q == 0:
                    out.append((i, w))      # no wrap in r: beyond r = R the tangential E vanishes
                continue
            out.append((i - q * n, w * setup.bloch[a] ** q))
        per_axis.append(out)
    nx, ny, _ = problem["n"]
    res = []
    for i, wi in per_axis[0]:
        for j, wj in per_axis[1]:
            for k, wk in per_axis[2]:
                res.append(((k * ny + j) * nx + i, wi * wj * wk))
    return res


# ---------------------------------------------------------------------------
# Sims: one per (k-point, face, harmonic, source kind and component)
# ---------------------------------------------------------------------------

_TM = (("J", 2), ("K", 0), ("K", 1))
_TE = (("J", 0), ("J", 1), ("K", 2))
_FULL = (("J", 0), ("J", 1), ("J", 2), ("K", 0), ("K", 1), ("K", 2))


def _families(problem):
    pol = problem["polarization"]
    if problem["dims"] == 2 and pol in ("TM", "TE", "TE+TM"):
        fam = []
        if "TM" in pol:
            fam += [("TM",) + x for x in _TM]
        if "TE" in pol:
            fam += [("TE",) + x for x in _TE]
        return fam
    return [("full",) + x for x in _FULL]


def harmonic_list(problem, face):
    tang, counts, _, _ = face_pixels(problem, face)
    if problem.get("basis", "cosine") == "point":
        return [(k,) for k in range(int(np.prod(counts)))]
    nh = [min(problem["n_harm"], c) for c in counts]
    if len(tang) == 1:
        return [(n,) for n in range(nh[0])]
    return [(n1, n2) for n1 in range(nh[0]) for n2 in range(nh[1])]


def enumerate_sims(problem):
    """All contributing sims.  For force axis i, a face with normal axis a needs every
    source component when a == i, otherwise only c == a (the other terms of
    n_c E_i - 1/2 n_i E_c vanish identically)."""
    fa = problem["force_axis"]
    sims = []
    for ki, _ in enumerate(problem["k_points"]):
        for fi, face in enumerate(problem["faces"]):
            for nvec in harmonic_list(problem, face):
                for pol, kind, c in _families(problem):
                    if face["axis"] == fa or c == face["axis"]:
                        sims.append({"k": ki, "face": fi, "harm": nvec, "pol": pol, "kind": kind, "comp": c})
    return sims


def _sim_vectors(problem, setup, sim):
    """Source flux at t = 0+ and the measurement functional of one sim (Sec. II, Eqs. (3)-(6))."""
    face = problem["faces"][sim["face"]]
    _, _, centres, dA = face_pixels(problem, face)
    f = harmonic(problem, face, sim["harm"])
    d = setup.d
    c = sim["comp"]
    magnetic = sim["kind"] == "K"
    offs = H_OFF if magnetic else E_OFF
    # source: D_c(p) = -(dA/dV) sum_k conj(W_c(k,p)) f(x_k); in cylindrical coordinates the
    # surface current f e^{i m phi} on the surface of revolution, averaged over the ring of the
    # site, carries r(x_k) / w(p) (ring area over ring volume)
    cyl = is_cyl(problem)
    nx = problem["n"][0]
    src = {}
    for k in range(centres.shape[0]):
        for idx, w in interp_weights(problem, setup, centres[k], offs[c]):
            scale = centres[k][0] / cyl_site_weight(problem, offs[c][0], idx % nx) if cyl else 1.0
            src[idx] = src.get(idx, 0.0) - np.conj(w) * f[k] * scale / d
    # measurement: s_i = sum_k dA w_S f(x_k) [n_c F_i(x_k) - 1/2 n_i F_c(x_k)]
    i = problem["force_axis"]
    a = face["axis"]
    nvec = [0.0, 0.0, 0.0]
    nvec[a] = float(face["sign"])
    eps, mu, _, _, _, _ = _materials(problem, [centres[:, 0], centres[:, 1], centres[:, 2]])
    wS = mu if magnetic else eps
    meas = {}
    for k in range(centres.shape[0]):
        base = dA * wS[k] * f[k]
        for q, coef in ((i, nvec[c]), (c, -0.5 * nvec[i])):
            if coef == 0.0:
                continue
            for idx, w in interp_weights(problem, setup, centres[k], offs[q]):
                key = (q, idx)
                meas[key] = meas.get(key, 0.0) + base * coef * w
    return src, meas


def _setups(problem):
    return [_Setup(problem, kp["k"], kp.get("m", 0)) for kp in problem["k_points"]]


def run_vectors(problem, setup, magnetic, src, meas, pol="full"):
    """Run the leapfrog from an explicit post-impulse flux and record an explicit
    functional: src maps (component, site) -> D (or B) value, meas maps
    (component, site) -> weight.  Returns s(n), n = 1..T."""
    sim = {"kind": "K" if magnetic else "J", "pol": pol, "comp": 0}
    return _run(problem, setup, sim, src, meas)


def run_sim(problem, sim, setup=None):
    """Run one sim; return the complex series s(n), n = 1..T."""
    if setup is None:
        kp = problem["k_points"][sim["k"]]
        setup = _Setup(problem, kp["k"], kp.get("m", 0))
    src, meas = _sim_vectors(problem, setup, sim)
    src = {(sim["comp"], k): v for k, v in src.items()}
    return _run(problem, setup, sim, src, meas)


def _run(problem, setup, sim, src, meas):
    s = _OgSim()
    s.magnetic = 1 if sim["kind"] == "K" else 0
    s.nsteps = problem["n_steps"]
    skeys = sorted(src)
    sk = np.array([k[1] for k in skeys], dtype=np.int32)
    sv = np.array([src[k] for k in skeys], dtype=np.complex128)
    scomp = np.array([k[0] for k in skeys], dtype=np.int32)
    sre, sim_ = np.ascontiguousarray(sv.real), np.ascontiguousarray(sv.imag)
    s.nsrc = len(sk)
    s.src_comp, s.src_idx, s.src_re, s.src_im = _ip(scomp), _ip(sk), _dp(sre), _dp(sim_)
    keys = sorted(meas)
    mcomp = np.array([k[0] for k in keys], dtype=np.int32)
    midx = np.array([k[1] for k in keys], dtype=np.int32)
    mv = np.array([meas[k] for k in keys], dtype=np.complex128)
    mre, mim = np.ascontiguousarray(mv.real), np.ascontiguousarray(mv.imag)
    ptr = np.array([0, len(keys)], dtype=np.int32)
    s.nset = 1
    s.set_ptr, s.m_comp, s.m_idx, s.m_re, s.m_im = _ip(ptr), _ip(mcomp), _ip(midx), _dp(mre), _dp(mim)
    T = problem["n_steps"]
    ore = np.zeros(T)
    oim = np.zeros(T)
    g = _OgGrid.from_buffer_copy(setup.grid)
    if sim["pol"] in ("TM", "TE"):
        # at k_z = 0 the TE and TM sets decouple exactly; only one set is ever non-zero
        tm = sim["pol"] == "TM"
        for q in range(3):
            g.eact[q] = int((q == 2) == tm)
            g.hact[q] = int((q == 2) != tm)
    rc = _lib(setup.real).oracle_run(ctypes.byref(g), ctypes.byref(s), _dp(ore), _dp(oim))
    if rc != 0:
        raise MemoryError("oracle_run failed")
    return ore + 1j * oim


def force(problem, sims=None, threads=None, return_parts=False):
    """F_i = sum_k weight_k sum_sims sum_{n>=1} w_n Re s(n)  (Eq. (1) with Sec. III B/D sums).

    Returns the force, or (force, per-sim contributions, sims) with return_parts."""
    if sims is None:
        sims = enumerate_sims(problem)
    setups = _setups(problem)
    w = g_weights(problem)
    kw = [kp["weight"] for kp in problem["k_points"]]
    nthr = threads or os.cpu_count() or 1

    def one(sim):
        s = run_sim(problem, sim, setups[sim["k"]])
        return math.fsum(w * s.real) * kw[sim["k"]]

    if nthr > 1 and len(sims) > 1:
        with ThreadPoolExecutor(max_workers=nthr) as ex:
            parts = list(ex.map(one, sims))
    else:
        parts = [one(s) for s in sims]
    F = math.fsum(parts)
    if return_parts:
        return F, parts, sims
    return F


def grid_setup(problem, kvec=(0.0, 0.0, 0.0), m=0):
    return _Setup(problem, list(kvec), m)


def evolve(problem, E0, H0, nsteps, kvec=(0.0, 0.0, 0.0), setup=None):
    """Source-free evolution of given fields (electric ordering, sigma on D, half-step start).
    E0, H0: complex arrays (3, N).  Returns (E^T, H^{T-1/2}, H^{T-3/2})."""
    if setup is None:
        setup = _Setup(problem, list(kvec))
    N = setup.N
    e = np.ascontiguousarray(np.asarray(E0, dtype=np.complex128).reshape(3, N))
    h = np.ascontiguousarray(np.asarray(H0, dtype=np.complex128).reshape(3, N))
    ere, eim = np.ascontiguousarray(e.real), np.ascontiguousarray(e.imag)
    hre, him = np.ascontiguousarray(h.real), np.ascontiguousarray(h.imag)
    pre, pim = np.zeros(3 * N), np.zeros(3 * N)
    rc = _lib(False).oracle_evolve(ctypes.byref(setup.grid), int(nsteps), _dp(ere), _dp(eim), _dp(hre), _dp(him),
                              _dp(pre), _dp(pim))
    if rc != 0:
        raise MemoryError("oracle_evolve failed")
    return ((ere + 1j * eim).reshape(3, N), (hre + 1j * him).reshape(3, N), (pre + 1j * pim).reshape(3, N))
