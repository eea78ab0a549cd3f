"""ctypes binding of include/casimir.h: argument marshalling only.

Every step of the computation runs inside libcasimir.so (host planner and CUDA
kernels).  Loading fails loudly when the library has not been built; there is
no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import weakref

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libcasimir.so")

OK, NOTREADY = 0, 1
EINVAL, ENOMEM, ECUDA, EBUSY, ETIMEOUT, ECANCELED = -1, -2, -3, -4, -5, -6

BC = {"pec": 0, "pml": 1, "periodic": 2}
SHAPE = {"box": 0, "sphere": 1, "grid": 2}
KIND = {"pec": 0, "pmc": 1, "dielectric": 2, "lorentz": 3}
POL = {"TM": 1, "TE": 2, "TE+TM": 3, "full": 4}
GVAR = {"plain": 0, "zinv": 1}
PREC = {"fp32": 0, "fp64": 1}
BASIS = {"cosine": 0, "point": 1}
COORDS = {"cartesian": 0, "cylindrical": 1}

D3 = ctypes.c_double * 3
I3 = ctypes.c_int * 3
MAX_POLES = 3      # CASIMIR_MAX_POLES
DP3 = ctypes.c_double * MAX_POLES


class Object(ctypes.Structure):
    _fields_ = [("shape", ctypes.c_int), ("kind", ctypes.c_int), ("lo", D3), ("hi", D3),
                ("center", D3), ("radius", ctypes.c_double), ("eps", ctypes.c_double),
                ("mu", ctypes.c_double), ("eps_inf", ctypes.c_double), ("delta_eps", DP3),
                ("omega0", DP3), ("mask", ctypes.POINTER(ctypes.c_uint8)), ("mask_n", I3),
                ("reserved", ctypes.c_int)]


def _poles(o: dict):
    """delta_eps / omega0 of a Lorentz object: numbers (one pole) or equal-length sequences."""
    de, w0 = o.get("delta_eps", 0.0), o.get("omega0", 0.0)
    de = [de] if isinstance(de, (int, float)) else list(de)
    w0 = [w0] if isinstance(w0, (int, float)) else list(w0)
    if len(de) != len(w0) or not 1 <= len(de) <= MAX_POLES:
        raise ValueError(f"lorentz: delta_eps and omega0 need 1..{MAX_POLES} entries each")
    pad = [0.0] * (MAX_POLES - len(de))
    return DP3(*[float(x) for x in de], *pad), DP3(*[float(x) for x in w0], *pad)


def _mask_bytes(mask):
    """A grid object's mask, indexed mask[i, j] or mask[i, j, k], as C-ordered (k, j, i) bytes."""
    import numpy as np
    m = np.asarray(mask)
    if m.ndim == 2:
        m = m[:, :, None]
    if m.ndim != 3:
        raise ValueError("grid mask: 2 or 3 dimensions")
    return np.ascontiguousarray((m != 0).transpose(2, 1, 0), dtype=np.uint8)


class Face(ctypes.Structure):
    _fields_ = [("axis", ctypes.c_int), ("sign", ctypes.c_int), ("pos", ctypes.c_double),
                ("lo", D3), ("hi", D3)]


class KPoint(ctypes.Structure):
    _fields_ = [("k", D3), ("weight", ctypes.c_double), ("m", ctypes.c_int), ("reserved", ctypes.c_int)]


class Problem(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int), ("n", I3), ("resolution", ctypes.c_double),
                ("courant", ctypes.c_double), ("n_steps", ctypes.c_int), ("sigma", ctypes.c_double),
                ("bg_eps", ctypes.c_double), ("bg_mu", ctypes.c_double),
                ("n_objects", ctypes.c_int), ("objects", ctypes.POINTER(Object)),
                ("bc", I3), ("pml_cells", I3),
                ("n_faces", ctypes.c_int), ("faces", ctypes.POINTER(Face)),
                ("n_harm", ctypes.c_int), ("polarization", ctypes.c_int),
                ("n_kpoints", ctypes.c_int), ("kpoints", ctypes.POINTER(KPoint)),
                ("force_axis", ctypes.c_int), ("g_variant", ctypes.c_int),
                ("precision", ctypes.c_int), ("basis", ctypes.c_int), ("coords", ctypes.c_int)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("n_sims", ctypes.c_int64), ("n_cells", ctypes.c_int64), ("cell_updates", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("bytes_per_update", ctypes.c_int64),
                ("upload_bytes", ctypes.c_int64), ("bytes_per_step", ctypes.c_int64), ("launches", ctypes.c_int64)]


class PlanOptions(ctypes.Structure):
    _fields_ = [("steps_per_launch", ctypes.c_int), ("march_rows", ctypes.c_int), ("kernel_3d", ctypes.c_int),
                ("reserved", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("queue_ms", ctypes.c_double), ("device_ms", ctypes.c_double), ("total_ms", ctypes.c_double),
                ("cell_updates", ctypes.c_int64), ("kernel_launches", ctypes.c_int64)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

# every function declared in include/casimir.h, with its ctypes signature
SIGNATURES = {
    "casimir_ctx_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_uint64, ctypes.POINTER(ctypes.c_void_p)]),
    "casimir_ctx_destroy": (None, [ctypes.c_void_p]),
    "casimir_ctx_set_stream": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "casimir_ctx_set_allocator": (ctypes.c_int, [ctypes.c_void_p, ALLOC_FN, FREE_FN, ctypes.c_void_p]),
    "casimir_ctx_set_watchdog": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double]),
    "casimir_ctx_set_wave_bytes": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    "casimir_ctx_kernel_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                                ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                                ctypes.c_int]),
    "casimir_plan": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Problem), ctypes.POINTER(ctypes.c_void_p)]),
    "casimir_plan_get_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(PlanInfo)]),
    "casimir_plan_sim_entries": (ctypes.c_int64, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                                                 ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64),
                                                 ctypes.POINTER(ctypes.c_double), ctypes.c_int64]),
    "casimir_plan_site_poles": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "casimir_plan_pml": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "casimir_plan_site_coefs": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "casimir_plan_ex": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Problem), ctypes.POINTER(PlanOptions),
                                       ctypes.POINTER(ctypes.c_void_p)]),
    "casimir_plan_get_options": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(PlanOptions)]),
    "casimir_ctx_set_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "casimir_plan_destroy": (None, [ctypes.c_void_p]),
    "casimir_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(ctypes.c_void_p)]),
    "casimir_force": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double), ctypes.POINTER(Stats)]),
    "casimir_cancel": (ctypes.c_int, [ctypes.c_void_p]),
    "casimir_run": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_double), ctypes.POINTER(Stats)]),
    "casimir_run_plain": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_double), ctypes.POINTER(Stats)]),
    "casimir_plan_sims": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32), ctypes.c_int64]),
    "casimir_plan_weights": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int64]),
    "casimir_run_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "casimir_last_error": (ctypes.c_char_p, []),
}

_lib = None


class CasimirError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"casimir error {code}: {msg}")
        self.code = code


def lib():
    """Load libcasimir.so (built by paper_0906_5170_gb300.build); raise if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run paper_0906_5170_gb300.build.build() first "
                              "(there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(rc):
    if rc < 0:
        raise CasimirError(rc, lib().casimir_last_error().decode(errors="replace"))
    return rc


def _d3(v):
    v = list(v) + [0.0] * (3 - len(v))
    return D3(*[float(x) for x in v[:3]])


class MarshalledProblem:
    """A casimir_problem struct and the arrays it points to, kept alive together."""

    def __init__(self, p: dict):
        objs = p.get("objects", [])
        self.masks = []                      # voxel masks of grid objects, kept alive with the struct
        self.objects = (Object * max(1, len(objs)))()
        for i, o in enumerate(objs):
            ob = self.objects[i]
            ob.shape = SHAPE[o["shape"]]
            ob.kind = KIND[o["kind"]]
            ob.lo = _d3(o.get("lo", [0, 0, 0]))
            ob.hi = _d3(o.get("hi", [0, 0, 0]))
            ob.center = _d3(o.get("center", [0, 0, 0]))
            ob.radius = float(o.get("radius", 0.0))
            ob.eps = float(o.get("eps", 1.0))
            ob.mu = float(o.get("mu", 1.0))
            ob.eps_inf = float(o.get("eps_inf", 1.0))
            ob.delta_eps, ob.omega0 = _poles(o)
            if o["shape"] == "grid":
                m = _mask_bytes(o["mask"])
                self.masks.append(m)
                ob.mask = m.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
                ob.mask_n = I3(*[int(x) for x in m.shape[::-1]])
        faces = p["faces"]
        self.faces = (Face * max(1, len(faces)))()
        for i, f in enumerate(faces):
            self.faces[i].axis = int(f["axis"])
            self.faces[i].sign = int(f["sign"])
            self.faces[i].pos = float(f["pos"])
            self.faces[i].lo = _d3(f["lo"])
            self.faces[i].hi = _d3(f["hi"])
        kps = p["k_points"]
        self.kpoints = (KPoint * max(1, len(kps)))()
        for i, k in enumerate(kps):
            self.kpoints[i].k = _d3(k["k"])
            self.kpoints[i].weight = float(k["weight"])
            self.kpoints[i].m = int(k.get("m", 0))
        s = Problem()
        s.dims = int(p["dims"])
        s.n = I3(*[int(x) for x in p["n"]])
        s.resolution = float(p["resolution"])
        s.courant = float(p["courant"])
        s.n_steps = int(p["n_steps"])
        s.sigma = float(p["sigma"])
        s.bg_eps = float(p["background"]["eps"])
        s.bg_mu = float(p["background"]["mu"])
        s.n_objects = len(objs)
        s.objects = self.objects
        s.bc = I3(*[BC[b] for b in p["bc"]])
        s.pml_cells = I3(*[int(x) for x in p.get("pml_cells", [0, 0, 0])])
        s.n_faces = len(faces)
        s.faces = self.faces
        s.n_harm = int(p["n_harm"])
        s.polarization = POL[p["polarization"]]
        s.n_kpoints = len(kps)
        s.kpoints = self.kpoints
        s.force_axis = int(p["force_axis"])
        s.g_variant = GVAR[p.get("g_variant", "plain")]
        s.precision = PREC[p.get("precision", "fp32")]
        s.basis = BASIS[p.get("basis", "cosine")]
        s.coords = COORDS[p.get("coords", "cartesian")]
        self.struct = s


class Context:
    """casimir_ctx_t: one device, one stream, an HBM budget and a request executor."""

    def __init__(self, device=0, hbm_budget_bytes=0, stream=None):
        h = ctypes.c_void_p()
        check(lib().casimir_ctx_create(int(device), int(hbm_budget_bytes), ctypes.byref(h)))
        self.h = h
        self._plans = weakref.WeakSet()
        if stream is not None:
            check(lib().casimir_ctx_set_stream(self.h, ctypes.c_void_p(int(stream))))

    def set_stream(self, stream):
        check(lib().casimir_ctx_set_stream(self.h, ctypes.c_void_p(int(stream) if stream else None)))

    def set_watchdog(self, ms):
        check(lib().casimir_ctx_set_watchdog(self.h, float(ms)))

    def set_allocator(self, alloc, free):
        self._alloc = ALLOC_FN(lambda b, u: alloc(b))
        self._free = FREE_FN(lambda p, u: free(p))
        check(lib().casimir_ctx_set_allocator(self.h, self._alloc, self._free, None))

    def set_wave_bytes(self, nbytes):
        check(lib().casimir_ctx_set_wave_bytes(self.h, int(nbytes)))

    def set_autotune(self, on=True):
        check(lib().casimir_ctx_set_autotune(self.h, 1 if on else 0))

    def kernel_stats(self, reset=False):
        ms = ctypes.c_double()
        nl = ctypes.c_int64()
        cu = ctypes.c_int64()
        check(lib().casimir_ctx_kernel_stats(self.h, ctypes.byref(ms), ctypes.byref(nl), ctypes.byref(cu), int(reset)))
        return ms.value, nl.value, cu.value

    def plan(self, problem: dict, options: dict | None = None):
        return Plan(problem, self, options)

    def close(self):
        if self.h:
            for p in list(self._plans):      # plans must be released before their context
                p.close()
            lib().casimir_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan:
    """casimir_plan_t built from a problem dictionary (ctx None: host-only plan)."""

    def __init__(self, problem: dict, ctx: Context | None = None, options: dict | None = None):
        self.problem = problem
        self.ctx = ctx
        self._m = MarshalledProblem(problem)
        h = ctypes.c_void_p()
        if options is None:
            check(lib().casimir_plan(ctx.h if ctx else None, ctypes.byref(self._m.struct), ctypes.byref(h)))
        else:
            o = PlanOptions(**{k: int(v) for k, v in options.items()})
            check(lib().casimir_plan_ex(ctx.h if ctx else None, ctypes.byref(self._m.struct), ctypes.byref(o),
                                        ctypes.byref(h)))
        self.h = h
        if ctx is not None:
            ctx._plans.add(self)

    def options(self):
        o = PlanOptions()
        check(lib().casimir_plan_get_options(self.h, ctypes.byref(o)))
        return {f: getattr(o, f) for f, _ in PlanOptions._fields_ if f != "reserved"}

    def info(self):
        i = PlanInfo()
        check(lib().casimir_plan_get_info(self.h, ctypes.byref(i)))
        return {f: getattr(i, f) for f, _ in PlanInfo._fields_}

    def site_coefs(self, kpoint, field, comp):
        """The rasterised coefficient (1/eps or 1/mu, 0 where masked) of the array storing
        component `comp` of E (field 0) or H (field 1) at k-point `kpoint`, as an array
        indexed [i, j, k], and the sites' offsets within a cell (in cells)."""
        nx, ny, nz = (int(v) for v in self.problem["n"])
        out = np.zeros(nx * ny * nz)
        off = (ctypes.c_double * 3)()
        check(lib().casimir_plan_site_coefs(self.h, int(kpoint), int(field), int(comp), off,
                                            out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out.reshape(nz, ny, nx).transpose(2, 1, 0), tuple(off)

    def pml(self, axis, half):
        """CPML b, c, 1/kappa along PML axis `axis` at integer (half 0) or half-integer sites."""
        n = int(self.problem["n"][axis]) if 0 <= axis < 3 else 1   # the library rejects a bad axis
        b, c, ik = np.zeros(n), np.zeros(n), np.zeros(n)
        P = ctypes.POINTER(ctypes.c_double)
        check(lib().casimir_plan_pml(self.h, int(axis), int(half), b.ctypes.data_as(P), c.ctypes.data_as(P),
                                     ik.ctypes.data_as(P)))
        return b, c, ik

    def site_poles(self, kpoint, comp, pole):
        """Strength and frequency of Lorentz pole slot `pole` at the sites of E component
        `comp` (arrays indexed [i, j, k]; present poles fill the first slots, 0 elsewhere)."""
        nx, ny, nz = (int(v) for v in self.problem["n"])
        de, w0 = np.zeros(nx * ny * nz), np.zeros(nx * ny * nz)
        check(lib().casimir_plan_site_poles(self.h, int(kpoint), int(comp), int(pole),
                                            de.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                            w0.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return (de.reshape(nz, ny, nx).transpose(2, 1, 0), w0.reshape(nz, ny, nx).transpose(2, 1, 0))

    def sim_entries(self, sim, which):
        """Source (which 0) or measurement (which 1) entries of simulation `sim`: arrays of
        3 * field + component, cell index on that array's lattice, and complex value."""
        L = lib()
        n = check(L.casimir_plan_sim_entries(self.h, int(sim), int(which), None, None, None, 0))
        comp = np.zeros(n, np.int32)
        idx = np.zeros(n, np.int64)
        val = np.zeros(2 * n)
        check(L.casimir_plan_sim_entries(self.h, int(sim), int(which),
                                         comp.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                         idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                         val.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n))
        return comp, idx, val[0::2] + 1j * val[1::2]

    def sims(self):
        n = self.info()["n_sims"]
        d = np.zeros(6 * n, dtype=np.int32)
        check(lib().casimir_plan_sims(self.h, d.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), n))
        return d.reshape(n, 6)

    def weights(self):
        T = int(self.problem["n_steps"])
        w = np.zeros(T)
        check(lib().casimir_plan_weights(self.h, w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), T))
        return w

    def run(self, per_sim=False, plain=False):
        """Synchronous run: returns (F[3], per-sim contributions or None, stats dict).
        plain=True uses the unbatched comparison path (casimir_run_plain)."""
        F = (ctypes.c_double * 3)()
        st = Stats()
        ps = None
        ptr = None
        if per_sim:
            ps = np.zeros(self.info()["n_sims"])
            ptr = ps.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        fn = lib().casimir_run_plain if plain else lib().casimir_run
        check(fn(self.h, F, ptr, ctypes.byref(st)))
        return np.array(F[:]), ps, {f: getattr(st, f) for f, _ in Stats._fields_}

    def submit(self, tag=0):
        t = ctypes.c_void_p()
        check(lib().casimir_submit(self.h, int(tag), ctypes.byref(t)))
        return Ticket(t, self)

    def close(self):
        if self.h:
            lib().casimir_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Ticket:
    def __init__(self, h, plan):
        self.h = h
        self.plan = plan        # the plan must outlive its requests
        self.done = False

    def force(self, wait_ms=-1):
        """Returns None while running, else (F[3], err_est, stats dict); raises on failure."""
        F = (ctypes.c_double * 3)()
        err = ctypes.c_double()
        st = Stats()
        rc = lib().casimir_force(self.h, int(wait_ms), F, ctypes.byref(err), ctypes.byref(st))
        if rc == NOTREADY:
            return None
        self.done = True
        check(rc)
        return np.array(F[:]), err.value, {f: getattr(st, f) for f, _ in Stats._fields_}

    def cancel(self):
        check(lib().casimir_cancel(self.h))


def header_functions(path=None):
    """Names of the functions declared in include/casimir.h."""
    import re
    path = path or os.path.join(os.path.dirname(HERE), "include", "casimir.h")
    txt = open(path).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(casimir_\w+)\s*\(", txt)) - {"casimir_alloc_fn", "casimir_free_fn"})
