"""ctypes binding of the C ABI in ``include/fempic.h``.

Argument marshalling only: every step of the method runs in the CUDA library.
The module-level functions carry the C names (``femPIC_create``,
``femPIC_step``, ...); ``Simulation`` wraps one handle with numpy in/out.
Loading fails loudly (ImportError) when ``libfempic.so`` has not been built.
"""

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# FEMPIC_LIB selects another build of the library (the test variants of build.py)
LIB_PATH = os.environ.get("FEMPIC_LIB") or os.path.join(_HERE, "libfempic.so")

FEMPIC_OK, FEMPIC_ERR_ARG, FEMPIC_ERR_MESH, FEMPIC_ERR_OOM, FEMPIC_ERR_CUDA = 0, 1, 2, 3, 4
FEMPIC_ERR_CG, FEMPIC_ERR_WALK, FEMPIC_ERR_SIZE, FEMPIC_ERR_STATE, FEMPIC_ERR_BARRIER = 5, 6, 7, 8, 9
FEMPIC_ERR_BOUNDS = 10
ERROR_NAMES = {0: "OK", 1: "ERR_ARG", 2: "ERR_MESH", 3: "ERR_OOM", 4: "ERR_CUDA", 5: "ERR_CG",
               6: "ERR_WALK", 7: "ERR_SIZE", 8: "ERR_STATE", 9: "ERR_BARRIER", 10: "ERR_BOUNDS"}
PRECISION = {"fp64_strict": 0, "fp64": 1, "mixed": 2}
SCHEME = {"trapezoid": 0, "wave": 1}
PUSH = {"boris": 0, "ab4": 1}
QUANTITY = {"E": 0, "B": 1, "DG": 2, "RHO": 3, "X": 4, "V": 5, "TET": 6, "NCROSS": 7, "HASH": 8,
            "E_PREV": 9, "DG_PREV": 10, "DIAG": 11, "PHI": 12, "SPECIES": 13, "B_IMPRESSED": 14, "J": 15}
MAX_SPECIES = 8
OPERATOR = {"M1": 0, "K": 1, "C": 2, "D": 3, "DT": 4, "M2": 5, "A": 6, "L": 7, "PI": 8, "PIT": 9}


class femPIC_mesh(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int32), ("n_tets", ctypes.c_int32),
                ("xyz_host", ctypes.c_void_p), ("tets_host", ctypes.c_void_p)]


class femPIC_species(ctypes.Structure):
    _fields_ = [("q", ctypes.c_double), ("m", ctypes.c_double), ("weight", ctypes.c_double),
                ("n", ctypes.c_int64), ("x_host", ctypes.c_void_p), ("v_host", ctypes.c_void_p),
                ("tet_host", ctypes.c_void_p)]


class femPIC_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("scheme", ctypes.c_int32),
                ("gamma", ctypes.c_double), ("beta", ctypes.c_double), ("cg_rtol", ctypes.c_double),
                ("cg_max_it", ctypes.c_int32), ("max_cross", ctypes.c_int32),
                ("sort_period", ctypes.c_int32), ("B0", ctypes.c_double * 3),
                ("rho_ion", ctypes.c_double), ("es_init", ctypes.c_int32),
                ("diagnostics", ctypes.c_int32), ("device", ctypes.c_int32),
                ("stream", ctypes.c_void_p), ("push", ctypes.c_int32)]


class femPIC_diag(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("status", ctypes.c_int32),
                ("cg_iterations", ctypes.c_int32), ("cg_residual", ctypes.c_double),
                ("continuity_abs", ctypes.c_double), ("continuity_ref", ctypes.c_double),
                ("gauss_abs", ctypes.c_double), ("gauss_ref", ctypes.c_double),
                ("crossings", ctypes.c_double), ("absorbed", ctypes.c_double),
                ("divb_abs", ctypes.c_double), ("divb_ref", ctypes.c_double)]


class femPIC_info(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int32), ("n_tets", ctypes.c_int32),
                ("n_edges", ctypes.c_int32), ("n_faces", ctypes.c_int32),
                ("order", ctypes.c_int32), ("n0", ctypes.c_int32), ("n1", ctypes.c_int32),
                ("n2", ctypes.c_int32), ("nl0", ctypes.c_int32), ("nl1", ctypes.c_int32),
                ("nl2", ctypes.c_int32), ("n_particles", ctypes.c_int64),
                ("nnz_A", ctypes.c_int64), ("nnz_C", ctypes.c_int64), ("nnz_Q", ctypes.c_int64),
                ("nnz_D", ctypes.c_int64), ("nnz_DT", ctypes.c_int64), ("nnz_Pi", ctypes.c_int64),
                ("n_boundary_faces", ctypes.c_int32), ("device_bytes", ctypes.c_size_t),
                ("nnz_L", ctypes.c_int64), ("nnz_V", ctypes.c_int64), ("aux_cheb_degree", ctypes.c_int32),
                ("n_species", ctypes.c_int32), ("n_impedance_faces", ctypes.c_int32),
                ("n_absorb_faces", ctypes.c_int32), ("n_inject_faces", ctypes.c_int32),
                ("device_allocations", ctypes.c_int64), ("cg_fp32_products", ctypes.c_int32),
                ("cg_replace_period", ctypes.c_int32), ("cg_smooth_degree", ctypes.c_int32)]


# (name, restype, argtypes) of every exported symbol declared in include/fempic.h
_P = ctypes.c_void_p
class femPIC_batch_tuning(ctypes.Structure):
    _fields_ = [("particle_block", ctypes.c_int32), ("particle_grid", ctypes.c_int32),
                ("cg_ctas_per_sm", ctypes.c_int32), ("particle_candidates", ctypes.c_int32),
                ("cg_candidates", ctypes.c_int32), ("steps", ctypes.c_int32),
                ("particle_ms", ctypes.c_double), ("cg_ms", ctypes.c_double),
                ("particle_ms_default", ctypes.c_double), ("cg_ms_default", ctypes.c_double)]


class femPIC_injector(ctypes.Structure):
    _fields_ = [("species", ctypes.c_int32), ("v_drift", ctypes.c_double * 3), ("v_sigma", ctypes.c_double * 3)]


class femPIC_projection(ctypes.Structure):
    _fields_ = [("outer_iterations", ctypes.c_int32), ("inner_iterations", ctypes.c_int32),
                ("div_residual", ctypes.c_double), ("host_ms", ctypes.c_double), ("device_ms", ctypes.c_double),
                ("inner_ms", ctypes.c_double), ("bytes_per_inner_iteration", ctypes.c_double)]


EXPORTS = [
    ("femPIC_default_opts", None, [ctypes.POINTER(femPIC_opts)]),
    ("femPIC_create", ctypes.c_int, [ctypes.POINTER(femPIC_mesh), ctypes.c_int32,
                                     ctypes.POINTER(femPIC_species), ctypes.POINTER(femPIC_opts),
                                     ctypes.POINTER(_P)]),
    ("femPIC_create_ext", ctypes.c_int, [ctypes.POINTER(femPIC_mesh), ctypes.c_int32,
                                         ctypes.POINTER(femPIC_species), ctypes.c_int32, _P,
                                         ctypes.POINTER(femPIC_opts), ctypes.POINTER(_P)]),
    ("femPIC_step", ctypes.c_int, [_P, ctypes.c_double, ctypes.c_int32]),
    ("femPIC_step_async", ctypes.c_int, [_P, ctypes.c_double, ctypes.c_int32]),
    ("femPIC_sync", ctypes.c_int, [_P]),
    ("femPIC_get", ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_size_t]),
    ("femPIC_set", ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_size_t]),
    ("femPIC_get_device", ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_size_t]),
    ("femPIC_set_device", ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_size_t]),
    ("femPIC_apply", ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_size_t, _P, ctypes.c_size_t]),
    ("femPIC_eval_fields", ctypes.c_int, [_P, ctypes.c_int64, _P, _P, _P, _P]),
    ("femPIC_eval_fields_noalloc", ctypes.c_int, [_P, ctypes.c_int64, _P, _P, _P, _P]),
    ("femPIC_get_info", ctypes.c_int, [_P, ctypes.POINTER(femPIC_info)]),
    ("femPIC_impressed_points", ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_int64)]),
    ("femPIC_set_injection", ctypes.c_int, [_P, ctypes.POINTER(femPIC_injector), ctypes.c_int32, ctypes.c_uint64]),
    ("femPIC_set_impressed_B", ctypes.c_int, [_P, _P, ctypes.c_int64, ctypes.c_int32,
                                              ctypes.POINTER(femPIC_projection)]),
    ("femPIC_last_timing", ctypes.c_int, [_P, _P, ctypes.c_int32]),
    ("femPIC_destroy", None, [_P]),
    ("femPIC_last_error", ctypes.c_char_p, [_P]),
    ("femPIC_measure_alu", ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]),
    ("femPIC_batch_create", ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(_P)]),
    ("femPIC_batch_step", ctypes.c_int, [_P, _P, ctypes.c_int32]),
    ("femPIC_batch_timing", ctypes.c_int, [_P, _P, ctypes.c_int32]),
    ("femPIC_batch_autotune", ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.POINTER(femPIC_batch_tuning)]),
    ("femPIC_batch_destroy", None, [_P]),
    ("femPIC_batch_last_error", ctypes.c_char_p, [_P]),
]

_lib = None


def load(path=LIB_PATH):
    """Load the library (once); raises ImportError if it was not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} not found: build it with paper_2111_12411_gb300.build.build() "
                          "(there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    for name, res, args in EXPORTS:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class FemPICError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def default_opts():
    o = femPIC_opts()
    load().femPIC_default_opts(ctypes.byref(o))
    return o


# ---- thin functions with the C names -----------------------------------------
def femPIC_create(xyz, tets, order, q, m, weight, x, v, tet, opts=None):
    lib = load()
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    tets = np.ascontiguousarray(tets, dtype=np.int32)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1, 3)
    tet = np.ascontiguousarray(tet, dtype=np.int32)
    mesh = femPIC_mesh(len(xyz), len(tets), _ptr(xyz), _ptr(tets))
    sp = femPIC_species(q, m, weight, len(x), _ptr(x), _ptr(v), _ptr(tet))
    h = ctypes.c_void_p()
    rc = lib.femPIC_create(ctypes.byref(mesh), order, ctypes.byref(sp),
                           ctypes.byref(opts) if opts is not None else None, ctypes.byref(h))
    if rc != FEMPIC_OK:
        msg = lib.femPIC_last_error(h).decode() if h.value else "create failed"
        if h.value:
            lib.femPIC_destroy(h)
        raise FemPICError(rc, msg)
    return h


def femPIC_create_ext(xyz, tets, order, species, bface_tag=None, opts=None):
    """species: list of dicts with q, m, weight, x, v, tet; bface_tag:
    int32[n_tets, 4] (0 PEC, 1 impedance) or None."""
    lib = load()
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    tets = np.ascontiguousarray(tets, dtype=np.int32)
    mesh = femPIC_mesh(len(xyz), len(tets), _ptr(xyz), _ptr(tets))
    keep = []
    arr = (femPIC_species * max(1, len(species)))()
    for k, spc in enumerate(species):
        x = np.ascontiguousarray(spc["x"], dtype=np.float64).reshape(-1, 3)
        v = np.ascontiguousarray(spc["v"], dtype=np.float64).reshape(-1, 3)
        tet = np.ascontiguousarray(spc["tet"], dtype=np.int32)
        keep += [x, v, tet]
        arr[k] = femPIC_species(spc["q"], spc["m"], spc["weight"], len(x), _ptr(x), _ptr(v), _ptr(tet))
    tag = None
    if bface_tag is not None:
        tag = np.ascontiguousarray(bface_tag, dtype=np.int32).reshape(len(tets), 4)
        keep.append(tag)
    h = ctypes.c_void_p()
    rc = lib.femPIC_create_ext(ctypes.byref(mesh), order, arr, len(species), _ptr(tag) if tag is not None else None,
                               ctypes.byref(opts) if opts is not None else None, ctypes.byref(h))
    if rc != FEMPIC_OK:
        msg = lib.femPIC_last_error(h).decode() if h.value else "create failed"
        if h.value:
            lib.femPIC_destroy(h)
        raise FemPICError(rc, msg)
    return h


def _check(h, rc):
    if rc != FEMPIC_OK:
        raise FemPICError(rc, load().femPIC_last_error(h).decode())


def femPIC_step(h, dt, n_steps=1):
    _check(h, load().femPIC_step(h, dt, n_steps))


def femPIC_step_async(h, dt, n_steps=1):
    _check(h, load().femPIC_step_async(h, dt, n_steps))


def femPIC_sync(h):
    _check(h, load().femPIC_sync(h))


def femPIC_get(h, what, out):
    _check(h, load().femPIC_get(h, QUANTITY.get(what, what), _ptr(out), out.nbytes))
    return out


def femPIC_set(h, what, arr):
    arr = np.ascontiguousarray(arr)
    _check(h, load().femPIC_set(h, QUANTITY.get(what, what), _ptr(arr), arr.nbytes))


def femPIC_get_device(h, what, dev_ptr, nbytes):
    _check(h, load().femPIC_get_device(h, QUANTITY.get(what, what), ctypes.c_void_p(dev_ptr), nbytes))


def femPIC_set_device(h, what, dev_ptr, nbytes):
    _check(h, load().femPIC_set_device(h, QUANTITY.get(what, what), ctypes.c_void_p(dev_ptr), nbytes))


def femPIC_apply(h, op, x, n_out):
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(n_out)
    _check(h, load().femPIC_apply(h, OPERATOR.get(op, op), _ptr(x), len(x), _ptr(y), len(y)))
    return y


def femPIC_eval_fields(h, x, tet):
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    tet = np.ascontiguousarray(tet, dtype=np.int32)
    E = np.empty_like(x)
    B = np.empty_like(x)
    _check(h, load().femPIC_eval_fields(h, len(x), _ptr(x), _ptr(tet), _ptr(E), _ptr(B)))
    return E, B


FEMPIC_PROBE_MAX_POINTS = 65536


def femPIC_eval_fields_noalloc(h, x, tet):
    """E and B at points, like femPIC_eval_fields, staged in the library's fixed
    device array instead of per-call allocations (at most
    FEMPIC_PROBE_MAX_POINTS points; calls that overlap on the GPU race)."""
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    tet = np.ascontiguousarray(tet, dtype=np.int32)
    E = np.empty_like(x)
    B = np.empty_like(x)
    _check(h, load().femPIC_eval_fields_noalloc(h, len(x), _ptr(x), _ptr(tet), _ptr(E), _ptr(B)))
    return E, B


def femPIC_set_injection(h, injectors, seed):
    """injectors: list of dicts with species, v_drift[3], v_sigma[3]."""
    arr = (femPIC_injector * max(1, len(injectors)))()
    for k, d in enumerate(injectors):
        arr[k].species = int(d["species"])
        for c in range(3):
            arr[k].v_drift[c] = float(d["v_drift"][c])
            arr[k].v_sigma[c] = float(d["v_sigma"][c])
    _check(h, load().femPIC_set_injection(h, arr, len(injectors), int(seed) & ((1 << 64) - 1)))


def femPIC_impressed_points(h):
    """[n_points, 3] quadrature points at which to evaluate an impressed B."""
    n = ctypes.c_int64(0)
    _check(h, load().femPIC_impressed_points(h, None, ctypes.byref(n)))
    xyz = np.empty((n.value, 3), dtype=np.float64)
    _check(h, load().femPIC_impressed_points(h, _ptr(xyz), ctypes.byref(n)))
    return xyz


def femPIC_set_impressed_B(h, B, constrained=True):
    """Project B [n_points, 3] (values at femPIC_impressed_points) onto W2;
    None clears it.  Returns the solver statistics as a dict."""
    st = femPIC_projection()
    if B is None:
        _check(h, load().femPIC_set_impressed_B(h, None, 0, int(constrained), ctypes.byref(st)))
    else:
        B = np.ascontiguousarray(B, dtype=np.float64).reshape(-1, 3)
        _check(h, load().femPIC_set_impressed_B(h, _ptr(B), len(B), int(constrained), ctypes.byref(st)))
    return {k: getattr(st, k) for k, _ in femPIC_projection._fields_}


def femPIC_get_info(h):
    info = femPIC_info()
    _check(h, load().femPIC_get_info(h, ctypes.byref(info)))
    return info


TIMING_KEYS = ("particle_ms", "field_ms", "launches", "sort_ms", "push_ms", "rhs_ms", "pcg_ms",
               "bupdate_ms", "cg_iterations")


def femPIC_last_timing(h):
    t = np.zeros(len(TIMING_KEYS))
    _check(h, load().femPIC_last_timing(h, _ptr(t), len(t)))
    return dict(zip(TIMING_KEYS, t.tolist()))


def femPIC_destroy(h):
    if h is not None and h.value:
        load().femPIC_destroy(h)


def femPIC_last_error(h):
    return load().femPIC_last_error(h).decode()


# ---- convenience wrapper --------------------------------------------------------
class Simulation:
    """One EM-FEMPIC instance on the GPU."""

    def __init__(self, xyz, tets, order, q, m, weight, x, v, tet, precision="fp64",
                 scheme="trapezoid", gamma=0.5, beta=0.25, cg_rtol=1e-12, cg_max_it=2000,
                 max_cross=4096, sort_period=1, B0=(0.0, 0.0, 0.0), rho_ion=0.0, es_init=True,
                 diagnostics=False, device=0, stream=None, species=None, bface_tag=None, push="boris"):
        o = default_opts()
        o.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
        o.scheme = SCHEME[scheme] if isinstance(scheme, str) else int(scheme)
        o.gamma, o.beta, o.cg_rtol = gamma, beta, cg_rtol
        o.cg_max_it, o.max_cross, o.sort_period = cg_max_it, max_cross, sort_period
        for k in range(3):
            o.B0[k] = B0[k]
        o.rho_ion = rho_ion
        o.es_init, o.diagnostics, o.device = int(es_init), int(diagnostics), device
        o.stream = stream
        o.push = PUSH[push] if isinstance(push, str) else int(push)
        if species is None and bface_tag is None:
            self.h = femPIC_create(xyz, tets, order, q, m, weight, x, v, tet, o)
        else:
            if species is None:
                species = [dict(q=q, m=m, weight=weight, x=x, v=v, tet=tet)]
            self.h = femPIC_create_ext(xyz, tets, order, species, bface_tag, o)
        self.info = femPIC_get_info(self.h)
        self.n_particles = int(self.info.n_particles)

    @classmethod
    def from_config(cls, cfg, **kw):
        """A config's instance, with its face tags and injectors when it has them."""
        args = dict(precision=cfg.get("precision", "fp64"), B0=cfg["B0"], rho_ion=cfg["rho_ion"])
        if cfg.get("bface_tag") is not None:
            args["bface_tag"] = cfg["bface_tag"]
        args.update(kw)
        sim = cls(cfg["xyz"], cfg["tets"], cfg["order"], cfg["q"], cfg["m"], cfg["weight"],
                  cfg["x"], cfg["v"], cfg["tet"], **args)
        if cfg.get("injectors") and args.get("bface_tag") is not None:
            sim.set_injection(cfg["injectors"], cfg["inject_seed"])
        return sim

    def _shape(self, what):
        i = self.info
        n1, n2, n0, npart = i.n1, i.n2, i.n0, self.n_particles
        return {"E": (n1, np.float64), "E_PREV": (n1, np.float64), "DG": (n1, np.float64),
                "DG_PREV": (n1, np.float64), "J": (n1, np.float64), "B": (n2, np.float64),
                "B_IMPRESSED": (n2, np.float64),
                "RHO": (n0, np.float64),
                "PHI": (n0, np.float64), "X": ((npart, 3), np.float64),
                "V": ((npart, 3), np.float64), "TET": (npart, np.int32), "SPECIES": (npart, np.int32),
                "NCROSS": (npart, np.int32), "HASH": (npart, np.uint64)}[what]

    def step(self, dt, n=1):
        femPIC_step(self.h, dt, n)

    def step_async(self, dt, n=1):
        femPIC_step_async(self.h, dt, n)

    def sync(self):
        femPIC_sync(self.h)

    def get(self, what, out=None):
        """The quantity as a new array, or written into ``out`` (e.g. pinned
        host memory: the copy then goes straight to it)."""
        shape, dt = self._shape(what)
        if out is None:
            return femPIC_get(self.h, what, np.empty(shape, dtype=dt))
        want = shape if isinstance(shape, tuple) else (shape,)
        if out.shape != want or out.dtype != np.dtype(dt) or not out.flags.c_contiguous:
            raise ValueError(f"{what}: out must be a C-contiguous {np.dtype(dt)} array of shape {want}")
        return femPIC_get(self.h, what, out)

    def set(self, what, arr):
        shape, dt = self._shape(what)
        arr = np.ascontiguousarray(arr, dtype=dt)
        if arr.shape != (shape if isinstance(shape, tuple) else (shape,)):
            raise ValueError(f"{what}: expected shape {shape}, got {arr.shape}")
        femPIC_set(self.h, what, arr)

    def diag(self):
        d = femPIC_diag()
        _check(self.h, load().femPIC_get(self.h, QUANTITY["DIAG"], ctypes.cast(ctypes.byref(d), ctypes.c_void_p),
                                         ctypes.sizeof(d)))
        return {k: getattr(d, k) for k, _ in femPIC_diag._fields_}

    def apply(self, op, x):
        i = self.info
        rows = {"M1": i.n1, "K": i.n1, "C": i.n2, "D": i.n1, "DT": i.n0, "M2": i.n2, "A": i.n1,
                "L": i.n0, "PI": i.n1, "PIT": 3 * i.n_nodes}[op]
        return femPIC_apply(self.h, op, x, rows)

    def eval_fields(self, x, tet):
        return femPIC_eval_fields(self.h, x, tet)

    def set_injection(self, injectors, seed):
        femPIC_set_injection(self.h, injectors, seed)

    def impressed_points(self):
        return femPIC_impressed_points(self.h)

    def set_impressed_B(self, B, constrained=True):
        """B: [n_points, 3] values at impressed_points(), or a callable of the
        points; None clears the impressed field."""
        if callable(B):
            B = B(self.impressed_points())
        return femPIC_set_impressed_B(self.h, B, constrained)

    def last_timing(self):
        return femPIC_last_timing(self.h)

    def close(self):
        femPIC_destroy(self.h)
        self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            if self.h is not None:
                self.close()
        except Exception:
            pass


# ---- batching ------------------------------------------------------------------
def femPIC_batch_create(handles):
    arr = (ctypes.c_void_p * len(handles))(*[h.value for h in handles])
    b = ctypes.c_void_p()
    rc = load().femPIC_batch_create(ctypes.cast(arr, ctypes.c_void_p), len(handles), ctypes.byref(b))
    if rc != FEMPIC_OK:
        msg = load().femPIC_batch_last_error(b).decode() if b.value else "batch create failed"
        if b.value:
            load().femPIC_batch_destroy(b)
        raise FemPICError(rc, msg)
    return b


def femPIC_batch_step(b, dts, n_steps=1):
    dts = np.ascontiguousarray(dts, dtype=np.float64)
    rc = load().femPIC_batch_step(b, _ptr(dts), n_steps)
    if rc != FEMPIC_OK:
        raise FemPICError(rc, load().femPIC_batch_last_error(b).decode())


def femPIC_batch_timing(b):
    t = np.zeros(4)
    load().femPIC_batch_timing(b, _ptr(t), 4)
    return dict(zip(("ms", "launches_per_step", "graph", "cg_ctas"), t.tolist()))


def femPIC_batch_autotune(b, dts, steps_per_candidate=2):
    dts = np.ascontiguousarray(dts, dtype=np.float64)
    t = femPIC_batch_tuning()
    rc = load().femPIC_batch_autotune(b, _ptr(dts), int(steps_per_candidate), ctypes.byref(t))
    if rc != FEMPIC_OK:
        raise FemPICError(rc, femPIC_batch_last_error(b))
    return {k: getattr(t, k) for k, _ in femPIC_batch_tuning._fields_}


def femPIC_batch_destroy(b):
    if b is not None and b.value:
        load().femPIC_batch_destroy(b)


def femPIC_batch_last_error(b):
    return load().femPIC_batch_last_error(b).decode()


class Batch:
    """Several Simulations advanced together (one launch per kernel for all)."""

    def __init__(self, sims):
        self.sims = list(sims)
        self.b = femPIC_batch_create([s.h for s in self.sims])

    def step(self, dts, n=1):
        femPIC_batch_step(self.b, dts, n)

    def timing(self):
        return femPIC_batch_timing(self.b)

    def autotune(self, dts, steps_per_candidate=2):
        """Pick the launch shapes of the batched kernels by timing real steps."""
        return femPIC_batch_autotune(self.b, dts, steps_per_candidate)

    def close(self):
        femPIC_batch_destroy(self.b)
        self.b = None

    def __del__(self):
        try:
            if self.b is not None:
                self.close()
        except Exception:
            pass


ALU_KIND = {"fp64_fma": 0, "fp32_fma": 1, "fp64_div": 2}


def measure_alu(kind, device=0):
    """Arithmetic throughput of the device (operations per second of the whole
    GPU; one fused multiply-add or one division counts as one operation)."""
    out = ctypes.c_double(0.0)
    rc = load().femPIC_measure_alu(int(device), ALU_KIND[kind], ctypes.byref(out))
    if rc != 0:
        raise FemPICError(rc, f"femPIC_measure_alu({kind}) failed")
    return out.value
