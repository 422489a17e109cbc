"""Thin ctypes binding of the pdmts C ABI (include/pdmts.h).

Function names match the C entry points; this module only marshals arguments
(numpy arrays or torch tensors in, numpy arrays out) and turns negative status
codes into exceptions. Every step of the computation runs in libpdmts.so. If
the library has not been built, load() raises instead of falling back to
anything else. PyTorch provides the CUDA stream and, through
pdmts_set_allocator, the device memory (its caching allocator).
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libpdmts.so")

PDMTS_OK = 0
ERRORS = {-1: "PDMTS_ERR_ARG", -2: "PDMTS_ERR_MASS", -3: "PDMTS_ERR_STABILITY", -4: "PDMTS_ERR_CUDA",
          -5: "PDMTS_ERR_TIMEOUT", -6: "PDMTS_ERR_STATE", -7: "PDMTS_ERR_NOMEM", -8: "PDMTS_ERR_UNSUPPORTED"}
PDMTS_FP64, PDMTS_FP32_BULK, PDMTS_FP32_BULK_SELL = 0, 1, 2
PDMTS_MICRO_POWER, PDMTS_MICRO_EXP = 0, 1
PDMTS_FORCE_LINEAR, PDMTS_FORCE_PMB = 0, 1
PDMTS_WEIGHT_CONSTANT, PDMTS_WEIGHT_LINEAR, PDMTS_WEIGHT_CUBIC = 0, 1, 2
PDMTS_LATTICE_TILES, PDMTS_LATTICE_TILE_AUTO = 10, -1
PDMTS_PRODUCT_AUTO, PDMTS_PRODUCT_FP64 = 0, 1


class PdmtsError(RuntimeError):
    def __init__(self, code, where, msg):
        super().__init__(f"{where}: {ERRORS.get(code, code)}: {msg}")
        self.code = code


class PDInfo(C.Structure):
    _fields_ = [("dim", C.c_int32), ("precision", C.c_int32), ("n", C.c_int64), ("n_bonds", C.c_int64),
                ("n_slots", C.c_int64), ("max_degree", C.c_int32), ("on_lattice", C.c_int32),
                ("layout", C.c_int32), ("lattice_nx", C.c_int32), ("lattice_ny", C.c_int32),
                ("lattice_tile", C.c_int32), ("lattice_h", C.c_double), ("steps_done", C.c_int64), ("device_bytes", C.c_int64),
                ("lattice_nz", C.c_int32), ("link_tile", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("pd_substeps", C.c_int64), ("bond_updates", C.c_int64), ("coarse_steps", C.c_int64),
                ("bonds_broken", C.c_int64), ("kernel_launches", C.c_int64), ("graph_launches", C.c_int64)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)

_lib = None
_lock = threading.Lock()
_V, _I, _I64, _D = C.c_void_p, C.c_int, C.c_int64, C.c_double

# (name, restype, argtypes) for every function declared in include/pdmts.h
SIGNATURES = [
    ("pdmts_ctx_create", _I, [C.POINTER(_V), _I, _V]),
    ("pdmts_ctx_destroy", _I, [_V]),
    ("pdmts_last_error", C.c_char_p, []),
    ("pdmts_set_allocator", _I, [_V, ALLOC_FN, FREE_FN, _V]),
    ("pdmts_ctx_synchronize", _I, [_V]),
    ("pd_create", _I, [_V, _I, _I64, _V, _V, _D, _D, _I, _D, _D, _D, _D, _I, C.POINTER(_V)]),
    ("pd_destroy", _I, [_V]),
    ("pd_set_precrack", _I, [_V, _I, _V]),
    ("pd_set_body_force", _I, [_V, _V]),
    ("pd_set_state", _I, [_V, _V, _V]),
    ("pd_set_weights", _I, [_V, _V]),
    ("pd_set_breaking", _I, [_V, _I]),
    ("pd_set_force_law", _I, [_V, _I]),
    ("pd_set_lattice_tile", _I, [_V, _I]),
    ("pd_info", _I, [_V, C.POINTER(PDInfo)]),
    ("pd_read_displacement", _I, [_V, _V]),
    ("pd_read_velocity", _I, [_V, _V]),
    ("pd_read_acceleration", _I, [_V, _V]),
    ("pd_read_damage", _I, [_V, _V]),
    ("pd_read_damage_static", _I, [_V, _V]),
    ("pd_read_bond_status", _I, [_V, _V, C.POINTER(_I64)]),
    ("pd_read_family", _I, [_V, _V, _V]),
    ("mts_set_time", _I, [_V, _D, _I, _D, _D, _I]),
    ("mts_advance", _I, [_V, _I64]),
    ("fem_create", _I, [_V, _I, _I64, _V, _I64, _I, _V, _D, _D, _D, _D, C.POINTER(_V)]),
    ("fem_set_traction", _I, [_V, _I64, _V, _V]),
    ("fem_set_state", _I, [_V, _V, _V]),
    ("fem_set_fixed", _I, [_V, _I64, _V]),
    ("fem_destroy", _I, [_V]),
    ("fem_read_displacement", _I, [_V, _V]),
    ("fem_read_velocity", _I, [_V, _V]),
    ("fem_read_acceleration", _I, [_V, _V]),
    ("arlequin_bind", _I, [_V, _V, _V, _I, _I, _V, C.POINTER(_V)]),
    ("arlequin_destroy", _I, [_V]),
    ("arlequin_read_lambda", _I, [_V, _V, C.POINTER(_I64)]),
    ("arlequin_constraint_residual", _I, [_V, C.POINTER(_D), C.POINTER(_D)]),
    ("arlequin_info", _I, [_V, _V]),
    ("arlequin_set_multiplier_product", _I, [_V, _I]),
    ("mts_batch_create", _I, [_I, C.POINTER(_V), C.POINTER(_V)]),
    ("mts_batch_advance", _I, [_V, _I64]),
    ("mts_batch_info", _I, [_V, _V]),
    ("mts_batch_destroy", _I, [_V]),
    ("pdmts_set_timing", _I, [_V, _I]),
    ("pdmts_set_debug_poll_limit", _I, [_V, _I64]),
    ("pdmts_get_timing", _I, [_V, C.POINTER(_D), C.POINTER(_I64)]),
    ("mts_get_phase_timing", _I, [_V, C.POINTER(_D), C.POINTER(_I64)]),
    ("pdmts_get_stats", _I, [_V, C.POINTER(Stats)]),
    ("mts_state_size", _I, [_V, C.POINTER(_I64)]),
    ("mts_state_save", _I, [_V, _V, _I64]),
    ("mts_state_load", _I, [_V, _V, _I64]),
]


def load():
    """Load libpdmts.so (built by paper_2403_03605_gb300.build). No fallback."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2403_03605_gb300.build.build()")
            lib = C.CDLL(LIB_PATH)
            for name, res, args in SIGNATURES:
                fn = getattr(lib, name, None)
                if fn is None:
                    continue
                fn.restype = res
                fn.argtypes = args
            _lib = lib
        return _lib


def _check(code, where):
    if code != PDMTS_OK:
        msg = load().pdmts_last_error()
        raise PdmtsError(code, where, msg.decode() if msg else "")


def _ptr(a):
    """Address of a numpy array or torch tensor (host or device), or None."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous()
        return a.data_ptr()
    assert a.flags.c_contiguous
    return a.ctypes.data


def _f64(a):
    if a is None or hasattr(a, "data_ptr"):
        return a
    return np.ascontiguousarray(a, dtype=np.float64)


# ------------------------------------------------------------------ context
class _TorchAllocator:
    """PyTorch's caching allocator exposed through pdmts_set_allocator."""

    def __init__(self, device, stream):
        import torch
        self.torch = torch
        self.device = device
        self.stream = stream
        self.alloc = ALLOC_FN(self._alloc)
        self.free = FREE_FN(self._free)

    def _alloc(self, size, user):
        try:
            return self.torch.cuda.caching_allocator_alloc(int(size), self.device, self.stream)
        except Exception:
            return None

    def _free(self, ptr, user):
        self.torch.cuda.caching_allocator_delete(ptr)


_allocators = {}


def pdmts_ctx_create(device=0, stream=None, torch_allocator=True):
    """Create a context. `stream` is a cudaStream_t integer (default: torch's
    current stream on `device`); with torch_allocator the library draws its
    device memory from PyTorch's caching allocator."""
    L = load()
    if stream is None:
        import torch
        stream = torch.cuda.current_stream(device).cuda_stream
    h = _V()
    _check(L.pdmts_ctx_create(C.byref(h), int(device), _V(stream) if stream else None), "pdmts_ctx_create")
    if torch_allocator:
        al = _TorchAllocator(device, stream)
        _check(L.pdmts_set_allocator(h, al.alloc, al.free, None), "pdmts_set_allocator")
        _allocators[h.value] = al
    return h.value


def pdmts_ctx_destroy(ctx):
    _check(load().pdmts_ctx_destroy(ctx), "pdmts_ctx_destroy")
    _allocators.pop(ctx, None)


def pdmts_last_error():
    m = load().pdmts_last_error()
    return m.decode() if m else ""


def pdmts_ctx_synchronize(ctx):
    _check(load().pdmts_ctx_synchronize(ctx), "pdmts_ctx_synchronize")


def pdmts_get_stats(ctx):
    s = Stats()
    _check(load().pdmts_get_stats(ctx, C.byref(s)), "pdmts_get_stats")
    return {k: getattr(s, k) for k, _ in Stats._fields_}


def pdmts_set_timing(ctx, enabled):
    _check(load().pdmts_set_timing(ctx, int(bool(enabled))), "pdmts_set_timing")


def pdmts_set_debug_poll_limit(ctx, polls):
    """Poll limit of each lattice tile's first tensor-copy wait (tests of the
    give-up path; negative restores the default)."""
    _check(load().pdmts_set_debug_poll_limit(ctx, int(polls)), "pdmts_set_debug_poll_limit")


def pdmts_get_timing(ctx):
    """(summed substep-chain milliseconds, substeps timed) since the last call."""
    ms, cnt = _D(), _I64()
    _check(load().pdmts_get_timing(ctx, C.byref(ms), C.byref(cnt)), "pdmts_get_timing")
    return ms.value, cnt.value


MTS_PHASES = ("free", "interface", "link", "correction", "step")


def mts_get_phase_timing(ctx):
    """({phase: summed milliseconds}, coarse steps timed) since the last call."""
    ms = (_D * 5)()
    cnt = _I64()
    _check(load().mts_get_phase_timing(ctx, ms, C.byref(cnt)), "mts_get_phase_timing")
    return dict(zip(MTS_PHASES, list(ms))), cnt.value


# ------------------------------------------------------------------------ PD
def pd_create(ctx, X, *, horizon, c, s0, rho, vol=None, vol_uniform=0.0, micro_kind=PDMTS_MICRO_POWER, l=0.0,
              precision=PDMTS_FP64):
    """X: (dim, n) reference positions. Returns the PD handle."""
    X = _f64(X)
    dim, n = X.shape
    vol = _f64(vol)
    h = _V()
    _check(load().pd_create(ctx, int(dim), int(n), _ptr(X), _ptr(vol), float(vol_uniform), float(horizon),
                            int(micro_kind), float(c), float(l), float(s0), float(rho), int(precision),
                            C.byref(h)), "pd_create")
    return h.value


def pd_destroy(pd):
    _check(load().pd_destroy(pd), "pd_destroy")


def pd_set_precrack(pd, cuts):
    """cuts: iterable of (normal axis, level, along axis, lo, hi) in metres."""
    arr = np.ascontiguousarray(np.asarray(list(cuts), dtype=np.float64).reshape(-1, 5))
    _check(load().pd_set_precrack(pd, len(arr), _ptr(arr) if len(arr) else None), "pd_set_precrack")


def pd_set_body_force(pd, b):
    b = _f64(b)
    _check(load().pd_set_body_force(pd, _ptr(b)), "pd_set_body_force")


def pd_set_state(pd, u=None, v=None):
    u, v = _f64(u), _f64(v)
    _check(load().pd_set_state(pd, _ptr(u), _ptr(v)), "pd_set_state")


def pd_set_weights(pd, alpha):
    alpha = _f64(alpha)
    _check(load().pd_set_weights(pd, _ptr(alpha)), "pd_set_weights")


def pd_set_breaking(pd, enabled):
    _check(load().pd_set_breaking(pd, int(bool(enabled))), "pd_set_breaking")


def pd_set_force_law(pd, kind):
    _check(load().pd_set_force_law(pd, int(kind)), "pd_set_force_law")


def pd_set_lattice_tile(pd, tile):
    _check(load().pd_set_lattice_tile(pd, int(tile)), "pd_set_lattice_tile")


def pd_info(pd):
    s = PDInfo()
    _check(load().pd_info(pd, C.byref(s)), "pd_info")
    return {k: getattr(s, k) for k, _ in PDInfo._fields_}


def _read(fn, pd, shape, out=None, dtype=np.float64):
    if out is None:
        out = np.empty(shape, dtype=dtype)
    _check(getattr(load(), fn)(pd, _ptr(out)), fn)
    return out


def pd_read_displacement(pd, out=None):
    i = pd_info(pd)
    return _read("pd_read_displacement", pd, (i["dim"], i["n"]), out)


def pd_read_velocity(pd, out=None):
    i = pd_info(pd)
    return _read("pd_read_velocity", pd, (i["dim"], i["n"]), out)


def pd_read_acceleration(pd, out=None):
    i = pd_info(pd)
    return _read("pd_read_acceleration", pd, (i["dim"], i["n"]), out)


def pd_read_damage(pd, out=None):
    i = pd_info(pd)
    return _read("pd_read_damage", pd, (i["n"],), out)


def pd_read_damage_static(pd, out=None):
    """Damage through the non-allocating entry point (static device scratch)."""
    i = pd_info(pd)
    return _read("pd_read_damage_static", pd, (i["n"],), out)


def pd_read_bond_status(pd):
    i = pd_info(pd)
    mu = np.empty(i["n_bonds"], dtype=np.uint8)
    cnt = _I64()
    _check(load().pd_read_bond_status(pd, _ptr(mu), C.byref(cnt)), "pd_read_bond_status")
    return mu, cnt.value


def pd_read_family(pd):
    i = pd_info(pd)
    rp = np.empty(i["n"] + 1, dtype=np.int64)
    col = np.empty(max(i["n_bonds"], 1), dtype=np.int32)
    _check(load().pd_read_family(pd, _ptr(rp), _ptr(col)), "pd_read_family")
    return rp, col[: i["n_bonds"]]


# ------------------------------------------------------------------- time
def mts_set_time(ctx, dt_pd, m_ratio=1, gamma_fe=0.5, beta_fe=0.25, check_stability=True):
    _check(load().mts_set_time(ctx, float(dt_pd), int(m_ratio), float(gamma_fe), float(beta_fe),
                               int(bool(check_stability))), "mts_set_time")


def mts_advance(ctx, n_coarse):
    _check(load().mts_advance(ctx, int(n_coarse)), "mts_advance")


# --------------------------------------------------------- FE and coupling
class ArlInfo(C.Structure):
    _fields_ = [("n_lambda", C.c_int64), ("n_overlap_pd", C.c_int64), ("fe_dofs", C.c_int64),
                ("colors", C.c_int64), ("rebuilds", C.c_int64), ("cheb_iterations", C.c_int64),
                ("device_bytes", C.c_int64)]


def fem_create(ctx, X, conn, *, E, nu, rho, thickness):
    """X: (dim, n) node positions; conn: (ne, 4) Q4 (2D) or (ne, 8) Hex8 (3D) int32 connectivity."""
    X = _f64(X)
    conn = np.ascontiguousarray(conn, dtype=np.int32)
    h = _V()
    _check(load().fem_create(ctx, int(X.shape[0]), int(X.shape[1]), _ptr(X), int(conn.shape[0]),
                             int(conn.shape[1]), _ptr(conn), float(E), float(nu), float(rho), float(thickness),
                             C.byref(h)), "fem_create")
    return h.value


def fem_set_traction(fe, faces, traction):
    faces = np.ascontiguousarray(faces, dtype=np.int32)
    traction = _f64(traction)
    _check(load().fem_set_traction(fe, int(faces.shape[0]), _ptr(faces), _ptr(traction)), "fem_set_traction")


def fem_set_fixed(fe, dofs):
    """dofs: FE dof ids d * n_nodes + node held at zero (Dirichlet)."""
    d = np.ascontiguousarray(np.asarray(dofs, dtype=np.int64).reshape(-1))
    _check(load().fem_set_fixed(fe, len(d), _ptr(d) if len(d) else None), "fem_set_fixed")


def fem_set_state(fe, u=None, v=None):
    u, v = _f64(u), _f64(v)
    _check(load().fem_set_state(fe, _ptr(u), _ptr(v)), "fem_set_state")


def fem_destroy(fe):
    _check(load().fem_destroy(fe), "fem_destroy")


def _fe_read(fn, fe, ndof, out=None):
    if out is None:
        out = np.empty(ndof, dtype=np.float64)
    _check(getattr(load(), fn)(fe, _ptr(out)), fn)
    return out


def fem_read_displacement(fe, ndof, out=None):
    return _fe_read("fem_read_displacement", fe, ndof, out)


def fem_read_velocity(fe, ndof, out=None):
    return _fe_read("fem_read_velocity", fe, ndof, out)


def fem_read_acceleration(fe, ndof, out=None):
    return _fe_read("fem_read_acceleration", fe, ndof, out)


def arlequin_bind(ctx, pd, fe, weight_kind, bands):
    """bands: iterable of (axis, lo, hi, fe_side, 0)."""
    b = np.ascontiguousarray(np.asarray(list(bands), dtype=np.float64).reshape(-1, 5))
    h = _V()
    _check(load().arlequin_bind(ctx, pd, fe, int(weight_kind), len(b), _ptr(b), C.byref(h)), "arlequin_bind")
    return h.value


def arlequin_destroy(arl):
    _check(load().arlequin_destroy(arl), "arlequin_destroy")


def arlequin_info(arl):
    s = ArlInfo()
    _check(load().arlequin_info(arl, C.byref(s)), "arlequin_info")
    return {k: getattr(s, k) for k, _ in ArlInfo._fields_}


class BatchInfo(C.Structure):
    _fields_ = [("n_members", C.c_int32), ("lattice_tile", C.c_int32), ("rounds", C.c_int64),
                ("work_items", C.c_int64), ("batched_launches", C.c_int64), ("kernel_launches", C.c_int64),
                ("last_round_ms", C.c_double * 5)]


def mts_batch_create(members):
    """A batch over the contexts `members` (each with a coupled problem bound)."""
    arr = (_V * len(members))(*members)
    out = _V()
    _check(load().mts_batch_create(len(members), arr, C.byref(out)), "mts_batch_create")
    return out


def mts_batch_advance(batch, n_rounds):
    _check(load().mts_batch_advance(batch, int(n_rounds)), "mts_batch_advance")


def mts_batch_info(batch):
    s = BatchInfo()
    _check(load().mts_batch_info(batch, C.byref(s)), "mts_batch_info")
    d = {k: getattr(s, k) for k, _ in BatchInfo._fields_}
    d["last_round_ms"] = list(d["last_round_ms"])
    return d


def mts_batch_destroy(batch):
    _check(load().mts_batch_destroy(batch), "mts_batch_destroy")


def arlequin_set_multiplier_product(arl, kind):
    """AUTO: FP32-pair product of lambda_m = (-H)^-1 y in FP32-bulk, FP64 in FP64; FP64: always FP64."""
    _check(load().arlequin_set_multiplier_product(arl, int(kind)), "arlequin_set_multiplier_product")


def arlequin_read_lambda(arl):
    n = arlequin_info(arl)["n_lambda"]
    lam = np.empty(n, dtype=np.float64)
    cnt = _I64()
    _check(load().arlequin_read_lambda(arl, _ptr(lam), C.byref(cnt)), "arlequin_read_lambda")
    return lam


def arlequin_constraint_residual(arl):
    r, f = _D(), _D()
    _check(load().arlequin_constraint_residual(arl, C.byref(r), C.byref(f)), "arlequin_constraint_residual")
    return r.value, f.value


# ------------------------------------------------------ checkpoint / resume
def mts_state_save(ctx):
    """The context's time-stepping state as a uint8 image (host memory)."""
    n = _I64()
    _check(load().mts_state_size(ctx, C.byref(n)), "mts_state_size")
    img = np.empty(n.value, dtype=np.uint8)
    _check(load().mts_state_save(ctx, _ptr(img), n.value), "mts_state_save")
    return img


def mts_state_load(ctx, image):
    """Restore an image from mts_state_save into a context with the same set-up."""
    img = np.ascontiguousarray(image, dtype=np.uint8)
    _check(load().mts_state_load(ctx, _ptr(img), img.size), "mts_state_load")
