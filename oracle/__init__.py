"""FP64 CPU oracle for the PD / MTS-Arlequin method (test infrastructure only).

This package is the reference that the CUDA library is checked against. Only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it. It shares no code with the CUDA library and never
calls it. The arithmetic lives in the C sources next to this file; this module
only compiles them with gcc (``-O2 -ffp-contract=off``, no fast-math) and
marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liborc.so")
_SOURCES = ["pd_oracle.c"]
_lock = threading.Lock()
_lib = None

MICRO_POWER, MICRO_EXP = 0, 1
FORCE_LINEAR, FORCE_PMB = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liborc.so`` (plain gcc, FP64)."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES if os.path.exists(os.path.join(_HERE, s))]
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB):
        newest = max(os.path.getmtime(s) for s in srcs + [os.path.join(_HERE, "oracle.h")])
        if os.path.getmtime(_LIB) >= newest:
            return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    base = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-o", tmp]
    # OpenMP spreads the node loops over host threads (same bits for any count);
    # without it the oracle runs on one thread
    r = subprocess.run([*base, "-fopenmp", *srcs, "-lm"], cwd=_HERE, capture_output=True, text=True)
    if r.returncode != 0:
        subprocess.run([*base, *srcs, "-lm"], check=True, cwd=_HERE)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _declare(_lib)
        return _lib


class PDParams(C.Structure):
    _fields_ = [("dim", C.c_int32), ("micro_kind", C.c_int32), ("force_kind", C.c_int32),
                ("breaking", C.c_int32), ("n", C.c_int64), ("c", C.c_double), ("l", C.c_double),
                ("s0", C.c_double), ("rho", C.c_double), ("dt", C.c_double)]


_P = C.c_void_p


def _declare(L):
    L.orc_family.argtypes = [C.c_int, C.c_int64, _P, C.c_double, _P, _P]
    L.orc_family.restype = C.c_int
    L.orc_precrack.argtypes = [C.c_int, C.c_int64, _P, _P, _P, C.c_int, _P, _P]
    L.orc_precrack.restype = C.c_int64
    L.orc_stretch_literal.argtypes = [C.c_int, _P, _P]
    L.orc_stretch_literal.restype = C.c_double
    L.orc_pd_forces.argtypes = [C.POINTER(PDParams), _P, _P, _P, _P, _P, _P, _P, _P]
    L.orc_pd_forces.restype = C.c_int64
    L.orc_pd_run.argtypes = [C.POINTER(PDParams), _P, _P, _P, _P, _P, _P, _P, _P, _P,
                             C.c_double, C.c_int, _P, _P, _P, C.c_int64]
    L.orc_pd_run.restype = C.c_int64
    L.orc_damage.argtypes = [C.c_int64, _P, _P, _P, _P, _P]
    L.orc_damage.restype = None
    L.orc_strain_energy.argtypes = [C.POINTER(PDParams), _P, _P, _P, _P, _P, _P, _P]
    L.orc_strain_energy.restype = C.c_double
    L.orc_kinetic_energy.argtypes = [C.POINTER(PDParams), _P, _P, _P]
    L.orc_kinetic_energy.restype = C.c_double
    L.orc_set_threads.argtypes = [C.c_int]
    L.orc_set_threads.restype = C.c_int
    L.orc_set_threads(1)


def set_threads(n: int) -> int:
    """Host threads of the oracle's node loops (n <= 0: every core). The result
    does not depend on it. Returns the count in effect (1 without OpenMP)."""
    return int(lib().orc_set_threads(int(n)))


def _ptr(a):
    return None if a is None else a.ctypes.data


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


@dataclass
class PD:
    """Inputs of one PD subdomain, as the oracle sees them.

    X: (dim, n) reference positions [m]; V: (n,) nodal volumes [m^3];
    c, s0, rho: micromodulus constant, critical stretch, density;
    micro: MICRO_POWER (c/|xi|^3) or MICRO_EXP (c exp(-|xi|/l)).
    """
    X: np.ndarray
    V: np.ndarray
    delta: float
    c: float
    s0: float
    rho: float
    dt: float
    micro: int = MICRO_POWER
    l: float = 0.0
    force: int = FORCE_LINEAR
    breaking: bool = True

    def __post_init__(self):
        self.X = np.ascontiguousarray(self.X, dtype=np.float64)
        self.V = np.ascontiguousarray(np.broadcast_to(self.V, (self.X.shape[1],)), dtype=np.float64)

    @property
    def dim(self):
        return self.X.shape[0]

    @property
    def n(self):
        return self.X.shape[1]

    def params(self, breaking=None) -> PDParams:
        b = self.breaking if breaking is None else breaking
        return PDParams(self.dim, self.micro, self.force, int(bool(b)), self.n, self.c, self.l,
                        self.s0, self.rho, self.dt)


def family(X: np.ndarray, delta: float):
    """CSR family H_delta (closed ball), rows sorted ascending."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    dim, n = X.shape
    L = lib()
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    if L.orc_family(dim, n, _ptr(X), delta, _ptr(row_ptr), None) != 0:
        raise ValueError("orc_family failed")
    col = np.zeros(max(int(row_ptr[-1]), 1), dtype=np.int32)
    if L.orc_family(dim, n, _ptr(X), delta, _ptr(row_ptr), _ptr(col)) != 0:
        raise ValueError("orc_family failed")
    return row_ptr, col[: int(row_ptr[-1])]


def precrack(P: np.ndarray, row_ptr, col, cuts, mu=None):
    """Cut bonds crossing axis-aligned cuts given in integer lattice units.

    P: (dim, n) int64 node coordinates; cuts: iterable of
    (normal_axis, level, along_axis, lo, hi). Returns (mu uint8, n_cut).
    """
    P = np.ascontiguousarray(P, dtype=np.int64)
    dim, n = P.shape
    if mu is None:
        mu = np.ones(len(col), dtype=np.uint8)
    cuts = np.ascontiguousarray(np.asarray(list(cuts), dtype=np.int64).reshape(-1, 5))
    cnt = lib().orc_precrack(dim, n, _ptr(P), _ptr(row_ptr), _ptr(col), len(cuts), _ptr(cuts), _ptr(mu))
    return mu, int(cnt)


def stretch_literal(xi, eta) -> float:
    xi = _f64(xi)
    eta = _f64(eta)
    return lib().orc_stretch_literal(len(xi), _ptr(xi), _ptr(eta))


def pd_forces(pd: PD, row_ptr, col, mu, u, alpha=None, breaking=None):
    """Force density (dim, n) at displacement u; updates mu in place if breaking."""
    u = _f64(u).reshape(pd.dim, pd.n)
    f = np.zeros_like(u)
    p = pd.params(breaking)
    alpha = _f64(alpha)
    nb = lib().orc_pd_forces(C.byref(p), _ptr(pd.X), _ptr(pd.V), _ptr(row_ptr), _ptr(col), _ptr(mu),
                             _ptr(alpha), _ptr(u), _ptr(f))
    return f, int(nb)


def pd_run(pd: PD, row_ptr, col, mu, u, v, a, nsteps, *, alpha=None, b=None, g=None, theta=None,
           theta_init=0.0, init=False, breaking=None):
    """Advance (u, v, a) in place by nsteps velocity-Verlet steps. Returns bonds broken."""
    for arr in (u, v, a):
        assert arr.dtype == np.float64 and arr.flags.c_contiguous and arr.shape == (pd.dim, pd.n)
    p = pd.params(breaking)
    alpha, b, g = _f64(alpha), _f64(b), _f64(g)
    theta = None if theta is None else _f64(theta)
    if theta is not None:
        assert theta.shape[0] >= nsteps
    nb = lib().orc_pd_run(C.byref(p), _ptr(pd.X), _ptr(pd.V), _ptr(row_ptr), _ptr(col), _ptr(mu),
                          _ptr(alpha), _ptr(b), _ptr(g), _ptr(theta), float(theta_init), int(bool(init)),
                          _ptr(u), _ptr(v), _ptr(a), int(nsteps))
    if nb < 0:
        raise ValueError("orc_pd_run failed")
    return int(nb)


def damage(pd: PD, row_ptr, col, mu):
    phi = np.zeros(pd.n)
    lib().orc_damage(pd.n, _ptr(pd.V), _ptr(row_ptr), _ptr(col), _ptr(mu), _ptr(phi))
    return phi


def strain_energy(pd: PD, row_ptr, col, mu, u, alpha=None) -> float:
    u = _f64(u)
    alpha = _f64(alpha)
    p = pd.params()
    return lib().orc_strain_energy(C.byref(p), _ptr(pd.X), _ptr(pd.V), _ptr(row_ptr), _ptr(col),
                                   _ptr(mu), _ptr(alpha), _ptr(u))


def kinetic_energy(pd: PD, v, alpha=None) -> float:
    v = _f64(v)
    alpha = _f64(alpha)
    p = pd.params()
    return lib().orc_kinetic_energy(C.byref(p), _ptr(pd.V), _ptr(alpha), _ptr(v))


def crack_tip(X, phi, normal: int, level: float, along: int, band: float, threshold: float = 0.35):
    """Extreme crack-tip positions of a damage field (damage as in Eq. 5).

    The paper does not define a crack tip; the reading taken here: among the
    nodes whose damage is at least `threshold` and whose distance to the crack
    plane x[normal] = level is at most `band`, the smallest and the largest
    coordinate along axis `along`. Returns (lo, hi), or (nan, nan) when no node
    qualifies. The default threshold sits below 11/28 (2D) and 47/122 (3D),
    the damage of a node next to a fully separated lattice plane at
    delta = 3.015 dx, and above 6/28, that of the second row. A plain loop
    over the nodes: for the small cases of the tests.
    """
    X = np.asarray(X, dtype=np.float64)
    phi = np.asarray(phi, dtype=np.float64)
    lo, hi = float("inf"), float("-inf")
    for i in range(X.shape[1]):
        if phi[i] >= threshold and abs(X[normal, i] - level) <= band:
            x = float(X[along, i])
            if x < lo:
                lo = x
            if x > hi:
                hi = x
    if hi == float("-inf"):
        return float("nan"), float("nan")
    return lo, hi
