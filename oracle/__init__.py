"""RES-PCA oracle -- TEST INFRASTRUCTURE ONLY.

A plain, slow, single-threaded FP64 CPU statement of the RES-PCA method
(Peng et al., arXiv 1904.07497) written in C (``respca_oracle.c``) and loaded
here with ctypes.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
The product library (``paper_1904_07497_gb300``) never imports, links or
executes anything in this folder, and this folder never imports the product.

Every function mirrors one passage of the paper (see the C file for the
citations).  Arrays are numpy, column-major (Fortran order) d x n, float64.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_SRC = os.path.join(_HERE, "respca_oracle.c")

_lib = None

CFLAGS = ["-O3", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-Wall", "-Wextra"]


def compiler_version() -> str:
    """First line of `gcc --version` (recorded beside oracle timings)."""
    try:
        out = subprocess.run(["gcc", "--version"], capture_output=True, text=True, check=True)
        return out.stdout.splitlines()[0].strip()
    except (OSError, subprocess.CalledProcessError):
        return "unknown"


def build(force: bool = False) -> str:
    """Compile the oracle with gcc: -O3, ISO C11, no FMA contraction and no
    -march=native, so that the x86_64 and aarch64 builds round every
    operation the same way and give the same bits."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)
            and os.path.getmtime(_LIB) >= os.path.getmtime(os.path.join(_HERE, "respca_oracle.h"))):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.run(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"], check=True)
    os.replace(tmp, _LIB)
    return _LIB


class OracleStats(ctypes.Structure):
    _fields_ = [
        ("iters", ctypes.c_int32),
        ("converged", ctypes.c_int32),
        ("err", ctypes.c_double),
        ("err_resid", ctypes.c_double),
        ("err_dL", ctypes.c_double),
        ("err_dS", ctypes.c_double),
        ("rho_final", ctypes.c_double),
        ("label_changes", ctypes.c_int64),
        ("lloyd_steps", ctypes.c_int64),
        ("init_lloyd_steps", ctypes.c_int32),
    ]


_D = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.POINTER(ctypes.c_int32)
_I64 = ctypes.POINTER(ctypes.c_int64)
_U8 = ctypes.POINTER(ctypes.c_uint8)
_U64 = ctypes.POINTER(ctypes.c_uint64)


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.oracle_splitmix64.argtypes = [_U64]
        lib.oracle_splitmix64.restype = ctypes.c_uint64
        lib.oracle_uniform.argtypes = [_U64]
        lib.oracle_uniform.restype = ctypes.c_double
        lib.oracle_fro.argtypes = [_D, ctypes.c_int64]
        lib.oracle_fro.restype = ctypes.c_double
        lib.oracle_column_norms.argtypes = [_D, ctypes.c_int64, ctypes.c_int64, _D]
        lib.oracle_column_norms.restype = None
        lib.oracle_cluster_means.argtypes = [_D, ctypes.c_int64, ctypes.c_int64, _I32,
                                             ctypes.c_int32, _D, _I64]
        lib.oracle_cluster_means.restype = None
        lib.oracle_l_step.argtypes = [_D, _D, _D, ctypes.c_double, ctypes.c_double, _I32,
                                      ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, _D, _D, _I64]
        lib.oracle_l_step.restype = None
        lib.oracle_assign.argtypes = [_D, ctypes.c_int64, ctypes.c_int64, _D, _U8,
                                      ctypes.c_int32, _I32]
        lib.oracle_assign.restype = ctypes.c_int64
        lib.oracle_lloyd.argtypes = [_D, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, _I32,
                                     _D, _U8, ctypes.c_int32, _I64]
        lib.oracle_lloyd.restype = ctypes.c_int32
        lib.oracle_kmeanspp.argtypes = [_D, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                                        ctypes.c_uint64, _I64]
        lib.oracle_kmeanspp.restype = None
        lib.oracle_init_labels.argtypes = [_D, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                                           ctypes.c_uint64, ctypes.c_int32, _I32]
        lib.oracle_init_labels.restype = ctypes.c_int32
        lib.oracle_s_step.argtypes = [_D, _D, _D, ctypes.c_double, ctypes.c_int64, _D]
        lib.oracle_s_step.restype = None
        lib.oracle_theta_step.argtypes = [_D, _D, _D, ctypes.c_double, ctypes.c_int64, _D]
        lib.oracle_theta_step.restype = None
        lib.oracle_iteration.argtypes = [_D, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_int32,
                                         _D, _D, _D, _I32, _D, _D, _I32]
        lib.oracle_iteration.restype = ctypes.c_int64
        lib.oracle_objective.argtypes = [_D, _D, _I32, ctypes.c_int32, ctypes.c_double,
                                         ctypes.c_int64, ctypes.c_int64]
        lib.oracle_objective.restype = ctypes.c_double
        lib.oracle_lagrangian.argtypes = [_D, _D, _D, _D, _I32, ctypes.c_int32, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_int64, ctypes.c_int64]
        lib.oracle_lagrangian.restype = ctypes.c_double
        lib.oracle_solve.argtypes = [_D, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_int32, ctypes.c_int32,
                                     ctypes.c_uint64, _I32, ctypes.c_int32, _D,
                                     _D, _D, _D, _I32, ctypes.POINTER(OracleStats)]
        lib.oracle_solve.restype = ctypes.c_int32
        lib.oracle_s_step_l21.argtypes = [_D, _D, _D, ctypes.c_double, ctypes.c_int64, ctypes.c_int64, _D]
        lib.oracle_s_step_l21.restype = None
        lib.oracle_iteration_ex.argtypes = lib.oracle_iteration.argtypes + [ctypes.c_int32]
        lib.oracle_iteration_ex.restype = ctypes.c_int64
        lib.oracle_solve_ex.argtypes = lib.oracle_solve.argtypes + [ctypes.c_int32]
        lib.oracle_solve_ex.restype = ctypes.c_int32
        _lib = lib
    return _lib


def _f64(a) -> np.ndarray:
    return np.asfortranarray(np.asarray(a, dtype=np.float64))


def _ptr(a: np.ndarray, typ):
    return a.ctypes.data_as(typ)


def _labels(p, n) -> np.ndarray:
    p = np.ascontiguousarray(np.asarray(p, dtype=np.int32))
    assert p.shape == (n,)
    return p


# ---------------------------------------------------------------- generators
def splitmix64_stream(seed: int, count: int) -> list[int]:
    lib = _load()
    st = ctypes.c_uint64(seed)
    return [int(lib.oracle_splitmix64(ctypes.byref(st))) for _ in range(count)]


def uniform_stream(seed: int, count: int) -> list[float]:
    lib = _load()
    st = ctypes.c_uint64(seed)
    return [float(lib.oracle_uniform(ctypes.byref(st))) for _ in range(count)]


# ---------------------------------------------------------------- steps
def fro(A) -> float:
    A = _f64(A)
    return _load().oracle_fro(_ptr(A, _D), A.size)


def column_norms(S) -> np.ndarray:
    """Sec. 6 anomaly score ||S_j||_2 per column."""
    S = _f64(S)
    d, n = S.shape
    out = np.zeros(n)
    _load().oracle_column_norms(_ptr(S, _D), d, n, _ptr(out, _D))
    return out


def cluster_means(Y, labels, c, mu=None):
    Y = _f64(Y)
    d, n = Y.shape
    p = _labels(labels, n)
    mu = np.zeros((d, c), order="F") if mu is None else _f64(mu).copy(order="F")
    cnt = np.zeros(c, dtype=np.int64)
    _load().oracle_cluster_means(_ptr(Y, _D), d, n, _ptr(p, _I32), c, _ptr(mu, _D), _ptr(cnt, _I64))
    return mu, cnt


def l_step(X, S, Theta, rho, lam, labels, c):
    X, S, Theta = _f64(X), _f64(S), _f64(Theta)
    d, n = X.shape
    p = _labels(labels, n)
    L = np.zeros((d, n), order="F")
    mu = np.zeros((d, c), order="F")
    cnt = np.zeros(c, dtype=np.int64)
    _load().oracle_l_step(_ptr(X, _D), _ptr(S, _D), _ptr(Theta, _D), rho, lam, _ptr(p, _I32), c,
                          d, n, _ptr(L, _D), _ptr(mu, _D), _ptr(cnt, _I64))
    return L, mu, cnt


def assign(Y, mu, labels, active=None):
    Y, mu = _f64(Y), _f64(mu)
    d, n = Y.shape
    c = mu.shape[1]
    p = _labels(labels, n).copy()
    act = np.ones(c, dtype=np.uint8) if active is None else np.ascontiguousarray(active, dtype=np.uint8)
    ch = _load().oracle_assign(_ptr(Y, _D), d, n, _ptr(mu, _D), _ptr(act, _U8), c, _ptr(p, _I32))
    return p, int(ch)


def lloyd(Y, labels, mu, active=None, km_max=100):
    Y = _f64(Y)
    d, n = Y.shape
    mu = _f64(mu).copy(order="F")
    c = mu.shape[1]
    p = _labels(labels, n).copy()
    act = np.ones(c, dtype=np.uint8) if active is None else np.ascontiguousarray(active, dtype=np.uint8).copy()
    ch = ctypes.c_int64(0)
    steps = _load().oracle_lloyd(_ptr(Y, _D), d, n, c, _ptr(p, _I32), _ptr(mu, _D), _ptr(act, _U8),
                                 km_max, ctypes.byref(ch))
    return p, mu, act, int(steps), int(ch.value)


def kmeanspp(X, c, seed):
    X = _f64(X)
    d, n = X.shape
    centers = np.zeros(c, dtype=np.int64)
    _load().oracle_kmeanspp(_ptr(X, _D), d, n, c, seed, _ptr(centers, _I64))
    return centers


def init_labels(X, c, seed, km_max=100):
    X = _f64(X)
    d, n = X.shape
    p = np.zeros(n, dtype=np.int32)
    steps = _load().oracle_init_labels(_ptr(X, _D), d, n, c, seed, km_max, _ptr(p, _I32))
    return p, int(steps)


def s_step(X, L, Theta, rho):
    X, L, Theta = _f64(X), _f64(L), _f64(Theta)
    S = np.zeros(X.shape, order="F")
    _load().oracle_s_step(_ptr(X, _D), _ptr(L, _D), _ptr(Theta, _D), rho, X.size, _ptr(S, _D))
    return S


def theta_step(X, L, S, Theta, rho):
    X, L, S = _f64(X), _f64(L), _f64(S)
    T = _f64(Theta).copy(order="F")
    _load().oracle_theta_step(_ptr(X, _D), _ptr(L, _D), _ptr(S, _D), rho, X.size, _ptr(T, _D))
    return T


@dataclass
class State:
    L: np.ndarray
    S: np.ndarray
    Theta: np.ndarray
    labels: np.ndarray
    rho: float

    def copy(self) -> "State":
        return State(self.L.copy(order="F"), self.S.copy(order="F"), self.Theta.copy(order="F"),
                     self.labels.copy(), float(self.rho))


def s_step_l21(X, L, Theta, rho):
    """S step with the l2,1 norm (block soft-thresholding of every column)."""
    X, L, Theta = _f64(X), _f64(L), _f64(Theta)
    d, n = X.shape
    S = np.zeros(X.shape, order="F")
    _load().oracle_s_step_l21(_ptr(X, _D), _ptr(L, _D), _ptr(Theta, _D), rho, d, n, _ptr(S, _D))
    return S


def iteration(X, state: State, c, lam, kappa=1.5, km_max=100, snorm=0):
    """One ALM iteration (L, p, S, Theta/rho) applied to a copy of ``state``."""
    X = _f64(X)
    d, n = X.shape
    s = state.copy()
    rho = ctypes.c_double(s.rho)
    norms = np.zeros(3)
    steps = ctypes.c_int32(0)
    ch = _load().oracle_iteration_ex(_ptr(X, _D), d, n, c, lam, kappa, km_max, _ptr(s.L, _D),
                                  _ptr(s.S, _D), _ptr(s.Theta, _D), _ptr(s.labels, _I32),
                                  ctypes.byref(rho), _ptr(norms, _D), ctypes.byref(steps), int(snorm))
    s.rho = rho.value
    return s, norms, int(ch), int(steps.value)


def objective(L, S, labels, c, lam):
    L, S = _f64(L), _f64(S)
    d, n = L.shape
    p = _labels(labels, n)
    return _load().oracle_objective(_ptr(L, _D), _ptr(S, _D), _ptr(p, _I32), c, lam, d, n)


def lagrangian(X, L, S, Theta, labels, c, lam, rho):
    X, L, S, Theta = _f64(X), _f64(L), _f64(S), _f64(Theta)
    d, n = X.shape
    p = _labels(labels, n)
    return _load().oracle_lagrangian(_ptr(X, _D), _ptr(L, _D), _ptr(S, _D), _ptr(Theta, _D),
                                     _ptr(p, _I32), c, lam, rho, d, n)


def solve(X, c, lam=0.0, rho0=1e-4, kappa=1.5, tol=1e-6, max_iter=500, km_max=100, seed=0,
          p0=None, warm: State | None = None, snorm=0):
    """Whole RES-PCA solve. Returns (State, stats dict)."""
    X = _f64(X)
    d, n = X.shape
    if warm is not None:
        s = warm.copy()
    else:
        s = State(np.zeros((d, n), order="F"), np.zeros((d, n), order="F"),
                  np.zeros((d, n), order="F"), np.zeros(n, dtype=np.int32), rho0)
    p0a = None if p0 is None else _labels(p0, n)
    rho = ctypes.c_double(s.rho)
    st = OracleStats()
    rc = _load().oracle_solve_ex(_ptr(X, _D), d, n, c, lam, rho0, kappa, tol, max_iter, km_max, seed,
                              None if p0a is None else _ptr(p0a, _I32), 1 if warm is not None else 0,
                              ctypes.byref(rho), _ptr(s.L, _D), _ptr(s.S, _D), _ptr(s.Theta, _D),
                              _ptr(s.labels, _I32), ctypes.byref(st), int(snorm))
    if rc != 0:
        raise ValueError("oracle_solve: invalid arguments")
    s.rho = rho.value
    stats = {f: getattr(st, f) for f, _ in OracleStats._fields_}
    return s, stats
