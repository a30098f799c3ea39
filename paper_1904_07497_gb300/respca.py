"""Python binding of librespca.so (the C ABI in include/respca.h).

Argument marshalling only: every step of the solver runs in the CUDA library.
The functions carry the C names.  Matrices are torch tensors on the handle's
device, column-major d x n: ``X.stride(0) == 1`` and the leading dimension is
``X.stride(1)`` (a contiguous (n, d) tensor transposed is such a view).
If the compiled library is missing this module raises; there is no other
code path.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "_lib", "librespca.so")

RESPCA_OK = 0
RESPCA_ERR_INVALID_ARG = 1
RESPCA_ERR_NONFINITE_INPUT = 2
RESPCA_ERR_OOM = 3
RESPCA_ERR_CUDA = 4
RESPCA_ERR_TIMEOUT = 5
RESPCA_ERR_UNSUPPORTED = 6

RESPCA_F32, RESPCA_BF16, RESPCA_F16 = 0, 1, 2


class respca_config(ctypes.Structure):
    _fields_ = [("rho0", ctypes.c_double), ("kappa", ctypes.c_double),
                ("kmeans_max_iter", ctypes.c_int32), ("timing", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("stream", ctypes.c_void_p),
                ("device", ctypes.c_int32), ("search_impl", ctypes.c_int32),
                ("ramp_skip", ctypes.c_int32), ("batch_lanes", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("s_norm", ctypes.c_int32),
                ("switch_tol", ctypes.c_double), ("stop_after_ramp", ctypes.c_int32),
                ("p_step", ctypes.c_int32), ("spectral_scale", ctypes.c_double)]


class respca_spectral_info(ctypes.Structure):
    _fields_ = [("outer_iters", ctypes.c_int32), ("matvecs", ctypes.c_int32),
                ("residual", ctypes.c_double), ("sigma2", ctypes.c_double),
                ("theta_c", ctypes.c_double), ("theta_next", ctypes.c_double),
                ("lloyd_passes", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("ms_gram", ctypes.c_double), ("ms_products", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class respca_stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("err", ctypes.c_double), ("err_resid", ctypes.c_double),
                ("err_dL", ctypes.c_double), ("err_dS", ctypes.c_double),
                ("rho_final", ctypes.c_double), ("lambda_", ctypes.c_double),
                ("label_changes", ctypes.c_int64), ("lloyd_passes", ctypes.c_int64),
                ("assigned_columns", ctypes.c_int64), ("rechecked_columns", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64),
                ("init_lloyd_passes", ctypes.c_int32), ("fused_launches", ctypes.c_int32),
                ("ms_total", ctypes.c_float), ("ms_init", ctypes.c_float),
                ("ms_fused", ctypes.c_float), ("ms_dense", ctypes.c_float),
                ("dense_passes", ctypes.c_int32), ("bf16_iters", ctypes.c_int32),
                ("x_norm", ctypes.c_double), ("ms_dense16", ctypes.c_float),
                ("dense16_passes", ctypes.c_int32), ("copy16_iters", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {(k[:-1] if k.endswith("_") else k): getattr(self, k) for k, _ in self._fields_
                if not k.startswith("reserved")}


class respca_warm(ctypes.Structure):
    _fields_ = [("Theta", ctypes.c_void_p), ("rho", ctypes.c_double),
                ("warm", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class respca_problem(ctypes.Structure):
    _fields_ = [("x_dtype", ctypes.c_int32), ("c", ctypes.c_int32), ("X", ctypes.c_void_p),
                ("d", ctypes.c_int64), ("n", ctypes.c_int64), ("ldx", ctypes.c_int64),
                ("lambda_", ctypes.c_double), ("tol", ctypes.c_double),
                ("max_iter", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("p0", ctypes.c_void_p), ("L", ctypes.c_void_p), ("S", ctypes.c_void_p),
                ("lds", ctypes.c_int64), ("p", ctypes.c_void_p)]


class respca_batch_options(ctypes.Structure):
    _fields_ = [("tile_rows", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("spin_limit", ctypes.c_int64), ("tuned_rows", ctypes.c_int32),
                ("tuned_ctas_per_sm", ctypes.c_int32), ("ms_kernel", ctypes.c_float),
                ("reserved", ctypes.c_int32)]


_lib = None
_I64 = ctypes.c_int64
_VP = ctypes.c_void_p


def load():
    """Load librespca.so (build it first with __graft_entry__.build() or
    paper_1904_07497_gb300._build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"RES-PCA CUDA library not built: {LIB_PATH} is missing")
    lib = ctypes.CDLL(LIB_PATH)
    lib.respca_config_default.argtypes = [ctypes.POINTER(respca_config)]
    lib.respca_config_default.restype = None
    lib.respca_create.argtypes = [ctypes.POINTER(_VP), ctypes.POINTER(respca_config)]
    lib.respca_create.restype = ctypes.c_int
    lib.respca_destroy.argtypes = [_VP]
    lib.respca_destroy.restype = ctypes.c_int
    solve_args = [_VP, ctypes.c_int32, _VP, _I64, _I64, _I64, ctypes.c_double, ctypes.c_int32,
                  ctypes.c_double, ctypes.c_int32, _VP, _VP, _VP, _I64, _VP]
    lib.respca_solve.argtypes = solve_args + [ctypes.POINTER(respca_warm), ctypes.POINTER(respca_stats)]
    lib.respca_solve.restype = ctypes.c_int
    lib.respca_solve_host.argtypes = solve_args + [ctypes.POINTER(respca_stats)]
    lib.respca_solve_host.restype = ctypes.c_int
    lib.respca_init_labels.argtypes = [_VP, ctypes.c_int32, _VP, _I64, _I64, _I64, ctypes.c_int32,
                                       _VP, ctypes.POINTER(ctypes.c_int32)]
    lib.respca_init_labels.restype = ctypes.c_int
    lib.respca_solve_batched.argtypes = [_VP, ctypes.c_int32, ctypes.POINTER(respca_problem),
                                         ctypes.POINTER(respca_stats)]
    lib.respca_solve_batched.restype = ctypes.c_int
    lib.respca_solve_batched_persistent.argtypes = [_VP, ctypes.c_int32, ctypes.POINTER(respca_problem),
                                                    ctypes.POINTER(respca_stats),
                                                    ctypes.POINTER(respca_batch_options)]
    lib.respca_solve_batched_persistent.restype = ctypes.c_int
    lib.respca_init_labels_noalloc.argtypes = [ctypes.c_int32, _VP, _I64, _I64, _I64, ctypes.c_int32,
                                               ctypes.c_uint64, ctypes.c_int32, _VP,
                                               ctypes.POINTER(ctypes.c_int32), _VP]
    lib.respca_init_labels_noalloc.restype = ctypes.c_int
    lib.respca_column_norms.argtypes = [_VP, _I64, _I64, _I64, _VP, _VP]
    lib.respca_column_norms.restype = ctypes.c_int
    _D = ctypes.c_double
    _PD = ctypes.POINTER(ctypes.c_double)
    _PF = ctypes.POINTER(ctypes.c_float)
    lib.respca_net_create.argtypes = [ctypes.POINTER(_VP), ctypes.c_int32, _VP]
    lib.respca_net_create.restype = ctypes.c_int
    lib.respca_net_destroy.argtypes = [_VP]
    lib.respca_net_destroy.restype = ctypes.c_int
    lib.respca_net_schedule.argtypes = [_D, _D, ctypes.c_int32, _PF, _PD, _PD]
    lib.respca_net_schedule.restype = ctypes.c_int
    lib.respca_net_forward.argtypes = [_VP, _VP, _I64, _I64, _I64, _VP, ctypes.c_int32, _D, _VP, _VP,
                                       _I64, ctypes.c_int32, _PD, _PD, _VP, _VP, _VP]
    lib.respca_net_forward.restype = ctypes.c_int
    lib.respca_net_infer.argtypes = [_VP, ctypes.c_int32, _VP, _I64, _I64, _I64, _VP, ctypes.c_int32, _D,
                                     _VP, _VP, _I64, ctypes.c_int32, _PD, _PD, ctypes.c_int32, _VP, _VP, _VP]
    lib.respca_net_infer.restype = ctypes.c_int
    lib.respca_net_backward.argtypes = [_VP, _VP, _VP, _I64, _D, _PD, _PD, _PD, _PF]
    lib.respca_net_backward.restype = ctypes.c_int
    lib.respca_mlp_forward.argtypes = [_VP, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _VP, _VP,
                                       _VP, _VP]
    lib.respca_mlp_forward.restype = ctypes.c_int
    lib.respca_mlp_backward.argtypes = [_VP, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _VP, _VP,
                                        _VP, _VP, ctypes.c_int32, _VP]
    lib.respca_mlp_backward.restype = ctypes.c_int
    lib.respca_adam_step.argtypes = [_VP, _VP, _VP, _VP, _I64, _D, _D, _D, _D, ctypes.c_int32, _VP]
    lib.respca_adam_step.restype = ctypes.c_int
    lib.respca_spectral_labels.argtypes = [_VP, _VP, _I64, _I64, _I64, ctypes.c_int32, _VP,
                                           ctypes.POINTER(respca_spectral_info)]
    lib.respca_spectral_labels.restype = ctypes.c_int
    lib.respca_status_string.argtypes = [ctypes.c_int]
    lib.respca_status_string.restype = ctypes.c_char_p
    lib.respca_last_error.argtypes = [_VP]
    lib.respca_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


class RespcaError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


def _check(h, rc: int, where: str):
    if rc != RESPCA_OK:
        lib = load()
        detail = lib.respca_last_error(h).decode() if h else ""
        raise RespcaError(rc, f"{where}: {lib.respca_status_string(rc).decode()}"
                              + (f" -- {detail}" if detail else ""))


def _dtype_code(t) -> int:
    import torch
    return {torch.float32: RESPCA_F32, torch.bfloat16: RESPCA_BF16,
            torch.float16: RESPCA_F16}[t.dtype]


def _colmajor(t, name):
    if t.dim() != 2 or t.stride(0) != 1:
        raise ValueError(f"{name} must be a column-major (d, n) view (stride(0) == 1)")
    return max(t.stride(1), t.shape[0])


def _state_out(L, S, d: int, n: int, like):
    import torch
    for t, name in ((L, "L"), (S, "S")):
        if t.dtype != torch.float32 or t.device != like.device or tuple(t.shape) != (d, n):
            raise ValueError(f"{name} must be a float32 ({d}, {n}) tensor on {like.device}")


def _labels_out(p, n: int, like, name: str = "p"):
    """Check an int32 label buffer before its pointer is handed to a kernel:
    a wrong dtype, length, layout or device would be written out of bounds."""
    import torch
    if p.dtype != torch.int32:
        raise ValueError(f"{name} must be int32")
    if not p.is_cuda or p.device != like.device:
        raise ValueError(f"{name} must be a CUDA tensor on {like.device}")
    if not p.is_contiguous() or p.numel() < n:
        raise ValueError(f"{name} must be contiguous with at least {n} elements")


# ------------------------------------------------------------------ C names
def respca_config_default() -> respca_config:
    cfg = respca_config()
    load().respca_config_default(ctypes.byref(cfg))
    return cfg


def respca_create(cfg: respca_config | None = None):
    h = _VP()
    _check(None, load().respca_create(ctypes.byref(h), ctypes.byref(cfg) if cfg else None),
           "respca_create")
    return h


def respca_destroy(h) -> None:
    _check(None, load().respca_destroy(h), "respca_destroy")


def respca_solve(h, X, c: int, L, S, p, *, lam: float = 0.0, tol: float = 1e-6,
                 max_iter: int = 500, p0=None, warm: respca_warm | None = None) -> dict:
    """X, L, S: (d, n) column-major CUDA tensors; p, p0: int32 (n,) CUDA tensors."""
    d, n = X.shape
    ldx = _colmajor(X, "X")
    lds = _colmajor(L, "L")
    if _colmajor(S, "S") != lds:
        raise ValueError("L and S must share a leading dimension")
    _state_out(L, S, d, n, X)
    _labels_out(p, n, X)
    if p0 is not None:
        _labels_out(p0, n, X, "p0")
    st = respca_stats()
    rc = load().respca_solve(h, _dtype_code(X), X.data_ptr(), d, n, ldx, float(lam), int(c),
                             float(tol), int(max_iter), p0.data_ptr() if p0 is not None else None,
                             L.data_ptr(), S.data_ptr(), lds, p.data_ptr(),
                             ctypes.byref(warm) if warm is not None else None, ctypes.byref(st))
    _check(h, rc, "respca_solve")
    return st.as_dict()


def respca_solve_host(h, X, c: int, L, S, p, *, lam: float = 0.0, tol: float = 1e-6,
                      max_iter: int = 500, p0=None) -> dict:
    """X, L, S: (d, n) column-major CPU tensors (pinned or not); p: int32 CPU."""
    d, n = X.shape
    ldx = _colmajor(X, "X")
    lds = _colmajor(L, "L")
    st = respca_stats()
    rc = load().respca_solve_host(h, _dtype_code(X), X.data_ptr(), d, n, ldx, float(lam), int(c),
                                  float(tol), int(max_iter),
                                  p0.data_ptr() if p0 is not None else None, L.data_ptr(),
                                  S.data_ptr(), lds, p.data_ptr(), ctypes.byref(st))
    _check(h, rc, "respca_solve_host")
    return st.as_dict()


def respca_init_labels(h, X, c: int, p) -> int:
    d, n = X.shape
    ldx = _colmajor(X, "X")
    _labels_out(p, n, X)
    passes = ctypes.c_int32(0)
    rc = load().respca_init_labels(h, _dtype_code(X), X.data_ptr(), d, n, ldx, int(c),
                                   p.data_ptr(), ctypes.byref(passes))
    _check(h, rc, "respca_init_labels")
    return passes.value


def respca_init_labels_noalloc(X, c: int, p, *, seed: int = 0, kmeans_max_iter: int = 100,
                               stream=None) -> int:
    """Initial labels with no device allocation (scratch in the library's
    static device array), for callers whose device memory belongs to their
    own pool or budget.  Synchronous.  X: (d, n) column-major CUDA tensor;
    p: int32 (n,) CUDA tensor on X's device.  Returns the number of Lloyd
    passes."""
    import torch
    d, n = X.shape
    ldx = _colmajor(X, "X")
    _labels_out(p, n, X)
    passes = ctypes.c_int32(0)
    s = stream.cuda_stream if stream is not None else None
    with torch.cuda.device(X.device):          # the entry point works on the current device
        rc = load().respca_init_labels_noalloc(_dtype_code(X), X.data_ptr(), d, n, ldx, int(c),
                                               int(seed), int(kmeans_max_iter), p.data_ptr(),
                                               ctypes.byref(passes), s)
    _check(None, rc, "respca_init_labels_noalloc")
    return passes.value


def respca_column_norms(S, out=None, stream=None):
    """Sec. 6 anomaly score ||S_j||_2 of every column of a column-major CUDA
    tensor S (d, n).  Returns a float32 tensor of n scores."""
    import torch
    d, n = S.shape
    if out is None:
        out = torch.empty(n, device=S.device, dtype=torch.float32)
    s = stream if stream is not None else torch.cuda.current_stream(S.device)
    rc = load().respca_column_norms(ctypes.c_void_p(S.data_ptr()), d, n, _colmajor(S, "S"),
                                    ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(s.cuda_stream))
    _check(None, rc, "respca_column_norms")
    return out


def _problem_table(problems: list[dict]):
    arr = (respca_problem * len(problems))()
    for i, q in enumerate(problems):
        X = q["X"]
        d, n = X.shape
        arr[i].x_dtype = _dtype_code(X)
        arr[i].c = int(q["c"])
        arr[i].X = X.data_ptr()
        arr[i].d, arr[i].n, arr[i].ldx = d, n, _colmajor(X, "X")
        arr[i].lambda_ = float(q.get("lam", 0.0))
        arr[i].tol = float(q.get("tol", 1e-6))
        arr[i].max_iter = int(q.get("max_iter", 500))
        arr[i].p0 = q["p0"].data_ptr() if q.get("p0") is not None else None
        arr[i].L = q["L"].data_ptr()
        arr[i].S = q["S"].data_ptr()
        arr[i].lds = _colmajor(q["L"], "L")
        arr[i].p = q["p"].data_ptr()
    return arr


def respca_solve_batched(h, problems: list[dict]) -> list[dict]:
    """problems: dicts with X, c, L, S, p (and optional lam, tol, max_iter, p0)."""
    arr = _problem_table(problems)
    stats = (respca_stats * len(problems))()
    rc = load().respca_solve_batched(h, len(problems), arr, stats)
    _check(h, rc, "respca_solve_batched")
    return [s.as_dict() for s in stats]


def respca_solve_batched_persistent(h, problems: list[dict], opt: respca_batch_options | None = None):
    """All problems in one persistent launch (respca_solve_batched_persistent).
    Returns (per-problem stats, options with the tile choice and kernel time)."""
    arr = _problem_table(problems)
    for q in problems:
        _state_out(q["L"], q["S"], q["X"].shape[0], q["X"].shape[1], q["X"])
        _labels_out(q["p"], q["X"].shape[1], q["X"])
    stats = (respca_stats * len(problems))()
    o = opt if opt is not None else respca_batch_options()
    rc = load().respca_solve_batched_persistent(h, len(problems), arr, stats, ctypes.byref(o))
    _check(h, rc, "respca_solve_batched_persistent")
    return [s.as_dict() for s in stats], o


# ------------------------------------------------------------------ convenience
@dataclass
class Result:
    L: object
    S: object
    p: object
    stats: dict


class Solver:
    """Owns a handle bound to the current torch CUDA stream."""

    def __init__(self, rho0: float = 1e-4, kappa: float = 1.5, kmeans_max_iter: int = 100,
                 seed: int = 0, stream=None, device: int | None = None, timing: bool = False,
                 search_impl: int = 0, ramp_skip: bool = True, batch_lanes: int = 0,
                 precision: int = 0, switch_tol: float | None = None, s_norm: int = 0,
                 stop_after_ramp: bool = False, p_step: int = 0, spectral_scale: float | None = None):
        import torch
        cfg = respca_config_default()
        cfg.stop_after_ramp = 1 if stop_after_ramp else 0
        cfg.p_step = p_step
        if spectral_scale is not None:
            cfg.spectral_scale = spectral_scale
        cfg.search_impl = search_impl
        cfg.ramp_skip = 1 if ramp_skip else 0
        cfg.batch_lanes = batch_lanes
        cfg.precision = precision
        cfg.s_norm = s_norm
        if switch_tol is not None:
            cfg.switch_tol = switch_tol
        cfg.rho0, cfg.kappa, cfg.kmeans_max_iter, cfg.seed = rho0, kappa, kmeans_max_iter, seed
        cfg.timing = 1 if timing else 0
        dev = torch.cuda.current_device() if device is None else device
        s = stream if stream is not None else torch.cuda.current_stream(dev)
        cfg.stream = s.cuda_stream
        cfg.device = dev
        self.stream = s
        self.device = dev
        self.h = respca_create(cfg)

    def close(self):
        if self.h:
            respca_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, X, c: int, *, lam: float = 0.0, tol: float = 1e-6, max_iter: int = 500,
              p0=None, warm=None, out=None) -> Result:
        import torch
        d, n = X.shape
        if out is None:
            L = torch.empty((n, d), device=X.device, dtype=torch.float32).T
            S = torch.empty((n, d), device=X.device, dtype=torch.float32).T
            p = torch.empty(n, device=X.device, dtype=torch.int32)
        else:
            L, S, p = out
        st = respca_solve(self.h, X, c, L, S, p, lam=lam, tol=tol, max_iter=max_iter, p0=p0,
                          warm=warm)
        return Result(L, S, p, st)

    def init_labels(self, X, c: int):
        import torch
        p = torch.empty(X.shape[1], device=X.device, dtype=torch.int32)
        passes = respca_init_labels(self.h, X, c, p)
        return p, passes


def respca_spectral_labels(h, Y, c: int, p=None) -> tuple[object, dict]:
    """Spectral p step alone (Sec. 4.2 alternative to K-means): labels of the
    columns of a column-major FP32 CUDA tensor Y (d, n).  Returns (p, info)."""
    import torch
    d, n = Y.shape
    ldy = _colmajor(Y, "Y")
    if p is None:
        p = torch.empty(n, device=Y.device, dtype=torch.int32)
    _labels_out(p, n, Y)
    info = respca_spectral_info()
    rc = load().respca_spectral_labels(h, Y.data_ptr(), d, n, ldy, int(c), p.data_ptr(), ctypes.byref(info))
    _check(h, rc, "respca_spectral_labels")
    return p, info.as_dict()


# ------------------------------------------------------------------ learned warm start
def respca_net_create(device: int = -1, stream=None):
    net = _VP()
    _check(None, load().respca_net_create(ctypes.byref(net), int(device),
                                          stream.cuda_stream if stream is not None else None),
           "respca_net_create")
    return net


def respca_net_destroy(net) -> None:
    _check(None, load().respca_net_destroy(net), "respca_net_destroy")


def respca_net_schedule(rho: float, kappa: float, m) -> tuple[list[float], list[float]]:
    """(rho_k, tau_k) from the 2 K log multipliers m (a sequence of floats)."""
    K = len(m) // 2
    mm = (ctypes.c_float * (2 * K))(*[float(v) for v in m])
    r = (ctypes.c_double * K)()
    t = (ctypes.c_double * K)()
    _check(None, load().respca_net_schedule(float(rho), float(kappa), K, mm, r, t),
           "respca_net_schedule")
    return list(r), list(t)


def respca_net_forward(net, X, p, c: int, lam: float, S0, Theta0, rho_k, tau_k, L=None, S=None,
                       Theta=None) -> None:
    """X, S0, Theta0 (and the outputs): (d, n) column-major FP32 CUDA tensors;
    p: int32 (n,) labels.  S0, Theta0 and the outputs share a leading dimension."""
    d, n = X.shape
    ldx = _colmajor(X, "X")
    lds = _colmajor(S0, "S0")
    for name, t in (("Theta0", Theta0), ("L", L), ("S", S), ("Theta", Theta)):
        if t is not None and _colmajor(t, name) != lds:
            raise ValueError(f"{name} must share the leading dimension of S0")
    K = len(rho_k)
    r = (ctypes.c_double * K)(*rho_k)
    t = (ctypes.c_double * K)(*tau_k)
    ptr = (lambda a: a.data_ptr() if a is not None else None)
    rc = load().respca_net_forward(net, X.data_ptr(), d, n, ldx, p.data_ptr(), int(c), float(lam),
                                   S0.data_ptr(), Theta0.data_ptr(), lds, K, r, t, ptr(L), ptr(S),
                                   ptr(Theta))
    _check(None, rc, "respca_net_forward")


def respca_net_infer(net, X, p, c: int, lam: float, S0, Theta0, rho_k, tau_k, L, S, Theta,
                     storage: int = 0) -> None:
    """Inference-only forward pass (respca_net_infer): X in FP32, BF16 or FP16;
    intermediate layer states in FP32 (storage 0) or BF16 (storage 1); the
    last layer's L, S, Theta (FP32, column-major like S0) are written."""
    d, n = X.shape
    ldx = _colmajor(X, "X")
    lds = _colmajor(S0, "S0")
    for t, name in ((Theta0, "Theta0"), (L, "L"), (S, "S"), (Theta, "Theta")):
        if _colmajor(t, name) != lds:
            raise ValueError(f"{name} must share S0's leading dimension")
    _labels_out(p, n, X)
    K = len(rho_k)
    rk = (ctypes.c_double * K)(*rho_k)
    tk = (ctypes.c_double * K)(*tau_k)
    rc = load().respca_net_infer(net, _dtype_code(X), X.data_ptr(), d, n, ldx, p.data_ptr(), int(c),
                                 float(lam), S0.data_ptr(), Theta0.data_ptr(), lds, K, rk, tk, int(storage),
                                 L.data_ptr(), S.data_ptr(), Theta.data_ptr())
    _check(None, rc, "respca_net_infer")


def respca_net_backward(net, Lt, St, scale: float, layers: int):
    """Loss and gradients of the last forward pass: returns
    (loss, g_rho [K], g_tau [K], g_m [2K])."""
    ldt = _colmajor(Lt, "Lt")
    if _colmajor(St, "St") != ldt:
        raise ValueError("Lt and St must share a leading dimension")
    K = int(layers)
    loss = ctypes.c_double(0.0)
    gr = (ctypes.c_double * K)()
    gt = (ctypes.c_double * K)()
    gm = (ctypes.c_float * (2 * K))()
    rc = load().respca_net_backward(net, Lt.data_ptr(), St.data_ptr(), ldt, float(scale),
                                    ctypes.byref(loss), gr, gt, gm)
    _check(None, rc, "respca_net_backward")
    return loss.value, list(gr), list(gt), list(gm)


def respca_mlp_forward(params, nz: int, H: int, nout: int, z, out, hidden, stream=None) -> None:
    s = stream.cuda_stream if stream is not None else None
    _check(None, load().respca_mlp_forward(params.data_ptr(), nz, H, nout, z.data_ptr(),
                                           out.data_ptr(), hidden.data_ptr(), s),
           "respca_mlp_forward")


def respca_mlp_backward(params, nz: int, H: int, nout: int, z, hidden, gout, grad,
                        accumulate: bool = False, stream=None) -> None:
    s = stream.cuda_stream if stream is not None else None
    _check(None, load().respca_mlp_backward(params.data_ptr(), nz, H, nout, z.data_ptr(),
                                            hidden.data_ptr(), gout.data_ptr(), grad.data_ptr(),
                                            1 if accumulate else 0, s),
           "respca_mlp_backward")


def respca_adam_step(params, grad, m, v, *, lr: float, t: int, beta1: float = 0.9,
                     beta2: float = 0.999, eps: float = 1e-8, stream=None) -> None:
    s = stream.cuda_stream if stream is not None else None
    _check(None, load().respca_adam_step(params.data_ptr(), grad.data_ptr(), m.data_ptr(),
                                         v.data_ptr(), params.numel(), float(lr), float(beta1),
                                         float(beta2), float(eps), int(t), s),
           "respca_adam_step")
