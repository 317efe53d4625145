"""Thin ctypes binding of libpavg.so (C-ABI declared in include/pavg.h).

Argument marshalling only: every step of the computation runs in the
library's CUDA kernels.  States are torch float64 CUDA tensors laid out as in
pavg.h ([n] or [B][n], u first then eta); torch supplies device memory and the
current stream.  Importing this module loads the library and raises when it
is missing or fails to load: there is no fallback path.
"""

import ctypes
import os

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libpavg.so")

PAVG_QUAD_MIDPOINT = 0
PAVG_QUAD_CLOSED = 1
PAVG_UPWIND_STANDARD = 0
PAVG_UPWIND_AS_PRINTED = 1
PAVG_SOLVER_MIXED = 0
PAVG_SOLVER_FP64 = 1
PAVG_SOLVER_SUBDOMAIN = 2
PAVG_PRECISION_FP64 = 0
PAVG_PRECISION_MIXED = 1
PAVG_MAX_CHEB_ARG = 16384.0  # widest exponential accepted: lambda_max |t|

ERRORS = {
    -1: "PAVG_ERR_INVAL", -2: "PAVG_ERR_NOMEM", -3: "PAVG_ERR_CUDA", -4: "PAVG_ERR_NOCONV",
    -5: "PAVG_ERR_NONFINITE", -6: "PAVG_ERR_TIMEOUT",
}

EXPORTED = [
    "pavg_default_params", "pavg_create", "pavg_destroy", "pavg_sizes", "pavg_mesh_export",
    "pavg_set_topography", "pavg_lambda_max", "pavg_linear", "pavg_nonlinear", "pavg_expL_apply",
    "pavg_averaged_rhs", "pavg_averaged_rhs_group", "pavg_averaged_rhs_literal", "pavg_averaged_rhs_marching", "pavg_timestep", "pavg_sync", "pavg_norms", "pavg_get_stats",
    "pavg_reset_stats", "pavg_last_error", "pavg_kernel_timing", "pavg_kernel_time", "pavg_linear_noalloc", "pavg_measure_fma_peak", "pavg_test_stall",
    "pavg_batch_create", "pavg_batch_destroy", "pavg_batch_averaged_rhs", "pavg_batch_autotune",
    "pavg_batch_set_config", "pavg_batch_get_config", "pavg_batch_kernel_time", "pavg_batch_sync",
    "pavg_batch_last_error", "pavg_batch_timestep",
    "pavg_surrogate_create", "pavg_surrogate_destroy", "pavg_surrogate_nparams", "pavg_surrogate_get_params",
    "pavg_surrogate_set_params", "pavg_surrogate_get_scaling", "pavg_surrogate_set_scaling",
    "pavg_surrogate_add_pairs", "pavg_surrogate_rows", "pavg_surrogate_fit_scaling", "pavg_surrogate_train",
    "pavg_surrogate_gradient", "pavg_surrogate_adam_step", "pavg_surrogate_features", "pavg_surrogate_apply",
    "pavg_surrogate_averaged_rhs", "pavg_surrogate_last_error",
]


class Params(ctypes.Structure):
    _fields_ = [
        ("refinement", ctypes.c_int),
        ("radius", ctypes.c_double),
        ("omega", ctypes.c_double),
        ("g", ctypes.c_double),
        ("H", ctypes.c_double),
        ("cheb_tol", ctypes.c_double),
        ("cg_rtol", ctypes.c_double),
        ("cg_maxit", ctypes.c_int),
        ("lambda_max", ctypes.c_double),
        ("quad_rule", ctypes.c_int),
        ("upwind_convention", ctypes.c_int),
        ("solver", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("sd_part_cells", ctypes.c_int),
        ("geometry_degree", ctypes.c_int),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("lambda_max", ctypes.c_double),
        ("last_degree", ctypes.c_int),
        ("cg_solves", ctypes.c_int),
        ("cg_iters_max", ctypes.c_int),
        ("cg_iters_mean", ctypes.c_double),
        ("error_flags", ctypes.c_int),
        ("kernel_launches", ctypes.c_int),
        ("cg_sweeps_mean", ctypes.c_double),
        ("solver_in_use", ctypes.c_int),
    ]


class BatchConfig(ctypes.Structure):
    _fields_ = [
        ("threads", ctypes.c_int),
        ("blocks_per_sm", ctypes.c_int),
        ("resident", ctypes.c_int),
        ("weighting", ctypes.c_int),
        ("predicted_ms", ctypes.c_double),
        ("strategy", ctypes.c_int),
    ]


class PavgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


def load(path=LIB_PATH):
    if not os.path.exists(path):
        raise RuntimeError(f"libpavg.so not found at {path}: build it with "
                           "`python -m paper_2103_07706_gb300.build` (no CPU fallback exists)")
    lib = ctypes.CDLL(path)
    P, D, I, I64, V = ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
    sig = {
        "pavg_default_params": (I, [ctypes.POINTER(Params)]),
        "pavg_create": (I, [ctypes.POINTER(Params), ctypes.POINTER(P)]),
        "pavg_destroy": (I, [P]),
        "pavg_sizes": (I, [P] + [ctypes.POINTER(I64)] * 5),
        "pavg_mesh_export": (I, [P, P, P]),
        "pavg_set_topography": (I, [P, P]),
        "pavg_lambda_max": (I, [P, ctypes.POINTER(D)]),
        "pavg_linear": (I, [P, P, P, I, V]),
        "pavg_nonlinear": (I, [P, P, P, I, V]),
        "pavg_expL_apply": (I, [P, D, P, P, I, V]),
        "pavg_averaged_rhs": (I, [P, D, I, P, P, V]),
        "pavg_averaged_rhs_group": (I, [P, D, I, I, I, P, P, V]),
        "pavg_averaged_rhs_literal": (I, [P, D, I, P, P, V]),
        "pavg_averaged_rhs_marching": (I, [P, D, I, P, P, V]),
        "pavg_timestep": (I, [P, D, D, I, P, I, V]),
        "pavg_sync": (I, [P, V]),
        "pavg_norms": (I, [P, P, P, V]),
        "pavg_get_stats": (I, [P, ctypes.POINTER(Stats)]),
        "pavg_reset_stats": (I, [P]),
        "pavg_last_error": (ctypes.c_char_p, [P]),
        "pavg_kernel_timing": (I, [P, I]),
        "pavg_kernel_time": (I, [P, ctypes.POINTER(D), ctypes.POINTER(I)]),
        "pavg_linear_noalloc": (I, [P, P, P, V]),
        "pavg_measure_fma_peak": (I, [I, ctypes.POINTER(D), V]),
        "pavg_test_stall": (I, [P, I, I, D]),
        "pavg_batch_create": (I, [P, I, ctypes.POINTER(P)]),
        "pavg_batch_destroy": (I, [P]),
        "pavg_batch_averaged_rhs": (I, [P, P, P, P, P, V]),
        "pavg_batch_autotune": (I, [P, P, P, P, V, ctypes.POINTER(BatchConfig)]),
        "pavg_batch_set_config": (I, [P, ctypes.POINTER(BatchConfig)]),
        "pavg_batch_get_config": (I, [P, ctypes.POINTER(BatchConfig)]),
        "pavg_batch_kernel_time": (I, [P, ctypes.POINTER(D), ctypes.POINTER(D)]),
        "pavg_batch_sync": (I, [P, V]),
        "pavg_batch_last_error": (ctypes.c_char_p, [P]),
        "pavg_batch_timestep": (I, [P, P, P, P, P, I, V]),
        "pavg_surrogate_create": (I, [I, ctypes.c_uint64, ctypes.POINTER(P)]),
        "pavg_surrogate_destroy": (I, [P]),
        "pavg_surrogate_nparams": (I, [P, ctypes.POINTER(I64)]),
        "pavg_surrogate_get_params": (I, [P, P]),
        "pavg_surrogate_set_params": (I, [P, P]),
        "pavg_surrogate_get_scaling": (I, [P, P, P, P, P]),
        "pavg_surrogate_set_scaling": (I, [P, P, P, P, P]),
        "pavg_surrogate_add_pairs": (I, [P, P, I, P, P, P, V]),
        "pavg_surrogate_rows": (I, [P, ctypes.POINTER(I64)]),
        "pavg_surrogate_fit_scaling": (I, [P, V]),
        "pavg_surrogate_train": (I, [P, I, I, D, ctypes.c_uint64, P, V]),
        "pavg_surrogate_gradient": (I, [P, P, P, I, P, ctypes.POINTER(D), V]),
        "pavg_surrogate_adam_step": (I, [P, P, D, V]),
        "pavg_surrogate_features": (I, [P, P, P, P, P, I, V]),
        "pavg_surrogate_apply": (I, [P, P, P, P, P, I, V]),
        "pavg_surrogate_averaged_rhs": (I, [P, P, D, I, I, D, I, I, P, P, ctypes.POINTER(I), ctypes.POINTER(D), V]),
        "pavg_surrogate_last_error": (ctypes.c_char_p, [P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        _LIB = load()
    return _LIB


def default_params(**overrides):
    p = Params()
    rc = lib().pavg_default_params(ctypes.byref(p))
    if rc:
        raise PavgError(rc, "pavg_default_params")
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def _ptr(t, n, B=None):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    want = n if B is None else B * n
    if t.numel() != want:
        raise ValueError(f"expected {want} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr() or None)


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def measure_fma_peak(fp64):
    """Measured FP64 (fp64=True) or FP32 fused multiply-add rate of the current GPU, TFLOP/s."""
    v = ctypes.c_double()
    rc = lib().pavg_measure_fma_peak(1 if fp64 else 0, ctypes.byref(v), _stream())
    if rc:
        raise PavgError(rc, "pavg_measure_fma_peak")
    return v.value


class Model:
    """One library context: mesh, FE operators and workspace on the current device."""

    def __init__(self, refinement=3, **params):
        self._lib = lib()
        torch.cuda.init()
        p = default_params(refinement=refinement, **params)
        h = ctypes.c_void_p()
        rc = self._lib.pavg_create(ctypes.byref(p), ctypes.byref(h))
        if rc:
            raise PavgError(rc, "pavg_create failed")
        self._h = h
        self.params = p
        vals = [ctypes.c_int64() for _ in range(5)]
        self._check(self._lib.pavg_sizes(h, *[ctypes.byref(v) for v in vals]))
        self.n_u, self.n_eta, self.n_cells, self.n_edges, self.n_verts = [v.value for v in vals]
        self.n = self.n_u + self.n_eta

    def _check(self, rc):
        if rc:
            raise PavgError(rc, self._lib.pavg_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.pavg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- info
    def mesh(self):
        import numpy as np
        verts = np.zeros((self.n_verts, 3))
        cells = np.zeros((self.n_cells, 3), dtype=np.int32)
        self._check(self._lib.pavg_mesh_export(self._h, verts.ctypes.data_as(ctypes.c_void_p),
                                               cells.ctypes.data_as(ctypes.c_void_p)))
        return verts, cells

    @property
    def lambda_max(self):
        v = ctypes.c_double()
        self._check(self._lib.pavg_lambda_max(self._h, ctypes.byref(v)))
        return v.value

    def stats(self):
        s = Stats()
        self._check(self._lib.pavg_get_stats(self._h, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in Stats._fields_}

    def kernel_timing(self, enable=True):
        self._check(self._lib.pavg_kernel_timing(self._h, 1 if enable else 0))

    def kernel_time(self):
        """(total ms, launches) of the CG launches of the most recent call."""
        ms, k = ctypes.c_double(), ctypes.c_int()
        self._check(self._lib.pavg_kernel_time(self._h, ctypes.byref(ms), ctypes.byref(k)))
        return ms.value, k.value

    def reset_stats(self):
        self._check(self._lib.pavg_reset_stats(self._h))

    def test_stall(self, mode, part=0, wait_us=0.0):
        """Test aid: make one block of the subdomain solver stall (pavg.h)."""
        self._check(self._lib.pavg_test_stall(self._h, int(mode), int(part), float(wait_us)))

    def norms(self, U):
        """(||u||_L2, ||u||_H(div), ||eta||_L2) of a state (the paper's error norms)."""
        import numpy as np
        out = np.zeros(3)
        self._check(self._lib.pavg_norms(self._h, _ptr(U, self.n), out.ctypes.data_as(ctypes.c_void_p), _stream()))
        return tuple(float(x) for x in out)

    def sync(self):
        self._check(self._lib.pavg_sync(self._h, _stream()))

    def set_topography(self, b):
        self._check(self._lib.pavg_set_topography(self._h, _ptr(b, self.n_eta)))

    # ---------------------------------------------------------------- operators
    def _out(self, U, out):
        return torch.empty_like(U) if out is None else out

    def _batch(self, U):
        if U.numel() % self.n:
            raise ValueError("state size is not a multiple of n")
        return U.numel() // self.n

    def linear(self, U, out=None):
        out = self._out(U, out)
        B = self._batch(U)
        self._check(self._lib.pavg_linear(self._h, _ptr(U, self.n, B), _ptr(out, self.n, B), B, _stream()))
        return out

    def linear_noalloc(self, U, out=None):
        """L U for one state through the entry point that allocates no device
        memory (scratch in a static device array; refinement <= 5)."""
        out = self._out(U, out)
        self._check(self._lib.pavg_linear_noalloc(self._h, _ptr(U, self.n), _ptr(out, self.n), _stream()))
        return out

    def nonlinear(self, U, out=None):
        out = self._out(U, out)
        B = self._batch(U)
        self._check(self._lib.pavg_nonlinear(self._h, _ptr(U, self.n, B), _ptr(out, self.n, B), B, _stream()))
        return out

    def expL(self, t, U, out=None):
        out = self._out(U, out)
        B = self._batch(U)
        self._check(self._lib.pavg_expL_apply(self._h, float(t), _ptr(U, self.n, B), _ptr(out, self.n, B), B,
                                              _stream()))
        return out

    def averaged_rhs(self, T, M, U, out=None):
        out = self._out(U, out)
        self._check(self._lib.pavg_averaged_rhs(self._h, float(T), int(M), _ptr(U, self.n), _ptr(out, self.n),
                                                _stream()))
        return out

    def averaged_rhs_group(self, T, M, m0, m1, U, out=None):
        """Terms m0 .. m1-1 of the M-shift average (weights of the whole rule)."""
        out = self._out(U, out)
        self._check(self._lib.pavg_averaged_rhs_group(self._h, float(T), int(M), int(m0), int(m1), _ptr(U, self.n),
                                                      _ptr(out, self.n), _stream()))
        return out

    def averaged_rhs_marching(self, T, M, U, out=None):
        """The average by shift marching (pavg.h)."""
        out = self._out(U, out)
        self._check(self._lib.pavg_averaged_rhs_marching(self._h, float(T), int(M), _ptr(U, self.n),
                                                         _ptr(out, self.n), _stream()))
        return out

    def averaged_rhs_literal(self, T, M, U, out=None):
        out = self._out(U, out)
        self._check(self._lib.pavg_averaged_rhs_literal(self._h, float(T), int(M), _ptr(U, self.n),
                                                        _ptr(out, self.n), _stream()))
        return out

    def timestep(self, dt, T, M, U, nsteps=1):
        self._check(self._lib.pavg_timestep(self._h, float(dt), float(T), int(M), _ptr(U, self.n), int(nsteps),
                                            _stream()))
        return U


class Batch:
    """Independent instances (Models) evaluated together: their Chebyshev
    chains and Clenshaw sums each in one persistent launch (pavg.h, batches)."""

    def __init__(self, models):
        self._lib = lib()
        self.models = list(models)
        n = len(self.models)
        arr = (ctypes.c_void_p * n)(*[m._h for m in self.models])
        h = ctypes.c_void_p()
        rc = self._lib.pavg_batch_create(arr, n, ctypes.byref(h))
        if rc:
            raise PavgError(rc, "pavg_batch_create failed")
        self._h = h

    def _check(self, rc):
        if rc:
            raise PavgError(rc, self._lib.pavg_batch_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.pavg_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _arrays(self, T, M, U):
        n = len(self.models)
        if not (len(T) == len(M) == len(U) == n):
            raise ValueError("one T, M and state per instance")
        Ta = (ctypes.c_double * n)(*[float(t) for t in T])
        Ma = (ctypes.c_int * n)(*[int(m) for m in M])
        Ua = (ctypes.c_void_p * n)(*[_ptr(u, m.n).value for u, m in zip(U, self.models)])
        return Ta, Ma, Ua

    def averaged_rhs(self, T, M, U, out=None):
        """out_i = N-bar_i(U_i) for every instance; returns the list of outputs."""
        Ta, Ma, Ua = self._arrays(T, M, U)
        out = [torch.empty_like(u) for u in U] if out is None else out
        Oa = (ctypes.c_void_p * len(out))(*[_ptr(o, m.n).value for o, m in zip(out, self.models)])
        self._check(self._lib.pavg_batch_averaged_rhs(self._h, Ta, Ma, Ua, Oa, _stream()))
        return out

    def timestep(self, dt, T, M, U, nsteps=1):
        """nsteps averaged Lawson RK4 steps of every instance, in place on U."""
        Ta, Ma, Ua = self._arrays(T, M, U)
        Da = (ctypes.c_double * len(U))(*[float(x) for x in dt])
        self._check(self._lib.pavg_batch_timestep(self._h, Da, Ta, Ma, Ua, int(nsteps), _stream()))
        return U

    def autotune(self, T, M, U):
        Ta, Ma, Ua = self._arrays(T, M, U)
        c = BatchConfig()
        self._check(self._lib.pavg_batch_autotune(self._h, Ta, Ma, Ua, _stream(), ctypes.byref(c)))
        return {k: getattr(c, k) for k, _ in BatchConfig._fields_}

    def set_config(self, threads, blocks_per_sm, resident=0, weighting=0, strategy=0):
        c = BatchConfig(threads, blocks_per_sm, resident, weighting, 0.0, strategy)
        self._check(self._lib.pavg_batch_set_config(self._h, ctypes.byref(c)))

    def config(self):
        c = BatchConfig()
        self._check(self._lib.pavg_batch_get_config(self._h, ctypes.byref(c)))
        return {k: getattr(c, k) for k, _ in BatchConfig._fields_}

    def kernel_time(self):
        """(forward ms, backward ms) of the two persistent launches of the last call."""
        f, g = ctypes.c_double(), ctypes.c_double()
        self._check(self._lib.pavg_batch_kernel_time(self._h, ctypes.byref(f), ctypes.byref(g)))
        return f.value, g.value

    def norms(self, U):
        """(||u||_L2, ||u||_H(div), ||eta||_L2) of a state (the paper's error norms)."""
        import numpy as np
        out = np.zeros(3)
        self._check(self._lib.pavg_norms(self._h, _ptr(U, self.n), out.ctypes.data_as(ctypes.c_void_p), _stream()))
        return tuple(float(x) for x in out)

    def sync(self):
        self._check(self._lib.pavg_batch_sync(self._h, _stream()))


N_SUR_IN = 124
N_SUR_OUT = 15


def _fptr(t, n=None):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise TypeError("expected a contiguous float32 CUDA tensor")
    if n is not None and t.numel() != n:
        raise ValueError(f"expected {n} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


class Surrogate:
    """Learned mesh-local correction of a cheap few-shift average towards the
    large-M average (pavg.h, learned surrogate)."""

    def __init__(self, hidden=128, seed=2103):
        import numpy as np
        self._lib = lib()
        h = ctypes.c_void_p()
        rc = self._lib.pavg_surrogate_create(int(hidden), ctypes.c_uint64(seed), ctypes.byref(h))
        if rc:
            raise PavgError(rc, "pavg_surrogate_create failed")
        self._h = h
        self.hidden = hidden
        n = ctypes.c_int64()
        self._check(self._lib.pavg_surrogate_nparams(h, ctypes.byref(n)))
        self.nparams = n.value
        self._np = np

    def _check(self, rc):
        if rc:
            raise PavgError(rc, self._lib.pavg_surrogate_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.pavg_surrogate_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self):
        out = self._np.zeros(self.nparams, dtype=self._np.float32)
        self._check(self._lib.pavg_surrogate_get_params(self._h, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def set_params(self, p):
        p = self._np.ascontiguousarray(p, dtype=self._np.float32)
        if p.size != self.nparams:
            raise ValueError("wrong parameter count")
        self._check(self._lib.pavg_surrogate_set_params(self._h, p.ctypes.data_as(ctypes.c_void_p)))

    def scaling(self):
        np = self._np
        mx, sx = np.zeros(N_SUR_IN, np.float32), np.zeros(N_SUR_IN, np.float32)
        my, sy = np.zeros(N_SUR_OUT, np.float32), np.zeros(N_SUR_OUT, np.float32)
        self._check(self._lib.pavg_surrogate_get_scaling(self._h, *[a.ctypes.data_as(ctypes.c_void_p)
                                                                    for a in (mx, sx, my, sy)]))
        return mx, sx, my, sy

    def set_scaling(self, mx, sx, my, sy):
        np = self._np
        arrs = [np.ascontiguousarray(a, dtype=np.float32) for a in (mx, sx, my, sy)]
        self._check(self._lib.pavg_surrogate_set_scaling(self._h, *[a.ctypes.data_as(ctypes.c_void_p)
                                                                    for a in arrs]))

    def add_pairs(self, model, U, Vc, Vf):
        n = len(U)
        arr = lambda L: (ctypes.c_void_p * n)(*[_ptr(x, model.n).value for x in L])
        self._check(self._lib.pavg_surrogate_add_pairs(self._h, model._h, n, arr(U), arr(Vc), arr(Vf), _stream()))

    def rows(self):
        r = ctypes.c_int64()
        self._check(self._lib.pavg_surrogate_rows(self._h, ctypes.byref(r)))
        return r.value

    def fit_scaling(self):
        self._check(self._lib.pavg_surrogate_fit_scaling(self._h, _stream()))

    def train(self, epochs, batch=8192, lr=1e-3, seed=7706):
        loss = (ctypes.c_double * max(epochs, 1))()
        self._check(self._lib.pavg_surrogate_train(self._h, int(epochs), int(batch), float(lr), ctypes.c_uint64(seed),
                                                   loss, _stream()))
        return list(loss)[:epochs]

    def gradient(self, X, Z):
        B = X.shape[0]
        g = torch.empty(self.nparams, dtype=torch.float32, device=X.device)
        loss = ctypes.c_double()
        self._check(self._lib.pavg_surrogate_gradient(self._h, _fptr(X, B * N_SUR_IN), _fptr(Z, B * N_SUR_OUT), int(B),
                                                      _fptr(g), ctypes.byref(loss), _stream()))
        return loss.value, g

    def adam_step(self, grad, lr):
        self._check(self._lib.pavg_surrogate_adam_step(self._h, _fptr(grad, self.nparams), float(lr), _stream()))

    def features(self, model, U, V, standardised=False):
        X = torch.empty((model.n_cells, N_SUR_IN), dtype=torch.float32, device=U.device)
        self._check(self._lib.pavg_surrogate_features(self._h, model._h, _ptr(U, model.n), _ptr(V, model.n), _fptr(X),
                                                      1 if standardised else 0, _stream()))
        return X

    def apply(self, model, U, V, out=None, bf16=False):
        out = torch.empty_like(U) if out is None else out
        self._check(self._lib.pavg_surrogate_apply(self._h, model._h, _ptr(U, model.n), _ptr(V, model.n),
                                                   _ptr(out, model.n), 1 if bf16 else 0, _stream()))
        return out

    def averaged_rhs(self, model, T, Mc, Mf, U, out=None, threshold=1e-3, check=True, bf16=False):
        """(out, used_fallback, rel_err): the surrogate form of N-bar(U) judged by the Mf-shift sum."""
        out = torch.empty_like(U) if out is None else out
        fb, err = ctypes.c_int(), ctypes.c_double()
        self._check(self._lib.pavg_surrogate_averaged_rhs(self._h, model._h, float(T), int(Mc), int(Mf),
                                                          float(threshold), 1 if check else 0, 1 if bf16 else 0,
                                                          _ptr(U, model.n), _ptr(out, model.n), ctypes.byref(fb),
                                                          ctypes.byref(err), _stream()))
        return out, bool(fb.value), err.value
