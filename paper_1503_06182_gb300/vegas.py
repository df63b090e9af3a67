"""Thin ctypes binding of libgvegas.so (include/vegas.h).

The functions keep the C names and only marshal arguments: every step of the
VEGAS iteration runs in the library's CUDA kernels.  Errors raise
``VegasError`` carrying the status code.  The library is loaded on first use;
if it has not been built, that raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgvegas.so")

VEGAS_OK = 0
VEGAS_EINVAL, VEGAS_ENOMEM, VEGAS_ECUDA, VEGAS_EGRID = -1, -2, -3, -4
VEGAS_ENONFINITE, VEGAS_EDEVICE, VEGAS_ESTATE = -5, -6, -7
VEGAS_GAUSS, VEGAS_DY, VEGAS_EE3J, VEGAS_DY_NLO = 0, 1, 2, 3
VEGAS_OPT_ALPHA, VEGAS_OPT_PRECISION, VEGAS_OPT_ADAPT, VEGAS_OPT_EPT = 0, 1, 2, 3
VEGAS_OPT_NONFINITE, VEGAS_OPT_GRAPH, VEGAS_OPT_TIMING, VEGAS_OPT_BATCH_ID = 4, 5, 6, 7
VEGAS_OPT_PDL, VEGAS_OPT_STRAT, VEGAS_OPT_BETA, VEGAS_OPT_BATCH_GRID = 8, 9, 10, 11
VEGAS_KERNEL_FILL, VEGAS_KERNEL_REDUCE, VEGAS_KERNEL_REFINE = 0, 1, 2
VEGAS_NGRAD = 5
VEGAS_MAX_PARAMS = 16
VEGAS_TILE = 1024
VEGAS_NOALLOC_MAX_WORDS = 1 << 18
VEGAS_HIST_MAX_BINS = 1000
VEGAS_PIPE_FFMA, VEGAS_PIPE_DFMA, VEGAS_PIPE_IMAD, VEGAS_PIPE_MUFU = 0, 1, 2, 3

_lock = threading.Lock()
_lib = None


class VegasError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {strerror(status)} ({status})")


_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_vp = C.c_void_p


_RAW = None


def _raw():
    """A second handle on the library whose per-stage entry points take plain
    pointers (the checked signatures of lib() cost microseconds per call)."""
    global _RAW
    if _RAW is None:
        R = C.CDLL(lib()._name)
        R.vegas_iterate.argtypes = [_vp, C.c_int64, C.c_int, C.c_int, C.c_void_p, C.c_int,
                                    C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        R.vegas_iterate.restype = C.c_int
        _RAW = R
    return _RAW


def lib():
    """The loaded library (raises if it is not built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built: call paper_1503_06182_gb300.build.build() "
                               "(needs nvcc); the VEGAS path has no CPU fallback")
        L = C.CDLL(LIB_PATH)
        sig = {
            "vegas_init": ([C.c_int, C.c_int, C.c_uint64, C.POINTER(_vp)], C.c_int),
            "vegas_free": ([_vp], None),
            "vegas_set_option": ([_vp, C.c_int, C.c_double], C.c_int),
            "vegas_set_stream": ([_vp, _vp], C.c_int),
            "vegas_workspace_size": ([_vp, C.c_int64, C.c_int, C.POINTER(C.c_size_t)], C.c_int),
            "vegas_set_workspace": ([_vp, _vp, C.c_size_t], C.c_int),
            "vegas_iterate": ([_vp, C.c_int64, C.c_int, C.c_int, _dp, C.c_int, C.POINTER(C.c_double),
                               C.POINTER(C.c_double), C.POINTER(C.c_double), _vp], C.c_int),
            "vegas_launch": ([_vp, C.c_int64, C.c_int, C.c_int, _dp, C.c_int], C.c_int),
            "vegas_fetch": ([_vp, C.POINTER(C.c_double), C.POINTER(C.c_double),
                             C.POINTER(C.c_double), _vp, C.POINTER(C.c_int64)], C.c_int),
            "vegas_grid_get": ([_vp, _dp], C.c_int),
            "vegas_grid_set": ([_vp, _dp], C.c_int),
            "vegas_state_size": ([_vp, C.POINTER(C.c_size_t)], C.c_int),
            "vegas_state_get": ([_vp, _vp, C.c_size_t], C.c_int),
            "vegas_state_set": ([_vp, _vp, C.c_size_t], C.c_int),
            "vegas_adjoint": ([_vp, C.c_int64, C.c_int, C.c_int, _dp, C.c_int, _dp, _dp,
                               C.POINTER(C.c_double), C.POINTER(C.c_double), _vp], C.c_int),
            "vegas_eval_events": ([_vp, C.c_int, _dp, C.c_int, C.c_uint32, _i64p, C.c_int64, _dp,
                                   _i32p], C.c_int),
            "vegas_rng_words": ([C.c_uint64, C.c_uint32, C.c_uint32, C.c_int64, C.c_int64, C.c_int,
                                 _u32p], C.c_int),
            "vegas_rng_words_noalloc": ([C.c_uint64, C.c_uint32, C.c_uint32, C.c_int64, C.c_int64,
                                         C.c_int, _u32p], C.c_int),
            "vegas_last_sums": ([_vp, _dp], C.c_int),
            "vegas_pipe_peak": ([C.c_int, C.c_double, C.POINTER(C.c_double)], C.c_int),
            "vegas_hist_set": ([_vp, C.c_int, C.c_double, C.c_double], C.c_int),
            "vegas_strat_get": ([_vp, C.POINTER(C.c_int), C.POINTER(C.c_int64), _vp, _vp], C.c_int),
            "vegas_strat_set": ([_vp, C.c_int64, _vp], C.c_int),
            "vegas_hist_get": ([_vp, _vp, _vp, _vp], C.c_int),
            "vegas_kernel_time": ([_vp, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int64),
                                   C.c_int], C.c_int),
            "vegas_get_ept": ([_vp, C.POINTER(C.c_int)], C.c_int),
            "vegas_batch_create": ([C.c_int, _i32p, _i64p, _i32p, _dp, _i32p, C.c_int, C.c_uint64,
                                    C.c_int, C.POINTER(_vp)], C.c_int),
            "vegas_batch_free": ([_vp], None),
            "vegas_batch_set_option": ([_vp, C.c_int, C.c_double], C.c_int),
            "vegas_batch_set_stream": ([_vp, _vp], C.c_int),
            "vegas_batch_iterate": ([_vp, C.c_int, _dp, _dp, _dp, _vp], C.c_int),
            "vegas_batch_grid_get": ([_vp, C.c_int, _dp], C.c_int),
            "vegas_strerror": ([C.c_int], C.c_char_p),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
        return L


def strerror(status: int) -> str:
    try:
        return lib().vegas_strerror(int(status)).decode()
    except RuntimeError:
        return "library not loaded"


def _check(st: int, what: str, allow=()):
    if st != VEGAS_OK and st not in allow:
        raise VegasError(st, what)
    return st


def _params(params) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(params, dtype=np.float64).reshape(-1))


def _ptr(a):
    return None if a is None else a.ctypes.data


# ---------------------------------------------------------------------------- context calls
def vegas_init(ndim: int, nbins: int, seed: int):
    h = _vp()
    _check(lib().vegas_init(ndim, nbins, seed, C.byref(h)), "vegas_init")
    return h


def vegas_free(h) -> None:
    if h:
        lib().vegas_free(h)


def vegas_set_option(h, key: int, value: float) -> None:
    _check(lib().vegas_set_option(h, key, float(value)), "vegas_set_option")


def vegas_set_stream(h, stream: int | None) -> None:
    _check(lib().vegas_set_stream(h, stream or None), "vegas_set_stream")


def vegas_workspace_size(h, ncall: int, itmx: int) -> int:
    n = C.c_size_t()
    _check(lib().vegas_workspace_size(h, ncall, itmx, C.byref(n)), "vegas_workspace_size")
    return n.value


def vegas_set_workspace(h, device_ptr: int | None, nbytes: int) -> None:
    _check(lib().vegas_set_workspace(h, device_ptr or None, nbytes), "vegas_set_workspace")


def _params_fast(params) -> np.ndarray:
    if (type(params) is np.ndarray and params.dtype == np.float64 and params.ndim == 1
            and params.flags.c_contiguous):
        return params
    return _params(params)


_PARAM_PTR = [None, 0]  # the last parameter array passed and its data address


def _params_ptr(params):
    """A float64 parameter array and its address; the address of the array
    object passed last is kept (an array's data does not move)."""
    if params is _PARAM_PTR[0]:
        return params, _PARAM_PTR[1]
    p = _params_fast(params)
    a = p.ctypes.data
    if p is params:
        _PARAM_PTR[0], _PARAM_PTR[1] = p, a
    return p, a


def vegas_iterate(h, ncall: int, itmx: int, integrand_id: int, params, allow_nonfinite=False):
    """Returns (integral, error, chi2_dof, per_iter[itmx, 2], status).  This is
    the per-stage call, so it passes raw pointers (no per-call argument
    checking by ctypes); the three scalars and the records share one buffer."""
    p, pa = _params_ptr(params)
    buf = np.empty(3 + 2 * itmx)
    a = buf.ctypes.data
    st = _raw().vegas_iterate(h, ncall, itmx, integrand_id, pa, p.shape[0], a, a + 8, a + 16,
                              a + 24)
    _check(st, "vegas_iterate", (VEGAS_ENONFINITE,) if allow_nonfinite else ())
    return float(buf[0]), float(buf[1]), float(buf[2]), buf[3:].reshape(itmx, 2), st


def vegas_launch(h, ncall: int, itmx: int, integrand_id: int, params) -> None:
    p = _params(params)
    _check(lib().vegas_launch(h, ncall, itmx, integrand_id, p, len(p)), "vegas_launch")


def vegas_fetch(h, itmx: int, allow_nonfinite=False):
    """Returns (integral, error, chi2_dof, per_iter[itmx, 2], nonfinite, status)."""
    I, e, c = C.c_double(), C.c_double(), C.c_double()
    nf = C.c_int64()
    per = np.zeros((itmx, 2))
    st = lib().vegas_fetch(h, C.byref(I), C.byref(e), C.byref(c), _ptr(per), C.byref(nf))
    _check(st, "vegas_fetch", (VEGAS_ENONFINITE,) if allow_nonfinite else ())
    return I.value, e.value, c.value, per, nf.value, st


def vegas_grid_get(h, ndim: int, nbins: int) -> np.ndarray:
    out = np.zeros((ndim, nbins + 1))
    _check(lib().vegas_grid_get(h, out.reshape(-1)), "vegas_grid_get")
    return out


def vegas_grid_set(h, edges) -> None:
    e = np.ascontiguousarray(edges, dtype=np.float64)
    _check(lib().vegas_grid_set(h, e.reshape(-1)), "vegas_grid_set")


def vegas_state_get(h) -> bytes:
    n = C.c_size_t()
    _check(lib().vegas_state_size(h, C.byref(n)), "vegas_state_size")
    buf = (C.c_char * n.value)()
    _check(lib().vegas_state_get(h, buf, n.value), "vegas_state_get")
    return bytes(buf)


def vegas_state_set(h, blob: bytes) -> None:
    buf = (C.c_char * len(blob)).from_buffer_copy(blob)
    _check(lib().vegas_state_set(h, buf, len(blob)), "vegas_state_set")


def vegas_adjoint(h, ncall: int, itmx: int, integrand_id: int, params):
    """Returns (grad[5], grad_err[5], integral, error, per_iter_grad[itmx, 5, 2])."""
    p = _params(params)
    g = np.zeros(VEGAS_NGRAD)
    ge = np.zeros(VEGAS_NGRAD)
    I, e = C.c_double(), C.c_double()
    per = np.zeros((itmx, VEGAS_NGRAD, 2))
    _check(lib().vegas_adjoint(h, ncall, itmx, integrand_id, p, len(p), g, ge, C.byref(I),
                               C.byref(e), _ptr(per)), "vegas_adjoint")
    return g, ge, I.value, e.value, per


def vegas_eval_events(h, ndim: int, integrand_id: int, params, iteration: int, events):
    """Returns (w[n], bins[n, ndim]) for the given event indices."""
    p = _params(params)
    ev = np.ascontiguousarray(events, dtype=np.int64)
    w = np.zeros(len(ev))
    b = np.zeros((len(ev), ndim), np.int32)
    _check(lib().vegas_eval_events(h, integrand_id, p, len(p), iteration, ev, len(ev), w,
                                   b.reshape(-1)), "vegas_eval_events")
    return w, b


def vegas_rng_words(seed: int, iteration: int, batch: int, first_event: int, n: int,
                    ndim: int) -> np.ndarray:
    out = np.zeros((n, ndim), np.uint32)
    _check(lib().vegas_rng_words(seed, iteration, batch, first_event, n, ndim, out.reshape(-1)),
           "vegas_rng_words")
    return out


def vegas_rng_words_noalloc(seed: int, iteration: int, batch: int, first_event: int, n: int,
                            ndim: int) -> np.ndarray:
    """vegas_rng_words through the library's fixed device buffer (no device
    allocation); n * ndim is limited to VEGAS_NOALLOC_MAX_WORDS."""
    out = np.zeros((n, ndim), np.uint32)
    st = lib().vegas_rng_words_noalloc(seed, iteration, batch, first_event, n, ndim,
                                       out.reshape(-1))
    if st == VEGAS_EINVAL and ndim >= 1 and n * ndim > VEGAS_NOALLOC_MAX_WORDS:
        raise VegasError(st, f"vegas_rng_words_noalloc: n*ndim = {n * ndim} exceeds the fixed "
                             f"buffer of {VEGAS_NOALLOC_MAX_WORDS} words")
    _check(st, "vegas_rng_words_noalloc")
    return out


def vegas_pipe_peak(pipe: int, ms: float = 50.0) -> float:
    """Measured rate of one arithmetic pipe (VEGAS_PIPE_*), flops or ops per second."""
    r = C.c_double()
    _check(lib().vegas_pipe_peak(int(pipe), float(ms), C.byref(r)), "vegas_pipe_peak")
    return r.value


def vegas_last_sums(h, ndim: int, nbins: int) -> np.ndarray:
    out = np.zeros(2 + ndim * nbins)
    _check(lib().vegas_last_sums(h, out), "vegas_last_sums")
    return out


def vegas_hist_set(h, nbins: int, lo: float = 0.0, hi: float = 1.0) -> None:
    _check(lib().vegas_hist_set(h, int(nbins), float(lo), float(hi)), "vegas_hist_set")


def vegas_hist_get(h, nbins: int):
    """(value, error, last_sums[2, nbins + 2]) of the last stage's histogram;
    index 0 is the underflow bin, nbins + 1 the overflow bin."""
    hb = nbins + 2
    val, err, last = np.zeros(hb), np.zeros(hb), np.zeros((2, hb))
    _check(lib().vegas_hist_get(h, _ptr(val), _ptr(err), _ptr(last)), "vegas_hist_get")
    return val, err, last


def vegas_strat_get(h):
    """(strata per axis, counts[nh] for the next iteration, var[nh] of the last)."""
    s, nh = C.c_int(), C.c_int64()
    _check(lib().vegas_strat_get(h, C.byref(s), C.byref(nh), None, None), "vegas_strat_get")
    counts = np.zeros(nh.value, np.int32)
    var = np.zeros(nh.value)
    _check(lib().vegas_strat_get(h, None, None, _ptr(counts), _ptr(var)), "vegas_strat_get")
    return s.value, counts, var


def vegas_strat_set(h, ncall: int, counts) -> None:
    counts = np.ascontiguousarray(counts, np.int32)
    _check(lib().vegas_strat_set(h, int(ncall), _ptr(counts)), "vegas_strat_set")


def vegas_kernel_time(h, kernel: int, reset: bool = False):
    ms = C.c_double()
    n = C.c_int64()
    _check(lib().vegas_kernel_time(h, kernel, C.byref(ms), C.byref(n), int(reset)),
           "vegas_kernel_time")
    return ms.value, n.value


def vegas_get_ept(h) -> int:
    v = C.c_int()
    _check(lib().vegas_get_ept(h, C.byref(v)), "vegas_get_ept")
    return v.value


# ---------------------------------------------------------------------------- batch calls
def vegas_batch_create(ndim, ncall, integrand_id, params, nbins: int, seed: int, precision: int):
    n = len(ndim)
    P = np.zeros((n, VEGAS_MAX_PARAMS))
    npar = np.zeros(n, np.int32)
    for i, p in enumerate(params):
        P[i, :len(p)] = p
        npar[i] = len(p)
    h = _vp()
    _check(lib().vegas_batch_create(n, np.ascontiguousarray(ndim, np.int32),
                                    np.ascontiguousarray(ncall, np.int64),
                                    np.ascontiguousarray(integrand_id, np.int32), P.reshape(-1),
                                    npar, nbins, seed, precision, C.byref(h)),
           "vegas_batch_create")
    return h


def vegas_batch_free(h) -> None:
    if h:
        lib().vegas_batch_free(h)


def vegas_batch_set_option(h, key: int, value: float) -> None:
    _check(lib().vegas_batch_set_option(h, key, float(value)), "vegas_batch_set_option")


def vegas_batch_set_stream(h, stream) -> None:
    _check(lib().vegas_batch_set_stream(h, stream or None), "vegas_batch_set_stream")


def vegas_batch_iterate(h, n: int, itmx: int):
    """Returns (integral[n], error[n], chi2_dof[n], per_iter[n, itmx, 2])."""
    I = np.zeros(n)
    e = np.zeros(n)
    c = np.zeros(n)
    per = np.zeros((n, itmx, 2))
    _check(lib().vegas_batch_iterate(h, itmx, I, e, c, _ptr(per)), "vegas_batch_iterate")
    return I, e, c, per


def vegas_batch_grid_get(h, index: int, ndim: int, nbins: int) -> np.ndarray:
    out = np.zeros((ndim, nbins + 1))
    _check(lib().vegas_batch_grid_get(h, index, out.reshape(-1)), "vegas_batch_grid_get")
    return out


# ---------------------------------------------------------------------------- convenience
class Vegas:
    """One VEGAS integration on the current CUDA device (owns a context).

    If ``torch_workspace`` is true, the device workspace is a torch tensor from
    PyTorch's caching allocator and the work runs on torch's current stream."""

    def __init__(self, ndim: int, nbins: int, seed: int = 1234, *, precision: str = "fp64",
                 alpha: float = 1.5, torch_workspace: bool = False, stream=None):
        self.ndim, self.nbins, self.seed = ndim, nbins, seed
        self.h = vegas_init(ndim, nbins, seed)
        self._ws = None
        self._ws_for = None  # the (ncall, itmx) the workspace was last checked for
        self._torch_ws = torch_workspace
        self.set(VEGAS_OPT_PRECISION, 1 if precision == "fp32" else 0)
        self.set(VEGAS_OPT_ALPHA, alpha)
        if stream is not None:
            vegas_set_stream(self.h, stream)

    def set(self, key: int, value: float) -> "Vegas":
        vegas_set_option(self.h, key, value)
        self._ws_for = None  # options can change the workspace a stage needs
        return self

    def _workspace(self, ncall: int, itmx: int):
        if not self._torch_ws or (ncall, itmx) == self._ws_for:
            return
        import torch

        need = vegas_workspace_size(self.h, ncall, itmx)
        self._ws_for = (ncall, itmx)
        if self._ws is None or self._ws.numel() < need:
            self._ws = torch.empty(need + 256, dtype=torch.uint8, device="cuda")
            ptr = self._ws.data_ptr()
            ptr = (ptr + 255) & ~255
            vegas_set_workspace(self.h, ptr, need)

    def iterate(self, ncall: int, itmx: int, integrand_id: int, params, allow_nonfinite=False):
        self._workspace(ncall, itmx)
        return vegas_iterate(self.h, ncall, itmx, integrand_id, params, allow_nonfinite)

    def launch(self, ncall: int, itmx: int, integrand_id: int, params):
        self._workspace(ncall, itmx)
        vegas_launch(self.h, ncall, itmx, integrand_id, params)

    def fetch(self, itmx: int, allow_nonfinite=False):
        return vegas_fetch(self.h, itmx, allow_nonfinite)

    def adjoint(self, ncall: int, itmx: int, params, integrand_id: int = VEGAS_DY):
        self._workspace(ncall, itmx)
        return vegas_adjoint(self.h, ncall, itmx, integrand_id, params)

    @property
    def grid(self) -> np.ndarray:
        return vegas_grid_get(self.h, self.ndim, self.nbins)

    @grid.setter
    def grid(self, edges) -> None:
        vegas_grid_set(self.h, edges)

    def state(self) -> bytes:
        return vegas_state_get(self.h)

    def restore(self, blob: bytes) -> None:
        vegas_state_set(self.h, blob)

    def eval_events(self, integrand_id: int, params, iteration: int, events):
        return vegas_eval_events(self.h, self.ndim, integrand_id, params, iteration, events)

    def last_sums(self) -> np.ndarray:
        return vegas_last_sums(self.h, self.ndim, self.nbins)

    def hist_set(self, nbins: int, lo: float = 0.0, hi: float = 1.0) -> "Vegas":
        """Fill a histogram of the integrand's observable in later stages
        (nbins = 0: none)."""
        vegas_hist_set(self.h, nbins, lo, hi)
        self._hist_n = int(nbins)
        self._ws_for = None
        return self

    def strat(self):
        """VEGAS+ state: (strata per axis, allocation, last per-hypercube variances)."""
        return vegas_strat_get(self.h)

    def strat_set(self, ncall: int, counts) -> None:
        vegas_strat_set(self.h, ncall, counts)

    def hist(self):
        """(value, error, last_sums) of the last stage's histogram."""
        return vegas_hist_get(self.h, getattr(self, "_hist_n", 0))

    def close(self) -> None:
        if self.h:
            vegas_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class VegasBatch:
    """Many independent VEGAS integrations advanced together (owns a batch).

    ``members`` is a list of ``(ndim, ncall, integrand_id, params)``; member b
    draws its events with Philox batch word b."""

    def __init__(self, members, nbins: int, seed: int = 1234, *, precision: str = "fp64",
                 alpha: float = 1.5):
        self.members = [(int(d), int(c), int(i), tuple(p)) for d, c, i, p in members]
        self.nbins, self.seed = nbins, seed
        self.h = vegas_batch_create([m[0] for m in self.members], [m[1] for m in self.members],
                                    [m[2] for m in self.members], [m[3] for m in self.members],
                                    nbins, seed, 1 if precision == "fp32" else 0)
        self.set(VEGAS_OPT_ALPHA, alpha)

    def __len__(self) -> int:
        return len(self.members)

    def set(self, key: int, value: float) -> "VegasBatch":
        vegas_batch_set_option(self.h, key, value)
        return self

    def iterate(self, itmx: int):
        """(integral[n], error[n], chi2_dof[n], per_iter[n, itmx, 2])."""
        return vegas_batch_iterate(self.h, len(self.members), itmx)

    def grid(self, index: int) -> np.ndarray:
        return vegas_batch_grid_get(self.h, index, self.members[index][0], self.nbins)

    def close(self) -> None:
        if self.h:
            vegas_batch_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
