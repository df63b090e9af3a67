"""Oracle: plain FP64 CPU VEGAS (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference leg of ``bench.py`` may import this package.  It wraps
``vegas_oracle.c`` (plain C99 + OpenMP, built with gcc) through ctypes and
shares no code with the CUDA library.

Functions follow the VEGAS method that the paper parallelises (Abstract;
Section 2.1: events of one iteration evaluated independently, all events
combined, serial grid optimisation; Section 2.2: per-event groups of random
numbers, Kahan summation, results independent of the thread count).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vegas_oracle.c")
_LIB = os.environ.get("ORACLE_LIB_OVERRIDE") or os.path.join(_HERE, "liboracle_vegas.so")
_SRC = os.environ.get("ORACLE_SRC_OVERRIDE") or _SRC
_lock = threading.Lock()
_lib = None

GAUSS, DY, EE3J, DYNLO = 0, 1, 2, 3
NGRAD = 5
CHUNK = 4096

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_up = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no CUDA involved)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c99", "-fopenmp", "-ffp-contract=off", "-fPIC",
               "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = C.CDLL(_LIB)
        lib.oracle_philox4x32_10.argtypes = [_up, _up, _up]
        lib.oracle_event_words.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint64,
                                           C.c_int, _up]
        lib.oracle_bin_map.argtypes = [C.c_uint32, C.c_int, C.POINTER(C.c_int32),
                                       C.POINTER(C.c_double)]
        lib.oracle_grid_map.argtypes = [_dp, C.c_int, C.c_uint32, C.POINTER(C.c_double)]
        lib.oracle_grid_map.restype = C.c_double
        lib.oracle_integrand.argtypes = [C.c_int, C.c_int, _dp, _dp, C.c_int,
                                         C.POINTER(C.c_double), C.c_void_p, C.c_void_p]
        lib.oracle_dy_dsigma_domega.argtypes = [C.c_int, C.c_double, C.c_double, _dp]
        lib.oracle_dy_dsigma_domega.restype = C.c_double
        lib.oracle_event.argtypes = [C.c_int, C.c_int, C.c_int, _dp, _dp, C.c_int, C.c_uint64,
                                     C.c_uint32, C.c_uint32, C.c_uint64,
                                     C.POINTER(C.c_double), _ip, _dp]
        lib.oracle_combine.argtypes = [C.c_int, _dp, _dp, C.POINTER(C.c_double),
                                       C.POINTER(C.c_double), C.POINTER(C.c_double)]
        lib.oracle_refine.argtypes = [C.c_int, C.c_int, C.c_double, _dp, _dp]
        lib.oracle_iterate.argtypes = [C.c_int, C.c_int, C.c_uint64, C.c_uint32,
                                       C.POINTER(C.c_uint64), C.c_int64, C.c_int, C.c_int, _dp,
                                       C.c_int, C.c_double, C.c_int, _dp,
                                       C.POINTER(C.c_double), C.POINTER(C.c_double),
                                       C.POINTER(C.c_double), C.c_void_p, C.c_void_p,
                                       C.POINTER(C.c_int64)]
        lib.oracle_iterate_hist.argtypes = [C.c_int, C.c_int, C.c_uint64, C.c_uint32,
                                            C.POINTER(C.c_uint64), C.c_int64, C.c_int, C.c_int,
                                            _dp, C.c_int, C.c_double, C.c_int, _dp, C.c_int,
                                            C.c_double, C.c_double, C.POINTER(C.c_double),
                                            C.POINTER(C.c_double), C.POINTER(C.c_double),
                                            C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                            C.c_void_p, C.POINTER(C.c_int64)]
        lib.oracle_observable.argtypes = [C.c_int, C.c_int, _dp, _dp, C.c_int,
                                          C.POINTER(C.c_double)]
        lib.oracle_hist_bin.argtypes = [C.c_double, C.c_int, C.c_double, C.c_double]
        lib.oracle_hist_combine.argtypes = [C.c_int, C.c_int, _dp, _dp, _dp, _dp, _dp]
        lib.oracle_plus_nstrat.argtypes = [C.c_int, C.c_int64]
        lib.oracle_plus_word.argtypes = [C.c_uint32, C.c_uint32, C.c_uint32]
        lib.oracle_plus_word.restype = C.c_uint32
        lib.oracle_plus_weight.argtypes = [C.c_double, C.c_int]
        lib.oracle_plus_weight.restype = C.c_double
        lib.oracle_plus_allocate.argtypes = [C.c_int64, C.c_int64, C.c_int, _dp, _ip]
        lib.oracle_iterate_plus.argtypes = [C.c_int, C.c_int, C.c_uint64, C.c_uint32,
                                            C.POINTER(C.c_uint64), C.c_int64, C.c_int, C.c_int,
                                            _dp, C.c_int, C.c_double, C.c_int, C.c_int, C.c_int,
                                            _dp, _ip, C.POINTER(C.c_double),
                                            C.POINTER(C.c_double), C.POINTER(C.c_double),
                                            C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                            C.c_void_p, C.POINTER(C.c_int64)]
        lib.oracle_adjoint.argtypes = [C.c_int, C.c_int, C.c_uint64, C.c_uint32,
                                       C.POINTER(C.c_uint64), C.c_int64, C.c_int, C.c_int, _dp,
                                       C.c_int, _dp, _dp, _dp, C.POINTER(C.c_double),
                                       C.POINTER(C.c_double), C.c_void_p, C.c_void_p]
        lib.oracle_set_threads.argtypes = [C.c_int]
        lib.oracle_get_threads.restype = C.c_int
        _lib = lib
        return lib


def _check(st: int, what: str):
    if st != 0:
        raise ValueError(f"oracle {what} failed with status {st}")


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def get_threads() -> int:
    return int(_load().oracle_get_threads())


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 (Salmon et al., SC'11) of one counter/key pair."""
    out = np.zeros(4, np.uint32)
    _load().oracle_philox4x32_10(np.ascontiguousarray(ctr, np.uint32),
                                 np.ascontiguousarray(key, np.uint32), out)
    return out


def event_words(seed: int, iteration: int, batch: int, event: int, ndim: int) -> np.ndarray:
    """The event's group of random words: one 32-bit word per axis."""
    out = np.zeros(max(ndim, 1), np.uint32)
    _load().oracle_event_words(seed, iteration, batch, event, ndim, out)
    return out[:ndim]


def bin_map(r: int, nbins: int):
    b = C.c_int32()
    f = C.c_double()
    _load().oracle_bin_map(r, nbins, C.byref(b), C.byref(f))
    return b.value, f.value


def grid_map(edges_axis, nbins: int, r: int):
    """One axis of the adaptive-grid map: returns (x, N * bin width)."""
    x = C.c_double()
    jac = _load().oracle_grid_map(np.ascontiguousarray(edges_axis, np.float64), nbins, r,
                                  C.byref(x))
    return x.value, jac


def integrand(iid: int, x, params, mom: bool = False, grad: bool = False):
    """g(x) at a point of the unit cube; optionally the momenta and dg/dtheta."""
    x = np.ascontiguousarray(x, np.float64)
    params = np.ascontiguousarray(params, np.float64)
    g = C.c_double()
    m = np.zeros(16, np.float64)
    gr = np.zeros(NGRAD, np.float64)
    st = _load().oracle_integrand(iid, len(x), x, params, len(params), C.byref(g),
                                  m.ctypes.data if mom else None,
                                  gr.ctypes.data if grad else None)
    _check(st, "integrand")
    out = [g.value]
    if mom:
        out.append(m.reshape(4, 4))
    if grad:
        out.append(gr)
    return out[0] if len(out) == 1 else tuple(out)


def dy_dsigma_domega(up_type: bool, shat: float, c: float, params) -> float:
    return _load().oracle_dy_dsigma_domega(int(up_type), shat, c,
                                           np.ascontiguousarray(params, np.float64))


def event(iid, ndim, nbins, edges, params, seed, iteration, batch, ev):
    """One event: returns (w, bins[ndim], x[ndim])."""
    edges = np.ascontiguousarray(edges, np.float64)
    params = np.ascontiguousarray(params, np.float64)
    w = C.c_double()
    bins = np.zeros(ndim, np.int32)
    x = np.zeros(ndim, np.float64)
    st = _load().oracle_event(iid, ndim, nbins, edges, params, len(params), seed, iteration,
                              batch, ev, C.byref(w), bins, x)
    _check(st, "event")
    return w.value, bins, x


def combine(Ik, sk):
    Ik = np.ascontiguousarray(Ik, np.float64)
    sk = np.ascontiguousarray(sk, np.float64)
    I, e, c = C.c_double(), C.c_double(), C.c_double()
    _load().oracle_combine(len(Ik), Ik, sk, C.byref(I), C.byref(e), C.byref(c))
    return I.value, e.value, c.value


def uniform_edges(ndim: int, nbins: int) -> np.ndarray:
    return np.tile(np.arange(nbins + 1, dtype=np.float64) / nbins, (ndim, 1))


def refine(d, edges, alpha: float = 1.5) -> np.ndarray:
    """Refined copy of edges (ndim x (nbins+1)) from bin sums d (ndim x nbins)."""
    d = np.ascontiguousarray(d, np.float64)
    out = np.ascontiguousarray(np.array(edges, np.float64, copy=True))
    ndim, nbins = d.shape
    _check(_load().oracle_refine(ndim, nbins, alpha, d.ravel(), out.reshape(-1)), "refine")
    return out


class Result(dict):
    __getattr__ = dict.__getitem__


def observable(iid: int, x, params) -> float:
    """The histogram observable of an event at x: Gauss x_0, Drell-Yan m_ll
    (GeV), 3-jet thrust."""
    x = np.ascontiguousarray(x, np.float64)
    params = np.ascontiguousarray(params, np.float64)
    v = C.c_double()
    _check(_load().oracle_observable(iid, len(x), x, params, len(params), C.byref(v)),
           "observable")
    return v.value


def hist_bin(v: float, nh: int, lo: float, hi: float) -> int:
    """Bin of v among nh bins over [lo, hi): 0 underflow, nh + 1 overflow."""
    return int(_load().oracle_hist_bin(float(v), int(nh), float(lo), float(hi)))


def hist_combine(sk, H, V):
    """Combined histogram (value, error) of per-iteration bin estimates H and
    variances V (m x hb) with the integral's weights."""
    sk = np.ascontiguousarray(sk, np.float64)
    H = np.ascontiguousarray(H, np.float64)
    V = np.ascontiguousarray(V, np.float64)
    m, hb = H.shape
    val, err = np.zeros(hb), np.zeros(hb)
    _load().oracle_hist_combine(m, hb, sk, H.ravel(), V.ravel(), val, err)
    return val, err


def iterate(ndim, nbins, seed, ncall, itmx, iid, params, *, edges=None, iteration=0, batch=0,
            alpha=1.5, adapt=True, want_sums=False, hist=None) -> Result:
    """itmx VEGAS iterations (one stage).  Returns integral, error, chi2dof,
    per_iter (itmx x 2), edges after the stage, the next iteration counter,
    and (optionally) the last iteration's sums.  hist = (nh, lo, hi) adds the
    combined histogram of the observable (hist_value, hist_error: nh + 2
    entries with underflow first and overflow last) and the last iteration's
    per-bin sums (hist_last: sum w then sum w^2)."""
    if edges is None:
        edges = uniform_edges(ndim, nbins)
    edges = np.ascontiguousarray(np.array(edges, np.float64, copy=True))
    params = np.ascontiguousarray(params, np.float64)
    it = C.c_uint64(iteration)
    I, e, c = C.c_double(), C.c_double(), C.c_double()
    per = np.zeros((itmx, 2), np.float64)
    sums = np.zeros(2 + ndim * nbins, np.float64)
    bad = C.c_int64()
    nh, lo, hi = (0, 0.0, 0.0) if hist is None else (int(hist[0]), float(hist[1]), float(hist[2]))
    hb = nh + 2 if nh > 0 else 0
    hval, herr, hlast = np.zeros(max(hb, 1)), np.zeros(max(hb, 1)), np.zeros(max(2 * hb, 1))
    st = _load().oracle_iterate_hist(ndim, nbins, seed, batch, C.byref(it), ncall, itmx, iid,
                                     params, len(params), alpha, int(adapt), edges.reshape(-1),
                                     nh, lo, hi, C.byref(I), C.byref(e), C.byref(c),
                                     per.ctypes.data, sums.ctypes.data if want_sums else None,
                                     hval.ctypes.data, herr.ctypes.data, hlast.ctypes.data,
                                     C.byref(bad))
    _check(st, "iterate")
    r = Result(integral=I.value, error=e.value, chi2dof=c.value, per_iter=per, edges=edges,
               iteration=it.value, nonfinite=bad.value)
    if want_sums:
        r["sums"] = sums
    if hb:
        r["hist_value"], r["hist_error"] = hval, herr
        r["hist_last"] = hlast.reshape(2, hb)
    return r


def adjoint(ndim, nbins, seed, ncall, itmx, params, *, edges=None, iteration=0, batch=0) -> Result:
    """Drell-Yan gradient d sigma / d(M_Z, Gamma_Z, sw2, a, b) on a frozen grid."""
    if edges is None:
        edges = uniform_edges(ndim, nbins)
    edges = np.ascontiguousarray(edges, np.float64)
    params = np.ascontiguousarray(params, np.float64)
    it = C.c_uint64(iteration)
    grad = np.zeros(NGRAD)
    gerr = np.zeros(NGRAD)
    I, e = C.c_double(), C.c_double()
    per = np.zeros((itmx, 2))
    perg = np.zeros((itmx, NGRAD, 2))
    st = _load().oracle_adjoint(ndim, nbins, seed, batch, C.byref(it), ncall, itmx, DY, params,
                                len(params), edges.reshape(-1), grad, gerr, C.byref(I),
                                C.byref(e), per.ctypes.data, perg.ctypes.data)
    _check(st, "adjoint")
    return Result(grad=grad, grad_err=gerr, integral=I.value, error=e.value, per_iter=per,
                  per_iter_grad=perg, iteration=it.value)


# ---------------------------------------------------------------------------- VEGAS+
def plus_nstrat(ndim: int, ncall: int) -> int:
    """Strata per axis: the largest s with 4 s^ndim <= ncall (and s^ndim <= 2^22)."""
    return int(_load().oracle_plus_nstrat(ndim, ncall))


def plus_word(r: int, c: int, s: int) -> int:
    """Stratified word floor((c 2^32 + r) / s)."""
    return int(_load().oracle_plus_word(r, c, s))


def plus_weight(v: float, beta: float) -> float:
    """Allocation weight v^(beta/2) as the stage forms it."""
    return float(_load().oracle_plus_weight(float(v), _beta_j(beta)))


def _beta_j(beta: float) -> int:
    j = int(round(4 * beta))
    if not (0 <= j <= 4 and abs(4 * beta - j) < 1e-12):
        raise ValueError("beta must be one of 0, 1/4, 1/2, 3/4, 1")
    return j


def plus_allocate(ncall: int, var, beta: float = 0.75) -> np.ndarray:
    var = np.ascontiguousarray(var, np.float64)
    n = np.zeros(len(var), np.int32)
    _check(_load().oracle_plus_allocate(len(var), ncall, _beta_j(beta), var, n), "plus_allocate")
    return n


def iterate_plus(ndim, nbins, seed, ncall, itmx, iid, params, *, edges=None, alloc=None,
                 iteration=0, batch=0, alpha=1.5, beta=0.75, nstrat=0, adapt=True) -> Result:
    """itmx VEGAS+ iterations (one stage) from a grid and an allocation
    (None: uniform).  Returns integral, error, chi2dof, per_iter, edges,
    alloc (for the next iteration), calls per iteration, the last
    iteration's sums, per-hypercube variances and means, nstrat."""
    s = nstrat if nstrat > 0 else plus_nstrat(ndim, ncall)
    nh = s ** ndim
    if edges is None:
        edges = uniform_edges(ndim, nbins)
    edges = np.ascontiguousarray(np.array(edges, np.float64, copy=True))
    a = np.zeros(nh, np.int32) if alloc is None else np.array(alloc, np.int32, copy=True)
    params = np.ascontiguousarray(params, np.float64)
    it = C.c_uint64(iteration)
    I, e, c = C.c_double(), C.c_double(), C.c_double()
    per = np.zeros((itmx, 2))
    calls = np.zeros(itmx, np.int64)
    sums = np.zeros(2 + ndim * nbins)
    var = np.zeros(nh)
    mean = np.zeros(nh)
    bad = C.c_int64()
    st = _load().oracle_iterate_plus(ndim, nbins, seed, batch, C.byref(it), ncall, itmx, iid,
                                     params, len(params), alpha, int(adapt), _beta_j(beta), s,
                                     edges.reshape(-1), a, C.byref(I), C.byref(e), C.byref(c),
                                     per.ctypes.data, calls.ctypes.data, sums.ctypes.data,
                                     var.ctypes.data, mean.ctypes.data, C.byref(bad))
    _check(st, "iterate_plus")
    return Result(integral=I.value, error=e.value, chi2dof=c.value, per_iter=per, edges=edges,
                  alloc=a, calls=calls, sums=sums, var=var, mean=mean, nstrat=s,
                  iteration=it.value, nonfinite=bad.value)
