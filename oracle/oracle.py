"""Python entry points of the FP64 CPU oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  It compiles ``vup_oracle.c`` with gcc
(``-O2 -ffp-contract=off -fopenmp``) into ``oracle/_build`` on first use and
wraps it with ctypes.  It shares no code with the CUDA library.

Each wrapper documents the paper passage its C routine follows; see the
header of ``vup_oracle.c``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vup_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libvup_oracle.so")
_lock = threading.Lock()
_lib = None

GAUSS, UNIFORM, TRUNCNORM = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle shared library (plain C, host compiler only)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
               "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            l = C.CDLL(build())
            dp, ip64, ip32, up8 = (C.POINTER(C.c_double), C.POINTER(C.c_int64),
                                   C.POINTER(C.c_int32), C.POINTER(C.c_uint8))
            l.oracle_grid_coord.restype = C.c_double
            l.oracle_grid_coord.argtypes = [C.c_double, C.c_double, C.c_int64, C.c_int64]
            l.oracle_eval_model.restype = C.c_int
            l.oracle_eval_model.argtypes = [C.c_int, dp, C.c_int, ip64, dp, dp, dp]
            l.oracle_bins.restype = None
            l.oracle_bins.argtypes = [C.c_int64, dp, C.c_int, ip32, dp, dp]
            dens = [C.c_int64, up8, dp, dp, dp, dp]
            l.oracle_weights.restype = C.c_int
            l.oracle_weights.argtypes = [C.c_int, ip64, dp, dp] + dens + [C.c_int64, dp, dp]
            l.oracle_propagate.restype = C.c_int
            l.oracle_propagate.argtypes = ([C.c_int, ip64, dp, dp, dp, ip32, C.c_int, C.c_int,
                                            C.c_int64, ip64] + dens + [dp, dp, dp, dp, C.c_int])
            l.oracle_ipsa.restype = C.c_int
            l.oracle_ipsa.argtypes = ([C.c_int, ip64, dp, dp, dp, C.c_int, C.c_int64, ip64]
                                      + dens + [dp, dp, C.c_int])
            l.oracle_ipsa_scale.restype = C.c_int
            l.oracle_ipsa_scale.argtypes = ([C.c_int, ip64, dp, dp, dp, C.c_int, C.c_int64, ip64]
                                            + dens + [dp, dp, C.c_int])
            l.oracle_model_at.restype = C.c_int
            l.oracle_model_at.argtypes = [C.c_int, dp, C.c_int, C.c_int64, dp, dp]
            l.oracle_deviation_moments.restype = C.c_int
            l.oracle_deviation_moments.argtypes = ([C.c_int, ip64, dp, dp, dp, C.c_int, C.c_int64, ip64, dp]
                                                   + dens + [dp])
            l.oracle_ipsa_matrix.restype = None
            l.oracle_ipsa_matrix.argtypes = [C.c_int64, C.c_int, C.c_double, C.c_double, dp, dp, C.c_int,
                                             C.c_double, C.c_double, dp]
            l.oracle_posterior_means.restype = C.c_int
            l.oracle_posterior_means.argtypes = ([C.c_int, ip64, dp, dp, ip32, C.c_int, C.c_int64, ip64] + dens
                                                 + [dp])
            l.oracle_sa_fields.restype = None
            l.oracle_sa_fields.argtypes = [C.c_int64, C.c_int, dp, C.c_double, dp, ip32, ip32, dp]
            _lib = l
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class OracleError(RuntimeError):
    pass


def grid_coords(n, lo, hi):
    """Per-axis midpoints x_{d,a} = lo + (a + 1/2)(hi - lo)/n (Sec. 3)."""
    L = lib()
    return [np.array([L.oracle_grid_coord(lo[d], hi[d], n[d], a) for a in range(n[d])])
            for d in range(len(n))]


def eval_model(model_id, theta, n, lo, hi):
    """y_i = M(x_i; theta) over the tensor grid, row-major (Sec. 2, Eq. modelfunction)."""
    n64 = np.asarray(n, np.int64)
    th = _f64(list(theta) + [0.0] * (8 - len(theta)))
    y = np.empty(int(np.prod(n64)), np.float64)
    rc = lib().oracle_eval_model(int(model_id), _p(th, C.c_double), len(n), _p(n64, C.c_int64),
                                 _p(_f64(lo), C.c_double), _p(_f64(hi), C.c_double),
                                 _p(y, C.c_double))
    if rc:
        raise OracleError(f"model {model_id} does not take {len(n)} axes")
    return y


def bins(y, B):
    """Equal-width output bins over [min y, max y] (Eq. 4), half-open, last closed."""
    y = _f64(y)
    out = np.empty(y.size, np.int32)
    ymin, ymax = C.c_double(), C.c_double()
    lib().oracle_bins(y.size, _p(y, C.c_double), int(B), _p(out, C.c_int32), C.byref(ymin),
                      C.byref(ymax))
    return out, ymin.value, ymax.value


def _dens_args(dens):
    kind = np.ascontiguousarray(dens.kind, np.uint8)
    return [dens.K, _p(kind, C.c_uint8), _p(_f64(dens.mu), C.c_double),
            _p(_f64(dens.sigma), C.c_double), _p(_f64(dens.lo), C.c_double),
            _p(_f64(dens.hi), C.c_double)], (kind,)


def weights(n, lo, hi, dens, k):
    """Normalised input probability vector W[k, :] over the grid (Algorithm VUP)."""
    N = int(np.prod(n))
    W = np.empty(N, np.float64)
    Z = C.c_double()
    n64 = np.asarray(n, np.int64)
    dargs, keep = _dens_args(dens)
    lo64, hi64 = _f64(lo), _f64(hi)
    rc = lib().oracle_weights(len(n), _p(n64, C.c_int64), _p(lo64, C.c_double),
                              _p(hi64, C.c_double), *dargs, int(k), _p(W, C.c_double),
                              C.byref(Z))
    if rc:
        raise OracleError(f"distribution {k} has an empty support on the grid")
    return W, Z.value


def propagate(n, lo, hi, y, bin_ids, B, J, dens, rows=None, threads=0):
    """Raw/central moments, histograms and weight sums for rows ``rows`` (Eq. VUP, Eq. 4).

    Returns dict(raw=[S,J], central=[S,J], hist=[S,B], wsum=[S]).
    """
    K = dens.K
    rows = np.arange(K, dtype=np.int64) if rows is None else np.asarray(rows, np.int64)
    S = rows.size
    raw = np.empty((S, J)); central = np.empty((S, J)); hist = np.empty((S, B)); wsum = np.empty(S)
    n64 = np.asarray(n, np.int64)
    y = _f64(y)
    bi = np.ascontiguousarray(bin_ids, np.int32)
    lo64, hi64 = _f64(lo), _f64(hi)
    dargs, keep = _dens_args(dens)
    rc = lib().oracle_propagate(len(n), _p(n64, C.c_int64), _p(lo64, C.c_double),
                                _p(hi64, C.c_double), _p(y, C.c_double), _p(bi, C.c_int32),
                                int(B), int(J), S, _p(rows, C.c_int64), *dargs,
                                _p(raw, C.c_double), _p(central, C.c_double),
                                _p(hist, C.c_double), _p(wsum, C.c_double), int(threads))
    if rc:
        raise OracleError("a selected distribution has an empty support on the grid")
    return dict(raw=raw, central=central, hist=hist, wsum=wsum)


def ipsa(n, lo, hi, y, J, dens, rows=None, threads=0):
    """Analytic dM_j/dmu and dM_j/dsigma, shape [S, ndim, J] each (IPSA sensitivities)."""
    K = dens.K
    rows = np.arange(K, dtype=np.int64) if rows is None else np.asarray(rows, np.int64)
    S, nd = rows.size, len(n)
    dmu = np.empty((S, nd, J)); dsg = np.empty((S, nd, J))
    n64 = np.asarray(n, np.int64)
    y = _f64(y)
    lo64, hi64 = _f64(lo), _f64(hi)
    dargs, keep = _dens_args(dens)
    rc = lib().oracle_ipsa(nd, _p(n64, C.c_int64), _p(lo64, C.c_double), _p(hi64, C.c_double),
                           _p(y, C.c_double), int(J), S, _p(rows, C.c_int64), *dargs,
                           _p(dmu, C.c_double), _p(dsg, C.c_double), int(threads))
    if rc:
        raise OracleError("a selected distribution has an empty support on the grid")
    return dmu, dsg


def ipsa_scale(n, lo, hi, y, J, dens, rows=None, threads=0):
    """Condition scale of the IPSA sensitivities, shape [S, ndim, J] each:
    sum_i W |s_p| |y|^j + |sbar_p| sum_i W |y|^j for p = mu and sigma (the sum
    of the absolute values of the products that make up dM_j/dp)."""
    K = dens.K
    rows = np.arange(K, dtype=np.int64) if rows is None else np.asarray(rows, np.int64)
    S, nd = rows.size, len(n)
    cmu = np.empty((S, nd, J)); csg = np.empty((S, nd, J))
    n64 = np.asarray(n, np.int64)
    y = _f64(y)
    lo64, hi64 = _f64(lo), _f64(hi)
    dargs, keep = _dens_args(dens)
    rc = lib().oracle_ipsa_scale(nd, _p(n64, C.c_int64), _p(lo64, C.c_double), _p(hi64, C.c_double),
                                 _p(y, C.c_double), int(J), S, _p(rows, C.c_int64), *dargs,
                                 _p(cmu, C.c_double), _p(csg, C.c_double), int(threads))
    if rc:
        raise OracleError("a selected distribution has an empty support on the grid")
    return cmu, csg


def solve(problem, rows=None, threads=0):
    """Full oracle pipeline for a ``Problem``: y, bins, moments, histograms."""
    y = eval_model(problem.model_id, problem.theta, problem.n, problem.lo, problem.hi)
    b, ymin, ymax = bins(y, problem.n_bins)
    out = propagate(problem.n, problem.lo, problem.hi, y, b, problem.n_bins, problem.n_moments,
                    problem.dens, rows=rows, threads=threads)
    out.update(y=y, bins=b, ymin=ymin, ymax=ymax)
    return out


# ---------------------------------------------------------------- Sec. 5.2 IPSA
def model_at(model_id, theta, x):
    """The model at arbitrary points x [K][ndim] (e.g. the estimated values
    y(l) = M(l, 0) at the densities' centres)."""
    x = _f64(np.atleast_2d(x))
    K, nd = x.shape
    th = np.zeros(8)
    th[:len(theta)] = theta
    y = np.empty(K)
    if lib().oracle_model_at(int(model_id), _p(th, C.c_double), nd, K, _p(x, C.c_double), _p(y, C.c_double)):
        raise OracleError("model not defined for this dimension")
    return y


def deviation_moments(n, lo, hi, y, J, dens, yref, rows=None):
    """sum_i W[k,i] (y_i - yref[k])^j, j = 1..J (Eq. IPSAvar: Delta^2 = half of j = 2)."""
    K = dens.K
    rows = np.arange(K, dtype=np.int64) if rows is None else np.asarray(rows, np.int64)
    out = np.empty((rows.size, J))
    n64 = np.asarray(n, np.int64)
    y, yref = _f64(y), _f64(yref)
    lo64, hi64 = _f64(lo), _f64(hi)
    dargs, keep = _dens_args(dens)
    rc = lib().oracle_deviation_moments(len(n), _p(n64, C.c_int64), _p(lo64, C.c_double), _p(hi64, C.c_double),
                                        _p(y, C.c_double), int(J), rows.size, _p(rows, C.c_int64),
                                        _p(yref, C.c_double), *dargs, _p(out, C.c_double))
    if rc:
        raise OracleError("a selected distribution has an empty support on the grid")
    return out


def ipsa_matrix(H, ymin, ymax, yref, nd, dlo, dhi):
    """IPSA probability matrix (Eq. IPSA): columns translated by -yref onto nd deviation bins."""
    H = _f64(H)
    K, B = H.shape
    yref = _f64(yref)
    out = np.empty((K, nd))
    lib().oracle_ipsa_matrix(K, B, float(ymin), float(ymax), _p(H, C.c_double), _p(yref, C.c_double), int(nd),
                             float(dlo), float(dhi), _p(out, C.c_double))
    return out


def sa_fields(H, level, rho=None):
    """Argmax bin, confidence-interval bins and the rho-marginalised global vector (Sec. 5.2)."""
    H = _f64(H)
    K, nb = H.shape
    am = np.empty(K, np.int32)
    ci = np.empty((K, 2), np.int32)
    g = np.empty(nb)
    r = None if rho is None else _f64(rho)
    lib().oracle_sa_fields(K, nb, _p(H, C.c_double), float(level), None if r is None else _p(r, C.c_double),
                           _p(am, C.c_int32), _p(ci, C.c_int32), _p(g, C.c_double))
    return am, ci, g


def posterior_means(n, lo, hi, bin_ids, B, dens, rows=None):
    """Bayes-inverted model matrix applied to the coordinates (Sec. 3):
    E[x_d | y in bin b, l_k], shape [S][B][ndim] (0 for empty bins)."""
    K = dens.K
    rows = np.arange(K, dtype=np.int64) if rows is None else np.asarray(rows, np.int64)
    nd = len(n)
    out = np.empty((rows.size, B, nd))
    n64 = np.asarray(n, np.int64)
    b32 = np.ascontiguousarray(bin_ids, np.int32)
    lo64, hi64 = _f64(lo), _f64(hi)
    dargs, keep = _dens_args(dens)
    rc = lib().oracle_posterior_means(nd, _p(n64, C.c_int64), _p(lo64, C.c_double), _p(hi64, C.c_double),
                                      _p(b32, C.c_int32), int(B), rows.size, _p(rows, C.c_int64), *dargs,
                                      _p(out, C.c_double))
    if rc:
        raise OracleError("a selected distribution has an empty support on the grid")
    return out
