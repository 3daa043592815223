"""Thin Python binding of libvup (see ``include/vup.h``).

The functions below carry the C ABI names and only marshal arguments: every
step of the propagation runs in the library's CUDA kernels.  PyTorch supplies
device memory and streams.  Importing this module loads the in-tree
``_lib/libvup.so``; if it is missing the import fails loudly -- there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# VUP_DEBUG=1 selects the debug build (device bounds checks that record
# VUP_ERR_BOUNDS instead of trapping; built by build(debug=True))
LIB_PATH = os.path.join(_PKG, "_lib", "libvup_debug.so" if os.environ.get("VUP_DEBUG") == "1" else "libvup.so")

VUP_OK, VUP_ERR_INVALID_ARG, VUP_ERR_CUDA, VUP_ERR_OOM, VUP_ERR_STATE = 0, 1, 2, 3, 4
VUP_ERR_EMPTY_SUPPORT, VUP_ERR_TIMEOUT, VUP_ERR_UNSUPPORTED, VUP_ERR_BOUNDS = 5, 6, 7, 8
VUP_GAUSS, VUP_UNIFORM, VUP_TRUNCNORM = 0, 1, 2
VUP_FP64, VUP_FP32, VUP_BF16X3, VUP_TF32, VUP_TF32X3 = 0, 1, 2, 3, 4
PRECISIONS = {"fp64": VUP_FP64, "fp32": VUP_FP32, "bf16x3": VUP_BF16X3, "tf32": VUP_TF32, "tf32x3": VUP_TF32X3}

# exported symbols declared in include/vup.h
ABI_SYMBOLS = [
    "vup_grid_create", "vup_grid_destroy", "vup_eval_model", "vup_set_outputs", "vup_propagate",
    "vup_propagate_weights", "vup_propagate_weights_noalloc", "vup_ipsa_sensitivity", "vup_propagate_ipsa", "vup_propagate_batched", "vup_batched_report", "vup_sync", "vup_selftest_wait", "vup_model_at",
    "vup_deviation_moments", "vup_ipsa_matrix", "vup_sa_fields", "vup_posterior_means",
    "vup_grid_info", "vup_set_hist_stream", "vup_set_weights_form", "vup_grid_copy", "vup_status_string", "vup_version", "vup_profile",
    "vup_profile_read", "vup_profile_timeline", "vup_last_error_detail", "vup_debug_fail_alloc",
    "vup_measure_peak",
]


class vup_densities(C.Structure):
    _fields_ = [("K", C.c_int64), ("ndim", C.c_int32), ("kind", C.c_void_p), ("mu", C.c_void_p),
                ("sigma", C.c_void_p), ("lo", C.c_void_p), ("hi", C.c_void_p)]


class vup_grid_info_t(C.Structure):
    _fields_ = [("ndim", C.c_int32), ("n", C.c_int64 * 3), ("N", C.c_int64), ("n_bins", C.c_int32),
                ("n_moments", C.c_int32), ("ymin", C.c_double), ("ymax", C.c_double),
                ("yscale", C.c_double), ("have_model", C.c_int32), ("hist_layout", C.c_int32),
                ("hist_stream", C.c_int32), ("hist_runs", C.c_int64), ("hist_intervals", C.c_int64),
                ("hist_records", C.c_int64), ("yshift", C.c_double)]


class VUPError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {vup_status_string(status)}")


_lib = None


def lib():
    """Load libvup.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libvup.so not built ({LIB_PATH}); run paper_1908_11246_gb300.build.build()")
        l = C.CDLL(LIB_PATH)
        vp, i64, i32, dp = C.c_void_p, C.c_int64, C.c_int32, C.POINTER(C.c_double)
        l.vup_grid_create.argtypes = [C.c_int, C.POINTER(C.c_int64), dp, dp, C.POINTER(vp)]
        l.vup_grid_destroy.argtypes = [vp]
        l.vup_eval_model.argtypes = [vp, C.c_int, dp, C.c_int, C.c_int, C.c_int, vp]
        l.vup_set_outputs.argtypes = [vp, vp, C.c_int, C.c_int, vp]
        l.vup_propagate.argtypes = [vp, C.POINTER(vup_densities), C.c_int, vp, vp, vp, vp]
        l.vup_propagate_weights.argtypes = [vp, i64, vp, vp, vp, vp]
        l.vup_propagate_weights_noalloc.argtypes = [vp, i64, vp, vp, vp, vp]
        l.vup_ipsa_sensitivity.argtypes = [vp, C.POINTER(vup_densities), C.c_int, vp, vp, vp, vp]
        l.vup_propagate_ipsa.argtypes = [vp, C.POINTER(vup_densities), C.c_int, vp, vp, vp, vp, vp, vp, vp]
        l.vup_propagate_batched.argtypes = [C.c_int, C.POINTER(vp), C.POINTER(vup_densities), C.c_int,
                                            C.POINTER(vp), C.POINTER(vp), vp]
        l.vup_batched_report.argtypes = [C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_double)]
        l.vup_sync.argtypes = [vp, vp]
        l.vup_selftest_wait.argtypes = [vp, C.c_uint32, vp]
        l.vup_model_at.argtypes = [vp, i64, vp, vp, vp]
        l.vup_deviation_moments.argtypes = [vp, i64, vp, vp, vp, vp]
        l.vup_ipsa_matrix.argtypes = [vp, i64, vp, vp, C.c_int, C.c_double, C.c_double, vp, vp]
        l.vup_sa_fields.argtypes = [i64, C.c_int, vp, C.c_double, vp, vp, vp, vp, vp]
        l.vup_posterior_means.argtypes = [vp, C.POINTER(vup_densities), vp, vp, vp]
        l.vup_grid_info.argtypes = [vp, C.POINTER(vup_grid_info_t)]
        l.vup_set_hist_stream.argtypes = [vp, C.c_int32, vp]
        l.vup_set_weights_form.argtypes = [vp, C.c_int32]
        l.vup_grid_copy.argtypes = [vp, C.c_int, vp, C.c_size_t, vp]
        l.vup_profile.argtypes = [C.c_int]
        l.vup_profile_read.argtypes = [C.c_char_p, C.c_size_t]
        l.vup_profile_timeline.argtypes = [C.c_char_p, C.c_size_t]
        l.vup_debug_fail_alloc.argtypes = [i64]
        l.vup_measure_peak.argtypes = [C.c_int, vp, C.POINTER(C.c_double)]
        for f in ABI_SYMBOLS:
            if f not in ("vup_status_string", "vup_version", "vup_last_error_detail"):
                getattr(l, f).restype = C.c_int
        l.vup_status_string.argtypes = [C.c_int]
        l.vup_status_string.restype = C.c_char_p
        l.vup_version.restype = C.c_char_p
        l.vup_last_error_detail.restype = C.c_char_p
        _lib = l
    return _lib


def vup_last_error_detail() -> str:
    return lib().vup_last_error_detail().decode()


def vup_measure_peak(kind: int, stream=None) -> float:
    """Measured ceiling: kind 0 FP32 FMA FLOP/s, kind 1 shared-memory row
    gathers in bytes/s (see include/vup.h)."""
    v = C.c_double()
    _check(lib().vup_measure_peak(int(kind), _stream(stream), C.byref(v)), "vup_measure_peak")
    return v.value


def vup_debug_fail_alloc(after: int):
    """Make every device allocation of the library fail after `after` more
    succeed (after < 0 disarms): a test hook for the out-of-memory paths."""
    _check(lib().vup_debug_fail_alloc(int(after)), "vup_debug_fail_alloc")


def vup_status_string(status: int) -> str:
    return lib().vup_status_string(int(status)).decode()


def vup_version() -> str:
    return lib().vup_version().decode()


def _check(st: int, where: str):
    if st != VUP_OK:
        detail = lib().vup_last_error_detail().decode() if st in (VUP_ERR_CUDA, VUP_ERR_OOM) else ""
        err = VUPError(st, where + (f" [{detail}]" if detail else ""))
        raise err


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


# ------------------------------------------------------------ ABI functions
def vup_grid_create(n, lo, hi):
    nd = len(n)
    n64 = (C.c_int64 * nd)(*[int(v) for v in n])
    lo_ = (C.c_double * nd)(*[float(v) for v in lo])
    hi_ = (C.c_double * nd)(*[float(v) for v in hi])
    h = C.c_void_p()
    _check(lib().vup_grid_create(nd, n64, lo_, hi_, C.byref(h)), "vup_grid_create")
    return h


def vup_grid_destroy(h):
    _check(lib().vup_grid_destroy(h), "vup_grid_destroy")


def vup_eval_model(h, model_id, theta, n_bins, n_moments, stream=None):
    th = (C.c_double * max(1, len(theta)))(*[float(v) for v in theta])
    _check(lib().vup_eval_model(h, int(model_id), th, len(theta), int(n_bins), int(n_moments),
                                _stream(stream)), "vup_eval_model")


def vup_set_outputs(h, y, n_bins, n_moments, stream=None):
    _check(lib().vup_set_outputs(h, _ptr(y), int(n_bins), int(n_moments), _stream(stream)),
           "vup_set_outputs")


def make_densities(dev):
    """Pack a dict of device tensors {kind, mu, sigma, lo, hi} into the ABI struct."""
    K, nd = dev["mu"].shape
    d = vup_densities(K, nd, dev["kind"].data_ptr(), dev["mu"].data_ptr(), dev["sigma"].data_ptr(),
                      dev["lo"].data_ptr() if dev.get("lo") is not None else None,
                      dev["hi"].data_ptr() if dev.get("hi") is not None else None)
    return d


def vup_propagate(h, dens, precision, moments_raw=None, moments_central=None, hist=None, stream=None):
    _check(lib().vup_propagate(h, C.byref(dens), int(precision), _ptr(moments_raw), _ptr(moments_central),
                               _ptr(hist), _stream(stream)), "vup_propagate")


def vup_propagate_weights(h, W, moments_raw=None, hist=None, stream=None):
    _check(lib().vup_propagate_weights(h, int(W.shape[0]), _ptr(W), _ptr(moments_raw), _ptr(hist),
                                       _stream(stream)), "vup_propagate_weights")


def vup_propagate_weights_noalloc(h, W, moments_raw=None, hist=None, stream=None):
    """Same as vup_propagate_weights, with the library's fixed device scratch array."""
    _check(lib().vup_propagate_weights_noalloc(h, int(W.shape[0]), _ptr(W), _ptr(moments_raw), _ptr(hist),
                                               _stream(stream)), "vup_propagate_weights_noalloc")


def vup_ipsa_sensitivity(h, dens, precision, dmu, dsigma, grad_moments=None, stream=None):
    _check(lib().vup_ipsa_sensitivity(h, C.byref(dens), int(precision), _ptr(grad_moments), _ptr(dmu),
                                      _ptr(dsigma), _stream(stream)), "vup_ipsa_sensitivity")


def vup_propagate_ipsa(h, dens, precision, moments_raw, moments_central, hist, dmu, dsigma, grad_moments=None,
                       stream=None):
    """vup_propagate and vup_ipsa_sensitivity of the same densities in one call."""
    _check(lib().vup_propagate_ipsa(h, C.byref(dens), int(precision), _ptr(moments_raw), _ptr(moments_central),
                                    _ptr(hist), _ptr(grad_moments), _ptr(dmu), _ptr(dsigma), _stream(stream)),
           "vup_propagate_ipsa")


class BatchedArgs:
    """The host arrays of one vup_propagate_batched call, marshalled once."""

    def __init__(self, handles, dens_list, raws, hists):
        n = self.n = len(handles)
        self.hs = (C.c_void_p * n)(*[h.value for h in handles])
        self.ds = (vup_densities * n)(*dens_list)
        self.rs = (C.c_void_p * n)(*[None if r is None else r.data_ptr() for r in raws])
        self.hh = (C.c_void_p * n)(*[None if x is None else x.data_ptr() for x in hists])

    def __call__(self, precision, stream=None):
        _check(lib().vup_propagate_batched(self.n, self.hs, self.ds, int(precision), self.rs, self.hh,
                                           _stream(stream)), "vup_propagate_batched")


def vup_propagate_batched(handles, dens_list, precision, raws, hists, stream=None):
    BatchedArgs(handles, dens_list, raws, hists)(precision, stream)


def vup_batched_report():
    cap, src, ms = C.c_int(), C.c_int(), C.c_double()
    _check(lib().vup_batched_report(C.byref(cap), C.byref(src), C.byref(ms)), "vup_batched_report")
    return {"bn_cap": cap.value, "source": src.value, "tune_ms": ms.value}


def batched_outputs(grids, dev_dens_list, moments=True, hist=True):
    """Per-instance output tensors (raw moments [K][J], histograms [K][B])."""
    import torch
    raws, hists = [], []
    for g, dd in zip(grids, dev_dens_list):
        K = dd["mu"].shape[0]
        dev = dd["mu"].device
        raws.append(torch.empty((K, g.n_moments or 1), dtype=torch.float64, device=dev) if moments else None)
        hists.append(torch.empty((K, g.n_bins or 1), dtype=torch.float32, device=dev) if hist else None)
    return raws, hists


def propagate_batched(grids, dev_dens_list, precision="bf16x3", moments=True, hist=True, out=None,
                      stream=None):
    """Propagate many (grid, densities) instances in one batched call; returns
    per-instance lists of raw moments and histograms (``out`` reuses a pair of
    lists from ``batched_outputs``, which lets later calls replay the batch's
    graph)."""
    raws, hists = out if out is not None else batched_outputs(grids, dev_dens_list, moments, hist)
    ds = [make_densities(dd) for dd in dev_dens_list]
    vup_propagate_batched([g.h for g in grids], ds, PRECISIONS[precision], raws, hists, stream)
    return raws, hists


def vup_selftest_wait(h, polls, stream=None):
    _check(lib().vup_selftest_wait(h, int(polls), _stream(stream)), "vup_selftest_wait")


def vup_model_at(h, x, y, stream=None):
    _check(lib().vup_model_at(h, int(x.shape[0]), _ptr(x), _ptr(y), _stream(stream)), "vup_model_at")


def vup_deviation_moments(h, moments_raw, y_ref, out, stream=None):
    _check(lib().vup_deviation_moments(h, int(moments_raw.shape[0]), _ptr(moments_raw), _ptr(y_ref), _ptr(out),
                                       _stream(stream)), "vup_deviation_moments")


def vup_ipsa_matrix(h, hist, y_ref, n_dbins, dlo, dhi, out, stream=None):
    _check(lib().vup_ipsa_matrix(h, int(hist.shape[0]), _ptr(hist), _ptr(y_ref), int(n_dbins), float(dlo),
                                 float(dhi), _ptr(out), _stream(stream)), "vup_ipsa_matrix")


def vup_sa_fields(hist, level, rho=None, argmax=None, ci=None, global_=None, stream=None):
    _check(lib().vup_sa_fields(int(hist.shape[0]), int(hist.shape[1]), _ptr(hist), float(level), _ptr(rho),
                               _ptr(argmax), _ptr(ci), _ptr(global_), _stream(stream)), "vup_sa_fields")


def vup_posterior_means(h, dens, hist, post, stream=None):
    _check(lib().vup_posterior_means(h, C.byref(dens), _ptr(hist), _ptr(post), _stream(stream)),
           "vup_posterior_means")


def vup_sync(h, stream=None):
    """Wait for queued work; raise on a condition recorded on the device."""
    _check(lib().vup_sync(h, _stream(stream)), "vup_sync")


def vup_sync_status(h, stream=None) -> int:
    return lib().vup_sync(h, _stream(stream))


def vup_grid_info(h):
    info = vup_grid_info_t()
    _check(lib().vup_grid_info(h, C.byref(info)), "vup_grid_info")
    return info


def vup_set_hist_stream(h, kind: int, stream=None):
    """Histogram stream choice: -1 auto, 0 sorted points, 1 sorted intervals, 2 records."""
    _check(lib().vup_set_hist_stream(h, int(kind), _stream(stream)), "vup_set_hist_stream")


def vup_set_weights_form(h, form: int):
    """Supplied-W form: -1 auto, 0 sorted block walk, 1 row per lane, 2 general."""
    _check(lib().vup_set_weights_form(h, int(form)), "vup_set_weights_form")


def vup_grid_copy(h, which, out, stream=None):
    _check(lib().vup_grid_copy(h, int(which), _ptr(out), out.numel() * out.element_size(), _stream(stream)),
           "vup_grid_copy")


def vup_profile(enable: bool):
    _check(lib().vup_profile(1 if enable else 0), "vup_profile")


def vup_profile_read() -> dict:
    """{kernel: (launches, total_ms)} recorded since vup_profile(True)."""
    import json
    buf = C.create_string_buffer(1 << 16)
    _check(lib().vup_profile_read(buf, len(buf)), "vup_profile_read")
    return {k: (int(v[0]), float(v[1])) for k, v in json.loads(buf.value.decode()).items()}


def vup_profile_timeline() -> list:
    """[(kernel group, stream number, launches, begin_ms, end_ms)] in launch
    order, relative to the first record, since vup_profile(True)."""
    import json
    buf = C.create_string_buffer(1 << 22)
    _check(lib().vup_profile_timeline(buf, len(buf)), "vup_profile_timeline")
    return [(str(n), int(s), int(l), float(a), float(b)) for n, s, l, a, b in json.loads(buf.value.decode())]


# ------------------------------------------------------ torch-facing helpers
def densities_to_device(dens, device="cuda"):
    """Copy a ``inputs.Densities`` (numpy SoA) to device tensors."""
    import torch
    return dict(kind=torch.as_tensor(np.ascontiguousarray(dens.kind), device=device),
                mu=torch.as_tensor(np.ascontiguousarray(dens.mu), device=device),
                sigma=torch.as_tensor(np.ascontiguousarray(dens.sigma), device=device),
                lo=torch.as_tensor(np.ascontiguousarray(dens.lo), device=device),
                hi=torch.as_tensor(np.ascontiguousarray(dens.hi), device=device))


class Grid:
    """Owning wrapper of a vup_grid handle."""

    def __init__(self, n, lo, hi):
        self.n, self.lo, self.hi = tuple(n), tuple(lo), tuple(hi)
        self.h = vup_grid_create(n, lo, hi)
        self.n_bins = self.n_moments = None

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            vup_grid_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def N(self):
        return int(np.prod(self.n))

    def eval_model(self, model_id, theta, n_bins, n_moments=4, stream=None):
        vup_eval_model(self.h, model_id, theta, n_bins, n_moments, stream)
        self.n_bins, self.n_moments = n_bins, n_moments

    def set_outputs(self, y, n_bins, n_moments=4, stream=None):
        vup_set_outputs(self.h, y, n_bins, n_moments, stream)
        self.n_bins, self.n_moments = n_bins, n_moments

    def propagate(self, dev_dens, precision="fp32", moments=True, central=True, hist=True, stream=None):
        import torch
        K = dev_dens["mu"].shape[0]
        dev = dev_dens["mu"].device
        J, B = self.n_moments or 1, self.n_bins or 1   # before eval_model the library reports VUP_ERR_STATE
        raw = torch.empty((K, J), dtype=torch.float64, device=dev) if moments else None
        cen = torch.empty((K, J), dtype=torch.float64, device=dev) if central else None
        hs = torch.empty((K, B), dtype=torch.float32, device=dev) if hist else None
        d = make_densities(dev_dens)
        vup_propagate(self.h, d, PRECISIONS[precision], raw, cen, hs, stream)
        return raw, cen, hs

    def ipsa(self, dev_dens, precision="fp32", grad=None, stream=None):
        import torch
        K, nd = dev_dens["mu"].shape
        dev = dev_dens["mu"].device
        shape = (K, nd) if grad is not None else (K, nd, self.n_moments)
        dmu = torch.empty(shape, dtype=torch.float32, device=dev)
        dsg = torch.empty(shape, dtype=torch.float32, device=dev)
        vup_ipsa_sensitivity(self.h, make_densities(dev_dens), PRECISIONS[precision], dmu, dsg, grad, stream)
        return dmu, dsg

    def sync(self, stream=None):
        vup_sync(self.h, stream)

    def info(self):
        return vup_grid_info(self.h)

    def set_hist_stream(self, kind: int, stream=None):
        """-1: automatic choice; 0: sorted points; 1: sorted intervals; 2: records."""
        vup_set_hist_stream(self.h, kind, stream)

    def set_weights_form(self, form: int):
        """-1: automatic choice; 0: sorted block walk; 1: row per lane; 2: general form."""
        vup_set_weights_form(self.h, form)

    def array(self, which):
        import torch
        info = self.info()
        if which in ("y", 0):
            out = torch.empty(info.N, dtype=torch.float64, device="cuda"); w = 0
        elif which in ("bins", 1):
            out = torch.empty(info.N, dtype=torch.int32, device="cuda"); w = 1
        elif which in ("perm", 2):
            out = torch.empty(info.N, dtype=torch.int32, device="cuda"); w = 2
        else:
            out = torch.empty(info.n_bins + 1, dtype=torch.int32, device="cuda"); w = 3
        vup_grid_copy(self.h, w, out)
        return out
