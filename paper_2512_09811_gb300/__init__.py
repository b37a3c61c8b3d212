"""Python binding of the GB300 polarization-propagator window solver.

Thin ctypes marshalling over the C ABI in ``include/pp.h``: every function
here has the C name, converts arguments, calls the library and turns a
non-zero status into ``PPError``.  All arithmetic happens in the CUDA
library; if it is not built, ``load()`` raises -- there is no CPU fallback.
"""

from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libpp_gb300.so")

PP_OK, PP_EINVAL, PP_ENOMEM, PP_ECUDA, PP_ENOTCONV, PP_ETIMEOUT, PP_EMETRIC, PP_EUNSTABLE = range(8)
PP_FP64, PP_BF16, PP_BF16X3 = 0, 2, 3
STATUS_NAMES = {
    PP_OK: "PP_OK", PP_EINVAL: "PP_EINVAL", PP_ENOMEM: "PP_ENOMEM", PP_ECUDA: "PP_ECUDA",
    PP_ENOTCONV: "PP_ENOTCONV", PP_ETIMEOUT: "PP_ETIMEOUT", PP_EMETRIC: "PP_EMETRIC",
    PP_EUNSTABLE: "PP_EUNSTABLE",
}

# every symbol declared in include/pp.h
EXPORTS = (
    "pp_default_options", "pp_create", "pp_sigma", "pp_metric_noalloc", "pp_diagonal", "pp_solve_window",
    "pp_solve_windows", "pp_solve_window_contour", "pp_polarizability", "pp_spectrum", "pp_windows_begin", "pp_windows_step",
    "pp_windows_end", "pp_last_stats", "pp_profile", "pp_profile_read", "pp_autotune_report",
    "pp_kernel_launches", "pp_destroy", "pp_last_error", "pp_server_create", "pp_server_add_dot",
    "pp_server_submit", "pp_server_wait", "pp_server_stats", "pp_server_last_error", "pp_server_destroy",
)


class pp_options(C.Structure):
    _fields_ = [
        ("prec", C.c_int), ("order", C.c_int), ("block", C.c_int), ("m_max", C.c_int),
        ("max_iter", C.c_int), ("res_tol", C.c_double), ("jacobi_floor", C.c_double),
        ("select", C.c_int), ("refine", C.c_int), ("seed", C.c_uint64), ("cuda_stream", C.c_void_p),
        ("workspace_gb", C.c_double), ("tda", C.c_int), ("graphs", C.c_int),
    ]


class pp_server_stats_t(C.Structure):
    _fields_ = [
        ("submitted", C.c_longlong), ("completed", C.c_longlong), ("failed", C.c_longlong),
        ("ctx_created", C.c_longlong), ("ctx_evicted", C.c_longlong), ("steps", C.c_longlong),
        ("max_concurrent_dots", C.c_int), ("max_windows_per_step", C.c_int), ("resident_dots", C.c_int),
        ("resident_bytes", C.c_longlong),
    ]


class PPError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None
_lock = threading.Lock()
_dp = C.POINTER(C.c_double)


def load(path: str | None = None):
    """Load the built library (``__graft_entry__.build()`` or ``_build.py`` makes it)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"CUDA library not built: {p} is missing (run paper_2512_09811_gb300._build)")
        lib = C.CDLL(p)
        vp = C.c_void_p
        lib.pp_default_options.argtypes = [C.POINTER(pp_options)]
        lib.pp_default_options.restype = None
        lib.pp_create.argtypes = [C.c_int, C.c_int, C.c_int, _dp, vp, C.c_int, _dp,
                                  C.POINTER(pp_options), C.POINTER(vp)]
        lib.pp_create.restype = C.c_int
        lib.pp_sigma.argtypes = [vp, C.c_int, vp, vp, vp, C.c_int, C.c_int]
        lib.pp_sigma.restype = C.c_int
        lib.pp_metric_noalloc.argtypes = [vp, C.c_int, vp, vp]
        lib.pp_metric_noalloc.restype = C.c_int
        lib.pp_diagonal.argtypes = [vp, _dp, _dp]
        lib.pp_diagonal.restype = C.c_int
        lib.pp_solve_window.argtypes = [vp, C.c_double, C.c_double, C.c_int, _dp, _dp, _dp, vp,
                                        C.POINTER(C.c_int)]
        lib.pp_solve_window.restype = C.c_int
        lib.pp_solve_windows.argtypes = [vp, C.c_int, _dp, _dp, C.POINTER(C.c_int), _dp, _dp, _dp,
                                         C.POINTER(C.c_int)]
        lib.pp_solve_windows.restype = C.c_int
        lib.pp_solve_window_contour.argtypes = [vp, C.c_double, C.c_double, C.c_int, C.c_int, _dp, _dp, _dp,
                                                C.POINTER(C.c_int)]
        lib.pp_solve_window_contour.restype = C.c_int
        lib.pp_polarizability.argtypes = [vp, C.c_int, _dp, C.c_double, C.c_int, _dp, _dp, C.POINTER(C.c_int)]
        lib.pp_polarizability.restype = C.c_int
        lib.pp_spectrum.argtypes = [vp, C.c_double, C.c_double, C.c_int, C.c_int, C.c_double, C.c_int, _dp, _dp,
                                    C.c_int, _dp, _dp, _dp, C.POINTER(C.c_int)]
        lib.pp_spectrum.restype = C.c_int
        lib.pp_windows_begin.argtypes = [vp, C.c_int, _dp, _dp, C.POINTER(C.c_int)]
        lib.pp_windows_begin.restype = C.c_int
        lib.pp_windows_step.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_longlong), C.POINTER(C.c_int)]
        lib.pp_windows_step.restype = C.c_int
        lib.pp_windows_end.argtypes = [vp, _dp, _dp, _dp, C.POINTER(C.c_int)]
        lib.pp_windows_end.restype = C.c_int
        lib.pp_last_stats.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_longlong),
                                      C.POINTER(C.c_double), C.POINTER(C.c_double)]
        lib.pp_last_stats.restype = C.c_int
        lib.pp_profile.argtypes = [vp, C.c_int]
        lib.pp_profile.restype = C.c_int
        lib.pp_profile_read.argtypes = [vp, C.c_int, C.POINTER(C.c_longlong), C.POINTER(C.c_double),
                                        C.POINTER(C.c_double)]
        lib.pp_profile_read.restype = C.c_int
        lib.pp_autotune_report.argtypes = [C.c_char_p, C.c_longlong]
        lib.pp_autotune_report.restype = C.c_longlong
        lib.pp_kernel_launches.argtypes = []
        lib.pp_kernel_launches.restype = C.c_longlong
        lib.pp_destroy.argtypes = [vp]
        lib.pp_destroy.restype = None
        lib.pp_last_error.argtypes = [vp]
        lib.pp_last_error.restype = C.c_char_p
        lib.pp_server_create.argtypes = [C.c_size_t, C.POINTER(pp_options), C.c_int, C.c_int, C.POINTER(vp)]
        lib.pp_server_create.restype = C.c_int
        lib.pp_server_add_dot.argtypes = [vp, C.c_int, C.c_int, C.c_int, _dp, vp, C.c_int, _dp,
                                          C.POINTER(C.c_int)]
        lib.pp_server_add_dot.restype = C.c_int
        lib.pp_server_submit.argtypes = [vp, C.c_int, C.c_double, C.c_double, C.c_int, C.POINTER(C.c_ulonglong)]
        lib.pp_server_submit.restype = C.c_int
        lib.pp_server_wait.argtypes = [vp, C.c_ulonglong, C.c_int, _dp, _dp, _dp, C.POINTER(C.c_int), _dp]
        lib.pp_server_wait.restype = C.c_int
        lib.pp_server_stats.argtypes = [vp, C.POINTER(pp_server_stats_t)]
        lib.pp_server_stats.restype = C.c_int
        lib.pp_server_last_error.argtypes = [vp]
        lib.pp_server_last_error.restype = C.c_char_p
        lib.pp_server_destroy.argtypes = [vp]
        lib.pp_server_destroy.restype = None
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def pp_default_options(**kw) -> pp_options:
    lib = load()
    opt = pp_options()
    lib.pp_default_options(C.byref(opt))
    for k, v in kw.items():
        if not hasattr(opt, k):
            raise KeyError(k)
        setattr(opt, k, v)
    return opt


def _check(st: int, ctx=None):
    if st not in (PP_OK,):
        msg = load().pp_last_error(ctx).decode(errors="replace")
        raise PPError(st, msg)


def pp_create(nocc: int, nvir: int, naux: int, eps, B, mu=None, opt: pp_options | None = None):
    """Returns an opaque context handle (int).  B may be float64 or float32 [naux, n, n]."""
    lib = load()
    eps = _f64(eps)
    B = np.ascontiguousarray(B)
    if B.dtype == np.float64:
        bdt = 0
    elif B.dtype == np.float32:
        bdt = 1
    else:
        B = _f64(B)
        bdt = 0
    mu_a = _f64(mu) if mu is not None else None
    if opt is None:
        opt = pp_default_options()
    out = C.c_void_p()
    st = lib.pp_create(nocc, nvir, naux, _ptr(eps), B.ctypes.data_as(C.c_void_p), bdt,
                       _ptr(mu_a) if mu_a is not None else None, C.byref(opt), C.byref(out))
    _check(st, None)
    return out.value


def pp_sigma(ctx, Z, prec: int = PP_FP64, metric: bool = False):
    """sigma = M z (and Sigma z) for Z[nvec, 2, nocc, nvir].

    Z may be a numpy array (host path) or a CUDA torch tensor of float64
    (device path: the library reads and writes device memory directly).
    """
    lib = load()
    if hasattr(Z, "is_cuda") and Z.is_cuda:
        import torch

        Zc = Z.contiguous()
        if Zc.dtype != torch.float64:
            raise TypeError("device Z must be float64")
        sig = torch.empty_like(Zc)
        met = torch.empty_like(Zc) if metric else None
        st = lib.pp_sigma(ctx, Zc.shape[0], Zc.data_ptr(), sig.data_ptr(),
                          met.data_ptr() if metric else None, prec, 1)
        _check(st, ctx)
        return (sig, met) if metric else sig
    Zh = _f64(Z)
    sig = np.empty_like(Zh)
    met = np.empty_like(Zh) if metric else None
    st = lib.pp_sigma(ctx, Zh.shape[0], Zh.ctypes.data, sig.ctypes.data,
                      met.ctypes.data if metric else None, prec, 0)
    _check(st, ctx)
    return (sig, met) if metric else sig


PP_METRIC_NOALLOC_MAX_ELEMS = 1 << 19
PP_METRIC_NOALLOC_MAX_NVEC = 32767


def pp_metric_noalloc(ctx, Z, out, nocc: int, nvir: int):
    """out = Sigma z without any device allocation in the library.

    Z and out are CUDA float64 tensors [nvec, 2, nocc, nvir] on the current device (the
    context's device) that the caller owns (nothing is allocated here either);
    nvec * nocc * nvir <= PP_METRIC_NOALLOC_MAX_ELEMS and nvec <= PP_METRIC_NOALLOC_MAX_NVEC.
    The C side cannot see shapes or devices, so they are checked here before the call: a
    mis-shaped tensor would make the kernels read and write past its end.  Calls that
    overlap in time on one device share the library's fixed scratch array and must be
    serialised by the caller.
    """
    lib = load()
    import torch

    dev = torch.cuda.current_device()
    for t in (Z, out):
        if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
            raise TypeError("pp_metric_noalloc needs contiguous CUDA float64 tensors")
        if t.device.index != dev:
            raise ValueError(f"pp_metric_noalloc: tensor on cuda:{t.device.index}, current device is cuda:{dev}")
        if t.dim() != 4 or tuple(t.shape[1:]) != (2, int(nocc), int(nvir)):
            raise ValueError(f"pp_metric_noalloc: expected [nvec, 2, {nocc}, {nvir}], got {tuple(t.shape)}")
    if Z.shape != out.shape:
        raise ValueError("Z and out must have the same shape")
    st = lib.pp_metric_noalloc(ctx, int(Z.shape[0]), Z.data_ptr(), out.data_ptr())
    _check(st, ctx)
    return out


def pp_diagonal(ctx, nocc: int, nvir: int):
    lib = load()
    dA = np.empty((nocc, nvir))
    dS = np.empty((nocc, nvir))
    _check(lib.pp_diagonal(ctx, _ptr(dA), _ptr(dS)), ctx)
    return dA, dS


def pp_solve_window(ctx, omega0: float, delta: float, k: int, nocc: int = 0, nvir: int = 0,
                    want_vectors: bool = False, allow_notconv: bool = False):
    lib = load()
    om = np.zeros(k)
    osc = np.zeros(k)
    res = np.zeros(k)
    nf = C.c_int(0)
    vecs = np.zeros((k, 2, nocc, nvir)) if want_vectors else None
    st = lib.pp_solve_window(ctx, float(omega0), float(delta), int(k), _ptr(om), _ptr(osc), _ptr(res),
                             vecs.ctypes.data if want_vectors else None, C.byref(nf))
    if not (allow_notconv and st == PP_ENOTCONV):
        _check(st, ctx)
    n = nf.value
    out = dict(omega=om[:n], osc=osc[:n], resid=res[:n], status=st)
    if want_vectors:
        out["vectors"] = vecs[:n]
    return out


def pp_solve_windows(ctx, omega0, delta, k, allow_notconv: bool = False):
    lib = load()
    omega0 = _f64(omega0)
    delta = _f64(delta)
    kk = np.ascontiguousarray(k, dtype=np.int32)
    nwin = omega0.size
    tot = int(kk.sum())
    om = np.zeros(tot)
    osc = np.zeros(tot)
    res = np.zeros(tot)
    nf = np.zeros(nwin, dtype=np.int32)
    st = lib.pp_solve_windows(ctx, nwin, _ptr(omega0), _ptr(delta), kk.ctypes.data_as(C.POINTER(C.c_int)),
                              _ptr(om), _ptr(osc), _ptr(res), nf.ctypes.data_as(C.POINTER(C.c_int)))
    if not (allow_notconv and st == PP_ENOTCONV):
        _check(st, ctx)
    out = []
    off = 0
    for w in range(nwin):
        n = int(nf[w])
        out.append(dict(omega=om[off:off + n], osc=osc[off:off + n], resid=res[off:off + n]))
        off += int(kk[w])
    return out, st


def pp_solve_window_contour(ctx, omega0: float, delta: float, k: int, nquad: int = 8, allow_notconv: bool = False):
    """All roots in [omega0, omega0 + delta] by the contour (Riesz projector) filter."""
    lib = load()
    om = np.zeros(k)
    osc = np.zeros(k)
    res = np.zeros(k)
    nf = C.c_int(0)
    st = lib.pp_solve_window_contour(ctx, float(omega0), float(delta), int(nquad), int(k), _ptr(om), _ptr(osc),
                                     _ptr(res), C.byref(nf))
    if not (allow_notconv and st == PP_ENOTCONV):
        _check(st, ctx)
    n = nf.value
    return dict(omega=om[:n], osc=osc[:n], resid=res[:n], status=st)


def pp_polarizability(ctx, omega, tol: float = 1e-8, max_iter: int = 2000, allow_notconv: bool = False):
    """Dipole polarizability alpha[f][c][c'] at real frequencies: dict(alpha, resid, iterations, status)."""
    lib = load()
    w = _f64(omega).ravel()
    alpha = np.zeros((w.size, 3, 3))
    res = np.zeros(w.size)
    its = np.zeros(w.size, dtype=np.int32)
    st = lib.pp_polarizability(ctx, int(w.size), _ptr(w), float(tol), int(max_iter), _ptr(alpha), _ptr(res),
                               its.ctypes.data_as(C.POINTER(C.c_int)))
    if not (allow_notconv and st == PP_ENOTCONV):
        _check(st, ctx)
    return dict(alpha=alpha, resid=res, iterations=its, status=st)


def pp_spectrum(ctx, w_lo: float, w_hi: float, nwin: int, kmax: int, eta: float, grid, cap: int = 4096,
                allow_notconv: bool = False):
    """Roots and Lorentzian-broadened absorption spectrum of [w_lo, w_hi]: dict(spec, omega, osc,
    resid, status)."""
    lib = load()
    g = _f64(grid).ravel()
    spec = np.zeros_like(g)
    om = np.zeros(cap)
    osc = np.zeros(cap)
    res = np.zeros(cap)
    n = C.c_int(0)
    st = lib.pp_spectrum(ctx, float(w_lo), float(w_hi), int(nwin), int(kmax), float(eta), int(g.size),
                         _ptr(g) if g.size else None, _ptr(spec) if g.size else None, int(cap), _ptr(om), _ptr(osc),
                         _ptr(res), C.byref(n))
    if not (allow_notconv and st == PP_ENOTCONV):
        _check(st, ctx)
    k = n.value
    return dict(spec=spec, omega=om[:k], osc=osc[:k], resid=res[:k], status=st)


class WindowRun:
    """pp_windows_begin / pp_windows_step / pp_windows_end: a batched window solve driven one
    block iteration at a time."""

    def __init__(self, ctx, omega0, delta, k):
        self.ctx = ctx
        self.omega0 = _f64(omega0)
        self.delta = _f64(delta)
        self.k = np.ascontiguousarray(k, dtype=np.int32)
        self.nwin = self.omega0.size
        _check(load().pp_windows_begin(ctx, self.nwin, _ptr(self.omega0), _ptr(self.delta),
                                       self.k.ctypes.data_as(C.POINTER(C.c_int))), ctx)

    def step(self):
        """One iteration of every unfinished window: (unfinished, sigma supervectors, sigma calls)."""
        un = C.c_int()
        nv = C.c_longlong()
        nc = C.c_int()
        _check(load().pp_windows_step(self.ctx, C.byref(un), C.byref(nv), C.byref(nc)), self.ctx)
        return un.value, nv.value, nc.value

    def end(self, allow_notconv: bool = False):
        tot = int(self.k.sum())
        om = np.zeros(tot)
        osc = np.zeros(tot)
        res = np.zeros(tot)
        nf = np.zeros(self.nwin, dtype=np.int32)
        st = load().pp_windows_end(self.ctx, _ptr(om), _ptr(osc), _ptr(res), nf.ctypes.data_as(C.POINTER(C.c_int)))
        if not (allow_notconv and st == PP_ENOTCONV):
            _check(st, self.ctx)
        out, off = [], 0
        for w in range(self.nwin):
            n = int(nf[w])
            out.append(dict(omega=om[off:off + n], osc=osc[off:off + n], resid=res[off:off + n]))
            off += int(self.k[w])
        return out, st


def pp_last_stats(ctx):
    lib = load()
    it = C.c_int()
    nv = C.c_longlong()
    sms = C.c_double()
    tms = C.c_double()
    _check(lib.pp_last_stats(ctx, C.byref(it), C.byref(nv), C.byref(sms), C.byref(tms)), ctx)
    return dict(iterations=it.value, sigma_vectors=nv.value, sigma_ms=sms.value, solve_ms=tms.value)


def pp_profile(ctx, enable: bool):
    _check(load().pp_profile(ctx, 1 if enable else 0), ctx)


def pp_profile_read(ctx, kernel_id: int):
    lib = load()
    n = C.c_longlong()
    ms = C.c_double()
    fl = C.c_double()
    _check(lib.pp_profile_read(ctx, int(kernel_id), C.byref(n), C.byref(ms), C.byref(fl)), ctx)
    return dict(launches=n.value, ms=ms.value, flops=fl.value)


def pp_autotune_report() -> str:
    """The tensor-core GEMM autotuner's table (text)."""
    lib = load()
    n = int(lib.pp_autotune_report(None, 0))
    buf = C.create_string_buffer(n)
    lib.pp_autotune_report(buf, n)
    return buf.value.decode(errors="replace")


def pp_kernel_launches() -> int:
    return int(load().pp_kernel_launches())


def pp_destroy(ctx):
    if ctx:
        load().pp_destroy(ctx)


def pp_last_error(ctx=None) -> str:
    return load().pp_last_error(ctx).decode(errors="replace")


class Dot:
    """Owning wrapper: one context per synthetic dot."""

    def __init__(self, inp, **opts):
        self.nocc, self.nvir, self.naux = inp.nocc, inp.nvir, inp.naux
        self.opt = pp_default_options(**opts)
        self.ctx = pp_create(inp.nocc, inp.nvir, inp.naux, inp.eps, inp.B, inp.mu, self.opt)

    def sigma(self, Z, prec=PP_FP64, metric=False):
        return pp_sigma(self.ctx, Z, prec, metric)

    def metric_noalloc(self, Z, out):
        return pp_metric_noalloc(self.ctx, Z, out, self.nocc, self.nvir)

    def diagonal(self):
        return pp_diagonal(self.ctx, self.nocc, self.nvir)

    def solve_window(self, omega0, delta, k, **kw):
        return pp_solve_window(self.ctx, omega0, delta, k, self.nocc, self.nvir, **kw)

    def solve_windows(self, omega0, delta, k, **kw):
        return pp_solve_windows(self.ctx, omega0, delta, k, **kw)

    def windows(self, omega0, delta, k):
        return WindowRun(self.ctx, omega0, delta, k)

    def solve_window_contour(self, omega0, delta, k, **kw):
        return pp_solve_window_contour(self.ctx, omega0, delta, k, **kw)

    def polarizability(self, omega, **kw):
        return pp_polarizability(self.ctx, omega, **kw)

    def spectrum(self, w_lo, w_hi, nwin, kmax, eta, grid, **kw):
        return pp_spectrum(self.ctx, w_lo, w_hi, nwin, kmax, eta, grid, **kw)

    def stats(self):
        return pp_last_stats(self.ctx)

    def close(self):
        if self.ctx:
            pp_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# serving
# ---------------------------------------------------------------------------
def pp_server_create(hbm_budget: int, opt: pp_options | None = None, slots_per_dot: int = 4, nworkers: int = 0):
    lib = load()
    if opt is None:
        opt = pp_default_options()
    out = C.c_void_p()
    st = lib.pp_server_create(int(hbm_budget), C.byref(opt), int(slots_per_dot), int(nworkers), C.byref(out))
    if st != PP_OK:
        raise PPError(st, "pp_server_create failed")
    return out.value


def pp_server_add_dot(srv, nocc: int, nvir: int, naux: int, eps, B, mu=None) -> int:
    lib = load()
    eps = _f64(eps)
    B = np.ascontiguousarray(B)
    if B.dtype == np.float32:
        bdt = 1
    else:
        B = _f64(B)
        bdt = 0
    mu_a = _f64(mu) if mu is not None else None
    did = C.c_int()
    st = lib.pp_server_add_dot(srv, nocc, nvir, naux, _ptr(eps), B.ctypes.data_as(C.c_void_p), bdt,
                               _ptr(mu_a) if mu_a is not None else None, C.byref(did))
    if st != PP_OK:
        raise PPError(st, lib.pp_server_last_error(srv).decode(errors="replace") or "pp_server_add_dot failed")
    return did.value


def pp_server_submit(srv, dot_id: int, omega0: float, delta: float, k: int) -> int:
    rid = C.c_ulonglong()
    st = load().pp_server_submit(srv, int(dot_id), float(omega0), float(delta), int(k), C.byref(rid))
    if st != PP_OK:
        raise PPError(st, "pp_server_submit failed")
    return rid.value


def pp_server_wait(srv, req_id: int, k: int, timeout_ms: int = -1, allow_notconv: bool = False):
    """Returns None on PP_ETIMEOUT, else dict(omega, osc, resid, latency_ms, queue_ms, status)."""
    lib = load()
    om = np.zeros(k)
    osc = np.zeros(k)
    res = np.zeros(k)
    lat = np.zeros(2)
    nf = C.c_int(0)
    st = lib.pp_server_wait(srv, C.c_ulonglong(req_id), int(timeout_ms), _ptr(om), _ptr(osc), _ptr(res),
                            C.byref(nf), _ptr(lat))
    if st == PP_ETIMEOUT:
        return None
    if st != PP_OK and not (allow_notconv and st == PP_ENOTCONV):
        raise PPError(st, lib.pp_server_last_error(srv).decode(errors="replace"))
    n = nf.value
    return dict(omega=om[:n], osc=osc[:n], resid=res[:n], latency_ms=float(lat[0]), queue_ms=float(lat[1]),
                status=st)


def pp_server_stats(srv) -> dict:
    stt = pp_server_stats_t()
    _check(load().pp_server_stats(srv, C.byref(stt)))
    return {name: getattr(stt, name) for name, _ in pp_server_stats_t._fields_}


def pp_server_last_error(srv) -> str:
    return load().pp_server_last_error(srv).decode(errors="replace")


def pp_server_destroy(srv):
    if srv:
        load().pp_server_destroy(srv)


class Server:
    """Owning wrapper of a serving loop."""

    def __init__(self, hbm_budget: int, slots_per_dot: int = 4, nworkers: int = 0, **opts):
        self.opt = pp_default_options(**opts)
        self.srv = pp_server_create(hbm_budget, self.opt, slots_per_dot, nworkers)
        self.dims = {}

    def add_dot(self, inp) -> int:
        did = pp_server_add_dot(self.srv, inp.nocc, inp.nvir, inp.naux, inp.eps, inp.B, inp.mu)
        self.dims[did] = (inp.nocc, inp.nvir)
        return did

    def submit(self, dot_id: int, omega0: float, delta: float, k: int) -> int:
        return pp_server_submit(self.srv, dot_id, omega0, delta, k)

    def wait(self, req_id: int, k: int, timeout_ms: int = -1, **kw):
        return pp_server_wait(self.srv, req_id, k, timeout_ms, **kw)

    def stats(self) -> dict:
        return pp_server_stats(self.srv)

    def close(self):
        if self.srv:
            pp_server_destroy(self.srv)
            self.srv = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
