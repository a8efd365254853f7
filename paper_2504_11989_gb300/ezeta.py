"""ctypes binding of the C ABI in include/ezeta.h (argument marshalling only).

Every numerical step runs in libezeta.so; this module converts Python/numpy/torch
arguments to pointers and sizes.  Loading fails loudly when the library has not
been built (call :func:`paper_2504_11989_gb300.build.build`).

Pointers: numpy arrays are passed as host pointers, torch CUDA tensors as device
pointers; the library detects which.  ``stream`` is a ``torch.cuda.Stream``, a raw
``cudaStream_t`` integer, or None (legacy default stream).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from .build import LIB

EZ_OK, EZ_EINVAL, EZ_EDOMAIN, EZ_EUNSUPPORTED, EZ_ENOMEM, EZ_ECUDA, EZ_ETIMEOUT, EZ_EBUSY = range(8)
EZ_FP64, EZ_MIXED = 0, 1
EZ_MAX_NU, EZ_MAX_PROD = 8, 4

_lock = threading.Lock()
_lib = None


class EzError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"ezeta error {code}: {msg}")
        self.code = code


class ez_quadrature(ctypes.Structure):
    _fields_ = [
        ("n_u", ctypes.c_int),
        ("n_v", ctypes.c_int),
        ("u_rule", ctypes.c_int),
        ("eps", ctypes.c_double),
        ("ell", ctypes.c_int),
        ("lam", ctypes.c_double),
        ("r_real", ctypes.c_double),
        ("r_recip", ctypes.c_double),
        ("prec", ctypes.c_int),
        ("dedupe", ctypes.c_int),
        ("part", ctypes.c_int),
        ("n_parts", ctypes.c_int),
    ]


class ez_sum_spec(ctypes.Structure):
    _fields_ = [
        ("n_distinct", ctypes.c_int),
        ("nu", ctypes.c_double * EZ_MAX_NU),
        ("n_prod", ctypes.c_int),
        ("expo", (ctypes.c_int * EZ_MAX_NU) * EZ_MAX_PROD),
    ]


EZ_REQ_ERR_EST = 1


class ez_request(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("A", ctypes.c_double * 9), ("spec", ez_sum_spec),
                ("quad", ez_quadrature), ("tag", ctypes.c_ulonglong), ("flags", ctypes.c_int)]


class ez_result(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_ulonglong), ("tag", ctypes.c_ulonglong), ("status", ctypes.c_int),
                ("value", ctypes.c_double * EZ_MAX_PROD), ("t_submit", ctypes.c_double),
                ("t_start", ctypes.c_double), ("t_done", ctypes.c_double),
                ("err_est", ctypes.c_double * EZ_MAX_PROD)]


class ez_serve_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_longlong), ("completed", ctypes.c_longlong), ("failed", ctypes.c_longlong),
                ("ticks", ctypes.c_longlong), ("max_batch_seen", ctypes.c_longlong),
                ("busy_seconds", ctypes.c_double), ("peak_device_bytes", ctypes.c_longlong),
                ("phi_tables_built", ctypes.c_longlong), ("phi_tables_reused", ctypes.c_longlong)]


EZ_SERVER_DRYRUN = 1


def lib():
    """The loaded libezeta.so; raises if it is missing (no fallback path exists)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB):
                raise RuntimeError(f"libezeta.so not built at {LIB}; run paper_2504_11989_gb300.build.build()")
            L = ctypes.CDLL(LIB)
            vp, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
            L.ez_last_error.restype = ctypes.c_char_p
            L.ez_launch_count.restype = ctypes.c_longlong
            L.ez_launch_count.argtypes = [ctypes.c_int]
            L.ez_lattice_create.argtypes = [ctypes.c_int, dp, ctypes.c_double, ctypes.POINTER(vp)]
            L.ez_lattice_destroy.argtypes = [vp]
            L.ez_quadrature_default.argtypes = [ctypes.POINTER(ez_quadrature)]
            L.ez_epstein_zeta.argtypes = [vp, ctypes.c_double, dp, vp, ctypes.c_size_t, vp, vp, ctypes.c_int, vp]
            L.ez_epstein_zeta_static.argtypes = [vp, ctypes.c_double, dp, vp, ctypes.c_size_t, vp, vp, vp]
            L.ez_lattice_sum_nbody.argtypes = [vp, dp, ctypes.c_int, ctypes.POINTER(ez_quadrature), vp, vp, vp]
            L.ez_atm_energy.argtypes = [vp, ctypes.POINTER(ez_quadrature), dp, dp, vp]
            L.ez_lattice_sum_adaptive.argtypes = [vp, ctypes.POINTER(ez_sum_spec), ctypes.POINTER(ez_quadrature),
                                                  ctypes.c_double, ctypes.c_int, dp, dp,
                                                  ctypes.POINTER(ctypes.c_longlong), vp]
            L.ez_lattice_sums.argtypes = [ctypes.c_int, ctypes.POINTER(vp), ctypes.POINTER(ez_sum_spec),
                                          ctypes.POINTER(ez_quadrature), vp, vp,
                                          ctypes.POINTER(ctypes.c_longlong), vp]
            L.ez_batch_create.argtypes = [ctypes.c_int, ctypes.POINTER(vp), ctypes.POINTER(ez_sum_spec),
                                          ctypes.POINTER(ez_quadrature), vp, ctypes.POINTER(vp)]
            L.ez_batch_run.argtypes = [vp, vp, vp]
            L.ez_batch_n_lines.restype = ctypes.c_longlong
            L.ez_batch_n_lines.argtypes = [vp]
            L.ez_batch_lines.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_longlong), vp]
            L.ez_batch_destroy.argtypes = [vp]
            L.ez_batch_timing.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_float),
                                          ctypes.POINTER(ctypes.c_float)]
            L.ez_batch_far_flops.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong),
                                             ctypes.POINTER(ctypes.c_longlong)]
            L.ez_batch_sizes.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]
            L.ez_diag_fp64_peak.argtypes = [ctypes.POINTER(ctypes.c_double), vp]
            L.ez_diag_fp32_peak.argtypes = [ctypes.POINTER(ctypes.c_double), vp]
            L.ez_server_create.argtypes = [ctypes.c_size_t, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.POINTER(vp)]
            L.ez_server_submit.argtypes = [vp, ctypes.POINTER(ez_request), ctypes.POINTER(ctypes.c_ulonglong)]
            L.ez_server_poll.argtypes = [vp, ctypes.POINTER(ez_result), ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
            L.ez_server_wait.argtypes = [vp, ctypes.c_ulonglong, ctypes.c_int, ctypes.POINTER(ez_result)]
            L.ez_server_stats.argtypes = [vp, ctypes.POINTER(ez_serve_stats)]
            L.ez_server_destroy.argtypes = [vp, ctypes.c_int]
            L.ez_layout.argtypes = [ctypes.c_int, ctypes.POINTER(ez_sum_spec), ctypes.POINTER(ez_quadrature),
                                    ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_int)]
            L.ez_plan_describe.argtypes = [ctypes.c_void_p, ctypes.POINTER(ez_sum_spec), ctypes.POINTER(ez_quadrature),
                                           ctypes.POINTER(ez_plan_info)]
            _lib = L
    return _lib


def _check(rc: int):
    if rc != EZ_OK:
        raise EzError(rc, lib().ez_last_error().decode())


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(a):
    """(pointer, keepalive) for a numpy array or torch tensor (any device)."""
    if a is None:
        return None, None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"] or a.dtype != np.float64:
            raise ValueError("numpy arguments must be C-contiguous float64")
        return ctypes.c_void_p(a.ctypes.data), a
    # torch.Tensor
    if a.dtype.__repr__() != "torch.float64" or not a.is_contiguous():
        raise ValueError("tensor arguments must be contiguous float64")
    return ctypes.c_void_p(a.data_ptr()), a


def ez_launch_count(reset: bool = False) -> int:
    return int(lib().ez_launch_count(1 if reset else 0))


def quadrature(q=None, **kw) -> ez_quadrature:
    """Build an ez_quadrature from a workloads.Quad (or keyword overrides)."""
    Q = ez_quadrature()
    lib().ez_quadrature_default(ctypes.byref(Q))
    if q is not None:
        Q.n_u, Q.n_v, Q.u_rule = q.n_u, q.n_v, q.u_rule
        Q.eps, Q.ell, Q.lam, Q.r_real, Q.r_recip = q.eps, q.ell, q.lam, q.r_real, q.r_recip
    for k, v in kw.items():
        setattr(Q, k, v)
    return Q


def sum_spec(nu, expo) -> ez_sum_spec:
    S = ez_sum_spec()
    S.n_distinct = len(nu)
    for j, v in enumerate(nu):
        S.nu[j] = float(v)
    S.n_prod = len(expo)
    for p, row in enumerate(expo):
        for j, e in enumerate(row):
            S.expo[p][j] = int(e)
    return S


class Lattice:
    """Owning wrapper of an ez_lattice handle (Def. "Lattices")."""

    def __init__(self, A, scale: float = 1.0):
        A = np.ascontiguousarray(A, dtype=np.float64)
        self.d = A.shape[0]
        self.A = A * float(scale)
        h = ctypes.c_void_p()
        _check(lib().ez_lattice_create(self.d, A.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), float(scale),
                                       ctypes.byref(h)))
        self.handle = h

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and _lib is not None:
            _lib.ez_lattice_destroy(h)
            self.handle = None


def _numel(a) -> int:
    return int(a.size) if isinstance(a, np.ndarray) else int(a.numel())


def _check_zeta_buffers(lat: "Lattice", xv, y, re, im, device_only: bool) -> int:
    """Checks the caller's buffers of an Epstein zeta call against each other and returns m.

    The C ABI receives bare pointers and cannot see sizes, so an undersized output or a
    point array of the wrong dimension would make the kernels read or write past the
    caller's buffers; every such case is rejected here with ValueError."""
    d = lat.d
    if xv.size != d:
        raise ValueError(f"x has {xv.size} components; the lattice has dimension {d}")
    if isinstance(y, np.ndarray):
        if y.ndim > 2 or (y.ndim == 2 and y.shape[1] != d) or y.size % d:
            raise ValueError(f"y must have shape (m, {d}); got {y.shape}")
    else:
        if y.dim() > 2 or (y.dim() == 2 and y.shape[1] != d) or y.numel() % d:
            raise ValueError(f"y must have shape (m, {d}); got {tuple(y.shape)}")
    m = _numel(y) // d
    for name, buf in (("re", re), ("im", im)):
        if buf is not None and _numel(buf) < m:
            raise ValueError(f"{name} holds {_numel(buf)} values; {m} are needed")
    bufs = [b for b in (y, re, im) if b is not None]
    on_gpu = [not isinstance(b, np.ndarray) and b.device.type == "cuda" for b in bufs]
    if device_only and not all(on_gpu):
        raise ValueError("y, re and im must be CUDA tensors")
    if any(on_gpu):
        import torch

        cur = torch.cuda.current_device()
        for b, g in zip(bufs, on_gpu):
            if not g and not isinstance(b, np.ndarray):
                raise ValueError(f"tensor on {b.device}: use a CUDA tensor or a numpy array")
            if g and b.device.index != cur:
                raise ValueError(f"tensor on {b.device}, but the current CUDA device is cuda:{cur}")
    elif not all(isinstance(b, np.ndarray) for b in bufs):
        raise ValueError("CPU tensors are not accepted: pass numpy arrays or CUDA tensors")
    return m


def ez_epstein_zeta(lat: Lattice, nu: float, x, y, re=None, im=None, prec: int = EZ_FP64, stream=None):
    """Z_{Lambda,nu}(x, y_i).  y: (m, d) numpy array or CUDA tensor.  Returns (re, im)
    in the same kind of container as y (allocated if not given)."""
    xv = np.ascontiguousarray(np.atleast_1d(np.asarray(x, dtype=np.float64)))
    if isinstance(y, np.ndarray):
        y = np.ascontiguousarray(y, dtype=np.float64)
        m = y.shape[0] if y.ndim > 1 else (y.size // lat.d)
        if re is None:
            re = np.zeros(m)
        if im is None:
            im = np.zeros(m)
    else:
        m = y.shape[0] if y.dim() > 1 else y.numel() // lat.d
        if re is None:
            re = y.new_zeros(m)
        if im is None:
            im = y.new_zeros(m)
    m = _check_zeta_buffers(lat, xv, y, re, im, device_only=False)
    yp, _ = _ptr(y)
    rp, _ = _ptr(re)
    ip, _ = _ptr(im)
    _check(lib().ez_epstein_zeta(lat.handle, float(nu), xv.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), yp,
                                 int(m), rp, ip, int(prec), _stream_ptr(stream)))
    return re, im


def ez_epstein_zeta_static(lat: Lattice, nu: float, x, y, re, im=None, stream=None):
    """Z_{Lambda,nu}(x, y_i) without any allocation: y, re, im are CUDA tensors owned by
    the caller; the library's scratch is a 256 KiB static device array (see ezeta.h)."""
    xv = np.ascontiguousarray(np.atleast_1d(np.asarray(x, dtype=np.float64)))
    m = _check_zeta_buffers(lat, xv, y, re, im, device_only=True)
    yp, _ = _ptr(y)
    rp, _ = _ptr(re)
    ip, _ = _ptr(im)
    _check(lib().ez_epstein_zeta_static(lat.handle, float(nu), xv.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                        yp, int(m), rp, ip, _stream_ptr(stream)))
    return re, im


def ez_lattice_sum_nbody(lat: Lattice, nu, q: ez_quadrature, out=None, stream=None, err_est: bool = False):
    """zeta^(n)(nu_1..nu_n).  Returns the value (float), or `out` when a numpy array or CUDA
    tensor of one double is given; with err_est=True returns (value, error estimate)."""
    nuv = np.ascontiguousarray(np.asarray(nu, dtype=np.float64))
    nup = nuv.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    e = ctypes.c_double()
    ep = ctypes.byref(e) if err_est else None
    if out is None:
        v = ctypes.c_double()
        _check(lib().ez_lattice_sum_nbody(lat.handle, nup, int(nuv.size), ctypes.byref(q), ctypes.byref(v), ep,
                                          _stream_ptr(stream)))
        return (v.value, e.value) if err_est else v.value
    if _numel(out) < 1:
        raise ValueError("out holds no value")
    op, _ = _ptr(out)
    _check(lib().ez_lattice_sum_nbody(lat.handle, nup, int(nuv.size), ctypes.byref(q), op, ep, _stream_ptr(stream)))
    return (out, e.value) if err_est else out


def ez_lattice_sum_adaptive(lat: Lattice, spec: ez_sum_spec, q: ez_quadrature, tol: float, max_rounds: int = 30,
                            stream=None):
    """Adaptive u integration (see ezeta.h): (values per product, error estimates, u nodes used)."""
    n = spec.n_prod
    v = (ctypes.c_double * n)()
    e = (ctypes.c_double * n)()
    used = ctypes.c_longlong()
    _check(lib().ez_lattice_sum_adaptive(lat.handle, ctypes.byref(spec), ctypes.byref(q), float(tol), int(max_rounds),
                                         v, e, ctypes.byref(used), _stream_ptr(stream)))
    return np.array(v[:]), np.array(e[:]), used.value


def ez_atm_energy(lat: Lattice, q: ez_quadrature, stream=None):
    """(E, [zeta(3,3,3), zeta(-1,5,5), zeta(1,3,5)]) -- Prop. in Sec. 2."""
    E = ctypes.c_double()
    parts = (ctypes.c_double * 3)()
    _check(lib().ez_atm_energy(lat.handle, ctypes.byref(q), ctypes.byref(E), parts, _stream_ptr(stream)))
    return E.value, np.array(parts[:])


def ez_lattice_sums(lats, specs, quads, out=None, lines: bool = False, stream=None):
    """Batched sums.  Returns out[(n_req, EZ_MAX_PROD)] and, if lines, (lines array
    [n_lines, EZ_MAX_PROD], offsets[n_req + 1])."""
    n = len(lats)
    harr = (ctypes.c_void_p * n)(*[l.handle for l in lats])
    sarr = (ez_sum_spec * n)(*specs)
    qarr = (ez_quadrature * n)(*quads)
    if out is None:
        out = np.zeros((n, EZ_MAX_PROD))
    op, _ = _ptr(out)
    offs = (ctypes.c_longlong * (n + 1))()
    lp = None
    lbuf = None
    if lines:
        # size from a first pass of the layout
        total = 0
        for l, s, q in zip(lats, specs, quads):
            ns, nu_t, ur = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
            _check(lib().ez_layout(l.d, ctypes.byref(s), ctypes.byref(q), ctypes.byref(ns), ctypes.byref(nu_t),
                                   ctypes.byref(ur)))
            total += ns.value * nu_t.value + (ns.value if ur.value == 2 else 0)
        lbuf = np.zeros((total, EZ_MAX_PROD))
        lp = ctypes.c_void_p(lbuf.ctypes.data)
    _check(lib().ez_lattice_sums(n, harr, sarr, qarr, op, lp, offs, _stream_ptr(stream)))
    if lines:
        return out, lbuf, np.array(offs[:])
    return out


class ez_plan_info(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_double), ("r_real", ctypes.c_double), ("r_recip", ctypes.c_double),
                ("M", ctypes.c_int * 3), ("m_hp", ctypes.c_int * 3), ("n_sectors", ctypes.c_int),
                ("n_u_total", ctypes.c_int), ("u_rule", ctypes.c_int), ("vchunk", ctypes.c_int),
                ("n_chunks", ctypes.c_int), ("line_lo", ctypes.c_longlong), ("line_hi", ctypes.c_longlong),
                ("n_far_items", ctypes.c_longlong), ("far_smem_bytes", ctypes.c_size_t), ("t_mix", ctypes.c_float),
                ("t_mid", ctypes.c_float), ("n_alpha", ctypes.c_int)]


def ez_plan_describe(lat: "Lattice", spec: ez_sum_spec, q: ez_quadrature) -> ez_plan_info:
    """The host-side plan of one sum (diagnostic; no GPU needed)."""
    info = ez_plan_info()
    _check(lib().ez_plan_describe(lat.handle, ctypes.byref(spec), ctypes.byref(q), ctypes.byref(info)))
    return info


def ez_layout(d: int, spec: ez_sum_spec, q: ez_quadrature):
    ns, nu_t, ur = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().ez_layout(int(d), ctypes.byref(spec), ctypes.byref(q), ctypes.byref(ns), ctypes.byref(nu_t),
                           ctypes.byref(ur)))
    return ns.value, nu_t.value, ur.value


class Batch:
    """ez_batch: resident plans and device tables of n sums (one upload); run() launches
    every kernel of the path again and returns the values."""

    def __init__(self, lats, specs, quads, stream=None):
        n = len(lats)
        self.n = n
        self._lats = list(lats)  # keep the lattice handles alive
        harr = (ctypes.c_void_p * n)(*[l.handle for l in lats])
        sarr = (ez_sum_spec * n)(*specs)
        qarr = (ez_quadrature * n)(*quads)
        h = ctypes.c_void_p()
        _check(lib().ez_batch_create(n, harr, sarr, qarr, _stream_ptr(stream), ctypes.byref(h)))
        self.handle = h

    def run(self, out=None, stream=None):
        """out: None (host array returned), numpy array or CUDA tensor of n*EZ_MAX_PROD."""
        if out is None:
            out = np.zeros((self.n, EZ_MAX_PROD))
        op, _ = _ptr(out)
        _check(lib().ez_batch_run(self.handle, op, _stream_ptr(stream)))
        return out

    def timing(self, enable: bool = True):
        """Enable event timing for following runs; returns (far_ms, total_ms) of the last timed run."""
        f, t = ctypes.c_float(), ctypes.c_float()
        _check(lib().ez_batch_timing(self.handle, 1 if enable else 0, ctypes.byref(f), ctypes.byref(t)))
        return f.value, t.value

    def far_flops(self):
        """(algorithmic FP64 flops of the far kernels of the last run, reciprocal terms, coefficients)."""
        f, t, c = ctypes.c_double(), ctypes.c_longlong(), ctypes.c_longlong()
        _check(lib().ez_batch_far_flops(self.handle, ctypes.byref(f), ctypes.byref(t), ctypes.byref(c)))
        return f.value, t.value, c.value

    def sizes(self):
        """(device bytes, host staging bytes) of the batch."""
        a, b = ctypes.c_longlong(), ctypes.c_longlong()
        _check(lib().ez_batch_sizes(self.handle, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def lines(self, stream=None):
        n_lines = int(lib().ez_batch_n_lines(self.handle))
        buf = np.zeros((n_lines, EZ_MAX_PROD))
        offs = (ctypes.c_longlong * (self.n + 1))()
        _check(lib().ez_batch_lines(self.handle, ctypes.c_void_p(buf.ctypes.data), offs, _stream_ptr(stream)))
        return buf, np.array(offs[:])

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and _lib is not None:
            _lib.ez_batch_destroy(h)
            self.handle = None


def ez_diag_fp64_peak(stream=None) -> float:
    v = ctypes.c_double()
    _check(lib().ez_diag_fp64_peak(ctypes.byref(v), _stream_ptr(stream)))
    return v.value


def ez_diag_fp32_peak(stream=None) -> float:
    v = ctypes.c_double()
    _check(lib().ez_diag_fp32_peak(ctypes.byref(v), _stream_ptr(stream)))
    return v.value


def make_request(A, nu, expo, q: ez_quadrature, tag: int = 0, err_est: bool = False) -> ez_request:
    A = np.asarray(A, dtype=np.float64)
    R = ez_request()
    R.d = A.shape[0]
    flat = np.zeros(9)
    flat[: A.size] = A.reshape(-1)
    for i in range(9):
        R.A[i] = flat[i]
    R.spec = sum_spec(nu, expo)
    R.quad = q
    R.tag = tag
    R.flags = EZ_REQ_ERR_EST if err_est else 0
    return R


class Server:
    """ez_server: continuous batching of lattice sums on a worker thread (see ezeta.h)."""

    def __init__(self, mem_budget_bytes: int, n_streams: int = 2, max_batch: int = 256, max_pending: int = 1 << 20,
                 dryrun: bool = False):
        h = ctypes.c_void_p()
        _check(lib().ez_server_create(int(mem_budget_bytes), int(n_streams), int(max_batch), int(max_pending),
                                      EZ_SERVER_DRYRUN if dryrun else 0, ctypes.byref(h)))
        self.handle = h

    def submit(self, req: ez_request) -> int:
        t = ctypes.c_ulonglong()
        _check(lib().ez_server_submit(self.handle, ctypes.byref(req), ctypes.byref(t)))
        return t.value

    def poll(self, max_results: int = 4096):
        buf = (ez_result * max_results)()
        n = ctypes.c_int()
        _check(lib().ez_server_poll(self.handle, buf, max_results, ctypes.byref(n)))
        return [buf[i] for i in range(n.value)]

    def wait(self, ticket: int, timeout_ms: int = 60000) -> ez_result:
        r = ez_result()
        _check(lib().ez_server_wait(self.handle, ticket, int(timeout_ms), ctypes.byref(r)))
        return r

    def stats(self) -> ez_serve_stats:
        st = ez_serve_stats()
        _check(lib().ez_server_stats(self.handle, ctypes.byref(st)))
        return st

    def close(self, timeout_ms: int = 60000):
        if getattr(self, "handle", None) is not None:
            _check(lib().ez_server_destroy(self.handle, int(timeout_ms)))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
