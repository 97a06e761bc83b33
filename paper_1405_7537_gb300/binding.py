"""Thin ctypes binding of the C ABI in include/dpr1.h.

Argument marshalling only: PyTorch provides device memory and the current CUDA
stream; every step of the computation runs in the library's CUDA kernels.  The
library must have been built (``__graft_entry__.build()`` or ``_build.build()``);
there is no CPU fallback, and every call fails loudly if the library or a GPU is
missing.
"""
import ctypes
import os

import numpy as np
import torch

from . import _build

_LIB = None


class Options(ctypes.Structure):
    _fields_ = [("T_Knu", ctypes.c_double), ("T_zero", ctypes.c_double), ("lanes", ctypes.c_int),
                ("warps_per_block", ctypes.c_int), ("blocks_per_sm", ctypes.c_int), ("max_bisect", ctypes.c_int),
                ("phase_events", ctypes.POINTER(ctypes.c_void_p)), ("zero_finder", ctypes.c_int),
                ("dd_mode", ctypes.c_int), ("T_kappa", ctypes.c_double), ("screen", ctypes.c_int)]

BISECTION, ACCELERATED = 0, 1   # dpr1_options.zero_finder


STATUS = {0: "ok", 1: "invalid argument", 2: "d is not sorted non-increasingly", 3: "rho must be finite and >= 0",
          4: "non-finite input", 5: "bisection did not converge", 6: "CUDA error", 7: "workspace error",
          8: "an eigenpair needs values outside the binary64 range"}


class DPR1Error(RuntimeError):
    def __init__(self, code, where):
        self.code = int(code)
        super().__init__("%s: %s (status %d)" % (where, STATUS.get(self.code, "unknown"), self.code))


_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_dbl = ctypes.c_double


def lib():
    """Loads libdpr1.so from the package tree (raises if it was not built)."""
    global _LIB
    if _LIB is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError("CUDA library %s is missing: run __graft_entry__.build() first" % path)
        L = ctypes.CDLL(path)
        L.dpr1_default_options.argtypes = [ctypes.POINTER(Options)]
        L.dpr1_default_options.restype = None
        L.dpr1_status_string.argtypes = [ctypes.c_int]
        L.dpr1_status_string.restype = ctypes.c_char_p
        L.dpr1_workspace_size.argtypes = [_i64]
        L.dpr1_workspace_size.restype = ctypes.c_size_t
        L.dpr1_eig.argtypes = [_i64, _vp, _vp, _dbl, _vp, _vp, _i64, _vp, _vp, _vp, _vp, ctypes.c_size_t,
                               ctypes.POINTER(Options), _vp]
        L.dpr1_eig.restype = ctypes.c_int
        L.dpr1_stream_status.argtypes = [_vp, _vp]
        L.dpr1_stream_status.restype = ctypes.c_int
        L.dpr1_probe_reciprocal.argtypes = [_i64, _vp, _vp, _vp]
        L.dpr1_probe_reciprocal.restype = ctypes.c_int
        L.dpr1_workspace_stats.argtypes = [_vp, ctypes.POINTER(ctypes.c_int64), _vp]
        L.dpr1_workspace_stats.restype = ctypes.c_int
        L.dpr1_probe_dfma.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp]
        L.dpr1_probe_dfma.restype = ctypes.c_int
        L.dpr1_backward_workspace_size.argtypes = [_i64]
        L.dpr1_backward_workspace_size.restype = ctypes.c_size_t
        L.dpr1_batched_workspace_size.argtypes = [_i64, _i64]
        L.dpr1_batched_workspace_size.restype = ctypes.c_size_t
        L.dpr1_hermitian_workspace_size.argtypes = [_i64]
        L.dpr1_hermitian_workspace_size.restype = ctypes.c_size_t
        L.dpr1_tridiag_workspace_size.argtypes = [_i64]
        L.dpr1_tridiag_workspace_size.restype = ctypes.c_size_t
        L.dpr1_arrow_workspace_size.argtypes = [_i64]
        L.dpr1_arrow_workspace_size.restype = ctypes.c_size_t
        for name, argt in _extra_signatures().items():
            if hasattr(L, name):
                getattr(L, name).argtypes = argt
                getattr(L, name).restype = ctypes.c_int
        _LIB = L
    return _LIB


def _extra_signatures():
    return {
        "dpr1_eig_batched": [_i64, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                             ctypes.c_size_t, ctypes.POINTER(Options), _vp],
        "dpr1_eig_backward": [_i64, _vp, _vp, _dbl, _vp, _vp, _vp, _vp, _i64, _vp, _vp, _vp, _vp,
                              ctypes.c_size_t, ctypes.POINTER(Options), _vp],
        "dpr1_eig_hermitian": [_i64, _vp, _vp, _dbl, _vp, _vp, _i64, _vp, _vp, _vp, _vp, ctypes.c_size_t,
                               ctypes.POINTER(Options), _vp],
        "dpr1_tridiag_eig": [_i64, _vp, _vp, _vp, _vp, _i64, _vp, ctypes.c_size_t, ctypes.POINTER(Options), _vp],
        "dpr1_arrow_eig": [_i64, _vp, _vp, _dbl, _vp, _vp, _i64, _vp, _vp, _vp, _vp, ctypes.c_size_t,
                           ctypes.POINTER(Options), _vp],
    }


def default_options(**kw):
    o = Options()
    lib().dpr1_default_options(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _check(code, where):
    if code != 0:
        raise DPR1Error(code, where)


def _dev_f64(t, device):
    if not isinstance(t, torch.Tensor):
        t = torch.from_numpy(np.array(t, dtype=np.float64, copy=True))
    if t.dtype != torch.float64 or t.device != device or not t.is_contiguous():
        t = t.to(device=device, dtype=torch.float64, non_blocking=t.is_pinned()).contiguous()
    return t


def workspace_size(n):
    return int(lib().dpr1_workspace_size(int(n)))


def workspace(n, device="cuda"):
    """A workspace tensor for dpr1_eig on order n (the caching allocator aligns to 512 B)."""
    return torch.empty(max(workspace_size(n), 256), dtype=torch.uint8, device=device)


def stream_status(ws, stream=None):
    """Synchronises the stream and returns the device-recorded status of the last call."""
    return int(lib().dpr1_stream_status(_ptr(ws), _stream(stream)))


def eig(d, z, rho, want_vectors=True, options=None, ws=None, out=None, check=True, stream=None):
    """All eigenpairs of D + rho z z^T (d non-increasing, rho >= 0) on the current CUDA device.

    Returns dict(lam, Vt, sigma, mu, xnorm) of float64 CUDA tensors; row k of Vt is v_k.
    ``check`` synchronises and raises DPR1Error on a device-detected problem."""
    dev = torch.device("cuda", torch.cuda.current_device()) if not (isinstance(d, torch.Tensor) and d.is_cuda) \
        else d.device
    d = _dev_f64(d, dev)
    z = _dev_f64(z, dev)
    n = d.numel()
    if z.numel() != n:
        raise ValueError("d and z must have the same length")
    if out is None:
        out = dict(lam=torch.empty(n, dtype=torch.float64, device=dev),
                   Vt=torch.empty((n, n), dtype=torch.float64, device=dev) if want_vectors else None,
                   sigma=torch.empty(n, dtype=torch.float64, device=dev),
                   mu=torch.empty(n, dtype=torch.float64, device=dev),
                   xnorm=torch.empty(n, dtype=torch.float64, device=dev))
    if ws is None:
        ws = workspace(n, dev)
    o = options if options is not None else default_options()
    Vt = out.get("Vt")
    code = lib().dpr1_eig(n, _ptr(d), _ptr(z), float(rho), _ptr(out["lam"]), _ptr(Vt), n if Vt is not None else 0,
                          _ptr(out.get("sigma")), _ptr(out.get("mu")), _ptr(out.get("xnorm")), _ptr(ws),
                          ws.numel(), ctypes.byref(o), _stream(stream))
    _check(code, "dpr1_eig")
    if check and n > 0:
        _check(stream_status(ws, stream), "dpr1_eig (device)")
    return out


def hermitian_workspace(n, device="cuda"):
    return torch.empty(max(int(lib().dpr1_hermitian_workspace_size(int(n))), 256), dtype=torch.uint8, device=device)


def eig_hermitian(d, z, rho, want_vectors=True, options=None, ws=None, check=True, stream=None):
    """All eigenpairs of the Hermitian D + rho z z^* (d real non-increasing, z complex, rho >= 0).

    Returns dict(lam, Vt, sigma, mu, xnorm); Vt is complex128 with row k = v_k."""
    dev = d.device if isinstance(d, torch.Tensor) and d.is_cuda else torch.device("cuda", torch.cuda.current_device())
    d = _dev_f64(d, dev)
    if not isinstance(z, torch.Tensor):
        z = torch.from_numpy(np.array(z, dtype=np.complex128, copy=True))
    z = z.to(device=dev, dtype=torch.complex128).contiguous()
    n = d.numel()
    if z.numel() != n:
        raise ValueError("d and z must have the same length")
    f64 = dict(dtype=torch.float64, device=dev)
    out = dict(lam=torch.empty(n, **f64), sigma=torch.empty(n, **f64), mu=torch.empty(n, **f64),
               xnorm=torch.empty(n, **f64),
               Vt=torch.empty((n, n), dtype=torch.complex128, device=dev) if want_vectors else None)
    if ws is None:
        ws = hermitian_workspace(n, dev)
    o = options if options is not None else default_options()
    Vt = out["Vt"]
    code = lib().dpr1_eig_hermitian(n, _ptr(d), _ptr(z), float(rho), _ptr(out["lam"]), _ptr(Vt),
                                    n if Vt is not None else 0, _ptr(out["sigma"]), _ptr(out["mu"]),
                                    _ptr(out["xnorm"]), _ptr(ws), ws.numel(), ctypes.byref(o), _stream(stream))
    _check(code, "dpr1_eig_hermitian")
    if check and n > 0:
        _check(stream_status(ws, stream), "dpr1_eig_hermitian (device)")
    return out


def tridiag_workspace(n, device="cuda"):
    return torch.empty(max(int(lib().dpr1_tridiag_workspace_size(int(n))), 256), dtype=torch.uint8, device=device)


def eigh_tridiagonal(a, b, want_vectors=True, options=None, ws=None, check=True, stream=None):
    """All eigenpairs of the symmetric tridiagonal matrix with diagonal a and off-diagonal b
    (divide and conquer with DPR1 merges).  Returns (lam non-increasing, Qt) with Qt[k] the
    k-th eigenvector (None when want_vectors is False)."""
    dev = a.device if isinstance(a, torch.Tensor) and a.is_cuda else torch.device("cuda", torch.cuda.current_device())
    a = _dev_f64(a, dev)
    n = a.numel()
    b = _dev_f64(b, dev) if n > 1 else None
    if n > 1 and b.numel() != n - 1:
        raise ValueError("b must have n - 1 entries")
    lam = torch.empty(n, dtype=torch.float64, device=dev)
    Qt = torch.empty((n, n), dtype=torch.float64, device=dev) if want_vectors else None
    if ws is None:
        ws = tridiag_workspace(n, dev)
    o = options if options is not None else default_options()
    code = lib().dpr1_tridiag_eig(n, _ptr(a), _ptr(b), _ptr(lam), _ptr(Qt), n if Qt is not None else 0, _ptr(ws),
                                  ws.numel(), ctypes.byref(o), _stream(stream))
    _check(code, "dpr1_tridiag_eig")
    if check and n > 0:
        _check(stream_status(ws, stream), "dpr1_tridiag_eig (device)")
    return lam, Qt


def arrow_workspace(n, device="cuda"):
    return torch.empty(max(int(lib().dpr1_arrow_workspace_size(int(n))), 256), dtype=torch.uint8, device=device)


def eig_arrowhead(d, z, alpha, want_vectors=True, options=None, ws=None, check=True, stream=None):
    """All n + 1 eigenpairs of the arrowhead [diag(d) z; z^T alpha] (d strictly decreasing, no
    zero weight), with the K_nu remedies and the near-zero recompute.  Returns dict(lam, Vt,
    sigma, mu, xnorm); Vt is (n+1) x (n+1), row k = v_k.  ``workspace_stats(ws)`` gives the
    counters of the call."""
    dev = d.device if isinstance(d, torch.Tensor) and d.is_cuda else torch.device("cuda", torch.cuda.current_device())
    d = _dev_f64(d, dev)
    z = _dev_f64(z, dev)
    n = d.numel()
    if z.numel() != n:
        raise ValueError("d and z must have the same length")
    f64 = dict(dtype=torch.float64, device=dev)
    out = dict(lam=torch.empty(n + 1, **f64), sigma=torch.empty(n + 1, **f64), mu=torch.empty(n + 1, **f64),
               xnorm=torch.empty(n + 1, **f64), Vt=torch.empty((n + 1, n + 1), **f64) if want_vectors else None)
    if ws is None:
        ws = arrow_workspace(n, dev)
    o = options if options is not None else default_options()
    Vt = out["Vt"]
    code = lib().dpr1_arrow_eig(n, _ptr(d), _ptr(z), float(alpha), _ptr(out["lam"]), _ptr(Vt),
                                n + 1 if Vt is not None else 0, _ptr(out["sigma"]), _ptr(out["mu"]),
                                _ptr(out["xnorm"]), _ptr(ws), ws.numel(), ctypes.byref(o), _stream(stream))
    _check(code, "dpr1_arrow_eig")
    if check:
        _check(stream_status(ws, stream), "dpr1_arrow_eig (device)")
    return out


def probe_reciprocal(x):
    x = _dev_f64(x, torch.device("cuda", torch.cuda.current_device()))
    out = torch.empty_like(x)
    _check(lib().dpr1_probe_reciprocal(x.numel(), _ptr(x), _ptr(out), _stream()), "dpr1_probe_reciprocal")
    torch.cuda.synchronize()
    return out


STAT_NAMES = ("solved", "flagged", "r1", "r2", "evals_solve", "evals_fix", "zero_path", "deflated", "double_double",
              "screened", "r2_double_double", "screened_near_bound", "screened_double_float", "inferred",
              "probes", "shift_binary32", "tail_rows", "vector_rows")


def workspace_stats(ws, stream=None):
    """Counters of the last dpr1_eig / dpr1_eig_batched / dpr1_arrow_eig call on ``ws``
    (synchronises the stream)."""
    buf = (ctypes.c_int64 * len(STAT_NAMES))()
    _check(lib().dpr1_workspace_stats(_ptr(ws), buf, _stream(stream)), "dpr1_workspace_stats")
    return dict(zip(STAT_NAMES, list(buf)))


class PhaseEvents:
    """Four CUDA events the library records around its phases (see dpr1_options.phase_events)."""

    def __init__(self):
        self.events = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        for e in self.events:          # torch creates the CUDA event lazily, on first record
            e.record()
        torch.cuda.synchronize()
        self._arr = (ctypes.c_void_p * 4)(*[ctypes.c_void_p(e.cuda_event) for e in self.events])

    def attach(self, options):
        options.phase_events = ctypes.cast(self._arr, ctypes.POINTER(ctypes.c_void_p))
        return options

    def times_ms(self):
        """(bisection kernel, remedies, eigenvectors) in ms for the last recorded call."""
        e = self.events
        return e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2]), e[2].elapsed_time(e[3])


def probe_dfma(blocks, threads, iters, sink, stream=None):
    _check(lib().dpr1_probe_dfma(int(blocks), int(threads), int(iters), _ptr(sink), _stream(stream)),
           "dpr1_probe_dfma")


def backward_workspace(n, device="cuda"):
    return torch.empty(max(int(lib().dpr1_backward_workspace_size(int(n))), 256), dtype=torch.uint8, device=device)


def eig_backward(d, z, rho, sigma, mu, grad_lam=None, grad_Vt=None, ws=None, check=True, stream=None):
    """(grad_d, grad_z, grad_rho) of L given dL/dlambda and dL/dVt (rows = dL/dv_k)."""
    dev = d.device
    n = d.numel()
    gd = torch.empty(n, dtype=torch.float64, device=dev)
    gz = torch.empty(n, dtype=torch.float64, device=dev)
    gr = torch.empty(1, dtype=torch.float64, device=dev)
    if ws is None:
        ws = backward_workspace(n, dev)
    gl = grad_lam.contiguous() if grad_lam is not None else None
    gV = grad_Vt.contiguous() if grad_Vt is not None else None
    code = lib().dpr1_eig_backward(n, _ptr(d), _ptr(z), float(rho), _ptr(sigma), _ptr(mu), _ptr(gl), _ptr(gV),
                                   n if gV is not None else 0, _ptr(gd), _ptr(gz), _ptr(gr), _ptr(ws), ws.numel(),
                                   None, _stream(stream))
    _check(code, "dpr1_eig_backward")
    if check and n > 0:
        _check(stream_status(ws, stream), "dpr1_eig_backward (device)")
    return gd, gz, gr[0]


class DPR1Eig(torch.autograd.Function):
    """(lambda, V) = eig(D + rho z z^T) with V[:, k] = v_k, lambda non-increasing.

    Saves d, z, rho and the pairs (sigma, mu) only; the backward recomputes the
    eigenvector columns from them (V is not kept for the backward)."""

    @staticmethod
    def forward(ctx, d, z, rho):
        r = rho.item() if isinstance(rho, torch.Tensor) else float(rho)
        out = eig(d.detach(), z.detach(), r)
        ctx.save_for_backward(d.detach(), z.detach(), out["sigma"], out["mu"])
        ctx.rho = r
        ctx.rho_is_tensor = isinstance(rho, torch.Tensor)
        return out["lam"], out["Vt"].t()

    @staticmethod
    def backward(ctx, g_lam, g_V):
        d, z, sig, mu = ctx.saved_tensors
        gVt = g_V.t().contiguous() if g_V is not None else None
        gd, gz, gr = eig_backward(d, z, ctx.rho, sig, mu, g_lam, gVt)
        return gd, gz, (gr.reshape(()) if ctx.rho_is_tensor else None)


def eigh_dpr1(d, z, rho):
    """Differentiable eigen-decomposition of D + rho z z^T: returns (lambda, V), V[:, k] = v_k."""
    return DPR1Eig.apply(d, z, rho)


def batched_workspace(nprob, total_n, device="cuda"):
    nb = int(lib().dpr1_batched_workspace_size(int(nprob), int(total_n)))
    return torch.empty(max(nb, 256), dtype=torch.uint8, device=device)


class Batch:
    """A batch of independent DPR1 problems laid out for dpr1_eig_batched.

    sizes: problem orders n_p; d, z: concatenated (device, float64); rho: per problem.
    Allocates the outputs (eigenvalues and eigenvector blocks) and the workspace once,
    so that repeated solves and CUDA-graph replays reuse them."""

    def __init__(self, sizes, device="cuda", want_vectors=True):
        sizes = np.asarray(sizes, dtype=np.int64)
        self.P = int(sizes.size)
        offs = np.zeros(self.P + 1, dtype=np.int64)
        offs[1:] = np.cumsum(sizes)
        voffs = np.zeros(self.P + 1, dtype=np.int64)
        voffs[1:] = np.cumsum(sizes * sizes)
        self.total = int(offs[-1])
        self.sizes = sizes
        self.offs_host, self.voffs_host = offs, voffs
        self.device = torch.device(device)
        self.offs = torch.tensor(offs, device=device)
        self.voffs = torch.tensor(voffs, device=device)
        f64 = dict(dtype=torch.float64, device=device)
        self.lam = torch.empty(self.total, **f64)
        self.sigma = torch.empty(self.total, **f64)
        self.mu = torch.empty(self.total, **f64)
        self.xnorm = torch.empty(self.total, **f64)
        self.Vt = torch.empty(int(voffs[-1]), **f64) if want_vectors else None
        self.ws = batched_workspace(self.P, self.total, device)

    def solve(self, d, z, rho, options=None, check=False, stream=None):
        o = options if options is not None else default_options()
        code = lib().dpr1_eig_batched(self.P, self.total, _ptr(self.offs), _ptr(self.voffs), _ptr(d), _ptr(z),
                                      _ptr(rho), _ptr(self.lam), _ptr(self.Vt), _ptr(self.sigma), _ptr(self.mu),
                                      _ptr(self.xnorm), _ptr(self.ws), self.ws.numel(), ctypes.byref(o),
                                      _stream(stream))
        _check(code, "dpr1_eig_batched")
        if check:
            _check(stream_status(self.ws, stream), "dpr1_eig_batched (device)")

    def block(self, p):
        """(lambda, Vt) views of problem p."""
        a, b = int(self.offs_host[p]), int(self.offs_host[p + 1])
        n = b - a
        va = int(self.voffs_host[p])
        Vt = self.Vt[va:va + n * n].view(n, n) if self.Vt is not None else None
        return self.lam[a:b], Vt
