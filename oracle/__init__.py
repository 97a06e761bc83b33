"""CPU oracle for the DPR1 eigensolver (arXiv 1405.7537) -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package.  The CUDA library never calls it, and it never calls the
CUDA library.

Two references live here:

* ``dpr1eig`` / ``eig_all``: Algorithm 1 (dpr1eig) step by step in binary64 with
  its own double-double code (``dpr1_oracle.c``).
* ``quad_eig``: the plain definition of the eigenpairs -- the zeros of the secular
  function Eq. (Pick) bisected in binary128, and x = (D - lambda I)^{-1} z
  (``quad_ref.c``).

``eig_full`` adds the paper's deflation (Sec. 1: zeta_j = 0 gives the eigenpair
(d_j, e_j); d_i = d_j gives the eigenvalue d_i after a Givens rotation in the
(i, j) plane) and the sign flip for rho < 0 (Sec. 1) around ``eig_all``.
``backward`` is the adjoint of (lambda, V) with respect to (d, z, rho).
``eig_hermitian`` reduces the complex Hermitian D + rho z z^* to the real problem with
weights |z_j| by the diagonal unitary of the phases of z.
"""
import ctypes
import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from .build import build_oracle

_LIB = None


class Opts(ctypes.Structure):
    _fields_ = [("dd_mode", ctypes.c_int), ("T_kappa", ctypes.c_double), ("T_Knu", ctypes.c_double),
                ("T_zero", ctypes.c_double), ("remedies", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [("shift", ctypes.c_int), ("first_shift", ctypes.c_int), ("used_dd", ctypes.c_int),
                ("remedy", ctypes.c_int), ("zero_path", ctypes.c_int), ("steps", ctypes.c_int),
                ("sigma", ctypes.c_double), ("mu", ctypes.c_double), ("nu", ctypes.c_double),
                ("lam", ctypes.c_double), ("b", ctypes.c_double), ("K_nu", ctypes.c_double),
                ("K_nu_final", ctypes.c_double), ("kappa_nu", ctypes.c_double), ("r2_dd", ctypes.c_int)]


_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


class OracleRangeError(ValueError):
    """The eigenpair needs values outside the binary64 range of the normalised problem (the
    oracle's code 4): mu zero, subnormal or not finite, or lambda or the vector not finite."""


def _raise(fn, rc):
    if rc == 4:
        raise OracleRangeError("%s: outside the binary64 range (code 4)" % fn)
    raise ValueError("%s failed with code %d" % (fn, rc))


def lib():
    global _LIB
    if _LIB is None:
        path = build_oracle()
        L = ctypes.CDLL(path)
        L.oracle_dpr1eig.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_double, ctypes.c_int,
                                     ctypes.POINTER(Opts), _dp, _dp, ctypes.POINTER(Info)]
        L.oracle_dpr1eig_range.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_double, ctypes.c_int,
                                           ctypes.c_int, ctypes.POINTER(Opts), _dp, _dp, _dp, _dp,
                                           _ip, _ip]
        L.oracle_backward.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_double, _dp, _dp, _dp, _dp,
                                      _dp, _dp, _dp]
        L.oracle_backward_rows.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_double, ctypes.c_int, _ip, _dp, _dp,
                                           _dp, _dp, _dp, _dp, _dp]
        L.quad_eigpair.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_double, ctypes.c_int, _dp, _dp, _dp]
        L.quad_eigpair2.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_double, ctypes.c_int, _dp, _dp, _dp,
                                    _dp, _ip, _dp]
        L.quad_backward.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_double, ctypes.c_int, _ip, _dp, _dp, _dp,
                                    _dp, _dp]
        L.quad_secular.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double]
        L.quad_secular.restype = ctypes.c_double
        for name in ("oracle_dd_add", "oracle_dd_mul", "oracle_dd_div"):
            getattr(L, name).argtypes = [ctypes.c_double] * 4 + [_dp]
        L.oracle_default_opts.argtypes = [ctypes.POINTER(Opts)]
        L.oracle_arroweig.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_double, ctypes.c_int, ctypes.POINTER(Opts),
                                      _dp, _dp, _dp, _dp, _ip, _ip, _dp]
        L.quad_arrow_eigpair.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_double, ctypes.c_int, _dp, _dp, _dp]
        for name in ("oracle_dpr1_r2", "oracle_arrow_r2"):
            getattr(L, name).argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                         _dp, _dp, _dp]
        _LIB = L
    return _LIB


def _ptr(a):
    return a.ctypes.data_as(_dp) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def default_opts(**kw):
    o = Opts()
    lib().oracle_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def dpr1eig(d, z, rho, k, opts=None):
    """Algorithm 1 for the k-th eigenpair (0-based, lambda_0 the largest).

    Returns (lambda, v, info) where info is a dict of the decisions taken."""
    d, z = _f64(d), _f64(z)
    n = d.size
    v = np.empty(n)
    lam = ctypes.c_double()
    info = Info()
    o = opts if opts is not None else default_opts()
    rc = lib().oracle_dpr1eig(n, _ptr(d), _ptr(z), float(rho), int(k), ctypes.byref(o),
                              ctypes.byref(lam), _ptr(v), ctypes.byref(info))
    if rc:
        _raise("oracle_dpr1eig", rc)
    return lam.value, v, {f[0]: getattr(info, f[0]) for f in Info._fields_}


def eig_all(d, z, rho, opts=None, ks=None, threads=1, want_vectors=True):
    """All (or the listed) eigenpairs of an irreducible, strictly ordered problem.

    Returns dict(lam, Vt, sigma, mu, shift, flags) indexed by the position in ks.
    flags: bit0-1 remedy (1 = R1, 2 = R2), bit2 near-zero recompute, bit3 double-double used,
    bit4 the R2 shift formed in double the working precision.
    The eigenpairs are independent; ``threads`` > 1 splits them over host threads
    (the C calls release the interpreter lock)."""
    d, z = _f64(d), _f64(z)
    n = d.size
    ks = np.arange(n) if ks is None else np.asarray(ks, dtype=np.int64)
    m = ks.size
    o = opts if opts is not None else default_opts()
    out = dict(lam=np.empty(m), sigma=np.empty(m), mu=np.empty(m),
               shift=np.empty(m, dtype=np.int32), flags=np.empty(m, dtype=np.int32),
               Vt=np.empty((m, n)) if want_vectors else None)

    def run(idx):
        v = np.empty(n)
        lam = ctypes.c_double()
        info = Info()
        L = lib()
        for p in idx:
            rc = L.oracle_dpr1eig(n, _ptr(d), _ptr(z), float(rho), int(ks[p]), ctypes.byref(o),
                                  ctypes.byref(lam), _ptr(v), ctypes.byref(info))
            if rc:
                _raise("oracle_dpr1eig", rc)
            out["lam"][p] = lam.value
            out["sigma"][p] = info.sigma
            out["mu"][p] = info.mu
            out["shift"][p] = info.shift
            out["flags"][p] = info.remedy | (info.zero_path << 2) | (info.used_dd << 3) | (info.r2_dd << 4)
            if want_vectors:
                out["Vt"][p] = v

    if threads <= 1 or m < 2:
        run(range(m))
    else:
        parts = np.array_split(np.arange(m), threads)
        with ThreadPoolExecutor(threads) as ex:
            list(ex.map(run, parts))
    return out


def backward(d, z, rho, sigma, mu, grad_lam=None, grad_Vt=None):
    """Adjoint of (lambda, V) -> (d, z, rho) from the pairs (sigma, mu); returns (gd, gz, grho)."""
    d, z, sigma, mu = _f64(d), _f64(z), _f64(sigma), _f64(mu)
    n = d.size
    gl = _f64(grad_lam) if grad_lam is not None else None
    gV = _f64(grad_Vt) if grad_Vt is not None else None
    gd, gz, gr = np.empty(n), np.empty(n), ctypes.c_double()
    rc = lib().oracle_backward(n, _ptr(d), _ptr(z), float(rho), _ptr(sigma), _ptr(mu), _ptr(gl),
                               _ptr(gV), _ptr(gd), _ptr(gz), ctypes.byref(gr))
    if rc:
        raise ValueError("oracle_backward failed with code %d" % rc)
    return gd, gz, gr.value


def backward_rows(d, z, rho, sigma, mu, grad_lam=None, grad_Vt=None):
    """The adjoint summed over the eigenpairs whose (sigma, mu) are given (any subset);
    grad_lam[t] and grad_Vt[t] belong to the pair (sigma[t], mu[t])."""
    d, z, sigma, mu = _f64(d), _f64(z), _f64(sigma), _f64(mu)
    n, m = d.size, sigma.size
    gl = _f64(grad_lam) if grad_lam is not None else None
    gV = _f64(grad_Vt) if grad_Vt is not None else None
    gd, gz, gr = np.empty(n), np.empty(n), ctypes.c_double()
    rc = lib().oracle_backward_rows(n, _ptr(d), _ptr(z), float(rho), m, None, _ptr(sigma), _ptr(mu), _ptr(gl),
                                    _ptr(gV), _ptr(gd), _ptr(gz), ctypes.byref(gr))
    if rc:
        raise ValueError("oracle_backward_rows failed with code %d" % rc)
    return gd, gz, gr.value


def quad_eig(d, z, rho, k, want_vector=True, full=False):
    """binary128 reference for eigenpair k: (lam_hi, lam_lo, v).

    With full=True returns dict(hi, lo, mu_hi, mu_lo, pole, v): lambda = d[pole] + mu."""
    d, z = _f64(d), _f64(z)
    n = d.size
    v = np.empty(n) if want_vector else None
    hi, lo, mh, ml = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    pole = ctypes.c_int()
    rc = lib().quad_eigpair2(n, _ptr(d), _ptr(z), float(rho), int(k), ctypes.byref(hi), ctypes.byref(lo),
                             ctypes.byref(mh), ctypes.byref(ml), ctypes.byref(pole), _ptr(v))
    if rc < 0:
        raise ValueError("quad_eigpair: bad arguments")
    if full:
        return dict(hi=hi.value, lo=lo.value, mu_hi=mh.value, mu_lo=ml.value, pole=pole.value, v=v)
    return hi.value, lo.value, v


def quad_all(d, z, rho, ks=None, threads=1, want_vectors=True):
    """binary128 reference for several eigenpairs: dict(hi, lo, mu_hi, mu_lo, pole, Vt)."""
    d, z = _f64(d), _f64(z)
    n = d.size
    ks = np.arange(n) if ks is None else np.asarray(ks, dtype=np.int64)
    m = ks.size
    out = dict(hi=np.empty(m), lo=np.empty(m), mu_hi=np.empty(m), mu_lo=np.empty(m),
               pole=np.empty(m, dtype=np.int64), Vt=np.empty((m, n)) if want_vectors else None)

    def run(idx):
        for p in idx:
            r = quad_eig(d, z, rho, ks[p], want_vectors, full=True)
            for key in ("hi", "lo", "mu_hi", "mu_lo", "pole"):
                out[key][p] = r[key]
            if want_vectors:
                out["Vt"][p] = r["v"]

    if threads <= 1 or m < 2:
        run(range(m))
    else:
        with ThreadPoolExecutor(threads) as ex:
            list(ex.map(run, np.array_split(np.arange(m), threads)))
    return out


def quad_backward(d, z, rho, grad_lam=None, grad_Vt=None, ks=None):
    """binary128 adjoint summed over eigenpairs ks (default all); grad rows belong to ks."""
    d, z = _f64(d), _f64(z)
    n = d.size
    ks = np.arange(n, dtype=np.int32) if ks is None else np.ascontiguousarray(ks, dtype=np.int32)
    gl = _f64(grad_lam) if grad_lam is not None else None
    gV = _f64(grad_Vt) if grad_Vt is not None else None
    gd, gz, gr = np.empty(n), np.empty(n), ctypes.c_double()
    rc = lib().quad_backward(n, _ptr(d), _ptr(z), float(rho), ks.size, ks.ctypes.data_as(_ip), _ptr(gl), _ptr(gV),
                             _ptr(gd), _ptr(gz), ctypes.byref(gr))
    if rc:
        raise ValueError("quad_backward failed")
    return gd, gz, gr.value


def quad_secular(d, z, rho, lam_hi, lam_lo=0.0):
    d, z = _f64(d), _f64(z)
    return lib().quad_secular(d.size, _ptr(d), _ptr(z), float(rho), float(lam_hi), float(lam_lo))


def dd_op(name, a, b):
    """Double-double add/mul/div of the oracle on (hi, lo) pairs, for its own pins."""
    out = np.empty(2)
    getattr(lib(), "oracle_dd_" + name)(a[0], a[1], b[0], b[1], _ptr(out))
    return out[0], out[1]


def zero_weight(z, zmax=None):
    """A weight that is below 2^-511 after the normalisation max|zeta| in [1/2, 1) counts as zero:
    |zeta_j| < 2^(e - 511) with max|zeta| = m 2^e (m in [1/2, 1); ``zmax`` gives the maximum when
    z is a part of the problem).  The secular function of the normalised problem sees only
    zeta_j^2, which is then not a normal binary64 number, and deflating it changes
    A = D + rho z z^T by less than 2^-510 rho ||z||."""
    z = np.asarray(z)
    m = float(np.max(np.abs(z))) if zmax is None and z.size else (0.0 if zmax is None else float(zmax))
    e = math.frexp(m)[1] if (m > 0.0 and math.isfinite(m)) else 0
    return np.abs(z) < math.ldexp(1.0, e - 511)


def eig_full(d, z, rho, opts=None, threads=1):
    """Eigen-decomposition of D + rho z z^T for any d sorted non-increasingly.

    Handles rho == 0 (lambda = d, V = I), rho < 0 (Sec. 1: solve -D - rho z z^T),
    zeta_j == 0 and d_j == d_{j+1} (Sec. 1 deflation, exact tests only; a weight below 2^-511
    times the power of two above the largest weight counts as zero, see ``zero_weight``) and returns
    dict(lam, Vt, sigma, mu) with lam non-increasing and Vt[k] = v_k.  Deflated pairs
    carry sigma = lambda and mu = 0."""
    d = _f64(d).copy()
    z = _f64(z).copy()
    n = d.size
    if n == 0:
        return dict(lam=np.empty(0), Vt=np.empty((0, 0)), sigma=np.empty(0), mu=np.empty(0))
    if np.any(d[:-1] < d[1:]):
        raise ValueError("d must be sorted non-increasingly")
    if rho == 0.0:
        return dict(lam=d.copy(), Vt=np.eye(n), sigma=d.copy(), mu=np.zeros(n))
    if rho < 0.0:
        # A = -( (-D) + |rho| z z^T ); -D is increasing, so reverse to keep the order
        r = eig_full(-d[::-1], z[::-1], -rho, opts, threads)
        lam = -r["lam"][::-1]
        Vt = r["Vt"][::-1, ::-1]
        return dict(lam=lam.copy(), Vt=np.ascontiguousarray(Vt), sigma=-r["sigma"][::-1].copy(),
                    mu=-r["mu"][::-1].copy())
    # --- deflation (exact tests only) ---
    Q = np.eye(n)              # accumulated rotations: z_rot = Q z, A = Q^T (D + rho z_rot z_rot^T) Q
    zr = z.copy()
    zmax = float(np.max(np.abs(z)))   # the zero-weight rule is relative to the largest weight
    defl = []                  # (position, eigenvalue) of deflated pairs in the rotated basis
    for j in range(n):
        if zero_weight(zr[j], zmax):
            defl.append(j)
    # ties: rotate each later member of a group of equal d's into the first non-zero member
    j = 0
    while j < n:
        g = j
        while g + 1 < n and d[g + 1] == d[j]:
            g += 1
        members = [p for p in range(j, g + 1) if not zero_weight(zr[p], zmax)]
        if len(members) > 1:
            a = members[0]
            for p in members[1:]:
                r = np.hypot(zr[a], zr[p])
                c, s = zr[a] / r, zr[p] / r
                G = np.eye(n)
                G[a, a], G[a, p], G[p, a], G[p, p] = c, s, -s, c
                zr = G @ zr
                zr[p] = 0.0
                Q = G @ Q
                defl.append(p)
        j = g + 1
    keep = np.array([p for p in range(n) if p not in set(defl)], dtype=np.int64)
    lam_all, vec_all, sig_all, mu_all = [], [], [], []
    if keep.size:
        r = eig_all(d[keep], zr[keep], rho, opts, threads=threads)
        for t in range(keep.size):
            x = np.zeros(n)
            x[keep] = r["Vt"][t]
            lam_all.append(r["lam"][t]); vec_all.append(Q.T @ x)
            sig_all.append(r["sigma"][t]); mu_all.append(r["mu"][t])
    for p in defl:
        e = np.zeros(n); e[p] = 1.0
        lam_all.append(d[p]); vec_all.append(Q.T @ e); sig_all.append(d[p]); mu_all.append(0.0)
    lam_all = np.array(lam_all)
    order = np.argsort(-lam_all, kind="stable")
    return dict(lam=lam_all[order], Vt=np.array(vec_all)[order], sigma=np.array(sig_all)[order],
                mu=np.array(mu_all)[order])


def hermitian_abs(z):
    """|z_j| of complex z as one fixed sequence of correctly rounded binary64 operations:
    sqrt(x'^2 + y'^2) / s with x' = s Re z_j, y' = s Im z_j and s = 2^-600 (max(|Re|, |Im|) >
    2^500), 2^600 (below 2^-500) or 1 (separate numpy operations, so no contraction).  This is
    the reading the Hermitian reduction fixes for its real weights."""
    z = np.ascontiguousarray(z, dtype=np.complex128)
    re, im = z.real.copy(), z.imag.copy()
    m = np.maximum(np.abs(re), np.abs(im))
    s = np.where(m > 2.0 ** 500, 2.0 ** -600, np.where(m < 2.0 ** -500, 2.0 ** 600, 1.0))
    inv = np.where(m > 2.0 ** 500, 2.0 ** 600, np.where(m < 2.0 ** -500, 2.0 ** -600, 1.0))
    x = re * s
    y = im * s
    xx = x * x
    yy = y * y
    return np.sqrt(xx + yy) * inv


def eig_hermitian(d, z, rho, opts=None, threads=1, ks=None):
    """Eigenpairs of the complex Hermitian D + rho z z^* (d real, non-increasing).

    With phi_j = z_j / |z_j| (phi_j = 1 for z_j = 0; |z_j| from ``hermitian_abs``) and Phi = diag(phi),
    Phi^* (D + rho z z^*) Phi = D + rho |z| |z|^T: the eigenvalues are those of the real
    problem with weights |z_j| (Algorithm 1 through ``eig_all``, or ``eig_full`` when it
    deflates) and v_k = Phi u_k.  Returns dict(lam, Vt, sigma, mu) with complex Vt[k] = v_k."""
    d = _f64(d)
    z = np.ascontiguousarray(z, dtype=np.complex128)
    a = hermitian_abs(z)
    phi = np.ones(z.size, dtype=np.complex128)
    nz = a > 0
    phi[nz] = z.real[nz] / a[nz] + 1j * (z.imag[nz] / a[nz])   # each part correctly rounded
    irreducible = rho > 0 and not np.any(zero_weight(a)) and np.all(d[:-1] > d[1:])
    if irreducible:
        r = eig_all(d, a, rho, opts, ks=ks, threads=threads)
    else:
        if ks is not None:
            raise ValueError("sampled rows need an irreducible problem")
        r = eig_full(d, a, rho, opts, threads=threads)
    out = dict(r)
    out["Vt"] = r["Vt"] * phi[None, :]
    return out


def tridiag_tree(n, t):
    """Node boundaries at depth t of the divide-and-conquer tree of order n:
    node i covers [s_i, s_{i+1}), s_i = floor(i n / 2^t); its children are nodes 2i and
    2i + 1 at depth t + 1, so every boundary between consecutive indices is split once."""
    return [(i * n) >> t for i in range((1 << t) + 1)]


def tridiag_dc(a, b, threads=1):
    """Eigen-decomposition of the symmetric tridiagonal T (diagonal a, off-diagonal b) by
    divide and conquer down to single elements, every merge a DPR1 problem (Sec. 1: the
    merges of Cuppen's method are DPR1 eigenproblems).

    Tear at the boundary between m - 1 and m of a node: T = diag(T1, T2) + rho v v^T with
    rho = |b_{m-1}|, v = e_{m-1} + sign(b_{m-1}) e_m, and T1, T2 with |b_{m-1}| taken off
    their corner diagonal entries; so a single element i carries a_i - |b_{i-1}| - |b_i|.
    Merge: with T1 = Q1 L1 Q1^T and T2 = Q2 L2 Q2^T, T = Q (L + rho u u^T) Q^T,
    Q = diag(Q1, Q2), u = Q^T v = (last row of Q1, sign * first row of Q2).  Weights with
    rho |u_j| <= 8 u ||T|| (u = 2^-53, ||T|| the largest Gershgorin row sum) are set to zero,
    the usual backward-stable deflation of divide and conquer; beyond the exact deflation
    of Sec. 1 it keeps the squares u_j^2 in the normal range of binary64.  The poles
    L1, L2 are merged into one non-increasing order (stable: T1's entry first on ties),
    the DPR1 problem is solved by ``eig_full`` (Algorithm 1 with the paper's deflation),
    and the eigenvectors of T are Q times the DPR1 eigenvectors mapped back to the
    unsorted order.  Returns (lam non-increasing, Qt) with Qt[k] the k-th eigenvector."""
    a = _f64(a)
    b = _f64(b)
    n = a.size
    if n == 0:
        return np.empty(0), np.empty((0, 0))
    if b.size != max(n - 1, 0):
        raise ValueError("b must have n - 1 entries")
    bl = np.concatenate([[0.0], np.abs(b)])
    br = np.concatenate([np.abs(b), [0.0]])
    leaf = (a - bl) - br
    # deflation tolerance of every merge: 8 u ||T||, u = 2^-53, ||T|| bounded by the largest
    # Gershgorin row sum (|a_i| + |b_{i-1}|) + |b_i|
    tol = np.ldexp(np.max((np.abs(a) + bl) + br), -50)
    T = 0
    while (1 << T) < n:
        T += 1
    # depth T: every node has at most one element
    lam = leaf.copy()
    blocks = {}
    s = tridiag_tree(n, T)
    for i in range(1 << T):
        if s[i + 1] - s[i] == 1:
            blocks[i] = np.ones((1, 1))
    for t in range(T - 1, -1, -1):
        s = tridiag_tree(n, t)
        lam_t = np.empty(n)
        new = {}
        for i in range(1 << t):
            lo, hi = s[i], s[i + 1]
            N = hi - lo
            if N == 0:
                continue
            if N == 1:
                lam_t[lo] = leaf[lo]
                new[i] = np.ones((1, 1))
                continue
            mid = ((2 * i + 1) * n) >> (t + 1)
            n1 = mid - lo
            Q1, Q2 = blocks[2 * i], blocks[2 * i + 1]
            beta = b[mid - 1]
            rho = abs(beta)
            sgn = 1.0 if beta >= 0 else -1.0
            vals = lam[lo:hi]
            u = np.concatenate([Q1[:, n1 - 1], sgn * Q2[:, 0]])
            # a weight with rho |u_j| <= tol is deflated (its pole is an eigenvalue of T to
            # within the backward error 8 u ||T|| of the whole method)
            u[rho * np.abs(u) <= tol] = 0.0
            order = np.argsort(-vals, kind="stable")
            r = eig_full(vals[order], u[order], rho, threads=threads)
            pos = np.empty(N, dtype=np.int64)
            pos[order] = np.arange(N)
            Gt = r["Vt"][:, pos]                      # Gt[k, src] = w_k at the sorted position of src
            Qt = np.empty((N, N))
            Qt[:, :n1] = Gt[:, :n1] @ Q1
            Qt[:, n1:] = Gt[:, n1:] @ Q2
            lam_t[lo:hi] = r["lam"]
            new[i] = Qt
        lam, blocks = lam_t, new
    return lam, blocks[0]


def _split_run(run, m, threads):
    if threads <= 1 or m < 2:
        run(range(m))
    else:
        with ThreadPoolExecutor(threads) as ex:
            list(ex.map(run, np.array_split(np.arange(m), threads)))


def arrow_eig_all(d, z, alpha, ks=None, threads=1, opts=None):
    """Eigenpairs of the arrowhead [diag(d) z; z^T alpha] (order n + 1, irreducible) by the
    steps of Algorithm 1 on its shifted inverse, with the remedies of Sec. 2 for large K_nu
    and the near-zero recompute (``oracle_arroweig``; opts as for ``dpr1eig``): dict(lam,
    sigma, mu, shift, flags, K_nu, Vt) with rows of length n + 1, for k in ks (default 0..n).
    flags: 1 R1, 2 R2, | 4 recomputed from A^{-1}, | 8 the R2 shift formed in double the working
    precision; shift -1 for a non-pole shift; K_nu of the
    first shift."""
    d, z = _f64(d), _f64(z)
    n = d.size
    ks = np.arange(n + 1) if ks is None else np.asarray(ks, dtype=np.int64)
    m = ks.size
    o = default_opts() if opts is None else opts
    out = dict(lam=np.empty(m), sigma=np.empty(m), mu=np.empty(m), shift=np.empty(m, dtype=np.int32),
               flags=np.empty(m, dtype=np.int32), K_nu=np.empty(m), Vt=np.empty((m, n + 1)))

    def run(idx):
        v = np.empty(n + 1)
        lam, sig, mu, K = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        sh, fl = ctypes.c_int(), ctypes.c_int()
        for p in idx:
            rc = lib().oracle_arroweig(n, _ptr(d), _ptr(z), float(alpha), int(ks[p]), ctypes.byref(o),
                                       ctypes.byref(lam), _ptr(v), ctypes.byref(sig), ctypes.byref(mu),
                                       ctypes.byref(sh), ctypes.byref(fl), ctypes.byref(K))
            if rc:
                _raise("oracle_arroweig", rc)
            out["lam"][p], out["sigma"][p], out["mu"][p], out["shift"][p] = lam.value, sig.value, mu.value, sh.value
            out["flags"][p], out["K_nu"][p] = fl.value, K.value
            out["Vt"][p] = v

    _split_run(run, m, threads)
    return out


def r2(d, z, rho_or_alpha, k, lam_est, arrow=False):
    """Remedy R2 alone from an estimate lam_est of eigenvalue k (0-based) of D + rho z z^T, or of
    the arrowhead [D z; z^T alpha] with arrow=True: dict(lam, sigma, mu, rounds)."""
    d, z = _f64(d), _f64(z)
    lam, sig, mu = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    fn = lib().oracle_arrow_r2 if arrow else lib().oracle_dpr1_r2
    rc = fn(d.size, _ptr(d), _ptr(z), float(rho_or_alpha), int(k), float(lam_est), ctypes.byref(lam),
            ctypes.byref(sig), ctypes.byref(mu))
    if rc < 0:
        raise ValueError("r2: bad arguments")
    return dict(lam=lam.value, sigma=sig.value, mu=mu.value, rounds=rc)


def quad_arrow_all(d, z, alpha, ks=None, threads=1):
    """binary128 reference for the arrowhead: dict(hi, lo, Vt), lambda_k = hi + lo."""
    d, z = _f64(d), _f64(z)
    n = d.size
    ks = np.arange(n + 1) if ks is None else np.asarray(ks, dtype=np.int64)
    m = ks.size
    out = dict(hi=np.empty(m), lo=np.empty(m), Vt=np.empty((m, n + 1)))

    def run(idx):
        v = np.empty(n + 1)
        hi, lo = ctypes.c_double(), ctypes.c_double()
        for p in idx:
            rc = lib().quad_arrow_eigpair(n, _ptr(d), _ptr(z), float(alpha), int(ks[p]), ctypes.byref(hi),
                                          ctypes.byref(lo), _ptr(v))
            if rc < 0:
                raise ValueError("quad_arrow_eigpair failed")
            out["hi"][p], out["lo"][p] = hi.value, lo.value
            out["Vt"][p] = v

    _split_run(run, m, threads)
    return out
