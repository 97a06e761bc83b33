"""Helpers for the GPU parity tests: error measures against the oracle and the binary128 reference."""
import math

import numpy as np

U53 = 2.0 ** -53


def tol(n):
    """The bound every eigenvalue and eigenvector component must meet: 16 n 2^-53 relative."""
    return 16 * max(n, 1) * U53


def two_sum(a, b):
    s = a + b
    bb = s - a
    return s, (a - (s - bb)) + (b - bb)


def pair_minus_ref(s, m, hi, lo):
    """(s + m) - (hi + lo) evaluated with error-free transformations (vectorised), relative to hi."""
    a, ea = two_sum(s, -hi)
    b, eb = two_sum(a, m)
    diff = b + (ea + eb - lo)
    return np.abs(diff) / np.abs(hi + lo)


def lam_minus_ref(x, hi, lo):
    a, ea = two_sum(x, -hi)
    return np.abs(a + (ea - lo)) / np.abs(hi + lo)


def vec_rel(V, Vref):
    return np.abs(V - Vref) / np.maximum(np.abs(Vref), 1e-300)


def eig_errors(gpu, ref_kind, ref, ks=None):
    """Max relative errors of the GPU results on rows ks against the oracle ('oracle') or
    binary128 ('quad') results computed on the same rows."""
    ks = np.arange(gpu["lam"].shape[0]) if ks is None else np.asarray(ks)
    lam = gpu["lam"][ks]
    sig = gpu["sigma"][ks]
    mu = gpu["mu"][ks]
    V = gpu["Vt"][ks] if gpu.get("Vt") is not None else None
    if ref_kind == "quad":
        e_lam = lam_minus_ref(lam, ref["hi"], ref["lo"])
        e_pair = pair_minus_ref(sig, mu, ref["hi"], ref["lo"])
        e_vec = vec_rel(V, ref["Vt"]).max(axis=1) if V is not None else np.zeros(len(ks))
    else:
        # the oracle's (sigma, mu) and lambda in binary64; compare pairs exactly through two_sum
        rs, rm = ref["sigma"], ref["mu"]
        hi, lo = two_sum(rs, rm)
        e_pair = pair_minus_ref(sig, mu, hi, lo)
        e_lam = np.abs(lam - ref["lam"]) / np.abs(ref["lam"])
        e_vec = vec_rel(V, ref["Vt"]).max(axis=1) if V is not None else np.zeros(len(ks))
    return e_lam, e_pair, e_vec


def zero_path_mask(gpu, d):
    """Rows whose lambda was recomputed from A^{-1} (lambda differs from sigma + mu)."""
    return gpu["lam"] != (gpu["sigma"] + gpu["mu"])


def strict_interlacing_ok(sig, mu, d):
    """lambda_k = sigma_k + mu_k lies in (d_k, d_{k-1}), decided exactly with two_sum."""
    n = d.size
    a, ea = two_sum(sig, -d)
    up = a + (ea + mu)
    okl = up > 0
    ok = okl.copy()
    b, eb = two_sum(sig[1:], -d[:-1])
    dn = b + (eb + mu[1:])
    ok[1:] &= dn < 0
    return bool(ok.all())


def trace_defect(sig, mu, d, z, rho):
    """|sum lambda - trace(A)| / sum |lambda| with compensated sums."""
    tr = math.fsum(list(d) + list(rho * z * z))
    sl = math.fsum(list(sig) + list(mu))
    return abs(sl - tr) / math.fsum(list(np.abs(sig + mu)))
