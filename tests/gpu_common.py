"""Helpers for the GPU parity tests: error measures against the oracle and the binary128 reference."""
import math

import numpy as np

import oracle

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


def run_gpu(B, d, z, rho, **opt):
    import torch
    o = B.default_options(**opt) if opt else None
    r = B.eig(torch.tensor(np.array(d), device="cuda"), torch.tensor(np.array(z), device="cuda"), rho, options=o)
    torch.cuda.synchronize()
    return {k: (v.cpu().numpy() if v is not None else None) for k, v in r.items()}


def check_full(B, d, z, rho, threads=16, **opt):
    """All rows against the oracle and binary128 (sizes the oracle finishes in seconds)."""
    n = d.size
    g = run_gpu(B, d, z, rho, **opt)
    q = oracle.quad_all(d, z, rho, threads=threads)
    r = oracle.eig_all(d, z, rho, threads=threads)
    el, ep, ev = eig_errors(g, "quad", q)
    # rows recomputed from A^{-1}: lambda is accurate, sigma + mu need not be
    zp = g["lam"] != g["sigma"] + g["mu"]
    ep = np.where(zp, 0.0, ep)
    assert el.max() <= tol(n), ("lambda vs quad", el.max(), tol(n), int(el.argmax()))
    assert ep.max() <= tol(n), ("pair vs quad", ep.max(), tol(n), int(ep.argmax()))
    assert ev.max() <= tol(n), ("vector vs quad", ev.max(), tol(n), int(ev.argmax()))
    ol, op, ov = eig_errors(g, "oracle", r)
    assert ol.max() <= tol(n), ("lambda vs oracle", ol.max())
    assert ov.max() <= tol(n), ("vector vs oracle", ov.max())
    assert strict_interlacing_ok(np.where(zp, g["lam"], g["sigma"]), np.where(zp, 0.0, g["mu"]), d)
    return g, r


def sampled(B, d, z, rho, nsample_oracle=48, nsample_quad=12, seed=0, **opt):
    """Sampled rows against the oracle and binary128, and whole-spectrum properties (full sizes)."""
    import torch
    n = d.size
    g = run_gpu(B, d, z, rho, **opt)
    rng = np.random.default_rng(seed)
    ks = np.unique(np.concatenate([[0, 1, n // 2, n - 2, n - 1], rng.choice(n, nsample_oracle, replace=False)]))
    r = oracle.eig_all(d, z, rho, ks=ks, threads=16)
    ol, op, ov = eig_errors(g, "oracle", r, ks)
    assert ol.max() <= tol(n) and ov.max() <= tol(n), (ol.max(), ov.max(), tol(n))
    kq = ks[:: max(1, ks.size // nsample_quad)]
    q = oracle.quad_all(d, z, rho, ks=kq, threads=16)
    ql, qp, qv = eig_errors(g, "quad", q, kq)
    assert ql.max() <= tol(n) and qv.max() <= tol(n), (ql.max(), qv.max(), tol(n))
    # properties at full size
    zp = g["lam"] != g["sigma"] + g["mu"]
    assert strict_interlacing_ok(np.where(zp, g["lam"], g["sigma"]), np.where(zp, 0.0, g["mu"]), d)
    assert trace_defect(g["sigma"], g["mu"], d, z, rho) <= 4 * n * 2.0 ** -52
    Vt = torch.tensor(g["Vt"], device="cuda")
    idx = torch.tensor(rng.choice(n, 256, replace=False), device="cuda")
    blk = Vt[idx] @ Vt[idx].T - torch.eye(256, dtype=torch.float64, device="cuda")
    assert blk.abs().max().item() <= n * 2.0 ** -52
    nrm = torch.linalg.vector_norm(Vt, dim=1)
    assert (nrm - 1).abs().max().item() <= 64 * 2.0 ** -52
    return g
