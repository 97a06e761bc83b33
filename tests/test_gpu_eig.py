"""GPU parity of dpr1_eig (through the C ABI) against the CPU oracle and the binary128 reference.

Bound (BASELINE the benchmark spec): every eigenvalue and every eigenvector component within
relative 16 n 2^-53 of the binary128 reference, and of the oracle.
"""
import numpy as np
import pytest

import oracle
from gpu_common import (eig_errors, strict_interlacing_ok, tol, trace_defect, two_sum, vec_rel,
                        lam_minus_ref, pair_minus_ref)
from paper_1405_7537_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1405_7537_gb300 import binding
    binding.lib()
    return binding


def run_gpu(B, d, z, rho, **opt):
    o = B.default_options(**opt) if opt else None
    r = B.eig(torch.tensor(np.array(d), device="cuda"), torch.tensor(np.array(z), device="cuda"), rho, options=o)
    torch.cuda.synchronize()
    return {k: (v.cpu().numpy() if v is not None else None) for k, v in r.items()}


def check_full(B, d, z, rho, threads=16, **opt):
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


def test_reciprocal_within_one_ulp(B):
    rng = np.random.default_rng(0)
    m = rng.uniform(1, 2, 1 << 20)
    e = rng.integers(-1000, 1000, m.size)
    x = np.ldexp(m, e) * rng.choice([-1.0, 1.0], m.size)
    r = B.probe_reciprocal(torch.tensor(x, device="cuda")).cpu().numpy()
    exact = 1.0 / x
    ulps = np.abs(r - exact) / np.spacing(np.abs(exact))
    assert ulps.max() <= 1.0


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (3, 2), (5, 3), (17, 4), (31, 5), (33, 6), (100, 7)])
def test_ragged_small_sizes(B, n, seed):
    d, z, rho = W.uniform(n, seed)
    check_full(B, d, z, rho)


@pytest.mark.parametrize("lanes", [8, 16, 32])
def test_lane_groups(B, lanes):
    d, z, rho = W.hard(200, 11)
    check_full(B, d, z, rho, lanes=lanes)


def test_paper_example1(B):
    d, z, rho = W.example1()
    g, _ = check_full(B, d, z, rho)
    assert abs(g["lam"][3] - 9.999999998999999e-25) <= 1e-15 * 1e-24


def test_paper_example2_pairs(B):
    mp = pytest.importorskip("mpmath").mp
    d, z, rho = W.example2()
    g, _ = check_full(B, d, z, rho)


def test_paper_example3_and_4(B):
    for d, z, rho in (W.example3(), W.example4(1e-3), W.example4(1e-8), W.example4(1e-15)):
        check_full(B, d, z, rho)


@pytest.mark.parametrize("gen,n,seed", [("uniform", 512, 0), ("hard", 512, 1), ("hard", 1000, 9),
                                        ("large", 700, 4)])
def test_workload_families(B, gen, n, seed):
    if gen == "large":
        d, z, rho, _ = W.large(n, seed, with_W=False)
    else:
        d, z, rho = getattr(W, gen)(n, seed)
    check_full(B, d, z, rho)


def test_uniform_512_full_config(B):
    """The n = 512 workload exactly as benchmarked: all pairs vs oracle and binary128."""
    d, z, rho = W.uniform(512, 0)
    check_full(B, d, z, rho)


def _sampled(B, d, z, rho, nsample_oracle=48, nsample_quad=12, seed=0):
    n = d.size
    g = run_gpu(B, d, z, rho)
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


def test_hard_16384_sampled(B):
    """The n = 16384 hard-spectrum workload as benchmarked, sampled against the oracle."""
    d, z, rho = W.hard(16384, 1)
    _sampled(B, d, z, rho)


def test_large_32768_sampled(B):
    d, z, rho, _ = W.large(32768, 4, with_W=False)
    _sampled(B, d, z, rho, nsample_oracle=24, nsample_quad=6)


def test_edge_cases(B):
    # n = 0
    out = B.eig(torch.empty(0, dtype=torch.float64, device="cuda"), torch.empty(0, dtype=torch.float64,
                                                                                 device="cuda"), 1.0)
    assert out["lam"].numel() == 0
    # rho = 0: lambda = d, V = I
    d, z, _ = W.uniform(9, 1)
    g = run_gpu(B, d, z, 0.0)
    assert np.array_equal(g["lam"], d) and np.array_equal(g["Vt"], np.eye(9))
    # rho < 0 is rejected on the host
    with pytest.raises(B.DPR1Error) as e:
        run_gpu(B, d, z, -1.0)
    assert e.value.code == 3
    # unsorted / non-finite are detected on the device
    with pytest.raises(B.DPR1Error) as e:
        run_gpu(B, d[::-1].copy(), z, 1.0)
    assert e.value.code == 2
    zb = z.copy(); zb[3] = np.nan
    with pytest.raises(B.DPR1Error) as e:
        run_gpu(B, d, zb, 1.0)
    assert e.value.code == 4


def test_deflation(B):
    d = np.array([3.0, 2.0, 2.0, 2.0, 1.0, 0.5, -1.0, -1.0])
    z = np.array([1.0, 0.5, 0.7, -0.2, 0.0, 1.0, 0.3, 0.0])
    for rho in (0.8, 2.5):
        g = run_gpu(B, d, z, rho)
        r = oracle.eig_full(d, z, rho)
        n = d.size
        assert np.max(np.abs(g["lam"] - r["lam"]) / np.abs(r["lam"])) <= tol(n)
        A = np.diag(d) + rho * np.outer(z, z)
        V = g["Vt"].T
        assert np.max(np.abs(V.T @ V - np.eye(n))) < 1e-14
        assert np.max(np.abs(A @ V - V * g["lam"])) < 1e-14
        # eigenvectors of simple eigenvalues are unique up to sign: compare them
        simple = [k for k in range(n) if np.sum(r["lam"] == r["lam"][k]) == 1]
        for k in simple:
            s = np.sign(np.dot(g["Vt"][k], r["Vt"][k]))
            assert np.max(np.abs(s * g["Vt"][k] - r["Vt"][k])) <= 1e-14
