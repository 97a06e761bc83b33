"""dpr1_eig_batched (through the C ABI): many uneven problems in one launch sequence, checked
per problem against dpr1_eig and the CPU oracle, at the 4096-problem workload on sampled
problems, under CUDA-graph capture, and for its argument errors."""
import numpy as np
import pytest

import oracle
from gpu_common import tol
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


def cu(a, dtype=torch.float64):
    return torch.tensor(np.array(a), dtype=dtype, device="cuda")


def make_batch(problems):
    sizes = [p[0].size for p in problems]
    d = np.concatenate([p[0] for p in problems]) if problems else np.zeros(0)
    z = np.concatenate([p[1] for p in problems]) if problems else np.zeros(0)
    rho = np.array([p[2] for p in problems])
    return sizes, d, z, rho


def rel(a, b):
    return np.abs(a - b) / np.maximum(np.abs(b), 1e-300)


def test_mixed_batch_matches_single_calls(B):
    probs = [W.uniform(1, 1), W.uniform(2, 2), W.uniform(3, 3), W.hard(17, 4), W.uniform(64, 5),
             (np.zeros(0), np.zeros(0), 1.0), W.hard(200, 6), W.uniform(33, 7)]
    dz, zz, _ = W.uniform(9, 8)
    probs.append((dz, zz, 0.0))                                      # rho = 0: lambda = d, V = I
    dd_ = np.array([3.0, 2.0, 2.0, 1.0, 0.5]); zd = np.array([1.0, 0.5, 0.7, 0.0, 1.0])
    probs.append((dd_, zd, 0.8))                                     # deflation: tie and zero weight
    sizes, d, z, rho = make_batch(probs)
    bt = B.Batch(sizes)
    for lanes in (0, 8, 16, 32):
        bt.solve(cu(d), cu(z), cu(rho), options=B.default_options(lanes=lanes), check=True)
        torch.cuda.synchronize()
        for p, (dp, zp, rp) in enumerate(probs):
            n = dp.size
            if n == 0:
                continue
            lam, Vt = bt.block(p)
            ref = B.eig(cu(dp), cu(zp), rp)
            assert np.max(rel(lam.cpu().numpy(), ref["lam"].cpu().numpy())) <= tol(n)
            V1, V0 = Vt.cpu().numpy(), ref["Vt"].cpu().numpy()
            if rp > 0 and np.all(zp != 0) and np.all(np.diff(dp) < 0):
                assert np.max(rel(V1, V0)) <= tol(n), p
            else:
                # deflated / trivial problems: eigenvectors of repeated eigenvalues are a basis choice
                A = np.diag(dp) + rp * np.outer(zp, zp)
                Vc = V1.T
                assert np.max(np.abs(Vc.T @ Vc - np.eye(n))) < 1e-14
                assert np.max(np.abs(A @ Vc - Vc * lam.cpu().numpy())) < 1e-14


def test_small_batch_workload_against_oracle(B):
    offs, d, z, rho = W.batch(P=48, seed=3, nmin=16, nmax=400)
    sizes = np.diff(offs)
    bt = B.Batch(sizes)
    bt.solve(cu(d), cu(z), cu(rho), check=True)
    torch.cuda.synchronize()
    for p in range(bt.P):
        a, b = offs[p], offs[p + 1]
        n = b - a
        r = oracle.eig_all(d[a:b], z[a:b], rho[p], threads=8)
        lam, Vt = bt.block(p)
        assert np.max(rel(lam.cpu().numpy(), r["lam"])) <= tol(n), p
        assert np.max(rel(Vt.cpu().numpy(), r["Vt"])) <= tol(n), p


def test_batch_4096_sampled(B):
    """The 4096-problem workload as benchmarked: every problem's trace, sampled problems in
    full against the oracle, orthogonality of sampled blocks."""
    offs, d, z, rho = W.batch()
    sizes = np.diff(offs)
    bt = B.Batch(sizes)
    bt.solve(cu(d), cu(z), cu(rho), check=True)
    torch.cuda.synchronize()
    lam_all = bt.lam.cpu().numpy()
    sig_all = bt.sigma.cpu().numpy()
    mu_all = bt.mu.cpu().numpy()
    import math
    for p in range(bt.P):
        a, b = offs[p], offs[p + 1]
        tr = math.fsum(list(d[a:b]) + list(rho[p] * z[a:b] ** 2))
        sl = math.fsum(list(sig_all[a:b]) + list(mu_all[a:b]))
        assert abs(sl - tr) <= 4 * (b - a) * 2.0 ** -52 * np.sum(np.abs(lam_all[a:b])), p
    rng = np.random.default_rng(0)
    for p in rng.choice(bt.P, 12, replace=False):
        a, b = offs[p], offs[p + 1]
        n = b - a
        r = oracle.eig_all(d[a:b], z[a:b], rho[p], threads=16)
        lam, Vt = bt.block(p)
        assert np.max(rel(lam.cpu().numpy(), r["lam"])) <= tol(n), p
        assert np.max(rel(Vt.cpu().numpy(), r["Vt"])) <= tol(n), p
        G = Vt @ Vt.T - torch.eye(n, dtype=torch.float64, device="cuda")
        assert G.abs().max().item() <= n * 2.0 ** -52


def test_graph_capture_replay(B):
    offs, d, z, rho = W.batch(P=200, seed=11, nmin=16, nmax=300)
    sizes = np.diff(offs)
    bt = B.Batch(sizes)
    dt, zt, rt = cu(d), cu(z), cu(rho)
    bt.solve(dt, zt, rt)
    torch.cuda.synchronize()
    lam0, Vt0 = bt.lam.clone(), bt.Vt.clone()
    bt.lam.zero_(); bt.Vt.zero_()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        bt.solve(dt, zt, rt)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    with torch.cuda.graph(g):
        bt.solve(dt, zt, rt)
    bt.lam.zero_(); bt.Vt.zero_()
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    assert torch.equal(bt.lam, lam0) and torch.equal(bt.Vt, Vt0)
    assert B.stream_status(bt.ws) == 0


def test_batch_argument_errors(B):
    sizes = [5, 7]
    bt = B.Batch(sizes)
    d = np.concatenate([W.uniform(5, 1)[0], W.uniform(7, 2)[0]])
    z = np.concatenate([W.uniform(5, 1)[1], W.uniform(7, 2)[1]])
    with pytest.raises(B.DPR1Error) as e:
        bt.solve(cu(d), cu(z), cu([1.0, -2.0]), check=True)
    assert e.value.code == 3
    bt.offs.copy_(torch.tensor([0, 13, 12], device="cuda"))          # decreasing offsets
    with pytest.raises(B.DPR1Error) as e:
        bt.solve(cu(d), cu(z), cu([1.0, 2.0]), check=True)
    assert e.value.code == 1


def test_autotuner_per_zero_finder(B, tmp_path, monkeypatch):
    """The tuner times every candidate shape on a sample of the size mix, caches the winner
    under a key of the size histogram, the GPU and the zero finder, and the tuned options
    solve the batch to the same results as the default shape."""
    from paper_1405_7537_gb300 import tune
    monkeypatch.setattr(tune, "CACHE", str(tmp_path / "tune_cache.json"))
    offs, d, z, rho = W.batch(P=64, seed=4, nmin=16, nmax=300)
    sizes = np.diff(offs)
    shapes = {}
    for zf in (0, 1):
        shapes[zf] = tune.tune(sizes, max_total=20_000, reps=1, zero_finder=zf)
        assert shapes[zf] in tune.CANDIDATES
        assert tune.tune(sizes, zero_finder=zf) == shapes[zf]          # cached
    import json
    keys = list(json.load(open(tune.CACHE)).keys())
    assert len(keys) == 2 and any("|zf0|" in k for k in keys) and any("|zf1|" in k for k in keys)
    bt = B.Batch(sizes)
    dt, zt, rt = cu(d), cu(z), cu(rho)
    bt.solve(dt, zt, rt, options=tune.options_for(sizes, zero_finder=1), check=True)
    lam1 = bt.lam.clone()
    bt.solve(dt, zt, rt, check=True)
    assert torch.max(torch.abs(lam1 - bt.lam) / torch.abs(bt.lam)).item() <= tol(int(sizes.max()))


@pytest.mark.parametrize("lanes", [0, 8, 32])
def test_every_pair_written_once(B, lanes):
    """Every (problem, k) of a batch is solved exactly once and every output slot is written: the
    outputs start as NaN, the work counter's solved count equals the number of eigenpairs (each
    index leaves the queue once), and for every problem (not a sample) each row of V is a unit
    vector, the eigenvalues keep the order of the poles (strict interlacing on the pairs), and
    their sum is the trace sum(d) + rho ||z||^2."""
    offs, d, z, rho = W.batch(P=384, seed=31, nmin=1, nmax=400)
    sizes = np.diff(offs)
    bt = B.Batch(sizes)
    for t in (bt.lam, bt.sigma, bt.mu, bt.xnorm, bt.Vt):
        t.fill_(float("nan"))
    bt.solve(cu(d), cu(z), cu(rho), options=B.default_options(lanes=lanes), check=True)
    torch.cuda.synchronize()
    st = B.workspace_stats(bt.ws)
    assert st["solved"] + st["deflated"] == bt.total, st
    lam, sig, mu, Vt = (t.cpu().numpy() for t in (bt.lam, bt.sigma, bt.mu, bt.Vt))
    assert np.all(np.isfinite(lam)) and np.all(np.isfinite(sig)) and np.all(np.isfinite(mu))
    assert np.all(np.isfinite(Vt))
    for p in range(bt.P):
        a, b = int(offs[p]), int(offs[p + 1])
        n = b - a
        if n == 0:
            continue
        dp, zp, rp = d[a:b], z[a:b], float(rho[p])
        V = Vt[int(bt.voffs_host[p]):int(bt.voffs_host[p]) + n * n].reshape(n, n)
        assert np.max(np.abs(np.sum(V * V, axis=1) - 1.0)) <= 1e-13 * max(n, 8), p
        lp = lam[a:b]
        assert np.all(lp[:-1] >= lp[1:]), p                  # decreasing, with the poles
        assert np.all(lp >= dp) and np.all(lp[1:] <= dp[:-1]), p
        scale = np.sum(np.abs(dp)) + rp * np.sum(zp * zp)
        assert abs(np.sum(lp) - (np.sum(dp) + rp * np.sum(zp * zp))) <= 64 * n * 2.0 ** -53 * scale, p
