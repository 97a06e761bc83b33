"""The accelerated bracketed solve (dpr1_options.zero_finder = 1, a fast zero finder in place
of bisection, Sec. 2.2) through the C ABI: the same parity bar as bisection against the
oracle and the binary128 reference, agreement with bisection, and far fewer evaluations of
the secular function."""
import numpy as np
import pytest

from gpu_common import check_full, run_gpu, sampled, tol, two_sum
from paper_1405_7537_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ACCEL = 1


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1405_7537_gb300 import binding
    binding.lib()
    assert binding.ACCELERATED == ACCEL
    return binding


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (3, 2), (5, 3), (17, 4), (33, 6), (100, 7)])
def test_ragged_small_sizes(B, n, seed):
    d, z, rho = W.uniform(n, seed)
    check_full(B, d, z, rho, zero_finder=ACCEL)


@pytest.mark.parametrize("lanes", [8, 16, 32])
def test_lane_groups(B, lanes):
    d, z, rho = W.hard(200, 11)
    check_full(B, d, z, rho, lanes=lanes, zero_finder=ACCEL)


def test_paper_examples(B):
    for d, z, rho in (W.example1(), W.example2(), W.example3(), W.example4(1e-3), W.example4(1e-8),
                      W.example4(1e-15)):
        check_full(B, d, z, rho, zero_finder=ACCEL)


@pytest.mark.parametrize("gen,n,seed", [("uniform", 512, 0), ("hard", 512, 1), ("hard", 1000, 9),
                                        ("large", 700, 4)])
def test_workload_families(B, gen, n, seed):
    if gen == "large":
        d, z, rho, _ = W.large(n, seed, with_W=False)
    else:
        d, z, rho = getattr(W, gen)(n, seed)
    check_full(B, d, z, rho, zero_finder=ACCEL)


def test_hard_16384_sampled(B):
    d, z, rho = W.hard(16384, 1)
    sampled(B, d, z, rho, zero_finder=ACCEL)


def _pairs_agree(a, b):
    """Rows whose (sigma, mu) pairs are bit-identical, and the max relative pair difference."""
    same = (a["sigma"] == b["sigma"]) & (a["mu"] == b["mu"])
    hi, lo = two_sum(b["sigma"], b["mu"])
    x, ex = two_sum(a["sigma"], -hi)
    y, ey = two_sum(x, a["mu"])
    diff = np.abs(y + (ex + ey - lo)) / np.abs(hi + lo)
    return same, diff


def test_agrees_with_bisection_and_saves_evaluations(B):
    """Both solvers stop at the adjacent pair of doubles across the sign change, so the pairs
    agree bit for bit except where the computed sign is not monotone within a few ulps (the two
    solvers group the secular sum differently: two terms over one reciprocal in bisection, one
    term with its slope in the accelerated solve, so |g| within rounding of zero at the final
    pair can pick the neighbouring double); the accelerated solve needs a fraction of the
    evaluations."""
    d, z, rho = W.hard(4096, 1)
    n = d.size
    dt, zt = torch.tensor(d, device="cuda"), torch.tensor(z, device="cuda")
    res, stats = {}, {}
    for zf in (0, ACCEL):
        ws = B.workspace(n)
        r = B.eig(dt, zt, rho, options=B.default_options(zero_finder=zf), ws=ws)
        torch.cuda.synchronize()
        res[zf] = {k: v.cpu().numpy() for k, v in r.items() if v is not None}
        stats[zf] = B.workspace_stats(ws)
    same, diff = _pairs_agree(res[ACCEL], res[0])
    assert same.mean() >= 0.97, same.mean()
    assert diff.max() <= tol(n), diff.max()
    assert np.max(np.abs(res[ACCEL]["Vt"] - res[0]["Vt"]) / np.maximum(np.abs(res[0]["Vt"]), 1e-300)) <= tol(n)
    assert stats[ACCEL]["solved"] == stats[0]["solved"] == n
    assert stats[ACCEL]["evals_solve"] <= 0.4 * stats[0]["evals_solve"], (stats[ACCEL], stats[0])


def test_batched(B):
    offs, d, z, rho = W.batch(P=64, seed=3, nmin=16, nmax=400)
    sizes = np.diff(offs)
    bt = B.Batch(sizes)
    dt, zt, rt = (torch.tensor(a, device="cuda") for a in (d, z, rho))
    bt.solve(dt, zt, rt, options=B.default_options(zero_finder=ACCEL), check=True)
    torch.cuda.synchronize()
    lam1, Vt1 = bt.lam.clone(), bt.Vt.clone()
    bt.solve(dt, zt, rt, check=True)
    torch.cuda.synchronize()
    for p in range(bt.P):
        a, b = offs[p], offs[p + 1]
        n = b - a
        l0 = bt.lam[a:b].cpu().numpy()
        assert np.max(np.abs(lam1[a:b].cpu().numpy() - l0) / np.abs(l0)) <= tol(n), p
        v0 = bt.block(p)[1].cpu().numpy()
        v1 = Vt1[bt.voffs_host[p]:bt.voffs_host[p] + n * n].view(n, n).cpu().numpy()
        assert np.max(np.abs(v1 - v0) / np.maximum(np.abs(v0), 1e-300)) <= tol(n), p


def test_deflated_and_edge_inputs(B):
    d = np.array([3.0, 2.0, 2.0, 2.0, 1.0, 0.5, -1.0, -1.0])
    z = np.array([1.0, 0.5, 0.7, -0.2, 0.0, 1.0, 0.3, 0.0])
    g0 = run_gpu(B, d, z, 0.8)
    g1 = run_gpu(B, d, z, 0.8, zero_finder=ACCEL)
    assert np.max(np.abs(g1["lam"] - g0["lam"]) / np.abs(g0["lam"])) <= tol(d.size)
    # poles that straddle zero: the near-zero recompute runs the non-pole solve at sigma = 0
    d2 = np.array([2.0, 1e-9, -1e-9, -3.0])
    z2 = np.array([1e-3, 1.0, 1.0, 1e-3])
    check_full(B, d2, z2, 1e-12, zero_finder=ACCEL)
