"""Data of any magnitude through the C ABI: the exact power-of-two normalisation (results scale
exactly with the data, bit for bit), and no silent failure -- every problem either meets
16 n 2^-53 against binary128 or the call reports DPR1_ERR_RANGE (an eigenpair that needs values
outside the binary64 range of the normalised problem)."""
import math

import numpy as np
import pytest

import oracle
from gpu_common import run_gpu, tol
from paper_1405_7537_gb300 import workloads as W
from test_oracle import _harsh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
RANGE = 8


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1405_7537_gb300 import binding
    binding.lib()
    return binding


@pytest.mark.parametrize("zf", [0, 1])
def test_scale_invariance_is_exact(B, zf):
    """d -> 2^s d, z -> 2^t z, rho -> 2^(s - 2t) rho: lambda, sigma, mu scale by 2^s and V is the
    same, bit for bit, including scales where the unnormalised data over- or underflow."""
    d, z, rho = W.hard(300, 4)
    base = run_gpu(B, d, z, rho, zero_finder=zf)
    for s, t in ((0, 300), (600, 0), (-600, 0), (900, 400), (-900, -400), (37, -11)):
        g = run_gpu(B, np.ldexp(d, s), np.ldexp(z, t), math.ldexp(rho, s - 2 * t), zero_finder=zf)
        assert np.array_equal(g["lam"], np.ldexp(base["lam"], s)), (s, t)
        assert np.array_equal(g["sigma"], np.ldexp(base["sigma"], s)), (s, t)
        assert np.array_equal(g["mu"], np.ldexp(base["mu"], s)), (s, t)
        assert np.array_equal(g["Vt"], base["Vt"]), (s, t)


def _status(B, d, z, rho, zf):
    try:
        return 0, run_gpu(B, d, z, rho, zero_finder=zf)
    except B.DPR1Error as ex:
        return ex.code, None


@pytest.mark.parametrize("zf", [0, 1])
def test_harsh_data_meets_the_bound_or_reports_range(B, zf):
    """The oracle's harsh generator (poles scaled by up to 2^700, weights over up to 2^150 and
    scaled by up to 2^300, rank-one part 2^-300 to 2^300 times the poles' scale): each call
    meets the bound against binary128 (components relative to max(|v|, 2^-1022)) or reports
    DPR1_ERR_RANGE; none fails silently."""
    rng = np.random.default_rng(3141 + zf)
    ok = 0
    seen = 0
    while seen < 80:
        d, z, rho = _harsh(rng)
        n = d.size
        if not (np.all(d[:-1] > d[1:]) and np.all(np.isfinite(d)) and not np.any(oracle.zero_weight(z))
                and rho > 0 and np.isfinite(rho)):
            continue
        seen += 1
        code, g = _status(B, d, z, rho, zf)
        if code == RANGE:
            continue
        assert code == 0, code
        q = oracle.quad_all(d, z, rho, threads=8)
        lq = q["hi"] + q["lo"]
        assert np.max(np.abs(g["lam"] - lq) / np.abs(lq)) <= tol(n), seen
        err = np.abs(g["Vt"] - q["Vt"]) / np.maximum(np.abs(q["Vt"]), 2.0 ** -1022)
        assert err.max() <= tol(n), (seen, float(err.max() / tol(n)))
        ok += 1
    assert ok >= 60


def test_out_of_range_pair_is_reported(B):
    """A weight of 1e-152 next to weights of 1 (above the zero-weight cut): lambda_0 - d_0 is
    below the normal binary64 range of the normalised problem; the call reports DPR1_ERR_RANGE
    instead of a vector without precision."""
    d = np.array([2.0e-3, 3.0e-4, 2.0e-12])
    z = np.array([1e-152, 1.0, -0.5])
    for zf in (0, 1):
        code, _ = _status(B, d, z, 4e-10, zf)
        assert code == RANGE


def test_batched_harsh_problems_equal_single_calls(B):
    """A batch of harsh problems (all in range, each with its own normalisation) gives each
    problem's single-call results."""
    rng = np.random.default_rng(99)
    probs = []
    while len(probs) < 24:
        d, z, rho = _harsh(rng, wmax=60)
        if not (np.all(d[:-1] > d[1:]) and np.all(np.isfinite(d)) and not np.any(oracle.zero_weight(z))
                and rho > 0 and np.isfinite(rho)):
            continue
        code, g = _status(B, d, z, rho, 0)
        if code == 0:
            probs.append((d, z, rho, g))
    bt = B.Batch([p[0].size for p in probs])
    bt.solve(torch.tensor(np.concatenate([p[0] for p in probs]), device="cuda"),
             torch.tensor(np.concatenate([p[1] for p in probs]), device="cuda"),
             torch.tensor(np.array([p[2] for p in probs]), device="cuda"), check=True)
    torch.cuda.synchronize()
    for i, (d, z, rho, g) in enumerate(probs):
        lam, Vt = (x.cpu().numpy() for x in bt.block(i)[:2])
        n = d.size
        # the launch shapes differ (lane groups sum in another order), so within the bound
        assert np.max(np.abs(lam - g["lam"]) / np.abs(g["lam"])) <= tol(n), i
        assert np.max(np.abs(Vt - g["Vt"]) / np.maximum(np.abs(g["Vt"]), 2.0 ** -1022)) <= tol(n), i


def test_arrowhead_scale_invariance_is_exact(B):
    """The arrowhead scales as a whole: A -> 2^s A gives 2^s lambda and the same V, bit for bit."""
    d, z, alpha = W.arrowhead(200, 3)
    cu = lambda a: torch.tensor(np.array(a, copy=True), device="cuda")
    base = B.eig_arrowhead(cu(d), cu(z), alpha)
    lam0, V0 = base["lam"].cpu().numpy(), base["Vt"].cpu().numpy()
    for s in (700, -700, 300, -13):
        r = B.eig_arrowhead(cu(np.ldexp(d, s)), cu(np.ldexp(z, s)), math.ldexp(alpha, s))
        assert np.array_equal(r["lam"].cpu().numpy(), np.ldexp(lam0, s)), s
        assert np.array_equal(r["Vt"].cpu().numpy(), V0), s


def test_harsh_arrowheads(B):
    """Arrowheads of any magnitude (the oracle's harsh generator): each call meets the bound
    against binary128 or reports DPR1_ERR_RANGE."""
    from test_oracle_arrow import _harsh_arrow
    rng = np.random.default_rng(707)
    cu = lambda a: torch.tensor(np.array(a, copy=True), device="cuda")
    ok = seen = 0
    while seen < 60:
        d, z, alpha = _harsh_arrow(rng)
        n = d.size
        if not (np.all(d[:-1] > d[1:]) and np.all(np.isfinite(d)) and np.isfinite(alpha) and not np.any(z == 0)):
            continue
        seen += 1
        for zf in (0, 1):
            try:
                r = B.eig_arrowhead(cu(d), cu(z), alpha, options=B.default_options(zero_finder=zf))
            except B.DPR1Error as ex:
                assert ex.code in (RANGE, 1), ex.code      # 1: a weight below the zero-weight cut
                continue
            q = oracle.quad_arrow_all(d, z, alpha, threads=8)
            lq = q["hi"] + q["lo"]
            t = 16 * (n + 1) * 2.0 ** -53
            lam, Vt = r["lam"].cpu().numpy(), r["Vt"].cpu().numpy()
            assert np.max(np.abs(lam - lq) / np.abs(lq)) <= t, (seen, zf)
            assert np.max(np.abs(Vt - q["Vt"]) / np.maximum(np.abs(q["Vt"]), 2.0 ** -1022)) <= t, (seen, zf)
            ok += 1
    assert ok >= 80


def test_backward_scale_invariance_is_exact(B):
    """The backward is normalised like the forward.  With d -> 2^s d, z -> 2^t z and
    rho -> 2^(s - 2t) rho, lambda scales by 2^s and V is unchanged, so a loss on lambda alone
    gives gradients scaled by (1, 2^(s - t), 2^(2t)) for (d, z, rho), and a loss on V alone by
    (2^-s, 2^-t, 2^(2t - s)) -- bit for bit, also where the unnormalised data over- or underflow."""
    d, z, rho = W.uniform(200, 5)
    rng = np.random.default_rng(5)
    gl = torch.tensor(rng.standard_normal(d.size), device="cuda")
    gV = torch.tensor(rng.standard_normal((d.size, d.size)), device="cuda")

    def grads(dd, zz, rr, lam_part):
        dt, zt = torch.tensor(dd, device="cuda"), torch.tensor(zz, device="cuda")
        r = B.eig(dt, zt, rr)
        g = B.eig_backward(dt, zt, rr, r["sigma"], r["mu"], gl if lam_part else None, None if lam_part else gV)
        torch.cuda.synchronize()
        return [g[0].cpu().numpy(), g[1].cpu().numpy(), float(g[2])]

    base = {lp: grads(d, z, rho, lp) for lp in (True, False)}
    for s, t in ((600, 0), (-600, 0), (0, 300), (300, -300), (-37, 11)):
        ds, zs, rs = np.ldexp(d, s), np.ldexp(z, t), math.ldexp(rho, s - 2 * t)
        a = grads(ds, zs, rs, True)
        b0 = base[True]
        assert np.array_equal(a[0], b0[0]), (s, t)
        assert np.array_equal(a[1], np.ldexp(b0[1], s - t)), (s, t)
        assert a[2] == math.ldexp(b0[2], 2 * t), (s, t)
        v = grads(ds, zs, rs, False)
        b1 = base[False]
        assert np.array_equal(v[0], np.ldexp(b1[0], -s)), (s, t)
        assert np.array_equal(v[1], np.ldexp(b1[1], -t)), (s, t)
        assert v[2] == math.ldexp(b1[2], 2 * t - s), (s, t)


def test_tridiagonal_scale_invariance_is_exact(B):
    """Divide and conquer scales with the matrix: every step (the tear, the deflation tolerance
    relative to ||T||, the normalised DPR1 merges, the products of the eigenvector blocks) is
    homogeneous, so T -> 2^s T gives 2^s lambda and the same Q, bit for bit."""
    rng = np.random.default_rng(12)
    a, b = rng.uniform(-1, 1, 700), rng.uniform(-1, 1, 699)
    cu = lambda x: torch.tensor(np.array(x, copy=True), device="cuda")
    lam0, Q0 = (x.cpu().numpy() for x in B.eigh_tridiagonal(cu(a), cu(b)))
    for s in (640, -640, 17):
        lam, Q = (x.cpu().numpy() for x in B.eigh_tridiagonal(cu(np.ldexp(a, s)), cu(np.ldexp(b, s))))
        assert np.array_equal(lam, np.ldexp(lam0, s)), s
        assert np.array_equal(Q, Q0), s


def test_hermitian_scale_invariance_is_exact(B):
    """The Hermitian reduction scales too: z -> 2^t z (its modulus is a fixed sequence of
    correctly rounded operations with a power-of-two scaling) and d -> 2^s d, rho -> 2^(s-2t) rho
    give 2^s lambda and the same complex V."""
    d, z, rho = W.hermitian(150, 3, base="uniform")
    cu = lambda x: torch.tensor(np.array(x, copy=True), device="cuda")
    base = B.eig_hermitian(cu(d), cu(z), rho)
    lam0, V0 = base["lam"].cpu().numpy(), base["Vt"].cpu().numpy()
    for s, t in ((500, -200), (-500, -200), (600, 320)):      # rho * 2^(s - 2t) stays normal
        zs = np.ldexp(z.real, t) + 1j * np.ldexp(z.imag, t)
        r = B.eig_hermitian(cu(np.ldexp(d, s)), cu(zs), math.ldexp(rho, s - 2 * t))
        assert np.array_equal(r["lam"].cpu().numpy(), np.ldexp(lam0, s)), (s, t)
        assert np.array_equal(r["Vt"].cpu().numpy(), V0), (s, t)
