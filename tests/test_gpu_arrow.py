"""dpr1_arrow_eig (real symmetric arrowhead [D z; z^T alpha]) through the C ABI against the
oracle's arrowhead solver and the binary128 reference: every eigenvalue and every eigenvector
component within relative 16 (n+1) 2^-53, for both zero finders."""
import numpy as np
import pytest

import oracle
from paper_1405_7537_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
EPS = 2.0 ** -53


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1405_7537_gb300 import binding
    binding.lib()
    return binding


def cu(x):
    return torch.tensor(np.array(x, dtype=np.float64, copy=True, order="C"), device="cuda")


def run(B, d, z, alpha, **opt):
    o = B.default_options(**opt) if opt else None
    r = B.eig_arrowhead(cu(d), cu(z), alpha, options=o)
    torch.cuda.synchronize()
    return {k: (v.cpu().numpy() if v is not None else None) for k, v in r.items()}


def rel(a, b):
    return np.abs(a - b) / np.maximum(np.abs(b), 1e-300)


def check(B, d, z, alpha, ks=None, **opt):
    n = d.size
    tol = 16 * (n + 1) * EPS
    g = run(B, d, z, alpha, **opt)
    rows = np.arange(n + 1) if ks is None else np.asarray(ks)
    r = oracle.arrow_eig_all(d, z, alpha, ks=rows, threads=16)
    assert np.max(rel(g["lam"][rows], r["lam"])) <= tol
    assert np.max(rel(g["Vt"][rows], r["Vt"])) <= tol
    kq = rows[:: max(1, rows.size // 24)]
    q = oracle.quad_arrow_all(d, z, alpha, ks=kq, threads=16)
    lq = q["hi"] + q["lo"]
    assert np.max(rel(g["lam"][kq], lq)) <= tol
    assert np.max(rel(g["Vt"][kq], q["Vt"])) <= tol
    # interlacing on the exact pairs: lambda_k - d_k > 0 > lambda_{k+1} - d_k
    sig, mu = g["sigma"], g["mu"]
    above = (sig[:-1] - d) + mu[:-1]
    below = (sig[1:] - d) + mu[1:]
    assert np.all(above > 0) and np.all(below < 0)
    return g


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (3, 2), (17, 3), (100, 4), (511, 5)])
@pytest.mark.parametrize("zf", [0, 1])
def test_sizes(B, n, seed, zf):
    d, z, alpha = W.arrowhead(n, seed)
    check(B, d, z, alpha, zero_finder=zf)


@pytest.mark.parametrize("lanes", [8, 16, 32])
def test_lane_groups(B, lanes):
    d, z, alpha = W.arrowhead(200, 7)
    check(B, d, z, alpha, lanes=lanes)


def test_graded_poles(B):
    n = 60
    d = np.sort(10.0 ** -np.arange(n, dtype=np.float64) * 0.5)[::-1]
    z = 1e-3 * np.sqrt(d)
    for zf in (0, 1):
        check(B, d, z, 1e-30, zero_finder=zf)


def test_16384_sampled_and_dense_properties(B):
    d, z, alpha = W.arrowhead(16384, 6)
    rng = np.random.default_rng(1)
    ks = np.unique(np.concatenate([[0, 1, 8192, 16383, 16384], rng.choice(16385, 40, replace=False)]))
    g = check(B, d, z, alpha, ks=ks)
    Vt = torch.tensor(g["Vt"], device="cuda")
    idx = torch.tensor(rng.choice(16385, 256, replace=False), device="cuda")
    blk = Vt[idx] @ Vt[idx].T - torch.eye(256, dtype=torch.float64, device="cuda")
    assert blk.abs().max().item() <= 16385 * 2.0 ** -52
    # trace: sum lambda = sum d + alpha
    import math
    assert abs(math.fsum(g["sigma"]) + math.fsum(g["mu"]) - (math.fsum(d) + alpha)) <= 64 * 16385 * EPS


def test_edges_and_errors(B):
    g = run(B, np.zeros(0), np.zeros(0), 0.25)
    assert g["lam"].tolist() == [0.25] and abs(g["Vt"][0, 0]) == 1.0
    d, z, alpha = W.arrowhead(20, 8)
    r = B.eig_arrowhead(cu(d), cu(z), alpha, want_vectors=False)
    assert np.max(rel(r["lam"].cpu().numpy(), oracle.arrow_eig_all(d, z, alpha)["lam"])) <= 16 * 21 * EPS
    dd = d.copy(); dd[5] = dd[4]                        # equal poles: reducible
    with pytest.raises(B.DPR1Error) as e:
        B.eig_arrowhead(cu(dd), cu(z), alpha)
    assert e.value.code == 1
    zz = z.copy(); zz[3] = 0.0                          # zero weight: reducible
    with pytest.raises(B.DPR1Error) as e:
        B.eig_arrowhead(cu(d), cu(zz), alpha)
    assert e.value.code == 1
    with pytest.raises(B.DPR1Error) as e:
        B.eig_arrowhead(cu(d[::-1]), cu(z), alpha)
    assert e.value.code == 2
    with pytest.raises(B.DPR1Error) as e:
        B.eig_arrowhead(cu(d), cu(z), float("nan"))
    assert e.value.code == 4


@pytest.mark.parametrize("alpha", [0.3, 1e-8, -2.0])
def test_hard_spectrum(B, alpha):
    d, z, _ = W.hard(1000, 2)
    for zf in (0, 1):
        check(B, d, z, alpha, zero_finder=zf)


def _clustered(n, seed):
    # the recipe of the oracle's remedy pin: tight pole clusters, weights over twelve decades
    rng = np.random.default_rng(seed)
    c = rng.uniform(-1, 1, max(1, n // 6))
    d = rng.choice(c, n) + rng.choice([1.0, -1.0], n) * 10.0 ** rng.uniform(-12, -3, n)
    d = np.sort(d)[::-1].copy()
    z = rng.choice([1.0, -1.0], n) * 10.0 ** rng.uniform(-12, 0, n)
    return d, z, float(10.0 ** rng.uniform(-10, -3))


@pytest.mark.parametrize("seed", [0, 3])
@pytest.mark.parametrize("zf", [0, 1])
def test_clustered_poles_use_remedies(B, seed, zf):
    """K_nu >> 1 next to pole clusters: R1 and R2 on the GPU give every eigenvalue and
    component within the bound of the oracle and of binary128; the counters show both
    remedies and the flagged count matches the oracle's K_nu > 16 count (up to the rounding of
    the two K_nu estimates)."""
    d, z, alpha = _clustered(240, seed)
    check(B, d, z, alpha, zero_finder=zf)
    ws = B.arrow_workspace(d.size, torch.device("cuda"))
    B.eig_arrowhead(cu(d), cu(z), alpha, options=B.default_options(zero_finder=zf), ws=ws)
    st = B.workspace_stats(ws)
    r = oracle.arrow_eig_all(d, z, alpha, threads=16)
    assert st["solved"] == d.size + 1
    assert st["r1"] > 0 and st["r2"] > 0
    assert abs(st["flagged"] - int(np.sum(r["K_nu"] > 16.0))) <= 2
    assert st["r1"] + st["r2"] <= st["flagged"]


def _near_singular(seed):
    rng = np.random.default_rng(seed)
    n = 3
    d = np.concatenate([rng.uniform(0.5, 1, 2), -rng.uniform(0.5, 1, 1)])
    d = np.sort(d)[::-1].copy()
    z = rng.choice([1.0, -1.0], n) * rng.uniform(0.3, 1.0, n)
    return d, z, float(np.sum(z * z / d)) * (1 + 1e-13)


def _lam_small_by_det(d, z, alpha, q):
    """The eigenvalue nearest zero from det(A) = prod_j d_j f(0) and the other eigenvalues
    (binary128), in exact rationals."""
    from fractions import Fraction as Fr
    lq = q["hi"] + q["lo"]
    k0 = int(np.argmin(np.abs(lq)))
    det = Fr(alpha) - sum(Fr(float(zj)) ** 2 / Fr(float(dj)) for dj, zj in zip(d, z))
    for dj in d:
        det *= Fr(float(dj))
    others = Fr(1)
    for k in range(d.size + 1):
        if k != k0:
            others *= Fr(float(q["hi"][k])) + Fr(float(q["lo"][k]))
    return k0, float(det / others)


@pytest.mark.parametrize("case", ["s1", "s2", "s4", "tiny"])
@pytest.mark.parametrize("zf", [0, 1])
def test_near_zero_recompute(B, case, zf):
    """Nearly singular arrowheads: the eigenvalue between the positive and the negative poles
    is far smaller than its distance to them; the GPU recomputes it from A^{-1} (sigma = 0) and
    meets the bound against det(A) = prod_j d_j f(0) in exact rationals."""
    if case == "tiny":
        d = np.array([float.fromhex("0x1.bf656f89b0670p-1"), float.fromhex("-0x1.c35f000a6603ap-1")])
        z = np.array([float.fromhex("0x1.4c82cd5918a9ap-15"), float.fromhex("0x1.5cb9c1af8ca60p-29")])
        alpha = float.fromhex("0x1.ee40d73254cdfp-30")
    else:
        d, z, alpha = _near_singular(int(case[1:]))
    n = d.size
    q = oracle.quad_arrow_all(d, z, alpha)
    k0, lam = _lam_small_by_det(d, z, alpha, q)
    ws = B.arrow_workspace(n, torch.device("cuda"))
    r = B.eig_arrowhead(cu(d), cu(z), alpha, options=B.default_options(zero_finder=zf), ws=ws)
    g = r["lam"].cpu().numpy()
    assert B.workspace_stats(ws)["zero_path"] >= 1
    tol = 16 * (n + 1) * EPS
    assert abs(g[k0] - lam) <= tol * abs(lam)
    check(B, d, z, alpha, zero_finder=zf)
