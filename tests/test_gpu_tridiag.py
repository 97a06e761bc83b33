"""dpr1_tridiag_eig (divide and conquer with batched DPR1 merges) through the C ABI, against the
oracle's divide and conquer (same tree and merge rules), LAPACK's tridiagonal solver, closed
forms, and the residual / orthogonality bounds."""
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


def run(B, a, b, **opt):
    o = B.default_options(**opt) if opt else None
    lam, Qt = B.eigh_tridiagonal(cu(a), cu(b), options=o)
    torch.cuda.synchronize()
    return lam.cpu().numpy(), Qt.cpu().numpy()


def norm_t(a, b):
    return np.max(np.abs(a)) + 2 * (np.max(np.abs(b)) if b.size else 0.0)


def props_gpu(B, a, b, lam, Qt, c=16):
    """Residual, orthogonality (on the GPU) and LAPACK eigenvalues."""
    n = a.size
    nT = norm_t(a, b)
    Q = cu(Qt).T
    at, bt = cu(a), cu(b)
    TQ = at[:, None] * Q
    TQ[:-1] += bt[:, None] * Q[1:]
    TQ[1:] += bt[:, None] * Q[:-1]
    R = TQ - Q * cu(lam)[None, :]
    assert torch.linalg.vector_norm(R, dim=0).max().item() <= c * n * EPS * nT
    G = Q.T @ Q - torch.eye(n, dtype=torch.float64, device="cuda")
    assert G.abs().max().item() <= c * n * EPS
    import scipy.linalg
    ref = np.sort(scipy.linalg.eigh_tridiagonal(a, b, eigvals_only=True))[::-1]
    assert np.max(np.abs(lam - ref)) <= c * n * EPS * nT


@pytest.mark.parametrize("n", [1, 2, 3, 5, 17, 64, 65, 200])
def test_small_against_oracle(B, n):
    a, b = W.tridiagonal(n, 10 + n)
    lam, Qt = run(B, a, b)
    lo, Qo = oracle.tridiag_dc(a, b, threads=8)
    nT = norm_t(a, b)
    assert np.max(np.abs(lam - lo)) <= 16 * n * EPS * nT
    # eigenvectors of simple, separated eigenvalues: bound by the gap (Davis-Kahan)
    for k in range(n):
        gap = np.min(np.abs(np.delete(lo, k) - lo[k])) if n > 1 else 1.0
        s = np.sign(np.dot(Qt[k], Qo[k]))
        assert np.max(np.abs(s * Qt[k] - Qo[k])) <= 64 * n * EPS * nT / gap + 1e-15, k
    if n > 1:
        props_gpu(B, a, b, lam, Qt)


def test_second_difference_closed_form(B):
    n = 1000
    a, b = 2.0 * np.ones(n), -np.ones(n - 1)
    lam, Qt = run(B, a, b)
    k = np.arange(1, n + 1)
    exact = np.sort(2 - 2 * np.cos(k * np.pi / (n + 1)))[::-1]
    assert np.max(np.abs(lam - exact)) <= 16 * n * EPS * 4
    props_gpu(B, a, b, lam, Qt)


@pytest.mark.parametrize("zf", [0, 1])
def test_random_4096(B, zf):
    a, b = W.tridiagonal(4096, 5)
    lam, Qt = run(B, a, b, zero_finder=zf)
    props_gpu(B, a, b, lam, Qt)


def test_random_1024_against_oracle(B):
    a, b = W.tridiagonal(1024, 6)
    lam, Qt = run(B, a, b)
    lo, Qo = oracle.tridiag_dc(a, b, threads=16)
    assert np.max(np.abs(lam - lo)) <= 16 * 1024 * EPS * norm_t(a, b)
    props_gpu(B, a, b, lam, Qt)


def test_wilkinson_glued_and_reducible(B):
    for a, b in (W.wilkinson(21), W.glued_wilkinson(21, 40, 1e-10), W.glued_wilkinson(101, 10, 1e-14)):
        lam, Qt = run(B, a, b)
        props_gpu(B, a, b, lam, Qt)
    a, b = W.tridiagonal(300, 7)
    b = b.copy()
    b[149] = 0.0
    b[10] = -abs(b[10])
    lam, Qt = run(B, a, b)
    props_gpu(B, a, b, lam, Qt)


def test_eigenvalues_only_and_errors(B):
    a, b = W.tridiagonal(500, 8)
    lam, Qt = B.eigh_tridiagonal(cu(a), cu(b), want_vectors=False)
    assert Qt is None
    lam2, _ = run(B, a, b)
    assert np.array_equal(lam.cpu().numpy(), lam2)
    bb = b.copy()
    bb[7] = np.nan
    with pytest.raises(B.DPR1Error) as e:
        B.eigh_tridiagonal(cu(a), cu(bb))
    assert e.value.code in (2, 3, 4)      # |NaN| coupling: a NaN weight rho of the merge
