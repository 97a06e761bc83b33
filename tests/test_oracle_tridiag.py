"""The oracle's divide-and-conquer tridiagonal eigensolver (every merge a DPR1 problem),
pinned against closed forms, LAPACK's tridiagonal solver and the defining properties."""
import numpy as np
import pytest

import oracle
from paper_1405_7537_gb300 import workloads as W

scipy_linalg = pytest.importorskip("scipy.linalg")
EPS = 2.0 ** -53


def dense(a, b):
    return np.diag(a) + np.diag(b, 1) + np.diag(b, -1)


def check_props(a, b, lam, Qt, c=16):
    n = a.size
    T = dense(a, b)
    nT = np.linalg.norm(T, 2)
    Q = Qt.T
    assert np.all(np.diff(lam) <= 0)
    assert np.max(np.linalg.norm(T @ Q - Q * lam[None, :], axis=0)) <= c * n * EPS * nT
    assert np.max(np.abs(Q.T @ Q - np.eye(n))) <= c * n * EPS
    ref = np.sort(scipy_linalg.eigh_tridiagonal(a, b, eigvals_only=True))[::-1]
    assert np.max(np.abs(lam - ref)) <= c * n * EPS * nT


def test_tree_splits_every_boundary_once():
    for n in (1, 2, 3, 5, 7, 100, 129):
        T = 0
        while (1 << T) < n:
            T += 1
        splits = []
        for t in range(T):
            s = oracle.tridiag_tree(n, t)
            for i in range(1 << t):
                if s[i + 1] - s[i] >= 2:
                    mid = ((2 * i + 1) * n) >> (t + 1)
                    assert s[i] < mid < s[i + 1]
                    splits.append(mid)
        assert sorted(splits) == list(range(1, n))
        s = oracle.tridiag_tree(n, T)
        assert all(s[i + 1] - s[i] <= 1 for i in range(1 << T))


@pytest.mark.parametrize("n", [1, 2, 3, 17, 64])
def test_second_difference_closed_form(n):
    """tridiag(-1, 2, -1): lambda_k = 2 - 2 cos(k pi / (n + 1)), v_k[j] ~ sin(j k pi / (n + 1))."""
    a, b = 2.0 * np.ones(n), -np.ones(n - 1)
    lam, Qt = oracle.tridiag_dc(a, b)
    k = np.arange(1, n + 1)
    exact = np.sort(2 - 2 * np.cos(k * np.pi / (n + 1)))[::-1]
    assert np.max(np.abs(lam - exact)) <= 16 * n * EPS * 4
    j = np.arange(1, n + 1)
    for r in range(n):
        kk = n - r                                   # lam is non-increasing
        v = np.sqrt(2.0 / (n + 1)) * np.sin(j * kk * np.pi / (n + 1))
        s = np.sign(np.dot(v, Qt[r]))
        gap = np.min(np.abs(np.delete(exact, r) - exact[r])) if n > 1 else 1.0
        assert np.max(np.abs(s * Qt[r] - v)) <= 64 * n * EPS / gap


def test_two_by_two_closed_form():
    a, b = np.array([0.3, -1.2]), np.array([0.7])
    lam, Qt = oracle.tridiag_dc(a, b)
    m, h = (a[0] + a[1]) / 2, np.hypot((a[0] - a[1]) / 2, b[0])
    assert np.allclose(lam, [m + h, m - h], rtol=0, atol=4 * EPS)
    check_props(a, b, lam, Qt)


@pytest.mark.parametrize("n,seed", [(10, 0), (100, 1), (257, 2)])
def test_random(n, seed):
    a, b = W.tridiagonal(n, seed)
    lam, Qt = oracle.tridiag_dc(a, b, threads=4)
    check_props(a, b, lam, Qt)


def test_wilkinson_and_glued():
    """Wilkinson W21+ (pairs of eigenvalues that agree to ~1e-14) and glued copies of it."""
    for a, b in (W.wilkinson(21), W.glued_wilkinson(21, 4, 1e-10)):
        lam, Qt = oracle.tridiag_dc(a, b)
        check_props(a, b, lam, Qt)


def test_reducible_and_signs():
    """A zero coupling splits T exactly (rho = 0 merge); negative couplings exercise the
    sign of the tear vector."""
    rng = np.random.default_rng(3)
    a = rng.uniform(-1, 1, 40)
    b = rng.uniform(-1, 1, 39)
    b[19] = 0.0
    b[5] = -abs(b[5])
    lam, Qt = oracle.tridiag_dc(a, b)
    check_props(a, b, lam, Qt)
    # the two blocks are independent: their spectra union is the whole spectrum
    l1 = scipy_linalg.eigh_tridiagonal(a[:20], b[:19], eigvals_only=True)
    l2 = scipy_linalg.eigh_tridiagonal(a[20:], b[20:], eigvals_only=True)
    assert np.max(np.abs(np.sort(np.concatenate([l1, l2]))[::-1] - lam)) <= 64 * 40 * EPS * 4
