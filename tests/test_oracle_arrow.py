"""The oracle's arrowhead eigensolver (Algorithm 1's steps on the shifted arrowhead inverse)
pinned against the dense eigenproblem, the 2 x 2 closed form and the binary128 bisection of
the arrowhead's secular function."""
import numpy as np
import pytest

import oracle
from paper_1405_7537_gb300 import workloads as W

EPS = 2.0 ** -53


def dense(d, z, alpha):
    n = d.size
    A = np.zeros((n + 1, n + 1))
    A[:n, :n] = np.diag(d)
    A[:n, n] = z
    A[n, :n] = z
    A[n, n] = alpha
    return A


def test_two_by_two_closed_form():
    d, z, alpha = np.array([0.4]), np.array([0.3]), -0.7
    r = oracle.arrow_eig_all(d, z, alpha)
    m, h = (d[0] + alpha) / 2, np.hypot((d[0] - alpha) / 2, z[0])
    assert np.allclose(r["lam"], [m + h, m - h], rtol=0, atol=4 * EPS)
    A = dense(d, z, alpha)
    V = r["Vt"].T
    assert np.max(np.abs(A @ V - V * r["lam"])) <= 8 * EPS


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (5, 2), (40, 3), (300, 4)])
def test_against_dense_and_binary128(n, seed):
    d, z, alpha = W.arrowhead(n, seed)
    r = oracle.arrow_eig_all(d, z, alpha, threads=4)
    A = dense(d, z, alpha)
    nA = np.linalg.norm(A, 2)
    V = r["Vt"].T
    m = n + 1
    # interlacing lambda_0 > d_0 > lambda_1 > ... > d_{n-1} > lambda_n, residual, orthogonality
    assert np.all(r["lam"][:-1] > d) and np.all(d > r["lam"][1:])
    assert np.max(np.linalg.norm(A @ V - V * r["lam"], axis=0)) <= 8 * m * EPS * nA
    assert np.max(np.abs(V.T @ V - np.eye(m))) <= 8 * m * EPS
    assert np.max(np.abs(np.sort(np.linalg.eigvalsh(A))[::-1] - r["lam"])) <= 8 * m * EPS * nA
    # every eigenvalue and every eigenvector component to high relative accuracy
    q = oracle.quad_arrow_all(d, z, alpha, threads=4)
    lq = q["hi"] + q["lo"]
    assert np.max(np.abs(r["lam"] - lq) / np.abs(lq)) <= 16 * m * EPS
    assert np.max(np.abs(r["Vt"] - q["Vt"]) / np.abs(q["Vt"])) <= 16 * m * EPS


def test_graded_spectrum_relative_accuracy():
    """Poles graded over many decades with small weights: the eigenvalues next to the small
    poles are tiny and must still carry high relative accuracy."""
    n = 60
    d = np.sort(10.0 ** -np.arange(n, dtype=np.float64) * 0.5 + 0.0)[::-1]
    z = 1e-3 * np.sqrt(d)
    alpha = 1e-30
    r = oracle.arrow_eig_all(d, z, alpha)
    q = oracle.quad_arrow_all(d, z, alpha)
    lq = q["hi"] + q["lo"]
    assert np.max(np.abs(r["lam"] - lq) / np.abs(lq)) <= 16 * (n + 1) * EPS


@pytest.mark.parametrize("alpha", [0.3, 1e-8, -2.0])
def test_hard_spectrum_without_remedies(alpha):
    """Graded poles and weights down to 1e-10 (the hard DPR1 spectrum): every eigenvalue and
    eigenvector component within the bound of binary128 with the plain pole solves."""
    d, z, _ = W.hard(300, 1)
    r = oracle.arrow_eig_all(d, z, alpha, threads=8)
    q = oracle.quad_arrow_all(d, z, alpha, threads=8)
    lq = q["hi"] + q["lo"]
    tol = 16 * 301 * EPS
    assert np.max(np.abs(r["lam"] - lq) / np.abs(lq)) <= tol
    assert np.max(np.abs(r["Vt"] - q["Vt"]) / np.maximum(np.abs(q["Vt"]), 1e-300)) <= tol
