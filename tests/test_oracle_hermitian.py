"""The oracle's complex Hermitian DPR1 (D + rho z z^*), pinned against the dense Hermitian
eigenproblem: residuals and orthonormality in complex arithmetic, eigenvalues against
numpy's eigvalsh and the binary128 reference, and the eigenvector formula
v = (D - lambda I)^{-1} z / ||.|| with the complex z evaluated directly."""
import numpy as np
import pytest

import oracle
from paper_1405_7537_gb300 import workloads as W

EPS = 2.0 ** -53


def dense(d, z, rho):
    return np.diag(d).astype(np.complex128) + rho * np.outer(z, np.conj(z))


@pytest.mark.parametrize("n,seed", [(2, 0), (7, 1), (40, 2), (120, 3)])
def test_residual_orthonormality_and_eigenvalues(n, seed):
    d, z, rho = W.hermitian(n, seed, base="uniform")
    r = oracle.eig_hermitian(d, z, rho)
    A = dense(d, z, rho)
    nA = np.linalg.norm(A, 2)
    V = r["Vt"].T
    res = A @ V - V * r["lam"][None, :]
    assert np.max(np.linalg.norm(res, axis=0)) <= 8 * n * EPS * nA
    assert np.max(np.abs(V.conj().T @ V - np.eye(n))) <= 8 * n * EPS
    ev = np.sort(np.linalg.eigvalsh(A))[::-1]
    assert np.max(np.abs(ev - r["lam"])) <= 8 * n * EPS * nA
    # every eigenvalue to high relative accuracy against the binary128 bisection of the
    # secular function with weights |z_j|
    q = oracle.quad_all(d, np.abs(z), rho)
    rel = np.abs(r["lam"] - (q["hi"] + q["lo"])) / np.abs(q["hi"])
    assert rel.max() <= 16 * n * EPS


def test_eigenvector_formula_with_complex_z():
    d, z, rho = W.hermitian(30, 5, base="uniform")
    r = oracle.eig_hermitian(d, z, rho)
    for k in (0, 7, 29):
        lam = r["sigma"][k] + r["mu"][k]
        x = z / ((d - r["sigma"][k]) - r["mu"][k])
        x = x / np.linalg.norm(x)
        assert np.max(np.abs(x - r["Vt"][k])) <= 64 * EPS, k
        assert abs(lam - r["lam"][k]) <= 4 * EPS * abs(lam)


def test_real_z_reduces_to_the_real_problem():
    d, z, rho = W.uniform(50, 6)
    rc = oracle.eig_hermitian(d, z.astype(np.complex128), rho)
    rr = oracle.eig_all(d, np.abs(z), rho)
    assert np.array_equal(rc["lam"], rr["lam"])
    # phases of a real z are +-1: v_k = diag(sign z) u_k
    assert np.max(np.abs(rc["Vt"] - rr["Vt"] * np.sign(z)[None, :])) == 0.0


def test_deflation_with_complex_weights():
    d = np.array([3.0, 2.0, 2.0, 1.0, 0.5])
    z = np.array([1 + 1j, 0.5j, 0.7 - 0.2j, 0.0, -1.0])
    rho = 0.9
    r = oracle.eig_hermitian(d, z, rho)
    A = dense(d, z, rho)
    V = r["Vt"].T
    assert np.max(np.abs(A @ V - V * r["lam"][None, :])) <= 1e-14
    assert np.max(np.abs(V.conj().T @ V - np.eye(5))) <= 1e-14
