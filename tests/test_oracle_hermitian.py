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
    q = oracle.quad_all(d, oracle.hermitian_abs(z), rho)
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
    rr = oracle.eig_all(d, oracle.hermitian_abs(z), rho)
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


def test_hermitian_abs_reading():
    """The weights |z_j| of the reduction: one fixed sequence of correctly rounded binary64
    operations (sqrt of the sum of squares, scaled by a power of two outside [2^-500, 2^500]).
    Within 1.5 ulps of the exact modulus (exact rational square, correctly rounded square root
    by integer arithmetic) over ordinary, huge, tiny and subnormal components; exactly |x| for
    real input; 0 for 0."""
    import math
    from fractions import Fraction as Fr

    def exact_abs(x, y):
        s = Fr(x) ** 2 + Fr(y) ** 2
        if s == 0:
            return 0.0
        # floor(sqrt(s) 2^k) by isqrt on a scaled integer, k large enough for 60 bits beyond
        k = 64 - (s.numerator.bit_length() - s.denominator.bit_length()) // 2 + 60
        if k >= 0:
            r = math.isqrt((s.numerator << (2 * k)) // s.denominator)
            return float(Fr(r, 1 << k))
        r = math.isqrt(s.numerator // (s.denominator << (-2 * k)))
        return float(r << -k)

    rng = np.random.default_rng(9)
    cases = [(3.0, 4.0), (0.0, 0.0), (-2.5, 0.0), (0.0, -1e-300), (5e-324, 5e-324), (1e308, 1e308),
             (1e-310, 3e-310), (2.0 ** 520, 1.0), (2.0 ** -520, 2.0 ** -530)]
    for _ in range(400):
        e = rng.uniform(-320, 300)
        x, y = rng.uniform(-1, 1, 2) * 10.0 ** np.array([e, e + rng.uniform(-20, 20)])
        cases.append((float(x), float(y)))
    z = np.array([complex(x, y) for x, y in cases])
    a = oracle.hermitian_abs(z)
    for (x, y), got in zip(cases, a):
        ref = exact_abs(x, y)
        if ref == 0.0:
            assert got == 0.0
            continue
        ulp = math.ulp(ref)
        assert abs(got - ref) <= 1.5 * ulp, (x, y, got, ref)
    xs = rng.uniform(-1, 1, 200) * 10.0 ** rng.uniform(-300, 300, 200)
    assert np.array_equal(oracle.hermitian_abs(xs.astype(np.complex128)), np.abs(xs))
