"""Seeded randomized parity on problems of many shapes.  dpr1_eig (both zero finders): uniform,
clustered and graded poles, exact ties, zero and tiny weights, rho over twelve decades;
irreducible problems are compared eigenvalue by eigenvalue and component by component with
the oracle and binary128, deflated ones by eigenvalues, residual and orthogonality
(eigenvectors of repeated eigenvalues are a basis choice).  dpr1_arrow_eig: random
arrowheads against binary128.  dpr1_tridiag_eig: random tridiagonal matrices against LAPACK.
dpr1_eig_batched: a batch of fuzz problems against the single calls."""
import numpy as np
import pytest

import oracle
from gpu_common import run_gpu, tol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1405_7537_gb300 import binding
    binding.lib()
    return binding


def random_problem(rng):
    n = int(rng.integers(1, 81))
    kind = rng.integers(0, 4)
    if kind == 0:                                   # uniform
        d = rng.uniform(-1, 1, n)
    elif kind == 1:                                 # clusters of close poles
        c = rng.uniform(-1, 1, max(1, n // 6))
        d = rng.choice(c, n) + rng.choice([1.0, -1.0], n) * 10.0 ** rng.uniform(-12, -3, n)
    elif kind == 2:                                 # graded over many decades
        d = np.sign(rng.uniform(-1, 1, n)) * 10.0 ** rng.uniform(-10, 0, n)
    else:                                           # exact ties
        d = rng.choice(rng.uniform(-1, 1, max(1, n // 3)), n)
    d = np.sort(d)[::-1].copy()
    zk = rng.integers(0, 3)
    if zk == 0:
        z = rng.uniform(-1, 1, n)
    elif zk == 1:
        z = rng.choice([1.0, -1.0], n) * 10.0 ** rng.uniform(-12, 0, n)
    else:
        z = rng.uniform(-1, 1, n)
        z[rng.random(n) < 0.2] = 0.0
    rho = float(10.0 ** rng.uniform(-6, 6))
    return d, z, rho


def irreducible(d, z, rho):
    return rho > 0 and not np.any(oracle.zero_weight(z)) and np.all(d[:-1] > d[1:])


@pytest.mark.parametrize("zf", [0, 1])
def test_fuzz_small_problems(B, zf):
    rng = np.random.default_rng(20261203 + zf)
    n_irr = 0
    for case in range(160):
        d, z, rho = random_problem(rng)
        n = d.size
        g = run_gpu(B, d, z, rho, zero_finder=zf)
        lam = g["lam"]
        if irreducible(d, z, rho):
            n_irr += 1
            r = oracle.eig_all(d, z, rho)
            q = oracle.quad_all(d, z, rho)
            lq = q["hi"] + q["lo"]
            scale = np.maximum(np.abs(lq), 1e-300)
            assert np.max(np.abs(lam - lq) / scale) <= tol(n), (case, "lambda vs binary128")
            assert np.max(np.abs(lam - r["lam"]) / scale) <= tol(n), (case, "lambda vs oracle")
            Vq = q["Vt"]
            err = np.abs(g["Vt"] - Vq) / np.maximum(np.abs(Vq), 1e-300)
            assert err.max() <= tol(n), (case, "vector vs binary128", float(err.max()))
        else:
            r = oracle.eig_full(d, z, rho)
            A = np.diag(d) + rho * np.outer(z, z)
            nA = max(np.linalg.norm(A, 2), 1e-300)
            assert np.max(np.abs(lam - r["lam"])) <= tol(n) * nA, (case, "lambda (deflated)")
            V = g["Vt"].T
            assert np.max(np.abs(A @ V - V * lam[None, :])) <= 64 * n * 2.0 ** -53 * nA, (case, "residual")
            assert np.max(np.abs(V.T @ V - np.eye(n))) <= 64 * n * 2.0 ** -53, (case, "orthogonality")
    assert n_irr >= 40


@pytest.mark.parametrize("zf", [0, 1])
def test_fuzz_larger_irreducible(B, zf):
    """Irreducible problems of 100 to 600 poles with clustered or graded poles and weights over
    twelve decades: every eigenvalue and component against binary128."""
    rng = np.random.default_rng(4242 + zf)
    done = 0
    while done < 12:
        d, z, rho = random_problem(rng)
        n = int(rng.integers(100, 601))
        kind = rng.integers(0, 2)
        if kind == 0:
            c = rng.uniform(-1, 1, n // 8)
            d = rng.choice(c, n) + rng.choice([1.0, -1.0], n) * 10.0 ** rng.uniform(-12, -3, n)
        else:
            d = np.sign(rng.uniform(-1, 1, n)) * 10.0 ** rng.uniform(-10, 0, n)
        d = np.sort(d)[::-1].copy()
        z = rng.choice([1.0, -1.0], n) * 10.0 ** rng.uniform(-12, 0, n)
        if not irreducible(d, z, rho):
            continue
        done += 1
        g = run_gpu(B, d, z, rho, zero_finder=zf)
        q = oracle.quad_all(d, z, rho, threads=16)
        lq = q["hi"] + q["lo"]
        assert np.max(np.abs(g["lam"] - lq) / np.abs(lq)) <= tol(n), (done, n, rho)
        err = np.abs(g["Vt"] - q["Vt"]) / np.maximum(np.abs(q["Vt"]), 1e-300)
        assert err.max() <= tol(n), (done, n, rho, float(err.max()))


@pytest.mark.parametrize("zf", [0, 1])
def test_fuzz_arrowhead(B, zf):
    """Random irreducible arrowheads: clustered or graded poles, weights over twelve decades,
    alpha over many decades and both signs, against binary128."""
    rng = np.random.default_rng(777 + zf)
    done = 0
    while done < 40:
        n = int(rng.integers(1, 300))
        kind = rng.integers(0, 3)
        if kind == 0:
            d = rng.uniform(-1, 1, n)
        elif kind == 1:
            c = rng.uniform(-1, 1, max(1, n // 6))
            d = rng.choice(c, n) + rng.choice([1.0, -1.0], n) * 10.0 ** rng.uniform(-12, -3, n)
        else:
            d = np.sign(rng.uniform(-1, 1, n)) * 10.0 ** rng.uniform(-10, 0, n)
        d = np.sort(d)[::-1].copy()
        z = rng.choice([1.0, -1.0], n) * 10.0 ** rng.uniform(-12 if rng.random() < 0.5 else -2, 0, n)
        alpha = float(rng.choice([1.0, -1.0]) * 10.0 ** rng.uniform(-12, 2))
        if not (np.all(d[:-1] > d[1:]) and not np.any(oracle.zero_weight(z))):
            continue
        done += 1
        r = B.eig_arrowhead(torch.tensor(d, device="cuda"), torch.tensor(z, device="cuda"), alpha,
                            options=B.default_options(zero_finder=zf))
        lam, Vt = r["lam"].cpu().numpy(), r["Vt"].cpu().numpy()
        q = oracle.quad_arrow_all(d, z, alpha, threads=16)
        lq = q["hi"] + q["lo"]
        t = 16 * (n + 1) * 2.0 ** -53
        assert np.max(np.abs(lam - lq) / np.abs(lq)) <= t, (done, n, alpha)
        err = np.abs(Vt - q["Vt"]) / np.maximum(np.abs(q["Vt"]), 1e-300)
        assert err.max() <= t, (done, n, alpha, float(err.max()))


def test_fuzz_tridiagonal(B):
    """Random symmetric tridiagonal matrices (uniform, graded diagonals, tiny and zero couplings)
    by divide and conquer: eigenvalues against LAPACK, residual and orthogonality."""
    import scipy.linalg
    rng = np.random.default_rng(99)
    for case in range(30):
        n = int(rng.integers(1, 400))
        a = rng.uniform(-1, 1, n) * (10.0 ** rng.uniform(-6, 0, n) if rng.random() < 0.3 else 1.0)
        b = rng.uniform(-1, 1, max(n - 1, 0))
        if rng.random() < 0.3 and n > 1:
            b *= 10.0 ** rng.uniform(-14, 0, n - 1)
        if rng.random() < 0.2 and n > 2:
            b[rng.integers(0, n - 1)] = 0.0
        lam, Qt = B.eigh_tridiagonal(torch.tensor(a, device="cuda"), torch.tensor(b, device="cuda"),
                                     options=B.default_options(zero_finder=int(rng.integers(0, 2))))
        lam, Qt = lam.cpu().numpy(), Qt.cpu().numpy()
        nT = np.max(np.abs(a)) + 2 * (np.max(np.abs(b)) if n > 1 else 0.0)
        if n > 1:
            ref = np.sort(scipy.linalg.eigh_tridiagonal(a, b, eigvals_only=True))[::-1]
        else:
            ref = a.copy()
        assert np.max(np.abs(lam - ref)) <= 16 * n * 2.0 ** -53 * nT, case
        T = np.diag(a) + (np.diag(b, 1) + np.diag(b, -1) if n > 1 else 0.0)
        Q = Qt.T
        assert np.max(np.abs(T @ Q - Q * lam[None, :])) <= 16 * n * 2.0 ** -53 * nT, case
        assert np.max(np.abs(Q.T @ Q - np.eye(n))) <= 16 * n * 2.0 ** -53, case


def test_fuzz_batched_against_single(B):
    """A batch of random problems of the fuzz shapes solved in one call equals the single
    calls (both zero finders)."""
    rng = np.random.default_rng(31)
    probs = [random_problem(rng) for _ in range(96)]
    sizes = [p[0].size for p in probs]
    d = np.concatenate([p[0] for p in probs])
    z = np.concatenate([p[1] for p in probs])
    rho = np.array([p[2] for p in probs])
    bt = B.Batch(sizes)
    for zf in (0, 1):
        bt.solve(torch.tensor(d, device="cuda"), torch.tensor(z, device="cuda"), torch.tensor(rho, device="cuda"),
                 options=B.default_options(zero_finder=zf), check=True)
        torch.cuda.synchronize()
        for p, (dp, zp, rp) in enumerate(probs):
            n = dp.size
            lam = bt.block(p)[0].cpu().numpy()
            g = run_gpu(B, dp, zp, rp, zero_finder=zf)
            scale = np.maximum(np.abs(g["lam"]), np.max(np.abs(g["lam"])) * 2.0 ** -52)
            assert np.max(np.abs(lam - g["lam"]) / scale) <= tol(n), (zf, p)


@pytest.mark.parametrize("zf", [0, 1])
def test_fuzz_hermitian(B, zf):
    """Complex Hermitian D + rho z z^* with the fuzz shapes and random phases (some weights
    purely real or purely imaginary, some zero): irreducible problems against the oracle's
    phase reduction and binary128 component by component, deflated ones by eigenvalues,
    residual and unitarity."""
    rng = np.random.default_rng(555 + zf)
    n_irr = 0
    for case in range(60):
        d, zr, rho = random_problem(rng)
        n = d.size
        ph = np.exp(1j * rng.uniform(-np.pi, np.pi, n))
        pick = rng.random(n)
        ph[pick < 0.1] = 1.0
        ph[(pick >= 0.1) & (pick < 0.2)] = 1j
        z = np.abs(zr) * ph
        z[zr == 0] = 0.0
        r = B.eig_hermitian(torch.tensor(d, device="cuda"), torch.tensor(z, device="cuda"), rho,
                            options=B.default_options(zero_finder=zf))
        lam, Vt = r["lam"].cpu().numpy(), r["Vt"].cpu().numpy()
        a = oracle.hermitian_abs(z)
        if irreducible(d, a, rho):
            n_irr += 1
            o = oracle.eig_hermitian(d, z, rho)
            scale = np.abs(o["lam"])
            assert np.max(np.abs(lam - o["lam"]) / scale) <= tol(n), (case, "lambda vs oracle")
            err = np.abs(Vt - o["Vt"]) / np.maximum(np.abs(o["Vt"]), 1e-300)
            assert err.max() <= tol(n), (case, "vector vs oracle", float(err.max()))
            q = oracle.quad_all(d, a, rho)
            lq = q["hi"] + q["lo"]
            assert np.max(np.abs(lam - lq) / np.abs(lq)) <= tol(n), (case, "lambda vs binary128")
        else:
            A = np.diag(d).astype(np.complex128) + rho * np.outer(z, z.conj())
            nA = max(np.linalg.norm(A, 2), 1e-300)
            ref = np.sort(np.linalg.eigvalsh(A))[::-1]
            assert np.max(np.abs(lam - ref)) <= 64 * n * 2.0 ** -53 * nA, (case, "lambda (deflated)")
            V = Vt.T
            assert np.max(np.abs(A @ V - V * lam[None, :])) <= 64 * n * 2.0 ** -53 * nA, (case, "residual")
            assert np.max(np.abs(V.conj().T @ V - np.eye(n))) <= 64 * n * 2.0 ** -53, (case, "unitarity")
    assert n_irr >= 15
