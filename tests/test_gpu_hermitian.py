"""dpr1_eig_hermitian (complex Hermitian D + rho z z^*) through the C ABI against the oracle's
Hermitian reduction and the binary128 reference: every eigenvalue and every complex
eigenvector component within relative 16 n 2^-53."""
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


def cu(a):
    return torch.tensor(np.array(a, copy=True, order="C"), device="cuda")


def run(B, d, z, rho, **opt):
    o = B.default_options(**opt) if opt else None
    r = B.eig_hermitian(cu(d), cu(z), rho, options=o)
    torch.cuda.synchronize()
    return {k: (v.cpu().numpy() if v is not None else None) for k, v in r.items()}


def crel(a, b):
    return np.abs(a - b) / np.maximum(np.abs(b), 1e-300)


def check(B, d, z, rho, ks=None, **opt):
    n = d.size
    g = run(B, d, z, rho, **opt)
    r = oracle.eig_hermitian(d, z, rho, ks=ks, threads=16)
    rows = np.arange(n) if ks is None else np.asarray(ks)
    assert np.max(crel(g["lam"][rows], r["lam"])) <= tol(n)
    assert np.max(crel(g["Vt"][rows], r["Vt"])) <= tol(n)
    # binary128: eigenvalues, and the vectors through the same phases
    kq = rows[:: max(1, rows.size // 16)]
    q = oracle.quad_all(d, oracle.hermitian_abs(z), rho, ks=kq, threads=16)
    lam_q = q["hi"] + q["lo"]
    assert np.max(np.abs(g["lam"][kq] - lam_q) / np.abs(lam_q)) <= tol(n)
    a = oracle.hermitian_abs(z)
    phi = z.real / a + 1j * (z.imag / a)
    assert np.max(crel(g["Vt"][kq], q["Vt"] * phi[None, :])) <= tol(n)
    return g


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (5, 2), (33, 3), (512, 0)])
def test_uniform_sizes(B, n, seed):
    d, z, rho = W.hermitian(n, seed, base="uniform")
    check(B, d, z, rho)


@pytest.mark.parametrize("zf", [0, 1])
def test_hard_spectrum(B, zf):
    d, z, rho = W.hermitian(1000, 9, base="hard")
    check(B, d, z, rho, zero_finder=zf)


def test_hard_16384_sampled(B):
    d, z, rho = W.hermitian(16384, 1)
    rng = np.random.default_rng(0)
    ks = np.unique(np.concatenate([[0, 1, 8191, 16382, 16383], rng.choice(16384, 40, replace=False)]))
    g = check(B, d, z, rho, ks=ks)
    # unitary rows at full size: a sampled block of V^* V
    Vt = torch.tensor(g["Vt"], device="cuda")
    idx = torch.tensor(rng.choice(16384, 256, replace=False), device="cuda")
    blk = Vt[idx] @ Vt[idx].conj().T - torch.eye(256, dtype=torch.complex128, device="cuda")
    assert blk.abs().max().item() <= 16384 * 2.0 ** -52


def test_residual_dense(B):
    d, z, rho = W.hermitian(200, 4, base="uniform")
    g = run(B, d, z, rho)
    A = np.diag(d).astype(np.complex128) + rho * np.outer(z, np.conj(z))
    V = g["Vt"].T
    nA = np.linalg.norm(A, 2)
    assert np.max(np.linalg.norm(A @ V - V * g["lam"][None, :], axis=0)) <= 8 * 200 * 2.0 ** -53 * nA
    assert np.max(np.abs(V.conj().T @ V - np.eye(200))) <= 8 * 200 * 2.0 ** -53


def test_deflation_and_edges(B):
    d = np.array([3.0, 2.0, 2.0, 1.0, 0.5])
    z = np.array([1 + 1j, 0.5j, 0.7 - 0.2j, 0.0, -1.0])
    g = run(B, d, z, 0.9)
    A = np.diag(d).astype(np.complex128) + 0.9 * np.outer(z, np.conj(z))
    V = g["Vt"].T
    assert np.max(np.abs(A @ V - V * g["lam"][None, :])) <= 1e-14
    assert np.max(np.abs(V.conj().T @ V - np.eye(5))) <= 1e-14
    # eigenvalues only
    dd, zz, rho = W.hermitian(64, 3, base="uniform")
    r = B.eig_hermitian(cu(dd), cu(zz), rho, want_vectors=False)
    ref = oracle.eig_hermitian(dd, zz, rho)
    assert np.max(crel(r["lam"].cpu().numpy(), ref["lam"])) <= tol(64)
    # a non-finite imaginary part is reported by the device check
    zb = zz.copy()
    zb[5] = complex(0.3, np.inf)
    with pytest.raises(B.DPR1Error) as e:
        B.eig_hermitian(cu(dd), cu(zb), rho)
    assert e.value.code == 4
