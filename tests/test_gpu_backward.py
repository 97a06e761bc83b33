"""GPU adjoint (dpr1_eig_backward through the C ABI, and the autograd Function) against the
oracle's adjoint, central finite differences and the trace identities."""
import numpy as np
import pytest

import oracle
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
    return torch.tensor(np.array(a), dtype=torch.float64, device="cuda")


def nrel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


def gpu_grads(B, d, z, rho, w, Wm):
    r = B.eig(cu(d), cu(z), rho)
    gd, gz, gr = B.eig_backward(cu(d), cu(z), rho, r["sigma"], r["mu"],
                                cu(w) if w is not None else None, cu(Wm) if Wm is not None else None)
    return gd.cpu().numpy(), gz.cpu().numpy(), gr.item(), r


@pytest.mark.parametrize("gen,n,seed", [("uniform", 7, 1), ("uniform", 64, 2), ("hard", 300, 3), ("uniform", 257, 9)])
def test_backward_matches_oracle_adjoint(B, gen, n, seed):
    d, z, rho = getattr(W, gen)(n, seed)
    rng = np.random.default_rng(seed)
    w, Wm = rng.standard_normal(n), rng.standard_normal((n, n))
    gd, gz, gr, r = gpu_grads(B, d, z, rho, w, Wm)
    ro = oracle.eig_all(d, z, rho, threads=8)
    od, oz, orho = oracle.backward(d, z, rho, ro["sigma"], ro["mu"], w, Wm)
    assert nrel(gd, od) <= 1e-10 and nrel(gz, oz) <= 1e-10 and abs(gr - orho) <= 1e-10 * abs(orho), \
        (nrel(gd, od), nrel(gz, oz), gr, orho)


@pytest.mark.parametrize("gen,n,seed", [("hard", 200, 5), ("large", 300, 4)])
def test_backward_matches_binary128_adjoint(B, gen, n, seed):
    if gen == "large":
        d, z, rho, _ = W.large(n, seed, with_W=False)
    else:
        d, z, rho = getattr(W, gen)(n, seed)
    rng = np.random.default_rng(seed)
    w, Wm = rng.standard_normal(n), rng.standard_normal((n, n))
    gd, gz, gr, _ = gpu_grads(B, d, z, rho, w, Wm)
    qd, qz, qr = oracle.quad_backward(d, z, rho, w, Wm)
    assert nrel(gd, qd) <= 1e-10 and nrel(gz, qz) <= 1e-10 and abs(gr - qr) <= 1e-10 * abs(qr), \
        (nrel(gd, qd), nrel(gz, qz), gr, qr)


def test_backward_central_differences(B):
    n = 10
    d, z, rho = W.uniform(n, 17)
    rng = np.random.default_rng(17)
    w, Wm = rng.standard_normal(n), rng.standard_normal((n, n))
    gd, gz, gr, _ = gpu_grads(B, d, z, rho, w, Wm)

    def loss(dd_, zz_, rr_):
        r = B.eig(cu(dd_), cu(zz_), rr_)
        return float(np.dot(w, r["lam"].cpu().numpy()) + np.sum(Wm * r["Vt"].cpu().numpy()))

    h = 1e-6 * min(1.0, float(np.min(-np.diff(d))))
    for t in range(4):
        a, b_, c = rng.standard_normal(n), rng.standard_normal(n), rng.standard_normal()
        fd = (loss(d + h * a, z + h * b_, rho + h * c) - loss(d - h * a, z - h * b_, rho - h * c)) / (2 * h)
        an = np.dot(gd, a) + np.dot(gz, b_) + gr * c
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (fd, an)


def test_trace_identities_full_size(B):
    """d(sum lambda)/dd = 1, /dz = 2 rho z, /drho = ||z||^2 (trace(A) = sum lambda) at n = 4096."""
    d, z, rho, _, _ = W.diff(4096, 2)
    n = d.size
    gd, gz, gr, _ = gpu_grads(B, d, z, rho, np.ones(n), None)
    assert np.max(np.abs(gd - 1.0)) <= 1e-11
    assert np.max(np.abs(gz - 2 * rho * z)) <= 1e-11 * np.max(np.abs(2 * rho * z)) * 10
    assert abs(gr - np.dot(z, z)) <= 1e-11 * np.dot(z, z)


def test_differentiated_4096_config(B):
    """The n = 4096 fwd+bwd workload: loss = w . lambda + sum W o V, gradients vs the oracle."""
    d, z, rho, w, Wm = W.diff(4096, 2)
    gd, gz, gr, r = gpu_grads(B, d, z, rho, w, Wm)
    ro = oracle.eig_all(d, z, rho, threads=16, want_vectors=False)
    od, oz, orho = oracle.backward(d, z, rho, ro["sigma"], ro["mu"], w, Wm)
    assert nrel(gd, od) <= 1e-10 and nrel(gz, oz) <= 1e-10 and abs(gr - orho) <= 1e-10 * abs(orho)


def test_large_32768_sampled_rows(B):
    """n = 32768 (recompute in the backward): W nonzero on 48 sampled rows only, so the oracle sums
    exactly those rows."""
    d, z, rho, _ = W.large(32768, 4, with_W=False)
    n = d.size
    rng = np.random.default_rng(5)
    ks = np.sort(rng.choice(n, 48, replace=False))
    Wrows = rng.standard_normal((ks.size, n))
    r = B.eig(cu(d), cu(z), rho, want_vectors=False)
    gV = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    gV[torch.tensor(ks, device="cuda")] = cu(Wrows)
    gd, gz, gr = B.eig_backward(cu(d), cu(z), rho, r["sigma"], r["mu"], None, gV)
    sig, mu = r["sigma"].cpu().numpy()[ks], r["mu"].cpu().numpy()[ks]
    od, oz, orho = oracle.backward_rows(d, z, rho, sig, mu, None, Wrows)
    assert nrel(gd.cpu().numpy(), od) <= 1e-10 and nrel(gz.cpu().numpy(), oz) <= 1e-10
    assert abs(gr.item() - orho) <= 1e-10 * abs(orho)


def test_autograd_function(B):
    n = 8
    d, z, rho = W.uniform(n, 23)
    dt = cu(d).requires_grad_(True)
    zt = cu(z).requires_grad_(True)
    rt = torch.tensor(rho, dtype=torch.float64, device="cuda", requires_grad=True)
    rng = np.random.default_rng(23)
    w, Wm = cu(rng.standard_normal(n)), cu(rng.standard_normal((n, n)))
    lam, V = B.eigh_dpr1(dt, zt, rt)
    loss = (w * lam).sum() + (Wm * V).sum()
    loss.backward()
    # reference: oracle adjoint with V[:, k] = v_k, i.e. dL/dVt = Wm^T
    ro = oracle.eig_all(d, z, rho)
    od, oz, orho = oracle.backward(d, z, rho, ro["sigma"], ro["mu"], w.cpu().numpy(), Wm.cpu().numpy().T)
    assert nrel(dt.grad.cpu().numpy(), od) <= 1e-10
    assert nrel(zt.grad.cpu().numpy(), oz) <= 1e-10
    assert abs(rt.grad.item() - orho) <= 1e-10 * abs(orho)
    # double check with torch's finite-difference gradcheck on the same function
    def f(dd_, zz_):
        lam_, V_ = B.eigh_dpr1(dd_, zz_, rho)
        return (w * lam_).sum() + (Wm * V_).sum()
    assert torch.autograd.gradcheck(f, (cu(d).requires_grad_(True), cu(z).requires_grad_(True)), eps=1e-7,
                                    atol=1e-6, rtol=1e-5)
