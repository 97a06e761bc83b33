"""GPU adjoint (dpr1_eig_backward through the C ABI, and the autograd Function) against the
oracle's adjoint and the binary128 adjoint component by component, per-coordinate central
finite differences and the trace identities.  The componentwise bound: every component of
dL/dd, dL/dz and dL/drho within 16 n 2^-53 of its error scale (tests/adjoint_scale.py), and to
rel 1e-10 wherever that scale is within 100 times the component."""
import numpy as np
import pytest

import oracle
from adjoint_scale import adjoint_scales, central_differences, componentwise
from paper_1405_7537_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
U53 = 2.0 ** -53


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1405_7537_gb300 import binding
    binding.lib()
    return binding


def cu(a):
    return torch.tensor(np.array(a), dtype=torch.float64, device="cuda")


def gpu_grads(B, d, z, rho, w, Wm):
    r = B.eig(cu(d), cu(z), rho)
    gd, gz, gr = B.eig_backward(cu(d), cu(z), rho, r["sigma"], r["mu"],
                                cu(w) if w is not None else None, cu(Wm) if Wm is not None else None)
    return gd.cpu().numpy(), gz.cpu().numpy(), gr.item(), r


def check_components(got, ref, scales, n, what):
    """Every component of (dbar, zbar, rhobar) within 16 n 2^-53 of its error scale, and to rel 1e-10
    wherever the scale is within 100 times the component."""
    tau = 16 * n * U53
    for name, g, r, sc in zip(("d", "z", "rho"), got, ref, scales):
        res = componentwise(g, r, sc, tau)
        assert res["ok"], (what, name, res)


def load(gen, n, seed):
    if gen == "large":
        d, z, rho, _ = W.large(n, seed, with_W=False)
    else:
        d, z, rho = getattr(W, gen)(n, seed)[:3]
    return d, z, rho


@pytest.mark.parametrize("gen,n,seed", [("uniform", 7, 1), ("uniform", 64, 2), ("hard", 300, 3), ("uniform", 257, 9),
                                        ("hard", 2000, 3), ("large", 1000, 4)])
def test_backward_matches_oracle_adjoint(B, gen, n, seed):
    d, z, rho = load(gen, n, seed)
    rng = np.random.default_rng(seed)
    w, Wm = rng.standard_normal(n), rng.standard_normal((n, n))
    gd, gz, gr, r = gpu_grads(B, d, z, rho, w, Wm)
    ro = oracle.eig_all(d, z, rho, threads=16, want_vectors=False)
    od, oz, orho = oracle.backward(d, z, rho, ro["sigma"], ro["mu"], w, Wm)
    sc = adjoint_scales(d, z, rho, ro["sigma"], ro["mu"], w, Wm)
    check_components((gd, gz, gr), (od, oz, orho), sc, n, "oracle")


@pytest.mark.parametrize("gen,n,seed", [("uniform", 64, 2), ("hard", 200, 5), ("hard", 300, 3), ("large", 300, 4)])
def test_backward_matches_binary128_adjoint(B, gen, n, seed):
    d, z, rho = load(gen, n, seed)
    rng = np.random.default_rng(seed)
    w, Wm = rng.standard_normal(n), rng.standard_normal((n, n))
    gd, gz, gr, r = gpu_grads(B, d, z, rho, w, Wm)
    qd, qz, qr = oracle.quad_backward(d, z, rho, w, Wm)
    sc = adjoint_scales(d, z, rho, r["sigma"].cpu().numpy(), r["mu"].cpu().numpy(), w, Wm)
    check_components((gd, gz, gr), (qd, qz, qr), sc, n, "binary128")


@pytest.mark.parametrize("gen,n,seed", [("uniform", 16, 3), ("uniform", 32, 4), ("hard", 16, 5), ("hard", 32, 6)])
def test_backward_per_coordinate_central_differences(B, gen, n, seed):
    """Every component of the GPU adjoint against a central difference of the GPU forward in that
    one coordinate (Richardson-extrapolated; steps 1e-4 of the local pole gap for d_j, of |z_j| for
    z_j, of rho for rho), rel 1e-6.  The loss is sensitive at each component's own scale:
    sum_k w_k mu_k with mu_k = lambda_k - d_{i(k)} (the unperturbed shift; on the hard spectrum
    lambda_k rounds onto its pole, mu_k does not) plus sum W_kj V_kj / |V_kj|, whose adjoint is that
    of (lambda, V) with dL/dlambda = w, dL/dVt = W / |V|, less w_k at d_{i(k)}."""
    d, z, rho = load(gen, n, seed)
    rng = np.random.default_rng(seed)
    w, Wm = rng.standard_normal(n), rng.standard_normal((n, n))
    r0 = {k: v.cpu().numpy() for k, v in B.eig(cu(d), cu(z), rho).items()}
    sidx = np.array([int(np.flatnonzero(d == s)[0]) if np.any(d == s) else -1 for s in r0["sigma"]])
    pole = sidx >= 0
    Wh = Wm / np.abs(r0["Vt"])

    def loss(dd_, zz_, rr_):
        r = B.eig(cu(dd_), cu(zz_), rr_)
        sig, mu, Vt = r["sigma"].cpu().numpy(), r["mu"].cpu().numpy(), r["Vt"].cpu().numpy()
        base = np.where(pole, dd_[np.maximum(sidx, 0)], r0["sigma"])
        return float(np.dot(w, (sig - base) + mu) + np.sum(Wh * Vt))

    gd, gz, gr = B.eig_backward(cu(d), cu(z), rho, cu(r0["sigma"]), cu(r0["mu"]), cu(w), cu(Wh))
    gd, gz, gr = gd.cpu().numpy(), gz.cpu().numpy(), gr.item()
    np.subtract.at(gd, sidx[pole], w[pole])
    fd_d, fd_z, fd_r = central_differences(loss, d, z, rho)
    assert np.max(np.abs(fd_d - gd) / np.abs(gd)) <= 1e-6
    assert np.max(np.abs(fd_z - gz) / np.abs(gz)) <= 1e-6
    assert abs(fd_r - gr) <= 1e-6 * abs(gr)


def test_trace_identities_full_size(B):
    """d(sum lambda)/dd = 1, /dz = 2 rho z, /drho = ||z||^2 (trace(A) = sum lambda) at n = 4096."""
    d, z, rho, _, _ = W.diff(4096, 2)
    n = d.size
    gd, gz, gr, _ = gpu_grads(B, d, z, rho, np.ones(n), None)
    assert np.max(np.abs(gd - 1.0)) <= 1e-11
    assert np.max(np.abs(gz - 2 * rho * z)) <= 1e-11 * np.max(np.abs(2 * rho * z)) * 10
    assert abs(gr - np.dot(z, z)) <= 1e-11 * np.dot(z, z)


def test_differentiated_4096_config(B):
    """The n = 4096 fwd+bwd workload: loss = w . lambda + sum W o V, every gradient component
    against the oracle's adjoint."""
    d, z, rho, w, Wm = W.diff(4096, 2)
    n = d.size
    gd, gz, gr, r = gpu_grads(B, d, z, rho, w, Wm)
    ro = oracle.eig_all(d, z, rho, threads=16, want_vectors=False)
    od, oz, orho = oracle.backward(d, z, rho, ro["sigma"], ro["mu"], w, Wm)
    sc = adjoint_scales(d, z, rho, ro["sigma"], ro["mu"], w, Wm)
    check_components((gd, gz, gr), (od, oz, orho), sc, n, "oracle n=4096")


def test_large_32768_sampled_rows(B):
    """n = 32768 (recompute in the backward): W nonzero on 48 sampled rows only, so the oracle sums
    exactly those rows; every component of the gradients against it."""
    d, z, rho, _ = W.large(32768, 4, with_W=False)
    n = d.size
    rng = np.random.default_rng(5)
    ks = np.sort(rng.choice(n, 48, replace=False))
    Wrows = rng.standard_normal((ks.size, n))
    r = B.eig(cu(d), cu(z), rho, want_vectors=False)
    gV = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    gV[torch.tensor(ks, device="cuda")] = cu(Wrows)
    gd, gz, gr = B.eig_backward(cu(d), cu(z), rho, r["sigma"], r["mu"], None, gV)
    del gV
    sig, mu = r["sigma"].cpu().numpy()[ks], r["mu"].cpu().numpy()[ks]
    od, oz, orho = oracle.backward_rows(d, z, rho, sig, mu, None, Wrows)
    sc = adjoint_scales(d, z, rho, sig, mu, None, Wrows)
    check_components((gd.cpu().numpy(), gz.cpu().numpy(), gr.item()), (od, oz, orho), sc, n, "oracle n=32768 rows")


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
    wn, Wt = w.cpu().numpy(), Wm.cpu().numpy().T
    od, oz, orho = oracle.backward(d, z, rho, ro["sigma"], ro["mu"], wn, Wt)
    sc = adjoint_scales(d, z, rho, ro["sigma"], ro["mu"], wn, Wt)
    check_components((dt.grad.cpu().numpy(), zt.grad.cpu().numpy(), rt.grad.item()), (od, oz, orho), sc, n,
                     "autograd")
    # double check with torch's finite-difference gradcheck on the same function
    def f(dd_, zz_):
        lam_, V_ = B.eigh_dpr1(dd_, zz_, rho)
        return (w * lam_).sum() + (Wm * V_).sum()
    assert torch.autograd.gradcheck(f, (cu(d).requires_grad_(True), cu(z).requires_grad_(True)), eps=1e-7,
                                    atol=1e-6, rtol=1e-5)
