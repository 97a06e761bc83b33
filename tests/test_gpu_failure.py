"""Failure detection on the GPU without a fault: a solve that reaches its iteration cap stops,
records DPR1_ERR_NOT_CONVERGED in the workspace's status word and returns; dpr1_stream_status
reports it promptly and clears it, and the next call on the same workspace with the default cap
is correct.  Every wait in the kernels is a bounded loop, so a tiny cap (3 bisection steps, or
1 + 1 evaluations of the accelerated solve) makes every eigenvalue give up early -- nothing spins,
traps or faults."""
import time

import numpy as np
import pytest

import oracle
from paper_1405_7537_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NOT_CONVERGED = 5
U53 = 2.0 ** -53


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1405_7537_gb300 import binding
    binding.lib()
    return binding


def cu(x):
    return torch.tensor(np.array(x, dtype=np.float64, copy=True), device="cuda")


def rel(a, b):
    return np.abs(a - b) / np.maximum(np.abs(b), 1e-300)


CAPS = [(0, 3), (1, 1)]   # (zero_finder, max_bisect): bisection, accelerated solve


@pytest.mark.parametrize("zf,cap", CAPS)
def test_cap_single_problem_then_default(B, zf, cap):
    d, z, rho = W.uniform(512, 0)
    n = d.size
    ws = B.workspace(n)
    t0 = time.monotonic()
    with pytest.raises(B.DPR1Error) as e:
        B.eig(cu(d), cu(z), rho, options=B.default_options(zero_finder=zf, max_bisect=cap), ws=ws)
    assert e.value.code == NOT_CONVERGED
    assert time.monotonic() - t0 < 30.0
    # dpr1_stream_status cleared the word: nothing is pending on this workspace
    assert B.stream_status(ws) == 0
    # the same workspace, default cap: correct against the oracle
    r = B.eig(cu(d), cu(z), rho, options=B.default_options(zero_finder=zf), ws=ws)
    ref = oracle.eig_all(d, z, rho, threads=16)
    tol = 16 * n * U53
    assert np.max(rel(r["lam"].cpu().numpy(), ref["lam"])) <= tol
    assert np.max(rel(r["Vt"].cpu().numpy(), ref["Vt"])) <= tol


@pytest.mark.parametrize("zf,cap", CAPS)
def test_cap_batched_then_default(B, zf, cap):
    offs, d, z, rho = W.batch(64, 7, nmin=16, nmax=300)
    bt = B.Batch(np.diff(offs))
    dt, zt, rt = cu(d), cu(z), cu(rho)
    t0 = time.monotonic()
    with pytest.raises(B.DPR1Error) as e:
        bt.solve(dt, zt, rt, options=B.default_options(zero_finder=zf, max_bisect=cap), check=True)
    assert e.value.code == NOT_CONVERGED
    assert time.monotonic() - t0 < 30.0
    assert B.stream_status(bt.ws) == 0
    bt.solve(dt, zt, rt, options=B.default_options(zero_finder=zf), check=True)
    for p in (0, 17, 63):
        a, b_ = int(offs[p]), int(offs[p + 1])
        lam, Vt = bt.block(p)
        ref = oracle.eig_all(d[a:b_], z[a:b_], float(rho[p]), threads=16)
        tol = 16 * (b_ - a) * U53
        assert np.max(rel(lam.cpu().numpy(), ref["lam"])) <= tol
        assert np.max(rel(Vt.cpu().numpy(), ref["Vt"])) <= tol


@pytest.mark.parametrize("zf,cap", CAPS)
def test_cap_arrowhead_then_default(B, zf, cap):
    d, z, alpha = W.arrowhead(300, 8)
    n = d.size
    ws = B.arrow_workspace(n)
    t0 = time.monotonic()
    with pytest.raises(B.DPR1Error) as e:
        B.eig_arrowhead(cu(d), cu(z), alpha, options=B.default_options(zero_finder=zf, max_bisect=cap), ws=ws)
    assert e.value.code == NOT_CONVERGED
    assert time.monotonic() - t0 < 30.0
    assert B.stream_status(ws) == 0
    r = B.eig_arrowhead(cu(d), cu(z), alpha, options=B.default_options(zero_finder=zf), ws=ws)
    ref = oracle.arrow_eig_all(d, z, alpha, threads=16)
    tol = 16 * (n + 1) * U53
    assert np.max(rel(r["lam"].cpu().numpy(), ref["lam"])) <= tol
    assert np.max(rel(r["Vt"].cpu().numpy(), ref["Vt"])) <= tol
