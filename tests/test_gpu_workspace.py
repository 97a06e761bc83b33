"""The bisection's stored-element buffers at the end of the workspace are optional.

The size functions include one buffer per lane group, where each group stores the elements
of the inverse of its shifted matrix (Delta_j and zeta_j^2 / Delta_j) once per eigenvalue and
every bisection step reads them.  A workspace cut to the required part makes every step
form the elements from d and zeta^2 again.  Both ways meet the bound against the oracle and
the binary128 reference (the remedies included), agree with each other within it, and a
workspace below the required part is rejected before any launch."""
import numpy as np
import pytest

import oracle
from gpu_common import eig_errors, tol
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


def cu(x):
    return torch.tensor(np.array(x, dtype=np.float64, copy=True), device="cuda")


def host(r):
    return {k: (v.cpu().numpy() if v is not None else None) for k, v in r.items()}


# The required part of the dpr1_eig workspace is a 256-byte header and 25 arrays of 8- or
# 4-byte entries per eigenpair (140 B in all), each padded to 256 B; of the arrowhead's, 92 B
# per eigenpair of the order n + 1 in 13 arrays.  16 KiB above that leaves too little for one
# buffer of 2 n doubles at the orders used here (n >= 1024).
def min_bytes(n):
    return 140 * n + 16384


def arrow_min_bytes(n):
    return 92 * (n + 1) + 16384


def test_dpr1_with_and_without_buffers(B):
    d, z, rho = W.hard(2048, 5)
    n = d.size
    res, stats = {}, {}
    for name, nbytes in (("full", B.workspace_size(n)), ("cut", min_bytes(n))):
        ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        res[name] = host(B.eig(cu(d), cu(z), rho, ws=ws))
        stats[name] = B.workspace_stats(ws)
    rng = np.random.default_rng(0)
    r2 = np.nonzero(~np.isin(res["cut"]["sigma"], d))[0]          # rows of the non-pole shift (R2)
    ks = np.unique(np.concatenate([[0, 1, n // 2, n - 1], rng.choice(n, 40, replace=False), r2[:8]]))
    r = oracle.eig_all(d, z, rho, ks=ks, threads=16)
    q = oracle.quad_all(d, z, rho, ks=ks[::4], threads=16)
    for name in res:
        ol, _, ov = eig_errors(res[name], "oracle", r, ks)
        ql, _, qv = eig_errors(res[name], "quad", q, ks[::4])
        assert max(ol.max(), ov.max(), ql.max(), qv.max()) <= tol(n), name
        assert stats[name]["solved"] == n
        assert stats[name]["r1"] > 0 and stats[name]["r2"] > 0, (name, stats[name])
    a, b = res["full"], res["cut"]
    assert np.max(np.abs(a["lam"] - b["lam"]) / np.abs(b["lam"])) <= tol(n)
    assert np.max(np.abs(a["Vt"] - b["Vt"]) / np.maximum(np.abs(b["Vt"]), 1e-300)) <= tol(n)
    # below the required part: rejected (DPR1_ERR_WORKSPACE) before any launch
    with pytest.raises(B.DPR1Error) as e:
        B.eig(cu(d), cu(z), rho, ws=torch.empty(256 * 1024, dtype=torch.uint8, device="cuda"))
    assert e.value.code == 7


def test_arrowhead_with_and_without_buffers(B):
    d, z, alpha = W.arrowhead(1500, 9)
    n = d.size
    res = {}
    for name, nbytes in (("full", int(B.lib().dpr1_arrow_workspace_size(n))), ("cut", arrow_min_bytes(n))):
        ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        res[name] = host(B.eig_arrowhead(cu(d), cu(z), alpha, ws=ws))
    rng = np.random.default_rng(1)
    ks = np.unique(np.concatenate([[0, 1, n // 2, n - 1, n], rng.choice(n + 1, 40, replace=False)]))
    r = oracle.arrow_eig_all(d, z, alpha, ks=ks, threads=16)
    t = 16 * (n + 1) * 2.0 ** -53
    for name, g in res.items():
        assert np.max(np.abs(g["lam"][ks] - r["lam"]) / np.abs(r["lam"])) <= t, name
        assert np.max(np.abs(g["Vt"][ks] - r["Vt"]) / np.maximum(np.abs(r["Vt"]), 1e-300)) <= t, name
    a, b = res["full"], res["cut"]
    assert np.max(np.abs(a["lam"] - b["lam"]) / np.abs(b["lam"])) <= t
    assert np.max(np.abs(a["Vt"] - b["Vt"]) / np.maximum(np.abs(b["Vt"]), 1e-300)) <= t
    with pytest.raises(B.DPR1Error) as e:
        B.eig_arrowhead(cu(d), cu(z), alpha, ws=torch.empty(4096, dtype=torch.uint8, device="cuda"))
    assert e.value.code == 7
