"""dpr1_eig_noalloc: the entry point for callers that cannot allocate device memory.

It runs the same launch sequence as dpr1_eig on a static scratch array inside the
library.  Checked through the C ABI against dpr1_eig (which uses a caller workspace) on
two calls in a row -- the array keeps the previous call's contents, so the second call
must not depend on them -- and for the size limit."""
import ctypes

import numpy as np
import pytest

from paper_1405_7537_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U53 = 2.0 ** -53


def test_noalloc_matches_dpr1_eig_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1405_7537_gb300 import binding as B
    L = B.lib()
    vp = ctypes.c_void_p
    L.dpr1_eig_noalloc.argtypes = [ctypes.c_int64, vp, vp, ctypes.c_double, vp, vp, ctypes.c_int64, vp, vp, vp, vp,
                                   ctypes.c_int, vp]
    L.dpr1_eig_noalloc.restype = ctypes.c_int
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # two different problems in a row (the second smaller, so stale entries of the first
    # remain in the static array), then the maximum size
    cases = [W.hard(1500, 3), W.uniform(700, 4), W.uniform(4096, 5)]
    for d, z, rho in cases:
        n = d.size
        dt = torch.tensor(np.array(d), device="cuda")
        zt = torch.tensor(np.array(z), device="cuda")
        ref = B.eig(dt, zt, rho)
        lam = torch.empty(n, dtype=torch.float64, device="cuda")
        Vt = torch.empty((n, n), dtype=torch.float64, device="cuda")
        sig = torch.empty(n, dtype=torch.float64, device="cuda")
        mu = torch.empty(n, dtype=torch.float64, device="cuda")
        xn = torch.empty(n, dtype=torch.float64, device="cuda")
        rc = L.dpr1_eig_noalloc(n, dt.data_ptr(), zt.data_ptr(), rho, lam.data_ptr(), Vt.data_ptr(), n,
                                sig.data_ptr(), mu.data_ptr(), xn.data_ptr(), None, 1, stream)
        assert rc == 0
        torch.cuda.synchronize()
        tol = 16 * n * U53
        l0, l1 = ref["lam"].cpu().numpy(), lam.cpu().numpy()
        V0, V1 = ref["Vt"].cpu().numpy(), Vt.cpu().numpy()
        assert np.max(np.abs(l1 - l0) / np.abs(l0)) <= tol
        assert np.max(np.abs(V1 - V0) / np.maximum(np.abs(V0), 1e-300)) <= tol
        # shifts: the same poles; a non-pole shift (remedy R2) is the computed eigenvalue.  The
        # static array leaves no room for the bisection's stored-element buffers, so this call
        # forms the secular sums at every evaluation -- a different grouping of the terms from
        # dpr1_eig with a full workspace -- and a non-pole shift may differ in its last bits
        s0, s1 = ref["sigma"].cpu().numpy(), sig.cpu().numpy()
        pole0, pole1 = np.isin(s0, d), np.isin(s1, d)
        assert np.array_equal(pole0, pole1) and np.array_equal(s0[pole0], s1[pole1])
        assert np.max(np.abs(s1 - s0) / np.abs(s0), initial=0.0) <= tol
    # beyond the static scratch: rejected before any launch
    n = 4097
    big = torch.zeros(n, dtype=torch.float64, device="cuda")
    rc = L.dpr1_eig_noalloc(n, big.data_ptr(), big.data_ptr(), 1.0, big.data_ptr(), None, 0, None, None, None, None,
                            1, stream)
    assert rc == 1
