"""The remedy thresholds are readings of the paper ("K_nu >> 1" and "|lambda| << min(...)" have no
constant): T_Knu = 16 and T_zero = 64 by default.  No choice in a wide range may change whether
a result meets the bound: with T_Knu in {4, 16, 64} and T_zero in {16, 64, 256}, every
eigenvalue, shift pair and eigenvector component of the GPU path stays within relative
16 n 2^-53 of binary128 on the hard spectrum (n = 2000), on clustered poles with weights over
twelve decades, on poles at consecutive binary64 numbers, and on nearly singular problems
(the near-zero recompute).  The oracle is held to the same bound on CPU for the same settings."""
import numpy as np
import pytest

import oracle
from gpu_common import pair_minus_ref, run_gpu, tol
from paper_1405_7537_gb300 import workloads as W

torch = pytest.importorskip("torch")

SETTINGS = [(tk, tz) for tk in (4.0, 16.0, 64.0) for tz in (16.0, 64.0, 256.0)]


def clustered(seed, n=240):
    rng = np.random.default_rng(seed)
    c = rng.uniform(-1, 1, max(1, n // 6))
    d = np.sort(rng.choice(c, n) + rng.choice([1.0, -1.0], n) * 10.0 ** rng.uniform(-12, -3, n))[::-1].copy()
    z = rng.choice([1.0, -1.0], n) * 10.0 ** rng.uniform(-12, 0, n)
    assert np.all(d[:-1] > d[1:])
    return d, z, float(10.0 ** rng.uniform(-3, 3))


def near_singular(seed, n=40):
    """Poles of both signs and rho chosen so that f(0) = 1 + rho sum zeta_j^2 / d_j is about 1e-12:
    one eigenvalue lies far closer to zero than to its poles."""
    rng = np.random.default_rng(seed)
    d = np.sort(np.concatenate([rng.uniform(0.1, 1, n // 2), -rng.uniform(0.1, 1, n - n // 2)]))[::-1].copy()
    z = rng.uniform(0.3, 1.0, n) * rng.choice([1.0, -1.0], n)
    s = float(np.sum(z * z / d))
    if s >= 0:
        d = -d[::-1].copy()
        z = z[::-1].copy()
        s = float(np.sum(z * z / d))
    return d, z, -1.0 / s * (1 - 1e-12)


def cases():
    out = [("hard", W.hard(2000, 3))]
    out += [("clustered", clustered(s)) for s in (1, 2)]
    out += [("adjacent", W.adjacent_poles(s)) for s in (0, 8, 11, 13)]
    out += [("near-singular", near_singular(s)) for s in (1, 2)]
    return out


def max_errors(g, q):
    lq = q["hi"] + q["lo"]
    zp = g["lam"] != g["sigma"] + g["mu"]             # rows recomputed from A^{-1}
    e_lam = np.max(np.abs(g["lam"] - lq) / np.abs(lq))
    e_pair = np.max(np.where(zp, 0.0, pair_minus_ref(g["sigma"], g["mu"], q["hi"], q["lo"])))
    e_vec = np.max(np.abs(g["Vt"] - q["Vt"]) / np.maximum(np.abs(q["Vt"]), 1e-300))
    return e_lam, e_pair, e_vec


@pytest.fixture(scope="module")
def references():
    return [(name, d, z, rho, oracle.quad_all(d, z, rho, threads=16)) for name, (d, z, rho) in cases()]


@pytest.mark.gpu
def test_gpu_meets_bound_for_every_threshold(references):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1405_7537_gb300 import binding as B
    B.lib()
    for name, d, z, rho, q in references:
        n = d.size
        for tk, tz in SETTINGS:
            for zf in (0, 1):
                g = run_gpu(B, d, z, rho, T_Knu=tk, T_zero=tz, zero_finder=zf)
                e = max_errors(g, q)
                assert max(e) <= tol(n), (name, tk, tz, zf, e, tol(n))


def test_oracle_meets_bound_for_every_threshold():
    for name, (d, z, rho) in cases():
        if name == "hard":
            d, z, rho = W.hard(400, 3)                # the CPU suite stays short
        n = d.size
        q = oracle.quad_all(d, z, rho, threads=8)
        for tk, tz in SETTINGS:
            r = oracle.eig_all(d, z, rho, opts=oracle.default_opts(T_Knu=tk, T_zero=tz), threads=8)
            e = max_errors(r, q)
            assert max(e) <= tol(n), (name, tk, tz, e, tol(n))
