"""The seeded input generators (host code, no GPU) keep the recipes the tests and the bench are
quoted on: strictly decreasing poles, the stated gaps and weight ranges, and the same arrays for
the same seed."""
import numpy as np

from paper_1405_7537_gb300 import workloads as W


def strictly_decreasing(d):
    return bool(np.all(d[:-1] > d[1:]))


def test_uniform():
    d, z, rho = W.uniform(4096, 0)
    assert strictly_decreasing(d) and np.all(np.abs(d) < 1.0)
    assert np.all(np.abs(z) > 1e-3) and np.all(np.abs(z) < 1.0)
    assert rho == 1.0
    d2, z2, _ = W.uniform(4096, 0)
    assert np.array_equal(d, d2) and np.array_equal(z, z2)


def test_hard_spectrum():
    n = 16384
    d, z, rho = W.hard(n, 1)
    assert d.size == n and strictly_decreasing(d)
    assert np.min(d[:-1] - d[1:]) >= 1e-14
    # half the poles are the graded values 10^(-12 j / n), j = 1..n/2
    graded = 10.0 ** (-12.0 * np.arange(1, n // 2 + 1) / n)
    assert np.all(np.isin(graded, d))
    assert np.all(np.abs(z) >= 1e-10) and np.all(np.abs(z) <= 1.0)
    assert 0.45 < np.mean(z > 0) < 0.55
    assert rho == 1e3
    d2, z2, _ = W.hard(n, 1)
    assert np.array_equal(d, d2) and np.array_equal(z, z2)
    d3, _, _ = W.hard(n, 2)
    assert not np.array_equal(d, d3)


def test_diff():
    n = 512
    d, z, rho, w, Wm = W.diff(n, 2)
    assert strictly_decreasing(d) and rho == 0.5
    assert z.shape == (n,) and w.shape == (n,) and Wm.shape == (n, n)


def test_batch():
    offs, d, z, rho = W.batch(P=256, seed=3)
    sizes = np.diff(offs)
    assert offs[0] == 0 and offs[-1] == d.size == z.size
    assert sizes.min() >= 16 and sizes.max() <= 2048
    assert np.all((rho >= 0.1) & (rho <= 10.0))
    for p in range(sizes.size):
        assert strictly_decreasing(d[offs[p]:offs[p + 1]])
    # the sizes are those of batch_sizes with the same seed
    s2, _ = W.batch_sizes(P=256, seed=3)
    assert np.array_equal(sizes, s2)


def test_large():
    n = 32768
    d, z, rho, Wm = W.large(n, 4, with_W=False)
    assert Wm is None and rho == 1.0
    assert strictly_decreasing(d)
    gaps = d[:-1] - d[1:]
    tight = np.sum(np.abs(gaps - 1e-13) < 1e-15)
    # up to 1% of the gaps are tightened to 1e-13 (a pick is skipped when its pair is taken)
    assert 0.5 * (n // 100) <= tight <= n // 100
    assert np.all(np.abs(z) >= 1e-8) and np.all(np.abs(z) <= 1.0)


def test_hermitian_phases():
    d, zc, rho = W.hermitian(1024, 1)
    dr, zr, rr = W.hard(1024, 1)
    assert np.array_equal(d, dr) and rho == rr
    assert np.allclose(np.abs(zc), np.abs(zr), rtol=1e-15, atol=0.0)
