"""Seeded synthetic DPR1 problems: the paper's worked examples and the five workloads.

This module only draws inputs; it contains none of the method's arithmetic, so that
both the CUDA path and the CPU oracle can be fed from it.  Every problem is
``(d, z, rho)`` with ``d`` sorted strictly decreasingly, as the paper assumes
(Sec. 1, Eq. (order)).

Worked examples (Sec. 3):
  example1()            Example 1, n = 6, pole at zero, eigenvalue 1e-24
  example2()            Example 2, n = 4, poles 1 + 40e, ..., 1 + 10e, e = 2^-52
  example3(beta)        Example 3, n = 4, beta = 1e-7
  example4(beta)        Example 4, n = 202, beta in {1e-3, 1e-8, 1e-15}
Workloads (seeded, numpy default_rng):
  uniform(n, seed)      d ~ U(-1, 1), z ~ U(-1, 1) with |z| > 1e-3, rho = 1
  hard(n, seed)         half the poles graded 10^(-12 j/n), half U(-1, 1), gaps >= 1e-14,
                        |z| log-uniform in [1e-10, 1] with random sign, rho = 1e3
  diff(n, seed)         d ~ U(-1, 1), z ~ U(-1, 1), rho = 0.5, plus w ~ N(0,1)^n, W ~ N(0,1)^{n x n}
  batch(P, seed)        P problems, n_k log-uniform in [16, 2048], rho_k ~ U(0.1, 10)
  large(n, seed)        d ~ U(-1, 1) with 1% of adjacent gaps set to 1e-13,
                        |z| log-uniform in [1e-8, 1] with random sign, rho = 1, W ~ N(0,1)^{n x n}
"""
import numpy as np

EPS = 2.0 ** -52


def example1():
    d = np.array([1e10, 5.0, 4e-3, 0.0, -4e-3, -5.0])
    z = np.array([1e10, 1.0, 1.0, 1e-7, 1.0, 1.0])
    return d, z, 1.0


def example2():
    d = np.array([1 + 40 * EPS, 1 + 30 * EPS, 1 + 20 * EPS, 1 + 10 * EPS])
    z = np.array([1.0, 2.0, 2.0, 1.0])
    return d, z, 1.0


def example3(beta=1e-7):
    d = np.array([10.0 / 3.0, 2 + beta, 2 - beta, 1.0])
    z = np.array([2.0, beta, beta, 2.0])
    return d, z, 1.0


def example4(beta):
    """D = diag(1, 2 +- k beta (k = 1..100), 10/3), z = (2, beta, ..., beta, 2), sorted decreasingly."""
    dd = [1.0]
    for k in range(1, 101):
        dd += [2 + k * beta, 2 - k * beta]
    dd.append(10.0 / 3.0)
    d = np.array(dd)
    z = np.full(202, beta)
    z[0] = 2.0
    z[-1] = 2.0
    order = np.argsort(-d, kind="stable")
    return d[order], z[order], 1.0


def _sorted_distinct_uniform(rng, n, lo=-1.0, hi=1.0):
    d = rng.uniform(lo, hi, n)
    while True:
        d = np.sort(d)[::-1]
        dup = np.nonzero(d[:-1] == d[1:])[0]
        if dup.size == 0:
            return np.ascontiguousarray(d)
        d[dup] = rng.uniform(lo, hi, dup.size)


def uniform(n=512, seed=0):
    rng = np.random.default_rng(seed)
    d = _sorted_distinct_uniform(rng, n)
    z = rng.uniform(-1.0, 1.0, n)
    small = np.abs(z) <= 1e-3
    while small.any():
        z[small] = rng.uniform(-1.0, 1.0, int(small.sum()))
        small = np.abs(z) <= 1e-3
    return d, z, 1.0


def hard(n=16384, seed=1):
    """Half graded poles 10^(-12 j / n), j = 1..n/2 (so in [1e-6, 1)), half U(-1, 1);
    any adjacent gap below 1e-14 is removed by redrawing the uniform member."""
    rng = np.random.default_rng(seed)
    h = n // 2
    graded = 10.0 ** (-12.0 * np.arange(1, h + 1) / n)
    uni = rng.uniform(-1.0, 1.0, n - h)
    while True:
        allv = np.concatenate([graded, uni])
        src = np.concatenate([np.zeros(h, dtype=bool), np.ones(n - h, dtype=bool)])
        order = np.argsort(-allv, kind="stable")
        dv, sv = allv[order], src[order]
        bad = np.nonzero(dv[:-1] - dv[1:] < 1e-14)[0]
        if bad.size == 0:
            break
        # redraw a uniform member of every offending pair
        idx = set()
        for b in bad:
            p = b if sv[b] else b + 1
            idx.add(order[p] - h)
        idx = np.array(sorted(idx), dtype=np.int64)
        uni[idx] = rng.uniform(-1.0, 1.0, idx.size)
    mag = 10.0 ** rng.uniform(-10.0, 0.0, n)
    sign = np.where(rng.random(n) < 0.5, -1.0, 1.0)
    return np.ascontiguousarray(dv), mag * sign, 1e3


def diff(n=4096, seed=2):
    rng = np.random.default_rng(seed)
    d = _sorted_distinct_uniform(rng, n)
    z = rng.uniform(-1.0, 1.0, n)
    w = rng.standard_normal(n)
    W = rng.standard_normal((n, n))
    return d, z, 0.5, w, W


def batch_sizes(P=4096, seed=3, nmin=16, nmax=2048):
    rng = np.random.default_rng(seed)
    return np.rint(np.exp(rng.uniform(np.log(nmin), np.log(nmax), P))).astype(np.int64), rng


def batch(P=4096, seed=3, nmin=16, nmax=2048):
    """Returns (offs[P+1], d, z, rho[P]) with problem p in d[offs[p]:offs[p+1]]."""
    sizes, rng = batch_sizes(P, seed, nmin, nmax)
    offs = np.zeros(P + 1, dtype=np.int64)
    offs[1:] = np.cumsum(sizes)
    d = np.empty(offs[-1])
    z = np.empty(offs[-1])
    rho = np.empty(P)
    for p in range(P):
        n = int(sizes[p])
        d[offs[p]:offs[p + 1]] = _sorted_distinct_uniform(rng, n)
        z[offs[p]:offs[p + 1]] = rng.uniform(-1.0, 1.0, n)
        rho[p] = rng.uniform(0.1, 10.0)
    return offs, d, z, rho


def large(n=32768, seed=4, with_W=True):
    """1% of the adjacent gaps are set to 1e-13 by moving d_{j+1} to d_j - 1e-13
    (skipped where that would reach d_{j+2} or touch an already tightened pair)."""
    rng = np.random.default_rng(seed)
    d = _sorted_distinct_uniform(rng, n)
    m = n // 100
    picks = rng.choice(n - 2, size=m, replace=False)
    used = np.zeros(n, dtype=bool)
    for j in np.sort(picks):
        if used[j] or used[j + 1]:
            continue
        nd = d[j] - 1e-13
        if nd > d[j + 2] and nd < d[j]:
            d[j + 1] = nd
            used[j] = used[j + 1] = True
    mag = 10.0 ** rng.uniform(-8.0, 0.0, n)
    sign = np.where(rng.random(n) < 0.5, -1.0, 1.0)
    W = rng.standard_normal((n, n)) if with_W else None
    return d, mag * sign, 1.0, W


def hermitian(n=16384, seed=1, base="hard"):
    """A complex Hermitian DPR1 problem: the real workload `base` (its d, rho and |z|) with a
    phase exp(i theta_j), theta_j ~ U(0, 2 pi) from an independent stream, on every z_j."""
    d, z, rho = (hard if base == "hard" else uniform)(n, seed)
    rng = np.random.default_rng(seed + 1000)
    theta = rng.uniform(0.0, 2.0 * np.pi, n)
    return d, np.abs(z) * np.exp(1j * theta), rho


def tridiagonal(n=4096, seed=5):
    """A symmetric tridiagonal matrix: diagonal a and off-diagonal b ~ U(-1, 1)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, n), rng.uniform(-1.0, 1.0, max(n - 1, 0))


def wilkinson(n=21):
    """Wilkinson's W_n^+ (n = 2m + 1): diagonal |m - j|, j = 0..n-1, off-diagonal ones."""
    m = (n - 1) // 2
    return np.abs(m - np.arange(n)).astype(np.float64), np.ones(n - 1)


def glued_wilkinson(n=21, copies=4, glue=1e-10):
    """`copies` Wilkinson W_n^+ blocks coupled by off-diagonal entries `glue`: clusters of
    very close eigenvalues, a hard case for divide and conquer."""
    a0, b0 = wilkinson(n)
    a = np.tile(a0, copies)
    b = np.concatenate([np.concatenate([b0, [glue]]) for _ in range(copies)])[:-1]
    return a, b


def adjacent_poles(seed):
    """Poles at consecutive binary64 numbers: a cluster of 3 to 5 of them in [0.5, 1) with weights
    +-10^U(-30, -15), except one of size sqrt(c 2^-52), c ~ U(0.2, 4), which puts the zero of the
    rest of the secular function inside the cluster; 1 to 3 poles U(-1, 0.4) and as many
    U(1.2, 2) with weights +-U(0.1, 1); rho = 10^U(-1, 1).  Eigenvalues then lie within a fraction
    of an ulp of a pole, and their neighbours hug the poles more closely still (K_nu >> 1 at
    both poles), so that no binary64 number lies between such an eigenvalue and its pole."""
    rng = np.random.default_rng(seed)
    eps = 2.0 ** -52
    m = int(rng.integers(3, 6))
    q = [float(rng.uniform(0.5, 1.0))]
    for _ in range(m - 1):
        q.append(float(np.nextafter(q[-1], 2.0)))
    nfar = int(rng.integers(1, 4))
    far = list(rng.uniform(-1.0, 0.4, nfar)) + list(rng.uniform(1.2, 2.0, nfar))
    d = np.array(sorted(q + far, reverse=True))
    inq = np.isin(d, q)
    z = np.where(inq, 10.0 ** rng.uniform(-30.0, -15.0, d.size), rng.uniform(0.1, 1.0, d.size))
    z *= np.where(rng.random(d.size) < 0.5, 1.0, -1.0)
    z[np.flatnonzero(inq)[rng.integers(0, m)]] = np.sqrt(eps * rng.uniform(0.2, 4.0))
    return d, z, float(10.0 ** rng.uniform(-1.0, 1.0))


def screen_stress(seed):
    """Problems that put the binary32 screen of the bisection at its limits (kind = seed % 3):
    0: clusters of poles at relative spacing 2^-s, s ~ U{18..22}, weights +-10^U(-8, 0) and
       rho = 10^U(-2, 2);
    1: a cluster of tiny poles 2^-70 (1 + j 2^-9) (differences near 2^-79) among poles of size
       about 1, weights +-2^U(-40, -10): the stored differences and weights over differences
       reach both ends of the screen's binary32 range (2^-80 and 2^60);
    2: weights +-2^U(-31, -27) next to O(1) ones with rho = 1: eigenvalues within about 2^-58 of
       their poles, so |nu| lies on both sides of the screen's limit 2^60."""
    rng = np.random.default_rng(seed)
    kind = seed % 3
    if kind == 0:
        n = int(rng.integers(200, 600))
        cs = rng.uniform(-1.0, 1.0, max(1, n // 20))
        d = []
        while len(d) < n:
            c = float(rng.choice(cs))
            s = int(rng.integers(18, 23))
            m = int(rng.integers(2, 12))
            d += [c * (1.0 + k * 2.0 ** -s) for k in range(m)]
        d = np.unique(np.array(d[:n]))[::-1].copy()
        z = rng.choice([1.0, -1.0], d.size) * 10.0 ** rng.uniform(-8.0, 0.0, d.size)
        return d, z, float(10.0 ** rng.uniform(-2.0, 2.0))
    if kind == 1:
        m = int(rng.integers(20, 60))
        tiny = 2.0 ** -70 * (1.0 + np.arange(m) * 2.0 ** -9)
        big = rng.uniform(-1.0, 1.0, int(rng.integers(40, 120)))
        d = np.unique(np.concatenate([tiny, big]))[::-1].copy()
        z = rng.choice([1.0, -1.0], d.size) * 2.0 ** rng.uniform(-40.0, -10.0, d.size)
        return d, z, 1.0
    n = int(rng.integers(100, 400))
    d = _sorted_distinct_uniform(rng, n)
    small = rng.random(n) < 0.5
    z = np.where(small, 2.0 ** rng.uniform(-31.0, -27.0, n), rng.uniform(0.1, 1.0, n))
    z *= rng.choice([1.0, -1.0], n)
    return d, z, 1.0


def arrowhead(n=16384, seed=6):
    """A real symmetric arrowhead [diag(d) z; z^T alpha] of order n + 1: d ~ U(-1, 1) sorted
    decreasing and distinct, z ~ U(-1, 1) redrawn while |z| <= 1e-3, alpha ~ U(-1, 1)."""
    d, z, _ = uniform(n, seed)
    rng = np.random.default_rng(seed + 2000)
    return d, z, float(rng.uniform(-1.0, 1.0))
