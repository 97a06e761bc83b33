"""The oracle's arrowhead eigensolver (Algorithm 1's steps on the shifted arrowhead inverse)
pinned against the dense eigenproblem, the 2 x 2 closed form and the binary128 bisection of
the arrowhead's secular function."""
import numpy as np
import pytest

import oracle
from paper_1405_7537_gb300 import workloads as W

EPS = 2.0 ** -53


def dense(d, z, alpha):
    n = d.size
    A = np.zeros((n + 1, n + 1))
    A[:n, :n] = np.diag(d)
    A[:n, n] = z
    A[n, :n] = z
    A[n, n] = alpha
    return A


def test_two_by_two_closed_form():
    d, z, alpha = np.array([0.4]), np.array([0.3]), -0.7
    r = oracle.arrow_eig_all(d, z, alpha)
    m, h = (d[0] + alpha) / 2, np.hypot((d[0] - alpha) / 2, z[0])
    assert np.allclose(r["lam"], [m + h, m - h], rtol=0, atol=4 * EPS)
    A = dense(d, z, alpha)
    V = r["Vt"].T
    assert np.max(np.abs(A @ V - V * r["lam"])) <= 8 * EPS


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (5, 2), (40, 3), (300, 4)])
def test_against_dense_and_binary128(n, seed):
    d, z, alpha = W.arrowhead(n, seed)
    r = oracle.arrow_eig_all(d, z, alpha, threads=4)
    A = dense(d, z, alpha)
    nA = np.linalg.norm(A, 2)
    V = r["Vt"].T
    m = n + 1
    # interlacing lambda_0 > d_0 > lambda_1 > ... > d_{n-1} > lambda_n, residual, orthogonality
    assert np.all(r["lam"][:-1] > d) and np.all(d > r["lam"][1:])
    assert np.max(np.linalg.norm(A @ V - V * r["lam"], axis=0)) <= 8 * m * EPS * nA
    assert np.max(np.abs(V.T @ V - np.eye(m))) <= 8 * m * EPS
    assert np.max(np.abs(np.sort(np.linalg.eigvalsh(A))[::-1] - r["lam"])) <= 8 * m * EPS * nA
    # every eigenvalue and every eigenvector component to high relative accuracy
    q = oracle.quad_arrow_all(d, z, alpha, threads=4)
    lq = q["hi"] + q["lo"]
    assert np.max(np.abs(r["lam"] - lq) / np.abs(lq)) <= 16 * m * EPS
    assert np.max(np.abs(r["Vt"] - q["Vt"]) / np.abs(q["Vt"])) <= 16 * m * EPS


def test_graded_spectrum_relative_accuracy():
    """Poles graded over many decades with small weights: the eigenvalues next to the small
    poles are tiny and must still carry high relative accuracy."""
    n = 60
    d = np.sort(10.0 ** -np.arange(n, dtype=np.float64) * 0.5 + 0.0)[::-1]
    z = 1e-3 * np.sqrt(d)
    alpha = 1e-30
    r = oracle.arrow_eig_all(d, z, alpha)
    q = oracle.quad_arrow_all(d, z, alpha)
    lq = q["hi"] + q["lo"]
    assert np.max(np.abs(r["lam"] - lq) / np.abs(lq)) <= 16 * (n + 1) * EPS


@pytest.mark.parametrize("alpha", [0.3, 1e-8, -2.0])
def test_hard_spectrum_without_remedies(alpha):
    """Graded poles and weights down to 1e-10 (the hard DPR1 spectrum): every eigenvalue and
    eigenvector component within the bound of binary128 with the plain pole solves."""
    d, z, _ = W.hard(300, 1)
    r = oracle.arrow_eig_all(d, z, alpha, threads=8)
    q = oracle.quad_arrow_all(d, z, alpha, threads=8)
    lq = q["hi"] + q["lo"]
    tol = 16 * 301 * EPS
    assert np.max(np.abs(r["lam"] - lq) / np.abs(lq)) <= tol
    assert np.max(np.abs(r["Vt"] - q["Vt"]) / np.maximum(np.abs(q["Vt"]), 1e-300)) <= tol


def _clustered(n, seed):
    """Poles in tight clusters (spreads 1e-12 to 1e-3), weights over twelve decades, small
    alpha: eigenvalues next to a cluster see K_nu >> 1 at the nearer pole."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(-1, 1, max(1, n // 6))
    d = rng.choice(c, n) + rng.choice([1.0, -1.0], n) * 10.0 ** rng.uniform(-12, -3, n)
    d = np.sort(d)[::-1].copy()
    z = rng.choice([1.0, -1.0], n) * 10.0 ** rng.uniform(-12, 0, n)
    assert np.all(d[:-1] > d[1:])
    return d, z, float(10.0 ** rng.uniform(-10, -3))


def _errors(r, q):
    lq = q["hi"] + q["lo"]
    e = np.max(np.abs(r["lam"] - lq) / np.abs(lq))
    ev = np.max(np.abs(r["Vt"] - q["Vt"]) / np.maximum(np.abs(q["Vt"]), 1e-300))
    return e, ev


@pytest.mark.parametrize("seed", [0, 3])
def test_remedies_restore_accuracy_on_clustered_poles(seed):
    """K_nu >> 1 (Eq. (K0)): the plain pole solves miss the bound on clustered poles; R1 (the
    other neighbouring pole) and R2 (a non-pole shift, the arrowhead form of Eq. (gamma)) bring
    every eigenvalue and component back within 16(n+1)2^-53 of binary128."""
    d, z, alpha = _clustered(240, seed)
    n = d.size
    tol = 16 * (n + 1) * EPS
    q = oracle.quad_arrow_all(d, z, alpha, threads=8)
    plain = oracle.arrow_eig_all(d, z, alpha, threads=8, opts=oracle.default_opts(remedies=0))
    full = oracle.arrow_eig_all(d, z, alpha, threads=8)
    assert max(_errors(plain, q)) > tol
    e, ev = _errors(full, q)
    assert e <= tol and ev <= tol, (e, ev)
    flags = full["flags"] & 3
    assert np.any(flags == 1) and np.any(flags == 2)
    assert np.all((flags != 0) == (full["K_nu"] > 16.0))
    assert np.all(full["shift"][flags == 2] == -1)


def _near_singular(seed):
    # few poles with O(1) weights keep K_nu small, so the pole solve is taken as it stands and
    # only d_i + mu cancels
    rng = np.random.default_rng(seed)
    n = 3
    d = np.concatenate([rng.uniform(0.5, 1, 2), -rng.uniform(0.5, 1, 1)])
    d = np.sort(d)[::-1].copy()
    z = rng.choice([1.0, -1.0], n) * rng.uniform(0.3, 1.0, n)
    alpha = float(np.sum(z * z / d)) * (1 + 1e-13)
    return d, z, alpha


def _det_times_inverse_f(d, z, alpha):
    """det(A) = prod_j d_j * f(0), f(0) = alpha - sum_j zeta_j^2 / d_j (Schur complement of D),
    exact in rationals."""
    from fractions import Fraction as Fr
    f0 = Fr(alpha) - sum(Fr(float(zj)) ** 2 / Fr(float(dj)) for dj, zj in zip(d, z))
    det = f0
    for dj in d:
        det *= Fr(float(dj))
    return det


@pytest.mark.parametrize("seed", [1, 2, 4])
def test_near_zero_eigenvalue(seed):
    """An arrowhead with alpha next to sum zeta_j^2/d_j is nearly singular: one eigenvalue,
    between the positive and the negative poles, is far smaller than its distance to them.  The
    product of the eigenvalues is det(A) = prod_j d_j f(0) (exact in rationals), which pins that
    eigenvalue independently of any secular solve; the oracle reaches it only with the
    recompute from A^{-1} (sigma = 0), and the binary128 reference agrees."""
    from fractions import Fraction as Fr
    d, z, alpha = _near_singular(seed)
    n = d.size
    tol = 16 * (n + 1) * EPS
    q = oracle.quad_arrow_all(d, z, alpha)
    lq = q["hi"] + q["lo"]
    kz = int(np.argmin(np.abs(lq)))
    assert 0 < kz < n and d[kz] < 0 < d[kz - 1]
    others = Fr(1)
    for k in range(n + 1):
        if k != kz:
            others *= Fr(float(q["hi"][k])) + Fr(float(q["lo"][k]))
    lam_det = float(_det_times_inverse_f(d, z, alpha) / others)
    assert abs(lq[kz] - lam_det) <= 4 * EPS * abs(lam_det)
    assert abs(lam_det) < 1e-6 * min(d[kz - 1], -d[kz])
    r = oracle.arrow_eig_all(d, z, alpha)
    assert r["flags"][kz] & 4
    assert abs(r["lam"][kz] - lam_det) <= tol * abs(lam_det)
    no_zero = oracle.arrow_eig_all(d, z, alpha, opts=oracle.default_opts(remedies=1))
    assert abs(no_zero["lam"][kz] - lam_det) > tol * abs(lam_det)


def test_random_arrowheads_against_binary128():
    """Seeded random arrowheads of many shapes (uniform, clustered, graded, nearly singular;
    alpha over fourteen decades, both signs), all remedies on: every eigenvalue and component
    within 16(n+1)2^-53 of binary128."""
    rng = np.random.default_rng(2026)
    done = 0
    while done < 60:
        n = int(rng.integers(1, 60))
        kind = rng.integers(0, 4)
        if kind == 0:
            d = rng.uniform(-1, 1, n)
        elif kind == 1:
            c = rng.uniform(-1, 1, max(1, n // 6))
            d = rng.choice(c, n) + rng.choice([1.0, -1.0], n) * 10.0 ** rng.uniform(-12, -3, n)
        elif kind == 2:
            d = np.sign(rng.uniform(-1, 1, n)) * 10.0 ** rng.uniform(-10, 0, n)
        else:
            d = np.concatenate([rng.uniform(0.5, 1, n - n // 2), -rng.uniform(0.5, 1, n // 2)])
        d = np.sort(d)[::-1].copy()
        z = rng.choice([1.0, -1.0], n) * 10.0 ** rng.uniform(-12 if rng.random() < 0.5 else -2, 0, n)
        if kind == 3:
            alpha = float(np.sum(z * z / d)) * (1 + 10.0 ** rng.uniform(-14, -2))
        else:
            alpha = float(rng.choice([1.0, -1.0]) * 10.0 ** rng.uniform(-12, 2))
        if not (np.all(d[:-1] > d[1:]) and not np.any(oracle.zero_weight(z))):
            continue
        done += 1
        r = oracle.arrow_eig_all(d, z, alpha, threads=4)
        q = oracle.quad_arrow_all(d, z, alpha, threads=4)
        e, ev = _errors(r, q)
        tol = 16 * (n + 1) * EPS
        assert e <= tol and ev <= tol, (done, n, kind, alpha, e, ev)


def test_near_zero_eigenvalue_with_tiny_weights():
    """Weights 4e-5 and 2.5e-9 against poles of size 0.9: the middle eigenvalue is about
    2.4e-22.  det(A) = prod_j d_j f(0) (exact in rationals) fixes it; the binary128 reference
    (bisection on lambda itself: d_i + mu would carry 2^-113 |d_i|, about 4e-13 of lambda) and
    the oracle both reach it."""
    from fractions import Fraction as Fr
    d = np.array([float.fromhex("0x1.bf656f89b0670p-1"), float.fromhex("-0x1.c35f000a6603ap-1")])
    z = np.array([float.fromhex("0x1.4c82cd5918a9ap-15"), float.fromhex("0x1.5cb9c1af8ca60p-29")])
    alpha = float.fromhex("0x1.ee40d73254cdfp-30")
    q = oracle.quad_arrow_all(d, z, alpha)
    others = (Fr(float(q["hi"][0])) + Fr(float(q["lo"][0]))) * (Fr(float(q["hi"][2])) + Fr(float(q["lo"][2])))
    lam_det = _det_times_inverse_f(d, z, alpha) / others
    assert 1e-23 < abs(float(lam_det)) < 1e-21
    # attainable in binary128 here: 2^-113 (|alpha| + sum_j |zeta_j^2/d_j|) / |f'|, about 1e-21 of
    # lambda; the shifted d_i + mu would be about 4e-13 off
    assert abs(Fr(float(q["hi"][1])) + Fr(float(q["lo"][1])) - lam_det) <= Fr(2.0 ** -60) * abs(lam_det)
    r = oracle.arrow_eig_all(d, z, alpha)
    assert r["flags"][1] & 4
    assert abs(Fr(float(r["lam"][1])) - lam_det) <= Fr(16 * 3 * EPS) * abs(lam_det)


def test_r2_from_any_estimate():
    """R2 for the arrowhead from any starting estimate (absurd values, the interval ends,
    random points inside; the exterior intervals end at Weyl's bounds): lambda_k within
    16(n+1)2^-53 of binary128, and no cancelling difference of the pair (sigma, mu) to a
    neighbouring pole (where no binary64 shift achieves that, the shift is formed in double the
    working precision: at most 3 more solves)."""
    rng = np.random.default_rng(78)
    for case in range(12):
        n = int(rng.integers(1, 40))
        if case % 2:
            c = rng.uniform(-1, 1, max(1, n // 5))
            d = rng.choice(c, n) + rng.choice([1.0, -1.0], n) * 10.0 ** rng.uniform(-12, -3, n)
        else:
            d = rng.uniform(-1, 1, n)
        d = np.sort(d)[::-1].copy()
        if not np.all(d[:-1] > d[1:]):
            continue
        z = rng.choice([1.0, -1.0], n) * 10.0 ** rng.uniform(-6, 0, n)
        alpha = float(rng.choice([1.0, -1.0]) * 10.0 ** rng.uniform(-8, 2))
        q = oracle.quad_arrow_all(d, z, alpha)
        lq = q["hi"] + q["lo"]
        zn = float(np.sqrt(np.sum(z * z)))
        for k in rng.choice(n + 1, size=min(n + 1, 4), replace=False):
            lo = d[k] if k < n else min(d[-1], alpha) - zn
            hi = d[k - 1] if k > 0 else max(d[0], alpha) + zn
            ests = [1e293, -1e293, float("nan"), 0.0, lo, hi, lq[k]] + list(lo + (hi - lo) * rng.random(3))
            for est in ests:
                r = oracle.r2(d, z, alpha, k, est, arrow=True)
                assert 1 <= r["rounds"] <= 6
                assert abs(r["lam"] - lq[k]) <= 16 * (n + 1) * EPS * abs(lq[k]), (case, k, est, r, lq[k])
                for p in [p for p in (k - 1, k) if 0 <= p < n]:
                    dp = d[p] - r["sigma"]
                    assert 16 * abs(dp - r["mu"]) >= abs(dp) + abs(r["mu"]), (case, k, p, est, r)


def test_r2_shift_in_double_the_working_precision():
    """The arrowhead's R2 with the shift in double the working precision (Sec. 2, last sentence
    of remedy (R2)): arrowheads whose poles include a cluster of consecutive binary64 numbers
    (the adjacent-poles workload with alpha ~ U(-2, 2)) put eigenvalues within a fraction of an
    ulp of a pole with K_nu >> 1 at both of their poles; every eigenvalue and component meets
    16(n+1)2^-53 against binary128, and more than 12 of 150 problems take the branch."""
    hits = 0
    for seed in range(150):
        d, z, _ = W.adjacent_poles(seed)
        alpha = float(np.random.default_rng(seed + 500).uniform(-2, 2))
        n = d.size
        r = oracle.arrow_eig_all(d, z, alpha)
        q = oracle.quad_arrow_all(d, z, alpha)
        hits += int(np.any(r["flags"] & 8))
        e, ev = _errors(r, q)
        assert e <= 16 * (n + 1) * EPS and ev <= 16 * (n + 1) * EPS, (seed, e, ev)
    assert hits > 12


def _harsh_arrow(rng, wmax=100):
    """Arrowheads of any magnitude: the matrix scaled by 2^U(-600, 600), weights spread over up
    to 2^wmax and scaled by 2^U(-60, 60) against the poles, alpha from 2^-200 to 2^200 times them."""
    import math
    n = int(rng.integers(1, 40))
    kind = rng.integers(0, 3)
    if kind == 0:
        d = rng.uniform(-1, 1, n)
    elif kind == 1:
        c = rng.uniform(-1, 1, max(1, n // 5))
        d = rng.choice(c, n) + rng.choice([1.0, -1.0], n) * 10.0 ** rng.uniform(-12, -3, n)
    else:
        d = np.sign(rng.uniform(-1, 1, n)) * 10.0 ** rng.uniform(-12, 0, n)
    d = np.sort(d)[::-1].copy()
    z = rng.choice([1.0, -1.0], n) * 2.0 ** rng.uniform(-rng.uniform(0, wmax), 0, n) * 2.0 ** rng.uniform(-60, 60)
    alpha = float(rng.choice([1.0, -1.0]) * 2.0 ** rng.uniform(-200, 200))
    s = int(rng.integers(-600, 600))
    return np.ldexp(d, s), np.ldexp(z, s), math.ldexp(alpha, s)


def test_harsh_arrowheads():
    """Arrowheads of any magnitude meet 16(n+1)2^-53 against binary128 (components relative to
    max(|v|, 2^-1022)) or are reported as out of range -- none fails silently.  This also pins
    the binary128 reference at such scales (its square root and brackets are scale-free)."""
    rng = np.random.default_rng(606)
    ok = 0
    seen = 0
    while seen < 120:
        d, z, alpha = _harsh_arrow(rng)
        n = d.size
        if not (np.all(d[:-1] > d[1:]) and np.all(np.isfinite(d)) and np.isfinite(alpha) and not np.any(z == 0)):
            continue
        seen += 1
        try:
            r = oracle.arrow_eig_all(d, z, alpha, threads=4)
        except oracle.OracleRangeError:
            continue
        q = oracle.quad_arrow_all(d, z, alpha, threads=4)
        lq = q["hi"] + q["lo"]
        tol = 16 * (n + 1) * EPS
        assert np.max(np.abs(r["lam"] - lq) / np.abs(lq)) <= tol, seen
        assert np.max(np.abs(r["Vt"] - q["Vt"]) / np.maximum(np.abs(q["Vt"]), 2.0 ** -1022)) <= tol, seen
        ok += 1
    assert ok >= 100
