"""Pins of the CPU oracle against values fixed by the paper and by mathematics.

Nothing here calls the CUDA library.  Each pin is chosen so that a plausible slip
in the oracle (a dropped term, a wrong sign or index, a transposed operand, a
missing double-double step, a missing remedy) fails at least one of them:

* double-double add/mul/div against exact rationals;
* the binary128 reference against an independent mpmath bisection;
* the n = 2 closed form;
* Examples 1-3 (printed eigenvalues, eigenvectors and the corner element b);
* Example 4 / Table 1 (orthogonality and residual measures, with and without
  double-double, and the double-double counts);
* interlacing, trace, orthogonality and residual invariants;
* accuracy of every eigenvalue and eigenvector component against binary128
  within 16 n 2^-53 on seeded workloads, with and without the remedies;
* the adjoint against finite differences, the dense eigen-decomposition
  adjoint and the trace identities.
"""
from fractions import Fraction as Fr

import math

import numpy as np
import pytest

import oracle
from adjoint_scale import adjoint_scales, central_differences, componentwise
from conftest import read_golden
from paper_1405_7537_gb300 import workloads as W

U53 = 2.0 ** -53


def tol(n):
    return 16 * n * U53


def fr_rel(a_parts, b_parts):
    """|sum(a) - sum(b)| / |sum(b)| computed exactly."""
    a = sum(Fr(x) for x in a_parts)
    b = sum(Fr(x) for x in b_parts)
    return abs(float((a - b) / b)) if b != 0 else abs(float(a))


# ---------------------------------------------------------------- double-double
def _rand_dd(rng, scale_exp=0):
    hi = rng.uniform(0.5, 1.0) * 2.0 ** rng.integers(-40 + scale_exp, 40 + scale_exp)
    hi *= rng.choice([-1.0, 1.0])
    lo = rng.uniform(-0.5, 0.5) * np.spacing(abs(hi))
    s = hi + lo
    return (s, lo - (s - hi))


@pytest.mark.parametrize("op", ["add", "mul", "div"])
def test_dd_ops_against_exact_rationals(op):
    """Sec. 2.3: double the working precision; each dd operation must be accurate to ~2^-100."""
    rng = np.random.default_rng(7)
    cases = [_rand_dd(rng) for _ in range(400)]
    worst = 0.0
    for t in range(0, 400, 2):
        a, b = cases[t], cases[t + 1]
        if op == "add" and t % 8 == 0:
            # heavy cancellation: b = -a + small
            b = (-a[0], rng.uniform(-0.5, 0.5) * np.spacing(abs(a[0])) * 2.0 ** -int(rng.integers(1, 30)))
        A, B = Fr(a[0]) + Fr(a[1]), Fr(b[0]) + Fr(b[1])
        exact = {"add": A + B, "mul": A * B, "div": A / B}[op]
        r = oracle.dd_op(op, a, b)
        got = Fr(r[0]) + Fr(r[1])
        if exact == 0:
            assert got == 0
            continue
        err = abs(float((got - exact) / exact))
        worst = max(worst, err)
    assert worst <= 2.0 ** -100, worst


# ---------------------------------------------------------------- binary128 reference
def _mp_eigpair(d, z, rho, k, mp):
    """Brute-force bisection of f(lambda) in mpmath inside the interlacing interval."""
    n = len(d)
    D = [mp.mpf(x) for x in d]
    Z = [mp.mpf(x) for x in z]
    R = mp.mpf(rho)

    def f(lam):
        return 1 + R * sum(Z[j] ** 2 / (D[j] - lam) for j in range(n))

    if k == 0:
        lo, hi = D[0], D[0] + 2 * R * sum(x * x for x in Z)
    else:
        lo, hi = D[k], D[k - 1]
    for _ in range(400):
        mid = (lo + hi) / 2
        if f(mid) < 0:
            lo = mid
        else:
            hi = mid
    lam = (lo + hi) / 2
    x = [Z[j] / (D[j] - lam) for j in range(n)]
    nx = mp.sqrt(sum(t * t for t in x))
    return lam, [t / nx for t in x]


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (3, 2), (5, 3), (6, 4)])
def test_quad_reference_against_mpmath(n, seed):
    mp = pytest.importorskip("mpmath").mp
    mp.dps = 60
    rng = np.random.default_rng(seed)
    d = np.sort(rng.uniform(-3, 3, n))[::-1]
    z = rng.uniform(-2, 2, n)
    rho = float(rng.uniform(0.2, 3))
    for k in range(n):
        hi, lo, v = oracle.quad_eig(d, z, rho, k)
        lam, vm = _mp_eigpair(d, z, rho, k, mp)
        assert abs((mp.mpf(hi) + mp.mpf(lo) - lam) / lam) < 1e-30
        for j in range(n):
            assert abs(v[j] - float(vm[j])) <= 2 * U53 * abs(float(vm[j])) + 1e-300


def test_n2_closed_form():
    """n = 2: lambda = (t +- sqrt((d1 - d2 + rho(z1^2 - z2^2))^2 + 4 rho^2 z1^2 z2^2)) / 2."""
    mp = pytest.importorskip("mpmath").mp
    mp.dps = 50
    rng = np.random.default_rng(11)
    for _ in range(40):
        d = np.sort(rng.uniform(-2, 2, 2))[::-1]
        z = rng.uniform(-1, 1, 2) * 10.0 ** rng.uniform(-6, 0, 2)
        rho = float(10.0 ** rng.uniform(-2, 2))
        d1, d2, z1, z2, r = (mp.mpf(float(x)) for x in (d[0], d[1], z[0], z[1], rho))
        t = d1 + d2 + r * (z1 ** 2 + z2 ** 2)
        s = mp.sqrt((d1 - d2 + r * (z1 ** 2 - z2 ** 2)) ** 2 + 4 * r ** 2 * z1 ** 2 * z2 ** 2)
        l1 = (t + s) / 2
        det = d1 * d2 + r * (z1 ** 2 * d2 + z2 ** 2 * d1)
        l2 = det / l1 if abs(l1) > abs((t - s) / 2) else (t - s) / 2
        for k, lex in enumerate((l1, l2)):
            lam, v, info = oracle.dpr1eig(d, z, rho, k)
            assert abs((mp.mpf(info["sigma"]) + mp.mpf(info["mu"]) - lex) / lex) <= tol(2)
            x = [mp.mpf(float(z[j])) / (mp.mpf(float(d[j])) - lex) for j in range(2)]
            nx = mp.sqrt(x[0] ** 2 + x[1] ** 2)
            for j in range(2):
                assert abs(v[j] - float(x[j] / nx)) <= tol(2) * abs(float(x[j] / nx))


# ---------------------------------------------------------------- worked examples
def test_example1_printed_values():
    g = read_golden("example1.txt")
    lam_p = [float(v[0]) for k, v in g if k == "lambda"]
    v4_p = np.array([float(v[0]) for k, v in g if k == "v4"])
    d, z, rho = W.example1()
    for k in range(6):
        lam, v, info = oracle.dpr1eig(d, z, rho, k)
        assert abs(lam - lam_p[k]) <= 1e-15 * abs(lam_p[k]), (k, lam, lam_p[k])
        h, l, vq = oracle.quad_eig(d, z, rho, k)
        assert abs(h - lam_p[k]) <= 1e-15 * abs(lam_p[k])
        if k == 3:
            assert np.all(np.abs(v - v4_p) <= 1e-15 * np.abs(v4_p))
            assert np.all(np.abs(vq - v4_p) <= 1e-15 * np.abs(v4_p))


def test_example2_32_digit_pairs():
    mp = pytest.importorskip("mpmath").mp
    mp.dps = 50
    g = read_golden("example2.txt")
    lam32 = [mp.mpf(v[0]) for k, v in g if k == "lambda32"]
    lam64 = [(int(v[0]), int(v[1])) for k, v in g if k == "lambda64"]
    pair_ks = [int(x) - 1 for k, v in g if k == "pair32" for x in v]
    d, z, rho = W.example2()
    e = 2.0 ** -52
    for k in range(4):
        lam, v, info = oracle.dpr1eig(d, z, rho, k)
        # binary64 result printed by the paper for dpr1eig (within one unit in the last place)
        base, mult = lam64[k]
        assert abs(lam - (base + mult * e)) <= np.spacing(lam)
        # binary128 reference reproduces the 32 printed digits
        h, l, _ = oracle.quad_eig(d, z, rho, k)
        assert abs((mp.mpf(h) + mp.mpf(l) - lam32[k]) / lam32[k]) < 1e-31
        if k in pair_ks:
            s = mp.mpf(info["sigma"]) + mp.mpf(info["mu"])
            assert abs((s - lam32[k]) / lam32[k]) < 2e-31


def test_example3_corner_element_and_vector():
    g = dict((k, v) for k, v in read_golden("example3.txt") if k.startswith("b_"))
    v2_p = np.array([float(v[0]) for k, v in read_golden("example3.txt") if k == "v2"])
    d, z, rho = W.example3()
    lam, v, info = oracle.dpr1eig(d, z, rho, 1, oracle.default_opts(dd_mode=2))
    assert info["first_shift"] == 1 and info["shift"] == 1
    assert abs(info["b"] - float(g["b_dd"][0])) <= 1e-16 * abs(info["b"])
    assert np.all(np.abs(v - v2_p) <= 2e-16 * np.abs(v2_p) + 1e-17)
    lam_nd, v_nd, info_nd = oracle.dpr1eig(d, z, rho, 1, oracle.default_opts(dd_mode=0))
    assert abs(info_nd["b"] - float(g["b_fp64"][0])) <= 2 * np.spacing(info_nd["b"])
    # without double-double the eigenvector loses about 7 digits (kappa_nu ~ 1e7)
    assert np.max(np.abs(v_nd - v2_p) / np.abs(v2_p)) > 1e-11
    # the threshold mode decides to use double-double here
    _, _, info_thr = oracle.dpr1eig(d, z, rho, 1, oracle.default_opts(dd_mode=1))
    assert info_thr["used_dd"] == 1


def _measures(d, z, rho, lam, Vt):
    n = d.size
    A = np.diag(d) + rho * np.outer(z, z)
    V = Vt.T
    O = np.max(np.linalg.norm(V.T @ V - np.eye(n), axis=0)) / (n * 2.0 ** -52)
    R = np.max(np.linalg.norm(A @ V - V * lam, axis=0)) / (n * 2.0 ** -52 * np.linalg.norm(A, 2))
    return O, R


def test_example4_table1():
    rows = read_golden("example4_table1.txt")
    for beta_s, vals in rows:
        beta = float(beta_s)
        O_nd_p, O_dd_p, R_dd_p, dv_p, n_dd_p = (float(x) for x in vals)
        d, z, rho = W.example4(beta)
        r = oracle.eig_all(d, z, rho)
        O, R = _measures(d, z, rho, r["lam"], r["Vt"])
        assert O < 0.2 and R < 0.2, (beta, O, R)
        rn = oracle.eig_all(d, z, rho, oracle.default_opts(dd_mode=0))
        On, _ = _measures(d, z, rho, rn["lam"], rn["Vt"])
        assert O_nd_p / 2 < On < O_nd_p * 2, (beta, On, O_nd_p)
        dv = np.max(np.abs(rn["Vt"] - r["Vt"]) / np.abs(r["Vt"]))
        assert dv_p / 1.5 < dv < dv_p * 1.5, (beta, dv, dv_p)
        rt = oracle.eig_all(d, z, rho, oracle.default_opts(dd_mode=1))
        assert int(np.sum((rt["flags"] >> 3) & 1)) == int(n_dd_p)


# ---------------------------------------------------------------- accuracy against binary128
def _check_against_quad(d, z, rho, opts=None, ks=None, threads=8):
    n = d.size
    r = oracle.eig_all(d, z, rho, opts, ks=ks, threads=threads)
    q = oracle.quad_all(d, z, rho, ks=ks, threads=threads)
    e_pair = max(fr_rel([s, m], [h, l]) for s, m, h, l in zip(r["sigma"], r["mu"], q["hi"], q["lo"]))
    e_lam = max(fr_rel([a], [h, l]) for a, h, l in zip(r["lam"], q["hi"], q["lo"]))
    e_vec = np.max(np.abs(r["Vt"] - q["Vt"]) / np.maximum(np.abs(q["Vt"]), 1e-300))
    return r, e_pair, e_lam, e_vec


@pytest.mark.parametrize("gen,n,seed", [("uniform", 64, 0), ("uniform", 300, 5), ("hard", 256, 1),
                                        ("hard", 512, 9), ("large", 400, 4)])
def test_all_components_within_bound_of_binary128(gen, n, seed):
    if gen == "large":
        d, z, rho, _ = W.large(n, seed, with_W=False)
    else:
        d, z, rho = getattr(W, gen)(n, seed)
    r, e_pair, e_lam, e_vec = _check_against_quad(d, z, rho)
    assert e_pair <= tol(n) and e_lam <= tol(n) and e_vec <= tol(n), (e_pair, e_lam, e_vec, tol(n))


def _pair_err(lam, info, h, l):
    if info["zero_path"]:
        return fr_rel([lam], [h, l])
    return fr_rel([info["sigma"], info["mu"]], [h, l])


# (d, z, rho, k, remedy expected): lambda_k's nearest pole has K_nu >> 1
REMEDY_CASES = [
    # k = 1: lambda_1 = 1e3-ish far above d_1 while lambda_2 hugs d_1 -> only R2 is possible
    ([1.0, 0.0, -1.0], [1e-4, 1.0, 1.0], 1e3, 0, 2),
    # interior eigenvalue whose nearer pole is hugged from the other side; the other pole works (R1)
    ([0.11277631052444313, -8.602631907875167e-05, -0.001417447836908407, -0.36653735387592706],
     [-0.000393655760729729, 0.19487579738160088, -0.0009440805320101989, 0.3107416582357829],
     4.915271596018554, 3, 1),
]


@pytest.mark.parametrize("case", REMEDY_CASES)
def test_remedies_fix_large_K_nu(case):
    d, z, rho, k, rem = case
    d, z = np.array(d), np.array(z)
    n = d.size
    h, l, vq = oracle.quad_eig(d, z, rho, k)
    lam0, v0, i0 = oracle.dpr1eig(d, z, rho, k, oracle.default_opts(remedies=2))
    e0 = max(_pair_err(lam0, i0, h, l), np.max(np.abs(v0 - vq) / np.abs(vq)))
    assert i0["K_nu"] > 16 and e0 > tol(n)         # without R1/R2 the bound is missed
    lam1, v1, i1 = oracle.dpr1eig(d, z, rho, k)
    e1 = max(_pair_err(lam1, i1, h, l), np.max(np.abs(v1 - vq) / np.abs(vq)))
    assert i1["remedy"] == rem and e1 <= tol(n)


def test_other_pole_not_taken_when_its_eigenvector_formula_cancels():
    """lambda_2 lies 1.3e-4 from d_2 and 0.11 from d_1; K_nu at d_2 is 2e7 because lambda_3
    hugs d_2 from below.  At d_1 K_nu = 1, but x_2 = zeta_2 / ((d_2 - d_1) - mu) cancels by
    0.11 / 1.3e-4, so R1 would lose ~900 ulps in v_2[2]; R2 keeps every component."""
    d = np.array([0.11194228395448386, 0.0014323237359187434, -0.0012032856196724088,
                  -0.0020923462965340453, -0.021922411152150944])
    z = np.array([0.23955894133815114, 3.595254856845261e-07, 3.0836878960918116e-08,
                  0.04739602608944186, -0.004540811583072913])
    rho, k, n = 10.417883351109507, 1, 5
    h, l, vq = oracle.quad_eig(d, z, rho, k)
    lam, v, info = oracle.dpr1eig(d, z, rho, k)
    assert info["K_nu"] > 1e6 and info["remedy"] == 2
    assert max(_pair_err(lam, info, h, l), np.max(np.abs(v - vq) / np.abs(vq))) <= tol(n)


def test_hard_spectrum_uses_both_remedies():
    d, z, rho = W.hard(256, 1)
    r, e_pair, e_lam, e_vec = _check_against_quad(d, z, rho)
    assert e_vec <= tol(256)
    fl = r["flags"] & 3
    assert np.sum(fl == 1) > 0 and np.sum(fl == 2) > 0


def test_double_double_keeps_example4_within_bound():
    d, z, rho = W.example4(1e-8)
    _, _, _, e_vec = _check_against_quad(d, z, rho)
    assert e_vec <= tol(d.size)


def _near_zero_problem():
    d = np.array([3.0, 1.5, -1.0, -2.5])
    z = np.array([1.0, 1.0, 2.0, 1.0])
    lam_star = 1e-13
    s = sum(z[j] ** 2 / (d[j] - lam_star) for j in range(4))
    return d, z, -1.0 / s


def test_near_zero_eigenvalue_path():
    """Eq. (gamma): lambda << distance to the poles is recomputed from A^{-1}."""
    d, z, rho = _near_zero_problem()
    lam, v, info = oracle.dpr1eig(d, z, rho, 2)
    h, l, vq = oracle.quad_eig(d, z, rho, 2)
    assert info["zero_path"] == 1
    assert abs(h) < 1e-12
    assert fr_rel([lam], [h, l]) <= tol(4)
    lam0, _, _ = oracle.dpr1eig(d, z, rho, 2, oracle.default_opts(remedies=1))
    assert fr_rel([lam0], [h, l]) > 1e-6          # sigma + mu cancels without it


def test_near_zero_eigenvalue_by_determinant():
    """An eigenvalue of about 4e-26 between poles of size 1: with dyadic data
    1 + rho sum_j zeta_j^2 / d_j = -2^-80 exactly, and the product of the eigenvalues is
    det(D + rho z z^T) = prod_j d_j (1 + rho sum_j zeta_j^2 / d_j) (exact in rationals), which
    fixes the small one without any secular solve.  The oracle's recompute from A^{-1}
    (Eq. (gamma): at sigma = 0 every term of f is exact here) reaches it to the bound; binary128
    cannot (f cancels O(1) terms near lambda: 2^-113 absolute, about 3e-10 of lambda), so the
    reference is held to that absolute accuracy only."""
    from fractions import Fraction as Fr
    d = np.array([1.0, 0.5, -0.25, -1.0])
    z = np.array([1.0, 1.0, 1.0, 2.0 ** -40])
    rho = 1.0
    n = d.size
    q = oracle.quad_all(d, z, rho)
    k0 = int(np.argmin(np.abs(q["hi"])))
    det = 1 + Fr(rho) * sum(Fr(float(zj)) ** 2 / Fr(float(dj)) for dj, zj in zip(d, z))
    for dj in d:
        det *= Fr(float(dj))
    others = Fr(1)
    for k in range(n):
        if k != k0:
            others *= Fr(float(q["hi"][k])) + Fr(float(q["lo"][k]))
    lam_det = det / others
    assert 1e-27 < abs(float(lam_det)) < 1e-24
    assert abs(Fr(float(q["hi"][k0])) + Fr(float(q["lo"][k0])) - lam_det) <= Fr(2.0 ** -110)
    lam, _, info = oracle.dpr1eig(d, z, rho, k0)
    assert info["zero_path"] == 1
    assert abs(Fr(float(lam)) - lam_det) <= Fr(tol(n)) * abs(lam_det)


# ---------------------------------------------------------------- invariants
@pytest.mark.parametrize("gen,n,seed", [("uniform", 200, 3), ("hard", 300, 2)])
def test_interlacing_trace_orthogonality(gen, n, seed):
    d, z, rho = getattr(W, gen)(n, seed)
    r = oracle.eig_all(d, z, rho, threads=8)
    for k in range(n):
        s, m = Fr(r["sigma"][k]), Fr(r["mu"][k])
        lam = s + m
        # strict interlacing on the exact pairs, Eq. (interlace)
        assert lam > Fr(d[k])
        if k > 0:
            assert lam < Fr(d[k - 1])
        if r["shift"][k] == k:
            assert r["mu"][k] > 0
        elif r["shift"][k] >= 0 and r["shift"][k] == k - 1:
            assert r["mu"][k] < 0
        # non-strict on the rounded eigenvalues
        assert r["lam"][k] >= d[k] and (k == 0 or r["lam"][k] <= d[k - 1])
    # trace(A) = sum(lambda)
    tr = sum(Fr(x) for x in d) + Fr(rho) * sum(Fr(x) * Fr(x) for x in z)
    sl = sum(Fr(s) + Fr(m) for s, m in zip(r["sigma"], r["mu"]))
    assert abs(float(sl - tr)) <= 4 * n * 2.0 ** -52 * float(np.sum(np.abs(r["lam"])))
    O, R = _measures(d, z, rho, r["lam"], r["Vt"])
    assert O < 1.0 and R < 1.0


def test_dense_solver_crosscheck():
    d, z, rho = W.uniform(80, 12)
    r = oracle.eig_all(d, z, rho)
    A = np.diag(d) + rho * np.outer(z, z)
    w, V = np.linalg.eigh(A)
    nA = np.linalg.norm(A, 2)
    assert np.max(np.abs(np.sort(r["lam"]) - w)) <= 1e-13 * nA
    # same vectors up to sign (well separated spectrum)
    Vs = V[:, ::-1].T
    sgn = np.sign(np.sum(Vs * r["Vt"], axis=1))
    assert np.max(np.abs(Vs * sgn[:, None] - r["Vt"])) < 1e-10


# ---------------------------------------------------------------- deflation and rho <= 0
def test_deflation_and_sign_flip():
    d = np.array([3.0, 2.0, 2.0, 2.0, 1.0, 0.5, -1.0])
    z = np.array([1.0, 0.5, 0.7, -0.2, 0.0, 1.0, 0.3])
    for rho in (0.8, -0.7, 0.0):
        r = oracle.eig_full(d, z, rho)
        A = np.diag(d) + rho * np.outer(z, z)
        w = np.linalg.eigvalsh(A)[::-1]
        assert np.max(np.abs(r["lam"] - w)) <= 1e-14 * np.linalg.norm(A, 2)
        assert np.all(np.diff(r["lam"]) <= 0)
        V = r["Vt"].T
        assert np.max(np.abs(V.T @ V - np.eye(7))) < 1e-14
        assert np.max(np.abs(A @ V - V * r["lam"])) < 1e-14
    r = oracle.eig_full(d, z, 0.8)
    assert np.sum(r["lam"] == 2.0) == 2          # tie group of three keeps two deflated copies
    assert np.sum(r["lam"] == 1.0) == 1          # zeta = 0


# ---------------------------------------------------------------- adjoint
def _loss(d, z, rho, w, Wm):
    r = oracle.eig_all(d, z, rho)
    return float(np.dot(w, r["lam"]) + np.sum(Wm * r["Vt"]))


def test_backward_against_finite_differences():
    rng = np.random.default_rng(21)
    n = 7
    d, z, rho = W.uniform(n, 21)
    w = rng.standard_normal(n)
    Wm = rng.standard_normal((n, n))
    r = oracle.eig_all(d, z, rho)
    gd, gz, gr = oracle.backward(d, z, rho, r["sigma"], r["mu"], w, Wm)
    gap = np.min(-np.diff(d))
    for t in range(4):
        dd_ = rng.standard_normal(n)
        dz = rng.standard_normal(n)
        dr = rng.standard_normal()
        h = 1e-6 * min(1.0, gap)
        lp = _loss(d + h * dd_, z + h * dz, rho + h * dr, w, Wm)
        lm = _loss(d - h * dd_, z - h * dz, rho - h * dr, w, Wm)
        fd = (lp - lm) / (2 * h)
        an = np.dot(gd, dd_) + np.dot(gz, dz) + gr * dr
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (fd, an)


def test_backward_against_dense_adjoint():
    """Standard adjoint of A = V diag(lambda) V^T: Abar = V (diag(lbar) + F o (V^T Vbar)) V^T."""
    rng = np.random.default_rng(5)
    n = 9
    d, z, rho = W.uniform(n, 33)
    r = oracle.eig_all(d, z, rho)
    lam, V = r["lam"], r["Vt"].T
    lb = rng.standard_normal(n)
    Vb = rng.standard_normal((n, n))        # dL/dV, columns = eigenvectors
    F = lam[None, :] - lam[:, None]
    np.fill_diagonal(F, np.inf)
    F = 1.0 / F
    Ab = V @ (np.diag(lb) + F * (V.T @ Vb)) @ V.T
    Ab = 0.5 * (Ab + Ab.T)
    gd_ref = np.diag(Ab).copy()
    gz_ref = 2 * rho * Ab @ z
    gr_ref = z @ Ab @ z
    gd, gz, gr = oracle.backward(d, z, rho, r["sigma"], r["mu"], lb, Vb.T)
    assert np.linalg.norm(gd - gd_ref) <= 1e-10 * np.linalg.norm(gd_ref)
    assert np.linalg.norm(gz - gz_ref) <= 1e-10 * np.linalg.norm(gz_ref)
    assert abs(gr - gr_ref) <= 1e-10 * abs(gr_ref)


def test_backward_trace_identities():
    d, z, rho = W.hard(64, 3)
    r = oracle.eig_all(d, z, rho)
    n = d.size
    gd, gz, gr = oracle.backward(d, z, rho, r["sigma"], r["mu"], np.ones(n), None)
    # d(sum lambda)/d d_j = sum_k v_k[j]^2 = 1, d/dz = 2 rho z, d/drho = ||z||^2
    assert np.max(np.abs(gd - 1.0)) <= 1e-12
    assert np.max(np.abs(gz - 2 * rho * z) / np.abs(2 * rho * z)) <= 1e-9
    assert abs(gr - np.dot(z, z)) <= 1e-12 * np.dot(z, z)


@pytest.mark.parametrize("gen,n,seed", [("uniform", 64, 2), ("hard", 200, 5), ("large", 300, 4)])
def test_backward_against_binary128_adjoint(gen, n, seed):
    """The adjoint formulas evaluated in binary128 at binary128 eigenpairs; the hard and
    large spectra have eigenvectors within 1e-10 of a unit vector, where the plain
    binary64 evaluation of g = vbar - v (v . vbar) cancels."""
    if gen == "large":
        d, z, rho, _ = W.large(n, seed, with_W=False)
    else:
        d, z, rho = getattr(W, gen)(n, seed)
    rng = np.random.default_rng(seed)
    w, Wm = rng.standard_normal(n), rng.standard_normal((n, n))
    r = oracle.eig_all(d, z, rho, threads=8)
    od, oz, orho = oracle.backward(d, z, rho, r["sigma"], r["mu"], w, Wm)
    qd, qz, qrho = oracle.quad_backward(d, z, rho, w, Wm)
    # component by component: within 16 n 2^-53 of each component's error scale, and to rel 1e-10
    # wherever the scale is within 100 times the component (no cancellation worth the name)
    sd, sz, sr = adjoint_scales(d, z, rho, r["sigma"], r["mu"], w, Wm)
    tau = 16 * n * 2.0 ** -53
    for got, ref, sc in ((od, qd, sd), (oz, qz, sz), (orho, qrho, sr)):
        res = componentwise(got, ref, sc, tau)
        assert res["ok"], res


@pytest.mark.parametrize("gen,n,seed", [("uniform", 16, 3), ("uniform", 32, 4), ("hard", 16, 5), ("hard", 32, 6)])
def test_backward_per_coordinate_central_differences(gen, n, seed):
    """Every component of dL/dd, dL/dz and dL/drho against a central difference in that one
    coordinate (Richardson-extrapolated, steps 1e-4 of the local pole gap for d_j and of |z_j|
    for z_j).  The loss is sensitive at each component's own scale: sum_k w_k mu_k with
    mu_k = lambda_k - d_{i(k)} (the shift index of the unperturbed solve; on the hard spectrum
    lambda_k rounds onto its pole, mu_k does not) plus sum W_kj V_kj / |V_kj| (tiny components
    count as much as large ones).  Its adjoint is the adjoint of (lambda, V) with dL/dlambda = w,
    dL/dVt = W / |V|, less w_k at d_{i(k)}."""
    d, z, rho = getattr(W, gen)(n, seed)
    rng = np.random.default_rng(seed)
    w, Wm = rng.standard_normal(n), rng.standard_normal((n, n))
    r0 = oracle.eig_all(d, z, rho)
    # the pole index of each shift (-1 for a non-pole shift of R2, which stays fixed)
    sidx = np.array([int(np.flatnonzero(d == s)[0]) if np.any(d == s) else -1 for s in r0["sigma"]])
    pole = sidx >= 0
    Wh = Wm / np.abs(r0["Vt"])

    def loss(dd_, zz_, rr_):
        r = oracle.eig_all(dd_, zz_, rr_)
        base = np.where(pole, dd_[np.maximum(sidx, 0)], r0["sigma"])
        return float(np.dot(w, (r["sigma"] - base) + r["mu"]) + np.sum(Wh * r["Vt"]))

    gd, gz, gr = oracle.backward(d, z, rho, r0["sigma"], r0["mu"], w, Wh)
    np.subtract.at(gd, sidx[pole], w[pole])
    fd_d, fd_z, fd_r = central_differences(loss, d, z, rho)
    assert np.max(np.abs(fd_d - gd) / np.abs(gd)) <= 1e-6
    assert np.max(np.abs(fd_z - gz) / np.abs(gz)) <= 1e-6
    assert abs(fd_r - gr) <= 1e-6 * abs(gr)


def test_tiny_weights_are_zero_weights():
    """A weight whose square is not a normal binary64 number after the normalisation
    max|zeta| in [1/2, 1) is deflated (the secular function cannot see it): the remaining
    eigenvalues equal the binary128 eigenvalues of the reduced problem, the deflated ones are
    their poles, and A V = V diag(lambda).  The rule is relative to the largest weight."""
    d, z, rho = W.uniform(64, 3)
    z = z.copy()
    z[[5, 20, 40]] = [1e-170, 1e-200, 1e-155]
    z[[6, 30]] = [3e-162, -2e-158]
    r = oracle.eig_full(d, z, rho)
    A = np.diag(d) + rho * np.outer(z, z)
    V = r["Vt"].T
    assert np.max(np.abs(A @ V - V * r["lam"])) <= 1e-14
    assert np.max(np.abs(V.T @ V - np.eye(64))) <= 1e-14
    keep = ~oracle.zero_weight(z)
    assert keep.sum() == 59
    assert oracle.zero_weight(2.0 ** -512, zmax=0.9) and not oracle.zero_weight(2.0 ** -511, zmax=0.9)
    assert np.array_equal(oracle.zero_weight(z * 2.0 ** 300), ~keep)
    assert np.array_equal(oracle.zero_weight(z * 2.0 ** -300), ~keep)
    q = oracle.quad_all(d[keep], z[keep], rho)
    lk = np.sort(np.concatenate([q["hi"] + q["lo"], d[~keep]]))[::-1]
    assert np.max(np.abs(r["lam"] - lk) / np.abs(lk)) <= 16 * 64 * 2.0 ** -53


def _r2_estimates(rng, lo, hi, true):
    """Estimates an R2 shift may start from: absurd values, the interval ends, random points
    inside it (uniform and next to either end), and the eigenvalue itself."""
    est = [1e293, -1e293, float("nan"), 0.0, lo, hi, true]
    if np.isfinite(hi):
        w = hi - lo
        est += list(lo + w * rng.random(3)) + [lo + w * 1e-9, hi - w * 1e-9]
    else:
        est += list(lo + abs(true - lo) * 10.0 ** rng.uniform(-3, 3, 4))
    return est


def test_r2_from_any_estimate():
    """Remedy R2 (Sec. 2) from any starting estimate: the shift is moved into the interlacing
    interval of lambda_k, where the sign of f picks the side whose exterior eigenvalue of
    (A - sigma I)^{-1} is 1/(lambda_k - sigma); the solve repeats while sigma is not nearer to
    lambda_k than to the interval's poles.  Every estimate, absurd ones included, gives
    lambda_k within 16 n 2^-53 of binary128 on clustered, graded and uniform problems, and a pair
    (sigma, mu) whose differences to the neighbouring poles do not cancel (where no binary64
    shift achieves that, the shift is formed in double the working precision: at most 3 more
    solves)."""
    rng = np.random.default_rng(77)
    for case in range(12):
        n = int(rng.integers(2, 40))
        kind = case % 3
        if kind == 0:
            d = rng.uniform(-1, 1, n)
        elif kind == 1:
            c = rng.uniform(-1, 1, max(1, n // 5))
            d = rng.choice(c, n) + rng.choice([1.0, -1.0], n) * 10.0 ** rng.uniform(-12, -3, n)
        else:
            d = np.sign(rng.uniform(-1, 1, n)) * 10.0 ** rng.uniform(-10, 0, n)
        d = np.sort(d)[::-1].copy()
        if not np.all(d[:-1] > d[1:]):
            continue
        z = rng.choice([1.0, -1.0], n) * 10.0 ** rng.uniform(-6, 0, n)
        rho = float(10.0 ** rng.uniform(-3, 6))
        q = oracle.quad_all(d, z, rho, want_vectors=False)
        lq = q["hi"] + q["lo"]
        for k in rng.choice(n, size=min(n, 4), replace=False):
            hi = d[k - 1] if k > 0 else d[0] + rho * float(np.sum(z * z))
            for est in _r2_estimates(rng, d[k], hi, lq[k]):
                r = oracle.r2(d, z, rho, k, est)
                assert 1 <= r["rounds"] <= 6
                assert abs(r["lam"] - lq[k]) <= tol(n) * abs(lq[k]), (case, k, est, r, lq[k])
                for p in ([k - 1, k] if k > 0 else [k]):
                    dp = d[p] - r["sigma"]
                    assert 16 * abs(dp - r["mu"]) >= abs(dp) + abs(r["mu"]), (case, k, p, est, r)


def _pair_error(sig, mu, hi, lo):
    """|(sigma + mu) - (hi + lo)| / |hi + lo| with error-free transformations."""
    def two_sum(a, b):
        t = a + b
        bb = t - a
        return t, (a - (t - bb)) + (b - bb)
    a, ea = two_sum(sig, -hi)
    b, eb = two_sum(a, mu)
    return np.abs(b + (ea + eb - lo)) / np.abs(hi + lo)


def test_r2_shift_in_double_the_working_precision():
    """Remedy R2, last sentence of Sec. 2: when no binary64 number lies between lambda_k and a
    neighbouring pole, the shift and its DPR1 matrix are formed in double the working precision.
    The fixed case: lambda_1 lies 5.2e-18 (1/20 ulp) above the pole d_1, K_nu ~ 1e33 there
    (lambda_2 hugs d_1 from below within 4e-51), the other pole d_0 is far, and the nearest binary64
    shift next to lambda_1, nextup(d_1), leaves (d_1 - sigma) - mu cancelling by a factor 20.  With
    the double-double shift the pair, lambda_1 and every component meet the bound against binary128,
    as do all eigenpairs of 120 seeded problems with poles at consecutive binary64 numbers, of which
    more than 20 take the branch."""
    d = np.array([1.2309301857926847, 0.8071443705564947, 0.8071443705564946, 0.8071443705564945,
                  -0.7174580783727836])
    z = np.array([-6.0703694565774058e-01, -3.4635323545170545e-26, 2.6021119607883683e-08,
                  -1.5544665423687004e-15, 6.2430810708415818e-01])
    rho = 0.1918407481797008
    cases = [(d, z, rho)] + [W.adjacent_poles(seed) for seed in range(120)]
    hits = 0
    for c, (d, z, rho) in enumerate(cases):
        n = d.size
        r = oracle.eig_all(d, z, rho)
        q = oracle.quad_all(d, z, rho)
        dd = (r["flags"] & 16) != 0
        hits += int(dd.any())
        if c == 0:
            assert dd[1] and not dd[[0, 2, 3, 4]].any()
            assert r["sigma"][1] == d[1] and 0 < r["mu"][1] < 2.0 ** -53 * d[1]
        lq = q["hi"] + q["lo"]
        assert np.max(np.abs(r["lam"] - lq) / np.abs(lq)) <= tol(n), c
        assert np.max(_pair_error(r["sigma"], r["mu"], q["hi"], q["lo"])) <= tol(n), c
        assert np.max(np.abs(r["Vt"] - q["Vt"]) / np.abs(q["Vt"])) <= tol(n), c
        # the returned pair is against the nearer pole: its pole differences do not cancel
        for k in np.flatnonzero(dd):
            assert np.any(d == r["sigma"][k])
    assert hits > 20


def test_scale_invariance_is_exact():
    """The exact power-of-two normalisation: D + rho z z^T with d -> 2^s d, z -> 2^t z and
    rho -> 2^(s - 2t) rho is 2^s times the same matrix, and the oracle returns exactly 2^s times
    the eigenvalues and the same eigenvectors, bit for bit, even where the unscaled data would
    over- or underflow (s, t up to +-900)."""
    d, z, rho = W.hard(120, 4)
    base = oracle.eig_all(d, z, rho)
    for s, t in ((0, 300), (600, 0), (-600, 0), (900, 400), (-900, -400), (37, -11)):
        ds, zs, rs = np.ldexp(d, s), np.ldexp(z, t), math.ldexp(rho, s - 2 * t)
        r = oracle.eig_all(ds, zs, rs)
        assert np.array_equal(r["lam"], np.ldexp(base["lam"], s)), (s, t)
        assert np.array_equal(r["Vt"], base["Vt"]), (s, t)


def _harsh(rng, wmax=150):
    """Data of any magnitude: poles scaled by 2^U(-700, 700), weights over up to 2^wmax within a
    problem and scaled by 2^U(-300, 300), and a rank-one part from 2^-300 to 2^300 times the
    poles' scale; poles uniform, clustered or graded."""
    n = int(rng.integers(2, 40))
    kind = rng.integers(0, 3)
    if kind == 0:
        d = rng.uniform(-1, 1, n)
    elif kind == 1:
        c = rng.uniform(-1, 1, max(1, n // 5))
        d = rng.choice(c, n) + rng.choice([1.0, -1.0], n) * 10.0 ** rng.uniform(-12, -3, n)
    else:
        d = np.sign(rng.uniform(-1, 1, n)) * 10.0 ** rng.uniform(-12, 0, n)
    d = np.sort(d)[::-1].copy()
    z = rng.choice([1.0, -1.0], n) * 2.0 ** rng.uniform(-rng.uniform(0, wmax), 0, n)
    rho = 2.0 ** rng.uniform(-300, 300) / float(np.sum(z * z)) * float(np.max(np.abs(d)))
    s, t = int(rng.integers(-700, 700)), int(rng.integers(-300, 300))
    e = math.frexp(rho)[1] + s - 2 * t
    if not -1000 < e < 1000:          # keep rho itself a normal binary64 number
        return _harsh(rng, wmax)
    return np.ldexp(d, s), np.ldexp(z, t), math.ldexp(rho, s - 2 * t)


def test_harsh_data_meets_the_bound_or_reports_range():
    """No silent failure on data of any magnitude: every eigenpair either meets 16 n 2^-53
    against binary128 (components compared relative to max(|v|, 2^-1022), the binary64 normal
    range) or the oracle reports that it needs values outside the binary64 range."""
    rng = np.random.default_rng(2718)
    ok = rng_err = 0
    while ok + rng_err < 150:
        d, z, rho = _harsh(rng)
        n = d.size
        if not (np.all(d[:-1] > d[1:]) and np.all(np.isfinite(d)) and not np.any(oracle.zero_weight(z))
                and rho > 0 and np.isfinite(rho)):
            continue
        try:
            r = oracle.eig_all(d, z, rho, threads=4)
        except oracle.OracleRangeError:
            rng_err += 1
            continue
        q = oracle.quad_all(d, z, rho, threads=4)
        lq = q["hi"] + q["lo"]
        assert np.max(np.abs(r["lam"] - lq) / np.abs(lq)) <= tol(n)
        err = np.abs(r["Vt"] - q["Vt"]) / np.maximum(np.abs(q["Vt"]), 2.0 ** -1022)
        assert err.max() <= tol(n), float(err.max() / tol(n))
        ok += 1
    assert ok >= 120


def test_out_of_range_pair_is_reported():
    """A weight of 1e-152 next to weights of 1 (above the zero-weight cut, 2^-511 of the largest):
    lambda_0 - d_0 is about rho zeta_0^2 ~ 1e-314, below the normal binary64 range even after
    the normalisation, so the pair cannot be formed with full precision and the oracle reports
    it instead of returning it."""
    d = np.array([2.0e-3, 3.0e-4, 2.0e-12])
    z = np.array([1e-152, 1.0, -0.5])
    with pytest.raises(oracle.OracleRangeError):
        oracle.dpr1eig(d, z, 4e-10, 0)
    lam, _, _ = oracle.dpr1eig(d, z, 4e-10, 1)        # the other pairs are in range
    q = oracle.quad_eig(d, z, 4e-10, 1, want_vector=False)
    assert abs(lam - (q[0] + q[1])) <= tol(3) * abs(lam)
