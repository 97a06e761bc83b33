/*
 * dpr1_oracle.c -- plain, slow, single-thread CPU oracle of the forward-stable
 * DPR1 eigensolver of Jakovcevic Stor, Slapnicar and Barlow (arXiv 1405.7537).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the reference the CUDA path is checked
 * against.  Only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark load it.  It shares no code with the CUDA library: it has its own
 * double-double arithmetic, its own bisection and its own eigenvector formula.
 *
 * It follows Algorithm 1 (dpr1eig) step by step, in IEEE binary64 ("FP64"), in
 * the paper's notation:
 *   A = D + rho z z^T, d_1 > d_2 > ... > d_n, rho > 0, zeta_j != 0     (Sec. 1, Eq. (A), (order))
 *   shift sigma = d_i, A_i = A - d_i I                                  (Sec. 2)
 *   A_i^{-1} = arrowhead with diagonal delta_j = 1/(d_j - d_i),
 *              border w_j = -zeta_j / (zeta_i (d_j - d_i)) and corner b  (Eq. (invAi), (b_ob))
 *   g(nu) = b - nu - sum_j w_j^2 / (delta_j - nu)                       (Eq. (secAi))
 *   x = [(D_1 - mu I)^{-1} z_1; -zeta_i/mu; (D_2 - mu I)^{-1} z_2], v = x/||x||  (Eq. (eigenvecAi))
 *   lambda = mu + sigma, mu = 1/nu                                      (Eq. (8))
 *   kappa_nu, K_b, K_z                                                  (Eq. (knu2))
 *   K_nu = ||A_i^{-1}||_2 / |nu|, remedies R1 and R2                    (Eq. (K0))
 *   lambda near zero: lambda = 1/nu, nu extreme eigenvalue of
 *       A^{-1} = D^{-1} + gamma D^{-1} z z^T D^{-1}                     (Eq. (gamma))
 *   double the working precision as double-double                      (Sec. 2.3)
 *
 * Readings of points the paper leaves open (each also listed in the design notes):
 *   - Eq. (secAi) prints Delta = diag(D_1, D_2); the arrowhead's diagonal is
 *     diag(D_1^{-1}, D_2^{-1}), so delta_j = 1/(d_j - d_i) is used.
 *   - "kappa_nu >> O(n)": b is recomputed in double-double when
 *     kappa_nu > T_kappa * n (mode 1), always (mode 2, default) or never (mode 0).
 *   - Bisection bracket (the paper only cites Olver-Stewart): the Weyl bracket
 *     [max(b, max delta), max(b, max delta) + ||w||] for the rightmost eigenvalue,
 *     mirrored for the leftmost, intersected with the known sign of nu; bisection on
 *     the bit patterns of |nu| until the end points are adjacent doubles; the end
 *     point with the smaller |g| is returned.
 *   - "K_nu >> 1": K_nu > T_Knu.  ||A_i^{-1}||_2 is computed exactly as
 *     max(|leftmost|, |rightmost|) of the arrowhead, each by bisection.
 *   - R1 is taken when the other neighbouring pole gives a smaller K_nu that is within
 *     T_Knu and lambda is not more than T_Knu times farther from that pole than from
 *     the first one (otherwise the eigenvector formula at the other pole cancels);
 *     else R2.  R2 shifts to sigma = fl(lambda) of the better pole solution moved into the
 *     interlacing interval of lambda_k ((d_k, d_{k-1}), or (d_0, d_0 + rho ||z||^2] for
 *     k = 0), computes f(sigma) in double-double and finds the exterior eigenvalue of the
 *     DPR1 matrix
 *     (A - sigma I)^{-1} = (D - sigma I)^{-1} + gamma (D - sigma I)^{-1} z z^T (D - sigma I)^{-1},
 *     gamma = -rho / f(sigma), by bisection; when sigma was not nearer to lambda_k than to
 *     the interval's poles, again from the midpoint (the Weyl bound for k = 0) and then
 *     from the lambda found there (o_r2).  When no binary64 number lies between lambda_k and
 *     a neighbouring pole (the interval holds none, or the binary64 result's difference to a
 *     pole cancels by more than 16), the shift is formed in double the working precision:
 *     sigma = d_k + t, the DPR1 matrix from the double-double differences d_j - sigma, and the
 *     result is returned against the nearer pole (o_r2_dd).  A pole solve that left the
 *     binary64 range counts as K_nu = inf.
 *   - "|lambda| << min(|lambda - d_k|, |lambda - d_{k-1}|)": T_zero |lambda| < min(...).
 *     The denominator of gamma is formed in double-double; if it is zero, lambda = 0.
 *   - Shift test tie F == 0 takes the else branch (sigma = d_{k-1}), as printed.
 *   - Data of any magnitude: each problem is solved after the exact power-of-two
 *     normalisation D' = 2^-a D, z' = 2^-b z, rho' = 2^(2b-a) rho (oracle_dpr1eig), and a
 *     pair that needs values outside the binary64 range (mu zero, subnormal or not finite;
 *     lambda or v not finite) returns code 4.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* Double-double arithmetic: an unevaluated sum hi + lo of two binary64       */
/* numbers, |lo| <= ulp(hi)/2.  Error-free transformations: TwoSum (Knuth),  */
/* FastTwoSum and the product split (Dekker 1971), the latter through fma.   */
/* ------------------------------------------------------------------------- */
typedef struct { double hi, lo; } odd_t;

static odd_t o_two_sum(double a, double b) {
  odd_t r;
  double s = a + b;
  double bb = s - a;
  double err = (a - (s - bb)) + (b - bb);
  r.hi = s; r.lo = err;
  return r;
}

static odd_t o_fast_two_sum(double a, double b) { /* requires |a| >= |b| or a == 0 */
  odd_t r;
  double s = a + b;
  r.hi = s; r.lo = b - (s - a);
  return r;
}

static odd_t o_two_prod(double a, double b) {
  odd_t r;
  double p = a * b;
  r.hi = p; r.lo = fma(a, b, -p);
  return r;
}

static odd_t o_from(double a) { odd_t r; r.hi = a; r.lo = 0.0; return r; }

static odd_t o_add(odd_t a, odd_t b) {
  odd_t s = o_two_sum(a.hi, b.hi);
  odd_t t = o_two_sum(a.lo, b.lo);
  double lo = s.lo + t.hi;
  s = o_fast_two_sum(s.hi, lo);
  lo = s.lo + t.lo;
  return o_fast_two_sum(s.hi, lo);
}

static odd_t o_neg(odd_t a) { a.hi = -a.hi; a.lo = -a.lo; return a; }

static odd_t o_mul(odd_t a, odd_t b) {
  odd_t p = o_two_prod(a.hi, b.hi);
  double lo = p.lo + (a.hi * b.lo + a.lo * b.hi);
  return o_fast_two_sum(p.hi, lo);
}

static odd_t o_mul_d(odd_t a, double b) {
  odd_t p = o_two_prod(a.hi, b);
  double lo = p.lo + a.lo * b;
  return o_fast_two_sum(p.hi, lo);
}

/* a / b: long division with three binary64 quotient digits. */
static odd_t o_div(odd_t a, odd_t b) {
  double q1 = a.hi / b.hi;
  odd_t r = o_add(a, o_neg(o_mul_d(b, q1)));
  double q2 = r.hi / b.hi;
  r = o_add(r, o_neg(o_mul_d(b, q2)));
  double q3 = r.hi / b.hi;
  odd_t q = o_fast_two_sum(q1, q2);
  return o_add(q, o_from(q3));
}

/* Exported for the tests that pin the double-double layer against exact rationals. */
void oracle_dd_add(double ah, double al, double bh, double bl, double* out) {
  odd_t a = {ah, al}, b = {bh, bl}; odd_t r = o_add(a, b); out[0] = r.hi; out[1] = r.lo;
}
void oracle_dd_mul(double ah, double al, double bh, double bl, double* out) {
  odd_t a = {ah, al}, b = {bh, bl}; odd_t r = o_mul(a, b); out[0] = r.hi; out[1] = r.lo;
}
void oracle_dd_div(double ah, double al, double bh, double bl, double* out) {
  odd_t a = {ah, al}, b = {bh, bl}; odd_t r = o_div(a, b); out[0] = r.hi; out[1] = r.lo;
}

/* ------------------------------------------------------------------------- */
/* Options and per-eigenpair report                                          */
/* ------------------------------------------------------------------------- */
typedef struct {
  int dd_mode;        /* 0: never, 1: when kappa_nu > T_kappa * n, 2: always (default) */
  double T_kappa;     /* threshold factor for mode 1 (default 1500: with it mode 1 uses
                         double-double for 25 / 201 / 201 eigenvalues of Example 4, the
                         counts the paper reports) */
  double T_Knu;       /* remedies when K_nu > T_Knu */
  double T_zero;      /* near-zero test factor */
  int remedies;       /* bit 0: R1/R2, bit 1: near-zero recompute (3 = both, default) */
} oracle_opts;

typedef struct {
  int shift;          /* 0-based pole index i of the final shift, -1 for a non-pole shift (R2) */
  int first_shift;    /* pole chosen by the shift test */
  int used_dd;        /* b (or f(sigma)) formed in double-double */
  int remedy;         /* 0 none, 1 R1, 2 R2 */
  int zero_path;      /* lambda recomputed from A^{-1} */
  int steps;          /* bisection steps of the final solve */
  double sigma, mu, nu, lambda;
  double b;           /* corner element of the final arrowhead (binary64) */
  double K_nu;        /* K_nu of the first shift */
  double K_nu_final;  /* K_nu of the final shift (1 for R2) */
  double kappa_nu;    /* Eq. (knu2) of the first shift */
  int r2_dd;          /* R2 took its shift in double the working precision */
} oracle_info;

void oracle_default_opts(oracle_opts* o) {
  o->dd_mode = 2; o->T_kappa = 1500.0; o->T_Knu = 16.0; o->T_zero = 64.0; o->remedies = 3;
}

/* ------------------------------------------------------------------------- */
/* Bisection on the bit patterns of |nu|.                                     */
/* ------------------------------------------------------------------------- */
static uint64_t o_bits(double a) { uint64_t u; memcpy(&u, &a, 8); return u; }
static double o_from_bits(uint64_t u) { double a; memcpy(&a, &u, 8); return a; }

/* Evaluates a secular function at nu; the callee decides the sign convention. */
typedef double (*o_secular_fn)(const void* ctx, double nu);

/*
 * Finds the root of a secular function that has exactly one sign change for
 * nu = s*a, a in [a_lo, a_hi]; phi(s*a) "below" the root has sign below_sign
 * (+1 or -1).  a_lo is known to lie on the near side of the root (it may be a
 * pole, where phi is not evaluated); a_hi is checked and pushed out until phi
 * changes sign.  Returns s*a for the end point of the final adjacent pair with
 * the smaller |phi|.
 */
static double o_bisect(o_secular_fn phi, const void* ctx, double s, double a_lo, double a_hi,
                       int below_sign, int* steps_out) {
  int steps = 0;
  /* the bracket is on |nu| >= 0; -0.0 (and NaN) become +0.0 so that the bit patterns of the
     two ends are ordered like their values */
  if (!(a_lo > 0.0)) a_lo = 0.0;
  if (!(a_hi > a_lo)) a_hi = (a_lo > 0.0) ? a_lo * 2.0 : 1.0;
  /* make sure the far end is past the root */
  for (int t = 0; t < 2100; t++) {
    double g = phi(ctx, s * a_hi);
    if (g * below_sign <= 0.0) break;
    double w = a_hi - a_lo;
    a_lo = a_hi;
    a_hi = a_hi + 2.0 * w;
    if (isinf(a_hi)) break;
  }
  uint64_t lo = o_bits(a_lo), hi = o_bits(a_hi);
  double glo = NAN, ghi = NAN;
  while (hi - lo > 1) {
    uint64_t mid = lo + (hi - lo) / 2;
    double g = phi(ctx, s * o_from_bits(mid));
    steps++;
    if (g * below_sign > 0.0) { lo = mid; glo = g; }
    else { hi = mid; ghi = g; }
  }
  if (steps_out) *steps_out = steps;
  if (lo == hi) return s * o_from_bits(lo);
  if (isnan(glo)) glo = phi(ctx, s * o_from_bits(lo));
  if (isnan(ghi)) ghi = phi(ctx, s * o_from_bits(hi));
  double alo = fabs(glo), ahi = fabs(ghi);
  if (isnan(alo)) alo = INFINITY;
  if (isnan(ahi)) ahi = INFINITY;
  return s * o_from_bits(ahi < alo ? hi : lo);
}

/* ------------------------------------------------------------------------- */
/* The arrowhead inverse of the shifted matrix, Eq. (invAi), (b_ob).          */
/* ------------------------------------------------------------------------- */
typedef struct {
  int n, i;
  const double* delta; /* [n], delta[i] unused */
  const double* w;     /* [n], w[i] unused */
  double b;
} o_arrow_ctx;

/* g(nu) = b - nu - w^T (Delta - nu I)^{-1} w, Eq. (secAi). */
static double o_g_arrow(const void* vctx, double nu) {
  const o_arrow_ctx* c = (const o_arrow_ctx*)vctx;
  double s = 0.0;
  for (int j = 0; j < c->n; j++) {
    if (j == c->i) continue;
    s += c->w[j] * c->w[j] / (c->delta[j] - nu);
  }
  return (c->b - nu) - s;
}

typedef struct {
  double b;           /* binary64 corner element */
  double Kb, Kz, kappa_nu;
  int used_dd;
} o_arrow_info;

/*
 * Forms delta_j = 1/(d_j - d_i), w_j = -(delta_j zeta_j)/zeta_i and b of Eq. (b_ob),
 * computes K_b, K_z and kappa_nu of Eq. (knu2) and, depending on dd_mode,
 * recomputes b in double-double (Sec. 2.3).
 */
static void o_arrowhead(int n, const double* d, const double* z, double rho, int i,
                        const oracle_opts* opt, double* delta, double* w, o_arrow_info* out) {
  double P = 0.0, N = 0.0;          /* z_1^T D_1^{-1} z_1 >= 0 and z_2^T D_2^{-1} z_2 <= 0 */
  double sumz = 0.0;
  for (int j = 0; j < n; j++) {
    if (j == i) { delta[j] = 0.0; w[j] = 0.0; continue; }
    double dj = d[j] - d[i];
    delta[j] = 1.0 / dj;
    w[j] = -(delta[j] * z[j]) / z[i];
    double t = z[j] * (delta[j] * z[j]);
    if (j < i) P += t; else N += t;
    sumz += fabs(z[j]);
  }
  double b = (1.0 / (z[i] * z[i])) * ((1.0 / rho + P) + N);
  double Kb = (1.0 + rho * P - rho * N) / fabs(1.0 + rho * P + rho * N);
  double Kz = sumz / fabs(z[i]);
  double sn = sqrt((double)n);
  double k1 = (n + 4) * sn * Kb;
  double k2 = 3.0 * sn + (n + 4) * (1.0 + 2.0 * Kz);
  double kappa = k1 < k2 ? k1 : k2;
  int use_dd = (opt->dd_mode == 2) || (opt->dd_mode == 1 && kappa > opt->T_kappa * n);
  if (use_dd) {
    /* b = (1/zeta_i^2) (1/rho + sum_{j != i} zeta_j^2 / (d_j - d_i)), all in double-double */
    odd_t acc = o_div(o_from(1.0), o_from(rho));
    for (int j = 0; j < n; j++) {
      if (j == i) continue;
      odd_t dj = o_two_sum(d[j], -d[i]);
      odd_t zz = o_two_prod(z[j], z[j]);
      acc = o_add(acc, o_div(zz, dj));
    }
    odd_t bb = o_div(acc, o_two_prod(z[i], z[i]));
    b = bb.hi + bb.lo;
  }
  out->b = b; out->Kb = Kb; out->Kz = Kz; out->kappa_nu = kappa; out->used_dd = use_dd;
}

/* Extreme eigenvalue of the arrowhead: side = +1 rightmost, -1 leftmost. */
static double o_arrow_extreme(int n, int i, const double* delta, const double* w, double b,
                              int side, int* steps) {
  o_arrow_ctx c = {n, i, delta, w, b};
  double wn2 = 0.0;
  double dmax = -INFINITY, dmin = INFINITY;
  for (int j = 0; j < n; j++) {
    if (j == i) continue;
    wn2 += w[j] * w[j];
    if (delta[j] > dmax) dmax = delta[j];
    if (delta[j] < dmin) dmin = delta[j];
  }
  double wn = sqrt(wn2);
  if (side > 0) {
    /* rightmost: nu in [max(b, max delta), max(b, max delta) + ||w||], and nu > 0 */
    double lo = b > dmax ? b : dmax;
    double hi = lo + wn;
    /* g > 0 below the root */
    return o_bisect(o_g_arrow, &c, 1.0, lo, hi, +1, steps);
  } else {
    /* leftmost: nu in [min(b, min delta) - ||w||, min(b, min delta)], and nu < 0 */
    double up = b < dmin ? b : dmin;
    double a_lo = -up, a_hi = -up + wn;
    /* in |nu|: g < 0 on the pole side (small |nu|), g > 0 beyond the root */
    return o_bisect(o_g_arrow, &c, -1.0, a_lo, a_hi, -1, steps);
  }
}

/* Eigenvector of A_i from mu, Eq. (eigenvecAi), normalised with a scaled 2-norm. */
static void o_vector_pole(int n, const double* d, const double* z, int i, double mu, double* v) {
  double m = 0.0;
  for (int j = 0; j < n; j++) {
    double x = (j == i) ? -z[i] / mu : z[j] / ((d[j] - d[i]) - mu);
    v[j] = x;
    if (fabs(x) > m) m = fabs(x);
  }
  double s = 0.0;
  for (int j = 0; j < n; j++) { double t = v[j] / m; s += t * t; }
  double r = sqrt(s);
  for (int j = 0; j < n; j++) v[j] = (v[j] / m) / r;
}

/* Eigenvector x = (D - lambda I)^{-1} z with lambda = sigma + mu, sigma not a pole. */
static void o_vector_shift(int n, const double* d, const double* z, double sigma, double mu, double* v) {
  double m = 0.0;
  for (int j = 0; j < n; j++) {
    double x = z[j] / ((d[j] - sigma) - mu);
    v[j] = x;
    if (fabs(x) > m) m = fabs(x);
  }
  double s = 0.0;
  for (int j = 0; j < n; j++) { double t = v[j] / m; s += t * t; }
  double r = sqrt(s);
  for (int j = 0; j < n; j++) v[j] = (v[j] / m) / r;
}

/* ------------------------------------------------------------------------- */
/* Solve at pole i for eigenvalue k: the extreme eigenvalue of A_i^{-1} on    */
/* the side that belongs to lambda_k, and K_nu of Eq. (K0).                   */
/* ------------------------------------------------------------------------- */
typedef struct {
  double nu, mu, b, K_nu, kappa_nu;
  int steps, used_dd;
} o_pole_solve;

static void o_solve_at_pole(int n, const double* d, const double* z, double rho, int k, int i,
                            const oracle_opts* opt, double* delta, double* w, o_pole_solve* r) {
  o_arrow_info ai;
  o_arrowhead(n, d, z, rho, i, opt, delta, w, &ai);
  /* sigma = d_k (i == k): lambda_k - d_k > 0 is the smallest positive mu, nu rightmost.
     sigma = d_{k-1} (i == k-1): lambda_k - d_{k-1} < 0, nu leftmost. */
  int side = (i == k) ? +1 : -1;
  int steps = 0;
  double nu = o_arrow_extreme(n, i, delta, w, ai.b, side, &steps);
  /* ||A_i^{-1}||_2 = max(|leftmost|, |rightmost|); the leftmost exists when i < n-1 */
  double other = 0.0;
  if (side > 0) {
    if (i < n - 1) other = o_arrow_extreme(n, i, delta, w, ai.b, -1, NULL);
  } else {
    other = o_arrow_extreme(n, i, delta, w, ai.b, +1, NULL);
  }
  double nrm = fabs(nu) > fabs(other) ? fabs(nu) : fabs(other);
  r->nu = nu; r->mu = 1.0 / nu; r->b = ai.b;
  r->K_nu = nrm / fabs(nu); r->kappa_nu = ai.kappa_nu;
  /* a solve that left the binary64 range (nu infinite or NaN, mu zero) is no solution: it
     counts as K_nu = inf, so the remedies take over */
  if (!(r->K_nu >= 1.0) || !isfinite(nu) || r->mu == 0.0) r->K_nu = INFINITY;
  r->steps = steps; r->used_dd = ai.used_dd;
}

/* ------------------------------------------------------------------------- */
/* Non-pole shift: exterior eigenvalue of (A - sigma I)^{-1}, used by R2      */
/* (sigma near lambda) and by the near-zero recompute (sigma = 0), Eq. (gamma) */
/* ------------------------------------------------------------------------- */
typedef struct {
  int n;
  const double* e;   /* 1/(d_j - sigma) */
  const double* u;   /* zeta_j/(d_j - sigma) */
  double gamma;
} o_dpr1inv_ctx;

/* h(nu) = 1 + gamma sum_j u_j^2 / (e_j - nu), the secular function of E + gamma u u^T. */
static double o_h_dpr1(const void* vctx, double nu) {
  const o_dpr1inv_ctx* c = (const o_dpr1inv_ctx*)vctx;
  double s = 0.0;
  for (int j = 0; j < c->n; j++) s += c->u[j] * c->u[j] / (c->e[j] - nu);
  return 1.0 + c->gamma * s;
}

/* d_j - sigma in double-double for a shift sigma = s + t (s, t binary64; t = 0 for a shift
   in working precision, when this is the exact difference of two binary64 numbers). */
static odd_t o_diff(double dj, double s, double t) {
  odd_t r = o_two_sum(dj, -s);
  return (t != 0.0) ? o_add(r, o_from(-t)) : r;
}

/* f(sigma) = 1 + rho sum zeta_j^2/(d_j - sigma) in double-double, Eq. (Pick), sigma = s + t. */
static odd_t o_f_dd(int n, const double* d, const double* z, double rho, double s, double t) {
  odd_t acc = o_from(0.0);
  for (int j = 0; j < n; j++) {
    odd_t dj = o_diff(d[j], s, t);
    odd_t zz = o_two_prod(z[j], z[j]);
    acc = o_add(acc, o_div(zz, dj));
  }
  return o_add(o_from(1.0), o_mul_d(acc, rho));
}

/*
 * Exterior eigenvalue of (A - sigma I)^{-1} for the shift sigma = s + t.  The elements of the
 * DPR1 matrix are formed from the differences d_j - sigma rounded to binary64 (for t = 0 the
 * plain binary64 difference d_j - s; for t != 0 the double-double difference, the shift in
 * double the working precision of remedy R2); f(sigma) is formed in double-double.
 * Returns 1 and mu (lambda = sigma + mu) on success, 0 if f(sigma) is zero in
 * double-double (lambda = sigma, mu = 0).
 */
static int o_solve_nonpole(int n, const double* d, const double* z, double rho, double s, double t,
                           double* e, double* u, double* mu_out, int* steps) {
  odd_t f = o_f_dd(n, d, z, rho, s, t);
  if (f.hi == 0.0 && f.lo == 0.0) { *mu_out = 0.0; if (steps) *steps = 0; return 0; }
  odd_t gdd = o_div(o_from(-rho), f);
  double gamma = gdd.hi + gdd.lo;
  double emax = -INFINITY, emin = INFINITY, un2 = 0.0;
  for (int j = 0; j < n; j++) {
    double dj = o_diff(d[j], s, t).hi;
    e[j] = 1.0 / dj;
    u[j] = z[j] / dj;
    un2 += u[j] * u[j];
    if (e[j] > emax) emax = e[j];
    if (e[j] < emin) emin = e[j];
  }
  o_dpr1inv_ctx c = {n, e, u, gamma};
  double nu;
  /* gamma > 0: rightmost eigenvalue in [max e, max e + gamma ||u||^2], positive;
     gamma < 0: leftmost in [min e - |gamma| ||u||^2, min e], negative.
     In both cases h < 0 on the pole side (small |nu|). */
  if (gamma > 0) {
    nu = o_bisect(o_h_dpr1, &c, 1.0, emax, emax + gamma * un2, -1, steps);
  } else {
    nu = o_bisect(o_h_dpr1, &c, -1.0, -emin, -emin - gamma * un2, -1, steps);
  }
  *mu_out = 1.0 / nu;
  return 1;
}

/* After a non-pole shift (R2): the difference d_p - lambda = (d_p - sigma) - mu to a
   neighbouring pole p cancels by more than a factor 16.  Then lambda lies much nearer to the
   pole than any binary64 shift can: no floating-point number lies between lambda and the pole,
   and the shift must be formed in double the working precision (o_r2_dd). */
static int o_pole_difference_cancels(double dp, double sigma, double mu) {
  const double t = (dp - sigma) - mu;
  return 16.0 * fabs(t) < fabs(dp - sigma) + fabs(mu);
}

/*
 * (R2) with the shift in double the working precision (Sec. 2, the last sentence of remedy
 * (R2)): sigma = d_k + t, the binary64 offset t inside the interlacing interval of lambda_k
 * measured from its lower pole: t in (0, g), g = d_{k-1} - d_k (exact in double-double), or for
 * k = 0 t in (0, rho ||z||^2] (Weyl).  The DPR1 matrix (A - sigma I)^{-1} is formed from the
 * double-double differences d_j - sigma (o_solve_nonpole).  The rounds follow o_r2: first the
 * estimate est_s + est_m (an unevaluated pair), then the midpoint of the interval (the Weyl end
 * for k = 0), then the lambda found there, until |mu| is below half the distance from sigma to
 * the nearer pole end.  lambda - d_k = t + mu is then returned against the nearer pole:
 * sigma_out = d_k, mu_out = fl(t + mu), or sigma_out = d_{k-1}, mu_out = fl((t - g) + mu), so
 * that every pole difference (d_j - sigma_out) - mu_out keeps its relative accuracy.
 */
static int o_r2_dd(int n, const double* d, const double* z, double rho, int k, double est_s, double est_m,
                   double* e, double* u, double* sigma_out, double* mu_out) {
  const double base = d[k];
  odd_t g;
  if (k > 0) {
    g = o_two_sum(d[k - 1], -base);
  } else {
    double zz = 0.0;
    for (int j = 0; j < n; j++) zz += z[j] * z[j];
    g = o_from(rho * zz);
  }
  const double gw = g.hi + g.lo;
  odd_t te = o_add(o_two_sum(est_s, -base), o_from(est_m));
  double t = te.hi + te.lo, mu = 0.0;
  const double mid = (k > 0) ? 0.5 * gw : gw;
  int rounds = 0;
  for (;;) {
    if (!(t > 0.0) || (k > 0 && !(t < gw)) || (k == 0 && t > gw)) t = mid;   /* also a NaN estimate */
    o_solve_nonpole(n, d, z, rho, base, t, e, u, &mu, NULL);
    rounds++;
    double room = t;
    if (k > 0 && gw - t < room) room = gw - t;
    if (rounds >= 3 || fabs(mu) < 0.5 * room) break;
    t = (rounds == 1) ? mid : t + mu;
  }
  odd_t lm = o_two_sum(t, mu);                  /* lambda - d_k */
  if (k > 0 && lm.hi > 0.5 * gw) {
    odd_t up = o_add(lm, o_neg(g));             /* lambda - d_{k-1} */
    *sigma_out = d[k - 1];
    *mu_out = up.hi + up.lo;
  } else {
    *sigma_out = base;
    *mu_out = lm.hi + lm.lo;
  }
  return rounds;
}

/*
 * (R2) from an estimate est_s + est_m of lambda_k (an unevaluated pair, e.g. a pole and its mu).
 * The shift is fl(est_s + est_m) moved into the interlacing interval of lambda_k: (d_k, d_{k-1}),
 * or (d_0, d_0 + rho ||z||^2] for k = 0.
 * Any sigma inside gives lambda_k: f(sigma) < 0 exactly when sigma < lambda_k, and the
 * exterior eigenvalue on that side of (A - sigma I)^{-1} is 1/(lambda_k - sigma).  It is
 * computed to high relative accuracy when lambda_k is the eigenvalue nearest to sigma, which
 * holds when |mu| < (distance from sigma to the nearer pole end of the interval) / 2, since
 * every other eigenvalue lies beyond those poles.  Otherwise (the estimate was far off: K_nu
 * of both pole solves near 1/eps) the next shift is the midpoint of the interval (the Weyl
 * bound for k = 0), from which lambda_k is at least as near as any other eigenvalue, and the
 * one after is the lambda found there (at most 3 solves).
 * When the interval holds no binary64 number, or the result's difference to a neighbouring pole
 * cancels (no binary64 number lies between lambda_k and that pole), the shift is formed in
 * double the working precision instead (o_r2_dd; *dd_out = 1).
 * Returns the number of solves.
 */
static int o_r2(int n, const double* d, const double* z, double rho, int k, double est_s, double est_m, double* e,
                double* u, double* sigma_out, double* mu_out, int* dd_out) {
  double lo = d[k], hi;
  if (k > 0) {
    hi = d[k - 1];
  } else {
    double zz = 0.0;
    for (int j = 0; j < n; j++) zz += z[j] * z[j];
    hi = d[0] + rho * zz;
  }
  double s = est_s + est_m, mu = 0.0;
  int rounds = 0;
  *dd_out = 0;
  for (;;) {
    if (!(s > lo)) s = nextafter(lo, INFINITY);           /* also a NaN estimate */
    if (k > 0 && s >= hi) s = nextafter(hi, -INFINITY);
    if (k == 0 && s > hi) s = hi;
    if (!(s > lo) || (k > 0 && !(s < hi))) {
      /* no binary64 number inside the interval */
      *dd_out = 1;
      return rounds + o_r2_dd(n, d, z, rho, k, est_s, est_m, e, u, sigma_out, mu_out);
    }
    o_solve_nonpole(n, d, z, rho, s, 0.0, e, u, &mu, NULL);
    rounds++;
    double room = s - lo;
    if (k > 0 && hi - s < room) room = hi - s;
    if (rounds >= 3 || fabs(mu) < 0.5 * room) break;
    /* not reliable from this shift (the estimate was far off).  Next, a shift from which
       lambda_k is at least as near as any other eigenvalue, so that the solve there is
       accurate: the midpoint of (d_k, d_{k-1}), or for k = 0 the Weyl bound (every other
       eigenvalue lies below lambda_0); then, if still needed, the lambda found there */
    s = (rounds == 1) ? (k > 0 ? lo + 0.5 * (hi - lo) : hi) : s + mu;
  }
  if (o_pole_difference_cancels(d[k], s, mu) || (k > 0 && o_pole_difference_cancels(d[k - 1], s, mu))) {
    *dd_out = 1;
    return rounds + o_r2_dd(n, d, z, rho, k, s, mu, e, u, sigma_out, mu_out);
  }
  *sigma_out = s;
  *mu_out = mu;
  return rounds;
}

/* Test entry point for o_r2: lambda_k by R2 from the estimate lam_est. */
int oracle_dpr1_r2(int n, const double* d, const double* z, double rho, int k, double lam_est, double* lambda,
                   double* sigma, double* mu) {
  if (n < 1 || k < 0 || k >= n || !(rho > 0.0)) return -1;
  double* e = (double*)malloc(sizeof(double) * n);
  double* u = (double*)malloc(sizeof(double) * n);
  if (!e || !u) { free(e); free(u); return -1; }
  int dd;
  int r = o_r2(n, d, z, rho, k, lam_est, 0.0, e, u, sigma, mu, &dd);
  if (r) *lambda = *sigma + *mu;
  free(e); free(u);
  return r;
}

/* ------------------------------------------------------------------------- */
/* Algorithm 1: the k-th eigenpair (k is 0-based here).                      */
/* ------------------------------------------------------------------------- */
/* The eigenpair needs values outside the binary64 range (of the normalised problem): mu is
   zero, subnormal or not finite (lambda lies within 2^-1022 of its shift, where mu and with it
   the eigenvector's components lose precision), or lambda or a component of v is not finite. */
static int o_out_of_range(int n, double mu, double lambda, const double* v) {
  if (!(fabs(mu) >= 0x1p-1022) || !isfinite(mu) || !isfinite(lambda)) return 1;
  if (v)
    for (int j = 0; j < n; j++)
      if (!isfinite(v[j])) return 1;
  return 0;
}

static int o_dpr1eig_core(int n, const double* d, const double* z, double rho, int k,
                          const oracle_opts* opt_in, double* lambda_out, double* v, oracle_info* info) {
  oracle_opts opt;
  if (opt_in) opt = *opt_in; else oracle_default_opts(&opt);
  if (n < 1 || k < 0 || k >= n || !(rho > 0.0)) return 1;
  double* delta = (double*)malloc(sizeof(double) * n);
  double* w = (double*)malloc(sizeof(double) * n);
  if (!delta || !w) { free(delta); free(w); return 2; }
  oracle_info inf;
  memset(&inf, 0, sizeof(inf));

  /* Shift choice: k = 1 -> sigma = d_1; otherwise evaluate f at the midpoint
     tau of (d_k, d_{k-1}) in coordinates shifted by d_k. */
  int i;
  if (k == 0) {
    i = 0;
  } else {
    double tau = (d[k - 1] - d[k]) / 2.0;
    double s = 0.0;
    for (int j = 0; j < n; j++) {
      double dbar = d[j] - d[k];
      s += z[j] * z[j] / (dbar - tau);
    }
    double F = 1.0 + rho * s;
    i = (F > 0.0) ? k : k - 1;
  }
  inf.first_shift = i;

  o_pole_solve ps;
  o_solve_at_pole(n, d, z, rho, k, i, &opt, delta, w, &ps);
  inf.used_dd = ps.used_dd;
  inf.K_nu = ps.K_nu;
  inf.kappa_nu = ps.kappa_nu;
  double sigma = d[i];
  double mu = ps.mu, nu = ps.nu;
  double K = ps.K_nu;
  int steps = ps.steps;
  double b = ps.b;
  int shift = i;

  if ((opt.remedies & 1) && K > opt.T_Knu) {
    /* (R1): the neighbouring pole on the other side of lambda, if there is one.  The
       eigenvector formula at that pole divides by (d_j - d_other) - mu, which cancels
       for the nearer pole j = i by the factor |lambda - d_other| / |lambda - d_i|; R1
       is taken when that factor and K_nu at the other pole are both within T_Knu. */
    int other = (i == k) ? k - 1 : k;
    double best_sigma = sigma, best_mu = mu, best_K = K;
    if (other >= 0 && other != i) {
      o_pole_solve p2;
      o_solve_at_pole(n, d, z, rho, k, other, &opt, delta, w, &p2);
      double ratio = fabs((d[i] - d[other]) + mu) / fabs(mu);
      inf.used_dd = inf.used_dd || p2.used_dd;
      if (p2.K_nu < K && p2.K_nu <= opt.T_Knu && ratio <= opt.T_Knu) {
        shift = other; sigma = d[other]; mu = p2.mu; nu = p2.nu; K = p2.K_nu;
        steps = p2.steps; b = p2.b; inf.remedy = 1;
      }
      if (p2.K_nu < best_K) { best_sigma = d[other]; best_mu = p2.mu; best_K = p2.K_nu; }
    }
    if (K > opt.T_Knu) {
      /* (R2): a non-pole shift next to lambda, from the better of the two pole solutions
         (the one with the smaller K_nu) */
      double s2, mu2;
      int dd2;
      if (o_r2(n, d, z, rho, k, best_sigma, best_mu, delta, w, &s2, &mu2, &dd2)) {
        shift = -1; sigma = s2; mu = mu2; nu = (mu2 != 0.0) ? 1.0 / mu2 : INFINITY; K = 1.0;
        steps = 0; inf.remedy = 2; inf.used_dd = 1; inf.r2_dd = dd2;
      }
    }
  }

  /* eigenvector and eigenvalue at the final shift */
  if (shift >= 0) o_vector_pole(n, d, z, shift, mu, v);
  else o_vector_shift(n, d, z, sigma, mu, v);
  double lambda = mu + sigma;

  /* lambda much closer to zero than to its neighbouring poles: recompute from A^{-1} */
  if (opt.remedies & 2) {
    int allnz = 1;
    for (int j = 0; j < n; j++) if (d[j] == 0.0) { allnz = 0; break; }
    double m1 = fabs(lambda - d[k]);
    if (k > 0) { double m2 = fabs(lambda - d[k - 1]); if (m2 < m1) m1 = m2; }
    if (allnz && opt.T_zero * fabs(lambda) < m1) {
      double mu0;
      int ok = o_solve_nonpole(n, d, z, rho, 0.0, 0.0, delta, w, &mu0, NULL);
      lambda = ok ? mu0 : 0.0;
      inf.zero_path = 1;
    }
  }

  inf.shift = shift; inf.sigma = sigma; inf.mu = mu; inf.nu = nu; inf.lambda = lambda;
  inf.b = b; inf.K_nu_final = K; inf.steps = steps;
  *lambda_out = lambda;
  if (info) *info = inf;
  free(delta); free(w);
  if (shift < 0 && (o_pole_difference_cancels(d[k], sigma, mu) ||
                    (k > 0 && o_pole_difference_cancels(d[k - 1], sigma, mu))))
    return 4;
  return o_out_of_range(n, mu, lambda, v) ? 4 : 0;
}

/*
 * Exact power-of-two normalisation (the paper takes the data in range).  With
 * max|d_j| = m_d 2^e_d, max|zeta_j| = m_z 2^e_z and rho = m_r 2^e_r (m in [1/2, 1), e = 0 for
 * a zero), a = max(e_d, e_r + 2 e_z) and b = e_z: D' = 2^-a D, z' = 2^-b z,
 * rho' = 2^(2b - a) rho, and A = 2^a (D' + rho' z' z'^T) has the same eigenvectors and
 * lambda = 2^a lambda'.  Multiplying by a power of two changes no rounding while everything
 * stays in the normal range, so in range this gives the bits of the unnormalised computation;
 * outside it the matrix scale is about 1, rho' <= 4 and max|zeta'| is in [1/2, 1), which keeps
 * zeta_j^2, rho zeta_j^2 and the poles' differences away from overflow.
 */
void oracle_scale_exponents(int n, const double* d, const double* z, double rho, int* a_out, int* b_out) {
  double md = 0.0, mz = 0.0;
  for (int j = 0; j < n; j++) {
    if (fabs(d[j]) > md) md = fabs(d[j]);
    if (fabs(z[j]) > mz) mz = fabs(z[j]);
  }
  int ed = 0, ez = 0, er = 0;
  if (md > 0.0 && isfinite(md)) frexp(md, &ed);
  if (mz > 0.0 && isfinite(mz)) frexp(mz, &ez);
  if (rho > 0.0 && isfinite(rho)) frexp(rho, &er);
  int a = ed;
  if (!(md > 0.0) && mz > 0.0 && rho > 0.0) a = er + 2 * ez;
  *a_out = a;
  *b_out = ez;
}

int oracle_dpr1eig(int n, const double* d, const double* z, double rho, int k,
                   const oracle_opts* opt_in, double* lambda_out, double* v, oracle_info* info) {
  if (n < 1 || k < 0 || k >= n || !(rho > 0.0)) return 1;
  int a, b;
  oracle_scale_exponents(n, d, z, rho, &a, &b);
  double* ds = (double*)malloc(sizeof(double) * n);
  double* zs = (double*)malloc(sizeof(double) * n);
  if (!ds || !zs) { free(ds); free(zs); return 2; }
  for (int j = 0; j < n; j++) { ds[j] = ldexp(d[j], -a); zs[j] = ldexp(z[j], -b); }
  const double rs = ldexp(rho, 2 * b - a);
  /* rho' = 0 (the rank-one part below 2^-1074 of the poles' scale): outside the range */
  int rc = (rs > 0.0) ? o_dpr1eig_core(n, ds, zs, rs, k, opt_in, lambda_out, v, info) : 4;
  free(ds); free(zs);
  if (rc && rc != 4) return rc;
  if (rs == 0.0) return 4;
  *lambda_out = ldexp(*lambda_out, a);
  if (info) {
    info->sigma = ldexp(info->sigma, a);
    info->mu = ldexp(info->mu, a);
    info->lambda = ldexp(info->lambda, a);
    info->nu = ldexp(info->nu, -a);
    info->b = ldexp(info->b, -a);
  }
  return rc;
}

/* All eigenpairs k in [k0, k1): lambda[k], V row-major with row k = v_k, plus (sigma, mu). */
int oracle_dpr1eig_range(int n, const double* d, const double* z, double rho, int k0, int k1,
                         const oracle_opts* opt, double* lambda, double* Vt, double* sigma,
                         double* mu, int* shift, int* flags) {
  for (int k = k0; k < k1; k++) {
    oracle_info inf;
    int rc = oracle_dpr1eig(n, d, z, rho, k, opt, &lambda[k], Vt ? &Vt[(size_t)k * n] : NULL, &inf);
    if (rc) return rc;
    if (sigma) sigma[k] = inf.sigma;
    if (mu) mu[k] = inf.mu;
    if (shift) shift[k] = inf.shift;
    if (flags) flags[k] = inf.remedy | (inf.zero_path << 2) | (inf.used_dd << 3);
  }
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Adjoint of (lambda, V) with respect to (d, z, rho).                        */
/* From the implicit derivative of f(lambda_k) = 0 (Eq. (Pick)) and the        */
/* explicit x_k = (D - lambda_k I)^{-1} z, v_k = x_k/||x_k|| (Eq. (Aeigenvec)): */
/*   s_j = d_j - lambda_k = (d_j - sigma_k) - mu_k,                            */
/*   dlambda/dd_j = v_j^2, dlambda/dzeta_j = -2 x_j/||x||^2,                  */
/*   dlambda/drho = 1/(rho^2 ||x||^2);                                        */
/*   with vbar = dL/dv_k and c = v^T vbar, g = vbar - v c; gbar = g/||x||     */
/*   is the adjoint of x, and                                                 */
/*   lambda_bar = grad_lambda_k + sum_j g_j v_j / s_j,                         */
/*   dbar_j += lambda_bar v_j^2 - g_j v_j / s_j,                               */
/*   zbar_j += (g_j / s_j - 2 lambda_bar v_j) / ||x||,                         */
/*   rhobar += lambda_bar / (rho ||x||)^2.                                     */
/* Evaluation: let p be the index of the largest |v_p|.  When v is close to   */
/* e_p (lambda_k next to the pole d_p), g_p and the two parts of dbar_p cancel */
/* at the scale 1/s_p; with S2 = sum_{j != p} v_j^2 = 1 - v_p^2 and            */
/* P = sum_{j != p} v_j vbar_j the same quantities are                         */
/*   g_p = vbar_p S2 - v_p P,                                                  */
/*   lambda_bar = Lam + T_p, Lam = grad_lambda_k + sum_{j != p} g_j v_j / s_j,  */
/*   T_p = g_p v_p / s_p,                                                      */
/*   dbar_p += Lam v_p^2 - T_p S2,                                             */
/*   zbar_p += (g_p / s_p (S2 - v_p^2) - 2 Lam v_p) / ||x||,                   */
/* which have no such cancellation.                                            */
/* grad_lambda or grad_Vt may be NULL (zero).  Rows of grad_Vt are dL/dv_k.   */
/* ------------------------------------------------------------------------- */
int oracle_backward_rows(int n, const double* d, const double* z, double rho, int m, const int* rows,
                         const double* sigma, const double* mu,
                         const double* grad_lambda, const double* grad_Vt,
                         double* grad_d, double* grad_z, double* grad_rho);

int oracle_backward(int n, const double* d, const double* z, double rho,
                    const double* sigma, const double* mu,
                    const double* grad_lambda, const double* grad_Vt,
                    double* grad_d, double* grad_z, double* grad_rho) {
  return oracle_backward_rows(n, d, z, rho, n, NULL, sigma, mu, grad_lambda, grad_Vt, grad_d, grad_z, grad_rho);
}

/* The same sum restricted to m eigenpairs; sigma, mu, grad_lambda and the rows of grad_Vt
   are indexed by position in that list (rows is unused and may be NULL). */
int oracle_backward_rows(int n, const double* d, const double* z, double rho, int m, const int* rows,
                         const double* sigma, const double* mu,
                         const double* grad_lambda, const double* grad_Vt,
                         double* grad_d, double* grad_z, double* grad_rho) {
  double* s = (double*)malloc(sizeof(double) * n);
  double* v = (double*)malloc(sizeof(double) * n);
  double* g = (double*)malloc(sizeof(double) * n);
  if (!s || !v || !g) { free(s); free(v); free(g); return 2; }
  (void)rows;
  for (int j = 0; j < n; j++) { grad_d[j] = 0.0; grad_z[j] = 0.0; }
  double grho = 0.0;
  for (int k = 0; k < m; k++) {
    double mx = 0.0;
    int p = 0;
    for (int j = 0; j < n; j++) {
      s[j] = (d[j] - sigma[k]) - mu[k];
      v[j] = z[j] / s[j];
      if (fabs(v[j]) > mx) { mx = fabs(v[j]); p = j; }
    }
    double q = 0.0;
    for (int j = 0; j < n; j++) { double t = v[j] / mx; q += t * t; }
    double xn = mx * sqrt(q);                /* ||x|| */
    for (int j = 0; j < n; j++) v[j] = (v[j] / mx) / sqrt(q);
    const double* vb = grad_Vt ? &grad_Vt[(size_t)k * n] : NULL;
    double S2 = 0.0, P = 0.0;
    for (int j = 0; j < n; j++) {
      if (j == p) continue;
      S2 += v[j] * v[j];
      if (vb) P += v[j] * vb[j];
    }
    double c = vb ? v[p] * vb[p] + P : 0.0;
    for (int j = 0; j < n; j++) g[j] = vb ? vb[j] - v[j] * c : 0.0;
    if (vb) g[p] = vb[p] * S2 - v[p] * P;
    double Lam = grad_lambda ? grad_lambda[k] : 0.0;
    for (int j = 0; j < n; j++) if (j != p) Lam += g[j] * v[j] / s[j];
    double Tp = g[p] * v[p] / s[p];
    double lb = Lam + Tp;
    for (int j = 0; j < n; j++) {
      if (j == p) {
        grad_d[j] += Lam * v[j] * v[j] - Tp * S2;
        grad_z[j] += ((g[j] / s[j]) * (S2 - v[j] * v[j]) - 2.0 * Lam * v[j]) / xn;
      } else {
        grad_d[j] += lb * v[j] * v[j] - g[j] * v[j] / s[j];
        grad_z[j] += (g[j] / s[j] - 2.0 * lb * v[j]) / xn;
      }
    }
    double t = 1.0 / (rho * xn);
    grho += lb * t * t;
  }
  *grad_rho = grho;
  free(s); free(v); free(g);
  return 0;
}

/* Real symmetric arrowhead matrices A = [D z; z^T alpha] of order n + 1      */
/* (the companion problem the paper relates its method to, Sec. 1).  The same */
/* steps as Algorithm 1: shift to the nearer pole d_i, form the inverse of    */
/* A - d_i I, which is again an arrowhead, bisect its secular equation for    */
/* the extreme eigenvalue nu, lambda = d_i + 1/nu, v = [x; -1] / ||.||,       */
/* x = (D - lambda I)^{-1} z; then the remedies of Sec. 2 when K_nu is large  */
/* and the near-zero recompute.  Irreducible input only (d strictly           */
/* decreasing, no zero weight).                                               */
/*                                                                            */
/* (A - d_i I)^{-1}: with Delta_j = d_j - d_i (j != i) it has the diagonal    */
/* delta_j = 1/Delta_j, b at position i and 0 at position n, and the border   */
/* (row i) w_j = -zeta_j / (zeta_i Delta_j), 1/zeta_i at position n, where    */
/*   b = (1/zeta_i^2) (sum_{j != i} zeta_j^2 / Delta_j - (alpha - d_i))       */
/* (the DPR1 corner of Eq. (b_ob) with 1/rho replaced by d_i - alpha).  Its   */
/* secular function has one more pole, at 0, of weight 1/zeta_i^2:            */
/*   g(nu) = b - nu - sum_{j != i} w_j^2/(delta_j - nu) + (1/zeta_i^2)/nu.    */
/*                                                                            */
/* (A - sigma I)^{-1} for sigma not a pole (R2, and sigma = 0 for the         */
/* near-zero recompute): with the Schur complement                            */
/*   f(sigma) = alpha - sigma - sum_j zeta_j^2 / (d_j - sigma)                */
/* of D - sigma I it equals diag(e, 0) + gamma u u^T, e_j = 1/(d_j - sigma),  */
/* u = [zeta_j/(d_j - sigma); -1], gamma = 1/f(sigma): a DPR1 matrix of order */
/* n + 1 whose extreme eigenvalue is 1/(lambda - sigma) for the eigenvalue    */
/* lambda next to sigma (the arrowhead form of Eq. (gamma)).                  */
/* ------------------------------------------------------------------------- */
typedef struct {
  int n, i;
  const double* delta;
  const double* w;
  double b, wz2;       /* corner and 1/zeta_i^2 */
} o_ah_ctx;

static double o_g_ah(const void* vctx, double nu) {
  const o_ah_ctx* c = (const o_ah_ctx*)vctx;
  double s = 0.0;
  for (int j = 0; j < c->n; j++) {
    if (j == c->i) continue;
    s += c->w[j] * c->w[j] / (c->delta[j] - nu);
  }
  return ((c->b - nu) - s) + c->wz2 / nu;
}

/* Forms the arrowhead inverse of A - d_i I: delta, w and the corner b (double-double). */
static void o_ah_form(int n, const double* d, const double* z, double alpha, int i, double* delta, double* w,
                      o_ah_ctx* c) {
  odd_t acc = o_two_sum(d[i], -alpha);
  for (int j = 0; j < n; j++) {
    if (j == i) { delta[j] = 0.0; w[j] = 0.0; continue; }
    delta[j] = 1.0 / (d[j] - d[i]);
    w[j] = -(delta[j] * z[j]) / z[i];
    acc = o_add(acc, o_div(o_two_prod(z[j], z[j]), o_two_sum(d[j], -d[i])));
  }
  odd_t bb = o_div(acc, o_two_prod(z[i], z[i]));
  double wz = 1.0 / z[i];
  c->n = n; c->i = i; c->delta = delta; c->w = w;
  c->b = bb.hi + bb.lo;
  c->wz2 = wz * wz;
}

/* Extreme eigenvalue of the arrowhead inverse, side = +1 rightmost, -1 leftmost.  Weyl
   bracket: within ||border|| of max(b, max delta, 0) (rightmost) or min(b, min delta, 0)
   (leftmost); the poles of g are the delta_j and 0. */
static double o_ah_extreme(const o_ah_ctx* c, int side, int* steps) {
  double wn2 = c->wz2, dmax = 0.0, dmin = 0.0;
  for (int j = 0; j < c->n; j++) {
    if (j == c->i) continue;
    wn2 += c->w[j] * c->w[j];
    if (c->delta[j] > dmax) dmax = c->delta[j];
    if (c->delta[j] < dmin) dmin = c->delta[j];
  }
  double wn = sqrt(wn2);
  if (side > 0) {
    double lo = c->b > dmax ? c->b : dmax;
    return o_bisect(o_g_ah, c, 1.0, lo, lo + wn, +1, steps);
  }
  double up = c->b < dmin ? c->b : dmin;
  return o_bisect(o_g_ah, c, -1.0, -up, -up + wn, -1, steps);
}

typedef struct {
  double nu, mu, K_nu;
  int steps;
} o_ah_pole;

/* Solve at pole i for eigenvalue k: the extreme eigenvalue of (A - d_i I)^{-1} on the side
   of lambda_k (rightmost when i == k, lambda_k > d_i; leftmost when i == k - 1) and
   K_nu = ||(A - d_i I)^{-1}||_2 / |nu| (Eq. (K0)), the norm being the larger of the
   |extreme eigenvalues|, both by bisection. */
static void o_ah_solve_at_pole(int n, const double* d, const double* z, double alpha, int k, int i,
                               double* delta, double* w, o_ah_pole* r) {
  o_ah_ctx c;
  o_ah_form(n, d, z, alpha, i, delta, w, &c);
  int side = (i == k) ? +1 : -1;
  int steps = 0;
  double nu = o_ah_extreme(&c, side, &steps);
  double other = o_ah_extreme(&c, -side, NULL);
  double nrm = fabs(nu) > fabs(other) ? fabs(nu) : fabs(other);
  r->nu = nu; r->mu = 1.0 / nu; r->K_nu = nrm / fabs(nu); r->steps = steps;
  /* a solve that left the binary64 range counts as K_nu = inf (as for D + rho z z^T) */
  if (!(r->K_nu >= 1.0) || !isfinite(nu) || r->mu == 0.0) r->K_nu = INFINITY;
}

typedef struct {
  int n;
  const double* e;   /* 1/(d_j - sigma) */
  const double* u;   /* zeta_j/(d_j - sigma) */
  double gamma;
} o_ahinv_ctx;

/* h(nu) = 1 + gamma (sum_j u_j^2/(e_j - nu) + 1/(0 - nu)), the secular function of
   diag(e, 0) + gamma u u^T with u_n = -1. */
static double o_h_ahinv(const void* vctx, double nu) {
  const o_ahinv_ctx* c = (const o_ahinv_ctx*)vctx;
  double s = 0.0;
  for (int j = 0; j < c->n; j++) s += c->u[j] * c->u[j] / (c->e[j] - nu);
  return 1.0 + c->gamma * (s - 1.0 / nu);
}

/* Non-pole shift sigma = s + t (t = 0: a binary64 shift; t != 0: the shift in double the working
   precision, the elements from the double-double differences d_j - sigma rounded to binary64, as
   o_solve_nonpole): returns 1 and mu (lambda = sigma + mu), or 0 when f(sigma) is zero in
   double-double (lambda = sigma, mu = 0). */
static int o_ah_solve_nonpole(int n, const double* d, const double* z, double alpha, double s, double t, double* e,
                              double* u, double* mu_out, int* steps) {
  odd_t f = o_diff(alpha, s, t);
  for (int j = 0; j < n; j++)
    f = o_add(f, o_neg(o_div(o_two_prod(z[j], z[j]), o_diff(d[j], s, t))));
  if (f.hi == 0.0 && f.lo == 0.0) { *mu_out = 0.0; if (steps) *steps = 0; return 0; }
  odd_t gdd = o_div(o_from(1.0), f);
  double gamma = gdd.hi + gdd.lo;
  double emax = 0.0, emin = 0.0, un2 = 1.0;   /* the pole at 0 and u_n^2 = 1 */
  for (int j = 0; j < n; j++) {
    double dj = o_diff(d[j], s, t).hi;
    e[j] = 1.0 / dj;
    u[j] = z[j] / dj;
    un2 += u[j] * u[j];
    if (e[j] > emax) emax = e[j];
    if (e[j] < emin) emin = e[j];
  }
  o_ahinv_ctx c = {n, e, u, gamma};
  double nu;
  /* gamma > 0: rightmost eigenvalue in [max(e, 0), max(e, 0) + gamma ||u||^2];
     gamma < 0: leftmost, mirrored; h < 0 on the pole side in both cases */
  if (gamma > 0) nu = o_bisect(o_h_ahinv, &c, 1.0, emax, emax + gamma * un2, -1, steps);
  else nu = o_bisect(o_h_ahinv, &c, -1.0, -emin, -emin - gamma * un2, -1, steps);
  *mu_out = 1.0 / nu;
  return 1;
}

/* (R2) for the arrowhead with the shift in double the working precision, as o_r2_dd: sigma =
   base + t with base the pole end of the interlacing interval nearer the lower end (d_k; d_{n-1}
   for k = n, whose interval lies below it), tau = |t| in (0, g) between two poles, or up to the
   Weyl end for an exterior eigenvalue; the result is returned against the nearer pole. */
static int o_ah_r2_dd(int n, const double* d, const double* z, double alpha, int k, double wlo, double whi,
                      double est_s, double est_m, double* e, double* u, double* sigma_out, double* mu_out) {
  const int lo_pole = k < n, hi_pole = k > 0;
  const double sgn = lo_pole ? 1.0 : -1.0;
  const double base = lo_pole ? d[k] : d[n - 1];
  odd_t g;
  if (lo_pole && hi_pole) g = o_two_sum(d[k - 1], -base);
  else g = o_from(lo_pole ? whi - base : base - wlo);   /* to the Weyl end */
  const double gw = g.hi + g.lo;
  const double mid = (lo_pole && hi_pole) ? 0.5 * gw : gw;
  odd_t te = o_add(o_two_sum(est_s, -base), o_from(est_m));
  double tau = sgn * (te.hi + te.lo), mu = 0.0;
  int rounds = 0;
  for (;;) {
    if (!(tau > 0.0) || !(tau <= gw) || (hi_pole && lo_pole && !(tau < gw))) tau = mid;
    o_ah_solve_nonpole(n, d, z, alpha, base, sgn * tau, e, u, &mu, NULL);
    rounds++;
    double room = tau;
    if (lo_pole && hi_pole && gw - tau < room) room = gw - tau;
    if (rounds >= 3 || fabs(mu) < 0.5 * room) break;
    tau = (rounds == 1) ? mid : tau + sgn * mu;
  }
  odd_t lm = o_two_sum(sgn * tau, mu);          /* lambda - base */
  if (lo_pole && hi_pole && lm.hi > 0.5 * gw) {
    odd_t up = o_add(lm, o_neg(g));             /* lambda - d_{k-1} */
    *sigma_out = d[k - 1];
    *mu_out = up.hi + up.lo;
  } else {
    *sigma_out = base;
    *mu_out = lm.hi + lm.lo;
  }
  return rounds;
}

/* (R2) for the arrowhead from an estimate est_s + est_m of lambda_k, as o_r2: the shift is moved
   into the interlacing interval of lambda_k, (d_k, d_{k-1}), with the exterior ends from
   Weyl's bounds, lambda_0 <= max(d_0, alpha) + ||z|| and lambda_n >= min(d_{n-1}, alpha) - ||z||;
   when |mu| is not below half the distance from sigma to the nearer pole end, the next shift
   is the midpoint (the Weyl bound of an exterior eigenvalue) and then the lambda found there
   (at most 3 solves).  When no binary64 shift lies between lambda_k and a neighbouring pole the
   shift is formed in double the working precision (o_ah_r2_dd; *dd_out = 1).  Returns the
   number of solves. */
static int o_ah_r2(int n, const double* d, const double* z, double alpha, int k, double est_s, double est_m,
                   double* e, double* u, double* sigma_out, double* mu_out, int* dd_out) {
  double zn = 0.0;
  for (int j = 0; j < n; j++) zn += z[j] * z[j];
  zn = sqrt(zn);
  const int lo_pole = k < n, hi_pole = k > 0;
  double lo = lo_pole ? d[k] : (d[n - 1] < alpha ? d[n - 1] : alpha) - zn;
  double hi = hi_pole ? d[k - 1] : (d[0] > alpha ? d[0] : alpha) + zn;
  double s = est_s + est_m, mu = 0.0;
  int rounds = 0;
  *dd_out = 0;
  for (;;) {
    if (lo_pole && !(s > lo)) s = nextafter(lo, INFINITY);
    if (!lo_pole && !(s >= lo)) s = lo;                    /* also a NaN estimate */
    if (hi_pole && s >= hi) s = nextafter(hi, -INFINITY);
    if (!hi_pole && s > hi) s = hi;
    if ((lo_pole && !(s > lo)) || (hi_pole && !(s < hi))) {
      *dd_out = 1;
      return rounds + o_ah_r2_dd(n, d, z, alpha, k, lo, hi, est_s, est_m, e, u, sigma_out, mu_out);
    }
    o_ah_solve_nonpole(n, d, z, alpha, s, 0.0, e, u, &mu, NULL);
    rounds++;
    double room = INFINITY;
    if (lo_pole) room = s - lo;
    if (hi_pole && hi - s < room) room = hi - s;
    if (rounds >= 3 || fabs(mu) < 0.5 * room) break;
    /* as o_r2: next the midpoint, or the Weyl bound of an exterior eigenvalue */
    s = (rounds == 1) ? (lo_pole && hi_pole ? lo + 0.5 * (hi - lo) : (hi_pole ? lo : hi)) : s + mu;
  }
  if ((lo_pole && o_pole_difference_cancels(d[k], s, mu)) || (hi_pole && o_pole_difference_cancels(d[k - 1], s, mu))) {
    *dd_out = 1;
    return rounds + o_ah_r2_dd(n, d, z, alpha, k, lo, hi, s, mu, e, u, sigma_out, mu_out);
  }
  *sigma_out = s;
  *mu_out = mu;
  return rounds;
}

/* Test entry point for o_ah_r2: lambda_k of the arrowhead by R2 from the estimate lam_est. */
int oracle_arrow_r2(int n, const double* d, const double* z, double alpha, int k, double lam_est, double* lambda,
                    double* sigma, double* mu) {
  if (n < 1 || k < 0 || k > n) return -1;
  double* e = (double*)malloc(sizeof(double) * n);
  double* u = (double*)malloc(sizeof(double) * n);
  if (!e || !u) { free(e); free(u); return -1; }
  int dd;
  int r = o_ah_r2(n, d, z, alpha, k, lam_est, 0.0, e, u, sigma, mu, &dd);
  if (r) *lambda = *sigma + *mu;
  free(e); free(u);
  return r;
}

/* Eigenvector [x; -1] / ||.||, x_j = zeta_j / ((d_j - sigma) - mu), scaled 2-norm. */
static void o_ah_vector(int n, const double* d, const double* z, double sigma, double mu, double* v) {
  double m = 1.0;
  for (int j = 0; j < n; j++) {
    double x = z[j] / ((d[j] - sigma) - mu);
    v[j] = x;
    if (fabs(x) > m) m = fabs(x);
  }
  v[n] = -1.0;
  double s = 0.0;
  for (int j = 0; j <= n; j++) { double t = v[j] / m; s += t * t; }
  double r = sqrt(s);
  for (int j = 0; j <= n; j++) v[j] = (v[j] / m) / r;
}

/* Eigenvalue k (0-based, 0..n) of the arrowhead; v has n + 1 entries.  opt: T_Knu, T_zero
   and remedies as for oracle_dpr1eig (NULL: defaults).  flags_out: remedy (1 R1, 2 R2) |
   4 when lambda was recomputed from A^{-1} | 8 when the R2 shift was formed in double the
   working precision.  shift_out: final pole, -1 for a non-pole shift. */
static int o_arroweig_core(int n, const double* d, const double* z, double alpha, int k, const oracle_opts* opt_in,
                           double* lambda_out, double* v, double* sigma_out, double* mu_out, int* shift_out,
                           int* flags_out, double* K_out) {
  oracle_opts opt;
  if (opt_in) opt = *opt_in; else oracle_default_opts(&opt);
  if (n < 1 || k < 0 || k > n) return 1;
  for (int j = 0; j < n; j++) {
    if (z[j] == 0.0 || (j + 1 < n && !(d[j] > d[j + 1]))) return 3;   /* reducible */
  }
  double* delta = (double*)malloc(sizeof(double) * n);
  double* w = (double*)malloc(sizeof(double) * n);
  if (!delta || !w) { free(delta); free(w); return 2; }
  /* shift: lambda_0 > d_0 (pole 0), lambda_n < d_{n-1} (pole n-1); otherwise
     lambda_k lies in (d_k, d_{k-1}) and f(lambda) = alpha - lambda - sum z_j^2/(d_j - lambda),
     decreasing there, is evaluated at the midpoint: f < 0 puts lambda in the lower half */
  int i;
  if (k == 0) i = 0;
  else if (k == n) i = n - 1;
  else {
    double tau = (d[k - 1] - d[k]) / 2.0;
    double s = 0.0;
    for (int j = 0; j < n; j++) s += z[j] * z[j] / ((d[j] - d[k]) - tau);
    double F = (alpha - d[k]) - tau - s;
    i = (F < 0.0) ? k : k - 1;
  }
  o_ah_pole ps;
  o_ah_solve_at_pole(n, d, z, alpha, k, i, delta, w, &ps);
  double sigma = d[i], mu = ps.mu, K = ps.K_nu;
  int shift = i, flags = 0;
  if (K_out) *K_out = K;

  if ((opt.remedies & 1) && K > opt.T_Knu) {
    /* (R1) the neighbouring pole on the other side of lambda_k, when there is one (none for
       the exterior eigenvalues), under the same acceptance rule as oracle_dpr1eig */
    int other = (i == k) ? k - 1 : k;
    double best_sigma = sigma, best_mu = mu, best_K = K;
    if (other >= 0 && other < n && other != i) {
      o_ah_pole p2;
      o_ah_solve_at_pole(n, d, z, alpha, k, other, delta, w, &p2);
      double ratio = fabs((d[i] - d[other]) + mu) / fabs(mu);
      if (p2.K_nu < K && p2.K_nu <= opt.T_Knu && ratio <= opt.T_Knu) {
        shift = other; sigma = d[other]; mu = p2.mu; K = p2.K_nu; flags = 1;
      }
      if (p2.K_nu < best_K) { best_sigma = d[other]; best_mu = p2.mu; best_K = p2.K_nu; }
    }
    if (K > opt.T_Knu) {
      /* (R2) from the better pole solution */
      double s2, mu2;
      int dd2;
      if (o_ah_r2(n, d, z, alpha, k, best_sigma, best_mu, delta, w, &s2, &mu2, &dd2)) {
        shift = -1; sigma = s2; mu = mu2; flags = 2 | (dd2 << 3);
      }
    }
  }
  o_ah_vector(n, d, z, sigma, mu, v);
  double lambda = sigma + mu;

  /* lambda much closer to zero than to its neighbouring poles: lambda = 1/nu, nu the extreme
     eigenvalue of A^{-1} (sigma = 0) */
  if (opt.remedies & 2) {
    int allnz = 1;
    for (int j = 0; j < n; j++) if (d[j] == 0.0) { allnz = 0; break; }
    double m1 = INFINITY;
    if (k < n) m1 = fabs(lambda - d[k]);
    if (k > 0) { double m2 = fabs(lambda - d[k - 1]); if (m2 < m1) m1 = m2; }
    if (allnz && opt.T_zero * fabs(lambda) < m1) {
      double mu0;
      int ok = o_ah_solve_nonpole(n, d, z, alpha, 0.0, 0.0, delta, w, &mu0, NULL);
      lambda = ok ? mu0 : 0.0;
      flags |= 4;
    }
  }
  *lambda_out = lambda;
  if (sigma_out) *sigma_out = sigma;
  if (mu_out) *mu_out = mu;
  if (shift_out) *shift_out = shift;
  if (flags_out) *flags_out = flags;
  free(delta); free(w);
  if (shift < 0 && ((k < n && o_pole_difference_cancels(d[k], sigma, mu)) ||
                    (k > 0 && o_pole_difference_cancels(d[k - 1], sigma, mu))))
    return 4;
  return o_out_of_range(n + 1, mu, lambda, v) ? 4 : 0;
}

/* Exact power-of-two normalisation of the arrowhead (the whole matrix scales together):
   a = e of max(|d_j|, |zeta_j|, |alpha|) = m 2^e, A' = 2^-a A, lambda = 2^a lambda', the same
   eigenvectors; in range this gives the bits of the unnormalised computation. */
int oracle_arroweig(int n, const double* d, const double* z, double alpha, int k, const oracle_opts* opt_in,
                    double* lambda_out, double* v, double* sigma_out, double* mu_out, int* shift_out,
                    int* flags_out, double* K_out) {
  if (n < 1 || k < 0 || k > n) return 1;
  double m = fabs(alpha);
  for (int j = 0; j < n; j++) {
    if (fabs(d[j]) > m) m = fabs(d[j]);
    if (fabs(z[j]) > m) m = fabs(z[j]);
  }
  int a = 0;
  if (m > 0.0 && isfinite(m)) frexp(m, &a);
  double* ds = (double*)malloc(sizeof(double) * n);
  double* zs = (double*)malloc(sizeof(double) * n);
  if (!ds || !zs) { free(ds); free(zs); return 2; }
  for (int j = 0; j < n; j++) { ds[j] = ldexp(d[j], -a); zs[j] = ldexp(z[j], -a); }
  double sg = 0.0, mu = 0.0;
  int rc = o_arroweig_core(n, ds, zs, ldexp(alpha, -a), k, opt_in, lambda_out, v, &sg, &mu, shift_out, flags_out,
                           K_out);
  free(ds); free(zs);
  if (rc && rc != 4) return rc;
  *lambda_out = ldexp(*lambda_out, a);
  if (sigma_out) *sigma_out = ldexp(sg, a);
  if (mu_out) *mu_out = ldexp(mu, a);
  return rc;
}
