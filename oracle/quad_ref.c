/*
 * quad_ref.c -- binary128 reference for the eigenpairs of A = D + rho z z^T.
 *
 * TEST INFRASTRUCTURE ONLY (loaded by the tests and the smoke check).
 *
 * This is the plain definition of the result, not the paper's algorithm:
 *   lambda_k is the zero of the secular function
 *       f(lambda) = 1 + rho sum_j zeta_j^2 / (d_j - lambda)            (Eq. (Pick))
 *   in the interlacing interval (d_k, d_{k-1}), or (d_1, d_1 + rho ||z||^2] for k = 1
 *   (Eq. (interlace)); f is strictly increasing there for rho > 0.
 *   v_k = x / ||x||, x = (D - lambda_k I)^{-1} z                       (Eq. (Aeigenvec))
 * Everything is evaluated in IEEE binary128 (_Float128: 113-bit significand),
 * and lambda_k is found by bisection on the arithmetic midpoint until the two
 * end points are adjacent binary128 numbers (see quad_eigpair2 for the shifted
 * coordinates that keep the distance to the nearest pole accurate).
 *
 * k is 0-based.  lambda is returned as an unevaluated pair (hi, lo) of binary64
 * numbers (hi + lo carries about 106 bits); v is rounded to binary64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

typedef _Float128 q_t;

static q_t q_abs(q_t a) { return a < 0 ? -a : a; }

/* square root by Newton's iteration from the binary64 estimate, after an exact scaling by
   powers of four into [1, 4) (so that the estimate is neither zero nor infinite) */
static q_t q_sqrt(q_t a) {
  if (!(a > 0)) return 0;
  q_t s = 1;
  while (a >= (q_t)0x1p64) { a /= (q_t)0x1p64; s *= (q_t)0x1p32; }
  while (a < (q_t)0x1p-64) { a *= (q_t)0x1p64; s /= (q_t)0x1p32; }
  while (a >= 4) { a /= 4; s *= 2; }
  while (a < 1) { a *= 4; s /= 2; }
  q_t y = (q_t)sqrt((double)a);
  for (int t = 0; t < 3; t++) y = (y + a / y) / 2;
  return y * s;
}

/* f(d_i + mu) with D[j] = d_j - d_i formed in binary128 */
static q_t q_fshift(int n, const q_t* D, const double* z, double rho, q_t mu) {
  q_t s = 0;
  for (int j = 0; j < n; j++) {
    q_t zj = (q_t)z[j];
    s += zj * zj / (D[j] - mu);
  }
  return 1 + (q_t)rho * s;
}

static q_t q_f(int n, const double* d, const double* z, double rho, q_t lam) {
  q_t s = 0;
  for (int j = 0; j < n; j++) {
    q_t zj = (q_t)z[j];
    s += zj * zj / ((q_t)d[j] - lam);
  }
  return 1 + (q_t)rho * s;
}

/*
 * An arrowhead eigenvalue closer to zero than to its nearest pole (|lambda| < |mu|): d_i + mu
 * then carries an absolute error of about 2^-113 |d_i|, large next to |lambda|.  Instead lambda
 * is found by bisection of the secular function on lambda itself over [a, b] (an interlacing
 * interval); every d_j - lambda is then formed to 2^-113 relative, since no pole is nearer to
 * lambda than zero is, and the root carries 2^-113 (|alpha| + sum_j |zeta_j^2/(d_j - lambda)|)
 * divided by |f'| >= 1.  (For D + rho z z^T the same evaluation gains nothing: its secular
 * function 1 + rho sum_j ... cancels O(1) terms near such an eigenvalue.)  sgn_below is the
 * sign of the function between a and the root.
 */
typedef q_t (*q_secular_fn)(const void* ctx, q_t lam);

static q_t q_bisect_value(q_secular_fn fn, const void* ctx, q_t a, q_t b, int sgn_below) {
  for (int steps = 0; steps < 20000; steps++) {
    q_t mid = a + (b - a) / 2;
    if (!(mid > a && mid < b)) break;
    q_t f = fn(ctx, mid);
    if ((f > 0) == (sgn_below > 0) && f != 0) a = mid; else b = mid;
  }
  return a + (b - a) / 2;
}

/*
 * Bisection is done on mu = lambda - d_i in coordinates shifted by the nearer end
 * pole d_i of the interlacing interval, so that mu keeps 113 significant bits even
 * when lambda is within a few binary64 ulps of a pole: f(d_i + mu) is evaluated
 * as 1 + rho sum_j zeta_j^2 / ((d_j - d_i) - mu) with the pole differences formed
 * in binary128.  The nearer pole is found from the sign of f at the midpoint of
 * the interval (f > 0 there puts lambda in the lower half).
 * Returns the number of bisection steps, or -1 on bad arguments; *pole receives i.
 */
int quad_eigpair2(int n, const double* d, const double* z, double rho, int k,
                  double* lam_hi, double* lam_lo, double* mu_hi, double* mu_lo, int* pole, double* v) {
  if (n < 1 || k < 0 || k >= n || !(rho > 0)) return -1;
  q_t* D = (q_t*)malloc(sizeof(q_t) * n);
  if (!D) return -1;
  int i;
  q_t lo, hi;   /* bracket of mu */
  if (k == 0) {
    q_t zz = 0;
    for (int j = 0; j < n; j++) zz += (q_t)z[j] * (q_t)z[j];
    i = 0;
    lo = 0;
    hi = 2 * (q_t)rho * zz;
  } else {
    q_t tau = ((q_t)d[k - 1] - (q_t)d[k]) / 2;
    for (int j = 0; j < n; j++) D[j] = (q_t)d[j] - (q_t)d[k];
    q_t fm = q_fshift(n, D, z, rho, tau);
    if (fm > 0) { i = k; lo = 0; hi = tau; }
    else { i = k - 1; lo = -tau; hi = 0; }
  }
  for (int j = 0; j < n; j++) D[j] = (q_t)d[j] - (q_t)d[i];
  /* f(d_i + mu) is increasing in mu on the bracket */
  int steps = 0;
  q_t flo = NAN, fhi = NAN;
  int have_lo = 0, have_hi = 0;
  for (; steps < 20000; steps++) {
    q_t mid = lo + (hi - lo) / 2;
    if (!(mid > lo && mid < hi)) break;
    q_t fm = q_fshift(n, D, z, rho, mid);
    if (fm < 0) { lo = mid; flo = fm; have_lo = 1; }
    else { hi = mid; fhi = fm; have_hi = 1; }
  }
  q_t mu;
  if (have_lo && have_hi) mu = (q_abs(fhi) < q_abs(flo)) ? hi : lo;
  else if (have_hi) mu = hi;
  else mu = lo;
  q_t lam = (q_t)d[i] + mu;
  double h = (double)lam;
  *lam_hi = h;
  *lam_lo = (double)(lam - (q_t)h);
  h = (double)mu;
  *mu_hi = h;
  *mu_lo = (double)(mu - (q_t)h);
  *pole = i;
  if (v) {
    q_t m = 0;
    q_t* x = (q_t*)malloc(sizeof(q_t) * n);
    if (!x) { free(D); return -1; }
    for (int j = 0; j < n; j++) {
      x[j] = (q_t)z[j] / (D[j] - mu);
      if (q_abs(x[j]) > m) m = q_abs(x[j]);
    }
    q_t s = 0;
    for (int j = 0; j < n; j++) { q_t t = x[j] / m; s += t * t; }
    q_t r = q_sqrt(s);
    for (int j = 0; j < n; j++) v[j] = (double)((x[j] / m) / r);
    free(x);
  }
  free(D);
  return steps;
}

int quad_eigpair(int n, const double* d, const double* z, double rho, int k,
                 double* lam_hi, double* lam_lo, double* v) {
  double mh, ml; int pole;
  return quad_eigpair2(n, d, z, rho, k, lam_hi, lam_lo, &mh, &ml, &pole, v);
}

/*
 * Adjoint of (lambda, V) with respect to (d, z, rho) in binary128, from the plain
 * formulas (implicit derivative of f(lambda_k) = 0, explicit x = (D - lambda_k I)^{-1} z):
 *   s_j = d_j - lambda_k, v = x/||x||, c = v . vbar, g = vbar - v c,
 *   lambda_bar = grad_lambda_k + sum_j g_j v_j / s_j,
 *   dbar_j += lambda_bar v_j^2 - g_j v_j / s_j,
 *   zbar_j += (g_j / s_j - 2 lambda_bar v_j) / ||x||,  rhobar += lambda_bar / (rho ||x||)^2,
 * with lambda_k from the shifted binary128 bisection (s_j = (d_j - d_i) - mu).
 * Sums over the m eigenpairs ks[0..m); grad_lambda[t] and grad_Vt row t belong to ks[t].
 */
int quad_backward(int n, const double* d, const double* z, double rho, int m, const int* ks,
                  const double* grad_lambda, const double* grad_Vt, double* gd, double* gz, double* grho) {
  q_t* D = (q_t*)malloc(sizeof(q_t) * n);
  q_t* x = (q_t*)malloc(sizeof(q_t) * n);
  q_t* S = (q_t*)malloc(sizeof(q_t) * n);
  q_t* Gd = (q_t*)malloc(sizeof(q_t) * n);
  q_t* Gz = (q_t*)malloc(sizeof(q_t) * n);
  if (!D || !x || !S || !Gd || !Gz) { free(D); free(x); free(S); free(Gd); free(Gz); return -1; }
  for (int j = 0; j < n; j++) { Gd[j] = 0; Gz[j] = 0; }
  q_t Gr = 0;
  for (int t = 0; t < m; t++) {
    int k = ks ? ks[t] : t;
    double lh, ll, mh, ml;
    int pole;
    if (quad_eigpair2(n, d, z, rho, k, &lh, &ll, &mh, &ml, &pole, NULL) < 0) return -1;
    q_t mu = (q_t)mh + (q_t)ml;
    q_t mx = 0;
    for (int j = 0; j < n; j++) {
      S[j] = ((q_t)d[j] - (q_t)d[pole]) - mu;
      x[j] = (q_t)z[j] / S[j];
      if (q_abs(x[j]) > mx) mx = q_abs(x[j]);
    }
    q_t sq = 0;
    for (int j = 0; j < n; j++) { q_t u = x[j] / mx; sq += u * u; }
    q_t xn = mx * q_sqrt(sq);
    const double* vb = grad_Vt ? &grad_Vt[(size_t)t * n] : NULL;
    q_t c = 0;
    if (vb) for (int j = 0; j < n; j++) c += (x[j] / xn) * (q_t)vb[j];
    q_t lb = grad_lambda ? (q_t)grad_lambda[t] : 0;
    for (int j = 0; j < n; j++) {
      q_t v = x[j] / xn;
      q_t g = vb ? (q_t)vb[j] - v * c : 0;
      lb += g * v / S[j];
    }
    for (int j = 0; j < n; j++) {
      q_t v = x[j] / xn;
      q_t g = vb ? (q_t)vb[j] - v * c : 0;
      Gd[j] += lb * v * v - g * v / S[j];
      Gz[j] += (g / S[j] - 2 * lb * v) / xn;
    }
    q_t r = 1 / ((q_t)rho * xn);
    Gr += lb * r * r;
  }
  for (int j = 0; j < n; j++) { gd[j] = (double)Gd[j]; gz[j] = (double)Gz[j]; }
  *grho = (double)Gr;
  free(D); free(x); free(S); free(Gd); free(Gz);
  return 0;
}

/* f(lambda) at lambda = hi + lo, in binary128, rounded to binary64 (used by tests). */
double quad_secular(int n, const double* d, const double* z, double rho, double lam_hi, double lam_lo) {
  return (double)q_f(n, d, z, rho, (q_t)lam_hi + (q_t)lam_lo);
}

/*
 * Arrowhead A = [D z; z^T alpha] of order n + 1 (irreducible): lambda_k (k = 0..n) is the zero
 * of f(lambda) = alpha - lambda - sum_j zeta_j^2 / (d_j - lambda), strictly decreasing between
 * consecutive poles, in (d_0, inf) for k = 0, (d_k, d_{k-1}) for 0 < k < n and (-inf, d_{n-1})
 * for k = n; v_k = [x; -1] / ||.||, x = (D - lambda_k I)^{-1} z.  Bisection in binary128 on
 * mu = lambda - d_i, with the pole differences d_j - d_i formed in binary128, i the nearer end
 * pole of the interval (from the sign of f at its midpoint; the exterior intervals use the
 * pole they touch); an eigenvalue closer to zero than to that pole is then found by bisection
 * on lambda itself (q_bisect_value).  Returns the number of steps, or -1.
 */
static q_t q_fa(int n, const q_t* D, const double* z, q_t a, q_t mu) {
  q_t s = 0;
  for (int j = 0; j < n; j++) {
    q_t zj = (q_t)z[j];
    s += zj * zj / (D[j] - mu);
  }
  return (a - mu) - s;
}

typedef struct { int n; const double* d; const double* z; double alpha; } q_arrow_ctx;

/* f(lambda) = alpha - lambda - sum_j zeta_j^2 / (d_j - lambda), unshifted */
static q_t q_fa_ctx(const void* vc, q_t lam) {
  const q_arrow_ctx* c = (const q_arrow_ctx*)vc;
  q_t s = 0;
  for (int j = 0; j < c->n; j++) {
    q_t zj = (q_t)c->z[j];
    s += zj * zj / ((q_t)c->d[j] - lam);
  }
  return ((q_t)c->alpha - lam) - s;
}

int quad_arrow_eigpair(int n, const double* d, const double* z, double alpha, int k,
                       double* lam_hi, double* lam_lo, double* v) {
  if (n < 1 || k < 0 || k > n) return -1;
  q_t* D = (q_t*)malloc(sizeof(q_t) * n);
  if (!D) return -1;
  q_t zn = 0;
  for (int j = 0; j < n; j++) zn += (q_t)z[j] * (q_t)z[j];
  zn = q_sqrt(zn);
  int i;
  q_t lo, hi;
  if (k == 0 || k == n) {
    i = (k == 0) ? 0 : n - 1;
    q_t gap = (k == 0) ? (q_t)alpha - (q_t)d[0] : (q_t)d[n - 1] - (q_t)alpha;
    q_t U = (gap > 0 ? gap : 0) + zn;          /* Weyl: |lambda - d_i| <= max(0, gap) + ||z|| */
    if (k == 0) { lo = 0; hi = U; } else { lo = -U; hi = 0; }
  } else {
    q_t tau = ((q_t)d[k - 1] - (q_t)d[k]) / 2;
    for (int j = 0; j < n; j++) D[j] = (q_t)d[j] - (q_t)d[k];
    q_t fm = q_fa(n, D, z, (q_t)alpha - (q_t)d[k], tau);
    if (fm < 0) { i = k; lo = 0; hi = tau; }
    else { i = k - 1; lo = -tau; hi = 0; }
  }
  for (int j = 0; j < n; j++) D[j] = (q_t)d[j] - (q_t)d[i];
  q_t a = (q_t)alpha - (q_t)d[i];
  int steps = 0;
  /* f decreasing in mu on (lo, hi): f > 0 below the root */
  for (; steps < 20000; steps++) {
    q_t mid = lo + (hi - lo) / 2;
    if (!(mid > lo && mid < hi)) break;
    if (mid == 0) { /* never evaluate the pole itself */
      mid = (lo == 0) ? hi / 2 : lo / 2;
      if (!(mid > lo && mid < hi)) break;
    }
    q_t f = q_fa(n, D, z, a, mid);
    if (f > 0) lo = mid; else hi = mid;
  }
  q_t mu = lo + (hi - lo) / 2;
  q_t lam = (q_t)d[i] + mu;
  if (q_abs(lam) < q_abs(mu)) {
    q_arrow_ctx c = {n, d, z, alpha};
    q_t zn2 = 0;
    for (int j = 0; j < n; j++) zn2 += (q_t)z[j] * (q_t)z[j];
    q_t U = 2 * (q_abs((q_t)alpha) + q_abs((q_t)d[0]) + q_abs((q_t)d[n - 1]) + q_sqrt(zn2));
    q_t a = (k < n) ? (q_t)d[k] : -U, b = (k > 0) ? (q_t)d[k - 1] : U;
    lam = q_bisect_value(q_fa_ctx, &c, a, b, +1);   /* f decreasing: f > 0 below the root */
  }
  double h = (double)lam;
  *lam_hi = h;
  *lam_lo = (double)(lam - (q_t)h);
  if (v) {
    q_t nrm = 1;
    q_t* x = (q_t*)malloc(sizeof(q_t) * n);
    if (!x) { free(D); return -1; }
    for (int j = 0; j < n; j++) { x[j] = (q_t)z[j] / (D[j] - mu); nrm += x[j] * x[j]; }
    /* scale-safe square root: nrm >= 1 here */
    q_t r = q_sqrt(nrm);
    for (int j = 0; j < n; j++) v[j] = (double)(x[j] / r);
    v[n] = (double)(-1 / r);
    free(x);
  }
  free(D);
  return steps;
}
