// dpr1_solve.cuh -- per-eigenvalue solvers shared by the DPR1 kernels (sm_103a).
//
// A lane group of L threads (L = 8, 16 or 32) evaluates each secular function together:
// every lane sums its strided share of the terms and an xor-shuffle reduction gives every
// lane the bit-identical total, so all lanes take the same bisection decisions.
//   solve_pole     extreme eigenvalue nu of the arrowhead inverse of A - d_i I
//                  (Eq. (invAi), (b_ob), (secAi)); b in double-double (Sec. 2.3)
//   solve_nonpole  exterior eigenvalue of (A - sigma I)^{-1} for a non-pole shift sigma
//                  (remedy R2, and sigma = 0 for Eq. (gamma))
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "dpr1_device.cuh"

namespace dpr1 {

// ---------------------------------------------------------------------------------
// Secular sums
// ---------------------------------------------------------------------------------
// S(nu) = sum_{j != i} zz_j / (Delta_j (1 - nu Delta_j)),  Delta_j = d_j - d_i.
// With delta_j = 1/Delta_j and w_j = -zeta_j / (zeta_i Delta_j) (Eq. (invAi)) this is
// zeta_i^2 sum_j w_j^2 / (delta_j - nu), the sum of Eq. (secAi); multiplying the
// numerator and denominator by Delta_j leaves one division per term and forms
// 1 - nu Delta_j with a single rounding (fma).  For the extreme eigenvalue every term
// has the same sign.
// The hot sums use the fast reciprocal without a per-term range test; each lane records
// whether any denominator left the fast range and, if a lane of the group saw one, the
// group recomputes the sum with the range-safe reciprocal (never the case for sane data).
template <int L, bool SAFE>
__device__ __forceinline__ double arrow_sum_pass(const double* __restrict__ d, const double* __restrict__ zz, int n,
                                                 int i, double di, double nu, int lane, unsigned gm, bool* bad) {
  double s0 = 0.0, s1 = 0.0;
  bool b = false;
  int j = lane;
  for (; j + L < n; j += 2 * L) {
    double D0 = __dsub_rn(d[j], di), D1 = __dsub_rn(d[j + L], di);
    double t0 = __fma_rn(-nu, D0, 1.0), t1 = __fma_rn(-nu, D1, 1.0);
    double x0 = __dmul_rn(D0, t0), x1 = __dmul_rn(D1, t1);
    double r0, r1;
    if (SAFE) { r0 = rcp(x0); r1 = rcp(x1); }
    else {
      r0 = rcp_nr(x0); r1 = rcp_nr(x1);
      b |= (!rcp_in_range(x0) && j != i) || (!rcp_in_range(x1) && j + L != i);
    }
    // the excluded term j == i (0 * inf) is removed by selecting a zero reciprocal
    s0 = __fma_rn(zz[j], (j == i) ? 0.0 : r0, s0);
    s1 = __fma_rn(zz[j + L], (j + L == i) ? 0.0 : r1, s1);
  }
  if (j < n) {
    double D0 = __dsub_rn(d[j], di);
    double t0 = __fma_rn(-nu, D0, 1.0);
    double x0 = __dmul_rn(D0, t0);
    double r0;
    if (SAFE) r0 = rcp(x0);
    else { r0 = rcp_nr(x0); b |= !rcp_in_range(x0) && j != i; }
    s0 = __fma_rn(zz[j], (j == i) ? 0.0 : r0, s0);
  }
  *bad = b;
  return group_sum<L>(__dadd_rn(s0, s1), gm);
}

template <int L>
__device__ __forceinline__ double arrow_sum(const double* __restrict__ d, const double* __restrict__ zz, int n,
                                            int i, double di, double nu, int lane, unsigned gm) {
  bool bad;
  double s = arrow_sum_pass<L, false>(d, zz, n, i, di, nu, lane, gm, &bad);
  if (group_any<L>(bad, gm)) s = arrow_sum_pass<L, true>(d, zz, n, i, di, nu, lane, gm, &bad);
  return s;
}

// Same terms with Delta_j = d_j - sigma for a non-pole shift (no excluded index):
// sum_j u_j^2 / (e_j - nu), e_j = 1/(d_j - sigma), u_j = zeta_j/(d_j - sigma).
template <int L, bool SAFE>
__device__ __forceinline__ double shift_sum_pass(const double* __restrict__ d, const double* __restrict__ zz, int n,
                                                 double sigma, double nu, int lane, unsigned gm, bool* bad) {
  double s0 = 0.0, s1 = 0.0;
  bool b = false;
  int j = lane;
  for (; j + L < n; j += 2 * L) {
    double D0 = __dsub_rn(d[j], sigma), D1 = __dsub_rn(d[j + L], sigma);
    double t0 = __fma_rn(-nu, D0, 1.0), t1 = __fma_rn(-nu, D1, 1.0);
    double x0 = __dmul_rn(D0, t0), x1 = __dmul_rn(D1, t1);
    double r0, r1;
    if (SAFE) { r0 = rcp(x0); r1 = rcp(x1); }
    else { r0 = rcp_nr(x0); r1 = rcp_nr(x1); b |= !rcp_in_range(x0) || !rcp_in_range(x1); }
    s0 = __fma_rn(zz[j], r0, s0);
    s1 = __fma_rn(zz[j + L], r1, s1);
  }
  if (j < n) {
    double D0 = __dsub_rn(d[j], sigma);
    double t0 = __fma_rn(-nu, D0, 1.0);
    double x0 = __dmul_rn(D0, t0);
    double r0;
    if (SAFE) r0 = rcp(x0);
    else { r0 = rcp_nr(x0); b |= !rcp_in_range(x0); }
    s0 = __fma_rn(zz[j], r0, s0);
  }
  *bad = b;
  return group_sum<L>(__dadd_rn(s0, s1), gm);
}

template <int L>
__device__ __forceinline__ double shift_sum(const double* __restrict__ d, const double* __restrict__ zz, int n,
                                            double sigma, double nu, int lane, unsigned gm) {
  bool bad;
  double s = shift_sum_pass<L, false>(d, zz, n, sigma, nu, lane, gm, &bad);
  if (group_any<L>(bad, gm)) s = shift_sum_pass<L, true>(d, zz, n, sigma, nu, lane, gm, &bad);
  return s;
}

// sum_{j != skip} zeta_j^2 / (d_j - s) in double-double (skip = -1: all j); also returns
// sum_{j != skip} zeta_j^2 / (d_j - s)^2 in binary64 (the squared norm of the border).
template <int L>
__device__ __forceinline__ dd dd_pole_sum(const double* __restrict__ d, const double* __restrict__ z, int n,
                                          int skip, double s, int lane, unsigned gm, double* sq,
                                          double* cub = nullptr) {
  dd acc = {0.0, 0.0};
  double q = 0.0, c3 = 0.0;
  for (int j = lane; j < n; j += L) {
    if (j == skip) continue;
    dd D = two_sum(d[j], -s);
    dd Z = two_prod(z[j], z[j]);
    dd c = dd_div(Z, D);
    acc = dd_add(acc, c);
    double r = rcp(D.hi);
    double c2 = __dmul_rn(c.hi, r);
    q = __dadd_rn(q, c2);
    if (cub) c3 = __fma_rn(c2, r, c3);
  }
  *sq = group_sum<L>(q, gm);
  if (cub) *cub = group_sum<L>(c3, gm);
  return group_sum_dd<L>(acc, gm);
}

// ---------------------------------------------------------------------------------
// Bit-pattern bisection of a secular function on |nu| for nu = side*|nu|.
// phi(nu) has sign `below` for |nu| between `floor` and the root and the opposite sign
// beyond it.  `floor` is a pole of phi (or 0) that is known to lie below the root and
// is never evaluated; [alo, ahi] is an estimate of the bracket: its far end is checked
// and pushed out while it is still below the root, its near end (when above the floor)
// is checked and moved down towards the floor while it is above the root.  Every lane
// of the group runs the same loop (the sums are identical in every lane).  Returns nu
// with the smaller |phi| of the final adjacent pair; *ok = false if the cap was reached.
// ---------------------------------------------------------------------------------
template <class Phi>
__device__ double bisect(Phi phi, double side, double floor, double alo, double ahi, bool below_positive, int cap,
                         bool* ok, int* steps_out) {
  int steps = 0;
  bool good = true;
  if (!(floor >= 0.0)) floor = 0.0;
  if (!(alo >= floor)) alo = floor;
  if (!(ahi > alo)) ahi = (alo > 0.0) ? alo * 2.0 : 1.0;
  const uint64_t fl = dbits(floor);
  uint64_t lo = dbits(alo), hi = dbits(ahi);
  double glo = 0.0, ghi = 0.0;
  bool have_lo = false, have_hi = false;
  // far end: pushed out geometrically (in bit space) while it is still below the root
  for (int t = 0; t < 64; t++) {
    double g = phi(side * dfrom(hi));
    steps++;
    bool below = below_positive ? (g > 0.0) : (g < 0.0);
    if (!below) { ghi = g; have_hi = true; break; }
    uint64_t wd = hi - lo;
    lo = hi; glo = g; have_lo = true;
    hi = hi + 2 * wd + 64;
    if (hi >= 0x7ff0000000000000ull) { hi = 0x7fefffffffffffffull; }
  }
  // near end (when above the floor): if the root lies below it, fall back to the floor
  if (!have_lo && lo > fl) {
    double g = phi(side * dfrom(lo));
    steps++;
    bool below = below_positive ? (g > 0.0) : (g < 0.0);
    if (below) { glo = g; have_lo = true; }
    else { hi = lo; ghi = g; have_hi = true; lo = fl; }
  }
  int it = 0;
  while (hi - lo > 1) {
    if (it >= cap) { good = false; break; }
    uint64_t mid = lo + ((hi - lo) >> 1);
    double g = phi(side * dfrom(mid));
    bool below = below_positive ? (g > 0.0) : (g < 0.0);
    if (below) { lo = mid; glo = g; have_lo = true; }
    else { hi = mid; ghi = g; have_hi = true; }
    it++;
  }
  steps += it;
  if (!have_lo && lo > fl) { glo = phi(side * dfrom(lo)); steps++; have_lo = true; }
  if (!have_hi) { ghi = phi(side * dfrom(hi)); steps++; have_hi = true; }
  double alo_g = have_lo ? fabs(glo) : INFINITY;
  double ahi_g = fabs(ghi);
  if (isnan(alo_g)) alo_g = INFINITY;
  if (isnan(ahi_g)) ahi_g = INFINITY;
  *ok = good;
  if (steps_out) *steps_out = steps;
  return side * dfrom((ahi_g < alo_g) ? hi : lo);
}

// ---------------------------------------------------------------------------------
// Solve at a pole: extreme eigenvalue of the arrowhead inverse of A - d_i I.
// ---------------------------------------------------------------------------------
struct PoleResult {
  double mu, nu, b;
  bool ok;
  int steps;
};

// dd corner element of Eq. (b_ob): b = (1/zeta_i^2)(1/rho + sum_{j != i} zeta_j^2/(d_j - d_i)),
// rounded to binary64 (the arrowhead is formed in working precision).
template <int L>
__device__ __forceinline__ double corner_b(const double* __restrict__ d, const double* __restrict__ z, int n, int i,
                                           double rho, int lane, unsigned gm, double* wn2) {
  double sq;
  dd acc = dd_pole_sum<L>(d, z, n, i, d[i], lane, gm, &sq);
  dd B = dd_add(dd_div({1.0, 0.0}, {rho, 0.0}), acc);
  dd Zi = two_prod(z[i], z[i]);
  *wn2 = sq / Zi.hi;
  return dd_to_double(dd_div(B, Zi));
}

// Brackets of |nu| from the shift test (see the derivation in k_solve's comment).
template <int L>
__device__ PoleResult solve_pole(const double* __restrict__ d, const double* __restrict__ z,
                                 const double* __restrict__ zz, int n, double rho, int k, int i, double alo,
                                 double ahi, int cap, int lane, unsigned gm) {
  PoleResult r;
  double wn2;
  double b = corner_b<L>(d, z, n, i, rho, lane, gm, &wn2);
  double side = (i == k) ? 1.0 : -1.0;
  double di = d[i];
  double inv_zi2 = 1.0 / zz[i];
  // Weyl: the extreme eigenvalue lies within ||w|| of max(b, max delta) (rightmost) or
  // min(b, min delta) (leftmost); Rayleigh: nu >= b (rightmost), nu <= b (leftmost).
  double wn = sqrt(wn2);
  // floor: the pole of g next to the extreme eigenvalue (largest delta_j for the
  // rightmost, smallest for the leftmost), or 0 when all poles lie on the other side.
  double floor;
  // Corner bound: for the rightmost eigenvalue nu >= b and nu - b = sum_j w_j^2 / (nu - delta_j)
  // <= ||w||^2 / (b - max delta) when b > max delta (mirrored for the leftmost).  Next to a
  // pole b ~ 1/zeta_i^2 dominates and this bracket is narrow.
  if (side > 0) {
    // largest delta_j: the nearest pole above d_i, or for i = 0 the farthest pole below
    double dmax = (i > 0) ? 1.0 / (d[i - 1] - di) : (n > 1 ? 1.0 / (d[n - 1] - di) : -INFINITY);
    floor = fmax(dmax, 0.0);
    alo = fmax(alo, b);
    ahi = fmin(ahi, fmax(b, dmax) + wn);
    if (b > dmax) ahi = fmin(ahi, b + wn2 / (b - dmax));
  } else {
    double dmin = (i + 1 < n) ? 1.0 / (d[i + 1] - di) : INFINITY;
    floor = fmax(-dmin, 0.0);
    alo = fmax(alo, -b);
    ahi = fmin(ahi, -fmin(b, dmin) + wn);
    if (b < dmin) ahi = fmin(ahi, -b + wn2 / (dmin - b));
  }
  // a few ulps of margin for the rounding of the bounds; bisect() checks both ends
  alo = alo * (1.0 - 0x1p-48);
  ahi = ahi * (1.0 + 0x1p-48);
  auto phi = [&](double nu) {
    double S = arrow_sum<L>(d, zz, n, i, di, nu, lane, gm);
    return __dsub_rn(__dsub_rn(b, nu), __dmul_rn(S, inv_zi2));
  };
  bool ok;
  int steps;
  // g(nu) > 0 below the root for the rightmost; for the leftmost, |nu| below the root
  // means nu above it, where g < 0.
  double nu = bisect(phi, side, floor, alo, ahi, side > 0, cap, &ok, &steps);
  r.nu = nu;
  r.mu = 1.0 / nu;
  r.b = b;
  r.ok = ok;
  r.steps = steps;
  return r;
}

// ---------------------------------------------------------------------------------
// Non-pole shift sigma (R2, and sigma = 0 for Eq. (gamma)): form
//   f(sigma) = 1 + rho sum zeta_j^2 / (d_j - sigma) in double-double, gamma = -rho / f(sigma),
// and bisect h(nu) = 1 + gamma sum_j u_j^2 / (e_j - nu), e_j = 1/(d_j - sigma),
// u_j = zeta_j/(d_j - sigma), for the exterior eigenvalue of
// (A - sigma I)^{-1} = diag(e) + gamma u u^T: the rightmost (nu > 0) when gamma > 0, the
// leftmost when gamma < 0; h < 0 on the pole side in both cases.  Returns mu = 1/nu
// (lambda = sigma + mu); f(sigma) == 0 in double-double gives mu = 0.
// ---------------------------------------------------------------------------------
template <int L>
__device__ double solve_nonpole(const double* __restrict__ d, const double* __restrict__ z,
                                const double* __restrict__ zz, int n, double rho, double sigma, int above, int below,
                                int cap, int lane, unsigned gm, bool* ok, int* steps_out = nullptr) {
  // above / below: indices of the poles next to sigma (-1: none on that side)
  double un2, cub;
  dd acc = dd_pole_sum<L>(d, z, n, -1, sigma, lane, gm, &un2, &cub);
  dd f = dd_add({1.0, 0.0}, two_prod(acc.hi, rho));
  f = dd_add(f, {__dmul_rn(acc.lo, rho), 0.0});
  *ok = true;
  if (f.hi == 0.0 && f.lo == 0.0) return 0.0;
  double gamma = dd_to_double(dd_div({-rho, 0.0}, f));
  // extreme e_j = 1/(d_j - sigma): the poles next to sigma
  const double emax = above >= 0 ? 1.0 / __dsub_rn(d[above], sigma) : -INFINITY;
  const double emin = below >= 0 ? 1.0 / __dsub_rn(d[below], sigma) : INFINITY;
  // Rayleigh quotient of u: (sum_j e_j u_j^2)/||u||^2 + gamma ||u||^2, a lower bound of the
  // largest and an upper bound of the smallest eigenvalue of diag(e) + gamma u u^T; with
  // sigma next to lambda, gamma ||u||^2 dominates and the bracket below is narrow.
  const double rq = cub / un2 + gamma * un2;
  double side, floor, alo, ahi;
  if (gamma > 0.0) {
    side = 1.0;
    floor = fmax(emax, 0.0);
    alo = fmax(floor, rq * (1.0 - 0x1p-48));
    ahi = floor + gamma * un2;
  } else {
    side = -1.0;
    floor = fmax(-emin, 0.0);
    alo = fmax(floor, -rq * (1.0 - 0x1p-48));
    ahi = floor - gamma * un2;
  }
  ahi *= (1.0 + 0x1p-48);
  auto phi = [&](double nu) { return __fma_rn(gamma, shift_sum<L>(d, zz, n, sigma, nu, lane, gm), 1.0); };
  int steps;
  double nu = bisect(phi, side, floor, alo, ahi, false, cap, ok, &steps);
  if (steps_out) *steps_out = steps;
  return 1.0 / nu;
}

}  // namespace dpr1
