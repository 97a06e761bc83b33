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

// unrolling of the evaluation loop over the stored elements
#ifndef DPR1_STORED_UNROLL
#define DPR1_STORED_UNROLL 2
#endif
// consecutive bisection steps the binary32 screen may fail to settle before it is given up
// (a failure means the midpoint fell within the screen's error window of the root; after the
// binary64 step the next midpoint lies a quarter of the bracket away and is often settled)
#ifndef DPR1_SCREEN_TRIES
#define DPR1_SCREEN_TRIES 2
#endif
// the double-float screen after the binary32 one, which is left after this many consecutive
// failures
#ifndef DPR1_SCREEN_DF
#define DPR1_SCREEN_DF 1
#endif
// the checks of the bracket's ends also try the screen
#ifndef DPR1_SCREEN_ENDS
#define DPR1_SCREEN_ENDS 1
#endif
// screened probes before the bisection that certify bounds next to the root (at most
// DPR1_PREDICT_STEPS; they stop once the certified bracket is at most kPredictStop doubles wide)
#ifndef DPR1_PREDICT
#define DPR1_PREDICT 1
#endif
#ifndef DPR1_PREDICT_STEPS
#define DPR1_PREDICT_STEPS 12
#endif
#ifndef DPR1_SCREEN32_TRIES
#define DPR1_SCREEN32_TRIES 2
#endif


namespace dpr1 {

constexpr int kStoredUnroll = DPR1_STORED_UNROLL;
constexpr int kScreenTries = DPR1_SCREEN_TRIES;
constexpr bool kScreenDf = DPR1_SCREEN_DF != 0;
constexpr int kScreen32Tries = DPR1_SCREEN32_TRIES;
constexpr bool kScreenEnds = DPR1_SCREEN_ENDS != 0;
constexpr bool kPredict = DPR1_PREDICT != 0;
constexpr int kPredictSteps = DPR1_PREDICT_STEPS;
constexpr uint64_t kPredictStop = 4;

// ---------------------------------------------------------------------------------
// Shifts in double the working precision (remedy R2 when no binary64 number lies between
// lambda and a neighbouring pole, Sec. 2): sigma = s + t, an unevaluated pair of binary64
// numbers.  The difference d_j - sigma is formed in double-double and the matrix element
// is its binary64 rounding; with OFS = false the shift is the binary64 number s and the
// element is fl(d_j - s).
// ---------------------------------------------------------------------------------
__device__ __forceinline__ dd shift_diff(double dj, double s, double t) {
  return dd_add(two_sum(dj, -s), {-t, 0.0});
}

template <bool OFS>
__device__ __forceinline__ double elem_diff(double dj, double s, double t) {
  if constexpr (OFS) return shift_diff(dj, s, t).hi;
  else return __dsub_rn(dj, s);
}

// ---------------------------------------------------------------------------------
// Secular sums
// ---------------------------------------------------------------------------------
// S(nu) = sum_{j != i} zz_j / (Delta_j (1 - nu Delta_j)),  Delta_j = d_j - d_i.
// With delta_j = 1/Delta_j and w_j = -zeta_j / (zeta_i Delta_j) (Eq. (invAi)) this is
// zeta_i^2 sum_j w_j^2 / (delta_j - nu), the sum of Eq. (secAi); multiplying the
// numerator and denominator by Delta_j leaves one division per term and forms
// 1 - nu Delta_j with a single rounding (fma).  For the extreme eigenvalue every term
// has the same sign.
// The bisection sums (neither SAFE nor DERIV) take two terms over one reciprocal (below).
// The hot sums use the fast reciprocal without a per-term range test; each lane records
// whether any denominator left the fast range and, if a lane of the group saw one, the
// group recomputes the sum with the range-safe reciprocal (never the case for sane data).
// With DERIV the pass also returns dS/dnu = sum_{j != i} zz_j / (1 - nu Delta_j)^2 (for the
// accelerated solve); i = -1 excludes no term (non-pole shifts, Delta_j = d_j - sigma).
// With OFS the shift is di + dlo in double the working precision (elem_diff).
template <int L, bool SAFE, bool DERIV, bool OFS = false>
__device__ __forceinline__ double arrow_sum_pass(const double* __restrict__ d, const double* __restrict__ zz, int n,
                                                 int i, double di, double nu, int lane, unsigned gm, bool* bad,
                                                 double* dsum, double dlo = 0.0) {
  double s0 = 0.0, s1 = 0.0, q0 = 0.0, q1 = 0.0;
  bool b = false;
  int j = lane;
  for (; j + L < n; j += 2 * L) {
    double D0 = elem_diff<OFS>(d[j], di, dlo), D1 = elem_diff<OFS>(d[j + L], di, dlo);
    double t0 = __fma_rn(-nu, D0, 1.0), t1 = __fma_rn(-nu, D1, 1.0);
    double x0 = __dmul_rn(D0, t0), x1 = __dmul_rn(D1, t1);
    if (!SAFE && !DERIV) {
      // Two terms over one reciprocal: zz0/x0 + zz1/x1 = (zz0 x1 + zz1 x0) / (x0 x1).  Beyond
      // every pole (the only place the solvers evaluate) all x_j have one sign, so the
      // numerator does not cancel.  The excluded term j == i enters as zz = 0, x = 1.
      const double y0 = (j == i) ? 1.0 : x0, y1 = (j + L == i) ? 1.0 : x1;
      const double w0 = (j == i) ? 0.0 : zz[j], w1 = (j + L == i) ? 0.0 : zz[j + L];
      const double num = __fma_rn(w0, y1, __dmul_rn(w1, y0));
      const double den = __dmul_rn(y0, y1);
      b |= !rcp_in_range(den) || !rcp_in_range(num);
      s0 = __fma_rn(num, rcp_nr(den), s0);
      continue;
    }
    double r0, r1;
    if (SAFE) { r0 = rcp(x0); r1 = rcp(x1); }
    else {
      r0 = rcp_nr(x0); r1 = rcp_nr(x1);
      b |= (!rcp_in_range(x0) && j != i) || (!rcp_in_range(x1) && j + L != i);
    }
    // the excluded term j == i (0 * inf) is removed by selecting a zero reciprocal
    r0 = (j == i) ? 0.0 : r0;
    r1 = (j + L == i) ? 0.0 : r1;
    s0 = __fma_rn(zz[j], r0, s0);
    s1 = __fma_rn(zz[j + L], r1, s1);
    if (DERIV) {
      double u0 = __dmul_rn(D0, r0), u1 = __dmul_rn(D1, r1);   // 1 / (1 - nu Delta_j)
      q0 = __fma_rn(__dmul_rn(zz[j], u0), u0, q0);
      q1 = __fma_rn(__dmul_rn(zz[j + L], u1), u1, q1);
    }
  }
  if (j < n) {
    double D0 = elem_diff<OFS>(d[j], di, dlo);
    double t0 = __fma_rn(-nu, D0, 1.0);
    double x0 = __dmul_rn(D0, t0);
    double r0;
    if (SAFE) r0 = rcp(x0);
    else { r0 = rcp_nr(x0); b |= !rcp_in_range(x0) && j != i; }
    r0 = (j == i) ? 0.0 : r0;
    s0 = __fma_rn(zz[j], r0, s0);
    if (DERIV) {
      double u0 = __dmul_rn(D0, r0);
      q0 = __fma_rn(__dmul_rn(zz[j], u0), u0, q0);
    }
  }
  *bad = b;
  if (DERIV) *dsum = group_sum<L>(__dadd_rn(q0, q1), gm);
  return group_sum<L>(__dadd_rn(s0, s1), gm);
}

template <int L, bool OFS = false>
__device__ __forceinline__ double arrow_sum(const double* __restrict__ d, const double* __restrict__ zz, int n,
                                            int i, double di, double nu, int lane, unsigned gm, double dlo = 0.0) {
  bool bad;
  double s = arrow_sum_pass<L, false, false, OFS>(d, zz, n, i, di, nu, lane, gm, &bad, nullptr, dlo);
  if (group_any<L>(bad, gm))
    s = arrow_sum_pass<L, true, false, OFS>(d, zz, n, i, di, nu, lane, gm, &bad, nullptr, dlo);
  return s;
}

// the sum and its derivative with respect to nu
template <int L, bool OFS = false>
__device__ __forceinline__ double arrow_sum_d(const double* __restrict__ d, const double* __restrict__ zz, int n,
                                              int i, double di, double nu, int lane, unsigned gm, double* dsum,
                                              double dlo = 0.0) {
  bool bad;
  double s = arrow_sum_pass<L, false, true, OFS>(d, zz, n, i, di, nu, lane, gm, &bad, dsum, dlo);
  if (group_any<L>(bad, gm)) s = arrow_sum_pass<L, true, true, OFS>(d, zz, n, i, di, nu, lane, gm, &bad, dsum, dlo);
  return s;
}

// The same sum S(nu) from the elements of the inverse formed once per eigenvalue (Eq. (invAi)):
// Ds[j] = Delta_j and us[j] = zz_j / Delta_j (both 0 at the excluded index j = i, which then
// adds 0 / 1), so each evaluation forms only t_j = 1 - nu Delta_j (one fma) and sums
// u_j / t_j, four terms over one reciprocal:
//   u0/t0 + u1/t1 = (u0 t1 + u1 t0) / (t0 t1),  and two such pairs combined the same way.
// Every u_j / t_j = zz_j / (Delta_j t_j) has the sign of the sum, so each u_a t_b of a numerator
// has the sign of t_a t_b times that sign and no numerator cancels.  Each lane reads only the
// entries it wrote (index j = lane mod L).  A numerator or denominator outside the fast
// reciprocal's range (extreme data) sends the group to the range-safe sum from d and zz.
template <int L, bool OFS = false>
__device__ __forceinline__ double stored_sum(const double* __restrict__ Ds, const double* __restrict__ us,
                                             const double* __restrict__ d, const double* __restrict__ zz, int n,
                                             int i, double di, double nu, int lane, unsigned gm, double dlo = 0.0) {
  double s0 = 0.0;
  bool b = false;
  int j = lane;
#pragma unroll kStoredUnroll
  for (; j + 3 * L < n; j += 4 * L) {
    const double t0 = __fma_rn(-nu, Ds[j], 1.0), t1 = __fma_rn(-nu, Ds[j + L], 1.0);
    const double t2 = __fma_rn(-nu, Ds[j + 2 * L], 1.0), t3 = __fma_rn(-nu, Ds[j + 3 * L], 1.0);
    const double u0 = us[j], u1 = us[j + L], u2 = us[j + 2 * L], u3 = us[j + 3 * L];
    const double n01 = __fma_rn(u0, t1, __dmul_rn(u1, t0)), p01 = __dmul_rn(t0, t1);
    const double n23 = __fma_rn(u2, t3, __dmul_rn(u3, t2)), p23 = __dmul_rn(t2, t3);
    const double num = __fma_rn(n01, p23, __dmul_rn(n23, p01)), den = __dmul_rn(p01, p23);
    b |= !rcp_in_range(den) || !rcp_in_range(num);
    s0 = __fma_rn(num, rcp_nr(den), s0);
  }
  if (j + L < n) {
    const double t0 = __fma_rn(-nu, Ds[j], 1.0), t1 = __fma_rn(-nu, Ds[j + L], 1.0);
    const double num = __fma_rn(us[j], t1, __dmul_rn(us[j + L], t0)), den = __dmul_rn(t0, t1);
    b |= !rcp_in_range(den) || !rcp_in_range(num);
    s0 = __fma_rn(num, rcp_nr(den), s0);
    j += 2 * L;
  }
  if (j < n) {
    const double t0 = __fma_rn(-nu, Ds[j], 1.0), u0 = us[j];
    b |= !rcp_in_range(t0) || (u0 != 0.0 && !rcp_in_range(u0));
    s0 = __fma_rn(u0, rcp_nr(t0), s0);
  }
  const double s = group_sum<L>(s0, gm);
  if (group_any<L>(b, gm)) {
    bool bad;
    return arrow_sum_pass<L, true, false, OFS>(d, zz, n, i, di, nu, lane, gm, &bad, nullptr, dlo);
  }
  return s;
}

// A bound on |S64 - S| at a bisection step a screen settles: S is the exact sum of
// T_j = u_j / t_j, t_j = 1 - nu Delta_j, over the stored elements, S64 the sum stored_sum
// returns, A >= sum_j |T_j|, m = ceil(n / L) terms per lane, u = 2^-53.
//  - t_j is one fma (the exact 1 - nu Delta_j rounded once): u |T_j| per term.
//  - A group of four terms is one quotient of products of like sign: each numerator of a pair
//    2 roundings, each pair product 1, the numerator of the four 2 more (5 in all), the
//    denominator 3, the reciprocal within one ulp (2u) and the product exact inside the fma:
//    10u of the group's value; a pair or a single term fewer.  With t_j's: 11u of sum |T_j|.
//  - The fma accumulation rounds at most m/4 + 2 times by u of a partial sum of like-sign
//    terms (at most A), and the lane group's tree tree_roundings<L> times.
// In all (m/4 + 13 + tree_roundings<L>) u A to first order; the bound adds u A for the rest.
// The range-safe fallback of stored_sum does not run at such a step: the screens settle a step
// only for stored elements in their ranges (|Delta| in [2^-80, 2^40), |u| in [2^-80, 2^60),
// |nu| <= 2^60) and with |nu Delta_j / t_j| <= 2^20, so every |t_j| lies in [2^-22, 2^101) and
// every numerator and denominator of stored_sum between 2^-160 and 2^410, inside the fast
// reciprocal's range.
template <int L>
__device__ __forceinline__ double stored_sum_error(double m, double A) {
  return (0.25 * m + 14.0 + (double)tree_roundings<L>()) * 0x1p-53 * A;
}

// Binary32 screen of a bisection step.  From the binary32 copies Df_j = fl32(Delta_j) and
// uf_j = fl32(u_j) and vf = fl32(nu) (each within eps = 2^-24 relative) each lane forms
// t = fl(1 - vf Df) (one fma), r = 1/t (approximate reciprocal and one Newton step: within
// 1.07 eps for any seed within 2^-14, 1.0001 eps for the hardware's), a = fl(uf r), and sums the
// a_j with Sum2 (TwoSum, Ogita-Rump-Oishi 2005).
// With p = vf Df exactly and the exact term T_j = u_j / (1 - nu Delta_j):
//   |t - (1 - nu Delta_j)| <= eps (1.0001 |t| + 2.0002 |p|),
// so the relative error of a_j is at most eps (4.07 + 2.0005 |p / t|) and, with w = |fl(fl(p) r)|
// (|p / t| <= w (1 + 3.01 eps)) and Sum2's own eps per term,
//   |a_j - T_j| + (Sum2's share) <= e_j = |a_j| (6 + 2.5 w) eps,
// valid while w <= 2^20 (then t and 1 - nu Delta_j have one sign and the relative error
// stays below 1/8; a lane with a larger w turns the screen off for the step).  The returned
// bound E = 1.05 (1 + 2 (m + 2) eps) sum_j e_j + 8 n 2^-126 (m terms per lane: the roundings of
// the bound's own sum; the last term for results below the binary32 normal range) holds for
// |S - sum_j T_j|, and A = 1.02 sum_j e_j / (6 eps) + E >= sum_j |T_j|.  The copies and nu
// must lie in the ranges checked by store_elem and here (|nu| in [2^-60, 2^60], so |p| <= 2^100).
// Returns false when the screen does not apply (a range, w, or a non-finite sum or bound).
// With SLOPE it also returns *dS ~ dS/dnu = sum_j (u_j / t_j)(Delta_j / t_j) (no bound: the
// probes of the bisection only place points with it).
template <int L, bool SLOPE = false>
__device__ __forceinline__ bool screen_sum(const float* __restrict__ Df, const float* __restrict__ uf, int n,
                                           double nu, int lane, unsigned gm, double* S, double* E, double* A,
                                           double* dS = nullptr) {
  const float vf = __double2float_rn(nu);
  const float av = fabsf(vf);
  float sh = 0.0f, sl = 0.0f, e = 0.0f, sd = 0.0f;
  bool bad = !(av >= 0x1p-60f && av <= 0x1p60f);
  for (int j = lane; j < n; j += L) {
    const float D = Df[j], u = uf[j];
    const float t = __fmaf_rn(-vf, D, 1.0f);
    const float r0 = rcp_approx_f32(t);
    const float r = __fmaf_rn(r0, __fmaf_rn(-t, r0, 1.0f), r0);
    const float a = __fmul_rn(u, r);
    const float w = fabsf(__fmul_rn(__fmul_rn(vf, D), r));
    if (SLOPE) sd = __fmaf_rn(a, __fmul_rn(D, r), sd);
    bad |= !(w <= 0x1p20f);
    const float sn = __fadd_rn(sh, a);
    const float bb = __fsub_rn(sn, sh);
    sl = __fadd_rn(sl, __fadd_rn(__fsub_rn(sh, __fsub_rn(sn, bb)), __fsub_rn(a, bb)));
    sh = sn;
    e = __fmaf_rn(fabsf(a), __fmaf_rn(2.5f, w, 6.0f), e);
  }
  // the lane group's sums in binary32: the pairs (sh, sl) by TwoSum (the low parts' roundings
  // stay far below eps A, inside the bound's 5% margin), the bound's sum raised by 2^-20 to cover
  // its own tree_roundings (at most 16)
  group_sum2_f<L>(&sh, &sl, gm);
  const double sum = __dadd_rn((double)sh, (double)sl);
  const double es = (double)group_sum_f<L>(e, gm) * (1.0 + 0x1p-20);
  if (SLOPE) *dS = (double)group_sum_f<L>(sd, gm);
  bad = group_any<L>(bad, gm);
  const double m = (double)((n + L - 1) / L);
  *S = sum;
  *E = 1.05 * (1.0 + 2.0 * (m + 2.0) * 0x1p-24) * 0x1p-24 * es + 8.0 * (double)n * 0x1p-126;
  *A = (1.02 / 6.0) * es + *E;
  return !bad && m * 0x1p-24 < 0.25 && isfinite(sum) && isfinite(es);
}

// x = hi + lo with hi = RN32(x) (the binary32 number nearest x, ties to even) and lo = x - hi
// rounded to 24 bits, so |x - hi - lo| <= 2^-48 |x| (plus at most 2^-149 where lo is a subnormal
// binary32 number, rounded a second time).  Formed with integer arithmetic on the bits of x: on GB300 a binary64 ->
// binary32 conversion runs on the binary64 pipe at the fma rate, integer operations on their own
// pipe at 32 times that.  Valid for x = 0 and 2^-126 <= |x| < 2^128; other x give 0 (callers
// only use copies of x in the screens' ranges).
__device__ __forceinline__ void split_f32x2(double x, float* hi, float* lo) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const unsigned sgn = (unsigned)(bits >> 63) << 31;
  const int e = (int)((bits >> 52) & 0x7ffu);
  if (e < 897 || e > 1150) {
    *hi = 0.0f;
    *lo = 0.0f;
    return;
  }
  const long long m = (long long)((bits & 0xfffffffffffffull) | 0x10000000000000ull);   // 53 bits
  long long q = m >> 29;                                                                  // 24 bits
  const long long rem = m & 0x1fffffff;
  if (rem > 0x10000000 || (rem == 0x10000000 && (q & 1))) q++;
  const int rlo = (int)(m - (q << 29));            // x - hi in units of 2^(e - 1075), |.| <= 2^28
  int ef = e - 896;                                // binary32 exponent field of hi
  if (q == 0x1000000) {
    q = 0x800000;
    ef++;
  }
  *hi = (ef <= 254) ? __uint_as_float(sgn | ((unsigned)ef << 23) | (unsigned)(q & 0x7fffff)) : 0.0f;
  // lo = rlo 2^k, k = e - 1075: the conversion rounds rlo to 24 bits; for k >= -126 the power of
  // two is a normal binary32 number and the product is exact (|rlo| in [1, 2^28]); below, the
  // scaling goes through 2^(k + 64) (exact) and 2^-64, which rounds once where the result is
  // subnormal
  const int k = e - 1075;
  const float lf = __int2float_rn(rlo);
  const float lv = (k >= -126) ? lf * __uint_as_float((unsigned)(k + 127) << 23)
                               : (lf * __uint_as_float((unsigned)(k + 64 + 127) << 23)) * 0x1p-64f;
  *lo = sgn ? -lv : lv;
}

// RN32(x) (the binary32 number nearest x, ties to even) by integer operations, for x = 0 and
// 2^-126 <= |x| < 2^128; *ok = false for other x (the result is then 0).
__device__ __forceinline__ float rn32(double x, bool* ok) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const unsigned sgn = (unsigned)(bits >> 63) << 31;
  const int e = (int)((bits >> 52) & 0x7ffu);
  if (e < 897 || e > 1150) {
    *ok = (bits << 1) == 0;
    return 0.0f;
  }
  const unsigned long long m = (bits & 0xfffffffffffffull) | 0x10000000000000ull;   // 53 bits
  unsigned q = (unsigned)(m >> 29);                                                   // 24 bits
  const unsigned rem = (unsigned)(m & 0x1fffffffu);
  if (rem > 0x10000000u || (rem == 0x10000000u && (q & 1u))) q++;
  int ef = e - 896;
  if (q == 0x1000000u) {
    q = 0x800000u;
    ef++;
  }
  *ok = ef <= 254;
  return *ok ? __uint_as_float(sgn | ((unsigned)ef << 23) | (q & 0x7fffffu)) : 0.0f;
}

// Shift test of Algorithm 1 in binary32: F = 1 + rho sum_j zz_j / ((d_j - d_k) - tau).  Each lane
// forms Delta_j = fl(d_j - d_k) in binary64 (one subtraction) and the rest in binary32 from
// Df = RN32(Delta_j), zf = RN32(zz_j), tf = RN32(tau) (integer conversions): den = fl(Df - tf),
// r = 1/den (approximate reciprocal and one Newton step, 1.07 eps), t = fl(zf r), summed by Sum2.
// With eps = 2^-24, |den - ((d_j - d_k) - tau)| <= eps (|Df| + tf) (1 + 2^-28) + eps |den| and
// w = (|Df| + tf) |r|, the term is within e_j = |t| eps (1.01 w + 4.2) of zz_j / ((d_j - d_k) - tau)
// (the conversions of zz and Delta, the reciprocal, the product and Sum2's share), valid while
// w <= 2^20 (else the lane reports failure); a weight below the binary32 range (zf = 0) adds at
// most 2^-125 |r|.  shift_sum_f32 returns the sum S32 with es = sum e_j and as = sum |t_j| (each
// rounded up); the tests below bound |F32 - F| for the exact F and |F64 - F| for the binary64 pass
// of the solve kernel (two roundings of each difference, the one-ulp reciprocal and the product:
// u (w + 4) per term, m = ceil(n / L) accumulations per lane, the tree and the last sum), so a
// decision on the sign of F32 with |F32| > E is the binary64 pass's decision.
template <int L>
__device__ __forceinline__ bool shift_sum_f32(const double* __restrict__ d, const double* __restrict__ zz, int n,
                                              double dk, double tau, int lane, unsigned gm, double* S, double* es_out,
                                              double* as_out) {
  bool ok = true;
  const float tf = rn32(tau, &ok);
  float sh = 0.0f, sl = 0.0f, e = 0.0f, a1 = 0.0f;
  for (int j = lane; j < n; j += L) {
    bool okd, okz;
    const float Df = rn32(__dsub_rn(d[j], dk), &okd);
    const float zf = rn32(zz[j], &okz);
    const float den = __fsub_rn(Df, tf);
    const float r0 = rcp_approx_f32(den);
    const float r = __fmaf_rn(r0, __fmaf_rn(-den, r0, 1.0f), r0);
    const float t = __fmul_rn(zf, r);
    const float ar = fabsf(r);
    const float w = __fmul_rn(__fadd_rn(fabsf(Df), tf), ar);
    ok &= okd && (w <= 0x1p20f);
    const float at = fabsf(t);
    e = __fmaf_rn(at, __fmaf_rn(1.01f, w, 4.2f), e);
    if (!okz) e = __fmaf_rn(ar, 0x1p-125f, e);
    a1 = __fadd_rn(a1, at);
    float er;
    sh = two_sum_f(sh, t, &er);
    sl = __fadd_rn(sl, er);
  }
  // the lane group's sums in binary32 as in screen_sum
  group_sum2_f<L>(&sh, &sl, gm);
  *S = __dadd_rn((double)sh, (double)sl);
  *es_out = (double)group_sum_f<L>(e, gm) * (1.0 + 0x1p-20);
  *as_out = (double)group_sum_f<L>(a1, gm) * (1.0 + 0x1p-20);
  return !group_any<L>(!ok, gm);
}

// D + rho z z^T: F = 1 + rho S.
template <int L>
__device__ __noinline__ bool shift_test_f32(const double* __restrict__ d, const double* __restrict__ zz, int n,
                                            double dk, double tau, double rho, int lane, unsigned gm, double* F,
                                            double* E) {
  double S, es, as;
  const bool ok = shift_sum_f32<L>(d, zz, n, dk, tau, lane, gm, &S, &es, &as);
  const double m = (double)((n + L - 1) / L);
  const double g = 1.0 + 2.0 * (m + 2.0) * 0x1p-24;
  const double F32 = 1.0 + rho * S;
  const double E32 = rho * (1.05 * g * 0x1p-24 * es + (2.0 + tree_roundings<L>()) * 0x1p-53 * g * as +
                            4.0 * (double)n * 0x1p-149);
  const double E64 = 1.01 * 0x1p-53 * rho * g * (es + (m + 16.0 + tree_roundings<L>()) * as);
  *F = F32;
  *E = 1.01 * (E32 + E64 + 0x1p-50 * (1.0 + rho * g * as));
  return ok && isfinite(F32) && isfinite(*E);
}

// The arrowhead [D z; z^T alpha]: F = c - S with c = fl(fl(alpha - d_k) - tau), the value the
// binary64 pass subtracts its sum fl(sp + sn) from; fl(c - x) has the sign of c - x, so the
// binary64 decision is the sign of c - fl(sp + sn), within the same bound of c - S32.
template <int L>
__device__ __noinline__ bool shift_test_arrow_f32(const double* __restrict__ d, const double* __restrict__ zz, int n,
                                                  double dk, double tau, double c, int lane, unsigned gm, double* F,
                                                  double* E) {
  double S, es, as;
  const bool ok = shift_sum_f32<L>(d, zz, n, dk, tau, lane, gm, &S, &es, &as);
  const double m = (double)((n + L - 1) / L);
  const double g = 1.0 + 2.0 * (m + 2.0) * 0x1p-24;
  const double F32 = __dsub_rn(c, S);
  const double E32 = 1.05 * g * 0x1p-24 * es + (2.0 + tree_roundings<L>()) * 0x1p-53 * g * as +
                     4.0 * (double)n * 0x1p-149;
  const double E64 = 1.01 * 0x1p-53 * g * (es + (m + 16.0 + tree_roundings<L>()) * as);
  *F = F32;
  *E = 1.01 * (E32 + E64 + 0x1p-50 * (fabs(c) + g * as));
  return ok && isfinite(F32) && isfinite(*E);
}

// Stores the elements of the inverse at j: Delta_j and u_j = zz_j / Delta_j and, with F, their
// binary32 copies and the low parts (F[j] = RN32(Delta_j), F[n + j] = RN32(u_j), F[2n + j] and
// F[3n + j] the remainders: split_f32x2).  Returns false when a copy is not a normal binary32
// number in the screens' range (|Delta| in [2^-80, 2^40), |u| in [2^-80, 2^60), or zero), which
// turns the screens off.
__device__ __forceinline__ bool store_elem(double* __restrict__ Ds, double* __restrict__ us, float* __restrict__ F,
                                           int n, int j, double D, double u) {
  Ds[j] = D;
  us[j] = u;
  if (!F) return true;
  split_f32x2(D, F + j, F + 2 * n + j);
  split_f32x2(u, F + n + j, F + 3 * n + j);
  const unsigned eD = (unsigned)(__double_as_longlong(D) >> 52) & 0x7ffu;
  const unsigned eu = (unsigned)(__double_as_longlong(u) >> 52) & 0x7ffu;
  return (D == 0.0 || (eD >= 943u && eD <= 1062u)) && (u == 0.0 || (eu >= 943u && eu <= 1082u));
}

// Double-float screen of a bisection step, for the steps the binary32 screen cannot settle.
// The stored elements as pairs of binary32 numbers, Delta = Dh + Dl and u = uh + ul to 2^-48
// (store_elem), and nu = vh + vl likewise; eps = 2^-24, w = |nu Delta / t|.  Each term
// T_j = u_j / (1 - nu Delta_j) is formed as q1 + q2:
//   p = nu Delta: ph + pe = vh Dh exactly (fma), pl = vh Dl + vl Dh + pe (two fma);
//     |ph + pl - nu Delta| <= 8.01 eps^2 |nu Delta| (the splits of nu and Delta 2 eps^2, the
//     rounded cross terms 5 eps^2, the dropped vl Dl eps^2);
//   t = 1 - p: s + er = 1 - ph (TwoSum), (th, tl) = TwoSum(s, fl(er - pl));
//     |th + tl - t| <= eps^2 |t| (1 + 11.2 w);
//   a = u / t: r the binary32 reciprocal of th refined by one Newton step (within 1.07 eps),
//     q1 = fl(uh r), q2 = fl(R r) with R = fl(fl(fl(uh - q1 th) + ul) - q1 tl) (fma; the exact
//     residual u - q1 t is at most 4.1 eps |u|, its roundings 9.3 eps^2 |u|, the reciprocal's
//     error on it 12.6 eps^2 |u / t|);
//   so |q1 + q2 - T_j| <= eps^2 |T_j| (24 + 11.2 w) (1.001), bounded by eps^2 |q1| (32 + 16 w)
//   (|T_j| <= |q1| (1 + 2.2 eps), and the computed w is within 3.1 eps of |nu Delta / t|).
// Per lane the terms are summed in three binary32 levels (sh, sl, sll): q1 joins sh by TwoSum,
// its error er and q2 are added exactly (TwoSum: a + ae = er + q2) and a joins sl by TwoSum;
// only c = fl(ae + se) (se the last TwoSum's error) and sll = fl(sll + c) round, each by at
// most eps times |c| and |sll|, whose sum bl bounds them at run time (a running error bound).
// With two levels instead (fl(er + q2) added to sl), the roundings of sl grow like
// m^(3/2) eps^2 sum |q1| and, near the root, exceed the terms' own error.  The lane sum goes to
// binary64 with two roundings and is added in the lane group's tree (tree_roundings more), each
// at most 2^-53 of sum |q1|.  Accumulators of positive terms in binary32 (bl,
// sum |q1| (32 + 16 w), sum |q1|) are at most (m + 2) eps below their exact values (m terms per
// lane), hence the factor g = 1 + 2 (m + 2) eps.  Subnormal binary32 intermediates add at most
// 2^-150 per operation (48 n 2^-149 in all) and, where nu Delta lies below the binary32 normal
// range, relative errors below 2^-140.  The returned
//   E = 1.05 g (eps^2 sum e_j + eps sum bl) + g ((2 + tree_roundings) 2^-53 + 2^-140) sum |q1|
//       + 48 n 2^-149
// bounds |S - sum_j T_j|, and A = 1.001 g sum |q1| + E >= sum_j |T_j|.  Ranges as screen_sum
// (w <= 2^20: |t| >= 2^-21, every |q1| below 2^82).  Returns false when the screen does not
// apply (a range, w, or a non-finite sum or bound).
// With SLOPE it also returns *dS as screen_sum does (from the high parts).
template <int L, bool SLOPE = false>
__device__ __forceinline__ bool screen_df_sum(const float* __restrict__ F, int n, double nu, int lane, unsigned gm,
                                              double* S, double* E, double* A, double* dS = nullptr) {
  const float* __restrict__ Dh = F;
  const float* __restrict__ uh = F + n;
  const float* __restrict__ Dl = F + 2 * n;
  const float* __restrict__ ul = F + 3 * n;
  float vh, vl;
  split_f32x2(nu, &vh, &vl);
  const float av = fabsf(vh);
  bool bad = !(av >= 0x1p-60f && av <= 0x1p60f);
  float sh = 0.0f, sl = 0.0f, sll = 0.0f, bl = 0.0f, e = 0.0f, a1 = 0.0f, sd = 0.0f;
  for (int j = lane; j < n; j += L) {
    const float dh = Dh[j], dl = Dl[j], uhj = uh[j], ulj = ul[j];
    const float ph = __fmul_rn(vh, dh);
    const float pe = __fmaf_rn(vh, dh, -ph);
    const float pl = __fmaf_rn(vh, dl, __fmaf_rn(vl, dh, pe));
    const float s = __fsub_rn(1.0f, ph);
    const float b0 = __fsub_rn(s, 1.0f);
    const float er = __fadd_rn(__fsub_rn(1.0f, __fsub_rn(s, b0)), __fsub_rn(-ph, b0));
    const float tl0 = __fsub_rn(er, pl);
    const float th = __fadd_rn(s, tl0);
    const float b1 = __fsub_rn(th, s);
    const float tl = __fadd_rn(__fsub_rn(s, __fsub_rn(th, b1)), __fsub_rn(tl0, b1));
    const float r0 = rcp_approx_f32(th);
    const float r = __fmaf_rn(r0, __fmaf_rn(-th, r0, 1.0f), r0);
    const float q1 = __fmul_rn(uhj, r);
    if (SLOPE) sd = __fmaf_rn(q1, __fmul_rn(dh, r), sd);
    const float e1 = __fmaf_rn(-q1, th, uhj);
    const float R = __fmaf_rn(-q1, tl, __fadd_rn(e1, ulj));
    const float q2 = __fmul_rn(R, r);
    const float w = fabsf(__fmul_rn(ph, r));
    bad |= !(w <= 0x1p20f);
    float er2, a, ae, se;
    sh = two_sum_f(sh, q1, &er2);
    a = two_sum_f(er2, q2, &ae);
    sl = two_sum_f(sl, a, &se);
    const float c = __fadd_rn(ae, se);
    sll = __fadd_rn(sll, c);
    bl = __fadd_rn(bl, __fadd_rn(fabsf(c), fabsf(sll)));
    const float aq = fabsf(q1);
    a1 = __fadd_rn(a1, aq);
    e = __fmaf_rn(aq, __fmaf_rn(16.0f, w, 32.0f), e);
  }
  const double sum = group_sum<L>(__dadd_rn(__dadd_rn((double)sh, (double)sl), (double)sll), gm);
  // the bound's sums of positive terms in binary32, raised by 2^-20 to cover their own
  // tree_roundings (at most 16)
  const double es = (double)group_sum_f<L>(e, gm) * (1.0 + 0x1p-20);
  const double bs = (double)group_sum_f<L>(bl, gm) * (1.0 + 0x1p-20);
  const double as = (double)group_sum_f<L>(a1, gm) * (1.0 + 0x1p-20);
  if (SLOPE) *dS = (double)group_sum_f<L>(sd, gm);
  bad = group_any<L>(bad, gm);
  const double m = (double)((n + L - 1) / L);
  const double g = 1.0 + 2.0 * (m + 2.0) * 0x1p-24;
  *S = sum;
  *E = 1.05 * g * (0x1p-48 * es + 0x1p-24 * bs) + g * ((2.0 + tree_roundings<L>()) * 0x1p-53 + 0x1p-140) * as +
       48.0 * (double)n * 0x1p-149;
  *A = 1.001 * g * as + *E;
  return !bad && m * 0x1p-24 < 0.25 && isfinite(sum) && isfinite(es) && isfinite(bs) && isfinite(as);
}

// The loops over the stored elements as calls of their own (NI) or inlined.  Out of line, the
// caller's state is saved once per evaluation instead of crowding the loop's registers: the
// better form for the solve kernel of large problems, compiled for four blocks per SM (64
// registers), where the loops are long; inlined for problems of small order, where the loops are
// short and the call's cost counts.
template <int L, bool OFS>
__device__ __noinline__ double stored_sum_call(const double* __restrict__ Ds, const double* __restrict__ us,
                                               const double* __restrict__ d, const double* __restrict__ zz, int n,
                                               int i, double di, double nu, int lane, unsigned gm, double dlo) {
  return stored_sum<L, OFS>(Ds, us, d, zz, n, i, di, nu, lane, gm, dlo);
}
template <int L, bool SLOPE>
__device__ __noinline__ bool screen_sum_call(const float* __restrict__ Df, const float* __restrict__ uf, int n,
                                             double nu, int lane, unsigned gm, double* S, double* E, double* A,
                                             double* dS) {
  return screen_sum<L, SLOPE>(Df, uf, n, nu, lane, gm, S, E, A, dS);
}
template <int L, bool SLOPE>
__device__ __noinline__ bool screen_df_sum_call(const float* __restrict__ F, int n, double nu, int lane,
                                                unsigned gm, double* S, double* E, double* A, double* dS) {
  return screen_df_sum<L, SLOPE>(F, n, nu, lane, gm, S, E, A, dS);
}
template <bool NI, int L, bool SLOPE = false>
__device__ __forceinline__ bool screen_sum_x(const float* __restrict__ Df, const float* __restrict__ uf, int n,
                                             double nu, int lane, unsigned gm, double* S, double* E, double* A,
                                             double* dS = nullptr) {
  if constexpr (NI) return screen_sum_call<L, SLOPE>(Df, uf, n, nu, lane, gm, S, E, A, dS);
  else return screen_sum<L, SLOPE>(Df, uf, n, nu, lane, gm, S, E, A, dS);
}
template <bool NI, int L, bool SLOPE = false>
__device__ __forceinline__ bool screen_df_sum_x(const float* __restrict__ F, int n, double nu, int lane, unsigned gm,
                                                double* S, double* E, double* A, double* dS = nullptr) {
  if constexpr (NI) return screen_df_sum_call<L, SLOPE>(F, n, nu, lane, gm, S, E, A, dS);
  else return screen_df_sum<L, SLOPE>(F, n, nu, lane, gm, S, E, A, dS);
}

// The sum and its derivative dS/dnu = sum_j zz_j / t_j^2 = sum_j (u_j / t_j)(Delta_j / t_j) from
// the stored elements (the accelerated solve): one reciprocal of t_j per term, 8 binary64
// instructions against 10 when Delta_j and Delta_j t_j are formed at every evaluation.
template <int L, bool OFS = false>
__device__ __forceinline__ double stored_sum_d(const double* __restrict__ Ds, const double* __restrict__ us,
                                               const double* __restrict__ d, const double* __restrict__ zz, int n,
                                               int i, double di, double nu, int lane, unsigned gm, double* dsum,
                                               double dlo = 0.0) {
  double s0 = 0.0, s1 = 0.0, q0 = 0.0, q1 = 0.0;
  bool b = false;
  int j = lane;
  for (; j + L < n; j += 2 * L) {
    const double D0 = Ds[j], D1 = Ds[j + L];
    const double t0 = __fma_rn(-nu, D0, 1.0), t1 = __fma_rn(-nu, D1, 1.0);
    b |= !rcp_in_range(t0) || !rcp_in_range(t1);
    const double r0 = rcp_nr(t0), r1 = rcp_nr(t1);
    const double a0 = __dmul_rn(us[j], r0), a1 = __dmul_rn(us[j + L], r1);
    s0 = __dadd_rn(s0, a0);
    s1 = __dadd_rn(s1, a1);
    q0 = __fma_rn(a0, __dmul_rn(D0, r0), q0);
    q1 = __fma_rn(a1, __dmul_rn(D1, r1), q1);
  }
  if (j < n) {
    const double D0 = Ds[j];
    const double t0 = __fma_rn(-nu, D0, 1.0);
    b |= !rcp_in_range(t0);
    const double r0 = rcp_nr(t0);
    const double a0 = __dmul_rn(us[j], r0);
    s0 = __dadd_rn(s0, a0);
    q0 = __fma_rn(a0, __dmul_rn(D0, r0), q0);
  }
  const double s = group_sum<L>(__dadd_rn(s0, s1), gm);
  *dsum = group_sum<L>(__dadd_rn(q0, q1), gm);
  if (group_any<L>(b, gm)) {
    bool bad;
    return arrow_sum_pass<L, true, true, OFS>(d, zz, n, i, di, nu, lane, gm, &bad, dsum, dlo);
  }
  return s;
}

// The secular sums from the stored elements when the group has them (Ds != nullptr), else
// formed from d and zz at every evaluation.
template <int L, bool OFS = false, bool NI = false>
__device__ __forceinline__ double elem_sum(const double* __restrict__ Ds, const double* __restrict__ us,
                                           const double* __restrict__ d, const double* __restrict__ zz, int n, int i,
                                           double di, double nu, int lane, unsigned gm, double dlo = 0.0) {
  if (!Ds) return arrow_sum<L, OFS>(d, zz, n, i, di, nu, lane, gm, dlo);
  if constexpr (NI) return stored_sum_call<L, OFS>(Ds, us, d, zz, n, i, di, nu, lane, gm, dlo);
  else return stored_sum<L, OFS>(Ds, us, d, zz, n, i, di, nu, lane, gm, dlo);
}

template <int L, bool OFS = false>
__device__ __forceinline__ double elem_sum_d(const double* __restrict__ Ds, const double* __restrict__ us,
                                             const double* __restrict__ d, const double* __restrict__ zz, int n,
                                             int i, double di, double nu, int lane, unsigned gm, double* dsum,
                                             double dlo = 0.0) {
  return Ds ? stored_sum_d<L, OFS>(Ds, us, d, zz, n, i, di, nu, lane, gm, dsum, dlo)
            : arrow_sum_d<L, OFS>(d, zz, n, i, di, nu, lane, gm, dsum, dlo);
}

// Same terms with Delta_j = d_j - sigma for a non-pole shift (no excluded index):
// sum_j u_j^2 / (e_j - nu), e_j = 1/(d_j - sigma), u_j = zeta_j/(d_j - sigma).
template <int L>
__device__ __forceinline__ double shift_sum(const double* __restrict__ d, const double* __restrict__ zz, int n,
                                            double sigma, double nu, int lane, unsigned gm) {
  return arrow_sum<L>(d, zz, n, -1, sigma, nu, lane, gm);
}

// sum_{j != skip} zeta_j^2 / (d_j - s) in double-double (skip = -1: all j); also returns
// sum_{j != skip} zeta_j^2 / (d_j - s)^2 in binary64 (the squared norm of the border).
// Each term is formed from the exact difference D = Dh + Dl (FastTwoSum with the operands
// ordered by magnitude) and the exact square zeta_j^2 = zz_j + zl_j (stored once per problem)
// as q + e_q, q = zz_j / Dh rounded, with the first-order correction
// e_q = ((zz_j - q Dh) + (zl_j - q Dl)) / Dh.  The q are summed by compensated summation
// (Sum2 of Ogita, Rump and Oishi, SIAM J. Sci. Comput. 26 (2005)): two_sum keeps each
// rounding error, and the errors and the e_q go to a second binary64 accumulator, which
// gives the sum as accurately as accumulation in twice the working precision (Sec. 2.3).
// With Ds != nullptr it also stores Dh = fl(d_j - s) and q = zz_j / Dh (0 and 0 at skip): the
// elements of the inverse that stored_sum reads; with F their binary32 copies and low parts
// (store_elem), and *scr_ok tells whether the screens apply to them.
// With OFS the shift is s + slo in double the working precision: the difference is formed by
// shift_diff and the stored element is its binary64 rounding (elem_diff).
template <int L, bool OFS = false>
__device__ __forceinline__ dd dd_pole_sum(const double* __restrict__ d, const double* __restrict__ zz,
                                          const double* __restrict__ zl, int n, int skip, double s, int lane,
                                          unsigned gm, double* sq, double* cub = nullptr,
                                          double* __restrict__ Ds = nullptr, double* __restrict__ us = nullptr,
                                          float* __restrict__ F = nullptr, bool* scr_ok = nullptr,
                                          double slo = 0.0) {
  double hi = 0.0, lo = 0.0, q2 = 0.0, c3 = 0.0;
  const double ms = -s;
  bool ok = F != nullptr;
  for (int j = lane; j < n; j += L) {
    if (j == skip) {
      if (Ds) ok &= store_elem(Ds, us, F, n, j, 0.0, 0.0);
      continue;
    }
    const double dj = d[j];
    double Dh, Dl;
    if constexpr (OFS) {
      const dd D = shift_diff(dj, s, slo);
      Dh = D.hi;
      Dl = D.lo;
    } else {
      const bool ge = fabs(dj) >= fabs(ms);
      const double big = ge ? dj : ms, small = ge ? ms : dj;
      Dh = __dadd_rn(big, small);
      Dl = __dsub_rn(small, __dsub_rn(Dh, big));
    }
    const double Zh = zz[j], Zl = zl[j];
    const double r = rcp(Dh);
    const double q = __dmul_rn(Zh, r);
    if (Ds) ok &= store_elem(Ds, us, F, n, j, Dh, q);
    const double eq = __dmul_rn(__dadd_rn(__fma_rn(-q, Dh, Zh), __fma_rn(-q, Dl, Zl)), r);
    const dd t = two_sum(hi, q);
    hi = t.hi;
    lo = __dadd_rn(lo, __dadd_rn(t.lo, eq));
    const double c2 = __dmul_rn(q, r);
    q2 = __dadd_rn(q2, c2);
    if (cub) c3 = __fma_rn(c2, r, c3);
  }
  *sq = group_sum<L>(q2, gm);
  if (cub) *cub = group_sum<L>(c3, gm);
  if (scr_ok) *scr_ok = !group_any<L>(!ok, gm);
  return group_sum_dd<L>(two_sum(hi, lo), gm);
}

// ---------------------------------------------------------------------------------
// Bit-pattern bisection of a secular function on |nu| for nu = side*|nu|.
// phi(nu) has sign `below` for |nu| between `floor` and the root and the opposite sign
// beyond it.  `floor` is a pole of phi (or 0) that is known to lie below the root and
// is never evaluated; [alo, ahi] is an estimate of the bracket.  Ends from a soft estimate
// (eager_lo / eager_hi) are checked first; any other end that the bisection never moves is
// checked when the bisection has closed on it.  A far end still below the root is pushed
// out geometrically, a near end above the root falls back to the floor, and the bisection
// continues (each bisection phase has the iteration cap).  Every lane of the group runs the same loop (the
// sums are identical in every lane).  Returns nu with the smaller |phi| of the final
// adjacent pair; *ok = false if the cap was reached.
// ---------------------------------------------------------------------------------
// Root of the pole model of F = fscale (a0 - a1 t + Psi) fitted to Psi(t) and Psi'(t) (see the
// accelerated solve below); Newton's step where the model has no usable pole.
__device__ __forceinline__ double model_root(double t, double F, double psi, double dpsi, double E, double a0,
                                             double a1, double fscale) {
  const double x0 = __dsub_rn(t, E);
  if (x0 > 0.0 && x0 <= 1.0e300 && dpsi < 0.0) {
    const double s = -dpsi * x0 * x0;
    const double c = __fma_rn(dpsi, x0, psi);
    const double A = (a0 + c) - a1 * E;
    double x;
    if (a1 > 0.0) {
      const double disc = (A != 0.0) ? fabs(A) * sqrt(1.0 + (4.0 * a1 * s / A) / A) : sqrt(4.0 * a1 * s);
      x = (A > 0.0) ? (A + disc) / (2.0 * a1) : (2.0 * s) / (disc - A);
    } else {
      x = (A < 0.0) ? -s / A : INFINITY;
    }
    return E + x;
  }
  // no usable pole: Newton's step on F = fscale (a0 - a1 t + Psi)
  const double dF = fscale * (dpsi - a1);
  return (dF < 0.0) ? t - F / dF : NAN;
}

// No screen: every step evaluates phi.
struct NoScreen {
  __device__ bool operator()(double, double*, double*, int, double* = nullptr, double* = nullptr) const {
    return false;
  }
};

// screen(nu, &g, &tol, mode, psi, dpsi) may settle a step without phi: it returns true with g of
// the sign phi(nu) would have and |g| > tol (the bisection then takes the same decision); mode -1
// lets the screen choose its precision, 0 asks for binary32 only and 1 for the double-float
// screen only; with psi != nullptr it also returns Psi and Psi' (below) from the screened sums.
// Once it fails kScreenTries times in a row, the remaining steps (closer to the root) use phi
// only; an end whose value came from the screen is evaluated by phi before the final choice, so
// the result is the one of phi alone.  *screened counts the steps the screen settled.
//
// Certified bounds.  On t = |nu| the exact secular function of the stored elements has the form
// F(t) = a0 - t + Psi(t), Psi(t) = sum_j c_j / (t - e_j) > 0 with c_j > 0 and every pole e_j
// below the bracket, so F is strictly decreasing there, and the error of phi is at most
// alpha Psi(t) + beta |a0 - t| + gamma |F(t)| with alpha, beta, gamma far below 1 (the stored sum's
// bound, the roundings of b - nu, of the products and of the last difference).  Where F > 0,
// lowering t raises F by at least the change of t plus that of Psi, and the bound by at most
// beta times the first and alpha times the second, so F minus the bound only grows; where F < 0
// the same holds for raising t.  A point where a screen settled the step has |F| above the bound
// (its tolerance covers the screen's error, the bound and the roundings); hence every t below a
// point settled "below" (above a point settled "above") gets phi's decision "below" ("above")
// without an evaluation.  With `predict`, screened probes set such bounds cl and ch next to the
// root: from the upper end, the accelerated solve's pole model (model_root: pole `pole`, F =
// a0 - t + Psi) fitted to each probe's screened value and slope gives the next probe, first with
// the binary32 screen, then, once its steps shrink below twice its tolerance over the slope (or
// it cannot settle a probe), with the double-float screen; one double-float step later two probes
// at that estimate minus and plus twice the tolerance over the slope certify both sides.  The
// bisection then follows its own path from its own bracket and takes every midpoint outside
// (cl, ch) from them (*inferred counts those steps, *probes the screened probes).  The steps, the
// decisions and the result are those of the bisection without the probes.
template <class Phi, class Scr = NoScreen>
__device__ double bisect(Phi phi, double side, double floor, double alo, double ahi, bool below_positive, int cap,
                         bool* ok, int* steps_out, bool eager_lo = false, bool eager_hi = false, Scr screen = Scr(),
                         int* screened = nullptr, bool predict = false, double pole = 0.0, double a0 = 0.0,
                         int* inferred = nullptr, int* probes = nullptr) {
  int steps = 0;
  bool good = true;
  if (!(floor >= 0.0)) floor = 0.0;
  if (!(alo >= floor)) alo = floor;
  if (!(ahi > alo)) ahi = (alo > 0.0) ? alo * 2.0 : 1.0;
  const uint64_t fl = dbits(floor);
  const uint64_t top = 0x7fefffffffffffffull;
  uint64_t lo = dbits(alo), hi = dbits(ahi);
  uint64_t span = hi - lo + 64;
  double glo = 0.0, ghi = 0.0;
  bool have_lo = false, have_hi = false;    // the end point was evaluated (its side is known)
  bool scr_lo = false, scr_hi = false;      // its value came from the screen (or a certified bound)
  double llo = 0.0, lhi = 0.0;              // then a lower bound on |phi| there
  bool scr_on = true;
  int scr_fail = 0;                         // consecutive steps the screen did not settle
  int it = 0, pushes = 0, nscr = 0, ninf = 0, nprobe = 0;
  // certified bounds: phi decides "below" at every t <= dfrom(cl), "above" at every t >= dfrom(ch),
  // and |phi| is at least Lcl (Lch) there
  uint64_t cl = 0, ch = ~0ull;
  double Lcl = 0.0, Lch = 0.0;
  // a lower bound on |phi| from a screened value g and its tolerance: |phi - g| <= tol plus
  // roundings of g's size
  auto lower = [](double g, double tol) { return fmax(fabs(g) * (1.0 - 0x1p-50) - 2.0 * tol, 0.0); };
  // an end check: a certified bound, the screen when it settles the point, else phi (*sc: the
  // value is not phi's)
  auto check = [&](uint64_t x, bool* sc, double* lb) -> double {
    double g, tol;
    if (x <= cl || x >= ch) {
      *sc = true;
      *lb = (x <= cl) ? Lcl : Lch;
      steps++;
      ninf++;
      return ((x <= cl) == below_positive) ? 1.0 : -1.0;
    }
    *sc = kScreenEnds && screen(side * dfrom(x), &g, &tol, -1, nullptr, nullptr);
    if (*sc) {
      nscr++;
      *lb = lower(g, tol);
    } else {
      g = phi(side * dfrom(x));
    }
    steps++;
    return g;
  };
  // ends that come from a soft estimate (eager_*) are checked before the bisection
  if (eager_hi) {
    for (; pushes < 64; pushes++) {
      bool sc;
      double lb;
      double g = check(hi, &sc, &lb);
      bool below = below_positive ? (g > 0.0) : (g < 0.0);
      if (!below) { ghi = g; have_hi = true; scr_hi = sc; lhi = lb; break; }
      lo = hi; glo = g; have_lo = true; scr_lo = sc; llo = lb;
      if (hi >= top) break;
      hi = (top - hi > span) ? hi + span : top;
      span *= 2;
    }
  }
  if (eager_lo && !have_lo && lo > fl) {
    bool sc;
    double lb;
    double g = check(lo, &sc, &lb);
    bool below = below_positive ? (g > 0.0) : (g < 0.0);
    if (below) { glo = g; have_lo = true; scr_lo = sc; llo = lb; }
    else { hi = lo; ghi = g; have_hi = true; scr_hi = sc; lhi = lb; lo = fl; }
  }
  if (predict) {
    int level = 0;           // 0: binary32 probes, 1: double-float probes
    int phase = 0;           // 0: model steps, 1: certify below the estimate, 2: certify above it
    double est = 0.0, delta = 0.0;
    uint64_t x = hi;
    for (int p = 0; p < kPredictSteps; p++) {
      const uint64_t bl = cl > lo ? cl : lo, bh = ch < hi ? ch : hi;
      if (bh <= bl || bh - bl <= kPredictStop) break;
      if (x <= bl || x >= bh) {
        if (phase == 0 && x == bh && x == hi && !have_hi) {
          // the first probe: the upper end itself
        } else if (phase == 1) {
          phase = 2;                          // the lower side is certified already
          x = dbits(est + delta);
          continue;
        } else if (phase == 2) {
          break;
        } else {
          x = bl + ((bh - bl) >> 1);
        }
      }
      const double t = dfrom(x);
      double g, tol, psi = 0.0, dpsi = 0.0;
      nprobe++;
      const bool sc = screen(side * t, &g, &tol, level, phase == 0 ? &psi : nullptr, &dpsi);
      if (!sc) {
        if (phase == 0 && level == 0 && kScreenDf) {
          level = 1;                          // within the binary32 screen's reach of the root
          continue;
        }
        break;
      }
      const bool below = below_positive ? (g > 0.0) : (g < 0.0);
      if (below) {
        cl = x;
        Lcl = lower(g, tol);
      } else {
        ch = x;
        Lch = lower(g, tol);
      }
      if (phase == 1) {
        phase = 2;
        x = dbits(est + delta);
        continue;
      }
      if (phase == 2) break;
      const double F = below_positive ? g : -g;
      const double slope = dpsi - 1.0;
      if (!(slope < 0.0)) break;
      double tc = model_root(t, F, psi, dpsi, pole, a0, 1.0, 1.0);
      const double tl = dfrom(bl), th = dfrom(bh);
      if (!(tc > tl && tc < th)) tc = below ? fmin(t + fabs(F / slope), th) : fmax(t - fabs(F / slope), tl);
      const double dl = 2.0 * tol / -slope;
      if (level == 0 && kScreenDf && fabs(tc - t) <= dl) {
        level = 1;                            // converged at the binary32 screen's resolution
        x = dbits(tc);
        continue;
      }
      if (level == 1) {
        // one double-float model step from within the binary32 screen's reach: certify
        est = tc;
        delta = dl;
        phase = 1;
        x = dbits(est - delta);
        continue;
      }
      x = dbits(tc);
    }
  }
  for (;;) {
    // bisection on the bit patterns; every evaluation moves one end and makes it known
    int phase = 0;
    while (hi - lo > 1) {
      if (phase >= cap) { good = false; break; }
      phase++;
      uint64_t mid = lo + ((hi - lo) >> 1);
      double g, tol, lb = 0.0;
      bool sc = false;
      if (mid <= cl || mid >= ch) {
        // a certified bound decides the step
        sc = true;
        ninf++;
        g = ((mid <= cl) == below_positive) ? 1.0 : -1.0;
        lb = (mid <= cl) ? Lcl : Lch;
      } else {
        if (scr_on) {
          sc = screen(side * dfrom(mid), &g, &tol, -1, nullptr, nullptr);
          scr_fail = sc ? 0 : scr_fail + 1;
          scr_on = scr_fail < kScreenTries;
        }
        if (!sc) g = phi(side * dfrom(mid));
        else {
          nscr++;
          lb = lower(g, tol);
        }
      }
      bool below = below_positive ? (g > 0.0) : (g < 0.0);
      if (below) { lo = mid; glo = g; have_lo = true; scr_lo = sc; llo = lb; }
      else { hi = mid; ghi = g; have_hi = true; scr_hi = sc; lhi = lb; }
      it++;
    }
    if (!good) break;
    // an end the bisection never moved is only an estimate: check it now (usually the root
    // lies strictly inside and both ends have moved, so this costs nothing)
    if (!have_hi) {
      bool sc;
      double lb;
      double g = check(hi, &sc, &lb);
      bool below = below_positive ? (g > 0.0) : (g < 0.0);
      if (below && pushes < 64 && hi < top) {
        // the root lies beyond the estimate: push the far end out geometrically
        lo = hi; glo = g; have_lo = true; scr_lo = sc; llo = lb;
        hi = (top - hi > span) ? hi + span : top;
        span *= 2;
        pushes++;
        continue;
      }
      ghi = g; have_hi = !below; scr_hi = sc; lhi = lb;
      if (below) { good = false; break; }
    }
    if (!have_lo && lo > fl) {
      bool sc;
      double lb;
      double g = check(lo, &sc, &lb);
      bool below = below_positive ? (g > 0.0) : (g < 0.0);
      if (!below) {
        // the root lies below the near estimate: fall back to the floor
        hi = lo; ghi = g; have_hi = true; scr_hi = sc; lhi = lb; lo = fl;
        continue;
      }
      glo = g; have_lo = true; scr_lo = sc; llo = lb;
    }
    break;
  }
  // the final choice compares the values of phi at the two ends.  An end known only from a
  // screen or a certified bound is evaluated unless its lower bound on |phi| already exceeds the
  // other end's |phi| (then the other end is the choice, as it would be after the evaluation);
  // of two such ends the one with the smaller bound is evaluated first.
  if (have_lo && scr_lo && have_hi && scr_hi) {
    if (llo <= lhi) { glo = phi(side * dfrom(lo)); steps++; scr_lo = false; }
    else { ghi = phi(side * dfrom(hi)); steps++; scr_hi = false; }
  }
  if (have_lo && scr_lo) {
    if (have_hi && !scr_hi && llo > fabs(ghi)) glo = INFINITY;
    else { glo = phi(side * dfrom(lo)); steps++; }
  }
  if (have_hi && scr_hi) {
    if (have_lo && !scr_lo && lhi > fabs(glo)) ghi = INFINITY;
    else { ghi = phi(side * dfrom(hi)); steps++; }
  }
  steps += it;
  if (screened) *screened = nscr;
  if (inferred) *inferred = ninf;
  if (probes) *probes = nprobe;
  double alo_g = have_lo ? fabs(glo) : INFINITY;
  double ahi_g = have_hi ? fabs(ghi) : INFINITY;
  if (isnan(alo_g)) alo_g = INFINITY;
  if (isnan(ahi_g)) ahi_g = INFINITY;
  *ok = good;
  if (steps_out) *steps_out = steps;
  return side * dfrom((ahi_g < alo_g) ? hi : lo);
}

// ---------------------------------------------------------------------------------
// Accelerated bracketed solve (a fast zero finder in place of bisection, Sec. 2.2).
//
// On t = |nu| the secular functions of both solvers have the form
//   F(t) = a0 - a1 t + Psi(t),   Psi(t) = sum_j w_j^2 / (t - e_j),   every pole e_j < root,
// (a1 = 1 for the arrowhead function g, a1 = 0 for the non-pole function h after scaling),
// with F > 0 below the root.  Psi is positive, decreasing and convex above its poles.
// Model: Psi(t') ~ c + s / (t' - E), E the nearest pole (the largest e_j), with c and s
// fitted to Psi and Psi' at the current point t:  s = -Psi'(t) (t - E)^2,
// c = Psi(t) + Psi'(t) (t - E).  For one term w^2/(t' - e) with e <= E the fitted model
// minus the term is  c (t' - t)^2 / ((t' - E)(t' - e)) >= 0,  c = w^2 (E - e)/(t - e)^2 >= 0,
// so the model lies above Psi everywhere above E and the model's root
//   a1 x^2 - A x - s = 0,  x = t' - E,  A = a0 + c - a1 E
// lies at or above the true root, from any t: in exact arithmetic the iterates come down
// to the root from above (quadratically; exactly in one step when one pole carries all
// the weight).  The candidates are kept strictly inside the bracket [lo, hi] of doubles
// (bit patterns, as in bisect); when the model no longer moves the upper end by more than
// one double, back-off steps hi - 1, hi - 4, hi - 16, ... find a point below the root (and
// lo + 1, lo + 4, ... a point above it when the model puts the root at the lower end), and
// the loop ends, like bisect, with an adjacent pair of doubles across the sign change.
// ---------------------------------------------------------------------------------
// ev(t, want, &psi, &dpsi) returns F(t) times a positive constant fscale and, when want is
// set, Psi(t) and Psi'(t) (back-off steps, which usually close the bracket, skip them).
// floor, alo, ahi as in bisect.
template <class Ev>
__device__ double accel_solve(Ev ev, double floor, double alo, double ahi, double E, double a0, double a1,
                              double fscale, int cap, bool* ok, int* steps_out) {
  if (!(floor >= 0.0)) floor = 0.0;
  if (!(alo >= floor)) alo = floor;
  if (!(ahi > alo)) ahi = (alo > 0.0) ? alo * 2.0 : 1.0;
  const uint64_t top = 0x7fefffffffffffffull;
  uint64_t lo = dbits(floor), hi = top;
  bool have_lo = false, have_hi = false, good = true;
  double Flo = 0.0, Fhi = 0.0;
  uint64_t t = dbits(ahi);
  uint64_t span = dbits(ahi) - dbits(alo) + 64;
  uint64_t back = 1, back_lo = 1, wref = 0;
  int steps = 0, model_steps = 0, since = 0;
  bool want = true, from_lo = false;
  // the bracket halves at least every second step once both ends are known: a third more
  // evaluations than the bisection's cap (128 for the default cap of 96)
  const int limit = cap + (cap + 2) / 3;
  for (;;) {
    if (steps >= limit) { good = false; break; }
    const double tv = dfrom(t);
    double psi = 0.0, dpsi = 0.0;
    const double F = ev(tv, want, &psi, &dpsi);
    steps++;
    if (F > 0.0) { lo = t; Flo = F; have_lo = true; }
    else { hi = t; Fhi = F; have_hi = true; }
    if (hi - lo <= 1) break;
    const double tc = want ? model_root(tv, F, psi, dpsi, E, a0, a1, fscale) : NAN;
    const uint64_t c = (tc > 0.0 && tc <= 1.7e308) ? dbits(tc) : 0ull;
    want = true;
    uint64_t nxt;
    if (!have_hi) {
      // every point so far lies below the root; the model's root lies above it
      if (c > t) nxt = c;
      else { nxt = (top - t > span) ? t + span : top; span *= 2; }
    } else {
      const bool use_model = c > lo && c + 1 < hi && model_steps < 24;
      bool force_mid = false;
      if (have_lo) {
        // both ends evaluated: the bracket must halve at least every second step
        const uint64_t wdt = hi - lo;
        if (wref == 0 || wdt <= wref / 2) { wref = wdt; since = 0; }
        else if (++since >= 2) force_mid = true;
      }
      if (force_mid) nxt = lo + ((hi - lo) >> 1);
      else if (use_model) { nxt = c; model_steps++; }
      else if (have_lo && (c != 0ull ? c <= lo : from_lo)) {
        // the model puts the root at the lower end (within rounding): step up from it
        nxt = (hi - lo > back_lo) ? lo + back_lo : lo + ((hi - lo) >> 1);
        back_lo = (back_lo < (1ull << 60)) ? back_lo * 4 : back_lo;
        want = false;
        from_lo = true;
      } else {
        nxt = (hi - lo > back) ? hi - back : lo + ((hi - lo) >> 1);
        back = (back < (1ull << 60)) ? back * 4 : back;
        want = false;
        from_lo = false;
      }
    }
    if (nxt <= lo || nxt >= hi) nxt = lo + ((hi - lo) >> 1);
    t = nxt;
  }
  double alo_g = have_lo ? fabs(Flo) : INFINITY;
  double ahi_g = have_hi ? fabs(Fhi) : INFINITY;
  if (isnan(alo_g)) alo_g = INFINITY;
  if (isnan(ahi_g)) ahi_g = INFINITY;
  *ok = good && have_hi;
  if (steps_out) *steps_out = steps;
  return dfrom((ahi_g < alo_g || !have_lo) && have_hi ? hi : lo);
}

// Larger root t of (t - B)(t - E) = W (W >= 0), evaluated without cancellation; +-inf or
// NaN when an argument is not finite (callers then ignore the bound).
__device__ __forceinline__ double qroot(double B, double E, double W) {
  const double c = E - B;
  const double s = sqrt(__fma_rn(c, c, 4.0 * W));
  const double x = (c > 0.0) ? (2.0 * W) / (c + s) : 0.5 * (s - c);
  return E + x;
}

// Quadratic bracket of the extreme eigenvalue t = |nu| > every pole e_j of the secular
// function t - B = sum_j w_j^2 / (t - e_j), W = sum_j w_j^2, poles in [Efar, Enear]: every
// denominator lies in [t - Enear, t - Efar], so t - B lies between W / (t - Efar) and
// W / (t - Enear), and t between the larger roots of (t - B)(t - Efar) = W and
// (t - B)(t - Enear) = W.  (The corner bound B + W / (B - Enear) is this upper bound with
// t - Enear replaced by B - Enear.)
__device__ __forceinline__ void quad_bracket(double B, double Efar, double Enear, double W, double* alo,
                                             double* ahi) {
  const double lo = qroot(B, Efar, W), hi = qroot(B, Enear, W);
  if (isfinite(lo)) *alo = fmax(*alo, lo);
  if (isfinite(hi)) *ahi = fmin(*ahi, hi);
}

// ---------------------------------------------------------------------------------
// Solve at a pole: extreme eigenvalue of the arrowhead inverse of A - d_i I.
// ---------------------------------------------------------------------------------
struct PoleResult {
  double mu, nu, b;
  bool ok;
  bool dd;     // b was formed in double-double
  int steps;
  int screened;   // bisection steps settled by the binary32 screen
  int screened_near;   // of those, steps whose margin over the screen's bound was below 2
  int screened_df;     // of those, steps settled by the double-float screen
  int inferred;        // bisection steps decided by certified bounds (no evaluation)
  int probes;          // screened probes that placed those bounds
};

// How the corner b is formed (Sec. 2.3): mode 1 in double the working precision when kappa_nu of
// Eq. (knu2) exceeds T_kappa n, as Algorithm 1 does, mode 2 always; zsum = sum_j |zeta_j| of the
// problem (for K_z).
struct CornerRule {
  int mode;
  double T_kappa;
  double zsum;
};

// Corner element of Eq. (b_ob): b = (1/zeta_i^2)(1/rho + sum_{j != i} zeta_j^2/(d_j - d_i)),
// rounded to binary64 (the arrowhead is formed in working precision).  Mode 1 first sums the
// terms in binary64, P over j < i (positive) and N over j > i (negative), and takes
//   K_b = (1 + rho P - rho N) / |1 + rho P + rho N|,   K_z = sum_{j != i} |zeta_j| / |zeta_i|,
//   kappa_nu = min((n + 4) sqrt(n) K_b, 3 sqrt(n) + (n + 4)(1 + 2 K_z))     (Eq. (knu2));
// b is then recomputed in double-double only when kappa_nu > T_kappa n.
// With Ds != nullptr the pass also stores the elements Delta_j and zz_j / Delta_j of the
// inverse for stored_sum (a pass of its own in mode 2).
template <int L>
__device__ __forceinline__ double corner_b(const double* __restrict__ d, const double* __restrict__ zz,
                                           const double* __restrict__ zl, int n, int i,
                                           double rho, int lane, unsigned gm, double* wn2, CornerRule cr,
                                           bool* used_dd, double* __restrict__ Ds, double* __restrict__ us,
                                           float* __restrict__ F, bool* scr_ok) {
  const double di = d[i];
  bool ok = F != nullptr;
  if (cr.mode != 2) {
    double p = 0.0, q = 0.0, s2 = 0.0;
    for (int j = lane; j < n; j += L) {
      if (j == i) {
        if (Ds) ok &= store_elem(Ds, us, F, n, j, 0.0, 0.0);
        continue;
      }
      const double D = __dsub_rn(d[j], di);
      const double r = rcp(D);
      const double t = __dmul_rn(zz[j], r);
      if (Ds) ok &= store_elem(Ds, us, F, n, j, D, t);
      if (j < i) p = __dadd_rn(p, t);
      else q = __dadd_rn(q, t);
      s2 = __fma_rn(t, r, s2);
    }
    const double P = group_sum<L>(p, gm), N = group_sum<L>(q, gm);
    *wn2 = group_sum<L>(s2, gm) / zz[i];
    const double nn = (double)n, sn = sqrt(nn);
    const double Kb = (1.0 + rho * P - rho * N) / fabs(1.0 + rho * P + rho * N);
    const double zi = sqrt(zz[i]);
    const double Kz = (cr.zsum - zi) / zi;
    const double kappa = fmin((nn + 4.0) * sn * Kb, 3.0 * sn + (nn + 4.0) * (1.0 + 2.0 * Kz));
    *scr_ok = !group_any<L>(!ok, gm);
    if (kappa <= cr.T_kappa * nn) {
      *used_dd = false;
      return (1.0 / zz[i]) * ((1.0 / rho + P) + N);
    }
  }
  *used_dd = true;
  if (cr.mode == 2) {
    if (Ds) {
      for (int j = lane; j < n; j += L) {
        const double D = (j == i) ? 0.0 : __dsub_rn(d[j], di);
        ok &= store_elem(Ds, us, F, n, j, D, (j == i) ? 0.0 : __dmul_rn(zz[j], rcp(D)));
      }
    }
    *scr_ok = !group_any<L>(!ok, gm);
  }
  double sq;
  dd acc = dd_pole_sum<L>(d, zz, zl, n, i, di, lane, gm, &sq);
  dd B = dd_add(dd_div({1.0, 0.0}, {rho, 0.0}), acc);
  const dd Zi = {zz[i], zl[i]};
  *wn2 = sq / Zi.hi;
  return dd_to_double(dd_div(B, Zi));
}

// Brackets of |nu| from the shift test (see the derivation in k_solve's comment).  Ds, us: the
// lane group's private buffers of n doubles each for the elements of the inverse (evaluations
// with stored_sum), or nullptr (each evaluation forms them from d and zz).
template <int L, bool NI = false>
__device__ PoleResult solve_pole(const double* __restrict__ d, const double* __restrict__ zl,
                                 const double* __restrict__ zz, int n, double rho, int k, int i, double alo,
                                 double ahi, int cap, bool fast, int lane, unsigned gm, CornerRule cr,
                                 double* __restrict__ Ds = nullptr, double* __restrict__ us = nullptr,
                                 bool screen = false) {
  PoleResult r;
  r.screened = 0;
  r.screened_near = 0;
  r.screened_df = 0;
  r.inferred = 0;
  r.probes = 0;
  double wn2;
  bool used_dd, scr_ok = false;
  // the binary32 copies and low parts follow the two binary64 arrays (us = Ds + n)
  float* const F = (Ds && screen && !fast) ? (float*)(us + n) : nullptr;
  double b = corner_b<L>(d, zz, zl, n, i, rho, lane, gm, &wn2, cr, &used_dd, Ds, us, F, &scr_ok);
  double side = (i == k) ? 1.0 : -1.0;
  double di = d[i];
  double inv_zi2 = 1.0 / zz[i];
  // Weyl: the extreme eigenvalue lies within ||w|| of max(b, max delta) (rightmost) or
  // min(b, min delta) (leftmost); Rayleigh: nu >= b (rightmost), nu <= b (leftmost).
  double wn = sqrt(wn2);
  // floor: the pole of g next to the extreme eigenvalue (largest delta_j for the
  // rightmost, smallest for the leftmost), or 0 when all poles lie on the other side.
  double floor, E;   // E: the nearest pole on |nu| (the accelerated solve's model pole)
  // [alo, ahi] from the caller (the shift test) rests on its choice of pole and is checked
  // before the bisection where it is the binding bound; the bounds below are rigorous up to
  // rounding and are only checked if the bisection closes on them.
  const double alo_in = alo, ahi_in = ahi;
  double rlo, rhi = INFINITY;
  // Corner bound: for the rightmost eigenvalue nu >= b and nu - b = sum_j w_j^2 / (nu - delta_j)
  // <= ||w||^2 / (b - max delta) when b > max delta (mirrored for the leftmost).  Next to a
  // pole b ~ 1/zeta_i^2 dominates and this bracket is narrow.
  if (side > 0) {
    // largest delta_j: the nearest pole above d_i, or for i = 0 the farthest pole below
    double dmax = (i > 0) ? 1.0 / (d[i - 1] - di) : (n > 1 ? 1.0 / (d[n - 1] - di) : -INFINITY);
    floor = fmax(dmax, 0.0);
    E = dmax;
    rlo = b;
    rhi = fmax(b, dmax) + wn;
    if (b > dmax) rhi = fmin(rhi, b + wn2 / (b - dmax));
    // smallest delta_j: the nearest pole below d_i, or for i = n-1 the farthest pole above
    const double dmin = (i + 1 < n) ? 1.0 / (d[i + 1] - di) : (n > 1 ? 1.0 / (d[0] - di) : -INFINITY);
    quad_bracket(b, dmin, dmax, wn2, &rlo, &rhi);
  } else {
    double dmin = (i + 1 < n) ? 1.0 / (d[i + 1] - di) : INFINITY;
    floor = fmax(-dmin, 0.0);
    // smallest delta_j: the nearest pole below d_i, or for i = n-1 the farthest pole above
    E = (i + 1 < n) ? -dmin : (n > 1 ? -1.0 / (d[0] - di) : -INFINITY);
    rlo = -b;
    rhi = -fmin(b, dmin) + wn;
    if (b < dmin) rhi = fmin(rhi, -b + wn2 / (dmin - b));
    // on t = -nu the poles are -delta_j: the nearest is -dmin, the farthest -(largest delta_j)
    const double dmx = (i > 0) ? 1.0 / (d[i - 1] - di) : (n > 1 ? 1.0 / (d[n - 1] - di) : INFINITY);
    quad_bracket(-b, -dmx, -dmin, wn2, &rlo, &rhi);
  }
  alo = fmax(alo_in, rlo);
  ahi = fmin(ahi_in, rhi);
  const bool eager_lo = alo_in > rlo, eager_hi = ahi_in < rhi;
  // a few ulps of margin for the rounding of the bounds
  alo = alo * (1.0 - 0x1p-48);
  ahi = ahi * (1.0 + 0x1p-48);
  bool ok;
  int steps;
  double nu;
  if (fast) {
    // F(t) = side * g(side * t) = side b - t + Psi(t), Psi = -side S / zeta_i^2
    auto ev = [&](double t, bool want, double* psi, double* dpsi) {
      const double v = side * t;
      double dS = 0.0;
      const double S = want ? elem_sum_d<L>(Ds, us, d, zz, n, i, di, v, lane, gm, &dS)
                            : elem_sum<L>(Ds, us, d, zz, n, i, di, v, lane, gm);
      const double Sz = __dmul_rn(S, inv_zi2);
      *psi = -side * Sz;
      *dpsi = -__dmul_rn(dS, inv_zi2);
      const double g = __dsub_rn(__dsub_rn(b, v), Sz);
      return side > 0 ? g : -g;
    };
    nu = side * accel_solve(ev, floor, alo, ahi, E, side * b, 1.0, 1.0, cap, &ok, &steps);
  } else {
    auto phi = [&](double v) {
      double S = elem_sum<L, false, NI>(Ds, us, d, zz, n, i, di, v, lane, gm);
      return __dsub_rn(__dsub_rn(b, v), __dmul_rn(S, inv_zi2));
    };
    // The screen settles a step when its g = fl(fl(b - v) - fl(Sx inv_zi2)) exceeds every
    // way the decision could differ from phi's: |Sx - S| <= Ex (the screen's bound),
    // |S64 - S| <= stored_sum_error for phi's binary64 sum, and the roundings of the two
    // products.  fl(x - y) has the sign of x - y, so phi's sign then equals the sign of g.
    const double mlane = (double)((n + L - 1) / L);
    auto decide = [&](double Sx, double Ex, double aS, double v, double* g, double* tl) -> bool {
      const double E64 = stored_sum_error<L>(mlane, aS);
      const double tol = 1.01 * inv_zi2 * (Ex + E64 + 0x1p-51 * aS);
      const double G = __dsub_rn(__dsub_rn(b, v), __dmul_rn(Sx, inv_zi2));
      if (!(fabs(G) > tol)) return false;
      if (fabs(G) <= 2.0 * tol) r.screened_near++;
      *g = G;
      *tl = tol;
      return true;
    };
    // the binary32 screen first; after kScreenTries consecutive failures (its window is reached)
    // the double-float screen alone, whose window is narrower by about 2^22
    int f32_fail = 0;
    auto scr = [&](double v, double* g, double* tl, int mode, double* psi, double* dpsi) -> bool {
      if (!scr_ok) return false;
      double Sx, Ex, aS, dS = 0.0;
      bool ok = false;
      if (mode == 0 || (mode < 0 && f32_fail < kScreen32Tries)) {
        ok = (psi ? screen_sum_x<NI, L, true>(F, F + n, n, v, lane, gm, &Sx, &Ex, &aS, &dS)
                  : screen_sum_x<NI, L>(F, F + n, n, v, lane, gm, &Sx, &Ex, &aS)) &&
             decide(Sx, Ex, aS, v, g, tl);
        if (ok) {
          if (mode < 0) f32_fail = 0;
        } else {
          if (mode == 0) return false;
          f32_fail++;
        }
      }
      if (!ok) {
        if (mode == 1) f32_fail = kScreen32Tries;   // the probes have reached the binary32 window
        ok = kScreenDf &&
             (psi ? screen_df_sum_x<NI, L, true>(F, n, v, lane, gm, &Sx, &Ex, &aS, &dS)
                  : screen_df_sum_x<NI, L>(F, n, v, lane, gm, &Sx, &Ex, &aS)) &&
             decide(Sx, Ex, aS, v, g, tl);
        if (!ok) return false;
        r.screened_df++;
      }
      // Psi and Psi' on t = |nu| as the accelerated solve forms them (F = side b - t + Psi)
      if (psi) {
        *psi = -side * __dmul_rn(Sx, inv_zi2);
        *dpsi = -__dmul_rn(dS, inv_zi2);
      }
      return true;
    };
    // g(nu) > 0 below the root for the rightmost; for the leftmost, |nu| below the root
    // means nu above it, where g < 0.
    nu = bisect(phi, side, floor, alo, ahi, side > 0, cap, &ok, &steps, eager_lo, eager_hi, scr, &r.screened,
                kPredict && scr_ok, E, side * b, &r.inferred, &r.probes);
  }
  r.nu = nu;
  r.mu = 1.0 / nu;
  r.b = b;
  r.ok = ok;
  r.dd = used_dd;
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
// With OFS the shift is sigma + sigma_lo in double the working precision (remedy R2 when no
// binary64 number lies between lambda and a neighbouring pole): the elements of the DPR1 matrix
// are the binary64 roundings of the double-double differences d_j - sigma (elem_diff) and
// f(sigma) is formed from those differences in double-double.
template <int L, bool OFS = false, bool NI = false>
__device__ double solve_nonpole(const double* __restrict__ d, const double* __restrict__ zl,
                                const double* __restrict__ zz, int n, double rho, double sigma, int above, int below,
                                int cap, bool fast, int lane, unsigned gm, bool* ok, int* steps_out = nullptr,
                                double* __restrict__ Ds = nullptr, double* __restrict__ us = nullptr,
                                double sigma_lo = 0.0) {
  // above / below: indices of the poles next to sigma (-1: none on that side)
  double un2, cub;
  // the double-double pass also stores the elements d_j - sigma and zeta_j^2 / (d_j - sigma)
  // for the solve when the group has a buffer (Ds, us as for solve_pole)
  dd acc = dd_pole_sum<L, OFS>(d, zz, zl, n, -1, sigma, lane, gm, &un2, &cub, Ds, us, nullptr, nullptr,
                               sigma_lo);
  dd f = dd_add({1.0, 0.0}, two_prod(acc.hi, rho));
  f = dd_add(f, {__dmul_rn(acc.lo, rho), 0.0});
  *ok = true;
  if (f.hi == 0.0 && f.lo == 0.0) return 0.0;
  double gamma = dd_to_double(dd_div({-rho, 0.0}, f));
  // extreme e_j = 1/(d_j - sigma): the poles next to sigma
  const double emax = above >= 0 ? 1.0 / elem_diff<OFS>(d[above], sigma, sigma_lo) : -INFINITY;
  const double emin = below >= 0 ? 1.0 / elem_diff<OFS>(d[below], sigma, sigma_lo) : INFINITY;
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
  int steps;
  double nu;
  if (fast) {
    // F(t) = -h(side * t) = |gamma| (Psi(t) - 1/|gamma|), Psi = -side S; model pole: the
    // largest e_j on |nu| (with no pole above sigma, the one farthest below it)
    const double E = (gamma > 0.0) ? (above >= 0 ? emax : 1.0 / elem_diff<OFS>(d[n - 1], sigma, sigma_lo))
                                   : (below >= 0 ? -emin : -1.0 / elem_diff<OFS>(d[0], sigma, sigma_lo));
    const double ag = fabs(gamma);
    auto ev = [&](double t, bool want, double* psi, double* dpsi) {
      double dS = 0.0;
      const double S = want ? elem_sum_d<L, OFS>(Ds, us, d, zz, n, -1, sigma, side * t, lane, gm, &dS, sigma_lo)
                            : elem_sum<L, OFS, NI>(Ds, us, d, zz, n, -1, sigma, side * t, lane, gm, sigma_lo);
      *psi = -side * S;
      *dpsi = -dS;
      return -__fma_rn(gamma, S, 1.0);
    };
    nu = side * accel_solve(ev, floor, alo, ahi, E, -1.0 / ag, 0.0, ag, cap, ok, &steps);
  } else {
    auto phi = [&](double v) {
      const double S = elem_sum<L, OFS, NI>(Ds, us, d, zz, n, -1, sigma, v, lane, gm, sigma_lo);
      return __fma_rn(gamma, S, 1.0);
    };
    nu = bisect(phi, side, floor, alo, ahi, false, cap, ok, &steps);
  }
  if (steps_out) *steps_out = steps;
  return 1.0 / nu;
}

}  // namespace dpr1
