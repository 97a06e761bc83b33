// dpr1_eig.cu -- all eigenpairs of one DPR1 matrix A = D + rho z z^T on sm_103a.
//
// Launch sequence on the caller's stream (Algorithm 1, dpr1eig, for every k at once):
//   k_scan      input checks, copies d, z, z^2 into the workspace, deflation tests (Sec. 1)
//   k_deflate   exact deflation (zeta_j == 0, ties) when k_scan found any; else returns
//   k_solve     per eigenvalue (one lane group): shift test, corner b in double-double,
//               bisection for the extreme eigenvalue nu of the arrowhead inverse
//   k_classify  K_nu of Eq. (K0) from the neighbouring eigenvalues; picks R1 / R2 candidates
//   k_fix       R1 (the other pole) and R2 (non-pole shift, f(sigma) in double-double)
//   k_zero      eigenvalues much closer to zero than to their poles: lambda from A^{-1}
//   k_vectors   lambda, (sigma, mu), ||x|| and the rows of V^T, v = x / ||x||
// The shared-memory / register details of the hot loop are in the k_solve comment.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>

#include "../../include/dpr1.h"
#include "dpr1_device.cuh"
#include "dpr1_internal.cuh"

namespace dpr1 {

// ---------------------------------------------------------------------------------
// Workspace layout
// ---------------------------------------------------------------------------------
static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t ws_layout(int64_t n, Ws* w, char* base) {
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += align256(bytes);
    return base ? base + o : nullptr;
  };
  size_t nn = (size_t)(n > 0 ? n : 1);
  char* hdr = take(sizeof(unsigned) * 64);
  char* dr = take(sizeof(double) * nn);
  char* zr = take(sizeof(double) * nn);
  char* zz = take(sizeof(double) * nn);
  char* sig = take(sizeof(double) * nn);
  char* mu = take(sizeof(double) * nn);
  char* shift = take(sizeof(int) * nn);
  char* flag = take(sizeof(int) * nn);
  char* list = take(sizeof(int) * nn);
  char* lamz = take(sizeof(double) * nn);
  char* src = take(sizeof(int) * nn);
  char* coef = take(sizeof(double) * nn);
  char* rpos = take(sizeof(int) * nn);
  char* dpos = take(sizeof(int) * nn);
  char* gst = take(sizeof(int) * nn);
  char* rprev = take(sizeof(double) * nn);
  char* rcur = take(sizeof(double) * nn);
  char* dlist = take(sizeof(int) * nn);
  char* zlist = take(sizeof(int) * nn);
  char* fk = take(sizeof(double) * nn * 3);
  if (w && base) {
    w->hdr = (unsigned*)hdr;
    w->status = (unsigned*)hdr;
    w->counters = (unsigned*)hdr + 8;
    w->nred = (int*)((unsigned*)hdr + 32);
    w->ndefl = (int*)((unsigned*)hdr + 33);
    w->dr = (double*)dr; w->zr = (double*)zr; w->zz = (double*)zz;
    w->sig = (double*)sig; w->mu = (double*)mu;
    w->shift = (int*)shift; w->flag = (int*)flag; w->list = (int*)list;
    w->lamz = (double*)lamz;
    w->src = (int*)src; w->coef = (double*)coef; w->rpos = (int*)rpos; w->dpos = (int*)dpos;
    w->gst = (int*)gst; w->rprev = (double*)rprev; w->rcur = (double*)rcur; w->dlist = (int*)dlist;
    w->zlist = (int*)zlist;
    w->fixinfo = (double*)fk;
  }
  return off;
}

// ---------------------------------------------------------------------------------
// k_scan: checks and copies; one thread per j
// ---------------------------------------------------------------------------------
__global__ void k_scan(int n, const double* __restrict__ d, const double* __restrict__ z, Ws w) {
  unsigned bits = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) *w.nred = n;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    double dj = d[j], zj = z[j];
    if (!isfinite(dj) || !isfinite(zj)) bits |= ST_NONFINITE;
    if (j + 1 < n) {
      double dn = d[j + 1];
      if (dj < dn) bits |= ST_UNSORTED;
      if (dj == dn) bits |= ST_DEFLATED;
    }
    if (zj == 0.0) bits |= ST_DEFLATED;
    if (dj == 0.0) bits |= ST_ZERO_POLE;
    w.dr[j] = dj;
    w.zr[j] = zj;
    w.zz[j] = __dmul_rn(zj, zj);
  }
  bits = __reduce_or_sync(FULL, bits);
  if ((threadIdx.x & 31) == 0 && bits) atomicOr(w.status, bits);
}

// ---------------------------------------------------------------------------------
// k_deflate: exact deflation of Sec. 1, one thread (runs only when k_scan found a
// zero zeta_j or a tie d_j == d_{j+1}).  Ties: the non-zero weights of a group of
// equal poles are rotated into its first non-zero member by a chain of Givens
// rotations; the survivor keeps zeta = ||group||, every other member becomes an
// eigenpair (d_group, Q^T e_m).  Writes the reduced problem (dr, zr, zz, nred), for
// every position p its source reduced index src[p] (-1: none) and coefficient
// coef[p] = zeta_p / ||group|| (1 for singletons), the list of deflated positions,
// and for tie members the prefix norms rprev (before) and rcur (including) them.
// ---------------------------------------------------------------------------------
__global__ void k_deflate(int n, const double* __restrict__ d, const double* __restrict__ z, Ws w) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  unsigned st = *w.status;
  *w.ndefl = 0;
  if (!(st & ST_DEFLATED) || (st & (ST_UNSORTED | ST_NONFINITE))) return;
  int nr = 0, nd = 0;
  int j = 0;
  while (j < n) {
    int e = j;
    while (e + 1 < n && d[e + 1] == d[j]) e++;
    // group [j, e] of equal poles
    int first = -1;
    double r = 0.0;
    for (int p = j; p <= e; p++) {
      w.gst[p] = j;
      if (z[p] == 0.0) {
        w.src[p] = -1; w.coef[p] = 0.0; w.rprev[p] = 0.0; w.rcur[p] = 0.0;
        w.dlist[nd++] = p;
        continue;
      }
      double rp = r;
      r = hypot(r, z[p]);
      w.rprev[p] = rp; w.rcur[p] = r;
      if (first < 0) first = p;
      else w.dlist[nd++] = p;
    }
    if (first >= 0) {
      // survivor: the group's rotated weight; the signed weight of the first member keeps
      // the survivor's orientation (coef[first] > 0)
      double zs = (z[first] > 0.0) ? r : -r;
      for (int p = j; p <= e; p++) {
        if (z[p] == 0.0) continue;
        w.src[p] = nr;
        w.coef[p] = z[p] / zs;
      }
      w.dr[nr] = d[j];
      w.zr[nr] = zs;
      w.zz[nr] = __dmul_rn(zs, zs);
      nr++;
    }
    j = e + 1;
  }
  *w.nred = nr;
  *w.ndefl = nd;
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
template <int L>
__device__ __forceinline__ double arrow_sum(const double* __restrict__ d, const double* __restrict__ zz, int n,
                                            int i, double di, double nu, int lane, unsigned gm) {
  double s0 = 0.0, s1 = 0.0;
  int j = lane;
  for (; j + L < n; j += 2 * L) {
    double D0 = __dsub_rn(d[j], di), D1 = __dsub_rn(d[j + L], di);
    double t0 = __fma_rn(-nu, D0, 1.0), t1 = __fma_rn(-nu, D1, 1.0);
    double r0 = rcp(__dmul_rn(D0, t0)), r1 = rcp(__dmul_rn(D1, t1));
    double c0 = __dmul_rn(zz[j], r0), c1 = __dmul_rn(zz[j + L], r1);
    s0 = __dadd_rn(s0, (j == i) ? 0.0 : c0);
    s1 = __dadd_rn(s1, (j + L == i) ? 0.0 : c1);
  }
  if (j < n) {
    double D0 = __dsub_rn(d[j], di);
    double t0 = __fma_rn(-nu, D0, 1.0);
    double c0 = __dmul_rn(zz[j], rcp(__dmul_rn(D0, t0)));
    s0 = __dadd_rn(s0, (j == i) ? 0.0 : c0);
  }
  return group_sum<L>(__dadd_rn(s0, s1), gm);
}

// Same terms with Delta_j = d_j - sigma for a non-pole shift (no excluded index):
// sum_j u_j^2 / (e_j - nu), e_j = 1/(d_j - sigma), u_j = zeta_j/(d_j - sigma).
template <int L>
__device__ __forceinline__ double shift_sum(const double* __restrict__ d, const double* __restrict__ zz, int n,
                                            double sigma, double nu, int lane, unsigned gm) {
  double s0 = 0.0, s1 = 0.0;
  int j = lane;
  for (; j + L < n; j += 2 * L) {
    double D0 = __dsub_rn(d[j], sigma), D1 = __dsub_rn(d[j + L], sigma);
    double t0 = __fma_rn(-nu, D0, 1.0), t1 = __fma_rn(-nu, D1, 1.0);
    s0 = __fma_rn(zz[j], rcp(__dmul_rn(D0, t0)), s0);
    s1 = __fma_rn(zz[j + L], rcp(__dmul_rn(D1, t1)), s1);
  }
  if (j < n) {
    double D0 = __dsub_rn(d[j], sigma);
    double t0 = __fma_rn(-nu, D0, 1.0);
    s0 = __fma_rn(zz[j], rcp(__dmul_rn(D0, t0)), s0);
  }
  return group_sum<L>(__dadd_rn(s0, s1), gm);
}

// sum_{j != skip} zeta_j^2 / (d_j - s) in double-double (skip = -1: all j); also returns
// sum_{j != skip} zeta_j^2 / (d_j - s)^2 in binary64 (the squared norm of the border).
template <int L>
__device__ __forceinline__ dd dd_pole_sum(const double* __restrict__ d, const double* __restrict__ z, int n,
                                          int skip, double s, int lane, unsigned gm, double* sq) {
  dd acc = {0.0, 0.0};
  double q = 0.0;
  for (int j = lane; j < n; j += L) {
    if (j == skip) continue;
    dd D = two_sum(d[j], -s);
    dd Z = two_prod(z[j], z[j]);
    dd c = dd_div(Z, D);
    acc = dd_add(acc, c);
    q = __fma_rn(c.hi, rcp(D.hi), q);
  }
  *sq = group_sum<L>(q, gm);
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
  // far end
  for (int t = 0; t < 8; t++) {
    double g = phi(side * dfrom(hi));
    steps++;
    bool below = below_positive ? (g > 0.0) : (g < 0.0);
    if (!below) { ghi = g; have_hi = true; break; }
    uint64_t wd = hi - lo;
    lo = hi; glo = g; have_lo = true;
    hi = hi + 2 * wd + (1ull << 40);
    if (hi >= 0x7ff0000000000000ull) hi = 0x7fefffffffffffffull;
  }
  // near end, never below the floor
  for (int t = 0; t < 8 && !have_lo && lo > fl; t++) {
    double g = phi(side * dfrom(lo));
    steps++;
    bool below = below_positive ? (g > 0.0) : (g < 0.0);
    if (below) { glo = g; have_lo = true; break; }
    hi = lo; ghi = g; have_hi = true;
    lo = (lo > fl + (1ull << 52)) ? lo - (1ull << 52) : fl;
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
  if (side > 0) {
    // largest delta_j: the nearest pole above d_i, or for i = 0 the farthest pole below
    double dmax = (i > 0) ? 1.0 / (d[i - 1] - di) : (n > 1 ? 1.0 / (d[n - 1] - di) : -INFINITY);
    floor = fmax(dmax, 0.0);
    alo = fmax(alo, b * (1.0 - 0x1p-30));
    ahi = fmin(ahi, fmax(b, dmax) + wn);
  } else {
    double dmin = (i + 1 < n) ? 1.0 / (d[i + 1] - di) : INFINITY;
    floor = fmax(-dmin, 0.0);
    alo = fmax(alo, -b * (1.0 - 0x1p-30));
    ahi = fmin(ahi, -fmin(b, dmin) + wn);
  }
  alo = alo * (1.0 - 0x1p-30);
  ahi = ahi * (1.0 + 0x1p-30);
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
// k_solve: one lane group of L threads per eigenvalue; groups take eigenvalues from a
// global counter (persistent grid).
//
// Shift test (Algorithm 1): tau = (d_{k-1} - d_k)/2 and
//   F = 1 + rho sum_j zeta_j^2 / ((d_j - d_k) - tau);  F > 0 -> sigma = d_k, else d_{k-1}.
// The same pass gives rigorous brackets for nu (derived from f(d_i + mu) = 0):
//   sigma = d_k:     mu in (0, tau]   -> 1/tau <= nu <= (1 + rho P) / (rho zeta_k^2),
//                    P = sum_{j<k} zeta_j^2 / ((d_j - d_k) - tau)   (the positive terms of F)
//   sigma = d_{k-1}: mu in [-tau, 0)  -> 1/tau <= |nu| <= (-1 - rho N) / (rho zeta_{k-1}^2),
//                    N = sum_{j>=k} zeta_j^2 / ((d_j - d_k) - tau)  (the negative terms of F)
//   k = 1:           mu in [rho zeta_1^2, rho ||z||^2] -> nu in [1/(rho ||z||^2), 1/(rho zeta_1^2)]
// ---------------------------------------------------------------------------------
template <int L>
__global__ void __launch_bounds__(256) k_solve(Ws w, double rho, int cap) {
  const int n = *w.nred;
  if (*w.status & (ST_UNSORTED | ST_NONFINITE)) return;
  const int lane = threadIdx.x & (L - 1);
  const unsigned gm = group_mask<L>();
  const int leader = (threadIdx.x & 31) & ~(L - 1);
  const double* __restrict__ d = w.dr;
  const double* __restrict__ z = w.zr;
  const double* __restrict__ zz = w.zz;
  for (;;) {
    int k = 0;
    if (lane == 0) k = (int)atomicAdd(&w.counters[0], 1u);
    k = __shfl_sync(gm, k, leader, 32);
    if (k >= n) break;
    int i;
    double alo, ahi;
    if (k == 0) {
      double s = 0.0;
      for (int j = lane; j < n; j += L) s = __dadd_rn(s, zz[j]);
      s = group_sum<L>(s, gm);
      i = 0;
      alo = 1.0 / (rho * s);
      ahi = 1.0 / (rho * zz[0]);
    } else {
      double dk = d[k];
      double tau = __dmul_rn(__dsub_rn(d[k - 1], dk), 0.5);
      double sp = 0.0, sn = 0.0;
      for (int j = lane; j < n; j += L) {
        double den = __dsub_rn(__dsub_rn(d[j], dk), tau);
        double t = __dmul_rn(zz[j], rcp(den));
        if (j < k) sp = __dadd_rn(sp, t);
        else sn = __dadd_rn(sn, t);
      }
      sp = group_sum<L>(sp, gm);
      sn = group_sum<L>(sn, gm);
      double F = 1.0 + rho * (sp + sn);
      if (F > 0.0) {
        i = k;
        alo = 1.0 / tau;
        ahi = (1.0 + rho * sp) / (rho * zz[k]);
      } else {
        i = k - 1;
        alo = 1.0 / tau;
        ahi = (-1.0 - rho * sn) / (rho * zz[k - 1]);
      }
    }
    PoleResult pr = solve_pole<L>(d, z, zz, n, rho, k, i, alo, ahi, cap, lane, gm);
    if (lane == 0) {
      w.sig[k] = d[i];
      w.mu[k] = pr.mu;
      w.shift[k] = i;
      w.flag[k] = 0;
      atomicAdd(&w.counters[C_EVAL_SOLVE], (unsigned)pr.steps);
      if (!pr.ok) atomicOr(w.status, ST_NOT_CONVERGED);
    }
  }
}

// ---------------------------------------------------------------------------------
// k_classify: K_nu = ||A_i^{-1}||_2 / |nu| (Eq. (K0)).  ||A_i^{-1}||_2 is the reciprocal
// distance from d_i to the spectrum; the eigenvalues next to pole d_i are lambda_i
// (above) and lambda_{i+1} (below), one of which is lambda_k, so
//   K_nu = max(1, |mu_k| / |lambda_m - d_i|),  lambda_m the other neighbour of d_i.
// For K_nu > T_Knu the eigenvalue goes to k_fix with the candidate other pole o and
//   K'  = max(1, |lambda_k - d_o| / |lambda_m' - d_o|)   (m' the other neighbour of d_o),
//   ratio = |lambda_k - d_o| / |lambda_k - d_i|.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ double dist_to(const Ws& w, int m, double p) {
  // |lambda_m - p| from the pair (sig_m, mu_m)
  return fabs(__dadd_rn(__dsub_rn(w.sig[m], p), w.mu[m]));
}

__global__ void k_classify(Ws w, double T_Knu) {
  const int n = *w.nred;
  if (*w.status & (ST_UNSORTED | ST_NONFINITE)) return;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    int i = w.shift[k];
    double di = w.dr[i];
    double mu = w.mu[k];
    double mk = fabs(mu);
    int m = (i == k) ? k + 1 : k - 1;
    double K = 1.0;
    if (m >= 0 && m < n) K = fmax(1.0, mk / dist_to(w, m, di));
    if (K > T_Knu) {
      // the other neighbouring pole o of lambda_k, its K' and the distance ratio, all from
      // the results of k_solve (k_fix overwrites pairs, so they are captured here)
      int o = (i == k) ? k - 1 : k;
      double K2 = INFINITY, ratio = INFINITY;
      if (o >= 0 && o < n && o != i) {
        double dko = fabs(__dadd_rn(__dsub_rn(di, w.dr[o]), mu));
        int m2 = (o == k) ? k + 1 : k - 1;
        K2 = 1.0;
        if (m2 >= 0 && m2 < n) K2 = fmax(1.0, dko / dist_to(w, m2, w.dr[o]));
        ratio = dko / mk;
      }
      unsigned slot = atomicAdd(&w.counters[1], 1u);
      w.list[slot] = k;
      w.fixinfo[3 * (size_t)slot] = K;
      w.fixinfo[3 * (size_t)slot + 1] = K2;
      w.fixinfo[3 * (size_t)slot + 2] = ratio;
      w.flag[k] = 1;
    }
  }
}

// ---------------------------------------------------------------------------------
// k_fix: remedies for the flagged eigenvalues, one lane group each.
//  (R1) solve at the other neighbouring pole o; accept when K' < K, K' <= T_Knu and
//       ratio <= T_Knu (beyond that ratio the eigenvector formula at d_o cancels).
//  (R2) otherwise shift to sigma = fl(lambda) from the better pole solution, moved into
//       the open interval (d_k, d_{k-1}) if it falls on a pole; form
//       f(sigma) = 1 + rho sum zeta_j^2 / (d_j - sigma) in double-double,
//       gamma = -rho / f(sigma), and bisect
//       h(nu) = 1 + gamma sum_j u_j^2 / (e_j - nu),  e_j = 1/(d_j - sigma), u_j = zeta_j/(d_j - sigma),
//       for the exterior eigenvalue of (A - sigma I)^{-1} = diag(e) + gamma u u^T:
//       the rightmost (nu > 0) when gamma > 0, the leftmost when gamma < 0; h < 0 on
//       the pole side in both cases.  mu = 1/nu; f(sigma) == 0 gives mu = 0.
// ---------------------------------------------------------------------------------
template <int L>
__device__ double solve_nonpole(const double* __restrict__ d, const double* __restrict__ z,
                                const double* __restrict__ zz, int n, double rho, double sigma, int cap, int lane,
                                unsigned gm, bool* ok, int* steps_out = nullptr) {
  double un2;
  dd acc = dd_pole_sum<L>(d, z, n, -1, sigma, lane, gm, &un2);
  dd f = dd_add({1.0, 0.0}, two_prod(acc.hi, rho));
  f = dd_add(f, {__dmul_rn(acc.lo, rho), 0.0});
  *ok = true;
  if (f.hi == 0.0 && f.lo == 0.0) return 0.0;
  double gamma = dd_to_double(dd_div({-rho, 0.0}, f));
  // largest / smallest e_j: the poles next to sigma
  double emax = -INFINITY, emin = INFINITY;
  for (int j = lane; j < n; j += L) {
    double e = 1.0 / __dsub_rn(d[j], sigma);
    emax = fmax(emax, e);
    emin = fmin(emin, e);
  }
  emax = group_max<L>(emax, gm);
  emin = -group_max<L>(-emin, gm);
  double side, alo, ahi;
  if (gamma > 0.0) {
    side = 1.0;
    alo = fmax(emax, 0.0);
    ahi = fmax(emax, 0.0) + gamma * un2;
  } else {
    side = -1.0;
    alo = -emin;
    ahi = -emin - gamma * un2;
  }
  ahi *= (1.0 + 0x1p-30);
  auto phi = [&](double nu) { return __fma_rn(gamma, shift_sum<L>(d, zz, n, sigma, nu, lane, gm), 1.0); };
  int steps;
  // the floor is the pole e_max (or e_min), or 0 when all e_j lie on the other side
  double nu = bisect(phi, side, alo, alo, ahi, false, cap, ok, &steps);
  if (steps_out) *steps_out = steps;
  return 1.0 / nu;
}

template <int L>
__global__ void __launch_bounds__(256) k_fix(Ws w, double rho, double T_Knu, int cap) {
  const int n = *w.nred;
  if (*w.status & (ST_UNSORTED | ST_NONFINITE)) return;
  const int nfix = (int)w.counters[1];
  const int lane = threadIdx.x & (L - 1);
  const unsigned gm = group_mask<L>();
  const int leader = (threadIdx.x & 31) & ~(L - 1);
  const double* __restrict__ d = w.dr;
  const double* __restrict__ z = w.zr;
  const double* __restrict__ zz = w.zz;
  for (;;) {
    int t = 0;
    if (lane == 0) t = (int)atomicAdd(&w.counters[2], 1u);
    t = __shfl_sync(gm, t, leader, 32);
    if (t >= nfix) break;
    int k = w.list[t];
    int i = w.shift[k];
    double di = d[i];
    double mu = w.mu[k];
    const double K = w.fixinfo[3 * (size_t)t];
    const double K2 = w.fixinfo[3 * (size_t)t + 1];
    const double ratio = w.fixinfo[3 * (size_t)t + 2];
    double new_sig = di, new_mu = mu;
    int new_shift = i;
    bool done = false;
    double best_sig = di, best_mu = mu;
    int o = (i == k) ? k - 1 : k;
    if (o >= 0 && o < n && o != i && K2 < K) {
      // bracket of |nu| at the other pole: |lambda_k - d_o| < d_{k-1} - d_k
      double span = __dsub_rn(d[k - 1], d[k]);
      PoleResult pr = solve_pole<L>(d, z, zz, n, rho, k, o, 0.0, INFINITY, cap, lane, gm);
      (void)span;
      if (!pr.ok && lane == 0) atomicOr(w.status, ST_NOT_CONVERGED);
      if (lane == 0) atomicAdd(&w.counters[C_EVAL_FIX], (unsigned)pr.steps);
      best_sig = d[o];
      best_mu = pr.mu;
      if (K2 <= T_Knu && ratio <= T_Knu) {
        new_sig = d[o]; new_mu = pr.mu; new_shift = o; done = true;
      }
    }
    if (!done) {
      double s = __dadd_rn(best_sig, best_mu);
      double lo = d[k];
      double hi = (k > 0) ? d[k - 1] : INFINITY;
      if (s <= lo) s = dnext_up(lo);
      if (s >= hi) s = dnext_down(hi);
      if (s > lo && s < hi) {
        bool ok;
        int st2 = 0;
        double m2 = solve_nonpole<L>(d, z, zz, n, rho, s, cap, lane, gm, &ok, &st2);
        if (!ok && lane == 0) atomicOr(w.status, ST_NOT_CONVERGED);
        if (lane == 0) atomicAdd(&w.counters[C_EVAL_FIX], (unsigned)st2);
        new_sig = s; new_mu = m2; new_shift = -1;
      }
    }
    if (lane == 0) {
      w.sig[k] = new_sig;
      w.mu[k] = new_mu;
      w.shift[k] = new_shift;
      if (new_shift == -1) atomicAdd(&w.counters[C_R2], 1u);
      else if (new_shift != i) atomicAdd(&w.counters[C_R1], 1u);
      w.flag[k] = (new_shift == -1) ? 2 : (new_shift != i ? 1 : 0);
    }
  }
}

// ---------------------------------------------------------------------------------
// Eigenvalues much closer to zero than to their neighbouring poles,
// T_zero |lambda| < min(|lambda - d_k|, |lambda - d_{k-1}|), when no pole is zero:
// lambda = 1/nu, nu the extreme eigenvalue of A^{-1} = D^{-1} + gamma D^{-1} z z^T D^{-1}
// (Eq. (gamma)) -- the non-pole solve with sigma = 0.  k_zero_detect marks candidates
// (the paper notes there is at most one); k_zero_solve handles them one warp each.
// lamz[k] = NaN means "not recomputed".
// ---------------------------------------------------------------------------------
__global__ void k_zero_detect(Ws w, double T_zero) {
  const int n = *w.nred;
  if (*w.status & (ST_UNSORTED | ST_NONFINITE)) return;
  const bool zero_pole = (*w.status & ST_ZERO_POLE) != 0;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    w.lamz[k] = __longlong_as_double(0x7ff8000000000000ll);
    if (zero_pole) continue;
    double s = w.sig[k], m = w.mu[k];
    double lam = __dadd_rn(s, m);
    double m1 = fabs(__dadd_rn(__dsub_rn(s, w.dr[k]), m));
    if (k > 0) m1 = fmin(m1, fabs(__dadd_rn(__dsub_rn(s, w.dr[k - 1]), m)));
    if (T_zero * fabs(lam) < m1) {
      unsigned slot = atomicAdd(&w.counters[3], 1u);
      w.zlist[slot] = k;
    }
  }
}

__global__ void k_zero_solve(Ws w, double rho, int cap) {
  const int n = *w.nred;
  if (*w.status & (ST_UNSORTED | ST_NONFINITE)) return;
  const int nz = (int)w.counters[3];
  const int lane = threadIdx.x & 31;
  const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int t = wid; t < nz; t += nw) {
    int k = w.zlist[t];
    bool ok;
    double lam0 = solve_nonpole<32>(w.dr, w.zr, w.zz, n, rho, 0.0, cap, lane, FULL, &ok);
    if (lane == 0) {
      w.lamz[k] = lam0;
      if (!ok) atomicOr(w.status, ST_NOT_CONVERGED);
    }
  }
}

// ---------------------------------------------------------------------------------
// k_vectors: one warp per eigenvalue row.  x_j = zeta_j / ((d_j - sigma) - mu) (for a
// pole shift d_i this is Eq. (eigenvecAi), with x_i = -zeta_i / mu), ||x|| with a
// scaled fallback when the plain sum of squares over- or underflows, v = x / ||x||.
// Writes lambda, sigma, mu, ||x|| and row k of V^T (coalesced along j).  For a
// deflated problem the row of reduced eigenvalue k goes to output row rpos[k] and
// component p takes coef[p] * x_{src[p]}; deflated pairs are written by k_defl_rows.
// ---------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_vectors(Ws w, int n_full, double* __restrict__ lambda,
                                                 double* __restrict__ Vt, int64_t ldv, double* __restrict__ sigma_out,
                                                 double* __restrict__ mu_out, double* __restrict__ xnorm_out) {
  const int n = *w.nred;
  if (*w.status & (ST_UNSORTED | ST_NONFINITE)) return;
  const bool defl = (*w.ndefl > 0) || (n != n_full);
  const int lane = threadIdx.x & 31;
  const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const double* __restrict__ d = w.dr;
  const double* __restrict__ z = w.zr;
  for (int k = wid; k < n; k += nw) {
    double s = w.sig[k], m = w.mu[k];
    double mx = 0.0, q = 0.0;
    for (int j = lane; j < n; j += 32) {
      double x = __dmul_rn(z[j], rcp(__dsub_rn(__dsub_rn(d[j], s), m)));
      mx = fmax(mx, fabs(x));
      q = __fma_rn(x, x, q);
    }
    mx = group_max<32>(mx, FULL);
    q = group_sum<32>(q, FULL);
    double scale = 1.0;                  // v_j = x_j * scale / sqrt(q)
    if (!(q < 1e300) || !(mx > 1e-140)) {
      // rescale by the largest component
      scale = 1.0 / mx;
      q = 0.0;
      for (int j = lane; j < n; j += 32) {
        double x = __dmul_rn(z[j], rcp(__dsub_rn(__dsub_rn(d[j], s), m))) * scale;
        q = __fma_rn(x, x, q);
      }
      q = group_sum<32>(q, FULL);
    }
    double nrm = sqrt(q);                // ||x|| * scale
    double c = scale / nrm;
    int row = defl ? w.rpos[k] : k;
    if (lane == 0) {
      double lz = w.lamz[k];
      lambda[row] = isnan(lz) ? __dadd_rn(s, m) : lz;
      if (sigma_out) sigma_out[row] = s;
      if (mu_out) mu_out[row] = m;
      if (xnorm_out) xnorm_out[row] = nrm / scale;
    }
    if (!Vt) continue;
    double* vr = Vt + (int64_t)row * ldv;
    if (!defl) {
      for (int j = lane; j < n; j += 32) vr[j] = __dmul_rn(z[j], rcp(__dsub_rn(__dsub_rn(d[j], s), m))) * c;
    } else {
      for (int p = lane; p < n_full; p += 32) {
        int sj = w.src[p];
        double v = 0.0;
        if (sj >= 0) v = w.coef[p] * (__dmul_rn(z[sj], rcp(__dsub_rn(__dsub_rn(d[sj], s), m))) * c);
        vr[p] = v;
      }
    }
  }
}

// Output positions after deflation: reduced eigenvalue k goes after every deflated
// value above it; deflated position p after every reduced eigenvalue >= d_p.
// lambda_k > d_p is decided exactly from (sigma_k - d_p) + mu_k in double-double.
__device__ __forceinline__ bool lam_greater_equal(double s, double m, double dp) {
  dd t = two_sum(s, -dp);
  dd u = two_sum(t.lo, m);
  dd v = two_sum(t.hi, u.hi);
  double tot = v.hi + (v.lo + u.lo);
  return tot >= 0.0;
}

__global__ void k_defl_positions(Ws w, int n_full, const double* __restrict__ d_full) {
  const int n = *w.nred;
  const int nd = *w.ndefl;
  if (nd == 0 && n == n_full) return;
  int tid = blockIdx.x * blockDim.x + threadIdx.x;
  int stride = gridDim.x * blockDim.x;
  for (int k = tid; k < n; k += stride) {
    // deflated values (non-increasing in dlist order) strictly above lambda_k
    int lo = 0, hi = nd;
    while (lo < hi) {
      int mid = (lo + hi) >> 1;
      double dp = d_full[w.dlist[mid]];
      if (!lam_greater_equal(w.sig[k], w.mu[k], dp)) lo = mid + 1;  // d_p > lambda_k
      else hi = mid;
    }
    w.rpos[k] = k + lo;
  }
  for (int q = tid; q < nd; q += stride) {
    double dp = d_full[w.dlist[q]];
    int lo = 0, hi = n;   // reduced eigenvalues >= d_p (non-increasing in k)
    while (lo < hi) {
      int mid = (lo + hi) >> 1;
      if (lam_greater_equal(w.sig[mid], w.mu[mid], dp)) lo = mid + 1;
      else hi = mid;
    }
    w.dpos[q] = q + lo;
  }
}

// Rows of deflated pairs: e_p for zeta_p == 0; for the t-th non-zero member m_t of a
// tie group (t >= 1) the vector Q^T e_{m_t} of the Givens chain: -zeta_{m_t} zeta_j /
// (r_t r_{t-1}) at the earlier non-zero members j of the group and r_{t-1}/r_t at m_t.
__global__ void k_defl_rows(Ws w, int n_full, const double* __restrict__ d_full, const double* __restrict__ z_full,
                            double* __restrict__ lambda, double* __restrict__ Vt, int64_t ldv,
                            double* __restrict__ sigma_out, double* __restrict__ mu_out,
                            double* __restrict__ xnorm_out) {
  const int nd = *w.ndefl;
  const int lane = threadIdx.x & 31;
  const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int q = wid; q < nd; q += nw) {
    int p = w.dlist[q];
    int row = w.dpos[q];
    double dp = d_full[p];
    if (lane == 0) {
      lambda[row] = dp;
      if (sigma_out) sigma_out[row] = dp;
      if (mu_out) mu_out[row] = 0.0;
      if (xnorm_out) xnorm_out[row] = 0.0;
    }
    if (!Vt) continue;
    double* vr = Vt + (int64_t)row * ldv;
    double zp = z_full[p];
    int g0 = w.gst[p];
    double rc = w.rcur[p], rp = w.rprev[p];
    for (int j = lane; j < n_full; j += 32) {
      double v = 0.0;
      if (zp == 0.0) {
        v = (j == p) ? 1.0 : 0.0;
      } else if (j == p) {
        v = rp / rc;
      } else if (j >= g0 && j < p && z_full[j] != 0.0) {
        v = -(zp / rc) * (z_full[j] / rp);
      }
      vr[j] = v;
    }
  }
}

// rho == 0: lambda = d, V = I, sigma = d, mu = 0.
__global__ void k_trivial(int n, const double* __restrict__ d, double* __restrict__ lambda, double* __restrict__ Vt,
                          int64_t ldv, double* __restrict__ sigma_out, double* __restrict__ mu_out,
                          double* __restrict__ xnorm_out) {
  int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = tid; k < n; k += stride) {
    lambda[k] = d[k];
    if (sigma_out) sigma_out[k] = d[k];
    if (mu_out) mu_out[k] = 0.0;
    if (xnorm_out) xnorm_out[k] = 0.0;
  }
  if (Vt) {
    for (int64_t t = tid; t < (int64_t)n * n; t += stride) {
      int64_t r = t / n, c = t % n;
      Vt[r * ldv + c] = (r == c) ? 1.0 : 0.0;
    }
  }
}

__global__ void k_probe_dfma(int iters, double* sink) {
  int gid = blockIdx.x * blockDim.x + threadIdx.x;
  double a[8];
#pragma unroll
  for (int t = 0; t < 8; t++) a[t] = 1.0 + 1e-3 * (gid & 15) + 1e-4 * t;
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int t = 0; t < 8; t++) a[t] = __fma_rn(a[t], 0.999999, 1e-7);
  }
  double s = 0.0;
#pragma unroll
  for (int t = 0; t < 8; t++) s += a[t];
  sink[gid] = s;
}

__global__ void k_probe_rcp(int64_t count, const double* __restrict__ x, double* __restrict__ out) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x)
    out[t] = rcp(x[t]);
}

// ---------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------
int sm_count() {
  static int cached = 0;
  if (!cached) {
    int dev = 0;
    cudaGetDevice(&dev);
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cached = v > 0 ? v : 1;
  }
  return cached;
}

Options resolve(const dpr1_options* o) {
  Options r;
  dpr1_options def;
  dpr1_default_options(&def);
  const dpr1_options* s = o ? o : &def;
  r.T_Knu = s->T_Knu > 0 ? s->T_Knu : def.T_Knu;
  r.T_zero = s->T_zero > 0 ? s->T_zero : def.T_zero;
  r.lanes = (s->lanes == 8 || s->lanes == 16 || s->lanes == 32) ? s->lanes : 0;
  r.warps = s->warps_per_block > 0 && s->warps_per_block <= 8 ? s->warps_per_block : 8;
  r.bps = s->blocks_per_sm > 0 && s->blocks_per_sm <= 8 ? s->blocks_per_sm : 2;
  r.cap = s->max_bisect >= 64 && s->max_bisect <= 4096 ? s->max_bisect : def.max_bisect;
  r.events = s->phase_events;
  return r;
}

static void record(const Options& o, int t, cudaStream_t st) {
  if (o.events && o.events[t]) cudaEventRecord((cudaEvent_t)o.events[t], st);
}

template <int L>
static void launch_solve_fix(const Ws& w, double rho, const Options& o, int grid, cudaStream_t st) {
  record(o, 0, st);
  k_solve<L><<<grid, 32 * o.warps, 0, st>>>(w, rho, o.cap);
  record(o, 1, st);
  k_classify<<<sm_count() * 4, 256, 0, st>>>(w, o.T_Knu);
  k_fix<L><<<grid, 32 * o.warps, 0, st>>>(w, rho, o.T_Knu, o.cap);
  record(o, 2, st);
}

dpr1_status run_eig(int64_t n64, const double* d, const double* z, double rho, double* lambda, double* Vt,
                    int64_t ldv, double* sigma, double* mu, double* xnorm, void* workspace, size_t wbytes,
                    const dpr1_options* opt, cudaStream_t st) {
  int n = (int)n64;
  Ws w;
  ws_layout(n, &w, (char*)workspace);
  Options o = resolve(opt);
  if (cudaMemsetAsync(w.hdr, 0, sizeof(unsigned) * 64, st) != cudaSuccess) return DPR1_ERR_CUDA;
  int sms = sm_count();
  if (rho == 0.0) {
    k_trivial<<<sms * 4, 256, 0, st>>>(n, d, lambda, Vt, ldv, sigma, mu, xnorm);
    return cudaGetLastError() == cudaSuccess ? DPR1_OK : DPR1_ERR_CUDA;
  }
  int sgrid = (n + 255) / 256;
  if (sgrid > sms * 8) sgrid = sms * 8;
  k_scan<<<sgrid, 256, 0, st>>>(n, d, z, w);
  k_deflate<<<1, 32, 0, st>>>(n, d, z, w);
  int L = o.lanes ? o.lanes : (n <= 256 ? 8 : (n <= 1024 ? 16 : 32));
  int groups_per_block = (32 * o.warps) / L;
  int want_blocks = (n + groups_per_block - 1) / groups_per_block;
  int grid = sms * o.bps;
  if (want_blocks < grid) grid = want_blocks > 0 ? want_blocks : 1;
  if (L == 8) launch_solve_fix<8>(w, rho, o, grid, st);
  else if (L == 16) launch_solve_fix<16>(w, rho, o, grid, st);
  else launch_solve_fix<32>(w, rho, o, grid, st);
  k_zero_detect<<<sgrid, 256, 0, st>>>(w, o.T_zero);
  k_zero_solve<<<1, 128, 0, st>>>(w, rho, o.cap);
  k_defl_positions<<<sms, 256, 0, st>>>(w, n, d);
  int vgrid = (n + 7) / 8;
  if (vgrid > sms * 16) vgrid = sms * 16;
  k_vectors<<<vgrid, 256, 0, st>>>(w, n, lambda, Vt, ldv, sigma, mu, xnorm);
  record(o, 3, st);
  k_defl_rows<<<sms, 256, 0, st>>>(w, n, d, z, lambda, Vt, ldv, sigma, mu, xnorm);
  return cudaGetLastError() == cudaSuccess ? DPR1_OK : DPR1_ERR_CUDA;
}

}  // namespace dpr1

using namespace dpr1;

extern "C" {

void dpr1_default_options(dpr1_options* opt) {
  if (!opt) return;
  opt->T_Knu = 16.0;
  opt->T_zero = 64.0;
  opt->lanes = 0;
  opt->warps_per_block = 0;
  opt->blocks_per_sm = 0;
  opt->max_bisect = 96;
  opt->phase_events = nullptr;
}

const char* dpr1_status_string(dpr1_status s) {
  switch (s) {
    case DPR1_OK: return "ok";
    case DPR1_ERR_ARG: return "invalid argument";
    case DPR1_ERR_UNSORTED: return "d is not sorted non-increasingly";
    case DPR1_ERR_RHO: return "rho must be finite and >= 0";
    case DPR1_ERR_NONFINITE: return "non-finite input";
    case DPR1_ERR_NOT_CONVERGED: return "bisection did not converge within its iteration cap";
    case DPR1_ERR_CUDA: return "CUDA error";
    case DPR1_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
  }
  return "unknown status";
}

size_t dpr1_workspace_size(int64_t n) {
  if (n < 0) return 0;
  return ws_layout(n, nullptr, nullptr);
}

dpr1_status dpr1_eig(int64_t n, const double* d, const double* z, double rho, double* lambda, double* Vt, int64_t ldv,
                     double* sigma, double* mu, double* xnorm, void* workspace, size_t workspace_bytes,
                     const dpr1_options* opt, dpr1_stream_t stream) {
  if (n < 0 || n > (int64_t)0x3fffffff) return DPR1_ERR_ARG;
  if (!std::isfinite(rho) || rho < 0.0) return DPR1_ERR_RHO;
  if (n == 0) return DPR1_OK;
  if (!d || !z || !lambda) return DPR1_ERR_ARG;
  if (Vt && ldv < n) return DPR1_ERR_ARG;
  if (!workspace || ((uintptr_t)workspace & 255) || workspace_bytes < dpr1_workspace_size(n))
    return DPR1_ERR_WORKSPACE;
  return run_eig(n, d, z, rho, lambda, Vt, ldv, sigma, mu, xnorm, workspace, workspace_bytes, opt,
                 (cudaStream_t)stream);
}

dpr1_status dpr1_stream_status(void* workspace, dpr1_stream_t stream) {
  if (!workspace || ((uintptr_t)workspace & 255)) return DPR1_ERR_WORKSPACE;
  unsigned st = 0;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemcpyAsync(&st, workspace, sizeof(unsigned), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return DPR1_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return DPR1_ERR_CUDA;
  if (cudaMemsetAsync(workspace, 0, sizeof(unsigned), s) != cudaSuccess) return DPR1_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return DPR1_ERR_CUDA;
  if (st & ST_NONFINITE) return DPR1_ERR_NONFINITE;
  if (st & ST_UNSORTED) return DPR1_ERR_UNSORTED;
  if (st & ST_NOT_CONVERGED) return DPR1_ERR_NOT_CONVERGED;
  return DPR1_OK;
}

dpr1_status dpr1_workspace_stats(void* workspace, int64_t* out, dpr1_stream_t stream) {
  if (!workspace || ((uintptr_t)workspace & 255) || !out) return DPR1_ERR_ARG;
  unsigned h[64];
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemcpyAsync(h, workspace, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess) return DPR1_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return DPR1_ERR_CUDA;
  const unsigned* c = h + 8;
  out[0] = (int32_t)h[32];
  out[1] = c[C_FIX_N];
  out[2] = c[C_R1];
  out[3] = c[C_R2];
  out[4] = c[C_EVAL_SOLVE];
  out[5] = c[C_EVAL_FIX];
  out[6] = c[C_ZERO_N];
  out[7] = (int32_t)h[33];
  return DPR1_OK;
}

dpr1_status dpr1_probe_dfma(int blocks, int threads, int iters, double* sink, dpr1_stream_t stream) {
  if (blocks <= 0 || threads <= 0 || threads > 1024 || iters <= 0 || !sink) return DPR1_ERR_ARG;
  k_probe_dfma<<<blocks, threads, 0, (cudaStream_t)stream>>>(iters, sink);
  return cudaGetLastError() == cudaSuccess ? DPR1_OK : DPR1_ERR_CUDA;
}

dpr1_status dpr1_probe_reciprocal(int64_t count, const double* x, double* out, dpr1_stream_t stream) {
  if (count < 0 || (count > 0 && (!x || !out))) return DPR1_ERR_ARG;
  if (count == 0) return DPR1_OK;
  int64_t g = (count + 255) / 256;
  if (g > 4096) g = 4096;
  k_probe_rcp<<<(int)g, 256, 0, (cudaStream_t)stream>>>(count, x, out);
  return cudaGetLastError() == cudaSuccess ? DPR1_OK : DPR1_ERR_CUDA;
}

}  // extern "C"
