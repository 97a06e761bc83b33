// dpr1_eig.cu -- eigenpairs of DPR1 matrices A = D + rho z z^T on sm_103a, for one problem
// (dpr1_eig) or a batch of independent problems of uneven sizes (dpr1_eig_batched).
//
// A problem table maps every global element index g to its problem p (offsets into the
// concatenated d, z, lambda, sigma, mu, ||x|| arrays and into the Vt blocks); a single
// problem is the table with one entry.  Launch sequence on the caller's stream
// (Algorithm 1, dpr1eig, for every eigenpair of every problem at once):
//   k_owner     batch only: element -> problem map, offset checks
//   k_norm      exact power-of-two normalisation of each problem (D' = 2^-a D, z' = 2^-b z)
//   k_scan      input checks, scaled copies of d, z, z^2 in the workspace, deflation tests (Sec. 1)
//   k_deflate   exact deflation (zeta_j == 0, ties) for the problems that need it
//   k_solve     per eigenvalue (one lane group): shift test, corner b in double-double,
//               bisection for the extreme eigenvalue nu of the arrowhead inverse; once its
//               queue is empty, the eigenvector rows of the eigenvalues solved by then
//   k_classify  K_nu of Eq. (K0) from the neighbouring eigenvalues; picks R1 / R2 candidates
//   k_fix       R1 (the other pole) and R2 (non-pole shift, f(sigma) in double-double)
//   k_zero_*    eigenvalues much closer to zero than to their poles: lambda from A^{-1}
//   k_vectors   lambda, (sigma, mu), ||x|| (scaled back) and the rows of V^T, v = x / ||x||,
//               that k_solve did not write or whose pair changed since; pairs outside the
//               binary64 range are reported (DPR1_ERR_RANGE)
//   k_defl_*    output rows of deflated problems; k_trivial for rho == 0 (and rho' out of range)
// All work lists are global, so the persistent kernels balance the whole batch.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>

#include "../../include/dpr1.h"
#include "dpr1_device.cuh"
#include "dpr1_internal.cuh"
#include "dpr1_solve.cuh"

// launch shape of the remedies kernel: one block-wide group per flagged eigenvalue
#ifndef DPR1_FIX_THREADS
#define DPR1_FIX_THREADS 256
#endif
#ifndef DPR1_FIX_BLOCKS_PER_SM
#define DPR1_FIX_BLOCKS_PER_SM 2
#endif
// the upper bracket end from the shift test's partial sums (only with the binary64 pass)
#ifndef DPR1_SHIFT_AHI
#define DPR1_SHIFT_AHI 0
#endif
// the solve kernel for problems of mean order above DPR1_SOLVE_LARGE_N: compiled for
// DPR1_SOLVE_MIN_BLOCKS resident blocks per SM with its sums out of line; below, for
// DPR1_SOLVE_SMALL_BLOCKS with its sums inlined (the loops are short there and a call costs)
#ifndef DPR1_SOLVE_LARGE_N
#define DPR1_SOLVE_LARGE_N 2048
#endif
#ifndef DPR1_SOLVE_SMALL_BLOCKS
#define DPR1_SOLVE_SMALL_BLOCKS 2
#endif
// batches of 64 or more problems up to this mean size run the remedies one warp per item
#ifndef DPR1_FIX_WARP_MAX_N
#define DPR1_FIX_WARP_MAX_N 2048
#endif
// and so do fewer problems up to this mean size (each flagged eigenvalue's evaluations are then
// short, and a block-wide group would pay a barrier per evaluation)
#ifndef DPR1_FIX_SMALL_N
#define DPR1_FIX_SMALL_N 1024
#endif
// eigenvector rows as pairs of components with 16-byte accesses
#ifndef DPR1_VEC_PAIRS
#define DPR1_VEC_PAIRS 1
#endif

namespace dpr1 {

constexpr bool kShiftAhi = DPR1_SHIFT_AHI != 0;
constexpr bool kShift32 = DPR1_SHIFT32 != 0 && !kShiftAhi;
constexpr bool kVecPairs = DPR1_VEC_PAIRS != 0;

// ---------------------------------------------------------------------------------
// Workspace layout
// ---------------------------------------------------------------------------------
static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t ws_layout2(int64_t total, int64_t nprob, bool batched, Ws* w, char* base) {
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += align256(bytes);
    return base ? base + o : nullptr;
  };
  size_t nn = (size_t)(total > 0 ? total : 1);
  size_t pp = (size_t)(nprob > 0 ? nprob : 1);
  char* hdr = take(sizeof(unsigned) * 64);
  char* dr = take(sizeof(double) * nn);
  char* zr = take(sizeof(double) * nn);
  char* zz = take(sizeof(double) * nn);
  char* zl = take(sizeof(double) * nn);
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
  char* own = batched ? take(sizeof(int) * nn) : nullptr;
  char* pn = take(sizeof(int) * pp);
  char* pd = take(sizeof(int) * pp);
  char* ps = take(sizeof(unsigned) * pp);
  char* pe = take(sizeof(int) * 2 * pp);
  char* pr = take(sizeof(double) * pp);
  char* pzs = take(sizeof(double) * pp);
  if (w && base) {
    w->hdr = (unsigned*)hdr;
    w->status = (unsigned*)hdr;
    w->counters = (unsigned*)hdr + 8;
    w->counters64 = (unsigned long long*)((unsigned*)hdr + 24);
    w->nred = (int*)pn;
    w->ndefl = (int*)pd;
    w->pst = (unsigned*)ps;
    w->owner = (int*)own;
    w->dr = (double*)dr; w->zr = (double*)zr; w->zz = (double*)zz; w->zl = (double*)zl;
    w->sig = (double*)sig; w->mu = (double*)mu;
    w->shift = (int*)shift; w->flag = (int*)flag; w->list = (int*)list;
    w->lamz = (double*)lamz;
    w->src = (int*)src; w->coef = (double*)coef; w->rpos = (int*)rpos; w->dpos = (int*)dpos;
    w->gst = (int*)gst; w->rprev = (double*)rprev; w->rcur = (double*)rcur; w->dlist = (int*)dlist;
    w->zlist = (int*)zlist;
    w->fixinfo = (double*)fk;
    w->pexp = (int*)pe;
    w->prho = (double*)pr;
    w->pzsum = (double*)pzs;
    w->terms = nullptr;
    w->term_n = 0;
    w->term_slots = 0;
    w->vrow = nullptr;
    w->vstate = nullptr;
  }
  return off;
}

// Lane-group width of k_solve for an average problem order (when the options leave it open).  In a
// batch, eight lanes up to a mean order of 384 (problems of orders 96-384: 33.3 ms against 39.8 with
// 16 lanes and 48.3 with 32 for 425k eigenpairs; orders 16-96: 18.2 against 24.9 and 32.5) and a
// warp above (orders 384-2048: 108.4 ms against 115.8 with 16 lanes and 140.3 with 8).
static int default_lanes(double avg_n, int64_t nprob = 1) {
  if (nprob > 1) return avg_n <= 384 ? 8 : 32;
  return avg_n <= 96 ? 8 : (avg_n <= 384 ? 16 : 32);
}

// Bytes of the stored-element buffers appended to the workspace: TERM_BYTES term_n bytes for
// each lane group of k_solve's default launch (8 warps per block, DPR1_SOLVE_MIN_BLOCKS blocks per
// SM), term_n = n for
// one problem and max(2048, 4 n_avg) (at most total) for a batch; problems of larger order,
// and groups beyond the buffers under other launch options, form the elements per evaluation.
// Bytes of the records of the eigenvector rows the solve kernel's tail writes (after the buffers,
// 256-byte aligned): one problem of order above DPR1_SOLVE_LARGE_N.
static size_t tail_bytes(int64_t total, int64_t nprob) {
  if (!kTailRows || nprob != 1 || total <= DPR1_SOLVE_LARGE_N) return 0;
  return 256 + align256(sizeof(double) * 4 * (size_t)total) + align256(sizeof(unsigned) * (size_t)total);
}

size_t term_bytes(int64_t total, int64_t nprob) {
  if (total <= 0 || nprob <= 0) return 0;
  const double avg = (double)total / (double)nprob;
  const int64_t gpb = (32 * 8) / default_lanes(avg, nprob);
  int64_t groups = (int64_t)sm_count() * DPR1_SOLVE_MIN_BLOCKS * gpb;
  // a launch with blocks of gpb' <= gpb groups has at most total + gpb' - 1 of them
  const int64_t need = total + gpb - 1;
  if (groups > need) groups = need;
  int64_t tn = total;
  if (nprob > 1) {
    const int64_t cap = (int64_t)(4.0 * avg) + 1;
    tn = cap > 2048 ? cap : 2048;
    if (tn > total) tn = total;
  }
  tn = (tn + 31) & ~(int64_t)31;
  return (size_t)groups * TERM_BYTES * (size_t)tn + tail_bytes(total, nprob);
}

size_t ws_layout(int64_t n, Ws* w, char* base) { return ws_layout2(n, 1, false, w, base); }

// ---------------------------------------------------------------------------------
// Problem table
// ---------------------------------------------------------------------------------
struct Prob {
  int P;                    // number of problems
  int64_t total;            // elements of all problems
  const int64_t* offs;      // device [P+1], nullptr: one problem of size total
  const int64_t* voffs;     // device [P+1] element offsets of the Vt blocks (ld = n_p)
  const double* rhos;       // device [P], nullptr: rho0
  double rho0;
  int64_t ldv0;             // leading dimension of Vt for a single problem
  const double* d;
  const double* z;
  double* lambda;
  double* Vt;
  double* sigma;
  double* mu;
  double* xnorm;
};

__device__ __forceinline__ int p_owner(const Prob& pb, const Ws& w, int64_t g) { return pb.offs ? w.owner[g] : 0; }
__device__ __forceinline__ int64_t p_base(const Prob& pb, int p) { return pb.offs ? pb.offs[p] : 0; }
__device__ __forceinline__ int p_size(const Prob& pb, int p) {
  return pb.offs ? (int)(pb.offs[p + 1] - pb.offs[p]) : (int)pb.total;
}
__device__ __forceinline__ double p_rho(const Prob& pb, int p) { return pb.rhos ? pb.rhos[p] : pb.rho0; }
__device__ __forceinline__ int64_t p_vbase(const Prob& pb, int p) { return pb.voffs ? pb.voffs[p] : 0; }
__device__ __forceinline__ int64_t p_ld(const Prob& pb, int p) { return pb.offs ? (int64_t)p_size(pb, p) : pb.ldv0; }

constexpr unsigned ST_FATAL = ST_NONFINITE | ST_UNSORTED | ST_BADARG | ST_RHO;

// ---------------------------------------------------------------------------------
// k_owner (batch): element -> problem map and offset checks (a warp per problem)
// ---------------------------------------------------------------------------------
__global__ void k_owner(Prob pb, Ws w) {
  const int lane = threadIdx.x & 31;
  const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (pb.offs[0] != 0 || pb.offs[pb.P] != pb.total) atomicOr(w.status, ST_BADARG);
  }
  for (int p = wid; p < pb.P; p += nw) {
    int64_t b = pb.offs[p], e = pb.offs[p + 1];
    if (b < 0 || e < b || e > pb.total || e - b > 0x3fffffff) {
      if (lane == 0) atomicOr(w.status, ST_BADARG);
      continue;
    }
    if (pb.voffs && pb.voffs[p] < 0 && lane == 0) atomicOr(w.status, ST_BADARG);
    for (int64_t g = b + lane; g < e; g += 32) w.owner[g] = p;
  }
}

// ---------------------------------------------------------------------------------
// k_norm: exact power-of-two normalisation of each problem (one block per problem).  With
// max|d_j| = m 2^a and max|zeta_j| = m' 2^b (m, m' in [1/2, 1)): D' = 2^-a D, z' = 2^-b z,
// rho' = 2^(2b - a) rho, so A = 2^a (D' + rho' z' z'^T) has the same eigenvectors and
// lambda = 2^a lambda'.  Multiplying by a power of two changes no rounding in the normal range,
// so there the results are those of the unnormalised computation; for data of any magnitude
// it keeps the poles' differences and the weights at their own scale (zeta_j^2 cannot overflow
// or underflow) and leaves the ratio of the rank-one part to D in rho'.  With every pole zero,
// a comes from rho ||z||^2.  rho' outside the normal range marks the problem PT_RANGE.
// ---------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_norm(Prob pb, Ws w) {
  if (*w.status & ST_FATAL) return;
  for (int p = blockIdx.x; p < pb.P; p += gridDim.x) {
    const int64_t base = p_base(pb, p);
    const int n = p_size(pb, p);
    double md = 0.0, mz = 0.0;
    for (int j = threadIdx.x; j < n; j += 256) {
      md = fmax(md, fabs(pb.d[base + j]));
      mz = fmax(mz, fabs(pb.z[base + j]));
    }
    md = group_max<256>(md, FULL);
    mz = group_max<256>(mz, FULL);
    // sum_j |zeta'_j| of the normalised weights (K_z of Eq. (knu2)), in a fixed order
    int ezb = 0;
    if (mz > 0.0 && isfinite(mz)) frexp(mz, &ezb);
    double zs = 0.0;
    for (int j = threadIdx.x; j < n; j += 256) zs = __dadd_rn(zs, fabs(scalbn(pb.z[base + j], -ezb)));
    zs = group_sum<256>(zs, FULL);
    if (threadIdx.x == 0) {
      w.pzsum[p] = zs;
      const double rho = p_rho(pb, p);
      int ed = 0, ez = 0, er = 0;
      if (md > 0.0 && isfinite(md)) frexp(md, &ed);
      if (mz > 0.0 && isfinite(mz)) frexp(mz, &ez);
      if (rho > 0.0 && isfinite(rho)) frexp(rho, &er);
      const int a = (md > 0.0) ? ed : er + 2 * ez;
      w.pexp[2 * p] = a;
      w.pexp[2 * p + 1] = ez;
      const double rs = scalbn(rho, 2 * ez - a);
      w.prho[p] = rs;
      if (rho > 0.0 && isfinite(rho) && mz > 0.0 && isfinite(mz) && isfinite(md) && !(rs >= 0x1p-1022 && isfinite(rs))) {
        atomicOr(&w.pst[p], PT_RANGE | PT_TRIVIAL);
        atomicOr(w.status, ST_RANGE);
      }
    }
  }
}

// ---------------------------------------------------------------------------------
// k_scan: checks and scaled copies (d' = 2^-a d, z' = 2^-b z); one thread per element
// ---------------------------------------------------------------------------------
__global__ void k_scan(Prob pb, Ws w) {
  if (*w.status & ST_FATAL) return;
  unsigned bits = 0;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < pb.total;
       g += (int64_t)gridDim.x * blockDim.x) {
    int p = p_owner(pb, w, g);
    int64_t base = p_base(pb, p);
    int n = p_size(pb, p);
    int64_t j = g - base;
    double dj = pb.d[g], zj = pb.z[g];
    const double djs = scalbn(dj, -w.pexp[2 * p]), zjs = scalbn(zj, -w.pexp[2 * p + 1]);
    unsigned pbits = 0;
    if (j == 0) {
      double r = p_rho(pb, p);
      w.nred[p] = n;
      w.ndefl[p] = 0;
      if (!isfinite(r) || r < 0.0) bits |= ST_RHO;
      if (r == 0.0) pbits |= PT_TRIVIAL;
    }
    if (!isfinite(dj) || !isfinite(zj)) bits |= ST_NONFINITE;
    if (j + 1 < n) {
      double dn = pb.d[g + 1];
      if (dj < dn) bits |= ST_UNSORTED;
      if (dj == dn) pbits |= PT_DEFLATE;
    }
    if (zero_weight(zjs)) pbits |= PT_DEFLATE;
    if (dj == 0.0) pbits |= PT_ZERO_POLE;
    if (pbits) atomicOr(&w.pst[p], pbits);
    w.dr[g] = djs;
    w.zr[g] = zjs;
    const double zq = __dmul_rn(zjs, zjs);
    w.zz[g] = zq;
    w.zl[g] = __fma_rn(zjs, zjs, -zq);
  }
  bits = __reduce_or_sync(FULL, bits);
  if ((threadIdx.x & 31) == 0 && bits) atomicOr(w.status, bits);
}

// ---------------------------------------------------------------------------------
// k_deflate: exact deflation of Sec. 1 for the problems that need it.  Ties: the
// non-zero weights of a group of equal poles are rotated into its first non-zero member
// by a chain of Givens rotations; the survivor keeps zeta = +-||group||, every other
// member becomes an eigenpair (d_group, Q^T e_m).  Writes the reduced problem at the
// problem's offset (dr, zr, zz, nred), for every position its source reduced index src
// (-1: none) and coefficient coef = zeta_q / zeta_survivor, the deflated positions
// (dlist, local indices) and for tie members the prefix norms rprev (before) and rcur
// (including) them.
// ---------------------------------------------------------------------------------
// One group of equal poles, from position j to its end e (serial; lane 0).
__device__ int deflate_group(const Ws& w, int64_t base, const double* d, const double* z, int ea, int eb, int n,
                             int j, int* nr, int* nd) {
  int e = j;
  while (e + 1 < n && d[e + 1] == d[j]) e++;
  int first = -1;
  double r = 0.0;
  for (int q = j; q <= e; q++) {
    w.gst[base + q] = j;
    const double zq = scalbn(z[q], -eb);
    if (zero_weight(zq)) {
      w.src[base + q] = -1; w.coef[base + q] = 0.0; w.rprev[base + q] = 0.0; w.rcur[base + q] = 0.0;
      w.dlist[base + (*nd)++] = q;
      continue;
    }
    double rp = r;
    r = hypot(r, zq);
    w.rprev[base + q] = rp; w.rcur[base + q] = r;
    if (first < 0) first = q;
    else w.dlist[base + (*nd)++] = q;
  }
  if (first >= 0) {
    double zs = (z[first] > 0.0) ? r : -r;
    for (int q = j; q <= e; q++) {
      const double zq = scalbn(z[q], -eb);
      if (zero_weight(zq)) continue;
      w.src[base + q] = *nr;
      w.coef[base + q] = zq / zs;
    }
    w.dr[base + *nr] = scalbn(d[j], -ea);
    w.zr[base + *nr] = zs;
    const double zq = __dmul_rn(zs, zs);
    w.zz[base + *nr] = zq;
    w.zl[base + *nr] = __fma_rn(zs, zs, -zq);
    (*nr)++;
  }
  return e + 1;
}

// One warp per problem: chunks of 32 positions.  A chunk in which no pole equals a
// neighbour holds only single-member groups (a survivor with coef 1, or a zero weight),
// placed with ballot prefix counts; a chunk that a group of equal poles touches is done
// serially by lane 0, group by group, to the end of the last group it starts.  The
// outputs are those of the serial scan (same order of survivors and deflated positions).
__global__ void k_deflate(Prob pb, Ws w) {
  if (*w.status & ST_FATAL) return;
  const int lane = threadIdx.x & 31;
  const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int p = wid; p < pb.P; p += nw) {
    unsigned ps = w.pst[p];
    if (!(ps & PT_DEFLATE) || (ps & PT_TRIVIAL)) continue;
    const int64_t base = p_base(pb, p);
    const int n = p_size(pb, p);
    const double* d = pb.d + base;
    const double* z = pb.z + base;
    const int ea = w.pexp[2 * p], eb = w.pexp[2 * p + 1];
    int nr = 0, nd = 0, q0 = 0;
    while (q0 < n) {
      const int q = q0 + lane;
      const bool in = q < n;
      const double dq = in ? d[q] : 0.0, zq = in ? scalbn(z[q], -eb) : 0.0;
      const bool tie = in && ((q > 0 && d[q - 1] == dq) || (q + 1 < n && d[q + 1] == dq));
      if (__ballot_sync(FULL, tie) == 0u) {
        const bool zw = in && zero_weight(zq);
        const bool keep = in && !zw;
        const unsigned km = __ballot_sync(FULL, keep), dm = __ballot_sync(FULL, zw);
        const unsigned below = (1u << lane) - 1u;
        if (in) {
          w.gst[base + q] = q;
          if (zw) {
            w.src[base + q] = -1; w.coef[base + q] = 0.0; w.rprev[base + q] = 0.0; w.rcur[base + q] = 0.0;
            w.dlist[base + nd + __popc(dm & below)] = q;
          } else {
            const int r = nr + __popc(km & below);
            w.src[base + q] = r;
            w.coef[base + q] = 1.0;                       // zeta_q / zeta_q
            w.rprev[base + q] = 0.0;
            w.rcur[base + q] = fabs(zq);                  // hypot(0, zeta_q)
            w.dr[base + r] = scalbn(dq, -ea);
            w.zr[base + r] = zq;
            const double zz = __dmul_rn(zq, zq);
            w.zz[base + r] = zz;
            w.zl[base + r] = __fma_rn(zq, zq, -zz);
          }
        }
        nr += __popc(km);
        nd += __popc(dm);
        q0 += 32;
      } else {
        int j = q0;
        if (lane == 0) {
          while (j < q0 + 32 && j < n) j = deflate_group(w, base, d, z, ea, eb, n, j, &nr, &nd);
        }
        __syncwarp();
        nr = __shfl_sync(FULL, nr, 0);
        nd = __shfl_sync(FULL, nd, 0);
        q0 = __shfl_sync(FULL, j, 0);
      }
    }
    if (lane == 0) {
      w.nred[p] = nr;
      w.ndefl[p] = nd;
      atomicAdd(&w.counters[C_DEFL], (unsigned)nd);
    }
  }
}

// ---------------------------------------------------------------------------------
// k_solve: one lane group of L threads per eigenvalue; groups take global eigenvalue
// indices from a counter (persistent grid) and skip deflated slots.  A group with a buffer in
// the workspace stores the elements of the inverse there in the corner pass and evaluates the
// secular function from them (stored_sum, stored_sum_d).
//
// Shift test (Algorithm 1): tau = (d_{k-1} - d_k)/2 and
//   F = 1 + rho sum_j zeta_j^2 / ((d_j - d_k) - tau);  F > 0 -> sigma = d_k, else d_{k-1}.
// The same pass gives brackets for nu (from f(d_i + mu) = 0 and the sign of F):
//   sigma = d_k:     mu in (0, tau]   -> 1/tau <= nu <= (1 + rho P) / (rho zeta_k^2),
//                    P = sum_{j<k} zeta_j^2 / ((d_j - d_k) - tau)   (the positive terms of F)
//   sigma = d_{k-1}: mu in [-tau, 0)  -> 1/tau <= |nu| <= (-1 - rho N) / (rho zeta_{k-1}^2),
//                    N = sum_{j>=k} zeta_j^2 / ((d_j - d_k) - tau)  (the negative terms of F)
//   k = 1:           mu in [rho zeta_1^2, rho ||z||^2] -> nu in [1/(rho ||z||^2), 1/(rho zeta_1^2)]
// (solve_pole checks the near end, so a wrong sign of a rounded F costs steps, not accuracy).
// ---------------------------------------------------------------------------------
// ---------------------------------------------------------------------------------
// One eigenvector row by a warp (Eq. (eigenvecAi)): x_j = zeta_j / ((d_j - sigma) - mu) (for a
// pole shift d_i, x_i = -zeta_i / mu), ||x|| with a scaled fallback when the plain sum of squares
// over- or underflows.  With vr the row v = x / ||x|| is written there: the first pass stores
// x_j as it forms them (pairs of components from a 16-byte aligned position, lane 0 taking an
// unaligned first and an unpaired last one) and the second rescales them in place.  Returns
// *nrm = ||x|| scale and *scale (v_j = x_j scale / *nrm).
// ---------------------------------------------------------------------------------
__device__ __forceinline__ void row_values(const double* __restrict__ d, const double* __restrict__ z, int n,
                                           double s, double m, double* __restrict__ vr, int lane, double* nrm_out,
                                           double* scale_out) {
  const bool store = vr != nullptr;
  double q = 0.0;
  bool bad = false;
  const int j0 = (store && kVecPairs && (((uintptr_t)vr) & 15)) ? 1 : 0;
  const int npair = (store && kVecPairs) ? (n - j0) >> 1 : 0;
  const int jtail = j0 + 2 * npair;
  if (store && kVecPairs) {
    for (int t = lane; t < npair; t += 32) {
      const int j = j0 + 2 * t;
      const double den0 = __dsub_rn(__dsub_rn(d[j], s), m), den1 = __dsub_rn(__dsub_rn(d[j + 1], s), m);
      double2 x;
      x.x = __dmul_rn(z[j], rcp_nr(den0));
      x.y = __dmul_rn(z[j + 1], rcp_nr(den1));
      bad |= !rcp_in_range(den0) || !rcp_in_range(den1);
      *reinterpret_cast<double2*>(vr + j) = x;
      q = __fma_rn(x.x, x.x, q);
      q = __fma_rn(x.y, x.y, q);
    }
    if (lane == 0) {
      // the unaligned first component (j0 = 1) and the unpaired last one (jtail = n - 1)
      for (int e = 0; e < 2; e++) {
        const int j = e == 0 ? (j0 ? 0 : -1) : (jtail < n ? jtail : -1);
        if (j < 0) continue;
        const double den = __dsub_rn(__dsub_rn(d[j], s), m);
        const double x = __dmul_rn(z[j], rcp_nr(den));
        bad |= !rcp_in_range(den);
        vr[j] = x;
        q = __fma_rn(x, x, q);
      }
    }
  } else {
    for (int j = lane; j < n; j += 32) {
      const double den = __dsub_rn(__dsub_rn(d[j], s), m);
      const double x = __dmul_rn(z[j], rcp_nr(den));
      bad |= !rcp_in_range(den);
      if (store) vr[j] = x;
      q = __fma_rn(x, x, q);
    }
  }
  q = group_sum<32>(q, FULL);
  bad = group_any<32>(bad, FULL);
  double scale = 1.0;                  // v_j = x_j * scale / sqrt(q)
  bool rewrite = false;                // the stored x_j are not usable: write v_j from scratch
  if (bad || !(q < 1e300) || !(q > 1e-280)) {
    double mx = 0.0;
    for (int j = lane; j < n; j += 32) mx = fmax(mx, fabs(__dmul_rn(z[j], rcp(__dsub_rn(__dsub_rn(d[j], s), m)))));
    mx = group_max<32>(mx, FULL);
    scale = 1.0 / mx;
    q = 0.0;
    for (int j = lane; j < n; j += 32) {
      double x = __dmul_rn(z[j], rcp(__dsub_rn(__dsub_rn(d[j], s), m))) * scale;
      q = __fma_rn(x, x, q);
    }
    q = group_sum<32>(q, FULL);
    rewrite = true;
  }
  const double nrm = sqrt(q);          // ||x|| * scale
  const double c = scale / nrm;
  *nrm_out = nrm;
  *scale_out = scale;
  if (!store) return;
  if (!rewrite && kVecPairs) {
    for (int t = lane; t < npair; t += 32) {
      const int j = j0 + 2 * t;
      double2 x = *reinterpret_cast<const double2*>(vr + j);
      x.x = __dmul_rn(x.x, c);
      x.y = __dmul_rn(x.y, c);
      *reinterpret_cast<double2*>(vr + j) = x;
    }
    if (lane == 0) {
      if (j0) vr[0] = __dmul_rn(vr[0], c);
      if (jtail < n) vr[n - 1] = __dmul_rn(vr[n - 1], c);
    }
  } else if (!rewrite) {
    for (int j = lane; j < n; j += 32) vr[j] = __dmul_rn(vr[j], c);
  } else {
    for (int j = lane; j < n; j += 32) vr[j] = __dmul_rn(z[j], rcp(__dsub_rn(__dsub_rn(d[j], s), m))) * c;
  }
}

// A row written by the solve kernel's tail, out of line (the solve loop keeps its registers),
// and its record: the pair it was formed from, ||x|| scale and the scale.
__device__ __noinline__ void tail_row(const double* __restrict__ d, const double* __restrict__ z, int n, double s,
                                      double m, double* __restrict__ vr, int lane, double* __restrict__ rec) {
  double nrm, scale;
  row_values(d, z, n, s, m, vr, lane, &nrm, &scale);
  if (lane == 0) {
    rec[0] = s;
    rec[1] = m;
    rec[2] = nrm;
    rec[3] = scale;
  }
}

template <int L, int MINB, bool NI>
__global__ void __launch_bounds__(256, MINB)
    k_solve(Prob pb, Ws w, int cap, bool fast, int dd_mode, double T_kappa, bool screen) {
  if (*w.status & ST_FATAL) return;
  const int lane = threadIdx.x & (L - 1);
  const unsigned gm = group_mask<L>();
  const int leader = (threadIdx.x & 31) & ~(L - 1);
  const int64_t grp = (int64_t)blockIdx.x * (blockDim.x / L) + threadIdx.x / L;
  double* const Dbuf = (w.terms && grp < w.term_slots) ? w.terms + 4 * grp * w.term_n : nullptr;
  for (;;) {
    long long gl = 0;
    if (lane == 0) gl = (long long)atomicAdd(&w.counters64[0], 1ull);
    gl = __shfl_sync(gm, gl, leader, 32);
    if (gl >= pb.total) {
      if constexpr (kTailRows && L == 32 && NI) {
        // the queue is empty: write the eigenvector rows of the eigenvalues solved so far (one
        // problem without deflation), sweeping all rows once in order.  A row whose eigenvalue is
        // still being solved is left to k_vectors (writing it here would lengthen the kernel's
        // last, slowest solves), and so is one whose pair a later kernel changes.  Bisection
        // only: the accelerated solve's eigenvalues take even times and leave no idle tail.
        if (!fast && w.vstate && pb.P == 1 && pb.Vt && w.nred[0] == pb.total) {
          const int n = (int)pb.total;
          for (;;) {
            // lane 0 claims the next row and, once its acquire load sees the pair written, reads
            // the pair and passes it to the other lanes
            unsigned r = 0, st = 0;
            double sr = 0.0, mr = 0.0;
            if (lane == 0) {
              r = atomicAdd(&w.counters[C_TROW], 1u);
              if (r < (unsigned)n) st = ld_acquire(w.vstate + r);
              if (st == 1u) {
                sr = w.sig[r];
                mr = w.mu[r];
              }
            }
            r = __shfl_sync(gm, r, 0, 32);
            st = __shfl_sync(gm, st, 0, 32);
            if (r >= (unsigned)n) break;
            if (st != 1u) continue;
            sr = __shfl_sync(gm, sr, 0, 32);
            mr = __shfl_sync(gm, mr, 0, 32);
            tail_row(w.dr, w.zr, n, sr, mr, pb.Vt + (int64_t)r * pb.ldv0, lane, w.vrow + 4 * (int64_t)r);
            if (lane == 0) {
              w.vstate[r] = 2u;
              atomicAdd(&w.counters[C_TAILROWS], 1u);
            }
          }
        }
      }
      break;
    }
    const int64_t g = gl;
    const int p = p_owner(pb, w, g);
    if (w.pst[p] & PT_TRIVIAL) continue;
    const int64_t base = p_base(pb, p);
    const int n = w.nred[p];
    const int k = (int)(g - base);
    if (k >= n) continue;
    const double rho = w.prho[p];   // rho' of the normalised problem
    const double* __restrict__ d = w.dr + base;
    const double* __restrict__ zl = w.zl + base;
    const double* __restrict__ zz = w.zz + base;
    int i;
    double alo, ahi;
    bool shift32 = false;
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
      double sp = 0.0, sn = 0.0, F = 0.0, EF = 0.0;
      // the binary32 pass decides where its bound settles the sign (the binary64 pass's sign)
      const bool f32 = kShift32 && screen && shift_test_f32<L>(d, zz, n, dk, tau, rho, lane, gm, &F, &EF) &&
                       fabs(F) > EF;
      shift32 = f32;
      if (!f32) {
        for (int j = lane; j < n; j += L) {
          double den = __dsub_rn(__dsub_rn(d[j], dk), tau);
          double t = __dmul_rn(zz[j], rcp(den));
          if (j < k) sp = __dadd_rn(sp, t);
          else sn = __dadd_rn(sn, t);
        }
        sp = group_sum<L>(sp, gm);
        sn = group_sum<L>(sn, gm);
        F = 1.0 + rho * (sp + sn);
      }
      alo = 1.0 / tau;
      ahi = INFINITY;
      if (F > 0.0) {
        i = k;
        if (kShiftAhi) ahi = (1.0 + rho * sp) / (rho * zz[k]);
      } else {
        i = k - 1;
        if (kShiftAhi) ahi = (-1.0 - rho * sn) / (rho * zz[k - 1]);
      }
    }
    const bool stored = Dbuf && n <= w.term_n;
    PoleResult pr = solve_pole<L, NI>(d, zl, zz, n, rho, k, i, alo, ahi, cap, fast, lane, gm,
                                  CornerRule{dd_mode, T_kappa, w.pzsum[p]}, stored ? Dbuf : nullptr,
                                  stored ? Dbuf + n : nullptr, screen);
    if (lane == 0) {
      if (pr.dd) atomicAdd(&w.counters[C_DD], 1u);
      if (pr.screened) atomicAdd(&w.counters[C_SCREEN], (unsigned)pr.screened);
      if (pr.screened_near) atomicAdd(&w.counters[C_SCREEN_NEAR], (unsigned)pr.screened_near);
      if (pr.screened_df) atomicAdd(&w.counters[C_SCREEN_DF], (unsigned)pr.screened_df);
      if (pr.inferred) atomicAdd(&w.counters[C_INFER], (unsigned)pr.inferred);
      if (pr.probes) atomicAdd(&w.counters[C_PROBE], (unsigned)pr.probes);
      if (shift32) atomicAdd(&w.counters[C_SHIFT32], 1u);
      w.sig[g] = d[i];
      w.mu[g] = pr.mu;
      w.shift[g] = i;
      w.flag[g] = 0;
      atomicAdd(&w.counters[C_EVAL_SOLVE], (unsigned)pr.steps);
      atomicAdd(&w.counters[C_SOLVED], 1u);
      if (!pr.ok) atomicOr(w.status, ST_NOT_CONVERGED);
      if (w.vstate) st_release(w.vstate + g, 1u);     // (sigma, mu) written: the row may be formed
    }
  }
}

// ---------------------------------------------------------------------------------
// k_classify: K_nu = ||A_i^{-1}||_2 / |nu| (Eq. (K0)).  ||A_i^{-1}||_2 is the reciprocal
// distance from d_i to the spectrum; the eigenvalues next to pole d_i are lambda_i
// (above) and lambda_{i+1} (below), one of which is lambda_k, so
//   K_nu = max(1, |mu_k| / |lambda_m - d_i|),  lambda_m the other neighbour of d_i.
// For K_nu > T_Knu the eigenvalue goes to k_fix with the candidate other pole o,
//   K'  = max(1, |lambda_k - d_o| / |lambda_m' - d_o|)   (m' the other neighbour of d_o),
//   ratio = |lambda_k - d_o| / |lambda_k - d_i|,
// captured here because k_fix overwrites pairs.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ double dist_to(const Ws& w, int64_t m, double p) {
  return fabs(__dadd_rn(__dsub_rn(w.sig[m], p), w.mu[m]));
}

__global__ void k_classify(Prob pb, Ws w, double T_Knu) {
  if (*w.status & ST_FATAL) return;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < pb.total;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int p = p_owner(pb, w, g);
    if (w.pst[p] & PT_TRIVIAL) continue;
    const int64_t base = p_base(pb, p);
    const int n = w.nred[p];
    const int k = (int)(g - base);
    if (k >= n) continue;
    const double* d = w.dr + base;
    int i = w.shift[g];
    double di = d[i];
    double mu = w.mu[g];
    double mk = fabs(mu);
    int m = (i == k) ? k + 1 : k - 1;
    double K = 1.0;
    if (m >= 0 && m < n) K = fmax(1.0, mk / dist_to(w, base + m, di));
    // a pole solve that left the binary64 range (mu zero or not finite) is no solution
    if (!(mk > 0.0) || !isfinite(mk) || isnan(K)) K = INFINITY;
    if (K > T_Knu) {
      int o = (i == k) ? k - 1 : k;
      double K2 = INFINITY, ratio = INFINITY;
      if (o >= 0 && o < n && o != i) {
        double dko = fabs(__dadd_rn(__dsub_rn(di, d[o]), mu));
        int m2 = (o == k) ? k + 1 : k - 1;
        K2 = 1.0;
        if (m2 >= 0 && m2 < n) K2 = fmax(1.0, dko / dist_to(w, base + m2, d[o]));
        ratio = dko / mk;
      }
      unsigned slot = atomicAdd(&w.counters[C_FIX_N], 1u);
      w.list[slot] = (int)g;
      w.fixinfo[3 * (size_t)slot] = K;
      w.fixinfo[3 * (size_t)slot + 1] = K2;
      w.fixinfo[3 * (size_t)slot + 2] = ratio;
      w.flag[g] = 1;
    }
  }
}

// After a non-pole shift: the difference d_p - lambda = (d_p - sigma) - mu to a neighbouring
// pole p cancels by more than a factor 16 (lambda lies much nearer to the pole than sigma).
__device__ __forceinline__ bool pole_difference_cancels(double dp, double s, double m) {
  const double t = __dsub_rn(__dsub_rn(dp, s), m);
  return 16.0 * fabs(t) < __dadd_rn(fabs(__dsub_rn(dp, s)), fabs(m));
}

// ---------------------------------------------------------------------------------
// k_fix: remedies for the flagged eigenvalues, one lane group each.
//  (R1) solve at the other neighbouring pole o when K' < K, K' <= T_Knu and ratio <= T_Knu
//       (beyond that ratio the eigenvector formula at d_o cancels); K' and the ratio come
//       from k_classify, so the solve runs only when it is taken.
//  (R2) otherwise shift to sigma = fl(lambda) of the first pole solution, moved into the
//       interlacing interval of lambda_k ((d_k, d_{k-1}); (d_0, d_0 + rho ||z||^2] for k = 0),
//       and solve_nonpole.  Any sigma there yields lambda_k (the sign of f(sigma) picks the
//       side), accurately once lambda_k is the eigenvalue nearest to sigma; when |mu| is not
//       below half the distance to the nearer pole end, the next shift is the midpoint (the
//       Weyl bound for k = 0) and then the lambda found there (at most 3 solves: a first
//       estimate with K_nu near 1/eps is noise).  When no binary64 number lies between
//       lambda_k and a neighbouring pole, the shift is formed in double the working precision
//       (at most 3 more solves).
// A group with one of k_solve's buffers bisects from stored elements there, as k_solve does.
// ---------------------------------------------------------------------------------
template <int L, bool NI>
__global__ void __launch_bounds__(L > 256 ? L : 256) k_fix(Prob pb, Ws w, double T_Knu, int cap, bool fast,
                                                           int dd_mode, double T_kappa, bool screen) {
  if (*w.status & ST_FATAL) return;
  const int nfix = (int)w.counters[C_FIX_N];
  const int lane = threadIdx.x & (L - 1);
  const unsigned gm = group_mask<L>();
  const int leader = (threadIdx.x & 31) & ~(L - 1);
  // k_solve has finished: its lane-group buffers are free for the remedies' solves
  const int64_t grp = (int64_t)blockIdx.x * (blockDim.x / L) + threadIdx.x / L;
  double* const Dbuf = (w.terms && grp < w.term_slots) ? w.terms + 4 * grp * w.term_n : nullptr;
  __shared__ int item;
  for (;;) {
    int t = 0;
    if constexpr (L > 32) {
      if (threadIdx.x == 0) item = (int)atomicAdd(&w.counters[C_FIX_Q], 1u);
      __syncthreads();
      t = item;
      __syncthreads();
    } else {
      if (lane == 0) t = (int)atomicAdd(&w.counters[C_FIX_Q], 1u);
      t = __shfl_sync(gm, t, leader, 32);
    }
    if (t >= nfix) break;
    const int64_t g = w.list[t];
    const int p = p_owner(pb, w, g);
    const int64_t base = p_base(pb, p);
    const int n = w.nred[p];
    const int k = (int)(g - base);
    const double rho = w.prho[p];   // rho' of the normalised problem
    const double* __restrict__ d = w.dr + base;
    const double* __restrict__ zl = w.zl + base;
    const double* __restrict__ zz = w.zz + base;
    int i = w.shift[g];
    double di = d[i];
    double mu = w.mu[g];
    const double K = w.fixinfo[3 * (size_t)t];
    const double K2 = w.fixinfo[3 * (size_t)t + 1];
    const double ratio = w.fixinfo[3 * (size_t)t + 2];
    double new_sig = di, new_mu = mu;
    int new_shift = i;
    bool done = false;
    int o = (i == k) ? k - 1 : k;
    double* const Ds = (Dbuf && n <= w.term_n) ? Dbuf : nullptr;
    double* const us = Ds ? Dbuf + n : nullptr;
    // R1 is solved only when it will be taken (K' and the ratio come from k_classify); R2 starts
    // from the first estimate otherwise, and its clamp and safe second shift cover a poor one
    if (o >= 0 && o < n && o != i && K2 < K && K2 <= T_Knu && ratio <= T_Knu) {
      PoleResult pr = solve_pole<L, NI>(d, zl, zz, n, rho, k, o, 0.0, INFINITY, cap, fast, lane, gm,
                                    CornerRule{dd_mode, T_kappa, w.pzsum[p]}, Ds, us, screen);
      if (!pr.ok && lane == 0) atomicOr(w.status, ST_NOT_CONVERGED);
      if (lane == 0) atomicAdd(&w.counters[C_EVAL_FIX], (unsigned)pr.steps);
      if (lane == 0 && pr.screened) atomicAdd(&w.counters[C_SCREEN], (unsigned)pr.screened);
      if (lane == 0 && pr.screened_near) atomicAdd(&w.counters[C_SCREEN_NEAR], (unsigned)pr.screened_near);
      if (lane == 0 && pr.screened_df) atomicAdd(&w.counters[C_SCREEN_DF], (unsigned)pr.screened_df);
      if (lane == 0 && pr.inferred) atomicAdd(&w.counters[C_INFER], (unsigned)pr.inferred);
      if (lane == 0 && pr.probes) atomicAdd(&w.counters[C_PROBE], (unsigned)pr.probes);
      new_sig = d[o]; new_mu = pr.mu; new_shift = o; done = true;
    }
    if (!done) {
      // the interlacing interval of lambda_k, (d_k, d_{k-1}), or (d_0, d_0 + rho ||z||^2] (Weyl)
      const double lo = d[k];
      double hi;
      if (k > 0) {
        hi = d[k - 1];
      } else {
        double zs = 0.0;
        for (int j = lane; j < n; j += L) zs = __dadd_rn(zs, zz[j]);
        hi = __fma_rn(rho, group_sum<L>(zs, gm), d[0]);
      }
      double s = __dadd_rn(di, mu);                     // the first solution's lambda
      bool solved = false;
      for (int round = 0; round < 3; round++) {
        if (!(s > lo)) s = dnext_up(lo);
        if (k > 0 && s >= hi) s = dnext_down(hi);
        if (k == 0 && s > hi) s = hi;
        if (!(s > lo) || (k > 0 && !(s < hi))) break;
        bool ok;
        int st2 = 0;
        const double m2 =
            solve_nonpole<L, false, NI>(d, zl, zz, n, rho, s, k > 0 ? k - 1 : -1, k, cap, fast, lane, gm, &ok, &st2, Ds, us);
        if (!ok && lane == 0) atomicOr(w.status, ST_NOT_CONVERGED);
        if (lane == 0) atomicAdd(&w.counters[C_EVAL_FIX], (unsigned)st2);
        new_sig = s; new_mu = m2; new_shift = -1; solved = true;
        // accurate when lambda_k is the eigenvalue nearest to sigma: every other eigenvalue lies
        // beyond the interval's poles.  Otherwise the next shift is one from which lambda_k is at
        // least as near as any other eigenvalue -- the midpoint of (d_k, d_{k-1}), or for k = 0
        // the Weyl bound -- and the one after is the lambda found there
        const double room = (k > 0) ? fmin(s - lo, hi - s) : s - lo;
        if (fabs(m2) < 0.5 * room) break;
        s = (round == 0) ? (k > 0 ? __fma_rn(0.5, __dsub_rn(hi, lo), lo) : hi) : __dadd_rn(s, m2);
      }
      // no binary64 number between lambda_k and a neighbouring pole: the interval holds none, or
      // the result's difference to a pole cancels.  Then (Sec. 2, remedy R2) the shift and its
      // DPR1 matrix are formed in double the working precision: sigma = d_k + t, an unevaluated
      // pair with t in (0, g), g = d_{k-1} - d_k (or up to the Weyl bound for k = 0), the rounds
      // as above from the estimate; lambda - d_k = t + mu is returned against the nearer pole.
      if (!solved || pole_difference_cancels(lo, new_sig, new_mu) ||
          (k > 0 && pole_difference_cancels(hi, new_sig, new_mu))) {
        const dd g = (k > 0) ? two_sum(hi, -lo) : dd{__dsub_rn(hi, lo), 0.0};
        const double gw = __dadd_rn(g.hi, g.lo);
        const double mid = (k > 0) ? 0.5 * gw : gw;
        const dd te = dd_add(two_sum(new_sig, -lo), {new_mu, 0.0});
        double t = __dadd_rn(te.hi, te.lo), m2 = 0.0;
        for (int round = 0; round < 3; round++) {
          if (!(t > 0.0) || (k > 0 && !(t < gw)) || (k == 0 && t > gw)) t = mid;
          bool ok;
          int st2 = 0;
          m2 = solve_nonpole<L, true, NI>(d, zl, zz, n, rho, lo, k > 0 ? k - 1 : -1, k, cap, fast, lane, gm, &ok, &st2,
                                      Ds, us, t);
          if (!ok && lane == 0) atomicOr(w.status, ST_NOT_CONVERGED);
          if (lane == 0) atomicAdd(&w.counters[C_EVAL_FIX], (unsigned)st2);
          const double room = (k > 0) ? fmin(t, gw - t) : t;
          if (fabs(m2) < 0.5 * room) break;
          t = (round == 0) ? mid : __dadd_rn(t, m2);
        }
        const dd lm = two_sum(t, m2);                   // lambda - d_k
        if (k > 0 && lm.hi > 0.5 * gw) {
          const dd up = dd_add(lm, {-g.hi, -g.lo});     // lambda - d_{k-1}
          new_sig = hi;
          new_mu = __dadd_rn(up.hi, up.lo);
        } else {
          new_sig = lo;
          new_mu = __dadd_rn(lm.hi, lm.lo);
        }
        new_shift = -1;
        if (lane == 0) atomicAdd(&w.counters[C_R2DD], 1u);
      }
    }
    if (lane == 0) {
      w.sig[g] = new_sig;
      w.mu[g] = new_mu;
      w.shift[g] = new_shift;
      if (new_shift == -1) atomicAdd(&w.counters[C_R2], 1u);
      else if (new_shift != i) atomicAdd(&w.counters[C_R1], 1u);
      w.flag[g] = (new_shift == -1) ? 2 : (new_shift != i ? 1 : 0);
    }
  }
}

// ---------------------------------------------------------------------------------
// Eigenvalues much closer to zero than to their neighbouring poles,
// T_zero |lambda| < min(|lambda - d_k|, |lambda - d_{k-1}|), when no pole of the problem
// is zero: lambda = 1/nu, nu the extreme eigenvalue of A^{-1} = D^{-1} + gamma D^{-1} z z^T D^{-1}
// (Eq. (gamma)) -- the non-pole solve with sigma = 0.  k_zero_detect marks candidates
// (the paper notes there is at most one per problem); k_zero_solve handles them one warp
// each.  lamz[g] = NaN means "not recomputed".
// ---------------------------------------------------------------------------------
__global__ void k_zero_detect(Prob pb, Ws w, double T_zero) {
  if (*w.status & ST_FATAL) return;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < pb.total;
       g += (int64_t)gridDim.x * blockDim.x) {
    w.lamz[g] = __longlong_as_double(0x7ff8000000000000ll);
    const int p = p_owner(pb, w, g);
    const unsigned ps = w.pst[p];
    if (ps & (PT_TRIVIAL | PT_ZERO_POLE)) continue;
    const int64_t base = p_base(pb, p);
    const int k = (int)(g - base);
    if (k >= w.nred[p]) continue;
    double s = w.sig[g], m = w.mu[g];
    double lam = __dadd_rn(s, m);
    double m1 = fabs(__dadd_rn(__dsub_rn(s, w.dr[base + k]), m));
    if (k > 0) m1 = fmin(m1, fabs(__dadd_rn(__dsub_rn(s, w.dr[base + k - 1]), m)));
    if (T_zero * fabs(lam) < m1) {
      unsigned slot = atomicAdd(&w.counters[C_ZERO_N], 1u);
      w.zlist[slot] = (int)g;
    }
  }
}

__global__ void k_zero_solve(Prob pb, Ws w, int cap, bool fast) {
  if (*w.status & ST_FATAL) return;
  const int nz = (int)w.counters[C_ZERO_N];
  const int lane = threadIdx.x & 31;
  const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int t = wid; t < nz; t += nw) {
    const int64_t g = w.zlist[t];
    const int p = p_owner(pb, w, g);
    const int64_t base = p_base(pb, p);
    const int n = w.nred[p];
    const double* d = w.dr + base;
    // poles next to 0: the first negative pole and the one before it (no pole is zero here)
    int lo = 0, hi = n;
    while (lo < hi) {
      int mid = (lo + hi) >> 1;
      if (d[mid] > 0.0) lo = mid + 1;
      else hi = mid;
    }
    const int below = lo < n ? lo : -1;
    const int above = lo - 1;
    bool ok;
    double lam0 = solve_nonpole<32>(d, w.zl + base, w.zz + base, n, w.prho[p], 0.0, above, below, cap, fast, lane,
                                    FULL, &ok);
    if (lane == 0) {
      w.lamz[g] = lam0;
      if (!ok) atomicOr(w.status, ST_NOT_CONVERGED);
    }
  }
}

// ---------------------------------------------------------------------------------
// Output positions in deflated problems: reduced eigenvalue k goes after every deflated
// value above it; deflated position q after every reduced eigenvalue >= d_q.
// lambda_k >= d_q is decided exactly from (sigma_k - d_q) + mu_k in double-double.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ bool lam_greater_equal(double s, double m, double dq) {
  dd t = two_sum(s, -dq);
  dd u = two_sum(t.lo, m);
  dd v = two_sum(t.hi, u.hi);
  double tot = v.hi + (v.lo + u.lo);
  return tot >= 0.0;
}

__global__ void k_defl_positions(Prob pb, Ws w) {
  if (*w.status & ST_FATAL) return;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < pb.total;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int p = p_owner(pb, w, g);
    const int nd = w.ndefl[p];
    if (nd == 0 || (w.pst[p] & PT_TRIVIAL)) continue;
    const int64_t base = p_base(pb, p);
    const int n = w.nred[p];
    const int k = (int)(g - base);
    const double* dfull = pb.d + base;
    const int ea = w.pexp[2 * p];                       // (sigma, mu) are in normalised units
    if (k < n) {
      int lo = 0, hi = nd;   // deflated values strictly above lambda_k
      while (lo < hi) {
        int mid = (lo + hi) >> 1;
        double dq = scalbn(dfull[w.dlist[base + mid]], -ea);
        if (!lam_greater_equal(w.sig[base + k], w.mu[base + k], dq)) lo = mid + 1;
        else hi = mid;
      }
      w.rpos[g] = k + lo;
    }
    if (k < nd) {
      double dq = scalbn(dfull[w.dlist[base + k]], -ea);
      int lo = 0, hi = n;    // reduced eigenvalues >= d_q (non-increasing in k)
      while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (lam_greater_equal(w.sig[base + mid], w.mu[base + mid], dq)) lo = mid + 1;
        else hi = mid;
      }
      w.dpos[g] = k + lo;
    }
  }
}

// ---------------------------------------------------------------------------------
// k_vectors: one warp per eigenvalue row.  x_j = zeta_j / ((d_j - sigma) - mu) (for a
// pole shift d_i this is Eq. (eigenvecAi), with x_i = -zeta_i / mu), ||x|| with a
// scaled fallback when the plain sum of squares over- or underflows, v = x / ||x||.
// Each x_j is evaluated once: the first pass stores it in the output row while summing
// the squares, the second rescales the row in place (FP64 work once, the row written twice).
// Writes lambda, sigma, mu, ||x|| and row k of the problem's V^T block (coalesced along
// j).  In a deflated problem the row of reduced eigenvalue k goes to output row rpos and
// component q takes coef[q] * x_{src[q]}; deflated pairs are written by k_defl_rows.  A row the
// solve kernel's tail wrote (row_values, the same arithmetic) is kept when its record holds the
// final (sigma, mu); rows whose pair the remedies or the near-zero path changed are written anew.
// ---------------------------------------------------------------------------------
// Scalar outputs of eigenpair g (reduced index k, output row `row`) in the caller's units --
// lambda, sigma, mu times 2^a and ||x|| times 2^(b - a) -- and the range check: the pair needs
// values outside the binary64 range (mu zero, subnormal or not finite: lambda within 2^-1022 of
// its shift in normalised units; lambda or ||x|| not finite), or after a non-pole shift the
// difference to a neighbouring pole still cancels (R2 in double the working precision did not
// bring sigma next to lambda within its solves).
__device__ __forceinline__ void pair_outputs(const Prob& pb, const Ws& w, int p, int64_t g, int64_t base, int k,
                                             int row, const double* __restrict__ d, double s, double m, double nrm,
                                             double scale, double c) {
  const int ea = w.pexp[2 * p], eb = w.pexp[2 * p + 1];
  const double lz = w.lamz[g];
  const double lam = isnan(lz) ? __dadd_rn(s, m) : lz;
  const double xn = nrm / scale;
  pb.lambda[base + row] = scalbn(lam, ea);
  if (pb.sigma) pb.sigma[base + row] = scalbn(s, ea);
  if (pb.mu) pb.mu[base + row] = scalbn(m, ea);
  if (pb.xnorm) pb.xnorm[base + row] = scalbn(xn, eb - ea);
  bool out = !(fabs(m) >= 0x1p-1022) || !isfinite(m) || !isfinite(lam) || !(xn > 0.0) || !isfinite(xn) ||
             !isfinite(c);
  if (w.shift[g] < 0) out = out || pole_difference_cancels(d[k], s, m) ||
                            (k > 0 && pole_difference_cancels(d[k - 1], s, m));
  if (out) atomicOr(w.status, ST_RANGE);
}

__global__ void __launch_bounds__(256) k_vectors(Prob pb, Ws w) {
  if (*w.status & ST_FATAL) return;
  const int lane = threadIdx.x & 31;
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t g = wid; g < pb.total; g += nw) {
    const int p = p_owner(pb, w, g);
    if (w.pst[p] & PT_TRIVIAL) continue;
    const int64_t base = p_base(pb, p);
    const int n = w.nred[p];
    const int nfull = p_size(pb, p);
    const int k = (int)(g - base);
    if (k >= n) continue;
    const bool defl = (n != nfull);
    const double* __restrict__ d = w.dr + base;
    const double* __restrict__ z = w.zr + base;
    const double s = w.sig[g], m = w.mu[g];
    const int row = defl ? w.rpos[g] : k;
    double* vr = pb.Vt ? pb.Vt + p_vbase(pb, p) + (int64_t)row * p_ld(pb, p) : nullptr;
    if (w.vstate && vr && !defl && w.vstate[g] == 2u) {
      // the solve kernel's tail wrote the row: kept if it was formed from the final pair
      const double* rec = w.vrow + 4 * g;
      if (__double_as_longlong(rec[0]) == __double_as_longlong(s) &&
          __double_as_longlong(rec[1]) == __double_as_longlong(m)) {
        if (lane == 0) pair_outputs(pb, w, p, g, base, k, row, d, s, m, rec[2], rec[3], rec[3] / rec[2]);
        continue;
      }
    }
    // without deflation the row is written with its norm; a deflated row is written below
    double nrm, scale;
    row_values(d, z, n, s, m, defl ? nullptr : vr, lane, &nrm, &scale);
    const double c = scale / nrm;
    if (lane == 0) {
      pair_outputs(pb, w, p, g, base, k, row, d, s, m, nrm, scale, c);
      if (vr) atomicAdd(&w.counters[C_VECROWS], 1u);
    }
    if (!vr || !defl) continue;
    for (int qq = lane; qq < nfull; qq += 32) {
      int sj = w.src[base + qq];
      double v = 0.0;
      if (sj >= 0) v = w.coef[base + qq] * (__dmul_rn(z[sj], rcp(__dsub_rn(__dsub_rn(d[sj], s), m))) * c);
      vr[qq] = v;
    }
  }
}

// Rows of deflated pairs: e_q for zeta_q == 0; for the t-th non-zero member m_t of a tie
// group (t >= 1) the vector Q^T e_{m_t} of the Givens chain: -zeta_{m_t} zeta_j / (r_t r_{t-1})
// at the earlier non-zero members j of the group and r_{t-1}/r_t at m_t.
__global__ void k_defl_rows(Prob pb, Ws w) {
  if (*w.status & ST_FATAL) return;
  const int lane = threadIdx.x & 31;
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t g = wid; g < pb.total; g += nw) {
    const int p = p_owner(pb, w, g);
    if (w.pst[p] & PT_TRIVIAL) continue;
    const int64_t base = p_base(pb, p);
    const int qd = (int)(g - base);
    if (qd >= w.ndefl[p]) continue;
    const int nfull = p_size(pb, p);
    const double* dfull = pb.d + base;
    const double* zfull = pb.z + base;
    const int eb = w.pexp[2 * p + 1];                   // rcur, rprev are norms of scaled weights
    const int q = w.dlist[base + qd];
    const int row = w.dpos[g];
    const double dq = dfull[q];
    if (lane == 0) {
      pb.lambda[base + row] = dq;
      if (pb.sigma) pb.sigma[base + row] = dq;
      if (pb.mu) pb.mu[base + row] = 0.0;
      if (pb.xnorm) pb.xnorm[base + row] = 0.0;
    }
    if (!pb.Vt) continue;
    double* vr = pb.Vt + p_vbase(pb, p) + (int64_t)row * p_ld(pb, p);
    const double zq = scalbn(zfull[q], -eb);
    const int g0 = w.gst[base + q];
    const double rc = w.rcur[base + q], rp = w.rprev[base + q];
    for (int j = lane; j < nfull; j += 32) {
      double v = 0.0;
      if (zero_weight(zq)) {
        v = (j == q) ? 1.0 : 0.0;
      } else if (j == q) {
        v = rp / rc;
      } else if (j >= g0 && j < q) {
        const double zj = scalbn(zfull[j], -eb);
        if (!zero_weight(zj)) v = -(zq / rc) * (zj / rp);
      }
      vr[j] = v;
    }
  }
}

// rho_p == 0 (or rho' outside the normal range, reported): lambda = d, V = I, sigma = d,
// mu = 0 (one warp per row).
__global__ void k_trivial(Prob pb, Ws w) {
  if (*w.status & ST_FATAL) return;
  const int lane = threadIdx.x & 31;
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t g = wid; g < pb.total; g += nw) {
    const int p = p_owner(pb, w, g);
    if (!(w.pst[p] & PT_TRIVIAL)) continue;
    const int64_t base = p_base(pb, p);
    const int n = p_size(pb, p);
    const int k = (int)(g - base);
    if (lane == 0) {
      pb.lambda[g] = pb.d[g];
      if (pb.sigma) pb.sigma[g] = pb.d[g];
      if (pb.mu) pb.mu[g] = 0.0;
      if (pb.xnorm) pb.xnorm[g] = 0.0;
    }
    if (!pb.Vt) continue;
    double* vr = pb.Vt + p_vbase(pb, p) + (int64_t)k * p_ld(pb, p);
    for (int j = lane; j < n; j += 32) vr[j] = (j == k) ? 1.0 : 0.0;
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
  r.warps_auto = !(s->warps_per_block > 0 && s->warps_per_block <= 8);
  r.bps_auto = !(s->blocks_per_sm > 0 && s->blocks_per_sm <= 8);
  r.bps = s->blocks_per_sm > 0 && s->blocks_per_sm <= 8 ? s->blocks_per_sm : DPR1_SOLVE_MIN_BLOCKS;
  r.cap = s->max_bisect >= 1 && s->max_bisect <= 4096 ? s->max_bisect : def.max_bisect;
  r.events = s->phase_events;
  r.fast = s->zero_finder == 1;
  r.dd_mode = (s->dd_mode == 2) ? 2 : 1;
  r.T_kappa = s->T_kappa > 0 ? s->T_kappa : def.T_kappa;
  r.screen = s->screen != 0;
  return r;
}

static void record(const Options& o, int t, cudaStream_t st) {
  if (o.events && o.events[t]) cudaEventRecord((cudaEvent_t)o.events[t], st);
}

template <int L>
static void launch_solve_fix(const Prob& pb, const Ws& w, const Options& o, int grid, int warps, double avg_n,
                             cudaStream_t st) {
  record(o, 0, st);
  if (L == 32 && avg_n > DPR1_SOLVE_LARGE_N)
    k_solve<32, DPR1_SOLVE_MIN_BLOCKS, true><<<grid, 32 * warps, 0, st>>>(pb, w, o.cap, o.fast, o.dd_mode, o.T_kappa,
                                                                          o.screen);
  else
    k_solve<L, DPR1_SOLVE_SMALL_BLOCKS, false><<<grid, 32 * warps, 0, st>>>(pb, w, o.cap, o.fast, o.dd_mode, o.T_kappa,
                                                                           o.screen);
  record(o, 1, st);
  int64_t cg = (pb.total + 255) / 256;
  if (cg > sm_count() * 8) cg = sm_count() * 8;
  k_classify<<<cg > 0 ? (int)cg : 1, 256, 0, st>>>(pb, w, o.T_Knu);
  if ((pb.P < 64 && avg_n > DPR1_FIX_SMALL_N) || avg_n > DPR1_FIX_WARP_MAX_N) {
    // few flagged eigenvalues of large problems: a block-wide group each finishes every item
    // soonest
    int64_t fg = pb.total;                            // at most one block per eigenpair
    if (fg > sm_count() * DPR1_FIX_BLOCKS_PER_SM) fg = sm_count() * DPR1_FIX_BLOCKS_PER_SM;
    if (w.terms && fg > w.term_slots) fg = w.term_slots;   // every group with a buffer
    k_fix<DPR1_FIX_THREADS, true><<<fg > 0 ? (int)fg : 1, DPR1_FIX_THREADS, 0, st>>>(pb, w, o.T_Knu, o.cap, o.fast,
                                                                                  o.dd_mode, o.T_kappa, o.screen);
  } else {
    // small problems, or many of them: one warp each (a block-wide group would leave most of
    // its threads idle and pay a barrier per evaluation), in blocks of one warp, which the block
    // scheduler spreads over the SMs -- with 8-warp blocks the first warps to reach the work
    // counter, and so a few flagged eigenvalues, would share the binary64 pipes of a few SMs
    int64_t fg = pb.total;                            // at most one warp per eigenpair
    if (fg > sm_count() * 32) fg = sm_count() * 32;
    if (w.terms && fg > w.term_slots) fg = w.term_slots;   // every group with a buffer
    k_fix<32, false><<<fg > 0 ? (int)fg : 1, 32, 0, st>>>(pb, w, o.T_Knu, o.cap, o.fast, o.dd_mode, o.T_kappa, o.screen);
  }
  record(o, 2, st);
}

// Launch sequence for a problem table; `avg_n` picks the lane-group width when the
// options leave it open.
static dpr1_status run_table(const Prob& pb, void* workspace, size_t wbytes, const Options& o, double avg_n,
                             cudaStream_t st) {
  Ws w;
  const size_t base = ws_layout2(pb.total, pb.P, pb.offs != nullptr, &w, (char*)workspace);
  if (cudaMemsetAsync(w.hdr, 0, sizeof(unsigned) * 64, st) != cudaSuccess) return DPR1_ERR_CUDA;
  if (cudaMemsetAsync(w.pst, 0, sizeof(unsigned) * (size_t)(pb.P > 0 ? pb.P : 1), st) != cudaSuccess)
    return DPR1_ERR_CUDA;
  const int sms = sm_count();
  if (pb.offs) {
    int og = (pb.P + 7) / 8;
    if (og > sms * 8) og = sms * 8;
    k_owner<<<og > 0 ? og : 1, 256, 0, st>>>(pb, w);
  }
  int ng = pb.P;                                        // a block per problem
  if (ng > sms * 8) ng = sms * 8;
  k_norm<<<ng > 0 ? ng : 1, 256, 0, st>>>(pb, w);
  int64_t sg = (pb.total + 255) / 256;
  if (sg > sms * 8) sg = sms * 8;
  if (sg < 1) sg = 1;
  const int sgrid = (int)sg;
  k_scan<<<sgrid, 256, 0, st>>>(pb, w);
  int dg = (pb.P + 3) / 4;                              // a warp per problem
  if (dg > sms * 8) dg = sms * 8;
  k_deflate<<<dg > 0 ? dg : 1, 128, 0, st>>>(pb, w);
  int L = o.lanes ? o.lanes : default_lanes(avg_n, pb.P);
  // Shape of the solve kernel.  Its time is set by the binary64 pipe of the busiest SM, so the
  // eigenvalues must spread evenly over the SMs: with fewer lane groups than 8-warp blocks on
  // every SM can hold, blocks of fewer warps, at most one per SM; else as many 8-warp blocks per
  // SM (up to the default, all resident at once) as the lane groups fill completely, whose
  // groups take eigenvalues from the work counter (a partly filled extra block per SM would load
  // some SMs more than others).  Options may fix the shape.
  int warps = o.warps;
  int bps = o.bps;
  // problems of small order run the solve kernel compiled for fewer resident blocks (its sums
  // inlined; DPR1_SOLVE_LARGE_N)
  if (o.bps_auto && !(L == 32 && avg_n > DPR1_SOLVE_LARGE_N) && bps > DPR1_SOLVE_SMALL_BLOCKS)
    bps = DPR1_SOLVE_SMALL_BLOCKS;
  const int64_t lanes_total = pb.total * L;
  if (o.warps_auto) {
    const int64_t w_need = (lanes_total + 32 * (int64_t)sms - 1) / (32 * (int64_t)sms);
    warps = w_need >= 8 ? 8 : (int)(w_need > 0 ? w_need : 1);
    if (o.bps_auto) {
      const int64_t fill = lanes_total / ((int64_t)32 * 8 * sms);
      if (fill < bps) bps = fill > 1 ? (int)fill : 1;
    }
  }
  int groups_per_block = (32 * warps) / L;
  int64_t want_blocks = (pb.total + groups_per_block - 1) / groups_per_block;
  int grid = sms * bps;
  if (want_blocks < grid) grid = want_blocks > 0 ? (int)want_blocks : 1;
  // the rest of the workspace holds the stored elements of the inverse for the solves: one
  // buffer for every lane group of the launch (for one problem, of its order), or none at all.
  // Every group then forms the secular sums the same way, so the results do not depend on
  // which group takes which eigenvalue.
  if (wbytes > base) {
    const size_t tb = wbytes - base;
    const int64_t groups = (int64_t)grid * groups_per_block;
    int64_t tn = (int64_t)(tb / (TERM_BYTES * (size_t)groups)) & ~(int64_t)31;
    if (pb.P == 1) tn = (pb.total + 31) & ~(int64_t)31;
    if (tn >= 32 && (size_t)groups * TERM_BYTES * (size_t)tn <= tb) {
      w.terms = (double*)((char*)workspace + base);
      w.term_n = tn;
      w.term_slots = groups;
      // after the buffers, the records of the eigenvector rows the solve kernel's tail writes
      // (one problem, solved by the kernel's large form, with eigenvectors)
      if (kTailRows && pb.P == 1 && pb.Vt && L == 32 && avg_n > DPR1_SOLVE_LARGE_N) {
        const size_t at = align256(base + (size_t)groups * TERM_BYTES * (size_t)tn);
        const size_t rec = align256(sizeof(double) * 4 * (size_t)pb.total);
        if (at + rec + align256(sizeof(unsigned) * (size_t)pb.total) <= wbytes) {
          w.vrow = (double*)((char*)workspace + at);
          w.vstate = (unsigned*)((char*)workspace + at + rec);
          if (cudaMemsetAsync(w.vstate, 0, sizeof(unsigned) * (size_t)pb.total, st) != cudaSuccess)
            return DPR1_ERR_CUDA;
        }
      }
    }
  }
  if (L == 8) launch_solve_fix<8>(pb, w, o, grid, warps, avg_n, st);
  else if (L == 16) launch_solve_fix<16>(pb, w, o, grid, warps, avg_n, st);
  else launch_solve_fix<32>(pb, w, o, grid, warps, avg_n, st);
  k_zero_detect<<<sgrid, 256, 0, st>>>(pb, w, o.T_zero);
  k_zero_solve<<<4, 128, 0, st>>>(pb, w, o.cap, o.fast);
  k_defl_positions<<<sgrid, 256, 0, st>>>(pb, w);
  int64_t vg = (pb.total + 7) / 8;
  if (vg > sms * 16) vg = sms * 16;
  if (vg < 1) vg = 1;
  k_vectors<<<(int)vg, 256, 0, st>>>(pb, w);
  record(o, 3, st);
  k_defl_rows<<<(int)vg, 256, 0, st>>>(pb, w);
  k_trivial<<<(int)vg, 256, 0, st>>>(pb, w);
  return cudaGetLastError() == cudaSuccess ? DPR1_OK : DPR1_ERR_CUDA;
}

dpr1_status run_eig(int64_t n64, const double* d, const double* z, double rho, double* lambda, double* Vt,
                    int64_t ldv, double* sigma, double* mu, double* xnorm, void* workspace, size_t wbytes,
                    const dpr1_options* opt, cudaStream_t st) {
  Prob pb;
  pb.P = 1;
  pb.total = n64;
  pb.offs = nullptr;
  pb.voffs = nullptr;
  pb.rhos = nullptr;
  pb.rho0 = rho;
  pb.ldv0 = ldv;
  pb.d = d; pb.z = z;
  pb.lambda = lambda; pb.Vt = Vt; pb.sigma = sigma; pb.mu = mu; pb.xnorm = xnorm;
  Options o = resolve(opt);
  return run_table(pb, workspace, wbytes, o, (double)n64, st);
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
  opt->zero_finder = 0;
  opt->dd_mode = 1;
  opt->T_kappa = 1500.0;
  opt->screen = 1;
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
    case DPR1_ERR_RANGE: return "an eigenpair needs values outside the binary64 range";
  }
  return "unknown status";
}

size_t dpr1_workspace_size(int64_t n) {
  if (n < 0) return 0;
  return ws_layout(n, nullptr, nullptr) + term_bytes(n, 1);
}

size_t dpr1_batched_workspace_size(int64_t nprob, int64_t total_n) {
  if (nprob < 0 || total_n < 0) return 0;
  return ws_layout2(total_n, nprob, true, nullptr, nullptr) + term_bytes(total_n, nprob);
}

dpr1_status dpr1_eig(int64_t n, const double* d, const double* z, double rho, double* lambda, double* Vt, int64_t ldv,
                     double* sigma, double* mu, double* xnorm, void* workspace, size_t workspace_bytes,
                     const dpr1_options* opt, dpr1_stream_t stream) {
  if (n < 0 || n > (int64_t)0x3fffffff) return DPR1_ERR_ARG;
  if (!std::isfinite(rho) || rho < 0.0) return DPR1_ERR_RHO;
  if (n == 0) return DPR1_OK;
  if (!d || !z || !lambda) return DPR1_ERR_ARG;
  if (Vt && ldv < n) return DPR1_ERR_ARG;
  // the stored-element buffers at the end of the workspace are optional
  if (!workspace || ((uintptr_t)workspace & 255) || workspace_bytes < ws_layout(n, nullptr, nullptr))
    return DPR1_ERR_WORKSPACE;
  return run_eig(n, d, z, rho, lambda, Vt, ldv, sigma, mu, xnorm, workspace, workspace_bytes, opt,
                 (cudaStream_t)stream);
}

dpr1_status dpr1_eig_batched(int64_t nprob, int64_t total_n, const int64_t* offs, const int64_t* voffs,
                             const double* d, const double* z, const double* rho, double* lambda, double* Vt,
                             double* sigma, double* mu, double* xnorm, void* workspace, size_t workspace_bytes,
                             const dpr1_options* opt, dpr1_stream_t stream) {
  if (nprob < 0 || nprob > (int64_t)0x3fffffff || total_n < 0) return DPR1_ERR_ARG;
  if (nprob == 0 || total_n == 0) return DPR1_OK;
  if (!offs || !d || !z || !rho || !lambda) return DPR1_ERR_ARG;
  if (Vt && !voffs) return DPR1_ERR_ARG;
  if (!workspace || ((uintptr_t)workspace & 255) ||
      workspace_bytes < ws_layout2(total_n, nprob, true, nullptr, nullptr))
    return DPR1_ERR_WORKSPACE;
  Prob pb;
  pb.P = (int)nprob;
  pb.total = total_n;
  pb.offs = offs;
  pb.voffs = voffs;
  pb.rhos = rho;
  pb.rho0 = 0.0;
  pb.ldv0 = 0;
  pb.d = d; pb.z = z;
  pb.lambda = lambda; pb.Vt = Vt; pb.sigma = sigma; pb.mu = mu; pb.xnorm = xnorm;
  Options o = resolve(opt);
  return run_table(pb, workspace, workspace_bytes, o, (double)total_n / (double)nprob, (cudaStream_t)stream);
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
  if (st & ST_BADARG) return DPR1_ERR_ARG;
  if (st & ST_RHO) return DPR1_ERR_RHO;
  if (st & ST_NONFINITE) return DPR1_ERR_NONFINITE;
  if (st & ST_UNSORTED) return DPR1_ERR_UNSORTED;
  if (st & ST_RANGE) return DPR1_ERR_RANGE;
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
  out[0] = c[C_SOLVED];
  out[1] = c[C_FIX_N];
  out[2] = c[C_R1];
  out[3] = c[C_R2];
  out[4] = c[C_EVAL_SOLVE];
  out[5] = c[C_EVAL_FIX];
  out[6] = c[C_ZERO_N];
  out[7] = c[C_DEFL];
  out[8] = c[C_DD];
  out[9] = c[C_SCREEN];
  out[10] = c[C_R2DD];
  out[11] = c[C_SCREEN_NEAR];
  out[12] = c[C_SCREEN_DF];
  out[13] = c[C_INFER];
  out[14] = c[C_PROBE];
  out[15] = c[C_SHIFT32];
  out[16] = c[C_TAILROWS];
  out[17] = c[C_VECROWS];
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
