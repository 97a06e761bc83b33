// dpr1_tridiag.cu -- divide-and-conquer eigensolver for a symmetric tridiagonal matrix T
// (diagonal a, off-diagonal b) whose merges are DPR1 eigenproblems (Sec. 1: divide and
// conquer is where DPR1 problems arise), each level's merges solved by one batched
// dpr1_eig launch.
//
// Tree: node i at depth t covers [s_i, s_{i+1}), s_i = floor(i n / 2^t), and has children
// 2i and 2i+1 at depth t+1; at depth T = ceil(log2 n) every node holds at most one index,
// and every boundary between consecutive indices is the split of exactly one node.
// Tear at a node's split m: T = diag(T1, T2) + rho v v^T, rho = |b_{m-1}|,
// v = e_{m-1} + sign(b_{m-1}) e_m, with |b_{m-1}| taken off the two corner diagonal entries;
// so a single index i carries a_i - |b_{i-1}| - |b_i|.
// Merge: T1 = Q1 L1 Q1^T, T2 = Q2 L2 Q2^T give T = Q (L + rho u u^T) Q^T, Q = diag(Q1, Q2),
// u = (last components of Q1's eigenvectors, sign * first components of Q2's).  The poles
// L1, L2 (each non-increasing) are merged into one non-increasing order (T1's entry first
// on ties), the DPR1 problem is solved, and the eigenvectors of T are
//   Q^T_node[k, :] = [G^T[k, 0:N1] Q1^T, G^T[k, N1:N] Q2^T],  G^T[k, s] = W^T[k, pos(s)],
// W^T the DPR1 eigenvector rows (sorted basis) and pos(s) the merged position of pole s.
// Weights with rho |u_j| <= 8 u ||T|| (u = 2^-53, ||T|| the largest Gershgorin row sum) are
// set to zero, the usual backward-stable deflation of divide and conquer; beyond the exact
// deflation of Sec. 1 it keeps every surviving u_j^2 in the normal range of binary64.
// The products run in k_dc_gemm, a binary64 tiled GEMM that reads W^T through pos.
// Storage per depth: eigenvalues in index order (n doubles), and each node's Q^T as an
// N x N row-major block at voffs_t[i] = i q^2 + (2q + 1) floor(i r / 2^t), q = floor(n / 2^t),
// r = n mod 2^t (the node sizes are q or q + 1, so the prefix sums of N^2 have this form).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "../../include/dpr1.h"
#include "dpr1_device.cuh"
#include "dpr1_internal.cuh"

namespace dpr1 {

static size_t a256t(size_t x) { return (x + 255) & ~(size_t)255; }

static int tree_depth(int64_t n) {
  int T = 0;
  while (((int64_t)1 << T) < n) T++;
  return T;
}

// sum over the nodes at depth t of N_i^2
static int64_t level_blocks(int64_t n, int t) {
  int64_t P = (int64_t)1 << t;
  int64_t q = n >> t, r = n - (q << t);
  return P * q * q + (2 * q + 1) * r;
}

struct DcWs {
  unsigned* status;   // the call's status word (dpr1_stream_status reads it)
  double* tol;        // deflation tolerance of the merges
  double *leaf, *lamA, *lamB, *dm, *zm, *rho, *Qe, *Qo, *WT;
  int* pos;
  int64_t* tab;       // offs and voffs of every depth: depth t at tab + 2 (2^t - 1 + t), 2 (2^t + 1) entries
  void* bws;
  size_t bws_bytes;
};

__host__ __device__ __forceinline__ int64_t tab_index(int t) { return 2 * ((((int64_t)1) << t) - 1 + t); }

static size_t dc_layout(int64_t n, DcWs* w, char* base) {
  size_t nn = (size_t)(n > 0 ? n : 1);
  int T = tree_depth(n);
  size_t qe = 1, qo = 1, wt = 1;
  for (int t = 0; t <= T; t++) {
    size_t b = (size_t)level_blocks(n, t);
    if (t < T && b > wt) wt = b;
    if (t == 0) continue;
    if (t & 1) { if (b > qo) qo = b; }
    else if (b > qe) qe = b;
  }
  size_t tabn = (size_t)tab_index(T + 1);
  int64_t maxp = T > 0 ? ((int64_t)1 << (T - 1)) : 1;
  size_t bws = a256t(dpr1_batched_workspace_size(maxp, n > 0 ? n : 1));
  size_t off = 0;
  size_t o_st = off; off += 256;
  size_t o_leaf = off; off += a256t(8 * nn);
  size_t o_la = off; off += a256t(8 * nn);
  size_t o_lb = off; off += a256t(8 * nn);
  size_t o_dm = off; off += a256t(8 * nn);
  size_t o_zm = off; off += a256t(8 * nn);
  size_t o_rho = off; off += a256t(8 * nn);
  size_t o_pos = off; off += a256t(4 * nn);
  size_t o_tab = off; off += a256t(8 * tabn);
  size_t o_qe = off; off += a256t(8 * qe);
  size_t o_qo = off; off += a256t(8 * qo);
  size_t o_wt = off; off += a256t(8 * wt);
  size_t o_bws = off; off += bws;
  if (w && base) {
    w->status = (unsigned*)(base + o_st);
    w->tol = (double*)(base + o_st + 64);
    w->leaf = (double*)(base + o_leaf);
    w->lamA = (double*)(base + o_la);
    w->lamB = (double*)(base + o_lb);
    w->dm = (double*)(base + o_dm);
    w->zm = (double*)(base + o_zm);
    w->rho = (double*)(base + o_rho);
    w->pos = (int*)(base + o_pos);
    w->tab = (int64_t*)(base + o_tab);
    w->Qe = (double*)(base + o_qe);
    w->Qo = (double*)(base + o_qo);
    w->WT = (double*)(base + o_wt);
    w->bws = base + o_bws;
    w->bws_bytes = bws;
  }
  return off;
}

__device__ __forceinline__ int64_t d_start(int64_t i, int64_t n, int t) { return (i * n) >> t; }

__device__ __forceinline__ int64_t d_voff(int64_t i, int64_t n, int t) {
  const int64_t q = n >> t, r = n - (q << t);
  return i * q * q + (2 * q + 1) * ((i * r) >> t);
}

// node at depth t that holds index g: the largest i with floor(i n / 2^t) <= g
__device__ __forceinline__ int64_t d_node(int64_t g, int64_t n, int t) {
  return ((((g + 1) << t) + n - 1) / n) - 1;
}

// offs and voffs of every depth 0..T (the tables dpr1_eig_batched reads)
__global__ void k_dc_tables(int64_t n, int T, int64_t* __restrict__ tab) {
  const int64_t total = tab_index(T + 1);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int t = 0;
    while (tab_index(t + 1) <= e) t++;
    const int64_t loc = e - tab_index(t);
    const int64_t np1 = ((int64_t)1 << t) + 1;
    tab[e] = (loc < np1) ? d_start(loc, n, t) : d_voff(loc - np1, n, t);
  }
}

// single indices: leaf values, and the depth-T eigenvalues (leaf values) and 1x1 blocks
__global__ void k_dc_leaves(int64_t n, int T, const double* __restrict__ a, const double* __restrict__ b,
                            double* __restrict__ leaf, double* __restrict__ lamT, double* __restrict__ QT) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    const double bl = g > 0 ? fabs(b[g - 1]) : 0.0;
    const double br = g + 1 < n ? fabs(b[g]) : 0.0;
    const double v = __dsub_rn(__dsub_rn(a[g], bl), br);
    leaf[g] = v;
    lamT[g] = v;
    QT[d_voff(d_node(g, n, T), n, T)] = 1.0;
  }
}

// Deflation tolerance of every merge, 8 u ||T|| with u = 2^-53 and ||T|| bounded by the
// largest Gershgorin row sum (|a_i| + |b_{i-1}|) + |b_i| (one block).
__global__ void __launch_bounds__(1024) k_dc_norm(int64_t n, const double* __restrict__ a,
                                                  const double* __restrict__ b, double* __restrict__ tol) {
  __shared__ double part[32];
  double m = 0.0;
  for (int64_t g = threadIdx.x; g < n; g += blockDim.x) {
    const double bl = g > 0 ? fabs(b[g - 1]) : 0.0;
    const double br = g + 1 < n ? fabs(b[g]) : 0.0;
    m = fmax(m, __dadd_rn(__dadd_rn(fabs(a[g]), bl), br));
  }
  m = group_max<32>(m, FULL);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); k++) r = fmax(r, part[k]);
    *tol = scalbn(r, -50);
  }
}

// the status a batched call recorded, accumulated into the call's status word
__global__ void k_dc_status(const unsigned* __restrict__ level, unsigned* __restrict__ call) { *call |= *level; }

// number of entries of the non-increasing x[0..m) that are > v (strict) or >= v
__device__ __forceinline__ int count_above(const double* __restrict__ x, int m, double v, bool strict) {
  int lo = 0, hi = m;
  while (lo < hi) {
    const int md = (lo + hi) >> 1;
    const bool above = strict ? (x[md] > v) : (x[md] >= v);
    if (above) lo = md + 1;
    else hi = md;
  }
  return lo;
}

// DPR1 inputs of every node at depth t from its children at depth t+1
__global__ void k_dc_merge(int64_t n, int t, const double* __restrict__ b, const double* __restrict__ leaf,
                           const double* __restrict__ tolp, const double* __restrict__ lamc,
                           const double* __restrict__ QTc,
                           double* __restrict__ dm, double* __restrict__ zm, double* __restrict__ rho,
                           int* __restrict__ pos, double* __restrict__ QTt) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = d_node(g, n, t);
    const int64_t lo = d_start(i, n, t), hi = d_start(i + 1, n, t);
    const int N = (int)(hi - lo);
    if (N == 1) {
      dm[g] = leaf[g];
      zm[g] = 1.0;
      rho[i] = 0.0;
      pos[g] = 0;
      if (QTt) QTt[d_voff(i, n, t)] = 1.0;
      continue;
    }
    const int64_t mid = d_start(2 * i + 1, n, t + 1);
    const int N1 = (int)(mid - lo), N2 = (int)(hi - mid);
    const double beta = b[mid - 1];
    if (g == lo) rho[i] = fabs(beta);
    const double sgn = beta >= 0.0 ? 1.0 : -1.0;
    const double v = lamc[g];
    int p;
    double u;
    if (g < mid) {
      const int a_ = (int)(g - lo);
      p = a_ + count_above(lamc + mid, N2, v, true);
      u = QTc[d_voff(2 * i, n, t + 1) + (int64_t)a_ * N1 + (N1 - 1)];
    } else {
      const int b_ = (int)(g - mid);
      p = b_ + count_above(lamc + lo, N1, v, false);
      u = sgn * QTc[d_voff(2 * i + 1, n, t + 1) + (int64_t)b_ * N2];
    }
    // backward-stable deflation: rho |u| <= 8 u ||T|| drops the weight (and keeps every
    // surviving u^2 in the normal range of binary64)
    if (__dmul_rn(fabs(beta), fabs(u)) <= *tolp) u = 0.0;
    dm[lo + p] = v;
    zm[lo + p] = u;
    pos[g] = p;
  }
}

// C = A B per node and half h (h = 0: columns 0..N1 with Q1; h = 1: columns N1..N with Q2):
//   A[r, k] = W^T[r, pos(off_h + k)]  (N x N_h),  B = child's Q^T (N_h x N_h),
//   C[r, c] -> Q^T_node[r, off_h + c].
// One block computes a 64 x 64 tile of C with 256 threads (4 x 4 each), k in steps of 16.
constexpr int GT = 64, GK = 16;

__global__ void __launch_bounds__(256) k_dc_gemm(int64_t n, int t, int64_t tiles_per_node,
                                                 const double* __restrict__ WT, const int* __restrict__ pos,
                                                 const double* __restrict__ QTc, double* __restrict__ out,
                                                 int64_t ldo_root) {
  __shared__ double As[GK][GT + 1];
  __shared__ double Bs[GK][GT];
  __shared__ int ps[GK];
  const int64_t item = blockIdx.x;
  const int64_t i = item / tiles_per_node;
  int64_t loc = item - i * tiles_per_node;
  const int64_t lo = d_start(i, n, t), hi = d_start(i + 1, n, t);
  const int N = (int)(hi - lo);
  if (N < 2) return;
  const int64_t mid = d_start(2 * i + 1, n, t + 1);
  const int N1 = (int)(mid - lo), N2 = (int)(hi - mid);
  const int tr_ = (N + GT - 1) / GT;
  const int tc1 = (N1 + GT - 1) / GT, tc2 = (N2 + GT - 1) / GT;
  int h, Nh, off, tr, tc;
  if (loc < (int64_t)tr_ * tc1) { h = 0; Nh = N1; off = 0; tr = (int)(loc / tc1); tc = (int)(loc % tc1); }
  else {
    loc -= (int64_t)tr_ * tc1;
    if (loc >= (int64_t)tr_ * tc2) return;
    h = 1; Nh = N2; off = N1; tr = (int)(loc / tc2); tc = (int)(loc % tc2);
  }
  const double* __restrict__ W = WT + d_voff(i, n, t);
  const double* __restrict__ Bm = QTc + d_voff(2 * i + h, n, t + 1);
  const int* __restrict__ pl = pos + lo + off;
  double* C;
  int64_t ldc;
  if (t == 0) { C = out; ldc = ldo_root; }
  else { C = out + d_voff(i, n, t); ldc = N; }
  const int tid = threadIdx.x;
  const int ty = tid >> 4, tx = tid & 15;
  const int row0 = tr * GT, col0 = tc * GT;
  double acc[4][4];
#pragma unroll
  for (int p = 0; p < 4; p++)
#pragma unroll
    for (int q = 0; q < 4; q++) acc[p][q] = 0.0;
  for (int k0 = 0; k0 < Nh; k0 += GK) {
    if (tid < GK) ps[tid] = (k0 + tid < Nh) ? pl[k0 + tid] : 0;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < (GT * GK) / 256; q++) {
      const int e = tid + 256 * q;
      const int r = e / GK, kk = e % GK;
      const int row = row0 + r, k = k0 + kk;
      As[kk][r] = (row < N && k < Nh) ? W[(int64_t)row * N + ps[kk]] : 0.0;
      const int kb = e / GT, c = e % GT;
      const int col = col0 + c, kr = k0 + kb;
      Bs[kb][c] = (col < Nh && kr < Nh) ? Bm[(int64_t)kr * Nh + col] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; kk++) {
      double av[4], bv[4];
#pragma unroll
      for (int p = 0; p < 4; p++) av[p] = As[kk][ty * 4 + p];
#pragma unroll
      for (int q = 0; q < 4; q++) bv[q] = Bs[kk][tx * 4 + q];
#pragma unroll
      for (int p = 0; p < 4; p++)
#pragma unroll
        for (int q = 0; q < 4; q++) acc[p][q] = __fma_rn(av[p], bv[q], acc[p][q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < 4; p++) {
    const int row = row0 + ty * 4 + p;
    if (row >= N) continue;
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int col = col0 + tx * 4 + q;
      if (col < Nh) C[(int64_t)row * ldc + off + col] = acc[p][q];
    }
  }
}

}  // namespace dpr1

using namespace dpr1;

extern "C" {

size_t dpr1_tridiag_workspace_size(int64_t n) {
  if (n < 0) return 0;
  return dc_layout(n, nullptr, nullptr);
}

dpr1_status dpr1_tridiag_eig(int64_t n, const double* a, const double* b, double* lambda, double* Qt, int64_t ldq,
                             void* workspace, size_t workspace_bytes, const dpr1_options* opt,
                             dpr1_stream_t stream) {
  if (n < 0 || n > (int64_t)0x3fffffff) return DPR1_ERR_ARG;
  if (n == 0) return DPR1_OK;
  if (!a || !lambda || (n > 1 && !b)) return DPR1_ERR_ARG;
  if (Qt && ldq < n) return DPR1_ERR_ARG;
  if (!workspace || ((uintptr_t)workspace & 255) || workspace_bytes < dpr1_tridiag_workspace_size(n))
    return DPR1_ERR_WORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  DcWs w;
  dc_layout(n, &w, (char*)workspace);
  const int T = tree_depth(n);
  const int sms = sm_count();
  int64_t eg = (n + 255) / 256;
  if (eg > sms * 8) eg = sms * 8;
  if (cudaMemsetAsync(w.status, 0, 256, st) != cudaSuccess) return DPR1_ERR_CUDA;
  double* QTdepth[2] = {w.Qe, w.Qo};
  if (n == 1) {
    // T = 0: the single index is its own leaf, lambda = a_0, Q = [1]
    k_dc_leaves<<<1, 32, 0, st>>>(n, 0, a, b, w.leaf, lambda, Qt ? Qt : w.Qe);
    return cudaGetLastError() == cudaSuccess ? DPR1_OK : DPR1_ERR_CUDA;
  }
  const int64_t tabn = tab_index(T + 1);
  int tg = (int)((tabn + 255) / 256);
  if (tg > sms * 8) tg = sms * 8;
  k_dc_tables<<<tg, 256, 0, st>>>(n, T, w.tab);
  k_dc_norm<<<1, 1024, 0, st>>>(n, a, b, w.tol);
  k_dc_leaves<<<(int)eg, 256, 0, st>>>(n, T, a, b, w.leaf, w.lamA, QTdepth[T & 1]);
  double* lam_child = w.lamA;     // eigenvalues of depth t + 1, in index order
  double* lam_free = w.lamB;
  for (int t = T - 1; t >= 0; t--) {
    const int64_t P = (int64_t)1 << t;
    double* QTc = QTdepth[(t + 1) & 1];
    double* QTt = (t == 0) ? nullptr : QTdepth[t & 1];
    k_dc_merge<<<(int)eg, 256, 0, st>>>(n, t, b, w.leaf, w.tol, lam_child, QTc, w.dm, w.zm, w.rho, w.pos, QTt);
    if (cudaGetLastError() != cudaSuccess) return DPR1_ERR_CUDA;
    double* lam_out = (t == 0) ? lambda : lam_free;
    const int64_t* offs = w.tab + tab_index(t);
    const int64_t* voffs = offs + P + 1;
    dpr1_status s = dpr1_eig_batched(P, n, offs, voffs, w.dm, w.zm, w.rho, lam_out, w.WT, nullptr, nullptr,
                                     nullptr, w.bws, w.bws_bytes, opt, stream);
    if (s != DPR1_OK) return s;
    k_dc_status<<<1, 1, 0, st>>>((const unsigned*)w.bws, w.status);
    if (t > 0 || Qt) {
      const int64_t Nmax = (n + P - 1) / P;            // node sizes are floor or ceil of n / 2^t
      const int64_t Nh = (Nmax + 1) / 2;
      const int64_t tpn = ((Nmax + GT - 1) / GT) * 2 * ((Nh + GT - 1) / GT);
      const int64_t grid = P * tpn;
      if (grid > 0x7fffffffLL) return DPR1_ERR_ARG;
      k_dc_gemm<<<(unsigned)grid, 256, 0, st>>>(n, t, tpn, w.WT, w.pos, QTc, t == 0 ? Qt : QTt, ldq);
      if (cudaGetLastError() != cudaSuccess) return DPR1_ERR_CUDA;
    }
    if (t > 0) {
      lam_free = lam_child;
      lam_child = lam_out;
    }
  }
  return DPR1_OK;
}

}  // extern "C"
