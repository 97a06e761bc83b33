// dpr1_backward.cu -- adjoint of the DPR1 eigen-decomposition (no counterpart in the
// paper; built from its Eq. (Pick) and Eq. (Aeigenvec)).
//
// For eigenpair k with lambda_k = sigma_k + mu_k the columns are recomputed, not stored:
//   s_j = d_j - lambda_k = (d_j - sigma_k) - mu_k,  x_j = zeta_j / s_j,  v = x / ||x||.
// The implicit derivative of f(lambda_k) = 1 + rho sum zeta_j^2 / (d_j - lambda_k) = 0 gives
//   dlambda/dd_j = v_j^2,  dlambda/dzeta_j = -2 x_j / ||x||^2,  dlambda/drho = 1/(rho^2 ||x||^2),
// and with vbar = dL/dv_k, c = v . vbar, g = vbar - v c (so gbar = g / ||x|| is dL/dx):
//   lambdabar = dL/dlambda_k + sum_j g_j v_j / s_j
//   dbar_j   += lambdabar v_j^2 - g_j v_j / s_j
//   zbar_j   += (g_j / s_j - 2 lambdabar v_j) / ||x||
//   rhobar   += lambdabar / (rho ||x||)^2
// Evaluation (as in the oracle's reading): p is the index of the largest |v_p|.  Next to a
// pole v is within ~1e-10 of e_p; then g_p and the two parts of dbar_p cancel at the scale
// 1/s_p, so with S2 = sum_{j != p} v_j^2 (= 1 - v_p^2) and P = sum_{j != p} v_j vbar_j:
//   c = v_p vbar_p + P,  g_p = vbar_p S2 - v_p P,
//   Lam = dL/dlambda_k + sum_{j != p} g_j v_j / s_j,  T_p = g_p v_p / s_p,  lambdabar = Lam + T_p,
//   dbar_p += Lam v_p^2 - T_p S2,   zbar_p += (g_p / s_p (S2 - v_p^2) - 2 Lam v_p) / ||x||.
// Work split: warp w of a set of nwb(n) warps takes rows k = w, w + nwb, ... and keeps
// its own partial rows of dbar and zbar in the workspace (no atomics), and a final kernel
// sums the partials in warp order, so the result does not depend on scheduling.  Each warp
// also keeps the reciprocals 1/s_j of its current row, formed in the first pass and read by the
// other two (each lane reads back what it wrote): the three passes form them once instead of
// three times, 10 of 35 binary64 instructions per component.
// The problem is normalised as in the forward (D' = 2^-a D, z' = 2^-b z, rho' = 2^(2b-a) rho,
// sigma' = 2^-a sigma, mu' = 2^-a mu, dL/dlambda' = 2^a dL/dlambda) and the gradients are
// scaled back (dL/dd = 2^-a dL/dd', dL/dz = 2^-b dL/dz', dL/drho = 2^(2b-a) dL/drho'): in the
// normal range this changes no rounding, and it keeps data of any magnitude in range.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "../../include/dpr1.h"
#include "dpr1_device.cuh"
#include "dpr1_internal.cuh"

namespace dpr1 {

// warps of the row kernel: 152 blocks of wpb(n) warps, one block per SM of a GB300 (a number
// fixed by n, so that the partial sums and their order do not depend on the device).  Large
// orders take more warps: the kernel is latency-bound, and with enough rows per warp (10 at
// n = 32768 with 21 warps per block) the extra partial rows cost little (backward at n = 32768:
// 130.7 ms with 7 warps per block, 89.0 with 14, 83.7 with 21; at n = 4096 the 7-warp blocks
// are fastest, 1.88 against 2.33 and 3.32 ms).
__host__ __device__ inline int wpb(int64_t n) { return n > 24576 ? 21 : (n > 8192 ? 14 : 7); }
__host__ __device__ inline int nwb(int64_t n) { return 152 * wpb(n); }

static size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

struct BwdWs {
  unsigned* status;
  int* ex;      // status words 2, 3: the exponents a, b of the normalisation
  double* pd;   // [nwb][n]
  double* pz;   // [nwb][n]
  double* rb;   // [nwb][n] the reciprocals 1/s_j of each warp's current row
  double* pr;   // [nwb]
  double* ds;   // [n] d' = 2^-a d
  double* zs;   // [n] z' = 2^-b z
};

static size_t bwd_layout(int64_t n, BwdWs* w, char* base) {
  size_t nn = (size_t)(n > 0 ? n : 1);
  size_t off = 0;
  size_t o_st = off; off += 256;
  const size_t nw = (size_t)nwb(n);
  size_t o_pd = off; off += a256(sizeof(double) * nn * nw);
  size_t o_pz = off; off += a256(sizeof(double) * nn * nw);
  size_t o_rb = off; off += a256(sizeof(double) * nn * nw);
  size_t o_pr = off; off += a256(sizeof(double) * nw);
  size_t o_ds = off; off += a256(sizeof(double) * nn);
  size_t o_zs = off; off += a256(sizeof(double) * nn);
  if (w && base) {
    w->status = (unsigned*)(base + o_st);
    w->ex = (int*)(base + o_st) + 2;
    w->ds = (double*)(base + o_ds);
    w->zs = (double*)(base + o_zs);
    w->pd = (double*)(base + o_pd);
    w->pz = (double*)(base + o_pz);
    w->rb = (double*)(base + o_rb);
    w->pr = (double*)(base + o_pr);
  }
  return off;
}

// The exponents of the normalisation (one block): max|d_j| = m 2^a, max|z_j| = m' 2^b.
__global__ void k_bwd_norm(int n, const double* __restrict__ d, const double* __restrict__ z, BwdWs w) {
  double md = 0.0, mz = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    md = fmax(md, fabs(d[j]));
    mz = fmax(mz, fabs(z[j]));
  }
  md = group_max<256>(md, FULL);
  mz = group_max<256>(mz, FULL);
  if (threadIdx.x == 0) {
    int a = 0, b = 0;
    if (md > 0.0 && isfinite(md)) frexp(md, &a);
    if (mz > 0.0 && isfinite(mz)) frexp(mz, &b);
    w.ex[0] = a;
    w.ex[1] = b;
  }
}

// the normalised copies d' and z'
__global__ void k_bwd_scale(int n, const double* __restrict__ d, const double* __restrict__ z, BwdWs w) {
  const int a = w.ex[0], b = w.ex[1];
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    w.ds[j] = scalbn(d[j], -a);
    w.zs[j] = scalbn(z[j], -b);
  }
}

template <int WPB>
__global__ void __launch_bounds__(32 * WPB, 1) k_bwd_rows(int n, double rho_in, const double* __restrict__ sig,
                                                  const double* __restrict__ mu, const double* __restrict__ gl,
                                                  const double* __restrict__ gV, int64_t ldg, BwdWs w) {
  const int lane = threadIdx.x & 31;
  const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  constexpr int NWB = 152 * WPB;
  if (wid >= NWB) return;
  const int ea = w.ex[0], eb = w.ex[1];
  const double* __restrict__ d = w.ds;
  const double* __restrict__ z = w.zs;
  const double rho = scalbn(rho_in, 2 * eb - ea);
  double* __restrict__ pd = w.pd + (size_t)wid * n;
  double* __restrict__ pz = w.pz + (size_t)wid * n;
  double* __restrict__ rb = w.rb + (size_t)wid * n;
  double prho = 0.0;
  unsigned bad = 0;
  bool first = true;
  for (int k = wid; k < n; k += NWB) {
    const double s = scalbn(sig[k], -ea), m = scalbn(mu[k], -ea);
    // pass 1: ||x|| (scaled when the plain sum of squares leaves the safe range) and the
    // index p of the largest component (the smallest index among equal ones)
    double mx = 0.0, q = 0.0;
    int p = n;
    for (int j = lane; j < n; j += 32) {
      const double r = rcp(__dsub_rn(__dsub_rn(d[j], s), m));
      rb[j] = r;
      double x = __dmul_rn(z[j], r);
      double ax = fabs(x);
      if (ax > mx) { mx = ax; p = j; }
      q = __fma_rn(x, x, q);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      double omx = __shfl_xor_sync(FULL, mx, o);
      int op = __shfl_xor_sync(FULL, p, o);
      if (omx > mx || (omx == mx && op < p)) { mx = omx; p = op; }
    }
    q = group_sum<32>(q, FULL);
    double scale = 1.0;
    if (!(q < 1e300) || !(mx > 1e-140)) {
      scale = 1.0 / mx;
      q = 0.0;
      for (int j = lane; j < n; j += 32) {
        double x = __dmul_rn(z[j], rcp(__dsub_rn(__dsub_rn(d[j], s), m))) * scale;
        q = __fma_rn(x, x, q);
      }
      q = group_sum<32>(q, FULL);
    }
    const double nrm = sqrt(q);
    const double cv = scale / nrm;            // v_j = x_j * cv
    const double inv = cv;                    // 1 / ||x||
    if (p >= n) p = 0;
    const double sp = __dsub_rn(__dsub_rn(d[p], s), m);
    const double rp = rcp(sp);
    const double vp = __dmul_rn(z[p], rp) * cv;
    const double* __restrict__ grow = gV ? gV + (int64_t)k * ldg : nullptr;
    const double gvp = grow ? grow[p] : 0.0;
    // pass 2 (j != p): P, S2, A = sum vbar_j v_j / s_j, Bs = sum v_j^2 / s_j
    double P = 0.0, S2 = 0.0, A = 0.0, Bs = 0.0;
    for (int j = lane; j < n; j += 32) {
      if (j == p) continue;
      const double r = rb[j];
      double v = __dmul_rn(z[j], r) * cv;
      double vr = __dmul_rn(v, r);
      S2 = __fma_rn(v, v, S2);
      if (grow) {
        double gv = grow[j];
        P = __fma_rn(v, gv, P);
        A = __fma_rn(gv, vr, A);
        Bs = __fma_rn(v, vr, Bs);
      }
    }
    S2 = group_sum<32>(S2, FULL);
    if (grow) {
      P = group_sum<32>(P, FULL);
      A = group_sum<32>(A, FULL);
      Bs = group_sum<32>(Bs, FULL);
    }
    const double c = grow ? __fma_rn(vp, gvp, P) : 0.0;
    const double gp = grow ? __fma_rn(gvp, S2, -vp * P) : 0.0;
    const double Lam = (gl ? scalbn(gl[k], ea) : 0.0) + __fma_rn(-c, Bs, A);
    const double Tp = __dmul_rn(gp, vp) * rp;
    const double lb = Lam + Tp;
    // pass 3: contributions
    for (int j = lane; j < n; j += 32) {
      double db, zb;
      if (j == p) {
        db = __fma_rn(Lam * vp, vp, -Tp * S2);
        zb = inv * __fma_rn(gp * rp, __fma_rn(-vp, vp, S2), -2.0 * Lam * vp);
      } else {
        const double r = rb[j];
        double v = __dmul_rn(z[j], r) * cv;
        double g = grow ? __fma_rn(-v, c, grow[j]) : 0.0;
        double vr = __dmul_rn(v, r);
        db = __fma_rn(lb * v, v, -g * vr);
        zb = inv * __fma_rn(g, r, -2.0 * lb * v);
      }
      if (first) { pd[j] = db; pz[j] = zb; }
      else { pd[j] += db; pz[j] += zb; }
    }
    first = false;
    double t = inv / rho;
    prho = __fma_rn(lb, t * t, prho);
    if (!isfinite(lb) || !isfinite(nrm)) bad = 1;
  }
  if (lane == 0) {
    w.pr[wid] = prho;
    if (bad) atomicOr(w.status, ST_NONFINITE);
  }
}

// grad_d[j] = sum_w pd[w][j] in warp order (w < min(n, nwb(n))); likewise grad_z and grad_rho.
__global__ void k_bwd_reduce(int n, BwdWs w, double* __restrict__ gd, double* __restrict__ gz,
                             double* __restrict__ grho) {
  const int nwt = nwb(n);
  const int nw = n < nwt ? n : nwt;
  const int ea = w.ex[0], eb = w.ex[1];
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    double a = 0.0, b = 0.0;
    for (int t = 0; t < nw; t++) {
      a += w.pd[(size_t)t * n + j];
      b += w.pz[(size_t)t * n + j];
    }
    gd[j] = scalbn(a, -ea);
    gz[j] = scalbn(b, -eb);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    double r = 0.0;
    for (int t = 0; t < nw; t++) r += w.pr[t];
    *grho = scalbn(r, 2 * eb - ea);
  }
}

}  // namespace dpr1

using namespace dpr1;

extern "C" {

size_t dpr1_backward_workspace_size(int64_t n) {
  if (n < 0) return 0;
  return bwd_layout(n, nullptr, nullptr);
}

dpr1_status dpr1_eig_backward(int64_t n, const double* d, const double* z, double rho, const double* sigma,
                              const double* mu, const double* grad_lambda, const double* grad_Vt, int64_t ldg,
                              double* grad_d, double* grad_z, double* grad_rho, void* workspace,
                              size_t workspace_bytes, const dpr1_options* opt, dpr1_stream_t stream) {
  (void)opt;
  if (n < 0 || n > (int64_t)0x3fffffff) return DPR1_ERR_ARG;
  if (!std::isfinite(rho) || !(rho > 0.0)) return DPR1_ERR_RHO;
  if (n == 0) return DPR1_OK;
  if (!d || !z || !sigma || !mu || !grad_d || !grad_z || !grad_rho) return DPR1_ERR_ARG;
  if (grad_Vt && ldg < n) return DPR1_ERR_ARG;
  if (!workspace || ((uintptr_t)workspace & 255) || workspace_bytes < dpr1_backward_workspace_size(n))
    return DPR1_ERR_WORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  BwdWs w;
  bwd_layout(n, &w, (char*)workspace);
  if (cudaMemsetAsync(w.status, 0, 256, st) != cudaSuccess) return DPR1_ERR_CUDA;
  int g = (int)((n + 255) / 256);
  if (g > 4 * sm_count()) g = 4 * sm_count();
  k_bwd_norm<<<1, 256, 0, st>>>((int)n, d, z, w);
  k_bwd_scale<<<g, 256, 0, st>>>((int)n, d, z, w);
  const int wp = wpb(n);
  if (wp == 21) k_bwd_rows<21><<<152, 32 * 21, 0, st>>>((int)n, rho, sigma, mu, grad_lambda, grad_Vt, ldg, w);
  else if (wp == 14) k_bwd_rows<14><<<152, 32 * 14, 0, st>>>((int)n, rho, sigma, mu, grad_lambda, grad_Vt, ldg, w);
  else k_bwd_rows<7><<<152, 32 * 7, 0, st>>>((int)n, rho, sigma, mu, grad_lambda, grad_Vt, ldg, w);
  k_bwd_reduce<<<g, 256, 0, st>>>((int)n, w, grad_d, grad_z, grad_rho);
  return cudaGetLastError() == cudaSuccess ? DPR1_OK : DPR1_ERR_CUDA;
}

}  // extern "C"
