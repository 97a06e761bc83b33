// dpr1_hermitian.cu -- the complex Hermitian DPR1 matrix A = D + rho z z^* (the extension of
// Algorithm 1 to the Hermitian case that the paper states after Algorithm 1).
//
// Write z_j = |z_j| phi_j with |phi_j| = 1 and Phi = diag(phi).  Then Phi^* A Phi =
// D + rho |z| |z|^T is real, so A has the eigenvalues of that real DPR1 matrix, and
// v_k = Phi u_k for its eigenvectors u_k.  This is again Eq. (Aeigenvec) with the complex z:
// (D - lambda_k I)^{-1} z = Phi (D - lambda_k I)^{-1} |z|.  The real problem runs through the
// dpr1_eig launch sequence unchanged.  Its rows u_k are written with twice the row stride
// into the caller's complex output, and k_herm_expand turns each row into the complex entries
// u_kj phi_j in place.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "../../include/dpr1.h"
#include "dpr1_device.cuh"
#include "dpr1_internal.cuh"

namespace dpr1 {

dpr1_status run_eig(int64_t n64, const double* d, const double* z, double rho, double* lambda, double* Vt,
                    int64_t ldv, double* sigma, double* mu, double* xnorm, void* workspace, size_t wbytes,
                    const dpr1_options* opt, cudaStream_t st);

static size_t a256h(size_t x) { return (x + 255) & ~(size_t)255; }

// workspace: [the real dpr1_eig workspace (status word first)][|z|: n doubles][phi: n complex]
struct HermWs {
  void* real_ws;
  size_t real_bytes;
  double* zabs;
  double2* phase;
};

static size_t herm_layout(int64_t n, HermWs* w, char* base) {
  size_t nn = (size_t)(n > 0 ? n : 1);
  size_t off = 0;
  size_t o_real = off; size_t rb = a256h(dpr1_workspace_size(n)); off += rb;
  size_t o_abs = off; off += a256h(sizeof(double) * nn);
  size_t o_ph = off; off += a256h(sizeof(double2) * nn);
  if (w && base) {
    w->real_ws = base + o_real;
    w->real_bytes = rb;
    w->zabs = (double*)(base + o_abs);
    w->phase = (double2*)(base + o_ph);
  }
  return off;
}

// |x + iy| as one fixed sequence of correctly rounded binary64 operations,
// sqrt(x'^2 + y'^2) / s with x' = s x, y' = s y and s = 2^-600 (max(|x|, |y|) > 2^500),
// 2^600 (below 2^-500) or 1, so that every IEEE binary64 implementation of the same steps
// gives the same bits (within 1.5 ulps of the true modulus).  The real problem then has
// exactly the same weights wherever it is formed.
__device__ __forceinline__ double abs_binary64(double x, double y) {
  const double m = fmax(fabs(x), fabs(y));
  double s = 1.0, inv = 1.0;
  if (m > 0x1p500) { s = 0x1p-600; inv = 0x1p600; }
  else if (m < 0x1p-500) { s = 0x1p600; inv = 0x1p-600; }
  const double xs = __dmul_rn(x, s), ys = __dmul_rn(y, s);
  return __dmul_rn(__dsqrt_rn(__dadd_rn(__dmul_rn(xs, xs), __dmul_rn(ys, ys))), inv);
}

// |z_j| and phi_j = z_j / |z_j| (phi_j = 1 for z_j = 0, a deflated component whose eigenvector
// is e_j).  Non-finite entries give a non-finite |z_j|, which the real path reports as
// DPR1_ERR_NONFINITE.
__global__ void k_herm_prep(int n, const double2* __restrict__ z, double* __restrict__ zabs,
                            double2* __restrict__ phase) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const double2 c = z[j];
    const double a = abs_binary64(c.x, c.y);
    zabs[j] = a;
    phase[j] = (a > 0.0 && a <= 1.7976931348623157e308) ? make_double2(__ddiv_rn(c.x, a), __ddiv_rn(c.y, a))
                                                       : make_double2(1.0, 0.0);
  }
}

// Row k holds u_k as n doubles at the start of its complex row (stride 2 ldv doubles);
// one warp rewrites it as n complex numbers u_kj phi_j.  Chunks of 32 entries go from the
// end of the row to its start: chunk c reads doubles [32c, 32c + 32) and writes doubles
// [64c, 64c + 64), which no later (lower) chunk reads, and every lane reads its entry
// before any lane of the chunk writes.
__global__ void k_herm_expand(int n, int64_t ldv, double* __restrict__ Vt, const double2* __restrict__ phase) {
  const int lane = threadIdx.x & 31;
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t k = wid; k < n; k += nw) {
    double* row = Vt + k * 2 * ldv;
    double2* crow = reinterpret_cast<double2*>(row);
    for (int c = (n + 31) / 32 - 1; c >= 0; c--) {
      const int j = c * 32 + lane;
      const double u = (j < n) ? row[j] : 0.0;
      __syncwarp();
      if (j < n) {
        const double2 p = phase[j];
        crow[j] = make_double2(__dmul_rn(u, p.x), __dmul_rn(u, p.y));
      }
      __syncwarp();
    }
  }
}

}  // namespace dpr1

using namespace dpr1;

extern "C" {

size_t dpr1_hermitian_workspace_size(int64_t n) {
  if (n < 0) return 0;
  return herm_layout(n, nullptr, nullptr);
}

dpr1_status dpr1_eig_hermitian(int64_t n, const double* d, const double* z, double rho, double* lambda,
                               double* Vt, int64_t ldv, double* sigma, double* mu, double* xnorm, void* workspace,
                               size_t workspace_bytes, const dpr1_options* opt, dpr1_stream_t stream) {
  if (n < 0 || n > (int64_t)0x3fffffff) return DPR1_ERR_ARG;
  if (!std::isfinite(rho) || rho < 0.0) return DPR1_ERR_RHO;
  if (n == 0) return DPR1_OK;
  if (!d || !z || !lambda) return DPR1_ERR_ARG;
  if (((uintptr_t)z & 15) || (Vt && ((uintptr_t)Vt & 15))) return DPR1_ERR_ARG;
  if (Vt && ldv < n) return DPR1_ERR_ARG;
  if (!workspace || ((uintptr_t)workspace & 255) || workspace_bytes < dpr1_hermitian_workspace_size(n))
    return DPR1_ERR_WORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  HermWs w;
  herm_layout(n, &w, (char*)workspace);
  const int sms = sm_count();
  int g = (int)((n + 255) / 256);
  if (g > sms * 4) g = sms * 4;
  k_herm_prep<<<g, 256, 0, st>>>((int)n, reinterpret_cast<const double2*>(z), w.zabs, w.phase);
  if (cudaGetLastError() != cudaSuccess) return DPR1_ERR_CUDA;
  dpr1_status s = run_eig(n, d, w.zabs, rho, lambda, Vt, Vt ? 2 * ldv : 0, sigma, mu, xnorm, w.real_ws,
                          w.real_bytes, opt, st);
  if (s != DPR1_OK || !Vt) return s;
  int64_t vg = (n + 7) / 8;
  if (vg > sms * 16) vg = sms * 16;
  k_herm_expand<<<(int)vg, 256, 0, st>>>((int)n, ldv, Vt, w.phase);
  return cudaGetLastError() == cudaSuccess ? DPR1_OK : DPR1_ERR_CUDA;
}

}  // extern "C"
