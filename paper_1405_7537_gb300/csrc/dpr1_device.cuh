// dpr1_device.cuh -- device arithmetic shared by the DPR1 kernels (sm_103a).
//
// * double-double ("dd") numbers: unevaluated sums hi + lo of two binary64 numbers,
//   used for the paper's one element computed in double the working precision
//   (Sec. 2.3): the corner b of Eq. (b_ob), and f(sigma) / the denominator of gamma
//   for the non-pole shifts (R2, Eq. (gamma)).  Error-free transformations: Knuth's
//   TwoSum, Dekker's FastTwoSum and the exact product through fma.
// * a binary64 reciprocal: the sm_103a approximate reciprocal instruction
//   (rcp.approx.ftz.f64, about 20 correct bits) refined by one third-order
//   Newton-Raphson step r = r0 (1 + e + e^2), e = 1 - x r0; the result is within
//   one unit in the last place of 1/x for |x| in [2^-1020, 2^1020] (outside that
//   range the IEEE quotient is used).
// * lane-group reductions with xor shuffles: every lane of a group ends with the
//   bit-identical total (IEEE addition is commutative), so every lane takes the
//   same bisection decisions without a broadcast.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace dpr1 {

constexpr unsigned FULL = 0xffffffffu;

// status bits recorded on the device
enum : unsigned {
  ST_NONFINITE = 1u,
  ST_UNSORTED = 2u,
  ST_NOT_CONVERGED = 4u,
  ST_BADARG = 8u,       // inconsistent batch offsets
  ST_RHO = 16u,         // a rho_p < 0 or not finite
  ST_RANGE = 32u,       // an eigenpair needs values outside the binary64 range (normalised problem)
};

struct dd {
  double hi, lo;
};

__device__ __forceinline__ dd two_sum(double a, double b) {
  double s = __dadd_rn(a, b);
  double bb = __dsub_rn(s, a);
  double e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
  return {s, e};
}

// TwoSum in binary32: returns s = fl(a + b) and sets *e with s + *e = a + b exactly
__device__ __forceinline__ float two_sum_f(float a, float b, float* e) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  *e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return s;
}

__device__ __forceinline__ dd fast_two_sum(double a, double b) {  // |a| >= |b| or a == 0
  double s = __dadd_rn(a, b);
  return {s, __dsub_rn(b, __dsub_rn(s, a))};
}

__device__ __forceinline__ dd two_prod(double a, double b) {
  double p = __dmul_rn(a, b);
  return {p, __fma_rn(a, b, -p)};
}

// dd + dd with both the high and the low parts summed error-free
__device__ __forceinline__ dd dd_add(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi);
  dd t = two_sum(a.lo, b.lo);
  s = fast_two_sum(s.hi, __dadd_rn(s.lo, t.hi));
  return fast_two_sum(s.hi, __dadd_rn(s.lo, t.lo));
}

__device__ __forceinline__ double rcp_approx(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  return r;
}

// binary32 approximate reciprocal (flushes subnormal inputs and results to zero); the screen
// of the bisection refines it by one Newton step, after which any seed within 2^-14 relative
// gives the reciprocal within 1.07 2^-24
__device__ __forceinline__ float rcp_approx_f32(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// 1/x within one ulp for |x| in [2^-1020, 2^1021) (see the file comment); no range handling.
__device__ __forceinline__ double rcp_nr(double x) {
  double r0 = rcp_approx(x);
  double e = __fma_rn(-x, r0, 1.0);
  double p = __fma_rn(e, e, e);
  return __fma_rn(r0, p, r0);
}

// the exponent field of x lies in [1023-1020, 1023+1020]: rcp_nr is within one ulp
__device__ __forceinline__ bool rcp_in_range(double x) {
  unsigned ex = (unsigned)(__double_as_longlong(x) >> 52) & 0x7ffu;
  return ex - 3u <= 2040u;
}

// A normalised weight zeta (max|zeta| in [1/2, 1)) with zeta^2 below the normal range of
// binary64 (|zeta| < 2^-511) is a zero weight: its square, the only form in which the secular
// function sees it, is not representable, and deflating it changes A = D + rho z z^T by less
// than 2^-510 rho ||z||.
__device__ __forceinline__ bool zero_weight(double z) { return fabs(z) < 0x1p-511; }

// IEEE quotient for the rare out-of-range operands; kept out of line so that the compiler
// does not evaluate it speculatively next to every fast reciprocal
static __device__ __noinline__ double rcp_ieee(double x) { return 1.0 / x; }

// 1/x within one ulp for every x (the IEEE quotient outside the fast range)
__device__ __forceinline__ double rcp(double x) { return rcp_in_range(x) ? rcp_nr(x) : rcp_ieee(x); }

// dd / dd to about 2^-104 relative: q1 = a.hi/b.hi, then one correction digit from the
// exact residual a.hi - q1 b.hi (fma), the low parts and the divisor's reciprocal.
__device__ __forceinline__ dd dd_div(dd a, dd b) {
  double r = rcp(b.hi);
  double q1 = __dmul_rn(a.hi, r);
  // make q1 faithful so that the fma residual below is exact
  double res = __fma_rn(-q1, b.hi, a.hi);
  q1 = __fma_rn(res, r, q1);
  res = __fma_rn(-q1, b.hi, a.hi);                       // exact
  double rest = __dadd_rn(res, __fma_rn(-q1, b.lo, a.lo));
  double q2 = __dmul_rn(rest, r);
  return fast_two_sum(q1, q2);
}

__device__ __forceinline__ double dd_to_double(dd a) { return __dadd_rn(a.hi, a.lo); }

// A lane group is L consecutive lanes of a warp (L = 8, 16 or 32; gm is its lane mask, so
// groups of one warp may run different iterations independently), or the whole thread
// block (L = 64, 128 or 256 = blockDim.x; gm unused), whose reductions go through shared
// memory between two block barriers and sum the warp partials in warp order, so every
// thread again holds the bit-identical total.
template <int L>
__device__ __forceinline__ unsigned group_mask() {
  if (L >= 32) return FULL;
  return ((1u << (L & 31)) - 1u) << ((threadIdx.x & 31) & ~(L - 1));
}

template <int L>
__device__ __forceinline__ double group_sum(double v, unsigned gm) {
  constexpr int W = L < 32 ? L : 32;
#pragma unroll
  for (int o = W / 2; o > 0; o >>= 1) v = __dadd_rn(v, __shfl_xor_sync(gm, v, o));
  if constexpr (L > 32) {
    __shared__ double part[L / 32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
    __syncthreads();
    v = part[0];
#pragma unroll
    for (int t = 1; t < L / 32; t++) v = __dadd_rn(v, part[t]);
    __syncthreads();
  }
  return v;
}

// The same sum in binary32 (every lane gets the identical total: the xor tree adds the same two
// operands in both lanes of a pair, and the block path sums the warp partials in warp order).
// Each of the tree_roundings<L>() additions rounds once by at most 2^-24 of its result.
template <int L>
__device__ __forceinline__ float group_sum_f(float v, unsigned gm) {
  constexpr int W = L < 32 ? L : 32;
#pragma unroll
  for (int o = W / 2; o > 0; o >>= 1) v = __fadd_rn(v, __shfl_xor_sync(gm, v, o));
  if constexpr (L > 32) {
    __shared__ float part[L / 32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
    __syncthreads();
    v = part[0];
#pragma unroll
    for (int t = 1; t < L / 32; t++) v = __fadd_rn(v, part[t]);
    __syncthreads();
  }
  return v;
}

// The sum of the pairs hi + lo of binary32 numbers: each level adds the high parts by TwoSum
// (exact: its error is the same in both lanes of a pair) and the low parts and that error with
// two roundings, each at most 2^-24 of the low part; identical total in every lane.
template <int L>
__device__ __forceinline__ void group_sum2_f(float* hi, float* lo, unsigned gm) {
  constexpr int W = L < 32 ? L : 32;
  float h = *hi, l = *lo;
#pragma unroll
  for (int o = W / 2; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(gm, h, o), ol = __shfl_xor_sync(gm, l, o);
    float e;
    const float s = __fadd_rn(h, oh);
    const float bb = __fsub_rn(s, h);
    e = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(oh, bb));
    h = s;
    l = __fadd_rn(__fadd_rn(l, ol), e);
  }
  if constexpr (L > 32) {
    __shared__ float ph[L / 32], pl[L / 32];
    if ((threadIdx.x & 31) == 0) { ph[threadIdx.x >> 5] = h; pl[threadIdx.x >> 5] = l; }
    __syncthreads();
    h = ph[0];
    l = pl[0];
#pragma unroll
    for (int t = 1; t < L / 32; t++) {
      const float s = __fadd_rn(h, ph[t]);
      const float bb = __fsub_rn(s, h);
      const float e = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(ph[t], bb));
      h = s;
      l = __fadd_rn(__fadd_rn(l, pl[t]), e);
    }
    __syncthreads();
  }
  *hi = h;
  *lo = l;
}

// roundings on the path of group_sum from one lane's value to the total
template <int L>
__host__ __device__ constexpr int tree_roundings() {
  int t = 0;
  for (int o = (L < 32 ? L : 32) / 2; o > 0; o >>= 1) t++;
  return L > 32 ? t + L / 32 - 1 : t;
}

template <int L>
__device__ __forceinline__ dd group_sum_dd(dd v, unsigned gm) {
  constexpr int W = L < 32 ? L : 32;
#pragma unroll
  for (int o = W / 2; o > 0; o >>= 1) {
    dd w;
    w.hi = __shfl_xor_sync(gm, v.hi, o);
    w.lo = __shfl_xor_sync(gm, v.lo, o);
    v = dd_add(v, w);
  }
  if constexpr (L > 32) {
    __shared__ double ph[L / 32], pl[L / 32];
    if ((threadIdx.x & 31) == 0) { ph[threadIdx.x >> 5] = v.hi; pl[threadIdx.x >> 5] = v.lo; }
    __syncthreads();
    v.hi = ph[0]; v.lo = pl[0];
#pragma unroll
    for (int t = 1; t < L / 32; t++) v = dd_add(v, dd{ph[t], pl[t]});
    __syncthreads();
  }
  return v;
}

template <int L>
__device__ __forceinline__ double group_max(double v, unsigned gm) {
  constexpr int W = L < 32 ? L : 32;
#pragma unroll
  for (int o = W / 2; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(gm, v, o));
  if constexpr (L > 32) {
    __shared__ double part[L / 32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
    __syncthreads();
    v = part[0];
#pragma unroll
    for (int t = 1; t < L / 32; t++) v = fmax(v, part[t]);
    __syncthreads();
  }
  return v;
}

template <int L>
__device__ __forceinline__ bool group_any(bool b, unsigned gm) {
  if constexpr (L > 32) return __syncthreads_or(b) != 0;
  else return __any_sync(gm, b) != 0;
}

__device__ __forceinline__ uint64_t dbits(double a) { return (uint64_t)__double_as_longlong(a); }

// neighbouring binary64 numbers of a finite x
__device__ __forceinline__ double dnext_up(double x) {
  if (x == 0.0) return __longlong_as_double(1ll);
  long long b = __double_as_longlong(x);
  return __longlong_as_double(x > 0.0 ? b + 1 : b - 1);
}
__device__ __forceinline__ double dnext_down(double x) { return -dnext_up(-x); }
__device__ __forceinline__ double dfrom(uint64_t u) { return __longlong_as_double((long long)u); }

// a flag store that orders this thread's earlier writes before it, and a load that orders this
// thread's later reads after it (device scope): with them, a thread that sees the flag sees the
// data written before it
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

}  // namespace dpr1
