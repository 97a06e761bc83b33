// dpr1_internal.cuh -- host/device structures shared by the library's translation units.
#pragma once
#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/dpr1.h"

// resident blocks per SM that the solve kernels' register budget is compiled for (and their
// default launch and stored-element buffers are sized for)
#ifndef DPR1_SOLVE_MIN_BLOCKS
#define DPR1_SOLVE_MIN_BLOCKS 4
#endif
// the shift test's sign from the binary32 pass where its bound decides it
#ifndef DPR1_SHIFT32
#define DPR1_SHIFT32 1
#endif
// lane groups of a solve kernel that find its queue empty write the eigenvector rows of the
// eigenvalues solved so far (one problem of order above 2048, with eigenvectors)
#ifndef DPR1_TAIL_ROWS
#define DPR1_TAIL_ROWS 1
#endif

namespace dpr1 {

constexpr bool kTailRows = DPR1_TAIL_ROWS != 0;

// Views into the caller's workspace for one problem (see ws_layout).
struct Ws {
  unsigned* hdr;       // 64 words: status and counters
  unsigned* status;    // hdr[0]: ST_* bits
  unsigned* counters;  // hdr[8..]: see the C_* indices
  unsigned long long* counters64;  // hdr[24..25]: the solve queue
  int* nred;           // [P]: order of each reduced (deflated) problem
  int* ndefl;          // [P]: deflated pairs of each problem
  unsigned* pst;       // [P]: PT_* bits of each problem
  int* owner;          // [total]: problem of each element (batch only)
  double *dr, *zr, *zz, *zl;  // reduced problem: d, z, z^2 = zz + zl exactly
  double *sig, *mu;           // eigenvalue pairs of the reduced problem
  int *shift, *flag, *list;   // pole index (-1: non-pole shift), remedy flag, work lists
  double* lamz;               // eigenvalue from A^{-1} (NaN: not recomputed)
  int* src;                   // deflation: reduced index feeding position p (-1: none)
  double* coef;               // deflation: zeta_p / zeta_survivor
  int *rpos, *dpos;           // output rows of reduced / deflated pairs
  int* gst;                   // first position of p's group of equal poles
  double *rprev, *rcur;       // Givens chain prefix norms
  int* dlist;                 // deflated positions, increasing
  int* zlist;                 // near-zero candidates
  double* fixinfo;            // per flagged slot: K_nu, K_nu at the other pole, distance ratio
  int* pexp;                  // [2P]: exponents (a, b) of the normalisation D' = 2^-a D, z' = 2^-b z
  double* prho;               // [P]: rho' = 2^(2b - a) rho
  double* pzsum;              // [P]: sum_j |zeta'_j| (for K_z of Eq. (knu2))
  // elements of the inverse for the secular evaluations (k_solve, k_fix): lane group g < term_slots owns
  // TERM_BYTES term_n bytes at terms + 4 g term_n and uses them for problems of order n <= term_n:
  // n doubles Delta_j, n doubles zz_j / Delta_j, then their binary32 copies and the low parts of
  // the pairs (n floats each);
  // nullptr: every evaluation forms them from dr and zz
  double* terms;
  int64_t term_n;
  int64_t term_slots;
  // eigenvector rows written by the solve kernel's lane groups once its queue is empty (one
  // problem without deflation): vstate[g] 0 unsolved, 1 solved, 2 row written; vrow[4 g ..]
  // the sigma, mu, ||x|| (scaled) and scale it was formed with; nullptr: k_vectors writes every row
  double* vrow;
  unsigned* vstate;
};

struct Options {
  double T_Knu, T_zero;
  int lanes, warps, bps, cap;
  bool warps_auto;   // warps per block of the solve kernel left to the library
  bool bps_auto;     // and its blocks per SM
  void* const* events;
  bool fast;   // accelerated solve instead of bisection
  int dd_mode;       // corner b: 1 double-double when kappa_nu > T_kappa n, 2 always
  double T_kappa;
  bool screen;       // binary32 screen of the bisection steps (same results)
};

// hdr counters (Ws::counters index; 16 and 17 are hdr[24..25], the solve queue)
enum : int {
  C_FIX_N = 1, C_FIX_Q = 2, C_ZERO_N = 3, C_EVAL_SOLVE = 4, C_EVAL_FIX = 5,
  C_R2 = 6, C_R1 = 7, C_SOLVED = 8, C_DEFL = 9, C_DD = 10, C_SCREEN = 11, C_R2DD = 12,
  C_SCREEN_NEAR = 13, C_SCREEN_DF = 14, C_INFER = 18, C_PROBE = 19, C_SHIFT32 = 20, C_TROW = 21,
  C_TAILROWS = 22, C_VECROWS = 23
};

// per-problem bits (Ws::pst)
enum : unsigned {
  PT_TRIVIAL = 1u,     // rho == 0
  PT_DEFLATE = 2u,     // a zero weight or equal poles
  PT_ZERO_POLE = 4u,   // some d_j == 0 (the near-zero recompute is then skipped, Eq. (gamma))
  PT_RANGE = 8u,       // rho' outside the normal range: skipped (solved as rho = 0) and reported
};

// bytes per element of a lane group's buffer: Delta_j, zz_j / Delta_j (binary64), their binary32
// copies (the binary32 screen's) and the low parts of the pairs (the double-float screen's)
constexpr size_t TERM_BYTES = 32;

size_t ws_layout(int64_t n, Ws* w, char* base);
size_t term_bytes(int64_t total, int64_t nprob);
Options resolve(const dpr1_options* o);
int sm_count();

}  // namespace dpr1
