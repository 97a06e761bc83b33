/*
 * dpr1.h -- C ABI of the GB300 (sm_103a) forward-stable eigensolver for
 * diagonal-plus-rank-one (DPR1) matrices
 *
 *     A = D + rho z z^T,  D = diag(d_1, ..., d_n),  d_1 >= d_2 >= ... >= d_n,  rho >= 0,
 *
 * after N. Jakovcevic Stor, I. Slapnicar, J. L. Barlow, "Forward stable eigenvalue
 * decomposition of rank-one modifications of diagonal matrices" (arXiv 1405.7537).
 * Each eigenpair (lambda_k, v_k) is computed independently (Algorithm 1, dpr1eig):
 * shift to the nearer pole d_i of lambda_k, form the arrowhead inverse of A - d_i I
 * (Eq. (invAi)) with its corner element b (Eq. (b_ob)) in double-double, bisect its
 * secular equation (Eq. (secAi)) for the extreme eigenvalue nu, recover
 * lambda_k = d_i + 1/nu (Eq. (8)) and v_k = x / ||x||, x = (D - lambda_k I)^{-1} z
 * (Eq. (Aeigenvec), (eigenvecAi)); apply the remedies R1/R2 when K_nu (Eq. (K0)) is
 * large, and recompute lambda_k from A^{-1} (Eq. (gamma)) when it is much closer to
 * zero than to its poles.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Working precision is IEEE binary64.  All array arguments are DEVICE pointers
 *   owned by the caller, unless a parameter says "host".  The library allocates no
 *   memory: it works in the caller's workspace, sized by dpr1_workspace_size*().
 * - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy default
 *   stream).  The return value reports argument errors found on the host and launch
 *   failures.  Conditions found on the device (unsorted or non-finite input, an
 *   iteration cap reached) are recorded in a status word inside the workspace;
 *   dpr1_stream_status() synchronises the stream and returns it.
 * - Output order: lambda_1 >= lambda_2 >= ... (Eq. (interlace)); row k of Vt
 *   (Vt[k*ldv + j], 0-based) is v_k with the paper's sign, v = x / ||x||.
 * - Each eigenvalue is also returned as the unevaluated pair (sigma_k, mu_k),
 *   lambda_k = sigma_k + mu_k exactly in real arithmetic (the representation of
 *   Example 2): sigma_k is the shift (a pole, or a non-pole shift chosen by R2) and
 *   mu_k the computed eigenvalue of A - sigma_k I.  Components of v_k are formed as
 *   zeta_j / ((d_j - sigma_k) - mu_k).
 * - Deflation (Sec. 1): zeta_j == 0 gives the eigenpair (d_j, e_j); d_j == d_{j+1}
 *   gives the eigenvalue d_j after a Givens rotation in the (j, j+1) plane.  Both are
 *   exact tests.  A weight whose square, after the normalisation below, is not a normal
 *   binary64 number (|zeta_j| < 2^(b - 511), max|zeta| = m 2^b with m in [1/2, 1)) counts as
 *   zero: the secular function only sees zeta_j^2, and dropping it changes A by less than
 *   2^-510 rho ||z||.  Deflated pairs carry sigma = lambda, mu = 0.
 * - Normalisation: each problem is solved as A = 2^a (D' + rho' z' z'^T) with the exact
 *   powers of two D' = 2^-a D (max|d_j| = m 2^a), z' = 2^-b z and rho' = 2^(2b - a) rho, and
 *   the results are scaled back.  In the normal range this changes no rounding; it lets data
 *   of any magnitude through.  An eigenpair that still needs values outside the binary64
 *   range (mu below 2^-1022 in the normalised units: the eigenvalue closer to its pole than
 *   binary64 can resolve with full precision; or rho' itself outside the normal range) is
 *   reported as DPR1_ERR_RANGE, never returned silently.
 * - The functions never throw, never exit and never wait on the device except in
 *   dpr1_stream_status().
 */
#ifndef DPR1_H
#define DPR1_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define DPR1_API __attribute__((visibility("default")))
#else
#define DPR1_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* dpr1_stream_t; /* identical to cudaStream_t */

typedef enum {
  DPR1_OK = 0,
  DPR1_ERR_ARG = 1,            /* bad size, stride or NULL pointer (host check) */
  DPR1_ERR_UNSORTED = 2,       /* d is not non-increasing (device check) */
  DPR1_ERR_RHO = 3,            /* rho < 0 or not finite (host check); use A -> -(-D - rho z z^T) */
  DPR1_ERR_NONFINITE = 4,      /* d, z or a gradient holds Inf/NaN (device check) */
  DPR1_ERR_NOT_CONVERGED = 5,  /* a bisection did not close within its iteration cap (device) */
  DPR1_ERR_CUDA = 6,           /* a CUDA launch or runtime call failed */
  DPR1_ERR_WORKSPACE = 7,      /* workspace NULL, misaligned (256 B) or smaller than required */
  DPR1_ERR_RANGE = 8           /* an eigenpair needs values outside the binary64 range (device) */
} dpr1_status;

/* Tunables; pass NULL for the defaults (dpr1_default_options). */
typedef struct {
  double T_Knu;          /* remedies when K_nu > T_Knu (default 16) */
  double T_zero;         /* near-zero recompute when T_zero |lambda| < distance to its poles (64) */
  int lanes;             /* threads per eigenvalue in the solve kernels: 0 = auto, else 8, 16 or 32 */
  int warps_per_block;   /* 0 = auto */
  int blocks_per_sm;     /* 0 = auto (up to 4 blocks of the solve kernel per SM), else 1..8 */
  int max_bisect;        /* iteration cap per bisection (default 96; 1..4096 accepted, other values
                            give the default).  A bisection phase that reaches it stops and the
                            call reports DPR1_ERR_NOT_CONVERGED; bisection to adjacent doubles
                            needs up to 64 steps, so caps below 64 serve to test that path.  The
                            accelerated solve may take cap + cap/3 evaluations. */
  void* const* phase_events; /* instrumentation: NULL, or 4 cudaEvent_t recorded on `stream`
                                before the bisection kernel, after it, after the remedies and
                                after the eigenvector kernel */
  int zero_finder;       /* 0 (default): bisection of the arrowhead secular function, as
                            Algorithm 1 states; 1: the accelerated bracketed solve (a
                            rational model with the nearest pole, fitted to the value and
                            slope, kept inside the bisection bracket; the fast zero finder
                            alternative of Sec. 2.2).  Both stop at the
                            adjacent pair of doubles across the sign change. */
  int dd_mode;           /* the corner b of Eq. (b_ob): 1 (default) in double the working
                            precision when kappa_nu of Eq. (knu2) exceeds T_kappa * n, as
                            Algorithm 1 does, else in binary64; 2: always in double-double */
  double T_kappa;        /* "kappa_nu >> O(n)": double-double when kappa_nu > T_kappa * n (1500) */
  int screen;            /* 1 (default): a bisection step whose sign a binary32 evaluation of the
                            stored elements settles with a rigorous error bound -- the sign the
                            binary64 evaluation would give -- skips the binary64 evaluation, so
                            the results are the same bits as with 0 (every step in binary64) */
} dpr1_options;

DPR1_API void dpr1_default_options(dpr1_options* opt);

/* Human-readable name of a status code (static storage). */
DPR1_API const char* dpr1_status_string(dpr1_status s);

/*
 * Bytes of workspace for dpr1_eig on a problem of order n (the workspace must be
 * 256-byte aligned; its contents need not be initialised).  The size includes, at the end,
 * one buffer of 32n bytes per lane group of the solve kernel's default launch on the
 * current device (32 groups per SM for n > 384): there each group stores the elements of
 * the inverse of its shifted matrix, Delta_j = d_j - d_i and zeta_j^2 / Delta_j of Eq. (invAi),
 * once per eigenvalue (in binary64 and as pairs of binary32 numbers for the screens of the
 * bisection steps), and every bisection step reads them instead of forming them again.
 * For n > 2048 it also includes 36n bytes (and 256 of alignment) after the buffers, where
 * the solve kernel's lane groups that find its queue empty record the eigenvector rows they
 * write (Eq. (eigenvecAi)) for the eigenvalues solved by then.
 * These parts are optional: a smaller workspace is accepted down to the part without
 * them (every evaluation of the secular function then forms the elements again, with the same accuracy
 * bound, and the eigenvector kernel writes every row); below that part the call returns
 * DPR1_ERR_WORKSPACE.  The row records change no bit of the results; without the buffers the
 * sums group their terms differently, so a result may differ in its last bits, within the bound.
 */
DPR1_API size_t dpr1_workspace_size(int64_t n);

/*
 * dpr1_eig -- all eigenpairs of one DPR1 matrix (Algorithm 1 for k = 1..n).
 *
 *   n        order (n >= 0; n == 0 is a no-op)
 *   d, z     device double[n]; d non-increasing, any z (zeros and ties are deflated, and so is
 *            a weight below 2^-511 relative to the largest, see above)
 *   rho      rho >= 0 (rho == 0 gives lambda = d, V = I)
 *   lambda   device double[n], out: eigenvalues, non-increasing
 *   Vt       device double[n*ldv] or NULL, out: row k = v_k (ldv >= n)
 *   sigma,mu device double[n] or NULL, out: lambda_k = sigma_k + mu_k
 *   xnorm    device double[n] or NULL, out: ||x_k||_2, x_k = (D - lambda_k I)^{-1} z
 *   workspace, workspace_bytes: see dpr1_workspace_size
 *   opt      NULL or tunables
 *   stream   CUDA stream
 * Errors: DPR1_ERR_ARG, DPR1_ERR_RHO, DPR1_ERR_WORKSPACE, DPR1_ERR_CUDA synchronously;
 * DPR1_ERR_UNSORTED, DPR1_ERR_NONFINITE, DPR1_ERR_RANGE, DPR1_ERR_NOT_CONVERGED via
 * dpr1_stream_status.
 */
DPR1_API dpr1_status dpr1_eig(int64_t n, const double* d, const double* z, double rho,
                     double* lambda, double* Vt, int64_t ldv,
                     double* sigma, double* mu, double* xnorm,
                     void* workspace, size_t workspace_bytes,
                     const dpr1_options* opt, dpr1_stream_t stream);

/*
 * Bytes of workspace for dpr1_eig_batched on nprob problems with total_n eigenpairs in all.
 * As for dpr1_workspace_size, the size ends with optional buffers for the stored elements of
 * the inverse, here of order max(2048, 4 total_n / nprob) (at most total_n) per lane group; the
 * call divides whatever workspace lies beyond the required part among its lane groups, and
 * problems larger than a group's buffer form the elements at every evaluation.
 */
DPR1_API size_t dpr1_batched_workspace_size(int64_t nprob, int64_t total_n);

/*
 * dpr1_eig_batched -- all eigenpairs of nprob independent DPR1 problems of uneven sizes in
 * one launch sequence (no counterpart in the paper: divide-and-conquer merges produce
 * many such problems, Sec. 1).  Problem p occupies elements offs[p] .. offs[p+1]-1 of the
 * concatenated arrays d, z, lambda, sigma, mu, xnorm (n_p = offs[p+1] - offs[p], any n_p
 * >= 0), has weight rho[p], and its eigenvector block is Vt + voffs[p], an n_p x n_p
 * row-major matrix whose row k is v_k.  Every eigenpair of every problem is one work item
 * of the same persistent kernels (Algorithm 1 per item), so small and large problems
 * share the GPU without per-problem launches.  The call launches a fixed number of
 * kernels and never synchronises, so the whole sequence can be captured in a CUDA graph.
 *
 *   nprob, total_n   problem count, offs[nprob] (host values, must match the device offsets)
 *   offs, voffs      device int64[nprob+1]; voffs may be NULL when Vt is NULL
 *   d, z, rho        device double[total_n], double[total_n], double[nprob]
 *   lambda, ...      outputs as dpr1_eig, concatenated per problem
 * Errors: as dpr1_eig; inconsistent offsets are reported as DPR1_ERR_ARG and a bad rho[p]
 * as DPR1_ERR_RHO through dpr1_stream_status.
 */
DPR1_API dpr1_status dpr1_eig_batched(int64_t nprob, int64_t total_n, const int64_t* offs, const int64_t* voffs,
                                      const double* d, const double* z, const double* rho,
                                      double* lambda, double* Vt, double* sigma, double* mu, double* xnorm,
                                      void* workspace, size_t workspace_bytes,
                                      const dpr1_options* opt, dpr1_stream_t stream);

/*
 * Bytes of workspace for dpr1_eig_backward on order n (256-byte aligned, uninitialised):
 * three rows of n doubles (partial rows of the gradients of d and z, and the current row's
 * reciprocals) for each of 1064, 2128 or 3192 warps (n <= 8192, <= 24576, above).
 */
DPR1_API size_t dpr1_backward_workspace_size(int64_t n);

/*
 * dpr1_eig_backward -- adjoint of (lambda, V) with respect to (d, z, rho).  No
 * counterpart in the paper: it differentiates the secular equation f(lambda_k) = 0
 * (Eq. (Pick)) implicitly and the eigenvector formula x_k = (D - lambda_k I)^{-1} z,
 * v_k = x_k / ||x_k|| (Eq. (Aeigenvec)) explicitly; the eigenvectors are recomputed from
 * the pairs (sigma_k, mu_k) that dpr1_eig returned, V is not needed.
 *
 *   n, d, z, rho     the forward problem (irreducible: no zero zeta_j, no equal d_j)
 *   sigma, mu        device double[n] from dpr1_eig
 *   grad_lambda      device double[n] or NULL (zero): dL/dlambda_k
 *   grad_Vt, ldg     device double[n*ldg] or NULL (zero): row k = dL/dv_k
 *   grad_d, grad_z   device double[n], out (overwritten)
 *   grad_rho         device double[1], out
 * The sum over eigenpairs is done in a fixed order: results are reproducible.  The problem
 * is normalised by exact powers of two as in dpr1_eig and the gradients are scaled back
 * (in the normal range this changes no rounding).
 * Errors as dpr1_eig; a non-finite intermediate (e.g. a deflated input) is reported as
 * DPR1_ERR_NONFINITE through dpr1_stream_status on this workspace.
 */
DPR1_API dpr1_status dpr1_eig_backward(int64_t n, const double* d, const double* z, double rho,
                                       const double* sigma, const double* mu,
                                       const double* grad_lambda, const double* grad_Vt, int64_t ldg,
                                       double* grad_d, double* grad_z, double* grad_rho,
                                       void* workspace, size_t workspace_bytes,
                                       const dpr1_options* opt, dpr1_stream_t stream);

/*
 * Bytes of workspace for dpr1_eig_hermitian on order n (256-byte aligned, uninitialised).
 */
DPR1_API size_t dpr1_hermitian_workspace_size(int64_t n);

/*
 * dpr1_eig_hermitian -- all eigenpairs of the complex Hermitian DPR1 matrix A = D + rho z z^*
 * (the extension of Algorithm 1 to the Hermitian case that the paper states after it).
 * With z_j = |z_j| phi_j, |phi_j| = 1, A = Phi (D + rho |z| |z|^T) Phi^*, Phi = diag(phi): the
 * eigenvalues are those of the real DPR1 matrix with weights |z_j| (computed by the dpr1_eig
 * path) and v_k = Phi u_k = (D - lambda_k I)^{-1} z / ||.|| (Eq. (Aeigenvec) with complex z).
 *
 *   n, d, rho  as dpr1_eig (d real, non-increasing; rho >= 0)
 *   z          device complex double[n], interleaved (re, im), 16-byte aligned
 *   lambda, sigma, mu, xnorm   as dpr1_eig (real)
 *   Vt         device complex double[n*ldv] (interleaved, 16-byte aligned) or NULL; out: row k
 *              = v_k; ldv >= n counts complex entries
 *   workspace  dpr1_hermitian_workspace_size(n) bytes, 256-byte aligned; its first part is a
 *              dpr1_eig workspace, so dpr1_stream_status(workspace, stream) reports the
 *              device-detected conditions
 * Errors: as dpr1_eig (a non-finite re or im part gives DPR1_ERR_NONFINITE); a misaligned z or
 * Vt is DPR1_ERR_ARG.
 */
DPR1_API dpr1_status dpr1_eig_hermitian(int64_t n, const double* d, const double* z, double rho,
                                        double* lambda, double* Vt, int64_t ldv,
                                        double* sigma, double* mu, double* xnorm,
                                        void* workspace, size_t workspace_bytes,
                                        const dpr1_options* opt, dpr1_stream_t stream);

/*
 * Bytes of workspace for dpr1_tridiag_eig on order n (256-byte aligned, uninitialised):
 * about 22 n^2 bytes (the eigenvector blocks of two tree depths, the DPR1 eigenvectors of
 * one depth) plus O(n).
 */
DPR1_API size_t dpr1_tridiag_workspace_size(int64_t n);

/*
 * dpr1_tridiag_eig -- all eigenpairs of the symmetric tridiagonal matrix T with diagonal a
 * and off-diagonal b, by divide and conquer whose merges are DPR1 eigenproblems (Sec. 1:
 * divide and conquer is where DPR1 problems arise), each tree depth's merges solved by one
 * dpr1_eig_batched launch sequence (Algorithm 1 per eigenpair).  The tree halves down to
 * single indices; the tear at a split m is rho v v^T with rho = |b_{m-1}| >= 0 and
 * v = e_{m-1} + sign(b_{m-1}) e_m.  Eigenvector blocks are formed by binary64 products on
 * the GPU (no library GEMM).
 *
 *   n          order (n >= 0; n == 0 is a no-op)
 *   a, b       device double[n], double[n-1] (b may be NULL for n == 1)
 *   lambda     device double[n], out: eigenvalues, non-increasing
 *   Qt         device double[n*ldq] or NULL (eigenvalues only), out: row k = eigenvector k
 *   workspace  dpr1_tridiag_workspace_size(n) bytes, 256-byte aligned; dpr1_stream_status on
 *              it reports the device-detected conditions of all merge levels
 *   opt        NULL or tunables of the DPR1 solves (zero_finder, lanes, ...)
 * Errors: DPR1_ERR_ARG, DPR1_ERR_WORKSPACE, DPR1_ERR_CUDA synchronously; DPR1_ERR_NONFINITE,
 * DPR1_ERR_NOT_CONVERGED through dpr1_stream_status.
 */
DPR1_API dpr1_status dpr1_tridiag_eig(int64_t n, const double* a, const double* b, double* lambda,
                                      double* Qt, int64_t ldq, void* workspace, size_t workspace_bytes,
                                      const dpr1_options* opt, dpr1_stream_t stream);

/*
 * Bytes of workspace for dpr1_arrow_eig with n poles (256-byte aligned, uninitialised).  As
 * for dpr1_workspace_size, it ends with optional buffers in which the solves store the
 * elements of the inverse of each shifted matrix once per eigenvalue; a workspace down to
 * the part without them is accepted.
 */
DPR1_API size_t dpr1_arrow_workspace_size(int64_t n);

/*
 * dpr1_arrow_eig -- all n + 1 eigenpairs of the real symmetric arrowhead matrix
 * A = [D z; z^T alpha], D = diag(d), the companion problem the paper relates its method to
 * (Sec. 1), by the steps of Algorithm 1 on the shifted inverse: (A - d_i I)^{-1} is again an
 * arrowhead, with the corner b = (1/zeta_i^2)(sum_{j != i} zeta_j^2/(d_j - d_i) - (alpha - d_i))
 * formed in double-double and one more pole, at 0, of weight 1/zeta_i^2; lambda = d_i + 1/nu
 * for its extreme eigenvalue nu (bisection, or the accelerated solve with opt->zero_finder),
 * v = [x; -1] / ||.||, x = (D - lambda I)^{-1} z.  As in dpr1_eig, an eigenvalue whose K_nu
 * (Eq. (K0)) exceeds opt->T_Knu is recomputed at the other neighbouring pole (R1) or at a
 * non-pole shift sigma next to it (R2, Sec. 2), where (A - sigma I)^{-1} =
 * diag((D - sigma I)^{-1}, 0) + u u^T / f(sigma), u = [(D - sigma I)^{-1} z; -1],
 * f(sigma) = alpha - sigma - z^T (D - sigma I)^{-1} z in double-double, is a DPR1 matrix of
 * order n + 1; and an eigenvalue much closer to zero than to its neighbouring poles
 * (T_zero |lambda| < distance) is recomputed from A^{-1} (sigma = 0) when no pole is zero.
 *
 *   n          number of poles (n >= 0; the matrix has order n + 1)
 *   d, z       device double[n]: d strictly decreasing, every |z_j| >= 2^(a - 511) with
 *              max(|d_j|, |z_j|, |alpha|) = m 2^a, m in [1/2, 1) (the matrix is irreducible;
 *              deflate equal poles and zero weights before the call).  The matrix is solved
 *              as 2^a (2^-a A), an exact normalisation, as dpr1_eig does
 *   alpha      the corner entry
 *   lambda     device double[n+1], out: eigenvalues, non-increasing; they interlace d
 *   Vt         device double[(n+1)*ldv] or NULL, out: row k = v_k (n + 1 entries, ldv >= n + 1)
 *   sigma, mu  device double[n+1] or NULL, out: the shift sigma_k (a pole, or the R2 shift)
 *              and mu_k = 1/nu; lambda_k = sigma_k + mu_k except for an eigenvalue
 *              recomputed from A^{-1}, and v_k is formed from (sigma_k, mu_k)
 *   xnorm      device double[n+1] or NULL, out: ||[x; -1]||
 *   workspace  dpr1_arrow_workspace_size(n) bytes, 256-byte aligned; dpr1_workspace_stats
 *              reads its counters like those of dpr1_eig
 * Errors: DPR1_ERR_ARG, DPR1_ERR_WORKSPACE, DPR1_ERR_CUDA synchronously; through
 * dpr1_stream_status: DPR1_ERR_ARG (equal poles or a zero weight), DPR1_ERR_UNSORTED,
 * DPR1_ERR_NONFINITE, DPR1_ERR_RANGE, DPR1_ERR_NOT_CONVERGED.
 */
DPR1_API dpr1_status dpr1_arrow_eig(int64_t n, const double* d, const double* z, double alpha,
                                    double* lambda, double* Vt, int64_t ldv,
                                    double* sigma, double* mu, double* xnorm,
                                    void* workspace, size_t workspace_bytes,
                                    const dpr1_options* opt, dpr1_stream_t stream);

/*
 * Synchronises `stream` and returns the status the device recorded in `workspace`
 * during the last call that used it (DPR1_OK if none), then clears it.
 */
DPR1_API dpr1_status dpr1_stream_status(void* workspace, dpr1_stream_t stream);


/*
 * dpr1_eig_noalloc -- dpr1_eig without a caller-provided workspace.  The paper has no
 * counterpart: this is an interface for callers that cannot allocate device memory,
 * such as code running inside another framework's memory pool or a plugin that may
 * not grow the device footprint at run time.  The scratch memory is a static array
 * inside the library (640 KiB, held on every device that loads the library until the
 * process exits), so n is limited to DPR1_NOALLOC_MAX_N; larger n returns
 * DPR1_ERR_ARG without launching anything.  The call allocates nothing.
 *
 *   arguments     as dpr1_eig (same outputs, same conventions), without the workspace
 *   wait          0: asynchronous, like dpr1_eig (device-detected problems are then not
 *                 reported); non-zero: synchronise `stream` at the end and return the
 *                 device-detected status as dpr1_stream_status would
 *
 * The first call in each CUDA context of a device looks up the device address of the
 * static array (with that device current) and caches it under the context's unique ID;
 * make that first call before any stream capture.  If the context is destroyed and
 * rebuilt (cudaDeviceReset by the caller or by another library), the array's address
 * may change: the next call notices the new context and looks it up again, so a reset
 * invalidates nothing the caller holds for this entry point.  All calls
 * share the one array and it keeps the last call's contents (the call clears what must
 * start at zero).  Calls that overlap on the GPU -- on different streams or from
 * host threads without ordering -- race on it and give wrong results.
 */
#define DPR1_NOALLOC_MAX_N 4096
DPR1_API dpr1_status dpr1_eig_noalloc(int64_t n, const double* d, const double* z, double rho,
                                      double* lambda, double* Vt, int64_t ldv,
                                      double* sigma, double* mu, double* xnorm,
                                      const dpr1_options* opt, int wait, dpr1_stream_t stream);

/*
 * Instrumentation (no counterpart in the paper): synchronises `stream` and copies the
 * counters of the last dpr1_eig / dpr1_eig_batched / dpr1_arrow_eig call on `workspace` into
 * out[0..17]:
 *   0 eigenvalues solved by the bisection kernel, 1 eigenvalues flagged by K_nu,
 *   2 remedies taken with R1, 3 with R2, 4 secular-function evaluations in the bisection
 *   kernel, 5 evaluations in the remedy kernel, 6 eigenvalues recomputed from A^{-1},
 *   7 deflated pairs, 8 corners b formed in double-double by the bisection kernel,
 *   9 bisection steps (of those counted in 4 and 5) settled by the binary32 screen,
 *   10 R2 remedies that formed their shift in double the working precision (of those in 3),
 *   11 screened evaluations (bisection steps of 9 and probes of 14) whose screened value
 *   exceeded the screen's error bound by less than a factor 2, 12 screened evaluations (steps
 *   of 9 and probes of 14) settled by the double-float screen, 13 bisection steps (of those
 *   counted in 4 and 5) decided by bounds that screened probes certified, without an
 *   evaluation, 14 screened probes that placed those bounds (not counted in 4 and 5),
 *   15 shift tests of the bisection kernel whose sign the binary32 pass settled (the others
 *   take the binary64 pass), 16 eigenvector rows written by the bisection kernel's lane
 *   groups after its queue ran out (the eigenvector kernel writes the others), 17 eigenvector
 *   rows written by the eigenvector kernel (the others, and those of 16 whose pair a remedy or
 *   the near-zero path changed).  `out` holds 18 values.
 */
DPR1_API dpr1_status dpr1_workspace_stats(void* workspace, int64_t* out, dpr1_stream_t stream);

/*
 * Measurement helper (no counterpart in the paper): launches `blocks` x `threads`
 * threads that each run `iters` iterations of 8 independent binary64 fma chains
 * (8 * iters * blocks * threads fma in total) and write one double to sink[thread].
 * Timed by the caller, it gives the device's binary64 fma issue rate.
 */
DPR1_API dpr1_status dpr1_probe_dfma(int blocks, int threads, int iters, double* sink, dpr1_stream_t stream);

/*
 * Test hook (no counterpart in the paper): out[t] = the library's binary64
 * reciprocal of x[t] for t < count, as used in the secular sums.  Lets tests bound
 * its error against correctly rounded division.
 */
DPR1_API dpr1_status dpr1_probe_reciprocal(int64_t count, const double* x, double* out, dpr1_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* DPR1_H */
