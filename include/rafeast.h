/*
 * rafeast.h - C ABI of the GB300 (sm_103a) RA-FEAST hot path.
 *
 * RA-FEAST (arXiv 2512.01257) computes every eigenpair of a sparse symmetric
 * positive definite matrix A whose eigenvalue lies in [lmin, lmax] (Eq. 1):
 * a randomized warmstart (Algorithm 2, Phase 1) followed by FEAST subspace
 * iterations (Algorithm 1 / Algorithm 2, Phase 2). Each FEAST iteration
 * applies the quadrature projector of Eq. 3 by solving the complex symmetric
 * shifted systems (z_j I - A) X_j = Q for all N_c nodes at once with batched
 * COCG, accumulates Q~ = sum_j Re(w_j X_j), re-orthonormalises Q~ and runs a
 * Rayleigh-Ritz step.
 *
 * Conventions shared by every entry point:
 *  - A = L + diag_shift * I, where L is given in CSR form (int32 row_ptr[n+1],
 *    int32 col_idx[nnz], double values[nnz]) and must be symmetric. Keeping
 *    the shift out of the CSR keeps integer graph-Laplacian values exact when
 *    the mixed-precision path rounds them to float32.
 *  - Dense blocks (subspaces, eigenvectors, Omega) are column-major n x m
 *    arrays of double in the caller's row order: entry (i, k) is at
 *    ptr[k * n + i]. The library may reorder rows internally for locality;
 *    that never shows at this interface.
 *  - A pointer argument documented "device" must be a CUDA device pointer
 *    (or managed memory) on the handle's device; "host" means ordinary host
 *    memory. Inputs are copied or read; the caller keeps ownership of every
 *    buffer it passes and the library never frees it.
 *  - Every function returns an int status (RAFEAST_OK = 0; positive values
 *    are solver outcomes with valid outputs, negative values are errors with
 *    outputs unspecified). No function aborts the process or throws across
 *    the ABI. A handle is not thread safe; distinct handles may be used from
 *    distinct threads and streams.
 *  - Work is ordered after all prior work on the stream given to
 *    rafeast_create, and that stream is made to wait for the call's device
 *    work before the call returns. Calls with host outputs synchronise.
 */
#ifndef RAFEAST_H
#define RAFEAST_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes (in the spirit of FEAST's info output) ---------------- */
#define RAFEAST_OK 0
#define RAFEAST_NO_EIGENVALUE 1      /* no Ritz value inside [lmin, lmax]     */
#define RAFEAST_NO_CONVERGENCE 2     /* max_outer reached; best iterate out   */
#define RAFEAST_M0_TOO_SMALL 3       /* every Ritz value inside: m0 <= count  */
#define RAFEAST_ERR_INVALID_ARG (-1) /* bad size, pointer, CSR or parameter   */
#define RAFEAST_ERR_NOT_SYMMETRIC (-2)
#define RAFEAST_ERR_CUDA (-3)        /* a CUDA runtime call failed            */
#define RAFEAST_ERR_COCG_BREAKDOWN (-4)
#define RAFEAST_ERR_TIMEOUT (-5)     /* a bounded device wait ran out         */
#define RAFEAST_ERR_OUT_OF_MEMORY (-6)
#define RAFEAST_ERR_NOT_READY (-7)   /* e.g. START_SUBSPACE with no subspace  */
#define RAFEAST_ERR_CHOLESKY (-8)    /* Cholesky-QR failed even when shifted  */
#define RAFEAST_ERR_NO_DEVICE (-9)
#define RAFEAST_ERR_EXCHANGE (-10)   /* a sharded solve's sum callback failed */

/* ---- enums --------------------------------------------------------------- */
#define RAFEAST_FP64 0   /* every step in double                              */
#define RAFEAST_MIXED 1  /* shifted solves + their SpMM in float32; Gram,      *
                          * Cholesky-QR, Rayleigh-Ritz, residuals in double    *
                          * (the Gram of the first, preconditioning Cholesky-  *
                          * QR pass is summed in float; its products with the  *
                          * factor and the last pass stay double)              */

#define RAFEAST_FORM_DIRECT 0     /* COCG right-hand side Q (as printed)      */
#define RAFEAST_FORM_CORRECTION 1 /* COCG right-hand side A Q - Q diag(theta); *
                                   * X_j rebuilt as (Q + Y_j)/(z_j - theta):   *
                                   * the same X_j, with an inexact solve's    *
                                   * error proportional to the residual       */

#define RAFEAST_START_RANDOM 0   /* Algorithm 1: random orthonormal Q(0)      */
#define RAFEAST_START_SUBSPACE 1 /* the handle's subspace (warmstart / set)   */

#define RAFEAST_CREATE_NO_REORDER 1u      /* keep the caller's row order      */
#define RAFEAST_CREATE_FORCE_REORDER 2u   /* always apply the reordering      */
#define RAFEAST_CREATE_CHECK_SYMMETRY 4u  /* O(nnz) host check, -2 on failure */
#define RAFEAST_CREATE_RCM 8u             /* reverse Cuthill-McKee instead of *
                                           * the default recursive breadth-   *
                                           * first bisection                  */

/* option keys for rafeast_set_option */
#define RAFEAST_OPT_WARMSTART_MAP 1 /* 0 auto, 1 literal (A-lmin)/(lmax-lmin), *
                                     * 2 low-end (g I - A)/(g - lmin)          */
#define RAFEAST_OPT_CHUNK 2         /* COCG iterations per CUDA-graph replay   */
#define RAFEAST_OPT_AUTOTUNE 3      /* 1 (default) time SpMM shapes, 0 off     */
#define RAFEAST_OPT_LANES 4         /* force lanes per row (4,8,16,32), 0 auto */
#define RAFEAST_OPT_PROFILE 5       /* 1: time every COCG kernel in the graph  */
#define RAFEAST_OPT_KERNEL 6        /* COCG kernels: 0 auto (register gathers),*
                                     * 1 register gathers, 2 bulk-copy (TMA)   *
                                     * gathers (float32, N_c >= 2)             */
#define RAFEAST_OPT_MAXNZ 7         /* nonzeros per bulk-copy item (1..32)     */
#define RAFEAST_OPT_WAIT_LIMIT 8    /* clock cycles one device-side wait may   *
                                     * spin before the solve stops with        *
                                     * RAFEAST_ERR_TIMEOUT (default 2e9, ~1 s) */
#define RAFEAST_OPT_CPL 10          /* cap on subspace columns per lane in the *
                                     * register-gather kernels (0: automatic); *
                                     * a lower cap means narrower column       *
                                     * blocks, fewer registers, more warps     */
#define RAFEAST_OPT_SOLVER 11       /* shifted solves: 0 one COCG per shift,   *
                                     * 1 multi-shift COCG (one seed recurrence *
                                     * per column, other shifts from its       *
                                     * scalars; same iterates in exact         *
                                     * arithmetic)                              */
#define RAFEAST_OPT_UPDATE 12       /* multi-shift update kernel: 0 auto    *
                                     * (streamed), 1 gathered products (M p_k *
                                     * recomputed from gathered r and p), 2   *
                                     * streamed (the dot kernel stores M r_k, *
                                     * M p_k follows by its recurrence; no    *
                                     * gathers in the update). Batched solves *
                                     * follow the first handle's setting.     */
#define RAFEAST_OPT_VALUES_FREE 13  /* 0 (default): when the CSR part of A  *
                                     * is a unit-weight graph Laplacian (off- *
                                     * diagonal values -1, diagonal = degree) *
                                     * the multi-shift dot kernels gather on  *
                                     * its off-diagonal pattern alone, with   *
                                     * L r = deg r - sum of neighbours; 1:    *
                                     * always read the values                 */
#define RAFEAST_OPT_TILED 14        /* seed dot kernel of the multi-shift    *
                                     * float32 solve with the streamed update: *
                                     * 0 (default) tiled (row tiles whose      *
                                     * gathered rows are staged in shared      *
                                     * memory) when the matrix has tiles, the  *
                                     * autotuner choosing between it and the   *
                                     * register gathers; 1 register gathers    *
                                     * only; 2 tiled only (when it has tiles)  */
#define RAFEAST_OPT_TILE_CB 15      /* with RAFEAST_OPT_TILED = 2: column     *
                                     * pairs per block of the tiled dot kernel *
                                     * (4 or 8; 0 = autotuned)                 */
#define RAFEAST_OPT_DENSE 16        /* FP64 Gram matrices (Cholesky-QR,       *
                                     * Rayleigh-Ritz, rafeast_gram): 0 (default)*
                                     * on the tensor cores, FP64 values split   *
                                     * into exact BF16 digits with integer      *
                                     * accumulation (m <= 128); 1 on the FP64   *
                                     * pipe                                     */
#define RAFEAST_OPT_DEFER 17        /* float32 multi-shift solves with the    *
                                     * tiled dot kernel: 1 the update kernel   *
                                     * of step k leaves the shifted directions *
                                     * and their quadrature terms to the dot   *
                                     * kernel of step k + 1, which streams     *
                                     * them beside its gathers (residuals      *
                                     * ping-pong between two arrays); 0        *
                                     * (default) every update complete (the    *
                                     * deferred form moves more bytes and      *
                                     * measured slower)                        */
#define RAFEAST_OPT_TEST_STALL 9    /* test hook: bytes (multiple of 16) that  *
                                     * every bulk-copy stage waits for and no *
                                     * copy delivers, so the bounded wait     *
                                     * expires; 0 (default) disables it       */

typedef struct rafeast_ctx* rafeast_t;

/* Solver parameters (all host). Field order is part of the ABI. */
typedef struct rafeast_params {
  double lmin, lmax;     /* search interval, lmin < lmax                      */
  int32_t m0;            /* subspace size, 1..128, > eigenvalues inside       */
  int32_t nc;            /* quadrature nodes on the half contour, 1..16; one  *
                          * COCG per shift (RAFEAST_OPT_SOLVER = 0) runs up   *
                          * to 8, more run multi-shift with the streamed      *
                          * update                                            */
  double ellipse_ratio;  /* imaginary/real semi-axis ratio e, (0, 1]           */
  double solve_tol;      /* COCG: stop when ||r||_2 <= solve_tol * ||b||_2     */
  double outer_tol;      /* stop when max in-interval ||Av-lv||/||A||_1 <= tol */
  int32_t max_outer;     /* FEAST iterations cap (Algorithm 2: max_iter)       */
  int32_t max_inner;     /* COCG iterations cap per solve                      */
  int32_t precision;     /* RAFEAST_FP64 or RAFEAST_MIXED                      */
  int32_t solve_form;    /* RAFEAST_FORM_DIRECT or RAFEAST_FORM_CORRECTION     */
  int32_t start;         /* RAFEAST_START_RANDOM or RAFEAST_START_SUBSPACE     */
  int32_t reserved;      /* must be 0                                          */
  uint64_t seed;         /* seed of the random start (RAFEAST_START_RANDOM)    */
} rafeast_params;

/* Diagnostics filled by rafeast_solve / rafeast_filter (may be NULL). */
typedef struct rafeast_info {
  int32_t status;
  int32_t outer_iters;       /* FEAST iterations run                          */
  int32_t cocg_iters_total;  /* sum over iterations of the slowest system     */
  int32_t cocg_min_last;     /* last iteration: fewest COCG steps of a system */
  int32_t cocg_max_last;     /* last iteration: most COCG steps of a system   */
  int32_t cholqr_shifted;    /* Cholesky-QR passes that needed a shift        */
  int32_t kernel_launches;   /* kernels launched by this call                 */
  int32_t spmm_launches;     /* of which sparse-matrix products               */
  double max_resid;          /* max in-interval relative residual             */
  double t_warmstart_ms;     /* device time per phase (CUDA events). This one */
                             /* is the start phase of the solve call: random  */
                             /* start (Omega, orthonormalise, A Q) or the     */
                             /* check of the handle's subspace; the time of   */
                             /* a rafeast_warmstart call is not in it         */
  double t_filter_ms;
  double t_orth_ms;
  double t_rr_ms;
  double t_total_ms;
} rafeast_info;

/* ---- handle ------------------------------------------------------------- */

/* Create a solver for A = L + diag_shift*I (Eq. 1's symmetric positive
 * definite A; Section 5.1's graph Laplacians L = D - W with a shift).
 * row_ptr/col_idx/values are host pointers, or device pointers when
 * inputs_on_device != 0; they are copied and may be freed on return.
 * Column indices must lie in [0, n) and be sorted within each row; L must be
 * symmetric (checked only with RAFEAST_CREATE_CHECK_SYMMETRY). stream is a
 * cudaStream_t (NULL = legacy default stream) on the current device; flags
 * combine RAFEAST_CREATE_*. On success *out owns every device buffer the
 * library allocates for this matrix until rafeast_destroy. Errors: -1 for
 * n <= 0, nnz < 0, a NULL pointer or an invalid CSR; -2 for an asymmetric L
 * when checked; -6 when device memory runs out; -9 without a CUDA device. */
int rafeast_create(rafeast_t* out, int64_t n, int64_t nnz,
                   const int32_t* row_ptr, const int32_t* col_idx,
                   const double* values, double diag_shift,
                   int inputs_on_device, void* stream, uint32_t flags);

/* Release the handle and all its device memory. NULL is a no-op. */
void rafeast_destroy(rafeast_t h);

/* Static English text for a status code. */
const char* rafeast_status_string(int status);

/* Text of the last CUDA failure seen by this thread (empty when none): the
 * failing runtime call, its error string and source location. Valid until
 * the next call on the same thread. */
const char* rafeast_last_error(void);

/* Set a tuning option (RAFEAST_OPT_*). -1 for an unknown key or value. */
int rafeast_set_option(rafeast_t h, int key, int64_t value);

/* Cumulative device time and algorithmic bytes of the batched-COCG kernels
 * launched while RAFEAST_OPT_PROFILE was on (CUDA events recorded around each
 * kernel inside the replayed graphs). out (host, 8 doubles): dot-kernel
 * launches, milliseconds, bytes; update-kernel launches, milliseconds, bytes;
 * the kernel shapes of the last multi-shift solve as 10000*c + 100*lanes +
 * chunks per lane, c the CTAs per SM the chosen kernel instance is compiled
 * for (0: the default instance; dot kernel, update kernel; chosen by the
 * autotuner). Bytes count A once (nnz*(4+s) + 4(n+1), s = 4 or 8) plus each state
 * column the launch reads or writes once: the dot kernel reads r, the update
 * kernel reads r and p, writes r and p, and updates the quadrature sum. With
 * reset != 0 the counters restart at zero after being copied out. */
int rafeast_profile(rafeast_t h, int reset, double* out);

/* Per-step history of the last COCG solve run with RAFEAST_OPT_PROFILE on:
 * for step k, the number of subspace columns with a still-active shift, the
 * largest ||r_k||_2/||b||_2 over the active systems, and the milliseconds of
 * the step's dot kernel and update kernel (kernel_ms[2k], kernel_ms[2k+1]).
 * Copies at most max_len steps into the host arrays (any may be NULL) and
 * returns the history length (0 when nothing was profiled), or -1 for a NULL
 * handle. After a profiled rafeast_solve_batched the first handle holds the
 * whole batch's trace instead: per grouped COCG step, the active pairs of all
 * problems (active_cols), the number of active problems (max_relres) and the
 * step's grouped dot and update milliseconds. */
int rafeast_profile_history(rafeast_t h, int max_len, int* active_cols, double* max_relres,
                            double* kernel_ms);

/* Matrix facts: n, internal row order (0 the caller's, 1 recursive
 * breadth-first bisection, 2 reverse Cuthill-McKee), ||A||_1 and the
 * Gershgorin interval of A. Any output pointer may be NULL. */
int rafeast_matrix_info(rafeast_t h, int64_t* n, int* reordered,
                        double* norm1, double* gersh_lo, double* gersh_hi);

/* ---- hot-path steps ------------------------------------------------------ */

/* Quadrature nodes and weights on the upper half of the ellipse around
 * [lmin, lmax] (Section 2.1, Eq. 3): z_j = c + R(cos t_j + i e sin t_j),
 * w_j = (R om_j/2)(e cos t_j + i sin t_j), t_j = (pi/2)(1 + x_j) with
 * Gauss-Legendre points x_j and weights om_j; the projector is
 * Re sum_j w_j (z_j I - A)^{-1}. z and w are host arrays of 2*nc doubles
 * (re, im interleaved). -1 unless lmin < lmax, 1 <= nc <= 64, 0 < e <= 1. */
int rafeast_quadrature(double lmin, double lmax, int nc, double e,
                       double* z, double* w);

/* Raw Philox-4x64-10 words (Salmon et al., SC'11) for counters
 * (first_block + b, 0, 0, 0), b < nblocks, key (seed, 0): words[4b + t].
 * words is a device array of 4*nblocks uint64; stream a cudaStream_t. This is
 * the generator behind Omega (Algorithm 2, "Draw Omega"). */
int rafeast_philox(uint64_t seed, uint64_t first_block, int64_t nblocks,
                   uint64_t* words, void* stream);

/* Omega ~ N(0,1)^{n x k} (Algorithm 2; Assumption 1.6) from the Philox
 * words by Box-Muller; column-major linear index e = c*n + i, block e/4.
 * omega: device, n*k doubles, caller row order. */
int rafeast_draw_omega(rafeast_t h, uint64_t seed, int k, double* omega);

/* Y = alpha * (A X) + beta * X for k columns (the SpMM of every power step of
 * the warmstart, Algorithm 2 Phase 1, and of Rayleigh-Ritz). X, Y: device,
 * column-major n x k. precision RAFEAST_FP64 computes in double;
 * RAFEAST_MIXED rounds X and the CSR values to float32 and accumulates in
 * float32 (the inner-solve kernel's arithmetic). */
int rafeast_spmm(rafeast_t h, int k, double alpha, double beta,
                 const double* X, double* Y, int precision);

/* W_j = (z_j I - A) P_j for nc complex shifts and m complex columns
 * (the operator of the shifted systems of Algorithm 1). P, W: device arrays
 * of n*m*nc complex values as (re, im) double pairs, entry (i, col, j) at
 * 2*((col*nc + j)*n + i). z: host, 2*nc doubles. precision as rafeast_spmm. */
int rafeast_shifted_spmm(rafeast_t h, int nc, const double* z, int m,
                         const double* P, double* W, int precision);

/* One quadrature filter application (Algorithm 1 "Compute Q~",
 * Algorithm 2 Step 2a): for every node solve (z_j I - A) X_j = Q by batched
 * COCG to prm->solve_tol (cap prm->max_inner) in prm->precision and form
 * Qt = sum_j Re(w_j X_j) in double. Uses prm->lmin, lmax, nc,
 * ellipse_ratio, solve_form. Q, Qt: device, n x m0 column-major (m0 =
 * prm->m0). theta: host array of m0 Ritz values for the correction form
 * (NULL = Rayleigh quotients of Q). -4 on a COCG breakdown. */
int rafeast_filter(rafeast_t h, const rafeast_params* prm, const double* Q,
                   const double* theta, double* Qt, rafeast_info* info);

/* Orthonormalise in place, Q R = Q~ (Algorithm 1 QR step), by Cholesky-QR
 * in double, repeated (CholQR2) and shifted when the Gram matrix is not
 * numerically positive definite (shifted CholQR3). Q: device n x m in/out.
 * R: host m x m column-major upper-triangular factor, or NULL. -8 when the
 * block is rank deficient beyond what a shift repairs. */
int rafeast_orthonormalize(rafeast_t h, int m, double* Q, double* R);

/* Gram matrix G = X^T Y of two tall blocks (the Cholesky-QR Gram matrix
 * B_Q = Q~^T Q~ and the Rayleigh-Ritz matrix A_Q = Q^T (A Q) of Algorithm 1
 * are of this form). X, Y: device, n x m column-major (n of the handle);
 * G: device, m x m column-major, entry (a, b) = sum_i X(i, a) Y(i, b), FP64.
 * Per-CTA partial sums live in the handle's scratch. m in 1..128. */
int rafeast_gram(rafeast_t h, int m, const double* X, const double* Y, double* G);

/* Tall block product Y = X M (the products X R^{-1} of Cholesky-QR and
 * Q V of Rayleigh-Ritz in Algorithm 1 are of this form). X: device, n x m
 * column-major (n of the handle); M: device, m x mo column-major; Y: device,
 * n x mo column-major, entry (i, b) = sum_a X(i, a) M(a, b), FP64 accurate:
 * on the tensor cores through exact BF16 digits of the FP64 values unless
 * RAFEAST_OPT_DENSE = 1. m, mo in 1..128. */
int rafeast_block_product(rafeast_t h, int m, const double* X, const double* M, int mo,
                          double* Y);

/* Allocation-free Gram matrix (no counterpart in the paper; a service for
 * callers): the same G = X^T Y as rafeast_gram, without a handle and without
 * any device allocation during the call. Some callers cannot let a library
 * allocate: applications that reserve the whole device memory up front for
 * their own allocator, or code that must not stall on cudaMalloc/cudaFree
 * (both can synchronise the device). Here the per-CTA partial sums live in a
 * fixed 2 MiB device array compiled into the library, held by every GPU that
 * loads it until the process exits.
 *   X, Y: device, n x m column-major (leading dimension n); G: device, m x m
 *   column-major, entry (a, b) = sum_i X(i, a) Y(i, b); n >= 1, 1 <= m <= 64
 *   (larger m returns -1 and rafeast_last_error says why). stream: a
 *   cudaStream_t on the current device; the call only enqueues work, G is
 *   ready when the stream reaches it.
 *   The first call on a device sets up: it looks up the array's device
 *   address (cudaGetSymbolAddress) and caches it. CUDA loads modules lazily
 *   by default, so that first call is also the one that loads the array and
 *   the entry point's kernels onto the device, about 2 MiB plus code: it
 *   allocates, later calls do not. Make the first call (n = 1, m = 1 will do)
 *   before reserving device memory for another allocator and before any
 *   stream capture begins; no cudaDeviceReset may follow it. An error that
 *   was already pending when the call begins is returned as -3 and left
 *   pending. All calls share the array: calls whose work overlaps on the GPU
 *   (other streams, other threads) race on it and must be serialised by the
 *   caller. */
int rafeast_gram_noalloc(const double* X, const double* Y, int64_t n, int m, double* G,
                         void* stream);

/* Rayleigh-Ritz (Algorithm 1): A_Q = Q^T A Q = V L V^T with L ascending,
 * Q <- Q V in place; theta (host, m) receives L and resid (host, m, may be
 * NULL) the relative residuals ||A q_i - l_i q_i||_2 / ||A||_1. Q must have
 * orthonormal columns. Q: device n x m. */
int rafeast_rayleigh_ritz(rafeast_t h, int m, double* Q, double* theta,
                          double* resid);

/* Randomized warmstart (Algorithm 2 Phase 1; Eq. 6 applied to B): draw
 * Omega (n x (m0+p)) from seed, Y = B^(2q+1) Omega with B the affine map of
 * RAFEAST_OPT_WARMSTART_MAP, Q = orth(Y), then Rayleigh-Ritz on A keeps the
 * m0 Ritz vectors whose Ritz values are closest to (lmin+lmax)/2. The result
 * becomes the handle's subspace (used by RAFEAST_START_SUBSPACE). Y is
 * re-orthonormalised after each pair of products; each orthonormalisation is
 * a Cholesky-QR whose first, preconditioning pass sums its Gram in float
 * (products with the factor and the last pass in double). */
int rafeast_warmstart(rafeast_t h, double lmin, double lmax, int m0, int p,
                      int q, uint64_t seed);

/* Inject a subspace (the warm-start injection of Section 6; also a resume
 * point): Q0 is n x m0 column-major, host or device per on_device; it is
 * orthonormalised and Rayleigh-Ritz'ed into the handle. */
int rafeast_set_subspace(rafeast_t h, const double* Q0, int m0, int on_device);

/* Copy the handle's current subspace (n x m0) and its Ritz values (m0, host,
 * may be NULL) out; Q host or device per on_device. -7 without one. */
int rafeast_get_subspace(rafeast_t h, double* Q, double* theta, int m0,
                         int on_device);

/* FEAST / RA-FEAST Phase 2 (Algorithms 1 and 2): iterate filter, QR,
 * Rayleigh-Ritz until every Ritz pair inside [lmin, lmax] has relative
 * residual <= outer_tol or max_outer iterations ran. Outputs (host or device
 * per outputs_on_device): evals[m0] Ritz values, the first *m_found of which
 * lie inside the interval in ascending order; evecs[n*m0] the matching
 * vectors, column-major; resid[m0] their relative residuals. m_found is a
 * host int. Returns 0, or 1/2/3 with valid outputs (no eigenvalue inside, no
 * convergence, m0 too small), or a negative error. The final subspace stays
 * in the handle. */
int rafeast_solve(rafeast_t h, const rafeast_params* prm, int* m_found,
                  double* evals, double* evecs, double* resid,
                  int outputs_on_device, rafeast_info* info);

/* Solve count independent problems (distinct handles on one device, each
 * with its own params and outputs; arrays of count pointers) as one batch.
 * All problems share precision and nc. Every outer iteration runs the
 * filter of all problems still iterating together: multi-shift COCG (the
 * RAFEAST_OPT_SOLVER = 1 path, whatever the handles' options) whose steps
 * are grouped launches, one dot and one update launch per step covering
 * every problem, captured as one CUDA graph on the first handle's stream.
 * The per-problem CholQR, Rayleigh-Ritz and residual phases run on the
 * problems' own streams, driven from up to 16 host threads, so their short
 * kernels overlap. A problem stops when it converges or reaches its own
 * max_outer. Outputs and statuses as rafeast_solve, per problem;
 * statuses[count] receives each problem's status (host). The grouped
 * launches are counted in the first problem's info. Returns the first
 * negative status, or 0; -1 (with a message) for mixed precision, mixed nc,
 * mixed devices or a repeated handle. */
int rafeast_solve_batched(int count, rafeast_t const* hs,
                          const rafeast_params* prms, int* m_found,
                          double* const* evals, double* const* evecs,
                          double* const* resid, int outputs_on_device,
                          rafeast_info* infos, int* statuses);

/* ---- sharding over ranks (one process and one GPU per rank) ----------------
 * The filter step of the outer loop (Algorithm 1, Algorithm 2 Phase 2:
 * Q~ = sum_j w_j (z_j I - A)^{-1} Q, Eq. 2) splits into independent shifted
 * solves. A sharded solve gives each rank a share of them and adds the
 * ranks' partial blocks with one sum over ranks per outer iteration; every
 * rank then runs the same orthonormalisation, Rayleigh-Ritz and residual
 * steps on the same block. The paper runs on one CPU thread and has no
 * counterpart: this is the GPU layout of its independent solves. */
#define RAFEAST_SHARD_COLUMNS 0 /* each rank filters a range of Q's columns    *
                                 * (whole column pairs) with all N_c nodes;     *
                                 * the other columns of its block are zero, so *
                                 * the sum over ranks is exact                  */
#define RAFEAST_SHARD_SHIFTS 1  /* each rank filters every column with a range *
                                 * of the N_c nodes; the sum over ranks adds    *
                                 * partial quadrature sums (rounding differs   *
                                 * from one rank's sum in the last bits). With *
                                 * the multi-shift solver every rank runs the  *
                                 * seed recurrence of its nodes: the sparse    *
                                 * products are not divided, only the shifted  *
                                 * updates                                     */

/* [*lo, *hi) = rank's share in a world of `world` ranks: columns of m0 for
 * RAFEAST_SHARD_COLUMNS (pairs split as evenly as they go, rank order), or
 * quadrature nodes of nc for RAFEAST_SHARD_SHIFTS (nc * rank / world ..).
 * A share can be empty (more ranks than pairs or nodes). Host only; -1 for
 * a bad mode, rank, world, m0 or nc. */
int rafeast_shard_range(int mode, int m0, int nc, int rank, int world, int* lo, int* hi);

/* Instance sharding of many independent problems (the batched workload):
 * owner[i] = the rank (0 .. world-1) that solves problem i, chosen longest
 * first: by decreasing cost[i] (ties: lower index first) each problem goes
 * to the rank with the least cost so far (ties: the lower rank). Host only,
 * deterministic, so every rank computes the same owners; cost is any
 * non-negative work estimate (e.g. nnz). -1 for count < 0, world < 1, a
 * negative cost or null arrays with count > 0. */
int rafeast_partition_instances(int count, const int64_t* cost, int world, int32_t* owner);

/* The caller's sum over ranks: on return, buf (count doubles, device memory
 * of the handle's device) must hold on every rank the element-wise sum of
 * all ranks' buf, with the caller's device work finished. The library has
 * synchronised its stream before the call, and it resumes its own work on
 * that stream afterwards. Every rank must add in the same order, so that
 * all ranks hold the same bits (an NCCL or gloo all-reduce does). Return 0,
 * or non-zero on failure (the solve then returns RAFEAST_ERR_EXCHANGE). */
typedef int (*rafeast_sum_fn)(void* ctx, double* buf, int64_t count);

/* rafeast_solve on rank `rank` of `world`, each rank with its own handle of
 * the same matrix (same CSR, create flags and options), the same params and
 * the same starting subspace (after the same rafeast_warmstart or
 * set_subspace; START_RANDOM draws the same block on every rank). Per outer
 * iteration the rank filters its share (rafeast_shard_range of `mode`) into
 * an n x m0 block, zero elsewhere, and calls sum(ctx, block, n * ldq) once,
 * ldq = m0 rounded up to even; after the Rayleigh-Ritz step it calls
 * sum(ctx, flag, 1) with flag 1.0 when the rank's residual test passed: the
 * loop stops when every rank passed, so that all ranks make the same number
 * of calls. Each rank ends with the whole result (outputs as rafeast_solve);
 * info counts this rank's COCG steps. world = 1 is rafeast_solve (no call of
 * sum, which may be null). Returns as rafeast_solve, RAFEAST_ERR_EXCHANGE
 * when sum failed, -1 for a bad mode, rank or world (or world > 1 with a null
 * sum). */
int rafeast_solve_sharded(rafeast_t h, const rafeast_params* prm, int mode, int rank,
                          int world, rafeast_sum_fn sum, void* ctx, int* m_found,
                          double* evals, double* evecs, double* resid, int outputs_on_device,
                          rafeast_info* info);

#ifdef __cplusplus
}
#endif
#endif /* RAFEAST_H */
