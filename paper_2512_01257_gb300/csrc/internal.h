// Internal interfaces of librafeast: handle layout, workspace, kernel
// launchers. Not part of the public ABI (include/rafeast.h is).
#pragma once

#include <cstdint>
#include <string>
#include <type_traits>
#include <vector>
#include <cuda_runtime.h>

#include "../../include/rafeast.h"

namespace rafeast {

// ---- error plumbing ---------------------------------------------------------
struct Err {
  int code;
};
#define RF_CUDA(call)                                                      \
  do {                                                                     \
    cudaError_t e_ = (call);                                               \
    if (e_ != cudaSuccess) {                                               \
      ::rafeast::set_last_error(e_, #call, __FILE__, __LINE__);            \
      throw ::rafeast::Err{e_ == cudaErrorMemoryAllocation                 \
                               ? RAFEAST_ERR_OUT_OF_MEMORY                 \
                               : RAFEAST_ERR_CUDA};                        \
    }                                                                      \
  } while (0)
#define RF_LAUNCH() ::rafeast::check_launch(__FILE__, __LINE__)
#define RF_CHECK(cond, code)             \
  do {                                   \
    if (!(cond)) throw ::rafeast::Err{code}; \
  } while (0)

void set_last_error(cudaError_t e, const char* what, const char* file, int line);
void set_last_message(const char* msg);  // replaces the text of rafeast_last_error
void clear_last_error();
// after a kernel launch: the launch's own error; with RAFEAST_DEBUG_SYNC=1 in
// the environment also synchronises and reports execution errors here
void check_launch(const char* file, int line);

// ---- device control block of one batched COCG solve -------------------------
struct CocgCtl {
  unsigned int ticket;  // last-CTA election in the dot kernel
  int iter;             // COCG iteration k about to run
  int active;           // systems still iterating
  int done;             // 1: every kernel of the solve returns at once
  int breakdown;        // systems stopped by a vanishing p^T M p
  int capped;           // systems stopped by max_inner
  int max_iters;        // most iterations taken by any system
  int min_iters;        // fewest iterations taken by a system with b != 0
  int timeout;          // a bounded device wait ran out
  // tiled dot kernel: CTAs of each column block that have finished, column
  // blocks whose scalar step is done, and the step's counters summed over
  // the column blocks (all zero between steps)
  unsigned int cbticket[16];
  unsigned int ticket2;
  int g_active, g_brk, g_cap, g_mx, g_cols;
  int g_mn;                     // 0x7fffffff between steps
  unsigned long long g_worst;   // bits of a non-negative double
  // 1 when the last update kernel left its shifted-direction updates to the
  // next dot kernel (deferred form); cleared at the end of every scalar step
  int pend;
};

// per-system scalar state, double precision (one struct per system s)
struct SysState {
  double2 gamma_prev;   // r_{k-1}^T r_{k-1}
  double2 alpha_prev;   // alpha_{k-1}
  double bnorm2;        // ||b||_2^2
  int active;
  int iters;
};

// per-system coefficients consumed by the update kernel, in working precision
template <typename T> struct Coef {
  typename std::conditional<sizeof(T) == 4, float2, double2>::type beta, alpha, ca;
  T ar;
  T pad;
};

// multi-shift COCG: per (column i, non-seed shift j') scalar state and the
// coefficients the update kernel consumes
struct ShiftState {
  double2 zeta;       // zeta_k of the shifted system (residual = zeta_k r_k)
  double2 zeta_prev;  // zeta_{k-1}
  int active;
  int iters;
};
template <typename T> struct ShiftCoef {
  typename std::conditional<sizeof(T) == 4, float2, double2>::type zeta, beta, ca;
  T act;  // 1 while the shifted system iterates, else 0 (p_j frozen)
  T pad;
};

// arguments of the batched COCG kernels (one problem or a concatenation)
template <typename T> struct CocgArgs {
  int64_t n;
  const int32_t* rowptr;
  const int32_t* colidx;
  const T* val;
  int m0;          // subspace columns i
  int ldc;         // complex stride of one state row (>= m0 * NC, even)
  int lanes;       // G: lanes per row group (4, 8, 16, 32)
  int cpl;         // chunks per lane (<= kernel's MAXCPL)
  T* r[2];         // residual, ping-pong
  T* p[2];         // search direction, ping-pong
  T* dacc;         // quadrature accumulator, n x ldd (real)
  int ldd;
  const double* qin;     // Q, internal row-major n x ldq (init)
  const double* aqin;    // A Q, same layout (correction form), or null
  int ldq;
  const double* theta;   // Ritz values [m0] (correction form)
  const void* zs;        // c2<T>[NC]: z_j - sigma
  const double2* coef;   // [nsys]: quadrature coefficient of system s
  double* acc;           // [nsys * 5] dot partial sums (zeroed)
  SysState* st;          // [nsys]
  Coef<T>* cf;           // [nsys]
  int* colact;           // [m0]: 1 while any shift of column i is active
  CocgCtl* ctl;
  int* hist;             // [max_inner + 2]: active columns after step k, or null
  double* rhist;         // [max_inner + 2]: max ||r||/||b|| over active systems
  int nc_real;           // shifts with a right-hand side (<= NC)
  double tol2;           // solve_tol^2
  int max_inner;
  int form;              // RAFEAST_FORM_*
  long long wait_cycles; // bound of one bulk-copy wait (clock64 cycles)
  int stall_bytes;       // test hook: extra bytes each stage expects (0)
  // multi-shift mode (ms = 1): the dot kernel runs on column pairs of the
  // seed shift (m0 = pairs, NC = 2, both zs entries z_seed - sigma); systems
  // are the 2*pairs columns; the shifted systems live in ps/sst/scf
  int ms;
  int ns;                  // non-seed shifts
  int nc_total;            // real shifts (seed included)
  const double2* sigma;    // [ns]: z_j - z_seed
  const double2* scoef;    // [columns * ns]: quadrature coefficient c_j(i)
  ShiftState* sst;         // [columns * ns]
  ShiftCoef<T>* scf;       // [columns * ns]
  T* ps;                   // shifted directions, row r: pairs x ns x 2 complex
  int ldps;                // complex stride of a ps row
  // resident CTAs per SM the multi-shift kernels are compiled for (float,
  // at most two chunks per lane): 0 or 2 the default instances, 3 or 4
  // instances with fewer registers per thread (host-side choice)
  int occ;
  // streamed multi-shift update (wbuf != null): the dot kernel also stores
  // w_k = M r_k, and the update kernel forms s_k = M p_k by the recurrence
  // s_k = w_k + beta s_{k-1} instead of gathering; r and p are updated in
  // place (r[0] == r[1], p[0] == p[1]), s is kept in sbuf
  T* wbuf;
  T* sbuf;
  // deferred form of the streamed update (defer = 1, tiled dot kernel): the
  // update kernel of step k forms p_k, s_k, r_{k+1} (r ping-ponged between
  // r[0] and r[1]) and the seed's quadrature term, and leaves the shifted
  // directions and their quadrature terms of step k to the dot kernel of
  // step k + 1, which applies them from r_k while its gathered rows load
  int defer;
  // values-free Laplacian gathers (lcolidx != null): A = L + shift I with L a
  // unit-weight graph Laplacian (off-diagonal -1, diagonal = degree); lrowptr
  // and lcolidx hold the off-diagonal pattern only, L r = deg r - sum r_nbr
  const int32_t* lrowptr;
  const int32_t* lcolidx;
};

// ---- row tiles of the tiled sparse products (tiling.cpp, kernels_tiled.cu) ----
// Tile t holds rows [trow[t], trow[t+1]); its union (the rows its nonzeros
// name and its own rows, ascending) is ucol[uoff[t] .. uoff[t+1]); its first
// row sits at union position uself[t]; every nonzero has its column's
// position in its tile's union in lidx (parallel to the CSR column array).
struct TileHost {
  std::vector<int32_t> trow, uoff, ucol;
  int max_union = 0, max_rows = 0;
};
struct TileArgs {
  int ntiles;
  int max_union;
  const int32_t* trow;
  const int32_t* uoff;
  const int32_t* ucol;
  const int32_t* uself;
  const uint16_t* lidx;  // for the pattern the kernel gathers on
  int cb;                // column pairs per block (4 or 8)
  int ncb;               // column blocks
  double* part;          // [grid * cb * 10]: per-CTA sums
};
#ifndef RF_TILE_UCAP
#define RF_TILE_UCAP 512
#endif
constexpr int TILE_UCAP = RF_TILE_UCAP;  // most union rows of a tile
constexpr int TILE_TMAX = 256;    // most rows of a tile
constexpr int TILE_NNZCAP = 3072; // most nonzeros of a tile (full CSR)
constexpr int TILE_MAX_OCC = 8;   // most resident CTAs per SM of the tiled kernel

// ---- handle -----------------------------------------------------------------
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

struct Handle {
  int device = 0;
  int num_sms = 0;
  int64_t n = 0, nnz = 0;
  cudaStream_t user_stream = nullptr;
  cudaStream_t stream = nullptr;  // internal, non-blocking
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  // CSR in internal order
  int32_t* rowptr = nullptr;
  int32_t* colidx = nullptr;
  double* val64 = nullptr;
  float* val32 = nullptr;
  // the off-diagonal pattern when A's CSR part is a unit-weight Laplacian
  int32_t* lrowptr = nullptr;
  int32_t* lcolidx = nullptr;
  int64_t nnz_off = 0;
  // row tiles (ntiles = 0 when the matrix has a row that gathers from more
  // than TILE_UCAP rows): union arrays, and the local indices of the full
  // CSR and of the off-diagonal pattern
  int ntiles = 0, tile_max_union = 0, tile_max_rows = 0;
  int32_t* trow = nullptr;
  int32_t* uoff = nullptr;
  int32_t* ucol = nullptr;
  int32_t* uself = nullptr;
  uint16_t* lidx = nullptr;
  uint16_t* llidx = nullptr;
  double tile_ratio = 0.0;  // sum of union sizes / n
  int order_kind = 0;       // 0 caller's order, 1 bisection, 2 reverse Cuthill-McKee
  double shift = 0.0;
  double norm1 = 0.0, glo = 0.0, ghi = 0.0;
  bool reordered = false;
  int32_t* perm = nullptr;   // internal row r holds original row perm[r]
  int32_t* iperm = nullptr;  // original row o sits at internal row iperm[o]
  // current subspace (internal order, row-major n x ldq)
  int m0 = 0, ldq = 0;
  double* Q = nullptr;
  double* AQ = nullptr;
  std::vector<double> theta;  // host copy of Ritz values
  double* theta_d = nullptr;
  // options
  int opt_ws_map = 0;
  int opt_chunk = 16;
  int opt_autotune = 1;
  int opt_lanes = 0;
  int opt_cpl = 0;     // cap on column chunks per lane (0: kernel maximum)
  int opt_solver = 1;  // 0: COCG per shift, 1: multi-shift COCG (default)
  int opt_update = 0;  // multi-shift update: 0 auto, 1 gathered products, 2 streamed
  int opt_values_free = 0;  // 0: values-free gathers for unit Laplacians, 1: never
  int opt_tiled = 0;        // seed dot kernel: 0 auto (tiled when built), 1 never, 2 only tiled
  int opt_tile_cb = 0;      // tiled dot kernel: forced column pairs per block (0: autotuned)
  int opt_dense = 0;        // FP64 Gram matrices: 0 tensor cores (digit split), 1 FP64 pipe
  int opt_defer = 0;        // 1: deferred shifted updates with the tiled dot kernel, 0: never
  // quadrature nodes [shard_j0, shard_j1) of the N_c this filter sums over
  // (a shift-sharded solve); shard_j1 < 0: all of them
  int shard_j0 = 0, shard_j1 = -1;
  // autotuned kernel shapes (lanes, chunks per lane) of the multi-shift
  // kernels, keyed by (pairs, shifts, precision)
  struct Shape {
    int dl, dc, ul, uc;
    int dm = 0, um = 0;  // forced CTAs per SM (0: default instance)
    int dt = 0;          // tiled dot kernel: column pairs per block (0: register gathers)
  };
  std::vector<std::pair<int64_t, Shape>> tuned;
  int opt_profile = 0;
  int opt_kernel = 0;  // 0 auto, 1 register gathers, 2 bulk-copy gathers
  int opt_maxnz = 8;   // nonzeros per bulk-copy item
  long long opt_wait_cycles = 2000000000LL;  // ~1 s: bound of one device wait
  int opt_stall_bytes = 0;                   // test hook, see RAFEAST_OPT_TEST_STALL
  // kernel time / algorithmic bytes of the COCG kernels (profile option)
  double prof[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  std::vector<int> last_hist;        // last profiled filter: active columns per step
  std::vector<double> last_rhist;    // and the worst relative residual per step
  std::vector<float> last_tk;        // dot, update kernel milliseconds per step
  // scratch, grown on demand and kept
  std::vector<DevBuf> bufs;
  // launch accounting of the current call
  int launches = 0;
  int spmm_launches = 0;
};

void* scratch(Handle* h, int slot, size_t bytes);  // keep-alive buffer per slot
// raise a kernel's dynamic shared-memory limit to at least `bytes` on the
// current device; never lowers it, so threads launching the same kernel with
// different sizes cannot undercut one another
void ensure_dyn_smem(const void* fn, size_t bytes);
enum Slot {
  S_STATE = 0, S_DACC, S_QT, S_TMP1, S_TMP2, S_SCAL, S_GRAM, S_SMALL, S_OMEGA,
  S_AQ2, S_IO1, S_IO2, S_BATCH, S_TPART, S_SHARD, S_COUNT
};

// ---- host math (hostmath.cpp) ------------------------------------------------
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w);
void quadrature_nodes(double lmin, double lmax, int nc, double e,
                      std::vector<double>& zr, std::vector<double>& zi,
                      std::vector<double>& wr, std::vector<double>& wi);
// reverse Cuthill-McKee order of a symmetric CSR pattern: perm[new] = old
void rcm_order(int64_t n, const int32_t* rowptr, const int32_t* colidx,
               std::vector<int32_t>& perm);
int64_t bandwidth(int64_t n, const int32_t* rowptr, const int32_t* colidx,
                  const int32_t* perm /* may be null */);
// recursive breadth-first bisection of a symmetric pattern: perm[new] = old
void bisect_order(int64_t n, const int32_t* rowptr, const int32_t* colidx, int leaf,
                  std::vector<int32_t>& perm);
// row tiles with unions of at most ucap rows, at most tmax rows and at most
// nnzcap nonzeros; false when a single row exceeds a cap
bool build_tiles(int64_t n, const int32_t* rowptr, const int32_t* colidx, int ucap, int tmax,
                 int nnzcap, TileHost& t);
// union rows per row of the tiles of a few evenly spaced row windows (an
// estimate of the whole pattern's ratio; -1 when a row exceeds a cap)
double tile_union_ratio(int64_t n, const int32_t* rowptr, const int32_t* colidx, int ucap,
                        int tmax, int nnzcap, int windows);
// union positions of every nonzero of a pattern whose columns lie in the
// tiles' unions (the full CSR or its off-diagonal part); uself per tile.
// lidx gets 8 zero entries of padding after the last nonzero.
void tile_local_index(int64_t n, const int32_t* rowptr, const int32_t* colidx,
                      const TileHost& t, std::vector<uint16_t>& lidx,
                      std::vector<int32_t>& uself);
// tiled seed dot kernel of the multi-shift COCG (float32, streamed update);
// occ_cap: most CTAs per SM (0: as many as fit, at most TILE_MAX_OCC)
void launch_ms_dots_tiled(const CocgArgs<float>& a, const TileArgs& tl, int buf, int num_sms,
                          int occ_cap, cudaStream_t s);

// ---- kernel launchers (kernels_sparse.cu) --------------------------------------
int nc_pad(int nc);  // shifts rounded up to a compiled NC (1, 2, 4, 8)
int max_cpl(int NC, bool fp64);
void choose_shape(int m0, int NC, bool fp64, int forced_lanes, int& lanes, int& cpl,
                  int& colblocks, int forced_cpl);

template <typename T>
void launch_cocg_init(const CocgArgs<T>& a, int NC, int num_sms, cudaStream_t s);
template <typename T>
void launch_cocg_reset(const CocgArgs<T>& a, int NC, cudaStream_t s);
// multi-shift COCG (seed dot kernel = launch_cocg_dots with NC = 2)
template <typename T>
void launch_ms_init(const CocgArgs<T>& a, int m_real, int num_sms, cudaStream_t s);
template <typename T>
void launch_ms_update(const CocgArgs<T>& a, int buf, int num_sms, cudaStream_t s);
// streamed multi-shift update (needs a.wbuf, a.sbuf; no gathers)
template <typename T>
void launch_ms_update_stream(const CocgArgs<T>& a, int buf, int num_sms, cudaStream_t s);
int ms_max_cpl(bool fp64);
// bulk-copy (TMA) kernels, float32, NC in {2, 4, 8}, blocked state layout
// (kernels_tma.cu). which: 0 init, 1 dots, 2 update.
void launch_cocg_tma(const CocgArgs<float>& a, int NC, int which, int buf, int maxnz,
                     int num_sms, cudaStream_t s);
int tma_cpl(int m0);
int tma_ncb(int m0, int cpl);
template <typename T>
void launch_cocg_dots(const CocgArgs<T>& a, int NC, int buf, int num_sms, cudaStream_t s);
template <typename T>
void launch_cocg_update(const CocgArgs<T>& a, int NC, int buf, int num_sms, cudaStream_t s);

// grouped multi-shift COCG over many problems, one persistent launch per
// kernel per step (kernels_batched.cu): the CTAs drain a queue of work items
// (problem, row slice, column block) described by an item map (starts of the
// problems' items [count + 1], then gx per problem); the dot kernel's last
// CTA re-plans both maps on the device as problems finish.
struct GroupCtl {
  unsigned int ticket;  // CTAs of the current dot launch that have finished
  unsigned int next_d;  // queue heads of the dot and update launches
  unsigned int next_u;
  int grid_d, grid_u;   // persistent grid sizes of the two kernels
  int pad[3];
};
struct GroupPlan {
  int count = 0;
  int ns = 0;
  int mc_d = 2, mc_u = 2;  // compiled chunks per lane of the two kernels
  size_t smem_dots = 0, smem_upd = 0;
  const void* fn_dots = nullptr;
  const void* fn_upd = nullptr;
  std::vector<int> map_dots, map_upd;  // initial maps (every problem active)
  std::vector<int> gg_d, gg_u;  // per problem: row groups, column blocks, gathered KiB, 0
  int ctas_dots = 0, ctas_upd = 0;  // persistent grid sizes
};
// the two kernels may use different (lanes, chunks) shapes per problem
template <typename T> struct GroupDev {
  const CocgArgs<T>* args_d;
  const CocgArgs<T>* args_u;
  int* map_d;
  int* map_u;
  GroupCtl* gc;
  const CocgCtl* ctl;  // the problems' control blocks, contiguous
  const int4* gg_d;
  const int4* gg_u;
};
template <typename T>
void plan_ms_grouped(const std::vector<CocgArgs<T>>& args_d, const std::vector<CocgArgs<T>>& args_u,
                     int num_sms, GroupPlan& g);
// which: 0 dots (seed scalars of every problem, then the re-plan), 1 update
template <typename T>
void launch_ms_grouped(const GroupPlan& g, const GroupDev<T>& d, int which, int buf,
                       cudaStream_t s);

// W = zs_j P - L P over complex chunks (rafeast_shifted_spmm)
template <typename T>
void launch_shifted_spmm(int64_t n, const int32_t* rp, const int32_t* ci, const T* val,
                         int m, int ldc, int NC, const void* zs, const T* P, T* W,
                         int lanes, int cpl, int num_sms, cudaStream_t s);
// Y = sL * (L X) + sI * X, real, row-major n x ld (ld even)
template <typename T>
void launch_spmm_real(int64_t n, const int32_t* rp, const int32_t* ci, const T* val,
                      int k, int ld, double sL, double sI, const T* X, T* Y,
                      int num_sms, cudaStream_t s);

// ---- dense kernels (kernels_dense.cu) ------------------------------------------
void launch_philox(uint64_t seed, uint64_t first, int64_t nblocks, uint64_t* out,
                   cudaStream_t s);
void launch_omega(uint64_t seed, int64_t n, int k, double* out_colmajor, cudaStream_t s);
// caller col-major (n x m, ld n, original order) <-> internal row-major (ld)
void launch_to_internal(int64_t n, int m, const double* src, double* dst, int ld,
                        const int32_t* perm, cudaStream_t s);
void launch_from_internal(int64_t n, int m, const double* src, int ld, double* dst,
                          const int32_t* perm, const int32_t* cols /* may be null */,
                          cudaStream_t s);
// row-major tall blocks, FP64
// G = X^T Y (m x m, ld m); sym: X^T Y is symmetric (X^T X, X^T A X), only
// one triangle of tile blocks is formed and mirrored; f32 (sym only): products
// and per-CTA sums in float, for the preconditioning pass of a
// mixed-precision Cholesky-QR
void gram(const double* X, const double* Y, int64_t n, int m, int ld, double* G,
          double* partial, int num_sms, cudaStream_t s, bool sym = false, bool f32 = false);
// G = sum of the m x m partials in increasing order (sym: the 16-blocks below
// the diagonal taken from above it, so G is exactly symmetric)
void gram_sum(const double* part, int parts, int m, bool sym, double* G, cudaStream_t s);
// the same Gram on the tensor cores (kernels_tc.cu): FP64 values split into
// exact BF16 digits, tcgen05 products, exact integer accumulation; m <= 128,
// partial: num_sms * m * m doubles; err (may be null) set on a timed-out wait
bool gram_tc_fits(int m);
// Y = X M on the tensor cores (exact BF16 digits of FP64 values, TMEM
// levels): m, mo <= 128; err (device int) is set when a bounded wait ran out
bool tall_tc_fits(int m, int mo);
void tall_gemm_tc(const double* X, int64_t n, int m, int ldx, const double* M, int mo, double* Y,
                  int ldy, int num_sms, int* err, cudaStream_t s);
void gram_tc(const double* X, const double* Y, int64_t n, int m, int ld, double* G,
             double* partial, int num_sms, int* err, cudaStream_t s, bool sym);
// Y = X * M (M: m x mo, ld mo); upper: M is upper triangular (m == mo)
void tall_gemm(const double* X, int64_t n, int m, int ldx, const double* M, int mo,
               double* Y, int ldy, cudaStream_t s, bool upper = false);
// one-CTA Cholesky of G (+shift when needed) and inverse of the factor:
// Rinv (m x m, ld m, upper) with Q R = X -> Q = X Rinv. status[0] = 0 ok,
// 1 shifted, 2 failed; with check_id, bit 4 is added when an entry of G is
// off the identity by more than 1/4. status[1..] unused.
void chol_inv(double* G, int m, int64_t nrows, double* Rfac, double* Rinv, int* status,
              cudaStream_t s, bool check_id = false);
// one-CTA cyclic Jacobi: A (m x m, ld m, symmetric) -> eigenvalues ascending
// in w, eigenvectors (columns) in V (m x m, ld m)
// (work: 6 (m+1)^2 doubles; mixed-precision Jacobi, see kernels_dense.cu)
// m x m row-major C = alpha op(A) op(B) + gamma I (ta, tb: transpose); C must
// not alias A or B
void small_gemm(const double* A, int ta, const double* B, int tb, double* C, int m, double alpha,
                double gamma, cudaStream_t s);
void jacobi_eigh(double* A, int m, double* w, double* V, double* work, cudaStream_t s);
// res_i = ||AQ_i - theta_i Q_i||^2 (sums, m), FP64; part: workspace of
// 2 * num_sms * m doubles (per-block sums, added in a fixed order)
void col_resid2(const double* Q, const double* AQ, const double* theta, int64_t n, int m,
                int ld, double* out, double* part, int num_sms, cudaStream_t s);
// Qt = f_i * Q + D (D in T, ld ldd)
template <typename T>
void launch_combine(const double* Q, int ldq, const T* D, int ldd, const double* f,
                    int64_t n, int m, double* Qt, cudaStream_t s);
void launch_zero(void* p, size_t bytes, cudaStream_t s);
void launch_widen(const float* src, double* dst, int64_t count, cudaStream_t s);
// out[i] = sum_r X[r][i] Y[r][i] (part as for col_resid2)
void col_dot(const double* X, const double* Y, int64_t n, int m, int ld, double* out,
             double* part, int num_sms, cudaStream_t s);
void launch_cast_to_f32(const double* src, float* dst, int64_t count, cudaStream_t s);

}  // namespace rafeast
