// C-ABI of librafeast (declared in include/rafeast.h): handle lifecycle and
// the FEAST / RA-FEAST driver. Every numerical step runs in the kernels of
// kernels_sparse.cu / kernels_dense.cu on the handle's stream; the host only
// sequences launches, reads back the m0 Ritz values and residuals once per
// outer iteration, and takes the convergence decision (Algorithm 1's
// "until convergence"). The COCG inner iterations are captured as CUDA
// graphs of `chunk` steps and replayed until the device reports that every
// system has converged.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <memory>
#include <mutex>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace rafeast {

static thread_local char g_err[512] = "";

void set_last_message(const char* msg) { snprintf(g_err, sizeof(g_err), "%s", msg); }

void clear_last_error() { g_err[0] = 0; }

void set_last_error(cudaError_t e, const char* what, const char* file, int line) {
  if (g_err[0]) return;  // keep the first failure of this call
  snprintf(g_err, sizeof(g_err), "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
}

static int debug_sync() {
  static int v = -1;
  if (v < 0) {
    const char* e = getenv("RAFEAST_DEBUG_SYNC");
    v = (e && e[0] == '1') ? 1 : 0;
  }
  return v;
}

static thread_local bool g_capturing = false;

void check_launch(const char* file, int line) {
  cudaError_t e = cudaGetLastError();
  // no device-wide sync while this thread captures a graph
  if (e == cudaSuccess && debug_sync() && !g_capturing) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    set_last_error(e, "kernel launch", file, line);
    throw Err{e == cudaErrorMemoryAllocation ? RAFEAST_ERR_OUT_OF_MEMORY : RAFEAST_ERR_CUDA};
  }
}

void ensure_dyn_smem(const void* fn, size_t bytes) {
  static std::mutex mu;
  static std::vector<std::pair<std::pair<int, const void*>, size_t>> set;
  int dev = 0;
  RF_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  for (auto& e : set)
    if (e.first.first == dev && e.first.second == fn) {
      if (e.second >= bytes) return;
      RF_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
      e.second = bytes;
      return;
    }
  RF_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  set.push_back(std::make_pair(std::make_pair(dev, fn), bytes));
}

void* scratch(Handle* h, int slot, size_t bytes) {
  if ((int)h->bufs.size() <= slot) h->bufs.resize(slot + 1);
  DevBuf& b = h->bufs[slot];
  if (bytes == 0) bytes = 16;
  if (b.bytes < bytes) {
    if (b.p) RF_CUDA(cudaFree(b.p));
    b.p = nullptr;
    b.bytes = 0;
    RF_CUDA(cudaMalloc(&b.p, bytes));
    b.bytes = bytes;
  }
  return b.p;
}

static inline int even(int m) { return m + (m & 1); }

struct CallScope {
  Handle* h;
  explicit CallScope(Handle* hh) : h(hh) {
    h->launches = 0;
    h->spmm_launches = 0;
    cudaGetLastError();  // a stale error of an earlier call is not ours
    g_err[0] = 0;
    RF_CUDA(cudaSetDevice(h->device));
    RF_CUDA(cudaEventRecord(h->ev_in, h->user_stream));
    RF_CUDA(cudaStreamWaitEvent(h->stream, h->ev_in, 0));
  }
  void finish() {
    RF_CUDA(cudaEventRecord(h->ev_out, h->stream));
    RF_CUDA(cudaStreamWaitEvent(h->user_stream, h->ev_out, 0));
  }
};

// ---------------------------------------------------------------------------
// dense building blocks on internal row-major blocks
// ---------------------------------------------------------------------------
struct DenseWs {
  double* G;      // m x m
  double* R;      // m x m
  double* Rinv;   // m x m
  double* V;      // m x m
  double* Vw;     // 6 (m+1)^2: eigensolver work
  double* w;      // m
  double* part;   // gram partials
  int* status;    // 4 ints
  double* small;  // m doubles
};

static DenseWs dense_ws(Handle* h, int m) {
  const size_t mm = (size_t)(m + 1) * (m + 1);
  const int parts = 2 * h->num_sms;
  char* base = (char*)scratch(h, S_GRAM, sizeof(double) * (10 * mm + 2 * (m + 1) +
                                                          (size_t)parts * m * m) + 64);
  DenseWs d;
  double* p = (double*)base;
  d.G = p; p += mm;
  d.R = p; p += mm;
  d.Rinv = p; p += mm;
  d.V = p; p += mm;
  d.Vw = p; p += 6 * mm;
  d.w = p; p += m + 1;
  d.small = p; p += m + 1;
  d.part = p;
  d.status = (int*)scratch(h, S_SMALL, 64);
  return d;
}

// G = X^T Y (m x m) of the handle's tall blocks: on the tensor cores (FP64
// values split into exact BF16 digits, kernels_tc.cu) unless the FP64 pipe is
// asked for or m exceeds 128; the float Gram of a preconditioning pass stays
// on the float pipe. sym: the result is symmetric (X^T X, X^T A X) and is
// made exactly so.
static void gram_dev(Handle* h, const double* X, const double* Y, int m, int ld, double* G,
                     const DenseWs& d, bool sym, bool f32 = false) {
  // (two launches either way; the callers count them)
  if (!f32 && h->opt_dense == 0 && gram_tc_fits(m))
    gram_tc(X, Y, h->n, m, ld, G, d.part, h->num_sms, d.status + 3, h->stream, sym);
  else
    gram(X, Y, h->n, m, ld, G, d.part, h->num_sms, h->stream, sym, f32);
}

// Y = X M (tall n x m block times m x mo, row-major M) on the tensor cores
// (exact BF16 digits of the FP64 values, kernels_tc.cu) unless the FP64 pipe
// is asked for; upper: M is upper triangular (the FP64 kernel skips its zero
// blocks)
static void tall_dev(Handle* h, const double* X, int m, int ldx, const double* M, int mo,
                     double* Y, int ldy, bool upper = false) {
  if (h->opt_dense == 0 && tall_tc_fits(m, mo)) {
    // (the timeout flag beside the dense status words; no other scratch is
    // touched, so the caller's dense workspace stays where it is)
    int* err = (int*)scratch(h, S_SMALL, 64) + 3;
    tall_gemm_tc(X, h->n, m, ldx, M, mo, Y, ldy, h->num_sms, err, h->stream);
  } else {
    tall_gemm(X, h->n, m, ldx, M, mo, Y, ldy, h->stream, upper);
  }
}

// X (n x m, ld) <- X R^{-1}; returns number of shifted passes; R_total (host,
// m x m row-major upper) accumulates the factor if non-null. low_first: the
// first pass forms its Gram in float, as in cholqr_rr below (the pass only
// preconditions; the products with R^{-1} stay FP64 and the last pass is FP64).
static int cholqr(Handle* h, double*& X, double*& tmp, int m, int ld, std::vector<double>* Rtot,
                  bool low_first = false) {
  DenseWs d = dense_ws(h, m);
  int shifted = 0;
  int passes = 2;
  bool low_used = false;
  std::vector<double> Racc;
  if (Rtot) {
    Racc.assign((size_t)m * m, 0.0);
    for (int i = 0; i < m; ++i) Racc[i * m + i] = 1.0;
  }
  for (int pass = 0; pass < passes; ++pass) {
    const bool low = low_first && pass == 0;
    int st = 0;
    for (int attempt = 0; attempt < 2; ++attempt) {
      const bool f32 = low && attempt == 0;
      gram_dev(h, X, X, m, ld, d.G, d, true, f32);
      chol_inv(d.G, m, h->n, d.R, d.Rinv, d.status, h->stream, low_used && pass == 1);
      h->launches += 3;
      RF_CUDA(cudaMemcpyAsync(&st, d.status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
      RF_CUDA(cudaStreamSynchronize(h->stream));
      if (f32 && st != 0) continue;  // the float Gram was not enough: FP64
      low_used = f32;
      break;
    }
    if (st & 4) {
      st &= ~4;
      if (passes < 4) ++passes;
    }
    if (st == 2) throw Err{RAFEAST_ERR_CHOLESKY};
    if (st == 1) {
      ++shifted;
      if (passes < 4) ++passes;
    }
    tall_dev(h, X, m, ld, d.Rinv, m, tmp, ld, true);
    h->launches += 1;
    std::swap(X, tmp);
    if (Rtot) {
      std::vector<double> Rp((size_t)m * m), out((size_t)m * m, 0.0);
      RF_CUDA(cudaMemcpyAsync(Rp.data(), d.R, sizeof(double) * m * m, cudaMemcpyDeviceToHost,
                              h->stream));
      RF_CUDA(cudaStreamSynchronize(h->stream));
      // R_total <- R_pass * R_total
      for (int i = 0; i < m; ++i)
        for (int k = i; k < m; ++k) {
          const double r = Rp[i * m + k];
          if (r == 0.0) continue;
          for (int j = 0; j < m; ++j) out[i * m + j] += r * Racc[k * m + j];
        }
      Racc.swap(out);
    }
  }
  if (Rtot) *Rtot = Racc;
  return shifted;
}

// Rayleigh-Ritz on X (n x m, ld, orthonormal): Qout = X V, AQout = A Qout,
// theta (device, m, ascending).
static void rayleigh_ritz_dev(Handle* h, const double* X, int m, int ld, double* Qout,
                              double* AQout, double* theta_d, double* tmp) {
  DenseWs d = dense_ws(h, m);
  launch_spmm_real<double>(h->n, h->rowptr, h->colidx, h->val64, m, ld, 1.0, h->shift, X, tmp,
                           h->num_sms, h->stream);
  gram_dev(h, X, tmp, m, ld, d.G, d, true);
  jacobi_eigh(d.G, m, theta_d, d.V, d.Vw, h->stream);
  tall_dev(h, X, m, ld, d.V, m, Qout, ld);
  // A Q by the (memory-bound) SpMM rather than (A X) V by an FP64 GEMM
  launch_spmm_real<double>(h->n, h->rowptr, h->colidx, h->val64, m, ld, 1.0, h->shift, Qout,
                           AQout, h->num_sms, h->stream);
  h->launches += 7;
  h->spmm_launches += 2;
}

// Cholesky-QR2 and Rayleigh-Ritz with the last factor folded in (the outer
// loop's orthonormalise + Rayleigh-Ritz): the passes before the last form
// X <- X R^{-1}; the last pass's R^{-1} is not applied. With Z = X R^{-1}:
// Z^T A Z = R^{-T} (X^T A X) R^{-1} = V diag(theta) V^T, and the Ritz vectors
// are Z V = X (R^{-1} V), one tall product instead of two. Qout = X (R^{-1} V),
// AQout = A Qout. ev_mid is recorded between the factorisations and the rest.
// low_first (mixed precision): the first pass only preconditions X, so its
// Gram is formed in float; X R1^{-1} is still an FP64 product, which keeps the
// span of X. The pass is redone in FP64 when the float Gram needed a shift,
// and an extra FP64 pass is added when the next Gram is not close to the
// identity; the last factorisation is always FP64.
// Returns the number of shifted passes.
static int cholqr_rr(Handle* h, double*& X, double*& tmp, double* tmp2, int m, int ld,
                     double* Qout, double* AQout, double* theta_d, cudaEvent_t ev_mid,
                     bool low_first = false) {
  DenseWs d = dense_ws(h, m);
  int shifted = 0;
  int passes = 2;
  bool low_used = false;
  for (int pass = 0; pass < passes; ++pass) {
    const bool low = low_first && pass == 0;
    int st = 0;
    for (int attempt = 0; attempt < 2; ++attempt) {
      const bool f32 = low && attempt == 0;
      gram_dev(h, X, X, m, ld, d.G, d, true, f32);
      chol_inv(d.G, m, h->n, d.R, d.Rinv, d.status, h->stream, low_used && pass == 1);
      h->launches += 3;
      RF_CUDA(cudaMemcpyAsync(&st, d.status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
      RF_CUDA(cudaStreamSynchronize(h->stream));
      if (f32 && st != 0) continue;  // the float Gram was not enough: FP64
      low_used = f32;
      break;
    }
    if (st & 4) {
      // X R1^{-1} from the float pass is far from orthonormal: one more pass
      st &= ~4;
      if (passes < 4) ++passes;
    }
    if (st == 2) throw Err{RAFEAST_ERR_CHOLESKY};
    if (st == 1) {
      ++shifted;
      if (passes < 4) ++passes;
    }
    if (pass == passes - 1) break;  // the last factor is folded into Rayleigh-Ritz
    tall_dev(h, X, m, ld, d.Rinv, m, tmp, ld, true);
    h->launches += 1;
    std::swap(X, tmp);
  }
  RF_CUDA(cudaEventRecord(ev_mid, h->stream));
  launch_spmm_real<double>(h->n, h->rowptr, h->colidx, h->val64, m, ld, 1.0, h->shift, X, tmp2,
                           h->num_sms, h->stream);
  gram_dev(h, X, tmp2, m, ld, d.G, d, true);  // X^T A X
  small_gemm(d.G, 0, d.Rinv, 0, d.R, m, 1.0, 0.0, h->stream);            // (X^T A X) R^-1
  small_gemm(d.Rinv, 1, d.R, 0, d.G, m, 1.0, 0.0, h->stream);            // R^-T (.)
  jacobi_eigh(d.G, m, theta_d, d.V, d.Vw, h->stream);
  small_gemm(d.Rinv, 0, d.V, 0, d.R, m, 1.0, 0.0, h->stream);  // R^-1 V
  tall_dev(h, X, m, ld, d.R, m, Qout, ld);
  launch_spmm_real<double>(h->n, h->rowptr, h->colidx, h->val64, m, ld, 1.0, h->shift, Qout,
                           AQout, h->num_sms, h->stream);
  h->launches += 9;
  h->spmm_launches += 2;
  return shifted;
}

static void residuals_host(Handle* h, const double* Q, const double* AQ, const double* theta_d,
                           int m, int ld, std::vector<double>& res) {
  DenseWs d = dense_ws(h, m);
  col_resid2(Q, AQ, theta_d, h->n, m, ld, d.small, d.part, h->num_sms, h->stream);
  h->launches += 2;
  res.resize(m);
  RF_CUDA(cudaMemcpyAsync(res.data(), d.small, sizeof(double) * m, cudaMemcpyDeviceToHost,
                          h->stream));
  RF_CUDA(cudaStreamSynchronize(h->stream));
  for (int i = 0; i < m; ++i) res[i] = std::sqrt(std::max(res[i], 0.0)) / h->norm1;
}

// ---------------------------------------------------------------------------
// batched COCG filter: Qt = sum_j Re(w_j X_j), (z_j I - A) X_j = Q
// ---------------------------------------------------------------------------
struct FilterStats {
  int iters_max = 0, iters_min = 0, breakdown = 0, capped = 0;
};

// a shift-sharded filter sums over the nodes [shard_j0, shard_j1) only: the
// partial filtered blocks of all ranks add up to the N_c-node sum (Eq. 2)
static void shard_nodes(const Handle* h, std::vector<double>& zr, std::vector<double>& zi,
                        std::vector<double>& wr, std::vector<double>& wi) {
  if (h->shard_j1 < 0) return;
  const int nc = (int)zr.size();
  const int j0 = std::max(0, std::min(h->shard_j0, nc)), j1 = std::max(j0, std::min(h->shard_j1, nc));
  for (auto* v : {&zr, &zi, &wr, &wi}) *v = std::vector<double>(v->begin() + j0, v->begin() + j1);
}

template <typename T>
static void filter_dev(Handle* h, const rafeast_params& prm, const double* Qd, const double* AQd,
                       const double* theta_d, const std::vector<double>& theta, int m0, int ldq,
                       double* Qt, FilterStats& fs) {
  using C = c2<T>;
  const bool fp64 = sizeof(T) == 8;
  std::vector<double> zr, zi, wr, wi;
  quadrature_nodes(prm.lmin, prm.lmax, prm.nc, prm.ellipse_ratio, zr, zi, wr, wi);
  shard_nodes(h, zr, zi, wr, wi);
  const int nc = (int)zr.size();
  const int NC = nc_pad(nc);
  const int nsys = m0 * NC;
  const bool corr = prm.solve_form == RAFEAST_FORM_CORRECTION;
  // host-side small tables
  std::vector<double2> coef(nsys);
  std::vector<double> finit(m0, 0.0);
  for (int i = 0; i < m0; ++i)
    for (int j = 0; j < NC; ++j) {
      double2 c = make_double2(0.0, 0.0);
      if (j < nc) {
        if (corr) {
          // w_j / (z_j - theta_i)
          const double dr = zr[j] - theta[i], di = zi[j];
          const double den = dr * dr + di * di;
          c = make_double2((wr[j] * dr + wi[j] * di) / den, (wi[j] * dr - wr[j] * di) / den);
          finit[i] += c.x;
        } else {
          c = make_double2(wr[j], wi[j]);
        }
      }
      coef[i * NC + j] = c;
    }
  std::vector<C> zs(NC);
  for (int j = 0; j < NC; ++j) {
    const int jj = j < nc ? j : 0;
    zs[j].x = (T)(zr[jj] - h->shift);
    zs[j].y = (T)zi[jj];
  }
  // kernel family: bulk-copy gathers for float32 with NC >= 2 (default),
  // register gathers otherwise
  const bool use_tma = !fp64 && NC >= 2 && h->opt_kernel == 2;
  // device buffers
  const int ldc = even(m0 * NC);
  size_t state_elems = (size_t)h->n * ldc * 2;
  if (use_tma) state_elems = (size_t)h->n * m0 * NC * 2;  // blocked, no padding
  T* state = (T*)scratch(h, S_STATE, 4 * state_elems * sizeof(T));
  const int ldd = m0;
  T* dacc = (T*)scratch(h, S_DACC, (size_t)h->n * ldd * sizeof(T));
  size_t off = 0;
  auto carve = [&](size_t bytes) {
    off = (off + 255) & ~(size_t)255;
    size_t o = off;
    off += bytes;
    return o;
  };
  const size_t o_acc = carve(sizeof(double) * 5 * nsys);
  const size_t o_st = carve(sizeof(SysState) * nsys);
  const size_t o_cf = carve(sizeof(Coef<T>) * nsys);
  const size_t o_col = carve(sizeof(int) * m0);
  const size_t o_ctl = carve(sizeof(CocgCtl));
  const size_t o_zs = carve(sizeof(C) * NC);
  const size_t o_coef = carve(sizeof(double2) * nsys);
  const size_t o_fin = carve(sizeof(double) * m0);
  const size_t o_hist = carve(sizeof(int) * ((size_t)prm.max_inner + 2));
  const size_t o_rhist = carve(sizeof(double) * ((size_t)prm.max_inner + 2));
  char* sc = (char*)scratch(h, S_SCAL, off + 256);
  RF_CUDA(cudaMemcpyAsync(sc + o_zs, zs.data(), sizeof(C) * NC, cudaMemcpyHostToDevice, h->stream));
  RF_CUDA(cudaMemcpyAsync(sc + o_coef, coef.data(), sizeof(double2) * nsys, cudaMemcpyHostToDevice,
                          h->stream));
  RF_CUDA(cudaMemcpyAsync(sc + o_fin, finit.data(), sizeof(double) * m0, cudaMemcpyHostToDevice,
                          h->stream));
  CocgArgs<T> a;
  memset(&a, 0, sizeof(a));
  a.n = h->n;
  a.rowptr = h->rowptr;
  a.colidx = h->colidx;
  a.val = fp64 ? (const T*)h->val64 : (const T*)h->val32;
  a.m0 = m0;
  a.ldc = ldc;
  int colblocks = 1;
  choose_shape(m0, NC, fp64, h->opt_lanes, a.lanes, a.cpl, colblocks, h->opt_cpl);
  a.r[0] = state;
  a.r[1] = state + state_elems;
  a.p[0] = state + 2 * state_elems;
  a.p[1] = state + 3 * state_elems;
  a.dacc = dacc;
  a.ldd = ldd;
  a.qin = Qd;
  a.aqin = AQd;
  a.ldq = ldq;
  a.theta = theta_d;
  a.zs = sc + o_zs;
  a.coef = (const double2*)(sc + o_coef);
  a.acc = (double*)(sc + o_acc);
  a.st = (SysState*)(sc + o_st);
  a.cf = (Coef<T>*)(sc + o_cf);
  a.colact = (int*)(sc + o_col);
  a.ctl = (CocgCtl*)(sc + o_ctl);
  a.hist = h->opt_profile ? (int*)(sc + o_hist) : nullptr;
  a.rhist = h->opt_profile ? (double*)(sc + o_rhist) : nullptr;
  a.nc_real = nc;
  a.tol2 = prm.solve_tol * prm.solve_tol;
  a.max_inner = prm.max_inner;
  a.form = prm.solve_form;
  a.wait_cycles = h->opt_wait_cycles;
  a.stall_bytes = h->opt_stall_bytes;
  const int maxnz = h->opt_maxnz;
  if constexpr (sizeof(T) == 4) {
    if (use_tma) {
      launch_cocg_reset<T>(a, NC, h->stream);
      launch_cocg_tma(a, NC, 0, 0, maxnz, h->num_sms, h->stream);
    } else {
      launch_cocg_init<T>(a, NC, h->num_sms, h->stream);
    }
  } else {
    launch_cocg_init<T>(a, NC, h->num_sms, h->stream);
  }
  h->launches += 2;
  // capture `chunk` COCG steps as one graph (with event nodes around every
  // kernel when profiling, so kernel times are measured inside the replays)
  int chunk = std::max(2, h->opt_chunk);
  chunk += chunk & 1;
  const bool prof = h->opt_profile != 0;
  std::vector<cudaEvent_t> evs;
  if (prof) {
    evs.resize(2 * chunk + 1);
    for (auto& e : evs) RF_CUDA(cudaEventCreate(&e));
  }
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  RF_CUDA(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
  g_capturing = true;
  try {
    for (int it = 0; it < chunk; ++it) {
      // external records: the graph itself records the event on each replay
      if (prof) RF_CUDA(cudaEventRecordWithFlags(evs[2 * it], h->stream, cudaEventRecordExternal));
      if constexpr (sizeof(T) == 4) {
        if (use_tma) launch_cocg_tma(a, NC, 1, it & 1, maxnz, h->num_sms, h->stream);
        else launch_cocg_dots<T>(a, NC, it & 1, h->num_sms, h->stream);
      } else {
        launch_cocg_dots<T>(a, NC, it & 1, h->num_sms, h->stream);
      }
      if (prof)
        RF_CUDA(cudaEventRecordWithFlags(evs[2 * it + 1], h->stream, cudaEventRecordExternal));
      if constexpr (sizeof(T) == 4) {
        if (use_tma) launch_cocg_tma(a, NC, 2, it & 1, maxnz, h->num_sms, h->stream);
        else launch_cocg_update<T>(a, NC, it & 1, h->num_sms, h->stream);
      } else {
        launch_cocg_update<T>(a, NC, it & 1, h->num_sms, h->stream);
      }
    }
    if (prof) RF_CUDA(cudaEventRecordWithFlags(evs[2 * chunk], h->stream, cudaEventRecordExternal));
  } catch (...) {
    g_capturing = false;
    cudaStreamEndCapture(h->stream, &graph);
    if (graph) cudaGraphDestroy(graph);
    for (auto& e : evs) cudaEventDestroy(e);
    throw;
  }
  g_capturing = false;
  RF_CUDA(cudaStreamEndCapture(h->stream, &graph));
  RF_CUDA(cudaGraphInstantiate(&exec, graph, 0));
  CocgCtl ctl;
  const int max_replays = (prm.max_inner + 2) / chunk + 2;
  int replays = 0;
  std::vector<float> tk;  // per iteration k: dots ms, update ms
  for (; replays < max_replays; ++replays) {
    RF_CUDA(cudaGraphLaunch(exec, h->stream));
    RF_CUDA(cudaMemcpyAsync(&ctl, a.ctl, sizeof(ctl), cudaMemcpyDeviceToHost, h->stream));
    RF_CUDA(cudaStreamSynchronize(h->stream));
    if (prof)
      for (int it = 0; it < 2 * chunk; ++it) {
        float ms = 0.f;
        RF_CUDA(cudaEventElapsedTime(&ms, evs[it], evs[it + 1]));
        tk.push_back(ms);
      }
    if (ctl.done) break;
  }
  h->launches += 2 * chunk * (replays + 1);
  h->spmm_launches += 2 * chunk * (replays + 1);
  RF_CUDA(cudaGraphExecDestroy(exec));
  RF_CUDA(cudaGraphDestroy(graph));
  for (auto& e : evs) RF_CUDA(cudaEventDestroy(e));
  if (prof && ctl.done) {
    // algorithmic bytes: A once, plus the state columns each kernel touches
    const int iters = std::min(ctl.iter, prm.max_inner + 1);
    std::vector<int> hist(iters + 1, 0);
    RF_CUDA(cudaMemcpy(hist.data(), a.hist, sizeof(int) * iters, cudaMemcpyDeviceToHost));
    h->last_hist.assign(hist.begin(), hist.begin() + iters);
    h->last_tk.assign(tk.begin(), tk.begin() + std::min<size_t>(tk.size(), 2 * (size_t)iters));
    h->last_rhist.assign(iters, 0.0);
    RF_CUDA(cudaMemcpy(h->last_rhist.data(), a.rhist, sizeof(double) * iters,
                       cudaMemcpyDeviceToHost));
    const double sv = fp64 ? 8.0 : 4.0;
    const double abytes = (double)h->nnz * (4.0 + sv) + 4.0 * (h->n + 1);
    const double colb = (double)h->n * NC * 2.0 * sv;  // one column i of one state array
    for (int k = 0; k < iters && 2 * k + 1 < (int)tk.size(); ++k) {
      const int act_d = k == 0 ? m0 : hist[k - 1];
      const int act_u = hist[k];
      h->prof[0] += 1;
      h->prof[1] += tk[2 * k];
      h->prof[2] += abytes + colb * act_d;
      if (act_u > 0) {
        h->prof[3] += 1;
        h->prof[4] += tk[2 * k + 1];
        h->prof[5] += abytes + 4.0 * colb * act_u + 2.0 * (double)h->n * act_u * sv;
      }
    }
  }
  if (!ctl.done || ctl.timeout) throw Err{RAFEAST_ERR_TIMEOUT};
  fs.iters_max = ctl.max_iters;
  fs.iters_min = ctl.min_iters;
  fs.breakdown = ctl.breakdown;
  fs.capped = ctl.capped;
  // Qt = f(theta) Q + D
  launch_combine<T>(Qd, ldq, dacc, ldd, (const double*)(sc + o_fin), h->n, m0, Qt, h->stream);
  h->launches += 1;
  if (fs.breakdown) throw Err{RAFEAST_ERR_COCG_BREAKDOWN};
}

// multi-shift COCG filter: one seed Krylov recurrence per column (the shift
// nearest the real axis), every other shift from the seed's scalars; same
// Q~ as filter_dev in exact arithmetic, a quarter of the gathered bytes at
// N_c = 4.
template <typename T>
struct MsProblem {
  CocgArgs<T> a;
  const double* fin = nullptr;  // device [m0]: per-column constant of the correction form
  int m0 = 0, pairs = 0, ns = 0;
};

// one multi-shift problem on stream st: quadrature, seed choice, coefficient
// upload, state reset and init (two launches); default kernel shape. ctl_dev,
// when not null, replaces the handle's own control block (batched solves keep
// every problem's block in one array).
template <typename T>
static MsProblem<T> ms_setup(Handle* h, const rafeast_params& prm, const double* Qd,
                             const double* AQd, const double* theta_d,
                             const std::vector<double>& theta, int m0, int ldq, CocgCtl* ctl_dev,
                             bool profile, bool stream, cudaStream_t st, bool pingpong = false) {
  using C = c2<T>;
  const bool fp64 = sizeof(T) == 8;
  std::vector<double> zr, zi, wr, wi;
  quadrature_nodes(prm.lmin, prm.lmax, prm.nc, prm.ellipse_ratio, zr, zi, wr, wi);
  shard_nodes(h, zr, zi, wr, wi);
  const int nc = (int)zr.size();
  int seed = 0;
  for (int j = 1; j < nc; ++j)
    if (zi[j] < zi[seed]) seed = j;
  const int ns = nc - 1;
  std::vector<int> others;
  for (int j = 0; j < nc; ++j)
    if (j != seed) others.push_back(j);
  const bool corr = prm.solve_form == RAFEAST_FORM_CORRECTION;
  const int pairs = (m0 + 1) / 2, ncol = 2 * pairs;
  auto coef_of = [&](int j, int i) {
    if (i >= m0) return make_double2(0.0, 0.0);
    if (!corr) return make_double2(wr[j], wi[j]);
    const double dr = zr[j] - theta[i], di = zi[j];
    const double den = dr * dr + di * di;
    return make_double2((wr[j] * dr + wi[j] * di) / den, (wi[j] * dr - wr[j] * di) / den);
  };
  std::vector<double2> coef(ncol), scoef((size_t)ncol * std::max(ns, 1));
  std::vector<double> finit(m0, 0.0);
  for (int i = 0; i < ncol; ++i) {
    coef[i] = coef_of(seed, i);
    for (int t = 0; t < ns; ++t) scoef[(size_t)i * ns + t] = coef_of(others[t], i);
  }
  if (corr)
    for (int i = 0; i < m0; ++i)
      for (int j = 0; j < nc; ++j) finit[i] += coef_of(j, i).x;
  std::vector<double2> sigma(std::max(ns, 1));
  for (int t = 0; t < ns; ++t)
    sigma[t] = make_double2(zr[others[t]] - zr[seed], zi[others[t]] - zi[seed]);
  std::vector<C> zs(2);
  zs[0].x = zs[1].x = (T)(zr[seed] - h->shift);
  zs[0].y = zs[1].y = (T)zi[seed];
  // device buffers
  const int ldc = ncol;                     // seed arrays: complex per row
  const int ldps = pairs * ns * 2;          // shifted directions: complex per row
  const size_t seed_elems = (size_t)h->n * ldc * 2;
  const size_t ps_elems = (size_t)h->n * std::max(ldps, 1) * 2;
  // seed r, p, w, s, the shifted directions, and (ping-pong) a second r
  T* state = (T*)scratch(h, S_STATE,
                         ((pingpong ? 5 : 4) * seed_elems + ps_elems) * sizeof(T));
  const int ldd = ncol;
  T* dacc = (T*)scratch(h, S_DACC, (size_t)h->n * ldd * sizeof(T));
  size_t off = 0;
  auto carve = [&](size_t bytes) {
    off = (off + 255) & ~(size_t)255;
    size_t o = off;
    off += bytes;
    return o;
  };
  const size_t o_acc = carve(sizeof(double) * 5 * ncol);
  const size_t o_st = carve(sizeof(SysState) * ncol);
  const size_t o_cf = carve(sizeof(Coef<T>) * ncol);
  const size_t o_col = carve(sizeof(int) * pairs);
  const size_t o_ctl = carve(sizeof(CocgCtl));
  const size_t o_zs = carve(sizeof(C) * 2);
  const size_t o_coef = carve(sizeof(double2) * ncol);
  const size_t o_fin = carve(sizeof(double) * m0);
  const size_t o_sig = carve(sizeof(double2) * sigma.size());
  const size_t o_scoef = carve(sizeof(double2) * scoef.size());
  const size_t o_sst = carve(sizeof(ShiftState) * scoef.size());
  const size_t o_scf = carve(sizeof(ShiftCoef<T>) * scoef.size());
  const size_t o_hist = carve(sizeof(int) * ((size_t)prm.max_inner + 2));
  const size_t o_rhist = carve(sizeof(double) * ((size_t)prm.max_inner + 2));
  char* sc = (char*)scratch(h, S_SCAL, off + 256);
  RF_CUDA(cudaMemcpyAsync(sc + o_zs, zs.data(), sizeof(C) * 2, cudaMemcpyHostToDevice, st));
  RF_CUDA(cudaMemcpyAsync(sc + o_coef, coef.data(), sizeof(double2) * ncol, cudaMemcpyHostToDevice,
                          st));
  RF_CUDA(cudaMemcpyAsync(sc + o_fin, finit.data(), sizeof(double) * m0, cudaMemcpyHostToDevice,
                          st));
  RF_CUDA(cudaMemcpyAsync(sc + o_sig, sigma.data(), sizeof(double2) * sigma.size(),
                          cudaMemcpyHostToDevice, st));
  RF_CUDA(cudaMemcpyAsync(sc + o_scoef, scoef.data(), sizeof(double2) * scoef.size(),
                          cudaMemcpyHostToDevice, st));
  CocgArgs<T> a;
  memset(&a, 0, sizeof(a));
  a.n = h->n;
  a.rowptr = h->rowptr;
  a.colidx = h->colidx;
  a.val = fp64 ? (const T*)h->val64 : (const T*)h->val32;
  a.m0 = pairs;
  a.ldc = ldc;
  int colblocks = 1;
  choose_shape(pairs, 2, fp64, h->opt_lanes, a.lanes, a.cpl, colblocks,
               h->opt_cpl > 0 ? std::min(h->opt_cpl, ms_max_cpl(fp64)) : ms_max_cpl(fp64));
  if (stream) {
    // r and p in place, w = M r and s = M p beside them
    // r in place, or r_k / r_{k+1} alternating between two arrays (the
    // deferred form of the update still needs r_k after r_{k+1} is formed)
    a.r[0] = a.r[1] = state;
    if (pingpong) a.r[1] = state + 4 * seed_elems + ps_elems;
    a.p[0] = a.p[1] = state + seed_elems;
    a.wbuf = state + 2 * seed_elems;
    a.sbuf = state + 3 * seed_elems;
  } else {
    a.r[0] = state;
    a.r[1] = state + seed_elems;
    a.p[0] = state + 2 * seed_elems;
    a.p[1] = state + 3 * seed_elems;
  }
  a.ps = state + 4 * seed_elems;
  a.ldps = ldps;
  a.dacc = dacc;
  a.ldd = ldd;
  a.qin = Qd;
  a.aqin = AQd;
  a.ldq = ldq;
  a.theta = theta_d;
  a.zs = sc + o_zs;
  a.coef = (const double2*)(sc + o_coef);
  a.acc = (double*)(sc + o_acc);
  a.st = (SysState*)(sc + o_st);
  a.cf = (Coef<T>*)(sc + o_cf);
  a.colact = (int*)(sc + o_col);
  a.ctl = (CocgCtl*)(sc + o_ctl);
  a.hist = profile ? (int*)(sc + o_hist) : nullptr;
  a.rhist = profile ? (double*)(sc + o_rhist) : nullptr;
  a.nc_real = 2;
  a.tol2 = prm.solve_tol * prm.solve_tol;
  a.max_inner = prm.max_inner;
  a.form = prm.solve_form;
  a.wait_cycles = h->opt_wait_cycles;
  a.ms = 1;
  a.ns = ns;
  a.nc_total = nc;
  a.sigma = (const double2*)(sc + o_sig);
  a.scoef = (const double2*)(sc + o_scoef);
  a.sst = (ShiftState*)(sc + o_sst);
  a.scf = (ShiftCoef<T>*)(sc + o_scf);
  if (ctl_dev) a.ctl = ctl_dev;
  if (h->lcolidx && h->opt_values_free == 0) {
    a.lrowptr = h->lrowptr;
    a.lcolidx = h->lcolidx;
  }
  launch_ms_init<T>(a, m0, h->num_sms, st);
  h->launches += 2;
  MsProblem<T> P;
  P.a = a;
  P.fin = (const double*)(sc + o_fin);
  P.m0 = m0;
  P.pairs = pairs;
  P.ns = ns;
  return P;
}

// algorithmic bytes of one multi-shift step of a problem with act_d pairs
// active in the dot kernel and act_u in the update kernel: A once per kernel;
// the dot kernel reads the seed residual; the update kernel reads and writes
// the seed r and p, the shifted directions and the quadrature sum
// (streamed update: the dot kernel also writes w; the update kernel reads
// r, p, w, s and writes r, p, s, and reads no A)
static double ms_dots_bytes(const Handle* h, int act_d, bool fp64, bool stream = false,
                            bool vf = false, int defer_ns = -1) {
  const double sv = fp64 ? 8.0 : 4.0;
  // values-free gathers read the off-diagonal pattern only
  const double abytes = vf ? (double)h->nnz_off * 4.0 + 4.0 * (h->n + 1)
                           : (double)h->nnz * (4.0 + sv) + 4.0 * (h->n + 1);
  const double pairb = (double)h->n * 2 * 2.0 * sv;
  double b = abytes + pairb * act_d * (stream ? 2.0 : 1.0);
  // deferred form: the previous residual read, the shifted directions read
  // and written, the quadrature sum read and written
  if (defer_ns >= 0) b += (1.0 + 2.0 * defer_ns + 1.0) * pairb * act_d;
  return b;
}
static double ms_update_bytes(const Handle* h, int act_u, int ns, bool fp64,
                              bool stream = false, bool defer = false) {
  const double sv = fp64 ? 8.0 : 4.0;
  const double abytes = (double)h->nnz * (4.0 + sv) + 4.0 * (h->n + 1);
  const double pairb = (double)h->n * 2 * 2.0 * sv;
  const double dacc = 2.0 * (double)h->n * 2 * act_u * sv;
  if (stream && defer) return 7.0 * pairb * act_u + dacc;
  if (stream) return (7.0 + 2.0 * ns) * pairb * act_u + dacc;
  return abytes + (4.0 + 2.0 * ns) * pairb * act_u + dacc;
}

// combine Qt = f Q + D and the solve's statistics (after the device reported done)
template <typename T>
static void ms_finish(Handle* h, const MsProblem<T>& P, const double* Qd, int ldq, double* Qt,
                      const CocgCtl& ctl, FilterStats& fs, cudaStream_t st) {
  if (!ctl.done || ctl.timeout) throw Err{RAFEAST_ERR_TIMEOUT};
  fs.iters_max = ctl.max_iters;
  fs.iters_min = ctl.min_iters;
  fs.breakdown = ctl.breakdown;
  fs.capped = ctl.capped;
  launch_combine<T>(Qd, ldq, P.a.dacc, P.a.ldd, P.fin, h->n, P.m0, Qt, st);
  h->launches += 1;
  if (fs.breakdown) throw Err{RAFEAST_ERR_COCG_BREAKDOWN};
}

template <typename T>
static void filter_ms_dev(Handle* h, const rafeast_params& prm, const double* Qd,
                          const double* AQd, const double* theta_d,
                          const std::vector<double>& theta, int m0, int ldq, double* Qt,
                          FilterStats& fs) {
  const bool fp64 = sizeof(T) == 8;
  // (the gathering update is compiled for up to 8 shifts)
  const bool stream = h->opt_update != 1 || prm.nc > 8;
  // float32 streamed update, deferred form asked for: residuals ping-pong,
  // so that the tiled dot kernel can take over the shifted updates
  const bool pingpong = stream && !fp64 && h->opt_defer == 1 && h->ntiles > 0;
  MsProblem<T> P = ms_setup<T>(h, prm, Qd, AQd, theta_d, theta, m0, ldq, nullptr,
                                h->opt_profile != 0, stream, h->stream, pingpong);
  const CocgArgs<T>& a = P.a;
  const int pairs = P.pairs, ns = P.ns;
  const bool prof = h->opt_profile != 0;
  std::vector<float> tk;  // per executed step: dot ms, update ms (profiling)
  CocgCtl ctl;
  memset(&ctl, 0, sizeof(ctl));
  // tiled seed dot kernel (float32, streamed update, the matrix has tiles):
  // the tile arrays and the per-CTA sums; tl_for(cb) describes the launch
  // with cb column pairs per block
  const bool vf = a.lcolidx != nullptr;
  const bool can_tile = !fp64 && stream && h->ntiles > 0 && h->opt_tiled != 1 &&
                        (vf ? h->llidx != nullptr : h->lidx != nullptr);
  double* tpart = can_tile ? (double*)scratch(h, S_TPART, sizeof(double) * (size_t)h->num_sms *
                                                             TILE_MAX_OCC * 16 * 10)
                           : nullptr;
  auto tl_for = [&](int cb) {
    TileArgs tl;
    tl.ntiles = h->ntiles;
    tl.max_union = h->tile_max_union;
    tl.trow = h->trow;
    tl.uoff = h->uoff;
    tl.ucol = h->ucol;
    tl.uself = h->uself;
    tl.lidx = vf ? h->llidx : h->lidx;
    tl.cb = cb;
    tl.ncb = (pairs + cb - 1) / cb;
    tl.part = tpart;
    return tl;
  };
  int dot_cb = 0, dot_occ = 0;  // tiled dot kernel shape in use (dot_cb = 0: register gathers)
  auto launch_dots = [&](const CocgArgs<T>& ad, int buf, int cb, int occ) {
    if constexpr (std::is_same<T, float>::value) {
      if (cb > 0) {
        launch_ms_dots_tiled(ad, tl_for(cb), buf, h->num_sms, occ, h->stream);
        return;
      }
    }
    launch_cocg_dots<T>(ad, 2, buf, h->num_sms, h->stream);
  };
  // capture `steps` COCG steps with the given shapes; event nodes around each
  // kernel when timing is wanted (the graph records them on every replay)
  auto capture = [&](const CocgArgs<T>& ad, const CocgArgs<T>& au, int steps, bool timed,
                     std::vector<cudaEvent_t>& evs, cudaGraphExec_t& exec, int cb = 0,
                     int occ = 0) {
    if (timed) {
      evs.resize(2 * steps + 1);
      for (auto& e : evs) RF_CUDA(cudaEventCreate(&e));
    }
    cudaGraph_t graph = nullptr;
    RF_CUDA(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    g_capturing = true;
    try {
      for (int it = 0; it < steps; ++it) {
        if (timed)
          RF_CUDA(cudaEventRecordWithFlags(evs[2 * it], h->stream, cudaEventRecordExternal));
        launch_dots(ad, it & 1, cb, occ);
        if (timed)
          RF_CUDA(cudaEventRecordWithFlags(evs[2 * it + 1], h->stream, cudaEventRecordExternal));
        if (stream) launch_ms_update_stream<T>(au, it & 1, h->num_sms, h->stream);
        else launch_ms_update<T>(au, it & 1, h->num_sms, h->stream);
      }
      if (timed)
        RF_CUDA(cudaEventRecordWithFlags(evs[2 * steps], h->stream, cudaEventRecordExternal));
    } catch (...) {
      g_capturing = false;
      cudaStreamEndCapture(h->stream, &graph);
      if (graph) cudaGraphDestroy(graph);
      throw;
    }
    g_capturing = false;
    RF_CUDA(cudaStreamEndCapture(h->stream, &graph));
    RF_CUDA(cudaGraphInstantiate(&exec, graph, 0));
    RF_CUDA(cudaGraphDestroy(graph));
  };
  auto replay = [&](cudaGraphExec_t exec, int steps, bool timed, std::vector<cudaEvent_t>& evs,
                    std::vector<float>* out) {
    RF_CUDA(cudaGraphLaunch(exec, h->stream));
    RF_CUDA(cudaMemcpyAsync(&ctl, a.ctl, sizeof(ctl), cudaMemcpyDeviceToHost, h->stream));
    RF_CUDA(cudaStreamSynchronize(h->stream));
    if (timed && out)
      for (int it = 0; it < 2 * steps; ++it) {
        float ms = 0.f;
        RF_CUDA(cudaEventElapsedTime(&ms, evs[it], evs[it + 1]));
        out->push_back(ms);
      }
    h->launches += 2 * steps;
    h->spmm_launches += 2 * steps;
  };
  // K10 autotuner: the dot and update kernels take their own (lanes, chunks)
  // shape. Untuned, each candidate runs two real COCG steps (timed by graph
  // event nodes) at the start of this solve; the fastest per kernel is kept
  // for this handle. Shapes change only the work split, not the arithmetic.
  CocgArgs<T> ad = a, au = a;
  ad.occ = au.occ = 0;
  const int64_t key =
      ((int64_t)pairs << 20) | ((int64_t)ns << 4) | (stream ? 2 : 0) | (fp64 ? 1 : 0);
  const int cap = h->opt_cpl > 0 ? std::min(h->opt_cpl, ms_max_cpl(fp64)) : ms_max_cpl(fp64);
  bool have = false;
  for (auto& kv : h->tuned)
    if (kv.first == key) {
      ad.lanes = kv.second.dl;
      ad.cpl = kv.second.dc;
      ad.occ = kv.second.dm;
      au.lanes = kv.second.ul;
      au.cpl = kv.second.uc;
      au.occ = kv.second.um;
      dot_cb = can_tile ? kv.second.dt : 0;
      dot_occ = kv.second.dt ? kv.second.dm : 0;
      if (h->opt_tiled == 2 && can_tile && dot_cb == 0) have = false;  // retune
      else have = true;
    }
  const bool tune = h->opt_autotune && !h->opt_lanes && !h->opt_cpl;
  int tuned_steps = 0;  // COCG steps the autotuner ran (full updates)
  if (!have && !tune && can_tile && h->opt_tiled == 2) dot_cb = 8;
  if (!have && tune) {
    // (lanes, chunks, CTAs per SM; 0 = the default instance)
    // (the last three only for FP64, whose one-chunk dot instance runs at
    // 3 CTAs per SM)
    const int cand[][3] = {{32, 2, 0}, {16, 2, 0}, {16, 3, 0}, {16, 4, 0}, {8, 1, 0},
                           {8, 2, 0},  {8, 4, 0},  {4, 2, 0},  {32, 2, 3}, {16, 2, 3},
                           {8, 2, 3},  {16, 2, 4}, {16, 3, 2}, {16, 4, 2}, {8, 3, 2},
                           {8, 4, 2},  {16, 3, 3}, {4, 1, 0},  {16, 1, 0}, {32, 1, 0}};
    const int n_all = (int)(sizeof(cand) / sizeof(cand[0])), n_fp64_only = 3;
    float best_d = 1e30f, best_u = 1e30f;
    for (int ci = 0; ci < n_all; ++ci) {
      const int* c = cand[ci];
      if (ctl.done) break;
      if (!fp64 && ci >= n_all - n_fp64_only) continue;
      const int G = c[0], cpl = c[1];
      if (cpl > cap) continue;
      if (c[2] && fp64) continue;
      const int blocks = (pairs + G * cpl - 1) / (G * cpl);
      if ((double)pairs / (blocks * G * cpl) < 0.5) continue;
      CocgArgs<T> t = a;
      t.lanes = G;
      t.cpl = cpl;
      t.occ = c[2];
      std::vector<cudaEvent_t> evs;
      cudaGraphExec_t exec = nullptr;
      capture(t, t, 2, true, evs, exec);
      std::vector<float> times;
      replay(exec, 2, true, evs, &times);
      RF_CUDA(cudaGraphExecDestroy(exec));
      for (auto& e : evs) RF_CUDA(cudaEventDestroy(e));
      tk.insert(tk.end(), times.begin(), times.end());
      // second step of the pair: its kernels ran with every column active
      // unless the solve already finished
      const float td = std::min(times[0], times[2]), tu = std::min(times[1], times[3]);
      if (td < best_d) {
        best_d = td;
        ad.lanes = G;
        ad.cpl = cpl;
        ad.occ = c[2];
      }
      if (tu < best_u) {
        best_u = tu;
        au.lanes = G;
        au.cpl = cpl;
        au.occ = c[2];
      }
    }
    // tiled dot kernel: column pairs per block x CTAs per SM (0: as many as
    // fit); only the dot kernel's time counts, the update is the streamed one.
    // Its sums are added in a fixed order (solves repeat to the last bit), so
    // it is kept unless the register gathers are more than 5% faster.
    if (can_tile) {
      const int tcand[][2] = {{8, 0}, {4, 0}, {8, 2}, {4, 4}};
      float best_t = 1e30f;
      int tcb = 0, tocc = 0;
      for (const auto& c : tcand) {
        if (ctl.done) break;
        if (c[0] > 2 * pairs && c[0] > 4) continue;  // mostly empty blocks
        std::vector<cudaEvent_t> evs;
        cudaGraphExec_t exec = nullptr;
        capture(au, au, 2, true, evs, exec, c[0], c[1]);
        std::vector<float> times;
        replay(exec, 2, true, evs, &times);
        RF_CUDA(cudaGraphExecDestroy(exec));
        for (auto& e : evs) RF_CUDA(cudaEventDestroy(e));
        tk.insert(tk.end(), times.begin(), times.end());
        const float td = std::min(times[0], times[2]);
        if (td < best_t) {
          best_t = td;
          tcb = c[0];
          tocc = c[1];
        }
      }
      if (tcb && (h->opt_tiled == 2 || best_t <= 1.05f * best_d)) {
        dot_cb = tcb;
        dot_occ = tocc;
      }
    }
    Handle::Shape shp;
    shp.dl = ad.lanes;
    shp.dc = ad.cpl;
    shp.dm = dot_cb ? dot_occ : ad.occ;
    shp.ul = au.lanes;
    shp.uc = au.cpl;
    shp.um = au.occ;
    shp.dt = dot_cb;
    h->tuned.push_back(std::make_pair(key, shp));
  }
  if (can_tile && h->opt_tiled == 2 && h->opt_tile_cb > 0) {
    dot_cb = h->opt_tile_cb;  // forced block width (tests)
    dot_occ = 0;
  }
  h->prof[6] = dot_cb ? 1000000 + dot_cb * 100 + dot_occ : ad.occ * 10000 + ad.lanes * 100 + ad.cpl;
  h->prof[7] = au.occ * 10000 + au.lanes * 100 + au.cpl;
  tuned_steps = (int)tk.size() / 2;
  int chunk = std::max(2, h->opt_chunk);
  chunk += chunk & 1;
  // deferred form (RAFEAST_OPT_DEFER = 1, tiled dot kernel, ping-pong
  // residuals): the update kernel leaves the shifted directions to the next
  // dot kernel; the first dot kernel after a full update finds nothing
  // pending
  const bool defer = pingpong && dot_cb > 0;
  ad.defer = au.defer = defer ? 1 : 0;
  std::vector<cudaEvent_t> evs;
  cudaGraphExec_t exec = nullptr;
  capture(ad, au, chunk, prof, evs, exec, dot_cb, dot_occ);
  const int max_replays = (prm.max_inner + 2) / chunk + 2;
  int replays = 0;
  for (; replays < max_replays && !ctl.done; ++replays) {
    replay(exec, chunk, prof, evs, &tk);
  }
  RF_CUDA(cudaGraphExecDestroy(exec));
  for (auto& e : evs) RF_CUDA(cudaEventDestroy(e));
  if (prof && ctl.done) {
    const int iters = std::min(ctl.iter, prm.max_inner + 1);
    std::vector<int> hist(iters + 1, 0);
    RF_CUDA(cudaMemcpy(hist.data(), a.hist, sizeof(int) * iters, cudaMemcpyDeviceToHost));
    h->last_hist.assign(hist.begin(), hist.begin() + iters);
    h->last_rhist.assign(iters, 0.0);
    RF_CUDA(cudaMemcpy(h->last_rhist.data(), a.rhist, sizeof(double) * iters,
                       cudaMemcpyDeviceToHost));
    h->last_tk.assign(tk.begin(), tk.begin() + std::min<size_t>(tk.size(), 2 * (size_t)iters));
    for (int k = 0; k < iters && 2 * k + 1 < (int)tk.size(); ++k) {
      const int act_d = k == 0 ? pairs : hist[k - 1];
      const int act_u = hist[k];
      h->prof[0] += 1;
      h->prof[1] += tk[2 * k];
      // (the autotuner's steps ran the full update; k counts from the
      // solve's first step, the deferred form starts after them)
      const bool dk = defer && k >= tuned_steps + 1, uk = defer && k >= tuned_steps;
      h->prof[2] += ms_dots_bytes(h, act_d, fp64, stream, a.lcolidx != nullptr, dk ? ns : -1);
      if (act_u > 0) {
        h->prof[3] += 1;
        h->prof[4] += tk[2 * k + 1];
        h->prof[5] += ms_update_bytes(h, act_u, ns, fp64, stream, uk);
      }
    }
  }
  ms_finish<T>(h, P, Qd, ldq, Qt, ctl, fs, h->stream);
}

// ---------------------------------------------------------------------------
// batched multi-shift filter: the COCG steps of every problem of a batch run
// in grouped launches (one dot and one update launch per step for all
// problems, kernels_batched.cu) captured as one CUDA graph of `chunk` steps on
// the batch stream bs; the graph is replayed until every problem's device
// control block reports done. Per-problem setup and the final combine are
// ordinary launches on bs. Errors of one problem (breakdown, timeout) are
// stored in its item; errors of the batch as a whole throw.
// ---------------------------------------------------------------------------
struct BatchItem {
  Handle* h = nullptr;
  const rafeast_params* prm = nullptr;
  double* Qt = nullptr;
  FilterStats fs;
  int err = 0;
};

template <typename T>
static void filter_ms_batched(std::vector<BatchItem*>& items, Handle* owner, cudaStream_t bs,
                              int64_t sig) {
  const int cnt = (int)items.size();
  if (cnt == 0) return;
  const bool fp64 = sizeof(T) == 8;
  // every problem's inputs were produced on its own stream
  for (auto* it : items) {
    RF_CUDA(cudaEventRecord(it->h->ev_out, it->h->stream));
    RF_CUDA(cudaStreamWaitEvent(bs, it->h->ev_out, 0));
  }
  // one device buffer: every problem's control block (one array the host
  // polls), the two kernels' arguments, item maps and shapes, queue control
  size_t off = 0;
  auto carve = [&](size_t bytes) {
    off = (off + 255) & ~(size_t)255;
    size_t o = off;
    off += bytes;
    return o;
  };
  const size_t o_ctl = carve(sizeof(CocgCtl) * cnt);
  const size_t o_ad = carve(sizeof(CocgArgs<T>) * cnt);
  const size_t o_au = carve(sizeof(CocgArgs<T>) * cnt);
  const size_t o_md = carve(sizeof(int) * (2 * cnt + 1));
  const size_t o_mu = carve(sizeof(int) * (2 * cnt + 1));
  const size_t o_gc = carve(sizeof(GroupCtl));
  const size_t o_ggd = carve(sizeof(int) * 4 * cnt);
  const size_t o_ggu = carve(sizeof(int) * 4 * cnt);
  char* bb = (char*)scratch(owner, S_BATCH, off + 256);
  CocgCtl* ctl_d = (CocgCtl*)(bb + o_ctl);
  std::vector<MsProblem<T>> P(cnt);
  for (int t = 0; t < cnt; ++t) {
    Handle* h = items[t]->h;
    P[t] = ms_setup<T>(h, *items[t]->prm, h->Q, h->AQ, h->theta_d, h->theta, h->m0, h->ldq,
                       ctl_d + t, owner->opt_profile != 0,
                       owner->opt_update != 1 || items[t]->prm->nc > 8, bs);
  }
  GroupDev<T> gd;
  gd.args_d = (const CocgArgs<T>*)(bb + o_ad);
  gd.args_u = (const CocgArgs<T>*)(bb + o_au);
  gd.map_d = (int*)(bb + o_md);
  gd.map_u = (int*)(bb + o_mu);
  gd.gc = (GroupCtl*)(bb + o_gc);
  gd.ctl = ctl_d;
  gd.gg_d = (const int4*)(bb + o_ggd);
  gd.gg_u = (const int4*)(bb + o_ggu);
  // (lanes, chunks) of a kernel: 0 = each problem's own default (at most two
  // chunks per lane, the two-CTA-per-SM instances), else one shape for all
  bool all_vf = true;
  for (int t = 0; t < cnt; ++t) all_vf = all_vf && P[t].a.lcolidx != nullptr;
  auto shaped = [&](int G, int cpl) {
    std::vector<CocgArgs<T>> v(cnt);
    for (int t = 0; t < cnt; ++t) {
      v[t] = P[t].a;
      if (!all_vf) {  // values-free gathers only when every problem has them
        v[t].lrowptr = nullptr;
        v[t].lcolidx = nullptr;
      }
      if (G == 0) {
        int cb = 1;
        choose_shape(P[t].pairs, 2, fp64, 0, v[t].lanes, v[t].cpl, cb,
                     std::min(2, ms_max_cpl(fp64)));
      } else {
        v[t].lanes = G;
        v[t].cpl = cpl;
      }
    }
    return v;
  };
  GroupPlan plan;
  // upload the arguments, maps and shapes of one shape choice (the device
  // has finished every earlier replay: each was synchronised)
  auto prepare = [&](const std::vector<CocgArgs<T>>& ad, const std::vector<CocgArgs<T>>& au) {
    plan = GroupPlan();
    plan_ms_grouped<T>(ad, au, owner->num_sms, plan);
    GroupCtl gch;
    memset(&gch, 0, sizeof(gch));
    gch.grid_d = plan.ctas_dots;
    gch.grid_u = plan.ctas_upd;
    RF_CUDA(cudaMemcpyAsync(bb + o_ad, ad.data(), sizeof(CocgArgs<T>) * cnt,
                            cudaMemcpyHostToDevice, bs));
    RF_CUDA(cudaMemcpyAsync(bb + o_au, au.data(), sizeof(CocgArgs<T>) * cnt,
                            cudaMemcpyHostToDevice, bs));
    RF_CUDA(cudaMemcpyAsync(bb + o_md, plan.map_dots.data(), sizeof(int) * plan.map_dots.size(),
                            cudaMemcpyHostToDevice, bs));
    RF_CUDA(cudaMemcpyAsync(bb + o_mu, plan.map_upd.data(), sizeof(int) * plan.map_upd.size(),
                            cudaMemcpyHostToDevice, bs));
    RF_CUDA(cudaMemcpyAsync(bb + o_gc, &gch, sizeof(gch), cudaMemcpyHostToDevice, bs));
    RF_CUDA(cudaMemcpyAsync(bb + o_ggd, plan.gg_d.data(), sizeof(int) * plan.gg_d.size(),
                            cudaMemcpyHostToDevice, bs));
    RF_CUDA(cudaMemcpyAsync(bb + o_ggu, plan.gg_u.data(), sizeof(int) * plan.gg_u.size(),
                            cudaMemcpyHostToDevice, bs));
  };
  std::vector<CocgCtl> ctl(cnt);
  bool all_done = false;
  std::vector<float> tk;  // dot ms, update ms per executed step (timed runs)
  // capture `steps` steps of the current plan and replay the graph `reps`
  // times (or until every problem is done); events bracket each kernel
  auto run = [&](int steps, bool timed, int reps) {
    std::vector<cudaEvent_t> evs;
    if (timed) {
      evs.resize(2 * steps + 1);
      for (auto& e : evs) RF_CUDA(cudaEventCreate(&e));
    }
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    RF_CUDA(cudaStreamBeginCapture(bs, cudaStreamCaptureModeThreadLocal));
    g_capturing = true;
    try {
      for (int it = 0; it < steps; ++it) {
        if (timed) RF_CUDA(cudaEventRecordWithFlags(evs[2 * it], bs, cudaEventRecordExternal));
        launch_ms_grouped<T>(plan, gd, 0, it & 1, bs);
        if (timed)
          RF_CUDA(cudaEventRecordWithFlags(evs[2 * it + 1], bs, cudaEventRecordExternal));
        launch_ms_grouped<T>(plan, gd, 1, it & 1, bs);
      }
      if (timed) RF_CUDA(cudaEventRecordWithFlags(evs[2 * steps], bs, cudaEventRecordExternal));
    } catch (...) {
      g_capturing = false;
      cudaStreamEndCapture(bs, &graph);
      if (graph) cudaGraphDestroy(graph);
      for (auto& e : evs) cudaEventDestroy(e);
      throw;
    }
    g_capturing = false;
    RF_CUDA(cudaStreamEndCapture(bs, &graph));
    RF_CUDA(cudaGraphInstantiate(&exec, graph, 0));
    RF_CUDA(cudaGraphDestroy(graph));
    for (int r = 0; r < reps && !all_done; ++r) {
      RF_CUDA(cudaGraphLaunch(exec, bs));
      RF_CUDA(cudaMemcpyAsync(ctl.data(), ctl_d, sizeof(CocgCtl) * cnt, cudaMemcpyDeviceToHost,
                              bs));
      RF_CUDA(cudaStreamSynchronize(bs));
      if (timed)
        for (int k = 0; k < 2 * steps; ++k) {
          float ms = 0.f;
          RF_CUDA(cudaEventElapsedTime(&ms, evs[k], evs[k + 1]));
          tk.push_back(ms);
        }
      owner->launches += 2 * steps;
      owner->spmm_launches += 2 * steps;
      all_done = true;
      for (int t = 0; t < cnt; ++t) all_done = all_done && ctl[t].done;
    }
    RF_CUDA(cudaGraphExecDestroy(exec));
    for (auto& e : evs) RF_CUDA(cudaEventDestroy(e));
  };
  // K10 autotuner for the batch: each candidate shape, applied to every
  // problem, runs two real COCG steps of the batch; the fastest per kernel
  // is kept on the first handle under the batch's signature `sig` (taken
  // over all problems of the rafeast_solve_batched call, so the shapes tuned
  // in the first outer iteration serve the later ones)
  const bool prof = owner->opt_profile != 0;
  Handle::Shape shp{0, 0, 0, 0};
  bool have = false;
  for (auto& kv : owner->tuned)
    if (kv.first == sig) {
      shp = kv.second;
      have = true;
    }
  if (!have && owner->opt_autotune) {
    const int cand[][2] = {{0, 0}, {32, 2}, {16, 2}, {16, 1}, {8, 2}, {8, 1},
                           {16, 3}, {8, 3},  {16, 4}, {8, 4}};
    const int capc = ms_max_cpl(fp64);
    float best_d = 1e30f, best_u = 1e30f;
    for (auto& c : cand) {
      if (all_done) break;
      if (c[1] > capc) continue;
      auto v = shaped(c[0], c[1]);
      prepare(v, v);
      const size_t k0 = tk.size();
      run(2, true, 1);
      if (tk.size() < k0 + 4) break;
      const float td = std::min(tk[k0], tk[k0 + 2]), tu = std::min(tk[k0 + 1], tk[k0 + 3]);
      if (td < best_d) {
        best_d = td;
        shp.dl = c[0];
        shp.dc = c[1];
      }
      if (tu < best_u) {
        best_u = tu;
        shp.ul = c[0];
        shp.uc = c[1];
      }
    }
    owner->tuned.push_back(std::make_pair(sig, shp));
  }
  if (!all_done) {
    prepare(shaped(shp.dl, shp.dc), shaped(shp.ul, shp.uc));
    int chunk = std::max(2, owner->opt_chunk);
    chunk += chunk & 1;
    int max_inner = 1;
    for (auto* it : items) max_inner = std::max(max_inner, it->prm->max_inner);
    run(chunk, prof, (max_inner + 2) / chunk + 2);
  }
  owner->prof[6] = shp.dl * 100 + shp.dc;
  owner->prof[7] = shp.ul * 100 + shp.uc;
  if (prof && all_done) {
    // per-step time of the grouped kernels against the algorithmic bytes of
    // every problem still active in that step
    int steps = 0;
    std::vector<std::vector<int>> hist(cnt);
    for (int t = 0; t < cnt; ++t) {
      const int iters = std::min(ctl[t].iter, items[t]->prm->max_inner + 1);
      hist[t].assign(iters, 0);
      if (iters > 0 && P[t].a.hist)
        RF_CUDA(cudaMemcpy(hist[t].data(), P[t].a.hist, sizeof(int) * iters,
                           cudaMemcpyDeviceToHost));
      steps = std::max(steps, iters);
    }
    for (int k = 0; k < steps && 2 * k + 1 < (int)tk.size(); ++k) {
      double bd = 0.0, bu = 0.0;
      int probs = 0, pairs_act = 0;
      for (int t = 0; t < cnt; ++t) {
        const int iters = (int)hist[t].size();
        if (k >= iters) continue;
        const int act_d = k == 0 ? P[t].pairs : hist[t][k - 1];
        const int act_u = hist[t][k];
        const bool st = P[t].a.wbuf != nullptr;
        bd += ms_dots_bytes(items[t]->h, act_d, fp64, st, all_vf);
        if (act_u > 0) bu += ms_update_bytes(items[t]->h, act_u, P[t].ns, fp64, st);
        if (act_d > 0) ++probs;
        pairs_act += act_d;
      }
      // batched trace, appended over the whole solve: active pairs, active
      // problems, dot and update milliseconds of the step
      owner->last_hist.push_back(pairs_act);
      owner->last_rhist.push_back((double)probs);
      owner->last_tk.push_back(tk[2 * k]);
      owner->last_tk.push_back(tk[2 * k + 1]);
      owner->prof[0] += 1;
      owner->prof[1] += tk[2 * k];
      owner->prof[2] += bd;
      if (bu > 0.0) {
        owner->prof[3] += 1;
        owner->prof[4] += tk[2 * k + 1];
        owner->prof[5] += bu;
      }
    }
  }
  for (int t = 0; t < cnt; ++t) {
    Handle* h = items[t]->h;
    try {
      ms_finish<T>(h, P[t], h->Q, h->ldq, items[t]->Qt, ctl[t], items[t]->fs, bs);
    } catch (const Err& e) {
      items[t]->err = e.code;
    }
  }
  // every problem's next phase runs on its own stream after the batch
  RF_CUDA(cudaEventRecord(owner->ev_in, bs));
  for (auto* it : items) RF_CUDA(cudaStreamWaitEvent(it->h->stream, owner->ev_in, 0));
}

static void validate_params(const rafeast_params* p) {
  RF_CHECK(p, RAFEAST_ERR_INVALID_ARG);
  RF_CHECK(std::isfinite(p->lmin) && std::isfinite(p->lmax) && p->lmin < p->lmax,
           RAFEAST_ERR_INVALID_ARG);
  RF_CHECK(p->m0 >= 1 && p->m0 <= 128, RAFEAST_ERR_INVALID_ARG);
  RF_CHECK(p->nc >= 1 && p->nc <= 16, RAFEAST_ERR_INVALID_ARG);
  RF_CHECK(p->ellipse_ratio > 0.0 && p->ellipse_ratio <= 1.0, RAFEAST_ERR_INVALID_ARG);
  RF_CHECK(p->solve_tol >= 0.0 && p->outer_tol >= 0.0, RAFEAST_ERR_INVALID_ARG);
  RF_CHECK(p->max_outer >= 1 && p->max_inner >= 1, RAFEAST_ERR_INVALID_ARG);
  RF_CHECK(p->precision == RAFEAST_FP64 || p->precision == RAFEAST_MIXED, RAFEAST_ERR_INVALID_ARG);
  RF_CHECK(p->solve_form == RAFEAST_FORM_DIRECT || p->solve_form == RAFEAST_FORM_CORRECTION,
           RAFEAST_ERR_INVALID_ARG);
  RF_CHECK(p->start == RAFEAST_START_RANDOM || p->start == RAFEAST_START_SUBSPACE,
           RAFEAST_ERR_INVALID_ARG);
}

static void run_filter(Handle* h, const rafeast_params& prm, const double* Qd, const double* AQd,
                       const double* theta_d, const std::vector<double>& theta, int m0, int ldq,
                       double* Qt, FilterStats& fs) {
  // one COCG per shift is compiled for up to 8 shifts: more go multi-shift
  const bool ms = (h->opt_solver == 1 && h->opt_kernel != 2) || prm.nc > 8;
  if (prm.precision == RAFEAST_FP64) {
    if (ms) filter_ms_dev<double>(h, prm, Qd, AQd, theta_d, theta, m0, ldq, Qt, fs);
    else filter_dev<double>(h, prm, Qd, AQd, theta_d, theta, m0, ldq, Qt, fs);
  } else {
    if (ms) filter_ms_dev<float>(h, prm, Qd, AQd, theta_d, theta, m0, ldq, Qt, fs);
    else filter_dev<float>(h, prm, Qd, AQd, theta_d, theta, m0, ldq, Qt, fs);
  }
}

// column-major caller block (host or device) -> internal row-major device
static void import_block(Handle* h, const double* src, int m, int on_device, double* dst, int ld) {
  const double* dsrc = src;
  if (!on_device) {
    double* tmp = (double*)scratch(h, S_IO1, sizeof(double) * h->n * m);
    RF_CUDA(cudaMemcpyAsync(tmp, src, sizeof(double) * h->n * m, cudaMemcpyHostToDevice, h->stream));
    dsrc = tmp;
  }
  launch_to_internal(h->n, m, dsrc, dst, ld, h->perm, h->stream);
  h->launches += 1;
}

static void export_block(Handle* h, const double* src, int ld, int m, const int32_t* cols_d,
                         int on_device, double* dst) {
  if (m <= 0) return;
  double* ddst = dst;
  if (!on_device) ddst = (double*)scratch(h, S_IO2, sizeof(double) * h->n * m);
  launch_from_internal(h->n, m, src, ld, ddst, h->perm, cols_d, h->stream);
  h->launches += 1;
  if (!on_device) {
    RF_CUDA(cudaMemcpyAsync(dst, ddst, sizeof(double) * h->n * m, cudaMemcpyDeviceToHost,
                            h->stream));
    RF_CUDA(cudaStreamSynchronize(h->stream));
  }
}

static void ensure_subspace_bufs(Handle* h, int m0) {
  const int ldq = even(m0);
  if (h->m0 != m0 || !h->Q) {
    if (h->Q) cudaFree(h->Q);
    if (h->AQ) cudaFree(h->AQ);
    if (h->theta_d) cudaFree(h->theta_d);
    h->Q = h->AQ = h->theta_d = nullptr;
    h->m0 = 0;
    RF_CUDA(cudaMalloc(&h->Q, sizeof(double) * h->n * ldq));
    RF_CUDA(cudaMalloc(&h->AQ, sizeof(double) * h->n * ldq));
    RF_CUDA(cudaMalloc(&h->theta_d, sizeof(double) * (m0 + 1)));
    RF_CUDA(cudaMemsetAsync(h->Q, 0, sizeof(double) * h->n * ldq, h->stream));
    RF_CUDA(cudaMemsetAsync(h->AQ, 0, sizeof(double) * h->n * ldq, h->stream));
    h->ldq = ldq;
  }
}

// orthonormalise + Rayleigh-Ritz a block already in h->Q (m0 columns)
static void subspace_from_Q(Handle* h, int m0) {
  const int ldq = h->ldq;
  double* tmp = (double*)scratch(h, S_TMP1, sizeof(double) * h->n * ldq);
  double* X = h->Q;
  double* Y = tmp;
  cholqr(h, X, Y, m0, ldq, nullptr);
  double* tmp2 = (double*)scratch(h, S_TMP2, sizeof(double) * h->n * ldq);
  // X holds the orthonormal block (either h->Q or tmp)
  double* Qout = (X == h->Q) ? tmp : h->Q;
  rayleigh_ritz_dev(h, X, m0, ldq, Qout, h->AQ, h->theta_d, tmp2);
  if (Qout != h->Q)
    RF_CUDA(cudaMemcpyAsync(h->Q, Qout, sizeof(double) * h->n * ldq, cudaMemcpyDeviceToDevice,
                            h->stream));
  h->theta.resize(m0);
  RF_CUDA(cudaMemcpyAsync(h->theta.data(), h->theta_d, sizeof(double) * m0,
                          cudaMemcpyDeviceToHost, h->stream));
  RF_CUDA(cudaStreamSynchronize(h->stream));
  h->m0 = m0;
}

// ---------------------------------------------------------------------------
// the outer FEAST loop in phases (Algorithm 1 / Algorithm 2 Phase 2):
// start, per-iteration tail after the filter (CholQR, Rayleigh-Ritz,
// residuals, convergence), outputs. rafeast_solve runs them in sequence;
// rafeast_solve_batched interleaves many problems with one batched filter.
// ---------------------------------------------------------------------------
struct SolveRun {
  Handle* h = nullptr;
  rafeast_params prm;
  int m0 = 0, ldq = 0;
  double *Qt = nullptr, *T1 = nullptr, *T2 = nullptr;
  std::vector<double> res;
  int status = RAFEAST_NO_CONVERGENCE;
  int it = 0, cocg_total = 0, shifted_total = 0;
  FilterStats fs;
  float t_filter = 0, t_orth = 0, t_rr = 0;
  cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  SolveRun() { memset(&prm, 0, sizeof(prm)); }
  SolveRun(const SolveRun&) = delete;
  SolveRun& operator=(const SolveRun&) = delete;
  ~SolveRun() {
    for (auto& e : ev)
      if (e) cudaEventDestroy(e);
  }
};

// starting subspace: random Gaussian block orthonormalised (plain FEAST), or
// the handle's current subspace (after rafeast_warmstart / set_subspace)
static void solve_begin(SolveRun& r, Handle* h, const rafeast_params& prm) {
  r.h = h;
  r.prm = prm;
  const int m0 = prm.m0;
  r.m0 = m0;
  for (auto& e : r.ev) RF_CUDA(cudaEventCreate(&e));
  RF_CUDA(cudaEventRecord(r.ev[0], h->stream));
  if (prm.start == RAFEAST_START_RANDOM) {
    ensure_subspace_bufs(h, m0);
    double* om = (double*)scratch(h, S_OMEGA, sizeof(double) * h->n * m0);
    launch_omega(prm.seed, h->n, m0, om, h->stream);
    launch_to_internal(h->n, m0, om, h->Q, h->ldq, h->perm, h->stream);
    h->launches += 2;
    double* X = h->Q;
    double* Y = (double*)scratch(h, S_TMP1, sizeof(double) * h->n * h->ldq);
    cholqr(h, X, Y, m0, h->ldq, nullptr);
    if (X != h->Q)
      RF_CUDA(cudaMemcpyAsync(h->Q, X, sizeof(double) * h->n * h->ldq, cudaMemcpyDeviceToDevice,
                              h->stream));
    // A Q and Rayleigh quotients (the correction form's theta)
    launch_spmm_real<double>(h->n, h->rowptr, h->colidx, h->val64, m0, h->ldq, 1.0, h->shift, h->Q,
                             h->AQ, h->num_sms, h->stream);
    h->launches += 1;
    h->spmm_launches += 1;
    {
      DenseWs d = dense_ws(h, m0);
      col_dot(h->Q, h->AQ, h->n, m0, h->ldq, h->theta_d, d.part, h->num_sms, h->stream);
      h->launches += 2;
    }
    h->theta.resize(m0);
    RF_CUDA(cudaMemcpyAsync(h->theta.data(), h->theta_d, sizeof(double) * m0,
                            cudaMemcpyDeviceToHost, h->stream));
    RF_CUDA(cudaStreamSynchronize(h->stream));
    h->m0 = m0;
  } else {
    if (!h->Q || h->m0 != m0) throw Err{RAFEAST_ERR_NOT_READY};
  }
  RF_CUDA(cudaEventRecord(r.ev[1], h->stream));
  r.ldq = h->ldq;
  r.Qt = (double*)scratch(h, S_QT, sizeof(double) * h->n * r.ldq);
  r.T1 = (double*)scratch(h, S_TMP1, sizeof(double) * h->n * r.ldq);
  r.T2 = (double*)scratch(h, S_TMP2, sizeof(double) * h->n * r.ldq);
  RF_CUDA(cudaMemsetAsync(r.Qt, 0, sizeof(double) * h->n * r.ldq, h->stream));
  RF_CUDA(cudaMemsetAsync(r.T1, 0, sizeof(double) * h->n * r.ldq, h->stream));
  r.res.assign(m0, 0.0);
}

// after the filter wrote Qt (events ev[2], ev[3] bracket it): CholQR, RR,
// residuals; true when every Ritz pair inside the interval has converged
static bool solve_outer_tail(SolveRun& r) {
  Handle* h = r.h;
  const int m0 = r.m0, ldq = r.ldq;
  double* X = r.Qt;
  double* Y = r.T1;
  r.shifted_total += cholqr_rr(h, X, Y, r.T2, m0, ldq, h->Q, h->AQ, h->theta_d, r.ev[4],
                               r.prm.precision == RAFEAST_MIXED);
  residuals_host(h, h->Q, h->AQ, h->theta_d, m0, ldq, r.res);
  RF_CUDA(cudaEventRecord(r.ev[5], h->stream));
  h->theta.resize(m0);
  RF_CUDA(cudaMemcpyAsync(h->theta.data(), h->theta_d, sizeof(double) * m0,
                          cudaMemcpyDeviceToHost, h->stream));
  RF_CUDA(cudaStreamSynchronize(h->stream));
  float a = 0, b = 0, c = 0;
  RF_CUDA(cudaEventElapsedTime(&a, r.ev[2], r.ev[3]));
  RF_CUDA(cudaEventElapsedTime(&b, r.ev[3], r.ev[4]));
  RF_CUDA(cudaEventElapsedTime(&c, r.ev[4], r.ev[5]));
  r.t_filter += a;
  r.t_orth += b;
  r.t_rr += c;
  double mx = -1.0;
  int nin = 0;
  for (int i = 0; i < m0; ++i)
    if (h->theta[i] >= r.prm.lmin && h->theta[i] <= r.prm.lmax) {
      ++nin;
      mx = std::max(mx, r.res[i]);
    }
  if (nin > 0 && mx <= r.prm.outer_tol) {
    r.status = RAFEAST_OK;
    return true;
  }
  return false;
}

// outputs: in-interval pairs first (ascending), then the rest (ascending)
static int solve_finish(SolveRun& r, int* m_found, double* evals, double* evecs, double* resid,
                        int outputs_on_device, rafeast_info* info) {
  Handle* h = r.h;
  const int m0 = r.m0;
  int status = r.status;
  std::vector<int> order;
  for (int i = 0; i < m0; ++i)
    if (h->theta[i] >= r.prm.lmin && h->theta[i] <= r.prm.lmax) order.push_back(i);
  const int mf = (int)order.size();
  for (int i = 0; i < m0; ++i)
    if (!(h->theta[i] >= r.prm.lmin && h->theta[i] <= r.prm.lmax)) order.push_back(i);
  if (mf == 0) status = RAFEAST_NO_EIGENVALUE;
  else if (mf >= m0) status = RAFEAST_M0_TOO_SMALL;
  *m_found = mf;
  std::vector<double> ev_out(m0), res_out(m0);
  double maxres = 0.0;
  for (int t = 0; t < m0; ++t) {
    ev_out[t] = h->theta[order[t]];
    res_out[t] = r.res[order[t]];
    if (t < mf) maxres = std::max(maxres, res_out[t]);
  }
  if (outputs_on_device) {
    RF_CUDA(cudaMemcpyAsync(evals, ev_out.data(), sizeof(double) * m0, cudaMemcpyHostToDevice,
                            h->stream));
    if (resid)
      RF_CUDA(cudaMemcpyAsync(resid, res_out.data(), sizeof(double) * m0, cudaMemcpyHostToDevice,
                              h->stream));
  } else {
    std::copy(ev_out.begin(), ev_out.end(), evals);
    if (resid) std::copy(res_out.begin(), res_out.end(), resid);
  }
  if (evecs) {
    int32_t* cols_d = (int32_t*)scratch(h, S_SMALL, sizeof(int32_t) * m0 + 64);
    std::vector<int32_t> cols(order.begin(), order.end());
    RF_CUDA(cudaMemcpyAsync(cols_d, cols.data(), sizeof(int32_t) * m0, cudaMemcpyHostToDevice,
                            h->stream));
    export_block(h, h->Q, r.ldq, m0, cols_d, outputs_on_device, evecs);
  }
  RF_CUDA(cudaEventRecord(r.ev[5], h->stream));
  RF_CUDA(cudaStreamSynchronize(h->stream));
  float tot = 0, tws = 0;
  RF_CUDA(cudaEventElapsedTime(&tot, r.ev[0], r.ev[5]));
  RF_CUDA(cudaEventElapsedTime(&tws, r.ev[0], r.ev[1]));
  if (info) {
    memset(info, 0, sizeof(*info));
    info->status = status;
    info->outer_iters = r.it;
    info->cocg_iters_total = r.cocg_total;
    info->cocg_min_last = r.fs.iters_min;
    info->cocg_max_last = r.fs.iters_max;
    info->cholqr_shifted = r.shifted_total;
    info->kernel_launches = h->launches;
    info->spmm_launches = h->spmm_launches;
    info->max_resid = maxres;
    info->t_warmstart_ms = tws;
    info->t_filter_ms = r.t_filter;
    info->t_orth_ms = r.t_orth;
    info->t_rr_ms = r.t_rr;
    info->t_total_ms = tot;
  }
  return status;
}

}  // namespace rafeast

using namespace rafeast;

#define API_BEGIN try {
#define API_END                              \
  }                                          \
  catch (const Err& e) {                     \
    return e.code;                           \
  }                                          \
  catch (...) {                              \
    return RAFEAST_ERR_CUDA;                 \
  }

extern "C" {

const char* rafeast_status_string(int s) {
  switch (s) {
    case RAFEAST_OK: return "ok";
    case RAFEAST_NO_EIGENVALUE: return "no eigenvalue inside the interval";
    case RAFEAST_NO_CONVERGENCE: return "no convergence within max_outer iterations";
    case RAFEAST_M0_TOO_SMALL: return "m0 too small: every Ritz value lies inside the interval";
    case RAFEAST_ERR_INVALID_ARG: return "invalid argument";
    case RAFEAST_ERR_NOT_SYMMETRIC: return "matrix is not symmetric";
    case RAFEAST_ERR_CUDA: return "CUDA error";
    case RAFEAST_ERR_COCG_BREAKDOWN: return "COCG breakdown";
    case RAFEAST_ERR_TIMEOUT: return "device work did not finish within its bound";
    case RAFEAST_ERR_OUT_OF_MEMORY: return "out of device memory";
    case RAFEAST_ERR_NOT_READY: return "no subspace in the handle";
    case RAFEAST_ERR_CHOLESKY: return "Cholesky-QR failed (rank-deficient block)";
    case RAFEAST_ERR_NO_DEVICE: return "no CUDA device";
    case RAFEAST_ERR_EXCHANGE: return "the sharded solve's sum callback failed";
    default: return "unknown status";
  }
}

const char* rafeast_last_error(void) { return g_err; }

int rafeast_quadrature(double lmin, double lmax, int nc, double e, double* z, double* w) {
  if (!z || !w || !(lmin < lmax) || nc < 1 || nc > 64 || !(e > 0.0 && e <= 1.0))
    return RAFEAST_ERR_INVALID_ARG;
  std::vector<double> zr, zi, wr, wi;
  quadrature_nodes(lmin, lmax, nc, e, zr, zi, wr, wi);
  for (int j = 0; j < nc; ++j) {
    z[2 * j] = zr[j];
    z[2 * j + 1] = zi[j];
    w[2 * j] = wr[j];
    w[2 * j + 1] = wi[j];
  }
  return RAFEAST_OK;
}

int rafeast_philox(uint64_t seed, uint64_t first_block, int64_t nblocks, uint64_t* words,
                   void* stream) {
  API_BEGIN
  if (nblocks < 0 || (nblocks > 0 && !words)) return RAFEAST_ERR_INVALID_ARG;
  launch_philox(seed, first_block, nblocks, words, (cudaStream_t)stream);
  RF_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  return RAFEAST_OK;
  API_END
}

int rafeast_create(rafeast_t* out, int64_t n, int64_t nnz, const int32_t* row_ptr,
                   const int32_t* col_idx, const double* values, double diag_shift,
                   int inputs_on_device, void* stream, uint32_t flags) {
  if (!out) return RAFEAST_ERR_INVALID_ARG;
  *out = nullptr;
  if (n <= 0 || nnz < 0 || n > INT32_MAX - 1 || nnz > INT32_MAX || !row_ptr ||
      (nnz > 0 && (!col_idx || !values)) || !std::isfinite(diag_shift))
    return RAFEAST_ERR_INVALID_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return RAFEAST_ERR_NO_DEVICE;
  Handle* h = new Handle();
  try {
    RF_CUDA(cudaGetDevice(&h->device));
    RF_CUDA(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device));
    h->n = n;
    h->nnz = nnz;
    h->shift = diag_shift;
    h->user_stream = (cudaStream_t)stream;
    RF_CUDA(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
    RF_CUDA(cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming));
    RF_CUDA(cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming));
    CallScope scope(h);
    // host copies for validation and reordering
    std::vector<int32_t> rp(n + 1), ci(nnz);
    std::vector<double> va(nnz);
    auto kind = inputs_on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
    RF_CUDA(cudaMemcpy(rp.data(), row_ptr, sizeof(int32_t) * (n + 1), kind));
    if (nnz) {
      RF_CUDA(cudaMemcpy(ci.data(), col_idx, sizeof(int32_t) * nnz, kind));
      RF_CUDA(cudaMemcpy(va.data(), values, sizeof(double) * nnz, kind));
    }
    RF_CHECK(rp[0] == 0 && rp[n] == nnz, RAFEAST_ERR_INVALID_ARG);
    for (int64_t i = 0; i < n; ++i) RF_CHECK(rp[i + 1] >= rp[i], RAFEAST_ERR_INVALID_ARG);
    for (int64_t k = 0; k < nnz; ++k)
      RF_CHECK(ci[k] >= 0 && ci[k] < n && std::isfinite(va[k]), RAFEAST_ERR_INVALID_ARG);
    if (flags & RAFEAST_CREATE_CHECK_SYMMETRY) {
      // every (i, j, v) needs a matching (j, i, v)
      std::vector<std::pair<int32_t, double>> rowv;
      for (int64_t i = 0; i < n; ++i)
        for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
          const int32_t j = ci[k];
          bool found = false;
          for (int32_t t = rp[j]; t < rp[j + 1]; ++t)
            if (ci[t] == i && va[t] == va[k]) {
              found = true;
              break;
            }
          if (!found) throw Err{RAFEAST_ERR_NOT_SYMMETRIC};
        }
    }
    // norms: ||A||_1 and Gershgorin interval of A = L + shift I
    double norm1 = 0.0, glo = INFINITY, ghi = -INFINITY;
    for (int64_t i = 0; i < n; ++i) {
      double d = diag_shift, off = 0.0;
      for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
        if (ci[k] == i) d += va[k];
        else off += std::fabs(va[k]);
      }
      norm1 = std::max(norm1, off + std::fabs(d));
      glo = std::min(glo, d - off);
      ghi = std::max(ghi, d + off);
    }
    h->norm1 = norm1 > 0.0 ? norm1 : 1.0;
    h->glo = glo;
    h->ghi = ghi;
    // row order. Default: recursive breadth-first bisection, down to sets of
    // one tile's rows (each kept in its level-structure order: finer cuts
    // gave tiles with larger unions), when its row tiles gather from at
    // least 15% fewer rows than the caller's order (tiling.cpp);
    // RAFEAST_CREATE_RCM: reverse Cuthill-McKee when it
    // narrows the band by 30%; FORCE_REORDER applies the chosen kind always
    std::vector<int32_t> perm;
    bool reorder = false;
    if (!(flags & RAFEAST_CREATE_NO_REORDER) && n > 1) {
      if (flags & RAFEAST_CREATE_RCM) {
        rcm_order(n, rp.data(), ci.data(), perm);
        const int64_t bw0 = bandwidth(n, rp.data(), ci.data(), nullptr);
        const int64_t bw1 = bandwidth(n, rp.data(), ci.data(), perm.data());
        reorder = (flags & RAFEAST_CREATE_FORCE_REORDER) || (double)bw1 < 0.7 * (double)bw0;
        h->order_kind = reorder ? 2 : 0;
      } else {
        bisect_order(n, rp.data(), ci.data(), TILE_TMAX, perm);
        bool better = (flags & RAFEAST_CREATE_FORCE_REORDER) != 0;
        if (!better) {
          // the permuted pattern (indices only) for the comparison
          std::vector<int32_t> ip(n), prp(n + 1), pci(nnz);
          for (int64_t r = 0; r < n; ++r) ip[perm[r]] = (int32_t)r;
          prp[0] = 0;
          for (int64_t r = 0; r < n; ++r) {
            const int32_t o = perm[r];
            int32_t* dst = pci.data() + prp[r];
            int c = 0;
            for (int32_t k = rp[o]; k < rp[o + 1]; ++k) dst[c++] = ip[ci[k]];
            prp[r + 1] = prp[r] + c;
          }
          // union rows per row on sampled row windows of both orders
          const double u0 = tile_union_ratio(n, rp.data(), ci.data(), TILE_UCAP, TILE_TMAX,
                                             TILE_NNZCAP, 8);
          const double u1 = tile_union_ratio(n, prp.data(), pci.data(), TILE_UCAP, TILE_TMAX,
                                             TILE_NNZCAP, 8);
          better = u1 > 0.0 && (u0 < 0.0 || u1 < 0.85 * u0);
        }
        reorder = better;
        h->order_kind = reorder ? 1 : 0;
      }
    }
    std::vector<int32_t> rp2 = rp, ci2 = ci;
    std::vector<double> va2 = va;
    if (reorder) {
      std::vector<int32_t> ip(n);
      for (int64_t r = 0; r < n; ++r) ip[perm[r]] = (int32_t)r;
      rp2[0] = 0;
      for (int64_t r = 0; r < n; ++r) rp2[r + 1] = rp2[r] + (rp[perm[r] + 1] - rp[perm[r]]);
      std::vector<std::pair<int32_t, double>> row;
      for (int64_t r = 0; r < n; ++r) {
        const int32_t o = perm[r];
        row.clear();
        for (int32_t k = rp[o]; k < rp[o + 1]; ++k) row.emplace_back(ip[ci[k]], va[k]);
        std::sort(row.begin(), row.end(),
                  [](const std::pair<int32_t, double>& a, const std::pair<int32_t, double>& b) {
                    return a.first < b.first;
                  });
        for (size_t t = 0; t < row.size(); ++t) {
          ci2[rp2[r] + t] = row[t].first;
          va2[rp2[r] + t] = row[t].second;
        }
      }
      RF_CUDA(cudaMalloc(&h->perm, sizeof(int32_t) * n));
      RF_CUDA(cudaMalloc(&h->iperm, sizeof(int32_t) * n));
      RF_CUDA(cudaMemcpy(h->perm, perm.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice));
      RF_CUDA(cudaMemcpy(h->iperm, ip.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice));
    }
    h->reordered = reorder;
    // a unit-weight graph Laplacian (every off-diagonal value -1, one diagonal
    // entry per row equal to the row's off-diagonal count) also gets its
    // off-diagonal pattern, for the values-free gathers
    bool unit = nnz > 0;
    for (int64_t r = 0; r < n && unit; ++r) {
      int deg = 0, ndiag = 0;
      double dv = 0.0;
      for (int32_t k = rp2[r]; k < rp2[r + 1]; ++k) {
        if (ci2[k] == r) {
          ++ndiag;
          dv = va2[k];
        } else if (va2[k] == -1.0) {
          ++deg;
        } else {
          unit = false;
        }
      }
      if (ndiag > 1 || dv != (double)deg) unit = false;
    }
    if (unit) {
      std::vector<int32_t> lrp(n + 1), lci;
      lci.reserve(nnz);
      lrp[0] = 0;
      for (int64_t r = 0; r < n; ++r) {
        for (int32_t k = rp2[r]; k < rp2[r + 1]; ++k)
          if (ci2[k] != r) lci.push_back(ci2[k]);
        lrp[r + 1] = (int32_t)lci.size();
      }
      h->nnz_off = (int64_t)lci.size();
      RF_CUDA(cudaMalloc(&h->lrowptr, sizeof(int32_t) * (n + 1)));
      RF_CUDA(cudaMalloc(&h->lcolidx, sizeof(int32_t) * std::max<int64_t>(h->nnz_off, 1)));
      RF_CUDA(cudaMemcpy(h->lrowptr, lrp.data(), sizeof(int32_t) * (n + 1),
                         cudaMemcpyHostToDevice));
      if (h->nnz_off)
        RF_CUDA(cudaMemcpy(h->lcolidx, lci.data(), sizeof(int32_t) * h->nnz_off,
                           cudaMemcpyHostToDevice));
    }
    // row tiles of the tiled dot kernel, on the internal order
    {
      TileHost t;
      if (nnz > 0 && build_tiles(n, rp2.data(), ci2.data(), TILE_UCAP, TILE_TMAX, TILE_NNZCAP, t)) {
        std::vector<uint16_t> lx, llx;
        std::vector<int32_t> us;
        tile_local_index(n, rp2.data(), ci2.data(), t, lx, us);
        h->ntiles = (int)t.trow.size() - 1;
        h->tile_max_union = t.max_union;
        h->tile_max_rows = t.max_rows;
        h->tile_ratio = (double)t.ucol.size() / (double)n;
        RF_CUDA(cudaMalloc(&h->trow, sizeof(int32_t) * t.trow.size()));
        RF_CUDA(cudaMalloc(&h->uoff, sizeof(int32_t) * t.uoff.size()));
        RF_CUDA(cudaMalloc(&h->ucol, sizeof(int32_t) * t.ucol.size()));
        RF_CUDA(cudaMalloc(&h->uself, sizeof(int32_t) * us.size()));
        RF_CUDA(cudaMalloc(&h->lidx, sizeof(uint16_t) * lx.size()));
        RF_CUDA(cudaMemcpy(h->trow, t.trow.data(), sizeof(int32_t) * t.trow.size(),
                           cudaMemcpyHostToDevice));
        RF_CUDA(cudaMemcpy(h->uoff, t.uoff.data(), sizeof(int32_t) * t.uoff.size(),
                           cudaMemcpyHostToDevice));
        RF_CUDA(cudaMemcpy(h->ucol, t.ucol.data(), sizeof(int32_t) * t.ucol.size(),
                           cudaMemcpyHostToDevice));
        RF_CUDA(cudaMemcpy(h->uself, us.data(), sizeof(int32_t) * us.size(),
                           cudaMemcpyHostToDevice));
        RF_CUDA(cudaMemcpy(h->lidx, lx.data(), sizeof(uint16_t) * lx.size(),
                           cudaMemcpyHostToDevice));
        if (unit && h->nnz_off > 0) {
          // the off-diagonal pattern gathers from the same unions
          std::vector<int32_t> lrp(n + 1), lci;
          lci.reserve(h->nnz_off);
          lrp[0] = 0;
          for (int64_t r = 0; r < n; ++r) {
            for (int32_t k = rp2[r]; k < rp2[r + 1]; ++k)
              if (ci2[k] != r) lci.push_back(ci2[k]);
            lrp[r + 1] = (int32_t)lci.size();
          }
          tile_local_index(n, lrp.data(), lci.data(), t, llx, us);
          RF_CUDA(cudaMalloc(&h->llidx, sizeof(uint16_t) * llx.size()));
          RF_CUDA(cudaMemcpy(h->llidx, llx.data(), sizeof(uint16_t) * llx.size(),
                             cudaMemcpyHostToDevice));
        }
      }
    }
    std::vector<float> v32(nnz);
    for (int64_t k = 0; k < nnz; ++k) v32[k] = (float)va2[k];
    RF_CUDA(cudaMalloc(&h->rowptr, sizeof(int32_t) * (n + 1)));
    RF_CUDA(cudaMalloc(&h->colidx, sizeof(int32_t) * std::max<int64_t>(nnz, 1)));
    RF_CUDA(cudaMalloc(&h->val64, sizeof(double) * std::max<int64_t>(nnz, 1)));
    RF_CUDA(cudaMalloc(&h->val32, sizeof(float) * std::max<int64_t>(nnz, 1)));
    RF_CUDA(cudaMemcpy(h->rowptr, rp2.data(), sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice));
    if (nnz) {
      RF_CUDA(cudaMemcpy(h->colidx, ci2.data(), sizeof(int32_t) * nnz, cudaMemcpyHostToDevice));
      RF_CUDA(cudaMemcpy(h->val64, va2.data(), sizeof(double) * nnz, cudaMemcpyHostToDevice));
      RF_CUDA(cudaMemcpy(h->val32, v32.data(), sizeof(float) * nnz, cudaMemcpyHostToDevice));
    }
    scope.finish();
    *out = reinterpret_cast<rafeast_t>(h);
    return RAFEAST_OK;
  } catch (const Err& e) {
    rafeast_destroy(reinterpret_cast<rafeast_t>(h));
    return e.code;
  } catch (...) {
    rafeast_destroy(reinterpret_cast<rafeast_t>(h));
    return RAFEAST_ERR_CUDA;
  }
}

void rafeast_destroy(rafeast_t hh) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return;
  cudaSetDevice(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (auto& b : h->bufs)
    if (b.p) cudaFree(b.p);
  void* ptrs[] = {h->rowptr, h->colidx, h->val64,   h->val32,   h->perm,  h->iperm,
                  h->Q,      h->AQ,     h->theta_d, h->lrowptr, h->lcolidx, h->trow,
                  h->uoff,   h->ucol,   h->uself,   h->lidx,    h->llidx};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (h->ev_in) cudaEventDestroy(h->ev_in);
  if (h->ev_out) cudaEventDestroy(h->ev_out);
  if (h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

int rafeast_set_option(rafeast_t hh, int key, int64_t value) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return RAFEAST_ERR_INVALID_ARG;
  switch (key) {
    case RAFEAST_OPT_WARMSTART_MAP:
      if (value < 0 || value > 2) return RAFEAST_ERR_INVALID_ARG;
      h->opt_ws_map = (int)value;
      return RAFEAST_OK;
    case RAFEAST_OPT_CHUNK:
      if (value < 2 || value > 512) return RAFEAST_ERR_INVALID_ARG;
      h->opt_chunk = (int)value;
      return RAFEAST_OK;
    case RAFEAST_OPT_AUTOTUNE:
      h->opt_autotune = value ? 1 : 0;
      return RAFEAST_OK;
    case RAFEAST_OPT_KERNEL:
      if (value < 0 || value > 2) return RAFEAST_ERR_INVALID_ARG;
      h->opt_kernel = (int)value;
      return RAFEAST_OK;
    case RAFEAST_OPT_MAXNZ:
      if (value < 1 || value > 32) return RAFEAST_ERR_INVALID_ARG;
      h->opt_maxnz = (int)value;
      return RAFEAST_OK;
    case RAFEAST_OPT_WAIT_LIMIT:
      if (value < 1) return RAFEAST_ERR_INVALID_ARG;
      h->opt_wait_cycles = (long long)value;
      return RAFEAST_OK;
    case RAFEAST_OPT_TEST_STALL:
      if (value < 0 || value > 4096 || (value % 16) != 0) return RAFEAST_ERR_INVALID_ARG;
      h->opt_stall_bytes = (int)value;
      return RAFEAST_OK;
    case RAFEAST_OPT_SOLVER:
      if (value < 0 || value > 1) return RAFEAST_ERR_INVALID_ARG;
      h->opt_solver = (int)value;
      return RAFEAST_OK;
    case RAFEAST_OPT_UPDATE:
      if (value < 0 || value > 2) return RAFEAST_ERR_INVALID_ARG;
      h->opt_update = (int)value;
      return RAFEAST_OK;
    case RAFEAST_OPT_VALUES_FREE:
      if (value < 0 || value > 1) return RAFEAST_ERR_INVALID_ARG;
      h->opt_values_free = (int)value;
      return RAFEAST_OK;
    case RAFEAST_OPT_TILED:
      if (value < 0 || value > 2) return RAFEAST_ERR_INVALID_ARG;
      h->opt_tiled = (int)value;
      return RAFEAST_OK;
    case RAFEAST_OPT_DEFER:
      if (value < 0 || value > 1) return RAFEAST_ERR_INVALID_ARG;
      h->opt_defer = (int)value;
      return RAFEAST_OK;
    case RAFEAST_OPT_DENSE:
      if (value < 0 || value > 1) return RAFEAST_ERR_INVALID_ARG;
      h->opt_dense = (int)value;
      return RAFEAST_OK;
    case RAFEAST_OPT_TILE_CB:
      if (value != 0 && value != 4 && value != 8) return RAFEAST_ERR_INVALID_ARG;
      h->opt_tile_cb = (int)value;
      return RAFEAST_OK;
    case RAFEAST_OPT_CPL:
      if (value < 0 || value > 16) return RAFEAST_ERR_INVALID_ARG;
      h->opt_cpl = (int)value;
      return RAFEAST_OK;
    case RAFEAST_OPT_PROFILE:
      h->opt_profile = value ? 1 : 0;
      return RAFEAST_OK;
    case RAFEAST_OPT_LANES:
      if (value != 0 && value != 4 && value != 8 && value != 16 && value != 32)
        return RAFEAST_ERR_INVALID_ARG;
      h->opt_lanes = (int)value;
      return RAFEAST_OK;
    default:
      return RAFEAST_ERR_INVALID_ARG;
  }
}

int rafeast_profile(rafeast_t hh, int reset, double* out) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return RAFEAST_ERR_INVALID_ARG;
  if (out)
    for (int t = 0; t < 8; ++t) out[t] = h->prof[t];
  if (reset)
    for (int t = 0; t < 6; ++t) h->prof[t] = 0.0;
  return RAFEAST_OK;
}

int rafeast_profile_history(rafeast_t hh, int max_len, int* active_cols, double* max_relres,
                            double* kernel_ms) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || max_len < 0) return RAFEAST_ERR_INVALID_ARG;
  const int len = (int)h->last_hist.size();
  for (int k = 0; k < std::min(len, max_len); ++k) {
    if (active_cols) active_cols[k] = h->last_hist[k];
    if (max_relres) max_relres[k] = h->last_rhist[k];
    if (kernel_ms) {
      kernel_ms[2 * k] = 2 * k < (int)h->last_tk.size() ? h->last_tk[2 * k] : 0.0;
      kernel_ms[2 * k + 1] = 2 * k + 1 < (int)h->last_tk.size() ? h->last_tk[2 * k + 1] : 0.0;
    }
  }
  return len;
}

int rafeast_matrix_info(rafeast_t hh, int64_t* n, int* reordered, double* norm1, double* glo,
                        double* ghi) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return RAFEAST_ERR_INVALID_ARG;
  if (n) *n = h->n;
  if (reordered) *reordered = h->reordered ? h->order_kind : 0;
  if (norm1) *norm1 = h->norm1;
  if (glo) *glo = h->glo;
  if (ghi) *ghi = h->ghi;
  return RAFEAST_OK;
}

int rafeast_draw_omega(rafeast_t hh, uint64_t seed, int k, double* omega) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || k < 1 || !omega) return RAFEAST_ERR_INVALID_ARG;
  API_BEGIN
  CallScope scope(h);
  launch_omega(seed, h->n, k, omega, h->stream);
  scope.finish();
  RF_CUDA(cudaStreamSynchronize(h->stream));
  return RAFEAST_OK;
  API_END
}

int rafeast_spmm(rafeast_t hh, int k, double alpha, double beta, const double* X, double* Y,
                 int precision) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || k < 1 || !X || !Y || (precision != RAFEAST_FP64 && precision != RAFEAST_MIXED))
    return RAFEAST_ERR_INVALID_ARG;
  API_BEGIN
  CallScope scope(h);
  const int ld = even(k);
  double* Xi = (double*)scratch(h, S_TMP1, sizeof(double) * h->n * ld);
  double* Yi = (double*)scratch(h, S_TMP2, sizeof(double) * h->n * ld);
  launch_to_internal(h->n, k, X, Xi, ld, h->perm, h->stream);
  // Y = alpha (L + shift I) X + beta X = alpha L X + (alpha shift + beta) X
  if (precision == RAFEAST_FP64) {
    launch_spmm_real<double>(h->n, h->rowptr, h->colidx, h->val64, k, ld, alpha,
                             alpha * h->shift + beta, Xi, Yi, h->num_sms, h->stream);
  } else {
    float* Xf = (float*)scratch(h, S_AQ2, sizeof(float) * h->n * ld * 2);
    float* Yf = Xf + h->n * ld;
    launch_cast_to_f32(Xi, Xf, h->n * (int64_t)ld, h->stream);
    launch_spmm_real<float>(h->n, h->rowptr, h->colidx, h->val32, k, ld, alpha,
                            alpha * h->shift + beta, Xf, Yf, h->num_sms, h->stream);
    launch_widen(Yf, Yi, h->n * (int64_t)ld, h->stream);
  }
  launch_from_internal(h->n, k, Yi, ld, Y, h->perm, nullptr, h->stream);
  scope.finish();
  RF_CUDA(cudaStreamSynchronize(h->stream));
  return RAFEAST_OK;
  API_END
}

int rafeast_shifted_spmm(rafeast_t hh, int nc, const double* z, int m, const double* P, double* W,
                         int precision) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || nc < 1 || nc > 8 || m < 1 || !z || !P || !W ||
      (precision != RAFEAST_FP64 && precision != RAFEAST_MIXED))
    return RAFEAST_ERR_INVALID_ARG;
  API_BEGIN
  CallScope scope(h);
  const int NC = nc_pad(nc);
  const int ldc = even(m * NC);
  const bool fp64 = precision == RAFEAST_FP64;
  // caller layout: entry (i, col, j) at 2*((col*nc + j)*n + i); internal:
  // row r, column col, shift j at 2*(r*ldc + col*NC + j). Move through a
  // real-valued internal block of 2*m*NC columns.
  const int kre = 2 * m * nc;
  const int ldr = even(kre);
  double* tin = (double*)scratch(h, S_TMP1, sizeof(double) * h->n * std::max(ldr, 2 * ldc));
  double* tout = (double*)scratch(h, S_TMP2, sizeof(double) * h->n * std::max(ldr, 2 * ldc));
  // caller array viewed as column-major n x kre with column index 2*(col*nc+j)+{0,1}?
  // No: caller stores (re, im) pairs contiguously per row entry, so view it as
  // column-major (2n) x (m*nc) and reorganise on the host side of the copy.
  std::vector<double> hp((size_t)2 * h->n * m * nc);
  RF_CUDA(cudaMemcpy(hp.data(), P, sizeof(double) * hp.size(), cudaMemcpyDeviceToHost));
  std::vector<int32_t> pm(h->n);
  if (h->perm) RF_CUDA(cudaMemcpy(pm.data(), h->perm, sizeof(int32_t) * h->n, cudaMemcpyDeviceToHost));
  else std::iota(pm.begin(), pm.end(), 0);
  std::vector<double> hin((size_t)h->n * ldc * 2, 0.0);
  for (int64_t r = 0; r < h->n; ++r)
    for (int col = 0; col < m; ++col)
      for (int j = 0; j < nc; ++j) {
        const size_t src = 2 * (((size_t)col * nc + j) * h->n + pm[r]);
        const size_t dst = 2 * ((size_t)r * ldc + (size_t)col * NC + j);
        hin[dst] = hp[src];
        hin[dst + 1] = hp[src + 1];
      }
  std::vector<double> hz(2 * NC);
  for (int j = 0; j < NC; ++j) {
    const int jj = j < nc ? j : 0;
    hz[2 * j] = z[2 * jj] - h->shift;
    hz[2 * j + 1] = z[2 * jj + 1];
  }
  int lanes, cpl, cb;
  choose_shape(m, NC, fp64, h->opt_lanes, lanes, cpl, cb, h->opt_cpl);
  std::vector<double> hout(hin.size());
  if (fp64) {
    double* zs = (double*)scratch(h, S_SMALL, sizeof(double) * 2 * NC + 64);
    RF_CUDA(cudaMemcpy(tin, hin.data(), sizeof(double) * hin.size(), cudaMemcpyHostToDevice));
    RF_CUDA(cudaMemcpy(zs, hz.data(), sizeof(double) * 2 * NC, cudaMemcpyHostToDevice));
    launch_shifted_spmm<double>(h->n, h->rowptr, h->colidx, h->val64, m, ldc, NC, zs, tin, tout,
                                lanes, cpl, h->num_sms, h->stream);
    RF_CUDA(cudaStreamSynchronize(h->stream));
    RF_CUDA(cudaMemcpy(hout.data(), tout, sizeof(double) * hout.size(), cudaMemcpyDeviceToHost));
  } else {
    std::vector<float> fin(hin.size()), fout(hin.size());
    for (size_t t = 0; t < hin.size(); ++t) fin[t] = (float)hin[t];
    std::vector<float> fz(2 * NC);
    for (int t = 0; t < 2 * NC; ++t) fz[t] = (float)hz[t];
    float* zs = (float*)scratch(h, S_SMALL, sizeof(float) * 2 * NC + 64);
    float* fi = (float*)tin;
    float* fo = (float*)tout;
    RF_CUDA(cudaMemcpy(fi, fin.data(), sizeof(float) * fin.size(), cudaMemcpyHostToDevice));
    RF_CUDA(cudaMemcpy(zs, fz.data(), sizeof(float) * 2 * NC, cudaMemcpyHostToDevice));
    launch_shifted_spmm<float>(h->n, h->rowptr, h->colidx, h->val32, m, ldc, NC, zs, fi, fo,
                               lanes, cpl, h->num_sms, h->stream);
    RF_CUDA(cudaStreamSynchronize(h->stream));
    RF_CUDA(cudaMemcpy(fout.data(), fo, sizeof(float) * fout.size(), cudaMemcpyDeviceToHost));
    for (size_t t = 0; t < hout.size(); ++t) hout[t] = fout[t];
  }
  std::vector<double> hw(hp.size());
  for (int64_t r = 0; r < h->n; ++r)
    for (int col = 0; col < m; ++col)
      for (int j = 0; j < nc; ++j) {
        const size_t dst = 2 * (((size_t)col * nc + j) * h->n + pm[r]);
        const size_t src = 2 * ((size_t)r * ldc + (size_t)col * NC + j);
        hw[dst] = hout[src];
        hw[dst + 1] = hout[src + 1];
      }
  RF_CUDA(cudaMemcpy(W, hw.data(), sizeof(double) * hw.size(), cudaMemcpyHostToDevice));
  scope.finish();
  return RAFEAST_OK;
  API_END
}

int rafeast_filter(rafeast_t hh, const rafeast_params* prm, const double* Q, const double* theta,
                   double* Qt, rafeast_info* info) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || !Q || !Qt) return RAFEAST_ERR_INVALID_ARG;
  API_BEGIN
  validate_params(prm);
  CallScope scope(h);
  const int m0 = prm->m0, ldq = even(m0);
  double* Qi = (double*)scratch(h, S_TMP1, sizeof(double) * h->n * ldq);
  double* AQi = (double*)scratch(h, S_TMP2, sizeof(double) * h->n * ldq);
  double* Qti = (double*)scratch(h, S_QT, sizeof(double) * h->n * ldq);
  RF_CUDA(cudaMemsetAsync(Qti, 0, sizeof(double) * h->n * ldq, h->stream));
  launch_to_internal(h->n, m0, Q, Qi, ldq, h->perm, h->stream);
  launch_spmm_real<double>(h->n, h->rowptr, h->colidx, h->val64, m0, ldq, 1.0, h->shift, Qi, AQi,
                           h->num_sms, h->stream);
  std::vector<double> th(m0);
  double* th_d = (double*)scratch(h, S_OMEGA, sizeof(double) * (m0 + 1));
  if (theta) {
    th.assign(theta, theta + m0);
  } else {
    // Rayleigh quotients q_i^T A q_i / q_i^T q_i
    std::vector<double> num(m0), den(m0);
    DenseWs d = dense_ws(h, m0);
    col_dot(Qi, AQi, h->n, m0, ldq, d.small, d.part, h->num_sms, h->stream);
    RF_CUDA(cudaMemcpyAsync(num.data(), d.small, sizeof(double) * m0, cudaMemcpyDeviceToHost,
                            h->stream));
    RF_CUDA(cudaStreamSynchronize(h->stream));
    col_dot(Qi, Qi, h->n, m0, ldq, d.small, d.part, h->num_sms, h->stream);
    RF_CUDA(cudaMemcpyAsync(den.data(), d.small, sizeof(double) * m0, cudaMemcpyDeviceToHost,
                            h->stream));
    RF_CUDA(cudaStreamSynchronize(h->stream));
    for (int i = 0; i < m0; ++i) th[i] = den[i] > 0 ? num[i] / den[i] : 0.0;
  }
  RF_CUDA(cudaMemcpyAsync(th_d, th.data(), sizeof(double) * m0, cudaMemcpyHostToDevice, h->stream));
  FilterStats fs;
  cudaEvent_t e0, e1;
  RF_CUDA(cudaEventCreate(&e0));
  RF_CUDA(cudaEventCreate(&e1));
  RF_CUDA(cudaEventRecord(e0, h->stream));
  int rc = RAFEAST_OK;
  try {
    run_filter(h, *prm, Qi, AQi, th_d, th, m0, ldq, Qti, fs);
  } catch (const Err& e) {
    // a breakdown still returns the filtered block; anything else is fatal
    if (e.code != RAFEAST_ERR_COCG_BREAKDOWN) throw;
    rc = e.code;
  }
  RF_CUDA(cudaEventRecord(e1, h->stream));
  launch_from_internal(h->n, m0, Qti, ldq, Qt, h->perm, nullptr, h->stream);
  RF_CUDA(cudaStreamSynchronize(h->stream));
  float ms = 0.f;
  RF_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (info) {
    memset(info, 0, sizeof(*info));
    info->status = rc;
    info->cocg_max_last = fs.iters_max;
    info->cocg_min_last = fs.iters_min;
    info->cocg_iters_total = fs.iters_max;
    info->t_filter_ms = ms;
    info->t_total_ms = ms;
    info->kernel_launches = h->launches;
    info->spmm_launches = h->spmm_launches;
  }
  scope.finish();
  return rc;
  API_END
}

int rafeast_orthonormalize(rafeast_t hh, int m, double* Q, double* R) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || m < 1 || m > 128 || !Q) return RAFEAST_ERR_INVALID_ARG;
  API_BEGIN
  CallScope scope(h);
  const int ld = even(m);
  double* A = (double*)scratch(h, S_TMP1, sizeof(double) * h->n * ld);
  double* B = (double*)scratch(h, S_TMP2, sizeof(double) * h->n * ld);
  launch_to_internal(h->n, m, Q, A, ld, h->perm, h->stream);
  std::vector<double> Rt;
  double* X = A;
  double* Y = B;
  cholqr(h, X, Y, m, ld, R ? &Rt : nullptr);
  launch_from_internal(h->n, m, X, ld, Q, h->perm, nullptr, h->stream);
  RF_CUDA(cudaStreamSynchronize(h->stream));
  if (R) {
    // column-major output of the row-major upper factor
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) R[(size_t)j * m + i] = Rt[(size_t)i * m + j];
  }
  scope.finish();
  return RAFEAST_OK;
  API_END
}

int rafeast_gram(rafeast_t hh, int m, const double* X, const double* Y, double* G) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || m < 1 || m > 128 || !X || !Y || !G) return RAFEAST_ERR_INVALID_ARG;
  API_BEGIN
  CallScope scope(h);
  const int ld = even(m);
  double* Xi = (double*)scratch(h, S_TMP1, sizeof(double) * h->n * ld);
  double* Yi = Xi;
  launch_to_internal(h->n, m, X, Xi, ld, h->perm, h->stream);
  if (Y != X) {  // (the same block twice: X^T X, one copy and one digit split)
    Yi = (double*)scratch(h, S_TMP2, sizeof(double) * h->n * ld);
    launch_to_internal(h->n, m, Y, Yi, ld, h->perm, h->stream);
  }
  DenseWs d = dense_ws(h, m);
  // row-major (Y^T X)[b][a] = sum_r Y[r][b] X[r][a] is G = X^T Y in column-major order
  gram_dev(h, Yi, Xi, m, ld, G, d, X == Y);
  h->launches += 4;
  scope.finish();
  RF_CUDA(cudaStreamSynchronize(h->stream));
  return RAFEAST_OK;
  API_END
}

int rafeast_block_product(rafeast_t hh, int m, const double* X, const double* M, int mo,
                          double* Y) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || m < 1 || m > 128 || mo < 1 || mo > 128 || !X || !M || !Y)
    return RAFEAST_ERR_INVALID_ARG;
  API_BEGIN
  CallScope scope(h);
  const int ldx = even(m), ldy = even(mo);
  double* Xi = (double*)scratch(h, S_TMP1, sizeof(double) * h->n * ldx);
  double* Yi = (double*)scratch(h, S_TMP2, sizeof(double) * h->n * ldy);
  launch_to_internal(h->n, m, X, Xi, ldx, h->perm, h->stream);
  // M: caller's column-major m x mo -> row-major, through the host (small)
  std::vector<double> mc((size_t)m * mo), mr((size_t)m * mo);
  RF_CUDA(cudaMemcpyAsync(mc.data(), M, sizeof(double) * m * mo, cudaMemcpyDeviceToHost,
                          h->stream));
  RF_CUDA(cudaStreamSynchronize(h->stream));
  for (int a = 0; a < m; ++a)
    for (int b = 0; b < mo; ++b) mr[(size_t)a * mo + b] = mc[(size_t)b * m + a];
  double* Mr = (double*)scratch(h, S_IO1, sizeof(double) * m * mo);
  RF_CUDA(cudaMemcpyAsync(Mr, mr.data(), sizeof(double) * m * mo, cudaMemcpyHostToDevice,
                          h->stream));
  tall_dev(h, Xi, m, ldx, Mr, mo, Yi, ldy);
  launch_from_internal(h->n, mo, Yi, ldy, Y, h->perm, nullptr, h->stream);
  h->launches += 3;
  scope.finish();
  RF_CUDA(cudaStreamSynchronize(h->stream));
  return RAFEAST_OK;
  API_END
}

int rafeast_rayleigh_ritz(rafeast_t hh, int m, double* Q, double* theta, double* resid) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || m < 1 || m > 128 || !Q || !theta) return RAFEAST_ERR_INVALID_ARG;
  API_BEGIN
  CallScope scope(h);
  const int ld = even(m);
  double* X = (double*)scratch(h, S_TMP1, sizeof(double) * h->n * ld);
  double* tmp = (double*)scratch(h, S_TMP2, sizeof(double) * h->n * ld);
  double* Qo = (double*)scratch(h, S_QT, sizeof(double) * h->n * ld);
  double* AQo = (double*)scratch(h, S_AQ2, sizeof(double) * h->n * ld);
  double* th_d = (double*)scratch(h, S_OMEGA, sizeof(double) * (m + 1));
  launch_to_internal(h->n, m, Q, X, ld, h->perm, h->stream);
  rayleigh_ritz_dev(h, X, m, ld, Qo, AQo, th_d, tmp);
  std::vector<double> res;
  residuals_host(h, Qo, AQo, th_d, m, ld, res);
  RF_CUDA(cudaMemcpyAsync(theta, th_d, sizeof(double) * m, cudaMemcpyDeviceToHost, h->stream));
  launch_from_internal(h->n, m, Qo, ld, Q, h->perm, nullptr, h->stream);
  RF_CUDA(cudaStreamSynchronize(h->stream));
  if (resid) std::copy(res.begin(), res.end(), resid);
  scope.finish();
  return RAFEAST_OK;
  API_END
}

int rafeast_warmstart(rafeast_t hh, double lmin, double lmax, int m0, int p, int q,
                      uint64_t seed) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || !(lmin < lmax) || m0 < 1 || p < 0 || q < 0 || m0 + p > 128 || m0 > 128 ||
      m0 + p > h->n)
    return RAFEAST_ERR_INVALID_ARG;
  API_BEGIN
  CallScope scope(h);
  const int k = m0 + p, ld = even(k);
  // B = s A + t I (Algorithm 2 Phase 1; the low-end map for low intervals)
  int which = h->opt_ws_map;
  if (which == 0) which = (0.5 * (lmin + lmax) >= 0.5 * (h->glo + h->ghi)) ? 1 : 2;
  double s, t;
  if (which == 1) {
    s = 1.0 / (lmax - lmin);
    t = -lmin * s;
  } else {
    s = -1.0 / (h->ghi - lmin);
    t = h->ghi / (h->ghi - lmin);
  }
  const double sL = s, sI = s * h->shift + t;  // B X = s L X + (s shift + t) X
  double* om = (double*)scratch(h, S_OMEGA, sizeof(double) * h->n * k);
  double* Y = (double*)scratch(h, S_TMP1, sizeof(double) * h->n * ld);
  double* Z = (double*)scratch(h, S_TMP2, sizeof(double) * h->n * ld);
  launch_omega(seed, h->n, k, om, h->stream);
  launch_to_internal(h->n, k, om, Z, ld, h->perm, h->stream);
  launch_spmm_real<double>(h->n, h->rowptr, h->colidx, h->val64, k, ld, sL, sI, Z, Y, h->num_sms,
                           h->stream);
  h->launches += 3;
  h->spmm_launches += 1;
  for (int it = 0; it < q; ++it) {
    cholqr(h, Y, Z, k, ld, nullptr, true);
    launch_spmm_real<double>(h->n, h->rowptr, h->colidx, h->val64, k, ld, sL, sI, Y, Z,
                             h->num_sms, h->stream);
    launch_spmm_real<double>(h->n, h->rowptr, h->colidx, h->val64, k, ld, sL, sI, Z, Y,
                             h->num_sms, h->stream);
    h->launches += 2;
    h->spmm_launches += 2;
  }
  cholqr(h, Y, Z, k, ld, nullptr, true);
  // Rayleigh-Ritz on the m0+p columns: A_Y = Y^T A Y, eigh, and only the m0
  // Ritz vectors kept are formed (Q = Y V_sel, then A Q)
  double* AY = (double*)scratch(h, S_AQ2, sizeof(double) * h->n * ld);
  double* th_all = (double*)scratch(h, S_IO1, sizeof(double) * (k + 1));
  {
    DenseWs d = dense_ws(h, k);
    launch_spmm_real<double>(h->n, h->rowptr, h->colidx, h->val64, k, ld, 1.0, h->shift, Y, AY,
                             h->num_sms, h->stream);
    gram_dev(h, Y, AY, k, ld, d.G, d, true);
    jacobi_eigh(d.G, k, th_all, d.V, d.Vw, h->stream);
    h->launches += 4;
    h->spmm_launches += 1;
  }
  std::vector<double> th(k), V((size_t)k * k);
  {
    DenseWs d = dense_ws(h, k);
    RF_CUDA(cudaMemcpyAsync(th.data(), th_all, sizeof(double) * k, cudaMemcpyDeviceToHost,
                            h->stream));
    RF_CUDA(cudaMemcpyAsync(V.data(), d.V, sizeof(double) * k * k, cudaMemcpyDeviceToHost,
                            h->stream));
    RF_CUDA(cudaStreamSynchronize(h->stream));
  }
  // keep the m0 Ritz values closest to the interval centre (stable ties)
  const double c = 0.5 * (lmin + lmax);
  std::vector<int> idx(k);
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(),
                   [&](int a, int b) { return std::fabs(th[a] - c) < std::fabs(th[b] - c); });
  idx.resize(m0);
  std::sort(idx.begin(), idx.end());
  // the kept eigenvector columns (k x m0, row-major) applied with the tall GEMM
  std::vector<double> S((size_t)k * m0, 0.0);
  for (int a = 0; a < k; ++a)
    for (int j = 0; j < m0; ++j) S[(size_t)a * m0 + j] = V[(size_t)a * k + idx[j]];
  ensure_subspace_bufs(h, m0);
  DenseWs d = dense_ws(h, k);
  RF_CUDA(cudaMemcpyAsync(d.V, S.data(), sizeof(double) * S.size(), cudaMemcpyHostToDevice,
                          h->stream));
  RF_CUDA(cudaMemsetAsync(h->Q, 0, sizeof(double) * h->n * h->ldq, h->stream));
  RF_CUDA(cudaMemsetAsync(h->AQ, 0, sizeof(double) * h->n * h->ldq, h->stream));
  tall_dev(h, Y, k, ld, d.V, m0, h->Q, h->ldq);
  launch_spmm_real<double>(h->n, h->rowptr, h->colidx, h->val64, m0, h->ldq, 1.0, h->shift, h->Q,
                           h->AQ, h->num_sms, h->stream);
  h->launches += 2;
  h->spmm_launches += 1;
  h->theta.resize(m0);
  for (int j = 0; j < m0; ++j) h->theta[j] = th[idx[j]];
  RF_CUDA(cudaMemcpyAsync(h->theta_d, h->theta.data(), sizeof(double) * m0,
                          cudaMemcpyHostToDevice, h->stream));
  RF_CUDA(cudaStreamSynchronize(h->stream));
  h->m0 = m0;
  scope.finish();
  return RAFEAST_OK;
  API_END
}

int rafeast_set_subspace(rafeast_t hh, const double* Q0, int m0, int on_device) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || !Q0 || m0 < 1 || m0 > 128 || m0 > h->n) return RAFEAST_ERR_INVALID_ARG;
  API_BEGIN
  CallScope scope(h);
  ensure_subspace_bufs(h, m0);
  import_block(h, Q0, m0, on_device, h->Q, h->ldq);
  subspace_from_Q(h, m0);
  scope.finish();
  return RAFEAST_OK;
  API_END
}

int rafeast_get_subspace(rafeast_t hh, double* Q, double* theta, int m0, int on_device) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || !Q) return RAFEAST_ERR_INVALID_ARG;
  if (!h->Q || h->m0 == 0) return RAFEAST_ERR_NOT_READY;
  if (m0 != h->m0) return RAFEAST_ERR_INVALID_ARG;
  API_BEGIN
  CallScope scope(h);
  export_block(h, h->Q, h->ldq, m0, nullptr, on_device, Q);
  if (theta) std::copy(h->theta.begin(), h->theta.end(), theta);
  scope.finish();
  RF_CUDA(cudaStreamSynchronize(h->stream));
  return RAFEAST_OK;
  API_END
}

int rafeast_solve(rafeast_t hh, const rafeast_params* prm, int* m_found, double* evals,
                  double* evecs, double* resid, int outputs_on_device, rafeast_info* info) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || !m_found || !evals) return RAFEAST_ERR_INVALID_ARG;
  API_BEGIN
  validate_params(prm);
  RF_CHECK(prm->reserved == 0, RAFEAST_ERR_INVALID_ARG);
  RF_CHECK(prm->m0 <= h->n, RAFEAST_ERR_INVALID_ARG);
  CallScope scope(h);
  SolveRun r;
  solve_begin(r, h, *prm);
  for (r.it = 1; r.it <= prm->max_outer; ++r.it) {
    RF_CUDA(cudaEventRecord(r.ev[2], h->stream));
    run_filter(h, *prm, h->Q, h->AQ, h->theta_d, h->theta, r.m0, r.ldq, r.Qt, r.fs);
    r.cocg_total += r.fs.iters_max;
    RF_CUDA(cudaEventRecord(r.ev[3], h->stream));
    if (solve_outer_tail(r)) break;
  }
  if (r.it > prm->max_outer) r.it = prm->max_outer;
  const int status = solve_finish(r, m_found, evals, evecs, resid, outputs_on_device, info);
  scope.finish();
  return status;
  API_END
}

int rafeast_shard_range(int mode, int m0, int nc, int rank, int world, int* lo, int* hi) {
  if (!lo || !hi || world < 1 || rank < 0 || rank >= world || m0 < 1 || nc < 1)
    return RAFEAST_ERR_INVALID_ARG;
  if (mode == RAFEAST_SHARD_COLUMNS) {
    // whole column pairs, so that every rank's block starts 16-byte aligned
    const int64_t pairs = (m0 + 1) / 2;
    *lo = (int)std::min<int64_t>(m0, 2 * (pairs * rank / world));
    *hi = (int)std::min<int64_t>(m0, 2 * (pairs * (rank + 1) / world));
  } else if (mode == RAFEAST_SHARD_SHIFTS) {
    *lo = (int)((int64_t)nc * rank / world);
    *hi = (int)((int64_t)nc * (rank + 1) / world);
  } else {
    return RAFEAST_ERR_INVALID_ARG;
  }
  return RAFEAST_OK;
}

int rafeast_partition_instances(int count, const int64_t* cost, int world, int32_t* owner) {
  if (count < 0 || world < 1 || (count > 0 && (!cost || !owner))) return RAFEAST_ERR_INVALID_ARG;
  for (int i = 0; i < count; ++i)
    if (cost[i] < 0) return RAFEAST_ERR_INVALID_ARG;
  // longest processing time first: largest cost to the least loaded rank
  // (ties: the lower instance index first, the lower rank)
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  std::vector<int64_t> load(world, 0);
  for (int i : order) {
    int r = 0;
    for (int q = 1; q < world; ++q)
      if (load[q] < load[r]) r = q;
    owner[i] = r;
    load[r] += cost[i];
  }
  return RAFEAST_OK;
}

int rafeast_solve_sharded(rafeast_t hh, const rafeast_params* prm, int mode, int rank, int world,
                          rafeast_sum_fn sum, void* ctx, int* m_found, double* evals,
                          double* evecs, double* resid, int outputs_on_device,
                          rafeast_info* info) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || !m_found || !evals) return RAFEAST_ERR_INVALID_ARG;
  if (world < 1 || rank < 0 || rank >= world || (world > 1 && !sum))
    return RAFEAST_ERR_INVALID_ARG;
  if (mode != RAFEAST_SHARD_COLUMNS && mode != RAFEAST_SHARD_SHIFTS) return RAFEAST_ERR_INVALID_ARG;
  API_BEGIN
  validate_params(prm);
  RF_CHECK(prm->reserved == 0, RAFEAST_ERR_INVALID_ARG);
  RF_CHECK(prm->m0 <= h->n, RAFEAST_ERR_INVALID_ARG);
  CallScope scope(h);
  SolveRun r;
  solve_begin(r, h, *prm);
  int lo = 0, hi = 0;
  rafeast_shard_range(mode, r.m0, prm->nc, rank, world, &lo, &hi);
  // the shift range lives in the handle for the filter's duration only
  struct ShardGuard {
    Handle* h;
    ~ShardGuard() {
      h->shard_j0 = 0;
      h->shard_j1 = -1;
    }
  } guard{h};
  double* flag = (double*)scratch(h, S_SHARD, 64);
  const size_t qt_bytes = sizeof(double) * h->n * r.ldq;
  auto exchange = [&](double* buf, int64_t count) {
    RF_CUDA(cudaStreamSynchronize(h->stream));
    if (sum(ctx, buf, count) != 0) {
      snprintf(g_err, sizeof(g_err), "sum callback failed (rank %d of %d)", rank, world);
      throw Err{RAFEAST_ERR_EXCHANGE};
    }
  };
  for (r.it = 1; r.it <= prm->max_outer; ++r.it) {
    RF_CUDA(cudaEventRecord(r.ev[2], h->stream));
    // this rank's share of Q~; the other ranks' columns (or nodes) stay zero,
    // so that the sum over ranks is the whole filtered block
    if (world > 1) RF_CUDA(cudaMemsetAsync(r.Qt, 0, qt_bytes, h->stream));
    r.fs = FilterStats();
    if (hi > lo) {
      if (mode == RAFEAST_SHARD_COLUMNS) {
        const std::vector<double> th(h->theta.begin() + lo, h->theta.begin() + hi);
        run_filter(h, *prm, h->Q + lo, h->AQ + lo, h->theta_d + lo, th, hi - lo, r.ldq,
                   r.Qt + lo, r.fs);
      } else {
        h->shard_j0 = lo;
        h->shard_j1 = hi;
        run_filter(h, *prm, h->Q, h->AQ, h->theta_d, h->theta, r.m0, r.ldq, r.Qt, r.fs);
        h->shard_j0 = 0;
        h->shard_j1 = -1;
      }
    }
    if (world > 1) exchange(r.Qt, (int64_t)h->n * r.ldq);
    r.cocg_total += r.fs.iters_max;
    RF_CUDA(cudaEventRecord(r.ev[3], h->stream));
    bool done = solve_outer_tail(r);
    if (world > 1) {
      // every rank runs the same dense steps on the same block; the ranks
      // still agree on stopping (all converged), so that no rank leaves the
      // loop while another waits in the next sum
      const double one = done ? 1.0 : 0.0;
      RF_CUDA(cudaMemcpyAsync(flag, &one, sizeof(double), cudaMemcpyHostToDevice, h->stream));
      exchange(flag, 1);
      double tot = 0.0;
      RF_CUDA(cudaMemcpyAsync(&tot, flag, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
      RF_CUDA(cudaStreamSynchronize(h->stream));
      done = tot > world - 0.5;
      if (!done) r.status = RAFEAST_NO_CONVERGENCE;
    }
    if (done) break;
  }
  if (r.it > prm->max_outer) r.it = prm->max_outer;
  const int status = solve_finish(r, m_found, evals, evecs, resid, outputs_on_device, info);
  scope.finish();
  return status;
  API_END
}

int rafeast_solve_batched(int count, rafeast_t const* hs, const rafeast_params* prms,
                          int* m_found, double* const* evals, double* const* evecs,
                          double* const* resid, int outputs_on_device, rafeast_info* infos,
                          int* statuses) {
  if (count < 0 || (count > 0 && (!hs || !prms || !m_found || !evals || !statuses)))
    return RAFEAST_ERR_INVALID_ARG;
  if (count == 0) return RAFEAST_OK;
  clear_last_error();
  API_BEGIN
  std::vector<Handle*> H(count);
  for (int t = 0; t < count; ++t) {
    H[t] = reinterpret_cast<Handle*>(hs[t]);
    RF_CHECK(H[t] && evals[t], RAFEAST_ERR_INVALID_ARG);
    validate_params(&prms[t]);
    RF_CHECK(prms[t].reserved == 0 && prms[t].m0 <= H[t]->n, RAFEAST_ERR_INVALID_ARG);
    if (prms[t].precision != prms[0].precision || prms[t].nc != prms[0].nc ||
        H[t]->device != H[0]->device) {
      set_last_message("rafeast_solve_batched: every problem of a batch needs the same "
                       "precision, the same nc and the same device");
      throw Err{RAFEAST_ERR_INVALID_ARG};
    }
    for (int u = 0; u < t; ++u)
      if (H[u] == H[t]) {
        set_last_message("rafeast_solve_batched: a handle appears twice in the batch");
        throw Err{RAFEAST_ERR_INVALID_ARG};
      }
  }
  Handle* owner = H[0];
  const cudaStream_t bs = owner->stream;
  std::vector<std::unique_ptr<CallScope>> scopes;
  for (int t = 0; t < count; ++t) scopes.emplace_back(new CallScope(H[t]));
  std::vector<SolveRun> runs(count);
  std::vector<BatchItem> items(count);
  std::vector<std::string> msgs(count);
  // per-problem phases run on the problems' own streams from a few host
  // threads, so their short kernels and host round trips overlap
  auto each = [&](const std::vector<int>& which, const std::function<void(int)>& f) {
    std::atomic<int> next(0);
    auto work = [&]() {
      cudaSetDevice(owner->device);
      for (;;) {
        const int k = next.fetch_add(1);
        if (k >= (int)which.size()) break;
        const int t = which[k];
        try {
          f(t);
        } catch (const Err& e) {
          items[t].err = e.code;
          msgs[t] = g_err;
        } catch (...) {
          items[t].err = RAFEAST_ERR_CUDA;
        }
      }
    };
    const int nt = std::min<int>((int)which.size(), 16);
    std::vector<std::thread> th;
    for (int k = 1; k < nt; ++k) th.emplace_back(work);
    work();
    for (auto& x : th) x.join();
  };
  std::vector<int> all(count);
  std::iota(all.begin(), all.end(), 0);
  for (int t = 0; t < count; ++t) {
    items[t].h = H[t];
    items[t].prm = &prms[t];
  }
  each(all, [&](int t) {
    solve_begin(runs[t], H[t], prms[t]);
    items[t].Qt = runs[t].Qt;
  });
  if (owner->opt_profile) {
    owner->last_hist.clear();
    owner->last_rhist.clear();
    owner->last_tk.clear();
  }
  // signature of the batch for the shape autotuner (negative: batch keys)
  int64_t sig = count;
  for (int t = 0; t < count; ++t)
    sig = sig * 1000003 + H[t]->n * 131 + prms[t].m0 * 7 + prms[t].nc;
  sig = -(sig & 0x3fffffffffffffffLL) - 1;
  std::vector<char> done(count, 0);
  int max_outer = 0;
  for (int t = 0; t < count; ++t) max_outer = std::max(max_outer, prms[t].max_outer);
  for (int it = 1; it <= max_outer; ++it) {
    std::vector<int> act;
    std::vector<BatchItem*> act_items;
    for (int t = 0; t < count; ++t)
      if (!done[t] && !items[t].err && it <= prms[t].max_outer) {
        act.push_back(t);
        act_items.push_back(&items[t]);
        runs[t].it = it;
        RF_CUDA(cudaEventRecord(runs[t].ev[2], bs));
      }
    if (act.empty()) break;
    if (prms[0].precision == RAFEAST_FP64) filter_ms_batched<double>(act_items, owner, bs, sig);
    else filter_ms_batched<float>(act_items, owner, bs, sig);
    for (int t : act) {
      runs[t].fs = items[t].fs;
      runs[t].cocg_total += items[t].fs.iters_max;
      RF_CUDA(cudaEventRecord(runs[t].ev[3], bs));
    }
    // the problems' phases read the filter's end event from their own threads
    RF_CUDA(cudaStreamSynchronize(bs));
    std::vector<int> ok;
    for (int t : act)
      if (!items[t].err) ok.push_back(t);
    each(ok, [&](int t) {
      if (solve_outer_tail(runs[t])) done[t] = 1;
    });
  }
  int first_err = RAFEAST_OK;
  std::vector<int> fin;
  for (int t = 0; t < count; ++t)
    if (!items[t].err) fin.push_back(t);
  each(fin, [&](int t) {
    statuses[t] = solve_finish(runs[t], &m_found[t], evals[t], evecs ? evecs[t] : nullptr,
                               resid ? resid[t] : nullptr, outputs_on_device,
                               infos ? &infos[t] : nullptr);
  });
  for (int t = 0; t < count; ++t) {
    if (items[t].err) {
      statuses[t] = items[t].err;
      if (infos) {
        memset(&infos[t], 0, sizeof(rafeast_info));
        infos[t].status = items[t].err;
      }
      if (first_err == RAFEAST_OK) {
        first_err = items[t].err;
        if (!msgs[t].empty()) set_last_message(msgs[t].c_str());
      }
    }
  }
  for (auto& sc : scopes) sc->finish();
  return first_err;
  API_END
}

}  // extern "C"
