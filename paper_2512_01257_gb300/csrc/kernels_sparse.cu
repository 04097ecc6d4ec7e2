// Sparse kernels of the RA-FEAST hot path (sm_103a).
//
// 1. Batched COCG for the shifted systems (z_j I - A) X_j = B of Algorithm 1 /
//    Algorithm 2 Step 2a, all N_c shifts x m0 columns in one launch. Each
//    COCG step is two launches (Chronopoulos-Gear ordering of the CG scalars:
//    one global reduction per step):
//      dots   : w = M r_k with M = (z_j - sigma) I - L, gathered from r_k;
//               gamma = r^T r, delta = r^T w, nu = ||r||^2 (Hermitian) per
//               system; the last CTA turns them into alpha_k, beta_k in FP64.
//      update : p_k = r_k + beta_k p_{k-1}, s = M p_k recomputed from the
//               gathered r_k and p_{k-1} (no stored w/s vector),
//               r_{k+1} = r_k - alpha_k s, and the quadrature sum
//               D += Re(c_js alpha_k p_k) (x is never stored).
//    Per step the state is streamed 5.5 times (n x ldc complex) instead of the
//    11 times of the textbook three-kernel form with stored x and w.
// 2. Plain SpMM variants with the same gather core: W = zs P - L P (complex,
//    for rafeast_shifted_spmm) and Y = sL (L X) + sI X (real; warmstart powers
//    and Rayleigh-Ritz products).
//
// Work mapping: a CTA has 8 warps; a warp is split into groups of G lanes
// (G = 4..32); each group owns one row at a time (grid-stride over rows so
// all CTAs sweep A's rows together and gathered rows are reused in L2);
// lane l of a group owns column chunks i = base + l + c*G, c < cpl, each chunk
// holding the NC shifts of subspace column i.
#include <cstdio>
#include <type_traits>

#include "cocg_kernels.cuh"

namespace rafeast {

int nc_pad(int nc) {
  if (nc <= 1) return 1;
  if (nc <= 2) return 2;
  if (nc <= 4) return 4;
  return 8;
}
int max_cpl(int NC, bool fp64) { return fp64 ? maxcpl_of<double>(NC) : maxcpl_of<float>(NC); }

void choose_shape(int m0, int NC, bool fp64, int forced_lanes, int& lanes, int& cpl,
                  int& colblocks, int forced_cpl) {
  int mc = max_cpl(NC, fp64);
  if (forced_cpl > 0 && forced_cpl < mc) mc = forced_cpl;
  double best = -1.0;
  const int cands[4] = {32, 16, 8, 4};
  for (int t = 0; t < 4; ++t) {
    int G = cands[t];
    if (forced_lanes && G != forced_lanes) continue;
    int c = (m0 + G - 1) / G;
    if (c > mc) c = mc;
    int blocks = (m0 + G * c - 1) / (G * c);
    double eff = double(m0) / double(blocks * G * c);
    // prefer wide groups (fewer re-reads of A) unless much less efficient
    double score = eff - 0.02 * (blocks - 1);
    if (score > best + 1e-12) {
      best = score;
      lanes = G;
      cpl = c;
      colblocks = blocks;
    }
  }
}

// ---------------------------------------------------------------------------
// COCG: reset of the small per-system arrays
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_cocg_reset(CocgArgs<T> a, int NC) {
  const int nsys = a.m0 * NC;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nsys; s += gridDim.x * blockDim.x) {
    SysState st;
    st.gamma_prev = make_double2(1.0, 0.0);
    st.alpha_prev = make_double2(1.0, 0.0);
    st.bnorm2 = 0.0;
    st.active = 1;
    st.iters = 0;
    a.st[s] = st;
    for (int q = 0; q < 5; ++q) a.acc[5 * s + q] = 0.0;
    if (s % NC == 0) a.colact[s / NC] = 1;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    CocgCtl c = {};
    c.g_mn = 0x7fffffff;
    c.ticket = 0;
    c.iter = 0;
    c.active = nsys;
    c.done = 0;
    c.breakdown = 0;
    c.capped = 0;
    c.max_iters = 0;
    c.min_iters = 0;
    c.timeout = 0;
    *a.ctl = c;
  }
}

// init: r0 = b (real rhs, zero imaginary part), p_{-1} = 0, D = 0
template <typename T, int NC>
__global__ void __launch_bounds__(THREADS) k_cocg_init(CocgArgs<T> a) {
  using C = c2<T>;
  const int64_t total = a.n * (int64_t)a.m0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = e / a.m0;
    const int i = (int)(e - row * a.m0);
    double b = a.qin[row * a.ldq + i];
    if (a.form == RAFEAST_FORM_CORRECTION) b = a.aqin[row * a.ldq + i] - a.theta[i] * b;
    C rv[NC], pv[NC];
#pragma unroll
    for (int j = 0; j < NC; ++j) {
      rv[j] = mk<T>(j < a.nc_real ? (T)b : (T)0, (T)0);
      pv[j] = mk<T>((T)0, (T)0);
    }
    const int64_t off = (row * a.ldc + (int64_t)i * NC) * 2;
    st_chunk<NC>(a.r[0] + off, rv);
    st_chunk<NC>(a.p[0] + off, pv);
    a.dacc[row * a.ldd + i] = (T)0;
  }
}

// ---------------------------------------------------------------------------
// COCG dots kernel
// ---------------------------------------------------------------------------
template <typename T, int NC, int MAXCPL, bool VF = false>
__global__ void __launch_bounds__(THREADS, (MAXCPL * NC <= 4) ? 2 : 1)
    k_cocg_dots(CocgArgs<T> a, int buf) {
  cocg_dots_body<T, NC, MAXCPL, VF>(a, &a, buf, grid_blk());
}

// ---------------------------------------------------------------------------
// COCG update kernel
// ---------------------------------------------------------------------------
template <typename T, int NC, int MAXCPL>
__global__ void __launch_bounds__(THREADS, sizeof(T) == 4 ? 2 : 1)
    k_cocg_update(CocgArgs<T> a, int buf) {
  using C = c2<T>;
  if (__ldcg(&a.ctl->done)) return;
  const RowMap mp = row_map(a.lanes, a.cpl, grid_blk());
  const unsigned gmask = group_mask(mp.G);
  const int ibase = blockIdx.y * mp.G * mp.cpl + mp.lg;
  const T* __restrict__ R = a.r[buf];
  const T* __restrict__ P = a.p[buf];
  T* __restrict__ Rn = a.r[buf ^ 1];
  T* __restrict__ Pn = a.p[buf ^ 1];
  const int64_t ldt = (int64_t)a.ldc * 2;
  const C* zs = reinterpret_cast<const C*>(a.zs);
  C zv[NC];
#pragma unroll
  for (int j = 0; j < NC; ++j) zv[j] = zs[j];
  // stage this block's coefficients in shared memory
  extern __shared__ unsigned char smem_raw[];
  Coef<T>* scf = reinterpret_cast<Coef<T>*>(smem_raw);
  const int i0 = blockIdx.y * mp.G * mp.cpl;
  const int ncols = min(mp.G * mp.cpl, a.m0 - i0);
  for (int t = threadIdx.x; t < ncols * NC; t += blockDim.x) scf[t] = a.cf[i0 * NC + t];
  __syncthreads();
  int coff[MAXCPL];
  unsigned mask = 0;
#pragma unroll
  for (int c = 0; c < MAXCPL; ++c) {
    const int i = ibase + c * mp.G;
    coff[c] = i * NC * 2;
    if (c < mp.cpl && i < a.m0 && __ldcg(a.colact + i)) mask |= 1u << c;
  }
  // warp-uniform exit: the gathers shuffle across the whole lane group
  if (!__any_sync(0xffffffffu, mask != 0)) return;
  for (int64_t row = mp.gid; row < a.n; row += mp.gstride) {
    const int k0 = __ldg(a.rowptr + row), k1 = __ldg(a.rowptr + row + 1);
    C ar[MAXCPL][NC], ap[MAXCPL][NC];
#pragma unroll
    for (int c = 0; c < MAXCPL; ++c)
#pragma unroll
      for (int j = 0; j < NC; ++j) ar[c][j] = ap[c][j] = mk<T>((T)0, (T)0);
    gather_row2<T, NC, MAXCPL>(a.colidx, a.val, k0, k1, (int)row, mp.lg, mp.G, gmask, R, P, ldt,
                               coff, mask, ar, ap);
#pragma unroll
    for (int c = 0; c < MAXCPL; ++c)
      if (mask & (1u << c)) {
        C rv[NC], pv[NC];
        ld_chunk<NC>(R + row * ldt + coff[c], rv);
        ld_chunk<NC>(P + row * ldt + coff[c], pv);
        const int il = (ibase + c * mp.G) - i0;
        T dsum = (T)0;
#pragma unroll
        for (int j = 0; j < NC; ++j) {
          const Coef<T> cf = scf[il * NC + j];
          // p_k = ar r_k + beta p_{k-1};  L p_k from the gathered sums
          const C pn = cfma<T>(cf.beta, pv[j], mk<T>(cf.ar * rv[j].x, cf.ar * rv[j].y));
          const C lpn = cfma<T>(cf.beta, ap[c][j], mk<T>(cf.ar * ar[c][j].x, cf.ar * ar[c][j].y));
          const C s = csub<T>(cmul<T>(zv[j], pn), lpn);
          rv[j] = csub<T>(rv[j], cmul<T>(cf.alpha, s));
          pv[j] = pn;
          dsum = fma(cf.ca.x, pn.x, fma(-cf.ca.y, pn.y, dsum));
        }
        st_chunk<NC>(Rn + row * ldt + coff[c], rv);
        st_chunk<NC>(Pn + row * ldt + coff[c], pv);
        T* dp = a.dacc + row * a.ldd + (ibase + c * mp.G);
        *dp += dsum;
      }
  }
}

// ---------------------------------------------------------------------------
// multi-shift COCG: reset, init, update. The seed's R and P use the NC = 2
// chunk layout over column pairs (pair q = columns 2q, 2q+1, complex offset
// row*ldc + 2q); the shifted directions ps hold, for pair q and non-seed
// shift t, columns 2q and 2q+1 at complex offset row*ldps + 2*(q*ns + t).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_ms_reset(CocgArgs<T> a) {
  const int ncol = 2 * a.m0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ncol; i += gridDim.x * blockDim.x) {
    SysState st;
    st.gamma_prev = make_double2(1.0, 0.0);
    st.alpha_prev = make_double2(1.0, 0.0);
    st.bnorm2 = 0.0;
    st.active = 1;
    st.iters = 0;
    a.st[i] = st;
    for (int q = 0; q < 5; ++q) a.acc[5 * i + q] = 0.0;
    if ((i & 1) == 0) a.colact[i / 2] = 1;
    for (int t = 0; t < a.ns; ++t) {
      ShiftState ss;
      ss.zeta = make_double2(1.0, 0.0);
      ss.zeta_prev = make_double2(1.0, 0.0);
      ss.active = 1;
      ss.iters = 0;
      a.sst[i * a.ns + t] = ss;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    CocgCtl c = {};
    c.g_mn = 0x7fffffff;
    c.ticket = 0;
    c.iter = 0;
    c.active = ncol;
    c.done = 0;
    c.breakdown = 0;
    c.capped = 0;
    c.max_iters = 0;
    c.min_iters = 0;
    c.timeout = 0;
    *a.ctl = c;
  }
}

// r0 = b for every column (b = 0 in a padding column), p = ps = 0, D = 0;
// a.qin/aqin hold m_real = ldq-strided columns, a.m0 is the pair count
template <typename T>
__global__ void __launch_bounds__(THREADS) k_ms_init(CocgArgs<T> a, int m_real) {
  const int ncol = 2 * a.m0;
  const int64_t total = a.n * (int64_t)ncol;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = e / ncol;
    const int i = (int)(e - row * ncol);
    double b = 0.0;
    if (i < m_real) {
      b = a.qin[row * a.ldq + i];
      if (a.form == RAFEAST_FORM_CORRECTION) b = a.aqin[row * a.ldq + i] - a.theta[i] * b;
    }
    const int64_t off = (row * a.ldc + i) * 2;
    a.r[0][off] = (T)b;
    a.r[0][off + 1] = (T)0;
    a.p[0][off] = (T)0;
    a.p[0][off + 1] = (T)0;
    if (a.sbuf) {  // s_{-1} = M p_{-1} = 0
      a.sbuf[off] = (T)0;
      a.sbuf[off + 1] = (T)0;
    }
    a.dacc[row * a.ldd + i] = (T)0;
    const int q = i >> 1, h = i & 1;
    for (int t = 0; t < a.ns; ++t) {
      const int64_t po = (row * a.ldps + 2 * ((int64_t)q * a.ns + t) + h) * 2;
      a.ps[po] = (T)0;
      a.ps[po + 1] = (T)0;
    }
  }
}

template <typename T, int NS, int MAXCPL>
__global__ void __launch_bounds__(THREADS, sizeof(T) == 4 ? 2 : 1)
    k_ms_update(CocgArgs<T> a, int buf) {
  ms_update_body<T, NS, MAXCPL>(a, &a, buf, grid_blk());
}

// the same kernels compiled for MINB resident CTAs per SM (fewer registers
// per thread, more warps to hide the gathers' latency); the autotuner picks
// them when they measure faster
template <typename T, int NS, int MAXCPL, int MINB>
__global__ void __launch_bounds__(THREADS, MINB) k_ms_update_occ(CocgArgs<T> a, int buf) {
  ms_update_body<T, NS, MAXCPL>(a, &a, buf, grid_blk());
}
template <typename T, int MAXCPL, int MINB, bool VF = false>
__global__ void __launch_bounds__(THREADS, MINB) k_cocg_dots_occ(CocgArgs<T> a, int buf) {
  cocg_dots_body<T, 2, MAXCPL, VF>(a, &a, buf, grid_blk());
}

template <typename T, int NS>
__global__ void __launch_bounds__(THREADS) k_ms_update_stream(CocgArgs<T> a, int buf) {
  if (__ldcg(&a.ctl->done)) return;
  // deferred form: the next dot kernel finds this step's shifted updates
  // pending (it starts after this kernel ends)
  if (a.defer && blockIdx.x == 0 && threadIdx.x == 0) a.ctl->pend = 1;
  extern __shared__ unsigned char smem_raw[];
  ms_stream_stage<T, NS>(a, smem_raw);
  ms_stream_elems<T, NS>(a, smem_raw, blockIdx.x * (int64_t)blockDim.x + threadIdx.x,
                         a.n * (int64_t)a.m0, (int64_t)gridDim.x * blockDim.x, 0, true, buf);
}

template <typename T, int NS>
static void dispatch_ms_update_stream(const CocgArgs<T>& a, int buf, int num_sms,
                                      cudaStream_t s) {
  // (NS < 0: the instance reads the shift count a.ns at run time)
  const size_t smem = ms_stream_smem<T>(a.m0, NS < 0 ? a.ns : NS);
  auto kern = k_ms_update_stream<T, NS>;
  if (smem > 48 * 1024) ensure_dyn_smem(reinterpret_cast<const void*>(kern), smem);
  int occ = 0;
  RF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, THREADS, smem));
  if (occ < 1) occ = 1;
  int64_t blocks = (a.n * (int64_t)a.m0 + THREADS - 1) / THREADS;
  if (blocks > (int64_t)num_sms * occ) blocks = (int64_t)num_sms * occ;
  if (blocks < 1) blocks = 1;
  kern<<<(int)blocks, THREADS, smem, s>>>(a, buf);
  RF_LAUNCH();
}

template <typename T>
void launch_ms_update_stream(const CocgArgs<T>& a, int buf, int num_sms, cudaStream_t s) {
  // (r in place or ping-ponged; the deferred form needs both residuals)
  RF_CHECK(a.wbuf && a.sbuf && a.p[0] == a.p[1] && (!a.defer || a.r[0] != a.r[1]),
           RAFEAST_ERR_INVALID_ARG);
  switch (a.ns) {
    case 0: dispatch_ms_update_stream<T, 0>(a, buf, num_sms, s); break;
    case 1: dispatch_ms_update_stream<T, 1>(a, buf, num_sms, s); break;
    case 2: dispatch_ms_update_stream<T, 2>(a, buf, num_sms, s); break;
    case 3: dispatch_ms_update_stream<T, 3>(a, buf, num_sms, s); break;
    case 4: dispatch_ms_update_stream<T, 4>(a, buf, num_sms, s); break;
    case 5: dispatch_ms_update_stream<T, 5>(a, buf, num_sms, s); break;
    case 6: dispatch_ms_update_stream<T, 6>(a, buf, num_sms, s); break;
    case 7: dispatch_ms_update_stream<T, 7>(a, buf, num_sms, s); break;
    default:  // N_c = 9..16: the shift count read at run time
      if (a.ns < 0 || a.ns > 15) throw Err{RAFEAST_ERR_INVALID_ARG};
      dispatch_ms_update_stream<T, -1>(a, buf, num_sms, s);
      break;
  }
}
template void launch_ms_update_stream<float>(const CocgArgs<float>&, int, int, cudaStream_t);
template void launch_ms_update_stream<double>(const CocgArgs<double>&, int, int, cudaStream_t);

template <typename T, int NS>
static void dispatch_ms_update(const CocgArgs<T>& a, int buf, int num_sms, cudaStream_t s) {
  constexpr int MCS = 2, MCL = sizeof(T) == 4 ? 4 : 2;
  const size_t smem = (size_t)2 * a.lanes * a.cpl * (sizeof(Coef<T>) + NS * sizeof(ShiftCoef<T>)) + 16;
  const int colblocks = (a.m0 + a.lanes * a.cpl - 1) / (a.lanes * a.cpl);
  const int64_t groups = (a.n + (int64_t)WARPS * (32 / a.lanes) - 1) / ((int64_t)WARPS * (32 / a.lanes));
  bool done = false;
  if constexpr (sizeof(T) == 4) {
    if (a.occ >= 3 && a.cpl <= MCS) {
      auto kern = a.occ >= 4 ? k_ms_update_occ<T, NS, MCS, 4> : k_ms_update_occ<T, NS, MCS, 3>;
      if (smem > 48 * 1024) ensure_dyn_smem(reinterpret_cast<const void*>(kern), smem);
      dim3 grid(grid_x(kern, smem, num_sms, groups), colblocks);
      kern<<<grid, THREADS, smem, s>>>(a, buf);
      done = true;
    }
  }
  if (done) {
  } else if (a.cpl <= MCS) {
    auto kern = k_ms_update<T, NS, MCS>;
    if (smem > 48 * 1024) ensure_dyn_smem(reinterpret_cast<const void*>(kern), smem);
    dim3 grid(grid_x(kern, smem, num_sms, groups), colblocks);
    kern<<<grid, THREADS, smem, s>>>(a, buf);
  } else {
    if (a.cpl > MCL) throw Err{RAFEAST_ERR_INVALID_ARG};
    auto kern = k_ms_update<T, NS, MCL>;
    if (smem > 48 * 1024) ensure_dyn_smem(reinterpret_cast<const void*>(kern), smem);
    dim3 grid(grid_x(kern, smem, num_sms, groups), colblocks);
    kern<<<grid, THREADS, smem, s>>>(a, buf);
  }
  RF_LAUNCH();
}

int ms_max_cpl(bool fp64) { return fp64 ? 2 : 4; }

template <typename T>
void launch_ms_init(const CocgArgs<T>& a, int m_real, int num_sms, cudaStream_t s) {
  k_ms_reset<T><<<(2 * a.m0 + 255) / 256, 256, 0, s>>>(a);
  RF_LAUNCH();
  const int64_t total = a.n * (int64_t)(2 * a.m0);
  int64_t blocks = (total + THREADS - 1) / THREADS;
  if (blocks > (int64_t)num_sms * 8) blocks = (int64_t)num_sms * 8;
  if (blocks < 1) blocks = 1;
  k_ms_init<T><<<(int)blocks, THREADS, 0, s>>>(a, m_real);
  RF_LAUNCH();
}

template <typename T>
void launch_ms_update(const CocgArgs<T>& a, int buf, int num_sms, cudaStream_t s) {
  switch (a.ns) {
    case 0: dispatch_ms_update<T, 0>(a, buf, num_sms, s); break;
    case 1: dispatch_ms_update<T, 1>(a, buf, num_sms, s); break;
    case 2: dispatch_ms_update<T, 2>(a, buf, num_sms, s); break;
    case 3: dispatch_ms_update<T, 3>(a, buf, num_sms, s); break;
    case 4: dispatch_ms_update<T, 4>(a, buf, num_sms, s); break;
    case 5: dispatch_ms_update<T, 5>(a, buf, num_sms, s); break;
    case 6: dispatch_ms_update<T, 6>(a, buf, num_sms, s); break;
    case 7: dispatch_ms_update<T, 7>(a, buf, num_sms, s); break;
    default: throw Err{RAFEAST_ERR_INVALID_ARG};
  }
}

template void launch_ms_init<float>(const CocgArgs<float>&, int, int, cudaStream_t);
template void launch_ms_init<double>(const CocgArgs<double>&, int, int, cudaStream_t);
template void launch_ms_update<float>(const CocgArgs<float>&, int, int, cudaStream_t);
template void launch_ms_update<double>(const CocgArgs<double>&, int, int, cudaStream_t);

// ---------------------------------------------------------------------------
// plain SpMM variants
// ---------------------------------------------------------------------------
template <typename T, int NC, int MAXCPL>
__global__ void __launch_bounds__(THREADS) k_shifted_spmm(int64_t n, const int32_t* rp,
                                                          const int32_t* ci, const T* val,
                                                          int m, int ldc, const void* zsp,
                                                          const T* P, T* W, int G, int cpl) {
  using C = c2<T>;
  const RowMap mp = row_map(G, cpl, grid_blk());
  const unsigned gmask = group_mask(G);
  const int ibase = blockIdx.y * G * cpl + mp.lg;
  const int64_t ldt = (int64_t)ldc * 2;
  const C* zs = reinterpret_cast<const C*>(zsp);
  C zv[NC];
#pragma unroll
  for (int j = 0; j < NC; ++j) zv[j] = zs[j];
  int coff[MAXCPL];
  unsigned mask = 0;
#pragma unroll
  for (int c = 0; c < MAXCPL; ++c) {
    const int i = ibase + c * G;
    coff[c] = i * NC * 2;
    if (c < cpl && i < m) mask |= 1u << c;
  }
  // warp-uniform exit: the gathers shuffle across the whole lane group
  if (!__any_sync(0xffffffffu, mask != 0)) return;
  for (int64_t row = mp.gid; row < n; row += mp.gstride) {
    C acc[MAXCPL][NC];
#pragma unroll
    for (int c = 0; c < MAXCPL; ++c)
#pragma unroll
      for (int j = 0; j < NC; ++j) acc[c][j] = mk<T>((T)0, (T)0);
    gather_row<T, NC, MAXCPL>(ci, val, __ldg(rp + row), __ldg(rp + row + 1), (int)row, mp.lg, G,
                              gmask, P, ldt, coff, mask, acc);
#pragma unroll
    for (int c = 0; c < MAXCPL; ++c)
      if (mask & (1u << c)) {
        C pv[NC];
        ld_chunk<NC>(P + row * ldt + coff[c], pv);
#pragma unroll
        for (int j = 0; j < NC; ++j) pv[j] = csub<T>(cmul<T>(zv[j], pv[j]), acc[c][j]);
        st_chunk<NC>(W + row * ldt + coff[c], pv);
      }
  }
}

template <typename T, int MAXCPL>
__global__ void __launch_bounds__(THREADS) k_spmm_real(int64_t n, const int32_t* rp,
                                                       const int32_t* ci, const T* val, int mc,
                                                       int ld, T sL, T sI, const T* X, T* Y,
                                                       int G, int cpl) {
  using C = c2<T>;
  const RowMap mp = row_map(G, cpl, grid_blk());
  const unsigned gmask = group_mask(G);
  const int ibase = blockIdx.y * G * cpl + mp.lg;
  int coff[MAXCPL];
  unsigned mask = 0;
#pragma unroll
  for (int c = 0; c < MAXCPL; ++c) {
    const int i = ibase + c * G;
    coff[c] = i * 2;
    if (c < cpl && i < mc) mask |= 1u << c;
  }
  // warp-uniform exit: the gathers shuffle across the whole lane group
  if (!__any_sync(0xffffffffu, mask != 0)) return;
  for (int64_t row = mp.gid; row < n; row += mp.gstride) {
    C acc[MAXCPL][1];
#pragma unroll
    for (int c = 0; c < MAXCPL; ++c) acc[c][0] = mk<T>((T)0, (T)0);
    gather_row<T, 1, MAXCPL>(ci, val, __ldg(rp + row), __ldg(rp + row + 1), (int)row, mp.lg, G,
                             gmask, X, ld, coff, mask, acc);
#pragma unroll
    for (int c = 0; c < MAXCPL; ++c)
      if (mask & (1u << c)) {
        C xv[1];
        ld_chunk<1>(X + row * ld + coff[c], xv);
        C y = mk<T>(sL * acc[c][0].x + sI * xv[0].x, sL * acc[c][0].y + sI * xv[0].y);
        *reinterpret_cast<C*>(Y + row * ld + coff[c]) = y;
      }
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------


template <typename T, int NC, int MC>
static void dispatch_dots_mc(const CocgArgs<T>& a, int buf, int num_sms, cudaStream_t s) {
  auto kern = k_cocg_dots<T, NC, MC>;
  if constexpr (NC == 2) {
    // column pairs of the multi-shift seed: values-free instances for a
    // unit-weight Laplacian (a.lcolidx), occupancy-forced ones (a.occ)
    const bool vf = a.lcolidx != nullptr;
    if (vf) kern = k_cocg_dots<T, NC, MC, true>;
    if constexpr (MC == 2 && sizeof(T) == 4) {
      if (a.occ >= 3)
        kern = a.occ >= 4 ? (vf ? k_cocg_dots_occ<T, MC, 4, true> : k_cocg_dots_occ<T, MC, 4>)
                          : (vf ? k_cocg_dots_occ<T, MC, 3, true> : k_cocg_dots_occ<T, MC, 3>);
    }
    // double, one chunk per lane: compiled for 3 CTAs per SM
    if constexpr (MC == 1 && sizeof(T) == 8)
      kern = vf ? k_cocg_dots_occ<T, 1, 3, true> : k_cocg_dots_occ<T, 1, 3>;
    if constexpr ((MC == 3 || MC == 4) && sizeof(T) == 4) {
      if (a.occ >= 2)
        kern = a.occ >= 3 ? (vf ? k_cocg_dots_occ<T, MC, 3, true> : k_cocg_dots_occ<T, MC, 3>)
                          : (vf ? k_cocg_dots_occ<T, MC, 2, true> : k_cocg_dots_occ<T, MC, 2>);
    }
  }
  const size_t smem = (size_t)a.lanes * MC * NC * 5 * sizeof(double);
  const int colblocks = (a.m0 + a.lanes * a.cpl - 1) / (a.lanes * a.cpl);
  const int64_t groups = (a.n + (int64_t)WARPS * (32 / a.lanes) - 1) / ((int64_t)WARPS * (32 / a.lanes));
  dim3 grid(grid_x(kern, smem, num_sms, groups), colblocks);
  kern<<<grid, THREADS, smem, s>>>(a, buf);
  RF_LAUNCH();
}

template <typename T, int NC, int MC>
static void dispatch_update_mc(const CocgArgs<T>& a, int buf, int num_sms, cudaStream_t s) {
  auto kern = k_cocg_update<T, NC, MC>;
  const size_t smem = (size_t)a.lanes * MC * NC * sizeof(Coef<T>);
  const int colblocks = (a.m0 + a.lanes * a.cpl - 1) / (a.lanes * a.cpl);
  const int64_t groups = (a.n + (int64_t)WARPS * (32 / a.lanes) - 1) / ((int64_t)WARPS * (32 / a.lanes));
  dim3 grid(grid_x(kern, smem, num_sms, groups), colblocks);
  kern<<<grid, THREADS, smem, s>>>(a, buf);
  RF_LAUNCH();
}

template <typename T>
void launch_cocg_reset(const CocgArgs<T>& a, int NC, cudaStream_t s) {
  k_cocg_reset<T><<<(a.m0 * NC + 255) / 256, 256, 0, s>>>(a, NC);
  RF_LAUNCH();
}

template <typename T, int NC>
static void dispatch_dots(const CocgArgs<T>& a, int buf, int num_sms, cudaStream_t s) {
  constexpr int SC = small_cpl_of<T>(NC), MC = maxcpl_of<T>(NC);
  // float column pairs: 3- and 4-chunk instances between the 2- and 6-chunk ones,
  // used when the shape asks for fewer CTAs per SM than its default (occ >= 2)
  if constexpr (NC == 2 && sizeof(T) == 4) {
    if (a.occ >= 2 && a.cpl > SC && a.cpl <= 4) {
      if (a.cpl == 3) dispatch_dots_mc<T, NC, 3>(a, buf, num_sms, s);
      else dispatch_dots_mc<T, NC, 4>(a, buf, num_sms, s);
      return;
    }
  }
  // double column pairs, one chunk per lane: fewest registers, most warps
  if constexpr (NC == 2 && sizeof(T) == 8) {
    if (a.cpl == 1) {
      dispatch_dots_mc<T, NC, 1>(a, buf, num_sms, s);
      return;
    }
  }
  if (SC < MC && a.cpl <= SC) dispatch_dots_mc<T, NC, SC>(a, buf, num_sms, s);
  else dispatch_dots_mc<T, NC, MC>(a, buf, num_sms, s);
}

template <typename T, int NC>
static void dispatch_update(const CocgArgs<T>& a, int buf, int num_sms, cudaStream_t s) {
  constexpr int SC = small_cpl_of<T>(NC), MC = maxcpl_of<T>(NC);
  if (SC < MC && a.cpl <= SC) dispatch_update_mc<T, NC, SC>(a, buf, num_sms, s);
  else dispatch_update_mc<T, NC, MC>(a, buf, num_sms, s);
}

template <typename T>
void launch_cocg_init(const CocgArgs<T>& a, int NC, int num_sms, cudaStream_t s) {
  launch_cocg_reset<T>(a, NC, s);
  const int64_t total = a.n * (int64_t)a.m0;
  int64_t blocks = (total + THREADS - 1) / THREADS;
  if (blocks > (int64_t)num_sms * 8) blocks = (int64_t)num_sms * 8;
  if (blocks < 1) blocks = 1;
  switch (NC) {
    case 1: k_cocg_init<T, 1><<<(int)blocks, THREADS, 0, s>>>(a); break;
    case 2: k_cocg_init<T, 2><<<(int)blocks, THREADS, 0, s>>>(a); break;
    case 4: k_cocg_init<T, 4><<<(int)blocks, THREADS, 0, s>>>(a); break;
    case 8: k_cocg_init<T, 8><<<(int)blocks, THREADS, 0, s>>>(a); break;
    default: throw Err{RAFEAST_ERR_INVALID_ARG};
  }
  RF_LAUNCH();
}

template <typename T>
void launch_cocg_dots(const CocgArgs<T>& a, int NC, int buf, int num_sms, cudaStream_t s) {
  switch (NC) {
    case 1: dispatch_dots<T, 1>(a, buf, num_sms, s); break;
    case 2: dispatch_dots<T, 2>(a, buf, num_sms, s); break;
    case 4: dispatch_dots<T, 4>(a, buf, num_sms, s); break;
    case 8: dispatch_dots<T, 8>(a, buf, num_sms, s); break;
    default: throw Err{RAFEAST_ERR_INVALID_ARG};
  }
}

template <typename T>
void launch_cocg_update(const CocgArgs<T>& a, int NC, int buf, int num_sms, cudaStream_t s) {
  switch (NC) {
    case 1: dispatch_update<T, 1>(a, buf, num_sms, s); break;
    case 2: dispatch_update<T, 2>(a, buf, num_sms, s); break;
    case 4: dispatch_update<T, 4>(a, buf, num_sms, s); break;
    case 8: dispatch_update<T, 8>(a, buf, num_sms, s); break;
    default: throw Err{RAFEAST_ERR_INVALID_ARG};
  }
}

template <typename T, int NC>
static void dispatch_shifted(int64_t n, const int32_t* rp, const int32_t* ci, const T* val, int m,
                             int ldc, const void* zs, const T* P, T* W, int G, int cpl,
                             int num_sms, cudaStream_t s) {
  constexpr int MC = maxcpl_of<T>(NC);
  if (cpl > MC) throw Err{RAFEAST_ERR_INVALID_ARG};
  auto kern = k_shifted_spmm<T, NC, MC>;
  const int colblocks = (m + G * cpl - 1) / (G * cpl);
  const int64_t groups = (n + (int64_t)WARPS * (32 / G) - 1) / ((int64_t)WARPS * (32 / G));
  dim3 grid(grid_x(kern, 0, num_sms, groups), colblocks);
  kern<<<grid, THREADS, 0, s>>>(n, rp, ci, val, m, ldc, zs, P, W, G, cpl);
  RF_LAUNCH();
}

template <typename T>
void launch_shifted_spmm(int64_t n, const int32_t* rp, const int32_t* ci, const T* val, int m,
                         int ldc, int NC, const void* zs, const T* P, T* W, int lanes, int cpl,
                         int num_sms, cudaStream_t s) {
  switch (NC) {
    case 1: dispatch_shifted<T, 1>(n, rp, ci, val, m, ldc, zs, P, W, lanes, cpl, num_sms, s); break;
    case 2: dispatch_shifted<T, 2>(n, rp, ci, val, m, ldc, zs, P, W, lanes, cpl, num_sms, s); break;
    case 4: dispatch_shifted<T, 4>(n, rp, ci, val, m, ldc, zs, P, W, lanes, cpl, num_sms, s); break;
    case 8: dispatch_shifted<T, 8>(n, rp, ci, val, m, ldc, zs, P, W, lanes, cpl, num_sms, s); break;
    default: throw Err{RAFEAST_ERR_INVALID_ARG};
  }
}

template <typename T>
void launch_spmm_real(int64_t n, const int32_t* rp, const int32_t* ci, const T* val, int k,
                      int ld, double sL, double sI, const T* X, T* Y, int num_sms,
                      cudaStream_t s) {
  constexpr int MC = maxcpl_of<T>(1);
  const int mc = (k + 1) / 2;
  int G, cpl, blocks;
  choose_shape(mc, 1, sizeof(T) == 8, 0, G, cpl, blocks, 0);
  auto kern = k_spmm_real<T, MC>;
  const int64_t groups = (n + (int64_t)WARPS * (32 / G) - 1) / ((int64_t)WARPS * (32 / G));
  dim3 grid(grid_x(kern, 0, num_sms, groups), blocks);
  kern<<<grid, THREADS, 0, s>>>(n, rp, ci, val, mc, ld, (T)sL, (T)sI, X, Y, G, cpl);
  RF_LAUNCH();
}

// explicit instantiations
template void launch_cocg_init<float>(const CocgArgs<float>&, int, int, cudaStream_t);
template void launch_cocg_reset<float>(const CocgArgs<float>&, int, cudaStream_t);
template void launch_cocg_reset<double>(const CocgArgs<double>&, int, cudaStream_t);
template void launch_cocg_init<double>(const CocgArgs<double>&, int, int, cudaStream_t);
template void launch_cocg_dots<float>(const CocgArgs<float>&, int, int, int, cudaStream_t);
template void launch_cocg_dots<double>(const CocgArgs<double>&, int, int, int, cudaStream_t);
template void launch_cocg_update<float>(const CocgArgs<float>&, int, int, int, cudaStream_t);
template void launch_cocg_update<double>(const CocgArgs<double>&, int, int, int, cudaStream_t);
template void launch_shifted_spmm<float>(int64_t, const int32_t*, const int32_t*, const float*, int,
                                         int, int, const void*, const float*, float*, int, int,
                                         int, cudaStream_t);
template void launch_shifted_spmm<double>(int64_t, const int32_t*, const int32_t*, const double*,
                                          int, int, int, const void*, const double*, double*, int,
                                          int, int, cudaStream_t);
template void launch_spmm_real<float>(int64_t, const int32_t*, const int32_t*, const float*, int,
                                      int, double, double, const float*, float*, int,
                                      cudaStream_t);
template void launch_spmm_real<double>(int64_t, const int32_t*, const int32_t*, const double*, int,
                                       int, double, double, const double*, double*, int,
                                       cudaStream_t);

}  // namespace rafeast
