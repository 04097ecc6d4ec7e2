// Gather core and COCG kernel bodies shared by the single-problem kernels
// (kernels_sparse.cu) and the grouped kernels that run many problems in one
// launch (kernels_batched.cu). A kernel body takes its CTA coordinate as a
// Blk instead of reading blockIdx/gridDim, so a grouped launch can hand each
// problem a slice of its grid.
#pragma once

#include "cocg_common.cuh"
#include "common.cuh"
#include "internal.h"

namespace rafeast {

constexpr int WARPS = 8;
constexpr int THREADS = WARPS * 32;

template <typename T> constexpr int maxcpl_of(int NC);
template <> constexpr int maxcpl_of<float>(int NC) { return NC >= 12 ? 1 : 12 / NC; }
template <> constexpr int maxcpl_of<double>(int NC) { return NC >= 8 ? 1 : 8 / NC; }

// a narrower instantiation (fewer chunks per lane, fewer registers, more
// resident warps) used when the chosen shape needs no more chunks than it has
template <typename T> constexpr int small_cpl_of(int NC);
template <> constexpr int small_cpl_of<float>(int NC) { return NC >= 4 ? 1 : 4 / NC; }
// (double column pairs of the multi-shift seed: 2 chunks, which is all the
// FP64 shapes use, at 2 CTAs per SM instead of 4 chunks at 1)
template <> constexpr int small_cpl_of<double>(int NC) {
  return NC == 2 ? 2 : (NC >= 8 ? 1 : 8 / NC);
}


template <typename K>
static inline int grid_x(K kernel, size_t smem, int num_sms, int64_t rows_needed_groups) {
  int occ = 0;
  RF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, THREADS, smem));
  if (occ < 1) occ = 1;
  int64_t g = (int64_t)num_sms * occ;
  if (g > rows_needed_groups) g = rows_needed_groups;
  if (g < 1) g = 1;
  return (int)g;
}


// ---------------------------------------------------------------------------
// gather core. The G lanes of a group own one row: they load up to G CSR
// entries of the row at once (coalesced) and broadcast them with width-G
// shuffles, so the gathered loads of consecutive entries do not wait on each
// other's index loads; NB entries (2, or 4 in the narrow float dot kernels)
// are in flight per step.
// acc[c][j] += sum_k val_k * X[col_k][chunk c] for the lane's active chunks.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned group_mask(int G) {
  if (G == 32) return 0xffffffffu;
  const int grp = (threadIdx.x & 31) / G;
  return ((1u << G) - 1u) << (grp * G);
}

// NB entries of the row are gathered per step (their loads in flight
// together); the sums are accumulated entry by entry in CSR order for any NB,
// so NB changes the latency hiding, not the result. A missing entry at the end
// re-reads the first entry's row with weight zero.
template <typename T, int NC, int MAXCPL, int NB = 2>
__device__ __forceinline__ void gather_row(const int32_t* __restrict__ colidx,
                                           const T* __restrict__ val, int k0, int k1, int row,
                                           int lg, int G, unsigned gmask,
                                           const T* __restrict__ X, int64_t ldx_t,
                                           const int (&coff)[MAXCPL], unsigned mask,
                                           c2<T> (&acc)[MAXCPL][NC]) {
  using C = c2<T>;
  for (int kb = k0; kb < k1; kb += G) {
    const int kk = kb + lg;
    const int my_c = kk < k1 ? __ldg(colidx + kk) : row;
    const T my_v = kk < k1 ? __ldg(val + kk) : (T)0;
    const int cnt = min(G, k1 - kb);
    for (int e = 0; e < cnt; e += NB) {
      int ci[NB];
      T vi[NB];
#pragma unroll
      for (int u = 0; u < NB; ++u) {
        const bool ok = e + u < cnt;
        ci[u] = __shfl_sync(gmask, my_c, ok ? e + u : e, G);
        const T v = __shfl_sync(gmask, my_v, ok ? e + u : e, G);
        vi[u] = ok ? v : (T)0;
      }
      C xs[NB][MAXCPL][NC];
#pragma unroll
      for (int c = 0; c < MAXCPL; ++c)
        if (mask & (1u << c)) {
#pragma unroll
          for (int u = 0; u < NB; ++u)
            ld_chunk<NC>(X + (int64_t)ci[u] * ldx_t + coff[c], xs[u][c]);
        }
#pragma unroll
      for (int c = 0; c < MAXCPL; ++c)
        if (mask & (1u << c)) {
#pragma unroll
          for (int j = 0; j < NC; ++j)
#pragma unroll
            for (int u = 0; u < NB; ++u) acc[c][j] = crfma<T>(vi[u], xs[u][c][j], acc[c][j]);
        }
    }
  }
}

// values-free gather for a unit-weight Laplacian's off-diagonal pattern:
// acc[c][j] += sum_k X[col_k][chunk c] (weights all +1; the -1 sign and the
// degree term are applied by the caller). Entries are taken NB per step as in
// gather_row.
template <typename T, int NC, int MAXCPL, int NB = 2>
__device__ __forceinline__ void gather_row_vf(const int32_t* __restrict__ colidx, int k0, int k1,
                                              int row, int lg, int G, unsigned gmask,
                                              const T* __restrict__ X, int64_t ldx_t,
                                              const int (&coff)[MAXCPL], unsigned mask,
                                              c2<T> (&acc)[MAXCPL][NC]) {
  using C = c2<T>;
  for (int kb = k0; kb < k1; kb += G) {
    const int kk = kb + lg;
    const int my_c = kk < k1 ? __ldg(colidx + kk) : row;
    const int cnt = min(G, k1 - kb);
    for (int e = 0; e < cnt; e += NB) {
      int ci[NB];
      T vi[NB];
#pragma unroll
      for (int u = 0; u < NB; ++u) {
        const bool ok = e + u < cnt;
        ci[u] = __shfl_sync(gmask, my_c, ok ? e + u : e, G);
        vi[u] = ok ? (T)1 : (T)0;
      }
      C xs[NB][MAXCPL][NC];
#pragma unroll
      for (int c = 0; c < MAXCPL; ++c)
        if (mask & (1u << c)) {
#pragma unroll
          for (int u = 0; u < NB; ++u)
            ld_chunk<NC>(X + (int64_t)ci[u] * ldx_t + coff[c], xs[u][c]);
        }
#pragma unroll
      for (int c = 0; c < MAXCPL; ++c)
        if (mask & (1u << c)) {
#pragma unroll
          for (int j = 0; j < NC; ++j) {
            // the first entry of a step always exists (e < cnt)
            acc[c][j].x += xs[0][c][j].x;
            acc[c][j].y += xs[0][c][j].y;
#pragma unroll
            for (int u = 1; u < NB; ++u) acc[c][j] = crfma<T>(vi[u], xs[u][c][j], acc[c][j]);
          }
        }
    }
  }
}

// two arrays at once (update kernel): acc_r from R, acc_p from P
template <typename T, int NC, int MAXCPL>
__device__ __forceinline__ void gather_row2(const int32_t* __restrict__ colidx,
                                            const T* __restrict__ val, int k0, int k1, int row,
                                            int lg, int G, unsigned gmask,
                                            const T* __restrict__ R, const T* __restrict__ P,
                                            int64_t ldx_t, const int (&coff)[MAXCPL],
                                            unsigned mask, c2<T> (&ar)[MAXCPL][NC],
                                            c2<T> (&ap)[MAXCPL][NC]) {
  using C = c2<T>;
  for (int kb = k0; kb < k1; kb += G) {
    const int kk = kb + lg;
    const int my_c = kk < k1 ? __ldg(colidx + kk) : row;
    const T my_v = kk < k1 ? __ldg(val + kk) : (T)0;
    const int cnt = min(G, k1 - kb);
    for (int e = 0; e < cnt; ++e) {
      const int ca = __shfl_sync(gmask, my_c, e, G);
      const T va = __shfl_sync(gmask, my_v, e, G);
      C xr[MAXCPL][NC], xp[MAXCPL][NC];
#pragma unroll
      for (int c = 0; c < MAXCPL; ++c)
        if (mask & (1u << c)) {
          ld_chunk<NC>(R + (int64_t)ca * ldx_t + coff[c], xr[c]);
          ld_chunk<NC>(P + (int64_t)ca * ldx_t + coff[c], xp[c]);
        }
#pragma unroll
      for (int c = 0; c < MAXCPL; ++c)
        if (mask & (1u << c)) {
#pragma unroll
          for (int j = 0; j < NC; ++j) {
            ar[c][j] = crfma<T>(va, xr[c][j], ar[c][j]);
            ap[c][j] = crfma<T>(va, xp[c][j], ap[c][j]);
          }
        }
    }
  }
}

// CTA coordinate of a kernel body: (x, y) in a gx x gy grid. Plain kernels
// take the launch grid; a grouped kernel takes its problem's slice.
struct Blk {
  int x, y, gx, gy;
};
__device__ __forceinline__ Blk grid_blk() {
  Blk b;
  b.x = blockIdx.x;
  b.y = blockIdx.y;
  b.gx = gridDim.x;
  b.gy = gridDim.y;
  return b;
}

struct RowMap {
  int lg, G, cpl;
  int64_t gid, gstride;
};

__device__ __forceinline__ RowMap row_map(int G, int cpl, const Blk& b) {
  RowMap m;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gpw = 32 / G;
  m.G = G;
  m.cpl = cpl;
  m.lg = lane % G;
  m.gid = ((int64_t)b.x * WARPS + warp) * gpw + lane / G;
  m.gstride = (int64_t)b.gx * WARPS * gpw;
  return m;
}

// ---------------------------------------------------------------------------
// COCG dots body: w = M r gathered from r; per system gamma = r^T r,
// delta = r^T w, nu = ||r||^2 reduced into a.acc; the last CTA of the
// problem (ticket over blk.gx * blk.gy CTAs) runs the scalar step on *src.
// ---------------------------------------------------------------------------
template <typename T, int NC, int MAXCPL, bool VF = false>
__device__ __forceinline__ void cocg_dots_body(const CocgArgs<T>& a, const CocgArgs<T>* src, int buf,
    const Blk& blk) {
  using C = c2<T>;
  if (__ldcg(&a.ctl->done)) return;
  const RowMap mp = row_map(a.lanes, a.cpl, blk);
  const unsigned gmask = group_mask(mp.G);
  const int ibase = blk.y * mp.G * mp.cpl + mp.lg;
  const T* __restrict__ R = buf ? a.r[1] : a.r[0];
  const int64_t ldt = (int64_t)a.ldc * 2;
  const C* zs = reinterpret_cast<const C*>(a.zs);
  C zv[NC];
#pragma unroll
  for (int j = 0; j < NC; ++j) zv[j] = zs[j];
  int coff[MAXCPL];
  unsigned mask = 0;
#pragma unroll
  for (int c = 0; c < MAXCPL; ++c) {
    const int i = ibase + c * mp.G;
    coff[c] = i * NC * 2;
    if (c < mp.cpl && i < a.m0 && __ldcg(a.colact + i)) mask |= 1u << c;
  }
  // per-lane partial dots in working precision
  T dg_re[MAXCPL][NC], dg_im[MAXCPL][NC], dd_re[MAXCPL][NC], dd_im[MAXCPL][NC], dn[MAXCPL][NC];
#pragma unroll
  for (int c = 0; c < MAXCPL; ++c)
#pragma unroll
    for (int j = 0; j < NC; ++j) dg_re[c][j] = dg_im[c][j] = dd_re[c][j] = dd_im[c][j] = dn[c][j] = (T)0;

  // every lane of a group must run the row loop (its shuffles name the whole
  // group); lanes without a chunk take part but load nothing
  if (__any_sync(0xffffffffu, mask != 0)) {
    const int32_t* __restrict__ rowptr = VF ? a.lrowptr : a.rowptr;
    for (int64_t row = mp.gid; row < a.n; row += mp.gstride) {
      const int k0 = __ldg(rowptr + row), k1 = __ldg(rowptr + row + 1);
      C acc[MAXCPL][NC];
#pragma unroll
      for (int c = 0; c < MAXCPL; ++c)
#pragma unroll
        for (int j = 0; j < NC; ++j) acc[c][j] = mk<T>((T)0, (T)0);
      // float kernels with at most 2 chunks per lane have the registers to
      // keep 4 entries' loads in flight
      constexpr int NB = sizeof(T) == 4 ? (MAXCPL == 1 ? 8 : MAXCPL == 2 ? 4 : 2) : 2;
      if constexpr (VF)
        gather_row_vf<T, NC, MAXCPL, NB>(a.lcolidx, k0, k1, (int)row, mp.lg, mp.G, gmask, R,
                                         ldt, coff, mask, acc);
      else
        gather_row<T, NC, MAXCPL, NB>(a.colidx, a.val, k0, k1, (int)row, mp.lg, mp.G, gmask, R,
                                      ldt, coff, mask, acc);
      // values-free: L r = deg r - (sum over neighbours), deg = k1 - k0
      const T deg = (T)(k1 - k0);
#pragma unroll
      for (int c = 0; c < MAXCPL; ++c)
        if (mask & (1u << c)) {
          C rv[NC], wv[NC];
          ld_chunk<NC>(R + row * ldt + coff[c], rv);
#pragma unroll
          for (int j = 0; j < NC; ++j) {
            const C lr = VF ? mk<T>(deg * rv[j].x - acc[c][j].x, deg * rv[j].y - acc[c][j].y)
                            : acc[c][j];
            const C w = csub<T>(cmul<T>(zv[j], rv[j]), lr);
            wv[j] = w;
            // gamma += r r, delta += r w, nu += |r|^2
            dg_re[c][j] = fma(rv[j].x, rv[j].x, fma(-rv[j].y, rv[j].y, dg_re[c][j]));
            dg_im[c][j] = fma((T)2 * rv[j].x, rv[j].y, dg_im[c][j]);
            dd_re[c][j] = fma(rv[j].x, w.x, fma(-rv[j].y, w.y, dd_re[c][j]));
            dd_im[c][j] = fma(rv[j].x, w.y, fma(rv[j].y, w.x, dd_im[c][j]));
            dn[c][j] = fma(rv[j].x, rv[j].x, fma(rv[j].y, rv[j].y, dn[c][j]));
          }
          // streamed update: keep w = M r for the update kernel
          if (a.wbuf) st_chunk<NC>(a.wbuf + row * ldt + coff[c], wv);
        }
    }
  }
  // reduce: groups of a warp -> smem (double) -> global atomics
  extern __shared__ double sred[];  // [G * MAXCPL * NC * 5]
  const int nred = mp.G * MAXCPL * NC * 5;
  for (int t = threadIdx.x; t < nred; t += blockDim.x) sred[t] = 0.0;
  __syncthreads();
  // every lane of the warp takes part in every shuffle (lanes without work
  // hold zeros), so the full-mask shuffles are never divergent
#pragma unroll
  for (int c = 0; c < MAXCPL; ++c)
#pragma unroll
    for (int j = 0; j < NC; ++j) {
      double v[5] = {(double)dg_re[c][j], (double)dg_im[c][j], (double)dd_re[c][j],
                     (double)dd_im[c][j], (double)dn[c][j]};
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        double x = v[q];
        for (int o = mp.G; o < 32; o <<= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        v[q] = x;
      }
      if ((threadIdx.x & 31) < mp.G && (mask & (1u << c))) {
#pragma unroll
        for (int q = 0; q < 5; ++q) atomicAdd(&sred[((mp.lg * MAXCPL + c) * NC + j) * 5 + q], v[q]);
      }
    }
  __syncthreads();
  for (int t = threadIdx.x; t < nred; t += blockDim.x) {
    const int q = t % 5;
    const int j = (t / 5) % NC;
    const int c = (t / (5 * NC)) % MAXCPL;
    const int lg = t / (5 * NC * MAXCPL);
    const int i = blk.y * mp.G * mp.cpl + lg + c * mp.G;
    if (c < mp.cpl && i < a.m0 && sred[t] != 0.0) atomicAdd(&a.acc[5 * (i * NC + j) + q], sred[t]);
  }
  __threadfence();
  __syncthreads();
  __shared__ int s_last;
  if (threadIdx.x == 0) {
    const unsigned tot = (unsigned)blk.gx * blk.gy;
    s_last = (atomicAdd(&a.ctl->ticket, 1u) == tot - 1);
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    if (a.ms) ms_scalar_step<T>(*src);
    else cocg_scalar_step<T>(*src, NC);
  }
}

// ---------------------------------------------------------------------------
// multi-shift update body (layout: see k_ms_reset in kernels_sparse.cu)
// ---------------------------------------------------------------------------
template <typename T, int NS, int MAXCPL>
__device__ __forceinline__ void ms_update_body(const CocgArgs<T>& a, const CocgArgs<T>* src, int buf,
    const Blk& blk) {
  using C = c2<T>;
  if (__ldcg(&a.ctl->done)) return;
  const RowMap mp = row_map(a.lanes, a.cpl, blk);
  const unsigned gmask = group_mask(mp.G);
  const int qbase = blk.y * mp.G * mp.cpl + mp.lg;
  const T* __restrict__ R = buf ? a.r[1] : a.r[0];
  const T* __restrict__ P = buf ? a.p[1] : a.p[0];
  T* __restrict__ Rn = buf ? a.r[0] : a.r[1];
  T* __restrict__ Pn = buf ? a.p[0] : a.p[1];
  const int64_t ldt = (int64_t)a.ldc * 2;
  const C zsd = reinterpret_cast<const C*>(a.zs)[0];
  // stage the block's coefficients: seed (2 per pair), shifts (2*NS per pair)
  extern __shared__ unsigned char smem_raw[];
  Coef<T>* scf = reinterpret_cast<Coef<T>*>(smem_raw);
  const int q0 = blk.y * mp.G * mp.cpl;
  const int npair = min(mp.G * mp.cpl, a.m0 - q0);
  ShiftCoef<T>* ssc = reinterpret_cast<ShiftCoef<T>*>(smem_raw + sizeof(Coef<T>) * 2 * mp.G * mp.cpl);
  for (int t = threadIdx.x; t < 2 * npair; t += blockDim.x) scf[t] = a.cf[2 * q0 + t];
  if (NS > 0)
    for (int t = threadIdx.x; t < 2 * npair * NS; t += blockDim.x) ssc[t] = a.scf[2 * q0 * NS + t];
  __syncthreads();
  int coff[MAXCPL];
  unsigned mask = 0;
#pragma unroll
  for (int c = 0; c < MAXCPL; ++c) {
    const int q = qbase + c * mp.G;
    coff[c] = q * 2 * 2;
    if (c < mp.cpl && q < a.m0 && __ldcg(a.colact + q)) mask |= 1u << c;
  }
  if (!__any_sync(0xffffffffu, mask != 0)) return;  // warp-uniform
  for (int64_t row = mp.gid; row < a.n; row += mp.gstride) {
    const int k0 = __ldg(a.rowptr + row), k1 = __ldg(a.rowptr + row + 1);
    C ar[MAXCPL][2], ap[MAXCPL][2];
#pragma unroll
    for (int c = 0; c < MAXCPL; ++c)
#pragma unroll
      for (int h = 0; h < 2; ++h) ar[c][h] = ap[c][h] = mk<T>((T)0, (T)0);
    gather_row2<T, 2, MAXCPL>(a.colidx, a.val, k0, k1, (int)row, mp.lg, mp.G, gmask, R, P, ldt,
                              coff, mask, ar, ap);
#pragma unroll
    for (int c = 0; c < MAXCPL; ++c)
      if (mask & (1u << c)) {
        const int q = qbase + c * mp.G, ql = q - q0;
        C rv[2], pv[2], rn[2];
        ld_chunk<2>(R + row * ldt + coff[c], rv);
        ld_chunk<2>(P + row * ldt + coff[c], pv);
        T dsum[2] = {(T)0, (T)0};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const Coef<T> cf = scf[2 * ql + h];
          const C pn = cfma<T>(cf.beta, pv[h], mk<T>(cf.ar * rv[h].x, cf.ar * rv[h].y));
          const C lpn = cfma<T>(cf.beta, ap[c][h], mk<T>(cf.ar * ar[c][h].x, cf.ar * ar[c][h].y));
          const C sv = csub<T>(cmul<T>(zsd, pn), lpn);
          rn[h] = csub<T>(rv[h], cmul<T>(cf.alpha, sv));
          pv[h] = pn;
          dsum[h] = fma(cf.ca.x, pn.x, fma(-cf.ca.y, pn.y, dsum[h]));
        }
#pragma unroll
        for (int t = 0; t < NS; ++t) {
          const ShiftCoef<T> s0 = ssc[(2 * ql) * NS + t];
          const ShiftCoef<T> s1 = ssc[(2 * ql + 1) * NS + t];
          if (s0.act != (T)0 || s1.act != (T)0) {
            T* pp = a.ps + (row * a.ldps + 2 * ((int64_t)q * NS + t)) * 2;
            C pj[2];
            ldcg_chunk<2>(pp, pj);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const ShiftCoef<T>& sc = h ? s1 : s0;
              if (sc.act != (T)0) {
                // p_j^k = zeta_k r_k + beta_j p_j^{k-1}; x_j += alpha_j p_j^k
                pj[h] = cfma<T>(sc.beta, pj[h], cmul<T>(sc.zeta, rv[h]));
                dsum[h] = fma(sc.ca.x, pj[h].x, fma(-sc.ca.y, pj[h].y, dsum[h]));
              }
            }
            st_chunk<2>(pp, pj);
          }
        }
        st_chunk<2>(Rn + row * ldt + coff[c], rn);
        st_chunk<2>(Pn + row * ldt + coff[c], pv);
        T* dp = a.dacc + row * a.ldd + 2 * q;
        dp[0] += dsum[0];
        dp[1] += dsum[1];
      }
  }
}

// ---------------------------------------------------------------------------
// streamed multi-shift update: one thread per (row, column pair), no
// gathers. With w_k = M r_k stored by the dot kernel and s_{k-1} = M p_{k-1}
// kept from the previous step:
//   p_k = ar r_k + beta p_{k-1},  s_k = ar w_k + beta s_{k-1} (= M p_k),
//   r_{k+1} = r_k - alpha s_k,    D += Re(c alpha p_k),
// and the shifted directions p_j^k = zeta_k r_k + beta_j p_j^{k-1} as in the
// gathering update. A frozen column has ar = 0, beta = 1, alpha = 0: its
// state is left as it is. Every access is to the thread's own row.
// ---------------------------------------------------------------------------
template <typename T>
__host__ __device__ inline size_t ms_stream_smem(int pairs, int ns) {
  return (size_t)2 * pairs * (sizeof(Coef<T>) + ns * sizeof(ShiftCoef<T>)) +
         sizeof(int) * pairs + 16;
}

// the problem's coefficients and column activity into shared memory
// (NS < 0: the shift count a.ns is read at run time)
template <typename T, int NS>
__device__ __forceinline__ void ms_stream_stage(const CocgArgs<T>& a, unsigned char* smem) {
  const int P = a.m0;
  const int ns = NS < 0 ? a.ns : NS;
  Coef<T>* scf = reinterpret_cast<Coef<T>*>(smem);
  ShiftCoef<T>* ssc = reinterpret_cast<ShiftCoef<T>*>(smem + sizeof(Coef<T>) * 2 * P);
  int* sact = reinterpret_cast<int*>(smem + (sizeof(Coef<T>) + ns * sizeof(ShiftCoef<T>)) * 2 * P);
  for (int t = threadIdx.x; t < 2 * P; t += blockDim.x) scf[t] = a.cf[t];
  if (ns > 0)
    for (int t = threadIdx.x; t < 2 * P * ns; t += blockDim.x) ssc[t] = a.scf[t];
  for (int t = threadIdx.x; t < P; t += blockDim.x) sact[t] = __ldcg(a.colact + t);
  __syncthreads();
}

// elements of the range [lo, e1) of the n x pairs element grid: e0, e0 + step,
// ...; with `down`, taken from the top of the range (element lo + e1 - 1 - e).
// The dot kernel walks the rows upwards, so the w rows it wrote last are still
// in L2 when a top-down update starts on them, and the r rows the update
// writes last are the first ones the next dot kernel gathers. Elements are
// independent, so the order changes only the cache reuse.
template <typename T, int NS>
__device__ __forceinline__ void ms_stream_elems(const CocgArgs<T>& a, const unsigned char* smem,
                                                int64_t e0, int64_t e1, int64_t step,
                                                int64_t lo, bool down, int buf = 0) {
  using C = c2<T>;
  const int P = a.m0;
  const int ns = NS < 0 ? a.ns : NS;
  const Coef<T>* scf = reinterpret_cast<const Coef<T>*>(smem);
  const ShiftCoef<T>* ssc =
      reinterpret_cast<const ShiftCoef<T>*>(smem + sizeof(Coef<T>) * 2 * P);
  const int* sact = reinterpret_cast<const int*>(
      smem + (sizeof(Coef<T>) + ns * sizeof(ShiftCoef<T>)) * 2 * P);
  // r_k from r[buf], r_{k+1} into r[buf ^ 1] (the same array when r is
  // updated in place)
  const T* __restrict__ R = a.r[buf];
  T* __restrict__ Rn = a.r[buf ^ 1];
  T* __restrict__ Pd = a.p[0];
  const T* __restrict__ W = a.wbuf;
  T* __restrict__ S = a.sbuf;
  const int nsh = a.defer ? 0 : ns;  // deferred: the shifted directions wait
  for (int64_t e = e0; e < e1; e += step) {
    const int64_t ee = down ? lo + e1 - 1 - e : e;
    const int64_t row = ee / P;
    const int q = (int)(ee - row * P);
    if (!sact[q]) continue;
    const int64_t off = (row * a.ldc + 2 * q) * 2;
    C rv[2], pv[2], wv[2], sv[2], rn[2];
    ld_chunk<2>(R + off, rv);
    ld_chunk<2>(Pd + off, pv);
    ldcg_chunk<2>(W + off, wv);
    ld_chunk<2>(S + off, sv);
    T dsum[2] = {(T)0, (T)0};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const Coef<T> cf = scf[2 * q + h];
      const C pn = cfma<T>(cf.beta, pv[h], mk<T>(cf.ar * rv[h].x, cf.ar * rv[h].y));
      const C sn = cfma<T>(cf.beta, sv[h], mk<T>(cf.ar * wv[h].x, cf.ar * wv[h].y));
      rn[h] = csub<T>(rv[h], cmul<T>(cf.alpha, sn));
      pv[h] = pn;
      sv[h] = sn;
      dsum[h] = fma(cf.ca.x, pn.x, fma(-cf.ca.y, pn.y, dsum[h]));
    }
#pragma unroll
    for (int t = 0; t < (NS < 0 ? nsh : NS); ++t) {
      if (NS >= 0 && nsh == 0) break;  // deferred form
      const ShiftCoef<T> s0 = ssc[(2 * q) * ns + t];
      const ShiftCoef<T> s1 = ssc[(2 * q + 1) * ns + t];
      if (s0.act != (T)0 || s1.act != (T)0) {
        T* pp = a.ps + (row * a.ldps + 2 * ((int64_t)q * ns + t)) * 2;
        C pj[2];
        ldcg_chunk<2>(pp, pj);
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          const ShiftCoef<T>& sc = hh ? s1 : s0;
          if (sc.act != (T)0) {
            pj[hh] = cfma<T>(sc.beta, pj[hh], cmul<T>(sc.zeta, rv[hh]));
            dsum[hh] = fma(sc.ca.x, pj[hh].x, fma(-sc.ca.y, pj[hh].y, dsum[hh]));
          }
        }
        st_chunk<2>(pp, pj);
      }
    }
    st_chunk<2>(Rn + off, rn);
    st_chunk<2>(Pd + off, pv);
    st_chunk<2>(S + off, sv);
    T* dp = a.dacc + row * a.ldd + 2 * q;
    dp[0] += dsum[0];
    dp[1] += dsum[1];
  }
}

}  // namespace rafeast
