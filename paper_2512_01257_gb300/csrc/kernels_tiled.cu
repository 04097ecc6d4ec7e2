// Tiled seed dot kernel of the multi-shift COCG (float32 state).
//
// The dominant sparse product of the shifted solves (Algorithm 2 Step 2a:
// w = M r_k with M = (z_s - sigma) I - L on the seed shift s, every column of
// the subspace at once) and the three per-column sums of the COCG step
// (gamma = r^T r, delta = r^T w, nu = ||r||^2), with the rows cut into tiles
// (tiling.cpp). A work item is (tile, column block): its CTA copies the rows
// of the tile's union (every row any of its nonzeros names, and its own rows)
// restricted to the block's cb column pairs into shared memory with
// asynchronous 16-byte copies (cp.async), then every row of the tile gathers
// its neighbours from shared memory. The copies of a tile are independent of
// one another and hold no registers, so many of them are in flight at once;
// the gathers that follow are shared-memory reads.
//
// Work split: CTA b of a grid of G CTAs (G a multiple of the number of column
// blocks ncb) takes the items b, b + G, b + 2G, ..., all of column block
// b mod ncb, in increasing tile order. Several CTAs share an SM, so one CTA's
// copies are in flight while another computes. Lane j of a row slot owns column pair
// cbk * cb + j (one 16-byte chunk: two complex values); the TT / cb row slots
// of the CTA take the tile's rows in turn.
//
// Sums: each lane keeps float partial sums over all of its rows (the FP64 pipe
// of this part runs at 1/64 of the float rate, so nothing per row is FP64);
// the CTA then adds its lanes' partials in a fixed order, in FP64, into its
// own slot of `part`. The last CTA of each column block adds the slots of its
// block in a fixed order (lanes over CTAs, then a fixed shuffle tree) and runs
// the FP64 scalar step of the block's columns (on this part FP64 issues at
// 1/64 of the float rate, so the column blocks share that work); the last
// column block to finish ends the step. No atomic addition takes part in a
// floating-point sum, so a step's sums do not depend on the order in which
// CTAs run, and two runs of a solve with the same shapes give the same
// iterates.
//
// The gathered sums are accumulated entry by entry in CSR order, exactly as
// the register-gather kernel (cocg_kernels.cuh) does, so w is the same to the
// last bit in both.
#include <algorithm>
#include <cstddef>

#include "cocg_kernels.cuh"

namespace rafeast {

// threads per CTA and the CTAs per SM the kernel is compiled for
#ifndef RF_TILED_TT
#define RF_TILED_TT 256
#endif
constexpr int TT = RF_TILED_TT;
constexpr int TT_MINB = TT == 256 ? 3 : 6;

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// a 16-byte chunk as two packed float pairs; add.rn.f32x2 / fma.rn.f32x2
// (sm_100 and later) round each lane exactly as two scalar operations would
using u64 = unsigned long long;
struct __align__(16) P4 {
  u64 lo, hi;
};
__device__ __forceinline__ u64 add2(u64 a, u64 b) {
  u64 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c) {
  u64 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ P4 p4add(P4 a, P4 b) { return P4{add2(a.lo, b.lo), add2(a.hi, b.hi)}; }
__device__ __forceinline__ P4 p4fma(u64 s2, P4 b, P4 a) {
  return P4{fma2(s2, b.lo, a.lo), fma2(s2, b.hi, a.hi)};
}
__device__ __forceinline__ u64 splat2(float v) {
  const unsigned u = __float_as_uint(v);
  return ((u64)u << 32) | u;
}
__device__ __forceinline__ float2 lo2(u64 v) {
  return make_float2(__uint_as_float((unsigned)v), __uint_as_float((unsigned)(v >> 32)));
}

// per-lane float sums of one complex column: gamma (re, im), delta (re, im), nu
__device__ __forceinline__ void dots_add(float2 r, float2 w, float* d) {
  d[0] = fmaf(r.x, r.x, fmaf(-r.y, r.y, d[0]));
  d[1] = fmaf(2.0f * r.x, r.y, d[1]);
  d[2] = fmaf(r.x, w.x, fmaf(-r.y, w.y, d[2]));
  d[3] = fmaf(r.x, w.y, fmaf(r.y, w.x, d[3]));
  d[4] = fmaf(r.x, r.x, fmaf(r.y, r.y, d[4]));
}

// the staged index data of one tile (shared memory, one of two buffers)
// (slx first: the 16-byte copies into it need a 16-byte aligned start)
struct __align__(16) TileIdx {
  uint16_t slx[TILE_NNZCAP + 16]; // union positions of the nonzeros, from kbase
  int sidx[TILE_UCAP];            // union rows
  int srp[TILE_TMAX + 1];         // row pointers of the tile's rows
  int r0, nr, nu, us, kbase;
};
static_assert(offsetof(TileIdx, slx) == 0 && sizeof(TileIdx) % 16 == 0,
              "16-byte copies into TileIdx::slx of both buffers must be aligned");
static_assert(sizeof(P4) == 16 && alignof(P4) == 16, "a staged chunk is one aligned 16 bytes");
static_assert((TILE_NNZCAP + 16) % 8 == 0, "slx holds whole 16-byte pieces");

// the copies of one tile (after its indices are in `b` and a barrier): its
// local indices in 16-byte pieces from an aligned start (the array is padded,
// so the last piece stays inside it) and the union's chunks of this column
// block (active pairs only)
template <int CB>
__device__ __forceinline__ void tile_copies(const TileArgs& tl, TileIdx& b, P4* xs,
                                            const float* R, int64_t ldt, int cbk, const int* sact) {
  const int kbase = b.kbase;
  const int npiece = (b.srp[b.nr] - kbase + 7) >> 3;
  for (int c = threadIdx.x; c < npiece; c += TT) cp_async16(b.slx + 8 * c, tl.lidx + kbase + 8 * c);
  for (int idx = threadIdx.x; idx < b.nu * CB; idx += TT) {
    const int jj = idx % CB;
    if (sact[jj])
      cp_async16(xs + idx, R + (int64_t)b.sidx[idx / CB] * ldt + (int64_t)(cbk * CB + jj) * 4);
  }
}

// the shifted systems' coefficients of one column (deferred form), staged
struct DefCoef {
  float2 zeta, beta, ca;
};

template <int CB, bool VF>
__global__ void __launch_bounds__(TT, TT_MINB) k_ms_dots_tiled(CocgArgs<float> a, TileArgs tl,
                                                               int buf) {
  if (__ldcg(&a.ctl->done)) return;
  // [max_union * CB] staged chunks (reused for the sums), one zero row of
  // CB chunks (the gathers' padding entries read it), then, for the
  // deferred form, the block's shifted coefficients [CB][2][ns]
  extern __shared__ __align__(16) P4 xs[];
  __shared__ TileIdx tb;
  __shared__ int sact[CB];
  constexpr int NRS = TT / CB;  // row slots
  const int ncb = tl.ncb;
  const int cbk = blockIdx.x % ncb;
  const int j = threadIdx.x % CB, rs = threadIdx.x / CB;
  const int q = cbk * CB + j;  // this lane's column pair
  if (threadIdx.x < CB) {
    const int qq = cbk * CB + threadIdx.x;
    sact[threadIdx.x] = qq < a.m0 ? __ldcg(a.colact + qq) : 0;
  }
  __syncthreads();
  const bool on = sact[j] != 0;
  int any = 0;
#pragma unroll
  for (int t = 0; t < CB; ++t) any |= sact[t];
  const int64_t ldt = (int64_t)a.ldc * 2;  // floats per state row
  const float* __restrict__ R = a.r[buf];   // r_k
  const int32_t* __restrict__ rowptr = VF ? a.lrowptr : a.rowptr;
  const float2 z = reinterpret_cast<const float2*>(a.zs)[0];
  float d[10];
#pragma unroll
  for (int t = 0; t < 10; ++t) d[t] = 0.0f;
  // deferred form: the previous step's shifted directions and their
  // quadrature terms are applied here, from r_{k-1} (the other residual
  // buffer) and the coefficients of the previous scalar step (this block's
  // columns are rewritten only by this block's last CTA, after every CTA of
  // the block is done)
  const bool pend = a.defer && __ldcg(&a.ctl->pend) != 0;
  const int ns = a.ns;
  // the zero row, written once (no copy reaches it)
  const int zrow = tl.max_union;
  if (threadIdx.x < CB) xs[zrow * CB + threadIdx.x] = P4{0ull, 0ull};
  DefCoef* sdc = reinterpret_cast<DefCoef*>(xs + (tl.max_union + 1) * CB);
  if (pend) {
    for (int e = threadIdx.x; e < CB * 2 * ns; e += TT) {
      const int jj = e / (2 * ns), h = (e / ns) & 1, t = e % ns;
      const int qq = cbk * CB + jj;
      DefCoef c;
      c.zeta = make_float2(0.f, 0.f);
      c.beta = make_float2(1.f, 0.f);
      c.ca = make_float2(0.f, 0.f);
      if (qq < a.m0) {
        const ShiftCoef<float> sc = a.scf[(2 * qq + h) * ns + t];
        if (sc.act != 0.f) {
          c.zeta = sc.zeta;
          c.beta = sc.beta;
          c.ca = sc.ca;
        }
      }
      sdc[e] = c;
    }
    __syncthreads();
  }
  const float* __restrict__ Rprev = a.r[buf ^ 1];  // r_{k-1}
  const int nitems = tl.ntiles * ncb;
  // the index data of the next item is loaded into registers while this
  // item's rows gather (this thread's share: union rows u = tid + TT c, row
  // pointers r = tid + TT c), and stored into tb once the gathers are done
  constexpr int UPT = (TILE_UCAP + TT - 1) / TT, RPT = (TILE_TMAX + 1 + TT - 1) / TT;
  int f_r0 = 0, f_nr = 0, f_nu = 0, f_us = 0;
  int f_sidx[UPT], f_srp[RPT];
  auto fetch = [&](int it) {
    const int t = it / ncb;
    f_r0 = __ldg(tl.trow + t);
    f_nr = __ldg(tl.trow + t + 1) - f_r0;
    const int u0 = __ldg(tl.uoff + t);
    f_nu = __ldg(tl.uoff + t + 1) - u0;
    f_us = __ldg(tl.uself + t);
#pragma unroll
    for (int c = 0; c < UPT; ++c) {
      const int u = threadIdx.x + TT * c;
      f_sidx[c] = u < f_nu ? __ldg(tl.ucol + u0 + u) : 0;
    }
#pragma unroll
    for (int c = 0; c < RPT; ++c) {
      const int r = threadIdx.x + TT * c;
      f_srp[c] = r <= f_nr ? __ldg(rowptr + f_r0 + r) : 0;
    }
  };
  if (any && (int)blockIdx.x < nitems) fetch(blockIdx.x);
  for (int item = blockIdx.x; any && item < nitems; item += gridDim.x) {
    // the tile's indices (fetched during the last item's gathers), then the
    // copies, which no longer wait on a global load each
    const int r0 = f_r0, nr = f_nr, nu = f_nu;
#pragma unroll
    for (int c = 0; c < UPT; ++c) {
      const int u = threadIdx.x + TT * c;
      if (u < nu) tb.sidx[u] = f_sidx[c];
    }
#pragma unroll
    for (int c = 0; c < RPT; ++c) {
      const int r = threadIdx.x + TT * c;
      if (r <= nr) tb.srp[r] = f_srp[c];
    }
    if (threadIdx.x == 0) {
      tb.r0 = r0;
      tb.nr = nr;
      tb.nu = nu;
      tb.us = f_us;
      tb.kbase = f_srp[0] & ~7;
    }
    __syncthreads();
    tile_copies<CB>(tl, tb, xs, R, ldt, cbk, sact);
    cp_async_wait_all();
    __syncthreads();
    if (item + (int)gridDim.x < nitems) fetch(item + gridDim.x);
    const uint16_t* slx = tb.slx;
    const int kbase = tb.kbase, us = tb.us;
    if (on) {
      for (int lr = rs; lr < nr; lr += NRS) {
        const int64_t row = r0 + lr;
        const int k0 = tb.srp[lr] - kbase, k1 = tb.srp[lr + 1] - kbase;
        // eight entries at a time, all their loads in flight together; the
        // entries past the row's end read the zero row and add +0 (the sum
        // starts at +0 and is never -0, so this leaves it unchanged: the
        // same sum, entry by entry in CSR order, as without padding)
        P4 acc = {0ull, 0ull};
        for (int k = k0; k < k1; k += 8) {
          int id[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) id[e] = k + e < k1 ? (int)slx[k + e] : zrow;
          P4 x[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) x[e] = xs[id[e] * CB + j];
          if constexpr (VF) {
#pragma unroll
            for (int e = 0; e < 8; ++e) acc = p4add(acc, x[e]);
          } else {
            const float* v = a.val + kbase + k;
            float vv[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) vv[e] = k + e < k1 ? __ldg(v + e) : 0.0f;
#pragma unroll
            for (int e = 0; e < 8; ++e) acc = p4fma(splat2(vv[e]), x[e], acc);
          }
        }
        const P4 rv = xs[(us + lr) * CB + j];
        const float2 r2[2] = {lo2(rv.lo), lo2(rv.hi)};
        const float2 l2v[2] = {lo2(acc.lo), lo2(acc.hi)};
        float2 w2[2];
        const float deg = (float)(k1 - k0);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          // values-free: L r = deg r - (sum over neighbours)
          const float2 lr2 =
              VF ? make_float2(deg * r2[h].x - l2v[h].x, deg * r2[h].y - l2v[h].y) : l2v[h];
          w2[h] = csub<float>(cmul<float>(z, r2[h]), lr2);
          dots_add(r2[h], w2[h], d + 5 * h);
        }
        if (a.wbuf)
          *reinterpret_cast<float4*>(a.wbuf + row * ldt + (int64_t)q * 4) =
              make_float4(w2[0].x, w2[0].y, w2[1].x, w2[1].y);
        // deferred form: this row's shifted directions and quadrature terms
        // of the previous step (streamed; its loads interleave with the
        // next row's shared-memory gathers)
        if (pend) {
          const DefCoef* dc = sdc + j * 2 * ns;
          const float4 rp4 = __ldcg(reinterpret_cast<const float4*>(Rprev + row * ldt) + q);
          const float2 rp[2] = {make_float2(rp4.x, rp4.y), make_float2(rp4.z, rp4.w)};
          float dsum[2] = {0.f, 0.f};
          for (int t = 0; t < ns; ++t) {
            const DefCoef c0 = dc[t], c1 = dc[ns + t];
            if (c0.ca.x == 0.f && c0.ca.y == 0.f && c0.zeta.x == 0.f && c0.zeta.y == 0.f &&
                c1.ca.x == 0.f && c1.ca.y == 0.f && c1.zeta.x == 0.f && c1.zeta.y == 0.f)
              continue;  // both systems of the pair stopped: p_j stays as it is
            float* pp = a.ps + (row * a.ldps + 2 * ((int64_t)q * ns + t)) * 2;
            const float4 p4 = __ldcg(reinterpret_cast<const float4*>(pp));
            float2 pj[2] = {make_float2(p4.x, p4.y), make_float2(p4.z, p4.w)};
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const DefCoef& c = h ? c1 : c0;
              // p_j^k = zeta_k r_k + beta_j p_j^{k-1};  D += Re(c_j alpha_j p_j^k)
              pj[h] = cfma<float>(c.beta, pj[h], cmul<float>(c.zeta, rp[h]));
              dsum[h] = fmaf(c.ca.x, pj[h].x, fmaf(-c.ca.y, pj[h].y, dsum[h]));
            }
            *reinterpret_cast<float4*>(pp) = make_float4(pj[0].x, pj[0].y, pj[1].x, pj[1].y);
          }
          float2* dp = reinterpret_cast<float2*>(a.dacc + row * a.ldd + 2 * q);
          float2 dv = *dp;
          dv.x += dsum[0];
          dv.y += dsum[1];
          *dp = dv;
        }
      }
    }
    __syncthreads();  // the next item's copies overwrite the staged data
  }
  // CTA sums in a fixed order: row slots of each lane position j in turn
  double* sred = reinterpret_cast<double*>(xs);  // [NRS][CB][10]
#pragma unroll
  for (int t = 0; t < 10; ++t) sred[(rs * CB + j) * 10 + t] = (double)d[t];
  __syncthreads();
  if (threadIdx.x < CB * 10) {
    const int jj = threadIdx.x / 10, t = threadIdx.x % 10;
    double s = 0.0;
    for (int r = 0; r < NRS; ++r) s += sred[(r * CB + jj) * 10 + t];
    tl.part[((int64_t)blockIdx.x * CB + jj) * 10 + t] = s;
    // (only the writers of part fence before the ticket: the other threads'
    // stores of w need not be waited for here)
    __threadfence();
  }
  __syncthreads();
  // the last CTA of this column block adds the block's CTA sums and runs
  // the scalar step of the block's columns; the last column block to finish
  // ends the step
  const int per_block = (int)gridDim.x / ncb;
  __shared__ int s_last;
  if (threadIdx.x == 0) s_last = atomicAdd(&a.ctl->cbticket[cbk], 1u) == (unsigned)per_block - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // the block's sums, per column: gamma (re, im), delta (re, im), nu, and the
  // seed records of the scalar step, in the (now free) staging area
  double* s_acc = reinterpret_cast<double*>(xs);
  MsSeed* s_seed = reinterpret_cast<MsSeed*>(s_acc + 2 * CB * 5);
  {
    // value v = (pair jj, sum t): lane l adds the CTAs l, l + 32, ... of the
    // block in that order, then the warp adds its lanes by a fixed tree. A
    // warp takes the values warp, warp + TT/32, ...; the loads of all of them
    // are issued before any is added.
    constexpr int NW = TT / 32, VPW = (CB * 10 + NW - 1) / NW;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double sv[VPW];
#pragma unroll
    for (int u = 0; u < VPW; ++u) sv[u] = 0.0;
    for (int b0 = 0; b0 < per_block; b0 += 32) {
      const int b = b0 + lane;
      double pv[VPW];
#pragma unroll
      for (int u = 0; u < VPW; ++u) {
        const int v = warp + NW * u;
        pv[u] = (v < CB * 10 && b < per_block)
                    ? __ldcg(tl.part + ((int64_t)(cbk + b * ncb) * CB + v / 10) * 10 + v % 10)
                    : 0.0;
      }
      if (b < per_block) {
#pragma unroll
        for (int u = 0; u < VPW; ++u) sv[u] += pv[u];
      }
    }
#pragma unroll
    for (int u = 0; u < VPW; ++u) {
      const int v = warp + NW * u;
      double x = sv[u];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (lane == 0 && v < CB * 10) s_acc[5 * (2 * (v / 10) + (v % 10) / 5) + (v % 10) % 5] = x;
    }
  }
  __shared__ MsCount cnt;
  if (threadIdx.x == 0) ms_count_init(cnt);
  __syncthreads();
  const int k = __ldcg(&a.ctl->iter);
  const int p0 = cbk * CB, p1 = min(a.m0, p0 + CB);
  double worst = 0.0;
  ms_scalar_cols_wide<float>(a, k, 2 * p0, 2 * p1, s_acc, s_seed, cnt, &worst);
  __syncthreads();
  ms_colact<float>(a, p0, p1, cnt);
  __syncthreads();
  if (a.hist) {
    const double w = block_max(worst);
    if (threadIdx.x == 0) cnt.worst = w;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  CocgCtl* c = a.ctl;
  atomicAdd(&c->g_active, cnt.active);
  atomicAdd(&c->g_brk, cnt.brk);
  atomicAdd(&c->g_cap, cnt.cap);
  atomicMax(&c->g_mx, cnt.mx);
  atomicMin(&c->g_mn, cnt.mn);
  atomicAdd(&c->g_cols, cnt.cols);
  atomicMax(&c->g_worst, (u64)__double_as_longlong(cnt.worst));
  c->cbticket[cbk] = 0;
  __threadfence();
  if (atomicAdd(&c->ticket2, 1u) != (unsigned)ncb - 1) return;
  __threadfence();
  MsCount tot;
  tot.active = __ldcg(&c->g_active);
  tot.brk = __ldcg(&c->g_brk);
  tot.cap = __ldcg(&c->g_cap);
  tot.mx = __ldcg(&c->g_mx);
  tot.mn = __ldcg(&c->g_mn);
  tot.cols = __ldcg(&c->g_cols);
  tot.worst = __longlong_as_double((long long)__ldcg(&c->g_worst));
  c->g_active = c->g_brk = c->g_cap = c->g_mx = c->g_cols = 0;
  c->g_mn = 0x7fffffff;
  c->g_worst = 0ull;
  c->ticket2 = 0;
  ms_scalar_finish<float>(a, k, tot);
}

template <int CB, bool VF>
static void launch_cb(const CocgArgs<float>& a, const TileArgs& tl, int buf, int num_sms,
                      int occ_cap, cudaStream_t s) {
  auto kern = k_ms_dots_tiled<CB, VF>;
  const size_t stage = (size_t)(tl.max_union + 1) * CB * sizeof(float4);
  const size_t red = std::max((size_t)TT * 10 * sizeof(double),
                              2 * CB * 5 * sizeof(double) + 2 * CB * sizeof(MsSeed));
  const size_t coef = a.defer ? (size_t)CB * 2 * a.ns * sizeof(DefCoef) : 0;
  const size_t smem = (stage > red ? stage : red) + coef;
  ensure_dyn_smem(reinterpret_cast<const void*>(kern), smem);
  int occ = 0;
  RF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, TT, smem));
  if (occ < 1) occ = 1;
  if (occ > TILE_MAX_OCC) occ = TILE_MAX_OCC;  // tl.part holds num_sms * TILE_MAX_OCC CTAs
  if (occ_cap > 0 && occ > occ_cap) occ = occ_cap;
  int g = (num_sms * occ / tl.ncb) * tl.ncb;
  if (g < tl.ncb) g = tl.ncb;
  kern<<<g, TT, smem, s>>>(a, tl, buf);
  RF_LAUNCH();
}

void launch_ms_dots_tiled(const CocgArgs<float>& a, const TileArgs& tl, int buf, int num_sms,
                          int occ_cap, cudaStream_t s) {
  const bool vf = a.lcolidx != nullptr;
  RF_CHECK(a.ms == 1 && (!a.defer || a.r[0] != a.r[1]), RAFEAST_ERR_INVALID_ARG);
  switch (tl.cb) {
    case 4: vf ? launch_cb<4, true>(a, tl, buf, num_sms, occ_cap, s)
               : launch_cb<4, false>(a, tl, buf, num_sms, occ_cap, s); break;
    case 8: vf ? launch_cb<8, true>(a, tl, buf, num_sms, occ_cap, s)
               : launch_cb<8, false>(a, tl, buf, num_sms, occ_cap, s); break;
    default: throw Err{RAFEAST_ERR_INVALID_ARG};
  }
}

}  // namespace rafeast
