// Batched-COCG kernels with TMA bulk-copy row gathers (sm_103a, float32).
//
// Same arithmetic as the register-gather kernels of kernels_sparse.cu (the
// shifted systems of Algorithm 1 / Algorithm 2 Step 2a in the Chronopoulos-
// Gear ordering; see there), but every gathered row slice is fetched by the
// bulk-copy engine: `cp.async.bulk.shared::cluster.global.mbarrier::
// complete_tx::bytes` into a ring of shared-memory stages owned by one warp,
// completion tracked by an mbarrier per stage. In-flight bytes then cost no
// registers, so each SM keeps ~150-200 KB of gathers in flight.
//
// State layout (float32 complex, blocked for conflict-free shared reads):
// a row holds m0*NC complex values (K*m0 float4, K = NC/2) split into ncb
// column blocks of bw = ceil(m0/ncb) <= CBW = 32*CPL subspace columns (the
// last one only as wide as the columns left, Wb = min(bw, m0 - cb*bw)), so
// the warps of different blocks get even work. Block cb is K planes of Wb
// float4, float4 (row, cb, k, il) at
//   row*K*m0 + K*cb*bw + k*Wb + il,
// holding shifts (2k, 2k+1) of column i = cb*bw + il. One block of one row
// (a "slice", K*Wb*16 bytes) is what a gather copies.
//
// Work mapping: warp w owns column block cb = w % ncb and rows
// w/ncb, w/ncb + nw/ncb, ... (nw = total warps, a multiple of ncb). Lane l
// owns columns cb*CBW + l + 32c, c < CPL. A row's nonzeros are processed in
// items of at most maxnz entries; the warp's ring keeps S items in flight.
//
// Every mbarrier wait is bounded (about one second of clock64 cycles); on
// expiry the kernel records RAFEAST_ERR_TIMEOUT in the control block, ends
// the solve, waits (bounded) for its own copies in flight, and returns.
#include <cstdint>

#include "cocg_common.cuh"
#include "common.cuh"
#include "internal.h"

namespace rafeast {

namespace tma {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// after a timeout: fixed drain time (~10 ms) for copies still in flight
constexpr long long DRAIN_CYCLES = 20000000LL;

// wait for phase `parity` of `bar`; false on timeout. Lane 0 alone polls
// (with the bound) and broadcasts its verdict, so the whole warp takes the same
// branch; on success every lane then observes the completed phase itself
// (acquire), which succeeds at once.
__device__ __forceinline__ bool wait_bounded(uint64_t* bar, uint32_t parity, int lane,
                                             long long limit) {
  int ok = 1;
  if (lane == 0 && !mbar_try_wait(bar, parity)) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
      if (clock64() - t0 > limit) {
        ok = 0;
        break;
      }
    }
  }
  ok = __shfl_sync(0xffffffffu, ok, 0);
  if (ok && lane != 0) mbar_try_wait(bar, parity);
  return ok != 0;
}

// row cursor over (row, [kb, ke)) items
struct Cursor {
  int64_t row;
  int kb, ke, k1;
  bool valid;
};
__device__ __forceinline__ void cur_start(Cursor& c, int64_t row, int64_t n,
                                          const int32_t* __restrict__ rp, int maxnz) {
  c.row = row;
  c.valid = row < n;
  if (c.valid) {
    c.kb = __ldg(rp + row);
    c.k1 = __ldg(rp + row + 1);
    c.ke = min(c.kb + maxnz, c.k1);
  }
}
__device__ __forceinline__ void cur_next(Cursor& c, int64_t stride, int64_t n,
                                         const int32_t* __restrict__ rp, int maxnz) {
  if (c.ke < c.k1) {
    c.kb = c.ke;
    c.ke = min(c.kb + maxnz, c.k1);
  } else {
    cur_start(c, c.row + stride, n, rp, maxnz);
  }
}

// issue the copies of one item into a stage: lane 0 arrives with the byte
// count, then lanes e < nz each copy slice e of every array
template <int NARR>
__device__ __forceinline__ void issue_item(const Cursor& c, unsigned char* stage, uint64_t* bar,
                                          const int32_t* __restrict__ colidx,
                                          const float* const (&arr)[NARR], int64_t row_f4,
                                          int64_t blk_f4, uint32_t slot_bytes,
                                          uint32_t slice_bytes, int maxnz, int lane,
                                          int stall_bytes) {
  const int nz = c.ke - c.kb;
  // stall_bytes > 0 (test hook) makes the stage expect bytes that never come
  if (lane == 0) mbar_arrive_expect_tx(bar, (uint32_t)nz * NARR * slice_bytes + stall_bytes);
  __syncwarp();
  // the warp's earlier generic reads of this stage precede the new async writes
  fence_proxy_async();
  for (int e = lane; e < nz; e += 32) {
    const int64_t col = __ldg(colidx + c.kb + e);
#pragma unroll
    for (int t = 0; t < NARR; ++t)
      bulk_g2s(stage + ((size_t)t * maxnz + e) * slot_bytes,
               arr[t] + (col * row_f4 + blk_f4) * 4, slice_bytes, bar);
  }
}

}  // namespace tma

using namespace tma;

// ---------------------------------------------------------------------------
// init for the blocked layout: r0 = b, p = 0, D = 0
// ---------------------------------------------------------------------------
template <int NC, int CPL>
__global__ void __launch_bounds__(256) k_init_blocked(CocgArgs<float> a, int bw) {
  constexpr int K = NC / 2, CBW = 32 * CPL;
  const int64_t total = a.n * (int64_t)a.m0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = e / a.m0;
    const int i = (int)(e - row * a.m0);
    double b = a.qin[row * a.ldq + i];
    if (a.form == RAFEAST_FORM_CORRECTION) b = a.aqin[row * a.ldq + i] - a.theta[i] * b;
    const int cb = i / bw, il = i % bw;
    const int wb = min(bw, a.m0 - cb * bw);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int64_t f4 = row * K * a.m0 + (int64_t)K * cb * bw + k * wb + il;
      const float b0 = 2 * k < a.nc_real ? (float)b : 0.f;
      const float b1 = 2 * k + 1 < a.nc_real ? (float)b : 0.f;
      reinterpret_cast<float4*>(a.r[0])[f4] = make_float4(b0, 0.f, b1, 0.f);
      reinterpret_cast<float4*>(a.p[0])[f4] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    a.dacc[row * a.ldd + i] = 0.f;
  }
}

// ---------------------------------------------------------------------------
// dots kernel
// ---------------------------------------------------------------------------
template <int NC, int CPL>
__global__ void __launch_bounds__(256, 1) k_dots_tma(CocgArgs<float> a, int buf, int ncb,
                                                     int bw, int maxnz, int S) {
  constexpr int K = NC / 2, CBW = 32 * CPL;
  constexpr uint32_t SLOT = CBW * NC * 8;  // shared-memory slot of one slice
  if (__ldcg(&a.ctl->done)) return;
  extern __shared__ __align__(128) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
  const size_t stage_bytes = (size_t)maxnz * SLOT;
  unsigned char* ring = smem + (size_t)warp * S * stage_bytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)W * S * stage_bytes) + warp * S;
  const int64_t gw = (int64_t)blockIdx.x * W + warp, nw = (int64_t)gridDim.x * W;
  const int cb = (int)(gw % ncb);
  const int64_t rstart = gw / ncb, rstride = nw / ncb;
  const int wb = min(bw, a.m0 - cb * bw);  // this block's width (<= CBW)
  const uint32_t SLICE = (uint32_t)(K * wb * 16);
  const int64_t row_f4 = (int64_t)K * a.m0, blk_f4 = (int64_t)K * cb * bw;
  const float* R = a.r[buf];
  const float* arrs[1] = {R};
  const float2* zs = reinterpret_cast<const float2*>(a.zs);
  float2 zv[NC];
#pragma unroll
  for (int j = 0; j < NC; ++j) zv[j] = zs[j];
  unsigned mask = 0;
#pragma unroll
  for (int c = 0; c < CPL; ++c) {
    const int il = lane + 32 * c, i = cb * bw + il;
    if (il < wb && __ldcg(a.colact + i)) mask |= 1u << c;
  }
  float dg_re[CPL][NC], dg_im[CPL][NC], dd_re[CPL][NC], dd_im[CPL][NC], dn[CPL][NC];
#pragma unroll
  for (int c = 0; c < CPL; ++c)
#pragma unroll
    for (int j = 0; j < NC; ++j) dg_re[c][j] = dg_im[c][j] = dd_re[c][j] = dd_im[c][j] = dn[c][j] = 0.f;

  bool timed_out = false;
  if (__any_sync(0xffffffffu, mask != 0)) {
    if (lane == 0) {
      for (int s = 0; s < S; ++s) mbar_init(bars + s, 1);
      fence_mbar_init();
      fence_proxy_async();
    }
    __syncwarp();
    Cursor pc, cc;
    cur_start(pc, rstart, a.n, a.rowptr, maxnz);
    cur_start(cc, rstart, a.n, a.rowptr, maxnz);
    for (int s = 0; s < S && pc.valid; ++s) {
      issue_item<1>(pc, ring + s * stage_bytes, bars + s, a.colidx, arrs, row_f4, blk_f4, SLOT, SLICE,
                    maxnz, lane, a.stall_bytes);
      cur_next(pc, rstride, a.n, a.rowptr, maxnz);
    }
    uint32_t phase = 0;  // bit s: parity to wait for on stage s
    int s = 0;
    float4 acc[CPL][K], own[CPL][K];
    bool have_own = false;
#pragma unroll
    for (int c = 0; c < CPL; ++c)
#pragma unroll
      for (int k = 0; k < K; ++k) acc[c][k] = make_float4(0.f, 0.f, 0.f, 0.f);
    while (cc.valid) {
      if (!wait_bounded(bars + s, (phase >> s) & 1u, lane, a.wait_cycles)) {
        timed_out = true;
        break;
      }
      phase ^= 1u << s;
      const unsigned char* stage = ring + s * stage_bytes;
      const int nz = cc.ke - cc.kb;
      const int my_c = lane < nz ? __ldg(a.colidx + cc.kb + lane) : -1;
      const float my_v = lane < nz ? __ldg(a.val + cc.kb + lane) : 0.f;
      const unsigned diag = __ballot_sync(0xffffffffu, my_c == (int)cc.row);
      for (int e = 0; e < nz; ++e) {
        const float v = __shfl_sync(0xffffffffu, my_v, e);
        const float4* sl = reinterpret_cast<const float4*>(stage + (size_t)e * SLOT);
#pragma unroll
        for (int c = 0; c < CPL; ++c)
#pragma unroll
          for (int k = 0; k < K; ++k) {
            const float4 x = sl[k * wb + lane + 32 * c];
            acc[c][k].x = fmaf(v, x.x, acc[c][k].x);
            acc[c][k].y = fmaf(v, x.y, acc[c][k].y);
            acc[c][k].z = fmaf(v, x.z, acc[c][k].z);
            acc[c][k].w = fmaf(v, x.w, acc[c][k].w);
          }
      }
      if (diag) {
        const int ed = __ffs(diag) - 1;
        const float4* sl = reinterpret_cast<const float4*>(stage + (size_t)ed * SLOT);
#pragma unroll
        for (int c = 0; c < CPL; ++c)
#pragma unroll
          for (int k = 0; k < K; ++k) own[c][k] = sl[k * wb + lane + 32 * c];
        have_own = true;
      }
      __syncwarp();
      const bool row_done = cc.ke == cc.k1;
      const int64_t row = cc.row;
      if (pc.valid) {
        issue_item<1>(pc, ring + s * stage_bytes, bars + s, a.colidx, arrs, row_f4, blk_f4, SLOT, SLICE,
                      maxnz, lane, a.stall_bytes);
        cur_next(pc, rstride, a.n, a.rowptr, maxnz);
      }
      cur_next(cc, rstride, a.n, a.rowptr, maxnz);
      s = (s + 1 == S) ? 0 : s + 1;
      if (row_done) {
        if (!have_own) {
          const float4* g = reinterpret_cast<const float4*>(R) + row * row_f4 + blk_f4;
#pragma unroll
          for (int c = 0; c < CPL; ++c)
            if (lane + 32 * c < wb) {
#pragma unroll
              for (int k = 0; k < K; ++k) own[c][k] = g[k * wb + lane + 32 * c];
            }
        }
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
          if (mask & (1u << c)) {
#pragma unroll
            for (int k = 0; k < K; ++k) {
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                const int j = 2 * k + h;
                const float2 r = h ? make_float2(own[c][k].z, own[c][k].w)
                                   : make_float2(own[c][k].x, own[c][k].y);
                const float2 lr = h ? make_float2(acc[c][k].z, acc[c][k].w)
                                    : make_float2(acc[c][k].x, acc[c][k].y);
                const float2 w = csub<float>(cmul<float>(zv[j], r), lr);
                dg_re[c][j] = fmaf(r.x, r.x, fmaf(-r.y, r.y, dg_re[c][j]));
                dg_im[c][j] = fmaf(2.f * r.x, r.y, dg_im[c][j]);
                dd_re[c][j] = fmaf(r.x, w.x, fmaf(-r.y, w.y, dd_re[c][j]));
                dd_im[c][j] = fmaf(r.x, w.y, fmaf(r.y, w.x, dd_im[c][j]));
                dn[c][j] = fmaf(r.x, r.x, fmaf(r.y, r.y, dn[c][j]));
              }
            }
          }
#pragma unroll
          for (int k = 0; k < K; ++k) acc[c][k] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        have_own = false;
      }
    }
    if (timed_out) {
      if (lane == 0) {
        atomicExch(&a.ctl->timeout, 1);
        atomicExch(&a.ctl->done, 1);
      }
      // bounded wait for the copies still in flight in the other stages
      const long long t0 = clock64();
      while (clock64() - t0 < DRAIN_CYCLES) {
      }
    }
  }
  // block reduction: per (cb, lane, c, j, q) in shared memory, then global
  __syncthreads();
  double* sred = reinterpret_cast<double*>(smem);
  const int nred = ncb * 32 * CPL * NC * 5;
  for (int t = threadIdx.x; t < nred; t += blockDim.x) sred[t] = 0.0;
  __syncthreads();
  if (!timed_out) {
#pragma unroll
    for (int c = 0; c < CPL; ++c)
      if (mask & (1u << c)) {
#pragma unroll
        for (int j = 0; j < NC; ++j) {
          double* d = sred + ((((size_t)cb * 32 + lane) * CPL + c) * NC + j) * 5;
          atomicAdd(d + 0, (double)dg_re[c][j]);
          atomicAdd(d + 1, (double)dg_im[c][j]);
          atomicAdd(d + 2, (double)dd_re[c][j]);
          atomicAdd(d + 3, (double)dd_im[c][j]);
          atomicAdd(d + 4, (double)dn[c][j]);
        }
      }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nred; t += blockDim.x) {
    const int q = t % 5;
    const int j = (t / 5) % NC;
    const int c = (t / (5 * NC)) % CPL;
    const int ln = (t / (5 * NC * CPL)) % 32;
    const int cbb = t / (5 * NC * CPL * 32);
    const int il = ln + 32 * c, i = cbb * bw + il;
    if (il < min(bw, a.m0 - cbb * bw) && sred[t] != 0.0)
      atomicAdd(&a.acc[5 * (i * NC + j) + q], sred[t]);
  }
  __threadfence();
  __syncthreads();
  __shared__ int s_last;
  if (threadIdx.x == 0) s_last = (atomicAdd(&a.ctl->ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (s_last) {
    __threadfence();
    cocg_scalar_step<float>(a, NC);
  }
}

// ---------------------------------------------------------------------------
// update kernel
// ---------------------------------------------------------------------------
template <int NC, int CPL>
__global__ void __launch_bounds__(256, 1) k_update_tma(CocgArgs<float> a, int buf, int ncb,
                                                       int bw, int maxnz, int S) {
  constexpr int K = NC / 2, CBW = 32 * CPL;
  constexpr uint32_t SLOT = CBW * NC * 8;  // shared-memory slot of one slice
  if (__ldcg(&a.ctl->done)) return;
  extern __shared__ __align__(128) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
  const size_t stage_bytes = (size_t)maxnz * 2 * SLOT;
  unsigned char* ring = smem + (size_t)warp * S * stage_bytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)W * S * stage_bytes) + warp * S;
  const int64_t gw = (int64_t)blockIdx.x * W + warp, nw = (int64_t)gridDim.x * W;
  const int cb = (int)(gw % ncb);
  const int64_t rstart = gw / ncb, rstride = nw / ncb;
  const int wb = min(bw, a.m0 - cb * bw);  // this block's width (<= CBW)
  const uint32_t SLICE = (uint32_t)(K * wb * 16);
  const int64_t row_f4 = (int64_t)K * a.m0, blk_f4 = (int64_t)K * cb * bw;
  const float* R = a.r[buf];
  const float* P = a.p[buf];
  float4* Rn = reinterpret_cast<float4*>(a.r[buf ^ 1]);
  float4* Pn = reinterpret_cast<float4*>(a.p[buf ^ 1]);
  const float* arrs[2] = {R, P};
  const float2* zs = reinterpret_cast<const float2*>(a.zs);
  float2 zv[NC];
#pragma unroll
  for (int j = 0; j < NC; ++j) zv[j] = zs[j];
  unsigned mask = 0;
  Coef<float> cf[CPL][NC];
#pragma unroll
  for (int c = 0; c < CPL; ++c) {
    const int il = lane + 32 * c, i = cb * bw + il;
    if (il < wb && __ldcg(a.colact + i)) mask |= 1u << c;
#pragma unroll
    for (int j = 0; j < NC; ++j) {
      if (il < wb) {
        cf[c][j] = a.cf[i * NC + j];
      } else {
        cf[c][j].beta = make_float2(1.f, 0.f);
        cf[c][j].alpha = cf[c][j].ca = make_float2(0.f, 0.f);
        cf[c][j].ar = 0.f;
      }
    }
  }
  if (!__any_sync(0xffffffffu, mask != 0)) return;  // warp-uniform
  if (lane == 0) {
    for (int s = 0; s < S; ++s) mbar_init(bars + s, 1);
    fence_mbar_init();
    fence_proxy_async();
  }
  __syncwarp();
  Cursor pc, cc;
  cur_start(pc, rstart, a.n, a.rowptr, maxnz);
  cur_start(cc, rstart, a.n, a.rowptr, maxnz);
  for (int s = 0; s < S && pc.valid; ++s) {
    issue_item<2>(pc, ring + s * stage_bytes, bars + s, a.colidx, arrs, row_f4, blk_f4, SLOT, SLICE,
                  maxnz, lane, a.stall_bytes);
    cur_next(pc, rstride, a.n, a.rowptr, maxnz);
  }
  uint32_t phase = 0;
  int s = 0;
  float4 accr[CPL][K], accp[CPL][K], ownr[CPL][K], ownp[CPL][K];
  bool have_own = false;
#pragma unroll
  for (int c = 0; c < CPL; ++c)
#pragma unroll
    for (int k = 0; k < K; ++k) accr[c][k] = accp[c][k] = make_float4(0.f, 0.f, 0.f, 0.f);
  while (cc.valid) {
    if (!wait_bounded(bars + s, (phase >> s) & 1u, lane, a.wait_cycles)) {
      if (lane == 0) {
        atomicExch(&a.ctl->timeout, 1);
        atomicExch(&a.ctl->done, 1);
      }
      const long long t0 = clock64();
      while (clock64() - t0 < DRAIN_CYCLES) {
      }
      return;
    }
    phase ^= 1u << s;
    const unsigned char* stage = ring + s * stage_bytes;
    const int nz = cc.ke - cc.kb;
    const int my_c = lane < nz ? __ldg(a.colidx + cc.kb + lane) : -1;
    const float my_v = lane < nz ? __ldg(a.val + cc.kb + lane) : 0.f;
    const unsigned diag = __ballot_sync(0xffffffffu, my_c == (int)cc.row);
    for (int e = 0; e < nz; ++e) {
      const float v = __shfl_sync(0xffffffffu, my_v, e);
      const float4* slr = reinterpret_cast<const float4*>(stage + (size_t)e * SLOT);
      const float4* slp = reinterpret_cast<const float4*>(stage + ((size_t)maxnz + e) * SLOT);
#pragma unroll
      for (int c = 0; c < CPL; ++c)
#pragma unroll
        for (int k = 0; k < K; ++k) {
          const float4 xr = slr[k * wb + lane + 32 * c];
          const float4 xp = slp[k * wb + lane + 32 * c];
          accr[c][k].x = fmaf(v, xr.x, accr[c][k].x);
          accr[c][k].y = fmaf(v, xr.y, accr[c][k].y);
          accr[c][k].z = fmaf(v, xr.z, accr[c][k].z);
          accr[c][k].w = fmaf(v, xr.w, accr[c][k].w);
          accp[c][k].x = fmaf(v, xp.x, accp[c][k].x);
          accp[c][k].y = fmaf(v, xp.y, accp[c][k].y);
          accp[c][k].z = fmaf(v, xp.z, accp[c][k].z);
          accp[c][k].w = fmaf(v, xp.w, accp[c][k].w);
        }
    }
    if (diag) {
      const int ed = __ffs(diag) - 1;
      const float4* slr = reinterpret_cast<const float4*>(stage + (size_t)ed * SLOT);
      const float4* slp = reinterpret_cast<const float4*>(stage + ((size_t)maxnz + ed) * SLOT);
#pragma unroll
      for (int c = 0; c < CPL; ++c)
#pragma unroll
        for (int k = 0; k < K; ++k) {
          ownr[c][k] = slr[k * wb + lane + 32 * c];
          ownp[c][k] = slp[k * wb + lane + 32 * c];
        }
      have_own = true;
    }
    __syncwarp();
    const bool row_done = cc.ke == cc.k1;
    const int64_t row = cc.row;
    if (pc.valid) {
      issue_item<2>(pc, ring + s * stage_bytes, bars + s, a.colidx, arrs, row_f4, blk_f4, SLOT, SLICE,
                    maxnz, lane, a.stall_bytes);
      cur_next(pc, rstride, a.n, a.rowptr, maxnz);
    }
    cur_next(cc, rstride, a.n, a.rowptr, maxnz);
    s = (s + 1 == S) ? 0 : s + 1;
    if (row_done) {
      const int64_t base = row * row_f4 + blk_f4;
      if (!have_own) {
#pragma unroll
        for (int c = 0; c < CPL; ++c)
          if (lane + 32 * c < wb) {
#pragma unroll
            for (int k = 0; k < K; ++k) {
              ownr[c][k] = reinterpret_cast<const float4*>(R)[base + k * wb + lane + 32 * c];
              ownp[c][k] = reinterpret_cast<const float4*>(P)[base + k * wb + lane + 32 * c];
            }
          }
      }
#pragma unroll
      for (int c = 0; c < CPL; ++c) {
        if (mask & (1u << c)) {
          float dsum = 0.f;
#pragma unroll
          for (int k = 0; k < K; ++k) {
            float4 rn, pnv;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int j = 2 * k + h;
              const Coef<float>& q = cf[c][j];
              const float2 r = h ? make_float2(ownr[c][k].z, ownr[c][k].w)
                                 : make_float2(ownr[c][k].x, ownr[c][k].y);
              const float2 p = h ? make_float2(ownp[c][k].z, ownp[c][k].w)
                                 : make_float2(ownp[c][k].x, ownp[c][k].y);
              const float2 lr = h ? make_float2(accr[c][k].z, accr[c][k].w)
                                  : make_float2(accr[c][k].x, accr[c][k].y);
              const float2 lp = h ? make_float2(accp[c][k].z, accp[c][k].w)
                                  : make_float2(accp[c][k].x, accp[c][k].y);
              const float2 pn = cfma<float>(q.beta, p, make_float2(q.ar * r.x, q.ar * r.y));
              const float2 lpn = cfma<float>(q.beta, lp, make_float2(q.ar * lr.x, q.ar * lr.y));
              const float2 sv = csub<float>(cmul<float>(zv[j], pn), lpn);
              const float2 rr = csub<float>(r, cmul<float>(q.alpha, sv));
              dsum = fmaf(q.ca.x, pn.x, fmaf(-q.ca.y, pn.y, dsum));
              if (h) {
                rn.z = rr.x;
                rn.w = rr.y;
                pnv.z = pn.x;
                pnv.w = pn.y;
              } else {
                rn.x = rr.x;
                rn.y = rr.y;
                pnv.x = pn.x;
                pnv.y = pn.y;
              }
            }
            Rn[base + k * wb + lane + 32 * c] = rn;
            Pn[base + k * wb + lane + 32 * c] = pnv;
          }
          a.dacc[row * a.ldd + cb * bw + lane + 32 * c] += dsum;
        }
#pragma unroll
        for (int k = 0; k < K; ++k) accr[c][k] = accp[c][k] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      have_own = false;
    }
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
struct TmaShape {
  int warps = 0, grid = 0, S = 2, maxnz = 8;
  size_t smem = 0;
};

static TmaShape tma_shape(int num_sms, int narr, uint32_t slice, int maxnz, int ncb,
                          size_t red_bytes) {
  TmaShape t;
  t.maxnz = maxnz;
  t.S = 2;
  const size_t budget = 220 * 1024;
  const size_t per_warp = (size_t)t.S * maxnz * narr * slice + t.S * 8;
  int w = (int)std::min<size_t>(8, budget / per_warp);
  if (w < 1) w = 1;
  t.warps = w;
  t.smem = std::max((size_t)w * per_warp, red_bytes);
  // total warps must be a multiple of the column-block count
  int g = num_sms;
  while (g > 1 && ((int64_t)g * w) % ncb != 0) --g;
  if (((int64_t)g * w) % ncb != 0) {
    g = ncb;  // w == 1 fallback
  }
  t.grid = g;
  return t;
}

int tma_cpl(int m0) { return m0 > 32 * 2 ? 2 : 1; }
int tma_ncb(int m0, int cpl) { return (m0 + 32 * cpl - 1) / (32 * cpl); }

template <int NC, int CPL>
static void run_tma(const CocgArgs<float>& a, int which, int buf, int maxnz, int num_sms,
                    cudaStream_t s) {
  constexpr int CBW = 32 * CPL;
  constexpr uint32_t SLOT = CBW * NC * 8;
  const int ncb = (a.m0 + CBW - 1) / CBW;
  const int bw = (a.m0 + ncb - 1) / ncb;
  if (which == 0) {
    const int64_t total = a.n * (int64_t)a.m0;
    int64_t blocks = (total + 255) / 256;
    if (blocks > (int64_t)num_sms * 8) blocks = (int64_t)num_sms * 8;
    k_init_blocked<NC, CPL><<<(int)std::max<int64_t>(blocks, 1), 256, 0, s>>>(a, bw);
    RF_LAUNCH();
    return;
  }
  const int narr = which == 1 ? 1 : 2;
  const size_t red = (size_t)ncb * 32 * CPL * NC * 5 * sizeof(double);
  TmaShape t = tma_shape(num_sms, narr, SLOT, maxnz, ncb, which == 1 ? red : 0);
  if (which == 1) {
    ensure_dyn_smem(reinterpret_cast<const void*>(k_dots_tma<NC, CPL>), t.smem);
    k_dots_tma<NC, CPL><<<t.grid, 32 * t.warps, t.smem, s>>>(a, buf, ncb, bw, t.maxnz, t.S);
  } else {
    ensure_dyn_smem(reinterpret_cast<const void*>(k_update_tma<NC, CPL>), t.smem);
    k_update_tma<NC, CPL><<<t.grid, 32 * t.warps, t.smem, s>>>(a, buf, ncb, bw, t.maxnz, t.S);
  }
  RF_LAUNCH();
}

// which: 0 init, 1 dots, 2 update
void launch_cocg_tma(const CocgArgs<float>& a, int NC, int which, int buf, int maxnz,
                     int num_sms, cudaStream_t s) {
  const int cpl = tma_cpl(a.m0);
#define RF_TMA(NCV, CPLV)                                               \
  if (NC == NCV && cpl == CPLV) {                                       \
    run_tma<NCV, CPLV>(a, which, buf, maxnz, num_sms, s);               \
    return;                                                             \
  }
  RF_TMA(2, 1) RF_TMA(2, 2) RF_TMA(4, 1) RF_TMA(4, 2) RF_TMA(8, 1) RF_TMA(8, 2)
#undef RF_TMA
  throw Err{RAFEAST_ERR_INVALID_ARG};
}

}  // namespace rafeast
