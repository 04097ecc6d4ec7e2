// Persistent grouped multi-shift COCG kernels: the COCG steps of many
// independent problems (uneven n, their own CSR, shifts, columns and state)
// in one launch per kernel and step, for rafeast_solve_batched.
//
// A launch is a persistent grid (the resident CTA count) draining a queue of
// work items. Problem t contributes gx_t x gy_t items (row slices x column
// blocks), arranged exactly as the single-problem kernels arrange their 2-D
// grid, so the kernel bodies (cocg_kernels.cuh) run unchanged on an item's
// Blk coordinate; the dot kernel's per-problem ticket counts the problem's
// items, so its scalar step runs when its last item is done. Items are
// numbered problem by problem and taken in order from an atomic counter, so
// the CTAs in flight work on one or two problems at a time and those
// problems' gathered rows stay in L2, while every CTA stays busy until the
// queue is empty whatever the spread of n.
//
// The queue follows the problems that are still iterating: the last CTA of
// every dot launch (global ticket, taken after every item's work and every
// problem's scalar step of the step) re-plans both kernels' item maps over
// the problems whose COCG has not finished, choosing the rows per item so
// that the active problems fill about ITEMS_PER_CTA items per resident CTA.
#include <algorithm>
#include <cstdio>

#include "cocg_kernels.cuh"

namespace rafeast {

constexpr int ITEMS_PER_CTA = 4;        // fewest items per resident CTA
constexpr long long WINDOW_KB = 48 * 1024;  // gathered state the CTAs in flight may share
constexpr int SMEM_MAP = 512;            // problems whose item map is staged in smem

// exclusive scan over the block (blockDim.x == THREADS); returns the prefix,
// *total the block sum
__device__ __forceinline__ int block_scan(int v, int* total) {
  __shared__ int s_w[WARPS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_w[warp] = x;
  __syncthreads();
  int base = 0, tot = 0;
#pragma unroll
  for (int w = 0; w < WARPS; ++w) {
    const int sw = s_w[w];
    if (w < warp) base += sw;
    tot += sw;
  }
  __syncthreads();
  *total = tot;
  return base + x - v;
}

// item maps over the active problems (done == 0), computed by the whole
// block: rows per item R chosen so that the active problems make about
// mult x grid items, mult = max(ITEMS_PER_CTA, gathered state / WINDOW_KB),
// i.e. the items in flight at any time share about WINDOW_KB of gathered
// state. map[0..count] item starts, map[count + 1 + t] = gx_t (>= 1).
__device__ void plan_items(const CocgCtl* __restrict__ ctl, const int4* __restrict__ gg_d,
                           const int4* __restrict__ gg_u, int count, int grid_d, int grid_u,
                           int* __restrict__ map_d, int* __restrict__ map_u) {
  __shared__ long long s_red[3][WARPS];
  __shared__ long long s_R[2];
  long long work_d = 0, work_u = 0, wkb = 0;
  for (int t = threadIdx.x; t < count; t += blockDim.x)
    if (!__ldcg(&ctl[t].done)) {
      const int4 g = gg_d[t], h = gg_u[t];
      work_d += (long long)g.x * g.y;
      work_u += (long long)h.x * h.y;
      wkb += g.z;
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    work_d += __shfl_xor_sync(0xffffffffu, work_d, o);
    work_u += __shfl_xor_sync(0xffffffffu, work_u, o);
    wkb += __shfl_xor_sync(0xffffffffu, wkb, o);
  }
  if ((threadIdx.x & 31) == 0) {
    s_red[0][threadIdx.x >> 5] = work_d;
    s_red[1][threadIdx.x >> 5] = work_u;
    s_red[2][threadIdx.x >> 5] = wkb;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    long long Wd = 0, Wu = 0, K = 0;
    for (int w = 0; w < WARPS; ++w) {
      Wd += s_red[0][w];
      Wu += s_red[1][w];
      K += s_red[2][w];
    }
    long long mult = (K + WINDOW_KB - 1) / WINDOW_KB;
    if (mult < ITEMS_PER_CTA) mult = ITEMS_PER_CTA;
    const long long td = mult * grid_d, tu = mult * grid_u;
    s_R[0] = Wd > td ? (Wd + td - 1) / td : 1;
    s_R[1] = Wu > tu ? (Wu + tu - 1) / tu : 1;
  }
  __syncthreads();
  const long long Rd = s_R[0], Ru = s_R[1];
  int off_d = 0, off_u = 0;
  for (int base = 0; base < count; base += blockDim.x) {
    const int t = base + threadIdx.x;
    int nd = 0, nu = 0, gxd = 1, gxu = 1;
    if (t < count && !__ldcg(&ctl[t].done)) {
      const int4 g = gg_d[t], h = gg_u[t];
      gxd = (int)((g.x + Rd - 1) / Rd);
      gxu = (int)((h.x + Ru - 1) / Ru);
      if (gxd < 1) gxd = 1;
      if (gxu < 1) gxu = 1;
      nd = gxd * g.y;
      nu = gxu * h.y;
    }
  int tot_d = 0, tot_u = 0;
    const int pd = block_scan(nd, &tot_d);
    const int pu = block_scan(nu, &tot_u);
    if (t < count) {
      map_d[t] = off_d + pd;
      map_d[count + 1 + t] = gxd;
      map_u[t] = off_u + pu;
      map_u[count + 1 + t] = gxu;
    }
    off_d += tot_d;
    off_u += tot_u;
  }
  if (threadIdx.x == 0) {
    map_d[count] = off_d;
    map_u[count] = off_u;
  }
}

// the item map, staged in shared memory when it fits
struct MapView {
  const int* p;
  __device__ __forceinline__ int operator[](int i) const { return p[i]; }
};
__device__ __forceinline__ MapView stage_map(const int* __restrict__ map, int count, int* smap) {
  MapView v;
  if (count <= SMEM_MAP) {
    for (int i = threadIdx.x; i < 2 * count + 1; i += blockDim.x) smap[i] = __ldcg(map + i);
    __syncthreads();
    v.p = smap;
  } else {
    v.p = map;
  }
  return v;
}

__device__ __forceinline__ int item_owner(const MapView& m, int count, int item) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (m[mid] <= item) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ Blk item_blk(const MapView& m, int count, int t, int item) {
  const int start = m[t], end = m[t + 1], gx = m[count + 1 + t];
  const int local = item - start;
  Blk b;
  b.x = local % gx;
  b.y = local / gx;
  b.gx = gx;
  b.gy = (end - start) / gx;
  return b;
}

// next item for this CTA (block-uniform), or -1 when the queue is empty
__device__ __forceinline__ int next_item(unsigned int* counter, int total) {
  __shared__ int s_item;
  __syncthreads();  // every thread is done with the previous item
  if (threadIdx.x == 0) {
    const unsigned int i = atomicAdd(counter, 1u);
    s_item = i < (unsigned int)total ? (int)i : -1;
  }
  __syncthreads();
  return s_item;
}

template <typename T, int MAXCPL, bool VF>
__global__ void __launch_bounds__(THREADS, (sizeof(T) == 4 && MAXCPL * 2 <= 4) ? 2 : 1)
    k_ms_dots_grouped(const CocgArgs<T>* __restrict__ args, int* __restrict__ map_d,
                      int* __restrict__ map_u, GroupCtl* __restrict__ gc,
                      const CocgCtl* __restrict__ ctl, const int4* __restrict__ gg_d,
                      const int4* __restrict__ gg_u, int count, int buf) {
  __shared__ int smap[2 * SMEM_MAP + 1];
  __shared__ int s_glast;
  const MapView m = stage_map(map_d, count, smap);
  const int total = m[count];
  for (;;) {
    const int item = next_item(&gc->next_d, total);
    if (item < 0) break;
    const int t = item_owner(m, count, item);
    const CocgArgs<T> a = args[t];
    cocg_dots_body<T, 2, MAXCPL, VF>(a, args + t, buf, item_blk(m, count, t, item));
  }
  // every CTA takes a global ticket once the queue is empty; all items (and
  // every problem's scalar step) are then done, and the last CTA re-plans
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_glast = atomicAdd(&gc->ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (s_glast) {
    __threadfence();
    plan_items(ctl, gg_d, gg_u, count, gc->grid_d, gc->grid_u, map_d, map_u);
    if (threadIdx.x == 0) {
      gc->next_d = 0;
      gc->next_u = 0;
      gc->ticket = 0;
      __threadfence();
    }
  }
}

template <typename T, int NS, int MAXCPL>
__global__ void __launch_bounds__(THREADS, sizeof(T) == 4 ? 2 : 1)
    k_ms_update_grouped(const CocgArgs<T>* __restrict__ args, const int* __restrict__ map,
                        GroupCtl* __restrict__ gc, int count, int buf) {
  __shared__ int smap[2 * SMEM_MAP + 1];
  const MapView m = stage_map(map, count, smap);
  const int total = m[count];
  for (;;) {
    const int item = next_item(&gc->next_u, total);
    if (item < 0) break;
    const int t = item_owner(m, count, item);
    const CocgArgs<T> a = args[t];
    ms_update_body<T, NS, MAXCPL>(a, args + t, buf, item_blk(m, count, t, item));
  }
}

// streamed update over a queue of items: an item is a contiguous range of
// one problem's n x pairs (row, column pair) elements; the problem's
// coefficients are staged in shared memory per item (buf is unused: the
// streamed state is updated in place)
template <typename T, int NS>
__global__ void __launch_bounds__(THREADS)
    k_ms_update_stream_grouped(const CocgArgs<T>* __restrict__ args, const int* __restrict__ map,
                               GroupCtl* __restrict__ gc, int count, int buf) {
  (void)buf;
  __shared__ int smap[2 * SMEM_MAP + 1];
  extern __shared__ unsigned char smem_raw[];
  const MapView m = stage_map(map, count, smap);
  const int total = m[count];
  for (;;) {
    const int item = next_item(&gc->next_u, total);
    if (item < 0) break;
    const int t = item_owner(m, count, item);
    const CocgArgs<T> a = args[t];
    const Blk b = item_blk(m, count, t, item);
    ms_stream_stage<T, NS>(a, smem_raw);
    const int64_t tot = a.n * (int64_t)a.m0;
    const int64_t chunk = (tot + b.gx - 1) / b.gx;
    const int64_t e0 = b.x * chunk;
    const int64_t e1 = e0 + chunk < tot ? e0 + chunk : tot;
    // (bottom-up here: walking the items and elements top-down measured
    // slower for the grouped launches)
    ms_stream_elems<T, NS>(a, smem_raw, e0 + threadIdx.x, e1, blockDim.x, e0, false);
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
template <typename T> constexpr int grouped_mc_large() { return sizeof(T) == 4 ? 4 : 2; }

template <typename T, int NS, int MC>
static const void* update_fn() {
  return reinterpret_cast<const void*>(k_ms_update_grouped<T, NS, MC>);
}

template <typename T, int MC>
static const void* update_fn_ns(int ns) {
  switch (ns) {
    case 0: return update_fn<T, 0, MC>();
    case 1: return update_fn<T, 1, MC>();
    case 2: return update_fn<T, 2, MC>();
    case 3: return update_fn<T, 3, MC>();
    case 4: return update_fn<T, 4, MC>();
    case 5: return update_fn<T, 5, MC>();
    case 6: return update_fn<T, 6, MC>();
    case 7: return update_fn<T, 7, MC>();
    default: throw Err{RAFEAST_ERR_INVALID_ARG};
  }
}

template <typename T>
static const void* stream_fn(int ns) {
  switch (ns) {
    case 0: return reinterpret_cast<const void*>(k_ms_update_stream_grouped<T, 0>);
    case 1: return reinterpret_cast<const void*>(k_ms_update_stream_grouped<T, 1>);
    case 2: return reinterpret_cast<const void*>(k_ms_update_stream_grouped<T, 2>);
    case 3: return reinterpret_cast<const void*>(k_ms_update_stream_grouped<T, 3>);
    case 4: return reinterpret_cast<const void*>(k_ms_update_stream_grouped<T, 4>);
    case 5: return reinterpret_cast<const void*>(k_ms_update_stream_grouped<T, 5>);
    case 6: return reinterpret_cast<const void*>(k_ms_update_stream_grouped<T, 6>);
    case 7: return reinterpret_cast<const void*>(k_ms_update_stream_grouped<T, 7>);
    default:  // N_c = 9..16: the shift count read at run time
      if (ns < 0 || ns > 15) throw Err{RAFEAST_ERR_INVALID_ARG};
      return reinterpret_cast<const void*>(k_ms_update_stream_grouped<T, -1>);
  }
}

template <typename T>
static const void* dots_fn(int mc, bool vf) {
  if (vf) {
    if (mc <= 2) return reinterpret_cast<const void*>(k_ms_dots_grouped<T, 2, true>);
    return reinterpret_cast<const void*>(k_ms_dots_grouped<T, grouped_mc_large<T>(), true>);
  }
  if (mc <= 2) return reinterpret_cast<const void*>(k_ms_dots_grouped<T, 2, false>);
  return reinterpret_cast<const void*>(k_ms_dots_grouped<T, grouped_mc_large<T>(), false>);
}

template <typename T>
static const void* upd_fn(int mc, int ns) {
  if (mc <= 2) return update_fn_ns<T, 2>(ns);
  return update_fn_ns<T, grouped_mc_large<T>()>(ns);
}

// initial item maps (every problem active), same rule as the device planner
static void plan_host(const std::vector<int>& gg, long long wkb, int grid, std::vector<int>& map) {
  const int cnt = (int)gg.size() / 4;
  long long work = 0;
  for (int t = 0; t < cnt; ++t) work += (long long)gg[4 * t] * gg[4 * t + 1];
  long long mult = std::max<long long>(ITEMS_PER_CTA, (wkb + WINDOW_KB - 1) / WINDOW_KB);
  const long long target = mult * grid;
  const long long R = work > target ? (work + target - 1) / target : 1;
  map.assign(2 * cnt + 1, 0);
  long long start = 0;
  for (int t = 0; t < cnt; ++t) {
    long long gx = (gg[4 * t] + R - 1) / R;
    if (gx < 1) gx = 1;
    map[t] = (int)start;
    map[cnt + 1 + t] = (int)gx;
    start += gx * gg[4 * t + 1];
  }
  if (start > 0x3fffffff) throw Err{RAFEAST_ERR_INVALID_ARG};
  map[cnt] = (int)start;
}

// per problem: row groups, column blocks, gathered state (KiB), 0
template <typename T>
static void shapes_of(const std::vector<CocgArgs<T>>& args, std::vector<int>& gg) {
  const int cnt = (int)args.size();
  gg.assign(4 * cnt, 0);
  for (int t = 0; t < cnt; ++t) {
    const auto& a = args[t];
    const int64_t per = (int64_t)WARPS * (32 / a.lanes);
    const int64_t groups = (a.n + per - 1) / per;
    RF_CHECK(groups < 0x7fffffff, RAFEAST_ERR_INVALID_ARG);
    gg[4 * t] = (int)groups;
    gg[4 * t + 1] = (a.m0 + a.lanes * a.cpl - 1) / (a.lanes * a.cpl);
    // seed r and p of every pair
    gg[4 * t + 2] = (int)std::min<int64_t>(
        0x7fffffff, (a.n * (int64_t)a.m0 * 2 * 2 * 2 * (int64_t)sizeof(T) + 1023) / 1024);
  }
}

template <typename T>
void plan_ms_grouped(const std::vector<CocgArgs<T>>& args_d, const std::vector<CocgArgs<T>>& args_u,
                     int num_sms, GroupPlan& g) {
  const int cnt = (int)args_d.size();
  RF_CHECK(cnt >= 1 && (int)args_u.size() == cnt, RAFEAST_ERR_INVALID_ARG);
  g.count = cnt;
  g.ns = args_d[0].ns;
  int cd = 1, cu = 1, ld = 4, lcu = 1;
  for (int t = 0; t < cnt; ++t) {
    const auto& a = args_d[t];
    const auto& b = args_u[t];
    RF_CHECK(a.ns == g.ns && b.ns == g.ns && a.ms == 1 && b.ms == 1, RAFEAST_ERR_INVALID_ARG);
    RF_CHECK(a.cpl >= 1 && a.cpl <= grouped_mc_large<T>() && b.cpl >= 1 &&
                 b.cpl <= grouped_mc_large<T>(),
             RAFEAST_ERR_INVALID_ARG);
    cd = std::max(cd, a.cpl);
    cu = std::max(cu, b.cpl);
    ld = std::max(ld, a.lanes);
    lcu = std::max(lcu, b.lanes * b.cpl);
  }
  const bool stream = args_u[0].wbuf != nullptr;
  int pmax = 1;
  for (int t = 0; t < cnt; ++t) {
    RF_CHECK((args_u[t].wbuf != nullptr) == stream && (args_d[t].wbuf != nullptr) == stream,
             RAFEAST_ERR_INVALID_ARG);
    pmax = std::max(pmax, args_u[t].m0);
  }
  g.mc_d = cd <= 2 ? 2 : grouped_mc_large<T>();
  g.mc_u = cu <= 2 ? 2 : grouped_mc_large<T>();
  g.smem_dots = (size_t)ld * g.mc_d * 2 * 5 * sizeof(double);
  // values-free dot instances when the problems carry the off-diagonal
  // pattern of a unit-weight Laplacian (all of them or none)
  const bool vf = args_d[0].lcolidx != nullptr;
  for (int t = 0; t < cnt; ++t)
    RF_CHECK((args_d[t].lcolidx != nullptr) == vf, RAFEAST_ERR_INVALID_ARG);
  g.fn_dots = dots_fn<T>(g.mc_d, vf);
  if (stream) {
    g.smem_upd = ms_stream_smem<T>(pmax, g.ns);
    g.fn_upd = stream_fn<T>(g.ns);
  } else {
    g.smem_upd = (size_t)2 * lcu * (sizeof(Coef<T>) + g.ns * sizeof(ShiftCoef<T>)) + 16;
    g.fn_upd = upd_fn<T>(g.mc_u, g.ns);
  }
  if (g.smem_upd > 48 * 1024) ensure_dyn_smem(g.fn_upd, g.smem_upd);
  int occ_d = 0, occ_u = 0;
  RF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_d, g.fn_dots, THREADS, g.smem_dots));
  RF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_u, g.fn_upd, THREADS, g.smem_upd));
  shapes_of(args_d, g.gg_d);
  shapes_of(args_u, g.gg_u);
  if (stream)
    for (int t = 0; t < cnt; ++t) {
      // element passes of one CTA over the problem's n x pairs elements
      const int64_t el = args_u[t].n * (int64_t)args_u[t].m0;
      RF_CHECK((el + THREADS - 1) / THREADS < 0x7fffffff, RAFEAST_ERR_INVALID_ARG);
      g.gg_u[4 * t] = (int)((el + THREADS - 1) / THREADS);
      g.gg_u[4 * t + 1] = 1;
    }
  long long wkb = 0;
  for (int t = 0; t < cnt; ++t) wkb += g.gg_d[4 * t + 2];
  g.ctas_dots = num_sms * std::max(occ_d, 1);
  g.ctas_upd = num_sms * std::max(occ_u, 1);
  plan_host(g.gg_d, wkb, g.ctas_dots, g.map_dots);
  plan_host(g.gg_u, wkb, g.ctas_upd, g.map_upd);
}

template <typename T>
void launch_ms_grouped(const GroupPlan& g, const GroupDev<T>& d, int which, int buf,
                       cudaStream_t s) {
  int cnt = g.count;
  GroupCtl* gc = d.gc;
  if (which == 0) {
    const CocgArgs<T>* ap = d.args_d;
    int* md = d.map_d;
    int* mu = d.map_u;
    const CocgCtl* ctl = d.ctl;
    const int4* ggd = d.gg_d;
    const int4* ggu = d.gg_u;
    void* params[] = {(void*)&ap,  (void*)&md,  (void*)&mu,  (void*)&gc, (void*)&ctl,
                      (void*)&ggd, (void*)&ggu, (void*)&cnt, (void*)&buf};
    RF_CUDA(cudaLaunchKernel(g.fn_dots, dim3(g.ctas_dots), dim3(THREADS), params, g.smem_dots, s));
  } else {
    const CocgArgs<T>* ap = d.args_u;
    const int* mu = d.map_u;
    void* params[] = {(void*)&ap, (void*)&mu, (void*)&gc, (void*)&cnt, (void*)&buf};
    RF_CUDA(cudaLaunchKernel(g.fn_upd, dim3(g.ctas_upd), dim3(THREADS), params, g.smem_upd, s));
  }
  RF_LAUNCH();
}

template void plan_ms_grouped<float>(const std::vector<CocgArgs<float>>&,
                                     const std::vector<CocgArgs<float>>&, int, GroupPlan&);
template void plan_ms_grouped<double>(const std::vector<CocgArgs<double>>&,
                                      const std::vector<CocgArgs<double>>&, int, GroupPlan&);
template void launch_ms_grouped<float>(const GroupPlan&, const GroupDev<float>&, int, int,
                                       cudaStream_t);
template void launch_ms_grouped<double>(const GroupPlan&, const GroupDev<double>&, int, int,
                                        cudaStream_t);

}  // namespace rafeast
