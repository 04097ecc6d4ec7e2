// Allocation-free Gram matrix, G = X^T Y (rafeast_gram_noalloc).
//
// Same result as rafeast_gram, for callers that must not have the library
// allocate device memory during the call. Its scratch (one m x m partial sum
// per CTA) lives in a file-scope device array of fixed size, compiled into
// the library. Host code never passes the array's symbol to a kernel (on the
// host the symbol is only a stand-in, not a device address); the device
// address is looked up once per device with cudaGetSymbolAddress, with that
// device current, and cached.
//
// The array belongs to this file's module. CUDA loads modules lazily by
// default (CUDA_MODULE_LOADING=LAZY), so the first call on a device is the one
// that loads the module: that call allocates the 2 MiB array and the code of
// the entry point's kernels on the device (it has all of them loaded), and
// later calls allocate nothing. From then on the
// device holds the array until the process exits. A caller that reserves
// device memory for its own allocator, or captures streams, makes a first call
// (n = 1, m = 1 is enough) before doing so. The cached address is only valid
// for the device context it was looked up in: no cudaDeviceReset may come
// after the first call on that device.
//
// Calls share the array, so two calls whose kernels overlap on the GPU (two
// streams, or two host threads) race on it. Each call overwrites every
// partial it later sums, so nothing needs clearing between calls.
#include <cstdio>
#include <mutex>

#include "internal.h"

namespace rafeast {

constexpr int NOALLOC_MAX_M = 64;   // largest m accepted
constexpr int NOALLOC_PARTS = 64;   // most per-CTA partial sums
constexpr size_t NOALLOC_DOUBLES = (size_t)NOALLOC_PARTS * NOALLOC_MAX_M * NOALLOC_MAX_M;

static __device__ __align__(256) double g_noalloc_partials[NOALLOC_DOUBLES];  // 2 MiB

constexpr int NA_RB = 16;  // rows staged per step

// partial[c] (column-major m x m) = X[rows of c]^T Y[rows of c]; X, Y
// column-major n x m. 16 x 16 threads, thread (tx, ty) owns entries
// (tx + 16u, ty + 16v).
template <int U>
__global__ void __launch_bounds__(256) k_gram_partial_noalloc(const double* __restrict__ X,
                                                              const double* __restrict__ Y,
                                                              int64_t n, int m,
                                                              double* __restrict__ part) {
  __shared__ double Xs[NA_RB][NOALLOC_MAX_M];
  __shared__ double Ys[NA_RB][NOALLOC_MAX_M];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[U][U];
#pragma unroll
  for (int u = 0; u < U; ++u)
#pragma unroll
    for (int v = 0; v < U; ++v) acc[u][v] = 0.0;
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = blockIdx.x * chunk;
  const int64_t r1 = min(n, r0 + chunk);
  for (int64_t rb = r0; rb < r1; rb += NA_RB) {
    const int rows = (int)min((int64_t)NA_RB, r1 - rb);
    __syncthreads();
    for (int t = threadIdx.x; t < NA_RB * m; t += blockDim.x) {
      const int rr = t % NA_RB, col = t / NA_RB;  // consecutive threads: consecutive rows
      Xs[rr][col] = rr < rows ? X[(int64_t)col * n + rb + rr] : 0.0;
      Ys[rr][col] = rr < rows ? Y[(int64_t)col * n + rb + rr] : 0.0;
    }
    __syncthreads();
    for (int rr = 0; rr < rows; ++rr) {
      double xa[U], yb[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int a = tx + 16 * u, b = ty + 16 * u;
        xa[u] = a < m ? Xs[rr][a] : 0.0;
        yb[u] = b < m ? Ys[rr][b] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int v = 0; v < U; ++v) acc[u][v] = fma(xa[u], yb[v], acc[u][v]);
    }
  }
  double* out = part + (int64_t)blockIdx.x * m * m;
#pragma unroll
  for (int u = 0; u < U; ++u)
#pragma unroll
    for (int v = 0; v < U; ++v) {
      const int a = tx + 16 * u, b = ty + 16 * v;
      if (a < m && b < m) out[(int64_t)b * m + a] = acc[u][v];
    }
}

__global__ void k_gram_sum_noalloc(const double* __restrict__ part, int nparts, int mm,
                                   double* __restrict__ G) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < mm; e += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < nparts; ++c) s += part[(int64_t)c * mm + e];
    G[e] = s;
  }
}

static std::mutex g_noalloc_mu;
static double* g_noalloc_addr[128] = {nullptr};

// device address of the array on device `dev`, the current device. The first
// call there sets up: it looks the address up (which loads this file's
// module, allocating the array) and has every kernel of the entry point
// loaded, so that all of the device memory the entry point ever takes is
// taken by that first call.
static cudaError_t noalloc_scratch(int dev, double** out) {
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    const void* fns[5] = {reinterpret_cast<const void*>(k_gram_partial_noalloc<1>),
                          reinterpret_cast<const void*>(k_gram_partial_noalloc<2>),
                          reinterpret_cast<const void*>(k_gram_partial_noalloc<3>),
                          reinterpret_cast<const void*>(k_gram_partial_noalloc<4>),
                          reinterpret_cast<const void*>(k_gram_sum_noalloc)};
    for (const void* f : fns) {
      e = cudaFuncGetAttributes(&fa, f);
      if (e != cudaSuccess) return e;
    }
    g_noalloc_addr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_addr[dev];
  return cudaSuccess;
}

}  // namespace rafeast

using namespace rafeast;

extern "C" int rafeast_gram_noalloc(const double* X, const double* Y, int64_t n, int m,
                                    double* G, void* stream) {
  clear_last_error();
  if (!X || !Y || !G || n < 1) return RAFEAST_ERR_INVALID_ARG;
  if (m < 1 || m > NOALLOC_MAX_M) {
    char msg[160];
    snprintf(msg, sizeof(msg),
             "rafeast_gram_noalloc: m = %d is outside 1..%d, the column limit of its fixed "
             "scratch array",
             m, NOALLOC_MAX_M);
    set_last_message(msg);
    return RAFEAST_ERR_INVALID_ARG;
  }
  // an error left pending by the caller's own earlier work is reported as
  // it is and left pending for the caller (not cleared, not launched over)
  cudaError_t e = cudaPeekAtLastError();
  if (e != cudaSuccess) {
    set_last_error(e, "rafeast_gram_noalloc: a CUDA error was pending before the call",
                   __FILE__, __LINE__);
    return RAFEAST_ERR_CUDA;
  }
  int dev = 0;
  e = cudaGetDevice(&dev);
  double* part = nullptr;
  if (e == cudaSuccess) e = noalloc_scratch(dev, &part);
  if (e != cudaSuccess) {
    set_last_error(e, "rafeast_gram_noalloc setup", __FILE__, __LINE__);
    return RAFEAST_ERR_CUDA;
  }
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  int64_t parts = (n + NA_RB - 1) / NA_RB;
  if (parts > NOALLOC_PARTS) parts = NOALLOC_PARTS;
  switch ((m + 15) / 16) {
    case 1: k_gram_partial_noalloc<1><<<(int)parts, 256, 0, s>>>(X, Y, n, m, part); break;
    case 2: k_gram_partial_noalloc<2><<<(int)parts, 256, 0, s>>>(X, Y, n, m, part); break;
    case 3: k_gram_partial_noalloc<3><<<(int)parts, 256, 0, s>>>(X, Y, n, m, part); break;
    default: k_gram_partial_noalloc<4><<<(int)parts, 256, 0, s>>>(X, Y, n, m, part); break;
  }
  e = cudaGetLastError();
  if (e == cudaSuccess) {
    k_gram_sum_noalloc<<<(m * m + 255) / 256, 256, 0, s>>>(part, (int)parts, m * m, G);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    set_last_error(e, "rafeast_gram_noalloc launch", __FILE__, __LINE__);
    return RAFEAST_ERR_CUDA;
  }
  return RAFEAST_OK;
}
