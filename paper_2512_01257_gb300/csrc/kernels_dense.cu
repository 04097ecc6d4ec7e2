// Dense FP64 kernels of the RA-FEAST outer loop (sm_103a).
//
// * Philox-4x64-10 words and Box-Muller normals for Omega (Algorithm 2,
//   "Draw Omega"; Salmon et al., SC'11).
// * Layout moves between the caller's column-major blocks and the internal
//   row-major, row-permuted blocks.
// * Tall-skinny Gram G = X^T Y (Cholesky-QR Gram B_Q = Q~^T Q~ and the
//   Rayleigh-Ritz matrix A_Q = Q^T (A Q), Algorithm 1), split over rows with
//   per-CTA partials and a deterministic second-stage sum.
// * One-CTA Cholesky of the m x m Gram matrix with the shift of shifted
//   Cholesky-QR when it is not numerically positive definite (Fukaya,
//   Kannan, Nakatsukasa, Yamamoto, Yanagisawa, SIAM J. Sci. Comput. 2020),
//   plus the inverse of the triangular factor, so Q = Q~ R^{-1} is a GEMM.
// * Tall GEMM Y = X M (Q R^{-1}, Q V, (A Q) V).
// * One-CTA cyclic Jacobi eigensolver for the reduced symmetric problem
//   (Rayleigh-Ritz, Algorithm 1): round-robin ordering of m/2 disjoint
//   rotations per round, rotation angles from the symmetric 2x2 Schur form.
// * Column norms of A Q - Q diag(theta) (residuals) and column dots.
#include <cfloat>
#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace rafeast {

// ---------------------------------------------------------------------------
// Philox-4x64-10
// ---------------------------------------------------------------------------
__device__ __forceinline__ void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += W0;
      k1 += W1;
    }
    const uint64_t hi0 = __umul64hi(M0, c[0]), lo0 = M0 * c[0];
    const uint64_t hi1 = __umul64hi(M1, c[2]), lo1 = M1 * c[2];
    const uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
}

__global__ void k_philox(uint64_t seed, uint64_t first, int64_t nblocks, uint64_t* out) {
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nblocks;
       b += (int64_t)gridDim.x * blockDim.x) {
    uint64_t c[4] = {first + (uint64_t)b, 0, 0, 0};
    philox4x64_10(c, seed, 0);
    out[4 * b + 0] = c[0];
    out[4 * b + 1] = c[1];
    out[4 * b + 2] = c[2];
    out[4 * b + 3] = c[3];
  }
}

__device__ __forceinline__ double u01(uint64_t x) {
  return ((double)(x >> 11) + 1.0) * 0x1.0p-53;
}

// Omega column-major n x k; linear index e = c*n + i; block e/4
__global__ void k_omega(uint64_t seed, int64_t total, double* out) {
  const int64_t nblk = (total + 3) / 4;
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nblk;
       b += (int64_t)gridDim.x * blockDim.x) {
    uint64_t c[4] = {(uint64_t)b, 0, 0, 0};
    philox4x64_10(c, seed, 0);
    double g[4];
    {
      const double rad = sqrt(-2.0 * log(u01(c[0])));
      double s, co;
      sincospi(2.0 * u01(c[1]), &s, &co);
      g[0] = rad * co;
      g[1] = rad * s;
    }
    {
      const double rad = sqrt(-2.0 * log(u01(c[2])));
      double s, co;
      sincospi(2.0 * u01(c[3]), &s, &co);
      g[2] = rad * co;
      g[3] = rad * s;
    }
#pragma unroll
    for (int t = 0; t < 4; ++t)
      if (4 * b + t < total) out[4 * b + t] = g[t];
  }
}

void launch_philox(uint64_t seed, uint64_t first, int64_t nblocks, uint64_t* out,
                   cudaStream_t s) {
  if (nblocks <= 0) return;
  int64_t blocks = (nblocks + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  k_philox<<<(int)blocks, 256, 0, s>>>(seed, first, nblocks, out);
  RF_LAUNCH();
}

void launch_omega(uint64_t seed, int64_t n, int k, double* out, cudaStream_t s) {
  const int64_t total = n * (int64_t)k;
  int64_t blocks = ((total + 3) / 4 + 255) / 256;
  if (blocks > 8192) blocks = 8192;
  if (blocks < 1) blocks = 1;
  k_omega<<<(int)blocks, 256, 0, s>>>(seed, total, out);
  RF_LAUNCH();
}

// ---------------------------------------------------------------------------
// layout moves
// ---------------------------------------------------------------------------
__global__ void k_to_internal(int64_t n, int m, const double* __restrict__ src,
                              double* __restrict__ dst, int ld, const int32_t* __restrict__ perm) {
  const int64_t total = n * (int64_t)ld;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / ld;
    const int c = (int)(e - r * ld);
    const int64_t o = perm ? perm[r] : r;
    dst[e] = c < m ? src[(int64_t)c * n + o] : 0.0;
  }
}

__global__ void k_from_internal(int64_t n, int m, const double* __restrict__ src, int ld,
                                double* __restrict__ dst, const int32_t* __restrict__ perm,
                                const int32_t* __restrict__ cols) {
  const int64_t total = n * (int64_t)m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / m;
    const int c = (int)(e - r * m);
    const int64_t o = perm ? perm[r] : r;
    const int sc = cols ? cols[c] : c;
    dst[(int64_t)c * n + o] = src[r * ld + sc];
  }
}

static int blocks_for(int64_t total, int per = 256, int cap = 16384) {
  int64_t b = (total + per - 1) / per;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

void launch_to_internal(int64_t n, int m, const double* src, double* dst, int ld,
                        const int32_t* perm, cudaStream_t s) {
  k_to_internal<<<blocks_for(n * (int64_t)ld), 256, 0, s>>>(n, m, src, dst, ld, perm);
  RF_LAUNCH();
}

void launch_from_internal(int64_t n, int m, const double* src, int ld, double* dst,
                          const int32_t* perm, const int32_t* cols, cudaStream_t s) {
  if (m <= 0) return;
  k_from_internal<<<blocks_for(n * (int64_t)m), 256, 0, s>>>(n, m, src, ld, dst, perm, cols);
  RF_LAUNCH();
}

__global__ void k_cast_f32(const double* __restrict__ src, float* __restrict__ dst, int64_t count) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = (float)src[e];
}
void launch_cast_to_f32(const double* src, float* dst, int64_t count, cudaStream_t s) {
  if (count <= 0) return;
  k_cast_f32<<<blocks_for(count), 256, 0, s>>>(src, dst, count);
  RF_LAUNCH();
}

__global__ void k_widen(const float* __restrict__ src, double* __restrict__ dst, int64_t count) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = (double)src[e];
}
void launch_widen(const float* src, double* dst, int64_t count, cudaStream_t s) {
  if (count <= 0) return;
  k_widen<<<blocks_for(count), 256, 0, s>>>(src, dst, count);
  RF_LAUNCH();
}

void launch_zero(void* p, size_t bytes, cudaStream_t s) {
  if (bytes) RF_CUDA(cudaMemsetAsync(p, 0, bytes, s));
}

// ---------------------------------------------------------------------------
// tall-skinny Gram: partial[cta] = X[rows]^T Y[rows], then a column sum
// ---------------------------------------------------------------------------
constexpr int GRAM_RB = 16;

// SYM: the result is symmetric, so the 16-strided tile blocks below the
// diagonal (u > v) are skipped; k_gram_sum mirrors them. A: the type the
// products are formed and summed in within a CTA (double; float for the
// preconditioning pass of a mixed-precision Cholesky-QR); the CTA partial
// sums are added in double.
template <int U, bool SYM, typename A = double>
__global__ void __launch_bounds__(256) k_gram_partial(const double* __restrict__ X,
                                                      const double* __restrict__ Y, int64_t n,
                                                      int m, int ld, double* __restrict__ part) {
  extern __shared__ double gsm[];
  double* Xs = gsm;                 // [GRAM_RB][ld]
  double* Ys = gsm + GRAM_RB * ld;  // [GRAM_RB][ld]
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  A acc[U][U];
#pragma unroll
  for (int u = 0; u < U; ++u)
#pragma unroll
    for (int v = 0; v < U; ++v) acc[u][v] = (A)0;
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = blockIdx.x * chunk;
  const int64_t r1 = min(n, r0 + chunk);
  for (int64_t rb = r0; rb < r1; rb += GRAM_RB) {
    const int rows = (int)min((int64_t)GRAM_RB, r1 - rb);
    __syncthreads();
    for (int t = threadIdx.x; t < GRAM_RB * ld; t += blockDim.x) {
      const int rr = t / ld;
      Xs[t] = rr < rows ? X[(rb + rr) * ld + (t - rr * ld)] : 0.0;
      Ys[t] = rr < rows ? Y[(rb + rr) * ld + (t - rr * ld)] : 0.0;
    }
    __syncthreads();
    for (int rr = 0; rr < rows; ++rr) {
      A xa[U], yb[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int a = tx + 16 * u;
        xa[u] = a < m ? (A)Xs[rr * ld + a] : (A)0;
        const int b = ty + 16 * u;
        yb[u] = b < m ? (A)Ys[rr * ld + b] : (A)0;
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int v = 0; v < U; ++v)
          if (!SYM || u <= v) acc[u][v] = fma(xa[u], yb[v], acc[u][v]);
    }
  }
  double* out = part + (int64_t)blockIdx.x * m * m;
#pragma unroll
  for (int u = 0; u < U; ++u)
#pragma unroll
    for (int v = 0; v < U; ++v) {
      const int a = tx + 16 * u, b = ty + 16 * v;
      if (a < m && b < m && (!SYM || u <= v)) out[a * m + b] = (double)acc[u][v];
    }
}

// sym: entries (a, b) with a / 16 > b / 16 were not computed; take (b, a).
// The partials are added in increasing order with Neumaier's compensated
// summation (A. Neumaier, ZAMM 54, 1974): the rounding error of every
// addition is carried along, so the sum of the CTAs' partials adds about
// two units of rounding instead of one per partial.
__global__ void k_gram_sum(const double* __restrict__ part, int nparts, int m, int sym,
                           double* G) {
  const int mm = m * m;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < mm; e += gridDim.x * blockDim.x) {
    const int a = e / m, b = e - a * m;
    const int src = (sym && (a >> 4) > (b >> 4)) ? b * m + a : e;
    double s = 0.0, c = 0.0;
    for (int p = 0; p < nparts; ++p) {
      const double v = part[(int64_t)p * mm + src];
      const double t = s + v;
      c += fabs(s) >= fabs(v) ? (s - t) + v : (v - t) + s;
      s = t;
    }
    G[e] = s + c;
  }
}

int gram_parts(int num_sms) { return 2 * num_sms; }

void gram_sum(const double* part, int parts, int m, bool sym, double* G, cudaStream_t s) {
  k_gram_sum<<<(m * m + 255) / 256, 256, 0, s>>>(part, parts, m, sym ? 1 : 0, G);
  RF_LAUNCH();
}

template <bool SYM, typename A = double>
static void gram_partials(const double* X, const double* Y, int64_t n, int m, int ld,
                          double* partial, int parts, size_t smem, cudaStream_t s) {
  switch ((m + 15) / 16) {
#define RF_GRAM(UU)                                                                      \
  case UU:                                                                               \
    ensure_dyn_smem(reinterpret_cast<const void*>(k_gram_partial<UU, SYM, A>), smem);   \
    k_gram_partial<UU, SYM, A><<<parts, 256, smem, s>>>(X, Y, n, m, ld, partial);        \
    break;
    RF_GRAM(1) RF_GRAM(2) RF_GRAM(3) RF_GRAM(4) RF_GRAM(5) RF_GRAM(6) RF_GRAM(7) RF_GRAM(8)
#undef RF_GRAM
    default: throw Err{RAFEAST_ERR_INVALID_ARG};
  }
}

void gram(const double* X, const double* Y, int64_t n, int m, int ld, double* G,
          double* partial, int num_sms, cudaStream_t s, bool sym, bool f32) {
  const int parts = gram_parts(num_sms);
  const size_t smem = 2 * GRAM_RB * (size_t)ld * sizeof(double);
  if (f32) {
    // only the symmetric X^T X of a preconditioning pass is formed in float
    if (!sym) throw Err{RAFEAST_ERR_INVALID_ARG};
    gram_partials<true, float>(X, Y, n, m, ld, partial, parts, smem, s);
  } else if (sym) {
    gram_partials<true>(X, Y, n, m, ld, partial, parts, smem, s);
  } else {
    gram_partials<false>(X, Y, n, m, ld, partial, parts, smem, s);
  }
  RF_LAUNCH();
  k_gram_sum<<<(m * m + 255) / 256, 256, 0, s>>>(partial, parts, m, sym ? 1 : 0, G);
  RF_LAUNCH();
}

// ---------------------------------------------------------------------------
// tall GEMM: Y[r][b] = sum_a X[r][a] M[a][b]   (M row-major m x mo)
// ---------------------------------------------------------------------------
// A row of Y is computed by L = ceil(mo / V) threads, V columns each
// (b = lane + L v), so that few lanes idle when mo is not a multiple of 32
// (mo = 80: 27 lanes, 81 slots); a CTA of 256 threads takes 256 / L rows
// (at most GEMM_MAX_ROWS) per tile. Rows of a tile may straddle warps.
constexpr int GEMM_MAX_ROWS = 32;

// UPPER: M is upper triangular (M[a][b] = 0 for a > b): column block v
// (b < L v + L) needs rows a < L v + L only, a bound shared by the row's lanes
template <int V, bool UPPER>
__global__ void __launch_bounds__(256) k_tall_gemm(const double* __restrict__ X, int64_t n, int m,
                                                   int ldx, const double* __restrict__ M, int mo,
                                                   double* __restrict__ Y, int ldy) {
  extern __shared__ double tsm[];
  const int L = (mo + V - 1) / V;
  const int rpt = min(GEMM_MAX_ROWS, (int)blockDim.x / L);  // rows per tile
  double* Ms = tsm;              // m * mo
  double* Xs = tsm + m * mo;     // rpt * m
  for (int t = threadIdx.x; t < m * mo; t += blockDim.x) Ms[t] = M[t];
  const int tr = threadIdx.x / L, tc = threadIdx.x - (threadIdx.x / L) * L;
  for (int64_t rb = blockIdx.x * (int64_t)rpt; rb < n; rb += (int64_t)gridDim.x * rpt) {
    __syncthreads();
    const int rows = (int)min((int64_t)rpt, n - rb);
    for (int t = threadIdx.x; t < rpt * m; t += blockDim.x) {
      const int rr = t / m;
      Xs[t] = rr < rows ? X[(rb + rr) * ldx + (t - rr * m)] : 0.0;
    }
    __syncthreads();
    if (tr < rows) {
      double acc[V];
#pragma unroll
      for (int v = 0; v < V; ++v) acc[v] = 0.0;
      for (int a = 0; a < m; ++a) {
        const double x = Xs[tr * m + a];
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const int b = tc + L * v;
          if (UPPER && a >= L * v + L) continue;
          if (b < mo) acc[v] = fma(x, Ms[a * mo + b], acc[v]);
        }
      }
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const int b = tc + L * v;
        if (b < mo) Y[(rb + tr) * ldy + b] = acc[v];
      }
    }
  }
}

void tall_gemm(const double* X, int64_t n, int m, int ldx, const double* M, int mo, double* Y,
               int ldy, cudaStream_t s, bool upper) {
  const int V = (mo + 31) / 32;
  const int L = (mo + V - 1) / V;
  const int rpt = std::min(GEMM_MAX_ROWS, 256 / L);
  const size_t smem = ((size_t)m * mo + (size_t)rpt * m) * sizeof(double);
  int dev = 0, sms = 0;
  RF_CUDA(cudaGetDevice(&dev));
  RF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int64_t tiles = (n + rpt - 1) / rpt;
  int blocks = (int)std::min<int64_t>(tiles, (int64_t)sms * 2);
  if (blocks < 1) blocks = 1;
  switch (V) {
#define RF_TG(VV)                                                                     \
  case VV:                                                                            \
    if (upper) {                                                                      \
      ensure_dyn_smem(reinterpret_cast<const void*>(k_tall_gemm<VV, true>), smem);   \
      k_tall_gemm<VV, true><<<blocks, 256, smem, s>>>(X, n, m, ldx, M, mo, Y, ldy);   \
    } else {                                                                          \
      ensure_dyn_smem(reinterpret_cast<const void*>(k_tall_gemm<VV, false>), smem);  \
      k_tall_gemm<VV, false><<<blocks, 256, smem, s>>>(X, n, m, ldx, M, mo, Y, ldy);  \
    }                                                                                 \
    break;
    RF_TG(1) RF_TG(2) RF_TG(3) RF_TG(4)
#undef RF_TG
    default: throw Err{RAFEAST_ERR_INVALID_ARG};
  }
  RF_LAUNCH();
}

// ---------------------------------------------------------------------------
// one-CTA Cholesky (+shift) and triangular inverse
// G: m x m (row-major, symmetric). Outputs R (upper, G = R^T R, row-major) and
// Rinv (upper, row-major); status: 0 ok, 1 shifted, 2 failed.
// ---------------------------------------------------------------------------
__device__ bool chol_inplace(double* S, int m) {
  __shared__ int s_bad;
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  for (int k = 0; k < m; ++k) {
    if (threadIdx.x == 0) {
      const double d = S[k * m + k];
      if (!(d > 0.0) || !isfinite(d)) s_bad = 1;
      else S[k * m + k] = sqrt(d);
    }
    __syncthreads();
    if (s_bad) return false;
    const double dk = S[k * m + k];
    for (int i = k + 1 + threadIdx.x; i < m; i += blockDim.x) S[i * m + k] /= dk;
    __syncthreads();
    const int rem = m - k - 1;
    const int tot = rem * rem;
    for (int t = threadIdx.x; t < tot; t += blockDim.x) {
      const int i = k + 1 + t / rem, j = k + 1 + t % rem;
      if (j <= i) S[i * m + j] -= S[i * m + k] * S[j * m + k];
    }
    __syncthreads();
  }
  return true;
}

__global__ void k_chol_inv(const double* __restrict__ G, int m, double shift_scale,
                           double* __restrict__ R, double* __restrict__ Rinv, int* status,
                           int check_id) {
  extern __shared__ double S[];  // m*m
  __shared__ double s_shift;
  __shared__ int s_far;
  if (threadIdx.x == 0) s_far = 0;
  __syncthreads();
  for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
    S[t] = G[t];
    // check_id: G is the Gram of a block that should be close to orthonormal;
    // flag (status bit 4) when an entry is off the identity by more than 1/4
    if (check_id && fabs(G[t] - ((t / m == t % m) ? 1.0 : 0.0)) > 0.25) s_far = 1;
  }
  __syncthreads();
  int st = 0;
  bool ok = chol_inplace(S, m);
  if (!ok) {
    // shifted Cholesky-QR: s = 11 (n m + m (m + 1)) u ||X||_2^2, ||X||_2^2 <= trace(G)
    if (threadIdx.x == 0) {
      double tr = 0.0;
      for (int i = 0; i < m; ++i) tr += fabs(G[i * m + i]);
      s_shift = shift_scale * tr;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
      const int i = t / m, j = t % m;
      S[t] = G[t] + (i == j ? s_shift : 0.0);
    }
    __syncthreads();
    ok = chol_inplace(S, m);
    st = ok ? 1 : 2;
  }
  if (!ok) {
    if (threadIdx.x == 0) status[0] = 2;
    return;
  }
  // R = L^T (upper)
  for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
    const int i = t / m, j = t % m;
    R[t] = j >= i ? S[j * m + i] : 0.0;
  }
  // Linv by forward substitution, one column per thread; Rinv = Linv^T
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    for (int i = 0; i < m; ++i) {
      double x;
      if (i < j) {
        x = 0.0;
      } else {
        double acc = (i == j) ? 1.0 : 0.0;
        for (int k = j; k < i; ++k) acc -= S[i * m + k] * Rinv[j * m + k];
        x = acc / S[i * m + i];
      }
      Rinv[j * m + i] = x;  // row j of Rinv holds column j of Linv^T... see below
    }
  }
  __syncthreads();
  // Rinv currently holds Linv^T stored as Rinv[j][i] = Linv[i][j] = (Linv^T)[j][i]
  if (threadIdx.x == 0) status[0] = st | (s_far ? 4 : 0);
}

void chol_inv(double* G, int m, int64_t nrows, double* Rfac, double* Rinv, int* status,
              cudaStream_t s, bool check_id) {
  const size_t smem = (size_t)m * m * sizeof(double);
  ensure_dyn_smem(reinterpret_cast<const void*>(k_chol_inv), smem);
  const double u = DBL_EPSILON / 2;
  const double scale = 11.0 * ((double)nrows * m + (double)m * (m + 1)) * u;
  k_chol_inv<<<1, 256, smem, s>>>(G, m, scale, Rfac, Rinv, status, check_id ? 1 : 0);
  RF_LAUNCH();
}

// ---------------------------------------------------------------------------
// one-CTA cyclic Jacobi (round-robin parallel order), in precision T
// ---------------------------------------------------------------------------
constexpr size_t JACOBI_SMEM_MAX = 216 * 1024;  // A and V in shared memory up to this size

// A (m x m, ld m, symmetric part taken) -> eigenvalues ascending in w, the
// matching eigenvectors as the columns of Vout (m x m, ld m). A pair (p, q)
// is rotated while |a_pq| > rot_tol sqrt(|a_pp a_qq|); the sweeps end when
// the off-diagonal mass is below off_tol of the total or a sweep rotated
// nothing. Vg: global fallback for the eigenvector accumulator (me * me).
template <typename T>
__global__ void k_jacobi(const double* __restrict__ Ain, int m, double* __restrict__ w,
                         double* __restrict__ Vout, T* __restrict__ Vg, int max_sweeps,
                         double rot_tol, double off_tol) {
  extern __shared__ unsigned char jsm[];
  T* A = reinterpret_cast<T*>(jsm);  // me * me (+ me * me for V when it fits)
  const int me = m + (m & 1);
  // the eigenvector accumulator in shared memory when both fit, else in the
  // global work buffer
  T* Vw = (2 * (size_t)me * me * sizeof(T) <= JACOBI_SMEM_MAX) ? A + me * me : Vg;
  __shared__ T cs[64 * 2];  // c, s per pair (me/2 <= 64)
  __shared__ int pq[64 * 2];
  __shared__ double s_off, s_tot;
  __shared__ double s_woff[32], s_wtot[32];  // per-warp sums, added in warp order
  __shared__ int s_order[128];
  __shared__ int s_rot;
  const T tiny = sizeof(T) == 4 ? (T)1e-37 : (T)1e-300;
  for (int t = threadIdx.x; t < me * me; t += blockDim.x) {
    const int i = t / me, j = t % me;
    A[t] = (i < m && j < m) ? (T)(0.5 * (Ain[i * m + j] + Ain[j * m + i])) : (T)0;
    Vw[t] = (i == j) ? (T)1 : (T)0;
  }
  __syncthreads();
  const int np = me / 2;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    // convergence test on the off-diagonal mass
    if (threadIdx.x == 0) {
      s_off = 0.0;
      s_tot = 0.0;
      s_rot = 0;
    }
    __syncthreads();
    double off = 0.0, tot = 0.0;
    for (int t = threadIdx.x; t < me * me; t += blockDim.x) {
      const int i = t / me, j = t % me;
      const double a2 = (double)A[t] * (double)A[t];
      tot += a2;
      if (i != j) off += a2;
    }
    off = warp_sum(off);
    tot = warp_sum(tot);
    if ((threadIdx.x & 31) == 0) {
      s_woff[threadIdx.x >> 5] = off;
      s_wtot[threadIdx.x >> 5] = tot;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double so = 0.0, st = 0.0;
      for (int wi = 0; wi < (int)(blockDim.x >> 5); ++wi) {
        so += s_woff[wi];
        st += s_wtot[wi];
      }
      s_off = so;
      s_tot = st;
    }
    __syncthreads();
    if (!(s_off > off_tol * s_tot) || s_tot == 0.0) break;
    for (int round = 0; round < me - 1; ++round) {
      for (int k = threadIdx.x; k < np; k += blockDim.x) {
        // circle method: position 0 fixed, others rotate
        auto player = [&](int pos) { return pos == 0 ? 0 : ((pos - 1 + round) % (me - 1)) + 1; };
        int p = player(k), q = player(me - 1 - k);
        if (p > q) {
          const int t = p;
          p = q;
          q = t;
        }
        const T apq = A[p * me + q];
        T c = (T)1, s = (T)0;
        const T app = A[p * me + p], aqq = A[q * me + q];
        if (apq != (T)0 && fabs(apq) > tiny && fabs(apq) > (T)rot_tol * sqrt(fabs(app * aqq))) {
          s_rot = 1;
          const T tau = (aqq - app) / ((T)2 * apq);
          const T at = fabs(tau);
          const T root = at > (T)1e15 ? at : sqrt((T)1 + tau * tau);
          const T t = (tau >= (T)0 ? (T)1 : (T)-1) / (at + root);
          c = (T)1 / sqrt((T)1 + t * t);
          s = t * c;
        }
        cs[2 * k] = c;
        cs[2 * k + 1] = s;
        pq[2 * k] = p;
        pq[2 * k + 1] = q;
      }
      __syncthreads();
      // the pairs of a round are disjoint, so every 2 x 2 block (rows of
      // pair j, columns of pair k) is updated on its own from its old
      // values: B <- L_j B R_k with L = [[c, -s], [s, c]], R = L^T; the
      // rotated diagonal blocks lose their off-diagonal entry
      for (int t = threadIdx.x; t < np * np; t += blockDim.x) {
        const int j = t / np, k = t % np;
        const T cj = cs[2 * j], sj = cs[2 * j + 1];
        const T ck = cs[2 * k], sk = cs[2 * k + 1];
        if (sj == (T)0 && sk == (T)0) continue;
        const int pj = pq[2 * j], qj = pq[2 * j + 1];
        const int pk = pq[2 * k], qk = pq[2 * k + 1];
        const T a11 = A[pj * me + pk], a12 = A[pj * me + qk];
        const T a21 = A[qj * me + pk], a22 = A[qj * me + qk];
        // rows: L_j B
        const T b11 = cj * a11 - sj * a21, b12 = cj * a12 - sj * a22;
        const T b21 = sj * a11 + cj * a21, b22 = sj * a12 + cj * a22;
        // columns: (L_j B) R_k
        A[pj * me + pk] = ck * b11 - sk * b12;
        A[pj * me + qk] = j == k ? (T)0 : sk * b11 + ck * b12;
        A[qj * me + pk] = j == k ? (T)0 : ck * b21 - sk * b22;
        A[qj * me + qk] = sk * b21 + ck * b22;
      }
      // V R_k
      for (int t = threadIdx.x; t < np * me; t += blockDim.x) {
        const int k = t / me, row = t % me;
        const T c = cs[2 * k], s = cs[2 * k + 1];
        if (s == (T)0) continue;
        const int p = pq[2 * k], q = pq[2 * k + 1];
        const T vp = Vw[row * me + p], vq = Vw[row * me + q];
        Vw[row * me + p] = c * vp - s * vq;
        Vw[row * me + q] = s * vp + c * vq;
      }
      __syncthreads();
    }
    if (s_rot == 0) break;  // nothing was above the threshold in this sweep
    __syncthreads();
  }
  // sort eigenvalues ascending (m <= 128), then write w and V columns
  if (threadIdx.x == 0) {
    for (int i = 0; i < m; ++i) s_order[i] = i;
    for (int i = 1; i < m; ++i) {
      const int key = s_order[i];
      const T kv = A[key * me + key];
      int j = i - 1;
      while (j >= 0 && A[s_order[j] * me + s_order[j]] > kv) {
        s_order[j + 1] = s_order[j];
        --j;
      }
      s_order[j + 1] = key;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < m; i += blockDim.x) w[i] = (double)A[s_order[i] * me + s_order[i]];
  for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
    const int r = t / m, c = t % m;
    Vout[r * m + c] = (double)Vw[r * me + s_order[c]];
  }
}

// small dense product, all m x m row-major: C = alpha op(A) op(B) + gamma I,
// op = transpose when the flag is set; one thread per entry of C
__global__ void k_small_gemm(const double* __restrict__ A, int ta, const double* __restrict__ B,
                             int tb, double* __restrict__ C, int m, double alpha, double gamma) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m * m) return;
  const int i = e / m, j = e - (e / m) * m;
  double acc = 0.0;
  for (int k = 0; k < m; ++k) {
    const double a = ta ? A[k * m + i] : A[i * m + k];
    const double b = tb ? B[j * m + k] : B[k * m + j];
    acc = fma(a, b, acc);
  }
  C[e] = alpha * acc + (i == j ? gamma : 0.0);
}

void small_gemm(const double* A, int ta, const double* B, int tb, double* C, int m, double alpha,
                double gamma, cudaStream_t s) {
  k_small_gemm<<<(m * m + 127) / 128, 128, 0, s>>>(A, ta, B, tb, C, m, alpha, gamma);
  RF_LAUNCH();
}

template <typename T>
static void jacobi_launch(const double* A, int m, double* w, double* V, T* Vg, int sweeps,
                          double rot_tol, double off_tol, cudaStream_t s) {
  const int me = m + (m & 1);
  size_t smem = (size_t)me * me * sizeof(T);
  if (2 * smem <= JACOBI_SMEM_MAX) smem *= 2;  // V beside A
  ensure_dyn_smem(reinterpret_cast<const void*>(k_jacobi<T>), smem);
  k_jacobi<T><<<1, 1024, smem, s>>>(A, m, w, V, Vg, sweeps, rot_tol, off_tol);
  RF_LAUNCH();
}

// Mixed-precision Jacobi. GB300's FP64 rate is a small fraction of its FP32
// rate, and a one-CTA Jacobi on an 80 x 80 matrix is bound by one SM's FP64
// issue. So: (1) float Jacobi to the float rounding floor gives V1 with
// V1^T A V1 diagonal to ~1e-7; (2) two Newton-Schulz steps
// V <- V (3 I - V^T V) / 2 make V1 orthonormal to working precision (its
// float error is ~1e-6, each step squares it); (3) the FP64 Jacobi on
// B = V^T A V, already nearly diagonal, needs a few sweeps; (4) V = V1 V_B.
// The final accuracy is that of the FP64 Jacobi, as with FP64 alone.
void jacobi_eigh(double* A, int m, double* w, double* V, double* work, cudaStream_t s) {
  if (m > 128) throw Err{RAFEAST_ERR_INVALID_ARG};
  const int me = m + (m & 1);
  const size_t mm = (size_t)me * me;
  double* W1 = work;
  double* W2 = work + mm;
  double* S = work + 2 * mm;
  double* B = work + 3 * mm;
  double* VB = work + 4 * mm;
  double* Vg = work + 5 * mm;  // also the float stage's fallback accumulator
  jacobi_launch<float>(A, m, w, W1, reinterpret_cast<float*>(Vg), 30, 1e-6, 1e-13, s);
  for (int it = 0; it < 2; ++it) {
    small_gemm(W1, 1, W1, 0, S, m, -0.5, 1.5, s);  // S = (3 I - V^T V) / 2
    small_gemm(W1, 0, S, 0, W2, m, 1.0, 0.0, s);   // V <- V S
    std::swap(W1, W2);
  }
  small_gemm(A, 0, W1, 0, S, m, 1.0, 0.0, s);  // A V
  small_gemm(W1, 1, S, 0, B, m, 1.0, 0.0, s);  // V^T A V
  jacobi_launch<double>(B, m, w, VB, Vg, 40, 1e-17, 1e-32, s);
  small_gemm(W1, 0, VB, 0, V, m, 1.0, 0.0, s);  // V1 V_B
}

// ---------------------------------------------------------------------------
// column reductions over rows
// mode 0: out[i] = sum_r X[r][i] Y[r][i];  mode 1: out[i] = sum_r (Y - th_i X)^2
// Block b sums the rows b, b + B, b + 2B, ... of every column into part[b];
// a second kernel adds the B partial sums of each column in increasing b, so
// the result does not depend on the order in which blocks run.
// ---------------------------------------------------------------------------
__global__ void k_colred(const double* __restrict__ X, const double* __restrict__ Y,
                         const double* __restrict__ th, int64_t n, int m, int ld, int mode,
                         double* part) {
  const int i = threadIdx.x;
  if (i >= m) return;
  const double t = mode ? th[i] : 0.0;
  double acc = 0.0;
  for (int64_t r = blockIdx.x; r < n; r += gridDim.x) {
    const double x = X[r * ld + i], y = Y[r * ld + i];
    if (mode) {
      const double d = y - t * x;
      acc = fma(d, d, acc);
    } else {
      acc = fma(x, y, acc);
    }
  }
  part[(int64_t)blockIdx.x * m + i] = acc;
}

__global__ void k_colsum(const double* __restrict__ part, int nparts, int m, double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  double s = 0.0;
  for (int b = 0; b < nparts; ++b) s += part[(int64_t)b * m + i];
  out[i] = s;
}

static void colred(const double* X, const double* Y, const double* th, int64_t n, int m, int ld,
                   int mode, double* out, double* part, int num_sms, cudaStream_t s) {
  const int threads = ((m + 31) / 32) * 32;
  const int blocks = (int)std::min<int64_t>(n, 2 * (int64_t)num_sms);
  k_colred<<<blocks, threads, 0, s>>>(X, Y, th, n, m, ld, mode, part);
  RF_LAUNCH();
  k_colsum<<<(m + 127) / 128, 128, 0, s>>>(part, blocks, m, out);
  RF_LAUNCH();
}

void col_dot(const double* X, const double* Y, int64_t n, int m, int ld, double* out,
             double* part, int num_sms, cudaStream_t s) {
  colred(X, Y, nullptr, n, m, ld, 0, out, part, num_sms, s);
}

void col_resid2(const double* Q, const double* AQ, const double* theta, int64_t n, int m, int ld,
                double* out, double* part, int num_sms, cudaStream_t s) {
  colred(Q, AQ, theta, n, m, ld, theta ? 1 : 0, out, part, num_sms, s);
}

// ---------------------------------------------------------------------------
// quadrature combine: Qt = f_i Q + D
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_combine(const double* __restrict__ Q, int ldq, const T* __restrict__ D, int ldd,
                          const double* __restrict__ f, int64_t n, int m, double* __restrict__ Qt) {
  const int64_t total = n * (int64_t)m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / m;
    const int i = (int)(e - r * m);
    Qt[r * ldq + i] = fma(f[i], Q[r * ldq + i], (double)D[r * ldd + i]);
  }
}

template <typename T>
void launch_combine(const double* Q, int ldq, const T* D, int ldd, const double* f, int64_t n,
                    int m, double* Qt, cudaStream_t s) {
  k_combine<T><<<blocks_for(n * (int64_t)m), 256, 0, s>>>(Q, ldq, D, ldd, f, n, m, Qt);
  RF_LAUNCH();
}
template void launch_combine<float>(const double*, int, const float*, int, const double*, int64_t,
                                    int, double*, cudaStream_t);
template void launch_combine<double>(const double*, int, const double*, int, const double*,
                                     int64_t, int, double*, cudaStream_t);

}  // namespace rafeast
