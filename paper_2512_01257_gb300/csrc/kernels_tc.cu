// FP64 Gram matrices G = X^T Y on the tensor cores (tcgen05, sm_103a), by
// splitting FP64 values into exact BF16 digits (the error-free splitting of
// Ozaki, Ogita, Oishi and Rump, "Error-free transformations of matrix
// multiplication by using fast routines of matrix multiplication and its
// applications", Numer. Algorithms 59, 2012).
//
// The Gram matrices of the Cholesky-QR and Rayleigh-Ritz steps (Algorithm 1)
// are n x m by n x m contractions with n up to 10^6 and m <= 128. On this part
// the FP64 pipe issues 2 operations per SM per clock; the BF16 tensor cores do
// several thousand. So:
//
// 1. Scaling. A CTA owns a range of rows. For every column of X (and of Y)
//    it takes the largest binary exponent over its rows, E, so that every
//    value of the column is below 2^E in magnitude, and writes each value as
//    the integer F = round(x 2^(55-E)), |F| <= 2^55 (the value to 2^-55
//    relative to the column's largest; integer operations only).
// 2. Digits. F = sum_{i=0..6} d_i 2^(8 (6-i)) with balanced digits
//    d_i in [-128, 128] (a carry moves every digit of 128 or more up), each
//    exact in BF16.
// 3. Products. x_a y_b = 2^(Ea+Eb-14) sum_{i,j} d_i d_j 2^(-8 (i+j)). The
//    pairs with i + j = l form level l; levels 0..6 are kept (the next would
//    change the result by 2^-56 of sum_k |x_ka y_kb|). A level is one TMEM
//    accumulator of FP32: its 28 pairs are 28 tcgen05.mma (M = 128 rows a,
//    N <= 64 columns b, K = 16 rows k) per 16 rows of X.
// 4. Exactness. A product of two digits is an integer of at most 2^14 and
//    level l adds l + 1 of them per row, so over 128 rows levels 0..3 stay
//    integers of magnitude <= 2^23 and FP32 holds them exactly. Every 128
//    rows those four levels are read out of TMEM and added, as one integer
//    sum_{l<=3} S_l 2^(8 (3-l)), into a 64-bit integer per entry; the next
//    MMAs restart them. Levels 4..6 keep accumulating in FP32 over the CTA's
//    rows: their rounding is below 2^-24 of terms that are themselves below
//    2^-32 of the result.
// 5. The CTA's partial Gram is (I + L 2^-8) 2^(Ea+Eb-38), I the integer and
//    L = S_4 + S_5 2^-8 + S_6 2^-16; the partials of all CTAs are added in a
//    fixed order (k_gram_sum), so the result does not depend on scheduling.
//
// Operands are staged in shared memory in the canonical K-major layout
// without swizzle (core matrices of 8 rows x 16 bytes; the descriptor's
// leading offset is the step between the two 8-element halves of a 16-wide
// K slice, its stride offset the step between 8-row groups), two buffers of
// 32 rows each: the digits of the next 32 rows are formed while the tensor
// cores multiply the last ones. One thread issues the MMAs and commits them
// to an mbarrier per buffer; every wait on it is bounded.
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace rafeast {

namespace {

constexpr int TC_THREADS = 256;
constexpr int TC_M = 128;               // MMA rows: Gram rows a (m <= 128)
constexpr int TC_KS = 32;               // rows of X per sub-chunk (two K = 16 steps)
constexpr int TC_SUB_PER_CHUNK = 4;     // sub-chunks per exact chunk (128 rows)
constexpr int TC_NB = 64;               // most Gram columns b per CTA
constexpr int TC_LEV = 7;               // levels kept (digit pairs with i + j <= 6)
constexpr int TC_DIG = 7;               // digits per value
constexpr uint32_t TC_LBO = 128;        // byte step between the two K halves of a K = 16 slice
constexpr uint32_t TC_SBO = 512;        // byte step between 8-row groups (32 rows of K = 4 cores)
constexpr int TC_APLANE = TC_M * TC_KS * 2;   // bytes of one digit plane of X^T (8 KB)
constexpr int TC_BPLANE = TC_NB * TC_KS * 2;  // bytes of one digit plane of Y^T (4 KB)
constexpr long long TC_WAIT = 200000000;      // bounded mbarrier polls (~ seconds)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// byte offset of (row r, k) in a K-major plane of 32 K columns
__device__ __forceinline__ uint32_t tc_off(int r, int k) {
  return (uint32_t)((r & 7) * 16 + (k & 7) * 2 + (k >> 3) * 128 + (r >> 3) * TC_SBO);
}

// shared-memory matrix descriptor: start, leading and stride byte offsets,
// descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((TC_LBO >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((TC_SBO >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N = n columns, M = 128
__device__ __forceinline__ uint32_t tc_idesc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(TC_M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tc_commit(uint64_t* mbar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(mbar))
      : "memory");
}

// bounded wait for phase `parity` of an mbarrier; false when it ran out
__device__ __forceinline__ bool tc_wait(uint64_t* mbar, uint32_t parity) {
  uint32_t done = 0;
  for (long long it = 0; it < TC_WAIT && !done; ++it)
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(mbar)), "r"(parity)
        : "memory");
  return done != 0;
}

// 8 FP32 columns of TMEM for this warp's 32 lanes
__device__ __forceinline__ void tc_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(taddr));
#pragma unroll
  for (int t = 0; t < 8; ++t) v[t] = __uint_as_float(r[t]);
}
__device__ __forceinline__ void tc_ld_wait() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// F = round(x 2^(55 - E)), E = ebias - 1022 for ebias the largest biased
// exponent of the column (|x| < 2^E); integer operations only
__device__ __forceinline__ long long tc_fixed(double x, int ebias) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF);
  if (e == 0) return 0;  // zero, or below 2^-1022
  const long long mant = (long long)((b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull);
  const int sh = e - ebias + 2;  // x = mant 2^(e-1075): F = mant 2^(e - 1075 + 55 - E)
  long long F;
  if (sh >= 0) F = mant << sh;  // sh <= 2: F < 2^55
  else if (sh > -54) F = (mant + (1ll << (-sh - 1))) >> (-sh);
  else F = 0;
  return (b >> 63) ? -F : F;
}

// balanced base-256 digits of |F| <= 2^55, d[0] most significant: the bytes
// of the two's complement, low to high, each moved into [-128, 128) by a
// carry into the next (32-bit operations on the two halves of F)
__device__ __forceinline__ void tc_digits(long long F, int (&d)[TC_DIG]) {
  const unsigned lo = (unsigned)(unsigned long long)F;
  const int hi = (int)(F >> 32);
  int c = 0;
#pragma unroll
  for (int i = TC_DIG - 1; i >= 3; --i) {
    const int v = (int)((lo >> (8 * (TC_DIG - 1 - i))) & 255u) + c;
    c = v >= 128;
    d[i] = v - (c << 8);
  }
#pragma unroll
  for (int i = 2; i >= 1; --i) {
    const int v = (int)(((unsigned)hi >> (8 * (2 - i))) & 255u) + c;
    c = v >= 128;
    d[i] = v - (c << 8);
  }
  d[0] = (hi >> 16) + c;
}

// two values at consecutive k of one row into the 7 digit planes (one 32-bit
// store per plane)
__device__ __forceinline__ void tc_store_pair(unsigned char* planes, int plane_bytes,
                                              uint32_t off, long long F0, long long F1) {
  int d0[TC_DIG], d1[TC_DIG];
  tc_digits(F0, d0);
  tc_digits(F1, d1);
#pragma unroll
  for (int i = 0; i < TC_DIG; ++i) {
    const __nv_bfloat162 p = __floats2bfloat162_rn((float)d0[i], (float)d1[i]);
    *reinterpret_cast<__nv_bfloat162*>(planes + i * plane_bytes + off) = p;
  }
}

// G partial of one CTA: rows [k_lo, k_hi) of X and Y, Gram rows a < m (all),
// Gram columns b0 .. b0 + nb (nb a multiple of 16, <= 64). SYM: Y == X, the
// B operand is read from X's digit planes.
template <bool SYM>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_tc_gram(const double* __restrict__ X, const double* __restrict__ Y, int64_t n, int m,
              int ld, int nb, double* __restrict__ part, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char tsm[];
  constexpr int BUF = TC_DIG * TC_APLANE + (SYM ? 0 : TC_DIG * TC_BPLANE);
  __shared__ int sEa[TC_M], sEb[TC_NB];
  __shared__ uint32_t s_tbase;
  __shared__ __align__(8) uint64_t s_mbar[2];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int b0 = blockIdx.y * nb;
  const int64_t k_lo = n * (int64_t)blockIdx.x / gridDim.x;
  const int64_t k_hi = n * (int64_t)(blockIdx.x + 1) / gridDim.x;
  // column exponents over this CTA's rows
  for (int t = tid; t < TC_M; t += TC_THREADS) sEa[t] = 0;
  for (int t = tid; t < TC_NB; t += TC_THREADS) sEb[t] = 0;
  __syncthreads();
  {
    const int a = tid & (TC_M - 1);
    int e = 0;
    if (a < m)
      for (int64_t r = k_lo + (tid >> 7); r < k_hi; r += 2)
        e = max(e, (int)(((unsigned long long)__double_as_longlong(X[r * ld + a]) >> 52) & 0x7FF));
    atomicMax(&sEa[a], e);
    if (!SYM) {
      const int b = tid & (TC_NB - 1);
      int f = 0;
      if (b < nb && b0 + b < m)
        for (int64_t r = k_lo + (tid >> 6); r < k_hi; r += 4)
          f = max(f, (int)(((unsigned long long)__double_as_longlong(Y[r * ld + b0 + b]) >> 52) &
                           0x7FF));
      atomicMax(&sEb[b], f);
    }
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&s_tbase)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_mbar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_mbar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tbase = s_tbase;
  const uint32_t idesc = tc_idesc(nb);
  // readout mapping: lane row a, half h of the nb columns
  const int ra = 32 * (warp & 3) + lane;
  const int h = warp >> 2, nh = nb >> 1;
  const uint32_t trow = tbase + ((uint32_t)(32 * (warp & 3)) << 16);
  long long acc[TC_NB / 2];
#pragma unroll
  for (int c = 0; c < TC_NB / 2; ++c) acc[c] = 0;
  bool ok = true;
  // levels 0..3 of the finished chunk into the integer sums
  auto read_exact = [&]() {
#pragma unroll
    for (int l = 0; l < 4; ++l) {
#pragma unroll
      for (int c8 = 0; c8 < TC_NB / 2; c8 += 8) {
        if (c8 < nh) {
          float v[8];
          tc_ld8(trow + l * nb + h * nh + c8, v);
          tc_ld_wait();
#pragma unroll
          for (int t = 0; t < 8; ++t) acc[c8 + t] += __float2ll_rn(v[t]) * (1ll << (8 * (3 - l)));
        }
      }
    }
  };
  const int64_t rows = k_hi - k_lo;
  const int nsub = (int)((rows + TC_KS - 1) / TC_KS);
  for (int s = 0; s < nsub && ok; ++s) {
    const int buf = s & 1;
    unsigned char* A = tsm + buf * BUF;
    unsigned char* B = A + TC_DIG * TC_APLANE;
    // (every wait's outcome is made CTA-uniform before anyone acts on it)
    if (s >= 2) ok = __syncthreads_and(tc_wait(&s_mbar[buf], ((s - 2) >> 1) & 1));
    if (!ok) break;
    // digits of rows k_lo + 32 s .. + 32 (zero past k_hi and for a >= m);
    // every load of the sub-chunk is issued before any digit is formed
    const int64_t rbase = k_lo + (int64_t)s * TC_KS;
    {
      const int a = tid & (TC_M - 1);
      const int eb = sEa[a];
      double xv[TC_KS / 2];
#pragma unroll
      for (int q = 0; q < TC_KS / 4; ++q) {
        const int kp = (tid >> 7) + 2 * q;
        const int64_t r = rbase + 2 * kp;
        xv[2 * q] = (a < m && r < k_hi) ? X[r * ld + a] : 0.0;
        xv[2 * q + 1] = (a < m && r + 1 < k_hi) ? X[(r + 1) * ld + a] : 0.0;
      }
#pragma unroll
      for (int q = 0; q < TC_KS / 4; ++q) {
        const int kp = (tid >> 7) + 2 * q;
        tc_store_pair(A, TC_APLANE, tc_off(a, 2 * kp), tc_fixed(xv[2 * q], eb),
                      tc_fixed(xv[2 * q + 1], eb));
      }
    }
    if (!SYM) {
      const int b = tid & (TC_NB - 1);
      const int eb = sEb[b];
      const bool on = b < nb && b0 + b < m;
      double yv[TC_KS / 4];
#pragma unroll
      for (int q = 0; q < TC_KS / 8; ++q) {
        const int kp = (tid >> 6) + 4 * q;
        const int64_t r = rbase + 2 * kp;
        yv[2 * q] = (on && r < k_hi) ? Y[r * ld + b0 + b] : 0.0;
        yv[2 * q + 1] = (on && r + 1 < k_hi) ? Y[(r + 1) * ld + b0 + b] : 0.0;
      }
      if (b < nb) {
#pragma unroll
        for (int q = 0; q < TC_KS / 8; ++q) {
          const int kp = (tid >> 6) + 4 * q;
          tc_store_pair(B, TC_BPLANE, tc_off(b, 2 * kp), tc_fixed(yv[2 * q], eb),
                        tc_fixed(yv[2 * q + 1], eb));
        }
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    const bool chunk_start = (s % TC_SUB_PER_CHUNK) == 0;
    if (s > 0 && chunk_start) {
      // the previous chunk is complete once the last sub-chunk's MMAs are
      ok = __syncthreads_and(tc_wait(&s_mbar[(s - 1) & 1], ((s - 1) >> 1) & 1));
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (ok) read_exact();
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      if (!ok) break;
    }
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a_base = smem_u32(A);
      const uint32_t b_base = SYM ? a_base + (uint32_t)(b0 >> 3) * TC_SBO : smem_u32(B);
      const int bplane = SYM ? TC_APLANE : TC_BPLANE;
      // descriptors differ only in their start address (16-byte units in the
      // low bits): one base per operand, plane and K-step offsets added
      const uint64_t ad0 = tc_desc(a_base), bd0 = tc_desc(b_base);
#pragma unroll
      for (int ks = 0; ks < TC_KS / 16; ++ks) {
#pragma unroll
        for (int l = 0; l < TC_LEV; ++l) {
          const bool fresh = ks == 0 && (l <= 3 ? chunk_start : s == 0);
#pragma unroll
          for (int i = 0; i <= l; ++i) {
            const int j = l - i;
            const uint64_t ad = ad0 + (uint64_t)((i * TC_APLANE + ks * 256) >> 4);
            const uint64_t bd = bd0 + (uint64_t)((j * bplane + ks * 256) >> 4);
            tc_mma(tbase + l * nb, ad, bd, idesc, (fresh && i == 0) ? 0u : 1u);
          }
        }
      }
      tc_commit(&s_mbar[buf]);
    }
  }
  // the last chunk: levels 0..3 into the integers, levels 4..6 as the
  // correction; the CTA's partial Gram scaled back
  if (ok && nsub > 0) ok = tc_wait(&s_mbar[(nsub - 1) & 1], ((nsub - 1) >> 1) & 1);
  ok = __syncthreads_and(ok);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok && nsub > 0) read_exact();
  const int a = ra;
  double* out = part + (int64_t)blockIdx.x * m * m;
#pragma unroll
  for (int c8 = 0; c8 < TC_NB / 2; c8 += 8) {
    if (c8 < nh) {
      float s4[8], s5[8], s6[8];
      if (ok && nsub > 0) {
        tc_ld8(trow + 4 * nb + h * nh + c8, s4);
        tc_ld8(trow + 5 * nb + h * nh + c8, s5);
        tc_ld8(trow + 6 * nb + h * nh + c8, s6);
        tc_ld_wait();
      }
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int b = b0 + h * nh + c8 + t;
        if (a < m && b < m) {
          double v = ok ? 0.0 : __longlong_as_double(0x7ff8000000000000ll);  // NaN on a timeout
          if (ok && nsub > 0) {
            const float lo = fmaf(s6[t], 0x1p-16f, fmaf(s5[t], 0x1p-8f, s4[t]));
            const int ea = sEa[a], ebb = SYM ? sEa[b] : sEb[h * nh + c8 + t];
            // (I + L 2^-8) 2^(Ea + Eb - 38), Ea = ea - 1022, Eb = eb - 1022
            const int p = ea + ebb - 2044 - 38;
            // two normal powers of two (results below 2^-2044 flush to zero)
            const int p1 = max(-1022, min(1023, p / 2)), p2 = max(-1022, min(1023, p - p / 2));
            v = fma((double)lo, 0x1p-8, (double)acc[c8 + t]);
            v = v * __longlong_as_double((long long)(p1 + 1023) << 52) *
                __longlong_as_double((long long)(p2 + 1023) << 52);
            if (ea == 0 || ebb == 0) v = 0.0;
          }
          out[(int64_t)a * m + b] = v;
        }
      }
    }
  }
  if (!ok && tid == 0 && err) atomicExch(err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(512));
}

// ---------------------------------------------------------------------------
// Tall product Y = X M (n x m times m x mo, m, mo <= 128) on the tensor cores,
// the same exact digit arithmetic with the contraction over the m columns:
//
// 1. Scaling. A CTA owns a range of rows. Column a of X is scaled by 2^-c_a,
//    c_a its largest exponent over those rows, and M's row a by 2^c_a (X M is
//    unchanged, and a small column of X keeps its own relative precision).
//    Row r of the scaled X is then written as integers F = round(x 2^(55-E_r))
//    with E_r its largest exponent, and column b of the scaled M as integers
//    G with its own exponent E_b; both are exact multiples of 2^-55 of their
//    row's or column's largest value.
// 2. Digits and levels as for the Gram: seven balanced base-256 digits per
//    integer, here the 34 digit pairs with i + j <= 7 as tcgen05.mma (M = 128
//    rows r, N = nb <= 64 columns b, K = 16 columns a) into eight FP32 levels
//    of TMEM (8 x 64 columns). With K = m <= 128 a level adds at most
//    7 x 128 products of at most 2^14: every level is an exact integer.
// 3. y_rb = (I + L 2^-8) 2^(E_r + E_b - 38), I = sum_{l<=3} S_l 2^(8 (3-l))
//    (an exact 64-bit integer) and L = S_4 + S_5 2^-8 + S_6 2^-16 + S_7 2^-24
//    (exact in FP64): one rounding to FP64; the dropped pairs (i + j >= 8)
//    change a product by less than 2^-61 of 2^(E_r + E_b), so the error is
//    that of writing the values as integers, 2^-55 of the row's and of the
//    column's largest scaled value per product.
//
// A row of X with a NaN or infinity gives a row of NaN, a column of M with
// one a column of NaN. Operands are staged as in the Gram (K-major, 32-wide K
// slices); the B digits of the CTA's columns are formed once, the A digits of
// the next 32 columns of a 128-row block while the tensor cores multiply the
// last ones.
constexpr int TT_LEV = 8;         // levels kept (digit pairs with i + j <= 7)
constexpr int TT_THREADS = 512;   // 16 warps: four threads per row of a 128-row block
constexpr int TT_NAN_ROW = -1000000;
constexpr int TT_ZERO_ROW = -0x40000000;

__global__ void __launch_bounds__(TT_THREADS, 1)
    k_tc_tall(const double* __restrict__ X, int64_t n, int m, int ldx,
              const double* __restrict__ Mm, int mo, double* __restrict__ Y, int ldy, int nb,
              int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char tsm[];
  constexpr int ABUF = TC_DIG * TC_APLANE;  // one buffer of A digit planes (56 KB)
  const int bpl = nb * 64;                  // bytes of one B digit plane of one K slice
  unsigned char* Bp = tsm + 2 * ABUF;       // [slice][digit] planes
  __shared__ int sCe[TC_M], sFb[TC_NB], sEr[TC_M];
  // the four partial row exponents of a block live in A buffer 0, which no
  // MMA reads while they are formed (the last block's MMAs have completed)
  int (*sEq)[TC_M] = reinterpret_cast<int (*)[TC_M]>(tsm);
  __shared__ uint32_t s_tbase;
  __shared__ __align__(8) uint64_t s_mbar[2];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int b0 = blockIdx.x * nb;
  const int parts = gridDim.y;
  const int64_t r_lo = n * (int64_t)blockIdx.y / parts;
  const int64_t r_hi = n * (int64_t)(blockIdx.y + 1) / parts;
  const int kp16 = (m + 15) & ~15, nsl = (kp16 + 31) / 32;
  // (1) column exponents of X over this CTA's rows (finite values); four
  // threads per column, eight rows in flight each
  for (int t = tid; t < TC_M; t += TT_THREADS) sCe[t] = 0;
  __syncthreads();
  {
    const int a = tid & (TC_M - 1), q4 = tid >> 7;
    int e = 0;
    if (a < m) {
      int64_t r = r_lo + q4;
      for (; r + 28 < r_hi; r += 32) {
        int ex[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
          ex[u] = (int)(((unsigned long long)__double_as_longlong(X[(r + 4 * u) * ldx + a]) >> 52) & 0x7FF);
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (ex[u] != 0x7FF) e = max(e, ex[u]);
      }
      for (; r < r_hi; r += 4) {
        const int ex = (int)(((unsigned long long)__double_as_longlong(X[r * ldx + a]) >> 52) & 0x7FF);
        if (ex != 0x7FF) e = max(e, ex);
      }
    }
    atomicMax(&sCe[a], e);
  }
  __syncthreads();
  // column exponents of the scaled M (0: the column is zero; -1: not finite)
  if (tid < TC_NB) {
    const int b = b0 + tid;
    int f = 0;
    bool bad = false;
    if (tid < nb && b < mo)
      for (int a = 0; a < m; ++a) {
        const int ex = (int)(((unsigned long long)__double_as_longlong(Mm[(int64_t)a * mo + b]) >> 52) & 0x7FF);
        if (ex == 0x7FF) bad = true;
        else if (ex != 0 && sCe[a] != 0) f = max(f, ex + sCe[a]);
      }
    sFb[tid] = bad ? -1 : f;
  }
  __syncthreads();
  // B digit planes of all K slices: scaled M^T (row b, K index a)
  for (int e = tid; e < nb * (kp16 / 2); e += TT_THREADS) {
    const int b = e % nb, ap = e / nb, a = 2 * ap;
    const int fb = sFb[b];
    long long F0 = 0, F1 = 0;
    if (b0 + b < mo && fb > 0) {
      if (a < m && sCe[a] != 0) F0 = tc_fixed(Mm[(int64_t)a * mo + b0 + b], fb - sCe[a]);
      if (a + 1 < m && sCe[a + 1] != 0) F1 = tc_fixed(Mm[(int64_t)(a + 1) * mo + b0 + b], fb - sCe[a + 1]);
    }
    tc_store_pair(Bp + (a >> 5) * TC_DIG * bpl, bpl, tc_off(b, a & 31), F0, F1);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&s_tbase)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_mbar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_mbar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tbase = s_tbase;
  const uint32_t idesc = tc_idesc(nb);
  // readout by warps 0..7: lane row ra, half h of the nb columns
  const int ra = 32 * (warp & 3) + lane, h = (warp >> 2) & 1, nh = nb >> 1;
  const uint32_t trow = tbase + ((uint32_t)(32 * (warp & 3)) << 16);
  // split mapping: row r of the block, eight of every 32 columns (quarter q4)
  const int sr = tid & (TC_M - 1), q4 = tid >> 7;
  bool ok = true;
  int g = 0;  // K slices issued so far (buffer g & 1, its commit's phase (g >> 1) & 1)
  for (int64_t rb = r_lo; rb < r_hi && ok; rb += TC_M) {
    // (2) row exponents of the scaled X over the columns this thread splits
    {
      const int64_t row = rb + sr;
      int e = TT_ZERO_ROW;
      bool bad = false;
      if (row < r_hi)
        for (int q = 0; q < nsl; ++q) {
          const int a0 = 32 * q + 8 * q4;
#pragma unroll
          for (int t = 0; t < 8; ++t)
            if (a0 + t < m) {
              const int ex =
                  (int)(((unsigned long long)__double_as_longlong(X[row * ldx + a0 + t]) >> 52) & 0x7FF);
              if (ex == 0x7FF) bad = true;
              else if (ex != 0) e = max(e, ex - sCe[a0 + t]);
            }
        }
      sEq[q4][sr] = bad ? TT_NAN_ROW : e;
      __syncthreads();
      if (q4 == 0) {
        int er = e;
        bool nan = bad;
#pragma unroll
        for (int u = 1; u < 4; ++u) {
          const int v = sEq[u][sr];
          nan = nan || v == TT_NAN_ROW;
          er = max(er, v);
        }
        sEr[sr] = nan ? TT_NAN_ROW : er;
      }
    }
    __syncthreads();
    const int er_s = sEr[sr];
    const bool on_s = rb + sr < r_hi && er_s != TT_NAN_ROW && er_s != TT_ZERO_ROW;
    // (3) K slices: digits of the next 32 columns while the last ones multiply
    for (int q = 0; q < nsl && ok; ++q, ++g) {
      const int buf = g & 1;
      unsigned char* A = tsm + buf * ABUF;
      if (g >= 2) ok = __syncthreads_and(tc_wait(&s_mbar[buf], ((g - 2) >> 1) & 1));
      if (!ok) break;
      {
        const int64_t row = rb + sr;
        const int a0 = 32 * q + 8 * q4;
        double xv[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) xv[t] = (on_s && a0 + t < m) ? X[row * ldx + a0 + t] : 0.0;
#pragma unroll
        for (int t = 0; t < 8; t += 2)
          tc_store_pair(A, TC_APLANE, tc_off(sr, 8 * q4 + t), tc_fixed(xv[t], sCe[a0 + t] + er_s),
                        tc_fixed(xv[t + 1], sCe[a0 + t + 1] + er_s));
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint64_t ad0 = tc_desc(smem_u32(A));
        const uint64_t bd0 = tc_desc(smem_u32(Bp + q * TC_DIG * bpl));
        const int nks = min(2, (kp16 - 32 * q) / 16);
        for (int ks = 0; ks < nks; ++ks) {
#pragma unroll
          for (int l = 0; l < TT_LEV; ++l) {
            const int i0 = l > TC_DIG - 1 ? l - (TC_DIG - 1) : 0;
#pragma unroll
            for (int i = i0; i <= l && i < TC_DIG; ++i) {
              const int j = l - i;
              const uint64_t ad = ad0 + (uint64_t)((i * TC_APLANE + ks * 256) >> 4);
              const uint64_t bd = bd0 + (uint64_t)((j * bpl + ks * 256) >> 4);
              tc_mma(tbase + l * nb, ad, bd, idesc, (q == 0 && ks == 0 && i == i0) ? 0u : 1u);
            }
          }
        }
        tc_commit(&s_mbar[buf]);
      }
    }
    if (!ok) break;
    // (4) the block's levels out of TMEM, combined and scaled, into Y
    ok = __syncthreads_and(tc_wait(&s_mbar[(g - 1) & 1], ((g - 1) >> 1) & 1));
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!ok) break;
    if (warp < 8) {
      const int64_t row = rb + ra;
      const int er = sEr[ra];
#pragma unroll 1
      for (int c8 = 0; c8 < nh; c8 += 8) {
        float S[TT_LEV][8];
#pragma unroll
        for (int l = 0; l < TT_LEV; ++l) tc_ld8(trow + l * nb + h * nh + c8, S[l]);
        tc_ld_wait();
        if (row < r_hi) {
#pragma unroll
          for (int t = 0; t < 8; ++t) {
            const int bl = h * nh + c8 + t, b = b0 + bl;
            if (b >= mo) continue;
            const int fb = sFb[bl];
            double v;
            if (er == TT_NAN_ROW || fb < 0) {
              v = __longlong_as_double(0x7ff8000000000000ll);
            } else if (er == TT_ZERO_ROW || fb == 0) {
              v = 0.0;
            } else {
              // every level is an integer below 2^24: I = sum_{l<=3} S_l 2^(8 (3-l))
              // and L' = sum_{l=4..7} S_l 2^(8 (7-l)) exactly in 64-bit integers,
              // then (I + L' 2^-32) 2^(E_r + E_b - 38) with one rounding
              const long long I = ((long long)__float2int_rn(S[0][t]) << 24) +
                                  ((long long)__float2int_rn(S[1][t]) << 16) +
                                  ((long long)__float2int_rn(S[2][t]) << 8) +
                                  (long long)__float2int_rn(S[3][t]);
              const long long Lq = ((long long)__float2int_rn(S[4][t]) << 24) +
                                   ((long long)__float2int_rn(S[5][t]) << 16) +
                                   ((long long)__float2int_rn(S[6][t]) << 8) +
                                   (long long)__float2int_rn(S[7][t]);
              const int p = er + fb - 2082;
              v = fma((double)Lq, 0x1p-32, (double)I);
              if (p >= -1022 && p <= 1023) {
                v *= __longlong_as_double((long long)(p + 1023) << 52);
              } else {
                const int p1 = max(-1022, min(1023, p / 2)), p2 = max(-1022, min(1023, p - p / 2));
                v = v * __longlong_as_double((long long)(p1 + 1023) << 52) *
                    __longlong_as_double((long long)(p2 + 1023) << 52);
              }
            }
            Y[row * ldy + b] = v;
          }
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }
  if (!ok) {
    // a wait ran out: this CTA's rows are NaN (the caller's next step fails)
    for (int64_t r = r_lo + tid; r < r_hi; r += TT_THREADS)
      for (int b = b0; b < min(mo, b0 + nb); ++b) Y[r * ldy + b] = __longlong_as_double(0x7ff8000000000000ll);
    if (tid == 0 && err) atomicExch(err, 1);
    // the MMAs in flight end before TMEM is released
    if (g > 0) tc_wait(&s_mbar[(g - 1) & 1], ((g - 1) >> 1) & 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(512));
}

}  // namespace

bool tall_tc_fits(int m, int mo) { return m >= 1 && m <= TC_M && mo >= 1 && mo <= 2 * TC_NB; }

void tall_gemm_tc(const double* X, int64_t n, int m, int ldx, const double* M, int mo, double* Y,
                  int ldy, int num_sms, int* err, cudaStream_t s) {
  RF_CHECK(tall_tc_fits(m, mo), RAFEAST_ERR_INVALID_ARG);
  const int nblk = (mo + TC_NB - 1) / TC_NB;
  int nb = (mo + nblk - 1) / nblk;
  nb = ((nb + 15) / 16) * 16;
  const int nbx = (mo + nb - 1) / nb;
  const int kp16 = (m + 15) & ~15, nsl = (kp16 + 31) / 32;
  int parts = num_sms / nbx;
  if (parts < 1) parts = 1;
  const int64_t blocks = (n + TC_M - 1) / TC_M;
  if (parts > blocks) parts = (int)std::max<int64_t>(1, blocks);
  const size_t smem = 2 * (size_t)TC_DIG * TC_APLANE + (size_t)nsl * TC_DIG * nb * 64;
  ensure_dyn_smem(reinterpret_cast<const void*>(k_tc_tall), smem);
  dim3 grid(nbx, parts);
  k_tc_tall<<<grid, TT_THREADS, smem, s>>>(X, n, m, ldx, M, mo, Y, ldy, nb, err);
  RF_LAUNCH();
}

bool gram_tc_fits(int m) { return m >= 1 && m <= TC_M; }

int gram_tc_parts(int num_sms) { return num_sms; }

void gram_tc(const double* X, const double* Y, int64_t n, int m, int ld, double* G,
             double* partial, int num_sms, int* err, cudaStream_t s, bool sym) {
  // X == Y: the B operand is read from X's digits (one split per value)
  const bool same = X == Y;
  RF_CHECK(gram_tc_fits(m), RAFEAST_ERR_INVALID_ARG);
  const int nblk = (m + TC_NB - 1) / TC_NB;
  int nb = (m + nblk - 1) / nblk;
  nb = ((nb + 15) / 16) * 16;
  const int nby = (m + nb - 1) / nb;
  const int parts = gram_tc_parts(num_sms);
  dim3 grid(parts, nby);
  if (same) {
    const size_t smem = 2 * (size_t)TC_DIG * TC_APLANE;
    ensure_dyn_smem(reinterpret_cast<const void*>(k_tc_gram<true>), smem);
    k_tc_gram<true><<<grid, TC_THREADS, smem, s>>>(X, X, n, m, ld, nb, partial, err);
  } else {
    const size_t smem = 2 * ((size_t)TC_DIG * TC_APLANE + (size_t)TC_DIG * TC_BPLANE);
    ensure_dyn_smem(reinterpret_cast<const void*>(k_tc_gram<false>), smem);
    k_tc_gram<false><<<grid, TC_THREADS, smem, s>>>(X, Y, n, m, ld, nb, partial, err);
  }
  RF_LAUNCH();
  gram_sum(partial, parts, m, sym, G, s);
}

}  // namespace rafeast
