// Scalar step of the batched COCG (shared by the register-gather and the
// bulk-copy kernels): executed by the last CTA of a dot-kernel launch, it
// turns the per-system sums gamma = r^T r, delta = r^T M r, nu = ||r||^2
// into alpha_k, beta_k (Chronopoulos-Gear ordering, FP64), applies the
// stopping rule ||r_k|| <= tol ||b|| and the step cap, freezes finished or
// broken-down systems, and refreshes the per-column activity flags.
#pragma once

#include "common.cuh"
#include "internal.h"

namespace rafeast {

template <typename T>
__device__ void cocg_scalar_step(const CocgArgs<T>& a, int NC) {
  using C = c2<T>;
  __shared__ int s_active, s_brk, s_cap, s_max, s_min;
  if (threadIdx.x == 0) {
    s_active = 0;
    s_brk = 0;
    s_cap = 0;
    s_max = 0;
    s_min = 0x7fffffff;
  }
  __syncthreads();
  const int k = __ldcg(&a.ctl->iter);
  const int nsys = a.m0 * NC;
  double worst = 0.0;  // max ||r||^2/||b||^2 over systems active at step k
  for (int s = threadIdx.x; s < nsys; s += blockDim.x) {
    SysState st = a.st[s];
    double* acc = a.acc + 5 * s;
    const double gre = __ldcg(acc + 0), gim = __ldcg(acc + 1);
    const double dre = __ldcg(acc + 2), dim = __ldcg(acc + 3), nu = __ldcg(acc + 4);
    acc[0] = acc[1] = acc[2] = acc[3] = acc[4] = 0.0;
    Coef<T> cf;
    cf.pad = (T)0;
    bool freeze = !st.active;
    if (st.active) {
      if (k == 0) st.bnorm2 = nu;
      if (st.bnorm2 > 0.0) worst = fmax(worst, nu / st.bnorm2);
      const bool conv = nu <= a.tol2 * st.bnorm2;
      if (conv || k >= a.max_inner) {
        st.active = 0;
        st.iters = k;
        freeze = true;
        if (!conv) atomicAdd(&s_cap, 1);
        if (st.bnorm2 > 0.0) {
          atomicMax(&s_max, k);
          atomicMin(&s_min, k);
        }
      } else {
        double bre = 0.0, bim = 0.0, mre = dre, mim = dim;
        if (k > 0) {
          // beta = gamma / gamma_prev
          const double2 gp = st.gamma_prev;
          const double den = gp.x * gp.x + gp.y * gp.y;
          bre = (gre * gp.x + gim * gp.y) / den;
          bim = (gim * gp.x - gre * gp.y) / den;
          // mu = delta - beta * gamma / alpha_prev
          const double2 ap = st.alpha_prev;
          const double da = ap.x * ap.x + ap.y * ap.y;
          const double bgr = bre * gre - bim * gim, bgi = bre * gim + bim * gre;
          mre = dre - (bgr * ap.x + bgi * ap.y) / da;
          mim = dim - (bgi * ap.x - bgr * ap.y) / da;
        }
        const double mabs = fabs(mre) + fabs(mim);
        if (!(mabs > 1e-300) || !isfinite(mabs) || !isfinite(bre) || !isfinite(bim)) {
          st.active = 0;
          st.iters = k;
          freeze = true;
          atomicAdd(&s_brk, 1);
        } else {
          const double mm = mre * mre + mim * mim;
          const double are = (gre * mre + gim * mim) / mm;
          const double aim = (gim * mre - gre * mim) / mm;
          st.gamma_prev = make_double2(gre, gim);
          st.alpha_prev = make_double2(are, aim);
          const double2 cq = a.coef[s];
          cf.ar = (T)1;
          cf.beta = mk<T>((T)bre, (T)bim);
          cf.alpha = mk<T>((T)are, (T)aim);
          cf.ca = mk<T>((T)(cq.x * are - cq.y * aim), (T)(cq.x * aim + cq.y * are));
          atomicAdd(&s_active, 1);
        }
      }
    }
    if (freeze) {
      cf.ar = (T)0;
      cf.beta = mk<T>((T)1, (T)0);
      cf.alpha = mk<T>((T)0, (T)0);
      cf.ca = mk<T>((T)0, (T)0);
    }
    a.st[s] = st;
    a.cf[s] = cf;
  }
  __syncthreads();
  __shared__ int s_cols;
  if (threadIdx.x == 0) s_cols = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < a.m0; i += blockDim.x) {
    int any = 0;
    for (int j = 0; j < NC; ++j) any |= a.st[i * NC + j].active;
    a.colact[i] = any;
    if (any) atomicAdd(&s_cols, 1);
  }
  __syncthreads();
  if (a.hist) {
    __shared__ double s_worst[32];
    worst = fmax(worst, __shfl_xor_sync(0xffffffffu, worst, 16));
    worst = fmax(worst, __shfl_xor_sync(0xffffffffu, worst, 8));
    worst = fmax(worst, __shfl_xor_sync(0xffffffffu, worst, 4));
    worst = fmax(worst, __shfl_xor_sync(0xffffffffu, worst, 2));
    worst = fmax(worst, __shfl_xor_sync(0xffffffffu, worst, 1));
    if ((threadIdx.x & 31) == 0) s_worst[threadIdx.x >> 5] = worst;
    __syncthreads();
    if (threadIdx.x == 0 && k <= a.max_inner) {
      double w = 0.0;
      for (int t = 0; t < (int)(blockDim.x >> 5); ++t) w = fmax(w, s_worst[t]);
      a.hist[k] = s_cols;
      a.rhist[k] = sqrt(w);
    }
  }
  if (threadIdx.x == 0) {
    CocgCtl* c = a.ctl;
    c->active = s_active;
    c->breakdown += s_brk;
    c->capped += s_cap;
    if (s_max > c->max_iters) c->max_iters = s_max;
    if (s_min != 0x7fffffff && (c->min_iters == 0 || s_min < c->min_iters)) c->min_iters = s_min;
    c->iter = k + 1;
    if (s_active == 0) c->done = 1;
    __threadfence();
    c->ticket = 0;
  }
}

}  // namespace rafeast
