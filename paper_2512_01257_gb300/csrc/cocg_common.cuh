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

// counters of one multi-shift scalar step (shared memory of the CTA that
// runs it, or combined over several CTAs)
struct MsCount {
  int active, brk, cap, mx, mn, cols;
  double worst;
};

__device__ inline void ms_count_init(MsCount& c) {
  c.active = 0;
  c.brk = 0;
  c.cap = 0;
  c.mx = 0;
  c.mn = 0x7fffffff;
  c.cols = 0;
  c.worst = 0.0;
}

// per-column part of the multi-shift scalar step for columns [c0, c1) at
// step k; counters into cnt (shared), the largest nu/||b||^2 of an active
// system into *worst (per thread). Columns are independent of one another.
template <typename T>
__device__ void ms_scalar_cols(const CocgArgs<T>& a, int k, int c0, int c1, MsCount& cnt,
                               double* worst_out) {
  const int ns = a.ns;
  double worst = 0.0;
  for (int i = c0 + (int)threadIdx.x; i < c1; i += blockDim.x) {
    SysState st = a.st[i];
    double* acc = a.acc + 5 * i;
    const double gre = __ldcg(acc + 0), gim = __ldcg(acc + 1);
    const double dre = __ldcg(acc + 2), dim = __ldcg(acc + 3), nu = __ldcg(acc + 4);
    acc[0] = acc[1] = acc[2] = acc[3] = acc[4] = 0.0;
    Coef<T> cf;
    cf.pad = (T)0;
    bool column_on = st.active != 0;
    if (column_on) {
      if (k == 0) st.bnorm2 = nu;
      if (st.bnorm2 > 0.0) worst = fmax(worst, nu / st.bnorm2);
      // seed scalars (beta_{k-1}, mu_k = p_k^T M p_k, alpha_k)
      double bre = 0.0, bim = 0.0, mre = dre, mim = dim;
      if (k > 0) {
        const double2 gp = st.gamma_prev;
        const double den = gp.x * gp.x + gp.y * gp.y;
        bre = (gre * gp.x + gim * gp.y) / den;
        bim = (gim * gp.x - gre * gp.y) / den;
        const double2 ap = st.alpha_prev;
        const double da = ap.x * ap.x + ap.y * ap.y;
        const double bgr = bre * gre - bim * gim, bgi = bre * gim + bim * gre;
        mre = dre - (bgr * ap.x + bgi * ap.y) / da;
        mim = dim - (bgi * ap.x - bgr * ap.y) / da;
      }
      const double mm = mre * mre + mim * mim;
      const bool seed_ok = mm > 1e-300 && isfinite(mm) && isfinite(bre) && isfinite(bim);
      const double are = seed_ok ? (gre * mre + gim * mim) / mm : 0.0;
      const double aim = seed_ok ? (gim * mre - gre * mim) / mm : 0.0;
      // the seed system's own stop: its quadrature contribution ends, its
      // recurrence continues while a shifted system of the column needs it.
      // st.iters is -1 while the seed runs, its stop step afterwards.
      const double thr = a.tol2 * st.bnorm2;
      bool any = false;
      bool seed_running = st.iters < 0 || k == 0;
      if (seed_running && (nu <= thr || k >= a.max_inner || !seed_ok)) {
        if (!(nu <= thr)) {
          if (!seed_ok) atomicAdd(&cnt.brk, 1);
          else atomicAdd(&cnt.cap, 1);
        }
        st.iters = k;
        seed_running = false;
        if (st.bnorm2 > 0.0) {
          atomicMax(&cnt.mx, k);
          atomicMin(&cnt.mn, k);
        }
      } else if (seed_running) {
        st.iters = -1;
        any = true;
      }
      // shifted systems
      for (int t = 0; t < ns; ++t) {
        ShiftState ss = a.sst[i * ns + t];
        ShiftCoef<T> sc;
        sc.pad = (T)0;
        sc.act = (T)0;
        sc.zeta = mk<T>((T)0, (T)0);
        sc.beta = mk<T>((T)1, (T)0);
        sc.ca = mk<T>((T)0, (T)0);
        if (ss.active) {
          const double zr = ss.zeta.x, zi = ss.zeta.y;
          const double nuj = (zr * zr + zi * zi) * nu;
          if (nuj <= thr || k >= a.max_inner || !seed_ok) {
            if (!(nuj <= thr)) {
              if (!seed_ok) atomicAdd(&cnt.brk, 1);
              else atomicAdd(&cnt.cap, 1);
            }
            ss.active = 0;
            ss.iters = k;
            if (st.bnorm2 > 0.0) {
              atomicMax(&cnt.mx, k);
              atomicMin(&cnt.mn, k);
            }
          } else {
            // zeta_{k+1}
            const double2 sg = a.sigma[t];
            const double2 ap = k == 0 ? make_double2(1.0, 0.0) : st.alpha_prev;
            const double2 zp = ss.zeta_prev, zc = ss.zeta;
            // numerator: zc * zp * ap
            double nre = zc.x * zp.x - zc.y * zp.y, nim = zc.x * zp.y + zc.y * zp.x;
            const double tr = nre * ap.x - nim * ap.y, ti = nre * ap.y + nim * ap.x;
            nre = tr;
            nim = ti;
            // 1 + sigma * a_k
            const double s1r = 1.0 + sg.x * are - sg.y * aim, s1i = sg.x * aim + sg.y * are;
            // zp * ap * (1 + sigma a_k)
            double d1r = zp.x * ap.x - zp.y * ap.y, d1i = zp.x * ap.y + zp.y * ap.x;
            const double t1r = d1r * s1r - d1i * s1i, t1i = d1r * s1i + d1i * s1r;
            // a_k * b_{k-1} * (zp - zc)
            const double abr = are * bre - aim * bim, abi = are * bim + aim * bre;
            const double dzr = zp.x - zc.x, dzi = zp.y - zc.y;
            const double t2r = abr * dzr - abi * dzi, t2i = abr * dzi + abi * dzr;
            const double der = t1r + t2r, dei = t1i + t2i;
            const double dd = der * der + dei * dei;
            const double znr = (nre * der + nim * dei) / dd, zni = (nim * der - nre * dei) / dd;
            const double zc2 = zc.x * zc.x + zc.y * zc.y;
            const double zp2 = zp.x * zp.x + zp.y * zp.y;
            if (!(dd > 1e-300) || !isfinite(znr) || !isfinite(zni) || !(zc2 > 1e-300) ||
                !(zp2 > 1e-300)) {
              ss.active = 0;
              ss.iters = k;
              atomicAdd(&cnt.brk, 1);
            } else {
              // alpha_k^j = a_k zeta_{k+1} / zeta_k
              const double qr = (znr * zc.x + zni * zc.y) / zc2, qi = (zni * zc.x - znr * zc.y) / zc2;
              const double ajr = are * qr - aim * qi, aji = are * qi + aim * qr;
              // beta_{k-1}^j = b_{k-1} (zeta_k / zeta_{k-1})^2
              const double rr = (zc.x * zp.x + zc.y * zp.y) / zp2, ri = (zc.y * zp.x - zc.x * zp.y) / zp2;
              const double r2r = rr * rr - ri * ri, r2i = 2.0 * rr * ri;
              const double bjr = bre * r2r - bim * r2i, bji = bre * r2i + bim * r2r;
              const double2 cq = a.scoef[i * ns + t];
              sc.act = (T)1;
              sc.zeta = mk<T>((T)zc.x, (T)zc.y);
              sc.beta = mk<T>((T)bjr, (T)bji);
              sc.ca = mk<T>((T)(cq.x * ajr - cq.y * aji), (T)(cq.x * aji + cq.y * ajr));
              ss.zeta_prev = zc;
              ss.zeta = make_double2(znr, zni);
              any = true;
            }
          }
        }
        a.sst[i * ns + t] = ss;
        a.scf[i * ns + t] = sc;
      }
      if (any) {
        st.gamma_prev = make_double2(gre, gim);
        st.alpha_prev = make_double2(are, aim);
        const double2 cq = a.coef[i];
        cf.ar = (T)1;
        cf.beta = mk<T>((T)bre, (T)bim);
        cf.alpha = mk<T>((T)are, (T)aim);
        cf.ca = seed_running ? mk<T>((T)(cq.x * are - cq.y * aim), (T)(cq.x * aim + cq.y * are))
                             : mk<T>((T)0, (T)0);
        atomicAdd(&cnt.active, 1);
      } else {
        st.active = 0;
        column_on = false;
      }
    }
    if (!column_on) {
      cf.ar = (T)0;
      cf.beta = mk<T>((T)1, (T)0);
      cf.alpha = mk<T>((T)0, (T)0);
      cf.ca = mk<T>((T)0, (T)0);
      for (int t = 0; t < ns; ++t) {
        ShiftCoef<T> sc;
        sc.pad = (T)0;
        sc.act = (T)0;
        sc.zeta = mk<T>((T)0, (T)0);
        sc.beta = mk<T>((T)1, (T)0);
        sc.ca = mk<T>((T)0, (T)0);
        a.scf[i * ns + t] = sc;
      }
    }
    a.st[i] = st;
    a.cf[i] = cf;
  }
  *worst_out = worst;
}

// the seed system's results of one column, handed from phase A to phases B
// and C of ms_scalar_cols_wide (shared memory)
struct MsSeed {
  SysState st;
  double gre, gim, are, aim, bre, bim, nu, thr;
  int on, seed_ok, seed_running, any;
};

// ms_scalar_cols for a whole CTA: the same arithmetic, value for value, in
// three phases so that the shifted systems of a column are computed side by
// side instead of one after another: (A) a thread per column takes the seed
// system (its sums from sacc[5 (i - c0) ..] in shared memory); (B) a thread
// per (column, shifted system) takes that system; (C) a thread per column
// writes the column's state and coefficients. sd: shared memory for c1 - c0
// MsSeed records. Every thread of the CTA calls it.
template <typename T>
__device__ void ms_scalar_cols_wide(const CocgArgs<T>& a, int k, int c0, int c1,
                                    const double* sacc, MsSeed* sd, MsCount& cnt,
                                    double* worst_out) {
  using Seed = MsSeed;
  const int ns = a.ns, nci = c1 - c0;
  double worst = 0.0;
  // (A) the seed system
  for (int ii = threadIdx.x; ii < nci; ii += blockDim.x) {
    const int i = c0 + ii;
    Seed s;
    s.st = a.st[i];
    s.gre = sacc[5 * ii + 0];
    s.gim = sacc[5 * ii + 1];
    const double dre = sacc[5 * ii + 2], dim = sacc[5 * ii + 3];
    s.nu = sacc[5 * ii + 4];
    s.on = s.st.active != 0;
    s.any = 0;
    s.are = s.aim = s.bre = s.bim = s.thr = 0.0;
    s.seed_ok = 0;
    s.seed_running = 0;
    if (s.on) {
      SysState& st = s.st;
      const double gre = s.gre, gim = s.gim, nu = s.nu;
      if (k == 0) st.bnorm2 = nu;
      if (st.bnorm2 > 0.0) worst = fmax(worst, nu / st.bnorm2);
      double bre = 0.0, bim = 0.0, mre = dre, mim = dim;
      if (k > 0) {
        const double2 gp = st.gamma_prev;
        const double den = gp.x * gp.x + gp.y * gp.y;
        bre = (gre * gp.x + gim * gp.y) / den;
        bim = (gim * gp.x - gre * gp.y) / den;
        const double2 ap = st.alpha_prev;
        const double da = ap.x * ap.x + ap.y * ap.y;
        const double bgr = bre * gre - bim * gim, bgi = bre * gim + bim * gre;
        mre = dre - (bgr * ap.x + bgi * ap.y) / da;
        mim = dim - (bgi * ap.x - bgr * ap.y) / da;
      }
      const double mm = mre * mre + mim * mim;
      const bool seed_ok = mm > 1e-300 && isfinite(mm) && isfinite(bre) && isfinite(bim);
      s.are = seed_ok ? (gre * mre + gim * mim) / mm : 0.0;
      s.aim = seed_ok ? (gim * mre - gre * mim) / mm : 0.0;
      s.bre = bre;
      s.bim = bim;
      s.seed_ok = seed_ok;
      s.thr = a.tol2 * st.bnorm2;
      bool seed_running = st.iters < 0 || k == 0;
      if (seed_running && (nu <= s.thr || k >= a.max_inner || !seed_ok)) {
        if (!(nu <= s.thr)) {
          if (!seed_ok) atomicAdd(&cnt.brk, 1);
          else atomicAdd(&cnt.cap, 1);
        }
        st.iters = k;
        seed_running = false;
        if (st.bnorm2 > 0.0) {
          atomicMax(&cnt.mx, k);
          atomicMin(&cnt.mn, k);
        }
      } else if (seed_running) {
        st.iters = -1;
        s.any = 1;
      }
      s.seed_running = seed_running;
    }
    sd[ii] = s;
  }
  __syncthreads();
  // (B) the shifted systems
  for (int e = threadIdx.x; e < nci * ns; e += blockDim.x) {
    const int ii = e / ns, t = e - (e / ns) * ns, i = c0 + ii;
    const Seed& s = sd[ii];
    if (!s.on) continue;
    const double nu = s.nu, thr = s.thr, are = s.are, aim = s.aim, bre = s.bre, bim = s.bim;
    const bool seed_ok = s.seed_ok != 0;
    ShiftState ss = a.sst[i * ns + t];
    ShiftCoef<T> sc;
    sc.pad = (T)0;
    sc.act = (T)0;
    sc.zeta = mk<T>((T)0, (T)0);
    sc.beta = mk<T>((T)1, (T)0);
    sc.ca = mk<T>((T)0, (T)0);
    if (ss.active) {
      const double zr = ss.zeta.x, zi = ss.zeta.y;
      const double nuj = (zr * zr + zi * zi) * nu;
      if (nuj <= thr || k >= a.max_inner || !seed_ok) {
        if (!(nuj <= thr)) {
          if (!seed_ok) atomicAdd(&cnt.brk, 1);
          else atomicAdd(&cnt.cap, 1);
        }
        ss.active = 0;
        ss.iters = k;
        if (s.st.bnorm2 > 0.0) {
          atomicMax(&cnt.mx, k);
          atomicMin(&cnt.mn, k);
        }
      } else {
        const double2 sg = a.sigma[t];
        const double2 ap = k == 0 ? make_double2(1.0, 0.0) : s.st.alpha_prev;
        const double2 zp = ss.zeta_prev, zc = ss.zeta;
        double nre = zc.x * zp.x - zc.y * zp.y, nim = zc.x * zp.y + zc.y * zp.x;
        const double tr = nre * ap.x - nim * ap.y, ti = nre * ap.y + nim * ap.x;
        nre = tr;
        nim = ti;
        const double s1r = 1.0 + sg.x * are - sg.y * aim, s1i = sg.x * aim + sg.y * are;
        double d1r = zp.x * ap.x - zp.y * ap.y, d1i = zp.x * ap.y + zp.y * ap.x;
        const double t1r = d1r * s1r - d1i * s1i, t1i = d1r * s1i + d1i * s1r;
        const double abr = are * bre - aim * bim, abi = are * bim + aim * bre;
        const double dzr = zp.x - zc.x, dzi = zp.y - zc.y;
        const double t2r = abr * dzr - abi * dzi, t2i = abr * dzi + abi * dzr;
        const double der = t1r + t2r, dei = t1i + t2i;
        const double dd = der * der + dei * dei;
        const double znr = (nre * der + nim * dei) / dd, zni = (nim * der - nre * dei) / dd;
        const double zc2 = zc.x * zc.x + zc.y * zc.y;
        const double zp2 = zp.x * zp.x + zp.y * zp.y;
        if (!(dd > 1e-300) || !isfinite(znr) || !isfinite(zni) || !(zc2 > 1e-300) ||
            !(zp2 > 1e-300)) {
          ss.active = 0;
          ss.iters = k;
          atomicAdd(&cnt.brk, 1);
        } else {
          const double qr = (znr * zc.x + zni * zc.y) / zc2, qi = (zni * zc.x - znr * zc.y) / zc2;
          const double ajr = are * qr - aim * qi, aji = are * qi + aim * qr;
          const double rr = (zc.x * zp.x + zc.y * zp.y) / zp2, ri = (zc.y * zp.x - zc.x * zp.y) / zp2;
          const double r2r = rr * rr - ri * ri, r2i = 2.0 * rr * ri;
          const double bjr = bre * r2r - bim * r2i, bji = bre * r2i + bim * r2r;
          const double2 cq = a.scoef[i * ns + t];
          sc.act = (T)1;
          sc.zeta = mk<T>((T)zc.x, (T)zc.y);
          sc.beta = mk<T>((T)bjr, (T)bji);
          sc.ca = mk<T>((T)(cq.x * ajr - cq.y * aji), (T)(cq.x * aji + cq.y * ajr));
          ss.zeta_prev = zc;
          ss.zeta = make_double2(znr, zni);
          atomicOr(&sd[ii].any, 1);
        }
      }
    }
    a.sst[i * ns + t] = ss;
    a.scf[i * ns + t] = sc;
  }
  __syncthreads();
  // (C) the column's state and coefficients
  for (int ii = threadIdx.x; ii < nci; ii += blockDim.x) {
    const int i = c0 + ii;
    const Seed& s = sd[ii];
    SysState st = s.st;
    Coef<T> cf;
    cf.pad = (T)0;
    bool column_on = s.on != 0;
    if (column_on) {
      if (s.any) {
        st.gamma_prev = make_double2(s.gre, s.gim);
        st.alpha_prev = make_double2(s.are, s.aim);
        const double2 cq = a.coef[i];
        cf.ar = (T)1;
        cf.beta = mk<T>((T)s.bre, (T)s.bim);
        cf.alpha = mk<T>((T)s.are, (T)s.aim);
        cf.ca = s.seed_running
                    ? mk<T>((T)(cq.x * s.are - cq.y * s.aim), (T)(cq.x * s.aim + cq.y * s.are))
                    : mk<T>((T)0, (T)0);
        atomicAdd(&cnt.active, 1);
      } else {
        st.active = 0;
        column_on = false;
      }
    }
    if (!column_on) {
      cf.ar = (T)0;
      cf.beta = mk<T>((T)1, (T)0);
      cf.alpha = mk<T>((T)0, (T)0);
      cf.ca = mk<T>((T)0, (T)0);
      for (int t = 0; t < ns; ++t) {
        ShiftCoef<T> sc;
        sc.pad = (T)0;
        sc.act = (T)0;
        sc.zeta = mk<T>((T)0, (T)0);
        sc.beta = mk<T>((T)1, (T)0);
        sc.ca = mk<T>((T)0, (T)0);
        a.scf[i * ns + t] = sc;
      }
    }
    a.st[i] = st;
    a.cf[i] = cf;
  }
  *worst_out = worst;
}

// column activity of the pairs [p0, p1) after their columns' step; counts
// the active pairs into cnt.cols
template <typename T>
__device__ void ms_colact(const CocgArgs<T>& a, int p0, int p1, MsCount& cnt) {
  for (int q = p0 + (int)threadIdx.x; q < p1; q += blockDim.x) {
    const int any = a.st[2 * q].active | a.st[2 * q + 1].active;
    a.colact[q] = any;
    if (any) atomicAdd(&cnt.cols, 1);
  }
}

// block-wide maximum of a per-thread value (every thread gets it)
__device__ inline double block_max(double v) {
  __shared__ double s_w[32];
  __shared__ double s_r;
  v = fmax(v, __shfl_xor_sync(0xffffffffu, v, 16));
  v = fmax(v, __shfl_xor_sync(0xffffffffu, v, 8));
  v = fmax(v, __shfl_xor_sync(0xffffffffu, v, 4));
  v = fmax(v, __shfl_xor_sync(0xffffffffu, v, 2));
  v = fmax(v, __shfl_xor_sync(0xffffffffu, v, 1));
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double w = 0.0;
    for (int t = 0; t < (int)(blockDim.x >> 5); ++t) w = fmax(w, s_w[t]);
    s_r = w;
  }
  __syncthreads();
  return s_r;
}

// the end of a multi-shift step (thread 0): profile history, statistics,
// the step counter, the done flag, the dot kernel's ticket
template <typename T>
__device__ void ms_scalar_finish(const CocgArgs<T>& a, int k, const MsCount& cnt) {
  CocgCtl* c = a.ctl;
  if (a.hist && k <= a.max_inner) {
    a.hist[k] = cnt.cols;
    a.rhist[k] = sqrt(cnt.worst);
  }
  c->active = cnt.active;
  c->breakdown += cnt.brk;
  c->capped += cnt.cap;
  if (cnt.mx > c->max_iters) c->max_iters = cnt.mx;
  if (cnt.mn != 0x7fffffff && (c->min_iters == 0 || cnt.mn < c->min_iters)) c->min_iters = cnt.mn;
  c->iter = k + 1;
  if (cnt.active == 0) c->done = 1;
  c->pend = 0;  // (the dot kernel that ends here applied any deferred updates)
  __threadfence();
  c->ticket = 0;
}

// Scalar step of the multi-shift COCG (last CTA of the seed's dot kernel).
// The seed system M_s = z_s I - A runs the same Chronopoulos-Gear recurrence
// as above (systems = columns i; the dot kernel treated column pairs as the
// two "shifts" of a chunk). Every other shift j, M_j = M_s + sigma_j I with
// sigma_j = z_j - z_s, shares the seed's Krylov space: its residual is
// zeta_k^j r_k, with (three-term residual-polynomial recurrence of CG at
// t = -sigma_j)
//   zeta_{k+1} = zeta_k zeta_{k-1} a_{k-1}
//                / (zeta_{k-1} a_{k-1} (1 + sigma a_k) + a_k b_{k-1} (zeta_{k-1} - zeta_k)),
//   alpha_k^j = a_k zeta_{k+1} / zeta_k,  beta_{k-1}^j = b_{k-1} (zeta_k / zeta_{k-1})^2,
// where a_k, b_{k-1} are the seed's alpha_k and beta_{k-1}. A shifted system
// stops when |zeta_k|^2 nu_k <= tol^2 ||b||^2; a column keeps iterating (the
// seed recurrence keeps running) while any of its shifts does.
template <typename T>
__device__ void ms_scalar_step(const CocgArgs<T>& a) {
  __shared__ MsCount cnt;
  if (threadIdx.x == 0) ms_count_init(cnt);
  __syncthreads();
  const int k = __ldcg(&a.ctl->iter);
  double worst = 0.0;
  ms_scalar_cols<T>(a, k, 0, 2 * a.m0, cnt, &worst);
  __syncthreads();
  ms_colact<T>(a, 0, a.m0, cnt);
  __syncthreads();
  if (a.hist) {
    const double w = block_max(worst);
    if (threadIdx.x == 0) cnt.worst = w;
  }
  __syncthreads();
  if (threadIdx.x == 0) ms_scalar_finish<T>(a, k, cnt);
}

}  // namespace rafeast
