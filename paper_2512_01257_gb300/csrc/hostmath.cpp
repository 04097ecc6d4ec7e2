// Host-side math of librafeast: quadrature nodes and row reordering.
//
// * Gauss-Legendre points/weights by Newton's method on the three-term
//   Legendre recurrence (P_{k+1} = ((2k+1) x P_k - k P_{k-1})/(k+1);
//   P_n' = n (x P_n - P_{n-1})/(x^2 - 1); weight 2/((1-x^2) P_n'(x)^2)),
//   then the half-ellipse nodes of the FEAST quadrature (Section 2.1, Eq. 3).
// * Reverse Cuthill-McKee ordering (Cuthill & McKee 1969; George & Liu,
//   "Computer Solution of Large Sparse Positive Definite Systems", 1981):
//   breadth-first search from a pseudo-peripheral vertex, neighbours visited
//   in increasing degree, order reversed. It narrows the band of rows that
//   the sparse products gather from, so gathered rows are reused from L2.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "internal.h"

namespace rafeast {

void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; ++i) {
    // initial guess for the i-th largest root
    double r = std::cos(pi * (i + 0.75) / (n + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = r;
      if (n == 0) p1 = 1.0;
      for (int k = 1; k < n; ++k) {
        const double p2 = ((2.0 * k + 1.0) * r * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
      }
      // p1 = P_n(r), p0 = P_{n-1}(r)
      dp = n * (r * p1 - p0) / (r * r - 1.0);
      const double dr = p1 / dp;
      r -= dr;
      if (std::fabs(dr) < 1e-16) break;
    }
    // recompute the derivative at the converged root
    double p0 = 1.0, p1 = r;
    for (int k = 1; k < n; ++k) {
      const double p2 = ((2.0 * k + 1.0) * r * p1 - k * p0) / (k + 1.0);
      p0 = p1;
      p1 = p2;
    }
    dp = n * (r * p1 - p0) / (r * r - 1.0);
    x[n - 1 - i] = r;  // ascending order
    w[n - 1 - i] = 2.0 / ((1.0 - r * r) * dp * dp);
  }
  if (n == 1) {
    x[0] = 0.0;
    w[0] = 2.0;
  }
}

void quadrature_nodes(double lmin, double lmax, int nc, double e, std::vector<double>& zr,
                      std::vector<double>& zi, std::vector<double>& wr, std::vector<double>& wi) {
  std::vector<double> x, om;
  gauss_legendre(nc, x, om);
  const double pi = 3.14159265358979323846;
  const double c = 0.5 * (lmin + lmax), R = 0.5 * (lmax - lmin);
  zr.resize(nc);
  zi.resize(nc);
  wr.resize(nc);
  wi.resize(nc);
  for (int j = 0; j < nc; ++j) {
    const double t = 0.5 * pi * (1.0 + x[j]);
    const double ct = std::cos(t), st = std::sin(t);
    zr[j] = c + R * ct;
    zi[j] = R * e * st;
    wr[j] = 0.5 * R * om[j] * e * ct;
    wi[j] = 0.5 * R * om[j] * st;
  }
}

static void bfs_levels(int64_t n, const int32_t* rp, const int32_t* ci, int32_t start,
                       std::vector<int32_t>& level, std::vector<int32_t>& order,
                       const std::vector<int32_t>& deg, bool sort_by_degree) {
  order.clear();
  order.push_back(start);
  level[start] = 0;
  std::vector<int32_t> nb;
  for (size_t h = 0; h < order.size(); ++h) {
    const int32_t v = order[h];
    nb.clear();
    for (int32_t k = rp[v]; k < rp[v + 1]; ++k) {
      const int32_t u = ci[k];
      if (u != v && level[u] < 0) {
        level[u] = level[v] + 1;
        nb.push_back(u);
      }
    }
    if (sort_by_degree)
      std::sort(nb.begin(), nb.end(), [&](int32_t a, int32_t b) {
        return deg[a] != deg[b] ? deg[a] < deg[b] : a < b;
      });
    order.insert(order.end(), nb.begin(), nb.end());
  }
}

void rcm_order(int64_t n, const int32_t* rp, const int32_t* ci, std::vector<int32_t>& perm) {
  std::vector<int32_t> deg(n);
  for (int64_t i = 0; i < n; ++i) deg[i] = rp[i + 1] - rp[i];
  std::vector<int32_t> cand(n);
  for (int64_t i = 0; i < n; ++i) cand[i] = (int32_t)i;
  std::stable_sort(cand.begin(), cand.end(), [&](int32_t a, int32_t b) { return deg[a] < deg[b]; });
  std::vector<char> done(n, 0);
  std::vector<int32_t> level(n, -1), order, result;
  result.reserve(n);
  for (int64_t t = 0; t < n; ++t) {
    int32_t s = cand[t];
    if (done[s]) continue;
    // pseudo-peripheral start: repeat BFS from a min-degree vertex of the
    // last level while the eccentricity grows
    int ecc = -1;
    for (int rep = 0; rep < 6; ++rep) {
      bfs_levels(n, rp, ci, s, level, order, deg, false);
      const int e = level[order.back()];
      int32_t best = order.back();
      for (auto it = order.rbegin(); it != order.rend() && level[*it] == e; ++it)
        if (deg[*it] < deg[best]) best = *it;
      for (int32_t v : order) level[v] = -1;
      if (e <= ecc) break;
      ecc = e;
      s = best;
    }
    bfs_levels(n, rp, ci, s, level, order, deg, true);
    for (int32_t v : order) {
      done[v] = 1;
      result.push_back(v);
    }
    // levels stay set (>= 0) for visited vertices: later BFSs skip them
  }
  perm.assign(result.rbegin(), result.rend());
}

int64_t bandwidth(int64_t n, const int32_t* rp, const int32_t* ci, const int32_t* perm) {
  std::vector<int32_t> ip;
  if (perm) {
    ip.resize(n);
    for (int64_t r = 0; r < n; ++r) ip[perm[r]] = (int32_t)r;
  }
  int64_t bw = 0;
  for (int64_t i = 0; i < n; ++i) {
    const int64_t pi = perm ? ip[i] : i;
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
      const int64_t pj = perm ? ip[ci[k]] : ci[k];
      const int64_t d = pi > pj ? pi - pj : pj - pi;
      if (d > bw) bw = d;
    }
  }
  return bw;
}

}  // namespace rafeast
