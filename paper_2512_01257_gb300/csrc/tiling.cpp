// Host-side preparation of the tiled sparse products: a locality ordering of
// the rows and the row tiles whose gathered rows are staged in shared memory.
//
// * Recursive bisection by breadth-first search: a vertex set is ordered by
//   the distance from a pseudo-peripheral vertex of it (the last vertex a
//   breadth-first search from an arbitrary vertex reaches) and cut at its
//   median; both halves are ordered the same way until they have at most
//   `leaf` vertices. This is the level-structure bisection of
//   George & Liu ("Computer Solution of Large Sparse Positive Definite
//   Systems", 1981, the one-way dissection / level-structure partitioning
//   chapters) applied recursively without keeping separators. Consecutive
//   rows of the result lie close together in the graph, so a tile of
//   consecutive rows gathers from few other rows.
// * Row tiles: consecutive rows are packed into a tile while the tile's
//   union of gathered rows (every column index of its rows plus the rows
//   themselves) stays within `ucap` rows and the tile within `tmax` rows and
//   `nnzcap` nonzeros.
//   The union is kept sorted; each nonzero gets its position in its tile's
//   union (16 bits). A kernel then stages the union's rows of a dense block
//   once per tile and gathers from shared memory.
#include <algorithm>
#include <atomic>
#include <cstdint>
#include <memory>
#include <thread>
#include <vector>

#include "internal.h"

namespace rafeast {

namespace {

struct BisectCtx {
  int64_t n;
  const int32_t* rp;
  const int32_t* ci;
  int leaf;
  std::unique_ptr<std::atomic<int32_t>[]> label;  // set id of each vertex
  std::unique_ptr<int32_t[]> seen;                // visit stamp per vertex
  std::atomic<int32_t> next_label{1};
  std::atomic<int32_t> next_stamp{1};
  int32_t* out;
};

// breadth-first order of the vertices of set `lab` reachable from `start`,
// appended to `order`; `stamp` marks visited vertices (each search of a set
// uses a fresh stamp, sets are disjoint, so searches running in parallel on
// other sets never touch the same entries: a vertex's stamp is read only
// after its label shows that it belongs to this set)
void bfs_in_set(BisectCtx& c, int32_t start, int32_t lab, int32_t stamp,
                std::vector<int32_t>& order) {
  size_t head = order.size();
  order.push_back(start);
  c.seen[start] = stamp;
  while (head < order.size()) {
    const int32_t v = order[head++];
    for (int32_t k = c.rp[v]; k < c.rp[v + 1]; ++k) {
      const int32_t u = c.ci[k];
      if (c.label[u].load(std::memory_order_relaxed) == lab && c.seen[u] != stamp) {
        c.seen[u] = stamp;
        order.push_back(u);
      }
    }
  }
}

// order of the whole set: every component, each by distance from a
// pseudo-peripheral vertex of it
void order_set(BisectCtx& c, const std::vector<int32_t>& S, int32_t lab,
               std::vector<int32_t>& order) {
  order.clear();
  order.reserve(S.size());
  const int32_t final_stamp = c.next_stamp.fetch_add(1);
  std::vector<int32_t> tmp;
  for (int32_t s : S) {
    if (c.seen[s] == final_stamp) continue;
    // probe search from s, then the real one from the farthest vertex
    tmp.clear();
    const int32_t ps = c.next_stamp.fetch_add(1);
    bfs_in_set(c, s, lab, ps, tmp);
    bfs_in_set(c, tmp.back(), lab, final_stamp, order);
  }
}

void bisect_rec(BisectCtx& c, std::vector<int32_t> S, int32_t lab, int64_t off, int depth) {
  if ((int64_t)S.size() <= c.leaf) {
    for (size_t i = 0; i < S.size(); ++i) c.out[off + (int64_t)i] = S[i];
    return;
  }
  std::vector<int32_t> order;
  order_set(c, S, lab, order);
  const size_t h = order.size() / 2;
  const int32_t l1 = c.next_label.fetch_add(1), l2 = c.next_label.fetch_add(1);
  std::vector<int32_t> A(order.begin(), order.begin() + h), B(order.begin() + h, order.end());
  for (int32_t v : A) c.label[v].store(l1, std::memory_order_relaxed);
  for (int32_t v : B) c.label[v].store(l2, std::memory_order_relaxed);
  std::vector<int32_t>().swap(S);
  std::vector<int32_t>().swap(order);
  if (depth < 4 && A.size() > 20000) {
    std::thread t([&c, A = std::move(A), l1, off, depth]() mutable {
      bisect_rec(c, std::move(A), l1, off, depth + 1);
    });
    bisect_rec(c, std::move(B), l2, off + (int64_t)h, depth + 1);
    t.join();
  } else {
    bisect_rec(c, std::move(A), l1, off, depth + 1);
    bisect_rec(c, std::move(B), l2, off + (int64_t)h, depth + 1);
  }
}

}  // namespace

void bisect_order(int64_t n, const int32_t* rp, const int32_t* ci, int leaf,
                  std::vector<int32_t>& perm) {
  perm.assign(n, 0);
  BisectCtx c;
  c.n = n;
  c.rp = rp;
  c.ci = ci;
  c.leaf = std::max(1, leaf);
  c.label.reset(new std::atomic<int32_t>[n]);
  c.seen.reset(new int32_t[n]);
  for (int64_t i = 0; i < n; ++i) {
    c.label[i].store(0, std::memory_order_relaxed);
    c.seen[i] = 0;
  }
  c.out = perm.data();
  std::vector<int32_t> all(n);
  for (int64_t i = 0; i < n; ++i) all[i] = (int32_t)i;
  bisect_rec(c, std::move(all), 0, 0, 0);
}

namespace {

// set of int32 keys of the current tile's union (open addressing, linear
// probing); cleared by resetting the slots it filled
struct USet {
  std::vector<int32_t> slot;
  std::vector<int32_t> used;
  unsigned mask;
  explicit USet(int cap) {
    unsigned c = 1;
    while (c < 4u * (unsigned)cap) c <<= 1;
    slot.assign(c, -1);
    mask = c - 1;
  }
  bool insert(int32_t k) {  // true when k was not in the set
    unsigned h = ((unsigned)k * 2654435761u) & mask;
    while (slot[h] != -1) {
      if (slot[h] == k) return false;
      h = (h + 1) & mask;
    }
    slot[h] = k;
    used.push_back((int32_t)h);
    return true;
  }
  void erase_last(size_t count) {  // undo the last `count` insertions
    for (size_t i = 0; i < count; ++i) {
      slot[used.back()] = -1;
      used.pop_back();
    }
  }
  void clear() {
    for (int32_t h : used) slot[h] = -1;
    used.clear();
  }
};

// greedy tiles of rows [lo, hi): appends row ends, union sizes and sorted
// unions; false when one row exceeds a cap
bool tiles_range(int64_t lo, int64_t hi, const int32_t* rp, const int32_t* ci, int ucap,
                 int tmax, int nnzcap, std::vector<int32_t>& ends, std::vector<int32_t>& sizes,
                 std::vector<int32_t>& ucol) {
  USet set(ucap);
  std::vector<int32_t> cur, added;
  int64_t r = lo;
  while (r < hi) {
    const int64_t t0 = r;
    cur.clear();
    set.clear();
    while (r < hi && r - t0 < tmax && (int64_t)rp[r + 1] - rp[t0] <= nnzcap) {
      added.clear();
      if (set.insert((int32_t)r)) added.push_back((int32_t)r);
      for (int32_t k = rp[r]; k < rp[r + 1]; ++k)
        if (set.insert(ci[k])) added.push_back(ci[k]);
      if ((int64_t)cur.size() + (int64_t)added.size() > ucap) {
        set.erase_last(added.size());
        break;
      }
      cur.insert(cur.end(), added.begin(), added.end());
      ++r;
    }
    if (r == t0) return false;  // one row gathers from more than ucap rows
    std::sort(cur.begin(), cur.end());
    ucol.insert(ucol.end(), cur.begin(), cur.end());
    ends.push_back((int32_t)r);
    sizes.push_back((int32_t)cur.size());
  }
  return true;
}

int host_threads() {
  const unsigned hc = std::thread::hardware_concurrency();
  return (int)std::max(1u, std::min(hc, 16u));
}

}  // namespace

bool build_tiles(int64_t n, const int32_t* rp, const int32_t* ci, int ucap, int tmax,
                 int nnzcap, TileHost& t) {
  // row chunks built in parallel (a tile never spans two chunks)
  const int nt = n > 65536 ? host_threads() : 1;
  std::vector<std::vector<int32_t>> ends(nt), sizes(nt), ucol(nt);
  std::vector<char> ok(nt, 1);
  auto work = [&](int c) {
    const int64_t lo = n * c / nt, hi = n * (c + 1) / nt;
    ok[c] = tiles_range(lo, hi, rp, ci, ucap, tmax, nnzcap, ends[c], sizes[c], ucol[c]);
  };
  std::vector<std::thread> th;
  for (int c = 1; c < nt; ++c) th.emplace_back(work, c);
  work(0);
  for (auto& x : th) x.join();
  for (int c = 0; c < nt; ++c)
    if (!ok[c]) return false;
  t.trow.assign(1, 0);
  t.uoff.assign(1, 0);
  t.ucol.clear();
  t.max_union = 0;
  t.max_rows = 0;
  for (int c = 0; c < nt; ++c) {
    t.ucol.insert(t.ucol.end(), ucol[c].begin(), ucol[c].end());
    for (size_t i = 0; i < ends[c].size(); ++i) {
      t.max_rows = std::max<int>(t.max_rows, ends[c][i] - t.trow.back());
      t.trow.push_back(ends[c][i]);
      t.uoff.push_back(t.uoff.back() + sizes[c][i]);
      t.max_union = std::max<int>(t.max_union, sizes[c][i]);
    }
  }
  return true;
}

double tile_union_ratio(int64_t n, const int32_t* rp, const int32_t* ci, int ucap, int tmax,
                        int nnzcap, int windows) {
  // rows of `windows` evenly spaced windows of n / (8 windows) rows each
  const int64_t w = std::max<int64_t>(1, n / (8 * (int64_t)windows));
  std::vector<double> sum(windows, 0.0), rows(windows, 0.0);
  std::vector<char> ok(windows, 1);
  auto work = [&](int c) {
    const int64_t lo = n * c / windows, hi = std::min(n, lo + w);
    std::vector<int32_t> e, sz, u;
    ok[c] = tiles_range(lo, hi, rp, ci, ucap, tmax, nnzcap, e, sz, u);
    sum[c] = (double)u.size();
    rows[c] = (double)(hi - lo);
  };
  std::vector<std::thread> th;
  for (int c = 1; c < windows; ++c) th.emplace_back(work, c);
  work(0);
  for (auto& x : th) x.join();
  double s = 0.0, r = 0.0;
  for (int c = 0; c < windows; ++c) {
    if (!ok[c]) return -1.0;
    s += sum[c];
    r += rows[c];
  }
  return s / r;
}

void tile_local_index(int64_t n, const int32_t* rp, const int32_t* ci, const TileHost& t,
                      std::vector<uint16_t>& lidx, std::vector<int32_t>& uself) {
  lidx.assign((size_t)rp[n] + 8, 0);
  const int64_t ntiles = (int64_t)t.trow.size() - 1;
  uself.assign(ntiles, 0);
  const int nt = n > 65536 ? host_threads() : 1;
  auto work = [&](int c) {
    // position of a union row within its (sorted) union: binary search
    for (int64_t tt = ntiles * c / nt; tt < ntiles * (c + 1) / nt; ++tt) {
      const int32_t* u0 = t.ucol.data() + t.uoff[tt];
      const int32_t* u1 = t.ucol.data() + t.uoff[tt + 1];
      uself[tt] = (int32_t)(std::lower_bound(u0, u1, t.trow[tt]) - u0);
      for (int64_t r = t.trow[tt]; r < t.trow[tt + 1]; ++r)
        for (int32_t k = rp[r]; k < rp[r + 1]; ++k)
          lidx[k] = (uint16_t)(std::lower_bound(u0, u1, ci[k]) - u0);
    }
  };
  std::vector<std::thread> th;
  for (int c = 1; c < nt; ++c) th.emplace_back(work, c);
  work(0);
  for (auto& x : th) x.join();
}

}  // namespace rafeast
