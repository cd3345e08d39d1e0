// renumber.cpp -- cell orders for data locality and their diagnostics.
//
// The paper renumbers the mesh so that an on-chip window of about twice the
// adjacency bandwidth holds every neighbour a cell needs (Sec. 3, Sec. 4).  On
// the GPU the hardware L2 plays that window; these orders decide its hit rate:
//   - reverse Cuthill-McKee from a pseudo-peripheral start found by repeated
//     breadth-first search (the GPS / George-Liu endpoint search the paper
//     cites in Sec. 4.2), neighbours visited by ascending degree, then index;
//   - a Hilbert space-filling curve through the cell centroids (16 bits per
//     axis of the bounding box), stable in the old index;
//   - Amoeba1, the paper's own constructive serial-bandwidth heuristic;
//   - a uniform shuffle (Fisher-Yates driven by SplitMix64) as the worst case.
// Diagnostics: bandwidth B_f(G) and serial bandwidth S_BW (Sec. 4.1).
#include <algorithm>
#include <cmath>
#include <numeric>

#include "fv_internal.h"

namespace fv {

namespace {

// SplitMix64 (Steele, Lea and Flood, 2014): a Weyl sequence passed through a
// 64-bit finaliser.
inline uint64_t splitmix64_next(uint64_t& state) {
  state += 0x9E3779B97F4A7C15ull;
  uint64_t z = state;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Cell-graph adjacency: up to three distinct neighbour ids, self loops and
// ghost faces dropped.
struct Adjacency {
  std::vector<int32_t> nb;   // [3n], -1 = none
  std::vector<int8_t> deg;   // [n]
};

Adjacency adjacency(const HostMesh& m) {
  Adjacency a;
  a.nb.assign(3 * m.n, -1);
  a.deg.assign(m.n, 0);
  for (int64_t c = 0; c < m.n; ++c) {
    int d = 0;
    for (int k = 0; k < 3; ++k) {
      int32_t x = m.nbr[3 * c + k];
      if (x < 0 || x == c) continue;
      bool dup = false;
      for (int j = 0; j < d; ++j) dup |= a.nb[3 * c + j] == x;
      if (!dup) a.nb[3 * c + d++] = x;
    }
    a.deg[c] = (int8_t)d;
  }
  return a;
}

// Breadth-first level structure from root; returns the nodes of the last
// level and the depth (number of levels - 1).  `mark` holds a per-search
// stamp so that repeated searches need no clearing.
int bfs_last_level(const Adjacency& a, int32_t root, std::vector<int32_t>& mark, int32_t stamp,
                   std::vector<int32_t>& queue, std::vector<int32_t>& last) {
  queue.clear();
  queue.push_back(root);
  mark[root] = stamp;
  size_t head = 0;
  int depth = 0;
  size_t level_begin = 0;
  while (head < queue.size()) {
    size_t level_end = queue.size();
    level_begin = head;
    for (; head < level_end; ++head) {
      int32_t c = queue[head];
      for (int k = 0; k < a.deg[c]; ++k) {
        int32_t x = a.nb[3 * c + k];
        if (mark[x] != stamp) {
          mark[x] = stamp;
          queue.push_back(x);
        }
      }
    }
    if (queue.size() > level_end) ++depth;
  }
  last.assign(queue.begin() + level_begin, queue.end());
  return depth;
}

}  // namespace

std::vector<int32_t> order_shuffle(int64_t n, uint64_t seed) {
  std::vector<int32_t> p(n);
  std::iota(p.begin(), p.end(), 0);
  uint64_t s = seed;
  for (int64_t i = n - 1; i > 0; --i) {
    uint64_t r = splitmix64_next(s);
    int64_t j = (int64_t)(((unsigned __int128)r * (unsigned __int128)(i + 1)) >> 64);
    std::swap(p[i], p[j]);
  }
  return p;
}

std::vector<int32_t> order_rcm(const HostMesh& m) {
  const int64_t n = m.n;
  Adjacency a = adjacency(m);
  std::vector<int32_t> order;
  order.reserve(n);
  std::vector<int32_t> mark(n, -1), queue, last;
  std::vector<char> placed(n, 0);
  int32_t stamp = 0;
  for (int64_t seed = 0; seed < n; ++seed) {
    if (placed[seed]) continue;
    // pseudo-peripheral start: move to a minimum-degree node of the last
    // level while that increases the eccentricity
    int32_t root = (int32_t)seed;
    int depth = bfs_last_level(a, root, mark, stamp++, queue, last);
    for (int iter = 0; iter < 64; ++iter) {
      int32_t cand = last[0];
      for (int32_t x : last)
        if (a.deg[x] < a.deg[cand] || (a.deg[x] == a.deg[cand] && x < cand)) cand = x;
      int d2 = bfs_last_level(a, cand, mark, stamp++, queue, last);
      if (d2 <= depth) break;
      root = cand;
      depth = d2;
    }
    // Cuthill-McKee from root
    size_t head = order.size();
    order.push_back(root);
    placed[root] = 1;
    int32_t buf[3];
    while (head < order.size()) {
      int32_t c = order[head++];
      int cnt = 0;
      for (int k = 0; k < a.deg[c]; ++k) {
        int32_t x = a.nb[3 * c + k];
        if (!placed[x]) {
          placed[x] = 1;
          buf[cnt++] = x;
        }
      }
      std::sort(buf, buf + cnt, [&](int32_t x, int32_t y) {
        return a.deg[x] != a.deg[y] ? a.deg[x] < a.deg[y] : x < y;
      });
      for (int j = 0; j < cnt; ++j) order.push_back(buf[j]);
    }
  }
  std::reverse(order.begin(), order.end());
  return order;
}

// Amoeba1 (Sec. 4.2): a constructive, breadth-first-like labelling aimed at a
// small serial bandwidth.  The labelled part P grows one node at a time.  For
// a labelled node i: s(i) is the largest label distance to a labelled
// neighbour below it, u(i) its unlabelled neighbours, and with n = |P| its
// importance is imp(i) = (n - i) + |u(i)| + s(i) (zero once u(i) is empty).
// I is the first label whose u() is not empty.  Among the nodes of u(I) the
// next label goes to the one with a labelled neighbour (other than I) of
// largest importance; ties keep the first candidate (the smallest node id
// of u(I), standing in for the paper's random choice).  Each component starts
// from a pseudo-peripheral node, as GPS finds one (Sec. 4.2).
std::vector<int32_t> order_am1(const HostMesh& m) {
  const int64_t n = m.n;
  Adjacency a = adjacency(m);
  std::vector<int32_t> order;  // label -> node
  order.reserve(n);
  std::vector<int64_t> label(n, -1), s(n, 0);
  std::vector<int8_t> uncovered(n, 0);  // |u(i)|
  for (int64_t c = 0; c < n; ++c) uncovered[c] = a.deg[c];
  std::vector<int32_t> mark(n, -1), queue, last;
  int32_t stamp = 0;
  auto add = [&](int32_t v) {
    const int64_t lv = (int64_t)order.size();
    label[v] = lv;
    order.push_back(v);
    for (int k = 0; k < a.deg[v]; ++k) {
      const int32_t x = a.nb[3 * v + k];
      if (label[x] >= 0) {
        s[v] = std::max<int64_t>(s[v], lv - label[x]);
        --uncovered[x];  // v is no longer uncovered for x
        --uncovered[v];
      }
    }
  };
  auto imp = [&](int32_t v) -> int64_t {
    if (uncovered[v] == 0) return 0;
    return ((int64_t)order.size() - label[v]) + uncovered[v] + s[v];
  };
  int64_t I = 0;  // label of the first node with uncovered neighbours
  for (int64_t seed = 0; seed < n; ++seed) {
    if (label[seed] >= 0) continue;
    int32_t root = (int32_t)seed;
    int depth = bfs_last_level(a, root, mark, stamp++, queue, last);
    for (int iter = 0; iter < 64; ++iter) {
      int32_t cand = last[0];
      for (int32_t x : last)
        if (a.deg[x] < a.deg[cand] || (a.deg[x] == a.deg[cand] && x < cand)) cand = x;
      int d2 = bfs_last_level(a, cand, mark, stamp++, queue, last);
      if (d2 <= depth) break;
      root = cand;
      depth = d2;
    }
    add(root);
    for (;;) {
      while (I < (int64_t)order.size() && uncovered[order[I]] == 0) ++I;
      if (I >= (int64_t)order.size()) break;  // component done
      const int32_t nodeI = order[I];
      int32_t first = -1, cand = -1;
      int64_t best = 0;
      for (int k = 0; k < a.deg[nodeI]; ++k) {
        const int32_t x = a.nb[3 * nodeI + k];
        if (label[x] >= 0) continue;
        if (first < 0 || x < first) first = x;
        int64_t local = 0;
        for (int j = 0; j < a.deg[x]; ++j) {
          const int32_t l = a.nb[3 * x + j];
          if (label[l] >= 0 && l != nodeI) local = std::max(local, imp(l));
        }
        if (local > best) {
          best = local;
          cand = x;
        }
      }
      add(best > 0 ? cand : first);
    }
  }
  return order;
}

namespace {

// Position of grid point (x, y) along the Hilbert curve filling a 2^bits x
// 2^bits grid: at each scale the quadrant gives two more bits of the
// position, and the coordinates are reflected / transposed so that the
// sub-curve in that quadrant has the canonical orientation.
uint64_t hilbert_index(uint32_t x, uint32_t y, int bits) {
  uint64_t d = 0;
  for (int b = bits - 1; b >= 0; --b) {
    uint32_t s = 1u << b;
    uint32_t qx = (x & s) ? 1u : 0u, qy = (y & s) ? 1u : 0u;
    d += (uint64_t)s * s * ((3u * qx) ^ qy);
    if (qy == 0) {
      uint32_t mask = s - 1u;
      if (qx == 1) {
        x = mask - (x & mask);
        y = mask - (y & mask);
      }
      std::swap(x, y);
    }
    x &= s - 1u;
    y &= s - 1u;
  }
  return d;
}

}  // namespace

std::vector<int32_t> order_hilbert(const HostMesh& m) {
  const int64_t n = m.n;
  double x0 = INFINITY, x1 = -INFINITY, y0 = INFINITY, y1 = -INFINITY;
  for (int64_t c = 0; c < n; ++c) {
    x0 = std::min(x0, m.cen[2 * c]);
    x1 = std::max(x1, m.cen[2 * c]);
    y0 = std::min(y0, m.cen[2 * c + 1]);
    y1 = std::max(y1, m.cen[2 * c + 1]);
  }
  const int bits = 16;
  const double top = (double)((1u << bits) - 1u);
  double sx = x1 > x0 ? top / (x1 - x0) : 0.0, sy = y1 > y0 ? top / (y1 - y0) : 0.0;
  std::vector<std::pair<uint64_t, int32_t>> key(n);
  for (int64_t c = 0; c < n; ++c) {
    uint32_t gx = (uint32_t)std::min(top, std::max(0.0, std::floor((m.cen[2 * c] - x0) * sx)));
    uint32_t gy = (uint32_t)std::min(top, std::max(0.0, std::floor((m.cen[2 * c + 1] - y0) * sy)));
    key[c] = {hilbert_index(gx, gy, bits), (int32_t)c};
  }
  std::sort(key.begin(), key.end());  // ties broken by the old index
  std::vector<int32_t> p(n);
  for (int64_t i = 0; i < n; ++i) p[i] = key[i].second;
  return p;
}

void apply_permutation(HostMesh& m, const std::vector<int32_t>& perm) {
  const int64_t n = m.n;
  if ((int64_t)perm.size() != n) throw Error{FV_EINVAL, "permutation size mismatch"};
  std::vector<int32_t> inv(n, -1);
  for (int64_t i = 0; i < n; ++i) {
    int32_t o = perm[i];
    if (o < 0 || o >= n || inv[o] != -1) throw Error{FV_EINVAL, "not a permutation"};
    inv[o] = (int32_t)i;
  }
  HostMesh r;
  r.n = n;
  r.nbr.resize(3 * n);
  r.nrm.resize(6 * n);
  r.vol.resize(n);
  r.inradius.resize(n);
  r.cen.resize(2 * n);
  r.vtx.resize(m.vtx.size());
  r.node_xy = std::move(m.node_xy);
  r.node_canon = std::move(m.node_canon);
  r.node_q = std::move(m.node_q);
  r.grid_e = m.grid_e;
  r.grid_cx = m.grid_cx;
  r.grid_cy = m.grid_cy;
  for (int64_t i = 0; i < n; ++i) {
    int64_t o = perm[i];
    for (int k = 0; k < 3; ++k) {
      int32_t x = m.nbr[3 * o + k];
      r.nbr[3 * i + k] = x >= 0 ? inv[x] : x;
    }
    for (int k = 0; k < 6; ++k) r.nrm[6 * i + k] = m.nrm[6 * o + k];
    r.vol[i] = m.vol[o];
    r.inradius[i] = m.inradius[o];
    r.cen[2 * i] = m.cen[2 * o];
    r.cen[2 * i + 1] = m.cen[2 * o + 1];
    if (!r.vtx.empty())
      for (int k = 0; k < 3; ++k) r.vtx[3 * i + k] = m.vtx[3 * o + k];
  }
  m = std::move(r);
}

int64_t graph_bandwidth(const HostMesh& m) {
  int64_t b = 0;
  for (int64_t c = 0; c < m.n; ++c)
    for (int k = 0; k < 3; ++k) {
      int32_t x = m.nbr[3 * c + k];
      if (x >= 0) b = std::max<int64_t>(b, x > c ? x - c : c - x);
    }
  return b;
}

int64_t serial_bandwidth(const HostMesh& m) {
  // s(i), e(i): smallest / largest neighbour label of the cell labelled i;
  // S = suffix minimum of s, E = prefix maximum of e; S_BW = max E(i) - S(i).
  const int64_t n = m.n;
  std::vector<int64_t> S(n + 1, INT64_MAX);
  for (int64_t i = n - 1; i >= 0; --i) {
    int64_t s = INT64_MAX;
    for (int k = 0; k < 3; ++k) {
      int32_t x = m.nbr[3 * i + k];
      if (x >= 0) s = std::min<int64_t>(s, x);
    }
    S[i] = std::min(S[i + 1], s);
  }
  int64_t E = INT64_MIN, best = 0;
  for (int64_t i = 0; i < n; ++i) {
    for (int k = 0; k < 3; ++k) {
      int32_t x = m.nbr[3 * i + k];
      if (x >= 0) E = std::max<int64_t>(E, x);
    }
    if (E != INT64_MIN && S[i] != INT64_MAX) best = std::max(best, E - S[i]);
  }
  return best;
}

}  // namespace fv
