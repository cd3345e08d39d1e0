// host_mesh.cpp -- builds the cell-centred mesh on the host: neighbour across
// each face, outward normals scaled by face length and triangle areas
// (Sec. 6.2.1), ghost faces tagged with their boundary kind (Sec. 7: each
// triangle has three neighbours, ghost nodes at boundaries).
//
// Edges are matched by sorting 64-bit keys of their (canonical) end nodes.
// Every face's normal is stored once per face and negated for the other side,
// so the two cells of a face always see exactly opposite normals -- also on
// periodic seams, where the two sides are different node copies.  The side
// that owns the normal is chosen from node ids alone (the smaller pair of raw
// node ids wins), which keeps the geometry independent of the cell numbering.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "fv_internal.h"

namespace fv {

namespace {

inline uint64_t edge_key(int32_t a, int32_t b) {
  uint32_t lo = (uint32_t)std::min(a, b), hi = (uint32_t)std::max(a, b);
  return ((uint64_t)lo << 32) | hi;
}

[[noreturn]] void fail(const std::string& msg) { throw Error{FV_EINVAL, msg}; }

}  // namespace

void build_host_mesh(const double* xy, int64_t n_nodes, const int32_t* tri, int64_t n_tri,
                     const int32_t* canon, const int32_t* bnd, int64_t n_bnd, int32_t default_bc,
                     HostMesh& m) {
  if (n_tri < 0 || n_nodes < 0 || n_bnd < 0) fail("negative size");
  if (n_tri > INT32_MAX / 3) fail("too many triangles for 32-bit cell ids");
  if (n_tri > 0 && (!xy || !tri)) fail("null xy or tri");
  if (n_bnd > 0 && !bnd) fail("null bnd_edges with n_bnd > 0");
  if (default_bc < FV_BC_NONE || default_bc > FV_BC_EXTRAP) fail("bad default_bc");
  for (int64_t j = 0; j < 3 * n_tri; ++j)
    if (tri[j] < 0 || tri[j] >= n_nodes) fail("node id out of range in tri");
  if (canon)
    for (int64_t j = 0; j < n_nodes; ++j)
      if (canon[j] < 0 || canon[j] >= n_nodes) fail("node id out of range in node_canon");
  const int64_t n = n_tri;
  m.n = n;
  m.nbr.assign(3 * n, 0);
  m.nrm.assign(6 * n, 0.0);
  m.vol.assign(n, 0.0);
  m.inradius.assign(n, 0.0);
  m.cen.assign(2 * n, 0.0);
  m.node_xy.assign(xy, xy + 2 * (n_tri > 0 ? n_nodes : 0));
  if (canon && n_tri > 0)
    m.node_canon.assign(canon, canon + n_nodes);
  else
    m.node_canon.clear();
  m.node_q.clear();
  m.grid_e = 0;
  m.grid_cx = m.grid_cy = 0.0;

  // oriented vertex triples
  std::vector<int32_t> v(3 * n);
  for (int64_t c = 0; c < n; ++c) {
    int32_t a = tri[3 * c], b = tri[3 * c + 1], d = tri[3 * c + 2];
    double ax = xy[2 * b] - xy[2 * a], ay = xy[2 * b + 1] - xy[2 * a + 1];
    double bx = xy[2 * d] - xy[2 * a], by = xy[2 * d + 1] - xy[2 * a + 1];
    double area = 0.5 * (ax * by - bx * ay);
    if (!(std::isfinite(area)) || area == 0.0)
      fail("zero-area or non-finite triangle " + std::to_string(c));
    if (area < 0.0) std::swap(b, d);
    v[3 * c] = a;
    v[3 * c + 1] = b;
    v[3 * c + 2] = d;
    m.vol[c] = std::fabs(area);
    m.cen[2 * c] = (xy[2 * a] + xy[2 * b] + xy[2 * d]) / 3.0;
    m.cen[2 * c + 1] = (xy[2 * a + 1] + xy[2 * b + 1] + xy[2 * d + 1]) / 3.0;
  }

  // faces sorted by canonical edge key
  struct Face {
    uint64_t key;
    int64_t slot;  // 3*cell + k
  };
  std::vector<Face> faces(3 * n);
  for (int64_t c = 0; c < n; ++c)
    for (int k = 0; k < 3; ++k) {
      int32_t a = v[3 * c + k], b = v[3 * c + (k + 1) % 3];
      int32_t ca = canon ? canon[a] : a, cb = canon ? canon[b] : b;
      if (ca == cb) fail("edge collapsed by node_canon in triangle " + std::to_string(c));
      faces[3 * c + k] = Face{edge_key(ca, cb), 3 * c + k};
    }
  std::sort(faces.begin(), faces.end(), [](const Face& x, const Face& y) {
    return x.key != y.key ? x.key < y.key : x.slot < y.slot;
  });

  std::vector<std::pair<uint64_t, int32_t>> tags;
  tags.reserve(n_bnd);
  for (int64_t j = 0; j < n_bnd; ++j) {
    int32_t a = bnd[3 * j], b = bnd[3 * j + 1], t = bnd[3 * j + 2];
    if (a < 0 || a >= n_nodes || b < 0 || b >= n_nodes) fail("node id out of range in bnd_edges");
    if (t < FV_BC_WALL || t > FV_BC_EXTRAP) fail("bad boundary tag in bnd_edges");
    int32_t ca = canon ? canon[a] : a, cb = canon ? canon[b] : b;
    tags.emplace_back(edge_key(ca, cb), t);
  }
  std::sort(tags.begin(), tags.end());

  auto raw_normal = [&](int64_t slot, double* out) {
    int64_t c = slot / 3;
    int k = (int)(slot % 3);
    int32_t a = v[3 * c + k], b = v[3 * c + (k + 1) % 3];
    out[0] = xy[2 * b + 1] - xy[2 * a + 1];
    out[1] = -(xy[2 * b] - xy[2 * a]);
  };
  auto raw_pair = [&](int64_t slot) {
    int64_t c = slot / 3;
    int k = (int)(slot % 3);
    int32_t a = v[3 * c + k], b = v[3 * c + (k + 1) % 3];
    return std::make_pair(std::min(a, b), std::max(a, b));
  };

  for (size_t j = 0; j < faces.size();) {
    size_t e = j + 1;
    while (e < faces.size() && faces[e].key == faces[j].key) ++e;
    if (e - j > 2) fail("edge shared by more than two triangles");
    if (e - j == 2) {
      int64_t s0 = faces[j].slot, s1 = faces[j + 1].slot;
      m.nbr[s0] = (int32_t)(s1 / 3);
      m.nbr[s1] = (int32_t)(s0 / 3);
      int64_t own = raw_pair(s0) <= raw_pair(s1) ? s0 : s1;
      int64_t other = own == s0 ? s1 : s0;
      raw_normal(own, &m.nrm[2 * own]);
      m.nrm[2 * other] = -m.nrm[2 * own];
      m.nrm[2 * other + 1] = -m.nrm[2 * own + 1];
    } else {
      int64_t s = faces[j].slot;
      int32_t tag = default_bc;
      auto it = std::lower_bound(tags.begin(), tags.end(), std::make_pair(faces[j].key, INT32_MIN));
      if (it != tags.end() && it->first == faces[j].key) tag = it->second;
      if (tag == FV_BC_NONE)
        fail("edge of triangle " + std::to_string(s / 3) + " has no neighbour and no boundary tag");
      m.nbr[s] = -tag;
      raw_normal(s, &m.nrm[2 * s]);
    }
    j = e;
  }

  for (int64_t c = 0; c < n; ++c) {
    double perim = 0.0;
    for (int k = 0; k < 3; ++k) perim += std::hypot(m.nrm[6 * c + 2 * k], m.nrm[6 * c + 2 * k + 1]);
    m.inradius[c] = 2.0 * m.vol[c] / perim;
  }
  m.vtx = std::move(v);
}

DeviceLayout pack_layout(const int32_t* nbr, const double* nrm, const double* vol,
                         const double* inradius, int64_t n, int32_t meta, bool f64) {
  DeviceLayout d;
  if (f64) {
    d.nbr.resize(n * 4 * sizeof(int32_t));
    d.geom.resize(n * 8 * sizeof(double));
    int32_t* nb = reinterpret_cast<int32_t*>(d.nbr.data());
    double* g = reinterpret_cast<double*>(d.geom.data());
    for (int64_t c = 0; c < n; ++c) {
      nb[4 * c] = nbr[3 * c];
      nb[4 * c + 1] = nbr[3 * c + 1];
      nb[4 * c + 2] = nbr[3 * c + 2];
      nb[4 * c + 3] = meta;
      for (int k = 0; k < 6; ++k) g[8 * c + k] = nrm[6 * c + k];
      g[8 * c + 6] = 1.0 / vol[c];
      g[8 * c + 7] = inradius[c];
    }
  } else {
    d.nbr.resize(n * 2 * sizeof(int32_t));
    d.geom.resize(n * 8 * sizeof(float));
    int32_t* nb = reinterpret_cast<int32_t*>(d.nbr.data());
    float* g = reinterpret_cast<float*>(d.geom.data());
    for (int64_t c = 0; c < n; ++c) {
      nb[2 * c] = nbr[3 * c + 1];
      nb[2 * c + 1] = nbr[3 * c + 2];
      for (int k = 0; k < 6; ++k) g[8 * c + k] = (float)nrm[6 * c + k];
      g[8 * c + 6] = (float)(1.0 / vol[c]);
      std::memcpy(&g[8 * c + 7], &nbr[3 * c], sizeof(int32_t));
    }
  }
  return d;
}

}  // namespace fv
