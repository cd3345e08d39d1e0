// vertex_geom.cpp -- normals and areas formed from vertex coordinates, the
// alternative to stored normals that the paper weighs for its FPGA design
// (Sec. 7: fewer bytes per cell for more arithmetic).
//
// The step kernel forms a face normal as the rotated edge vector of the
// cell's own nodes, n_k = (y_{k+1} - y_k, -(x_{k+1} - x_k)) (Sec. 6.2.1).
// Taken from floating-point coordinates that difference cancels: its error
// is the coordinates' rounding times L/h (domain over cell size), and the two
// node copies of a periodic seam round differently, so the two sides of a
// face would no longer see exactly opposite normals.  Here the nodes sit on a
// grid of spacing s = 2^e instead: grid coordinates are integers of at most
// 31 bits, edge vectors are exact integer differences, twice the area is an
// exact 64-bit cross product, and rounding happens once, when the exact value
// is converted to the kernel's precision.  The kernel's normals are then
// exactly the snapped mesh's stored normals rounded to FP32, and the two
// sides of every face (periodic seams included) are exact negations.
//
// Snapping moves each node by at most one grid step, s <= E / (2^31 - 16)
// for a mesh of extent E; periodic copies keep the integer offset of their
// canonical node, so a seam's edges stay translates of one another.
#include <algorithm>
#include <cmath>

#include "fv_internal.h"

namespace fv {

namespace {

[[noreturn]] void fail(const std::string& msg) { throw Error{FV_EINVAL, msg}; }

constexpr double kGridSpan = 2147483632.0;  // 2^31 - 16: grid steps across the extent
constexpr int64_t kQMax = (1LL << 30) - 1;  // |q| bound: edge components fit in 31 bits

}  // namespace

void snap_to_vertex_grid(HostMesh& m) {
  const int64_t n = m.n;
  const int64_t nn = (int64_t)m.node_xy.size() / 2;
  if (n == 0 || m.snapped()) return;
  if ((int64_t)m.vtx.size() != 3 * n) fail("vertex geometry: the mesh has no node lists");
  const std::vector<double>& xy = m.node_xy;
  std::vector<char> used(nn, 0);
  for (int32_t v : m.vtx) used[v] = 1;
  double x0 = INFINITY, x1 = -INFINITY, y0 = INFINITY, y1 = -INFINITY;
  for (int64_t j = 0; j < nn; ++j)
    if (used[j]) {
      x0 = std::min(x0, xy[2 * j]), x1 = std::max(x1, xy[2 * j]);
      y0 = std::min(y0, xy[2 * j + 1]), y1 = std::max(y1, xy[2 * j + 1]);
    }
  const double extent = std::max(x1 - x0, y1 - y0);
  if (!std::isfinite(extent) || !(extent > 0.0)) fail("vertex geometry: degenerate node extent");
  // the finest spacing 2^e with the extent within kGridSpan steps
  int e = (int)std::ceil(std::log2(extent / kGridSpan));
  while (std::ldexp(extent, -e) > kGridSpan) ++e;
  while (std::ldexp(extent, -(e - 1)) <= kGridSpan) --e;
  // the grid spacing 2^e scales FP32 normals: a normal float with room
  if (e < -62 || e > 62) fail("vertex geometry: mesh extent outside the grid's range");
  const double s = std::ldexp(1.0, e);
  const double cx = std::nearbyint(0.5 * (x0 + x1) / s) * s;
  const double cy = std::nearbyint(0.5 * (y0 + y1) / s) * s;
  // grid coordinates cx/s + q must be exact in FP64
  if (std::fabs(cx / s) > 0x1p52 || std::fabs(cy / s) > 0x1p52)
    fail("vertex geometry: mesh too far from the origin for its extent");
  std::vector<int32_t> q(2 * nn, 0);
  std::vector<double> out = xy;
  for (int64_t j = 0; j < nn; ++j) {
    if (!used[j]) continue;
    const int64_t r = m.node_canon.empty() ? j : m.node_canon[j];
    for (int d = 0; d < 2; ++d) {
      const double c = d == 0 ? cx : cy;
      // the canonical node's grid point plus this copy's offset in whole steps
      const int64_t qr = std::llround((xy[2 * r + d] - c) / s);
      const int64_t sh = r == j ? 0 : std::llround((xy[2 * j + d] - xy[2 * r + d]) / s);
      const int64_t qj = qr + sh;
      if (qj < -kQMax || qj > kQMax) fail("vertex geometry: node outside the grid's range");
      q[2 * j + d] = (int32_t)qj;
      out[2 * j + d] = c + (double)qj * s;
    }
  }
  // normals and areas from the grid coordinates (the mesh changes only once
  // every check has passed)
  std::vector<double> nrm(6 * n), vol(n), inradius(n);
  for (int64_t c = 0; c < n; ++c) {
    int64_t ex[3], ey[3];
    for (int k = 0; k < 3; ++k) {
      const int32_t a = m.vtx[3 * c + k], b = m.vtx[3 * c + (k + 1) % 3];
      ex[k] = (int64_t)q[2 * b] - q[2 * a];
      ey[k] = (int64_t)q[2 * b + 1] - q[2 * a + 1];
      nrm[6 * c + 2 * k] = (double)ey[k] * s;
      nrm[6 * c + 2 * k + 1] = (double)(-ex[k]) * s;
    }
    const int64_t cross = ex[0] * ey[1] - ey[0] * ex[1];  // twice the area, in grid units
    if (cross <= 0)
      fail("vertex geometry: triangle " + std::to_string(c) + " collapses on the grid");
    vol[c] = std::ldexp((double)cross, 2 * e - 1);
    if (!std::isnormal((float)(1.0 / vol[c]))) fail("vertex geometry: 1/V outside the FP32 range");
    double perim = 0.0;
    for (int k = 0; k < 3; ++k) perim += std::hypot(nrm[6 * c + 2 * k], nrm[6 * c + 2 * k + 1]);
    inradius[c] = 2.0 * vol[c] / perim;
  }
  // the two sides of every interior face: opposite edges, exactly
  auto canon = [&](int32_t v) { return m.node_canon.empty() ? v : m.node_canon[v]; };
  for (int64_t c = 0; c < n; ++c)
    for (int k = 0; k < 3; ++k) {
      const int32_t d = m.nbr[3 * c + k];
      if (d < 0) continue;
      const int32_t a = m.vtx[3 * c + k], b = m.vtx[3 * c + (k + 1) % 3];
      bool found = false;
      for (int j = 0; j < 3 && !found; ++j) {
        const int32_t a2 = m.vtx[3 * (int64_t)d + j], b2 = m.vtx[3 * (int64_t)d + (j + 1) % 3];
        if (m.nbr[3 * (int64_t)d + j] != (int32_t)c || canon(a2) != canon(b) ||
            canon(b2) != canon(a))
          continue;
        found = (int64_t)q[2 * b2] - q[2 * a2] == -((int64_t)q[2 * b] - q[2 * a]) &&
                (int64_t)q[2 * b2 + 1] - q[2 * a2 + 1] == -((int64_t)q[2 * b + 1] - q[2 * a + 1]);
      }
      if (!found)
        fail("vertex geometry: face " + std::to_string(k) + " of triangle " + std::to_string(c) +
             " is not the exact opposite of its neighbour's on the grid");
    }
  m.nrm = std::move(nrm);
  m.vol = std::move(vol);
  m.inradius = std::move(inradius);
  m.node_q = std::move(q);
  m.node_xy = std::move(out);
  m.grid_e = e;
  m.grid_cx = cx;
  m.grid_cy = cy;
}

TileVertices build_tile_vertices(const HostMesh& m, int32_t tile) {
  if (!m.snapped()) throw Error{FV_EINVAL, "vertex geometry: nodes not on the grid"};
  if (tile < 1) throw Error{FV_EINVAL, "tile size must be positive"};
  const int64_t n = m.n, nn = (int64_t)m.node_q.size() / 2;
  const int64_t n_tiles = (n + tile - 1) / tile;
  TileVertices T;
  T.voff.assign(n_tiles + 1, 0);
  T.cell_vl.assign(n, 0u);
  T.v0.assign(n, 0);
  std::vector<int32_t> stamp(nn, -1), local(nn, 0);
  for (int64_t b = 0; b < n_tiles; ++b) {
    const int64_t t0 = b * tile, t1 = std::min<int64_t>(t0 + tile, n);
    int32_t nv = 0;
    uint32_t id[3];
    for (int64_t c = t0; c < t1; ++c) {
      for (int k = 0; k < 3; ++k) {
        const int32_t v = m.vtx[3 * c + k];
        if (stamp[v] != (int32_t)b) {  // first use in this tile: next local id
          stamp[v] = (int32_t)b;
          local[v] = nv++;
          T.vq.push_back(m.node_q[2 * v]);
          T.vq.push_back(m.node_q[2 * v + 1]);
        }
        id[k] = (uint32_t)local[v];
      }
      T.v0[c] = (uint16_t)id[0];
      T.cell_vl[c] = id[1] | (id[2] << 16);
    }
    if (nv > 0xFFFF) throw Error{FV_EINVAL, "vertex geometry: too many nodes in a tile"};
    if ((int64_t)T.vq.size() / 2 > INT32_MAX)
      throw Error{FV_EINVAL, "vertex geometry: tile nodes exceed 32-bit offsets"};
    T.voff[b + 1] = (int32_t)(T.vq.size() / 2);
    T.v_cap = std::max(T.v_cap, nv);
  }
  return T;
}

}  // namespace fv
