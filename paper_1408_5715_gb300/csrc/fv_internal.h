// fv_internal.h -- host-side data structures shared by the library's
// translation units (mesh builder, renumbering, C ABI, kernels).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "fv.h"

namespace fv {

// Error raised inside the library and turned into a status at the C ABI.
struct Error {
  int code;
  std::string msg;
};

// A mesh as built on the host (Sec. 6.2.1 geometry, Sec. 7 neighbour
// structure).  Arrays are per cell in the current numbering.
struct HostMesh {
  int64_t n = 0;
  std::vector<int32_t> nbr;     // [3n] neighbour across face k, or -FV_BC_* tag
  std::vector<double> nrm;      // [6n] outward normal * face length, (x, y) per face
  std::vector<double> vol;      // [n]  triangle area V_T
  std::vector<double> inradius; // [n]  2 V_T / P_T (P_T perimeter): CFL length scale
  std::vector<double> cen;      // [2n] centroid (for the Hilbert order)
  std::vector<int32_t> vtx;     // [3n] nodes of each cell, counter-clockwise: face k runs
                                //      from vtx[3c+k] to vtx[3c+(k+1)%3]
  // nodes as given to fv_mesh_create (snapped by fv_mesh_set_geometry)
  std::vector<double> node_xy;     // [2 n_nodes]
  std::vector<int32_t> node_canon; // [n_nodes] periodic identification; empty: identity
  // vertex geometry (empty / 0 until the nodes are snapped to the grid)
  std::vector<int32_t> node_q;     // [2 n_nodes] grid coordinates: x = grid_cx + q * 2^grid_e
  int32_t grid_e = 0;
  double grid_cx = 0.0, grid_cy = 0.0;
  bool snapped() const { return !node_q.empty(); }
};

// Builds the host mesh; throws fv::Error{FV_EINVAL, ...} for malformed input.
void build_host_mesh(const double* xy, int64_t n_nodes, const int32_t* tri, int64_t n_tri,
                     const int32_t* canon, const int32_t* bnd, int64_t n_bnd, int32_t default_bc,
                     HostMesh& out);

// Cell orders (new -> old) for the current numbering of m (Sec. 4).
std::vector<int32_t> order_shuffle(int64_t n, uint64_t seed);
std::vector<int32_t> order_rcm(const HostMesh& m);
std::vector<int32_t> order_hilbert(const HostMesh& m);
std::vector<int32_t> order_am1(const HostMesh& m);

// Renumbers m in place with perm (new -> old), remapping neighbour ids.
void apply_permutation(HostMesh& m, const std::vector<int32_t>& perm);

// Device records of a cell range (byte buffers ready to copy):
//   FP64: nbr int4 (nbr0, nbr1, nbr2, 0); geom doubles n0x n0y n1x n1y n2x n2y 1/V 2V/P
//   FP32: nbr int2 (nbr1, nbr2); geom floats n0x n0y n1x n1y n2x n2y 1/V nbr0-bits
struct DeviceLayout {
  std::vector<unsigned char> nbr, geom;
};
DeviceLayout pack_layout(const int32_t* nbr, const double* nrm, const double* vol,
                         const double* inradius, int64_t n, int32_t meta, bool f64);

// Snaps the cells' nodes to a grid of spacing 2^e (vertex_geom.cpp) and
// rebuilds normals and areas from the grid coordinates; throws FV_EINVAL when
// the mesh does not fit the grid's 31-bit range or a face pair loses its
// exact negation.
void snap_to_vertex_grid(HostMesh& m);

// Partitioning into contiguous ranges of the current numbering (partition.cpp).
struct PartRange {
  int64_t begin = 0, end = 0;
};
struct LocalPart {
  int64_t n_owned = 0;
  std::vector<int64_t> global;      // [n_owned + n_halo] local -> global cell id
  std::vector<int32_t> halo_owner;  // [n_halo] part owning each halo cell
  std::vector<int32_t> nbr;         // [3 n_owned] local neighbour ids / ghost codes
  std::vector<double> nrm;          // [6 n_owned]
  std::vector<double> vol;          // [n_owned]
};
PartRange part_range(int64_t n, int32_t nparts, int32_t part);
LocalPart build_local_part(const HostMesh& m, int32_t nparts, int32_t part);

// Tiles and halos of the two-step update (tiles.cpp).  Per tile b:
// tile_info[2b] = offset of its halos in halo_id, tile_info[2b+1] = size of
// the first halo; the second halo runs to tile_info[2b+2].  cell_ln (per cell)
// and halo_ln (per first-halo entry; zero for second-halo entries) hold the
// three neighbours as 16-bit tile-local ids (ghost code c as 0x10000 + c),
// packed (f0 | f1 << 16, f2).
struct PairTiles {
  int32_t tile = 0;
  int64_t n_tiles = 0;
  std::vector<int32_t> tile_info;  // [2 (n_tiles + 1)]
  std::vector<int32_t> halo_id;    // global ids: first then second halo of each tile
  std::vector<uint32_t> halo_ln;   // [2 halo_id.size()]
  std::vector<uint32_t> cell_ln;   // [2 n]
  int32_t e_cap = 0;   // max over tiles of tile + both halos
  int32_t t1_cap = 0;  // max over tiles of tile + first halo
  // the faces each tile evaluates once (shape 7): tile b's are face_rec[2 f]
  // for f in [face_off[b], face_off[b + 1]): x = e | q << 16 | kq << 18 (face q
  // of tile cell e; kq the face of the cell across that points back, for a
  // cell of the tile), y = the 16-bit local id across (ring or ghost code)
  std::vector<int32_t> face_off;   // [n_tiles + 1]
  std::vector<uint32_t> face_rec;  // [2 faces]
};
PairTiles build_pair_tiles(const HostMesh& m, int32_t tile);

// The nodes of each tile for normals formed from vertex coordinates
// (vertex_geom.cpp).  Tile b's nodes are vq[2 voff[b] ..] (grid coordinates,
// duplicated where tiles share nodes); each cell's three nodes are 16-bit
// tile-local ids v0 (the high half of cell_ln's second word) and v1 | v2 << 16.
struct TileVertices {
  std::vector<int32_t> voff;      // [n_tiles + 1]
  std::vector<int32_t> vq;        // [2 voff[n_tiles]]
  std::vector<uint32_t> cell_vl;  // [n] v1 | v2 << 16
  std::vector<uint16_t> v0;       // [n]
  std::vector<float> inv_vol;     // [n] FP32 1/V (filled at upload)
  int32_t v_cap = 0;              // max nodes of a tile
};
TileVertices build_tile_vertices(const HostMesh& m, int32_t tile);

// Sec. 4.1 diagnostics on the cell graph of the current numbering.
int64_t graph_bandwidth(const HostMesh& m);
int64_t serial_bandwidth(const HostMesh& m);

}  // namespace fv
