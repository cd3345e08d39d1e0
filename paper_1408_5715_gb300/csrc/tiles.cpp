// tiles.cpp -- tiles and their halos for the two-step (temporally blocked)
// update.
//
// Chaining two updates of a cell without going back to memory (the paper's
// processor chaining, Sec. 7) needs, for a set of cells, the states of
// everything their two updates depend on.  Tile b is the contiguous range
// [b*T, min((b+1)*T, n)) of the current numbering (compact in space after a
// Hilbert renumbering).  Its first halo is every cell outside the tile that a
// tile cell has as a neighbour; its second halo every cell outside tile and
// first halo that a first-halo cell has as a neighbour.  The first step
// updates tile and first halo from states of tile and both halos; the second
// updates the tile from the first step's states of tile and first halo.
//
// Local numbering inside a tile: tile cells 0..nt-1 (nt cells in the tile),
// then the first halo (nt ..), then the second, each halo in ascending global
// id.  Neighbours are stored as 16-bit local ids; ghost faces keep their
// boundary code c < 0 as 0x10000 + c (0xFFFF wall, 0xFFFE far field, 0xFFFD
// extrapolation), so a tile with its halos holds at most 0xFFFD cells.
// Record of a tile cell: x = ids of faces 0 and 1, low half of y = id of
// face 2; bits 16 + 2k of y hold, for a face k whose neighbour is a cell of
// the same tile, the face of that neighbour that points back (the tile
// kernel that evaluates each face once writes the negated flux there).
#include <algorithm>

#include "fv_internal.h"

namespace fv {

namespace {

constexpr int32_t kLocalLimit = 0xFFFD;  // first code used by ghost faces

uint32_t local_code(int32_t nb, int64_t t0, int64_t t1, int32_t nt, const std::vector<int32_t>& halo_pos,
                    const std::vector<int32_t>& stamp, int32_t b) {
  if (nb < 0) return (uint32_t)(0x10000 + nb);
  if (nb >= t0 && nb < t1) return (uint32_t)(nb - t0);
  if (stamp[nb] != b) throw Error{FV_EINVAL, "tile halo construction: neighbour outside the halo"};
  return (uint32_t)(nt + halo_pos[nb]);
}

}  // namespace

PairTiles build_pair_tiles(const HostMesh& m, int32_t tile) {
  if (tile < 1) throw Error{FV_EINVAL, "tile size must be positive"};
  if (m.n / tile >= INT32_MAX) throw Error{FV_EINVAL, "too many tiles"};
  PairTiles L;
  L.tile = tile;
  const int64_t n = m.n;
  L.n_tiles = (n + tile - 1) / tile;
  L.tile_info.assign(2 * (L.n_tiles + 1), 0);
  L.cell_ln.assign(2 * (size_t)n, 0u);
  // stamp[c] == b: c belongs to tile b's halos; halo_pos[c]: its position there
  std::vector<int32_t> stamp(n, -1);
  std::vector<int32_t> halo_pos(n, 0);
  std::vector<int32_t> h1, h2;
  for (int32_t b = 0; b < (int32_t)L.n_tiles; ++b) {
    const int64_t t0 = (int64_t)b * tile, t1 = std::min<int64_t>(t0 + tile, n);
    const int32_t nt = (int32_t)(t1 - t0);
    h1.clear();
    h2.clear();
    for (int64_t c = t0; c < t1; ++c)
      for (int k = 0; k < 3; ++k) {
        const int32_t x = m.nbr[3 * c + k];
        if (x >= 0 && (x < t0 || x >= t1) && stamp[x] != b) {
          stamp[x] = b;
          h1.push_back(x);
        }
      }
    std::sort(h1.begin(), h1.end());
    // cells of the first halo are marked; the second halo excludes them
    for (int32_t x : h1)
      for (int k = 0; k < 3; ++k) {
        const int32_t y = m.nbr[3 * (int64_t)x + k];
        if (y >= 0 && (y < t0 || y >= t1) && stamp[y] != b) {
          stamp[y] = b;
          h2.push_back(y);
        }
      }
    std::sort(h2.begin(), h2.end());
    const int64_t e_size = (int64_t)nt + (int64_t)h1.size() + (int64_t)h2.size();
    if (e_size > kLocalLimit)
      throw Error{FV_EINVAL, "a tile with its halos exceeds 65533 cells; renumber the cells "
                             "with a compact order (Hilbert) or use smaller tiles"};
    for (size_t j = 0; j < h1.size(); ++j) halo_pos[h1[j]] = (int32_t)j;
    for (size_t j = 0; j < h2.size(); ++j) halo_pos[h2[j]] = (int32_t)(h1.size() + j);
    const int64_t hs = (int64_t)L.halo_id.size();
    if (hs + (int64_t)h1.size() + (int64_t)h2.size() > INT32_MAX)
      throw Error{FV_EINVAL, "tile halos too large for 32-bit offsets"};
    L.tile_info[2 * b] = (int32_t)hs;
    L.tile_info[2 * b + 1] = (int32_t)h1.size();
    auto pack = [&](int64_t c, uint32_t* out, bool tile_cell) {
      const uint32_t a0 = local_code(m.nbr[3 * c], t0, t1, nt, halo_pos, stamp, b);
      const uint32_t a1 = local_code(m.nbr[3 * c + 1], t0, t1, nt, halo_pos, stamp, b);
      const uint32_t a2 = local_code(m.nbr[3 * c + 2], t0, t1, nt, halo_pos, stamp, b);
      out[0] = a0 | (a1 << 16);
      out[1] = a2;
      if (!tile_cell) return;
      for (int k = 0; k < 3; ++k) {
        const int32_t x = m.nbr[3 * c + k];
        if (x < t0 || x >= t1) continue;
        int kx = -1;
        for (int q = 0; q < 3; ++q)
          if (m.nbr[3 * (int64_t)x + q] == (int32_t)c && !(x == c && q == k) &&
              m.nrm[6 * (int64_t)x + 2 * q] == -m.nrm[6 * c + 2 * k] &&
              m.nrm[6 * (int64_t)x + 2 * q + 1] == -m.nrm[6 * c + 2 * k + 1])
            kx = q;
        if (kx < 0) throw Error{FV_EINVAL, "tile construction: the two sides of a face differ"};
        out[1] |= (uint32_t)kx << (16 + 2 * k);
      }
    };
    for (int64_t c = t0; c < t1; ++c) pack(c, &L.cell_ln[2 * c], true);
    // faces the tile evaluates once: every face of a tile cell, except those
    // whose other side is a tile cell of lower local id (or, for a cell
    // bordering itself, its own lower face)
    L.face_off.push_back((int32_t)(L.face_rec.size() / 2));
    for (int64_t c = t0; c < t1; ++c) {
      const uint32_t e = (uint32_t)(c - t0);
      const uint32_t w0 = L.cell_ln[2 * c], w1 = L.cell_ln[2 * c + 1];
      const uint32_t v[3] = {w0 & 0xFFFFu, w0 >> 16, w1 & 0xFFFFu};
      for (uint32_t q = 0; q < 3; ++q) {
        const uint32_t kq = (w1 >> (16 + 2 * q)) & 3u;
        if (v[q] < (uint32_t)nt && (v[q] < e || (v[q] == e && kq < q))) continue;
        L.face_rec.push_back(e | q << 16 | kq << 18);
        L.face_rec.push_back(v[q]);
      }
    }
    L.halo_ln.resize(2 * (hs + h1.size() + h2.size()), 0u);
    for (size_t j = 0; j < h1.size(); ++j) pack(h1[j], &L.halo_ln[2 * (hs + j)], false);
    L.halo_id.insert(L.halo_id.end(), h1.begin(), h1.end());
    L.halo_id.insert(L.halo_id.end(), h2.begin(), h2.end());
    L.e_cap = std::max<int32_t>(L.e_cap, (int32_t)e_size);
    L.t1_cap = std::max<int32_t>(L.t1_cap, nt + (int32_t)h1.size());
  }
  L.tile_info[2 * L.n_tiles] = (int32_t)L.halo_id.size();
  L.face_off.push_back((int32_t)(L.face_rec.size() / 2));
  if (L.face_rec.size() / 2 > (size_t)INT32_MAX) throw Error{FV_EINVAL, "too many tile faces"};
  return L;
}

}  // namespace fv
