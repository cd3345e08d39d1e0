// tile_math.cuh -- the cell update on tiles staged in shared memory, shared by
// the one-step tile kernel (tile_step.cu) and the two-step kernels
// (pair_step.cu).  A tile holds the states of its cells and halo cells and,
// in the one-step kernel, their primitive variables (u, v, p, c), each
// computed once (the two-step kernels stage states only and form a
// neighbour's primitives at each use); neighbours are 16-bit tile-local ids
// (tiles.cpp), ghost faces the codes 0xFFFD..0xFFFF.
// The face arithmetic is cell_math.cuh's, so results are bitwise those of the
// one-step kernel that forms every neighbour's primitives itself.
#pragma once

#include "cell_math.cuh"

namespace fv {
namespace {

constexpr unsigned kGhostCodes = 0xFFFD;  // local ids at or above this are ghost faces

template <typename R>
__device__ __forceinline__ rec_t<R> prim_rec(const Prim<R>& w) {
  return Rec<R>::make(w.u, w.v, w.p, w.c);
}

template <typename R>
__device__ __forceinline__ Prim<R> rec_prim(const rec_t<R>& p) {
  return Prim<R>{p.x, p.y, p.z, p.w};
}

// One face of a cell whose neighbour state and primitives are in shared
// memory (entries [0, cap) of sU and sP).  PRIMS = false: only the states are
// staged (sP unused) and the neighbour's primitives are formed here.
template <typename R, int WAVE = kWaveAverage, bool PRIMS = true>
__device__ __forceinline__ R smem_face(const rec_t<R>& UL, const Prim<R>& L, unsigned v, R nx, R ny,
                                       const rec_t<R>* sU, const rec_t<R>* sP, const R* uinf,
                                       R acc[4], int cap, int* err) {
  rec_t<R> UR;
  Prim<R> W;
  if (v < kGhostCodes) {
    if (index_ok(v, cap, err)) {
      UR = sU[v];
      W = PRIMS ? rec_prim<R>(sP[v]) : primitive<R>(UR);
    } else {
      UR = UL;
      W = L;
    }
  } else {
    UR = ghost<R>((int)v - 0x10000, UL, nx, ny, uinf);
    W = primitive<R>(UR);
  }
  const R len = face_len<R>(nx, ny);
  face_flux_acc<R, false, WAVE>(UL, L, UR, W, nx, ny, len, R(1), acc);
  return len;
}

// Residual sum of one cell (faces in the order 0, 1, 2) and its perimeter;
// the tile-local ids of ln index entries [0, cap) of sU and sP.
template <typename R, int WAVE = kWaveAverage, bool PRIMS = true>
__device__ __forceinline__ R cell_fluxes(const rec_t<R>& g0, const rec_t<R>& g1, uint2 ln,
                                         const rec_t<R>& UL, const Prim<R>& L, const rec_t<R>* sU,
                                         const rec_t<R>* sP, const R* uinf, R acc[4], int cap,
                                         int* err) {
  R perim = smem_face<R, WAVE, PRIMS>(UL, L, ln.x & 0xffffu, g0.x, g0.y, sU, sP, uinf, acc, cap,
                                      err);
  perim = add(perim, smem_face<R, WAVE, PRIMS>(UL, L, ln.x >> 16, g0.z, g0.w, sU, sP, uinf, acc,
                                               cap, err));
  // the high half of ln.y holds a node id in the vertex-geometry layout
  perim = add(perim, smem_face<R, WAVE, PRIMS>(UL, L, ln.y & 0xffffu, g1.x, g1.y, sU, sP, uinf,
                                               acc, cap, err));
  return perim;
}

// Normals of a cell from the grid coordinates of its nodes q0, q1, q2
// (counter-clockwise; vertex_geom.cpp): face k's normal is its integer edge
// (dx, dy) rotated to (dy, -dx), converted with one rounding and scaled by
// the grid spacing vscale = 2^e -- bitwise the stored FP32 normals of the
// snapped mesh.  1/V is read (inv_vol), as stored for the snapped mesh;
// g1.w, unused here, is 0.
__device__ __forceinline__ void vertex_geometry(int2 q0, int2 q1, int2 q2, float vscale,
                                                float inv_vol, float4& g0, float4& g1) {
  g0.x = mul(__int2float_rn(q1.y - q0.y), vscale);
  g0.y = mul(__int2float_rn(q0.x - q1.x), vscale);
  g0.z = mul(__int2float_rn(q2.y - q1.y), vscale);
  g0.w = mul(__int2float_rn(q1.x - q2.x), vscale);
  g1.x = mul(__int2float_rn(q0.y - q2.y), vscale);
  g1.y = mul(__int2float_rn(q2.x - q0.x), vscale);
  g1.z = inv_vol;
  g1.w = 0.0f;
}

// Loads the states of a tile (nt cells from t0) and of its first halo (h1
// cells whose ids are halo[0 .. h1)) into shared memory with their primitive
// variables.  With PA > 0 each thread issues the loads of its first PA
// entries before it uses any, so it waits for about one memory round trip
// (two for halo cells, whose ids come first) rather than one per entry.
// The halo ids are global cell ids of the n cells (checked in the
// bounds-checked build; a bad id stages the tile's first cell).
template <typename R>
__device__ __forceinline__ int64_t staged_id(int64_t t0, int nt, int e, const int* halo,
                                             int64_t n, int* err) {
  if (e < nt) return t0 + e;
  const int64_t g = __ldg(halo + (e - nt));
  return index_ok(g, n, err) ? g : t0;
}

template <typename R, int THREADS, int PA>
__device__ __forceinline__ void stage_states(const rec_t<R>* __restrict__ U, int64_t t0, int nt,
                                             int h1, const int* __restrict__ halo, rec_t<R>* sU,
                                             rec_t<R>* sP, int64_t n, int* err) {
  const int ne = nt + h1;
  int e0 = threadIdx.x;
  if constexpr (PA > 0) {
    rec_t<R> u[PA];
#pragma unroll
    for (int k = 0; k < PA; ++k) {
      const int e = threadIdx.x + k * THREADS;
      if (e < ne) u[k] = Rec<R>::ld(U + staged_id<R>(t0, nt, e, halo, n, err));
    }
#pragma unroll
    for (int k = 0; k < PA; ++k) {
      const int e = threadIdx.x + k * THREADS;
      if (e < ne) {
        sU[e] = u[k];
        sP[e] = prim_rec<R>(primitive<R>(u[k]));
      }
    }
    e0 += PA * THREADS;
  }
  for (int e = e0; e < ne; e += THREADS) {
    const rec_t<R> u = Rec<R>::ld(U + staged_id<R>(t0, nt, e, halo, n, err));
    sU[e] = u;
    sP[e] = prim_rec<R>(primitive<R>(u));
  }
}

// Loads per thread issued together by stage_states: FP32 tiles with a ring
// of up to two block-widths of halo cells in one batch; FP64 (bound by its
// arithmetic, with twice the registers per state) one at a time.
template <typename R, int KMAX>
constexpr int kStageBatch = sizeof(R) == 4 ? KMAX + 2 : 0;

// The normal of face q of cell i from its geometry record (one 16-byte load).
template <typename R>
__device__ __forceinline__ void face_normal(const rec_t<R>* __restrict__ geom, int i, unsigned q,
                                            R& nx, R& ny);
template <>
__device__ __forceinline__ void face_normal<float>(const float4* __restrict__ geom, int i,
                                                   unsigned q, float& nx, float& ny) {
  const float4 g = __ldg(geom + 2 * i + (q == 2u));
  nx = q == 1u ? g.z : g.x;
  ny = q == 1u ? g.w : g.y;
}
template <>
__device__ __forceinline__ void face_normal<double>(const dq4* __restrict__ geom, int i,
                                                    unsigned q, double& nx, double& ny) {
  // record 2i holds faces 0 and 1, record 2i + 1 face 2 first: 16-byte halves
  const double2 g = __ldg(reinterpret_cast<const double2*>(geom + 2 * i + (q == 2u)) + (q == 1u));
  nx = g.x;
  ny = g.y;
}

}  // namespace
}  // namespace fv
