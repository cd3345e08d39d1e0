// tile_step.cu -- one step per launch on tiles staged in shared memory (shape
// variant 6 of the step kernel).
//
// A block owns a tile of consecutive cells.  It loads the states of the tile
// and of its first halo ring (the cells outside the tile adjacent to it,
// tiles.cpp) into shared memory and forms their primitive variables (Eq. 2)
// once per cell; the one-thread-per-cell kernels form them once per face,
// i.e. four times per cell.  Each tile cell then sums its three face fluxes
// from the shared-memory neighbours and finishes exactly as the other shapes
// do (finish_cell: forward Euler, Heun's stages or the residual, plain or
// compensated), so all shapes give the same bits.  The FP64 step, bound by
// its division and square-root sequences, gains most.
#include <cuda_runtime.h>

#include <cstdint>

#include "cell_math.cuh"
#include "kernels.h"
#include "launch_util.cuh"
#include "tile_math.cuh"

namespace fv {

namespace {

// VTX (FP32 only): normals from the grid coordinates of the tile's nodes,
// staged in shared memory after the states (vertex_geom.cpp), and 1/V from a
// 4-byte array, instead of each cell's 32-byte geometry record.
// FP32 keeps 1280 threads per SM resident (five blocks of 256: at most 48
// registers); FP64 needs its registers.
template <typename R, int MODE, bool COMP, int THREADS, int KMAX, int WAVE, bool VTX>
__global__ void __launch_bounds__(THREADS, sizeof(R) == 4 ? 1280 / THREADS : 1)
    k_step_tile(StepArgs a) {
  chain_entry();
  extern __shared__ __align__(128) unsigned char smem_raw[];
  rec_t<R>* sU = reinterpret_cast<rec_t<R>*>(smem_raw);  // [t1_cap] states
  rec_t<R>* sP = sU + a.t1_cap;                            // [t1_cap] (u, v, p, c)
  int2* sQ = reinterpret_cast<int2*>(sP + a.t1_cap);       // [v_cap] node grid coordinates
  const rec_t<R>* __restrict__ U = static_cast<const rec_t<R>*>(a.U);
  const rec_t<R>* __restrict__ geom = static_cast<const rec_t<R>*>(a.geom);
  rec_t<R>* out = static_cast<rec_t<R>*>(a.out);
  const int t0 = blockIdx.x * a.tile;  // cell ids are 32-bit
  const int nt = min(a.tile, (int)a.n - t0);
  const int hs = __ldg(a.tile_info + 2 * blockIdx.x);
  const int h1 = __ldg(a.tile_info + 2 * blockIdx.x + 1);
  // dt formed once per block (FP64 scalar work), read after the barrier
  __shared__ double s_t, s_dt;
  if (threadIdx.x == 0 && MODE != kModeResidual) block_dt(a, s_t, s_dt);
  // the tile's node coordinates: loads issued with the states', stored after
  constexpr int VA = KMAX / 2 + 1;  // per thread: 3 x 256 for the ~600 nodes of 1024 cells
  int2 qv[VTX ? VA : 1];
  int vb = 0, nv = 0;
  if constexpr (VTX) {
    vb = __ldg(a.tile_voff + blockIdx.x);
    nv = __ldg(a.tile_voff + blockIdx.x + 1) - vb;
#pragma unroll
    for (int k = 0; k < VA; ++k) {
      const int e = threadIdx.x + k * THREADS;
      if (e < nv) qv[k] = __ldg(a.tile_vq + vb + e);
    }
  }
  stage_states<R, THREADS, kStageBatch<R, KMAX>>(U, t0, nt, h1, a.halo_id + hs, sU, sP, a.n,
                                                 a.err);
  if constexpr (VTX) {
#pragma unroll
    for (int k = 0; k < VA; ++k) {
      const int e = threadIdx.x + k * THREADS;
      if (e < nv) sQ[e] = qv[k];
    }
    for (int e = threadIdx.x + VA * THREADS; e < nv; e += THREADS) sQ[e] = __ldg(a.tile_vq + vb + e);
  }
  __syncthreads();
  const double t = MODE != kModeResidual ? s_t : 0.0, dt = MODE != kModeResidual ? s_dt : 0.0;
  const R dtR = R(dt);
  R bmin = R(INFINITY);
  bool ok = true;
#pragma unroll
  for (int k = 0; k < KMAX; ++k) {
    const int e = threadIdx.x + k * THREADS;
    if (e < nt) {
      const int i = t0 + e;
      CellIn<R> c;
      const uint2 ln = __ldg(a.cell_ln + i);
      if constexpr (VTX) {
        const unsigned vl = __ldg(a.cell_vl + i);
        // node ids index the nv staged nodes (checked in the bounds-checked build)
        auto node = [&](unsigned q) { return index_ok(q, nv, a.err) ? sQ[q] : make_int2(0, 0); };
        vertex_geometry(node(ln.y >> 16), node(vl & 0xffffu), node(vl >> 16), a.vscale,
                        __ldg(a.inv_vol + i), c.g0, c.g1);
      } else {
        c.g0 = Rec<R>::ld(geom + 2 * i);
        c.g1 = Rec<R>::ld(geom + 2 * i + 1);
      }
      c.U = sU[e];
      if (MODE == kModeRK2b) c.base = static_cast<const rec_t<R>*>(a.Ubase)[i];
      if (COMP && MODE != kModeResidual) c.lo = a.lo[i];
      if (COMP && MODE == kModeRK2b) c.lo_stage = a.lo_stage[i];
      R acc[4] = {R(0), R(0), R(0), R(0)};
      const R perim = cell_fluxes<R, WAVE>(c.g0, c.g1, ln, c.U, rec_prim<R>(sP[e]), sU, sP,
                                           far_field<R>(a), acc, nt + h1, a.err);
      finish_cell<R, MODE, COMP>(a, out, i, c, acc, perim, dtR, bmin, ok);
    }
  }
  if (MODE == kModeFE || MODE == kModeRK2b) {
    if (!ok) atomicOr(a.err, 1);
    const double m = (double)block_min<R>(bmin);
    if (threadIdx.x == 0) {
      atomicMin(a.bmin_write, (unsigned long long)__double_as_longlong(m));
      if (blockIdx.x == 0) {
        *a.t_write = t + dt;
        *a.bmin_reset = kInfBits;
      }
    }
  }
}

// Shape 7: the tile shape with each face evaluated once.  Phase 1: the
// threads share the tile's face list (tiles.cpp): every face of a tile cell
// except those whose other side is a tile cell of lower local id (for a cell
// bordering itself across a periodic seam, its lower face); each writes the
// flux value to the slot sF[3e + q] of its cell and, across an inner face,
// the negation to the slot of the face pointing back.  The face
// fluxes are exactly antisymmetric (face_flux_value), so every slot holds the
// bits the cell would compute itself.  Phase 2: every tile cell adds its three
// slots in face order and finishes as the other shapes do: the same bits, with
// about half the face arithmetic.  It pays where the arithmetic is the
// bottleneck (FP64 on GB300); sF costs 3 records per tile cell of shared
// memory.
template <typename R, int MODE, bool COMP, int THREADS, int KMAX, int WAVE>
__global__ void __launch_bounds__(THREADS, 1) k_step_tile_faces(StepArgs a) {
  chain_entry();
  extern __shared__ __align__(128) unsigned char smem_raw[];
  rec_t<R>* sU = reinterpret_cast<rec_t<R>*>(smem_raw);  // [t1_cap] states
  rec_t<R>* sP = sU + a.t1_cap;                            // [t1_cap] (u, v, p, c)
  rec_t<R>* sF = sP + a.t1_cap;                            // [3 tile] face flux values
  const rec_t<R>* __restrict__ U = static_cast<const rec_t<R>*>(a.U);
  const rec_t<R>* __restrict__ geom = static_cast<const rec_t<R>*>(a.geom);
  rec_t<R>* out = static_cast<rec_t<R>*>(a.out);
  const int t0 = blockIdx.x * a.tile;  // cell ids are 32-bit
  const int nt = min(a.tile, (int)a.n - t0);
  const int hs = __ldg(a.tile_info + 2 * blockIdx.x);
  const int h1 = __ldg(a.tile_info + 2 * blockIdx.x + 1);
  __shared__ double s_t, s_dt;
  if (threadIdx.x == 0 && MODE != kModeResidual) block_dt(a, s_t, s_dt);
  stage_states<R, THREADS, kStageBatch<R, KMAX>>(U, t0, nt, h1, a.halo_id + hs, sU, sP, a.n,
                                                 a.err);
  __syncthreads();
  const R* uinf = far_field<R>(a);
  // phase 1: the tile's faces, each once, spread evenly over the threads
  const int f1 = __ldg(a.tile_face_off + blockIdx.x + 1);
  for (int f = __ldg(a.tile_face_off + blockIdx.x) + threadIdx.x; f < f1; f += THREADS) {
    const uint2 r = __ldg(a.tile_face + f);
    const unsigned e = r.x & 0xffffu, q = (r.x >> 16) & 3u, kv = (r.x >> 18) & 3u, v = r.y;
    if (!index_ok(e, nt, a.err)) continue;
    const int i = t0 + (int)e;
    R nx, ny;
    face_normal<R>(geom, i, q, nx, ny);
    const rec_t<R> UL = sU[e];
    const Prim<R> L = rec_prim<R>(sP[e]);
    const bool inner = v < (unsigned)nt;
    rec_t<R> UR;
    Prim<R> W;
    if (v < kGhostCodes) {
      if (index_ok(v, nt + h1, a.err)) {
        UR = sU[v];
        W = rec_prim<R>(sP[v]);
      } else {
        UR = UL;
        W = L;
      }
    } else {
      UR = ghost<R>((int)v - 0x10000, UL, nx, ny, uinf);
      W = primitive<R>(UR);
    }
    R X[4];
    face_flux_value<R, false, WAVE>(UL, L, UR, W, nx, ny, face_len<R>(nx, ny), R(1), X);
    sF[3 * e + q] = Rec<R>::make(X[0], X[1], X[2], X[3]);
    if (inner) sF[3 * v + kv] = Rec<R>::make(-X[0], -X[1], -X[2], -X[3]);
  }
  __syncthreads();
  const double t = MODE != kModeResidual ? s_t : 0.0, dt = MODE != kModeResidual ? s_dt : 0.0;
  const R dtR = R(dt);
  R bmin = R(INFINITY);
  bool ok = true;
  // phase 2: the three face values in face order, then the cell's update
#pragma unroll
  for (int k = 0; k < KMAX; ++k) {
    const int e = threadIdx.x + k * THREADS;
    if (e < nt) {
      const int i = t0 + e;
      CellIn<R> c;
      c.g0 = Rec<R>::ld(geom + 2 * i);
      c.g1 = Rec<R>::ld(geom + 2 * i + 1);
      c.U = sU[e];
      if (MODE == kModeRK2b) c.base = static_cast<const rec_t<R>*>(a.Ubase)[i];
      if (COMP && MODE != kModeResidual) c.lo = a.lo[i];
      if (COMP && MODE == kModeRK2b) c.lo_stage = a.lo_stage[i];
      R acc[4] = {R(0), R(0), R(0), R(0)};
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const rec_t<R> X = sF[3 * e + q];
        acc[0] = add(acc[0], X.x);
        acc[1] = add(acc[1], X.y);
        acc[2] = add(acc[2], X.z);
        acc[3] = add(acc[3], X.w);
      }
      // the perimeter (FP32 forms 2V/P from it; FP64 stores 2V/P)
      R perim = R(0);
      if constexpr (sizeof(R) == 4)
        perim = add(add(face_len<R>(c.g0.x, c.g0.y), face_len<R>(c.g0.z, c.g0.w)),
                    face_len<R>(c.g1.x, c.g1.y));
      finish_cell<R, MODE, COMP>(a, out, i, c, acc, perim, dtR, bmin, ok);
    }
  }
  if (MODE == kModeFE || MODE == kModeRK2b) {
    if (!ok) atomicOr(a.err, 1);
    const double m = (double)block_min<R>(bmin);
    if (threadIdx.x == 0) {
      atomicMin(a.bmin_write, (unsigned long long)__double_as_longlong(m));
      if (blockIdx.x == 0) {
        *a.t_write = t + dt;
        *a.bmin_reset = kInfBits;
      }
    }
  }
}

// Many meshes: each block is one tile of one mesh (tiles never span meshes)
// and uses that mesh's dt, time, far field and CFL-minimum slot; the mesh's
// first tile advances its time and clears its next slot.
template <typename R, int MODE, bool COMP, int THREADS, int KMAX>
__global__ void __launch_bounds__(THREADS) k_step_tile_batch(BatchArgs b) {
  chain_entry();
  const StepArgs& a = b.s;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  rec_t<R>* sU = reinterpret_cast<rec_t<R>*>(smem_raw);  // [t1_cap] states
  rec_t<R>* sP = sU + a.t1_cap;                            // [t1_cap] (u, v, p, c)
  const rec_t<R>* __restrict__ U = static_cast<const rec_t<R>*>(a.U);
  const rec_t<R>* __restrict__ geom = static_cast<const rec_t<R>*>(a.geom);
  rec_t<R>* out = static_cast<rec_t<R>*>(a.out);
  const int tile = blockIdx.x;
  const int m = __ldg(b.tile_mesh + tile);
  const int64_t t0 = __ldg(b.tile_start + tile);
  const int nt = __ldg(b.tile_cells + tile);
  const int hs = __ldg(a.tile_info + 2 * tile);
  const int h1 = __ldg(a.tile_info + 2 * tile + 1);
  __shared__ double s_t, s_dt;
  if (threadIdx.x == 0 && MODE != kModeResidual) {
    const double t = b.t[b.t_read * b.n_meshes + m];
    const unsigned long long bits = b.bmin[b.slot_read * b.n_meshes + m];
    double dt = a.cfl > 0.0 ? a.cfl * __longlong_as_double((long long)bits) : -a.cfl;
    if (a.t_stop > 0.0) {
      const double rem = a.t_stop - t;
      if (rem < dt) dt = rem;
      if (!(dt > 0.0)) dt = 0.0;
    }
    s_t = t;
    s_dt = dt;
  }
  stage_states<R, THREADS, kStageBatch<R, KMAX>>(U, t0, nt, h1, a.halo_id + hs, sU, sP, a.n,
                                                 a.err);
  __syncthreads();
  const double t = MODE != kModeResidual ? s_t : 0.0, dt = MODE != kModeResidual ? s_dt : 0.0;
  const R dtR = R(dt);
  const R* uinf = batch_far_field<R>(b, m);
  R bmin = R(INFINITY);
  bool ok = true;
#pragma unroll
  for (int k = 0; k < KMAX; ++k) {
    const int e = threadIdx.x + k * THREADS;
    if (e < nt) {
      const int64_t i = t0 + e;
      CellIn<R> c;
      c.g0 = Rec<R>::ld(geom + 2 * i);
      c.g1 = Rec<R>::ld(geom + 2 * i + 1);
      c.U = sU[e];
      if (MODE == kModeRK2b) c.base = static_cast<const rec_t<R>*>(a.Ubase)[i];
      if (COMP && MODE != kModeResidual) c.lo = a.lo[i];
      if (COMP && MODE == kModeRK2b) c.lo_stage = a.lo_stage[i];
      const uint2 ln = __ldg(a.cell_ln + i);
      R acc[4] = {R(0), R(0), R(0), R(0)};
      const R perim =
          cell_fluxes<R>(c.g0, c.g1, ln, c.U, rec_prim<R>(sP[e]), sU, sP, uinf, acc, nt + h1, a.err);
      finish_cell<R, MODE, COMP>(a, out, i, c, acc, perim, dtR, bmin, ok);
    }
  }
  if (MODE == kModeFE || MODE == kModeRK2b) {
    if (!ok) atomicOr(a.err, 1);
    const double mn = (double)block_min<R>(bmin);
    if (threadIdx.x == 0) {
      atomicMin(&b.bmin[b.slot_write * b.n_meshes + m], (unsigned long long)__double_as_longlong(mn));
      if (tile == __ldg(b.mesh_first_tile + m)) {
        b.t[b.t_write * b.n_meshes + m] = t + dt;
        b.bmin[b.slot_reset * b.n_meshes + m] = kInfBits;
      }
    }
  }
}

template <typename R, int MODE, bool COMP, int THREADS, int KMAX>
cudaError_t launch_tile_batch_t(const BatchArgs& b, cudaStream_t s) {
  auto k = k_step_tile_batch<R, MODE, COMP, THREADS, KMAX>;
  const size_t smem = tile_smem_bytes(sizeof(R) == 8, b.s.t1_cap);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return launch_chained(k, (unsigned)b.n_tiles, THREADS, smem, s, b.s.chained, b);
}

template <typename R, bool COMP>
cudaError_t launch_tile_batch_mode(int mode, const BatchArgs& b, cudaStream_t s) {
  if (b.s.tile != 1024) return cudaErrorInvalidValue;
  switch (mode) {
    case kModeFE: return launch_tile_batch_t<R, kModeFE, COMP, 256, 4>(b, s);
    case kModeRK2a: return launch_tile_batch_t<R, kModeRK2a, COMP, 256, 4>(b, s);
    case kModeRK2b: return launch_tile_batch_t<R, kModeRK2b, COMP, 256, 4>(b, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename R, int MODE, bool COMP, int THREADS, int KMAX, bool VTX>
cudaError_t launch_tile_t(const StepArgs& a, cudaStream_t s) {
  auto k = a.wave == kWaveMax ? k_step_tile<R, MODE, COMP, THREADS, KMAX, kWaveMax, VTX>
                              : k_step_tile<R, MODE, COMP, THREADS, KMAX, kWaveAverage, VTX>;
  const size_t smem = tile_smem_bytes(sizeof(R) == 8, a.t1_cap, VTX ? a.v_cap : 0);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t tiles = (a.n + a.tile - 1) / a.tile;
  return launch_chained(k, (unsigned)tiles, THREADS, smem, s, a.chained, a);
}

template <typename R, int MODE, bool COMP, int THREADS, int KMAX>
cudaError_t launch_faces_t(const StepArgs& a, cudaStream_t s) {
  auto k = a.wave == kWaveMax ? k_step_tile_faces<R, MODE, COMP, THREADS, KMAX, kWaveMax>
                              : k_step_tile_faces<R, MODE, COMP, THREADS, KMAX, kWaveAverage>;
  const size_t smem = tile_faces_smem_bytes(sizeof(R) == 8, a.t1_cap, a.tile);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t tiles = (a.n + a.tile - 1) / a.tile;
  return launch_chained(k, (unsigned)tiles, THREADS, smem, s, a.chained, a);
}

template <typename R, int MODE, bool COMP>
cudaError_t launch_faces_size(const StepArgs& a, cudaStream_t s) {
  if (a.tile < 1 || a.tile > kMaxTileCells) return cudaErrorInvalidValue;
  if (a.tile <= 512) return launch_faces_t<R, MODE, COMP, 256, 2>(a, s);
  if (a.tile <= 768) return launch_faces_t<R, MODE, COMP, 256, 3>(a, s);
  if (a.tile <= 1024) return launch_faces_t<R, MODE, COMP, 256, 4>(a, s);
  return launch_faces_t<R, MODE, COMP, 512, 4>(a, s);
}

template <typename R, bool COMP>
cudaError_t launch_faces_mode(int mode, const StepArgs& a, cudaStream_t s) {
  switch (mode) {
    case kModeFE: return launch_faces_size<R, kModeFE, COMP>(a, s);
    case kModeRK2a: return launch_faces_size<R, kModeRK2a, COMP>(a, s);
    case kModeRK2b: return launch_faces_size<R, kModeRK2b, COMP>(a, s);
    case kModeResidual: return launch_faces_size<R, kModeResidual, false>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

// Any tile size up to 2048 cells: the block shape whose KMAX x THREADS cells
// cover it (the cells of a tile beyond nt are skipped).
template <typename R, int MODE, bool COMP, bool VTX>
cudaError_t launch_tile_size(const StepArgs& a, cudaStream_t s) {
  if (a.tile < 1 || a.tile > kMaxTileCells) return cudaErrorInvalidValue;
  if (a.tile <= 512) return launch_tile_t<R, MODE, COMP, 256, 2, VTX>(a, s);
  if (a.tile <= 768) return launch_tile_t<R, MODE, COMP, 256, 3, VTX>(a, s);
  if (a.tile <= 1024) return launch_tile_t<R, MODE, COMP, 256, 4, VTX>(a, s);
  return launch_tile_t<R, MODE, COMP, 512, 4, VTX>(a, s);
}

template <typename R, bool COMP, bool VTX = false>
cudaError_t launch_tile_mode(int mode, const StepArgs& a, cudaStream_t s) {
  switch (mode) {
    case kModeFE: return launch_tile_size<R, kModeFE, COMP, VTX>(a, s);
    case kModeRK2a: return launch_tile_size<R, kModeRK2a, COMP, VTX>(a, s);
    case kModeRK2b: return launch_tile_size<R, kModeRK2b, COMP, VTX>(a, s);
    case kModeResidual: return launch_tile_size<R, kModeResidual, false, VTX>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_batch_step_tile(bool f64, int mode, const BatchArgs& b, cudaStream_t s) {
  if (b.n_tiles <= 0) return cudaSuccess;
  if (!b.s.cell_ln || !b.s.tile_info || !b.s.halo_id || !b.tile_mesh) return cudaErrorInvalidValue;
  if (f64) return launch_tile_batch_mode<double, false>(mode, b, s);
  if (b.s.lo) return launch_tile_batch_mode<float, true>(mode, b, s);
  return launch_tile_batch_mode<float, false>(mode, b, s);
}

cudaError_t launch_step_tile_faces(bool f64, int mode, const StepArgs& a, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  if (!a.cell_ln || !a.tile_info || !a.halo_id || a.tile_vq || !a.tile_face_off || !a.tile_face)
    return cudaErrorInvalidValue;
  if (f64) return launch_faces_mode<double, false>(mode, a, s);
  if (a.lo) return launch_faces_mode<float, true>(mode, a, s);
  return launch_faces_mode<float, false>(mode, a, s);
}

cudaError_t launch_step_tile(bool f64, int mode, const StepArgs& a, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  if (!a.cell_ln || !a.tile_info || !a.halo_id) return cudaErrorInvalidValue;
  if (a.tile_vq) {
    if (f64 || !a.cell_vl || !a.tile_voff || !a.inv_vol) return cudaErrorInvalidValue;
    if (a.lo) return launch_tile_mode<float, true, true>(mode, a, s);
    return launch_tile_mode<float, false, true>(mode, a, s);
  }
  if (f64) return launch_tile_mode<double, false>(mode, a, s);
  if (a.lo) return launch_tile_mode<float, true>(mode, a, s);
  return launch_tile_mode<float, false>(mode, a, s);
}

}  // namespace fv
