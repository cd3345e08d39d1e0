// tma_step.cu -- the fused step with its per-cell records staged through
// shared memory by the Tensor Memory Accelerator (shape variant 5).
//
// A persistent block owns tiles of kTile consecutive cells (tile = block,
// block + grid, ...).  For each tile one thread issues 1D bulk copies
// (cp.async.bulk) of the tile's slices of the state, geometry, neighbour ids
// and remainders into one of two shared-memory stages; the copies complete on
// that stage's mbarrier.  While the block computes tile k from one stage, the
// copies of tile k+1 are in flight into the other, so the loads stay in
// flight without holding registers.  A neighbour that lies in the current
// tile is read from shared memory; others come through L1/L2.
//
// Every wait on an mbarrier is bounded by a_.wait_limit polls.  When a wait
// gives up, the kernel sets bit 2 of the error word (the host reports
// FV_ETIMEOUT), stops computing, waits (bounded again) for its own copies
// still in flight and returns.  If that second wait gives up too it also sets
// bit 4 (the host reports FV_ESTATE: copies may still be landing).
#include <cuda_runtime.h>

#include <cstdint>

#include "cell_math.cuh"
#include "kernels.h"
#include "tma_util.cuh"

namespace fv {

namespace {

constexpr int kTile = kBlock;  // cells per tile = threads per block

template <typename R>
struct TileLayout {
  // byte sizes of one cell's records
  static constexpr unsigned kU = sizeof(rec_t<R>);
  static constexpr unsigned kGeom = 2 * sizeof(rec_t<R>);
  static constexpr unsigned kNbr = sizeof(R) == 8 ? 16 : 8;
  static constexpr unsigned kLo = 8;
};

template <typename R, int MODE, bool COMP>
struct __align__(128) TileStage {
  rec_t<R> U[kTile];
  rec_t<R> geom[2 * kTile];
  unsigned char nbr[kTile * TileLayout<R>::kNbr];
  rec_t<R> base[MODE == kModeRK2b ? kTile : 1];
  uint2 lo[COMP ? kTile : 1];
  uint2 lo_stage[(COMP && MODE == kModeRK2b) ? kTile : 1];
};

// Issues the copies of tile `t` into stage `st`; the tile holds `cnt` cells.
// Library-owned arrays are padded to whole tiles, so their slices are always
// whole multiples of 16 bytes; the caller's state is 16 or 32 bytes a cell.
template <typename R, int MODE, bool COMP>
__device__ __forceinline__ void issue_tile(const StepArgs& a, TileStage<R, MODE, COMP>& st,
                                           uint64_t* bar, int64_t t, unsigned cnt) {
  using L = TileLayout<R>;
  const int64_t c0 = t * kTile;
  const unsigned full = kTile;
  unsigned bytes = cnt * L::kU + full * (L::kGeom + L::kNbr);
  if (MODE == kModeRK2b) bytes += cnt * L::kU;
  if (COMP) bytes += full * L::kLo;
  if (COMP && MODE == kModeRK2b) bytes += full * L::kLo;
  mbar_expect_tx(bar, bytes);
  bulk_copy(st.U, static_cast<const rec_t<R>*>(a.U) + c0, cnt * L::kU, bar);
  bulk_copy(st.geom, static_cast<const rec_t<R>*>(a.geom) + 2 * c0, full * L::kGeom, bar);
  bulk_copy(st.nbr, static_cast<const unsigned char*>(a.nbr) + c0 * L::kNbr, full * L::kNbr, bar);
  if (MODE == kModeRK2b)
    bulk_copy(st.base, static_cast<const rec_t<R>*>(a.Ubase) + c0, cnt * L::kU, bar);
  if (COMP) bulk_copy(st.lo, a.lo + c0, full * L::kLo, bar);
  if (COMP && MODE == kModeRK2b) bulk_copy(st.lo_stage, a.lo_stage + c0, full * L::kLo, bar);
}

// dt and time of mesh m in a batch (lane 0 of each warp reads, then broadcast)
__device__ __forceinline__ double tma_batch_dt(const BatchArgs& b, int m, double& t) {
  double dt = 0.0;
  t = 0.0;
  if ((threadIdx.x & 31) == 0) {
    t = b.t[b.t_read * b.n_meshes + m];
    const unsigned long long bits = b.bmin[b.slot_read * b.n_meshes + m];
    dt = b.s.cfl > 0.0 ? b.s.cfl * __longlong_as_double((long long)bits) : -b.s.cfl;
    if (b.s.t_stop > 0.0) {
      const double rem = b.s.t_stop - t;
      if (rem < dt) dt = rem;
      if (!(dt > 0.0)) dt = 0.0;
    }
  }
  t = __shfl_sync(0xffffffffu, t, 0);
  return __shfl_sync(0xffffffffu, dt, 0);
}

// BATCH: the tiles are the 256-cell blocks of a batch; each tile uses its
// mesh's dt, time, free stream and CFL-minimum slot (see BatchArgs).
template <typename R, int MODE, bool COMP, bool BATCH>
__global__ void __launch_bounds__(kBlock) k_step_tma(BatchArgs b) {
  const StepArgs& a = b.s;
  using Stage = TileStage<R, MODE, COMP>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  Stage* stages = reinterpret_cast<Stage*>(smem_raw);
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ int abort_flag;
  const rec_t<R>* __restrict__ U = static_cast<const rec_t<R>*>(a.U);
  rec_t<R>* out = static_cast<rec_t<R>*>(a.out);
  const int tid = threadIdx.x;
  const int64_t ntiles = (a.n + kTile - 1) / kTile;
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    abort_flag = 0;
  }
  __syncthreads();
  double t = 0.0, dt = 0.0;
  if (!BATCH) dt = step_dt(a, t);
  R bmin = R(INFINITY);
  bool ok = true;
  auto tile_count = [&](int64_t tt) {
    const int64_t rem = a.n - tt * kTile;
    return (unsigned)(rem < kTile ? rem : kTile);
  };
  // prologue: the first two tiles of this block
  int64_t tile = blockIdx.x;
  if (tid == 0) {
    for (int s = 0; s < 2; ++s) {
      const int64_t tt = tile + (int64_t)s * gridDim.x;
      if (tt < ntiles) issue_tile<R, MODE, COMP>(a, stages[s], &bars[s], tt, tile_count(tt));
    }
  }
  unsigned phase[2] = {0u, 0u};
  int issued_not_waited[2] = {0, 0};
  for (int s = 0; s < 2; ++s) issued_not_waited[s] = (tile + (int64_t)s * gridDim.x) < ntiles;
  for (int k = 0; tile < ntiles; ++k, tile += gridDim.x) {
    const int s = k & 1;
    Stage& st = stages[s];
    // every thread waits for the stage (bounded)
    const bool arrived = mbar_wait(&bars[s], phase[s], a.wait_limit);
    if (!arrived) atomicExch(&abort_flag, 1);
    __syncthreads();
    if (abort_flag) break;
    phase[s] ^= 1u;
    issued_not_waited[s] = 0;
    const int64_t i = tile * kTile + tid;
    int m = 0;
    int64_t end = a.n;
    const R* uinf = far_field<R>(a);
    if (BATCH) {
      m = __ldg(b.block_mesh + tile);
      end = __ldg(b.mesh_end + m);
      uinf = batch_far_field<R>(b, m);
      dt = tma_batch_dt(b, m, t);
      bmin = R(INFINITY);
    }
    const R dtR = R(dt);
    if (i < end) {
      CellIn<R> c;
      c.g0 = st.geom[2 * tid];
      c.g1 = st.geom[2 * tid + 1];
      if constexpr (sizeof(R) == 8) {
        const int4 nb = reinterpret_cast<const int4*>(st.nbr)[tid];
        c.n0 = nb.x, c.n1 = nb.y, c.n2 = nb.z;
      } else {
        const int2 nb = reinterpret_cast<const int2*>(st.nbr)[tid];
        c.n0 = __float_as_int(c.g1.w), c.n1 = nb.x, c.n2 = nb.y;
      }
      c.U = st.U[tid];
      if (MODE == kModeRK2b) c.base = st.base[tid];
      if (COMP) c.lo = st.lo[tid];
      if (COMP && MODE == kModeRK2b) c.lo_stage = st.lo_stage[tid];
      const Prim<R> L = primitive<R>(c.U);
      R acc[4] = {R(0), R(0), R(0), R(0)};
      const int nb[3] = {c.n0, c.n1, c.n2};
      const R nx[3] = {c.g0.x, c.g0.z, c.g1.x};
      const R ny[3] = {c.g0.y, c.g0.w, c.g1.y};
      const int64_t t0 = tile * kTile;
      R perim = R(0);
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        rec_t<R> UR;
        if (nb[q] >= 0) {
          const int64_t local = (int64_t)nb[q] - t0;
          UR = (local >= 0 && local < kTile && (int64_t)nb[q] < end) ? st.U[local]
               : index_ok(nb[q], a.n, a.err)                         ? Rec<R>::ld(U + nb[q])
                                                                      : c.U;
        } else {
          UR = ghost<R>(nb[q], c.U, nx[q], ny[q], uinf);
        }
        const Prim<R> W = primitive<R>(UR);
        const R len = face_len<R>(nx[q], ny[q]);
        face_flux_acc<R, false>(c.U, L, UR, W, nx[q], ny[q], len, R(1), acc);
        perim = q == 0 ? len : add(perim, len);
      }
      finish_cell<R, MODE, COMP>(a, out, i, c, acc, perim, dtR, bmin, ok);
    }
    if (BATCH && (MODE == kModeFE || MODE == kModeRK2b)) {
      // this tile's mesh: its minimum, and (first tile of the mesh) its time
      const double mn = (double)block_min<R>(bmin);
      if (tid == 0) {
        atomicMin(&b.bmin[b.slot_write * b.n_meshes + m],
                  (unsigned long long)__double_as_longlong(mn));
        if (tile == 0 || __ldg(b.block_mesh + tile - 1) != m) {
          b.t[b.t_write * b.n_meshes + m] = t + dt;
          b.bmin[b.slot_reset * b.n_meshes + m] = kInfBits;
        }
      }
    }
    __syncthreads();  // the stage is free again
    if (tid == 0) {
      const int64_t nt = tile + 2 * (int64_t)gridDim.x;
      if (nt < ntiles) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue_tile<R, MODE, COMP>(a, st, &bars[s], nt, tile_count(nt));
        issued_not_waited[s] = 1;
      }
    }
  }
  if (abort_flag) {
    // record the timeout, then drain this block's copies still in flight
    if (tid == 0) {
      atomicOr(a.err, 2);
      for (int s = 0; s < 2; ++s)
        if (issued_not_waited[s] && !mbar_wait(&bars[s], phase[s], a.drain_limit))
          atomicOr(a.err, 4);  // copies may still land: the device state is suspect
    }
    __syncthreads();
    return;
  }
  if (MODE == kModeFE || MODE == kModeRK2b) {
    if (!ok) atomicOr(a.err, 1);
    if (!BATCH) {
      const double mn = (double)block_min<R>(bmin);
      if (tid == 0) {
        atomicMin(a.bmin_write, (unsigned long long)__double_as_longlong(mn));
        if (blockIdx.x == 0) {
          *a.t_write = t + dt;
          *a.bmin_reset = kInfBits;
        }
      }
    }
  }
}

template <typename R, int MODE, bool COMP, bool BATCH>
cudaError_t launch_tma_t(const BatchArgs& ba, cudaStream_t s) {
  const StepArgs& a = ba.s;
  auto kernel = k_step_tma<R, MODE, COMP, BATCH>;
  const size_t smem = 2 * sizeof(TileStage<R, MODE, COMP>);
  static int cap = 0;
  if (cap == 0) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBlock, smem) !=
            cudaSuccess ||
        per_sm < 1)
      return cudaErrorInvalidConfiguration;
    cap = sms * per_sm;
  }
  const int64_t ntiles = a.n > 0 ? (a.n + kTile - 1) / kTile : 1;
  const unsigned g = (unsigned)(ntiles < cap ? ntiles : cap);
  kernel<<<g, kBlock, smem, s>>>(ba);
  return cudaGetLastError();
}

}  // namespace

template <bool BATCH>
cudaError_t launch_tma_any(bool f64, int mode, const BatchArgs& b, cudaStream_t s) {
  const bool comp = !f64 && b.s.lo != nullptr;
#define FV_TMA_CASES(R, C)                                                   \
  switch (mode) {                                                            \
    case kModeFE: return launch_tma_t<R, kModeFE, C, BATCH>(b, s);           \
    case kModeRK2a: return launch_tma_t<R, kModeRK2a, C, BATCH>(b, s);       \
    case kModeRK2b: return launch_tma_t<R, kModeRK2b, C, BATCH>(b, s);       \
    default: return cudaErrorInvalidValue;                                   \
  }
  if (f64) {
    FV_TMA_CASES(double, false)
  } else if (comp) {
    FV_TMA_CASES(float, true)
  } else {
    FV_TMA_CASES(float, false)
  }
#undef FV_TMA_CASES
}

cudaError_t launch_step_tma(bool f64, int mode, const StepArgs& a, cudaStream_t s) {
  BatchArgs b{};
  b.s = a;
  return launch_tma_any<false>(f64, mode, b, s);
}

cudaError_t launch_batch_step_tma(bool f64, int mode, const BatchArgs& b, cudaStream_t s) {
  return launch_tma_any<true>(f64, mode, b, s);
}

}  // namespace fv
