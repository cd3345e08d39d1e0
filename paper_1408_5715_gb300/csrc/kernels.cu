// kernels.cu -- the fused cell-centred finite-volume step on sm_103a.
//
// One thread updates one triangle T (cell-centric, so no atomics on the
// state): it gathers its own state, its three neighbours' states (or builds
// ghost states at boundary faces), evaluates the Lax-Friedrichs flux of each
// face, sums them into the residual of Eq. 4 and applies the update of
// Sec. 6.2.2 (forward Euler, Eq. 6, or the second stage of Heun's scheme).
// The same thread then evaluates the CFL bound of its new state; a warp
// shuffle and shared-memory block minimum feed one 64-bit atomicMin per
// block, which gives the next step's dt without another pass over memory.
//
// The flux is evaluated without rotating into the face frame: with the
// unnormalised normal n (|n| = face length) and q = u.n,
//   |n| F(U).n-hat = (rho q, rho u q + p n_x, rho v q + p n_y, (E + p) q)
// and |n| (|u-bar_n| + c-bar) = (|q_L + q_R| + |n| (c_L + c_R)) / 2,
// which is algebraically the rotated form of Eq. 7a-7d (rotation R_n of the
// update equation), with the dissipation sign of Eq. 5.
//
// Data layout (all device arrays, one record per cell in the current order):
//   U     4 values per cell (rho, rho u, rho v, E), float4 or 32-byte doubles
//   nbr   int4 per cell: neighbour across faces 0..2, negative = ghost kind
//   geom  8 values per cell: n0x n0y n1x n1y n2x n2y 1/V 2V/P
#include <cuda_runtime.h>

#include <cstdint>

#include "cell_math.cuh"
#include "kernels.h"
#include "launch_util.cuh"

namespace fv {

namespace {

template <typename R, int MODE, bool COMP, int WAVE = kWaveAverage>
__device__ __forceinline__ void update_cell(const StepArgs& a, const rec_t<R>* __restrict__ U,
                                            rec_t<R>* out, int64_t i, const CellIn<R>& c, R dt,
                                            const R* uinf, R& bmin, bool& ok) {
  const rec_t<R>& UL = c.U;
  const Prim<R> L = primitive<R>(UL);
  R acc[4] = {R(0), R(0), R(0), R(0)};
  R perim = add_face_flux<R, WAVE>(UL, L, c.n0, c.g0.x, c.g0.y, U, uinf, acc, a.n, a.err);
  perim = add(perim, add_face_flux<R, WAVE>(UL, L, c.n1, c.g0.z, c.g0.w, U, uinf, acc, a.n, a.err));
  perim = add(perim, add_face_flux<R, WAVE>(UL, L, c.n2, c.g1.x, c.g1.y, U, uinf, acc, a.n, a.err));
  finish_cell<R, MODE, COMP>(a, out, i, c, acc, perim, dt, bmin, ok);
}

// The fused step.  Shape variants (chosen per mesh by the autotuner):
//   VAR 0: one thread per cell, a grid covering all cells;
//   VAR 1: a persistent grid (resident blocks only) walks the cells with a
//          grid stride; the own-cell loads of the next cell are issued before
//          the current cell gathers its neighbours and computes, so each
//          thread keeps two cells' worth of loads in flight;
//   VAR 2: VAR 1 limited to 64 registers (4 blocks of 256 per SM);
//   VAR 3: VAR 0 limited to 40 registers (6 blocks per SM);
//   VAR 4: VAR 0 limited to 32 registers (8 blocks per SM, full occupancy).
// One block minimum per block at the end feeds the next dt.
constexpr bool var_persistent(int v) { return v == 1 || v == 2; }
constexpr int var_min_blocks(int v) { return v == 2 ? 4 : v == 3 ? 6 : v == 4 ? 8 : 1; }

template <typename R, int MODE, bool COMP, int VAR, int WAVE>
__global__ void __launch_bounds__(kBlock, var_min_blocks(VAR)) k_step(StepArgs a) {
  chain_entry();
  const rec_t<R>* __restrict__ U = static_cast<const rec_t<R>*>(a.U);
  const rec_t<R>* __restrict__ geom = static_cast<const rec_t<R>*>(a.geom);
  rec_t<R>* out = static_cast<rec_t<R>*>(a.out);
  double t = 0.0, dt = 0.0;
  if (MODE != kModeResidual) dt = step_dt(a, t);
  const R dtR = R(dt);
  R bmin = R(INFINITY);
  bool ok = true;
  // cell ids are 32-bit (a mesh holds fewer than 2^31 / 3 cells): 32-bit
  // index arithmetic, one wide multiply-add per address
  const int n = (int)a.n;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (!var_persistent(VAR)) {
    if (i < n) {
      CellIn<R> cur;
      load_cell<R, MODE, COMP>(a, U, geom, i, cur);
      update_cell<R, MODE, COMP, WAVE>(a, U, out, i, cur, dtR, far_field<R>(a), bmin, ok);
    }
  } else {
    const int stride = gridDim.x * blockDim.x;
    CellIn<R> cur, nxt;
    if (i < n) load_cell<R, MODE, COMP>(a, U, geom, i, cur);
    for (; i < n; i += stride) {
      const int j = i + stride;
      if (j < n) load_cell<R, MODE, COMP>(a, U, geom, j, nxt);
      update_cell<R, MODE, COMP, WAVE>(a, U, out, i, cur, dtR, far_field<R>(a), bmin, ok);
      cur = nxt;
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

// ---------------------------------------------------------------------------
// Many meshes in one launch.  The meshes are concatenated into one cell range,
// each padded to a multiple of the block size, so every block belongs to one
// mesh; the block looks its mesh up, uses that mesh's dt, time and free
// stream, and feeds that mesh's minimum.  The per-cell work is the same
// load_cell / update_cell as the single-mesh kernel, so each mesh advances
// bit for bit as it would alone.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double batch_step_dt(const BatchArgs& b, int m, double& t) {
  double dt = 0.0;
  t = 0.0;
  if ((threadIdx.x & 31) == 0) {
    t = b.t[b.t_read * b.n_meshes + m];
    const unsigned long long bits = b.bmin[b.slot_read * b.n_meshes + m];
    dt = b.s.cfl > 0.0 ? b.s.cfl * __longlong_as_double((long long)bits) : -b.s.cfl;
    if (b.s.t_stop > 0.0) {
      double rem = b.s.t_stop - t;
      if (rem < dt) dt = rem;
      if (!(dt > 0.0)) dt = 0.0;
    }
  }
  t = __shfl_sync(0xffffffffu, t, 0);
  return __shfl_sync(0xffffffffu, dt, 0);
}

template <typename R, int MODE, bool COMP>
__global__ void __launch_bounds__(kBlock, sizeof(R) == 4 ? 6 : 1) k_step_batch(BatchArgs b) {
  const StepArgs& a = b.s;
  const rec_t<R>* __restrict__ U = static_cast<const rec_t<R>*>(a.U);
  const rec_t<R>* __restrict__ geom = static_cast<const rec_t<R>*>(a.geom);
  rec_t<R>* out = static_cast<rec_t<R>*>(a.out);
  const int m = __ldg(b.block_mesh + blockIdx.x);
  double t = 0.0;
  const double dt = batch_step_dt(b, m, t);
  R bmin = R(INFINITY);
  bool ok = true;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < __ldg(b.mesh_end + m)) {
    CellIn<R> cur;
    load_cell<R, MODE, COMP>(a, U, geom, i, cur);
    update_cell<R, MODE, COMP>(a, U, out, i, cur, R(dt), batch_far_field<R>(b, m), bmin, ok);
  }
  if (MODE == kModeFE || MODE == kModeRK2b) {
    if (!ok) atomicOr(a.err, 1);
    const double mn = (double)block_min<R>(bmin);
    if (threadIdx.x == 0) {
      atomicMin(&b.bmin[b.slot_write * b.n_meshes + m], (unsigned long long)__double_as_longlong(mn));
      if (blockIdx.x == 0 || __ldg(b.block_mesh + blockIdx.x - 1) != m) {  // first block of m
        b.t[b.t_write * b.n_meshes + m] = t + dt;
        b.bmin[b.slot_reset * b.n_meshes + m] = kInfBits;
      }
    }
  }
}

__global__ void k_batch_init(unsigned long long* bmin, double* t, int n_meshes, int* err) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < 3 * n_meshes) bmin[j] = kInfBits;
  if (j < 2 * n_meshes) t[j] = 0.0;
  if (j == 0) *err = 0;
}

template <typename R>
__global__ void __launch_bounds__(kBlock) k_batch_bound(const rec_t<R>* __restrict__ U,
                                                        const rec_t<R>* __restrict__ geom,
                                                        const int* block_mesh,
                                                        const int64_t* mesh_end, int n_meshes,
                                                        unsigned long long* bmin, int* err) {
  const int m = __ldg(block_mesh + blockIdx.x);
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  R bnd = R(INFINITY);
  bool ok = true;
  if (i < __ldg(mesh_end + m)) bnd = cell_bound<R>(Rec<R>::ld(U + i), geom_inradius<R>(geom, i), ok);
  if (!ok) atomicOr(err, 1);
  const double mn = (double)block_min<R>(bnd);
  if (threadIdx.x == 0) atomicMin(&bmin[m], (unsigned long long)__double_as_longlong(mn));
}

// per-mesh totals: one partial per block (blocks never span meshes), then one
// block per mesh adds its blocks' partials in a fixed order
template <typename R>
__global__ void __launch_bounds__(kBlock) k_batch_totals_partial(const rec_t<R>* __restrict__ U,
                                                                 const double* __restrict__ vol,
                                                                 const int* block_mesh,
                                                                 const int64_t* mesh_end,
                                                                 double* partials) {
  const int m = __ldg(block_mesh + blockIdx.x);
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  if (i < __ldg(mesh_end + m)) {
    const rec_t<R> u = Rec<R>::ld(U + i);
    const double v = __ldg(vol + i);
    s[0] = v * (double)u.x;
    s[1] = v * (double)u.y;
    s[2] = v * (double)u.z;
    s[3] = v * (double)u.w;
  }
  __shared__ double sm[4][kBlock / 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    for (int o = 16; o > 0; o >>= 1) s[q] += __shfl_xor_sync(0xffffffffu, s[q], o);
    if (lane == 0) sm[q][warp] = s[q];
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double acc = 0.0;
    for (int w = 0; w < kBlock / 32; ++w) acc += sm[threadIdx.x][w];
    partials[4 * blockIdx.x + threadIdx.x] = acc;
  }
}

__global__ void __launch_bounds__(kBlock) k_batch_totals_final(const double* partials,
                                                               const int* mesh_first_block,
                                                               double* out) {
  const int m = blockIdx.x;
  const int b0 = mesh_first_block[m], b1 = mesh_first_block[m + 1];
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  for (int j = b0 + threadIdx.x; j < b1; j += blockDim.x)
#pragma unroll
    for (int q = 0; q < 4; ++q) s[q] += partials[4 * j + q];
  __shared__ double sm[4][kBlock / 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    for (int o = 16; o > 0; o >>= 1) s[q] += __shfl_xor_sync(0xffffffffu, s[q], o);
    if (lane == 0) sm[q][warp] = s[q];
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double acc = 0.0;
    for (int w = 0; w < kBlock / 32; ++w) acc += sm[threadIdx.x][w];
    out[4 * m + threadIdx.x] = acc;
  }
}

__global__ void k_init_scalars(LoopScalars* d) {
  d->bmin[0] = d->bmin[1] = d->bmin[2] = kInfBits;
  d->t[0] = d->t[1] = 0.0;
  d->err = 0;
}

template <typename R>
__global__ void __launch_bounds__(kBlock) k_bound(const rec_t<R>* __restrict__ U,
                                                  const rec_t<R>* __restrict__ geom, int64_t n,
                                                  unsigned long long* bmin, int* err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  R b = R(INFINITY);
  bool ok = true;
  if (i < n) b = cell_bound<R>(Rec<R>::ld(U + i), geom_inradius<R>(geom, i), ok);
  if (!ok) atomicOr(err, 1);
  const double m = (double)block_min<R>(b);
  if (threadIdx.x == 0) atomicMin(bmin, (unsigned long long)__double_as_longlong(m));
}

__global__ void k_set_u64(unsigned long long* p, unsigned long long v, int* flag) {
  *p = v;
  if (flag) *flag = 0;
}

__global__ void k_dt_from_bound(const unsigned long long* bmin, double cfl, double* dt) {
  *dt = cfl > 0.0 ? cfl * __longlong_as_double((long long)*bmin) : -cfl;
}

// Deterministic totals sum_T V_T U_T in FP64: a fixed grid, a fixed
// thread-to-cell assignment and fixed reduction trees.
template <typename R>
__global__ void __launch_bounds__(kBlock) k_totals_partial(const rec_t<R>* __restrict__ U,
                                                           const double* __restrict__ vol,
                                                           int64_t n, double* partials) {
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const rec_t<R> u = Rec<R>::ld(U + i);
    const double v = __ldg(vol + i);
    s[0] += v * (double)u.x;
    s[1] += v * (double)u.y;
    s[2] += v * (double)u.z;
    s[3] += v * (double)u.w;
  }
  __shared__ double sm[4][kBlock / 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    for (int o = 16; o > 0; o >>= 1) s[q] += __shfl_xor_sync(0xffffffffu, s[q], o);
    if (lane == 0) sm[q][warp] = s[q];
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double acc = 0.0;
    for (int w = 0; w < kBlock / 32; ++w) acc += sm[threadIdx.x][w];
    partials[4 * blockIdx.x + threadIdx.x] = acc;
  }
}

__global__ void __launch_bounds__(kBlock) k_totals_final(const double* partials, int nparts,
                                                         double* out) {
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  for (int j = threadIdx.x; j < nparts; j += blockDim.x)
#pragma unroll
    for (int q = 0; q < 4; ++q) s[q] += partials[4 * j + q];
  __shared__ double sm[4][kBlock / 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    for (int o = 16; o > 0; o >>= 1) s[q] += __shfl_xor_sync(0xffffffffu, s[q], o);
    if (lane == 0) sm[q][warp] = s[q];
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double acc = 0.0;
    for (int w = 0; w < kBlock / 32; ++w) acc += sm[threadIdx.x][w];
    out[threadIdx.x] = acc;
  }
}

inline unsigned grid_for(int64_t n) { return (unsigned)((n + kBlock - 1) / kBlock); }

// Resident blocks of a kernel on the current device (cached per kernel).
template <typename K>
unsigned resident_blocks(K kernel) {
  static int cached = 0;
  if (cached == 0) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBlock, 0) != cudaSuccess ||
        per_sm < 1)
      return 1024;
    cached = sms * per_sm;
  }
  return (unsigned)cached;
}

template <typename R, int MODE, bool COMP, int VAR, int WAVE = kWaveAverage>
cudaError_t launch_one(const StepArgs& a, cudaStream_t s) {
  auto kernel = k_step<R, MODE, COMP, VAR, WAVE>;
  const int64_t want = a.n > 0 ? (a.n + kBlock - 1) / kBlock : 1;  // a time step always runs its scalars
  unsigned g = (unsigned)want;
  if (var_persistent(VAR)) {
    const unsigned cap = resident_blocks(kernel);
    g = (unsigned)(want < (int64_t)cap ? want : cap);
  }
  return launch_chained(kernel, g, kBlock, 0, s, a.chained, a);
}

template <typename R, int MODE, bool COMP>
cudaError_t launch_var(int var, const StepArgs& a, cudaStream_t s) {
  if (a.wave == kWaveMax)  // the Rusanov wave speed is built for shapes 0 and 1
    return var == 0 ? launch_one<R, MODE, COMP, 0, kWaveMax>(a, s)
                    : launch_one<R, MODE, COMP, 1, kWaveMax>(a, s);
  switch (var) {
    case 0: return launch_one<R, MODE, COMP, 0>(a, s);
    case 1: return launch_one<R, MODE, COMP, 1>(a, s);
    case 2: return launch_one<R, MODE, COMP, 2>(a, s);
    case 3: return launch_one<R, MODE, COMP, 3>(a, s);
    case 4: return launch_one<R, MODE, COMP, 4>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename R, bool COMP>
cudaError_t launch_step_t(int mode, int var, const StepArgs& a, cudaStream_t s) {
  if (a.n <= 0 && mode == kModeResidual) return cudaSuccess;
  switch (mode) {
    case kModeFE: return launch_var<R, kModeFE, COMP>(var, a, s);
    case kModeRK2a: return launch_var<R, kModeRK2a, COMP>(var, a, s);
    case kModeRK2b: return launch_var<R, kModeRK2b, COMP>(var, a, s);
    case kModeResidual:
      return a.wave == kWaveMax ? launch_one<R, kModeResidual, false, 0, kWaveMax>(a, s)
                                : launch_one<R, kModeResidual, false, 0>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_step(bool f64, int mode, int variant, const StepArgs& a, cudaStream_t s) {
  if (variant == 5 && a.wave == kWaveMax) variant = 1;  // the staged shape has the averages only
  if (variant == 5 && mode != kModeResidual && a.n > 0) return launch_step_tma(f64, mode, a, s);
  if (variant == kTileVariant && a.cell_ln) return launch_step_tile(f64, mode, a, s);
  if (variant == kFaceTileVariant && a.cell_ln && mode != kModeResidual)
    return launch_step_tile_faces(f64, mode, a, s);
  if (variant == 5 || variant == kTileVariant || variant == kFaceTileVariant) variant = 0;
  if (f64) return launch_step_t<double, false>(mode, variant, a, s);
  return a.lo ? launch_step_t<float, true>(mode, variant, a, s)
              : launch_step_t<float, false>(mode, variant, a, s);
}

cudaError_t launch_batch_step(bool f64, int mode, const BatchArgs& b, int64_t n_blocks,
                              cudaStream_t s) {
  const unsigned g = (unsigned)n_blocks;
  const bool comp = !f64 && b.s.lo != nullptr;
#define FV_BATCH_CASE(R, C)                                                              \
  switch (mode) {                                                                        \
    case kModeFE: k_step_batch<R, kModeFE, C><<<g, kBlock, 0, s>>>(b); break;            \
    case kModeRK2a: k_step_batch<R, kModeRK2a, C><<<g, kBlock, 0, s>>>(b); break;        \
    case kModeRK2b: k_step_batch<R, kModeRK2b, C><<<g, kBlock, 0, s>>>(b); break;        \
    default: return cudaErrorInvalidValue;                                               \
  }
  if (f64) {
    FV_BATCH_CASE(double, false)
  } else if (comp) {
    FV_BATCH_CASE(float, true)
  } else {
    FV_BATCH_CASE(float, false)
  }
#undef FV_BATCH_CASE
  return cudaGetLastError();
}

cudaError_t launch_batch_init(unsigned long long* bmin, double* t, int n_meshes, int* err,
                              cudaStream_t s) {
  k_batch_init<<<(3 * n_meshes + kBlock - 1) / kBlock, kBlock, 0, s>>>(bmin, t, n_meshes, err);
  return cudaGetLastError();
}

cudaError_t launch_batch_bound(bool f64, const void* U, const void* geom, const int* block_mesh,
                               const int64_t* mesh_end, int n_meshes, int64_t n_blocks,
                               unsigned long long* bmin, int* err, cudaStream_t s) {
  if (f64)
    k_batch_bound<double><<<(unsigned)n_blocks, kBlock, 0, s>>>(
        static_cast<const dq4*>(U), static_cast<const dq4*>(geom), block_mesh, mesh_end, n_meshes,
        bmin, err);
  else
    k_batch_bound<float><<<(unsigned)n_blocks, kBlock, 0, s>>>(
        static_cast<const float4*>(U), static_cast<const float4*>(geom), block_mesh, mesh_end,
        n_meshes, bmin, err);
  return cudaGetLastError();
}

cudaError_t launch_batch_totals(bool f64, const void* U, const double* vol, const int* block_mesh,
                                const int64_t* mesh_end, const int* mesh_first_block,
                                int n_meshes, int64_t n_blocks, double* partials, double* out,
                                cudaStream_t s) {
  if (f64)
    k_batch_totals_partial<double><<<(unsigned)n_blocks, kBlock, 0, s>>>(
        static_cast<const dq4*>(U), vol, block_mesh, mesh_end, partials);
  else
    k_batch_totals_partial<float><<<(unsigned)n_blocks, kBlock, 0, s>>>(
        static_cast<const float4*>(U), vol, block_mesh, mesh_end, partials);
  k_batch_totals_final<<<n_meshes, kBlock, 0, s>>>(partials, mesh_first_block, out);
  return cudaGetLastError();
}

cudaError_t launch_init_scalars(LoopScalars* d, cudaStream_t s) {
  k_init_scalars<<<1, 1, 0, s>>>(d);
  return cudaGetLastError();
}

cudaError_t launch_bound(bool f64, const void* U, const void* geom, int64_t n,
                         unsigned long long* bmin, int* err, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (f64)
    k_bound<double><<<grid_for(n), kBlock, 0, s>>>(static_cast<const dq4*>(U),
                                                   static_cast<const dq4*>(geom), n, bmin, err);
  else
    k_bound<float><<<grid_for(n), kBlock, 0, s>>>(static_cast<const float4*>(U),
                                                  static_cast<const float4*>(geom), n, bmin, err);
  return cudaGetLastError();
}

cudaError_t launch_totals(bool f64, const void* U, const double* vol, int64_t n, double* partials,
                          double* out, cudaStream_t s) {
  if (f64)
    k_totals_partial<double><<<kTotalsBlocks, kBlock, 0, s>>>(static_cast<const dq4*>(U), vol, n,
                                                              partials);
  else
    k_totals_partial<float><<<kTotalsBlocks, kBlock, 0, s>>>(static_cast<const float4*>(U), vol,
                                                             n, partials);
  k_totals_final<<<1, kBlock, 0, s>>>(partials, kTotalsBlocks, out);
  return cudaGetLastError();
}

// Restriction of a fine state to coarse cells: for coarse cell c, the
// area-weighted mean of its `kids` fine cells fine_of[c*kids + j], summed in
// FP64 in the order j = 0, 1, ... and written in the coarse precision.
template <typename RF, typename RC>
__global__ void __launch_bounds__(kBlock) k_restrict_mean(const rec_t<RF>* __restrict__ Uf,
                                                          const double* __restrict__ area,
                                                          const int* __restrict__ fine_of,
                                                          int64_t n_coarse, int kids,
                                                          rec_t<RC>* Uc) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_coarse) return;
  double s[4] = {0.0, 0.0, 0.0, 0.0}, v = 0.0;
  for (int j = 0; j < kids; ++j) {
    const int f = __ldg(fine_of + c * kids + j);
    const rec_t<RF> u = Rec<RF>::ld(Uf + f);
    const double a = __ldg(area + f);
    s[0] += a * (double)u.x;
    s[1] += a * (double)u.y;
    s[2] += a * (double)u.z;
    s[3] += a * (double)u.w;
    v += a;
  }
  Uc[c] = Rec<RC>::make((RC)(s[0] / v), (RC)(s[1] / v), (RC)(s[2] / v), (RC)(s[3] / v));
}

cudaError_t launch_restrict_mean(bool fine_f64, bool coarse_f64, const void* Uf, const double* area,
                                 const int* fine_of, int64_t n_coarse, int kids, void* Uc,
                                 cudaStream_t s) {
  if (n_coarse <= 0) return cudaSuccess;
  const unsigned g = grid_for(n_coarse);
  if (fine_f64 && coarse_f64)
    k_restrict_mean<double, double><<<g, kBlock, 0, s>>>(
        static_cast<const dq4*>(Uf), area, fine_of, n_coarse, kids, static_cast<dq4*>(Uc));
  else if (fine_f64)
    k_restrict_mean<double, float><<<g, kBlock, 0, s>>>(
        static_cast<const dq4*>(Uf), area, fine_of, n_coarse, kids, static_cast<float4*>(Uc));
  else if (coarse_f64)
    k_restrict_mean<float, double><<<g, kBlock, 0, s>>>(
        static_cast<const float4*>(Uf), area, fine_of, n_coarse, kids, static_cast<dq4*>(Uc));
  else
    k_restrict_mean<float, float><<<g, kBlock, 0, s>>>(
        static_cast<const float4*>(Uf), area, fine_of, n_coarse, kids, static_cast<float4*>(Uc));
  return cudaGetLastError();
}

cudaError_t launch_reset_min(unsigned long long* bmin, int* flag, cudaStream_t s) {
  k_set_u64<<<1, 1, 0, s>>>(bmin, kInfBits, flag);
  return cudaGetLastError();
}

cudaError_t launch_dt_from_bound(const unsigned long long* bmin, double cfl, double* dt_out,
                                 cudaStream_t s) {
  k_dt_from_bound<<<1, 1, 0, s>>>(bmin, cfl, dt_out);
  return cudaGetLastError();
}

}  // namespace fv
