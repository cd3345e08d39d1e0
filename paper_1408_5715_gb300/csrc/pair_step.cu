// pair_step.cu -- two forward-Euler steps per launch (temporal blocking).
//
// The paper chains processors so that the output of one update feeds the next
// without another trip through memory (Sec. 7).  Here one block owns a tile
// of consecutive cells.  It loads the states of the tile and of its two halo
// rings (tiles.cpp) into shared memory, then
//   step 1: updates tile and first halo, keeping U^{n+1} in shared memory and
//           the tile's remainders in registers;
//   step 2: updates the tile from U^{n+1} and writes U^{n+2}.
// Shared memory holds states only (16 bytes a cell per step); a cell forms
// the primitive variables (Eq. 2) of its neighbours from their states at
// each use, which costs instructions but halves the block's shared memory
// and so doubles the blocks an SM keeps resident.
// Per pair of updates a tile cell moves its state, remainder and geometry
// through DRAM once instead of twice; the price is the halo cells' extra
// loads and the first halo's repeated first step.
//
// Every cell update does exactly the arithmetic of the one-step kernel (the
// same helpers, explicitly rounded), and each primitive is computed by the
// same function from the same state, so a pair is bit for bit two single
// steps with the same dt.  dt: the CFL bound of the state at the start of the
// pair for both steps (or the fixed step), each clamped at t_stop as a single
// step would be.
//
// Two kernel shapes:
//   k_step_pair      one block per tile; every record is loaded through the
//                    caches when it is needed;
//   k_step_pair_tma  persistent blocks walk the tiles; the tile's own records
//                    (state, geometry, local neighbours, remainders: one
//                    contiguous slice of each array) arrive by bulk copies
//                    into one of two shared-memory stages while the block
//                    works on the previous tile, so only the halo cells are
//                    gathered with plain loads.  Waits on the copies are
//                    bounded (a.wait_limit polls); one that gives up sets
//                    error bit 2, the block drains its own copies (bounded)
//                    and returns; if that drain gives up too it sets bit 4
//                    (copies may still land in shared memory).
#include <cuda_runtime.h>

#include <cstdint>

#include "cell_math.cuh"
#include "kernels.h"
#include "launch_util.cuh"
#include "tile_math.cuh"
#include "tma_util.cuh"

namespace fv {

namespace {

// Residual sum of one cell from shared-memory neighbour states (tile_math.cuh):
// entries [0, cap) of sU, their primitives formed from the states.
__device__ __forceinline__ float cell_fluxes(const float4& g0, const float4& g1, uint2 ln,
                                             const float4& UL, const Prim<float>& L,
                                             const float4* sU, const float* uinf, float acc[4],
                                             int cap, int* err) {
  return cell_fluxes<float, kWaveAverage, false>(g0, g1, ln, UL, L, sU, nullptr, uinf, acc, cap,
                                                 err);
}

// Global id of halo entry j (checked in the bounds-checked build; a bad id
// reads cell 0 instead).
__device__ __forceinline__ int halo_cell(const PairArgs& a, int j) {
  const int g = __ldg(a.halo_id + j);
  return index_ok(g, a.n, a.err) ? g : 0;
}

// Forward-Euler update of one cell, plain or compensated (the arithmetic of
// the one-step kernel's update).
template <bool COMP>
__device__ __forceinline__ float4 fe_update(const float4& UL, float invV, const float acc[4],
                                            float dt, uint2 lo_in, uint2& lo_out) {
  // acc holds twice the flux sum (face_flux_acc)
  if (COMP) {
    const float f = mul(mul(-0.5f, dt), invV);
    const float u[4] = {UL.x, UL.y, UL.z, UL.w};
    float lo[4], s[4], e[4];
    unpack_rem(lo_in, lo);
#pragma unroll
    for (int q = 0; q < 4; ++q) s[q] = two_sum(u[q], fma_(f, acc[q], lo[q]), e[q]);
    lo_out = pack_rem(e);
    return make_float4(s[0], s[1], s[2], s[3]);
  }
  const float f = mul(mul(-0.5f, dt), invV);
  return make_float4(fma_(f, acc[0], UL.x), fma_(f, acc[1], UL.y), fma_(f, acc[2], UL.z),
                     fma_(f, acc[3], UL.w));
}

// dt of both steps of the pair, as the one-step kernel would take them
// in turn: the bound (or fixed step) read at the start of the pair, each step
// clamped so the time never passes t_stop.  One thread of the block forms
// them (FP64 scalar work; GB300's FP64 pipe is narrow) and the block reads
// them from shared memory after its next barrier.
struct PairDt {
  double t, dt1, dt2;
  float dt1f, dt2f;
};

__device__ __forceinline__ void pair_dt(const PairArgs& a, PairDt& d) {
  const double t = *a.t_read;
  const double dt = a.cfl > 0.0 ? a.cfl * __longlong_as_double((long long)*a.bmin_read) : -a.cfl;
  double dt1 = dt, dt2 = dt;
  if (a.t_stop > 0.0) {
    const double rem1 = a.t_stop - t;
    if (rem1 < dt1) dt1 = rem1;
    if (!(dt1 > 0.0)) dt1 = 0.0;
    const double rem2 = a.t_stop - (t + dt1);
    if (rem2 < dt2) dt2 = rem2;
    if (!(dt2 > 0.0)) dt2 = 0.0;
  }
  d.t = t;
  d.dt1 = dt1;
  d.dt2 = dt2;
  d.dt1f = (float)dt1;
  d.dt2f = (float)dt2;
}

// Step 1 of one cell (tile or first halo) from the states of the pair's start:
// writes U^{n+1} to shared memory, returns the remainder; `check` tests the
// new state as the one-step kernel does.
template <bool COMP>
__device__ __forceinline__ uint2 step1_cell(const float4& g0, const float4& g1, uint2 ln,
                                            uint2 lo0, int e, const float4* sU0, float4* sU1,
                                            const float* uinf, float dt, bool check, bool& ok,
                                            int cap, int* err) {
  const float4 UL = sU0[e];
  const Prim<float> L = primitive<float>(UL);
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  const float perim = cell_fluxes(g0, g1, ln, UL, L, sU0, uinf, acc, cap, err);
  uint2 lo1 = make_uint2(0u, 0u);
  const float4 U1 = fe_update<COMP>(UL, g1.z, acc, dt, lo0, lo1);
  sU1[e] = U1;
  if (check) {
    bool c_ok;
    bound_of<float>(U1, primitive<float>(U1), inradius<float>(g1, perim), c_ok);
    ok = ok && c_ok;
  }
  return lo1;
}

// Step 2 of one tile cell from U^{n+1}: the new state and remainder, the CFL
// bound folded into bmin.
template <bool COMP>
__device__ __forceinline__ float4 step2_cell(const float4& g0, const float4& g1, uint2 ln,
                                             uint2 lo1, int e, const float4* sU1,
                                             const float* uinf, float dt, uint2& lo2, float& bmin,
                                             bool& ok, int cap, int* err) {
  const float4 UL = sU1[e];
  const Prim<float> L = primitive<float>(UL);
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  const float perim = cell_fluxes(g0, g1, ln, UL, L, sU1, uinf, acc, cap, err);
  const float4 U2 = fe_update<COMP>(UL, g1.z, acc, dt, lo1, lo2);
  bool c_ok;
  bmin = fmin(bmin, cell_bound<float>(U2, inradius<float>(g1, perim), c_ok));
  ok = ok && c_ok;
  return U2;
}

// Step 1 of the first-halo cells of a tile (global gathers); their states are
// checked by the tiles that own them.
// ne: the entries staged in sU0 (tile and both halos).
template <int THREADS, bool COMP>
__device__ __forceinline__ void step1_halo(const PairArgs& a, int nt, int hs, int h1, int ne,
                                           const float4* sU0, float4* sU1, float dt) {
  for (int e = nt + threadIdx.x; e < nt + h1; e += THREADS) {
    const int j = hs + (e - nt);
    const int g = halo_cell(a, j);
    const float4 g0 = __ldg(a.geom + 2 * g), g1 = __ldg(a.geom + 2 * g + 1);
    const uint2 ln = __ldg(a.halo_ln + j);
    const uint2 lo0 = COMP ? __ldg(a.lo_in + g) : make_uint2(0u, 0u);
    bool unused = true;
    step1_cell<COMP>(g0, g1, ln, lo0, e, sU0, sU1, a.uinf, dt, false, unused, ne, a.err);
  }
}

// The pair's minimum and time (one block minimum per block).
__device__ __forceinline__ void pair_finish(const PairArgs& a, float bmin, bool ok, double t,
                                            double dt1, double dt2) {
  if (!ok) atomicOr(a.err, 1);
  const double m = (double)block_min<float>(bmin);
  if (threadIdx.x == 0) {
    atomicMin(a.bmin_write, (unsigned long long)__double_as_longlong(m));
    if (blockIdx.x == 0) {
      const double t1 = t + dt1;
      *a.t_write = t1 + dt2;
      *a.bmin_reset = kInfBits;
    }
  }
}

template <int THREADS, int KMAX, bool COMP>
__global__ void __launch_bounds__(THREADS) k_step_pair(PairArgs a) {
  chain_entry();
  extern __shared__ float4 smem[];
  float4* sU0 = smem;              // [e_cap]  U^n of tile + both halos
  float4* sU1 = smem + a.e_cap;    // [t1_cap] U^{n+1} of tile + first halo
  const int t0 = blockIdx.x * a.tile;  // cell ids are 32-bit
  const int nt = min(a.tile, (int)a.n - t0);
  const int hs = __ldg(a.tile_info + 2 * blockIdx.x);
  const int h1 = __ldg(a.tile_info + 2 * blockIdx.x + 1);
  const int h12 = __ldg(a.tile_info + 2 * blockIdx.x + 2) - hs;  // both halos
  __shared__ PairDt sdt;
  if (threadIdx.x == 0) pair_dt(a, sdt);

  // states at the start of the pair
  for (int e = threadIdx.x; e < nt + h12; e += THREADS) {
    const int g = e < nt ? t0 + e : halo_cell(a, hs + (e - nt));
    sU0[e] = __ldg(a.U + g);
  }
  __syncthreads();
  const float dt1f = sdt.dt1f, dt2f = sdt.dt2f;

  // step 1: tile cells (remainders stay in registers), then the first halo
  bool ok = true;
  uint2 lo1[KMAX];
#pragma unroll
  for (int k = 0; k < KMAX; ++k) {
    const int e = threadIdx.x + k * THREADS;
    lo1[k] = make_uint2(0u, 0u);
    if (e < nt) {
      const int g = t0 + e;
      const uint2 lo0 = COMP ? __ldg(a.lo_in + g) : make_uint2(0u, 0u);
      lo1[k] = step1_cell<COMP>(__ldg(a.geom + 2 * g), __ldg(a.geom + 2 * g + 1),
                                __ldg(a.cell_ln + g), lo0, e, sU0, sU1, a.uinf, dt1f, true, ok,
                                nt + h12, a.err);
    }
  }
  step1_halo<THREADS, COMP>(a, nt, hs, h1, nt + h12, sU0, sU1, dt1f);
  __syncthreads();

  // step 2: the tile, from U^{n+1}
  float bmin = INFINITY;
#pragma unroll
  for (int k = 0; k < KMAX; ++k) {
    const int e = threadIdx.x + k * THREADS;
    if (e < nt) {
      const int g = t0 + e;
      uint2 lo2;
      const float4 U2 = step2_cell<COMP>(__ldg(a.geom + 2 * g), __ldg(a.geom + 2 * g + 1),
                                         __ldg(a.cell_ln + g), lo1[k], e, sU1, a.uinf, dt2f, lo2,
                                         bmin, ok, nt + h1, a.err);
      a.out[g] = U2;
      if (COMP) a.lo_out[g] = lo2;
    }
  }
  pair_finish(a, bmin, ok, sdt.t, sdt.dt1, sdt.dt2);
}

// One stage of the staged kernel: a tile's slices of the state, geometry,
// local neighbours and remainders.
template <int TILE, bool COMP>
struct __align__(128) PairStage {
  float4 U[TILE];
  float4 geom[2 * TILE];
  uint2 ln[TILE];
  uint2 lo[COMP ? TILE : 2];
};

// Issues the bulk copies of tile b (nt cells) into stage st.  Sizes are
// multiples of 16 bytes: 16- and 32-byte records of nt cells, 8-byte records
// of nt rounded up to even (the library's arrays are padded to 256 cells).
template <int TILE, bool COMP>
__device__ __forceinline__ void issue_pair_tile(const PairArgs& a, PairStage<TILE, COMP>& st,
                                                uint64_t* bar, int64_t b, unsigned nt) {
  const int64_t c0 = b * TILE;
  const unsigned n2 = (nt + 1u) & ~1u;
  mbar_expect_tx(bar, nt * 16u + nt * 32u + n2 * 8u + (COMP ? n2 * 8u : 0u));
  bulk_copy(st.U, a.U + c0, nt * 16u, bar);
  bulk_copy(st.geom, a.geom + 2 * c0, nt * 32u, bar);
  bulk_copy(st.ln, a.cell_ln + c0, n2 * 8u, bar);
  if (COMP) bulk_copy(st.lo, a.lo_in + c0, n2 * 8u, bar);
}

template <int THREADS, int KMAX, bool COMP>
__global__ void __launch_bounds__(THREADS) k_step_pair_tma(PairArgs a) {
  constexpr int TILE = THREADS * KMAX;
  using Stage = PairStage<TILE, COMP>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  Stage* stages = reinterpret_cast<Stage*>(smem_raw);
  float4* sU0 = reinterpret_cast<float4*>(smem_raw + 2 * sizeof(Stage));
  float4* sU1 = sU0 + a.e_cap;
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ int abort_flag;
  __shared__ PairDt sdt;
  const int tid = threadIdx.x;
  const int64_t ntiles = (a.n + TILE - 1) / TILE;
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    abort_flag = 0;
    pair_dt(a, sdt);
  }
  __syncthreads();
  const float dt1f = sdt.dt1f, dt2f = sdt.dt2f;
  auto tile_count = [&](int64_t b) {
    const int64_t rem = a.n - b * TILE;
    return (unsigned)(rem < TILE ? rem : TILE);
  };
  int64_t b = blockIdx.x;
  // bit s: parity of stage s's barrier; copies issued into stage s, not yet waited for
  unsigned phase = 0u, pending = 0u;
  for (int s = 0; s < 2; ++s) {
    const int64_t bb = b + (int64_t)s * gridDim.x;
    if (bb < ntiles) {
      pending |= 1u << s;
      if (tid == 0) issue_pair_tile<TILE, COMP>(a, stages[s], &bars[s], bb, tile_count(bb));
    }
  }
  float bmin = INFINITY;
  bool ok = true;
  for (int k = 0; b < ntiles; ++k, b += gridDim.x) {
    const int s = k & 1;
    Stage& st = stages[s];
    if (!mbar_wait(&bars[s], (phase >> s) & 1u, a.wait_limit)) atomicExch(&abort_flag, 1);
    __syncthreads();
    if (abort_flag) break;
    phase ^= 1u << s;
    pending &= ~(1u << s);
    const int64_t t0 = b * TILE;
    const int nt = (int)tile_count(b);
    const int hs = __ldg(a.tile_info + 2 * b);
    const int h1 = __ldg(a.tile_info + 2 * b + 1);
    const int h12 = __ldg(a.tile_info + 2 * b + 2) - hs;
    for (int e = tid; e < nt + h12; e += THREADS)
      sU0[e] = e < nt ? st.U[e] : __ldg(a.U + halo_cell(a, hs + (e - nt)));
    __syncthreads();
    uint2 lo1[KMAX];
#pragma unroll
    for (int q = 0; q < KMAX; ++q) {
      const int e = tid + q * THREADS;
      lo1[q] = make_uint2(0u, 0u);
      if (e < nt)
        lo1[q] = step1_cell<COMP>(st.geom[2 * e], st.geom[2 * e + 1], st.ln[e],
                                  COMP ? st.lo[e] : make_uint2(0u, 0u), e, sU0, sU1, a.uinf,
                                  dt1f, true, ok, nt + h12, a.err);
    }
    step1_halo<THREADS, COMP>(a, nt, hs, h1, nt + h12, sU0, sU1, dt1f);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < KMAX; ++q) {
      const int e = tid + q * THREADS;
      if (e < nt) {
        uint2 lo2;
        const float4 U2 = step2_cell<COMP>(st.geom[2 * e], st.geom[2 * e + 1], st.ln[e], lo1[q],
                                           e, sU1, a.uinf, dt2f, lo2, bmin, ok, nt + h1, a.err);
        a.out[t0 + e] = U2;
        if (COMP) a.lo_out[t0 + e] = lo2;
      }
    }
    __syncthreads();  // the stage and the working arrays are free again
    if (tid == 0) {
      const int64_t nb = b + 2 * (int64_t)gridDim.x;
      if (nb < ntiles) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue_pair_tile<TILE, COMP>(a, st, &bars[s], nb, tile_count(nb));
      }
    }
    if (b + 2 * (int64_t)gridDim.x < ntiles) pending |= 1u << s;
  }
  if (abort_flag) {
    // record the timeout, then drain this block's copies still in flight
    if (tid == 0) {
      atomicOr(a.err, 2);
      for (int s = 0; s < 2; ++s)
        if (((pending >> s) & 1u) && !mbar_wait(&bars[s], (phase >> s) & 1u, a.drain_limit))
          atomicOr(a.err, 4);  // copies may still land: the device state is suspect
    }
    __syncthreads();
    return;
  }
  pair_finish(a, bmin, ok, sdt.t, sdt.dt1, sdt.dt2);
}

template <typename K>
cudaError_t smem_attr(K k, size_t smem) {
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <int THREADS, int KMAX, bool COMP>
cudaError_t launch_plain_t(const PairArgs& a, cudaStream_t s) {
  const size_t smem = pair_smem_bytes(a.e_cap, a.t1_cap, a.tile, false);
  const int64_t tiles = (a.n + a.tile - 1) / a.tile;
  auto k = k_step_pair<THREADS, KMAX, COMP>;
  cudaError_t e = smem_attr(k, smem);
  if (e != cudaSuccess) return e;
  return launch_chained(k, (unsigned)tiles, THREADS, smem, s, a.chained, a);
}

template <int THREADS, int KMAX, bool COMP>
cudaError_t launch_staged_t(const PairArgs& a, cudaStream_t s) {
  const size_t smem = pair_smem_bytes(a.e_cap, a.t1_cap, a.tile, true);
  const int64_t tiles = (a.n + a.tile - 1) / a.tile;
  auto k = k_step_pair_tma<THREADS, KMAX, COMP>;
  cudaError_t e = smem_attr(k, smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, THREADS, smem)) != cudaSuccess)
    return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int64_t cap = (int64_t)sms * per_sm;
  k<<<(unsigned)(tiles < cap ? tiles : cap), THREADS, smem, s>>>(a);
  return cudaGetLastError();
}

template <int THREADS, int KMAX>
cudaError_t launch_plain(const PairArgs& a, cudaStream_t s) {
  return a.lo_in ? launch_plain_t<THREADS, KMAX, true>(a, s)
                 : launch_plain_t<THREADS, KMAX, false>(a, s);
}

template <int THREADS, int KMAX>
cudaError_t launch_staged(const PairArgs& a, cudaStream_t s) {
  return a.lo_in ? launch_staged_t<THREADS, KMAX, true>(a, s)
                 : launch_staged_t<THREADS, KMAX, false>(a, s);
}

}  // namespace

cudaError_t launch_step_pair(const PairArgs& a, int staged, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  if (staged) {
    // the tile's records arrive by 16-byte-aligned bulk copies
    if ((reinterpret_cast<uintptr_t>(a.U) & 15u) != 0) return cudaErrorMisalignedAddress;
    switch (a.tile) {
      case 512: return launch_staged<512, 1>(a, s);
      case 1024: return launch_staged<1024, 1>(a, s);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (a.tile) {
    case 512: return launch_plain<256, 2>(a, s);
    case 768: return launch_plain<256, 3>(a, s);
    case 1024: return launch_plain<256, 4>(a, s);
    case 2048: return launch_plain<512, 4>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fv
