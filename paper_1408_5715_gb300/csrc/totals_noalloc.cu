// totals_noalloc.cu -- conserved totals for callers that cannot allocate
// device memory.
//
// fv_conserved_totals keeps its per-block partial sums in memory that the
// mesh allocates with cudaMalloc on first use.  Some callers must not
// allocate: a library running inside a framework whose caching allocator owns
// the device memory budget, or a latency-critical loop where cudaMalloc's
// implicit device-wide synchronisation would stall unrelated streams.  This
// variant keeps its partial sums in the file-scope array below instead: it
// is part of the loaded module, so every GPU that loads the library holds it
// (kNoAllocTiles * 4 doubles = 128 KiB) until the process exits.
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "fv.h"

// fv_last_error's storage lives in capi.cu.
namespace fv {
int record_error(int code, const std::string& msg);
}

namespace {

constexpr int kTileThreads = 256;
constexpr int kTileCellsPerThread = 16;
constexpr int64_t kTileCells = (int64_t)kTileThreads * kTileCellsPerThread;  // 4096
constexpr int kNoAllocTiles = 4096;

// One partial (mass, x-momentum, y-momentum, energy) per tile of 4096 cells.
static __device__ __align__(256) double g_noalloc_partials[kNoAllocTiles * 4];

struct __align__(32) dq4n {
  double x, y, z, w;
};

template <typename R>
struct Q;
template <>
struct Q<float> {
  using T = float4;
};
template <>
struct Q<double> {
  using T = dq4n;
};

// Each block sums V_T U_T over its tile in a fixed order and writes one partial.
template <typename R>
__global__ void __launch_bounds__(kTileThreads) k_tile_totals(const typename Q<R>::T* __restrict__ U,
                                                              const double* __restrict__ vol,
                                                              int64_t n, double* partials) {
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  const int64_t base = (int64_t)blockIdx.x * kTileCells;
  for (int j = 0; j < kTileCellsPerThread; ++j) {
    const int64_t i = base + (int64_t)j * kTileThreads + threadIdx.x;
    if (i < n) {
      const typename Q<R>::T u = U[i];
      const double v = vol[i];
      s[0] += v * (double)u.x;
      s[1] += v * (double)u.y;
      s[2] += v * (double)u.z;
      s[3] += v * (double)u.w;
    }
  }
  __shared__ double sm[4][kTileThreads / 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    for (int o = 16; o > 0; o >>= 1) s[q] += __shfl_xor_sync(0xffffffffu, s[q], o);
    if (lane == 0) sm[q][warp] = s[q];
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double acc = 0.0;
    for (int w = 0; w < kTileThreads / 32; ++w) acc += sm[threadIdx.x][w];
    partials[4 * blockIdx.x + threadIdx.x] = acc;
  }
}

// One block adds the tile partials in a fixed order.  Every partial it reads
// was written by k_tile_totals earlier in the same call, so nothing in the
// scratch array has to start at zero.
__global__ void __launch_bounds__(kTileThreads) k_tile_totals_final(const double* partials,
                                                                    int ntiles, double* out) {
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  for (int j = threadIdx.x; j < ntiles; j += blockDim.x)
#pragma unroll
    for (int q = 0; q < 4; ++q) s[q] += partials[4 * j + q];
  __shared__ double sm[4][kTileThreads / 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    for (int o = 16; o > 0; o >>= 1) s[q] += __shfl_xor_sync(0xffffffffu, s[q], o);
    if (lane == 0) sm[q][warp] = s[q];
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double acc = 0.0;
    for (int w = 0; w < kTileThreads / 32; ++w) acc += sm[threadIdx.x][w];
    out[threadIdx.x] = acc;
  }
}

// Device address of g_noalloc_partials for the current device.  In host code
// the array's name is only a host-side stand-in, so kernels must be given the
// address that cudaGetSymbolAddress returns with the device current.  The
// lookup is repeated on every call instead of cached: after cudaDeviceReset
// (or a release and re-creation of the primary context) the module is loaded
// again and an address kept from before would point at freed memory.  The
// first lookup on a device also loads the library's device code there.
cudaError_t scratch_address(double** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
  if (e != cudaSuccess) return e;
  *out = static_cast<double*>(p);
  return cudaSuccess;
}

int fail(int code, const std::string& msg) { return fv::record_error(code, msg); }

}  // namespace

extern "C" int fv_conserved_totals_noalloc(const void* U, const double* area, int64_t n_cells,
                                           int32_t precision, double* out, void* stream) {
  if (precision != FV_F32 && precision != FV_F64)
    return fail(FV_EINVAL, "precision must be FV_F32 or FV_F64");
  if (n_cells < 0) return fail(FV_EINVAL, "n_cells < 0");
  if (n_cells > (int64_t)kNoAllocTiles * kTileCells)
    return fail(FV_EINVAL, "n_cells = " + std::to_string(n_cells) +
                               " exceeds the no-allocation scratch capacity of " +
                               std::to_string((int64_t)kNoAllocTiles * kTileCells) + " cells");
  if (!out || (n_cells > 0 && (!U || !area))) return fail(FV_EINVAL, "null pointer");
  // the kernels read U as 16-byte (FP32) or 32-byte (FP64) records and the
  // areas and totals as doubles: a misaligned pointer would fault the device
  const uintptr_t u_align = precision == FV_F64 ? 32 : 16;
  if (n_cells > 0 && (reinterpret_cast<uintptr_t>(U) % u_align != 0 ||
                      reinterpret_cast<uintptr_t>(area) % 8 != 0))
    return fail(FV_EINVAL, "U must be " + std::to_string(u_align) +
                               "-byte aligned and area 8-byte aligned");
  if (reinterpret_cast<uintptr_t>(out) % 8 != 0) return fail(FV_EINVAL, "out must be 8-byte aligned");
  double* partials = nullptr;
  cudaError_t e = scratch_address(&partials);
  if (e != cudaSuccess)
    return fail(FV_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int ntiles = (int)((n_cells + kTileCells - 1) / kTileCells);
  if (ntiles > 0) {
    if (precision == FV_F64)
      k_tile_totals<double><<<ntiles, kTileThreads, 0, s>>>(static_cast<const dq4n*>(U), area,
                                                             n_cells, partials);
    else
      k_tile_totals<float><<<ntiles, kTileThreads, 0, s>>>(static_cast<const float4*>(U), area,
                                                            n_cells, partials);
  }
  k_tile_totals_final<<<1, kTileThreads, 0, s>>>(partials, ntiles, out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(FV_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
  return FV_OK;
}
