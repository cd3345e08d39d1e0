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
#include <mutex>
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
constexpr int kMaxDevices = 64;

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

// Device address of g_noalloc_partials, looked up once per device.  In host
// code the array's name is only a host-side stand-in, so kernels must be
// given the address that cudaGetSymbolAddress returns for the current device.
std::mutex g_addr_mutex;
double* g_addr[kMaxDevices] = {};

cudaError_t scratch_address(int dev, double** out) {
  std::lock_guard<std::mutex> lock(g_addr_mutex);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) return e;
    g_addr[dev] = static_cast<double*>(p);
  }
  *out = g_addr[dev];
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
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(FV_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(FV_EINVAL, "device id out of range");
  double* partials = nullptr;
  e = scratch_address(dev, &partials);
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
