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
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.h"

namespace fv {

namespace {

constexpr double kGamma = 1.4;           // Sec. 6.1
constexpr double kGammaM1 = kGamma - 1.0;
constexpr unsigned long long kInfBits = 0x7FF0000000000000ull;  // +inf as double bits

struct __align__(32) dq4 {
  double x, y, z, w;
};

template <typename R>
struct Rec;
template <>
struct Rec<float> {
  using T = float4;
  static __device__ __forceinline__ float4 ld(const float4* p) { return __ldg(p); }
  static __device__ __forceinline__ float4 make(float a, float b, float c, float d) {
    return make_float4(a, b, c, d);
  }
};
template <>
struct Rec<double> {
  using T = dq4;
  static __device__ __forceinline__ dq4 ld(const dq4* p) {
    const double2* q = reinterpret_cast<const double2*>(p);
    double2 a = __ldg(q), b = __ldg(q + 1);
    return dq4{a.x, a.y, b.x, b.y};
  }
  static __device__ __forceinline__ dq4 make(double a, double b, double c, double d) {
    return dq4{a, b, c, d};
  }
};

template <typename R>
using rec_t = typename Rec<R>::T;

// primitive variables of a state (Eq. 2 and the sound speed c = sqrt(gamma p / rho))
template <typename R>
struct Prim {
  R u, v, p, c;
};

template <typename R>
__device__ __forceinline__ Prim<R> primitive(const rec_t<R>& U) {
  Prim<R> w;
  R ir = R(1) / U.x;
  w.u = U.y * ir;
  w.v = U.z * ir;
  w.p = R(kGammaM1) * (U.w - R(0.5) * (U.y * w.u + U.z * w.v));
  w.c = sqrt(R(kGamma) * w.p * ir);
  return w;
}

// Ghost state across a boundary face (slip wall: mirrored normal momentum;
// far field: free stream; extrapolation: copy of the interior state).
template <typename R>
__device__ __forceinline__ rec_t<R> ghost(int code, const rec_t<R>& U, R nx, R ny,
                                          const double* uinf) {
  if (code == -1) {
    R m = (U.y * nx + U.z * ny) / (nx * nx + ny * ny);
    return Rec<R>::make(U.x, U.y - R(2) * m * nx, U.z - R(2) * m * ny, U.w);
  }
  if (code == -2) return Rec<R>::make(R(uinf[0]), R(uinf[1]), R(uinf[2]), R(uinf[3]));
  return U;
}

// Adds the Lax-Friedrichs flux of one face (times its length) to acc.
template <typename R>
__device__ __forceinline__ void add_face_flux(const rec_t<R>& UL, const Prim<R>& L, int nb, R nx,
                                              R ny, const rec_t<R>* __restrict__ Ucur,
                                              const double* uinf, R acc[4]) {
  rec_t<R> UR = nb >= 0 ? Rec<R>::ld(Ucur + nb) : ghost<R>(nb, UL, nx, ny, uinf);
  Prim<R> W = primitive<R>(UR);
  R len = sqrt(nx * nx + ny * ny);
  R qL = L.u * nx + L.v * ny;
  R qR = W.u * nx + W.v * ny;
  R a = R(0.25) * (fabs(qL + qR) + len * (L.c + W.c));
  acc[0] += R(0.5) * (UL.x * qL + UR.x * qR) - a * (UR.x - UL.x);
  acc[1] += R(0.5) * ((UL.y * qL + L.p * nx) + (UR.y * qR + W.p * nx)) - a * (UR.y - UL.y);
  acc[2] += R(0.5) * ((UL.z * qL + L.p * ny) + (UR.z * qR + W.p * ny)) - a * (UR.z - UL.z);
  acc[3] += R(0.5) * ((UL.w + L.p) * qL + (UR.w + W.p) * qR) - a * (UR.w - UL.w);
}

// CFL bound 2V/(P(|v|+c)) of a state, in the state's precision (a float
// bound converts exactly to the double used by the minimum); a bad state
// clears *ok and gives +inf.
template <typename R>
__device__ __forceinline__ R cell_bound(const rec_t<R>& U, R inradius, bool& ok) {
  Prim<R> w = primitive<R>(U);
  R lam = sqrt(w.u * w.u + w.v * w.v) + w.c;
  ok = (U.x > R(0)) && (w.p > R(0)) && isfinite(w.p) && isfinite(U.y) && isfinite(U.z) &&
       isfinite(lam);
  return ok ? inradius / lam : R(INFINITY);
}

// Minimum over the block; the result is valid in thread 0.
template <typename R>
__device__ __forceinline__ R block_min(R v) {
  __shared__ R sm[32];
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) sm[warp] = v;
  __syncthreads();
  if (warp == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    v = lane < nw ? sm[lane] : R(INFINITY);
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  }
  return v;
}

// Error-free sum (Knuth's TwoSum): s + e == a + b exactly, for any a, b.
__device__ __forceinline__ float two_sum(float a, float b, float& e) {
  const float s = a + b;
  const float ap = s - b;
  const float bp = s - ap;
  e = (a - ap) + (b - bp);
  return s;
}

__device__ __forceinline__ void unpack_lo(uint2 v, float l[4]) {
  l[0] = __uint_as_float(v.x << 16);
  l[1] = __uint_as_float(v.x & 0xffff0000u);
  l[2] = __uint_as_float(v.y << 16);
  l[3] = __uint_as_float(v.y & 0xffff0000u);
}

__device__ __forceinline__ unsigned bf16_bits(float x) {
  return (unsigned)__bfloat16_as_ushort(__float2bfloat16_rn(x));
}

__device__ __forceinline__ uint2 pack_lo(const float l[4]) {
  return make_uint2(bf16_bits(l[0]) | (bf16_bits(l[1]) << 16),
                    bf16_bits(l[2]) | (bf16_bits(l[3]) << 16));
}

// dt of the current step (CFL bound or fixed step, clamped so the loop's time
// never passes t_stop).  Lane 0 of each warp evaluates it and broadcasts, so
// the FP64 scalar work is per warp, not per cell.
__device__ __forceinline__ double step_dt(const StepArgs& a, double& t) {
  double dt = 0.0;
  t = 0.0;
  if ((threadIdx.x & 31) == 0) {
    t = *a.t_read;
    dt = a.cfl > 0.0 ? a.cfl * __longlong_as_double((long long)*a.bmin_read) : -a.cfl;
    if (a.t_stop > 0.0) {
      double rem = a.t_stop - t;
      if (rem < dt) dt = rem;
      if (!(dt > 0.0)) dt = 0.0;
    }
  }
  t = __shfl_sync(0xffffffffu, t, 0);
  return __shfl_sync(0xffffffffu, dt, 0);
}

template <typename R, int MODE, bool COMP>
__global__ void __launch_bounds__(kBlock) k_step(StepArgs a) {
  const rec_t<R>* __restrict__ U = static_cast<const rec_t<R>*>(a.U);
  const rec_t<R>* __restrict__ geom = static_cast<const rec_t<R>*>(a.geom);
  rec_t<R>* out = static_cast<rec_t<R>*>(a.out);
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double t = 0.0, dt = 0.0;
  if (MODE != kModeResidual) dt = step_dt(a, t);
  R bound = R(INFINITY);
  bool ok = true;
  if (i < a.n) {
    const int4 nb = __ldg(a.nbr + i);
    const rec_t<R> g0 = Rec<R>::ld(geom + 2 * i);
    const rec_t<R> g1 = Rec<R>::ld(geom + 2 * i + 1);
    const rec_t<R> UL = Rec<R>::ld(U + i);
    const Prim<R> L = primitive<R>(UL);
    R acc[4] = {R(0), R(0), R(0), R(0)};
    add_face_flux<R>(UL, L, nb.x, g0.x, g0.y, U, a.uinf, acc);
    add_face_flux<R>(UL, L, nb.y, g0.z, g0.w, U, a.uinf, acc);
    add_face_flux<R>(UL, L, nb.z, g1.x, g1.y, U, a.uinf, acc);
    const R invV = g1.z;
    if (MODE == kModeResidual) {
      out[i] = Rec<R>::make(-invV * acc[0], -invV * acc[1], -invV * acc[2], -invV * acc[3]);
    } else if (COMP) {
      // float state + bfloat16 remainder: the increment and the remainder are
      // added with an exact TwoSum, and what the float sum drops becomes the
      // new remainder (kept only by the stages that produce U^{n+1}).
      const float f = -(float)dt * (float)invV;
      float lo[4];
      unpack_lo(a.lo[i], lo);
      const float u[4] = {(float)UL.x, (float)UL.y, (float)UL.z, (float)UL.w};
      float base[4] = {u[0], u[1], u[2], u[3]};
      float inc[4];
      if (MODE == kModeRK2b) {
        // U^{n+1} = U^n + (U* - U^n)/2 + dt R(U*)/2, with U^n = base + lo and
        // U* = u + lo_stage
        const rec_t<R> B = static_cast<const rec_t<R>*>(a.Ubase)[i];
        base[0] = (float)B.x, base[1] = (float)B.y, base[2] = (float)B.z, base[3] = (float)B.w;
        float ls[4];
        unpack_lo(a.lo_stage[i], ls);
#pragma unroll
        for (int q = 0; q < 4; ++q)
          inc[q] = 0.5f * (u[q] - base[q]) + 0.5f * ((f * (float)acc[q] + ls[q]) + lo[q]);
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) inc[q] = f * (float)acc[q] + lo[q];
      }
      float s[4], e[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) s[q] = two_sum(base[q], inc[q], e[q]);
      const rec_t<R> Un = Rec<R>::make(R(s[0]), R(s[1]), R(s[2]), R(s[3]));
      out[i] = Un;
      if (MODE == kModeRK2a) {
        a.lo_stage[i] = pack_lo(e);
      } else {
        a.lo[i] = pack_lo(e);
        bound = cell_bound<R>(Un, g1.w, ok);
      }
    } else {
      const R f = -R(dt) * invV;
      rec_t<R> Un = Rec<R>::make(UL.x + f * acc[0], UL.y + f * acc[1], UL.z + f * acc[2],
                                 UL.w + f * acc[3]);
      if (MODE == kModeRK2b) {
        // plain load: Ubase may be the array this thread writes below
        const rec_t<R> B = static_cast<const rec_t<R>*>(a.Ubase)[i];
        Un = Rec<R>::make(R(0.5) * B.x + R(0.5) * Un.x, R(0.5) * B.y + R(0.5) * Un.y,
                          R(0.5) * B.z + R(0.5) * Un.z, R(0.5) * B.w + R(0.5) * Un.w);
      }
      out[i] = Un;
      if (MODE != kModeRK2a) bound = cell_bound<R>(Un, g1.w, ok);
    }
  }
  if (MODE == kModeFE || MODE == kModeRK2b) {
    if (!ok) atomicOr(a.err, 1);
    const double m = (double)block_min<R>(bound);
    if (threadIdx.x == 0) {
      atomicMin(a.bmin_write, (unsigned long long)__double_as_longlong(m));
      if (blockIdx.x == 0) {
        *a.t_write = t + dt;
        *a.bmin_reset = kInfBits;
      }
    }
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
  if (i < n) b = cell_bound<R>(Rec<R>::ld(U + i), Rec<R>::ld(geom + 2 * i + 1).w, ok);
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

template <typename R, bool COMP>
cudaError_t launch_step_t(int mode, const StepArgs& a, cudaStream_t s) {
  if (a.n <= 0 && mode == kModeResidual) return cudaSuccess;
  const unsigned g = a.n > 0 ? grid_for(a.n) : 1u;  // a time step always runs its scalars
  switch (mode) {
    case kModeFE: k_step<R, kModeFE, COMP><<<g, kBlock, 0, s>>>(a); break;
    case kModeRK2a: k_step<R, kModeRK2a, COMP><<<g, kBlock, 0, s>>>(a); break;
    case kModeRK2b: k_step<R, kModeRK2b, COMP><<<g, kBlock, 0, s>>>(a); break;
    case kModeResidual: k_step<R, kModeResidual, false><<<g, kBlock, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_step(bool f64, int mode, const StepArgs& a, cudaStream_t s) {
  if (f64) return launch_step_t<double, false>(mode, a, s);
  return a.lo ? launch_step_t<float, true>(mode, a, s) : launch_step_t<float, false>(mode, a, s);
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
