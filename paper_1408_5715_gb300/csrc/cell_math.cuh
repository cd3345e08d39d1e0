// cell_math.cuh -- device building blocks of the cell update shared by the
// step kernels (kernels.cu) and the learned-closure kernels (closure.cu):
// state records, explicitly rounded arithmetic, primitive variables (Eq. 2),
// ghost states, the Lax-Friedrichs face flux (Eq. 5 / Eq. 7), the CFL bound,
// block minimum, the float remainder codec and the per-cell loads.
#pragma once

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

// Reciprocal and square root.  FP64 keeps the correctly rounded operations
// (its results are held to 1e-12 of the FP64 oracle).  The FP32 path is
// memory-bound and its error budget is set by float rounding, so it uses the
// single-instruction approximations of the special-function unit
// (relative error about 2^-23).
template <typename R>
__device__ __forceinline__ R recip(R x);
template <>
__device__ __forceinline__ double recip<double>(double x) {
  return 1.0 / x;
}
template <>
__device__ __forceinline__ float recip<float>(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
template <typename R>
__device__ __forceinline__ R root(R x);
template <>
__device__ __forceinline__ double root<double>(double x) {
  return sqrt(x);
}
template <>
__device__ __forceinline__ float root<float>(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Explicitly rounded arithmetic.  Every multiply-add of the cell update is
// written out (fma / mul / add below, never left to contraction), so the
// compiler cannot fuse differently in different kernels: all kernel shapes and
// the batched kernel give bit-identical results.
__device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float fma_(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float div_(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ double div_(double a, double b) { return __ddiv_rn(a, b); }

template <typename R>
__device__ __forceinline__ R face_len(R nx, R ny) {
  return root<R>(fma_(nx, nx, mul(ny, ny)));
}

// primitive variables of a state (Eq. 2 and the sound speed c = sqrt(gamma p / rho))
template <typename R>
struct Prim {
  R u, v, p, c;
};

template <typename R>
__device__ __forceinline__ Prim<R> primitive(const rec_t<R>& U) {
  Prim<R> w;
  const R ir = recip<R>(U.x);
  w.u = mul(U.y, ir);
  w.v = mul(U.z, ir);
  const R m2 = fma_(U.y, w.u, mul(U.z, w.v));  // rho |v|^2
  w.p = mul(R(kGammaM1), fma_(R(-0.5), m2, U.w));
  w.c = root<R>(mul(mul(R(kGamma), w.p), ir));
  return w;
}

// Far-field state in the kernel's precision (rounded on the host, so no
// kernel converts: GB300's FP64 pipe is narrow).
template <typename R>
__device__ __forceinline__ const R* far_field(const StepArgs& a);
template <>
__device__ __forceinline__ const float* far_field<float>(const StepArgs& a) {
  return a.uinf_f;
}
template <>
__device__ __forceinline__ const double* far_field<double>(const StepArgs& a) {
  return a.uinf;
}

// ... and of mesh m of a batch
template <typename R>
__device__ __forceinline__ const R* batch_far_field(const BatchArgs& b, int m);
template <>
__device__ __forceinline__ const float* batch_far_field<float>(const BatchArgs& b, int m) {
  return b.uinf_f + 4 * m;
}
template <>
__device__ __forceinline__ const double* batch_far_field<double>(const BatchArgs& b, int m) {
  return b.uinf + 4 * m;
}

// Ghost state across a boundary face (slip wall: mirrored normal momentum;
// far field: free stream; extrapolation: copy of the interior state).
template <typename R>
__device__ __forceinline__ rec_t<R> ghost(int code, const rec_t<R>& U, R nx, R ny,
                                          const R* uinf) {
  if (code == -1) {
    const R m = div_(fma_(U.y, nx, mul(U.z, ny)), fma_(nx, nx, mul(ny, ny)));
    const R m2 = mul(R(-2), m);
    return Rec<R>::make(U.x, fma_(m2, nx, U.y), fma_(m2, ny, U.z), U.w);
  }
  if (code == -2) return Rec<R>::make(uinf[0], uinf[1], uinf[2], uinf[3]);
  return U;
}

// Index checks of the bounds-checked build (compiled with -DFV_DEBUG): every
// gather through a neighbour table (global cell ids, tile-local 16-bit ids,
// halo ids, node ids) tests its index against the array it reads; an index
// outside sets bit 8 of the error word (the host reports FV_EINDEX) and the
// access is skipped (the cell's own state stands in).  In the normal build
// the test is compiled out.
#ifdef FV_DEBUG
constexpr bool kIndexChecks = true;
#else
constexpr bool kIndexChecks = false;
#endif
constexpr int kErrIndex = 8;

__device__ __forceinline__ bool index_ok(int64_t i, int64_t n, int* err) {
  if (!kIndexChecks) return true;
  if (i >= 0 && i < n) return true;
  atomicOr(err, kErrIndex);
  return false;
}

// The state across face nb of a cell: the neighbour's (global id nb of n
// cells) or a ghost state.
template <typename R>
__device__ __forceinline__ rec_t<R> neighbour_state(const rec_t<R>& UL, int nb, R nx, R ny,
                                                    const rec_t<R>* __restrict__ Ucur,
                                                    const R* uinf, int64_t n, int* err) {
  if (nb >= 0) return index_ok(nb, n, err) ? Rec<R>::ld(Ucur + nb) : UL;
  return ghost<R>(nb, UL, nx, ny, uinf);
}

// Adds TWICE the flux of one face (times its length) to acc, given both
// states and their primitives: Eq. 5's factor 1/2 is applied once per cell,
// to dt/V (finish_cell).  Scaling by a power of two is exact, so the
// accumulated values are exactly twice those of the halved sum and every
// update is bitwise the same, for four multiplies fewer per face.  s scales
// the dissipation (the learned closure; SCALED = false is the paper's flux).
// WAVE selects the wave speed of the dissipation: kWaveAverage the paper's
// interface averages |u-bar_n| + c-bar; kWaveMax the larger one-sided speed
// max(|u_nL| + c_L, |u_nR| + c_R) (Rusanov), which keeps the first-order
// update positive in strong expansions.  Both are symmetric in L <-> R.
//
// Each term is written so that the two cells of a face compute exact
// opposites (the neighbour sees L and R swapped and the normal negated):
// every product involves one side only, rounding is symmetric in sign and the
// sums of the two sides' terms commute.  So the face flux is antisymmetric
// bit for bit -- discrete conservation is exact -- and a kernel may evaluate a
// face once and hand its negation to the cell across (k_step_tile_faces).
template <typename R, bool SCALED, int WAVE = kWaveAverage>
__device__ __forceinline__ void face_flux_value(const rec_t<R>& UL, const Prim<R>& L,
                                                const rec_t<R>& UR, const Prim<R>& W, R nx, R ny,
                                                R len, R s, R X[4]) {
  const R qL = fma_(L.u, nx, mul(L.v, ny));
  const R qR = fma_(W.u, nx, mul(W.v, ny));
  // na = -|n| (wave speed), twice the dissipation coefficient of Eq. 5
  R na;
  if (WAVE == kWaveAverage)
    na = mul(R(-0.5), fma_(len, add(L.c, W.c), fabs(add(qL, qR))));
  else
    na = -fmax(fma_(len, L.c, fabs(qL)), fma_(len, W.c, fabs(qR)));
  if (SCALED) na = mul(s, na);
  X[0] = fma_(na, sub(UR.x, UL.x), add(mul(UL.x, qL), mul(UR.x, qR)));
  X[1] = fma_(na, sub(UR.y, UL.y),
              add(fma_(UL.y, qL, mul(L.p, nx)), fma_(UR.y, qR, mul(W.p, nx))));
  X[2] = fma_(na, sub(UR.z, UL.z),
              add(fma_(UL.z, qL, mul(L.p, ny)), fma_(UR.z, qR, mul(W.p, ny))));
  X[3] = fma_(na, sub(UR.w, UL.w), add(mul(add(UL.w, L.p), qL), mul(add(UR.w, W.p), qR)));
}

template <typename R, bool SCALED, int WAVE = kWaveAverage>
__device__ __forceinline__ void face_flux_acc(const rec_t<R>& UL, const Prim<R>& L,
                                              const rec_t<R>& UR, const Prim<R>& W, R nx, R ny,
                                              R len, R s, R acc[4]) {
  R X[4];
  face_flux_value<R, SCALED, WAVE>(UL, L, UR, W, nx, ny, len, s, X);
#pragma unroll
  for (int q = 0; q < 4; ++q) acc[q] = add(acc[q], X[q]);
}

template <typename R, int WAVE = kWaveAverage>
__device__ __forceinline__ R add_face_flux(const rec_t<R>& UL, const Prim<R>& L, int nb, R nx,
                                           R ny, const rec_t<R>* __restrict__ Ucur,
                                           const R* uinf, R acc[4], int64_t n, int* err) {
  const rec_t<R> UR = neighbour_state<R>(UL, nb, nx, ny, Ucur, uinf, n, err);
  const Prim<R> W = primitive<R>(UR);
  const R len = face_len<R>(nx, ny);
  face_flux_acc<R, false, WAVE>(UL, L, UR, W, nx, ny, len, R(1), acc);
  return len;
}

// CFL bound 2V/(P(|v|+c)) of a state, in the state's precision (a float
// bound converts exactly to the double used by the minimum); a bad state
// clears *ok and gives +inf.
template <typename R>
__device__ __forceinline__ R bound_of(const rec_t<R>& U, const Prim<R>& w, R inradius, bool& ok) {
  const R lam = add(root<R>(fma_(w.u, w.u, mul(w.v, w.v))), w.c);
  // NaN fails every comparison; an infinite state gives an infinite lam
  ok = (U.x > R(0)) && (w.p > R(0)) && (lam < R(INFINITY));
  return ok ? mul(inradius, recip<R>(lam)) : R(INFINITY);
}

template <typename R>
__device__ __forceinline__ R cell_bound(const rec_t<R>& U, R inradius, bool& ok) {
  return bound_of<R>(U, primitive<R>(U), inradius, ok);
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

// The remainder of the four float state values is kept as four bfloat16
// values (8 bytes per cell): converting a pair is one instruction and
// unpacking is a shift, so the compensation costs few instructions.
__device__ __forceinline__ void unpack_rem(uint2 v, float l[4]) {
  l[0] = __uint_as_float(v.x << 16);
  l[1] = __uint_as_float(v.x & 0xffff0000u);
  l[2] = __uint_as_float(v.y << 16);
  l[3] = __uint_as_float(v.y & 0xffff0000u);
}

__device__ __forceinline__ uint2 pack_rem(const float e[4]) {
  __nv_bfloat162 a = __floats2bfloat162_rn(e[0], e[1]);
  __nv_bfloat162 b = __floats2bfloat162_rn(e[2], e[3]);
  return make_uint2(*reinterpret_cast<unsigned*>(&a), *reinterpret_cast<unsigned*>(&b));
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

// dt and time of the current step formed by one thread (the caller shares them).
__device__ __forceinline__ void block_dt(const StepArgs& a, double& t, double& dt) {
  t = *a.t_read;
  dt = a.cfl > 0.0 ? a.cfl * __longlong_as_double((long long)*a.bmin_read) : -a.cfl;
  if (a.t_stop > 0.0) {
    double rem = a.t_stop - t;
    if (rem < dt) dt = rem;
    if (!(dt > 0.0)) dt = 0.0;
  }
}

// Everything one cell's update reads from its own records.  Geometry layout:
//   FP64: geom[2i] = (n0x, n0y, n1x, n1y), geom[2i+1] = (n2x, n2y, 1/V, 2V/P),
//         nbr = int4 (nbr0, nbr1, nbr2, -);
//   FP32: geom[2i] = (n0x, n0y, n1x, n1y), geom[2i+1] = (n2x, n2y, 1/V, nbr0 as
//         bits), nbr = int2 (nbr1, nbr2); 2V/P is formed from the face lengths
//         that the flux computes anyway (40 bytes per cell instead of 48).
template <typename R>
struct CellIn {
  int n0, n1, n2;
  rec_t<R> g0, g1, U;
  rec_t<R> base;  // RK2 second stage: U^n of the cell
  uint2 lo, lo_stage;
};

template <typename R, int MODE, bool COMP>
__device__ __forceinline__ void load_cell(const StepArgs& a, const rec_t<R>* __restrict__ U,
                                          const rec_t<R>* __restrict__ geom, int64_t i,
                                          CellIn<R>& c) {
  c.g0 = Rec<R>::ld(geom + 2 * i);
  c.g1 = Rec<R>::ld(geom + 2 * i + 1);
  if constexpr (sizeof(R) == 8) {
    const int4 nb = __ldg(static_cast<const int4*>(a.nbr) + i);
    c.n0 = nb.x, c.n1 = nb.y, c.n2 = nb.z;
  } else {
    const int2 nb = __ldg(static_cast<const int2*>(a.nbr) + i);
    c.n0 = __float_as_int(c.g1.w), c.n1 = nb.x, c.n2 = nb.y;
  }
  c.U = Rec<R>::ld(U + i);
  // plain loads: Ubase and the remainders are rewritten in this kernel (each
  // only by the thread of its own cell)
  if (MODE == kModeRK2b) c.base = static_cast<const rec_t<R>*>(a.Ubase)[i];
  if (COMP && MODE != kModeResidual) c.lo = a.lo[i];
  if (COMP && MODE == kModeRK2b) c.lo_stage = a.lo_stage[i];
}

// 2V/P of a cell: stored for FP64, from the face lengths for FP32
template <typename R>
__device__ __forceinline__ R inradius(const rec_t<R>& g1, R perim) {
  if constexpr (sizeof(R) == 8) {
    return g1.w;
  } else {
    return mul(2.0f, recip<float>(mul(g1.z, perim)));
  }
}

template <typename R>
__device__ __forceinline__ R geom_inradius(const rec_t<R>* __restrict__ geom, int64_t i) {
  const rec_t<R> g0 = Rec<R>::ld(geom + 2 * i), g1 = Rec<R>::ld(geom + 2 * i + 1);
  if constexpr (sizeof(R) == 8) return g1.w;
  const R perim =
      add(add(face_len<R>(g0.x, g0.y), face_len<R>(g0.z, g0.w)), face_len<R>(g1.x, g1.y));
  return inradius<R>(g1, perim);
}

// Everything after the face fluxes: residual output, or the forward-Euler /
// Heun update (plain or compensated) and the CFL bound of the new state.
// acc holds twice the flux sum (face_flux_acc): the factors applied to it
// carry the 1/2 (exactly).
template <typename R, int MODE, bool COMP>
__device__ __forceinline__ void finish_cell(const StepArgs& a, rec_t<R>* out, int64_t i,
                                            const CellIn<R>& c, const R acc[4], R perim, R dt,
                                            R& bmin, bool& ok) {
  const rec_t<R>& UL = c.U;
  const R invV = c.g1.z;
  bool cell_ok = true;
  if (MODE == kModeResidual) {
    const R m = mul(R(-0.5), invV);
    out[i] = Rec<R>::make(mul(m, acc[0]), mul(m, acc[1]), mul(m, acc[2]), mul(m, acc[3]));
    return;
  }
  if (COMP) {
    // float state + bfloat16 remainder: the increment and the remainder are
    // added with an exact TwoSum, and what the float sum drops becomes the
    // new remainder (kept only by the stages that produce U^{n+1}).
    const float f = mul(mul(-0.5f, (float)dt), (float)invV);
    const float u[4] = {(float)UL.x, (float)UL.y, (float)UL.z, (float)UL.w};
    float base[4] = {u[0], u[1], u[2], u[3]};
    float inc[4];
    float lo[4];
    if (MODE == kModeRK2b) {
      base[0] = (float)c.base.x, base[1] = (float)c.base.y, base[2] = (float)c.base.z,
      base[3] = (float)c.base.w;
    }
    unpack_rem(c.lo, lo);  // the remainder of U^n
    if (MODE == kModeRK2b) {
      // U^{n+1} = U^n + (U* - U^n)/2 + dt R(U*)/2, with U^n = base + lo and
      // U* = u + lo_stage
      base[0] = (float)c.base.x, base[1] = (float)c.base.y, base[2] = (float)c.base.z,
      base[3] = (float)c.base.w;
      float ls[4];
      unpack_rem(c.lo_stage, ls);
#pragma unroll
      for (int q = 0; q < 4; ++q)
        inc[q] = fma_(0.5f, sub(u[q], base[q]),
                      mul(0.5f, add(fma_(f, (float)acc[q], ls[q]), lo[q])));
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) inc[q] = fma_(f, (float)acc[q], lo[q]);
    }
    float sm[4], e[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) sm[q] = two_sum(base[q], inc[q], e[q]);
    const rec_t<R> Un = Rec<R>::make(R(sm[0]), R(sm[1]), R(sm[2]), R(sm[3]));
    out[i] = Un;
    if (MODE == kModeRK2a) {
      a.lo_stage[i] = pack_rem(e);
    } else {
      a.lo[i] = pack_rem(e);
      bmin = fmin(bmin, cell_bound<R>(Un, inradius<R>(c.g1, perim), cell_ok));
    }
  } else {
    const R f = mul(mul(R(-0.5), dt), invV);
    rec_t<R> Un = Rec<R>::make(fma_(f, acc[0], UL.x), fma_(f, acc[1], UL.y),
                               fma_(f, acc[2], UL.z), fma_(f, acc[3], UL.w));
    if (MODE == kModeRK2b) {
      const rec_t<R>& B = c.base;
      const R h = R(0.5);
      Un = Rec<R>::make(add(mul(h, B.x), mul(h, Un.x)), add(mul(h, B.y), mul(h, Un.y)),
                        add(mul(h, B.z), mul(h, Un.z)), add(mul(h, B.w), mul(h, Un.w)));
    }
    out[i] = Un;
    if (MODE != kModeRK2a) bmin = fmin(bmin, cell_bound<R>(Un, inradius<R>(c.g1, perim), cell_ok));
  }
  ok = ok && cell_ok;
}

}  // namespace
}  // namespace fv
