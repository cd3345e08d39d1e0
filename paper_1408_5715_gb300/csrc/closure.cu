// closure.cu -- the learned per-face dissipation scale on tensor cores.
//
// Not part of the paper: an MLP 8 -> 32 -> 32 -> 1 (ReLU) maps eight features
// of a face that do not change when its two cells are swapped to a scale
// s = 0.2 + 1.3 sigmoid(z) of the Lax-Friedrichs dissipation of Eq. 5.
// Weights of the two hidden layers are bfloat16, accumulation is FP32.
//
// Each face is one row of the MLP, evaluated once: either by a pass over the
// mesh's face list that writes the scale to both cells' slots, followed by
// the step reading them (k_face_scales, k_step_scaled), or inside one kernel
// on shape 7's tiles (k_step_closure_tile).  Two tensor-core engines give the
// same bits.  mma.sync: a warp writes the bfloat16 features of 32 rows to
// shared memory; per 16-row tile, layer 1 is one m16n8k16 per 8 hidden units
// (K = 8 features, the bias parts, padding), layer 2 two per 8 units
// (K = 32) plus one for its bias parts, with the FP32 accumulators of layer 1
// re-packed in registers as the A operand of layer 2; layer 3 (32 -> 1) is an
// FP32 dot product finished with two quad shuffles.  tcgen05: 128 rows per
// MMA from shared-memory operands into tensor memory (the *_tc kernels
// below).  The training kernels (loss, gradient, Adam) use mma.sync.
//
// Conservation: the features are computed with explicitly rounded operations
// that give the same bits from either side of a face (the swap L <-> R,
// n -> -n), so both cells use the same scale and the face flux stays
// antisymmetric.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "cell_math.cuh"
#include "kernels.h"
#include "launch_util.cuh"
#include "tc_util.cuh"
#include "tile_math.cuh"

namespace fv {

namespace {

constexpr int kClWarps = 4;
constexpr int kClThreads = 32 * kClWarps;
constexpr int kRows = 96;  // 32 cells x 3 faces per warp

struct __align__(16) ClWarpSmem {
  uint4 feat[kRows];  // 8 bfloat16 features per row
  float s[kRows];     // scale per row
};

__device__ __forceinline__ unsigned pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<unsigned*>(&v);
}

// D += A (16x16, bf16, row) * B (16x8, bf16, col), FP32 accumulate.
__device__ __forceinline__ void mma_bf16(float d[4], unsigned a0, unsigned a1, unsigned a2,
                                         unsigned a3, unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float relu(float x) { return x > 0.0f ? x : 0.0f; }

// ReLU of two values packed to bfloat16 in one conversion that clamps
// negative results to zero: rounding keeps the sign, so this is the rounding
// of the ReLU (the next layer sees the same values).
__device__ __forceinline__ unsigned pack_bf16_relu(float lo, float hi) {
  unsigned d;
  asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}

// sigmoid(z) with the special-function unit's exponential and reciprocal
// (relative error a few 2^-22: far below the 1e-5 to which scales are held)
__device__ __forceinline__ float sigmoid(float z) {
  return recip<float>(add(1.0f, __expf(-z)));
}

__device__ __forceinline__ float scale_of(float z) { return fma_(1.3f, sigmoid(z), 0.2f); }

// The eight swap-invariant features of a face.
__device__ __forceinline__ void face_features(const float4& UL, const Prim<float>& L,
                                              const float4& UR, const Prim<float>& W, float nx,
                                              float ny, float len, float f[8]) {
  const float il = recip<float>(len);
  const float hx = mul(nx, il), hy = mul(ny, il);
  const float unL = fma_(L.u, hx, mul(L.v, hy));
  const float unR = fma_(W.u, hx, mul(W.v, hy));
  const float utL = fma_(L.v, hx, -mul(L.u, hy));
  const float utR = fma_(W.v, hx, -mul(W.u, hy));
  const float cbar = mul(0.5f, add(L.c, W.c));
  const float icb = recip<float>(cbar);
  f[0] = mul(fabsf(sub(UR.x, UL.x)), recip<float>(mul(0.5f, add(UL.x, UR.x))));
  f[1] = mul(fabsf(sub(unR, unL)), icb);
  f[2] = mul(fabsf(sub(utR, utL)), icb);
  f[3] = mul(fabsf(sub(W.p, L.p)), recip<float>(mul(0.5f, add(L.p, W.p))));
  f[4] = mul(fabsf(mul(0.5f, add(unL, unR))), icb);
  f[5] = fabsf(sub(mul(unR, recip<float>(W.c)), mul(unL, recip<float>(L.c))));
  f[6] = mul(fminf(L.c, W.c), icb);
  f[7] = mul(fmaxf(L.c, W.c), icb);
}

__device__ __forceinline__ uint4 pack_features(const float f[8]) {
  return make_uint4(pack_bf16(f[0], f[1]), pack_bf16(f[2], f[3]), pack_bf16(f[4], f[5]),
                    pack_bf16(f[6], f[7]));
}

// Weights as this thread's mma B fragments (loaded once per kernel).  The
// hidden-layer biases ride in the MMAs: each FP32 bias b is split into three
// bfloat16 parts hi + mid + lo (together its 24-bit significand) placed in
// three K rows of B, against A columns that hold 1.0 -- for layer 1 in the
// padding rows 8..10 of its K = 16 slice, for layer 2 in an extra K slice --
// so the tensor core adds them instead of 32 FP32 additions per row.
struct ClFrag {
  unsigned w1[4];   // layer 1, per n-tile: W1[n][2c..2c+1]
  unsigned w1b[4];  // layer 1, per n-tile: bias parts in K rows 8..10 (lanes c = 0, 1)
  unsigned w2[16];  // layer 2, per (n-tile, k-slice): two registers
  unsigned w2b[4];  // layer 2, per n-tile: bias parts in K rows 0..2 of the extra slice
  unsigned one;     // A columns of the bias rows: (1, 1) for c = 0, (1, 0) for c = 1
};

// The bias parts of unit n for lane quad position c: (hi, mid) for c = 0,
// (lo, 0) for c = 1, nothing for c = 2, 3.
__device__ __forceinline__ unsigned bias_parts(float b, int c) {
  const __nv_bfloat16 hi = __float2bfloat16_rn(b);
  const float r1 = sub(b, __bfloat162float(hi));
  const __nv_bfloat16 mid = __float2bfloat16_rn(r1);
  const float r2 = sub(r1, __bfloat162float(mid));
  if (c == 0) return pack_bf16(__bfloat162float(hi), __bfloat162float(mid));
  if (c == 1) return pack_bf16(r2, 0.0f);
  return 0u;
}

__device__ __forceinline__ void load_frags(const ClosureParams& cp, ClFrag& fr) {
  const int lane = threadIdx.x & 31, r = lane >> 2, c = lane & 3;
#pragma unroll
  for (int nt = 0; nt < 4; ++nt) {
    fr.w1[nt] = __ldg(cp.w1 + (nt * 8 + r) * 4 + c);
    fr.w1b[nt] = bias_parts(__ldg(cp.b1 + nt * 8 + r), c);
    fr.w2b[nt] = bias_parts(__ldg(cp.b2 + nt * 8 + r), c);
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
      fr.w2[(nt * 2 + kk) * 2] = __ldg(cp.w2 + (nt * 8 + r) * 16 + kk * 8 + c);
      fr.w2[(nt * 2 + kk) * 2 + 1] = __ldg(cp.w2 + (nt * 8 + r) * 16 + kk * 8 + 4 + c);
    }
  }
  fr.one = c == 0 ? 0x3F803F80u : c == 1 ? 0x00003F80u : 0u;  // bfloat16 1.0 = 0x3F80
}

// Layer-1 and layer-2 pre-activations of one 16-row tile, in accumulator
// fragment layout: g[nt][0..1] row r, g[nt][2..3] row r+8, columns
// nt*8 + 2c, +1.  h1 (bfloat16, as layer-2 A fragments) is returned too.
__device__ __forceinline__ void tile_forward(const ClWarpSmem& w, int t, const ClFrag& fr,
                                             float a1[4][4], unsigned A2[2][4], float g[4][4]) {
  const int lane = threadIdx.x & 31, r = lane >> 2, c = lane & 3;
  const unsigned* row0 = reinterpret_cast<const unsigned*>(&w.feat[16 * t + r]);
  const unsigned* row1 = reinterpret_cast<const unsigned*>(&w.feat[16 * t + r + 8]);
  const unsigned x0 = row0[c], x1 = row1[c];
#pragma unroll
  for (int nt = 0; nt < 4; ++nt) {
    a1[nt][0] = a1[nt][1] = a1[nt][2] = a1[nt][3] = 0.0f;
    // K columns 0..7 the features, 8..10 the bias rows against 1.0
    mma_bf16(a1[nt], x0, x1, fr.one, fr.one, fr.w1[nt], fr.w1b[nt]);
    const unsigned p0 = pack_bf16_relu(a1[nt][0], a1[nt][1]);
    const unsigned p1 = pack_bf16_relu(a1[nt][2], a1[nt][3]);
    A2[nt >> 1][(nt & 1) ? 2 : 0] = p0;
    A2[nt >> 1][(nt & 1) ? 3 : 1] = p1;
  }
#pragma unroll
  for (int nt = 0; nt < 4; ++nt) {
    g[nt][0] = g[nt][1] = g[nt][2] = g[nt][3] = 0.0f;
#pragma unroll
    for (int kk = 0; kk < 2; ++kk)
      mma_bf16(g[nt], A2[kk][0], A2[kk][1], A2[kk][2], A2[kk][3], fr.w2[(nt * 2 + kk) * 2],
               fr.w2[(nt * 2 + kk) * 2 + 1]);
    mma_bf16(g[nt], fr.one, fr.one, 0u, 0u, fr.w2b[nt], 0u);  // + b2
  }
}

// Layer 3 in a fixed order of explicitly rounded operations, the same in
// both tensor-core engines: four partial sums p_c, each a chain of fused
// multiply-adds over the column pairs (nt * 8 + 2c, +1), nt = 0..3, then
// ((p0 + p1) + (p2 + p3)) + b3.
__device__ __forceinline__ float out_pair(float acc, float g0, float g1, float w0, float w1) {
  return fma_(relu(g1), w1, fma_(relu(g0), w0, acc));
}

// z of rows r and r+8 of a tile (all four lanes of a quad get both).
__device__ __forceinline__ void tile_output(const float g[4][4], const float* w3, float b3,
                                            float& z0, float& z1) {
  const int c = threadIdx.x & 3;
  z0 = 0.0f;
  z1 = 0.0f;
#pragma unroll
  for (int nt = 0; nt < 4; ++nt) {
    const int col = nt * 8 + 2 * c;
    z0 = out_pair(z0, g[nt][0], g[nt][1], w3[col], w3[col + 1]);
    z1 = out_pair(z1, g[nt][2], g[nt][3], w3[col], w3[col + 1]);
  }
  z0 = add(z0, __shfl_xor_sync(0xffffffffu, z0, 1));
  z0 = add(z0, __shfl_xor_sync(0xffffffffu, z0, 2));
  z1 = add(z1, __shfl_xor_sync(0xffffffffu, z1, 1));
  z1 = add(z1, __shfl_xor_sync(0xffffffffu, z1, 2));
  z0 = add(z0, b3);
  z1 = add(z1, b3);
}

// Scales of the warp's first 16 * ntile rows, from the features in w.feat
// into w.s.
__device__ __forceinline__ void warp_mlp(ClWarpSmem& w, const ClFrag& fr, const float* w3, float b3,
                                         int ntile = kRows / 16) {
  const int lane = threadIdx.x & 31, r = lane >> 2, c = lane & 3;
  for (int t = 0; t < ntile; ++t) {
    float a1[4][4], g[4][4];
    unsigned A2[2][4];
    tile_forward(w, t, fr, a1, A2, g);
    float z0, z1;
    tile_output(g, w3, b3, z0, z1);
    // lane c = 0 of a quad forms row r's scale, lane c = 1 row r + 8's
    const float sv = scale_of((c & 1) ? z1 : z0);
    if (c < 2) w.s[16 * t + r + 8 * c] = sv;
  }
}

struct ClShared {
  ClWarpSmem warp[kClWarps];
  float b1[32], b2[32], w3[32];
};

__device__ __forceinline__ void load_small_params(const ClosureParams& cp, ClShared& sh) {
  if (threadIdx.x < 32) {
    sh.b1[threadIdx.x] = cp.b1[threadIdx.x];
    sh.b2[threadIdx.x] = cp.b2[threadIdx.x];
    sh.w3[threadIdx.x] = cp.w3[threadIdx.x];
  }
  __syncthreads();
}

// Face normals of a cell in the FP32 layout.
__device__ __forceinline__ void cell_normals(const CellIn<float>& c, float nx[3], float ny[3]) {
  nx[0] = c.g0.x, ny[0] = c.g0.y;
  nx[1] = c.g0.z, ny[1] = c.g0.w;
  nx[2] = c.g1.x, ny[2] = c.g1.y;
}

// The MLP alone on given FP32 features (rounded to bfloat16 like the step's).
__global__ void __launch_bounds__(kClThreads) k_closure_eval(const float* feats, float* s_out,
                                                             int64_t rows, ClosureParams cp) {
  __shared__ ClShared sh;
  load_small_params(cp, sh);
  ClFrag fr;
  load_frags(cp, fr);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  ClWarpSmem& w = sh.warp[warp];
  const int64_t wstride = (int64_t)gridDim.x * kClWarps * kRows;
  for (int64_t base = ((int64_t)blockIdx.x * kClWarps + warp) * kRows; base < rows;
       base += wstride) {
    for (int j = lane; j < kRows; j += 32) {
      float f[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      if (base + j < rows)
        for (int q = 0; q < 8; ++q) f[q] = feats[(base + j) * 8 + q];
      w.feat[j] = pack_features(f);
    }
    __syncwarp();
    warp_mlp(w, fr, sh.w3, cp.b3);
    __syncwarp();
    for (int j = lane; j < kRows; j += 32)
      if (base + j < rows) s_out[base + j] = w.s[j];
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// The scales as a pass of their own, then the step reading them.
//
// k_face_scales walks a list of the mesh's faces, each once (faces.cpp order:
// owner cell a, its face ka, the cell b across with its face kb, or a ghost
// code): a warp takes 32 faces, forms their features, evaluates the MLP on
// two 16-row tiles and writes each scale to both cells' slots s[3a + ka] and
// s[3b + kb].  The features are the same bits from either side of a face, so
// the scales are those of the fused kernel above.  k_step_scaled is the
// persistent one-thread-per-cell step with the flux's dissipation scaled by
// s[3i + k]: the per-cell state it keeps is that of the plain step, so it
// runs at the plain step's occupancy instead of carrying the cell across the
// MLP.
// ---------------------------------------------------------------------------
// What a face's row reads: its record and the two states (the state across
// is a ghost state at a boundary face).
struct FaceIn {
  FaceRec f;
  float4 UL, UR;
};

__device__ __forceinline__ void load_face(const StepArgs& a, const FaceRec* faces, int64_t row,
                                          FaceIn& x) {
  const float4* __restrict__ U = static_cast<const float4*>(a.U);
  x.f = faces[row];
  x.UL = __ldg(U + (x.f.a >> 2));
  const int nb = x.f.b >= 0 ? (x.f.b >> 2) : x.f.b;
  x.UR = neighbour_state<float>(x.UL, nb, x.f.nx, x.f.ny, U, a.uinf_f, a.n, a.err);
}

__global__ void __launch_bounds__(kClThreads) k_face_scales(StepArgs a, const FaceRec* faces,
                                                            int64_t nf, ClosureParams cp,
                                                            float* s_cf) {
  chain_entry();
  __shared__ ClShared sh;
  load_small_params(cp, sh);
  ClFrag fr;
  load_frags(cp, fr);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  ClWarpSmem& w = sh.warp[warp];
  const int64_t wstride = (int64_t)gridDim.x * kClWarps * 32;
  int64_t row = ((int64_t)blockIdx.x * kClWarps + warp) * 32 + lane;
  // this round's face and, issued before this round computes, the next's
  FaceIn cur, nxt;
  for (int64_t base = row - lane; base < nf; base += wstride, row += wstride) {
    const bool valid = row < nf;
    if (valid) load_face(a, faces, row, cur);
    float f[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (valid) {
      const Prim<float> L = primitive<float>(cur.UL), W = primitive<float>(cur.UR);
      face_features(cur.UL, L, cur.UR, W, cur.f.nx, cur.f.ny, face_len<float>(cur.f.nx, cur.f.ny),
                    f);
    }
    w.feat[lane] = pack_features(f);
    __syncwarp();
    warp_mlp(w, fr, sh.w3, cp.b3, 2);
    __syncwarp();
    if (valid) {
      const float sv = w.s[lane];
      s_cf[3 * (int64_t)(cur.f.a >> 2) + (cur.f.a & 3)] = sv;
      if (cur.f.b >= 0 && index_ok(cur.f.b >> 2, a.n, a.err))
        s_cf[3 * (int64_t)(cur.f.b >> 2) + (cur.f.b & 3)] = sv;
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// The MLP on the fifth-generation tensor cores (tcgen05), 128 rows at a time.
// A group of 128 threads owns 128 rows, one per thread.  Each thread writes
// its row's features (bfloat16, K columns 0..7; columns 8..10 hold 1.0
// against the bias parts of W1) into the layer-1 A operand in shared memory;
// one thread issues layer 1 (M 128, N 32, K 16) into the group's 32 TMEM
// columns and commits to the group's mbarrier; every thread reads its row of
// the accumulator (tcgen05.ld), applies ReLU, rounds to bfloat16 and writes
// its row of the layer-2 A operand (K 0..31; columns 32..34 hold 1.0 against
// the bias parts of W2); layer 2 (K 48, three MMAs) reuses the same TMEM
// columns; each thread reads its row back and forms layer 3 in registers
// (out_pair, the order of the mma.sync form).  The tensor core gives the
// accumulators of the mma.sync form bit for bit (tested: both forms give the
// same step), so the engines are interchangeable.
// Operands are K-major without swizzling (tc_util.cuh): element (r, k) of an
// operand of 16 k16 K columns sits at (r / 8) * 128 k16 + (k / 8) * 128 +
// (r % 8) * 16 + (k % 8) * 2 bytes.  Waits are bounded (polls); one that
// gives up (in any lane of a warp: the warp takes the result together) sets
// its group's abort flag, which the group's threads read only after the
// group's barrier, so the whole group stops there; the block records error
// bit 2, waits (bounded) for the group's MMAs still in flight (bit 4 if that
// gives up too) and frees its TMEM.
// ---------------------------------------------------------------------------
constexpr int kTcRows = 128;
constexpr unsigned kTcCols = 32;  // TMEM columns of one group: a 128 x 32 FP32 accumulator

struct __align__(128) TcRows {     // one group's A operands
  unsigned char a2[kTcRows * 96];  // layer 2: 128 x 48 (sbo 768)
  unsigned char a1[kTcRows * 32];  // layer 1: 128 x 16 (sbo 256)
};

struct __align__(128) TcWeights {  // B operands
  unsigned char w2[32 * 96];       // layer 2: 32 x 48 (sbo 768)
  unsigned char w1[32 * 32];       // layer 1: 32 x 16 (sbo 256)
  float w3[32];
};

struct TcBlock {
  uint64_t bar[2];  // per group
  int abort[2];     // per group: written by the group's threads only
  unsigned tmem;
};

__device__ __forceinline__ unsigned tc_off(int r, int k, int sbo) {
  return (unsigned)((r >> 3) * sbo + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ unsigned short bf16_bits(float x) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}

// The bias parts of b (hi, mid, lo: together its 24-bit significand), as
// bias_parts above.
__device__ __forceinline__ void bias3(float b, float p[3]) {
  p[0] = __bfloat162float(__float2bfloat16_rn(b));
  const float r1 = sub(b, p[0]);
  p[1] = __bfloat162float(__float2bfloat16_rn(r1));
  p[2] = sub(r1, p[1]);
}

// Barrier of group g's 128 threads (named barriers 1 and 2; literal ids, so
// the kernels reserve three barriers, not sixteen).
__device__ __forceinline__ void group_sync(int g) {
  if (g == 0)
    asm volatile("bar.sync 1, 128;" ::: "memory");
  else
    asm volatile("bar.sync 2, 128;" ::: "memory");
}

// Block setup for `groups` groups of 128 threads (blockDim = 128 groups):
// B operands, the constant columns of every row, TMEM (32 columns a group)
// and the groups' mbarriers.  Ends with a block barrier.
__device__ __forceinline__ void tc_setup(const ClosureParams& cp, TcWeights& w, TcRows* rows,
                                         TcBlock& tb, int groups) {
  const int tid = threadIdx.x, nthr = groups * kTcRows;
  const unsigned short* w1 = reinterpret_cast<const unsigned short*>(cp.w1);
  const unsigned short* w2 = reinterpret_cast<const unsigned short*>(cp.w2);
  for (int i = tid; i < 32 * 16; i += nthr) {
    const int n = i >> 4, k = i & 15;
    unsigned short v = 0;
    if (k < 8) {
      v = __ldg(w1 + n * 8 + k);
    } else if (k < 11) {
      float p[3];
      bias3(__ldg(cp.b1 + n), p);
      v = bf16_bits(p[k - 8]);
    }
    *reinterpret_cast<unsigned short*>(w.w1 + tc_off(n, k, 256)) = v;
  }
  for (int i = tid; i < 32 * 48; i += nthr) {
    const int n = i / 48, k = i % 48;
    unsigned short v = 0;
    if (k < 32) {
      v = __ldg(w2 + n * 32 + k);
    } else if (k < 35) {
      float p[3];
      bias3(__ldg(cp.b2 + n), p);
      v = bf16_bits(p[k - 32]);
    }
    *reinterpret_cast<unsigned short*>(w.w2 + tc_off(n, k, 768)) = v;
  }
  // this thread's row: A1 columns 8..15 = (1, 1, 1, 0, ...), A2 columns 32..47 likewise
  TcRows& r = rows[tid / kTcRows];
  const int row = tid % kTcRows;
  const uint4 ones = make_uint4(0x3F803F80u, 0x00003F80u, 0u, 0u);
  *reinterpret_cast<uint4*>(r.a1 + tc_off(row, 8, 256)) = ones;
  *reinterpret_cast<uint4*>(r.a2 + tc_off(row, 32, 768)) = ones;
  *reinterpret_cast<uint4*>(r.a2 + tc_off(row, 40, 768)) = make_uint4(0u, 0u, 0u, 0u);
  if (tid < 32) w.w3[tid] = __ldg(cp.w3 + tid);
  if (tid < 32) tc_alloc(&tb.tmem, kTcCols * (unsigned)groups);  // warp 0
  if (tid == 0) {
    for (int g = 0; g < groups; ++g) {
      mbar_init(&tb.bar[g], 1);
      tb.abort[g] = 0;
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
}

// One group's state across its chunks of 128 rows.
struct TcGroup {
  int id;          // group index (0 or 1)
  int row;         // this thread's row
  unsigned tmem;   // the group's first TMEM column, lane 0
  unsigned tlane;  // the same at this warp's 32 lanes
  unsigned phase;  // parity of the group's mbarrier
  bool pending;    // MMAs committed and not yet seen complete
};

__device__ __forceinline__ TcGroup tc_group(const TcBlock& tb) {
  TcGroup G;
  G.id = threadIdx.x / kTcRows;
  G.row = threadIdx.x % kTcRows;
  G.tmem = tb.tmem + kTcCols * (unsigned)G.id;
  G.tlane = G.tmem + ((unsigned)(32 * ((threadIdx.x >> 5) & 3)) << 16);
  G.phase = 0u;
  G.pending = false;
  return G;
}

// Layers 1-3 of the group's current 128 rows, whose features this group's
// threads wrote to rows.a1.  Returns false (in every thread of the group)
// when the group is stopping; else z of this thread's row, with ok = false
// if a wait gave up (z is then not formed; the group stops at its next call).
__device__ __forceinline__ bool tc_mlp(TcGroup& G, TcRows& r, const TcWeights& w, TcBlock& tb,
                                       float b3, unsigned limit, float& z, bool& ok) {
  constexpr unsigned idesc = tc_idesc_bf16(kTcRows, 32);
  volatile int* abort = &tb.abort[G.id];
  fence_async_smem();
  tc_fence_before();
  group_sync(G.id);
  if (*abort) return false;
  if (G.row == 0) {
    tc_fence_after();
    tc_mma(G.tmem, tc_desc(smem_addr(r.a1), 128, 256), tc_desc(smem_addr(w.w1), 128, 256), idesc,
           false);
    tc_commit(&tb.bar[G.id]);
  }
  G.pending = true;
  ok = __all_sync(0xffffffffu, mbar_wait(&tb.bar[G.id], G.phase, limit));
  float v[32];
  if (ok) {
    G.phase ^= 1u;
    G.pending = false;
    tc_fence_after();
    tc_ld32(G.tlane, v);
    uint4* dst = reinterpret_cast<uint4*>(r.a2 + tc_off(G.row, 0, 768));
#pragma unroll
    for (int g = 0; g < 4; ++g)
      dst[g * 8] = make_uint4(pack_bf16_relu(v[8 * g], v[8 * g + 1]),
                              pack_bf16_relu(v[8 * g + 2], v[8 * g + 3]),
                              pack_bf16_relu(v[8 * g + 4], v[8 * g + 5]),
                              pack_bf16_relu(v[8 * g + 6], v[8 * g + 7]));
  } else {
    *abort = 1;
  }
  fence_async_smem();
  tc_fence_before();
  group_sync(G.id);
  if (*abort) return false;
  if (G.row == 0) {
    tc_fence_after();
    const unsigned a2 = smem_addr(r.a2), w2 = smem_addr(w.w2);
#pragma unroll
    for (int k = 0; k < 3; ++k)
      tc_mma(G.tmem, tc_desc(a2 + 256 * k, 128, 768), tc_desc(w2 + 256 * k, 128, 768), idesc,
             k > 0);
    tc_commit(&tb.bar[G.id]);
  }
  G.pending = true;
  ok = __all_sync(0xffffffffu, mbar_wait(&tb.bar[G.id], G.phase, limit));
  if (!ok) {
    *abort = 1;  // the group stops at its next barrier
    return true;
  }
  G.phase ^= 1u;
  G.pending = false;
  tc_fence_after();
  tc_ld32(G.tlane, v);
  float p[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    p[c] = 0.0f;
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const int col = nt * 8 + 2 * c;
      p[c] = out_pair(p[c], v[col], v[col + 1], w.w3[col], w.w3[col + 1]);
    }
  }
  z = add(add(add(p[0], p[1]), add(p[2], p[3])), b3);
  return true;
}

// Block teardown: error bits of an abort, a bounded wait for each group's
// MMAs still in flight, TMEM freed.  Every thread of the block calls it.
__device__ __forceinline__ void tc_teardown(const TcGroup& G, TcBlock& tb, int groups, int* err,
                                            unsigned drain_limit) {
  if (tb.abort[G.id] && G.row == 0) {
    atomicOr(err, 2);
    if (G.pending && !mbar_wait(&tb.bar[G.id], G.phase, drain_limit)) atomicOr(err, 4);
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x < 32) {
    tc_fence_after();
    tc_dealloc(tb.tmem, kTcCols * (unsigned)groups);
  }
}

// k_face_scales with the MLP on tcgen05: one group per block, 128 faces at
// a time, persistent.
__global__ void __launch_bounds__(kTcRows) k_face_scales_tc(StepArgs a, const FaceRec* faces,
                                                            int64_t nf, ClosureParams cp,
                                                            float* s_cf) {
  chain_entry();
  __shared__ TcRows rows;
  __shared__ TcWeights w;
  __shared__ TcBlock tb;
  tc_setup(cp, w, &rows, tb, 1);
  TcGroup G = tc_group(tb);
  for (int64_t base = (int64_t)blockIdx.x * kTcRows; base < nf;
       base += (int64_t)gridDim.x * kTcRows) {
    const int64_t row = base + G.row;
    const bool valid = row < nf;
    FaceIn cur;
    float f[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (valid) {
      load_face(a, faces, row, cur);
      const Prim<float> L = primitive<float>(cur.UL), W = primitive<float>(cur.UR);
      face_features(cur.UL, L, cur.UR, W, cur.f.nx, cur.f.ny, face_len<float>(cur.f.nx, cur.f.ny),
                    f);
    }
    *reinterpret_cast<uint4*>(rows.a1 + tc_off(G.row, 0, 256)) = pack_features(f);
    float z;
    bool ok;
    if (!tc_mlp(G, rows, w, tb, cp.b3, a.wait_limit, z, ok)) break;
    if (ok && valid) {
      const float sv = scale_of(z);
      s_cf[3 * (int64_t)(cur.f.a >> 2) + (cur.f.a & 3)] = sv;
      if (cur.f.b >= 0 && index_ok(cur.f.b >> 2, a.n, a.err))
        s_cf[3 * (int64_t)(cur.f.b >> 2) + (cur.f.b & 3)] = sv;
    }
  }
  tc_teardown(G, tb, 1, a.err, a.drain_limit);
}

template <int MODE, bool COMP>
__global__ void __launch_bounds__(kBlock) k_step_scaled(StepArgs a, const float* s_cf) {
  chain_entry();
  const float4* __restrict__ U = static_cast<const float4*>(a.U);
  const float4* __restrict__ geom = static_cast<const float4*>(a.geom);
  float4* out = static_cast<float4*>(a.out);
  double t = 0.0, dt = 0.0;
  if (MODE != kModeResidual) dt = step_dt(a, t);
  float bmin = INFINITY;
  bool ok = true;
  const int n = (int)a.n;
  const int stride = gridDim.x * blockDim.x;
  CellIn<float> cur, nxt;
  float sc[3], sn[3];  // the scales of the cell, and of the next (loaded with its records)
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    load_cell<float, MODE, COMP>(a, U, geom, i, cur);
#pragma unroll
    for (int k = 0; k < 3; ++k) sc[k] = __ldg(s_cf + 3 * i + k);
  }
  for (; i < n; i += stride) {
    const int j = i + stride;
    if (j < n) {
      load_cell<float, MODE, COMP>(a, U, geom, j, nxt);
#pragma unroll
      for (int k = 0; k < 3; ++k) sn[k] = __ldg(s_cf + 3 * j + k);
    }
    const Prim<float> L = primitive<float>(cur.U);
    const int nb[3] = {cur.n0, cur.n1, cur.n2};
    const float nx[3] = {cur.g0.x, cur.g0.z, cur.g1.x}, ny[3] = {cur.g0.y, cur.g0.w, cur.g1.y};
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    float perim = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float4 UR = neighbour_state<float>(cur.U, nb[k], nx[k], ny[k], U, a.uinf_f, a.n, a.err);
      const Prim<float> W = primitive<float>(UR);
      const float len = face_len<float>(nx[k], ny[k]);
      face_flux_acc<float, true>(cur.U, L, UR, W, nx[k], ny[k], len, sc[k], acc);
      perim = k == 0 ? len : add(perim, len);
    }
    finish_cell<float, MODE, COMP>(a, out, i, cur, acc, perim, (float)dt, bmin, ok);
    cur = nxt;
#pragma unroll
    for (int k = 0; k < 3; ++k) sc[k] = sn[k];
  }
  if (MODE == kModeFE || MODE == kModeRK2b) {
    if (!ok) atomicOr(a.err, 1);
    const double m = (double)block_min<float>(bmin);
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
// The learned step on tiles (with shape 7): a block stages the states and
// primitives of its tile and the tile's ring in shared memory (tile_math.cuh)
// and walks the tile's face list (tiles.cpp) 32 faces per warp: features,
// the MLP on two 16-row tiles, then the scaled flux of each face, written to
// the slot of its cell and, negated, to the slot of the face pointing back
// (the face flux is antisymmetric bit for bit, and the features are the same
// bits from either side).  Every tile cell then adds its three slots in face
// order and finishes.  Each face's features, scale and flux are formed once
// and every primitive once per cell, in one launch -- the same bits as the
// two passes above.
// ---------------------------------------------------------------------------
template <int MODE, bool COMP, int THREADS, int KMAX>
__global__ void __launch_bounds__(THREADS) k_step_closure_tile(StepArgs a, ClosureParams cp) {
  chain_entry();
  constexpr int kWarps = THREADS / 32;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float4* sU = reinterpret_cast<float4*>(smem_raw);  // [t1_cap] states
  float4* sP = sU + a.t1_cap;                          // [t1_cap] (u, v, p, c)
  float4* sF = sP + a.t1_cap;                          // [3 tile] face flux values
  ClWarpSmem* wsm = reinterpret_cast<ClWarpSmem*>(sF + 3 * a.tile);  // [kWarps] MLP rows
  __shared__ float w3s[32];
  if (threadIdx.x < 32) w3s[threadIdx.x] = cp.w3[threadIdx.x];
  ClFrag fr;
  load_frags(cp, fr);
  const float4* __restrict__ U = static_cast<const float4*>(a.U);
  const float4* __restrict__ geom = static_cast<const float4*>(a.geom);
  float4* out = static_cast<float4*>(a.out);
  const int t0 = blockIdx.x * a.tile;  // cell ids are 32-bit
  const int nt = min(a.tile, (int)a.n - t0);
  const int hs = __ldg(a.tile_info + 2 * blockIdx.x);
  const int h1 = __ldg(a.tile_info + 2 * blockIdx.x + 1);
  __shared__ double s_t, s_dt;
  if (threadIdx.x == 0 && MODE != kModeResidual) block_dt(a, s_t, s_dt);
  stage_states<float, THREADS, kStageBatch<float, KMAX>>(U, t0, nt, h1, a.halo_id + hs, sU, sP,
                                                         a.n, a.err);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  ClWarpSmem& w = wsm[warp];
  const int fb = __ldg(a.tile_face_off + blockIdx.x), fe = __ldg(a.tile_face_off + blockIdx.x + 1);
  for (int base = fb + warp * 32; base < fe; base += kWarps * 32) {  // uniform in the warp
    const int f = base + lane;
    float feat[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    unsigned e = 0u, q = 0u, kv = 0u, v = 0u;
    float4 UL = make_float4(0.f, 0.f, 0.f, 0.f), UR = UL;
    Prim<float> L{0.f, 0.f, 0.f, 0.f}, W = L;
    float nx = 0.f, ny = 0.f, len = 0.f;
    bool use = false;
    if (f < fe) {
      const uint2 r = __ldg(a.tile_face + f);
      e = r.x & 0xffffu, q = (r.x >> 16) & 3u, kv = (r.x >> 18) & 3u, v = r.y;
      use = index_ok(e, nt, a.err);
      if (use) {
        face_normal<float>(geom, t0 + (int)e, q, nx, ny);
        UL = sU[e];
        L = rec_prim<float>(sP[e]);
        if (v < kGhostCodes) {
          if (index_ok(v, nt + h1, a.err)) {
            UR = sU[v];
            W = rec_prim<float>(sP[v]);
          } else {
            UR = UL;
            W = L;
          }
        } else {
          UR = ghost<float>((int)v - 0x10000, UL, nx, ny, a.uinf_f);
          W = primitive<float>(UR);
        }
        len = face_len<float>(nx, ny);
        face_features(UL, L, UR, W, nx, ny, len, feat);
      }
    }
    w.feat[lane] = pack_features(feat);
    __syncwarp();
    warp_mlp(w, fr, w3s, cp.b3, 2);
    __syncwarp();
    if (use) {
      float X[4];
      face_flux_value<float, true>(UL, L, UR, W, nx, ny, len, w.s[lane], X);
      sF[3 * e + q] = make_float4(X[0], X[1], X[2], X[3]);
      if (v < (unsigned)nt) sF[3 * v + kv] = make_float4(-X[0], -X[1], -X[2], -X[3]);
    }
    __syncwarp();
  }
  __syncthreads();
  const double t = MODE != kModeResidual ? s_t : 0.0, dt = MODE != kModeResidual ? s_dt : 0.0;
  float bmin = INFINITY;
  bool ok = true;
#pragma unroll
  for (int k = 0; k < KMAX; ++k) {
    const int e = threadIdx.x + k * THREADS;
    if (e < nt) {
      const int i = t0 + e;
      CellIn<float> c;
      c.g0 = __ldg(geom + 2 * i);
      c.g1 = __ldg(geom + 2 * i + 1);
      c.U = sU[e];
      if (MODE == kModeRK2b) c.base = static_cast<const float4*>(a.Ubase)[i];
      if (COMP && MODE != kModeResidual) c.lo = a.lo[i];
      if (COMP && MODE == kModeRK2b) c.lo_stage = a.lo_stage[i];
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const float4 X = sF[3 * e + q];
        acc[0] = add(acc[0], X.x);
        acc[1] = add(acc[1], X.y);
        acc[2] = add(acc[2], X.z);
        acc[3] = add(acc[3], X.w);
      }
      const float perim = add(add(face_len<float>(c.g0.x, c.g0.y), face_len<float>(c.g0.z, c.g0.w)),
                              face_len<float>(c.g1.x, c.g1.y));
      finish_cell<float, MODE, COMP>(a, out, i, c, acc, perim, (float)dt, bmin, ok);
    }
  }
  if (MODE == kModeFE || MODE == kModeRK2b) {
    if (!ok) atomicOr(a.err, 1);
    const double m = (double)block_min<float>(bmin);
    if (threadIdx.x == 0) {
      atomicMin(a.bmin_write, (unsigned long long)__double_as_longlong(m));
      if (blockIdx.x == 0) {
        *a.t_write = t + dt;
        *a.bmin_reset = kInfBits;
      }
    }
  }
}

// The learned step on shape 7's tiles with the MLP on tcgen05: as
// k_step_closure_tile, but the block's 256 threads are two groups of 128
// that take the tile's faces 128 at a time (group g: faces fb + 256 j + 128 g
// + row), one face per thread, whose features, scale and flux stay in that
// thread.  Dynamic shared memory: states, primitives and face fluxes as in
// k_step_closure_tile, then the groups' operands and the weights.
template <int MODE, bool COMP, int KMAX>
__global__ void __launch_bounds__(2 * kTcRows) k_step_closure_tile_tc(StepArgs a,
                                                                      ClosureParams cp) {
  chain_entry();
  constexpr int THREADS = 2 * kTcRows;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float4* sU = reinterpret_cast<float4*>(smem_raw);  // [t1_cap] states
  float4* sP = sU + a.t1_cap;                          // [t1_cap] (u, v, p, c)
  float4* sF = sP + a.t1_cap;                          // [3 tile] face flux values
  const size_t tc_at = ((size_t)(2 * a.t1_cap + 3 * a.tile) * 16 + 127) & ~(size_t)127;
  TcRows* rows = reinterpret_cast<TcRows*>(smem_raw + tc_at);  // [2]
  TcWeights& w = *reinterpret_cast<TcWeights*>(rows + 2);
  __shared__ TcBlock tb;
  tc_setup(cp, w, rows, tb, 2);
  TcGroup G = tc_group(tb);
  const float4* __restrict__ U = static_cast<const float4*>(a.U);
  const float4* __restrict__ geom = static_cast<const float4*>(a.geom);
  float4* out = static_cast<float4*>(a.out);
  const int t0 = blockIdx.x * a.tile;  // cell ids are 32-bit
  const int nt = min(a.tile, (int)a.n - t0);
  const int hs = __ldg(a.tile_info + 2 * blockIdx.x);
  const int h1 = __ldg(a.tile_info + 2 * blockIdx.x + 1);
  __shared__ double s_t, s_dt;
  if (threadIdx.x == 0 && MODE != kModeResidual) block_dt(a, s_t, s_dt);
  stage_states<float, THREADS, kStageBatch<float, KMAX>>(U, t0, nt, h1, a.halo_id + hs, sU, sP,
                                                         a.n, a.err);
  __syncthreads();
  TcRows& r = rows[G.id];
  const int fb = __ldg(a.tile_face_off + blockIdx.x), fe = __ldg(a.tile_face_off + blockIdx.x + 1);
  for (int base = fb + G.id * kTcRows; base < fe; base += THREADS) {  // uniform in the group
    const int f = base + G.row;
    float feat[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    unsigned e = 0u, q = 0u, kv = 0u, v = 0u;
    float4 UL = make_float4(0.f, 0.f, 0.f, 0.f), UR = UL;
    Prim<float> L{0.f, 0.f, 0.f, 0.f}, W = L;
    float nx = 0.f, ny = 0.f, len = 0.f;
    bool use = false;
    if (f < fe) {
      const uint2 rec = __ldg(a.tile_face + f);
      e = rec.x & 0xffffu, q = (rec.x >> 16) & 3u, kv = (rec.x >> 18) & 3u, v = rec.y;
      use = index_ok(e, nt, a.err);
      if (use) {
        face_normal<float>(geom, t0 + (int)e, q, nx, ny);
        UL = sU[e];
        L = rec_prim<float>(sP[e]);
        if (v < kGhostCodes) {
          if (index_ok(v, nt + h1, a.err)) {
            UR = sU[v];
            W = rec_prim<float>(sP[v]);
          } else {
            UR = UL;
            W = L;
          }
        } else {
          UR = ghost<float>((int)v - 0x10000, UL, nx, ny, a.uinf_f);
          W = primitive<float>(UR);
        }
        len = face_len<float>(nx, ny);
        face_features(UL, L, UR, W, nx, ny, len, feat);
      }
    }
    *reinterpret_cast<uint4*>(r.a1 + tc_off(G.row, 0, 256)) = pack_features(feat);
    float z;
    bool ok;
    if (!tc_mlp(G, r, w, tb, cp.b3, a.wait_limit, z, ok)) break;
    if (use && ok) {
      float X[4];
      face_flux_value<float, true>(UL, L, UR, W, nx, ny, len, scale_of(z), X);
      sF[3 * e + q] = make_float4(X[0], X[1], X[2], X[3]);
      if (v < (unsigned)nt) sF[3 * v + kv] = make_float4(-X[0], -X[1], -X[2], -X[3]);
    }
  }
  tc_teardown(G, tb, 2, a.err, a.drain_limit);  // ends with a block barrier
  const double t = MODE != kModeResidual ? s_t : 0.0, dt = MODE != kModeResidual ? s_dt : 0.0;
  float bmin = INFINITY;
  bool cell_ok = true;
#pragma unroll
  for (int k = 0; k < KMAX; ++k) {
    const int e = threadIdx.x + k * THREADS;
    if (e < nt) {
      const int i = t0 + e;
      CellIn<float> c;
      c.g0 = __ldg(geom + 2 * i);
      c.g1 = __ldg(geom + 2 * i + 1);
      c.U = sU[e];
      if (MODE == kModeRK2b) c.base = static_cast<const float4*>(a.Ubase)[i];
      if (COMP && MODE != kModeResidual) c.lo = a.lo[i];
      if (COMP && MODE == kModeRK2b) c.lo_stage = a.lo_stage[i];
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const float4 X = sF[3 * e + q];
        acc[0] = add(acc[0], X.x);
        acc[1] = add(acc[1], X.y);
        acc[2] = add(acc[2], X.z);
        acc[3] = add(acc[3], X.w);
      }
      const float perim = add(add(face_len<float>(c.g0.x, c.g0.y), face_len<float>(c.g0.z, c.g0.w)),
                              face_len<float>(c.g1.x, c.g1.y));
      finish_cell<float, MODE, COMP>(a, out, i, c, acc, perim, (float)dt, bmin, cell_ok);
    }
  }
  if (MODE == kModeFE || MODE == kModeRK2b) {
    if (!cell_ok) atomicOr(a.err, 1);
    const double m = (double)block_min<float>(bmin);
    if (threadIdx.x == 0) {
      atomicMin(a.bmin_write, (unsigned long long)__double_as_longlong(m));
      if (blockIdx.x == 0) {
        *a.t_write = t + dt;
        *a.bmin_reset = kInfBits;
      }
    }
  }
}

template <typename K>
unsigned cl_resident_blocks(K kernel) {
  static int cached = 0;
  if (cached == 0) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kClThreads, 0) !=
            cudaSuccess ||
        per_sm < 1)
      return 512;
    cached = sms * per_sm;
  }
  return (unsigned)cached;
}

template <typename K>
unsigned cl_grid(K kernel, int64_t items_per_warp_group, int64_t n) {
  const int64_t want = std::max<int64_t>(1, (n + items_per_warp_group * kClWarps - 1) /
                                                (items_per_warp_group * kClWarps));
  const unsigned cap = cl_resident_blocks(kernel);
  return (unsigned)std::min<int64_t>(want, cap);
}


// ---------------------------------------------------------------------------
// Training: one-step loss and its gradient.
//   U1 = U0 + dt R(U0; theta)   (forward Euler, fixed dt)
//   L  = sum_T V_T sum_q ((U1 - Ut)_q / w_q)^2
// dL/ds of a face = sum_q dL/dU1_q (-dt / V) dF_q/ds, where the flux is affine
// in s with dF/ds = -(|q_L + q_R| + |n| (c_L + c_R)) / 4 (U_R - U_L); then
// back through the MLP (FP32, straight through the bfloat16 roundings).
// ---------------------------------------------------------------------------
constexpr int kGrWarps = 2;
constexpr int kGrThreads = 32 * kGrWarps;

struct __align__(16) GrWarpSmem {
  ClWarpSmem f;               // features (bfloat16) and scales
  unsigned h1[kRows * 16];    // hidden layer 1 after ReLU, bfloat16 pairs
  float h2[kRows * 32];       // hidden layer 2 after ReLU
  float sig[kRows];           // sigmoid(z)
  float gs[kRows];            // dL/ds
};

struct GrShared {
  GrWarpSmem warp[kGrWarps];
  float b1[32], b2[32], w3[32];
  float W2[32 * 32];          // FP32 copy of the bfloat16 weights, [out][in]
};

__device__ __forceinline__ float bf16_lo(unsigned v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf16_hi(unsigned v) { return __uint_as_float(v & 0xffff0000u); }

__global__ void __launch_bounds__(kGrThreads) k_closure_grad(StepArgs a, const float4* Ut,
                                                             float dt, float4 wq,
                                                             ClosureParams cp, float* gpart,
                                                             double* lpart) {
  __shared__ GrShared sh;
  if (threadIdx.x < 32) {
    sh.b1[threadIdx.x] = cp.b1[threadIdx.x];
    sh.b2[threadIdx.x] = cp.b2[threadIdx.x];
    sh.w3[threadIdx.x] = cp.w3[threadIdx.x];
  }
  for (int j = threadIdx.x; j < 32 * 16; j += blockDim.x) {
    const unsigned v = cp.w2[j];
    sh.W2[2 * j] = bf16_lo(v);
    sh.W2[2 * j + 1] = bf16_hi(v);
  }
  __syncthreads();
  ClFrag fr;
  load_frags(cp, fr);
  const float4* __restrict__ U = static_cast<const float4*>(a.U);
  const float4* __restrict__ geom = static_cast<const float4*>(a.geom);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, r = lane >> 2, cq = lane & 3;
  GrWarpSmem& w = sh.warp[warp];
  const float iw2[4] = {1.0f / (wq.x * wq.x), 1.0f / (wq.y * wq.y), 1.0f / (wq.z * wq.z),
                        1.0f / (wq.w * wq.w)};
  // per-lane gradient accumulators: lane o owns layer-2 unit o and layer-1 unit o
  float gW2[32], gW1[8], gb1 = 0.0f, gb2 = 0.0f, gw3 = 0.0f, gb3 = 0.0f;
#pragma unroll
  for (int j = 0; j < 32; ++j) gW2[j] = 0.0f;
#pragma unroll
  for (int j = 0; j < 8; ++j) gW1[j] = 0.0f;
  double loss = 0.0;
  const int64_t wstride = (int64_t)gridDim.x * kGrWarps * 32;
  for (int64_t base = ((int64_t)blockIdx.x * kGrWarps + warp) * 32; base < a.n; base += wstride) {
    const int64_t i = base + lane;
    const bool valid = i < a.n;
    CellIn<float> c;
    float4 UR[3];
    Prim<float> L, W[3];
    float nx[3], ny[3], len[3];
    if (valid) {
      load_cell<float, kModeResidual, false>(a, U, geom, i, c);
      L = primitive<float>(c.U);
      cell_normals(c, nx, ny);
      const int nb[3] = {c.n0, c.n1, c.n2};
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        UR[k] = neighbour_state<float>(c.U, nb[k], nx[k], ny[k], U, a.uinf_f, a.n, a.err);
        W[k] = primitive<float>(UR[k]);
        len[k] = face_len<float>(nx[k], ny[k]);
        float f[8];
        face_features(c.U, L, UR[k], W[k], nx[k], ny[k], len[k], f);
        w.f.feat[k * 32 + lane] = pack_features(f);
      }
    } else {
#pragma unroll
      for (int k = 0; k < 3; ++k) w.f.feat[k * 32 + lane] = make_uint4(0u, 0u, 0u, 0u);
    }
    __syncwarp();
    // forward, keeping what the backward pass needs
    for (int t = 0; t < kRows / 16; ++t) {
      float a1[4][4], g[4][4];
      unsigned A2[2][4];
      tile_forward(w.f, t, fr, a1, A2, g);
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        w.h1[(16 * t + r) * 16 + nt * 4 + cq] = A2[nt >> 1][(nt & 1) ? 2 : 0];
        w.h1[(16 * t + r + 8) * 16 + nt * 4 + cq] = A2[nt >> 1][(nt & 1) ? 3 : 1];
        const int col = nt * 8 + 2 * cq;
        w.h2[(16 * t + r) * 32 + col] = relu(g[nt][0]);
        w.h2[(16 * t + r) * 32 + col + 1] = relu(g[nt][1]);
        w.h2[(16 * t + r + 8) * 32 + col] = relu(g[nt][2]);
        w.h2[(16 * t + r + 8) * 32 + col + 1] = relu(g[nt][3]);
      }
      float z0, z1;
      tile_output(g, sh.w3, cp.b3, z0, z1);
      if (cq == 0) {
        w.sig[16 * t + r] = sigmoid(z0);
        w.sig[16 * t + r + 8] = sigmoid(z1);
      }
    }
    __syncwarp();
    // one forward-Euler step of the own cell, its loss and dL/ds per face
    if (valid) {
      float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      float dFds[3][4];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float sk = fma_(1.3f, w.sig[k * 32 + lane], 0.2f);
        face_flux_acc<float, true>(c.U, L, UR[k], W[k], nx[k], ny[k], len[k], sk, acc);
        const float qL = fma_(L.u, nx[k], mul(L.v, ny[k]));
        const float qR = fma_(W[k].u, nx[k], mul(W[k].v, ny[k]));
        const float na = mul(-0.25f, fma_(len[k], add(L.c, W[k].c), fabsf(add(qL, qR))));
        dFds[k][0] = na * (UR[k].x - c.U.x);
        dFds[k][1] = na * (UR[k].y - c.U.y);
        dFds[k][2] = na * (UR[k].z - c.U.z);
        dFds[k][3] = na * (UR[k].w - c.U.w);
      }
      const float invV = c.g1.z;
      const float f = -dt * invV;
      const float fh = mul(0.5f, f);  // acc holds twice the flux sum
      const float V = 1.0f / invV;
      const float4 ut = Ut[i];
      const float d[4] = {fma_(fh, acc[0], c.U.x) - ut.x, fma_(fh, acc[1], c.U.y) - ut.y,
                          fma_(fh, acc[2], c.U.z) - ut.z, fma_(fh, acc[3], c.U.w) - ut.w};
      float gU[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        loss += (double)V * (double)d[q] * (double)d[q] * (double)iw2[q];
        gU[q] = 2.0f * V * d[q] * iw2[q];
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        float gsk = 0.0f;
#pragma unroll
        for (int q = 0; q < 4; ++q) gsk += gU[q] * f * dFds[k][q];
        w.gs[k * 32 + lane] = gsk;
      }
    } else {
#pragma unroll
      for (int k = 0; k < 3; ++k) w.gs[k * 32 + lane] = 0.0f;
    }
    __syncwarp();
    // backward through the MLP, row by row; lane o owns unit o of both layers
    const int o = lane;
    for (int row = 0; row < kRows; ++row) {
      const float sg = w.sig[row];
      const float dz = w.gs[row] * 1.3f * sg * (1.0f - sg);
      const float h2o = w.h2[row * 32 + o];
      gw3 += dz * h2o;
      gb3 += dz;  // every lane the same; lane 0's copy is used
      const float da2 = h2o > 0.0f ? dz * sh.w3[o] : 0.0f;
      gb2 += da2;
#pragma unroll
      for (int jj = 0; jj < 16; ++jj) {
        const unsigned hp = w.h1[row * 16 + jj];
        gW2[2 * jj] += da2 * bf16_lo(hp);
        gW2[2 * jj + 1] += da2 * bf16_hi(hp);
      }
      // dL/dh1 of unit j = o: sum over the outputs p of W2[p][o] da2_p
      float dh1 = 0.0f;
#pragma unroll
      for (int pp = 0; pp < 32; ++pp) dh1 += sh.W2[pp * 32 + o] * __shfl_sync(0xffffffffu, da2, pp);
      const unsigned hp = w.h1[row * 16 + (o >> 1)];
      const float h1o = (o & 1) ? bf16_hi(hp) : bf16_lo(hp);
      const float da1 = h1o > 0.0f ? dh1 : 0.0f;
      gb1 += da1;
      const uint4 xv = w.f.feat[row];
      const unsigned xs[4] = {xv.x, xv.y, xv.z, xv.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        gW1[2 * q] += da1 * bf16_lo(xs[q]);
        gW1[2 * q + 1] += da1 * bf16_hi(xs[q]);
      }
    }
    __syncwarp();
  }
  // deterministic block reduction: warps in order, through shared memory
  __syncthreads();
  float* red = reinterpret_cast<float*>(&sh.warp[0]);  // reuse: kGrWarps x kClosureParams floats
  {
    float* mine = red + warp * kClosureParams;
    const int o = lane;
    for (int j = 0; j < 8; ++j) mine[o * 8 + j] = gW1[j];           // W1[o][j]
    mine[256 + o] = gb1;                                            // b1[o]
    for (int j = 0; j < 32; ++j) mine[288 + o * 32 + j] = gW2[j];   // W2[o][j]
    mine[1312 + o] = gb2;                                           // b2[o]
    mine[1344 + o] = gw3;                                           // w3[o]
    if (o == 0) mine[1376] = gb3;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < kClosureParams; j += blockDim.x) {
    float sum = 0.0f;
    for (int wv = 0; wv < kGrWarps; ++wv) sum += red[wv * kClosureParams + j];
    gpart[(int64_t)blockIdx.x * kClosureParams + j] = sum;
  }
  // loss: warp shuffle, then warps in order
  for (int off = 16; off > 0; off >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, off);
  __shared__ double lw[kGrWarps];
  if (lane == 0) lw[warp] = loss;
  __syncthreads();
  if (threadIdx.x == 0) {
    double l = 0.0;
    for (int wv = 0; wv < kGrWarps; ++wv) l += lw[wv];
    lpart[blockIdx.x] = l;
  }
}

// Sums the per-block partials in block order (one thread per parameter).
__global__ void k_closure_grad_final(const float* gpart, const double* lpart, int nblocks,
                                     float* grad, double* loss) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < kClosureParams) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += (double)gpart[(int64_t)b * kClosureParams + j];
    grad[j] = (float)s;
  }
  if (j == 0) {
    double l = 0.0;
    for (int b = 0; b < nblocks; ++b) l += lpart[b];
    *loss = l;
  }
}

// Adam (Kingma and Ba, 2015) on FP32 master weights.
__global__ void k_adam(float* theta, const float* grad, float* m, float* v, int n, float lr,
                       float b1, float b2, float eps, float c1, float c2) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const float g = grad[j];
  const float mj = b1 * m[j] + (1.0f - b1) * g;
  const float vj = b2 * v[j] + (1.0f - b2) * g * g;
  m[j] = mj;
  v[j] = vj;
  theta[j] -= lr * (mj / c1) / (sqrtf(vj / c2) + eps);
}

__global__ void k_pack_closure(const float* theta, unsigned* w1, unsigned* w2, float* b) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const float* W1 = theta;
  const float* b1 = W1 + 32 * 8;
  const float* W2 = b1 + 32;
  const float* b2 = W2 + 32 * 32;
  const float* w3 = b2 + 32;
  const float* b3 = w3 + 32;
  if (j < 32 * 4) w1[j] = pack_bf16(W1[2 * j], W1[2 * j + 1]);  // row-major pairs
  if (j < 32 * 16) w2[j] = pack_bf16(W2[2 * j], W2[2 * j + 1]);
  if (j < 32) {
    b[j] = b1[j];
    b[32 + j] = b2[j];
    b[64 + j] = w3[j];
  }
  if (j == 0) b[96] = b3[0];
}

}  // namespace

cudaError_t launch_pack_closure(const float* theta, unsigned* w1, unsigned* w2, float* b,
                                cudaStream_t s) {
  k_pack_closure<<<2, 256, 0, s>>>(theta, w1, w2, b);
  return cudaGetLastError();
}


int closure_grad_blocks() {
  static int cached = 0;
  if (cached == 0) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_closure_grad, kGrThreads, 0) !=
            cudaSuccess ||
        per_sm < 1)
      return 256;
    cached = sms * per_sm;
  }
  return cached;
}

cudaError_t launch_closure_grad(const StepArgs& a, const float* Ut, double dt, const double* w,
                                const ClosureParams& cp, float* gpart, double* lpart,
                                int max_blocks, float* grad, double* loss, cudaStream_t s) {
  const int64_t want = std::max<int64_t>(1, (a.n + 32 * kGrWarps - 1) / (32 * kGrWarps));
  const int nb = (int)std::min<int64_t>(want, std::min(max_blocks, closure_grad_blocks()));
  k_closure_grad<<<nb, kGrThreads, 0, s>>>(a, reinterpret_cast<const float4*>(Ut), (float)dt,
                                           make_float4((float)w[0], (float)w[1], (float)w[2],
                                                       (float)w[3]),
                                           cp, gpart, lpart);
  k_closure_grad_final<<<(kClosureParams + 255) / 256, 256, 0, s>>>(gpart, lpart, nb, grad, loss);
  return cudaGetLastError();
}

cudaError_t launch_adam(float* theta, const float* grad, float* m, float* v, int n, double lr,
                        double b1, double b2, double eps, int64_t step, cudaStream_t s) {
  const double c1 = 1.0 - std::pow(b1, (double)step), c2 = 1.0 - std::pow(b2, (double)step);
  k_adam<<<(n + 255) / 256, 256, 0, s>>>(theta, grad, m, v, n, (float)lr, (float)b1, (float)b2,
                                         (float)eps, (float)c1, (float)c2);
  return cudaGetLastError();
}

cudaError_t launch_closure_eval(const float* feats, float* s_out, int64_t rows,
                                const ClosureParams& cp, cudaStream_t s) {
  if (rows <= 0) return cudaSuccess;
  k_closure_eval<<<cl_grid(k_closure_eval, kRows, rows), kClThreads, 0, s>>>(feats, s_out, rows,
                                                                              cp);
  return cudaGetLastError();
}


cudaError_t launch_face_scales(const StepArgs& a, const FaceRec* faces, int64_t nf,
                               const ClosureParams& cp, float* s_cf, cudaStream_t s) {
  if (nf <= 0) return cudaSuccess;
  if (cp.tc) {
    // eight resident blocks per SM (58 registers and 21 KB of shared memory
    // allow eight; each holds kTcCols of the SM's 512 TMEM columns)
    static unsigned cap = 0;
    if (cap == 0) {
      int dev = 0, sms = 0;
      cudaError_t e = cudaGetDevice(&dev);
      if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (e != cudaSuccess) return e;
      cap = (unsigned)sms * 8u;
    }
    const int64_t want = (nf + kTcRows - 1) / kTcRows;
    return launch_chained(k_face_scales_tc, (unsigned)std::min<int64_t>(want, cap), kTcRows, 0,
                          s, a.chained, a, faces, nf, cp, s_cf);
  }
  return launch_chained(k_face_scales, cl_grid(k_face_scales, 32, nf), kClThreads, 0, s,
                        a.chained, a, faces, nf, cp, s_cf);
}

namespace {
template <int MODE, bool COMP>
cudaError_t launch_scaled_t(const StepArgs& a, const float* s_cf, cudaStream_t s) {
  auto k = k_step_scaled<MODE, COMP>;
  static int per_sm = 0, sms = 0;
  if (per_sm == 0) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kBlock, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
  }
  const int64_t want = (a.n + kBlock - 1) / kBlock, cap = (int64_t)sms * per_sm;
  return launch_chained(k, (unsigned)std::max<int64_t>(1, std::min(want, cap)), kBlock, 0, s,
                        a.chained, a, s_cf);
}
}  // namespace

size_t closure_tile_smem_bytes(int t1_cap, int tile, bool tc) {
  if (tc) {
    const size_t at = (tile_faces_smem_bytes(false, t1_cap, tile) + 127) & ~(size_t)127;
    return at + 2 * sizeof(TcRows) + sizeof(TcWeights);
  }
  return tile_faces_smem_bytes(false, t1_cap, tile) + (size_t)8 * sizeof(ClWarpSmem);
}

namespace {
template <int MODE, bool COMP, int KMAX>
cudaError_t launch_cl_tile_t(const StepArgs& a, const ClosureParams& cp, cudaStream_t s) {
  auto k = cp.tc ? k_step_closure_tile_tc<MODE, COMP, KMAX>
                 : k_step_closure_tile<MODE, COMP, 256, KMAX>;
  const size_t smem = closure_tile_smem_bytes(a.t1_cap, a.tile, cp.tc);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t tiles = (a.n + a.tile - 1) / a.tile;
  return launch_chained(k, (unsigned)tiles, 256, smem, s, a.chained, a, cp);
}

template <int MODE, bool COMP>
cudaError_t launch_cl_tile_size(const StepArgs& a, const ClosureParams& cp, cudaStream_t s) {
  if (a.tile < 1 || a.tile > 1024) return cudaErrorInvalidValue;
  if (a.tile <= 256) return launch_cl_tile_t<MODE, COMP, 1>(a, cp, s);
  if (a.tile <= 512) return launch_cl_tile_t<MODE, COMP, 2>(a, cp, s);
  if (a.tile <= 768) return launch_cl_tile_t<MODE, COMP, 3>(a, cp, s);
  return launch_cl_tile_t<MODE, COMP, 4>(a, cp, s);
}
}  // namespace

cudaError_t launch_step_closure_tile(int mode, const StepArgs& a, const ClosureParams& cp,
                                     cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  if (!a.cell_ln || !a.tile_info || !a.halo_id || !a.tile_face_off || !a.tile_face || a.tile_vq)
    return cudaErrorInvalidValue;
  const bool comp = a.lo != nullptr;
  switch (mode) {
    case kModeFE:
      return comp ? launch_cl_tile_size<kModeFE, true>(a, cp, s)
                  : launch_cl_tile_size<kModeFE, false>(a, cp, s);
    case kModeRK2a:
      return comp ? launch_cl_tile_size<kModeRK2a, true>(a, cp, s)
                  : launch_cl_tile_size<kModeRK2a, false>(a, cp, s);
    case kModeRK2b:
      return comp ? launch_cl_tile_size<kModeRK2b, true>(a, cp, s)
                  : launch_cl_tile_size<kModeRK2b, false>(a, cp, s);
    case kModeResidual: return launch_cl_tile_size<kModeResidual, false>(a, cp, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_step_scaled(int mode, const StepArgs& a, const float* s_cf, cudaStream_t s) {
  if (a.n <= 0 && mode == kModeResidual) return cudaSuccess;
  const bool comp = a.lo != nullptr;
  switch (mode) {
    case kModeFE:
      return comp ? launch_scaled_t<kModeFE, true>(a, s_cf, s)
                  : launch_scaled_t<kModeFE, false>(a, s_cf, s);
    case kModeRK2a:
      return comp ? launch_scaled_t<kModeRK2a, true>(a, s_cf, s)
                  : launch_scaled_t<kModeRK2a, false>(a, s_cf, s);
    case kModeRK2b:
      return comp ? launch_scaled_t<kModeRK2b, true>(a, s_cf, s)
                  : launch_scaled_t<kModeRK2b, false>(a, s_cf, s);
    case kModeResidual: return launch_scaled_t<kModeResidual, false>(a, s_cf, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fv
