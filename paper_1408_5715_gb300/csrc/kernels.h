// kernels.h -- launch interface between the C ABI (capi.cu) and the device
// kernels (kernels.cu).  Plain structs of device pointers; no torch types.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace fv {

constexpr int kBlock = 256;        // threads per block of the cell kernels
constexpr int kTotalsBlocks = 1024; // fixed grid of the deterministic totals

// Wave speed of the Lax-Friedrichs dissipation (StepArgs::wave).
constexpr int kWaveAverage = 0;  // interface averages (Sec. 6.2.2, the default)
constexpr int kWaveMax = 1;      // larger one-sided speed (Rusanov)

// Step modes of the fused cell kernel.
enum StepMode : int {
  kModeFE = 0,       // U^{n+1} = U^n + dt R(U^n), plus the next-dt bound
  kModeRK2a = 1,     // U*      = U^n + dt R(U^n)
  kModeRK2b = 2,     // U^{n+1} = U^n/2 + (U* + dt R(U*))/2, plus the next-dt bound
  kModeResidual = 3  // R(U) = -(1/V) sum_f F_f
};

// Device-side scalars of a time loop.  bmin holds minima of the per-cell
// bound 2V/(P(|v|+c)) as the bit patterns of positive doubles (so that an
// unsigned 64-bit atomicMin orders them); three slots rotate so a step can
// read one, fill the next and clear the one after.
struct LoopScalars {
  unsigned long long bmin[3];
  double t[2];
  int err;
  int pad;
  double totals[4];
  double dt_out;
  unsigned long long aux_bmin;  // minimum of fv_compute_dt, apart from the loop's
  int aux_err;
  int pad2;
};

// Arguments of the fused step kernel (precision-independent view; the
// pointers are float or double records according to the launch).
struct StepArgs {
  const void* U;      // state whose fluxes are evaluated (neighbours and own cell)
  const void* Ubase;  // RK2 second stage: U^n of the own cell (may equal out)
  void* out;          // new state, or the residual in kModeResidual
  // Neighbours (negative = -FV_BC_* ghost) and geometry, by precision:
  //   FP64: nbr int4 (nbr0, nbr1, nbr2, -); geom 8 doubles n0x n0y n1x n1y n2x n2y 1/V 2V/P
  //   FP32: nbr int2 (nbr1, nbr2); geom 8 floats n0x n0y n1x n1y n2x n2y 1/V nbr0-bits
  const void* nbr;
  const void* geom;
  int64_t n;
  double uinf[4];     // far-field conserved state
  float uinf_f[4];    // the same rounded to float (FP32 kernels convert nothing)
  const unsigned long long* bmin_read;
  unsigned long long* bmin_write;
  unsigned long long* bmin_reset;
  const double* t_read;
  double* t_write;
  double cfl;         // > 0: CFL number; < 0: fixed dt = -cfl
  double t_stop;      // > 0: clamp the time advanced in this loop
  int* err;
  // FP32 compensated update: per cell, four bfloat16 values (8 bytes) holding
  // what the float state could not; read and rewritten in place by the cell's
  // own thread.  nullptr = plain float update.
  uint2* lo;
  // RK2 with lo: remainder of the stage state U* (written by the first stage,
  // read by the second).
  uint2* lo_stage;
  // Bounded waits of the TMA-staged variant: polls of an mbarrier before a
  // wait gives up (error bit 2), and polls allowed to drain copies in flight.
  unsigned wait_limit;
  unsigned drain_limit;
  // Tiles of the shared-memory variant (6): tile-local neighbours per cell,
  // per-tile halo offsets and ids (tiles.cpp), cells per tile, and the
  // capacity of a tile plus its first halo.
  const uint2* cell_ln;
  const int* tile_info;
  const int* halo_id;
  int tile;
  int t1_cap;
  // shape 7: each tile's faces evaluated once (tiles.cpp face_off / face_rec)
  const int* tile_face_off;
  const uint2* tile_face;
  // Vertex geometry of the tile variant (FP32; vertex_geom.cpp), or nullptr:
  // normals formed from grid coordinates of the tile's nodes and 1/V read
  // from inv_vol instead of the geom records.  tile_vq[2 tile_voff[b] ..]
  // are tile b's nodes (int32 x, y); a cell's nodes are tile-local ids
  // cell_ln[i].y >> 16 and the two halves of cell_vl[i]; v_cap is the most
  // nodes of a tile.  Normal = grid edge rotated, times vscale = 2^e.
  const unsigned* cell_vl;
  const int* tile_voff;
  const int2* tile_vq;
  const float* inv_vol;
  int v_cap;
  float vscale;
  // launch as part of a programmatic chain (launch_util.cuh)
  bool chained;
  // kWaveAverage or kWaveMax (shapes 0, 1 and 6; the others run shape 1)
  int wave;
};

// Arguments of the batched step kernel: many meshes concatenated into one
// cell range, each padded to a multiple of kBlock cells.
struct BatchArgs {
  StepArgs s;               // arrays over the whole range (n = padded total)
  const int* block_mesh;    // [n / kBlock] mesh of each block
  const int64_t* mesh_end;  // [n_meshes] one past the last real cell of each mesh
  const double* uinf;       // [4 * n_meshes] far-field conserved states
  const float* uinf_f;      // [4 * n_meshes] the same rounded to float
  unsigned long long* bmin; // [3 * n_meshes] CFL minima, slot-major
  double* t;                // [2 * n_meshes] time advanced, slot-major
  int n_meshes;
  int slot_read, slot_write, slot_reset;
  int t_read, t_write;
  // tiles of the shared-memory shape (6): per tile its mesh, first cell and
  // cell count; per mesh its first tile.  The tile-local neighbours, halo
  // offsets and ids and the capacity are in s (cell_ln, tile_info, halo_id,
  // t1_cap; s.tile = the largest tile).
  const int* tile_mesh;
  const int64_t* tile_start;
  const int* tile_cells;
  const int* mesh_first_tile;
  int n_tiles;
};

// Learned dissipation scale (closure.cu): MLP 8 -> 32 -> 32 -> 1 with
// bfloat16 hidden-layer weights.  Flat parameter order of theta (FP32, 1377
// values): W1[32][8], b1[32], W2[32][32], b2[32], w3[32], b3.
constexpr int kClosureParams = 32 * 8 + 32 + 32 * 32 + 32 + 32 + 1;

struct ClosureParams {
  const unsigned* w1;  // [32][4]: bfloat16 pairs (W1[n][2c], W1[n][2c+1])
  const unsigned* w2;  // [32][16]: bfloat16 pairs (W2[n][2c], W2[n][2c+1])
  const float* b1;     // [32]
  const float* b2;     // [32]
  const float* w3;     // [32]
  float b3;
  bool tc;             // MLP on tcgen05 (else mma.sync): same bits
};

cudaError_t launch_closure_eval(const float* feats, float* s_out, int64_t rows,
                                const ClosureParams& cp, cudaStream_t s);
// The scales of a face list (each face once, both cells' slots s_cf[3c + k]
// written) and the step that reads them (FP32; persistent one thread per cell).
// A face record: a = 4 c + k (cell c, its face k), b = 4 m + km for the cell
// m across (its face km) or a ghost code < 0, and face k's normal of cell c
// (times the face length) in FP32, as in the cell's geometry record.
struct __align__(16) FaceRec {
  int a, b;
  float nx, ny;
};
cudaError_t launch_face_scales(const StepArgs& a, const FaceRec* faces, int64_t nf,
                               const ClosureParams& cp, float* s_cf, cudaStream_t s);
cudaError_t launch_step_scaled(int mode, const StepArgs& a, const float* s_cf, cudaStream_t s);
// The learned step on tiles with each face once (shape 7's tiles and face
// lists; FP32; tiles of up to 1024 cells)
size_t closure_tile_smem_bytes(int t1_cap, int tile, bool tc);
cudaError_t launch_step_closure_tile(int mode, const StepArgs& a, const ClosureParams& cp,
                                     cudaStream_t s);
// Blocks the gradient kernel launches at most on this device.
int closure_grad_blocks();
// One-step loss and gradient; gpart [max_blocks * kClosureParams], lpart
// [max_blocks] scratch; grad [kClosureParams] and loss [1] device outputs.
cudaError_t launch_closure_grad(const StepArgs& a, const float* Ut, double dt, const double* w,
                                const ClosureParams& cp, float* gpart, double* lpart,
                                int max_blocks, float* grad, double* loss, cudaStream_t s);
cudaError_t launch_adam(float* theta, const float* grad, float* m, float* v, int n, double lr,
                        double b1, double b2, double eps, int64_t step, cudaStream_t s);
// theta (device, FP32, kClosureParams) -> w1, w2 (bfloat16 pairs), b (b1 b2 w3 b3)
cudaError_t launch_pack_closure(const float* theta, unsigned* w1, unsigned* w2, float* b,
                                cudaStream_t s);

// Shape variants of the step kernel (see k_step): 0 one thread per cell,
// 1 persistent grid with next-cell prefetch, 2 the same capped at 64
// registers, 3 and 4 one thread per cell capped at 40 and 32 registers,
// 5 persistent grid with TMA-staged cell records (tma_step.cu), 6 tiles with
// their first halo ring and primitives in shared memory (tile_step.cu).
constexpr int kStepVariants = 8;
constexpr int kTileVariant = 6;
constexpr int kFaceTileVariant = 7;
// shared memory of the tile variant: state and primitives of tile + halo
inline size_t tile_smem_bytes(bool f64, int t1_cap, int v_cap = 0) {
  return (size_t)t1_cap * 2 * (f64 ? 32 : 16) + (size_t)v_cap * 8;
}
cudaError_t launch_restrict_mean(bool fine_f64, bool coarse_f64, const void* Uf, const double* area,
                                 const int* fine_of, int64_t n_coarse, int kids, void* Uc,
                                 cudaStream_t s);
cudaError_t launch_step_tile(bool f64, int mode, const StepArgs& a, cudaStream_t s);
// shape 7: the tile shape with each face evaluated once (its states and
// primitives as shape 6, plus three face-flux records per tile cell)
inline size_t tile_faces_smem_bytes(bool f64, int t1_cap, int tile) {
  return tile_smem_bytes(f64, t1_cap) + (size_t)3 * tile * (f64 ? 32 : 16);
}
cudaError_t launch_step_tile_faces(bool f64, int mode, const StepArgs& a, cudaStream_t s);
cudaError_t launch_batch_step_tile(bool f64, int mode, const BatchArgs& b, cudaStream_t s);
// Library-owned per-cell arrays are allocated in whole tiles of this many
// cells (the TMA-staged variant copies whole tiles of them).
constexpr int64_t kPadCells = 256;
constexpr unsigned kDefaultWaitLimit = 1u << 24;

cudaError_t launch_step_tma(bool f64, int mode, const StepArgs& a, cudaStream_t s);
// the same for a batch (tiles = the batch's 256-cell blocks); needs the
// batch's library arrays padded to whole tiles, as fv_batch allocates them
cudaError_t launch_batch_step_tma(bool f64, int mode, const BatchArgs& b, cudaStream_t s);

// Two forward-Euler steps per launch on tiles staged in shared memory
// (pair_step.cu).  FP32 state; dt of both steps from the slots as for one
// step (CFL bound of the state at the start of the pair, or fixed).
struct PairArgs {
  const float4* U;        // state at the start of the pair (read only)
  float4* out;            // state after the pair
  const uint2* lo_in;     // compensated update: remainders at the start ...
  uint2* lo_out;          // ... and after the pair (both nullptr: plain update)
  const float4* geom;     // FP32 geometry, 2 records per cell
  const uint2* cell_ln;   // per cell: tile-local neighbours (16 bits each)
  const int* tile_info;   // [2 (n_tiles + 1)] halo offset, first-halo size
  const int* halo_id;     // global ids of the halos
  const uint2* halo_ln;   // tile-local neighbours of first-halo entries
  int64_t n;
  int tile;               // cells per tile
  int e_cap, t1_cap;      // shared-memory capacities (cells)
  float uinf[4];          // far-field conserved state, rounded to float
  const unsigned long long* bmin_read;
  unsigned long long* bmin_write;
  unsigned long long* bmin_reset;
  const double* t_read;
  double* t_write;
  double cfl, t_stop;
  int* err;
  // staged kernel: bounded mbarrier waits (error bit 2 when one gives up)
  unsigned wait_limit, drain_limit;
  bool chained;  // launch as part of a programmatic chain (launch_util.cuh)
};
// tile sizes with a kernel instantiation (the staged kernel: 512 and 1024)
constexpr int kPairTiles[4] = {512, 768, 1024, 2048};
// The one-step tile shape takes any tile size from 1 to this many cells.
constexpr int kMaxTileCells = 2048;
// dynamic shared memory of one block for the given capacities (the states
// only, 16 bytes a cell); the staged kernel adds two stages of the tile's own
// records (64 bytes a cell each)
inline size_t pair_smem_bytes(int e_cap, int t1_cap, int tile, bool staged) {
  return (size_t)(e_cap + t1_cap) * 16 + (staged ? (size_t)2 * 64 * tile : 0);
}
// staged: 0 loads through the caches; 1 persistent blocks whose tile records
// arrive by bulk copies (cp.async.bulk) into double-buffered stages
cudaError_t launch_step_pair(const PairArgs& a, int staged, cudaStream_t s);

// float (FV_F32) or double (FV_F64) instantiations
cudaError_t launch_step(bool f64, int mode, int variant, const StepArgs& a, cudaStream_t s);
cudaError_t launch_init_scalars(LoopScalars* d, cudaStream_t s);
cudaError_t launch_bound(bool f64, const void* U, const void* geom, int64_t n,
                         unsigned long long* bmin, int* err, cudaStream_t s);
cudaError_t launch_totals(bool f64, const void* U, const double* vol, int64_t n,
                          double* partials /*[kTotalsBlocks*4]*/, double* out /*[4]*/,
                          cudaStream_t s);
cudaError_t launch_batch_step(bool f64, int mode, const BatchArgs& b, int64_t n_blocks,
                              cudaStream_t s);
cudaError_t launch_batch_init(unsigned long long* bmin, double* t, int n_meshes, int* err,
                              cudaStream_t s);
cudaError_t launch_batch_bound(bool f64, const void* U, const void* geom, const int* block_mesh,
                               const int64_t* mesh_end, int n_meshes, int64_t n_blocks,
                               unsigned long long* bmin, int* err, cudaStream_t s);
cudaError_t launch_batch_totals(bool f64, const void* U, const double* vol, const int* block_mesh,
                                const int64_t* mesh_end, const int* mesh_first_block,
                                int n_meshes, int64_t n_blocks, double* partials, double* out,
                                cudaStream_t s);
// *bmin = +inf bits, *flag = 0 (flag nullable)
cudaError_t launch_reset_min(unsigned long long* bmin, int* flag, cudaStream_t s);
cudaError_t launch_dt_from_bound(const unsigned long long* bmin, double cfl, double* dt_out,
                                 cudaStream_t s);

}  // namespace fv
