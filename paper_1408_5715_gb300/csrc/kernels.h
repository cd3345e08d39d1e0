// kernels.h -- launch interface between the C ABI (capi.cu) and the device
// kernels (kernels.cu).  Plain structs of device pointers; no torch types.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace fv {

constexpr int kBlock = 256;        // threads per block of the cell kernels
constexpr int kTotalsBlocks = 1024; // fixed grid of the deterministic totals

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
  const int4* nbr;    // {nbr0, nbr1, nbr2, unused}; negative = -FV_BC_* ghost
  const void* geom;   // 8 values per cell: n0x n0y n1x n1y n2x n2y 1/V 2V/P
  int64_t n;
  double uinf[4];     // far-field conserved state
  const unsigned long long* bmin_read;
  unsigned long long* bmin_write;
  unsigned long long* bmin_reset;
  const double* t_read;
  double* t_write;
  double cfl;         // > 0: CFL number; < 0: fixed dt = -cfl
  double t_stop;      // > 0: clamp the time advanced in this loop
  int* err;
  // FP32 compensated update: per cell, four bfloat16 remainders (8 bytes)
  // that carry what the float state could not hold; read and rewritten in
  // place by the cell's own thread.  nullptr = plain float update.
  uint2* lo;
  // RK2 with lo: remainder of the stage state U* (written by the first stage,
  // read by the second).
  uint2* lo_stage;
};

// float (FV_F32) or double (FV_F64) instantiations
cudaError_t launch_step(bool f64, int mode, const StepArgs& a, cudaStream_t s);
cudaError_t launch_init_scalars(LoopScalars* d, cudaStream_t s);
cudaError_t launch_bound(bool f64, const void* U, const void* geom, int64_t n,
                         unsigned long long* bmin, int* err, cudaStream_t s);
cudaError_t launch_totals(bool f64, const void* U, const double* vol, int64_t n,
                          double* partials /*[kTotalsBlocks*4]*/, double* out /*[4]*/,
                          cudaStream_t s);
// *bmin = +inf bits, *flag = 0 (flag nullable)
cudaError_t launch_reset_min(unsigned long long* bmin, int* flag, cudaStream_t s);
cudaError_t launch_dt_from_bound(const unsigned long long* bmin, double cfl, double* dt_out,
                                 cudaStream_t s);

}  // namespace fv
