// Internal host-side interface between the C-ABI layer (api.cu) and the
// kernel translation units.
#pragma once

#include <cuda_runtime.h>

#include "qcams_device.cuh"

namespace qcams {

// Library-owned per-device scratch (created lazily, freed by qcams_shutdown).
struct Ctx {
  int device = -1;
  int sm_count = 0;
  DevShape* shapes = nullptr;          // [QCAMS_MAX_SYS][3]
  DevLevel* levels = nullptr;          // [kLevelCells]
  uint8_t* level_flag = nullptr;       // [kLevelCells] levels to solve in this call
  uint8_t* level_valid = nullptr;      // [kLevelCells] levels[] holds a solved level
  // per system slot: the AB-pair parameters and masses the cached levels
  // were solved for (levels depend on nothing else)
  double level_key[QCAMS_MAX_SYS][9] = {};
  bool level_key_set[QCAMS_MAX_SYS] = {};
  unsigned long long* counters = nullptr;  // [8]: 0 rhs, 1 steps, 2 queue head
  qcams_level* req_out = nullptr;      // [65536] qcams_levels output staging
  int32_t* req_in = nullptr;           // [3 * 65536] qcams_levels input staging
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};  // integrate / analyze timing
  bool timed = false;                  // ev[] hold a completed qcams_run_batch
};

struct IntegParams {
  double rtol, atol, r_stop2, t_stop, h_fixed;
  double gb_sigma;       // Gaussian-binning width of the product analysis
  long long max_steps;
  int fixed_step;
  float rtol_f, atol_f;  // error-norm constants in FP32
};

// Diagnostic: the integrator's table-driven exponential and CUDA's exp on n
// device arguments (integrate.cu; used by the accuracy test).
cudaError_t launch_exp_check(const double* x, double* mine, double* ref, long long n,
                             cudaStream_t st);

// Diagnostic: the integrator's pair-force 1/sqrt(s), exponent argument and
// exponential for one Morse pair (integrate.cu; used by the accuracy test).
cudaError_t launch_force_math_check(const double* s, double c0, double c1, double* ri,
                                    double* x, double* e, long long n, cudaStream_t st);

// Diagnostic: the integrator's float-float dot product (integrate.cu).
cudaError_t launch_ff_dot_check(const double* a, const double* w, int m, double* out,
                               float* out_f, long long n, cudaStream_t st);

// Validation and launch helpers defined in api.cu.
int prepare_run(const qcams_system* sys, int32_t n_sys, const qcams_integ* integ,
                const qcams_batch* batch, SysSet* ss, IntegParams* ip, DevBatch* d);
cudaError_t launch_shapes(const SysSet& ss, DevShape* shapes, cudaStream_t st);
cudaError_t launch_analyze(const SysSet& ss, const DevShape* shapes, double gb_sigma,
                           const DevBatch& d, cudaStream_t st);

// Launch the integrator over the batch (integrate.cu).
cudaError_t launch_integrate(const SysSet& sys, const DevShape* shapes, const IntegParams& ip,
                             const DevBatch& b, int precision, int persistent, int block,
                             int blocks_per_sm, Ctx& ctx, cudaStream_t st);

// FP64 integrator for small batches, `lanes` = 3 or 6 lanes per trajectory
// (integrate_grp.cu).
cudaError_t launch_integrate_grouped(const SysSet& sys, const DevShape* shapes,
                                     const IntegParams& ip, const DevBatch& b, int lanes,
                                     unsigned long long* counters, cudaStream_t st,
                                     bool all_morse);

// Registers per thread and resident blocks per SM of the lane-group kernel.
cudaError_t grouped_func_info(int lanes, bool all_morse, int* regs, int* blocks_per_sm);

// FP32 integrator with compensated state updates (integrate32.cu).
cudaError_t launch_integrate32(const SysSet& sys, const DevShape* shapes, const IntegParams& ip,
                               const DevBatch& b, int persistent, Ctx& ctx, cudaStream_t st,
                               bool all_morse);

// Drop the no-allocation entry point's cached scratch address for a device
// (noalloc.cu); qcams_shutdown calls it.
void noalloc_forget_device(int dev);

// Launch-shape variants of the integrator (integrate.cu), for the autotuner.
int integrate_variant_count();
void integrate_variant_shape(int v, int* block, int* blocks_per_sm);
bool integrate_shape_supported(int block, int blocks_per_sm);
cudaError_t integrate_variant_regs(int v, bool morse, int* regs);
cudaError_t integrate_variant_occupancy(int v, bool morse, int* blocks_per_sm);
bool integrate_all_morse(const SysSet& sys);

}  // namespace qcams
