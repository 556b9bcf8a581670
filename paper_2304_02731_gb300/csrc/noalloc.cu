// qcams_run_batch_noalloc: the integrate + analyse entry point for callers
// that must not allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs under a foreign memory
// pool or a fixed device-memory budget (where every allocation must come
// from the host application's own allocator), and callers that may not
// trigger the implicit device synchronisation a cudaMalloc can cause in the
// middle of their stream work.  qcams_run_batch creates a per-device context
// with cudaMalloc on first use; this variant instead keeps the integrator's
// scratch - the per-pair potential shape table and the work / statistics
// counters - in a fixed, file-scope device array, so it allocates nothing.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "qcams.h"
#include "qcams_device.cuh"
#include "qcams_internal.h"

namespace qcams {
namespace {

// Scratch layout: shape table for QCAMS_NOALLOC_MAX_SYS systems x 3 pairs,
// then 8 counters (0: rhs, 1: steps, 2: refill-queue head).
constexpr size_t kShapeBytes = sizeof(DevShape) * QCAMS_NOALLOC_MAX_SYS * 3;
constexpr size_t kCounterOffset = (kShapeBytes + 255) / 256 * 256;
static_assert(kCounterOffset + 8 * sizeof(unsigned long long) <= QCAMS_NOALLOC_SCRATCH_BYTES,
              "no-alloc scratch too small");
// SysSet holds QCAMS_MAX_SYS systems and the shape kernel writes n_sys * 3
// records: the no-alloc limit may not exceed the library's.
static_assert(QCAMS_NOALLOC_MAX_SYS <= QCAMS_MAX_SYS, "no-alloc system limit too large");

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[QCAMS_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the array for the current device, looked up once per
// device (host code cannot use the symbol's own address) and kept until
// qcams_shutdown on that device.
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

void noalloc_forget_device(int dev) {
  if (dev < 0 || dev >= kMaxDevices) return;
  std::lock_guard<std::mutex> lk(g_mu);
  g_scratch_ptr[dev] = nullptr;
}

}  // namespace qcams

using namespace qcams;

extern "C" int qcams_run_batch_noalloc(const qcams_system* sys, int32_t n_sys,
                                       const qcams_integ* integ, qcams_batch* batch,
                                       void* cuda_stream) {
  (void)cudaGetLastError();   // a stale error of an earlier runtime call is not ours
  if (n_sys > QCAMS_NOALLOC_MAX_SYS) return QCAMS_E_CAPACITY;
  SysSet ss;
  IntegParams ip;
  DevBatch d;
  int rc = prepare_run(sys, n_sys, integ, batch, &ss, &ip, &d);
  if (rc != QCAMS_OK) return rc;
  void* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return QCAMS_E_CUDA;
  if (batch->n == 0) return QCAMS_OK;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  Ctx scratch_ctx;   // no allocations: only the fields the integrator launch reads
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&scratch_ctx.sm_count, cudaDevAttrMultiProcessorCount, dev) !=
          cudaSuccess)
    return QCAMS_E_CUDA;
  DevShape* shapes = reinterpret_cast<DevShape*>(base);
  scratch_ctx.counters =
      reinterpret_cast<unsigned long long*>(static_cast<unsigned char*>(base) + kCounterOffset);
  // the counters start at zero on every call (launch_integrate clears them);
  // the shape table is rewritten on every call
  cudaError_t e = launch_shapes(ss, shapes, st);
  if (e == cudaSuccess)
    e = launch_integrate(ss, shapes, ip, d, integ->precision, integ->persistent, integ->block,
                         integ->blocks_per_sm, scratch_ctx, st);
  if (e != cudaSuccess) return QCAMS_E_CUDA;
  if (integ->fixed_step) return QCAMS_OK;
  e = launch_analyze(ss, shapes, ip.gb_sigma, d, st);
  return e == cudaSuccess ? QCAMS_OK : QCAMS_E_CUDA;
}
