// No-allocation variant of the 2D FP64 RVE batch solve (declared in include/fehmm.h as
// fehmm_rve2d_solve_fp64_noalloc; the paper has no counterpart).
//
// Some callers cannot call cudaMalloc: code that runs inside an allocator-free runtime
// (a host that hands the library only pre-registered buffers), code paths that must not
// allocate while a memory pool is being torn down or resized, and callers that need a
// predictable footprint fixed at load time.  For them this entry point uses no dynamic
// device memory at all: the per-block scratch the FP64 kernel needs (staged element
// tangents and the assembled stencil) and its work counter live in file-scope
// `static __device__` arrays of a fixed maximum size.  Every GPU on which the library is
// loaded holds that memory (kNoallocScratchBytes, about 22 MB) until the process exits.
//
// In host code the arrays' names are host-side stand-ins, not device addresses, so the
// set-up below asks the runtime for the real device addresses once per device, with that
// device current, and the kernel receives them as ordinary pointers.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "fehmm.h"
#include "fehmm_device.cuh"
#include "rve_args.h"

namespace fehmm {
namespace {

constexpr int kNoallocMaxNN = 256;      // grid_n <= 16
constexpr int kNoallocMaxBlocks = 152;  // one block per SM on a GB300, at most
constexpr size_t kNoallocScratchDoubles = (size_t)kNoallocMaxBlocks * 72 * kNoallocMaxNN;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kNoallocScratchDoubles];
static __device__ __align__(256) int32_t g_noalloc_queue[4];

struct DeviceSlots {
  double* scratch = nullptr;
  int32_t* queue = nullptr;
  int num_sms = 0;
};
DeviceSlots g_slots[kMaxDevices];
std::mutex g_mutex;

// Device addresses of the static arrays on the current device (set up on first use).
int device_slots(DeviceSlots* out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return FEHMM_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_mutex);
  DeviceSlots& s = g_slots[dev];
  if (!s.scratch) {
    void* scr = nullptr;
    void* q = nullptr;
    int sms = 0;
    if (cudaGetSymbolAddress(&scr, g_noalloc_scratch) != cudaSuccess ||
        cudaGetSymbolAddress(&q, g_noalloc_queue) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      return FEHMM_ERR_CUDA;
    }
    s.scratch = static_cast<double*>(scr);
    s.queue = static_cast<int32_t*>(q);
    s.num_sms = sms;
  }
  *out = s;
  return FEHMM_OK;
}

}  // namespace
}  // namespace fehmm

using namespace fehmm;

extern "C" int fehmm_rve2d_solve_fp64_noalloc(int n_qp, int grid_n, int phase_per_qp, const uint8_t* phase,
                                              const double* lame, double* w, const double* F, double* P,
                                              double* A, int32_t* status, int32_t* iters,
                                              const fehmm_options* opt, void* stream) {
  if (!opt || opt->dim != 2 || opt->precision != FEHMM_PREC_FP64) return FEHMM_ERR_ARG;
  if (n_qp <= 0 || !phase || !lame || !w || !F || !P || !status) return FEHMM_ERR_ARG;
  if (grid_n < 2 || (grid_n % 2) != 0) return FEHMM_ERR_ARG;
  if (grid_n * grid_n > kNoallocMaxNN) return FEHMM_ERR_TOO_LARGE;
  if (!(opt->cg_rtol > 0) || !(opt->cond_rtol > 0) || opt->max_cg <= 0 || opt->max_cond_cg <= 0 ||
      opt->max_newton < 0 || opt->retry_stages < 0 || opt->retry_stages > 64 ||
      (opt->bc != FEHMM_BC_PERIODIC && opt->bc != FEHMM_BC_KUBC))
    return FEHMM_ERR_ARG;
  if (opt->law != FEHMM_LAW_NEO_HOOKE) return FEHMM_ERR_UNSUPPORTED;  // one law in the static variant
  DeviceSlots slots;
  int rc = device_slots(&slots);
  if (rc != FEHMM_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  Rve2dArgs a{};
  a.n_qp = n_qp;
  a.nn_max = grid_n * grid_n;
  a.fixed_n = grid_n;
  a.phase_per_qp = phase_per_qp ? 1 : 0;
  a.phase = phase;
  a.rve_lame = lame;
  a.w_in = w;
  a.w_out = w;
  a.F = F;
  a.P = P;
  a.A = A;
  a.W = nullptr;
  a.status = status;
  a.iters = iters;
  a.queue = slots.queue;
  a.scratch = slots.scratch;
  a.newton_rtol = opt->newton_rtol;
  a.newton_atol = opt->newton_atol;
  a.cg_rtol = opt->cg_rtol;
  a.cond_rtol = opt->cond_rtol;
  a.max_newton = opt->max_newton;
  a.max_cg = opt->max_cg;
  a.max_cond_cg = opt->max_cond_cg;
  a.retry_stages = opt->retry_stages;
  a.mg = 0;  // block-Jacobi: the static scratch holds no multigrid levels
  a.bc = opt->bc == FEHMM_BC_KUBC ? 1 : 0;
  a.law = 0;
  a.mg_omega = 0.7f;
  a.mg_reuse = 0;
  a.X_in = nullptr;  // no kept transfer solutions: every transfer solve starts from zero
  a.X_out = nullptr;
  a.scratch_stride = 72LL * a.nn_max;
  a.flags = A ? 0 : kFlagNoTangent;
  // the shared work counter keeps the previous call's value: clear it on this stream
  // (a failed call is reported as FEHMM_ERR_CUDA with the runtime's last-error state
  // cleared, so that the caller's next CUDA call does not see it)
  if (cudaMemsetAsync(slots.queue, 0, sizeof(int32_t), s) != cudaSuccess) {
    cudaGetLastError();
    return FEHMM_ERR_CUDA;
  }
  const int blocks = std::min(std::min(n_qp, slots.num_sms), kNoallocMaxBlocks);
  if (rve2d_launch_fixed_fp64(a, blocks, s) != cudaSuccess) {
    cudaGetLastError();
    return FEHMM_ERR_CUDA;
  }
  return FEHMM_OK;
}
