// H.psi without any device allocation in the call.
//
// Some callers cannot call cudaMalloc while they run: code inside a
// pre-sized memory pool or arena allocator that owns the whole device
// memory, real-time or embedded loops where an allocation may stall or
// fail, and host code that must not touch the CUDA allocator after start-up.
// For them su2_apply_heff_static_scratch runs the native-FP64 H.psi with its
// intermediate T = E D^T in the fixed device array below instead of the
// environment's workspace.  The caller still passes psi in and out.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "su2_device.h"

namespace {

// Scratch for T of one term chunk: 64 MiB.  It is part of this library's
// device module, so a GPU holds it from the moment the module is loaded on it
// until the process exits (or the context is reset).  With CUDA's lazy module
// loading the load, and so the 64 MiB allocation by the driver, can happen at
// the first use on a device, i.e. inside the first call of the entry point on
// that device: a caller that must not allocate at all during its run makes
// one call at start-up.
constexpr size_t kScratchDoubles = size_t(8) << 20;
static __device__ __align__(256) double g_t_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
// per device: the array's device address, looked up once.  cudaDeviceReset
// destroys the context it belongs to; after a reset of a device the cached
// address is stale, so the library must not be used on a device after
// cudaDeviceReset in the same process.
double* g_scratch_ptr[kMaxDevices] = {};

}  // namespace

extern "C" int su2_apply_heff_static_scratch(su2_ctx* ctx, const su2_env* env, const double* psi_in_dev,
                                             double* psi_out_dev) {
  if (!ctx || !env || !psi_in_dev || !psi_out_dev) {
    if (ctx) ctx->err = "null argument";
    return SU2_EINVAL;
  }
  if (ctx->device < 0 || ctx->device >= kMaxDevices || env->ctx != ctx) {
    ctx->err = "needs a device context that owns the environment";
    return SU2_EINVAL;
  }
  if ((uintptr_t(psi_in_dev) | uintptr_t(psi_out_dev)) & 7) {
    ctx->err = "psi pointers must be 8-byte aligned";
    return SU2_EINVAL;
  }
  const int64_t n = env->psi_len;
  if (psi_in_dev < psi_out_dev + n && psi_out_dev < psi_in_dev + n) {
    ctx->err = "psi_in and psi_out overlap";
    return SU2_EINVAL;
  }
  if (env->t_elems > int64_t(kScratchDoubles)) {
    ctx->err = "a term chunk needs " + std::to_string(env->t_elems * 8) + " bytes of T, the static scratch holds " +
               std::to_string(kScratchDoubles * 8) + "; build the environment with t_budget_bytes <= " +
               std::to_string(kScratchDoubles * 8);
    return SU2_EINVAL;
  }
  if (env->os.on) {
    ctx->err = "the static-scratch entry point takes environments whose operators are all on the device";
    return SU2_EINVAL;
  }
  if (cudaSetDevice(ctx->device) != cudaSuccess) {
    ctx->err = "cudaSetDevice failed";
    return SU2_ECUDA;
  }
  double* scratch = nullptr;
  {
    // once per device, with that device current: the device address of the
    // array (its name in host code is only a host-side stand-in)
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_scratch_ptr[ctx->device]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_t_scratch);
      if (e != cudaSuccess || !p) {
        ctx->err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
        return SU2_ECUDA;
      }
      g_scratch_ptr[ctx->device] = static_cast<double*>(p);
    }
    scratch = g_scratch_ptr[ctx->device];
  }
  // F is the output and starts at zero; nothing in the scratch needs clearing:
  // K1 writes every element of T that K2 then reads.
  if (cudaMemsetAsync(psi_out_dev, 0, size_t(n) * sizeof(double), ctx->stream) != cudaSuccess) {
    ctx->err = "cudaMemsetAsync failed";
    return SU2_ECUDA;
  }
  su2::Profiler off;  // no event recording on this path
  for (const su2::Chunk& c : env->chunks)
    su2::launch_heff_fp64(ctx->stream, env->dL, env->dR, psi_in_dev, psi_out_dev, scratch, env->dk1, env->dk2,
                          env->dk2t, c, n, &off);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    ctx->err = std::string("launch: ") + cudaGetErrorString(e);
    return SU2_ECUDA;
  }
  return SU2_OK;
}
