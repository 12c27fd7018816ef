// noalloc.cu -- saa_eval_static: the value estimate of saa_eval for callers
// that cannot allocate device memory.
//
// saa_eval needs a caller-provided workspace and a context, and creating a
// context calls cudaMalloc.  Some callers cannot do either: real-time loops
// that cannot afford cudaMalloc's implicit device synchronisation, plug-ins
// inside a host framework that owns all device memory through its own
// allocator, and code running under a device-memory budget that another
// component enforces.  For them this entry point takes its scratch from one
// fixed array in device memory that the library defines at file scope.
// Every GPU that loads the library holds that array
// (SAA_STATIC_SCRATCH_BYTES) until the process exits.
//
// The scratch is shared by every call in the process: two calls whose work
// overlaps on the GPU (different streams, or different host threads) race
// on it and give wrong results.  Its first 256 bytes hold this path's
// device error word, which each call clears (cudaMemsetAsync) before its
// prologue checks C's diagonal; a call whose check fires writes NaN to its
// outputs.  The rest needs no clearing: the sample kernel writes each
// per-CTA partial on its first tile and the finalize kernels overwrite the
// totals, so the contents left by the last call are never read.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "internal.cuh"

namespace saa {

namespace {

static __device__ __align__(256) unsigned char g_static_scratch[SAA_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_dev[kMaxDevices];   // device address of g_static_scratch, per device

// Device address of the scratch array on the current device, looked up once
// per device (the name g_static_scratch is only a host-side stand-in).
saa_status scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("saa_eval_static: device ordinal out of range");
    return SAA_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return cuda_status(e, "saa_eval_static: cudaGetSymbolAddress(scratch)");
    g_scratch_dev[dev] = p;
  }
  *out = g_scratch_dev[dev];
  return SAA_OK;
}

// A call whose prologue flagged C's diagonal (not positive, or not finite)
// gives NaN outputs: this path has no context whose error word a later
// saa_ctx_sync could read.
__global__ void k_static_flag_out(const uint32_t* err, int K, double* f, double* pbar, double* var) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K || *err == 0u) return;
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  f[k] = nan;
  if (pbar) pbar[k] = nan;
  if (var) var[k] = nan;
}

constexpr size_t kErrBytes = 256;   // the error word's slot at the start of the scratch

}  // namespace
}  // namespace saa

using namespace saa;

extern "C" saa_status saa_eval_static(const saa_problem* prob, int32_t K, const double* X, saa_prec prec, double* f,
                                      double* pbar, double* var, void* stream) {
  saa::NvtxRange nvtx_range("saa_eval_static");
  if (!prob || prob->d < 1 || prob->N < 2 || prob->N > 0xffffffffll || prob->law < SAA_LAW_GAUSS ||
      prob->law > SAA_LAW_MIX || (prob->law == SAA_LAW_STUDENT_T && (prob->nu < 2 || (prob->nu & 1) || prob->nu > 64)) ||
      prob->reserved != 0 || !prob->mu || (!prob->chol && !prob->sd)) {
    set_error("saa_eval_static: invalid problem (see saa_eval for the rules)");
    return SAA_EINVAL;
  }
  if (!prob->chol) {
    set_error("saa_eval_static: the diagonal form (chol NULL, sd given) needs saa_eval and a workspace");
    return SAA_EUNSUPPORTED;
  }
  if (K < 1 || K > 65535 || !X || !f) {
    set_error("saa_eval_static: need 1 <= K <= 65535 and non-NULL X, f");
    return SAA_EINVAL;
  }
  if (prec != SAA_FP32 && prec != SAA_FP64) {
    set_error("saa_eval_static: only SAA_FP32 and SAA_FP64 are available without a workspace");
    return SAA_EUNSUPPORTED;
  }
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e, "saa_eval_static: cudaGetDevice");
  void* scratch = nullptr;
  saa_status s = scratch_address(dev, &scratch);
  if (s != SAA_OK) return s;

  // A context on the stack: device limits only, no device memory.
  saa_ctx c;
  std::memset(&c, 0, sizeof(c));
  c.device = dev;
  e = cudaDeviceGetAttribute(&c.sm_count, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return cuda_status(e, "saa_eval_static: cudaDeviceGetAttribute");

  Plan plan;
  s = make_plan(&c, prob, K, prec, 0, &plan);
  if (s != SAA_OK) return s;
  Workspace ws;
  uint32_t* err = (uint32_t*)scratch;
  const size_t need = carve(prob, K, plan, 0, (char*)scratch + kErrBytes, &ws);
  if (need > (size_t)SAA_STATIC_SCRATCH_BYTES - kErrBytes) {
    set_error("saa_eval_static: this d and K need " + std::to_string(need) + " bytes of scratch, more than the " +
              std::to_string((size_t)SAA_STATIC_SCRATCH_BYTES - kErrBytes) +
              " bytes the static array has for them; use saa_eval");
    return SAA_ENOMEM;
  }
  LawArgs la;
  la.d = prob->d;
  la.law = prob->law;
  la.nu = prob->nu;
  la.N = (uint32_t)prob->N;
  la.seed = prob->seed;
  la.instance = prob->instance;
  la.epoch = prob->epoch;
  la.t_dev = nullptr;
  la.M = 1;
  cudaStream_t st = (cudaStream_t)stream;
  s = cuda_status(cudaMemsetAsync(err, 0, sizeof(uint32_t), st), "saa_eval_static: clear the error word");
  if (s != SAA_OK) return s;
  s = cuda_status(launch_prologue(prob, K, X, prec, ws, err, st), "saa_eval_static: prologue launch");
  if (s != SAA_OK) return s;
  s = cuda_status(launch_simt(la, K, prec, 0, plan, ws, st), "saa_eval_static: sample kernel launch");
  if (s != SAA_OK) return s;
  s = cuda_status(launch_finalize(prob, K, prec, 0, plan, ws, f, pbar, var, nullptr, st),
                  "saa_eval_static: finalize launch");
  if (s != SAA_OK) return s;
  k_static_flag_out<<<(K + 255) / 256, 256, 0, st>>>(err, K, f, pbar, var);
  return cuda_status(cudaGetLastError(), "saa_eval_static: input-check launch");
}
