// tc.cu -- tcgen05 tensor-core path (BF16 hi/lo split contraction).
#include <cuda_runtime.h>

#include "internal.cuh"

namespace saa {

bool tc_supported(const saa_problem* p, int K, int want_grad) {
  (void)p; (void)K; (void)want_grad;
  return false;
}

saa_status tc_plan(const saa_ctx* ctx, const saa_problem* p, int K, Plan* plan) {
  (void)ctx; (void)p; (void)K; (void)plan;
  return SAA_EUNSUPPORTED;
}

cudaError_t launch_tc(const LawArgs& la, int K, const Plan& plan, const Workspace& ws, uint32_t* err,
                      cudaStream_t st) {
  (void)la; (void)K; (void)plan; (void)ws; (void)err; (void)st;
  return cudaErrorNotSupported;
}

}  // namespace saa
