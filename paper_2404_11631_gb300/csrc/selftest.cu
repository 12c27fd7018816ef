// selftest.cu -- exhaustive device check of the generator's shortened
// arithmetic: for every FP32 uniform u = (2k + 1) 2^-24, k < 2^23, the LOG
// quotient (m - 1)/(m + 1) by Markstein's correction against the IEEE
// round-to-nearest division, and the Box-Muller root sqrt(-2 LOG(u)) against
// the IEEE square root.  Counts of differing results go to a device array.
#include <cuda_runtime.h>

#include "gen.cuh"
#include "internal.cuh"

namespace saa {
namespace {

__global__ void k_selftest_arith(unsigned long long* bad) {
  unsigned long long nd = 0, ns = 0;
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < (1u << 23); k += gridDim.x * blockDim.x) {
    const float u = gen::unif24(k << 9);
    float m = __uint_as_float((__float_as_uint(u) & 0x007fffffu) | 0x3f800000u);
    if (m > 0x1.6a09e6p+0f) m = __fmul_rn(m, 0.5f);
    const float a = __fsub_rn(m, 1.0f), b = __fadd_rn(m, 1.0f);
    nd += __float_as_uint(gen::div_rn_gen(a, b)) != __float_as_uint(__fdiv_rn(a, b));
    const float x = __fmul_rn(-2.0f, gen::logf_own<false>(u));
    ns += __float_as_uint(gen::sqrt_rn_gen(x)) != __float_as_uint(__fsqrt_rn(x));
  }
  if (nd) atomicAdd(&bad[0], nd);
  if (ns) atomicAdd(&bad[1], ns);
}

}  // namespace
}  // namespace saa

using namespace saa;

extern "C" saa_status saa_selftest_arith(saa_ctx* ctx, unsigned long long* mismatches, void* stream) {
  if (!ctx || !mismatches) {
    set_error("saa_selftest_arith: ctx and mismatches must be non-NULL");
    return SAA_EINVAL;
  }
  if (cudaSetDevice(ctx->device) != cudaSuccess) {
    set_error("saa_selftest_arith: cudaSetDevice failed");
    return SAA_ECUDA;
  }
  const cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(mismatches, 0, 2 * sizeof(unsigned long long), st);
  if (e == cudaSuccess) {
    k_selftest_arith<<<4 * ctx->sm_count, 256, 0, st>>>(mismatches);
    e = cudaGetLastError();
  }
  return cuda_status(e, "saa_selftest_arith launch");
}
