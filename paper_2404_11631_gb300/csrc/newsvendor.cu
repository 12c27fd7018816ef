// newsvendor.cu -- saa_newsvendor_grad: the newsvendor's Monte Carlo
// gradient (Sec. 3.2, the approximated gradient), per product j and decision
// vector x_k:  k_j - v_j + (h_j + v_j) * (1/S) #{s : d_js <= x_kj},
// with S normal demand samples d_js = mu_j + sigma_j z_js per product.
//
// z_js are the in-kernel generator's FP32 normals on the demand tag
// (counter (s / 4, j, epoch, tag 3 | instance)); the indicator is decided on
// the standardised demand in FP32, z_js <= tau_kj = RN_f32((x_kj - mu_j) /
// sigma_j) with the subtraction and division in FP64, so the counts are
// exact integers.  There is no contraction: the work is the generator plus a
// compare and an add per sample and decision.
//
// Work units are (product, chunk of samples); a thread counts its chunk
// against every decision's threshold in registers and adds the counts to
// [K][n] with integer atomics (the sum does not depend on their order).  A
// second kernel forms the estimate in FP64.
#include <cuda_runtime.h>

#include "gen.cuh"
#include "internal.cuh"

namespace saa {
namespace {

constexpr int kNvMaxK = 8;
constexpr int kNvThreads = 256;

struct NvArgs {
  uint32_t n, S, chunks, sc;   // products, samples, chunks per product, samples per chunk (multiple of 4)
  uint64_t seed;
  uint32_t instance, epoch;
  const double* mu;
  const double* sigma;
  int K;
  const double* X;     // [K][n]
  uint32_t* counts;    // [K][n]
  uint32_t* err;
};

// KT = a.K rounded up to 1, 2, 4 or 8: the compare-and-count of every
// sample is unrolled over KT thresholds (padding thresholds count nothing).
template <int KT>
__global__ void __launch_bounds__(kNvThreads) k_nv_count(NvArgs a) {
  const uint64_t units = (uint64_t)a.n * a.chunks;
  const gen::Stream st = gen::make_stream(a.seed, a.epoch, a.instance);
  for (uint64_t u = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; u < units;
       u += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t j = (uint32_t)(u / a.chunks), c = (uint32_t)(u % a.chunks);
    const double mu = a.mu[j], sg = a.sigma[j];
    if (!(sg > 0.0)) {
      atomicOr(a.err, kErrInput);
      continue;
    }
    float tau[KT];
    uint32_t cnt[KT];
#pragma unroll
    for (int k = 0; k < KT; ++k) {
      tau[k] = (k < a.K) ? __double2float_rn(__ddiv_rn(__dsub_rn(a.X[(size_t)k * a.n + j], mu), sg)) : 0.0f;
      cnt[k] = 0u;
    }
    const uint32_t s0 = c * a.sc, s1 = min(a.S, s0 + a.sc);
    for (uint32_t s = s0; s < s1; s += 4) {
      const uint4 x = gen::philox(st, s >> 2, j, gen::kTagDemand);
      float z[4];
      gen::box_muller_f(x.x, x.y, &z[0], &z[1]);
      gen::box_muller_f(x.z, x.w, &z[2], &z[3]);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (s + q < s1) {
#pragma unroll
          for (int k = 0; k < KT; ++k) cnt[k] += (z[q] <= tau[k]) ? 1u : 0u;
        }
      }
    }
#pragma unroll
    for (int k = 0; k < KT; ++k)
      if (k < a.K && cnt[k]) atomicAdd(&a.counts[(size_t)k * a.n + j], cnt[k]);
  }
}

// grad_kj = (k_j - v_j) + (h_j + v_j) * (count_kj / S), FP64, in that order.
__global__ void k_nv_grad(uint32_t n, uint32_t S, int K, const double* __restrict__ kc,
                          const double* __restrict__ hc, const double* __restrict__ vc,
                          const uint32_t* __restrict__ counts, double* __restrict__ grad) {
  const uint64_t total = (uint64_t)K * n;
  for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < total;
       e += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t j = (uint32_t)(e % n);
    const double frac = __ddiv_rn((double)counts[e], (double)S);
    grad[e] = __dadd_rn(__dsub_rn(kc[j], vc[j]), __dmul_rn(__dadd_rn(hc[j], vc[j]), frac));
  }
}

saa_status nv_check(const saa_newsvendor* p, int32_t K) {
  if (!p) {
    set_error("saa_newsvendor: problem is NULL");
    return SAA_EINVAL;
  }
  if (p->n < 1 || p->n > 0xffffffffll || p->S < 1 || p->S > 0x3fffffffll) {
    set_error("saa_newsvendor: need 1 <= n < 2^32 products and 1 <= S < 2^30 samples");
    return SAA_EINVAL;
  }
  if (K < 1 || K > kNvMaxK) {
    set_error("saa_newsvendor: need 1 <= K <= 8 decision vectors");
    return SAA_EINVAL;
  }
  if (!p->mu || !p->sigma || !p->k || !p->h || !p->v) {
    set_error("saa_newsvendor: mu, sigma, k, h, v must be device pointers");
    return SAA_EINVAL;
  }
  return SAA_OK;
}

}  // namespace
}  // namespace saa

using namespace saa;

extern "C" size_t saa_newsvendor_workspace_size(const saa_newsvendor* prob, int32_t K) {
  if (nv_check(prob, K) != SAA_OK) return 0;
  return sizeof(uint32_t) * (size_t)K * (size_t)prob->n;
}

extern "C" saa_status saa_newsvendor_grad(saa_ctx* ctx, const saa_newsvendor* prob, int32_t K, const double* X,
                                          double* grad, void* ws, size_t ws_bytes, void* stream) {
  saa::NvtxRange nvtx_range("saa_newsvendor_grad");
  if (!ctx) {
    set_error("saa_newsvendor: ctx is NULL");
    return SAA_EINVAL;
  }
  saa_status s = nv_check(prob, K);
  if (s != SAA_OK) return s;
  if (!X || !grad || !ws) {
    set_error("saa_newsvendor: X, grad and ws must be device pointers");
    return SAA_EINVAL;
  }
  const size_t need = sizeof(uint32_t) * (size_t)K * (size_t)prob->n;
  if (ws_bytes < need || (((uintptr_t)ws) & 3u)) {
    set_error("saa_newsvendor: workspace smaller than saa_newsvendor_workspace_size() or misaligned");
    return SAA_ENOMEM;
  }
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != ctx->device && cudaSetDevice(ctx->device) != cudaSuccess) {
    set_error("saa_newsvendor: cudaSetDevice failed");
    return SAA_ECUDA;
  }
  NvArgs a;
  a.n = (uint32_t)prob->n;
  a.S = (uint32_t)prob->S;
  // enough (product, chunk) units to fill the GPU, chunks of at least 64 samples
  const uint64_t resident = (uint64_t)ctx->sm_count * 8 * kNvThreads;
  const uint64_t want_units = resident;
  uint64_t chunks = (want_units + a.n - 1) / a.n;
  const uint64_t max_chunks = ((uint64_t)a.S + 63) / 64;
  if (chunks > max_chunks) chunks = max_chunks;
  if (chunks < 1) chunks = 1;
  uint32_t sc = (uint32_t)(((uint64_t)a.S + chunks - 1) / chunks);
  sc = (sc + 3u) & ~3u;
  a.sc = sc;
  a.chunks = (uint32_t)(((uint64_t)a.S + sc - 1) / sc);
  a.seed = prob->seed;
  a.instance = prob->instance;
  a.epoch = prob->epoch;
  a.mu = prob->mu;
  a.sigma = prob->sigma;
  a.K = K;
  a.X = X;
  a.counts = (uint32_t*)ws;
  a.err = ctx->err;
  cudaStream_t st = (cudaStream_t)stream;
  s = cuda_status(cudaMemsetAsync(ws, 0, need, st), "saa_newsvendor: clear counts");
  if (s == SAA_OK) {
    const uint64_t units = (uint64_t)a.n * a.chunks;
    const uint64_t blocks = (units + kNvThreads - 1) / kNvThreads;
    const unsigned grid = (unsigned)(blocks < (uint64_t)ctx->sm_count * 32 ? blocks : (uint64_t)ctx->sm_count * 32);
    if (K == 1)
      k_nv_count<1><<<grid, kNvThreads, 0, st>>>(a);
    else if (K == 2)
      k_nv_count<2><<<grid, kNvThreads, 0, st>>>(a);
    else if (K <= 4)
      k_nv_count<4><<<grid, kNvThreads, 0, st>>>(a);
    else
      k_nv_count<8><<<grid, kNvThreads, 0, st>>>(a);
    const uint64_t total = (uint64_t)K * a.n;
    const uint64_t gb = (total + 255) / 256;
    k_nv_grad<<<(unsigned)(gb < 65535ull * 8 ? gb : 65535ull * 8), 256, 0, st>>>(a.n, a.S, K, prob->k, prob->h,
                                                                                  prob->v, a.counts, grad);
    ctx->kernels += 2;
    s = cuda_status(cudaGetLastError(), "saa_newsvendor: launch");
  }
  if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
  return s;
}
