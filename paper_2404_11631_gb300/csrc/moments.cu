// moments.cu -- saa_generate_moments: per-dimension sums of the innovations
// zhat_ij and of their squares over a scenario range, drawn by the same
// in-kernel generator as every estimator kernel (the samples of Sec. 3.1).
//
// It serves two purposes.  It checks the generator's law on the device at
// scales no host can reach (the standardised laws have mean 0 and variance
// 1 per coordinate).  It is also the generator-only kernel whose instruction
// count per normal (generation plus one add and one fma) is the per-unit
// figure of the ALU roofline.
//
// Layout: a row of nbp threads covers the dimension blocks of one scenario
// (block b = 4 dimensions in FP32 mode, 2 in FP64 mode); the CTA's rows walk
// the scenario range with a fixed stride.  Each thread keeps running sums in
// the mode's precision, the CTA folds its rows in row order into FP64
// partials [grid][d], and a second kernel adds the partials in CTA order,
// so the result is deterministic for a given device.
#include <cuda_runtime.h>

#include "gen.cuh"
#include "internal.cuh"

namespace saa {
namespace {

constexpr int kMomThreads = 256;
constexpr int kMomMaxDim = 2048;

template <typename T>
__global__ void __launch_bounds__(kMomThreads) k_gen_moments(LawArgs la, int64_t i0, int64_t n, int nbp,
                                                             double* __restrict__ part1, double* __restrict__ part2) {
  constexpr int PC = gen::Gen<T>::kPerCall;
  extern __shared__ double msm[];   // [rows][d] sums, then [rows][d] sums of squares
  const int d = la.d;
  const int nb = (d + PC - 1) / PC;
  const int rows = kMomThreads / nbp;
  const int row = threadIdx.x / nbp, bcol = threadIdx.x % nbp;
  double* m1 = msm;
  double* m2 = msm + (size_t)rows * d;
  const gen::Stream st = gen::make_stream(la.seed, la.epoch, la.instance);
  const uint32_t half = la.N / 2u;
  const uint32_t step = (uint32_t)gridDim.x * (uint32_t)rows;
  for (int b = bcol; b < nb; b += nbp) {
    T a1[PC], a2[PC];
#pragma unroll
    for (int q = 0; q < PC; ++q) a1[q] = a2[q] = T(0);
    for (uint32_t r = (uint32_t)blockIdx.x * (uint32_t)rows + (uint32_t)row; (int64_t)r < n; r += step) {
      const uint32_t i = (uint32_t)i0 + r;
      T z[PC];
      gen::Gen<T>::block(st, (uint32_t)b, i, gen::is_lognormal(la.law, i, half), z);
#pragma unroll
      for (int q = 0; q < PC; ++q) {
        a1[q] += z[q];
        a2[q] = fma(z[q], z[q], a2[q]);
      }
    }
#pragma unroll
    for (int q = 0; q < PC; ++q) {
      const int j = b * PC + q;
      if (j < d) {
        m1[(size_t)row * d + j] = (double)a1[q];
        m2[(size_t)row * d + j] = (double)a2[q];
      }
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < d; j += blockDim.x) {
    double t1 = 0.0, t2 = 0.0;
    for (int w = 0; w < rows; ++w) {
      t1 += m1[(size_t)w * d + j];
      t2 += m2[(size_t)w * d + j];
    }
    part1[(size_t)blockIdx.x * d + j] = t1;
    part2[(size_t)blockIdx.x * d + j] = t2;
  }
}

__device__ __forceinline__ void neumaier_add(double& s, double& c, double x) {
  const double t = s + x;
  if (fabs(s) >= fabs(x))
    c += (s - t) + x;
  else
    c += (x - t) + s;
  s = t;
}

// One block per 32 dimensions: warp w adds CTAs w, w + 8, ... and the eight
// warp sums are merged in warp order (deterministic).
__global__ void __launch_bounds__(256) k_moments_final(int grid, int d, const double* __restrict__ part1,
                                                       const double* __restrict__ part2, double* __restrict__ sum,
                                                       double* __restrict__ sumsq) {
  __shared__ double sh[4][8][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = blockIdx.x * 32 + lane;
  double s1 = 0.0, c1 = 0.0, s2 = 0.0, c2 = 0.0;
  if (j < d)
    for (int g = warp; g < grid; g += 8) {
      neumaier_add(s1, c1, part1[(size_t)g * d + j]);
      neumaier_add(s2, c2, part2[(size_t)g * d + j]);
    }
  sh[0][warp][lane] = s1;
  sh[1][warp][lane] = c1;
  sh[2][warp][lane] = s2;
  sh[3][warp][lane] = c2;
  __syncthreads();
  if (warp == 0 && j < d) {
    double t1 = 0.0, e1 = 0.0, t2 = 0.0, e2 = 0.0;
    for (int w = 0; w < 8; ++w) {
      neumaier_add(t1, e1, sh[0][w][lane]);
      neumaier_add(t1, e1, sh[1][w][lane]);
      neumaier_add(t2, e2, sh[2][w][lane]);
      neumaier_add(t2, e2, sh[3][w][lane]);
    }
    sum[j] = t1 + e1;
    if (sumsq) sumsq[j] = t2 + e2;
  }
}

struct MomPlan {
  int nbp, rows, grid;
  size_t smem, ws;
};

MomPlan mom_plan(const saa_ctx* ctx, int d, int64_t n, int prec) {
  const int PC = (prec == SAA_FP64) ? 2 : 4;
  const int nb = (d + PC - 1) / PC;
  MomPlan p;
  p.nbp = 1;
  while (p.nbp < nb && p.nbp < kMomThreads) p.nbp <<= 1;
  p.rows = kMomThreads / p.nbp;
  const int64_t want = (n + p.rows - 1) / p.rows;
  const int64_t cap = 4 * (int64_t)ctx->sm_count;
  p.grid = (int)(want < 1 ? 1 : want < cap ? want : cap);
  p.smem = sizeof(double) * 2 * (size_t)p.rows * d;
  p.ws = sizeof(double) * 2 * (size_t)p.grid * d;
  return p;
}

saa_status check_args(const saa_ctx* ctx, const saa_problem* prob, int64_t i0, int64_t n, saa_prec prec) {
  if (!ctx || !prob) {
    set_error("saa_generate_moments: ctx and prob must be non-NULL");
    return SAA_EINVAL;
  }
  if (prob->d < 1 || prob->d > kMomMaxDim || prob->N < 2 || prob->N > 0xffffffffll || prob->law < SAA_LAW_GAUSS ||
      prob->law > SAA_LAW_MIX) {
    set_error("saa_generate_moments: need 1 <= d <= 2048, 2 <= N < 2^32 and a known law");
    return SAA_EINVAL;
  }
  if (prec != SAA_FP32 && prec != SAA_FP64) {
    set_error("saa_generate_moments: takes SAA_FP32 or SAA_FP64");
    return SAA_EINVAL;
  }
  if (i0 < 0 || n < 1 || i0 + n > prob->N) {
    set_error("saa_generate_moments: scenario range outside [0, N)");
    return SAA_EINVAL;
  }
  return SAA_OK;
}

}  // namespace
}  // namespace saa

using namespace saa;

extern "C" size_t saa_generate_moments_workspace_size(const saa_ctx* ctx, const saa_problem* prob, int64_t i0,
                                                      int64_t n, saa_prec prec) {
  if (check_args(ctx, prob, i0, n, prec) != SAA_OK) return 0;
  return mom_plan(ctx, prob->d, n, prec).ws;
}

extern "C" saa_status saa_generate_moments(saa_ctx* ctx, const saa_problem* prob, int64_t i0, int64_t n,
                                           saa_prec prec, double* sum, double* sumsq, void* ws, size_t ws_bytes,
                                           void* stream) {
  saa::NvtxRange nvtx_range("saa_generate_moments");
  saa_status s = check_args(ctx, prob, i0, n, prec);
  if (s != SAA_OK) return s;
  if (!sum || !ws) {
    set_error("saa_generate_moments: sum and ws must be device pointers");
    return SAA_EINVAL;
  }
  const MomPlan p = mom_plan(ctx, prob->d, n, prec);
  if (ws_bytes < p.ws || (((uintptr_t)ws) & 7u)) {
    set_error("saa_generate_moments: workspace smaller than saa_generate_moments_workspace_size() or misaligned");
    return SAA_ENOMEM;
  }
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != ctx->device && cudaSetDevice(ctx->device) != cudaSuccess) {
    set_error("saa_generate_moments: cudaSetDevice failed");
    return SAA_ECUDA;
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
  double* part1 = (double*)ws;
  double* part2 = part1 + (size_t)p.grid * prob->d;
  cudaStream_t st = (cudaStream_t)stream;
  if (prec == SAA_FP64)
    k_gen_moments<double><<<p.grid, kMomThreads, p.smem, st>>>(la, i0, n, p.nbp, part1, part2);
  else
    k_gen_moments<float><<<p.grid, kMomThreads, p.smem, st>>>(la, i0, n, p.nbp, part1, part2);
  k_moments_final<<<(prob->d + 31) / 32, 256, 0, st>>>(p.grid, prob->d, part1, part2, sum, sumsq);
  ctx->kernels += 2;
  s = cuda_status(cudaGetLastError(), "saa_generate_moments: launch");
  if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
  return s;
}
