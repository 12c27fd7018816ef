// large_d.cu -- the estimator of Eq. 4 / Eq. 5 and its gradient for a
// diagonal covariance, Sigma = diag(sd^2) (the asset setup of Sec. 4.1), at
// any dimension: Sec. 4.1 runs 500 to 100000 assets, where a dense factor C
// no longer fits (80 GB at d = 10^5) and the sample tile of the CUDA-core
// kernels no longer fits shared memory.
//
// With C = diag(sd): w'R_i = c + s_i zhat_i'y, c = mu'w, y = sd o w.  Per
// call (FP32 normals, the generator of every other path, bit-exact):
//   forward  tiles of 8 scenarios, one warp each; the decisions y are
//            staged through shared memory 8192 / K dimensions at a time, so
//            a tile reads y once; lanes draw 4-dimension blocks and add each
//            block's FP32 dot product into a float-float sum; Q_ik = s_i
//            (sum) and s_i go to HBM, S1 and S2 to the CTA's FP64 partials;
//            with the sample store on, every normal is written out too.
//   adjoint  (gradient only) one thread per 4-dimension block over a slice
//            of the scenarios keeps Kahan-compensated FP32 sums of a_ij Q_ik
//            (G) and a_ij (m~), written per slice in FP64.  It takes its
//            normals from the sample store, [N][round_up(d, 4)] FP32 that the
//            forward pass wrote (26 GB at d = 10^5, N = 2^16: the write
//            hides under the generator's ALU time and the read is a plain
//            HBM stream), or, when the store is off or too small, draws its
//            block again (nothing of size N x d in memory).  Both give the
//            same bits.
//   finalize S1, S2 and the slices added in fixed order (FP64), then p_bar,
//            V, f_hat and grad = sd o [lambda 2/(N-1) (G - S1 m) - m] - mu.
// Every sum has a fixed order: results are bitwise deterministic.
#include <cuda_runtime.h>

#include <cstring>

#include "gen.cuh"
#include "internal.cuh"

namespace saa {
namespace {

constexpr int kLdThreads = 256;
constexpr int kLdWarps = kLdThreads / 32;
constexpr int kLdSPW = 1;                       // scenarios per warp in a forward tile
constexpr int kLdTile = kLdWarps * kLdSPW;     // 8 scenarios per forward tile (fine-grained rounds)
constexpr int kLdChunkFloats = 8192;            // y staged per pass: 8192 / K dimensions (32 KB)
constexpr int kLdMaxK = 4;

__device__ __forceinline__ void ld_ff_add(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bp = s - hi;
  lo += (hi - (s - bp)) + (x - bp);
  hi = s;
}

// y_kj = sd_j x_kj (FP32 copy for the contraction); c_k = mu'x_k (FP64, one
// block per decision, fixed-order tree).
__global__ void __launch_bounds__(kLdThreads) k_ld_prologue(int d, int K, const double* __restrict__ X,
                                                            const double* __restrict__ mu,
                                                            const double* __restrict__ sd, float* __restrict__ y,
                                                            double* __restrict__ c, uint32_t* __restrict__ err) {
  __shared__ double red[kLdWarps];
  const int k = blockIdx.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < d; j += gridDim.x * blockDim.x) {
    const double s = sd[j];
    if (k == 0 && (!(s > 0.0) || !isfinite(s))) atomicOr(err, kErrInput);
    y[(size_t)k * d + j] = (float)(s * X[(size_t)k * d + j]);
  }
  if (blockIdx.x != 0) return;
  double t = 0.0;
  for (int j = threadIdx.x; j < d; j += blockDim.x) t = fma(mu[j], X[(size_t)k * d + j], t);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if (lane == 0) red[warp] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double u = 0.0;
    for (int w = 0; w < kLdWarps; ++w) u += red[w];
    c[k] = u;
  }
}

template <int KT>
__global__ void __launch_bounds__(kLdThreads) k_ld_fwd(LawArgs la, int K, const float* __restrict__ y,
                                                       float* __restrict__ Q, float* __restrict__ S,
                                                       double* __restrict__ part_s1, double* __restrict__ part_s2,
                                                       int64_t tiles, float* __restrict__ zs, int dp) {
  constexpr int kLdChunk = kLdChunkFloats / KT;
  __shared__ __align__(16) float ys[KT][kLdChunk];
  __shared__ double red[kLdWarps][2][KT];
  const int d = la.d;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t epoch = la.epoch;
  if (la.t_dev) epoch += (uint32_t)(*la.t_dev / la.M);
  const gen::Stream st = gen::make_stream(la.seed, epoch, la.instance);
  const uint32_t half = la.N / 2u;
  double s1[KT], s2[KT];   // this warp's sums over its scenarios (FP64)
#pragma unroll
  for (int k = 0; k < KT; ++k) s1[k] = s2[k] = 0.0;
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    float hi[kLdSPW][KT], lo[kLdSPW][KT];
#pragma unroll
    for (int q = 0; q < kLdSPW; ++q)
#pragma unroll
      for (int k = 0; k < KT; ++k) hi[q][k] = lo[q][k] = 0.0f;
    const int64_t i_base = tile * kLdTile + warp * kLdSPW;
    for (int j0 = 0; j0 < d; j0 += kLdChunk) {
      const int dc = min(kLdChunk, d - j0);
      __syncthreads();   // the previous chunk is consumed
      for (int e = threadIdx.x; e < KT * kLdChunk; e += blockDim.x) {
        const int k = e / kLdChunk, j = e % kLdChunk;
        ys[k][j] = (k < K && j < dc) ? y[(size_t)k * d + j0 + j] : 0.0f;
      }
      __syncthreads();
      const int nbc = (dc + 3) / 4;   // 4-dimension blocks of the chunk
#pragma unroll
      for (int q = 0; q < kLdSPW; ++q) {
        const int64_t i = i_base + q;
        if (i >= (int64_t)la.N) break;   // warp-uniform
        const bool logn = gen::is_lognormal(la.law, (uint32_t)i, half);
        for (int bc = lane; bc < nbc; bc += 32) {
          float z[4];
          gen::Gen<float>::block(st, (uint32_t)((j0 >> 2) + bc), (uint32_t)i, logn, z);
          if (4 * bc + 4 > dc) {   // the chunk's ragged tail (ys is zero there too)
#pragma unroll
            for (int e = 0; e < 4; ++e)
              if (4 * bc + e >= dc) z[e] = 0.0f;
          }
          if (zs)   // the sample store: row i, dimensions j0 + 4 bc .. + 3 (< dp, 16-byte aligned)
            __stcs(reinterpret_cast<float4*>(zs + (size_t)i * dp + j0 + 4 * bc), make_float4(z[0], z[1], z[2], z[3]));
          // the block's 4-term FP32 dot product, then one float-float add: the
          // error stays at the FP32 rounding of each block's partial
#pragma unroll
          for (int k = 0; k < KT; ++k) {
            const float4 yv = *reinterpret_cast<const float4*>(&ys[k][4 * bc]);   // one 16-byte shared load
            float p = z[0] * yv.x;
            p = fmaf(z[1], yv.y, p);
            p = fmaf(z[2], yv.z, p);
            p = fmaf(z[3], yv.w, p);
            ld_ff_add(hi[q][k], lo[q][k], p);
          }
        }
      }
    }
    // per scenario: warp sum (float-float tree), the t-law scale, Q and S1/S2
#pragma unroll
    for (int q = 0; q < kLdSPW; ++q) {
      const int64_t i = i_base + q;
#pragma unroll
      for (int k = 0; k < KT; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const float oh = __shfl_xor_sync(0xffffffffu, hi[q][k], o);
          const float ol = __shfl_xor_sync(0xffffffffu, lo[q][k], o);
          ld_ff_add(hi[q][k], lo[q][k], oh);
          lo[q][k] += ol;
        }
      }
      if (i < (int64_t)la.N) {
        const float s = gen::Gen<float>::scale(st, (uint32_t)i, la.law, la.nu);
        if (lane == 0 && S) S[i] = s;
#pragma unroll
        for (int k = 0; k < KT; ++k) {
          if (k < K) {
            const double qv = (double)s * ((double)hi[q][k] + (double)lo[q][k]);
            if (lane == 0) Q[(size_t)i * K + k] = (float)qv;
            s1[k] += qv;
            s2[k] = fma(qv, qv, s2[k]);
          }
        }
      }
    }
  }
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < KT; ++k) {
      red[warp][0][k] = s1[k];
      red[warp][1][k] = s2[k];
    }
  }
  __syncthreads();
  if (threadIdx.x < K) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < kLdWarps; ++w) {
      a += red[w][0][threadIdx.x];
      b += red[w][1][threadIdx.x];
    }
    part_s1[(size_t)blockIdx.x * K + threadIdx.x] = a;
    part_s2[(size_t)blockIdx.x * K + threadIdx.x] = b;
  }
}

// Adjoint accumulation of one scenario into a thread's 4-dimension block:
// a = s_i zhat_ij; m~_j += a and G_kj += a Q_ik, Kahan-compensated (the
// compensation carries the lost low part).  Both adjoint kernels use it, so
// the stored and the redrawn samples give the same bits.
template <int KT>
__device__ __forceinline__ void ld_adj_add(const float z[4], float s, const float qk[KT], float ms[4], float mc[4],
                                           float gs[KT][4], float gc[KT][4]) {
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const float a = z[e] * s;
    {
      const float yv = a - mc[e];
      const float t = ms[e] + yv;
      mc[e] = (t - ms[e]) - yv;
      ms[e] = t;
    }
#pragma unroll
    for (int k = 0; k < KT; ++k) {
      const float yv = a * qk[k] - gc[k][e];
      const float t = gs[k][e] + yv;
      gc[k][e] = (t - gs[k][e]) - yv;
      gs[k][e] = t;
    }
  }
}

// The slice's sums of block b to part_m [slice][d] and part_g [slice][K][d].
template <int KT>
__device__ __forceinline__ void ld_adj_write(int b, int d, int K, int sl, const float ms[4], const float mc[4],
                                             const float gs[KT][4], const float gc[KT][4], double* part_g,
                                             double* part_m) {
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int j = 4 * b + e;
    if (j < d) {
      part_m[(size_t)sl * d + j] = (double)ms[e] - (double)mc[e];
#pragma unroll
      for (int k = 0; k < KT; ++k)
        if (k < K) part_g[((size_t)sl * K + k) * d + j] = (double)gs[k][e] - (double)gc[k][e];
    }
  }
}

// Adjoint drawing its samples again: thread t of block (x, slice) owns the
// 4-dimension block b = 256 x + t over the slice's scenarios.
template <int KT>
__global__ void __launch_bounds__(kLdThreads) k_ld_adj(LawArgs la, int K, int64_t per_slice,
                                                       const float* __restrict__ Q, const float* __restrict__ S,
                                                       double* __restrict__ part_g, double* __restrict__ part_m) {
  const int d = la.d;
  const int nb = (d + 3) / 4;
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  const int sl = blockIdx.y;
  uint32_t epoch = la.epoch;
  if (la.t_dev) epoch += (uint32_t)(*la.t_dev / la.M);
  const gen::Stream st = gen::make_stream(la.seed, epoch, la.instance);
  const uint32_t half = la.N / 2u;
  const bool tlaw = la.law == SAA_LAW_STUDENT_T;
  const int64_t i0 = (int64_t)sl * per_slice;
  const int64_t i1 = min((int64_t)la.N, i0 + per_slice);
  float gs[KT][4], gc[KT][4], ms[4], mc[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    ms[e] = mc[e] = 0.0f;
#pragma unroll
    for (int k = 0; k < KT; ++k) gs[k][e] = gc[k][e] = 0.0f;
  }
  if (b >= nb) return;
  for (int64_t i = i0; i < i1; ++i) {
    float z[4];
    gen::Gen<float>::block(st, (uint32_t)b, (uint32_t)i, gen::is_lognormal(la.law, (uint32_t)i, half), z);
    float qk[KT];
#pragma unroll
    for (int k = 0; k < KT; ++k) qk[k] = k < K ? Q[(size_t)i * K + k] : 0.0f;
    ld_adj_add<KT>(z, tlaw ? S[i] : 1.0f, qk, ms, mc, gs, gc);
  }
  ld_adj_write<KT>(b, d, K, sl, ms, mc, gs, gc, part_g, part_m);
}

// Adjoint reading the sample store: the same sums from zs [N][dp], four
// scenarios' loads issued ahead of their arithmetic (an HBM stream).
template <int KT>
__global__ void __launch_bounds__(kLdThreads) k_ld_adj_kept(LawArgs la, int K, int64_t per_slice,
                                                            const float* __restrict__ zs, int dp,
                                                            const float* __restrict__ Q, const float* __restrict__ S,
                                                            double* __restrict__ part_g,
                                                            double* __restrict__ part_m) {
  constexpr int U = 4;
  const int d = la.d;
  const int nb = (d + 3) / 4;
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  const int sl = blockIdx.y;
  const bool tlaw = la.law == SAA_LAW_STUDENT_T;
  const int64_t i0 = (int64_t)sl * per_slice;
  const int64_t i1 = min((int64_t)la.N, i0 + per_slice);
  float gs[KT][4], gc[KT][4], ms[4], mc[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    ms[e] = mc[e] = 0.0f;
#pragma unroll
    for (int k = 0; k < KT; ++k) gs[k][e] = gc[k][e] = 0.0f;
  }
  if (b >= nb) return;
  const float* col = zs + 4 * (size_t)b;
  int64_t i = i0;
  for (; i + U <= i1; i += U) {
    float4 zz[U];
    float sv[U], qk[U][KT];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      zz[u] = __ldcs(reinterpret_cast<const float4*>(col + (size_t)(i + u) * dp));
      sv[u] = tlaw ? __ldg(S + i + u) : 1.0f;
#pragma unroll
      for (int k = 0; k < KT; ++k) qk[u][k] = k < K ? __ldg(Q + (size_t)(i + u) * K + k) : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const float z[4] = {zz[u].x, zz[u].y, zz[u].z, zz[u].w};
      ld_adj_add<KT>(z, sv[u], qk[u], ms, mc, gs, gc);
    }
  }
  for (; i < i1; ++i) {
    const float4 v = __ldcs(reinterpret_cast<const float4*>(col + (size_t)i * dp));
    const float z[4] = {v.x, v.y, v.z, v.w};
    float qk[KT];
#pragma unroll
    for (int k = 0; k < KT; ++k) qk[k] = k < K ? __ldg(Q + (size_t)i * K + k) : 0.0f;
    ld_adj_add<KT>(z, tlaw ? __ldg(S + i) : 1.0f, qk, ms, mc, gs, gc);
  }
  ld_adj_write<KT>(b, d, K, sl, ms, mc, gs, gc, part_g, part_m);
}

// One warp per decision: S1, S2 over the forward CTAs (lane-strided, fixed
// tree), then p_bar, V and f_hat; S1 is kept for the gradient.
__global__ void k_ld_value_out(int grid, int K, double N, double lambda, const double* __restrict__ part_s1,
                               const double* __restrict__ part_s2, const double* __restrict__ c,
                               double* __restrict__ tot_s1, double* __restrict__ f, double* __restrict__ pbar,
                               double* __restrict__ var) {
  const int k = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (k >= K) return;
  double a = 0.0, b = 0.0;
  for (int g = lane; g < grid; g += 32) {
    a += part_s1[(size_t)g * K + k];
    b += part_s2[(size_t)g * K + k];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if (lane == 0) {
    tot_s1[k] = a;
    const double qbar = a / N;
    const double pb = c[k] + qbar;
    const double V = (b - a * qbar) / (N - 1.0);
    if (f) f[k] = lambda * V - pb;
    if (pbar) pbar[k] = pb;
    if (var) var[k] = V;
  }
}

// grad_kj = sd_j [lambda 2/(N-1) (G_kj - S1_k m_j) - m_j] - mu_j, m = m~/N,
// the slices added in order.
__global__ void k_ld_grad_out(int nsl, int K, int d, double N, double lambda, const double* __restrict__ part_g,
                              const double* __restrict__ part_m, const double* __restrict__ tot_s1,
                              const double* __restrict__ sd, const double* __restrict__ mu,
                              double* __restrict__ grad) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)K * d) return;
  const int k = (int)(e / d), j = (int)(e % d);
  double G = 0.0, m = 0.0;
  for (int sl = 0; sl < nsl; ++sl) {
    G += part_g[((size_t)sl * K + k) * d + j];
    m += part_m[(size_t)sl * d + j];
  }
  m /= N;
  const double u = lambda * 2.0 / (N - 1.0) * (G - tot_s1[k] * m) - m;
  grad[e] = sd[j] * u - mu[j];
}

template <int KT>
cudaError_t launch_ld_kt(const LawArgs& la, int K, int want_grad, const Plan& plan, const Workspace& w,
                         cudaStream_t st) {
  const int dp = (la.d + 3) & ~3;
  float* zs = (want_grad && plan.keep) ? w.zs : nullptr;
  k_ld_fwd<KT><<<plan.grid, kLdThreads, 0, st>>>(la, K, (const float*)w.Y, w.q_dev, w.s_dev, w.part_s1, w.part_s2,
                                                 plan.tiles, zs, dp);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !want_grad) return e;
  const int64_t per = (la.N + plan.nsplit - 1) / plan.nsplit;
  const dim3 ag((unsigned)plan.ablk, (unsigned)plan.nsplit);
  if (zs)
    k_ld_adj_kept<KT><<<ag, kLdThreads, 0, st>>>(la, K, per, zs, dp, w.q_dev, w.s_dev, w.part_gd, w.part_md);
  else
    k_ld_adj<KT><<<ag, kLdThreads, 0, st>>>(la, K, per, w.q_dev, w.s_dev, w.part_gd, w.part_md);
  return cudaGetLastError();
}

// Resident CTAs per SM of the forward (which = 0) or adjoint (1, from the
// store when kept) kernel for K decisions; 2 if the query fails.
int ld_occupancy(int which, int K, int kept) {
  int occ = 0;
  cudaError_t e;
  const int kt = K == 1 ? 1 : K == 2 ? 2 : 4;
  if (which == 0)
    e = kt == 1 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_ld_fwd<1>, kLdThreads, 0)
      : kt == 2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_ld_fwd<2>, kLdThreads, 0)
                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_ld_fwd<4>, kLdThreads, 0);
  else if (kept)
    e = kt == 1 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_ld_adj_kept<1>, kLdThreads, 0)
      : kt == 2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_ld_adj_kept<2>, kLdThreads, 0)
                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_ld_adj_kept<4>, kLdThreads, 0);
  else
    e = kt == 1 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_ld_adj<1>, kLdThreads, 0)
      : kt == 2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_ld_adj<2>, kLdThreads, 0)
                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_ld_adj<4>, kLdThreads, 0);
  if (e != cudaSuccess || occ < 1) {
    cudaGetLastError();
    return 2;
  }
  return occ;
}

}  // namespace

saa_status diag_plan(const saa_ctx* ctx, const saa_problem* p, int K, saa_prec prec, int want_grad, Plan* plan) {
  if (prec != SAA_FP32) {
    set_error("diagonal covariance (chol NULL, sd given): SAA_FP32 only");
    return SAA_EUNSUPPORTED;
  }
  if (K > kLdMaxK) {
    set_error("diagonal covariance path: K <= 4 decisions per call");
    return SAA_EUNSUPPORTED;
  }
  plan->prec = prec;
  plan->diag = 1;
  // forward: as many CTAs as fit on the SMs at once (the tiles are small,
  // so the last round is a small part of the work)
  plan->tiles = (p->N + kLdTile - 1) / kLdTile;
  const int64_t cap = (int64_t)ld_occupancy(0, K, 0) * ctx->sm_count;
  plan->grid = (int)(plan->tiles < cap ? plan->tiles : cap);
  const int nb = (p->d + 3) / 4;
  plan->ablk = (nb + kLdThreads - 1) / kLdThreads;
  if (want_grad) {
    const size_t store = (size_t)p->N * (size_t)((p->d + 3) & ~3) * sizeof(float);
    plan->keep = store <= ctx->store_cap;
    // adjoint: scenario slices for one full wave of CTAs (all equal work),
    // each slice at least 256 scenarios
    const int64_t slots = (int64_t)ld_occupancy(1, K, plan->keep) * ctx->sm_count;
    int64_t ns = slots / plan->ablk;
    const int64_t most = (p->N + 255) / 256;
    if (ns > most) ns = most;
    plan->nsplit = (int)(ns < 1 ? 1 : ns);
  }
  return SAA_OK;
}

size_t diag_carve(const saa_problem* p, int K, const Plan& plan, int want_grad, void* base, Workspace* ws) {
  const size_t d = (size_t)p->d, k = (size_t)K, g = (size_t)plan.grid, n = (size_t)p->N;
  char* b = (char*)base;
  size_t off = 0;
  auto take = [&](size_t bytes) -> void* {
    void* r = b ? (void*)(b + off) : nullptr;
    off = (off + bytes + 255) & ~(size_t)255;
    return r;
  };
  Workspace w;
  std::memset(&w, 0, sizeof(w));
  w.Y = take(k * d * 4);
  w.c = (double*)take(k * 8);
  w.part_s1 = (double*)take(g * k * 8);
  w.part_s2 = (double*)take(g * k * 8);
  w.tot_s1 = (double*)take(k * 8);
  w.q_dev = (float*)take(n * k * 4);
  w.s_dev = (float*)take(n * 4);
  if (want_grad) {
    w.part_gd = (double*)take((size_t)plan.nsplit * k * d * 8);
    w.part_md = (double*)take((size_t)plan.nsplit * d * 8);
    if (plan.keep) w.zs = (float*)take(n * ((d + 3) & ~(size_t)3) * 4);
  }
  if (want_grad == 2) {
    w.f_tmp = (double*)take(k * 8);
    w.t_dev = (int64_t*)take(8);
    w.grad_out = (double*)take(k * d * 8);
  }
  w.bytes = off;
  if (ws) *ws = w;
  return off;
}

cudaError_t launch_diag(const saa_problem* p, int K, const double* X, const LawArgs& la, int want_grad,
                        const Plan& plan, const Workspace& w, double* f, double* pbar, double* var, double* grad,
                        uint32_t* err, cudaStream_t st, cudaEvent_t ev0, cudaEvent_t ev1) {
  const int d = p->d;
  const dim3 pg((unsigned)min((d + kLdThreads - 1) / kLdThreads, 1024), (unsigned)K);
  k_ld_prologue<<<pg, kLdThreads, 0, st>>>(d, K, X, p->mu, p->sd, (float*)w.Y, w.c, err);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (ev0) cudaEventRecord(ev0, st);
  switch (K) {
    case 1: e = launch_ld_kt<1>(la, K, want_grad, plan, w, st); break;
    case 2: e = launch_ld_kt<2>(la, K, want_grad, plan, w, st); break;
    default: e = launch_ld_kt<4>(la, K, want_grad, plan, w, st); break;
  }
  if (ev1) cudaEventRecord(ev1, st);
  if (e != cudaSuccess) return e;
  k_ld_value_out<<<(K * 32 + 255) / 256, 256, 0, st>>>(plan.grid, K, (double)p->N, p->lambda, w.part_s1, w.part_s2,
                                                       w.c, w.tot_s1, f, pbar, var);
  e = cudaGetLastError();
  if (e != cudaSuccess || !want_grad || !grad) return e;
  const int64_t tot = (int64_t)K * d;
  k_ld_grad_out<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(plan.nsplit, K, d, (double)p->N, p->lambda, w.part_gd,
                                                               w.part_md, w.tot_s1, p->sd, p->mu, grad);
  return cudaGetLastError();
}

}  // namespace saa
