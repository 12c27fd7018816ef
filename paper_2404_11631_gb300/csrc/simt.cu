// simt.cu -- CUDA-core (FFMA / DFMA) path of the SAA estimator, the
// prologue that folds the law into the decisions, and the deterministic
// finalize kernels shared by every precision.
//
// Algebra (exact in real arithmetic; the CPU oracle does NOT use it, it forms
// R_i and evaluates Eq. 4 directly):
//   R_i = mu + C a_i with a_i = s_i zhat_i, so for decision w_k
//   w_k'R_i = c_k + Q_ik,  c_k = mu'w_k,  Q_ik = a_i'y_k,  y_k = C'w_k.
//   With S1_k = sum_i Q_ik, S2_k = sum_i Q_ik^2, m~ = sum_i a_i and
//   G_k = sum_i a_i Q_ik (the adjoint contraction A'Q):
//     pbar_k = c_k + S1_k/N                                          (Eq. 5)
//     V_k    = (S2_k - S1_k^2/N) / (N-1)
//     f_k    = lambda V_k - pbar_k                                   (Eq. 4)
//     grad_k = C [ lambda 2/(N-1) (G_k - S1_k m) - m ] - mu,  m = m~/N
// The hot loop therefore never forms R_i: it regenerates the tile of a_i,
// contracts it with Y, and reduces Q in the epilogue.
#include <cuda_runtime.h>

#include "gen.cuh"
#include "internal.cuh"
#include "simt_tile.cuh"

namespace saa {

// ------------------------------------------------------------------------
// Prologue: y_k = C' w_k (FP64), c_k = mu' w_k, and y rounded to the SIMT
// contraction precision, stored transposed [d][K].  One block per (group of
// 4 decisions, 32 consecutive j); the sum over l >= j is split over 8 warps
// (l = jc + w + 8t) and merged in warp order, so the result is deterministic.
// ------------------------------------------------------------------------
constexpr int kPrepK = 4;

template <typename T>
__global__ void __launch_bounds__(256) k_prologue(int d, int K, const double* __restrict__ X,
                                                  const double* __restrict__ mu, const double* __restrict__ C,
                                                  T* __restrict__ Yt, double* __restrict__ Y64,
                                                  double* __restrict__ c, uint32_t* __restrict__ err) {
  extern __shared__ double wsm[];            // [kPrepK][d] decisions
  __shared__ double red[8][kPrepK][32];
  const int k0 = blockIdx.x * kPrepK;
  const int jc = blockIdx.y * 32;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int idx = threadIdx.x; idx < kPrepK * d; idx += blockDim.x) {
    const int kk = idx / d, l = idx % d;
    wsm[idx] = (k0 + kk < K) ? X[(size_t)(k0 + kk) * d + l] : 0.0;
  }
  __syncthreads();
  const int j = jc + lane;
  double acc[kPrepK];
#pragma unroll
  for (int kk = 0; kk < kPrepK; ++kk) acc[kk] = 0.0;
  if (j < d) {
#pragma unroll 4
    for (int l = jc + warp; l < d; l += 8) {
      const double cl = (l >= j) ? C[(size_t)l * d + j] : 0.0;
#pragma unroll
      for (int kk = 0; kk < kPrepK; ++kk) acc[kk] = fma(cl, wsm[kk * d + l], acc[kk]);
    }
  }
#pragma unroll
  for (int kk = 0; kk < kPrepK; ++kk) red[warp][kk][lane] = acc[kk];
  __syncthreads();
  if (threadIdx.x < kPrepK * 32) {
    const int kk = threadIdx.x >> 5, jj = threadIdx.x & 31;
    const int k = k0 + kk, jo = jc + jj;
    if (k < K && jo < d) {
      double y = 0.0;
#pragma unroll
      for (int w = 0; w < 8; ++w) y += red[w][kk][jj];
      Y64[(size_t)k * d + jo] = y;
      if (Yt) Yt[(size_t)jo * K + k] = (T)y;
    }
  }
  // C must have a positive, finite diagonal (the factor of a positive definite Sigma)
  if (err && blockIdx.x == 0 && warp == 0 && j < d) {
    const double cjj = C[(size_t)j * d + j];
    if (!(cjj > 0.0) || !isfinite(cjj)) atomicOr(err, kErrInput);
  }
  if (blockIdx.y == 0 && warp < kPrepK && k0 + warp < K) {
    double sdot = 0.0;
    for (int l = lane; l < d; l += 32) sdot = fma(mu[l], wsm[warp * d + l], sdot);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sdot += __shfl_down_sync(0xffffffffu, sdot, o);
    if (lane == 0) c[k0 + warp] = sdot;
  }
}

cudaError_t launch_prologue(const saa_problem* p, int K, const double* X, int prec, const Workspace& ws,
                            uint32_t* err, cudaStream_t st) {
  const dim3 grid((K + kPrepK - 1) / kPrepK, (p->d + 31) / 32);
  const size_t smem = sizeof(double) * kPrepK * p->d;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(prec == SAA_FP64 ? (const void*)k_prologue<double>
                                                          : (const void*)k_prologue<float>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  if (prec == SAA_FP64)
    k_prologue<double><<<grid, 256, smem, st>>>(p->d, K, X, p->mu, p->chol, (double*)ws.Y, ws.Y64, ws.c, err);
  else
    k_prologue<float><<<grid, 256, smem, st>>>(p->d, K, X, p->mu, p->chol, is_tc(prec) ? nullptr : (float*)ws.Y,
                                               ws.Y64, ws.c, err);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------
// Main SIMT kernel.  Persistent over scenario tiles of BM rows; per tile:
//   1. scales s_i (t law) and the tile A' = [s_i zhat_i]' into shared memory
//      ([d][BMP], zero-filled past the ragged end of the scenario range);
//   2. m~ partial sums per dimension (FP64 registers);
//   3. per K-chunk of 64 decisions: Q = A Y by register tiling (TM x 4 per
//      thread), the S1/S2 column sums by a 16-lane shuffle tree, and for the
//      gradient the adjoint tile A'Q accumulated into the CTA's partial.
// Every partial element is owned by exactly one thread of one CTA, which
// writes it on the CTA's first tile and accumulates afterwards.
// ------------------------------------------------------------------------
// ------------------------------------------------------------------------
// Main SIMT kernel: persistent over scenario tiles of BM rows; each CTA owns
// one partial slot (its S1, S2, m~ and, for the gradient, G).
// ------------------------------------------------------------------------
template <typename T, int BM, int TN>
__global__ void __launch_bounds__(kThreads, 2) k_simt(LawArgs la, int K, int want_grad, const T* __restrict__ Yt,
                                                   double* __restrict__ part_s1, double* __restrict__ part_s2,
                                                   double* __restrict__ part_m, T* __restrict__ part_g,
                                                   T* __restrict__ part_gc, int64_t tiles) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int d = la.d;
  const SimtSmem<T, BM, TN> sm(smem_raw, d);
  uint32_t epoch = la.epoch;
  if (la.t_dev) epoch += (uint32_t)(*la.t_dev / la.M);
  const gen::Stream st = gen::make_stream(la.seed, epoch, la.instance);
  const uint32_t half = la.N / 2u;

  double macc[kMaxDimSimt / kThreads];
#pragma unroll
  for (int r = 0; r < kMaxDimSimt / kThreads; ++r) macc[r] = 0.0;
  double* p_s1 = part_s1 + (size_t)blockIdx.x * K;
  double* p_s2 = part_s2 + (size_t)blockIdx.x * K;
  T* p_g = want_grad ? part_g + (size_t)blockIdx.x * K * d : nullptr;
  T* p_gc = want_grad ? part_gc + (size_t)blockIdx.x * K * d : nullptr;

  bool first = true;
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const uint32_t i0 = la.i_base + (uint32_t)(tile * BM);
    const int nrow = (int)min((int64_t)BM, (int64_t)la.rows_end() - (int64_t)i0);
    simt_tile<T, BM, TN>(st, d, la.law, la.nu, half, i0, nrow, K, Yt, sm, macc, first, want_grad, p_s1, p_s2, p_g,
                     p_gc);
    first = false;
  }
  if (!first) {
#pragma unroll
    for (int r = 0; r < kMaxDimSimt / kThreads; ++r) {
      const int j = threadIdx.x + r * kThreads;
      if (j < d) part_m[(size_t)blockIdx.x * d + j] = macc[r];
    }
  }
}

int simt_bm(int prec, int d) {
  if (prec == SAA_FP64) return d <= 256 ? 64 : (d <= 512 ? 32 : 16);
  return d <= 512 ? 64 : 32;
}

// ------------------------------------------------------------------------
// Narrow kernel for K <= kNarrowK decisions (Algorithm 1 evaluates K = 1):
// each generating thread accumulates its partial dot products a_ij y_kj
// while drawing, the G = NT / BM threads sharing a scenario are summed in
// shared memory, and the adjoint sum_i a_i Q_ik is kept per dimension in
// Kahan-compensated registers for the whole CTA.  Partial slots have the
// same layout as k_simt, so the finalize is shared.  At large d the tile of
// samples fills shared memory, so one CTA runs per SM; it then uses NT =
// 1024 threads (SAA_NARROW_WIDE_THREADS) instead of 256 to keep the SM's
// warp slots busy.
// ------------------------------------------------------------------------
constexpr int kNarrowK = 4;
#ifndef SAA_NARROW_WIDE_THREADS
#define SAA_NARROW_WIDE_THREADS 1024
#endif
constexpr int kNarrowWide = SAA_NARROW_WIDE_THREADS;

// KN: decisions handled (K <= KN <= kNarrowK); the buffers keep the kNarrowK
// stride.
template <typename T, int BM, int NT, int KN>
__global__ void __launch_bounds__(NT, NT == kThreads ? 2 : 1) k_narrow(LawArgs la, int K, int want_grad,
                                                        const T* __restrict__ Yt, double* __restrict__ part_s1,
                                                        double* __restrict__ part_s2, double* __restrict__ part_m,
                                                        T* __restrict__ part_g, T* __restrict__ part_gc,
                                                        int64_t tiles) {
  constexpr int BMP = BM + Pad<T>::v;
  constexpr int G = NT / BM;                       // threads per scenario
  constexpr int PC = gen::Gen<T>::kPerCall;
  constexpr int JR = kMaxDimSimt / NT;             // dimensions per thread (adjoint, m~)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int d = la.d;
  T* As = reinterpret_cast<T*>(smem_raw);          // [d][BMP]
  T* Ys = As + (size_t)d * BMP;                    // [kNarrowK][d]
  T* qp = Ys + (size_t)kNarrowK * d;               // [G][BM][kNarrowK]
  T* Qs = qp + (size_t)G * BM * kNarrowK;          // [BM][kNarrowK]
  T* ss = Qs + (size_t)BM * kNarrowK;              // [BM]
  const int tid = threadIdx.x;
  const int i_own = tid % BM, g_own = tid / BM;
  uint32_t epoch = la.epoch;
  if (la.t_dev) epoch += (uint32_t)(*la.t_dev / la.M);
  const gen::Stream st = gen::make_stream(la.seed, epoch, la.instance);
  const uint32_t half = la.N / 2u;
  const int nb = (d + PC - 1) / PC;
  const bool tlaw = la.law == SAA_LAW_STUDENT_T;   // other laws have s = 1

  for (int idx = tid; idx < kNarrowK * d; idx += NT) {
    const int k = idx / d, j = idx % d;
    Ys[idx] = (k < K) ? Yt[(size_t)j * K + k] : T(0);
  }
  double macc[JR];
  T gs[JR][kNarrowK], gc[JR][kNarrowK];
#pragma unroll
  for (int r = 0; r < JR; ++r) {
    macc[r] = 0.0;
#pragma unroll
    for (int k = 0; k < KN; ++k) gs[r][k] = gc[r][k] = T(0);
  }
  double* p_s1 = part_s1 + (size_t)blockIdx.x * K;
  double* p_s2 = part_s2 + (size_t)blockIdx.x * K;

  bool first = true;
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const uint32_t i0 = la.i_base + (uint32_t)(tile * BM);
    const int nrow = (int)min((int64_t)BM, (int64_t)la.rows_end() - (int64_t)i0);
    __syncthreads();
    if (tid < BM) ss[tid] = (tid < nrow) ? gen::Gen<T>::scale(st, i0 + tid, la.law, la.nu) : T(0);
    __syncthreads();
    // draw the samples of scenario i_own, blocks g_own, g_own + G, ...
    T q[kNarrowK];
#pragma unroll
    for (int k = 0; k < KN; ++k) q[k] = T(0);
    const bool live = i_own < nrow;
    const uint32_t i = i0 + (uint32_t)i_own;
    const bool logn = gen::is_lognormal(la.law, i, half);
    const T s = ss[i_own];
    for (int b = g_own; b < nb; b += G) {
      T z[PC];
      if (live) {
        gen::Gen<T>::block(st, (uint32_t)b, i, logn, z);
        if (tlaw)
#pragma unroll
          for (int e = 0; e < PC; ++e) z[e] *= s;
      } else {
#pragma unroll
        for (int e = 0; e < PC; ++e) z[e] = T(0);
      }
#pragma unroll
      for (int e = 0; e < PC; ++e) {
        const int j = b * PC + e;
        if (j < d) {
          As[(size_t)j * BMP + i_own] = z[e];
#pragma unroll
          for (int k = 0; k < KN; ++k) q[k] = fma(z[e], Ys[k * d + j], q[k]);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < KN; ++k) qp[((size_t)g_own * BM + i_own) * kNarrowK + k] = q[k];
    __syncthreads();
    if (tid < BM * kNarrowK) {
      const int ii = tid / kNarrowK, k = tid % kNarrowK;
      T v = T(0);
      if (k < KN)
#pragma unroll
        for (int g = 0; g < G; ++g) v += qp[((size_t)g * BM + ii) * kNarrowK + k];
      Qs[ii * kNarrowK + k] = v;
    }
    __syncthreads();
    if (tid < K) {
      T s1 = T(0), s2 = T(0);
      for (int ii = 0; ii < nrow; ++ii) {
        const T v = Qs[ii * kNarrowK + tid];
        s1 += v;
        s2 = fma(v, v, s2);
      }
      p_s1[tid] = first ? (double)s1 : p_s1[tid] + (double)s1;
      p_s2[tid] = first ? (double)s2 : p_s2[tid] + (double)s2;
    }
#pragma unroll
    for (int r = 0; r < JR; ++r) {
      const int j = tid + r * NT;
      if (j < d) {
        T sum = T(0);
        T gt[kNarrowK];
#pragma unroll
        for (int k = 0; k < KN; ++k) gt[k] = T(0);
        for (int ii = 0; ii < nrow; ++ii) {
          const T a = As[(size_t)j * BMP + ii];
          sum += a;
          if (want_grad) {
#pragma unroll
            for (int k = 0; k < KN; ++k) gt[k] = fma(a, Qs[ii * kNarrowK + k], gt[k]);
          }
        }
        macc[r] += (double)sum;
        if (want_grad) {
#pragma unroll
          for (int k = 0; k < KN; ++k) {   // Kahan: gc carries the lost low part
            const T y = gt[k] - gc[r][k];
            const T t = gs[r][k] + y;
            gc[r][k] = (t - gs[r][k]) - y;
            gs[r][k] = t;
          }
        }
      }
    }
    first = false;
  }
  if (!first) {
#pragma unroll
    for (int r = 0; r < JR; ++r) {
      const int j = tid + r * NT;
      if (j < d) {
        part_m[(size_t)blockIdx.x * d + j] = macc[r];
        if (want_grad) {
#pragma unroll
          for (int k = 0; k < KN; ++k)
            if (k < K) {
              const size_t e = ((size_t)blockIdx.x * K + k) * d + j;
              part_g[e] = gs[r][k];
              part_gc[e] = gc[r][k];
            }
        }
      }
    }
  }
}

// Threads per CTA of the narrow kernel: the wide form for the FP32 tile of
// 32 scenarios (d > 512), where the tile's shared memory allows one CTA per SM.
int narrow_threads(int prec, int bm) { return (prec != SAA_FP64 && bm == 32) ? kNarrowWide : kThreads; }

size_t narrow_smem(int prec, int d, int bm) {
  const size_t es = (prec == SAA_FP64) ? 8 : 4;
  const int pad = (prec == SAA_FP64) ? 2 : 4;
  const size_t G = (size_t)narrow_threads(prec, bm) / bm;
  return es * ((size_t)d * (bm + pad) + (size_t)kNarrowK * d + G * bm * kNarrowK + (size_t)bm * kNarrowK + bm);
}

template <typename T, int BM, int NT>
static const void* narrow_fn() { return (const void*)k_narrow<T, BM, NT, kNarrowK>; }

static const void* narrow_kernel(int prec, int bm) {
  if (prec == SAA_FP64) return bm == 64 ? narrow_fn<double, 64, kThreads>()
                             : bm == 32 ? narrow_fn<double, 32, kThreads>() : narrow_fn<double, 16, kThreads>();
  return bm == 64 ? narrow_fn<float, 64, kThreads>() : narrow_fn<float, 32, kNarrowWide>();
}

int narrow_occupancy(int prec, int bm, int smem) {
  int n = 0;
  const void* f = narrow_kernel(prec, bm);
  if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, narrow_threads(prec, bm), smem) != cudaSuccess || n < 1)
    return 1;
  return n;
}

template <typename T, int BM, int NT>
static cudaError_t launch_narrow_t(const LawArgs& la, int K, int want_grad, const Plan& plan, const Workspace& ws,
                                   cudaStream_t st) {
  auto kern = K == 1 ? k_narrow<T, BM, NT, 1> : K == 2 ? k_narrow<T, BM, NT, 2> : k_narrow<T, BM, NT, kNarrowK>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, plan.smem);
  if (e != cudaSuccess) return e;
  kern<<<plan.grid, NT, plan.smem, st>>>(la, K, want_grad, (const T*)ws.Y, ws.part_s1, ws.part_s2, ws.part_m,
                                         (T*)ws.part_g, (T*)ws.part_gc, plan.tiles);
  return cudaGetLastError();
}

static cudaError_t launch_narrow(const LawArgs& la, int K, int prec, int want_grad, const Plan& plan,
                                 const Workspace& ws, cudaStream_t st) {
  if (prec == SAA_FP64) {
    switch (plan.bm) {
      case 64: return launch_narrow_t<double, 64, kThreads>(la, K, want_grad, plan, ws, st);
      case 32: return launch_narrow_t<double, 32, kThreads>(la, K, want_grad, plan, ws, st);
      default: return launch_narrow_t<double, 16, kThreads>(la, K, want_grad, plan, ws, st);
    }
  }
  return plan.bm == 64 ? launch_narrow_t<float, 64, kThreads>(la, K, want_grad, plan, ws, st)
                       : launch_narrow_t<float, 32, kNarrowWide>(la, K, want_grad, plan, ws, st);
}

int simt_tn(int K) { return K <= 16 ? 1 : 4; }

size_t simt_smem(int prec, int d, int bm, int tn) {
  const size_t es = (prec == SAA_FP64) ? 8 : 4;
  const int pad = (prec == SAA_FP64) ? 2 : 4;
  const size_t bn = 16 * (size_t)tn;
  return es * ((size_t)d * (bm + pad) + (size_t)kDK * bn + (size_t)bm * (bn + 1) + bm);
}

template <typename T, int BM, int TN>
static cudaError_t launch_simt_t(const LawArgs& la, int K, int want_grad, const Plan& plan, const Workspace& ws,
                                 cudaStream_t st) {
  auto kern = k_simt<T, BM, TN>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, plan.smem);
  if (e != cudaSuccess) return e;
  kern<<<plan.grid, kThreads, plan.smem, st>>>(la, K, want_grad, (const T*)ws.Y, ws.part_s1, ws.part_s2,
                                               ws.part_m, (T*)ws.part_g, (T*)ws.part_gc, plan.tiles);
  return cudaGetLastError();
}

template <int TN>
static cudaError_t launch_simt_tn(const LawArgs& la, int K, int prec, int want_grad, const Plan& plan,
                                  const Workspace& ws, cudaStream_t st) {
  if (prec == SAA_FP64) {
    switch (plan.bm) {
      case 64: return launch_simt_t<double, 64, TN>(la, K, want_grad, plan, ws, st);
      case 32: return launch_simt_t<double, 32, TN>(la, K, want_grad, plan, ws, st);
      default: return launch_simt_t<double, 16, TN>(la, K, want_grad, plan, ws, st);
    }
  }
  switch (plan.bm) {
    case 64: return launch_simt_t<float, 64, TN>(la, K, want_grad, plan, ws, st);
    default: return launch_simt_t<float, 32, TN>(la, K, want_grad, plan, ws, st);
  }
}

cudaError_t launch_simt(const LawArgs& la, int K, int prec, int want_grad, const Plan& plan, const Workspace& ws,
                        cudaStream_t st) {
  if (plan.narrow) return launch_narrow(la, K, prec, want_grad, plan, ws, st);
  return plan.tn == 1 ? launch_simt_tn<1>(la, K, prec, want_grad, plan, ws, st)
                      : launch_simt_tn<4>(la, K, prec, want_grad, plan, ws, st);
}

template <int TN>
static const void* simt_fn(int prec, int bm) {
  if (prec == SAA_FP64)
    return bm == 64 ? (const void*)k_simt<double, 64, TN> : bm == 32 ? (const void*)k_simt<double, 32, TN>
                                                                      : (const void*)k_simt<double, 16, TN>;
  return bm == 64 ? (const void*)k_simt<float, 64, TN> : (const void*)k_simt<float, 32, TN>;
}

int simt_occupancy(int prec, int bm, int tn, int smem) {
  int n = 0;
  const void* f = tn == 1 ? simt_fn<1>(prec, bm) : simt_fn<4>(prec, bm);
  if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, kThreads, smem) != cudaSuccess || n < 1) return 1;
  return n;
}

// ------------------------------------------------------------------------
// Finalize.  All cross-CTA sums are Neumaier-compensated FP64 sums in a
// fixed order (CTA index, then a fixed warp tree), so the result does not
// depend on scheduling.
// ------------------------------------------------------------------------
__device__ __forceinline__ void neumaier(double& s, double& c, double x) {
  const double t = s + x;
  if (fabs(s) >= fabs(x))
    c += (s - t) + x;
  else
    c += (x - t) + s;
  s = t;
}

// Items 0..K-1: part_s1, K..2K-1: part_s2, 2K..2K+d-1: part_m; one warp each.
__global__ void k_reduce_parts(const double* __restrict__ part_s1, const double* __restrict__ part_s2,
                               const double* __restrict__ part_m, int grid, int K, int d, int first,
                               double* __restrict__ s1, double* __restrict__ s2, double* __restrict__ m) {
  const int item = first + (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (item >= 2 * K + d) return;
  const double* src;
  int stride, off;
  double* dst;
  if (item < K) {
    src = part_s1; stride = K; off = item; dst = s1 + item;
  } else if (item < 2 * K) {
    src = part_s2; stride = K; off = item - K; dst = s2 + (item - K);
  } else {
    src = part_m; stride = d; off = item - 2 * K; dst = m + (item - 2 * K);
  }
  double s = 0.0, c = 0.0;
  for (int g = lane; g < grid; g += 32) neumaier(s, c, src[(size_t)g * stride + off]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double s_o = __shfl_down_sync(0xffffffffu, s, o);
    const double c_o = __shfl_down_sync(0xffffffffu, c, o);
    if (lane < o) {
      neumaier(s, c, s_o);
      c += c_o;
    }
  }
  if (lane == 0) *dst = s + c;
}

// Tensor path: S1_k = m~'y_k (FP64, fixed order) -- the row sums of Q are
// recovered from the per-dimension sums of a_i, sum_i Q_ik = (sum_i a_i)'y_k --
// then the value outputs.  One warp per decision.
__global__ void k_value_out_m(int K, int d, double N, double lambda, const double* __restrict__ m,
                              const double* __restrict__ Y64, const double* __restrict__ c,
                              const double* __restrict__ s2, double* __restrict__ s1_out, double* __restrict__ f,
                              double* __restrict__ pbar, double* __restrict__ var) {
  const int k = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (k >= K) return;
  double s = 0.0;
  for (int j = lane; j < d; j += 32) s = fma(m[j], Y64[(size_t)k * d + j], s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) {
    s1_out[k] = s;
    const double qbar = s / N;
    const double pb = c[k] + qbar;
    const double V = (s2[k] - s * qbar) / (N - 1.0);
    if (f) f[k] = lambda * V - pb;
    if (pbar) pbar[k] = pb;
    if (var) var[k] = V;
  }
}

__global__ void k_value_out(int K, double N, double lambda, const double* __restrict__ c,
                            const double* __restrict__ s1, const double* __restrict__ s2, double* __restrict__ f,
                            double* __restrict__ pbar, double* __restrict__ var) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  const double qbar = s1[k] / N;
  const double pb = c[k] + qbar;
  const double V = (s2[k] - s1[k] * qbar) / (N - 1.0);
  if (f) f[k] = lambda * V - pb;
  if (pbar) pbar[k] = pb;
  if (var) var[k] = V;
}

// u_k = lambda 2/(N-1) (G_k - S1_k m) - m.  G_kj is the sum of the CTAs'
// Kahan-carried partials (value part_g, compensation part_gc): one block per
// (32 dimensions, decision k), warp w sums CTAs w, w + 8, ... and the eight
// warp sums are merged in warp order, so the result is deterministic.  FP32
// partials are summed as float-float pairs (branch-free TwoSum, the running
// error and the Kahan compensations in a second float): about 2^-48 relative,
// without the narrow FP64 pipe.  FP64 partials use Neumaier's sum.
// With raw set it writes G_kj itself (the partial sums of saa_partials).
template <typename T>
__global__ void __launch_bounds__(256) k_grad_u(int grid, int K, int d, double N, double lambda,
                                                const T* __restrict__ part_g, const T* __restrict__ part_gc,
                                                const double* __restrict__ s1, const double* __restrict__ mt,
                                                double* __restrict__ u, int raw) {
  __shared__ double sh_s[8][32], sh_c[8][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = blockIdx.x * 32 + lane;
  const int k = blockIdx.y;
  double s = 0.0, c = 0.0;
  if (j < d) {
    if constexpr (sizeof(T) == 4) {
      float S = 0.0f, E = 0.0f;
#pragma unroll 4
      for (int g = warp; g < grid; g += 8) {
        const size_t e = ((size_t)g * K + k) * d + j;
        const float x = (float)part_g[e], xc = (float)part_gc[e];
        const float t = __fadd_rn(S, x);
        const float bb = __fsub_rn(t, S);
        const float err = __fadd_rn(__fsub_rn(S, __fsub_rn(t, bb)), __fsub_rn(x, bb));
        S = t;
        E = __fadd_rn(E, __fsub_rn(err, xc));
      }
      s = (double)S;
      c = (double)E;
    } else {
      for (int g = warp; g < grid; g += 8) {
        const size_t e = ((size_t)g * K + k) * d + j;
        neumaier(s, c, (double)part_g[e]);
        neumaier(s, c, -(double)part_gc[e]);
      }
    }
  }
  sh_s[warp][lane] = s;
  sh_c[warp][lane] = c;
  __syncthreads();
  if (warp == 0 && j < d) {
    double S = 0.0, C = 0.0;
    for (int w = 0; w < 8; ++w) {
      neumaier(S, C, sh_s[w][lane]);
      neumaier(S, C, sh_c[w][lane]);
    }
    const double G = S + C;
    if (raw) {
      u[(size_t)k * d + j] = G;
    } else {
      const double mj = mt[j] / N;
      u[(size_t)k * d + j] = lambda * (2.0 / (N - 1.0)) * (G - s1[k] * mj) - mj;
    }
  }
}

// grad_kj = sum_{l <= j} C_jl u_kl - mu_j (mu NULL: 0): one warp per (k, j).
__global__ void k_grad_out(int K, int d, const double* __restrict__ C, const double* __restrict__ mu,
                           const double* __restrict__ u, double* __restrict__ grad) {
  const int row = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= K * d) return;
  const int k = row / d, j = row % d;
  const double* cj = C + (size_t)j * d;
  const double* uk = u + (size_t)k * d;
  double s = 0.0;
  for (int l = lane; l <= j; l += 32) s = fma(cj[l], uk[l], s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) grad[(size_t)k * d + j] = mu ? s - mu[j] : s;
}

cudaError_t launch_grad_out(int K, int d, const double* chol, const double* mu, const double* u, double* grad,
                            cudaStream_t st) {
  const int64_t warps = (int64_t)K * d;
  k_grad_out<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(K, d, chol, mu, u, grad);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const saa_problem* p, int K, int prec, int want_grad, const Plan& plan,
                            const Workspace& ws, double* f, double* pbar, double* var, double* grad,
                            cudaStream_t st) {
  const int d = p->d;
  const int items = 2 * K + d;
  // the tensor path keeps no row sums of Q: items 0..K-1 (S1 partials) are skipped
  const int first = is_tc(prec) ? K : 0;
  k_reduce_parts<<<((items - first) * 32 + 255) / 256, 256, 0, st>>>(ws.part_s1, ws.part_s2, ws.part_m, plan.grid,
                                                                      K, d, first, ws.tot_s1, ws.tot_s2, ws.tot_m);
  const double N = (double)p->N;
  if (is_tc(prec))
    k_value_out_m<<<(K * 32 + 255) / 256, 256, 0, st>>>(K, d, N, p->lambda, ws.tot_m, ws.Y64, ws.c, ws.tot_s2,
                                                         ws.tot_s1, f, pbar, var);
  else if (f || pbar || var)
    k_value_out<<<(K + 255) / 256, 256, 0, st>>>(K, N, p->lambda, ws.c, ws.tot_s1, ws.tot_s2, f, pbar, var);
  if (want_grad && grad) {
    dim3 gu((d + 31) / 32, K);
    if (prec == SAA_FP64)
      k_grad_u<double><<<gu, 256, 0, st>>>(plan.grid, K, d, N, p->lambda, (const double*)ws.part_g,
                                           (const double*)ws.part_gc, ws.tot_s1, ws.tot_m, ws.grad_tmp, 0);
    else
      k_grad_u<float><<<gu, 256, 0, st>>>(plan.grid, K, d, N, p->lambda, (const float*)ws.part_g,
                                          (const float*)ws.part_gc, ws.tot_s1, ws.tot_m, ws.grad_tmp, 0);
    const int64_t warps = (int64_t)K * d;
    k_grad_out<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(K, d, p->chol, p->mu, ws.grad_tmp, grad);
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------------
// saa_partials: the CTA partials of a scenario range merged (the same fixed
// order as the finalize) and mapped from the whitened coordinates of the
// kernels to the paper's, D_i = R_i - mu = C a_i:
//   P1_k = S1_k, P2_k = S2_k, P3 = C m~, P4_k = C G_k.
// ------------------------------------------------------------------------
cudaError_t launch_partials_out(const saa_problem* p, int K, int prec, int want_grad, const Plan& plan,
                                const Workspace& ws, double* part, cudaStream_t st) {
  const int d = p->d;
  const int items = 2 * K + d;
  const int first = is_tc(prec) ? K : 0;
  double* P1 = part;
  double* P2 = part + K;
  double* P3 = part + 2 * K;
  double* P4 = part + 2 * K + d;
  k_reduce_parts<<<((items - first) * 32 + 255) / 256, 256, 0, st>>>(ws.part_s1, ws.part_s2, ws.part_m, plan.grid,
                                                                      K, d, first, P1, P2, ws.tot_m);
  if (is_tc(prec))   // S1 = m~'y_k (the tensor kernels keep no row sums of Q)
    k_value_out_m<<<(K * 32 + 255) / 256, 256, 0, st>>>(K, d, 2.0, p->lambda, ws.tot_m, ws.Y64, ws.c, P2, P1,
                                                         nullptr, nullptr, nullptr);
  k_grad_out<<<(unsigned)((d * 32 + 255) / 256), 256, 0, st>>>(1, d, p->chol, nullptr, ws.tot_m, P3);
  if (want_grad) {
    dim3 gu((d + 31) / 32, K);
    if (prec == SAA_FP64)
      k_grad_u<double><<<gu, 256, 0, st>>>(plan.grid, K, d, 2.0, p->lambda, (const double*)ws.part_g,
                                           (const double*)ws.part_gc, nullptr, nullptr, ws.grad_tmp, 1);
    else
      k_grad_u<float><<<gu, 256, 0, st>>>(plan.grid, K, d, 2.0, p->lambda, (const float*)ws.part_g,
                                          (const float*)ws.part_gc, nullptr, nullptr, ws.grad_tmp, 1);
    const int64_t warps = (int64_t)K * d;
    k_grad_out<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(K, d, p->chol, nullptr, ws.grad_tmp, P4);
  }
  return cudaGetLastError();
}

// saa_partials_merge: element e of the totals is the Neumaier-compensated
// sum of parts[r][e] over r = 0 .. R-1 in that order, one thread per
// element, so the totals do not depend on who computed which range when.
__global__ void k_merge_partials(int R, int64_t len, const double* __restrict__ parts, double* __restrict__ total) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= len) return;
  double s = 0.0, c = 0.0;
  for (int r = 0; r < R; ++r) neumaier(s, c, parts[(size_t)r * len + e]);
  total[e] = s + c;
}

cudaError_t launch_merge_partials(int R, int64_t len, const double* parts, double* total, cudaStream_t st) {
  k_merge_partials<<<(unsigned)((len + 255) / 256), 256, 0, st>>>(R, len, parts, total);
  return cudaGetLastError();
}

// saa_finalize_partials: Eq. 4, Eq. 5 and the gradient from the whole
// sample's partial sums, one warp per decision (FP64):
//   pbar = w'mu + P1/N, V = (P2 - P1^2/N)/(N-1), f = lambda V - pbar,
//   grad_j = lambda 2/(N-1) (P4_j - P1 P3_j/N) - (mu_j + P3_j/N).
__global__ void k_finalize_partials(int K, int d, double N, double lambda, const double* __restrict__ X,
                                    const double* __restrict__ mu, const double* __restrict__ part,
                                    double* __restrict__ f, double* __restrict__ pbar, double* __restrict__ var,
                                    double* __restrict__ grad) {
  const int k = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (k >= K) return;
  const double* x = X + (size_t)k * d;
  double c = 0.0;
  for (int j = lane; j < d; j += 32) c = fma(mu[j], x[j], c);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  const double P1 = part[k], P2 = part[K + k];
  const double* P3 = part + 2 * K;
  const double* P4 = part + 2 * K + d + (size_t)k * d;
  if (lane == 0) {
    const double pb = c + P1 / N;
    const double V = (P2 - P1 * (P1 / N)) / (N - 1.0);
    if (f) f[k] = lambda * V - pb;
    if (pbar) pbar[k] = pb;
    if (var) var[k] = V;
  }
  if (grad) {
    const double a = lambda * (2.0 / (N - 1.0));
    for (int j = lane; j < d; j += 32)
      grad[(size_t)k * d + j] = a * (P4[j] - P1 * (P3[j] / N)) - (mu[j] + P3[j] / N);
  }
}

cudaError_t launch_finalize_partials(int64_t N, int d, int K, double lambda, const double* X, const double* mu,
                                     const double* part, double* f, double* pbar, double* var, double* grad,
                                     cudaStream_t st) {
  k_finalize_partials<<<(K * 32 + 255) / 256, 256, 0, st>>>(K, d, (double)N, lambda, X, mu, part, f, pbar, var,
                                                             grad);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------
// saa_generate: innovations / scales (one thread per (scenario, block)),
// then the samples xi (one thread per (scenario, dimension)).
// ------------------------------------------------------------------------
template <typename T>
__global__ void k_gen_z(LawArgs la, int64_t i0, int64_t n, T* __restrict__ z, T* __restrict__ s) {
  constexpr int PC = gen::Gen<T>::kPerCall;
  const int d = la.d;
  const int nb = (d + PC - 1) / PC;
  const gen::Stream st = gen::make_stream(la.seed, la.epoch, la.instance);
  const uint32_t half = la.N / 2u;
  const int64_t total = n * nb;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = idx / nb;
    const int b = (int)(idx % nb);
    const uint32_t i = (uint32_t)(i0 + r);
    T v[PC];
    gen::Gen<T>::block(st, (uint32_t)b, i, gen::is_lognormal(la.law, i, half), v);
#pragma unroll
    for (int q = 0; q < PC; ++q) {
      const int j = b * PC + q;
      if (j < d) z[r * d + j] = v[q];
    }
    if (b == 0 && s) s[r] = gen::Gen<T>::scale(st, i, la.law, la.nu);
  }
}

__device__ __forceinline__ float fma_p(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_p(double a, double b, double c) { return __fma_rn(a, b, c); }

template <typename T>
__global__ void k_gen_xi(int d, int64_t n, const double* __restrict__ mu, const double* __restrict__ C,
                         const T* __restrict__ z, const T* __restrict__ s, T* __restrict__ xi) {
  const int64_t total = n * d;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = idx / d;
    const int j = (int)(idx % d);
    const T* zr = z + r * d;
    T acc = T(0);
    for (int l = 0; l <= j; ++l) acc = fma_p((T)C[(size_t)j * d + l], zr[l], acc);
    xi[idx] = fma_p(s[r], acc, (T)mu[j]);
  }
}

cudaError_t launch_generate(const LawArgs& la, int64_t i0, int64_t n, int prec, const double* mu,
                            const double* chol, void* z, void* s, void* xi, cudaStream_t st) {
  const int blocks = 1024;
  if (prec == SAA_FP64) {
    k_gen_z<double><<<blocks, 256, 0, st>>>(la, i0, n, (double*)z, (double*)s);
    if (xi) k_gen_xi<double><<<blocks, 256, 0, st>>>(la.d, n, mu, chol, (const double*)z, (const double*)s,
                                                     (double*)xi);
  } else {
    k_gen_z<float><<<blocks, 256, 0, st>>>(la, i0, n, (float*)z, (float*)s);
    if (xi) k_gen_xi<float><<<blocks, 256, 0, st>>>(la.d, n, mu, chol, (const float*)z, (const float*)s,
                                                    (float*)xi);
  }
  return cudaGetLastError();
}

}  // namespace saa
