// fw.cu -- the Frank-Wolfe update of Algorithm 1 (arXiv 2404.11631,
// Sec. 3.1) as one single-CTA FP64 kernel, so that a whole iteration
// (prologue, sample-average gradient, finalize, update) is a fixed sequence
// of launches that can be captured once as a CUDA graph and replayed.
//
// Given g = grad f_hat(w_t) and f_hat(w_t):
//   LMO over W = {w >= 0, 1'w <= 1}: the vertices of W are 0 and the unit
//   vectors, so s_t = e_j* for the first j* minimising g_j if g_j* < 0,
//   else s_t = 0;
//   gamma_t = 2 / (t + 2) (t = kM + m, the global iteration count);
//   w_{t+1} = w_t + gamma_t (s_t - w_t);  gap_t = g'(w_t - s_t) >= 0.
// The iteration counter lives in device memory and is advanced here, which
// also selects the next resample index floor(t / M) for the sample kernel.
#include <cuda_runtime.h>

#include "internal.cuh"

namespace saa {

constexpr int kFwThreads = 512;

__global__ void __launch_bounds__(kFwThreads) k_fw_step(int d, const double* __restrict__ g,
                                                        const double* __restrict__ f, double* __restrict__ w,
                                                        const int64_t* t_in, int64_t t_base,
                                                        double* __restrict__ f_trace, double* __restrict__ gap_trace,
                                                        int64_t* t_out) {
  __shared__ double sv[kFwThreads];
  __shared__ int si[kFwThreads];
  __shared__ double sg[kFwThreads];
  const int tid = threadIdx.x;
  const int64_t t = *t_in;
  double best = 0.0, gw = 0.0;
  int bi = -1;
  for (int j = tid; j < d; j += kFwThreads) {
    const double gj = g[j];
    if (bi < 0 || gj < best) {
      best = gj;
      bi = j;
    }
    gw = fma(gj, w[j], gw);
  }
  sv[tid] = best;
  si[tid] = bi;
  sg[tid] = gw;
  __syncthreads();
  for (int off = kFwThreads / 2; off > 0; off >>= 1) {
    if (tid < off) {
      const int oi = si[tid + off];
      const double ov = sv[tid + off];
      // smaller value wins; on equal values the smaller index wins
      if (oi >= 0 && (si[tid] < 0 || ov < sv[tid] || (ov == sv[tid] && oi < si[tid]))) {
        sv[tid] = ov;
        si[tid] = oi;
      }
      sg[tid] += sg[tid + off];
    }
    __syncthreads();
  }
  const double gmin = sv[0];
  const int js = (si[0] >= 0 && gmin < 0.0) ? si[0] : -1;
  const double gamma = 2.0 / ((double)t + 2.0);
  for (int j = tid; j < d; j += kFwThreads) {
    const double sj = (j == js) ? 1.0 : 0.0;
    w[j] = w[j] + gamma * (sj - w[j]);
  }
  if (tid == 0) {
    const int64_t it = t - t_base;
    if (f_trace) f_trace[it] = *f;
    if (gap_trace) gap_trace[it] = sg[0] - (js >= 0 ? gmin : 0.0);
  }
  __syncthreads();
  if (tid == 0) *t_out = t + 1;
}

__global__ void k_set_i64(int64_t* p, int64_t v) { *p = v; }

cudaError_t launch_fw_step(int d, const double* g, const double* f, double* w, const int64_t* t_dev,
                           int64_t t_base, double* f_trace, double* gap_trace, int64_t* t_next, cudaStream_t st) {
  k_fw_step<<<1, kFwThreads, 0, st>>>(d, g, f, w, t_dev, t_base, f_trace, gap_trace, t_next);
  return cudaGetLastError();
}

cudaError_t launch_set_i64(int64_t* p, int64_t v, cudaStream_t st) {
  k_set_i64<<<1, 1, 0, st>>>(p, v);
  return cudaGetLastError();
}

}  // namespace saa
