// chol.cu -- saa_cholesky: the lower Cholesky factor C of Sigma (C C' =
// Sigma), which maps standard normals to the samples of Sec. 3.1's normal
// law (R = mu + C z), computed on the device in FP64.
//
// Right-looking blocked factorization with 32-wide block columns.  For the
// block column starting at jb:
//   diag    one warp factorizes the 32 x 32 diagonal block in shared memory
//           (column by column: pivot square root, column scaling, update of
//           the block's trailing lower triangle);
//   panel   one thread per row below the block solves L_ib L_bb' = A_ib by
//           forward substitution;
//   update  the trailing lower triangle A_ik -= L_ib L_kb' in 32 x 32 tiles,
//           one CTA per tile of the lower triangle.
// Every step has a fixed summation order, so the factor is deterministic.
// A pivot that is not positive (Sigma not positive definite, or NaN) raises
// the input bit of the context's error word; the factor is then undefined.
#include <cuda_runtime.h>

#include "internal.cuh"

namespace saa {
namespace {

constexpr int kNB = 32;

// chol = lower triangle of Sigma, zeros above the diagonal (in place when the
// pointers are equal: only the upper triangle is written then).
__global__ void k_chol_copy(int d, const double* __restrict__ S, double* C) {
  const size_t n = (size_t)d * d;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / d), j = (int)(e % d);
    if (j > i)
      C[e] = 0.0;
    else if (S != C)
      C[e] = S[e];
  }
}

__global__ void __launch_bounds__(32) k_chol_diag(int d, int jb, double* A, uint32_t* err) {
  __shared__ double a[kNB][kNB + 1];
  const int b = min(kNB, d - jb);
  const int t = threadIdx.x;
  for (int j = 0; j < kNB; ++j) a[t][j] = (t < b && j <= t) ? A[(size_t)(jb + t) * d + jb + j] : 0.0;
  __syncwarp();
  for (int j = 0; j < b; ++j) {
    double piv = a[j][j];
    if (!(piv > 0.0)) {
      if (t == 0 && err) atomicOr(err, kErrInput);
      piv = 1.0;
    }
    const double r = sqrt(piv);
    __syncwarp();
    if (t == j) a[j][j] = r;
    if (t > j && t < b) a[t][j] = a[t][j] / r;
    __syncwarp();
    if (t > j && t < b) {
      const double ltj = a[t][j];
      for (int k = j + 1; k <= t; ++k) a[t][k] -= ltj * a[k][j];
    }
    __syncwarp();
  }
  for (int j = 0; j < kNB; ++j)
    if (t < b && j <= t) A[(size_t)(jb + t) * d + jb + j] = a[t][j];
}

// Rows i >= jb + 32 of the block column: x L_bb' = a, x_j = (a_j - sum_{l<j} x_l L_jl) / L_jj.
__global__ void __launch_bounds__(128) k_chol_panel(int d, int jb, double* A) {
  __shared__ double L[kNB][kNB + 1];
  for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x) {
    const int r = e / kNB, c = e % kNB;
    L[r][c] = (c <= r) ? A[(size_t)(jb + r) * d + jb + c] : 0.0;
  }
  __syncthreads();
  const int i = jb + kNB + blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d) return;
  double* row = A + (size_t)i * d + jb;
  double x[kNB];
#pragma unroll
  for (int j = 0; j < kNB; ++j) x[j] = row[j];
#pragma unroll
  for (int j = 0; j < kNB; ++j) {
    double s = x[j];
#pragma unroll
    for (int l = 0; l < j; ++l) s -= x[l] * L[j][l];
    x[j] = s / L[j][j];
  }
#pragma unroll
  for (int j = 0; j < kNB; ++j) row[j] = x[j];
}

// Trailing update of rows/columns >= s = jb + 32: A_ik -= sum_l L_il L_kl over
// the block column, for k <= i.  CTA `idx` takes the lower-triangle tile
// (ti, tk), tk <= ti, idx = ti (ti + 1) / 2 + tk.
__global__ void __launch_bounds__(256) k_chol_update(int d, int jb, double* A) {
  __shared__ double Pi[kNB][kNB + 1], Pk[kNB][kNB + 1];
  const int s = jb + kNB;
  const int idx = blockIdx.x;
  int ti = (int)((sqrt(8.0 * idx + 1.0) - 1.0) * 0.5);
  while (ti > 0 && ti * (ti + 1) / 2 > idx) --ti;
  while ((ti + 1) * (ti + 2) / 2 <= idx) ++ti;
  const int tk = idx - ti * (ti + 1) / 2;
  const int r0 = s + kNB * ti, c0 = s + kNB * tk;
  for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x) {
    const int r = e / kNB, l = e % kNB;
    Pi[r][l] = (r0 + r < d) ? A[(size_t)(r0 + r) * d + jb + l] : 0.0;
    Pk[r][l] = (c0 + r < d) ? A[(size_t)(c0 + r) * d + jb + l] : 0.0;
  }
  __syncthreads();
  const int c = threadIdx.x % kNB;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const int r = threadIdx.x / kNB + 8 * m;
    double acc = 0.0;
#pragma unroll
    for (int l = 0; l < kNB; ++l) acc += Pi[r][l] * Pk[c][l];
    const int i = r0 + r, k = c0 + c;
    if (i < d && k <= i) A[(size_t)i * d + k] -= acc;
  }
}

}  // namespace
}  // namespace saa

using namespace saa;

extern "C" saa_status saa_cholesky(saa_ctx* ctx, int32_t d, const double* Sigma, double* chol, void* stream) {
  saa::NvtxRange nvtx_range("saa_cholesky");
  if (!ctx) {
    set_error("saa_cholesky: ctx is NULL");
    return SAA_EINVAL;
  }
  if (d < 1 || d > 46340 || !Sigma || !chol) {
    set_error("saa_cholesky: need 1 <= d <= 46340 and non-NULL Sigma, chol");
    return SAA_EINVAL;
  }
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != ctx->device && cudaSetDevice(ctx->device) != cudaSuccess) {
    set_error("saa_cholesky: cudaSetDevice failed");
    return SAA_ECUDA;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const size_t n = (size_t)d * d;
  const int cblocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  k_chol_copy<<<cblocks, 256, 0, st>>>(d, Sigma, chol);
  int64_t launches = 1;
  for (int jb = 0; jb < d; jb += kNB) {
    k_chol_diag<<<1, 32, 0, st>>>(d, jb, chol, ctx->err);
    ++launches;
    if (jb + kNB < d) {
      const int rows = d - jb - kNB;
      k_chol_panel<<<(rows + 127) / 128, 128, 0, st>>>(d, jb, chol);
      const int T = (rows + kNB - 1) / kNB;
      k_chol_update<<<T * (T + 1) / 2, 256, 0, st>>>(d, jb, chol);
      launches += 2;
    }
  }
  ctx->kernels += launches;
  const saa_status s = cuda_status(cudaGetLastError(), "saa_cholesky: launch");
  if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
  return s;
}
