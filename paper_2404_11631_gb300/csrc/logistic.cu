// logistic.cu -- the binary-classification task of Sec. 3.3: the
// sample-average objective F(omega) of the logistic model, its gradient
// and the sub-sampled Hessian applied to a vector, over an index set S of a
// binary data set, for K parameter vectors at once.
//
//   t_ik = x_i'omega_k,  c = 1 / (1 + e^-t)
//   F_k    = (1/b) sum_{i in S} [ log(1 + e^t_ik) - z_i t_ik ]
//   grad_k = (1/b) sum_{i in S} (c_ik - z_i) x_i
//   hvp_k  = (1/b) sum_{i in S} c_ik (1 - c_ik) (x_i'v_k) x_i
//
// Features are bits: row i of the data set is nwp 32-bit words (feature j =
// bit j % 32 of word j / 32, padded with zero words to a multiple of 4).
// The forward contraction runs one thread per sample (the weights are read
// by all lanes of a warp at one shared-memory address, so every load is a
// broadcast) with masked FP32 adds folded into float-float sums once per
// word; the per-sample terms are FP64.  The adjoint runs one lane per
// feature word (32 features in registers) over a slice of the samples, so
// the bit loads are coalesced and the residuals are broadcast; the CTA
// merges its warps in fixed order into an FP64 partial per slice, and a
// final kernel adds the slices in order.  Every sum has a fixed order: the
// results are bitwise deterministic for a given device.
//
// The data set of Sec. 4.1's setup is generated by saa_logistic_generate:
// Bernoulli(1/2) features from Philox bits (counter tag 4) and labels from
// an integer linear rule z = [2 x'w* > 1'w*], flipped where the point's
// noise word (tag 5) is below a threshold.
#include <cuda_runtime.h>

#include "gen.cuh"
#include "internal.cuh"

namespace saa {
namespace {

constexpr int kLgThreads = 256;
constexpr int kLgMaxVec = 8;              // vectors in one forward pass (omega_k and v_k)
constexpr int kLgSmemFloats = 48 * 1024;  // shared-memory budget of the forward vectors (192 KB)
constexpr int kLgAdjSamples = 1024;       // samples per adjoint slice (128 per warp)

__host__ __device__ inline int lg_pitch(int n) { return ((n + 31) / 32 + 3) / 4 * 4; }

// ------------------------------------------------------------- data ------
__global__ void k_lg_features(int n, int nwp, uint64_t seed, uint32_t instance, int64_t i0, int64_t rows,
                              uint32_t* __restrict__ X) {
  const int nb = nwp / 4;   // 128-feature blocks per row (the padding words are whole blocks' tails)
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows * nb) return;
  const int64_t r = t / nb;
  const int b = (int)(t % nb);
  const gen::Stream st = gen::make_stream(seed, 0u, instance);
  const uint4 w = gen::philox(st, (uint32_t)b, (uint32_t)(i0 + r), gen::kTagFeature);
  uint32_t v[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int j0 = 128 * b + 32 * q;   // first feature of the word
    if (j0 >= n)
      v[q] = 0u;
    else if (n - j0 < 32)
      v[q] &= (1u << (n - j0)) - 1u;
  }
  *reinterpret_cast<uint4*>(X + (size_t)r * nwp + 4 * b) = make_uint4(v[0], v[1], v[2], v[3]);
}

// Labels: each block forms 1'w* once, then one warp per point takes the
// integer dot product of its bits with w*.
__global__ void __launch_bounds__(kLgThreads) k_lg_labels(int n, int nwp, uint64_t seed, uint32_t instance,
                                                          uint32_t flip, int64_t i0, int64_t rows,
                                                          const uint32_t* __restrict__ X,
                                                          const int32_t* __restrict__ wstar, uint8_t* __restrict__ z) {
  __shared__ long long sh[kLgThreads / 32];
  __shared__ long long s_tot;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long part = 0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) part += wstar[j];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if (lane == 0) sh[warp] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t = 0;
    for (int w = 0; w < kLgThreads / 32; ++w) t += sh[w];
    s_tot = t;
  }
  __syncthreads();
  const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (r >= rows) return;
  long long dot = 0;
  for (int q = lane; q < nwp; q += 32) {
    uint32_t bits = X[(size_t)r * nwp + q];
    while (bits) {
      const int t = __ffs(bits) - 1;
      bits &= bits - 1u;
      if (32 * q + t < n) dot += wstar[32 * q + t];
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
  if (lane == 0) {
    uint8_t lab = (uint8_t)(2 * dot > s_tot);
    const gen::Stream st = gen::make_stream(seed, 0u, instance);
    if (gen::philox(st, 0u, (uint32_t)(i0 + r), gen::kTagLabelNoise).x < flip) lab ^= 1u;
    z[r] = lab;
  }
}

// ------------------------------------------------------- estimator -------
// FP32 copies of the vectors the forward pass contracts: rows 0..K-1 are
// omega_k, rows K..2K-1 (with V) are v_k.
__global__ void k_lg_prep(int K, int n, int nv, const double* __restrict__ W, const double* __restrict__ V,
                          float* __restrict__ vec) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)nv * n) return;
  const int v = (int)(t / n), j = (int)(t % n);
  vec[t] = (float)(v < K ? W[(size_t)v * n + j] : V[(size_t)(v - K) * n + j]);
}

__device__ __forceinline__ void ff_add(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bp = s - hi;
  lo += (hi - (s - bp)) + (x - bp);
  hi = s;
}

// G threads per group of SPT samples (point i = idx[s], or s): thread c of
// the group takes the words q = c, c + G, ... of each of its samples, so
// every weight load serves SPT samples; t_v = x_i'vec_v for the NV = KC
// (HV ? 2 : 1) vectors, merged over the group by float-float shuffles;
// then the group's first thread forms the per-sample terms of F, the
// residual r = c - z and the Hessian weight h = c (1 - c) x'v from one
// FP32 exponential (the loss's large part exact in FP64).  (G, SPT) =
// (1, 2) for large samples (every weight load is a broadcast) or (8, 1)
// for small ones (eight threads share a point's features).  The weights
// are stored with a pitch of 36 floats per word, so the G threads' 16-byte
// loads fall in different banks.  The CTA's loss sums go to
// lossp[block][KC].
constexpr int kLgWordPitch = 36;

template <int KC, bool HV, int G, int SPT>
__global__ void __launch_bounds__(kLgThreads) k_lg_fwd(int n, int nwp, int64_t N, int64_t b,
                                                       const int64_t* __restrict__ idx, uint32_t* __restrict__ err,
                                                       const uint32_t* __restrict__ X, const uint8_t* __restrict__ z,
                                                       const float* __restrict__ vec, float* __restrict__ rs,
                                                       float* __restrict__ hs, double* __restrict__ lossp) {
  constexpr int NV = KC * (HV ? 2 : 1);
  constexpr int K = KC;
  extern __shared__ __align__(16) float svec[];   // [NV][nwp][36]
  __shared__ double sloss[kLgThreads / 32][KC];
  const int vpitch = kLgWordPitch * nwp;
  for (int e = threadIdx.x; e < NV * 32 * nwp; e += blockDim.x) {
    const int v = e / (32 * nwp), j = e % (32 * nwp);
    svec[v * vpitch + (j >> 5) * kLgWordPitch + (j & 31)] = j < n ? vec[(size_t)v * n + j] : 0.0f;
  }
  __syncthreads();
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int c = (int)(gt % G);
  int64_t sm[SPT], im[SPT];
  bool act[SPT];
#pragma unroll
  for (int m = 0; m < SPT; ++m) {
    sm[m] = (gt / G) * SPT + m;
    act[m] = sm[m] < b;
    im[m] = act[m] ? (idx ? idx[sm[m]] : sm[m]) : 0;
    if (act[m] && (im[m] < 0 || im[m] >= N)) {   // an index outside the data set: flagged, skipped
      if (c == 0) atomicOr(err, kErrInput);
      act[m] = false;
    }
  }
  float th[SPT][NV], tl[SPT][NV];
#pragma unroll
  for (int m = 0; m < SPT; ++m)
#pragma unroll
    for (int v = 0; v < NV; ++v) th[m][v] = tl[m][v] = 0.0f;
  {
    // 4-word groups c, c + G, ...; the next group's loads are issued before
    // the current one is processed
    const int ng = nwp / 4;
    const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
    const uint4* row4[SPT];
    uint4 cur[SPT];
#pragma unroll
    for (int m = 0; m < SPT; ++m) {
      row4[m] = reinterpret_cast<const uint4*>(X + (size_t)im[m] * nwp);
      cur[m] = (act[m] && c < ng) ? row4[m][c] : zero;
    }
    for (int gq = c; gq < ng; gq += G) {
      uint4 nxt[SPT];
#pragma unroll
      for (int m = 0; m < SPT; ++m) nxt[m] = (act[m] && gq + G < ng) ? row4[m][gq + G] : zero;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        uint32_t bits[SPT];
#pragma unroll
        for (int m = 0; m < SPT; ++m) bits[m] = u == 0 ? cur[m].x : u == 1 ? cur[m].y : u == 2 ? cur[m].z : cur[m].w;
        const float* wq = svec + (4 * gq + u) * kLgWordPitch;
        float p[SPT][NV];
#pragma unroll
        for (int m = 0; m < SPT; ++m)
#pragma unroll
          for (int v = 0; v < NV; ++v) p[m][v] = 0.0f;
#pragma unroll
        for (int t4 = 0; t4 < 8; ++t4) {
          float4 wv[NV];
#pragma unroll
          for (int v = 0; v < NV; ++v) wv[v] = *reinterpret_cast<const float4*>(wq + v * vpitch + 4 * t4);
#pragma unroll
          for (int m = 0; m < SPT; ++m)
#pragma unroll
            for (int v = 0; v < NV; ++v) {
              if (bits[m] & (1u << (4 * t4 + 0))) p[m][v] += wv[v].x;
              if (bits[m] & (1u << (4 * t4 + 1))) p[m][v] += wv[v].y;
              if (bits[m] & (1u << (4 * t4 + 2))) p[m][v] += wv[v].z;
              if (bits[m] & (1u << (4 * t4 + 3))) p[m][v] += wv[v].w;
            }
        }
#pragma unroll
        for (int m = 0; m < SPT; ++m)
#pragma unroll
          for (int v = 0; v < NV; ++v) ff_add(th[m][v], tl[m][v], p[m][v]);
      }
#pragma unroll
      for (int m = 0; m < SPT; ++m) cur[m] = nxt[m];
    }
  }
  // the group's partial sums, merged in a fixed tree (inactive lanes add 0)
#pragma unroll
  for (int o = 1; o < G; o <<= 1)
#pragma unroll
    for (int m = 0; m < SPT; ++m)
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const float oh = __shfl_xor_sync(0xffffffffu, th[m][v], o);
        const float ol = __shfl_xor_sync(0xffffffffu, tl[m][v], o);
        ff_add(th[m][v], tl[m][v], oh);
        tl[m][v] += ol;
      }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double loss = 0.0;
#pragma unroll
    for (int m = 0; m < SPT; ++m) {
      const int64_t s = sm[m];
      if (!act[m] && c == 0 && s < b) {   // a skipped (invalid) index contributes nothing
        rs[(size_t)s * K + k] = 0.0f;
        if (HV) hs[(size_t)s * K + k] = 0.0f;
      }
      if (act[m] && c == 0) {
        // with e = exp(-|t|): log(1 + e^t) - z t = log1p(e) + |t| [t and z
        // disagree] (the second term exact from the float-float t),
        // c = 1/(1 + e) or e/(1 + e), c (1 - c) = e / (1 + e)^2
        const bool zi = z[im[m]] != 0;
        const float tf = th[m][k] + tl[m][k];
        const float e = expf(-fabsf(tf));
        const float inv = 1.0f / (1.0f + e);
        const bool wrong = zi ? tf < 0.0f : tf > 0.0f;
        const double at = fabs((double)th[m][k] + (double)tl[m][k]);
        loss += (double)log1pf(e) + (wrong ? at : 0.0);
        const float cc = tf >= 0.0f ? inv : e * inv;
        rs[(size_t)s * K + k] = zi ? cc - 1.0f : cc;
        if (HV) {
          const float u = th[m][HV ? K + k : 0] + tl[m][HV ? K + k : 0];
          hs[(size_t)s * K + k] = e * inv * inv * u;
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, o);
    if (lane == 0) sloss[warp][k] = loss;
  }
  __syncthreads();
  if (threadIdx.x < K) {
    double t = 0.0;
    for (int w = 0; w < kLgThreads / 32; ++w) t += sloss[w][threadIdx.x];
    lossp[(size_t)blockIdx.x * K + threadIdx.x] = t;
  }
}

// Writes the warps' register sums to shared memory and adds them in warp
// order per feature (float-float) into the slice's FP64 partial.
__device__ __forceinline__ void lg_merge(const float (&acc)[32], float (&sh)[kLgThreads / 32][32][33],
                                         double* __restrict__ part, int n, int K, int sl, int k) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int t = 0; t < 32; ++t) sh[warp][t][lane] = acc[t];
  __syncthreads();
  // thread e (of 256) sums features e, e + 256, ... of the block's 1024
  for (int e = threadIdx.x; e < 1024; e += kLgThreads) {
    const int l = e >> 5, t = e & 31;   // word lane l, bit t
    const int j = 32 * (32 * blockIdx.x + l) + t;
    float hi = 0.0f, lo = 0.0f;   // float-float: the narrow FP64 pipe only converts the result
#pragma unroll
    for (int w = 0; w < kLgThreads / 32; ++w) ff_add(hi, lo, sh[w][t][l]);
    if (j < n) part[((size_t)sl * K + k) * n + j] = (double)hi + (double)lo;
  }
  __syncthreads();
}

// The adjoint's operands of sample s: its bits in word q (0 for an index
// outside the data set), its residual and its Hessian weight.
__device__ __forceinline__ void lg_adj_load(int64_t s, int64_t N, int nwp, int K, int k, int q,
                                            const int64_t* __restrict__ idx, const uint32_t* __restrict__ X,
                                            const float* __restrict__ rs, const float* __restrict__ hs,
                                            uint32_t& bits, float& r, float& hw) {
  const int64_t i = idx ? idx[s] : s;
  bits = (q < nwp && i >= 0 && i < N) ? X[(size_t)i * nwp + q] : 0u;
  r = rs[(size_t)s * K + k];
  hw = hs ? hs[(size_t)s * K + k] : 0.0f;
}

// Adjoint: block (word block wb, slice sl, vector k).  Lane l owns word
// 32 wb + l (features 32 (32 wb + l) + t); warp w adds the samples
// s = s0 + w, s0 + w + 8, ... of the slice.  part[sl][k][j] (FP64) gets the
// slice's sum of r x_j (and of h x_j in partH).
__global__ void __launch_bounds__(kLgThreads) k_lg_adj(int n, int nwp, int K, int64_t N, int64_t b,
                                                       const int64_t* __restrict__ idx,
                                                       const uint32_t* __restrict__ X, const float* __restrict__ rs,
                                                       const float* __restrict__ hs, double* __restrict__ partG,
                                                       double* __restrict__ partH) {
  __shared__ float sh[kLgThreads / 32][32][33];   // [warp][t][lane] (padded)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = 32 * blockIdx.x + lane;
  const int sl = blockIdx.y, k = blockIdx.z;
  const int64_t s0 = (int64_t)sl * kLgAdjSamples;
  const int64_t s1 = min(b, s0 + kLgAdjSamples);
  float g[32], h[32];
#pragma unroll
  for (int t = 0; t < 32; ++t) g[t] = h[t] = 0.0f;
  const bool want_h = hs != nullptr;
  // kB samples' bits and weights are loaded together, then added: enough
  // loads in flight per warp to cover the memory latency
  constexpr int kW = kLgThreads / 32, kB = 4;
  for (int64_t s = s0 + warp; s < s1; s += kB * kW) {
    uint32_t bits[kB];
    float r[kB], hw[kB];
#pragma unroll
    for (int u = 0; u < kB; ++u) {
      bits[u] = 0u;
      r[u] = hw[u] = 0.0f;
      if (s + u * kW < s1) lg_adj_load(s + u * kW, N, nwp, K, k, q, idx, X, rs, hs, bits[u], r[u], hw[u]);
    }
#pragma unroll
    for (int u = 0; u < kB; ++u)
#pragma unroll
      for (int t = 0; t < 32; ++t)
        if (bits[u] & (1u << t)) {
          g[t] += r[u];
          if (want_h) h[t] += hw[u];
        }
  }
  // merge the eight warps in warp order, one quantity at a time
  lg_merge(g, sh, partG, n, K, sl, k);
  if (want_h) lg_merge(h, sh, partH, n, K, sl, k);
}

// grad / hvp = (sum over slices) / b: one block per (32 features, vector,
// quantity); warp w adds the slices w, w + 8, ... and the eight warp sums
// are merged in warp order.  Block y = K * 2 (the F row) adds the forward
// blocks' loss sums for every k: F = (sum) / b.
__global__ void __launch_bounds__(256) k_lg_final(int n, int K, int nsl, int nfb, int64_t b,
                                                  const double* __restrict__ partG, const double* __restrict__ partH,
                                                  const double* __restrict__ lossp, double* __restrict__ F,
                                                  double* __restrict__ grad, double* __restrict__ hvp) {
  __shared__ double sh[8][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const double inv = 1.0 / (double)b;
  if (blockIdx.y == (unsigned)(2 * K)) {   // the objective
    if (blockIdx.x != 0) return;
    for (int k = warp; k < K; k += 8) {
      double t = 0.0;
      for (int fb = lane; fb < nfb; fb += 32) t += lossp[(size_t)fb * K + k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane == 0 && F) F[k] = t * inv;
    }
    return;
  }
  const int k = blockIdx.y >> 1, which = blockIdx.y & 1;
  const double* part = which ? partH : partG;
  double* out = which ? hvp : grad;
  if (!part || !out) return;
  const int j = 32 * blockIdx.x + lane;
  double t = 0.0;
  if (j < n)
    for (int sl = warp; sl < nsl; sl += 8) t += part[((size_t)sl * K + k) * n + j];
  sh[warp][lane] = t;
  __syncthreads();
  if (warp == 0 && j < n) {
    double u = 0.0;
#pragma unroll
    for (int w = 0; w < 8; ++w) u += sh[w][lane];
    out[(size_t)k * n + j] = u * inv;
  }
}

struct LgPlan {
  int nwp, nv, kchunk, nfb, nsl, g;
  size_t vec, rs, hs, lossp, partG, partH, total;
};

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

// One forward pass takes kchunk decisions (and their directions): the vectors
// must fit the shared-memory budget.
LgPlan lg_plan(int n, int64_t b, int K, int has_v) {
  LgPlan p;
  p.nwp = lg_pitch(n);
  const int per = has_v ? 2 : 1;
  int kc = kLgMaxVec / per;
  while (kc > 1 && kc * per * kLgWordPitch * p.nwp > kLgSmemFloats) --kc;
  p.kchunk = kc < K ? kc : K;
  p.nv = p.kchunk * per;
  // eight threads per point unless the points alone fill the GPU many times over
  p.g = b >= 64 * 1024 ? 1 : 8;
  const int64_t threads = p.g == 1 ? (b + 1) / 2 : b * p.g;   // (1 thread, 2 points) or (8 threads, 1 point)
  p.nfb = (int)((threads + kLgThreads - 1) / kLgThreads);
  p.nsl = (int)((b + kLgAdjSamples - 1) / kLgAdjSamples);
  size_t off = 0;
  p.vec = off; off = a256(off + 4 * (size_t)kLgMaxVec * n);
  p.rs = off; off = a256(off + 4 * (size_t)b * p.kchunk);
  p.hs = off; off = a256(off + (has_v ? 4 * (size_t)b * p.kchunk : 0));
  p.lossp = off; off = a256(off + 8 * (size_t)p.nfb * p.kchunk);
  p.partG = off; off = a256(off + 8 * (size_t)p.nsl * p.kchunk * n);
  p.partH = off; off = a256(off + (has_v ? 8 * (size_t)p.nsl * p.kchunk * n : 0));
  p.total = off;
  return p;
}

template <int KC, bool HV, int G, int SPT>
cudaError_t launch_fwd_g(const LgPlan& p, int n, int64_t N, int64_t b, const int64_t* idx, uint32_t* err,
                         const uint32_t* X, const uint8_t* z, const float* vec, float* rs, float* hs, double* lossp,
                         cudaStream_t st) {
  const size_t smem = sizeof(float) * KC * (HV ? 2 : 1) * kLgWordPitch * (size_t)p.nwp;
  cudaError_t e = cudaSuccess;
  if (smem > 48 * 1024)
    e = cudaFuncSetAttribute(k_lg_fwd<KC, HV, G, SPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_lg_fwd<KC, HV, G, SPT><<<p.nfb, kLgThreads, smem, st>>>(n, p.nwp, N, b, idx, err, X, z, vec, rs, hs, lossp);
  return cudaGetLastError();
}

template <int KC, bool HV>
cudaError_t launch_fwd(const LgPlan& p, int n, int64_t N, int64_t b, const int64_t* idx, uint32_t* err,
                       const uint32_t* X, const uint8_t* z, const float* vec, float* rs, float* hs, double* lossp,
                       cudaStream_t st) {
  if (p.g == 1) return launch_fwd_g<KC, HV, 1, 2>(p, n, N, b, idx, err, X, z, vec, rs, hs, lossp, st);
  return launch_fwd_g<KC, HV, 8, 1>(p, n, N, b, idx, err, X, z, vec, rs, hs, lossp, st);
}

template <bool HV>
cudaError_t launch_fwd_kc(int kc, const LgPlan& p, int n, int64_t N, int64_t b, const int64_t* idx, uint32_t* err,
                          const uint32_t* X, const uint8_t* z, const float* vec, float* rs, float* hs, double* lossp,
                          cudaStream_t st) {
  switch (kc) {
    case 1: return launch_fwd<1, HV>(p, n, N, b, idx, err, X, z, vec, rs, hs, lossp, st);
    case 2: return launch_fwd<2, HV>(p, n, N, b, idx, err, X, z, vec, rs, hs, lossp, st);
    case 3: return launch_fwd<3, HV>(p, n, N, b, idx, err, X, z, vec, rs, hs, lossp, st);
    case 4: return launch_fwd<4, HV>(p, n, N, b, idx, err, X, z, vec, rs, hs, lossp, st);
    default: break;
  }
  if (!HV) {
    switch (kc) {
      case 5: return launch_fwd<5, false>(p, n, N, b, idx, err, X, z, vec, rs, hs, lossp, st);
      case 6: return launch_fwd<6, false>(p, n, N, b, idx, err, X, z, vec, rs, hs, lossp, st);
      case 7: return launch_fwd<7, false>(p, n, N, b, idx, err, X, z, vec, rs, hs, lossp, st);
      case 8: return launch_fwd<8, false>(p, n, N, b, idx, err, X, z, vec, rs, hs, lossp, st);
      default: break;
    }
  }
  return cudaErrorInvalidValue;
}

saa_status lg_check(const saa_ctx* ctx, int n, int64_t N, int64_t b, int K) {
  if (!ctx) {
    set_error("saa_logistic: ctx is NULL");
    return SAA_EINVAL;
  }
  if (n < 1 || N < 1 || N > 0xffffffffll || b < 1 || K < 1) {
    set_error("saa_logistic: need n >= 1, 1 <= N < 2^32, b >= 1, K >= 1");
    return SAA_EINVAL;
  }
  if (kLgWordPitch * lg_pitch(n) > kLgSmemFloats) {
    set_error("saa_logistic: n too large for one forward pass (n <= 43648)");
    return SAA_EUNSUPPORTED;
  }
  return SAA_OK;
}

}  // namespace
}  // namespace saa

using namespace saa;

extern "C" int32_t saa_logistic_pitch(int32_t n) { return n < 1 ? 0 : lg_pitch(n); }

extern "C" saa_status saa_logistic_generate(saa_ctx* ctx, const saa_logistic* prob, int64_t i0, int64_t rows,
                                            uint32_t* X, uint8_t* z, void* stream) {
  saa::NvtxRange nvtx_range("saa_logistic_generate");
  if (!ctx || !prob) {
    set_error("saa_logistic_generate: ctx and prob must be non-NULL");
    return SAA_EINVAL;
  }
  if (prob->n < 1 || prob->N < 1 || prob->N > 0xffffffffll || i0 < 0 || rows < 0 || i0 + rows > prob->N || !X ||
      (((uintptr_t)X) & 15u) || (z && !prob->wstar)) {
    set_error("saa_logistic_generate: bad sizes, range or pointers (X 16-byte aligned; labels need wstar)");
    return SAA_EINVAL;
  }
  if (rows == 0) return SAA_OK;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != ctx->device) cudaSetDevice(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  const int nwp = lg_pitch(prob->n);
  const int64_t threads = rows * (nwp / 4);
  k_lg_features<<<(unsigned)((threads + kLgThreads - 1) / kLgThreads), kLgThreads, 0, st>>>(
      prob->n, nwp, prob->seed, prob->instance, i0, rows, X);
  cudaError_t e = cudaGetLastError();
  int launched = 1;
  if (e == cudaSuccess && z) {
    k_lg_labels<<<(unsigned)((rows * 32 + kLgThreads - 1) / kLgThreads), kLgThreads, 0, st>>>(
        prob->n, nwp, prob->seed, prob->instance, prob->flip, i0, rows, X, prob->wstar, z);
    e = cudaGetLastError();
    ++launched;
  }
  ctx->kernels += launched;
  if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
  return cuda_status(e, "saa_logistic_generate: launch");
}

extern "C" size_t saa_logistic_workspace_size(const saa_ctx* ctx, int32_t n, int64_t b, int32_t K, int has_v) {
  if (lg_check(ctx, n, 1, b, K) != SAA_OK) return 0;
  return lg_plan(n, b, K, has_v).total;
}

extern "C" saa_status saa_logistic_eval(saa_ctx* ctx, int32_t n, int64_t N, const uint32_t* X, const uint8_t* z,
                                        const int64_t* idx, int64_t b, int32_t K, const double* W, const double* V,
                                        double* F, double* grad, double* hvp, void* ws, size_t ws_bytes,
                                        void* stream) {
  saa::NvtxRange nvtx_range("saa_logistic_eval");
  if (!idx) b = N;
  saa_status s = lg_check(ctx, n, N, b, K);
  if (s != SAA_OK) return s;
  if (!X || (((uintptr_t)X) & 15u) || !z || !W || (hvp && !V) || !ws || (((uintptr_t)ws) & 255u)) {
    set_error("saa_logistic_eval: X (16-byte aligned), z, W, V (for hvp) and a 256-byte aligned ws are required");
    return SAA_EINVAL;
  }
  const int has_v = (V && hvp) ? 1 : 0;
  const LgPlan p = lg_plan(n, b, K, has_v);
  if (ws_bytes < p.total) {
    set_error("saa_logistic_eval: workspace smaller than saa_logistic_workspace_size()");
    return SAA_ENOMEM;
  }
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != ctx->device) cudaSetDevice(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  char* w = (char*)ws;
  float* vec = (float*)(w + p.vec);
  float* rs = (float*)(w + p.rs);
  float* hs = has_v ? (float*)(w + p.hs) : nullptr;
  double* lossp = (double*)(w + p.lossp);
  double* partG = (double*)(w + p.partG);
  double* partH = has_v ? (double*)(w + p.partH) : nullptr;
  cudaError_t e = cudaSuccess;
  int launched = 0;
  const bool want_adj = grad || hvp;
  // decisions in chunks that fit one forward pass
  for (int k0 = 0; e == cudaSuccess && k0 < K; k0 += p.kchunk) {
    const int kc = min(p.kchunk, K - k0);
    const int nv = kc * (has_v ? 2 : 1);
    k_lg_prep<<<(unsigned)(((int64_t)nv * n + 255) / 256), 256, 0, st>>>(kc, n, nv, W + (size_t)k0 * n,
                                                                        has_v ? V + (size_t)k0 * n : nullptr, vec);
    e = cudaGetLastError();
    if (e != cudaSuccess) break;
    const bool prof = ctx->prof_on && ctx->prof_n < 256;
    if (prof) cudaEventRecord(ctx->prof_ev[2 * ctx->prof_n], st);
    e = has_v ? launch_fwd_kc<true>(kc, p, n, N, b, idx, ctx->err, X, z, vec, rs, hs, lossp, st)
              : launch_fwd_kc<false>(kc, p, n, N, b, idx, ctx->err, X, z, vec, rs, hs, lossp, st);
    launched += 2;
    if (e == cudaSuccess && want_adj) {
      const dim3 grid((unsigned)((p.nwp + 31) / 32), (unsigned)p.nsl, (unsigned)kc);
      k_lg_adj<<<grid, kLgThreads, 0, st>>>(n, p.nwp, kc, N, b, idx, X, rs, has_v ? hs : nullptr, partG, partH);
      e = cudaGetLastError();
      ++launched;
    }
    if (prof) cudaEventRecord(ctx->prof_ev[2 * ctx->prof_n++ + 1], st);
    if (e == cudaSuccess) {
      const dim3 fgrid((unsigned)((n + 31) / 32), (unsigned)(2 * kc + 1));
      k_lg_final<<<fgrid, 256, 0, st>>>(n, kc, want_adj ? p.nsl : 0, p.nfb, b, want_adj ? partG : nullptr,
                                        has_v ? partH : nullptr, lossp, F ? F + k0 : nullptr,
                                        grad ? grad + (size_t)k0 * n : nullptr, hvp ? hvp + (size_t)k0 * n : nullptr);
      e = cudaGetLastError();
      ++launched;
    }
  }
  ctx->kernels += launched;
  if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
  return cuda_status(e, "saa_logistic_eval: launch");
}
