// simt_tile.cuh -- one scenario tile of the CUDA-core (FFMA / DFMA) SAA
// kernels, shared by the single-problem and the ragged-batch kernels.
//
// For the tile of scenarios i0 .. i0+nrow-1 (BM rows, zero-filled past nrow):
//   1. scales s_i (t law) and the tile A' = [s_i zhat_i]' into shared memory,
//      layout [d][BMP];
//   2. m~ partial sums per dimension into FP64 registers (macc);
//   3. per K-chunk of BN = 16 TN decisions: Q = A Y by register tiling
//      (TM x TN per thread), the S1/S2 column sums by a 16-lane shuffle tree into the
//      slot's FP64 partials, and for the gradient the adjoint tile A'Q
//      accumulated (Kahan) into the slot's partial G.
// Every partial element of a slot is owned by one thread, which writes it on
// the slot's first tile (first = true) and accumulates afterwards.
#pragma once
#include "gen.cuh"
#include "internal.cuh"

namespace saa {

template <typename T> struct Pad;
template <> struct Pad<float> { static constexpr int v = 4; };
template <> struct Pad<double> { static constexpr int v = 2; };

// TN decisions per thread column group: BN = 16 TN decisions per K-chunk
// (TN = 1 for K <= 16 so that narrow decision sets waste no FMAs).
template <typename T, int BM, int TN>
struct SimtSmem {
  static constexpr int BN = 16 * TN;
  static constexpr int BMP = BM + Pad<T>::v;
  static constexpr int QP = BN + 1;
  T* As;  // [d][BMP]
  T* Ys;  // [kDK][BN]
  T* Qs;  // [BM][QP]
  T* ss;  // [BM]
  __device__ SimtSmem(unsigned char* raw, int d) {
    As = reinterpret_cast<T*>(raw);
    Ys = As + (size_t)d * BMP;
    Qs = Ys + kDK * BN;
    ss = Qs + BM * QP;
  }
};

template <typename T, int BM, int TN>
__device__ __forceinline__ void simt_tile(const gen::Stream& st, int d, int law, int nu, uint32_t half, uint32_t i0,
                                          int nrow, int K, const T* __restrict__ Yt, const SimtSmem<T, BM, TN>& sm,
                                          double* macc, bool first, int want_grad, double* __restrict__ p_s1,
                                          double* __restrict__ p_s2, T* __restrict__ p_g, T* __restrict__ p_gc) {
  constexpr int TM = BM / 16;
  constexpr int BN = SimtSmem<T, BM, TN>::BN;
  constexpr int BMP = SimtSmem<T, BM, TN>::BMP;
  constexpr int QP = SimtSmem<T, BM, TN>::QP;
  constexpr int PC = gen::Gen<T>::kPerCall;
  T* As = sm.As;
  T* Ys = sm.Ys;
  T* Qs = sm.Qs;
  T* ss = sm.ss;
  const int tid = threadIdx.x;
  const int ty = tid & 15;  // scenario group
  const int tx = tid >> 4;  // decision group
  const int nb = (d + PC - 1) / PC;

  __syncthreads();
  if (tid < BM) ss[tid] = (tid < nrow) ? gen::Gen<T>::scale(st, i0 + tid, law, nu) : T(0);
  __syncthreads();
  for (int idx = tid; idx < nb * BM; idx += kThreads) {
    const int i = idx % BM;
    const int b = idx / BM;
    T z[PC];
    if (i < nrow) {
      gen::Gen<T>::block(st, (uint32_t)b, i0 + i, gen::is_lognormal(law, i0 + i, half), z);
      const T s = ss[i];
#pragma unroll
      for (int q = 0; q < PC; ++q) z[q] *= s;
    } else {
#pragma unroll
      for (int q = 0; q < PC; ++q) z[q] = T(0);
    }
#pragma unroll
    for (int q = 0; q < PC; ++q) {
      const int j = b * PC + q;
      if (j < d) As[(size_t)j * BMP + i] = z[q];
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kMaxDimSimt / kThreads; ++r) {
    const int j = tid + r * kThreads;
    if (j < d) {
      T sum = T(0);
      for (int i = 0; i < nrow; ++i) sum += As[(size_t)j * BMP + i];
      macc[r] += (double)sum;
    }
  }

  for (int k0 = 0; k0 < K; k0 += BN) {
    T acc[TM][TN];
#pragma unroll
    for (int m = 0; m < TM; ++m)
#pragma unroll
      for (int n = 0; n < TN; ++n) acc[m][n] = T(0);

    for (int j0 = 0; j0 < d; j0 += kDK) {
      __syncthreads();
      for (int idx = tid; idx < kDK * BN; idx += kThreads) {
        const int jj = idx / BN, kk = idx % BN;
        const int j = j0 + jj, k = k0 + kk;
        Ys[idx] = (j < d && k < K) ? Yt[(size_t)j * K + k] : T(0);
      }
      __syncthreads();
      const int jmax = min(kDK, d - j0);
      for (int jj = 0; jj < jmax; ++jj) {
        const T* arow = As + (size_t)(j0 + jj) * BMP + ty * TM;
        const T* yrow = Ys + jj * BN + tx * TN;
        T a[TM], y[TN];
#pragma unroll
        for (int m = 0; m < TM; ++m) a[m] = arow[m];
#pragma unroll
        for (int n = 0; n < TN; ++n) y[n] = yrow[n];
#pragma unroll
        for (int m = 0; m < TM; ++m)
#pragma unroll
          for (int n = 0; n < TN; ++n) acc[m][n] = fma(a[m], y[n], acc[m][n]);
      }
    }

    // S1 / S2 over the tile's rows: own rows, then the 16 lanes sharing tx.
#pragma unroll
    for (int n = 0; n < TN; ++n) {
      T s1 = T(0), s2 = T(0);
#pragma unroll
      for (int m = 0; m < TM; ++m) {
        s1 += acc[m][n];
        s2 = fma(acc[m][n], acc[m][n], s2);
      }
#pragma unroll
      for (int off = 8; off > 0; off >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, off);
        s2 += __shfl_xor_sync(0xffffffffu, s2, off);
      }
      const int k = k0 + tx * TN + n;
      if (ty == 0 && k < K) {
        p_s1[k] = first ? (double)s1 : p_s1[k] + (double)s1;
        p_s2[k] = first ? (double)s2 : p_s2[k] + (double)s2;
      }
    }

    if (want_grad) {
      __syncthreads();
#pragma unroll
      for (int m = 0; m < TM; ++m)
#pragma unroll
        for (int n = 0; n < TN; ++n) Qs[(ty * TM + m) * QP + tx * TN + n] = acc[m][n];
      __syncthreads();
      for (int jd0 = 0; jd0 < d; jd0 += 64) {
        T g[4][TN];
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int n = 0; n < TN; ++n) g[q][n] = T(0);
        for (int i = 0; i < nrow; ++i) {
          T a[4], qv[TN];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int j = jd0 + ty + 16 * q;
            a[q] = (j < d) ? As[(size_t)j * BMP + i] : T(0);
          }
#pragma unroll
          for (int n = 0; n < TN; ++n) qv[n] = Qs[i * QP + tx * TN + n];
#pragma unroll
          for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int n = 0; n < TN; ++n) g[q][n] = fma(a[q], qv[n], g[q][n]);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int j = jd0 + ty + 16 * q;
#pragma unroll
          for (int n = 0; n < TN; ++n) {
            const int k = k0 + tx * TN + n;
            if (j < d && k < K) {
              const size_t e = (size_t)k * d + j;
              if (first) {
                p_g[e] = g[q][n];
                p_gc[e] = T(0);
              } else {  // Kahan: the partial carries its lost low part in p_gc
                const T y = g[q][n] - p_gc[e];
                const T s = p_g[e];
                const T t = s + y;
                p_gc[e] = (t - s) - y;
                p_g[e] = t;
              }
            }
          }
        }
      }
    }
  }
}

}  // namespace saa
