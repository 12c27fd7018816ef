// batched.cu -- a ragged batch of independent SAA problems (Eq. 4 for each,
// Sec. 3.1) in one persistent launch.
//
// Each problem b has its own dimension d_b, sample count N_b, decisions K_b,
// law and Philox stream.  Its scenario range is cut into chunks ("items") of
// a fixed number of tiles; a persistent grid pulls items from an atomic
// counter (dynamic load balance across problems of very different sizes),
// and every item writes its own partial slot (S1, S2 per decision and m~ per
// dimension), so the result does not depend on which CTA took which item.
// A batched prologue computes every y_k = C_b'w_k; a finalize block per
// problem merges that problem's item partials in item order.  The tile work
// itself is the CUDA-core tile of the single-problem kernel (simt_tile).
// With gradients, every item also keeps Kahan-carried partials of
// G_k = sum_i a_i Q_ik, and two more kernels form u_k and grad_k = C u_k - mu.
//
// saa_batch_create plans a batch once (tile shape by the autotuner, the
// descriptor tables uploaded) and captures its launch sequence in a CUDA
// graph; saa_batch_launch replays that graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "gen.cuh"
#include "internal.cuh"
#include "simt_tile.cuh"

namespace saa {

struct BInst {
  int d, K, law, nu;
  uint32_t N, instance, epoch, pad;
  uint64_t seed;
  double lambda;
  const double* mu;
  const double* chol;
  const double* X;
  double* f;
  double* pbar;
  double* var;
  int64_t y_off;     // element offset of Yt ([d][K], contraction precision)
  int64_t y64_off;   // double offset of Y64 ([K][d])
  int64_t c_off;     // double offset of c ([K])
  int64_t part_off;  // double offset of this problem's item partials
  int item0, nitems;
  int pblock0, pad2;  // first prologue block
  double* grad;       // [K][d] output, or NULL (gradient batches)
  int64_t gpart_off;  // element offset of the item gradient partials: [nitems][2][K][d]
  int64_t u_off;      // double offset of u ([K][d])
  int ublock0, oblock0;  // first block of the u and C u kernels
};

struct BItem {
  int inst;
  uint32_t i0, n;
  int slot;  // item index within its problem
};

static_assert(sizeof(BInst) % 8 == 0, "descriptor alignment");

// ------------------------------------------------------------ prologue ---
constexpr int kBK = 4;   // decisions per prologue block

__device__ __forceinline__ int find_inst(const BInst* insts, int B, int blk) {
  int lo = 0, hi = B - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (insts[mid].pblock0 <= blk) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <typename T>
__global__ void __launch_bounds__(256) k_batched_prologue(const BInst* __restrict__ insts, int B, T* __restrict__ Yf,
                                                          double* __restrict__ Y64, double* __restrict__ cbuf) {
  extern __shared__ double wsm[];   // [kBK][d]
  __shared__ double red[8][kBK][32];
  const int b = find_inst(insts, B, blockIdx.x);
  const BInst in = insts[b];
  const int d = in.d, K = in.K;
  const int nj = (d + 31) / 32;
  const int local = blockIdx.x - in.pblock0;
  const int k0 = (local / nj) * kBK;
  const int jc = (local % nj) * 32;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int idx = threadIdx.x; idx < kBK * d; idx += blockDim.x) {
    const int kk = idx / d, l = idx % d;
    wsm[idx] = (k0 + kk < K) ? in.X[(size_t)(k0 + kk) * d + l] : 0.0;
  }
  __syncthreads();
  const int j = jc + lane;
  double acc[kBK];
#pragma unroll
  for (int kk = 0; kk < kBK; ++kk) acc[kk] = 0.0;
  if (j < d) {
#pragma unroll 4
    for (int l = jc + warp; l < d; l += 8) {
      const double cl = (l >= j) ? in.chol[(size_t)l * d + j] : 0.0;
#pragma unroll
      for (int kk = 0; kk < kBK; ++kk) acc[kk] = fma(cl, wsm[kk * d + l], acc[kk]);
    }
  }
#pragma unroll
  for (int kk = 0; kk < kBK; ++kk) red[warp][kk][lane] = acc[kk];
  __syncthreads();
  if (threadIdx.x < kBK * 32) {
    const int kk = threadIdx.x >> 5, jj = threadIdx.x & 31;
    const int k = k0 + kk, jo = jc + jj;
    if (k < K && jo < d) {
      double y = 0.0;
#pragma unroll
      for (int w = 0; w < 8; ++w) y += red[w][kk][jj];
      Y64[in.y64_off + (size_t)k * d + jo] = y;
      Yf[in.y_off + (size_t)jo * K + k] = (T)y;
    }
  }
  if (jc == 0 && warp < kBK && k0 + warp < K) {
    double s = 0.0;
    for (int l = lane; l < d; l += 32) s = fma(in.mu[l], wsm[warp * d + l], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) cbuf[in.c_off + k0 + warp] = s;
  }
}

// ---------------------------------------------------------------- main ---
template <typename T, int BM, int TN>
__global__ void __launch_bounds__(kThreads, 2) k_batched_main(const BInst* __restrict__ insts,
                                                              const BItem* __restrict__ items, int nitems,
                                                              const T* __restrict__ Yf, double* __restrict__ parts,
                                                              T* __restrict__ gparts, int want_grad,
                                                              uint32_t* __restrict__ counter) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_item;
  for (;;) {
    __syncthreads();   // the previous item's readers of s_item are done
    if (threadIdx.x == 0) s_item = (int)atomicAdd(counter, 1u);
    __syncthreads();
    const int it = s_item;
    if (it >= nitems) break;
    const BItem item = items[it];
    const BInst& in = insts[item.inst];
    const int d = in.d, K = in.K;
    const SimtSmem<T, BM, TN> sm(smem_raw, d);
    const gen::Stream st = gen::make_stream(in.seed, in.epoch, in.instance);
    double macc[kMaxDimSimt / kThreads];
#pragma unroll
    for (int r = 0; r < kMaxDimSimt / kThreads; ++r) macc[r] = 0.0;
    double* slot = parts + in.part_off + (size_t)item.slot * (2 * K + d);
    T* gslot = want_grad ? gparts + in.gpart_off + (size_t)item.slot * 2 * K * d : nullptr;
    const T* Yt = Yf + in.y_off;
    bool first = true;
    for (uint32_t off = 0; off < item.n; off += BM) {
      const int nrow = (int)min((uint32_t)BM, item.n - off);
      simt_tile<T, BM, TN>(st, d, in.law, in.nu, in.N / 2u, item.i0 + off, nrow, K, Yt, sm, macc, first, want_grad,
                           slot, slot + K, gslot, want_grad ? gslot + (size_t)K * d : nullptr);
      first = false;
    }
#pragma unroll
    for (int r = 0; r < kMaxDimSimt / kThreads; ++r) {
      const int j = threadIdx.x + r * kThreads;
      if (j < d) slot[2 * K + j] = macc[r];
    }
  }
}

// ----------------------------------------------------- fused value path ---
// Value-only batches with K_b <= 16 (the ragged workloads): no tile of
// samples is stored.  Each thread draws one scenario and accumulates its K
// dot products zhat_i'y_k while drawing, with y read from a padded copy in
// shared memory four decisions at a time; the 32 lanes of a warp read the
// same row of y, a broadcast.  The t-law scale s_i is applied once per
// scenario.  (The group reduction below is kept general: G = 1 here.)  S1 and S2 collect in
// shared memory per pass of 256/G scenarios: 16 parts per decision sum the
// pass in FP32 and carry the pass totals in FP64, and the parts are merged
// in order at the end of the item, so the result is deterministic.
constexpr int kFusedK = 16;

// four consecutive decisions' y_jk from shared memory (16-byte aligned)
__device__ __forceinline__ void load4(const float* p, float (&v)[4]) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void load4(const double* p, double (&v)[4]) {
  const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 2) k_batched_fused(
    const BInst* __restrict__ insts, const BItem* __restrict__ items, int nitems, const T* __restrict__ Yf,
    double* __restrict__ parts, uint32_t* __restrict__ counter) {
  constexpr int PC = gen::Gen<T>::kPerCall;
  extern __shared__ __align__(16) unsigned char fsm_raw[];
  T* Ys = reinterpret_cast<T*>(fsm_raw);   // [d][kFusedK] (decisions padded with zeros)
  __shared__ T Qs[256][kFusedK + 1];       // one row per scenario of the pass
  __shared__ double red[2][16][kFusedK];
  __shared__ int s_item;
  const int tid = threadIdx.x;
  const int kq = tid % kFusedK, part = tid / kFusedK;   // S1/S2 collection role
  for (;;) {
    __syncthreads();
    if (tid == 0) s_item = (int)atomicAdd(counter, 1u);
    __syncthreads();
    const int it = s_item;
    if (it >= nitems) break;
    const BItem item = items[it];
    const BInst& in = insts[item.inst];
    const int d = in.d, K = in.K;
    const int nb = (d + PC - 1) / PC;
    // one thread per scenario: the 32 lanes of a warp draw 32 scenarios
    // and read the same row of y (a shared-memory broadcast)
    const int G = 1;
    const int spp = 256 / G;   // scenarios per pass
    const int g = tid % G, sl = tid / G;
    for (int e = tid; e < d * kFusedK; e += 256) {
      const int j = e / kFusedK, k = e % kFusedK;
      Ys[e] = (k < K) ? Yf[in.y_off + (size_t)j * K + k] : T(0);
    }
    const gen::Stream st = gen::make_stream(in.seed, in.epoch, in.instance);
    const uint32_t half = in.N / 2u;
    const int kg = (K + 3) / 4;   // groups of four decisions (uniform over the CTA)
    double d1 = 0.0, d2 = 0.0;   // pass totals of this thread's (decision kq, part)
    for (uint32_t base = 0; base < item.n; base += (uint32_t)spp) {
      __syncthreads();   // Ys staged / the previous pass's Qs consumed
      const uint32_t r = base + (uint32_t)sl;
      const bool live = r < item.n;
      const uint32_t i = item.i0 + r;
      T q[kFusedK];
#pragma unroll
      for (int k = 0; k < kFusedK; ++k) q[k] = T(0);
      if (live) {
        const bool logn = gen::is_lognormal(in.law, i, half);
        for (int b = g; b < nb; b += G) {
          T z[PC];
          gen::Gen<T>::block(st, (uint32_t)b, i, logn, z);
#pragma unroll
          for (int e = 0; e < PC; ++e) {
            const int j = b * PC + e;
            if (j < d) {
              const T* yj = Ys + (size_t)j * kFusedK;
#pragma unroll
              for (int c = 0; c < kFusedK / 4; ++c)
                if (c < kg) {
                  T y4[4];
                  load4(yj + 4 * c, y4);
#pragma unroll
                  for (int u = 0; u < 4; ++u) q[4 * c + u] = fma(z[e], y4[u], q[4 * c + u]);
                }
            }
          }
        }
      }
      // the G threads of a scenario are consecutive lanes of one warp
      for (int o = G >> 1; o >= 1; o >>= 1) {
#pragma unroll
        for (int c = 0; c < kFusedK / 4; ++c)
          if (c < kg) {
#pragma unroll
            for (int u = 0; u < 4; ++u) q[4 * c + u] += __shfl_xor_sync(0xffffffffu, q[4 * c + u], o);
          }
      }
      if (g == 0) {
        const T s = (live && in.law == SAA_LAW_STUDENT_T) ? gen::Gen<T>::scale(st, i, in.law, in.nu) : T(1);
#pragma unroll
        for (int k = 0; k < kFusedK; ++k) Qs[sl][k] = live ? q[k] * s : T(0);
      }
      __syncthreads();
      if (kq < K) {
        T f1 = T(0), f2 = T(0);
        for (int x = part; x < spp; x += 16) {
          const T v = Qs[x][kq];
          f1 += v;
          f2 = fma(v, v, f2);
        }
        d1 += (double)f1;
        d2 += (double)f2;
      }
    }
    red[0][part][kq] = d1;
    red[1][part][kq] = d2;
    __syncthreads();
    if (tid < K) {
      double s1 = 0.0, s2 = 0.0;
      for (int pp = 0; pp < 16; ++pp) {
        s1 += red[0][pp][tid];
        s2 += red[1][pp][tid];
      }
      double* slot = parts + in.part_off + (size_t)item.slot * (2 * K + d);
      slot[tid] = s1;
      slot[K + tid] = s2;
    }
  }
}

// ------------------------------------------------------------ finalize ---
__device__ __forceinline__ void nsum_add(double& s, double& c, double x) {
  const double t = s + x;
  if (fabs(s) >= fabs(x))
    c += (s - t) + x;
  else
    c += (x - t) + s;
  s = t;
}

// One block per problem: merge its item partials in item order, then
// pbar_k = c_k + S1_k/N, V_k = (S2_k - S1_k^2/N)/(N-1), f_k = lambda V_k - pbar_k.
__global__ void k_batched_finalize(const BInst* __restrict__ insts, const double* __restrict__ parts,
                                   const double* __restrict__ cbuf) {
  const BInst in = insts[blockIdx.x];
  const int K = in.K, d = in.d;
  const int stride = 2 * K + d;
  const double* p = parts + in.part_off;
  const double N = (double)in.N;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    double s1 = 0.0, c1 = 0.0, s2 = 0.0, c2 = 0.0;
    for (int t = 0; t < in.nitems; ++t) {
      nsum_add(s1, c1, p[(size_t)t * stride + k]);
      nsum_add(s2, c2, p[(size_t)t * stride + K + k]);
    }
    const double S1 = s1 + c1, S2 = s2 + c2;
    const double qbar = S1 / N;
    const double pb = cbuf[in.c_off + k] + qbar;
    const double V = (S2 - S1 * qbar) / (N - 1.0);
    in.f[k] = in.lambda * V - pb;
    if (in.pbar) in.pbar[k] = pb;
    if (in.var) in.var[k] = V;
  }
}

// ------------------------------------------------------------- gradient ---
__device__ __forceinline__ int find_block(const BInst* insts, int B, int blk, bool outer) {
  int lo = 0, hi = B - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if ((outer ? insts[mid].oblock0 : insts[mid].ublock0) <= blk) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// u_kj = lambda 2/(N-1) (G_kj - S1_k m_j) - m_j for 32 dimensions of one
// decision of one problem: warp w sums items w, w + 8, ... of G (float-float
// pairs for FP32 partials, Neumaier for FP64), merged in warp order; S1_k
// and m_j are summed over items in item order.
template <typename T>
__global__ void __launch_bounds__(256) k_batched_grad_u(const BInst* __restrict__ insts, int B,
                                                        const double* __restrict__ parts,
                                                        const T* __restrict__ gparts, double* __restrict__ ubuf) {
  __shared__ double sh_s[8][32], sh_c[8][32];
  const int b = find_block(insts, B, blockIdx.x, false);
  const BInst in = insts[b];
  const int d = in.d, K = in.K;
  const int nj = (d + 31) / 32;
  const int local = blockIdx.x - in.ublock0;
  const int k = local / nj, jc = (local % nj) * 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = jc + lane;
  const size_t kd = (size_t)K * d;
  const T* gp = gparts + in.gpart_off;
  double s = 0.0, c = 0.0;
  if (j < d) {
    if constexpr (sizeof(T) == 4) {
      float S = 0.0f, E = 0.0f;
      for (int t = warp; t < in.nitems; t += 8) {
        const size_t e = (size_t)t * 2 * kd + (size_t)k * d + j;
        const float x = (float)gp[e], xc = (float)gp[e + kd];
        const float tt = __fadd_rn(S, x);
        const float bb = __fsub_rn(tt, S);
        const float err = __fadd_rn(__fsub_rn(S, __fsub_rn(tt, bb)), __fsub_rn(x, bb));
        S = tt;
        E = __fadd_rn(E, __fsub_rn(err, xc));
      }
      s = (double)S;
      c = (double)E;
    } else {
      for (int t = warp; t < in.nitems; t += 8) {
        const size_t e = (size_t)t * 2 * kd + (size_t)k * d + j;
        nsum_add(s, c, (double)gp[e]);
        nsum_add(s, c, -(double)gp[e + kd]);
      }
    }
  }
  sh_s[warp][lane] = s;
  sh_c[warp][lane] = c;
  __syncthreads();
  if (warp == 0 && j < d) {
    double G = 0.0, Gc = 0.0;
    for (int w = 0; w < 8; ++w) {
      nsum_add(G, Gc, sh_s[w][lane]);
      nsum_add(G, Gc, sh_c[w][lane]);
    }
    const int stride = 2 * K + d;
    const double* p = parts + in.part_off;
    double s1 = 0.0, c1 = 0.0, m = 0.0, cm = 0.0;
    for (int t = 0; t < in.nitems; ++t) {
      nsum_add(s1, c1, p[(size_t)t * stride + k]);
      nsum_add(m, cm, p[(size_t)t * stride + 2 * K + j]);
    }
    const double N = (double)in.N;
    const double mj = (m + cm) / N;
    ubuf[in.u_off + (size_t)k * d + j] = in.lambda * (2.0 / (N - 1.0)) * ((G + Gc) - (s1 + c1) * mj) - mj;
  }
}

// grad_kj = sum_{l <= j} C_jl u_kl - mu_j: one warp per (k, j) of one problem.
__global__ void __launch_bounds__(256) k_batched_grad_out(const BInst* __restrict__ insts, int B,
                                                          const double* __restrict__ ubuf) {
  const int b = find_block(insts, B, blockIdx.x, true);
  const BInst in = insts[b];
  const int d = in.d;
  const int lane = threadIdx.x & 31;
  const int64_t row = (int64_t)(blockIdx.x - in.oblock0) * 8 + (threadIdx.x >> 5);
  if (row >= (int64_t)in.K * d) return;
  const int k = (int)(row / d), j = (int)(row % d);
  const double* cj = in.chol + (size_t)j * d;
  const double* uk = ubuf + in.u_off + (size_t)k * d;
  double acc = 0.0;
  for (int l = lane; l <= j; l += 32) acc = fma(cj[l], uk[l], acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) in.grad[(size_t)k * d + j] = acc - in.mu[j];
}

// ------------------------------------------------------------------ host ---
struct BatchLayout {
  size_t insts, items, yf, y64, c, parts, gparts, u, counter, total;
  int nitems, pblocks, ublocks, oblocks, dmax, kmax;
};

static size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

// Fills the descriptor tables (host) and the workspace layout for a chunk of
// `chunk_tiles` tiles of BM scenarios per item.
static BatchLayout plan_batch(int B, const saa_problem* probs, const int32_t* K, const double* const* X,
                              double* const* f, double* const* pbar, double* const* var, double* const* grad,
                              int want_grad, int es, int bm, int chunk_tiles, std::vector<BInst>* hi,
                              std::vector<BItem>* hitems) {
  BatchLayout L;
  std::memset(&L, 0, sizeof(L));
  int64_t yf = 0, y64 = 0, c = 0, parts = 0, gparts = 0, u = 0;
  int nitems = 0, pblocks = 0, ublocks = 0, oblocks = 0, dmax = 1, kmax = 1;
  const uint32_t chunk = (uint32_t)(bm * chunk_tiles);
  if (hi) hi->resize(B);
  if (hitems) hitems->clear();
  for (int b = 0; b < B; ++b) {
    const saa_problem& p = probs[b];
    const int d = p.d, k = K[b];
    const int nit = (int)((p.N + chunk - 1) / chunk);
    if (hi) {
      BInst& in = (*hi)[b];
      std::memset(&in, 0, sizeof(in));
      in.d = d; in.K = k; in.law = p.law; in.nu = p.nu;
      in.N = (uint32_t)p.N; in.instance = p.instance; in.epoch = p.epoch;
      in.seed = p.seed; in.lambda = p.lambda;
      in.mu = p.mu; in.chol = p.chol; in.X = X[b];
      in.f = f[b]; in.pbar = pbar ? pbar[b] : nullptr; in.var = var ? var[b] : nullptr;
      in.y_off = yf; in.y64_off = y64; in.c_off = c; in.part_off = parts;
      in.item0 = nitems; in.nitems = nit; in.pblock0 = pblocks;
      in.grad = (want_grad && grad) ? grad[b] : nullptr;
      in.gpart_off = gparts; in.u_off = u; in.ublock0 = ublocks; in.oblock0 = oblocks;
    }
    if (hitems)
      for (int t = 0; t < nit; ++t) {
        BItem it;
        it.inst = b;
        it.i0 = (uint32_t)t * chunk;
        it.n = (uint32_t)std::min<int64_t>(chunk, p.N - (int64_t)t * chunk);
        it.slot = t;
        hitems->push_back(it);
      }
    yf += (int64_t)d * k;
    y64 += (int64_t)d * k;
    c += k;
    parts += (int64_t)nit * (2 * k + d);
    if (want_grad) {
      gparts += (int64_t)nit * 2 * k * d;
      u += (int64_t)k * d;
      ublocks += k * ((d + 31) / 32);
      oblocks += (int)(((int64_t)k * d + 7) / 8);
    }
    nitems += nit;
    pblocks += ((k + kBK - 1) / kBK) * ((d + 31) / 32);
    dmax = std::max(dmax, d);
    kmax = std::max(kmax, k);
  }
  size_t off = 0;
  L.insts = off; off = al(off + sizeof(BInst) * (size_t)B);
  L.items = off; off = al(off + sizeof(BItem) * (size_t)nitems);
  L.yf = off; off = al(off + (size_t)es * yf);
  L.y64 = off; off = al(off + 8 * (size_t)y64);
  L.c = off; off = al(off + 8 * (size_t)c);
  L.parts = off; off = al(off + 8 * (size_t)parts);
  L.gparts = off; off = al(off + (size_t)es * gparts);
  L.u = off; off = al(off + 8 * (size_t)u);
  L.counter = off; off = al(off + 8);
  L.total = off;
  L.nitems = nitems;
  L.pblocks = pblocks;
  L.ublocks = ublocks;
  L.oblocks = oblocks;
  L.dmax = dmax;
  L.kmax = kmax;
  return L;
}

template <typename T, int BM, int TN>
static cudaError_t launch_main(const saa_ctx* ctx, const BatchLayout& L, char* ws, int want_grad, cudaStream_t st) {
  const int prec = sizeof(T) == 8 ? SAA_FP64 : SAA_FP32;
  const int smem = (int)simt_smem(prec, L.dmax, BM, TN);
  auto kern = k_batched_main<T, BM, TN>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, smem);
  if (e != cudaSuccess) return e;
  const int grid = std::max(1, std::min(L.nitems, ctx->sm_count * std::max(occ, 1)));
  e = cudaMemsetAsync(ws + L.counter, 0, 8, st);
  if (e != cudaSuccess) return e;
  kern<<<grid, kThreads, smem, st>>>((const BInst*)(ws + L.insts), (const BItem*)(ws + L.items), L.nitems,
                                     (const T*)(ws + L.yf), (double*)(ws + L.parts), (T*)(ws + L.gparts), want_grad,
                                     (uint32_t*)(ws + L.counter));
  return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_fused(const saa_ctx* ctx, const BatchLayout& L, char* ws, cudaStream_t st) {
  const int smem = (int)(sizeof(T) * (size_t)L.dmax * kFusedK);
  auto kern = k_batched_fused<T>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 256, smem);
  if (e != cudaSuccess) return e;
  const int grid = std::max(1, std::min(L.nitems, ctx->sm_count * std::max(occ, 1)));
  e = cudaMemsetAsync(ws + L.counter, 0, 8, st);
  if (e != cudaSuccess) return e;
  kern<<<grid, 256, smem, st>>>((const BInst*)(ws + L.insts), (const BItem*)(ws + L.items), L.nitems,
                                (const T*)(ws + L.yf), (double*)(ws + L.parts), (uint32_t*)(ws + L.counter));
  return cudaGetLastError();
}

}  // namespace saa

using namespace saa;

namespace {

constexpr int kChunkChoices[3] = {16, 32, 64};   // tiles per item

struct TuneEntry {
  uint64_t key;
  int bm, chunk;
};
std::vector<TuneEntry> g_tune;   // per process: (batch-shape key) -> chosen tile shape
std::mutex g_tune_mu;

uint64_t shape_key(int B, const saa_problem* probs, const int32_t* K, int prec, int device) {
  uint64_t h = 1469598103934665603ull ^ (uint64_t)device ^ ((uint64_t)prec << 8) ^ ((uint64_t)B << 16);
  for (int b = 0; b < B; ++b) {
    h = (h ^ (uint64_t)probs[b].d) * 1099511628211ull;
    h = (h ^ (uint64_t)probs[b].N) * 1099511628211ull;
    h = (h ^ (uint64_t)K[b]) * 1099511628211ull;
  }
  return h;
}

saa_status validate(int B, const saa_problem* probs, const int32_t* K, const double* const* X, double* const* f,
                    saa_prec prec) {
  if (B < 1 || !probs || !K || !X || !f) {
    set_error("saa_eval_batched: need B >= 1 and non-NULL descriptor arrays");
    return SAA_EINVAL;
  }
  if (prec != SAA_FP32 && prec != SAA_FP64) {
    set_error("saa_eval_batched: SAA_FP32 or SAA_FP64");
    return SAA_EUNSUPPORTED;
  }
  for (int b = 0; b < B; ++b) {
    const saa_problem& p = probs[b];
    if (p.d < 1 || p.d > kMaxDimSimt || p.N < 2 || p.N > 0xffffffffll || p.law < 0 || p.law > 3 ||
        (p.law == SAA_LAW_STUDENT_T && (p.nu < 2 || (p.nu & 1) || p.nu > 64)) || p.reserved != 0 || !p.mu ||
        !p.chol || K[b] < 1 || K[b] > 65535 || !X[b] || !f[b]) {
      set_error("saa_eval_batched: invalid problem " + std::to_string(b));
      return SAA_EINVAL;
    }
  }
  return SAA_OK;
}

int pick_bm(int prec, int dmax) { return (prec == SAA_FP64) ? (dmax <= 256 ? 64 : 32) : (dmax <= 512 ? 64 : 32); }

}  // namespace

// The launch sequence of a planned batch (capturable): prologue, the
// persistent main kernel, the value finalize and, with gradients, the u and
// C u kernels.  Returns the number of kernels launched in *nk.
static saa_status launch_sequence(saa_ctx* ctx, int B, const BatchLayout& L, saa_prec prec, int bm, int want_grad,
                                  char* w, cudaStream_t st, int* nk) {
  const size_t psmem = sizeof(double) * kBK * L.dmax;
  if (prec == SAA_FP64) {
    if (psmem > 48 * 1024)
      cudaFuncSetAttribute(k_batched_prologue<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psmem);
    k_batched_prologue<double><<<L.pblocks, 256, psmem, st>>>((const BInst*)(w + L.insts), B, (double*)(w + L.yf),
                                                              (double*)(w + L.y64), (double*)(w + L.c));
  } else {
    if (psmem > 48 * 1024)
      cudaFuncSetAttribute(k_batched_prologue<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psmem);
    k_batched_prologue<float><<<L.pblocks, 256, psmem, st>>>((const BInst*)(w + L.insts), B, (float*)(w + L.yf),
                                                             (double*)(w + L.y64), (double*)(w + L.c));
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e, "batched prologue launch");
  const bool narrow = simt_tn(L.kmax) == 1;
  if (!want_grad && L.kmax <= kFusedK)
    e = (prec == SAA_FP64) ? launch_fused<double>(ctx, L, w, st) : launch_fused<float>(ctx, L, w, st);
  else if (prec == SAA_FP64)
    e = (bm == 64) ? (narrow ? launch_main<double, 64, 1>(ctx, L, w, want_grad, st)
                             : launch_main<double, 64, 4>(ctx, L, w, want_grad, st))
                   : (narrow ? launch_main<double, 32, 1>(ctx, L, w, want_grad, st)
                             : launch_main<double, 32, 4>(ctx, L, w, want_grad, st));
  else
    e = (bm == 64) ? (narrow ? launch_main<float, 64, 1>(ctx, L, w, want_grad, st)
                             : launch_main<float, 64, 4>(ctx, L, w, want_grad, st))
                   : (narrow ? launch_main<float, 32, 1>(ctx, L, w, want_grad, st)
                             : launch_main<float, 32, 4>(ctx, L, w, want_grad, st));
  if (e != cudaSuccess) return cuda_status(e, "batched sample kernel launch");
  k_batched_finalize<<<B, 64, 0, st>>>((const BInst*)(w + L.insts), (const double*)(w + L.parts),
                                       (const double*)(w + L.c));
  *nk = 3;
  if (want_grad && L.ublocks > 0) {
    if (prec == SAA_FP64)
      k_batched_grad_u<double><<<L.ublocks, 256, 0, st>>>((const BInst*)(w + L.insts), B,
                                                          (const double*)(w + L.parts),
                                                          (const double*)(w + L.gparts), (double*)(w + L.u));
    else
      k_batched_grad_u<float><<<L.ublocks, 256, 0, st>>>((const BInst*)(w + L.insts), B, (const double*)(w + L.parts),
                                                         (const float*)(w + L.gparts), (double*)(w + L.u));
    k_batched_grad_out<<<L.oblocks, 256, 0, st>>>((const BInst*)(w + L.insts), B, (const double*)(w + L.u));
    *nk += 2;
  }
  return cuda_status(cudaGetLastError(), "batched finalize launch");
}

// Plans the batch with tile shape (bm, chunk), optionally uploads its
// descriptor tables through the context's pinned staging buffer, and
// launches it.
static saa_status run_batch(saa_ctx* ctx, int B, const saa_problem* probs, const int32_t* K, const double* const* X,
                            saa_prec prec, double* const* f, double* const* pbar, double* const* var,
                            double* const* grad, int want_grad, void* ws, size_t ws_bytes, cudaStream_t st, int bm,
                            int chunk, bool upload, bool launch, BatchLayout* out_layout) {
  const int es = prec == SAA_FP64 ? 8 : 4;
  std::vector<BInst> hi;
  std::vector<BItem> hitems;
  const BatchLayout L = plan_batch(B, probs, K, X, f, pbar, var, grad, want_grad, es, bm, chunk, &hi, &hitems);
  if (out_layout) *out_layout = L;
  if (ws_bytes < L.total) {
    set_error("batched: workspace smaller than the workspace-size query");
    return SAA_ENOMEM;
  }
  char* w = (char*)ws;
  if (upload) {
    // descriptors go through a pinned staging buffer owned by the context
    const size_t bytes = L.yf;
    if (ctx->stage_bytes < bytes) {
      if (ctx->stage) {
        cudaEventSynchronize(ctx->stage_ready);
        cudaFreeHost(ctx->stage);
        ctx->stage = nullptr;
        ctx->stage_bytes = 0;
      }
      saa_status s = cuda_status(cudaHostAlloc(&ctx->stage, bytes, cudaHostAllocDefault), "pinned staging buffer");
      if (s != SAA_OK) return s;
      ctx->stage_bytes = bytes;
    } else {
      cudaEventSynchronize(ctx->stage_ready);   // the previous upload has been consumed
    }
    char* h = (char*)ctx->stage;
    std::memcpy(h + L.insts, hi.data(), sizeof(BInst) * hi.size());
    std::memcpy(h + L.items, hitems.data(), sizeof(BItem) * hitems.size());
    saa_status s = cuda_status(cudaMemcpyAsync(w, h, bytes, cudaMemcpyHostToDevice, st), "descriptor upload");
    if (s != SAA_OK) return s;
    s = cuda_status(cudaEventRecord(ctx->stage_ready, st), "stage event");
    if (s != SAA_OK) return s;
  }
  if (!launch) return SAA_OK;
  int nk = 0;
  saa_status s = launch_sequence(ctx, B, L, prec, bm, want_grad, w, st, &nk);
  ctx->kernels += nk;
  return s;
}

static size_t batch_ws(int32_t B, const saa_problem* probs, const int32_t* K, saa_prec prec, int want_grad) {
  const int es = prec == SAA_FP64 ? 8 : 4;
  size_t need = 0;
  // the largest layout over the tile shapes the autotuner may pick
  for (int bm : {32, 64})
    for (int ch : kChunkChoices)
      need = std::max(need, plan_batch(B, probs, K, nullptr, nullptr, nullptr, nullptr, nullptr, want_grad, es, bm, ch,
                                       nullptr, nullptr)
                                .total);
  return need;
}

// Tile shape for this batch shape: the autotuner's cached choice, else (when
// enabled and not capturing) time every candidate once, else a default.
static saa_status choose_shape(saa_ctx* ctx, int B, const saa_problem* probs, const int32_t* K, const double* const* X,
                               saa_prec prec, double* const* f, double* const* pbar, double* const* var,
                               double* const* grad, int want_grad, void* ws, size_t ws_bytes, cudaStream_t st,
                               int* bm_out, int* chunk_out) {
  int dmax = 1;
  for (int b = 0; b < B; ++b) dmax = std::max(dmax, probs[b].d);
  const uint64_t key = shape_key(B, probs, K, prec, ctx->device) ^ ((uint64_t)want_grad << 63);
  int bm = -1, chunk = -1;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    for (const TuneEntry& t : g_tune)
      if (t.key == key) {
        bm = t.bm;
        chunk = t.chunk;
      }
  }
  if (bm < 0 && ctx->autotune) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cs);
    if (cs == cudaStreamCaptureStatusNone) {
      cudaEvent_t e0, e1;
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      float best = 1e30f;
      saa_status s = SAA_OK;
      for (int cbm : {32, 64}) {
        if (prec == SAA_FP64 && cbm == 64 && dmax > 256) continue;
        if (prec == SAA_FP32 && cbm == 64 && dmax > 512) continue;
        for (int ch : kChunkChoices) {
          s = run_batch(ctx, B, probs, K, X, prec, f, pbar, var, grad, want_grad, ws, ws_bytes, st, cbm, ch, true,
                        true, nullptr);
          if (s != SAA_OK) break;
          cudaEventRecord(e0, st);
          s = run_batch(ctx, B, probs, K, X, prec, f, pbar, var, grad, want_grad, ws, ws_bytes, st, cbm, ch, false,
                        true, nullptr);
          cudaEventRecord(e1, st);
          cudaEventSynchronize(e1);
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          if (s == SAA_OK && ms < best) {
            best = ms;
            bm = cbm;
            chunk = ch;
          }
        }
        if (s != SAA_OK) break;
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      if (s != SAA_OK) return s;
      std::lock_guard<std::mutex> lock(g_tune_mu);
      g_tune.push_back({key, bm, chunk});
    }
  }
  if (bm < 0) {
    bm = pick_bm(prec, dmax);
    chunk = 32;
  }
  *bm_out = bm;
  *chunk_out = chunk;
  return SAA_OK;
}

// Makes ctx->device current for the duration of a call.
struct BatchDeviceGuard {
  int prev = -1;
  explicit BatchDeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~BatchDeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

struct saa_batch {
  saa_ctx* ctx;
  cudaGraphExec_t exec;
  int kernels;   // kernels per replay
};

extern "C" size_t saa_workspace_size_batched(const saa_ctx* ctx, int32_t B, const saa_problem* probs,
                                             const int32_t* K, saa_prec prec) {
  if (!ctx || B < 1 || !probs || !K) return 0;
  return batch_ws(B, probs, K, prec, 0);
}

extern "C" saa_status saa_eval_batched(saa_ctx* ctx, int32_t B, const saa_problem* probs, const int32_t* K,
                                       const double* const* X, saa_prec prec, double* const* f, double* const* pbar,
                                       double* const* var, void* ws, size_t ws_bytes, void* stream) {
  saa::NvtxRange nvtx_range("saa_eval_batched");
  if (!ctx) {
    set_error("ctx is NULL");
    return SAA_EINVAL;
  }
  saa_status s = validate(B, probs, K, X, f, prec);
  if (s != SAA_OK) return s;
  if (!ws || (((uintptr_t)ws) & 255u)) {
    set_error("workspace must be non-NULL and 256-byte aligned");
    return SAA_EINVAL;
  }
  BatchDeviceGuard g(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  int bm = 0, chunk = 0;
  s = choose_shape(ctx, B, probs, K, X, prec, f, pbar, var, nullptr, 0, ws, ws_bytes, st, &bm, &chunk);
  if (s != SAA_OK) return s;
  return run_batch(ctx, B, probs, K, X, prec, f, pbar, var, nullptr, 0, ws, ws_bytes, st, bm, chunk, true, true,
                   nullptr);
}

extern "C" size_t saa_batch_workspace_size(const saa_ctx* ctx, int32_t B, const saa_problem* probs, const int32_t* K,
                                           saa_prec prec, int want_grad) {
  if (!ctx || B < 1 || !probs || !K) return 0;
  return batch_ws(B, probs, K, prec, want_grad ? 1 : 0);
}

extern "C" saa_status saa_batch_create(saa_ctx* ctx, int32_t B, const saa_problem* probs, const int32_t* K,
                                       const double* const* X, saa_prec prec, double* const* f, double* const* pbar,
                                       double* const* var, double* const* grad, void* ws, size_t ws_bytes,
                                       void* stream, saa_batch** out) {
  saa::NvtxRange nvtx_range("saa_batch_create");
  if (!ctx || !out) {
    set_error("saa_batch_create: ctx and out must be non-NULL");
    return SAA_EINVAL;
  }
  *out = nullptr;
  saa_status s = validate(B, probs, K, X, f, prec);
  if (s != SAA_OK) return s;
  const int want_grad = grad ? 1 : 0;
  if (grad)
    for (int b = 0; b < B; ++b)
      if (!grad[b]) {
        set_error("saa_batch_create: grad[" + std::to_string(b) + "] is NULL");
        return SAA_EINVAL;
      }
  if (!ws || (((uintptr_t)ws) & 255u)) {
    set_error("workspace must be non-NULL and 256-byte aligned");
    return SAA_EINVAL;
  }
  if (ws_bytes < batch_ws(B, probs, K, prec, want_grad)) {
    set_error("saa_batch_create: workspace smaller than saa_batch_workspace_size()");
    return SAA_ENOMEM;
  }
  BatchDeviceGuard g(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  int bm = 0, chunk = 0;
  s = choose_shape(ctx, B, probs, K, X, prec, f, pbar, var, grad, want_grad, ws, ws_bytes, st, &bm, &chunk);
  if (s != SAA_OK) return s;
  // upload the descriptor tables once, and wait for them
  BatchLayout L;
  s = run_batch(ctx, B, probs, K, X, prec, f, pbar, var, grad, want_grad, ws, ws_bytes, st, bm, chunk, true, false,
                &L);
  if (s == SAA_OK) s = cuda_status(cudaStreamSynchronize(st), "saa_batch_create: descriptor upload");
  if (s != SAA_OK) return s;
  // capture the launch sequence on a private stream
  cudaStream_t cap;
  s = cuda_status(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "saa_batch_create: capture stream");
  if (s != SAA_OK) return s;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int nk = 0;
  s = cuda_status(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal), "saa_batch_create: begin capture");
  if (s == SAA_OK) {
    const saa_status r = launch_sequence(ctx, B, L, prec, bm, want_grad, (char*)ws, cap, &nk);
    const cudaError_t e = cudaStreamEndCapture(cap, &graph);
    s = (r != SAA_OK) ? r : cuda_status(e, "saa_batch_create: end capture");
  }
  if (s == SAA_OK) s = cuda_status(cudaGraphInstantiate(&exec, graph, 0), "saa_batch_create: instantiate");
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(cap);
  if (s != SAA_OK) return s;
  saa_batch* bt = new (std::nothrow) saa_batch();
  if (!bt) {
    cudaGraphExecDestroy(exec);
    set_error("saa_batch_create: host allocation failed");
    return SAA_ENOMEM;
  }
  bt->ctx = ctx;
  bt->exec = exec;
  bt->kernels = nk;
  *out = bt;
  return SAA_OK;
}

extern "C" saa_status saa_batch_launch(saa_batch* batch, void* stream) {
  saa::NvtxRange nvtx_range("saa_batch_launch");
  if (!batch) {
    set_error("saa_batch_launch: batch is NULL");
    return SAA_EINVAL;
  }
  BatchDeviceGuard g(batch->ctx->device);
  batch->ctx->kernels += batch->kernels;
  return cuda_status(cudaGraphLaunch(batch->exec, (cudaStream_t)stream), "saa_batch_launch: graph launch");
}

extern "C" void saa_batch_destroy(saa_batch* batch) {
  if (!batch) return;
  BatchDeviceGuard g(batch->ctx->device);
  cudaDeviceSynchronize();
  cudaGraphExecDestroy(batch->exec);
  delete batch;
}
