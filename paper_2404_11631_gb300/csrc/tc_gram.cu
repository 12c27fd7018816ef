// tc_gram.cu -- covariance-first form of the SAA estimate (Sec. 3.1: the
// sample mean and covariance of the R_i, formed once per resample) for
// d <= 1024, on tcgen05 tensor cores.
//
// With a_i = s_i zhat_i (whitened samples), every quantity of Eq. 4, Eq. 5
// and the gradient follows from two sums over the scenarios:
//   M = sum_i a_i a_i'   (d x d)      m~ = sum_i a_i   (d)
// as S1_k = m~'y_k, S2_k = y_k' M y_k and G_k = M y_k with y_k = C'w_k.
// saa_moments forms M and m~ (the work is independent of the number of
// decisions); saa_eval_moments then evaluates any K decisions, value and
// gradient, in FP64 at the cost of K d^2 multiply-adds.
//
// M is formed in 128 x 128 blocks M[p, q], p <= q, of the nb = ceil(d / 128)
// dimension slices (the rest by symmetry).  CTA g takes block pair
// g mod npairs over the scenario tiles t = g / npairs, + nrange, ... (nrange
// = the SMs the pairs leave, at least one), so that every SM works.  The
// generator draws any (scenario, slice) on its own, so each CTA draws the
// two slices of its pair: at d = 1024 every normal is drawn by up to 8 CTAs,
// the price of needing no exchange between them.
// Kernel (one CTA per SM, persistent over 64-scenario tiles):
//   generator warps draw slices p and q of each tile transposed --
//     [dims][scenarios], K-major over the scenarios, hi/lo of the operand
//     type -- into a 3-stage ring (one slice on a diagonal block), and the
//     diagonal blocks fold their draws into the CTA's partial of m~;
//   one thread issues A_p A_q^T (M = N = 128 dimensions, 4 k steps of 16
//     scenarios): hi*hi into one accumulator, hi*lo + lo*hi into another;
//   four epilogue warps fold each tile's hi*hi + corrections into a running
//     FP32 sum in TMEM with round-to-nearest adds, and at the end write the
//     CTA's partial of its block.
// TMEM: 3 x 128 columns.  The operands both change with the scenario, so
// their hi/lo representation error averages out; 4 k steps per tile keep the
// accumulator's rounding bias near two units in the last place per tile.
// Every wait is clock-bounded.
#include <cuda_runtime.h>

#include <cstring>

#include "gen.cuh"
#include "internal.cuh"
#include "tc_ptx.cuh"

namespace saa {
namespace tc {

constexpr int kQM = 64;                  // scenarios per tile of an off-diagonal block (diagonal: 2 kQM)
constexpr int kQD = 128;                 // dimensions per slice: MMA M and N
constexpr int kQMaxDim = 1024;
constexpr int kQStages = 3;
constexpr int kQSub = kQD * 128;         // one [128 dims][64 scenarios] 16-bit block
constexpr int kQStageBytes = 4 * kQSub;  // [slice p, slice q][hi, lo]
constexpr int kQEpi = 4;
constexpr int kQMma = 4;
constexpr int kQRng = 16;
constexpr int kQThreads = 32 * (5 + kQRng);
constexpr int kQSBufs = 4;

struct QArgs {
  LawArgs la;
  int64_t tiles;
  int nb, npairs, nrange;   // slices, block pairs p <= q, scenario ranges (CTA g: pair g % npairs, range g / npairs)
  float* part_M;    // [grid][128][128] row j (TMEM lane) of slice p, column l of slice q
  double* part_m;   // [grid][2 halves][d] (diagonal blocks: their slice's entries)
  uint32_t* err;
};

struct QSmem {
  uint64_t a_full[kQStages];
  uint64_t a_empty[kQStages];
  uint64_t s_ready[kQSBufs];
  uint64_t g_full, g_empty, drain;
  uint32_t tmem_base;
  uint32_t abort_flag;
  float s_buf[kQSBufs][2 * kQM];
};

size_t gram_smem_bytes() { return (size_t)kQStages * kQStageBytes + sizeof(QSmem); }

// D4: d is a multiple of 4, so every 4-dimension block below d is whole and
// the per-element guards drop out.
template <bool F16, bool D4>
__global__ void __launch_bounds__(kQThreads, 1) k_tc_gram(QArgs a) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  const uint32_t base = smem_u32(smem_raw);
  if (base & 1023u) {
    if (threadIdx.x == 0) atomicOr(a.err, kErrBounds);
    return;
  }
  uint8_t* ring = smem_raw;
  QSmem* sm = reinterpret_cast<QSmem*>(smem_raw + kQStages * kQStageBytes);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const LawArgs& la = a.la;
  const int d = la.d;
  volatile uint32_t* abort_flag = &sm->abort_flag;

  // this CTA's block pair (p, q), p <= q, in row order, and scenario range;
  // a diagonal block takes 128-scenario tiles (both halves of the stage hold
  // slice p), an off-diagonal one 64-scenario tiles (slices p and q)
  int bp = 0, bq = (int)(blockIdx.x % (uint32_t)a.npairs);
  while (bq >= a.nb - bp) {
    bq -= a.nb - bp;
    ++bp;
  }
  bq += bp;
  const bool diag = bp == bq;
  const int tm = diag ? 2 * kQM : kQM;
  const int64_t ntiles = ((int64_t)la.N + tm - 1) / tm;
  const int rg = (int)(blockIdx.x / (uint32_t)a.npairs);
  const int my_tiles = (rg < ntiles) ? (int)((ntiles - rg + a.nrange - 1) / a.nrange) : 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kQStages; ++s) {
      mbar_init(smem_u32(&sm->a_full[s]), kQRng);
      mbar_init(smem_u32(&sm->a_empty[s]), 1);
    }
    for (int s = 0; s < kQSBufs; ++s) mbar_init(smem_u32(&sm->s_ready[s]), tm / 32);
    mbar_init(smem_u32(&sm->g_full), 1);
    mbar_init(smem_u32(&sm->g_empty), kQEpi);
    mbar_init(smem_u32(&sm->drain), 1);
    sm->abort_flag = 0u;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kQMma) tmem_alloc(smem_u32(&sm->tmem_base), 512u);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sm->tmem_base;
  const uint32_t tg1a = tmem, tg1b = tmem + 128u, tg2 = tmem + 256u, tr = tmem + 384u;


  if (warp == kQMma) {
    // ------------------------------------------------------------ MMA ---
    if (lane == 0) {
      bool ok = true;
      const uint32_t idesc = idesc_f16(kQD, kQD, F16);
      int st = 0;
      uint32_t ph = 0;
      for (int tt = 0; ok && tt < my_tiles; ++tt) {
        ok = mbar_wait(smem_u32(&sm->g_empty), (uint32_t)((tt & 1) ^ 1), abort_flag, a.err) &&
             mbar_wait(smem_u32(&sm->a_full[st]), ph, abort_flag, a.err);
        if (!ok) break;
        tc_fence_after();
        const uint32_t stage = smem_u32(ring) + (uint32_t)(st * kQStageBytes);
        // off-diagonal: A = slice p, B = slice q, 4 k steps; diagonal: A = B,
        // 4 k steps on each half of the stage (the two halves' hi*hi in two
        // chunk accumulators)
        const int nk = diag ? 8 : 4;
        for (int kk = 0; kk < nk; ++kk) {   // 16 scenarios per k step
          const uint32_t o = (uint32_t)((kk & 3) * 32);
          const uint32_t ha = (uint32_t)((kk >> 2) * 2 * kQSub);           // diagonal: the stage half
          const uint32_t hb = diag ? ha : 2u * (uint32_t)kQSub;            // slice q (or the same half)
          const uint32_t ahi = stage + ha + o, alo = stage + ha + (uint32_t)kQSub + o;
          const uint32_t bhi = stage + hb + o, blo = stage + hb + (uint32_t)kQSub + o;
          const uint32_t g1 = (kk < 4) ? tg1a : tg1b;
          mma_bf16(g1, desc_sw128(ahi), desc_sw128(bhi), idesc, (kk & 3) == 0 ? 0u : 1u);
          mma_bf16(tg2, desc_sw128(ahi), desc_sw128(blo), idesc, kk == 0 ? 0u : 1u);
          mma_bf16(tg2, desc_sw128(alo), desc_sw128(bhi), idesc, 1u);
        }
        mma_commit(smem_u32(&sm->a_empty[st]));
        mma_commit(smem_u32(&sm->g_full));
        if (++st == kQStages) { st = 0; ph ^= 1u; }
      }
      mma_commit(smem_u32(&sm->drain));
      uint32_t never = 0u;
      mbar_wait(smem_u32(&sm->drain), 0, &never, a.err);
    }
    __syncwarp();
  } else if (warp < kQEpi) {
    // ------------------------------------------------------- epilogue ---
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    bool ok = true;
    for (int tt = 0; tt < my_tiles; ++tt) {
      if (!warp_wait(smem_u32(&sm->g_full), (uint32_t)(tt & 1), abort_flag, a.err)) {
        ok = false;
        break;
      }
      tc_fence_after();
#pragma unroll 1
      for (int c0 = 0; c0 < kQD; c0 += 16) {
        uint32_t x[16], y[16];
        tmem_ld16(tg1a + lane_base + (uint32_t)c0, x);
        if (diag) tmem_ld16(tg1b + lane_base + (uint32_t)c0, y);
        tmem_wait_ld();
        float p[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) p[i] = diag ? __uint_as_float(x[i]) + __uint_as_float(y[i]) : __uint_as_float(x[i]);
        tmem_ld16(tg2 + lane_base + (uint32_t)c0, x);
        if (tt > 0) tmem_ld16(tr + lane_base + (uint32_t)c0, y);
        tmem_wait_ld();
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          p[i] += __uint_as_float(x[i]);
          if (tt > 0) p[i] = __uint_as_float(y[i]) + p[i];
          x[i] = __float_as_uint(p[i]);
        }
        tmem_st16(tr + lane_base + (uint32_t)c0, x);
        tmem_wait_st();
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&sm->g_empty));
    }
    if (ok && my_tiles > 0) {
      tc_fence_after();
      const int j = warp * 32 + lane;   // this lane's row of M
      float* row = a.part_M + ((size_t)blockIdx.x * kQD + j) * kQD;
#pragma unroll 1
      for (int c0 = 0; c0 < kQD; c0 += 16) {
        uint32_t x[16];
        tmem_ld16(tr + lane_base + (uint32_t)c0, x);
        tmem_wait_ld();
#pragma unroll
        for (int i = 0; i < 16; i += 4)
          *reinterpret_cast<float4*>(row + c0 + i) = make_float4(__uint_as_float(x[i]), __uint_as_float(x[i + 1]),
                                                                 __uint_as_float(x[i + 2]), __uint_as_float(x[i + 3]));
      }
    }
  } else {
    // ------------------------------------------------------------ RNG ---
    const int rt = threadIdx.x - 32 * (kQMma + 1);   // 0 .. 511
    const gen::Stream gs = gen::make_stream(la.seed, la.epoch, la.instance);
    const uint32_t half = la.N / 2u;
    const bool tlaw = la.law == SAA_LAW_STUDENT_T;
    // stage half blk: slice p (blk 0) or q (blk 1) of the tile's 64
    // scenarios, or on a diagonal block slice p of scenarios 64 blk ..
    // 64 blk + 63; dimensions 4 b4 .. 4 b4 + 3 of the slice, scenarios
    // 8 g8 .. 8 g8 + 7 of the half, one scenario pair (4 bytes) per store,
    // pair order staggered by lane group
    const int blk = rt >> 8, b4 = (rt >> 3) & 31, g8 = rt & 7;
    const int pfirst = (lane >> 3) & 3;
    const int jb = 4 * b4;                                           // row of the stage (dimension within the slice)
    const int jg = ((diag || blk == 0) ? bp : bq) * kQD + jb;        // dimension
    const int sh = diag ? kQM * blk : 0;                             // first scenario of the half
    int st = 0;
    uint32_t ph = 0;
    for (int tt = 0; tt < my_tiles; ++tt) {
      const uint32_t tile = (uint32_t)rg + (uint32_t)tt * (uint32_t)a.nrange;
      const uint32_t i0 = tile * (uint32_t)tm;
      const int nrow = (int)min((uint32_t)tm, la.N - i0);
      const int sb4 = tt & (kQSBufs - 1);
      const uint32_t s_bar = smem_u32(&sm->s_ready[sb4]);
      if (tlaw && rt < tm) {
        sm->s_buf[sb4][rt] = (rt < nrow) ? gen::t_scale_f(gs, i0 + (uint32_t)rt, la.nu) : 0.0f;
        __syncwarp();
        if (lane == 0) mbar_arrive(s_bar);
      }
      if (!warp_wait(smem_u32(&sm->a_empty[st]), ph ^ 1u, abort_flag, a.err)) break;
      if (tlaw && !warp_wait(s_bar, (uint32_t)((tt >> 2) & 1), abort_flag, a.err)) break;
      uint8_t* stage = ring + st * kQStageBytes;
      float msum[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      {
#pragma unroll 1
        for (int p = 0; p < 4; ++p) {
          const int pq = (p + pfirst) & 3;   // scenarios 8 g8 + 2 pq, + 1 of the half
          const int r0 = sh + 8 * g8 + 2 * pq;
          float z0[4] = {0.0f, 0.0f, 0.0f, 0.0f}, z1[4] = {0.0f, 0.0f, 0.0f, 0.0f};
          if (jg < d) {
            if (r0 < nrow) {
              const uint32_t i = i0 + (uint32_t)r0;
              gen::Gen<float>::block(gs, (uint32_t)(jg >> 2), i, gen::is_lognormal(la.law, i, half), z0);
              if (tlaw) {
                const float s0 = sm->s_buf[sb4][r0];
#pragma unroll
                for (int e = 0; e < 4; ++e) z0[e] *= s0;
              }
#pragma unroll
              for (int e = 0; e < 4; ++e) z0[e] = (D4 || jg + e < d) ? z0[e] : 0.0f;
            }
            if (r0 + 1 < nrow) {
              const uint32_t i = i0 + (uint32_t)r0 + 1u;
              gen::Gen<float>::block(gs, (uint32_t)(jg >> 2), i, gen::is_lognormal(la.law, i, half), z1);
              if (tlaw) {
                const float s1 = sm->s_buf[sb4][r0 + 1];
#pragma unroll
                for (int e = 0; e < 4; ++e) z1[e] *= s1;
              }
#pragma unroll
              for (int e = 0; e < 4; ++e) z1[e] = (D4 || jg + e < d) ? z1[e] : 0.0f;
            }
          }
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            msum[e] += z0[e] + z1[e];
            const int jr = jb + e;   // row of the stage
            const uint32_t h = pack2<F16>(z0[e], z1[e]);
            const float2 f = unpack2<F16>(h);
            const uint32_t l = pack2<F16>(z0[e] - f.x, z1[e] - f.y);
            const uint32_t off = (uint32_t)(jr * 128 + ((g8 ^ (jr & 7)) << 4) + pq * 4);
            *reinterpret_cast<uint32_t*>(stage + (blk * 2 + 0) * kQSub + off) = h;
            *reinterpret_cast<uint32_t*>(stage + (blk * 2 + 1) * kQSub + off) = l;
          }
        }
      }
      // m~ (diagonal blocks): fold the 8 lanes that share these dimensions;
      // lane g8 == 0 of each half owns them in that half's partial row
      if (diag) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
#pragma unroll
          for (int o = 1; o < 8; o <<= 1) msum[e] += __shfl_xor_sync(0xffffffffu, msum[e], o);
        }
        if (g8 == 0) {
#pragma unroll
          for (int e = 0; e < 4; ++e)
            if (jg + e < d) {
              double* pm = a.part_m + ((size_t)blockIdx.x * 2 + blk) * d + jg + e;
              if (tt == 0)
                *pm = (double)msum[e];
              else
                atomicAdd(pm, (double)msum[e]);
            }
        }
      }
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&sm->a_full[st]));
      if (++st == kQStages) { st = 0; ph ^= 1u; }
    }
  }

  __syncthreads();
  if (warp == kQMma) {
    tc_fence_after();
    tmem_dealloc(tmem, 512u);
  }
}

}  // namespace tc

namespace {

__device__ __forceinline__ void nm_add(double& s, double& c, double x) {
  const double t = s + x;
  if (fabs(s) >= fabs(x))
    c += (s - t) + x;
  else
    c += (x - t) + s;
  s = t;
}

// M_jl = sum over the scenario ranges of block (p, q)'s partials, p = j / 128
// and q = l / 128 (or the transposed entry of block (q, p) when p > q), as
// float-float pairs (branch-free TwoSum); mt_j = sum over the ranges of the
// diagonal block's two partials of m~ (Neumaier).  One block per (row j, 32
// columns); warp w takes ranges w, w + 8, ..., merged in warp order.
__global__ void __launch_bounds__(256) k_gram_reduce(int nb, int npairs, int nrange, int d,
                                                     const float* __restrict__ part_M,
                                                     const double* __restrict__ part_m, double* __restrict__ M,
                                                     double* __restrict__ mt) {
  __shared__ double sh_s[8][32], sh_c[8][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = blockIdx.y;
  const int l = blockIdx.x * 32 + lane;
  // the block holding M_jl, and the entry's row / column within it
  const int pj = j >> 7, pl = l >> 7;
  const bool tr = pj > pl;
  const int p = tr ? pl : pj, q = tr ? pj : pl;
  const int jj = tr ? (l & 127) : (j & 127), ll = tr ? (j & 127) : (l & 127);
  const int pair = p * nb - p * (p - 1) / 2 + (q - p);   // row-order index of (p, q), p <= q
  float S = 0.0f, E = 0.0f;
  if (l < d)
    for (int r = warp; r < nrange; r += 8) {
      const float x = part_M[(((size_t)r * npairs + pair) * 128 + jj) * 128 + ll];
      const float t = __fadd_rn(S, x);
      const float bb = __fsub_rn(t, S);
      E = __fadd_rn(E, __fadd_rn(__fsub_rn(S, __fsub_rn(t, bb)), __fsub_rn(x, bb)));
      S = t;
    }
  sh_s[warp][lane] = (double)S;
  sh_c[warp][lane] = (double)E;
  __syncthreads();
  if (warp == 0 && l < d) {
    double s = 0.0, c = 0.0;
    for (int w = 0; w < 8; ++w) {
      nm_add(s, c, sh_s[w][lane]);
      nm_add(s, c, sh_c[w][lane]);
    }
    M[(size_t)j * d + l] = s + c;
  }
  if (blockIdx.x == 0 && warp == 1) {
    // lane L adds the partials of ranges L, L + 32, ... (both halves), then
    // the lanes' sums merge by a fixed shuffle tree
    const int dp = pj * nb - pj * (pj - 1) / 2;   // the diagonal block of j's slice
    double s = 0.0, c = 0.0;
    for (int r = lane; r < nrange; r += 32)
      for (int h = 0; h < 2; ++h) nm_add(s, c, part_m[(((size_t)r * npairs + dp) * 2 + h) * d + j]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double os = __shfl_down_sync(0xffffffffu, s, o), oc = __shfl_down_sync(0xffffffffu, c, o);
      nm_add(s, c, os);
      c += oc;
    }
    if (lane == 0) mt[j] = s + c;
  }
}

// Per decision k (one block of min(256, d rounded up to 32) threads, y_k in
// shared memory): S1 =
// mt'y_k, then t = M y_k row by row, S2 = y_k't; f, pbar, var; with a
// gradient, u_k = lambda 2/(N-1) (t - S1 m) - m with m = mt/N.  Sums in a
// fixed order (per thread, then a shuffle tree, then the warps in order).
__device__ __forceinline__ double gram_block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
  return t;
}
__global__ void __launch_bounds__(256) k_gram_eval(int K, int d, double N, double lambda, const double* __restrict__ M,
                                                   const double* __restrict__ mt, const double* __restrict__ Y64,
                                                   const double* __restrict__ c, double* __restrict__ f,
                                                   double* __restrict__ pbar, double* __restrict__ var,
                                                   double* __restrict__ u) {
  extern __shared__ double ys[];   // [d]
  __shared__ double red[8];
  const int k = blockIdx.x;
  for (int j = threadIdx.x; j < d; j += blockDim.x) ys[j] = Y64[(size_t)k * d + j];
  __syncthreads();
  double p1 = 0.0;
  for (int j = threadIdx.x; j < d; j += blockDim.x) p1 = fma(mt[j], ys[j], p1);
  const double S1 = gram_block_sum(p1, red);
  double p2 = 0.0;
  for (int j = threadIdx.x; j < d; j += blockDim.x) {
    const double* Mj = M + (size_t)j * d;
    double t = 0.0;
    for (int l = 0; l < d; ++l) t = fma(Mj[l], ys[l], t);
    p2 = fma(ys[j], t, p2);
    if (u) {
      const double mj = mt[j] / N;
      u[(size_t)k * d + j] = lambda * (2.0 / (N - 1.0)) * (t - S1 * mj) - mj;
    }
  }
  const double S2 = gram_block_sum(p2, red);
  if (threadIdx.x == 0) {
    const double qbar = S1 / N;
    const double pb = c[k] + qbar;
    const double V = (S2 - S1 * qbar) / (N - 1.0);
    if (f) f[k] = lambda * V - pb;
    if (pbar) pbar[k] = pb;
    if (var) var[k] = V;
  }
}

saa_status gram_check(const saa_ctx* ctx, const saa_problem* p, saa_prec prec) {
  if (!ctx || !p) {
    set_error("saa_moments: ctx and prob must be non-NULL");
    return SAA_EINVAL;
  }
  if (p->d < 1 || p->d > tc::kQMaxDim || p->N < 2 || p->N > 0xffffffffll || p->law < SAA_LAW_GAUSS ||
      p->law > SAA_LAW_MIX || (p->law == SAA_LAW_STUDENT_T && (p->nu < 2 || (p->nu & 1) || p->nu > 64)) ||
      p->reserved != 0 || !p->mu || !p->chol) {
    set_error("saa_moments: need 1 <= d <= 1024, 2 <= N < 2^32, a known law and device mu, chol");
    return SAA_EINVAL;
  }
  if (!is_tc(prec)) {
    set_error("saa_moments: the covariance-first form runs at SAA_F16X3 or SAA_BF16X3");
    return SAA_EUNSUPPORTED;
  }
  if ((int)tc::gram_smem_bytes() > ctx->smem_optin) {
    set_error("saa_moments: shared-memory ring does not fit");
    return SAA_EUNSUPPORTED;
  }
  return SAA_OK;
}

// Grid of the Gram kernel: every block pair p <= q of the nb slices, times
// as many scenario ranges as the SMs leave (at least one, at most the tiles).
struct GramPlan {
  int nb, npairs, nrange, grid;
  int64_t tiles;
};
GramPlan gram_plan(const saa_ctx* ctx, const saa_problem* p) {
  GramPlan g;
  g.nb = (p->d + tc::kQD - 1) / tc::kQD;
  g.npairs = g.nb * (g.nb + 1) / 2;
  g.tiles = (p->N + tc::kQM - 1) / tc::kQM;
  const int64_t dtiles = (p->N + 2 * tc::kQM - 1) / (2 * tc::kQM);   // a diagonal block's tiles
  int64_t nr = ctx->sm_count / g.npairs;
  if (nr < 1) nr = 1;
  if (nr > dtiles) nr = dtiles;   // every range has a tile of every block
  g.nrange = (int)nr;
  g.grid = g.npairs * g.nrange;
  return g;
}

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

struct DevGuard {
  int prev = -1;
  explicit DevGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DevGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

}  // namespace
}  // namespace saa

using namespace saa;

extern "C" size_t saa_moments_workspace_size(const saa_ctx* ctx, const saa_problem* prob, saa_prec prec) {
  if (gram_check(ctx, prob, prec) != SAA_OK) return 0;
  const size_t g = (size_t)gram_plan(ctx, prob).grid;
  return al256(sizeof(float) * g * tc::kQD * tc::kQD) + al256(sizeof(double) * g * 2 * prob->d);
}

extern "C" saa_status saa_moments(saa_ctx* ctx, const saa_problem* prob, saa_prec prec, double* M, double* mt,
                                  void* ws, size_t ws_bytes, void* stream) {
  saa::NvtxRange nvtx_range("saa_moments");
  saa_status s = gram_check(ctx, prob, prec);
  if (s != SAA_OK) return s;
  if (!M || !mt || !ws || (((uintptr_t)ws) & 255u)) {
    set_error("saa_moments: M, mt and a 256-byte aligned ws are required");
    return SAA_EINVAL;
  }
  const GramPlan gp = gram_plan(ctx, prob);
  const int grid = gp.grid;
  const size_t pm_off = al256(sizeof(float) * (size_t)grid * tc::kQD * tc::kQD);
  if (ws_bytes < pm_off + al256(sizeof(double) * (size_t)grid * 2 * prob->d)) {
    set_error("saa_moments: workspace smaller than saa_moments_workspace_size()");
    return SAA_ENOMEM;
  }
  DevGuard g(ctx->device);
  tc::QArgs a;
  a.la.d = prob->d;
  a.la.law = prob->law;
  a.la.nu = prob->nu;
  a.la.N = (uint32_t)prob->N;
  a.la.seed = prob->seed;
  a.la.instance = prob->instance;
  a.la.epoch = prob->epoch;
  a.la.t_dev = nullptr;
  a.la.M = 1;
  a.tiles = gp.tiles;
  a.nb = gp.nb;
  a.npairs = gp.npairs;
  a.nrange = gp.nrange;
  a.part_M = (float*)ws;
  a.part_m = (double*)((char*)ws + pm_off);
  a.err = ctx->err;
  const int smem = (int)tc::gram_smem_bytes();
  cudaStream_t st = (cudaStream_t)stream;
  const bool d4 = (prob->d & 3) == 0;
  auto kern = (prec == SAA_F16X3) ? (d4 ? tc::k_tc_gram<true, true> : tc::k_tc_gram<true, false>)
                                  : (d4 ? tc::k_tc_gram<false, true> : tc::k_tc_gram<false, false>);
  s = cuda_status(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
                  "saa_moments: shared-memory attribute");
  if (s != SAA_OK) return s;
  const bool prof = ctx->prof_on && ctx->prof_n < 256;
  if (prof) cudaEventRecord(ctx->prof_ev[2 * ctx->prof_n], st);
  kern<<<grid, tc::kQThreads, smem, st>>>(a);
  if (prof) cudaEventRecord(ctx->prof_ev[2 * ctx->prof_n++ + 1], st);
  k_gram_reduce<<<dim3((prob->d + 31) / 32, prob->d), 256, 0, st>>>(gp.nb, gp.npairs, gp.nrange, prob->d, a.part_M,
                                                                     a.part_m, M, mt);
  ctx->kernels += 2;
  return cuda_status(cudaGetLastError(), "saa_moments: launch");
}

extern "C" size_t saa_eval_moments_workspace_size(const saa_problem* prob, int32_t K) {
  if (!prob || prob->d < 1 || prob->d > tc::kQMaxDim || K < 1 || K > 65535) return 0;
  const size_t d = (size_t)prob->d, k = (size_t)K;
  return al256(8 * k * d) + al256(8 * k) + al256(8 * k * d);
}

extern "C" saa_status saa_eval_moments(saa_ctx* ctx, const saa_problem* prob, int32_t K, const double* X,
                                       const double* M, const double* mt, double* f, double* pbar, double* var,
                                       double* grad, void* ws, size_t ws_bytes, void* stream) {
  saa::NvtxRange nvtx_range("saa_eval_moments");
  if (!ctx || !prob || prob->d < 1 || prob->d > tc::kQMaxDim || prob->N < 2 || !prob->mu || !prob->chol) {
    set_error("saa_eval_moments: need ctx, and a problem with 1 <= d <= 1024, N >= 2, device mu, chol");
    return SAA_EINVAL;
  }
  if (K < 1 || K > 65535 || !X || !M || !mt || !ws || (((uintptr_t)ws) & 255u) || !(f || pbar || var || grad)) {
    set_error("saa_eval_moments: need 1 <= K <= 65535, X, M, mt, an output and a 256-byte aligned ws");
    return SAA_EINVAL;
  }
  if (ws_bytes < saa_eval_moments_workspace_size(prob, K)) {
    set_error("saa_eval_moments: workspace smaller than saa_eval_moments_workspace_size()");
    return SAA_ENOMEM;
  }
  DevGuard g(ctx->device);
  const size_t d = (size_t)prob->d, k = (size_t)K;
  Workspace w;
  std::memset(&w, 0, sizeof(w));
  w.Y64 = (double*)ws;
  w.c = (double*)((char*)ws + al256(8 * k * d));
  double* u = (double*)((char*)ws + al256(8 * k * d) + al256(8 * k));
  cudaStream_t st = (cudaStream_t)stream;
  // y_k = C'w_k and c_k = mu'w_k in FP64 (no contraction-precision copy)
  saa_status s = cuda_status(launch_prologue(prob, K, X, SAA_F16X3, w, ctx->err, st), "saa_eval_moments: prologue");
  if (s != SAA_OK) return s;
  const int et = (int)(d < 256 ? (d + 31) / 32 * 32 : 256);
  k_gram_eval<<<K, et, sizeof(double) * d, st>>>(K, prob->d, (double)prob->N, prob->lambda, M, mt, w.Y64, w.c, f,
                                                 pbar, var, grad ? u : nullptr);
  int launched = 2;
  if (grad) {
    launch_grad_out(K, prob->d, prob->chol, prob->mu, u, grad, st);
    ++launched;
  }
  ctx->kernels += launched;
  return cuda_status(cudaGetLastError(), "saa_eval_moments: launch");
}
