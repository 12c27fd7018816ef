// tc_grad.cu -- tcgen05 tensor-core path of the SAA estimate together with
// its gradient in w (Eq. 4 with Eq. 5, Sec. 3.1), for d <= 1024, K <= 64.
//
// With a_i = s_i zhat_i (the whitened samples), y_k = C'w_k and
// Q_ik = a_i'y_k, the gradient needs, per decision k, the d-vector
// G_k = sum_i a_i Q_ik besides S1_k, S2_k and m~ = sum_i a_i.  Per CTA (one
// per SM, persistent over 128-scenario tiles), per tile:
//   forward   the generator warps write the tile of a_i, 64 dimensions per
//             stage (K-major, 128-byte swizzle), while bulk TMA brings the
//             matching 64-dimension slice of the decision operand into the
//             same stage; one thread issues hi*hi and hi*lo + lo*hi (the
//             split-precision forward of the value kernel, FP16 or BF16).
//   epilogue  four warps read Q, keep S2_k in FP64 registers and write
//             W = Q 2^-f_k (2^f_k > |y_k|_2 in operand units, so |W_ik| <=
//             |a_i|_2) as hi/lo of the operand type into shared memory,
//             K-major over the tile's scenarios: the adjoint's second operand.
//   adjoint   the generator warps draw the same tile again, transposed: 128
//             dimensions x 128 scenarios per stage; the MMA thread issues
//             G += A' W (hi/lo, three products, hi*hi into G1 and the
//             corrections into G2) into one of two TMEM buffer pairs, and the
//             epilogue folds each 128-dimension block into the CTA's
//             Kahan-carried FP32 partial of G in global memory.  The same
//             stage also yields the CTA's partial of m~.
// The tensor core rounds every update of an accumulator with a bias toward
// zero, so a running sum over T k steps loses about T/2 of its low-order
// units in the last place: at d = 1024 (64 steps) that is 2e-6 of Q.  The
// hi*hi products therefore go, 8 k steps (128 dimensions) at a time, into
// one of two chunk accumulators that the epilogue folds into a running Q in
// TMEM with round-to-nearest FP32 additions; the small corrections keep one
// accumulator per tile.  The bias then stays near 4 units in the last
// place whatever d is.
// Drawing each tile twice costs a second pass of the generator but keeps
// A out of shared memory (a 128 x 1024 tile in hi/lo would need 512 KB).
// The adjoint's representation error changes sign and size from scenario to
// scenario, so it shrinks like sqrt(d / N) relative to G: FP16 hi/lo (2^-22
// per product) keeps it below 1e-6 from N ~ d upwards, where BF16 hi/lo
// (2^-17) would not.
// Every mbarrier wait is clock-bounded: on expiry the kernel raises the error
// word, drains its MMAs and copies, frees its TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "gen.cuh"
#include "internal.cuh"
#include "tc_ptx.cuh"

namespace saa {
namespace tc {

constexpr int kGM = 128;               // scenarios per tile (MMA M of the forward)
constexpr int kGKB = 64;               // dimensions per forward stage
constexpr int kGMB = 128;              // dimensions per adjoint stage (MMA M of the adjoint)
constexpr int kGStages = 3;
constexpr int kGStageBytes = 65536;    // forward: A hi+lo 32 KB + B slice <= 16 KB; adjoint: A' hi+lo 64 KB
constexpr int kGSubBytes = kGMB * 128; // adjoint: one [128 dims][64 scenarios] bf16 block
constexpr int kGEpiWarps = 4;
constexpr int kGMmaWarp = 4;           // warps 0..3 epilogue, 4 MMA, 5.. generator
constexpr int kGRngWarps = 16;
constexpr int kGThreads = 32 * (5 + kGRngWarps);
constexpr int kGRngThreads = 32 * kGRngWarps;
constexpr int kGMaxKp = 64;
constexpr int kGMaxDim = 1024;
constexpr int kGSBufs = 4;
constexpr int kGChunkStages = 2;       // forward stages (8 k steps) per hi*hi chunk accumulator
static_assert(kGRngThreads == 512, "adjoint stage mapping assumes 512 generator threads");

struct GArgs {
  LawArgs la;
  int K, Kp, nkb, nmb;
  int64_t tiles;
  const uint8_t* bimage;   // [nkb][hi, lo][Kp][128 B], swizzled
  const double* gaux;      // [2K]: 2^(e_k + f_k) (G at true scale), then 2^-f_k (W)
  const double* scale2;    // [K] 4^e_k  (S2 at true scale)
  double* part_s2;         // [grid][K]
  double* part_m;          // [grid][d]
  float* part_g;           // [grid][K][d]
  float* part_gc;          // [grid][K][d] Kahan compensation (true sum = part_g - part_gc)
  uint32_t* err;
};

struct GSmem {
  uint64_t a_full[kGStages];    // generator warps' stores into the stage
  uint64_t a_empty[kGStages];   // MMAs reading the stage done
  uint64_t b_full[kGStages];    // decision-operand slice landed (forward stages)
  uint64_t s_ready[kGSBufs];    // t-law scales of a tile
  uint64_t c_full[2], c_empty[2];   // hi*hi chunk accumulators
  uint64_t q_full, q_empty, w_full, w_empty;
  uint64_t g_full[2], g_empty[2];
  uint64_t drain;
  uint32_t tmem_base;
  uint32_t abort_flag;
  float s_buf[kGSBufs][kGM];
  float gsc_f[kGMaxKp];   // 2^(e_k + f_k)
  float wsc_f[kGMaxKp];   // 2^-f_k
};

// Layout: [stages][W: 2 scenario blocks x hi/lo x Kp rows x 128 B][GSmem]; 1024-byte aligned base.
size_t grad_smem_bytes(int Kp) { return (size_t)kGStages * kGStageBytes + (size_t)4 * Kp * 128 + sizeof(GSmem); }

// D8: d is a multiple of 8, so every unit below d is whole and the
// per-element guards drop out.
template <bool F16, bool D8>
__global__ void __launch_bounds__(kGThreads, 1) k_tc_grad(GArgs a) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  const uint32_t base = smem_u32(smem_raw);
  if (base & 1023u) {
    if (threadIdx.x == 0) atomicOr(a.err, kErrBounds);
    return;
  }
  const int Kp = a.Kp;
  uint8_t* ring = smem_raw;
  uint8_t* wbuf = smem_raw + kGStages * kGStageBytes;
  GSmem* sm = reinterpret_cast<GSmem*>(wbuf + 4 * Kp * 128);
  const uint32_t sRing = base, sW = base + (uint32_t)(kGStages * kGStageBytes);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const LawArgs& la = a.la;
  const int d = la.d;
  const uint32_t bslice = (uint32_t)(2 * Kp * 128);   // one forward slice of the decision operand
  volatile uint32_t* abort_flag = &sm->abort_flag;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kGStages; ++s) {
      mbar_init(smem_u32(&sm->a_full[s]), kGRngWarps);
      mbar_init(smem_u32(&sm->a_empty[s]), 1);
      mbar_init(smem_u32(&sm->b_full[s]), 1);
    }
    for (int s = 0; s < kGSBufs; ++s) mbar_init(smem_u32(&sm->s_ready[s]), kGM / 32);
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&sm->c_full[b]), 1);
      mbar_init(smem_u32(&sm->c_empty[b]), kGEpiWarps);
    }
    mbar_init(smem_u32(&sm->q_full), 1);
    mbar_init(smem_u32(&sm->q_empty), kGEpiWarps);
    mbar_init(smem_u32(&sm->w_full), kGEpiWarps);
    mbar_init(smem_u32(&sm->w_empty), 1);
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&sm->g_full[b]), 1);
      mbar_init(smem_u32(&sm->g_empty[b]), kGEpiWarps);
    }
    mbar_init(smem_u32(&sm->drain), 1);
    sm->abort_flag = 0u;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int k = threadIdx.x; k < kGMaxKp; k += blockDim.x) {
    sm->gsc_f[k] = (k < a.K) ? (float)a.gaux[k] : 0.0f;
    sm->wsc_f[k] = (k < a.K) ? (float)a.gaux[a.K + k] : 0.0f;
  }
  // TMEM, Kp columns each: two hi*hi chunk accumulators, the running Q, the
  // corrections D2, and two (G1, G2) pairs
  const uint32_t ncols = (8 * Kp <= 256) ? 256u : 512u;
  if (warp == kGMmaWarp) tmem_alloc(smem_u32(&sm->tmem_base), ncols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sm->tmem_base;
  const uint32_t tq = tmem + 2u * Kp, td2 = tmem + 3u * Kp;
  const int nchunk = (a.nkb + kGChunkStages - 1) / kGChunkStages;
  const int my_tiles = (int)((a.tiles - blockIdx.x + gridDim.x - 1) / gridDim.x);
  const int per_tile = a.nkb + a.nmb;
  double s2acc[kGMaxKp / 32];

  if (warp == kGMmaWarp) {
    // ------------------------------------------------------------ MMA ---
    if (lane == 0) {
      bool ok = true;
      const uint32_t idf = idesc_f16(kGM, Kp, F16);
      const uint32_t ida = idesc_f16(kGMB, Kp, F16);
      int st = 0, gcount = 0, ccount = 0;
      uint32_t ph = 0, bph = 0;   // bph: bit s = phase parity of b_full[s]
      for (int tt = 0; ok && tt < my_tiles; ++tt) {
        if (tt > 0) ok = mbar_wait(smem_u32(&sm->q_empty), (uint32_t)((tt - 1) & 1), abort_flag, a.err);
        for (int kb = 0; ok && kb < a.nkb; ++kb) {
          const int cb = ccount & 1;
          const bool c_first = (kb % kGChunkStages) == 0;
          const bool c_last = (kb % kGChunkStages) == kGChunkStages - 1 || kb == a.nkb - 1;
          if (c_first) {
            ok = mbar_wait(smem_u32(&sm->c_empty[cb]), (uint32_t)(((ccount >> 1) & 1) ^ 1), abort_flag, a.err);
            if (!ok) break;
          }
          const uint32_t tc1 = tmem + (uint32_t)(cb * Kp);
          ok = mbar_wait(smem_u32(&sm->a_full[st]), ph, abort_flag, a.err) &&
               mbar_wait(smem_u32(&sm->b_full[st]), (bph >> st) & 1u, abort_flag, a.err);
          if (!ok) break;
          bph ^= 1u << st;
          tc_fence_after();
          const uint32_t a_hi = sRing + (uint32_t)(st * kGStageBytes);
          const uint32_t a_lo = a_hi + kGM * 128;
          const uint32_t b_hi = a_hi + 2 * kGM * 128;
          const uint32_t b_lo = b_hi + (uint32_t)(Kp * 128);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {   // 16 dimensions per k step
            const uint32_t o = (uint32_t)(kk * 32);
            mma_bf16(tc1, desc_sw128(a_hi + o), desc_sw128(b_hi + o), idf, (c_first && kk == 0) ? 0u : 1u);
            mma_bf16(td2, desc_sw128(a_hi + o), desc_sw128(b_lo + o), idf, (kb == 0 && kk == 0) ? 0u : 1u);
            mma_bf16(td2, desc_sw128(a_lo + o), desc_sw128(b_hi + o), idf, 1u);
          }
          mma_commit(smem_u32(&sm->a_empty[st]));
          if (c_last) {
            mma_commit(smem_u32(&sm->c_full[cb]));
            ++ccount;
          }
          if (++st == kGStages) { st = 0; ph ^= 1u; }
        }
        if (!ok) break;
        mma_commit(smem_u32(&sm->q_full));
        ok = mbar_wait(smem_u32(&sm->w_full), (uint32_t)(tt & 1), abort_flag, a.err);
        for (int mb = 0; ok && mb < a.nmb; ++mb, ++gcount) {
          const int gb = gcount & 1;
          const uint32_t tg1 = tmem + (uint32_t)((4 + 2 * gb) * Kp), tg2 = tg1 + (uint32_t)Kp;
          ok = mbar_wait(smem_u32(&sm->g_empty[gb]), (uint32_t)(((gcount >> 1) & 1) ^ 1), abort_flag, a.err) &&
               mbar_wait(smem_u32(&sm->a_full[st]), ph, abort_flag, a.err);
          if (!ok) break;
          tc_fence_after();
          const uint32_t stage = sRing + (uint32_t)(st * kGStageBytes);
#pragma unroll
          for (int kk = 0; kk < 8; ++kk) {   // 16 scenarios per k step
            const int sb = kk >> 2;
            const uint32_t o = (uint32_t)((kk & 3) * 32);
            const uint32_t at_hi = stage + (uint32_t)((sb * 2 + 0) * kGSubBytes) + o;
            const uint32_t at_lo = stage + (uint32_t)((sb * 2 + 1) * kGSubBytes) + o;
            const uint32_t w_hi = sW + (uint32_t)((sb * 2 + 0) * Kp * 128) + o;
            const uint32_t w_lo = sW + (uint32_t)((sb * 2 + 1) * Kp * 128) + o;
            const uint32_t acc0 = (kk == 0) ? 0u : 1u;
            mma_bf16(tg1, desc_sw128(at_hi), desc_sw128(w_hi), ida, acc0);
            mma_bf16(tg2, desc_sw128(at_hi), desc_sw128(w_lo), ida, acc0);
            mma_bf16(tg2, desc_sw128(at_lo), desc_sw128(w_hi), ida, 1u);
          }
          mma_commit(smem_u32(&sm->a_empty[st]));
          mma_commit(smem_u32(&sm->g_full[gb]));
          if (++st == kGStages) { st = 0; ph ^= 1u; }
        }
        if (!ok) break;
        mma_commit(smem_u32(&sm->w_empty));
      }
      // every MMA issued above completes before TMEM is released
      mma_commit(smem_u32(&sm->drain));
      uint32_t never = 0u;
      mbar_wait(smem_u32(&sm->drain), 0, &never, a.err);
    }
    __syncwarp();
  } else if (warp < kGEpiWarps) {
    // ------------------------------------------------------- epilogue ---
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
#pragma unroll
    for (int g = 0; g < kGMaxKp / 32; ++g) s2acc[g] = 0.0;
    const int row = warp * 32 + lane;          // forward: scenario of this TMEM lane
    const int wsb = row >> 6, wil = row & 63;  // its 64-scenario block and position
    uint8_t* w_hi = wbuf + wsb * 2 * Kp * 128;
    uint8_t* w_lo = w_hi + Kp * 128;
    int gcount = 0, ccount = 0;
    for (int tt = 0; tt < my_tiles; ++tt) {
      // fold the hi*hi chunks into the running Q (round to nearest)
      bool cok = true;
      for (int c = 0; c < nchunk; ++c, ++ccount) {
        const int cb = ccount & 1;
        if (!warp_wait(smem_u32(&sm->c_full[cb]), (uint32_t)((ccount >> 1) & 1), abort_flag, a.err)) {
          cok = false;
          break;
        }
        tc_fence_after();
#pragma unroll 1
        for (int c0 = 0; c0 < Kp; c0 += 16) {
          uint32_t ra[16], rq[16];
          tmem_ld16(tmem + (uint32_t)(cb * Kp + c0) + lane_base, ra);
          if (c > 0) tmem_ld16(tq + (uint32_t)c0 + lane_base, rq);
          tmem_wait_ld();
          if (c > 0) {
#pragma unroll
            for (int i = 0; i < 16; ++i) ra[i] = __float_as_uint(__uint_as_float(ra[i]) + __uint_as_float(rq[i]));
          }
          tmem_st16(tq + (uint32_t)c0 + lane_base, ra);
          tmem_wait_st();
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&sm->c_empty[cb]));
      }
      if (!cok) break;
      if (!warp_wait(smem_u32(&sm->q_full), (uint32_t)(tt & 1), abort_flag, a.err)) break;
      if (tt > 0 && !warp_wait(smem_u32(&sm->w_empty), (uint32_t)((tt - 1) & 1), abort_flag, a.err)) break;
      tc_fence_after();
#pragma unroll 1
      for (int pc = 0; pc < Kp / 16; ++pc) {
        const uint32_t c0 = (uint32_t)(16 * pc);
        uint32_t r1[16], r2[16];
        tmem_ld16(tq + lane_base + c0, r1);
        tmem_ld16(td2 + lane_base + c0, r2);
        tmem_wait_ld();
        float v[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const float q = __uint_as_float(r1[i]) + __uint_as_float(r2[i]);
          const int k = (int)c0 + i;
          // element (k, row) of W: row k of the operand, 16-byte unit wil/8 swizzled by k
          const float wq = q * sm->wsc_f[k];   // power of two: exact
          const uint32_t hp = pack2<F16>(wq, 0.0f);
          const uint32_t lp = pack2<F16>(wq - unpack2<F16>(hp).x, 0.0f);
          const uint32_t off = (uint32_t)(k * 128 + (((wil >> 3) ^ (k & 7)) << 4) + (wil & 7) * 2);
          *reinterpret_cast<uint16_t*>(w_hi + off) = (uint16_t)(hp & 0xffffu);
          *reinterpret_cast<uint16_t*>(w_lo + off) = (uint16_t)(lp & 0xffffu);
          v[i] = q * q;
        }
        // reduce-scatter over the warp's 32 rows: lanes l and l + 16 end with column c0 + (l & 15)
#pragma unroll
        for (int w = 8; w >= 1; w >>= 1) {
          const bool upper = (lane & w) != 0;
#pragma unroll
          for (int i = 0; i < w; ++i) {
            const float send = upper ? v[i] : v[i + w];
            const float keep = upper ? v[i + w] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, w);
          }
        }
        v[0] += __shfl_xor_sync(0xffffffffu, v[0], 16);
        // lane l keeps column 32 g + l of s2acc[g]
#pragma unroll
        for (int h = 0; h < kGMaxKp / 32; ++h)
          if (h == (pc >> 1) && (lane >> 4) == (pc & 1)) s2acc[h] += (double)v[0];
      }
      fence_proxy_async();   // W: generic-proxy stores -> the MMA's async-proxy reads
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(smem_u32(&sm->w_full));
        mbar_arrive(smem_u32(&sm->q_empty));
      }
      // fold each adjoint block into the CTA's partial of G
      bool ok = true;
      for (int mb = 0; mb < a.nmb; ++mb, ++gcount) {
        const int gb = gcount & 1;
        const uint32_t tg1 = tmem + (uint32_t)((4 + 2 * gb) * Kp), tg2 = tg1 + (uint32_t)Kp;
        if (!warp_wait(smem_u32(&sm->g_full[gb]), (uint32_t)((gcount >> 1) & 1), abort_flag, a.err)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const int j = mb * kGMB + warp * 32 + lane;   // dimension of this TMEM lane
#pragma unroll 1
        for (int c0 = 0; c0 < Kp; c0 += 16) {
          uint32_t r1[16], r2[16];
          tmem_ld16(tg1 + lane_base + (uint32_t)c0, r1);
          tmem_ld16(tg2 + lane_base + (uint32_t)c0, r2);
          tmem_wait_ld();
          const int kn = a.K - c0;   // valid columns of this batch (may be <= 0)
          if (j < d && kn > 0) {
            float gv[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) gv[i] = (__uint_as_float(r1[i]) + __uint_as_float(r2[i])) * sm->gsc_f[c0 + i];
            const size_t e0 = ((size_t)blockIdx.x * a.K + c0) * d + j;
            if (tt == 0) {
#pragma unroll
              for (int i = 0; i < 16; ++i)
                if (i < kn) {
                  a.part_g[e0 + (size_t)i * d] = gv[i];
                  a.part_gc[e0 + (size_t)i * d] = 0.0f;
                }
            } else {
#pragma unroll
              for (int hb = 0; hb < 16; hb += 8) {   // two halves: 16 loads in flight, fewer live registers
                float ps[8], pc[8];
#pragma unroll
                for (int i = 0; i < 8; ++i)
                  if (hb + i < kn) {
                    ps[i] = a.part_g[e0 + (size_t)(hb + i) * d];
                    pc[i] = a.part_gc[e0 + (size_t)(hb + i) * d];
                  }
#pragma unroll
                for (int i = 0; i < 8; ++i)
                  if (hb + i < kn) {
                    const float y = gv[hb + i] - pc[i];
                    const float t = ps[i] + y;
                    a.part_gc[e0 + (size_t)(hb + i) * d] = (t - ps[i]) - y;
                    a.part_g[e0 + (size_t)(hb + i) * d] = t;
                  }
              }
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&sm->g_empty[gb]));
      }
      if (!ok) break;
    }
  } else {
    // ------------------------------------------------------------ RNG ---
    const int rt = threadIdx.x - 32 * (kGMmaWarp + 1);   // 0 .. 511
    uint32_t epoch = la.epoch;
    if (la.t_dev) epoch += (uint32_t)(*la.t_dev / la.M);
    const gen::Stream gs = gen::make_stream(la.seed, epoch, la.instance);
    const uint32_t half = la.N / 2u;
    const bool tlaw = la.law == SAA_LAW_STUDENT_T;
    // forward stage: 16-byte unit cu (8 dimensions) of rows rt/8 and rt/8 + 64
    const int cu = rt & 7;
    // adjoint stage: dimensions 4 b4 .. 4 b4 + 3 of the block, scenarios 8 g8 .. 8 g8 + 7,
    // written one scenario pair (4 bytes) at a time; the pair order is staggered by
    // lane group so that each store instruction covers all 32 banks once
    const int b4 = rt >> 4, g8 = rt & 15;
    const int asb = g8 >> 3, au = g8 & 7;
    const int pfirst = lane >> 3;
    int st = 0;
    uint32_t ph = 0;
    uint32_t bissued = 0, bpar = 0;   // copy issuer: stages with copies, parity of the next copy per stage
    const int iters = my_tiles * per_tile;
    for (int it = 0; it < iters; ++it) {
      const int tt = it / per_tile;
      const int pt = it - tt * per_tile;
      const uint32_t tile = blockIdx.x + (uint32_t)tt * gridDim.x;
      const uint32_t i0 = la.i_base + tile * (uint32_t)kGM;
      const int nrow = (int)min((uint32_t)kGM, la.rows_end() - i0);
      const int sb4 = tt & (kGSBufs - 1);
      const uint32_t s_bar = smem_u32(&sm->s_ready[sb4]);
      if (tlaw && pt == 0 && rt < kGM) {   // generator warps 0..3 draw the tile's scales
        sm->s_buf[sb4][rt] = (rt < nrow) ? gen::t_scale_f(gs, i0 + (uint32_t)rt, la.nu) : 0.0f;
        __syncwarp();
        if (lane == 0) mbar_arrive(s_bar);
      }
      if (!warp_wait(smem_u32(&sm->a_empty[st]), ph ^ 1u, abort_flag, a.err)) break;
      if (tlaw && !warp_wait(s_bar, (uint32_t)((tt >> 2) & 1), abort_flag, a.err)) break;
      uint8_t* stage = ring + st * kGStageBytes;
      if (pt < a.nkb) {
        // ---- forward stage: dimensions 64 kb .. 64 kb + 63 of the tile
        const int kb = pt;
        if (rt == 0) {
          const uint32_t bb = smem_u32(&sm->b_full[st]);
          mbar_expect_tx(bb, bslice);
          bulk_g2s(sRing + (uint32_t)(st * kGStageBytes) + 2u * kGM * 128u, a.bimage + (size_t)kb * bslice, bslice,
                   bb);
          bissued |= 1u << st;
          bpar ^= 1u << st;
        }
        const int j0 = kb * kGKB + cu * 8;
#pragma unroll 1
        for (int r = rt >> 3; r < kGM; r += kGRngThreads / 8) {
          float v[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) v[e] = 0.0f;
          if (r < nrow && j0 < d) {
            const uint32_t i = i0 + (uint32_t)r;
            const bool logn = gen::is_lognormal(la.law, i, half);
            float z[4];
            gen::Gen<float>::block(gs, (uint32_t)(j0 >> 2), i, logn, z);
#pragma unroll
            for (int e = 0; e < 4; ++e) v[e] = (D8 || j0 + e < d) ? z[e] : 0.0f;
            if (D8 || j0 + 4 < d) {
              gen::Gen<float>::block(gs, (uint32_t)(j0 >> 2) + 1u, i, logn, z);
#pragma unroll
              for (int e = 0; e < 4; ++e) v[4 + e] = (D8 || j0 + 4 + e < d) ? z[e] : 0.0f;
            }
            if (tlaw) {
              const float s = sm->s_buf[sb4][r];
#pragma unroll
              for (int e = 0; e < 8; ++e) v[e] *= s;
            }
          }
          uint32_t hi[4], lo[4];
#pragma unroll
          for (int e = 0; e < 8; e += 2) {
            hi[e / 2] = pack2<F16>(v[e], v[e + 1]);
            const float2 h = unpack2<F16>(hi[e / 2]);
            lo[e / 2] = pack2<F16>(v[e] - h.x, v[e + 1] - h.y);
          }
          const uint32_t off = sw_off(r, cu);
          *reinterpret_cast<uint4*>(stage + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
          *reinterpret_cast<uint4*>(stage + kGM * 128 + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
      } else {
        // ---- adjoint stage: dimensions 128 mb .. 128 mb + 127, transposed
        const int mb = pt - a.nkb;
        const int jb = mb * kGMB + 4 * b4;   // first of this thread's 4 dimensions
        float msum[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll 1
        for (int p = 0; p < 4; ++p) {
          const int pq = (p + pfirst) & 3;   // scenarios 8 g8 + 2 pq, + 1
          const int r0 = 8 * g8 + 2 * pq;
          float z0[4] = {0.0f, 0.0f, 0.0f, 0.0f}, z1[4] = {0.0f, 0.0f, 0.0f, 0.0f};
          if (jb < d) {
            if (r0 < nrow) {
              const uint32_t i = i0 + (uint32_t)r0;
              gen::Gen<float>::block(gs, (uint32_t)(jb >> 2), i, gen::is_lognormal(la.law, i, half), z0);
              if (tlaw) {
                const float s0 = sm->s_buf[sb4][r0];
#pragma unroll
                for (int e = 0; e < 4; ++e) z0[e] *= s0;
              }
#pragma unroll
              for (int e = 0; e < 4; ++e) z0[e] = (D8 || jb + e < d) ? z0[e] : 0.0f;
            }
            if (r0 + 1 < nrow) {
              const uint32_t i = i0 + (uint32_t)r0 + 1u;
              gen::Gen<float>::block(gs, (uint32_t)(jb >> 2), i, gen::is_lognormal(la.law, i, half), z1);
              if (tlaw) {
                const float s1 = sm->s_buf[sb4][r0 + 1];
#pragma unroll
                for (int e = 0; e < 4; ++e) z1[e] *= s1;
              }
#pragma unroll
              for (int e = 0; e < 4; ++e) z1[e] = (D8 || jb + e < d) ? z1[e] : 0.0f;
            }
          }
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            msum[e] += z0[e] + z1[e];
            const int jr = 4 * b4 + e;   // row of the stage
            const uint32_t h = pack2<F16>(z0[e], z1[e]);
            const float2 f = unpack2<F16>(h);
            const uint32_t l = pack2<F16>(z0[e] - f.x, z1[e] - f.y);
            const uint32_t off = (uint32_t)(jr * 128 + ((au ^ (jr & 7)) << 4) + pq * 4);
            *reinterpret_cast<uint32_t*>(stage + (asb * 2 + 0) * kGSubBytes + off) = h;
            *reinterpret_cast<uint32_t*>(stage + (asb * 2 + 1) * kGSubBytes + off) = l;
          }
        }
        // m~: fold the 16 lanes that share these dimensions; lane g8 == 0 owns
        // them for the whole kernel, so its additions reach part_m in program order
#pragma unroll
        for (int e = 0; e < 4; ++e) {
#pragma unroll
          for (int o = 1; o < 16; o <<= 1) msum[e] += __shfl_xor_sync(0xffffffffu, msum[e], o);
        }
        if (g8 == 0) {
#pragma unroll
          for (int e = 0; e < 4; ++e)
            if (jb + e < d) {
              double* pm = a.part_m + (size_t)blockIdx.x * d + jb + e;
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
      if (++st == kGStages) { st = 0; ph ^= 1u; }
    }
    if (rt == 0) {
      // the last copy into each stage has landed before the CTA moves on (after an abort too)
      uint32_t never = 0u;
      for (int s = 0; s < kGStages; ++s)
        if ((bissued >> s) & 1u) mbar_wait(smem_u32(&sm->b_full[s]), ((bpar >> s) & 1u) ^ 1u, &never, a.err);
    }
  }

  // ----------------------------------------------------- CTA reductions ---
  __syncthreads();   // MMAs and copies drained: the stages are free
  double* red_s2 = reinterpret_cast<double*>(ring);   // [kGEpiWarps][kGMaxKp]
  if (warp < kGEpiWarps) {
#pragma unroll
    for (int g = 0; g < kGMaxKp / 32; ++g)
      if (32 * g < Kp) red_s2[warp * kGMaxKp + 32 * g + lane] = s2acc[g];
  }
  __syncthreads();
  for (int k = threadIdx.x; k < a.K; k += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < kGEpiWarps; ++w) s += red_s2[w * kGMaxKp + k];
    a.part_s2[(size_t)blockIdx.x * a.K + k] = s * a.scale2[k];
  }
  if (warp == kGMmaWarp) {
    tc_fence_after();
    tmem_dealloc(tmem, ncols);
  }
}

}  // namespace tc

bool tc_grad_supported(const saa_problem* p, int K) { return p->d <= tc::kGMaxDim && K <= tc::kGMaxKp; }

static size_t grad_image_bytes(int K, int d) {
  const int Kp = (K + 31) / 32 * 32;
  const int nkb = (d + tc::kGKB - 1) / tc::kGKB;
  return (size_t)nkb * 2 * Kp * 128;
}

saa_status tc_grad_plan(const saa_ctx* ctx, const saa_problem* p, int K, Plan* plan) {
  const int Kp = (K + 31) / 32 * 32;
  plan->bm = tc::kGM;
  plan->tiles = (p->N + tc::kGM - 1) / tc::kGM;
  plan->grid = (int)(plan->tiles < ctx->sm_count ? plan->tiles : ctx->sm_count);
  plan->smem = (int)tc::grad_smem_bytes(Kp);
  // operand image, then scale2[K], gaux[2K]
  plan->tc_bytes = grad_image_bytes(K, p->d) + (size_t)24 * K;
  if (plan->smem > ctx->smem_optin) {
    set_error("tensor-core gradient tile does not fit in shared memory");
    return SAA_EUNSUPPORTED;
  }
  return SAA_OK;
}

cudaError_t launch_tc_grad(const LawArgs& la, int K, int prec, const Plan& plan, const Workspace& ws, uint32_t* err,
                           cudaStream_t st) {
  const bool f16 = (prec == SAA_F16X3);
  tc::GArgs a;
  a.la = la;
  a.K = K;
  a.Kp = (K + 31) / 32 * 32;
  a.nkb = (la.d + tc::kGKB - 1) / tc::kGKB;
  a.nmb = (la.d + tc::kGMB - 1) / tc::kGMB;
  a.tiles = plan.tiles;
  uint8_t* img = (uint8_t*)ws.tc;
  double* scale2 = (double*)(img + grad_image_bytes(K, la.d));
  double* gaux = scale2 + K;
  a.bimage = img;
  a.gaux = gaux;
  a.scale2 = scale2;
  a.part_s2 = ws.part_s2;
  a.part_m = ws.part_m;
  a.part_g = (float*)ws.part_g;
  a.part_gc = (float*)ws.part_gc;
  a.err = err;
  cudaError_t e = launch_tc_image(la.d, K, a.Kp, a.nkb, f16, ws.Y64, scale2, gaux, img, st);
  if (e != cudaSuccess) return e;
  const bool d8 = (la.d & 7) == 0;
  auto kern = f16 ? (d8 ? tc::k_tc_grad<true, true> : tc::k_tc_grad<true, false>)
                  : (d8 ? tc::k_tc_grad<false, true> : tc::k_tc_grad<false, false>);
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, plan.smem);
  if (e != cudaSuccess) return e;
  kern<<<plan.grid, tc::kGThreads, plan.smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace saa
