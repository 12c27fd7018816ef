// tc_stream.cu -- saa_eval_samples: Eq. 4 on samples held in device memory
// (the streamed form of the estimate: scenarios read from HBM instead of
// regenerated), on tcgen05 tensor cores fed by TMA tensor loads.
//
// For samples R_i (FP32, [N][d] row-major), a center c (the caller's mean
// estimate, or 0), per-column spreads sigma (or 1) and decisions x_k:
//   p_ik = c'x_k + sum_j v_ij x'_kj,  v_ij = (R_ij - c_j) 2^-a_j,
//   x'_kj = x_kj 2^a_j,  2^(a_j - 1) < sigma_j <= 2^a_j.
// The power-of-two scaling is exact; it keeps the operands of the split
// products in the normal range of the 16-bit types.  The contraction
// Q_ik = v_i'x'_k runs in split precision like the value kernel;
// S1_k = m~'x'_k with m~ = sum_i v_i and S2_k = sum_i Q_ik^2 give p_bar, V
// and f_hat as in saa_eval.  Centring keeps the variance well-conditioned
// when the samples' mean is far from 0.
//
// Per CTA (one per SM, persistent over 128-row tiles), per 64-column K block:
//   producer   one thread loads the block's two FP32 boxes (columns 0-31 and
//              32-63, 128 rows, 128-byte swizzle) by TMA tensor loads into
//              the two 16 KB halves of a stage;
//   converters 16 warps; the four threads of each row read their 16 values,
//              subtract c, split them into hi + lo of the operand type and,
//              after a warp sync, write hi over the first half's row and lo
//              over the second half's row -- exactly the K-major 128-byte
//              swizzled layout tcgen05.mma reads (no other thread touches the
//              row, so the conversion is in place);
//   MMA and epilogue as in the value kernel (hi*hi into D1, corrections
//              into D2, S2 reduce-scatter in FP64 registers).
// m~ comes from the converters: each warp reduce-scatters its 8 rows by
// shuffles, every lane keeps float-float running sums of its two columns per
// K block, and the CTA folds its 16 warps in warp order at the end
// (deterministic).  Every wait is bounded.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "internal.cuh"
#include "tc_ptx.cuh"

namespace saa {
namespace tc {

constexpr int kSM = 128;                  // rows (scenarios) per tile = MMA M
constexpr int kSKB = 64;                  // columns per K block
constexpr int kSMaxStages = 6;            // stages in flight: as many as shared memory holds
constexpr int kSStageBytes = 2 * kSM * 128;   // two 16 KB halves (FP32 boxes in, hi/lo out)
#ifndef SAA_STREAM_EPI_WARPS
#define SAA_STREAM_EPI_WARPS 8
#endif
constexpr int kSEpi = SAA_STREAM_EPI_WARPS;   // epilogue warps: 4 or 8 (two per TMEM lane quadrant)
constexpr int kSEpiStride = kSEpi / 4;        // column groups are dealt round-robin over a quadrant's warps
constexpr int kSMma = kSEpi;
constexpr int kSProd = kSEpi + 1;
constexpr int kSConv = 16;                // converter warps (8 rows each)
constexpr int kSThreads = 32 * (kSEpi + 2 + kSConv);
static_assert(kSEpi == 4 || kSEpi == 8, "4 or 8 epilogue warps");
constexpr int kSMaxKp = 256;

struct SArgs {
  int d, K, Kp, nkb, nst;
  uint32_t N;
  int64_t tiles;
  const float* ncs;       // [dpad] -fl32(c_j) 2^-a_j (0 past d)
  const float* isf;       // [dpad] 2^-a_j (0 past d)
  const uint8_t* bimage;  // [nkb][hi, lo][Kp][128 B]
  const double* scale2;   // [K]
  double* part_s2;        // [grid][K]
  double* part_m;         // [grid][dpad]
  uint32_t* err;
#ifdef SAA_BOUNDS_CHECK
  size_t n_s2, n_m;       // elements of part_s2 and part_m
#endif
};

// 16-byte aligned size: the FP32 center / scale arrays that follow it are
// read as float4.
struct alignas(16) SSmem {
  uint64_t ld_full[kSMaxStages];
  uint64_t a_full[kSMaxStages];
  uint64_t a_empty[kSMaxStages];
  uint64_t q_full[2], q_empty[2];   // accumulator slots: MMA -> epilogue, epilogue -> MMA
  uint64_t b_full, drain;
  uint32_t tmem_base;
  uint32_t abort_flag;
};

static_assert(sizeof(SSmem) % 16 == 0, "the arrays after SSmem are read as float4");

// Bytes of the decision image: per K block two planes (hi, lo) of Kp rows x
// 128 B for the 16-bit types; for E4M3 the 3 nkb 64-dimension halves (B1 of
// every block, then B2, then B3) packed two to a 128-byte row, half h in
// plane h / 2 at byte (h % 2) 64.
__host__ __device__ constexpr int img_bytes(int Kp, int nkb, bool f8) {
  return (f8 ? (3 * nkb + 1) / 2 : 2 * nkb) * Kp * 128;
}

size_t stream_smem_bytes(int Kp, int nkb, int nst, bool f8) {
  return (size_t)nst * kSStageBytes + (size_t)img_bytes(Kp, nkb, f8) + sizeof(SSmem) +
         2 * sizeof(float) * (size_t)nkb * kSKB;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void* tmap, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(tmap), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// P: 0 BF16 hi/lo, 1 FP16 hi/lo (three products each), 2 E4M3 (samples
// split hi/lo, decisions in three terms, four products).
template <int P, int NKB>
__global__ void __launch_bounds__(kSThreads, 1) k_tc_stream(SArgs a, const __grid_constant__ CUtensorMap tmap) {
  constexpr bool F16 = P == 1;
  constexpr bool F8 = P == 2;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  const uint32_t base = smem_u32(smem_raw);
  if (base & 1023u) {
    if (threadIdx.x == 0) atomicOr(a.err, kErrBounds);
    return;
  }
  const int bbytes = img_bytes(a.Kp, a.nkb, F8);
  uint8_t* As = smem_raw;
  const int nst = a.nst;
  SSmem* sm = reinterpret_cast<SSmem*>(smem_raw + nst * kSStageBytes + bbytes);
  const int dpad = a.nkb * kSKB;
  float* s_cf = reinterpret_cast<float*>(sm + 1);   // [dpad] -c_j 2^-a_j
  float* s_is = s_cf + dpad;                        // [dpad]
  const uint32_t sA = base, sB = base + (uint32_t)(nst * kSStageBytes);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  volatile uint32_t* abort_flag = &sm->abort_flag;

  if (threadIdx.x == 0) {
    for (int s = 0; s < nst; ++s) {
      mbar_init(smem_u32(&sm->ld_full[s]), 1);
      mbar_init(smem_u32(&sm->a_full[s]), kSConv);
      mbar_init(smem_u32(&sm->a_empty[s]), 1);
    }
    for (int q = 0; q < 2; ++q) {
      mbar_init(smem_u32(&sm->q_full[q]), 1);
      mbar_init(smem_u32(&sm->q_empty[q]), kSEpi);
    }
    mbar_init(smem_u32(&sm->b_full), 1);
    mbar_init(smem_u32(&sm->drain), 1);
    sm->abort_flag = 0u;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int j = threadIdx.x; j < dpad; j += blockDim.x) {
    s_cf[j] = a.ncs[j];
    s_is[j] = a.isf[j];
  }
  // TMEM: two accumulator slots of 256 columns, each D1 (hi*hi) at +0 and
  // D2 (hi*lo + lo*hi) at +128.  Kp <= 128: tiles alternate between the
  // slots.  Kp > 128: a tile's decision columns split into halves [0, 128)
  // (slot 0) and [128, Kp) (slot 1).  Either way the MMAs of the next slot
  // run while the epilogue drains the other one.
  const uint32_t ncols = 512u;
  if (warp == kSMma) tmem_alloc(smem_u32(&sm->tmem_base), ncols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sm->tmem_base;
  // One accumulator per tile (E4M3 always; the 16-bit types when the ring
  // holds a whole tile and a stage more, nkb < nst): the corrections of
  // every K block first, then hi*hi, in one 256-column slot.  Otherwise the
  // 16-bit types keep hi*hi and the corrections in two accumulators, a
  // tile's columns split over the slots at Kp > 128.
  const bool single = F8 || a.nkb < nst;
  const int nh = (!single && a.Kp > 128) ? 2 : 1;   // column halves per tile
  const int my_tiles = (int)((a.tiles - blockIdx.x + gridDim.x - 1) / gridDim.x);
  const int iters = my_tiles * a.nkb;
  float s2h[kSMaxKp / 32 / kSEpiStride], s2l[kSMaxKp / 32 / kSEpiStride];   // epilogue: S2 (float-float)
  float mh[NKB][2], ml[NKB][2];                   // converters: m~ of the lane's two columns per K block

  if (warp == kSMma) {
    // ------------------------------------------------------------ MMA ---
    if (lane == 0) {
      const uint32_t bb = smem_u32(&sm->b_full);
      mbar_expect_tx(bb, (uint32_t)bbytes);
      for (int off = 0; off < bbytes; off += 32768) {
        const int n = min(32768, bbytes - off);
        bulk_g2s(sB + (uint32_t)off, a.bimage + off, (uint32_t)n, bb);
      }
      bool ok = mbar_wait(bb, 0, abort_flag, a.err);
      const bool b_landed = ok;
      const uint32_t idesc0 = F8 ? idesc_e4m3(kSM, a.Kp) : idesc_f16(kSM, nh == 2 ? 128 : a.Kp, F16);
      const uint32_t idesc1 = F8 ? idesc0 : idesc_f16(kSM, nh == 2 ? a.Kp - 128 : a.Kp, F16);
      const uint32_t hl_b = (uint32_t)(a.Kp * 128);
      int tt = 0, kb = 0, st = 0;
      uint32_t ph = 0;
      for (int it = 0; ok && it < iters; ++it) {
        // slot of the first (or only) half; its n-th use waits for the
        // epilogue's (n-1)-th release
        const int s0 = nh == 2 ? 0 : (tt & 1);
        const int n0 = nh == 2 ? tt : (tt >> 1);
        if (kb == 0 && n0 > 0) {
          ok = mbar_wait(smem_u32(&sm->q_empty[s0]), (uint32_t)((n0 - 1) & 1), abort_flag, a.err);
          if (!ok) break;
        }
        ok = mbar_wait(smem_u32(&sm->a_full[st]), ph, abort_flag, a.err);
        if (!ok) break;
        tc_fence_after();
        const uint32_t a_hi = sA + (uint32_t)(st * kSStageBytes);
        const uint32_t a_lo = a_hi + kSM * 128;
        const uint32_t b_hi = sB + (uint32_t)(kb * 2) * hl_b;
        const uint32_t b_lo = b_hi + hl_b;
        for (int h = 0; h < nh; ++h) {
          const int sl = nh == 2 ? h : s0;
          if (h == 1 && kb == 0 && tt > 0) {
            ok = mbar_wait(smem_u32(&sm->q_empty[1]), (uint32_t)((tt - 1) & 1), abort_flag, a.err);
            if (!ok) break;
            tc_fence_after();
          }
          const uint32_t d1 = tmem + 256u * (uint32_t)sl, d2 = d1 + 128u;
          const uint32_t bo = (uint32_t)h * (128u * 128u);   // decision rows 128 h ..
          const uint32_t idesc = h == 0 ? idesc0 : idesc1;
          if constexpr (F8) {
            // A rows [A1 | A2] (64 dimensions per half, 32 per step) against
            // the image's halves B3, B2 and B1 of this block: the small
            // products A1 B3, A1 B2, A2 B1 first, then A1 B1
            const uint32_t acc0 = kb == 0 ? 0u : 1u;
            const uint32_t plane = (uint32_t)(a.Kp * 128);
            const int h1 = kb, h2 = a.nkb + kb, h3 = 2 * a.nkb + kb;
            const uint32_t b1 = sB + (uint32_t)(h1 >> 1) * plane + (uint32_t)(h1 & 1) * 64u;
            const uint32_t b2 = sB + (uint32_t)(h2 >> 1) * plane + (uint32_t)(h2 & 1) * 64u;
            const uint32_t b3 = sB + (uint32_t)(h3 >> 1) * plane + (uint32_t)(h3 & 1) * 64u;
            mma_e4m3(d1, desc_sw128(a_hi), desc_sw128(b3), idesc, acc0);
            mma_e4m3(d1, desc_sw128(a_hi + 32u), desc_sw128(b3 + 32u), idesc, 1u);
            mma_e4m3(d1, desc_sw128(a_hi), desc_sw128(b2), idesc, 1u);
            mma_e4m3(d1, desc_sw128(a_hi + 32u), desc_sw128(b2 + 32u), idesc, 1u);
            mma_e4m3(d1, desc_sw128(a_hi + 64u), desc_sw128(b1), idesc, 1u);
            mma_e4m3(d1, desc_sw128(a_hi + 96u), desc_sw128(b1 + 32u), idesc, 1u);
            mma_e4m3(d1, desc_sw128(a_hi), desc_sw128(b1), idesc, 1u);
            mma_e4m3(d1, desc_sw128(a_hi + 32u), desc_sw128(b1 + 32u), idesc, 1u);
          } else if (single) {
            // this K block's corrections now; the hi*hi of every K block of
            // the tile once its last block is in (the tile's stages are
            // consecutive in the ring and all still held)
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              const uint32_t o = (uint32_t)(kk * 32);
              mma_bf16(d1, desc_sw128(a_hi + o), desc_sw128(b_lo + o), idesc, (kb == 0 && kk == 0) ? 0u : 1u);
              mma_bf16(d1, desc_sw128(a_lo + o), desc_sw128(b_hi + o), idesc, 1u);
            }
            if (kb == a.nkb - 1) {
              for (int k2 = 0; k2 < a.nkb; ++k2) {
                const int s2 = (st - (a.nkb - 1 - k2) + nst) % nst;
                const uint32_t ah = sA + (uint32_t)(s2 * kSStageBytes);
                const uint32_t bh = sB + (uint32_t)(k2 * 2) * hl_b;
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                  const uint32_t o = (uint32_t)(kk * 32);
                  mma_bf16(d1, desc_sw128(ah + o), desc_sw128(bh + o), idesc, 1u);
                }
              }
            }
          } else {
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              const uint32_t o = (uint32_t)(kk * 32);
              const uint32_t acc0 = (kb == 0 && kk == 0) ? 0u : 1u;
              mma_bf16(d1, desc_sw128(a_hi + o), desc_sw128(b_hi + bo + o), idesc, acc0);
              mma_bf16(d2, desc_sw128(a_hi + o), desc_sw128(b_lo + bo + o), idesc, acc0);
              mma_bf16(d2, desc_sw128(a_lo + o), desc_sw128(b_hi + bo + o), idesc, 1u);
            }
          }
          if (kb == a.nkb - 1) mma_commit(smem_u32(&sm->q_full[sl]));
        }
        if (!ok) break;
        if (F8 || !single) {
          mma_commit(smem_u32(&sm->a_empty[st]));
        } else if (kb == a.nkb - 1) {   // the tile's stages, once its hi*hi are issued
          for (int k2 = 0; k2 < a.nkb; ++k2) mma_commit(smem_u32(&sm->a_empty[(st - (a.nkb - 1 - k2) + nst) % nst]));
        }
        if (++kb == a.nkb) { kb = 0; ++tt; }
        if (++st == nst) { st = 0; ph ^= 1u; }
      }
      mma_commit(smem_u32(&sm->drain));
      uint32_t never = 0u;
      mbar_wait(smem_u32(&sm->drain), 0, &never, a.err);
      if (!b_landed) mbar_wait(bb, 0, &never, a.err);
    }
    __syncwarp();
  } else if (warp == kSProd) {
    // ------------------------------------------------------- producer ---
    if (lane == 0) {
      int tt = 0, kb = 0, st = 0;
      uint32_t ph = 0, issued = 0, lpar = 0;   // stages with loads, parity of the next load per stage
      for (int it = 0; it < iters; ++it) {
        if (!mbar_wait(smem_u32(&sm->a_empty[st]), ph ^ 1u, abort_flag, a.err)) break;
        const uint32_t tile = blockIdx.x + (uint32_t)tt * gridDim.x;
        const uint32_t fb = smem_u32(&sm->ld_full[st]);
        mbar_expect_tx(fb, (uint32_t)kSStageBytes);
        const uint32_t dst = sA + (uint32_t)(st * kSStageBytes);
        tma_load_2d(dst, &tmap, kb * kSKB, (int)(tile * kSM), fb);
        tma_load_2d(dst + (uint32_t)(kSM * 128), &tmap, kb * kSKB + 32, (int)(tile * kSM), fb);
        issued |= 1u << st;
        lpar ^= 1u << st;
        if (++kb == a.nkb) { kb = 0; ++tt; }
        if (++st == nst) { st = 0; ph ^= 1u; }
      }
      // the last load into each stage has landed before the CTA moves on
      uint32_t never = 0u;
      for (int s = 0; s < nst; ++s)
        if ((issued >> s) & 1u) mbar_wait(smem_u32(&sm->ld_full[s]), ((lpar >> s) & 1u) ^ 1u, &never, a.err);
    }
    __syncwarp();
  } else if (warp < kSEpi) {
    // ------------------------------------------------------- epilogue ---
    // warp w reads TMEM lanes 32 (w % 4) .. + 31 and the column groups
    // g = w / 4, w / 4 + kSEpiStride, ...
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    const int g0 = warp >> 2;
#pragma unroll
    for (int g = 0; g < kSMaxKp / 32 / kSEpiStride; ++g) s2h[g] = s2l[g] = 0.0f;
    bool ok = true;
    for (int tt = 0; ok && tt < my_tiles; ++tt) {
      for (int h = 0; h < nh; ++h) {
        const int sl = nh == 2 ? h : (tt & 1);
        const int n = nh == 2 ? tt : (tt >> 1);
        if (!warp_wait(smem_u32(&sm->q_full[sl]), (uint32_t)(n & 1), abort_flag, a.err)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d1 = tmem + lane_base + 256u * (uint32_t)sl, d2 = d1 + 128u;
        // groups of this half: [0, 8) with one half, [4 h, 4 h + 4) with two.
        // The group loop stays rolled (register pressure); the running sums
        // rotate so that the current group's pair is s2h[0] / s2l[0], and
        // every warp visits 8 / kSEpiStride groups per tile.
        const int gb = nh == 2 ? 4 * h : 0, ge = nh == 2 ? 4 * h + 4 : 8;
#pragma unroll 1
        for (int g = gb + g0; g < ge; g += kSEpiStride) {
          if (32 * g < a.Kp) {
            const uint32_t c = (uint32_t)(32 * g - 128 * h);
            if (single)
              ff_add(s2h[0], s2l[0], epi_sq_colsum32_1(d1 + c, lane));
            else
              ff_add(s2h[0], s2l[0], epi_sq_colsum32_x2(d1 + c, d2 + c, lane));
          }
          rot_left(s2h);
          rot_left(s2l);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&sm->q_empty[sl]));
      }
    }
  } else {
    // ----------------------------------------------------- converters ---
    const int cw = warp - (kSProd + 1);            // 0 .. 15: rows 8 cw .. 8 cw + 7
    const int r = 8 * cw + (lane >> 2);            // row of the tile
    const int q = lane & 3;                        // columns 16 q .. 16 q + 15 of the K block
    const int box = q >> 1, u0 = (q & 1) * 4;      // FP32 box and its first 16-byte unit
    // Box-1 threads (q = 2, 3) visit their 16-byte units in the order
    // uu ^ 2, so that no two threads of a quarter-warp hit the same banks in
    // the two boxes; their v[] then holds the two 8-column halves swapped.
    const int hsw = q >> 1;
#pragma unroll
    for (int b = 0; b < NKB; ++b) mh[b][0] = mh[b][1] = ml[b][0] = ml[b][1] = 0.0f;
    bool in_range = true;
    int tt = 0, kb = 0, st = 0;
    uint32_t ph = 0;
    for (int it = 0; it < iters; ++it) {
      if (!warp_wait(smem_u32(&sm->ld_full[st]), ph, abort_flag, a.err)) break;
      const uint32_t tile = blockIdx.x + (uint32_t)tt * gridDim.x;
      const bool row_ok = (uint32_t)r < a.N - tile * (uint32_t)kSM;
      uint8_t* stage = As + st * kSStageBytes;
      const uint8_t* rowp = stage + box * (kSM * 128) + r * 128;
      const int j0 = kb * kSKB + 16 * q;
      float v[16];
#pragma unroll
      for (int uu = 0; uu < 4; ++uu) {
        const int uc = uu ^ (2 * hsw);
        const float4 t = *reinterpret_cast<const float4*>(rowp + (((u0 + uc) ^ (r & 7)) << 4));
        const float4 c = *reinterpret_cast<const float4*>(s_cf + j0 + 4 * uc);
        const float4 w = *reinterpret_cast<const float4*>(s_is + j0 + 4 * uc);
        // (R - c) 2^-a as one fma: both products are exact (power-of-two
        // scale), so the single rounding equals that of R - c, scaled
        v[4 * uu + 0] = fmaf(t.x, w.x, c.x);
        v[4 * uu + 1] = fmaf(t.y, w.y, c.y);
        v[4 * uu + 2] = fmaf(t.z, w.z, c.z);
        v[4 * uu + 3] = fmaf(t.w, w.w, c.w);
      }
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        v[e] = row_ok ? v[e] : 0.0f;
        if constexpr (F16) in_range = in_range && fabsf(v[e]) < 32768.0f;
        if constexpr (F8) in_range = in_range && fabsf(v[e]) <= 448.0f;
      }
      if constexpr (F8) {
        // E4M3 hi + lo of each value; the row's 128 bytes become [A1 | A2]:
        // this thread's 16 dimensions 16 q .. 16 q + 15 are unit q of A1 and
        // unit 4 + q of A2 (v[] holds their two 8-column halves swapped when
        // hsw is set)
        uint32_t h8[4], l8[4];   // byte quads: dims (of v) 4 w .. 4 w + 3
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          uint32_t hq = 0u, lq = 0u;
#pragma unroll
          for (int t = 0; t < 4; t += 2) {
            const int e = 4 * w + t;
            const uint32_t hp = e4m3x2(v[e], v[e + 1]);
            const float2 hf = e4m3x2_to_f2(hp);
            const uint32_t lp = e4m3x2(v[e] - hf.x, v[e + 1] - hf.y);
            hq |= hp << (8 * t);
            lq |= lp << (8 * t);
          }
          h8[w] = hq;
          l8[w] = lq;
        }
        __syncwarp();   // every thread of these rows has read its FP32 values
        const uint4 hu = hsw ? make_uint4(h8[2], h8[3], h8[0], h8[1]) : make_uint4(h8[0], h8[1], h8[2], h8[3]);
        const uint4 lu = hsw ? make_uint4(l8[2], l8[3], l8[0], l8[1]) : make_uint4(l8[0], l8[1], l8[2], l8[3]);
        if (bc_ok(sw_off(r, 4 + q) + 15u, (size_t)kSM * 128, a.err) && bc_ok(sw_off(r, q) + 15u, (size_t)kSM * 128, a.err)) {
          *reinterpret_cast<uint4*>(stage + sw_off(r, q)) = hu;
          *reinterpret_cast<uint4*>(stage + sw_off(r, 4 + q)) = lu;
        }
      } else {
      uint32_t hi[8], lo[8];
#pragma unroll
      for (int e = 0; e < 16; e += 2) {
        hi[e / 2] = pack2<F16>(v[e], v[e + 1]);
        const float2 h = unpack2<F16>(hi[e / 2]);
        lo[e / 2] = pack2<F16>(v[e] - h.x, v[e + 1] - h.y);
      }
      __syncwarp();   // every thread of these rows has read its FP32 values
      uint8_t* hrow = stage;                    // hi over the first half
      uint8_t* lrow = stage + kSM * 128;        // lo over the second half
      const int ua = 2 * q + hsw, ub = 2 * q + 1 - hsw;   // units of v[0..7] and v[8..15]
      if (bc_ok(sw_off(r, ua) + 15u, (size_t)kSM * 128, a.err) && bc_ok(sw_off(r, ub) + 15u, (size_t)kSM * 128, a.err)) {
        *reinterpret_cast<uint4*>(hrow + sw_off(r, ua)) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<uint4*>(hrow + sw_off(r, ub)) = make_uint4(hi[4], hi[5], hi[6], hi[7]);
        *reinterpret_cast<uint4*>(lrow + sw_off(r, ua)) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        *reinterpret_cast<uint4*>(lrow + sw_off(r, ub)) = make_uint4(lo[4], lo[5], lo[6], lo[7]);
      }
      }
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&sm->a_full[st]));
      // m~: reduce-scatter of the warp's 8 rows (lanes 4 apart share the
      // columns); lane (row rr, quarter q) ends with v[2 rr], v[2 rr + 1]
#pragma unroll
      for (int w = 16; w >= 4; w >>= 1) {
        const bool upper = (lane & w) != 0;
        const int hw = w >> 1;   // values kept: 8, 4, 2
#pragma unroll
        for (int e = 0; e < hw; ++e) {
          const float send = upper ? v[e] : v[e + hw];
          const float keep = upper ? v[e + hw] : v[e];
          v[e] = keep + __shfl_xor_sync(0xffffffffu, send, w);
        }
      }
#pragma unroll
      for (int b = 0; b < NKB; ++b)
        if (b == kb) {
          ff_add(mh[b][0], ml[b][0], v[0]);
          ff_add(mh[b][1], ml[b][1], v[1]);
        }
      if (++kb == a.nkb) { kb = 0; ++tt; }
      if (++st == nst) { st = 0; ph ^= 1u; }
    }
    if (!in_range) atomicOr(a.err, kErrInput);
  }

  // ----------------------------------------------------- CTA reductions ---
  __syncthreads();   // MMAs drained, loads landed: the A stages are free
  double* red_s2 = reinterpret_cast<double*>(As);   // [4 lane quadrants][Kp]
  double* red_m = red_s2 + 4 * a.Kp;                // [kSConv][dpad]
  if (warp < kSEpi) {
#pragma unroll
    for (int i = 0; i < kSMaxKp / 32 / kSEpiStride; ++i) {
      const int g = (warp >> 2) + i * kSEpiStride;
      if (32 * g < a.Kp) red_s2[(warp & 3) * a.Kp + 32 * g + epi_col(lane)] = (double)s2h[i] + (double)s2l[i];
    }
  } else if (warp > kSProd) {
    const int cw = warp - (kSProd + 1);
    const int col = 16 * (lane & 3) + (((lane >> 1) & 14) ^ (8 * ((lane & 3) >> 1)));
#pragma unroll
    for (int b = 0; b < NKB; ++b)
      if (b < a.nkb) {
        red_m[cw * dpad + b * kSKB + col] = (double)mh[b][0] + (double)ml[b][0];
        red_m[cw * dpad + b * kSKB + col + 1] = (double)mh[b][1] + (double)ml[b][1];
      }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < dpad; j += blockDim.x) {
    double t = 0.0;
#pragma unroll 4
    for (int w = 0; w < kSConv; ++w) t += red_m[w * dpad + j];
    if (bc_ok((size_t)blockIdx.x * dpad + j, SAA_BOUND(a.n_m), a.err)) a.part_m[(size_t)blockIdx.x * dpad + j] = t;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < a.K; k += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < 4; ++w) s += red_s2[w * a.Kp + k];
    if (bc_ok((size_t)blockIdx.x * a.K + k, SAA_BOUND(a.n_s2), a.err)) a.part_s2[(size_t)blockIdx.x * a.K + k] = s * a.scale2[k];
  }
  if (warp == kSMma) {
    tc_fence_after();
    tmem_dealloc(tmem, ncols);
  }
}

}  // namespace tc

namespace {

// Power-of-two exponent a with 2^(a-1) < sigma <= 2^a; -1000 for a spread
// that is not a positive finite number in [2^-100, 2^100].
__device__ __forceinline__ int spread_exp(double sigma) {
  if (!(sigma > 0.0) || !isfinite(sigma)) return -1000;
  int e;
  const double m = frexp(sigma, &e);   // sigma = m 2^e, m in [0.5, 1)
  if (m == 0.5) --e;                   // an exact power of two keeps its own exponent
  return (e < -100 || e > 100) ? -1000 : e;
}

// Operands of the streamed kernel: cf = center in FP32, isf = 2^-a_j,
// ncs = -cf isf (all 0 past d), Xs = x_kj 2^a_j.
__global__ void k_stream_prep(int K, int d, int dpad, const double* __restrict__ center,
                              const double* __restrict__ sigma, const double* __restrict__ X, float* __restrict__ cf,
                              float* __restrict__ isf, float* __restrict__ ncs, double* __restrict__ Xs,
                              uint32_t* err) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < dpad) {
    const int j = (int)t;
    int e = 0;
    if (j < d && sigma) {
      e = spread_exp(sigma[j]);
      if (e == -1000) {
        atomicOr(err, kErrInput);
        e = 0;
      }
    }
    cf[j] = (j < d && center) ? (float)center[j] : 0.0f;
    isf[j] = (j < d) ? ldexpf(1.0f, -e) : 0.0f;
    ncs[j] = -cf[j] * isf[j];
  } else if (t < dpad + (int64_t)K * d) {
    const int64_t u = t - dpad;
    const int j = (int)(u % d);
    int e = sigma ? spread_exp(sigma[j]) : 0;
    if (e == -1000) e = 0;
    Xs[u] = ldexp(X[u], e);
  }
}

// Decision operand image for the E4M3 products, one block per padded
// decision row n: e_n with max_j |x'_nj| 2^-e_n in [1, 2) (0 for a zero row),
// y = x'_n 2^(7 - e_n) (largest entry in [128, 256), inside E4M3's 448),
// split in FP64 into three E4M3 terms, y = B1 + B2 + B3 + r with |r| about
// 2^-12 |y| (each residual is exact in FP64), scale2[n] = 4^(e_n - 7).  The
// 64-dimension halves of the nkb K blocks, B1 of every block, then B2, then
// B3, are packed two to a 128-byte row (half h: plane h / 2 of Kp rows, bytes
// (h % 2) 64 .. + 63) in the 128-byte-swizzled K-major order.  Rows n >= K
// and dimensions j >= d are zero.
__global__ void __launch_bounds__(64) k_stream_image8(int d, int K, int Kp, int nkb, const double* __restrict__ Y64,
                                                      double* __restrict__ scale2, uint8_t* __restrict__ img) {
  __shared__ double wmax[2];
  const int n = blockIdx.x;
  const int lane = threadIdx.x & 31;
  double m = 0.0;
  if (n < K)
    for (int j = threadIdx.x; j < d; j += blockDim.x) m = fmax(m, fabs(Y64[(size_t)n * d + j]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) wmax[threadIdx.x >> 5] = m;
  __syncthreads();
  m = fmax(wmax[0], wmax[1]);
  const int e = (m > 0.0) ? ilogb(m) : 0;
  const double sc = ldexp(1.0, 7 - e);   // exact
  if (threadIdx.x == 0 && n < K) scale2[n] = ldexp(1.0, 2 * (e - 7));
  for (int grp = threadIdx.x; grp < nkb * 4; grp += blockDim.x) {
    const int kb = grp >> 2, g = grp & 3;   // dimensions 64 kb + 16 g .. + 15
    uint32_t w1[4], w2[4], w3[4];
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      uint32_t b1 = 0u, b2 = 0u, b3 = 0u;
#pragma unroll
      for (int t = 0; t < 4; t += 2) {
        double y[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int j = kb * tc::kSKB + 16 * g + 4 * w + t + u;
          y[u] = (n < K && j < d) ? Y64[(size_t)n * d + j] * sc : 0.0;
        }
        const uint32_t p1 = tc::e4m3x2((float)y[0], (float)y[1]);
        const float2 f1 = tc::e4m3x2_to_f2(p1);
        const double r0 = y[0] - (double)f1.x, r1 = y[1] - (double)f1.y;
        const uint32_t p2 = tc::e4m3x2((float)r0, (float)r1);
        const float2 f2 = tc::e4m3x2_to_f2(p2);
        const uint32_t p3 = tc::e4m3x2((float)(r0 - (double)f2.x), (float)(r1 - (double)f2.y));
        b1 |= p1 << (8 * t);
        b2 |= p2 << (8 * t);
        b3 |= p3 << (8 * t);
      }
      w1[w] = b1;
      w2[w] = b2;
      w3[w] = b3;
    }
    auto unit = [&](int h) {   // this row's 16-byte unit g of half h
      return (size_t)(h >> 1) * Kp * 128 + (size_t)n * 128 + (size_t)((((h & 1) * 4 + g) ^ (n & 7)) << 4);
    };
    *reinterpret_cast<uint4*>(img + unit(kb)) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
    *reinterpret_cast<uint4*>(img + unit(nkb + kb)) = make_uint4(w2[0], w2[1], w2[2], w2[3]);
    *reinterpret_cast<uint4*>(img + unit(2 * nkb + kb)) = make_uint4(w3[0], w3[1], w3[2], w3[3]);
  }
}

// m~_j = sum over CTAs of their slot-0 totals: one block per 32 columns,
// warp w adds CTAs w, w + 8, ... and the eight warp sums are merged in warp
// order (deterministic).  Plain FP64 adds: the partials are FP64 sums of
// FP32 values, so the rounding of a few hundred adds is far below FP32's.
__global__ void __launch_bounds__(256) k_stream_mfinal(int grid, int dpad, const double* __restrict__ part_m,
                                                       double* __restrict__ tot_m) {
  __shared__ double sh[8][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = blockIdx.x * 32 + lane;
  double s = 0.0;
  for (int g = warp; g < grid; g += 8) s += part_m[(size_t)g * dpad + j];
  sh[warp][lane] = s;
  __syncthreads();
  if (warp == 0) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < 8; ++w) t += sh[w][lane];
    tot_m[j] = t;
  }
}

// One warp per decision: S2_k over the CTAs' partials, c_k = fl32(center)'x_k
// (the center the kernel subtracted), S1_k = m~'x'_k, then the outputs of
// Eq. 4.  Lane-strided FP64 sums merged by a fixed shuffle tree.
__global__ void __launch_bounds__(256) k_stream_out(int grid, int K, int d, double N, double lambda,
                                                    const double* __restrict__ part_s2,
                                                    const double* __restrict__ tot_m, const float* __restrict__ cf,
                                                    const double* __restrict__ X, const double* __restrict__ Xs,
                                                    double* __restrict__ f, double* __restrict__ pbar,
                                                    double* __restrict__ var) {
  const int k = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (k >= K) return;
  double s2 = 0.0, c = 0.0, s1 = 0.0;
  for (int g = lane; g < grid; g += 32) s2 += part_s2[(size_t)g * K + k];
  for (int j = lane; j < d; j += 32) {
    c = fma((double)cf[j], X[(size_t)k * d + j], c);
    s1 = fma(tot_m[j], Xs[(size_t)k * d + j], s1);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
  }
  if (lane == 0) {
    const double qbar = s1 / N;
    const double pb = c + qbar;
    const double V = (s2 - s1 * qbar) / (N - 1.0);
    if (f) f[k] = lambda * V - pb;
    if (pbar) pbar[k] = pb;
    if (var) var[k] = V;
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

std::mutex g_enc_mu;
EncodeTiledFn g_encode = nullptr;

saa_status encode_fn(EncodeTiledFn* out) {
  std::lock_guard<std::mutex> lock(g_enc_mu);
  if (!g_encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
      set_error("saa_eval_samples: cuTensorMapEncodeTiled is not available");
      return SAA_ECUDA;
    }
    g_encode = (EncodeTiledFn)fn;
  }
  *out = g_encode;
  return SAA_OK;
}

struct SPlan {
  int Kp, nkb, nst, grid, smem, dpad;
  int64_t tiles;
  size_t img, s2, pm, cf, xs, tots, total;
};

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

SPlan stream_plan(const saa_ctx* ctx, int64_t N, int d, int K, saa_prec prec) {
  const bool f8 = prec == SAA_FP8X;
  SPlan p;
  p.Kp = (K + 31) / 32 * 32;
  p.nkb = (d + tc::kSKB - 1) / tc::kSKB;
  p.dpad = p.nkb * tc::kSKB;
  p.tiles = (N + tc::kSM - 1) / tc::kSM;
  p.grid = (int)(p.tiles < ctx->sm_count ? p.tiles : ctx->sm_count);
  // as many 32 KB stages as the shared memory left by the decision image holds
  p.nst = tc::kSMaxStages;
  while (p.nst > 2 && (int)tc::stream_smem_bytes(p.Kp, p.nkb, p.nst, f8) > ctx->smem_optin) --p.nst;
  p.smem = (int)tc::stream_smem_bytes(p.Kp, p.nkb, p.nst, f8);
  size_t off = 0;
  p.img = off; off = a256(off + (size_t)p.nkb * 2 * p.Kp * 128 + 8 * (size_t)K);
  p.s2 = off; off = a256(off + 8 * (size_t)p.grid * K);
  p.pm = off; off = a256(off + 8 * (size_t)p.grid * p.dpad);
  p.cf = off; off = a256(off + 4 * 3 * (size_t)p.dpad);
  p.xs = off; off = a256(off + 8 * (size_t)K * d);
  p.tots = off; off = a256(off + 8 * (size_t)p.dpad);
  p.total = off;
  return p;
}

saa_status stream_check(const saa_ctx* ctx, int64_t N, int d, int K, saa_prec prec) {
  if (!ctx) {
    set_error("saa_eval_samples: ctx is NULL");
    return SAA_EINVAL;
  }
  if (N < 2 || N >= (int64_t)1 << 31 || d < 4 || (d & 3) || K < 1) {
    set_error("saa_eval_samples: need 2 <= N < 2^31, d >= 4 a multiple of 4 (16-byte rows for TMA), K >= 1");
    return SAA_EINVAL;
  }
  if (!is_tc(prec) && prec != SAA_FP8X) {
    set_error("saa_eval_samples: streamed samples run at SAA_F16X3, SAA_BF16X3 or SAA_FP8X");
    return SAA_EUNSUPPORTED;
  }
  const SPlan p = stream_plan(ctx, N, d, K, prec);
  if (d > 256 || p.Kp > tc::kSMaxKp || tc::img_bytes(p.Kp, p.nkb, prec == SAA_FP8X) > 128 * 1024 ||
      p.smem > ctx->smem_optin) {
    set_error("saa_eval_samples: needs d <= 256, K <= 256 and a decision image of at most 128 KB");
    return SAA_EUNSUPPORTED;
  }
  return SAA_OK;
}

}  // namespace
}  // namespace saa

using namespace saa;

extern "C" size_t saa_eval_samples_workspace_size(const saa_ctx* ctx, int64_t N, int32_t d, int32_t K,
                                                  saa_prec prec) {
  if (stream_check(ctx, N, d, K, prec) != SAA_OK) return 0;
  return stream_plan(ctx, N, d, K, prec).total;
}

extern "C" saa_status saa_eval_samples(saa_ctx* ctx, int64_t N, int32_t d, const float* R, const double* center,
                                       const double* sigma, int32_t K, const double* X, double lambda,
                                       saa_prec prec, double* f, double* pbar, double* var, void* ws,
                                       size_t ws_bytes, void* stream) {
  saa::NvtxRange nvtx_range("saa_eval_samples");
  saa_status s = stream_check(ctx, N, d, K, prec);
  if (s != SAA_OK) return s;
  if (!R || (((uintptr_t)R) & 15u) || !X || !ws || (((uintptr_t)ws) & 255u)) {
    set_error("saa_eval_samples: R (16-byte aligned), X and a 256-byte aligned ws are required");
    return SAA_EINVAL;
  }
  if (prec == SAA_FP8X && (!center || !sigma)) {
    set_error("saa_eval_samples: SAA_FP8X needs center and sigma (E4M3 keeps 1e-4 only on centred, scaled samples)");
    return SAA_EINVAL;
  }
  const SPlan p = stream_plan(ctx, N, d, K, prec);
  if (ws_bytes < p.total) {
    set_error("saa_eval_samples: workspace smaller than saa_eval_samples_workspace_size()");
    return SAA_ENOMEM;
  }
  EncodeTiledFn encode = nullptr;
  s = encode_fn(&encode);
  if (s != SAA_OK) return s;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != ctx->device && cudaSetDevice(ctx->device) != cudaSuccess) {
    set_error("saa_eval_samples: cudaSetDevice failed");
    return SAA_ECUDA;
  }
  // 2-D map of R: inner dimension d (FP32, rows of 4 d bytes), outer N;
  // boxes of 32 columns x 128 rows with the 128-byte swizzle; zero fill
  CUtensorMap tmap;
  std::memset(&tmap, 0, sizeof(tmap));
  const cuuint64_t gdim[2] = {(cuuint64_t)d, (cuuint64_t)N};
  const cuuint64_t gstride[1] = {(cuuint64_t)d * 4};
  const cuuint32_t box[2] = {32, (cuuint32_t)tc::kSM};
  const cuuint32_t estr[2] = {1, 1};
  CUresult cr = encode(&tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)R, gdim, gstride, box, estr,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) {
    if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
    set_error("saa_eval_samples: cuTensorMapEncodeTiled failed (" + std::to_string((int)cr) + ")");
    return SAA_ECUDA;
  }
  char* w = (char*)ws;
  uint8_t* img = (uint8_t*)(w + p.img);
  double* scale2 = (double*)(img + (size_t)p.nkb * 2 * p.Kp * 128);
  double* part_s2 = (double*)(w + p.s2);
  double* part_m = (double*)(w + p.pm);
  float* cf = (float*)(w + p.cf);
  float* isf = cf + p.dpad;
  float* ncs = isf + p.dpad;
  double* Xs = (double*)(w + p.xs);
  double* tot_m = (double*)(w + p.tots);
  cudaStream_t st = (cudaStream_t)stream;
  const bool f16 = prec == SAA_F16X3;
  const bool f8 = prec == SAA_FP8X;
  const int64_t nprep = p.dpad + (int64_t)K * d;
  k_stream_prep<<<(unsigned)((nprep + 255) / 256), 256, 0, st>>>(K, d, p.dpad, center, sigma, X, cf, isf, ncs,
                                                                Xs, ctx->err);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {
    if (f8) {
      k_stream_image8<<<p.Kp, 64, 0, st>>>(d, K, p.Kp, p.nkb, Xs, scale2, img);
      e = cudaGetLastError();
    } else {
      e = launch_tc_image(d, K, p.Kp, p.nkb, f16, Xs, scale2, nullptr, img, st);
    }
  }
  tc::SArgs a;
  a.d = d;
  a.K = K;
  a.Kp = p.Kp;
  a.nkb = p.nkb;
  a.nst = p.nst;
  a.N = (uint32_t)N;
  a.tiles = p.tiles;
  a.ncs = ncs;
  a.isf = isf;
  a.bimage = img;
  a.scale2 = scale2;
  a.part_s2 = part_s2;
  a.part_m = part_m;
#ifdef SAA_BOUNDS_CHECK
  a.n_s2 = (size_t)p.grid * K;
  a.n_m = (size_t)p.grid * p.dpad;
#endif
  a.err = ctx->err;
  auto kern = f8 ? (p.nkb == 1 ? tc::k_tc_stream<2, 1> : p.nkb == 2 ? tc::k_tc_stream<2, 2> : tc::k_tc_stream<2, 4>)
            : f16 ? (p.nkb == 1 ? tc::k_tc_stream<1, 1> : p.nkb == 2 ? tc::k_tc_stream<1, 2> : tc::k_tc_stream<1, 4>)
                  : (p.nkb == 1 ? tc::k_tc_stream<0, 1> : p.nkb == 2 ? tc::k_tc_stream<0, 2> : tc::k_tc_stream<0, 4>);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, p.smem);
  const bool prof = ctx->prof_on && ctx->prof_n < 256;
  if (e == cudaSuccess) {
    if (prof) cudaEventRecord(ctx->prof_ev[2 * ctx->prof_n], st);
    kern<<<p.grid, tc::kSThreads, p.smem, st>>>(a, tmap);
    e = cudaGetLastError();
    if (prof) cudaEventRecord(ctx->prof_ev[2 * ctx->prof_n++ + 1], st);
  }
  if (e == cudaSuccess) {
    k_stream_mfinal<<<p.dpad / 32, 256, 0, st>>>(p.grid, p.dpad, part_m, tot_m);
    k_stream_out<<<(K * 32 + 255) / 256, 256, 0, st>>>(p.grid, K, d, (double)N, lambda, part_s2, tot_m, cf, X, Xs, f,
                                                       pbar, var);
    e = cudaGetLastError();
  }
  ctx->kernels += 5;
  if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
  return cuda_status(e, "saa_eval_samples: launch");
}
