// tc.cu -- tcgen05 tensor-core path of the SAA estimate (value): split
// precision contraction Q = A Y (BF16 or FP16 hi/lo operands, FP32
// accumulation in TMEM).  The decision operand is scaled per decision by a
// power of two so that its largest entry lies in [1, 2): exact, undone in
// the epilogue, and it keeps FP16 within range.  Systematic error: the
// representation error of y (identical for every scenario) does not average
// over N, so FP16 (2 x 11 bits, ~2^-22) is the 1e-6 variant and BF16
// (2 x 8 bits, ~2^-16) the 1e-4 variant.
//
// Two kernels: k_tc_value1 for d <= 128 (described above its definition:
// one double-buffered accumulator per tile, the MMAs issued by an epilogue
// thread) and k_tc_value for 128 < d <= 256, below.
//
// Per CTA (one per SM, persistent over 128-scenario tiles):
//   RNG warps   regenerate the tile of a_i = s_i zhat_i (Sec. 3.1 samples)
//               64 dimensions at a time, split each value into bf16 hi + lo
//               and write both straight into a shared-memory stage in the
//               128-byte-swizzled K-major layout tcgen05.mma reads; they
//               also keep the per-dimension sums m~ = sum_i a_i.
//   MMA warp    one thread issues, per 16-wide k step, the three products
//               hi*hi + hi*lo + lo*hi (M = 128 scenarios, N = K decisions)
//               into a TMEM accumulator, and commits stage releases.
//   epilogue    four warps (one per TMEM lane quadrant) read Q from TMEM,
//               square it and reduce each 32-row slice per decision with a
//               warp reduce-scatter, accumulating S2 in FP64 registers.
// The three products go to two accumulators: hi*hi into D1, the small
// corrections hi*lo + lo*hi into D2, added in FP32 round-to-nearest in the
// epilogue.  The tensor core's accumulation rounds each update of a running
// sum with a bias toward zero; keeping the large running sum to one update
// per 16-wide k step (instead of three) cuts that bias threefold.
// The decision operand (y_k = C'w_k as bf16 hi/lo, pre-swizzled in global
// memory by k_tc_image) is loaded once per CTA by bulk TMA and stays
// resident.  S1_k = sum_i Q_ik is recovered exactly as m~'y_k in the
// finalize.  Every wait on an mbarrier is bounded by a clock budget: on
// expiry the kernel raises the context's error word, drains its own MMAs
// and copies, frees its TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "gen.cuh"
#include "internal.cuh"
#include "tc_ptx.cuh"

namespace saa {
namespace tc {

constexpr int kM = 128;             // scenarios per tile = MMA M = TMEM lanes
constexpr int kKB = 64;             // dimensions per K block (128 B of bf16)
constexpr int kStages = 3;          // A stages in flight
constexpr int kStageBytes = 2 * kM * 128;   // hi + lo, 32 KB
constexpr int kEpiWarps = 4;
constexpr int kMmaWarp = 4;         // warps 0..3 epilogue, 4 MMA, 5.. RNG
#ifndef SAA_TC_RNG_WARPS
#define SAA_TC_RNG_WARPS 16
#endif
constexpr int kRngWarps = SAA_TC_RNG_WARPS;
constexpr int kThreadsTc = 32 * (5 + kRngWarps);
constexpr int kRngThreads = 32 * kRngWarps;
constexpr int kMaxKp = 256;         // MMA N limit (cta_group::1, M = 128)
constexpr int kMaxDim = 256;
constexpr int kMaxBBytes = 128 * 1024;

struct Args {
  LawArgs la;
  int K, Kp, nkb;             // decisions, padded to 32 (epilogue sweeps 32 columns), K blocks of 64 dims
  int64_t tiles;
  const uint8_t* bimage;      // [nkb][hi,lo][Kp][128 B], swizzled
  const double* scale2;       // [K] 4^e_k: undoes the operand scaling of Q^2
  double* part_s2;            // [grid][K]
  double* part_m;             // [grid][d]
  uint32_t* err;
#ifdef SAA_BOUNDS_CHECK
  size_t n_s2, n_m;           // elements of part_s2 and part_m
#endif
};

// ------------------------------------------------------------- kernel ----
constexpr int kSBufs = 4;   // t-law scale buffers (producers run at most kStages stages ahead)

struct Smem {
  uint64_t a_full[kStages];
  uint64_t a_empty[kStages];
  uint64_t s_ready[kSBufs];
  uint64_t q_full[2], q_empty[2], b_full, drain;   // accumulator buffers (one when K blocks > 2)
  uint32_t tmem_base;
  uint32_t abort_flag;
  float s_buf[kSBufs][kM];
};

// Layout: [A stages][B image][Smem]; the base must be 1024-byte aligned.
size_t smem_bytes(int Kp, int nkb) {
  return (size_t)kStages * kStageBytes + (size_t)nkb * 2 * Kp * 128 + sizeof(Smem);
}

// D8: d is a multiple of 8, so every 8-dimension unit below d is whole and
// the per-element guards drop out.
template <bool F16, int NKB, bool D8>
__global__ void __launch_bounds__(kThreadsTc, 1) k_tc_value(Args a) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  // The 128-byte swizzle is address based: operands need a 1024-byte aligned base.
  const uint32_t base = smem_u32(smem_raw);
  if (base & 1023u) {
    if (threadIdx.x == 0) atomicOr(a.err, kErrBounds);
    return;
  }
  const int bbytes = a.nkb * 2 * a.Kp * 128;
  uint8_t* As = smem_raw;
  Smem* sm = reinterpret_cast<Smem*>(smem_raw + kStages * kStageBytes + bbytes);
  const uint32_t sA = base, sB = base + (uint32_t)(kStages * kStageBytes);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const LawArgs& la = a.la;
  const int d = la.d;
  volatile uint32_t* abort_flag = &sm->abort_flag;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(smem_u32(&sm->a_full[s]), kRngWarps);
      mbar_init(smem_u32(&sm->a_empty[s]), 1);
    }
    for (int s = 0; s < kSBufs; ++s) mbar_init(smem_u32(&sm->s_ready[s]), kM / 32);
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&sm->q_full[b]), 1);
      mbar_init(smem_u32(&sm->q_empty[b]), kEpiWarps);
    }
    mbar_init(smem_u32(&sm->b_full), 1);
    mbar_init(smem_u32(&sm->drain), 1);
    sm->abort_flag = 0u;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  const uint32_t ncols = (2 * a.Kp <= 32) ? 32u : (2 * a.Kp <= 64) ? 64u : (2 * a.Kp <= 128) ? 128u
                       : (2 * a.Kp <= 256) ? 256u : 512u;
  if (warp == kMmaWarp) tmem_alloc(smem_u32(&sm->tmem_base), ncols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sm->tmem_base;
  const uint32_t td1 = tmem;                    // hi*hi accumulator: columns [0, Kp)
  const uint32_t td2 = tmem + (uint32_t)a.Kp;  // hi*lo + lo*hi accumulator: columns [Kp, 2 Kp)
  const int my_tiles = (int)((a.tiles - blockIdx.x + gridDim.x - 1) / gridDim.x);
  const int iters = my_tiles * a.nkb;
  float macc[NKB][8];             // RNG warps: per-dimension sums of a_i (NKB >= a.nkb)
  float s2h[kMaxKp / 32], s2l[kMaxKp / 32];   // epilogue warps: S2 of column 32 g + lane (float-float)

  if (warp == kMmaWarp) {
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
      const uint32_t idesc = idesc_f16(kM, a.Kp, F16);
      const uint32_t hl_b = (uint32_t)(a.Kp * 128);
      int tt = 0, kb = 0, st = 0;
      uint32_t ph = 0;
      for (int it = 0; ok && it < iters; ++it) {
        if (kb == 0 && tt > 0) {
          ok = mbar_wait(smem_u32(&sm->q_empty[0]), (uint32_t)((tt - 1) & 1), abort_flag, a.err);
          if (!ok) break;
        }
        ok = mbar_wait(smem_u32(&sm->a_full[st]), ph, abort_flag, a.err);
        if (!ok) break;
        tc_fence_after();
        const uint32_t a_hi = sA + (uint32_t)(st * kStageBytes);
        const uint32_t a_lo = a_hi + kM * 128;
        const uint32_t b_hi = sB + (uint32_t)(kb * 2) * hl_b;
        const uint32_t b_lo = b_hi + hl_b;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const uint32_t o = (uint32_t)(kk * 32);
          const uint32_t acc0 = (kb == 0 && kk == 0) ? 0u : 1u;
          mma_bf16(td1, desc_sw128(a_hi + o), desc_sw128(b_hi + o), idesc, acc0);
          mma_bf16(td2, desc_sw128(a_hi + o), desc_sw128(b_lo + o), idesc, acc0);
          mma_bf16(td2, desc_sw128(a_lo + o), desc_sw128(b_hi + o), idesc, 1u);
        }
        mma_commit(smem_u32(&sm->a_empty[st]));
        if (kb == a.nkb - 1) mma_commit(smem_u32(&sm->q_full[0]));
        if (++kb == a.nkb) { kb = 0; ++tt; }
        if (++st == kStages) { st = 0; ph ^= 1u; }
      }
      // every MMA issued above completes before TMEM is released; after an
      // abort, wait (bounded) for the operand copies still in flight too
      mma_commit(smem_u32(&sm->drain));
      uint32_t never = 0u;
      mbar_wait(smem_u32(&sm->drain), 0, &never, a.err);
      if (!b_landed) mbar_wait(bb, 0, &never, a.err);
    }
    __syncwarp();
  } else if (warp < kEpiWarps) {
    // ------------------------------------------------------- epilogue ---
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
#pragma unroll
    for (int g = 0; g < kMaxKp / 32; ++g) s2h[g] = s2l[g] = 0.0f;
    for (int tt = 0; tt < my_tiles; ++tt) {
      if (!warp_wait(smem_u32(&sm->q_full[0]), (uint32_t)(tt & 1), abort_flag, a.err)) break;
      tc_fence_after();
      // the group loop stays rolled (register pressure); the running sums
      // rotate so that group g's pair is s2h[0] / s2l[0] when it is added
#pragma unroll 1
      for (int g = 0; g < kMaxKp / 32; ++g) {
        if (32 * g < a.Kp) {
          const uint32_t c0 = (uint32_t)(32 * g);
          ff_add(s2h[0], s2l[0], epi_sq_colsum32_x2(td1 + lane_base + c0, td2 + lane_base + c0, lane));
        }
        rot_left(s2h);
        rot_left(s2l);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&sm->q_empty[0]));
    }
  } else {
    // ------------------------------------------------------------ RNG ---
    const int rt = threadIdx.x - 32 * (kMmaWarp + 1);   // 0 .. kRngThreads-1
    const int cu = rt & 7;                               // 16-byte unit (8 dims) within the K block
    const gen::Stream gs = gen::make_stream(la.seed, la.epoch, la.instance);
    const uint32_t half = la.N / 2u;
    const bool tlaw = la.law == SAA_LAW_STUDENT_T;
#pragma unroll
    for (int b = 0; b < NKB; ++b)
#pragma unroll
      for (int e = 0; e < 8; ++e) macc[b][e] = 0.0f;
    int tt = 0, kb = 0, st = 0;
    uint32_t ph = 0;
    for (int it = 0; it < iters; ++it) {
      const uint32_t tile = blockIdx.x + (uint32_t)tt * gridDim.x;
      const uint32_t i0 = la.i_base + tile * (uint32_t)kM;
      const int nrow = (int)min((uint32_t)kM, la.rows_end() - i0);
      const int sb = tt & (kSBufs - 1);
      const uint32_t s_bar = smem_u32(&sm->s_ready[sb]);
      if (tlaw && kb == 0 && rt < kM) {   // RNG warps 0..3 draw the tile's scales
        sm->s_buf[sb][rt] = (rt < nrow) ? gen::t_scale_f(gs, i0 + (uint32_t)rt, la.nu) : 0.0f;
        __syncwarp();
        if (lane == 0) mbar_arrive(s_bar);
      }
      if (!warp_wait(smem_u32(&sm->a_empty[st]), ph ^ 1u, abort_flag, a.err)) break;
      if (tlaw && !warp_wait(s_bar, (uint32_t)((tt >> 2) & 1), abort_flag, a.err)) break;
      uint8_t* stage = As + st * kStageBytes;
      const int j0 = kb * kKB + cu * 8;   // first dimension of this unit
      float vs[8];                         // this stage's rows, summed (m~)
#pragma unroll
      for (int e = 0; e < 8; ++e) vs[e] = 0.0f;
#pragma unroll 1
      for (int r = rt >> 3; r < kM; r += kRngThreads / 8) {
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
            const float s = sm->s_buf[sb][r];
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
        *reinterpret_cast<uint4*>(stage + kM * 128 + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
#pragma unroll
        for (int e = 0; e < 8; ++e) vs[e] += v[e];
      }
#pragma unroll
      for (int b = 0; b < NKB; ++b)
        if (b == kb)
#pragma unroll
          for (int e = 0; e < 8; ++e) macc[b][e] += vs[e];
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&sm->a_full[st]));
      if (++kb == a.nkb) { kb = 0; ++tt; }
      if (++st == kStages) { st = 0; ph ^= 1u; }
    }
    // lanes with equal rt & 7 hold the same unit: fold them (lanes 0..7 keep the sums)
#pragma unroll
    for (int b = 0; b < NKB; ++b)
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        float v = macc[b][e];
        v += __shfl_xor_sync(0xffffffffu, v, 8);
        v += __shfl_xor_sync(0xffffffffu, v, 16);
        macc[b][e] = v;
      }
  }

  // ----------------------------------------------------- CTA reductions ---
  __syncthreads();   // MMAs drained: the A stages are free for the reductions
  const int dpad = a.nkb * kKB;
  double* red_s2 = reinterpret_cast<double*>(As);      // [kEpiWarps][Kp]
  float* red_m = reinterpret_cast<float*>(red_s2 + kEpiWarps * a.Kp);   // [kRngWarps][dpad]
  if (warp > kMmaWarp && lane < 8) {
    const int rw = warp - (kMmaWarp + 1);
#pragma unroll
    for (int b = 0; b < NKB; ++b)
      if (b < a.nkb)
#pragma unroll
        for (int e = 0; e < 8; ++e) red_m[rw * dpad + b * kKB + lane * 8 + e] = macc[b][e];
  }
  if (warp < kEpiWarps) {
#pragma unroll
    for (int g = 0; g < kMaxKp / 32; ++g)
      if (32 * g < a.Kp) red_s2[warp * a.Kp + 32 * g + epi_col(lane)] = (double)s2h[g] + (double)s2l[g];
  }
  __syncthreads();
  for (int j = threadIdx.x; j < d; j += blockDim.x) {
    double s = 0.0;
    for (int rw = 0; rw < kRngWarps; ++rw) s += (double)red_m[rw * dpad + j];
    if (bc_ok((size_t)blockIdx.x * d + j, SAA_BOUND(a.n_m), a.err)) a.part_m[(size_t)blockIdx.x * d + j] = s;
  }
  for (int k = threadIdx.x; k < a.K; k += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < kEpiWarps; ++w) s += red_s2[w * a.Kp + k];
    if (bc_ok((size_t)blockIdx.x * a.K + k, SAA_BOUND(a.n_s2), a.err)) a.part_s2[(size_t)blockIdx.x * a.K + k] = s * a.scale2[k];
  }
  if (warp == kMmaWarp) {
    tc_fence_after();
    tmem_dealloc(tmem, ncols);
  }
}

// ------------------------------------------------------------------------
// k_tc_value1: the same estimate for d <= 128 (one or two K blocks of 64
// dimensions per tile), without a dedicated MMA warp: thread 0 of the
// epilogue issues each tile's MMAs once the tile's stages are drawn, then
// the four epilogue warps reduce the previous tile.  Fewer warps leave each
// thread up to 96 registers (no spills).  The three products go to
// one accumulator per tile, the small corrections hi*lo + lo*hi of every K
// block first and hi*hi last, so the running sum is large for only 4 nkb
// updates (the same rounding bias as a separate hi*hi accumulator); two
// accumulator buffers let the epilogue of one tile run under the MMAs of
// the next.  The tile's K blocks (at most two of the three stages) stay
// resident until its MMAs complete.
// ------------------------------------------------------------------------
// 16 generator warps, 96 registers: 20, 24 and 28 warps (80, 72 and 64
// registers, no spills) each measured slower.
constexpr int kRngWarps1 = 16;
constexpr int kRngThreads1 = 32 * kRngWarps1;
constexpr int kThreads1 = 32 * (kEpiWarps + kRngWarps1);
constexpr int kRowStep1 = kRngThreads1 / 8;   // rows between a generator thread's rows in a stage
static_assert(kRowStep1 % 8 == 0 && kM % kRowStep1 == 0,
              "every thread draws the same rows, all with one swizzle phase");

template <bool F16, int NKB, bool D8>
__global__ void __launch_bounds__(kThreads1, 1) k_tc_value1(Args a) {
  static_assert(NKB <= 2, "a tile's K blocks must fit in the stage ring with one to spare");
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  const uint32_t base = smem_u32(smem_raw);
  if (base & 1023u) {
    if (threadIdx.x == 0) atomicOr(a.err, kErrBounds);
    return;
  }
  const int bbytes = a.nkb * 2 * a.Kp * 128;
  uint8_t* As = smem_raw;
  Smem* sm = reinterpret_cast<Smem*>(smem_raw + kStages * kStageBytes + bbytes);
  const uint32_t sA = base, sB = base + (uint32_t)(kStages * kStageBytes);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const LawArgs& la = a.la;
  const int d = la.d;
  volatile uint32_t* abort_flag = &sm->abort_flag;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(smem_u32(&sm->a_full[s]), kRngWarps1);
      mbar_init(smem_u32(&sm->a_empty[s]), 1);
    }
    for (int s = 0; s < kSBufs; ++s) mbar_init(smem_u32(&sm->s_ready[s]), kM / 32);
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&sm->q_full[b]), 1);
      mbar_init(smem_u32(&sm->q_empty[b]), kEpiWarps);
    }
    mbar_init(smem_u32(&sm->b_full), 1);
    mbar_init(smem_u32(&sm->drain), 1);
    sm->abort_flag = 0u;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  const uint32_t ncols = (2 * a.Kp <= 32) ? 32u : (2 * a.Kp <= 64) ? 64u : (2 * a.Kp <= 128) ? 128u
                       : (2 * a.Kp <= 256) ? 256u : 512u;
  if (warp == 0) tmem_alloc(smem_u32(&sm->tmem_base), ncols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sm->tmem_base;
  const int my_tiles = (int)((a.tiles - blockIdx.x + gridDim.x - 1) / gridDim.x);
  float macc[NKB][8];                          // generator: per-dimension sums of a_i
  float s2h[kMaxKp / 32], s2l[kMaxKp / 32];    // epilogue: S2 of column 32 g + epi_col(lane)

  if (warp < kEpiWarps) {
    // ------------------------------------------- MMA issue + epilogue ---
    const bool issuer = threadIdx.x == 0;
    const uint32_t bb = smem_u32(&sm->b_full);
    bool mma_ok = true, b_landed = false;
    if (issuer) {
      mbar_expect_tx(bb, (uint32_t)bbytes);
      for (int off = 0; off < bbytes; off += 32768) {
        const int n = min(32768, bbytes - off);
        bulk_g2s(sB + (uint32_t)off, a.bimage + off, (uint32_t)n, bb);
      }
      mma_ok = b_landed = mbar_wait(bb, 0, abort_flag, a.err);
    }
    const uint32_t idesc = idesc_f16(kM, a.Kp, F16);
    const uint32_t hl_b = (uint32_t)(a.Kp * 128);
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
#pragma unroll
    for (int g = 0; g < kMaxKp / 32; ++g) s2h[g] = s2l[g] = 0.0f;
    int st = 0;
    uint32_t ph = 0;
    for (int tt = 0; tt <= my_tiles; ++tt) {
      if (issuer && mma_ok && tt < my_tiles) {
        // ---- the MMAs of tile tt into accumulator buffer tt & 1
        const int buf = tt & 1;
        if (tt >= 2)
          mma_ok = mbar_wait(smem_u32(&sm->q_empty[buf]), (uint32_t)(((tt - 2) >> 1) & 1), abort_flag, a.err);
        int sts[NKB];
#pragma unroll
        for (int kb = 0; kb < NKB; ++kb) {
          if (kb < a.nkb && mma_ok) {
            mma_ok = mbar_wait(smem_u32(&sm->a_full[st]), ph, abort_flag, a.err);
            sts[kb] = st;
            if (++st == kStages) { st = 0; ph ^= 1u; }
          }
        }
        if (mma_ok) {
          tc_fence_after();
          const uint32_t td = tmem + (uint32_t)(buf * a.Kp);
#pragma unroll
          for (int kb = 0; kb < NKB; ++kb) {
            if (kb < a.nkb) {
              const uint64_t dah = desc_sw128(sA + (uint32_t)(sts[kb] * kStageBytes));
              const uint64_t dal = dah + (uint64_t)((kM * 128) >> 4);
              const uint64_t dbh = desc_sw128(sB + (uint32_t)(kb * 2) * hl_b);
              const uint64_t dbl = dbh + (uint64_t)(hl_b >> 4);
#pragma unroll
              for (int kk = 0; kk < 4; ++kk) {
                const uint64_t o = (uint64_t)(kk * 2);   // 32 bytes in the descriptor's 16-byte units
                mma_bf16(td, dah + o, dbl + o, idesc, (kb == 0 && kk == 0) ? 0u : 1u);
                mma_bf16(td, dal + o, dbh + o, idesc, 1u);
              }
            }
          }
#pragma unroll
          for (int kb = 0; kb < NKB; ++kb) {
            if (kb < a.nkb) {
              const uint64_t dah = desc_sw128(sA + (uint32_t)(sts[kb] * kStageBytes));
              const uint64_t dbh = desc_sw128(sB + (uint32_t)(kb * 2) * hl_b);
#pragma unroll
              for (int kk = 0; kk < 4; ++kk)
                mma_bf16(td, dah + (uint64_t)(kk * 2), dbh + (uint64_t)(kk * 2), idesc, 1u);
            }
          }
#pragma unroll
          for (int kb = 0; kb < NKB; ++kb)
            if (kb < a.nkb) mma_commit(smem_u32(&sm->a_empty[sts[kb]]));
          mma_commit(smem_u32(&sm->q_full[buf]));
        }
      }
      __syncwarp();
      if (tt == 0) continue;
      // ---- S2 of tile tt - 1
      const int te = tt - 1, buf = te & 1;
      if (!warp_wait(smem_u32(&sm->q_full[buf]), (uint32_t)((te >> 1) & 1), abort_flag, a.err)) break;
      tc_fence_after();
      const uint32_t tq = tmem + (uint32_t)(buf * a.Kp) + lane_base;
      // the group loop stays rolled (register pressure; unrolled it measured
      // slower), two groups per pass: the running sums rotate by two so that
      // groups g, g + 1 are in s2h[0..1] / s2l[0..1] when they are added
#pragma unroll 1
      for (int g = 0; g < kMaxKp / 32; g += 2) {
        if (32 * g < a.Kp) ff_add(s2h[0], s2l[0], epi_sq_colsum32_1(tq + (uint32_t)(32 * g), lane));
        if (32 * g + 32 < a.Kp) ff_add(s2h[1], s2l[1], epi_sq_colsum32_1(tq + (uint32_t)(32 * g + 32), lane));
        rot_left2(s2h);
        rot_left2(s2l);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&sm->q_empty[buf]));
    }
    if (issuer) {
      // every MMA issued above completes before TMEM is released; after an
      // abort, wait (bounded) for the operand copies still in flight too
      mma_commit(smem_u32(&sm->drain));
      uint32_t never = 0u;
      mbar_wait(smem_u32(&sm->drain), 0, &never, a.err);
      if (!b_landed) mbar_wait(bb, 0, &never, a.err);
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ RNG ---
    // One pass per tile; the tile's K blocks (one stage each) in an
    // unrolled inner loop, so each stage's m~ sums go straight to their own
    // registers.  The sums are kept as f32x2 pairs (dimensions 2e, 2e + 1).
    const int rt = threadIdx.x - 32 * kEpiWarps;       // 0 .. kRngThreads1-1
    const int cu = rt & 7;                             // 16-byte unit (8 dims) within the K block
    const int r0 = rt >> 3;
    const gen::Stream gs = gen::make_stream(la.seed, la.epoch, la.instance);
    const uint32_t half = la.N / 2u;
    const bool tlaw = la.law == SAA_LAW_STUDENT_T;
    unsigned long long mp[NKB][4];
#pragma unroll
    for (int b = 0; b < NKB; ++b)
#pragma unroll
      for (int e = 0; e < 4; ++e) mp[b][e] = 0ull;   // +0.0f, +0.0f
    int st = 0;
    uint32_t ph = 0;
    bool ok = true;
    for (int tt = 0; tt < my_tiles && ok; ++tt) {
      const uint32_t tile = blockIdx.x + (uint32_t)tt * gridDim.x;
      const uint32_t i0 = la.i_base + tile * (uint32_t)kM;
      const int nrow = (int)min((uint32_t)kM, la.rows_end() - i0);
      const int sb = tt & (kSBufs - 1);
      const uint32_t s_bar = smem_u32(&sm->s_ready[sb]);
      if (tlaw && rt < kM) {   // generator warps 0..3 draw the tile's scales
        sm->s_buf[sb][rt] = (rt < nrow) ? gen::t_scale_f(gs, i0 + (uint32_t)rt, la.nu) : 0.0f;
        __syncwarp();
        if (lane == 0) mbar_arrive(s_bar);
      }
#pragma unroll
      for (int kb = 0; kb < NKB; ++kb) {
        if (!warp_wait(smem_u32(&sm->a_empty[st]), ph ^ 1u, abort_flag, a.err)) { ok = false; break; }
        if (kb == 0 && tlaw && !warp_wait(s_bar, (uint32_t)((tt >> 2) & 1), abort_flag, a.err)) {
          ok = false;
          break;
        }
        uint8_t* stage = As + st * kStageBytes;
        const int j0 = kb * kKB + cu * 8;   // first dimension of this unit
        const bool unit_ok = j0 < d;
#pragma unroll 1
        for (int r = r0; r < kM; r += kRowStep1) {
          float v[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) v[e] = 0.0f;
          if (r < nrow && unit_ok) {
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
              const float sv = sm->s_buf[sb][r];
#pragma unroll
              for (int e = 0; e < 8; ++e) v[e] *= sv;
            }
          }
          uint32_t hi[4], lo[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const unsigned long long vp = f2_pack(__float_as_uint(v[2 * e]), __float_as_uint(v[2 * e + 1]));
            hi[e] = pack2<F16>(v[2 * e], v[2 * e + 1]);
            const float2 h = unpack2<F16>(hi[e]);
            float l0, l1;
            f2_unpack(f2_sub(vp, f2_pack(__float_as_uint(h.x), __float_as_uint(h.y))), l0, l1);
            lo[e] = pack2<F16>(l0, l1);
            mp[kb][e] = f2_add(mp[kb][e], vp);
          }
          const uint32_t off = sw_off(r, cu);
          *reinterpret_cast<uint4*>(stage + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
          *reinterpret_cast<uint4*>(stage + kM * 128 + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&sm->a_full[st]));
        if (++st == kStages) { st = 0; ph ^= 1u; }
      }
    }
#pragma unroll
    for (int b = 0; b < NKB; ++b)
#pragma unroll
      for (int e = 0; e < 4; ++e) f2_unpack(mp[b][e], macc[b][2 * e], macc[b][2 * e + 1]);
    // lanes with equal rt & 7 hold the same unit: fold them (lanes 0..7 keep the sums)
#pragma unroll
    for (int b = 0; b < NKB; ++b)
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        float v = macc[b][e];
        v += __shfl_xor_sync(0xffffffffu, v, 8);
        v += __shfl_xor_sync(0xffffffffu, v, 16);
        macc[b][e] = v;
      }
  }

  // ----------------------------------------------------- CTA reductions ---
  __syncthreads();   // MMAs drained: the A stages are free for the reductions
  const int dpad = a.nkb * kKB;
  double* red_s2 = reinterpret_cast<double*>(As);      // [kEpiWarps][Kp]
  float* red_m = reinterpret_cast<float*>(red_s2 + kEpiWarps * a.Kp);   // [kRngWarps1][dpad]
  if (warp >= kEpiWarps && lane < 8) {
    const int rw = warp - kEpiWarps;
#pragma unroll
    for (int b = 0; b < NKB; ++b)
      if (b < a.nkb)
#pragma unroll
        for (int e = 0; e < 8; ++e) red_m[rw * dpad + b * kKB + lane * 8 + e] = macc[b][e];
  }
  if (warp < kEpiWarps) {
#pragma unroll
    for (int g = 0; g < kMaxKp / 32; ++g)
      if (32 * g < a.Kp) red_s2[warp * a.Kp + 32 * g + epi_col(lane)] = (double)s2h[g] + (double)s2l[g];
  }
  __syncthreads();
  for (int j = threadIdx.x; j < d; j += blockDim.x) {
    double s = 0.0;
    for (int rw = 0; rw < kRngWarps1; ++rw) s += (double)red_m[rw * dpad + j];
    if (bc_ok((size_t)blockIdx.x * d + j, SAA_BOUND(a.n_m), a.err)) a.part_m[(size_t)blockIdx.x * d + j] = s;
  }
  for (int k = threadIdx.x; k < a.K; k += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < kEpiWarps; ++w) s += red_s2[w * a.Kp + k];
    if (bc_ok((size_t)blockIdx.x * a.K + k, SAA_BOUND(a.n_s2), a.err)) a.part_s2[(size_t)blockIdx.x * a.K + k] = s * a.scale2[k];
  }
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, ncols);
  }
}

// Decision operand image, one block per padded decision row n: the scale
// e_n with max_j |y_nj| 2^-e_n in [1, 2) (e_n = 0 for a zero row; scale2[n] =
// 4^e_n undoes it on Q^2), then y_n 2^-e_n split into hi + lo of the operand
// type, laid out as [K block][hi, lo][Kp rows][128 B] in the
// 128-byte-swizzled K-major order; rows n >= K and dimensions j >= d are
// zero.  When gaux is given (gradient path) it also receives, with f_n the
// least integer such that 2^f_n > ||y_n 2^-e_n||_2 (0 for a zero row),
// gaux[n] = 2^(e_n + f_n) and gaux[K + n] = 2^-f_n: the adjoint's operand
// Q 2^-f_n is bounded by |a_i| and G is recovered exactly.
template <bool F16>
__global__ void __launch_bounds__(64) k_tc_image(int d, int K, int Kp, int nkb, const double* __restrict__ Y64,
                                                 double* __restrict__ scale2, double* __restrict__ gaux,
                                                 uint8_t* __restrict__ img) {
  __shared__ double wmax[2], wss[2];
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
  const double inv = ldexp(1.0, -e);   // exact
  if (gaux) {
    double ss = 0.0;
    if (n < K)
      for (int j = threadIdx.x; j < d; j += blockDim.x) {
        const double y = Y64[(size_t)n * d + j] * inv;
        ss = fma(y, y, ss);
      }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    if (lane == 0) wss[threadIdx.x >> 5] = ss;
    __syncthreads();
    ss = wss[0] + wss[1];
    // ||.||_2 < 2^f  <=>  ss < 4^f
    int f = 0;
    if (ss > 0.0) {
      f = ilogb(ss) / 2 + 1;
      while (ldexp(1.0, 2 * (f - 1)) > ss) --f;
    }
    if (threadIdx.x == 0 && n < K) {
      gaux[n] = ldexp(1.0, e + f);
      gaux[K + n] = ldexp(1.0, -f);
    }
  }
  if (threadIdx.x == 0 && n < K) scale2[n] = ldexp(1.0, 2 * e);
  for (int unit = threadIdx.x; unit < nkb * 8; unit += blockDim.x) {
    const int kb = unit >> 3, u = unit & 7;
    uint32_t hi[4], lo[4];
#pragma unroll
    for (int q = 0; q < 8; q += 2) {
      double y[2];
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const int j = kb * kKB + u * 8 + q + t;
        y[t] = (n < K && j < d) ? Y64[(size_t)n * d + j] * inv : 0.0;
      }
      hi[q / 2] = pack2<F16>((float)y[0], (float)y[1]);
      const float2 h = unpack2<F16>(hi[q / 2]);
      lo[q / 2] = pack2<F16>((float)(y[0] - (double)h.x), (float)(y[1] - (double)h.y));
    }
    const size_t blk = (size_t)kb * 2 * Kp * 128;
    const uint32_t off = (uint32_t)(n * 128 + ((u ^ (n & 7)) << 4));
    *reinterpret_cast<uint4*>(img + blk + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
    *reinterpret_cast<uint4*>(img + blk + (size_t)Kp * 128 + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
  }
}

// Self-test of the failure path: one warp waits, with the tensor kernel's
// bounded wait and a short budget, on an mbarrier that nothing completes.
// It gives up, raises the timeout bit of the error word and returns.
__global__ void k_selftest_timeout(uint32_t* err, long long budget) {
  __shared__ uint64_t bar;
  __shared__ uint32_t abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);
    abort_flag = 0u;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  mbar_wait_budget(smem_u32(&bar), 0u, &abort_flag, err, budget);
}

// Self-test of the index checks: each thread stores through bc_ok at an
// index at or past the declared capacity (32) of a 64-element array.  The
// checked build raises the bounds bit and skips every store; the indices
// stay inside the real array, so no build writes outside it.
__device__ float g_bc_probe[64];
__global__ void k_selftest_bounds(uint32_t* err) {
  const size_t i = 32u + threadIdx.x;
  if (bc_ok(i, 32u, err)) g_bc_probe[i] = 1.0f;
}

}  // namespace tc

cudaError_t launch_tc_image(int d, int K, int Kp, int nkb, bool f16, const double* Y64, double* scale2,
                            double* gaux, uint8_t* img, cudaStream_t st) {
  if (f16)
    tc::k_tc_image<true><<<Kp, 64, 0, st>>>(d, K, Kp, nkb, Y64, scale2, gaux, img);
  else
    tc::k_tc_image<false><<<Kp, 64, 0, st>>>(d, K, Kp, nkb, Y64, scale2, gaux, img);
  return cudaGetLastError();
}

cudaError_t launch_selftest_timeout(uint32_t* err, uint32_t budget_us, cudaStream_t st) {
  tc::k_selftest_timeout<<<1, 32, 0, st>>>(err, (long long)budget_us * 2100ll);
  return cudaGetLastError();
}

cudaError_t launch_selftest_bounds(uint32_t* err, cudaStream_t st) {
  tc::k_selftest_bounds<<<1, 32, 0, st>>>(err);
  return cudaGetLastError();
}

bool tc_supported(const saa_problem* p, int K, int want_grad) {
  if (want_grad) return false;
  const int Kp = (K + 31) / 32 * 32;
  const int nkb = (p->d + tc::kKB - 1) / tc::kKB;
  return p->d <= tc::kMaxDim && Kp <= tc::kMaxKp && (size_t)nkb * 2 * Kp * 128 <= (size_t)tc::kMaxBBytes;
}

static size_t bimage_bytes(int K, int d) {
  const int Kp = (K + 31) / 32 * 32;
  const int nkb = (d + tc::kKB - 1) / tc::kKB;
  return (size_t)nkb * 2 * Kp * 128;
}

saa_status tc_plan(const saa_ctx* ctx, const saa_problem* p, int K, Plan* plan) {
  const int Kp = (K + 31) / 32 * 32;
  const int nkb = (p->d + tc::kKB - 1) / tc::kKB;
  plan->bm = tc::kM;
  plan->tiles = (p->N + tc::kM - 1) / tc::kM;
  plan->grid = (int)(plan->tiles < ctx->sm_count ? plan->tiles : ctx->sm_count);
  plan->smem = (int)tc::smem_bytes(Kp, nkb);
  // operand image, then scale2[K]
  plan->tc_bytes = bimage_bytes(K, p->d) + (size_t)8 * K;
  if (plan->smem > ctx->smem_optin) {
    set_error("tensor-core tile does not fit in shared memory");
    return SAA_EUNSUPPORTED;
  }
  return SAA_OK;
}

cudaError_t launch_tc(const LawArgs& la, int K, int prec, const Plan& plan, const Workspace& ws, uint32_t* err,
                      cudaStream_t st) {
  const bool f16 = (prec == SAA_F16X3);
  tc::Args a;
  a.la = la;
  a.K = K;
  a.Kp = (K + 31) / 32 * 32;
  a.nkb = (la.d + tc::kKB - 1) / tc::kKB;
  a.tiles = plan.tiles;
  uint8_t* img = (uint8_t*)ws.tc;
  double* scale2 = (double*)(img + bimage_bytes(K, la.d));
  a.bimage = img;
  a.scale2 = scale2;
  a.part_s2 = ws.part_s2;
  a.part_m = ws.part_m;
#ifdef SAA_BOUNDS_CHECK
  a.n_s2 = ws.n_s2;
  a.n_m = ws.n_m;
#endif
  a.err = err;
  cudaError_t e = launch_tc_image(la.d, K, a.Kp, a.nkb, f16, ws.Y64, scale2, nullptr, img, st);
  if (e != cudaSuccess) return e;
  const bool d8 = (la.d & 7) == 0;
  void (*kern)(tc::Args);
  int threads = tc::kThreads1;
  if (a.nkb == 1)
    kern = f16 ? (d8 ? tc::k_tc_value1<true, 1, true> : tc::k_tc_value1<true, 1, false>)
               : (d8 ? tc::k_tc_value1<false, 1, true> : tc::k_tc_value1<false, 1, false>);
  else if (a.nkb == 2)
    kern = f16 ? (d8 ? tc::k_tc_value1<true, 2, true> : tc::k_tc_value1<true, 2, false>)
               : (d8 ? tc::k_tc_value1<false, 2, true> : tc::k_tc_value1<false, 2, false>);
  else {
    kern = f16 ? (d8 ? tc::k_tc_value<true, 4, true> : tc::k_tc_value<true, 4, false>)
               : (d8 ? tc::k_tc_value<false, 4, true> : tc::k_tc_value<false, 4, false>);
    threads = tc::kThreadsTc;
  }
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, plan.smem);
  if (e != cudaSuccess) return e;
  kern<<<plan.grid, threads, plan.smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace saa
