// tc_grad.cu -- tcgen05 tensor-core path of the SAA estimate together with
// its gradient in w (Eq. 4 with Eq. 5, Sec. 3.1), for d <= 1024, K <= 64,
// drawing every normal once.
//
// With a_i = s_i zhat_i (the whitened samples), y_k = C'w_k and
// Q_ik = a_i'y_k, the gradient needs, per decision k, the d-vector
// G_k = sum_i a_i Q_ik besides S2_k = sum_i Q_ik^2 and m~ = sum_i a_i.  G
// needs the whole Q_ik (all d dimensions) before any a_i can be folded into
// it, and a tile of 128 scenarios x 1024 dimensions in hi/lo takes 512 KB,
// more than one SM's shared memory.  So the dimensions are split across a
// thread-block cluster of C = ceil(d / 128) CTAs (at most 8): CTA r of a
// cluster owns dimensions 128 r .. 128 r + 127, and every CTA of the cluster
// works on the same 128-scenario tile at the same time.  Per tile:
//   draw      the generator warps of CTA r write a_i for its 128 dimensions
//             as hi/lo halves (K-major, 128-byte swizzle) into a 64 KB stage;
//             the stage is the operand of both contractions below.
//   forward   one thread issues Q^(r) = A^(r) Y^(r) over the CTA's 128
//             dimensions, with its slice of the decision operand resident in
//             shared memory, into one FP32 accumulator: the corrections
//             A_hi Y_lo and A_lo Y_hi of both chunks first, then A_hi Y_hi.
//   exchange  the epilogue warps write the rows of Q^(r) that CTA r reduces
//             into its own inbox and stage every other owner's rows in the
//             W buffer (free once the last tile's adjoint is done), in the
//             inbox's layout; one lane per half block bulk-copies it into
//             that owner's inbox (shared::cta -> shared::cluster, completing
//             bytes of the owner's x_full).  CTA r then adds the C partials
//             of its 128 / C rows in rank order, keeps S2 of those rows, and
//             writes W = Q 2^-f_k as hi/lo into its own W buffer (2^f_k >
//             |y_k|_2 in operand units, so |W_ik| <= |a_i|_2); each warp
//             bulk-copies its rows of W into every other CTA's W.
//   adjoint   with all rows of W in place, the thread issues
//             G^(r) = A^(r)' W for the tile, reading the same stage as an
//             MN-major operand (the dimensions of a 64-dimension chunk are
//             contiguous) against [W_hi; W_lo] and A_lo' W_hi, into a block
//             accumulator that spans four tiles.  The epilogue adds each
//             block (hi*hi + corrections) into a Kahan-compensated running
//             sum held in TMEM, so G never leaves the SM until the end.
// The draw of tile t + 1 overlaps the forward, exchange and adjoint of tile
// t (two stages), and the fold of a block overlaps the exchange of the
// tile after it; the exchange moves 2 x 28 KB of distributed shared memory per tile
// and CTA at C = 8.
//
// Accuracy.  The tensor core rounds every update of an accumulator with a
// bias toward zero, so a running sum over T k steps loses about T/2 units in
// the last place.  The forward's accumulator takes the 16 correction steps
// while it is still small and then the 8 hi*hi steps per CTA, and the C
// partials are added with round-to-nearest FP32 additions; the adjoint's blocks run 32 k
// steps (four tiles) before their compensated fold, so the bias stays near
// 16 units in the last place of a block (folding every tile, 4 units, took
// 3.8 % more time; the blocks' partial sums change sign from block to block,
// and G moved by 5e-9 relative to its largest entry).  The adjoint's representation
// error changes sign and size from scenario to scenario, so it shrinks like
// sqrt(d / N) relative to G: FP16 hi/lo (2^-22 per product) keeps it below
// 1e-6 from N ~ d upwards, where BF16 hi/lo (2^-17) would not.
//
// Every mbarrier wait is clock-bounded: on expiry the kernel raises the error
// word and falls through to the end; every thread of every CTA still reaches
// the closing cluster barriers (no CTA leaves while a peer may touch its
// shared memory), MMAs and copies are drained and TMEM is freed.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <mutex>

#include "gen.cuh"
#include "internal.cuh"
#include "tc_ptx.cuh"

namespace saa {
namespace tc {

constexpr int kGM = 128;                   // scenarios per tile (forward MMA M, adjoint MMA K)
constexpr int kGDims = 128;                // dimensions per CTA (adjoint MMA M)
constexpr int kGStages = 2;
constexpr int kGChunkBytes = kGM * 128;    // [128 rows][64 dims] of one half: 16 KB
constexpr int kGStageBytes = 4 * kGChunkBytes;   // [chunk 0: hi, lo][chunk 1: hi, lo]
constexpr int kGEpiWarps = 4;              // one per TMEM lane quadrant
constexpr int kGEpiThreads = 32 * kGEpiWarps;
constexpr int kGMmaWarp = kGEpiWarps;      // warps 0..7 epilogue, 8 forward MMA, 9.. generator
constexpr int kGRngWarps = 16;
constexpr int kGThreads = 32 * (kGEpiWarps + 1 + kGRngWarps);
constexpr int kGRngThreads = 32 * kGRngWarps;
constexpr int kGKp = 64;                   // decision columns (K <= 64; unused ones are zero)
constexpr int kGMaxCluster = 8;
constexpr int kGFoldTiles = 4;             // tiles per block of G between compensated folds
constexpr int kGMaxDim = kGDims * kGMaxCluster;
static_assert(kGRngThreads == 512, "stage mapping assumes 512 generator threads");

struct GArgs {
  LawArgs la;
  int K, C;
  int64_t tiles;
  const uint8_t* bimage;   // [2C blocks of 64 dims][hi, lo][64][128 B], swizzled
  const double* gaux;      // [2K]: 2^(e_k + f_k) (G at true scale), then 2^-f_k (W)
  const double* scale2;    // [K] 4^e_k  (S2 at true scale)
  double* part_s2;         // [clusters][K]
  double* part_m;          // [clusters][d]
  float* part_g;           // [clusters][K][d]
  float* part_gc;          // [clusters][K][d] (true sum = part_g - part_gc)
  uint32_t* err;
#ifdef SAA_BOUNDS_CHECK
  size_t n_s2, n_m, n_g;   // elements of part_s2, part_m, part_g
#endif
};

struct GSmem {
  uint64_t a_full[kGStages][2];  // generator warps' stores into each 64-dimension chunk of the stage
  uint64_t a_empty[kGStages];  // both contractions of the stage done
  uint64_t s_ready[2];         // t-law scales of a tile
  uint64_t y_full;             // decision-operand slice landed
  uint64_t q_full, q_empty;    // forward accumulators
  uint64_t x_full;             // every CTA's partial rows are in this CTA's inbox (4 arrivals + bytes)
  uint64_t w_full;             // every CTA's rows of W are in this CTA's W (4 arrivals + bytes)
  uint64_t w_free;             // every CTA's adjoint of the tile is done (C multicast commits)
  uint64_t g_full, g_empty;    // per-tile block of G
  uint64_t drain, drain_adj;   // forward / adjoint MMAs complete (end of kernel)
  uint32_t tmem_base;
  uint32_t abort_flag;
  float s_buf[2][kGM];
  float gsc_f[kGKp];   // 2^(e_k + f_k)
  float wsc_f[kGKp];   // 2^-f_k
};

// Layout (1024-byte aligned base):
//   [stages: 2 x 64 KB]
//   [Y slice: 2 chunks of 64 dims x (hi, lo) x 64 decisions x 128 B]     32 KB, K-major
//   [W: (hi, lo) x 128 scenarios x 64 decisions (128 B)]                 32 KB, MN-major
//   [inbox: C sources x (128 / C) rows x 64 FP32]                       32 KB
//   [GSmem]
constexpr int kGOpBytes = 2 * 2 * kGKp * 128;
size_t grad_smem_bytes() { return (size_t)kGStages * kGStageBytes + (size_t)3 * kGOpBytes + sizeof(GSmem); }

// Float offset in the inbox of column k of row l (of the owner's rows) from
// source CTA p: 16-byte units XOR-swizzled by the row, so a warp's stores
// (32 rows, one unit each) and the owner's 16-byte reads are free of bank
// conflicts.
__device__ __forceinline__ uint32_t inbox_off(int p, int nr, int l, int k) {
  return (uint32_t)((p * nr + l) * kGKp + ((((k >> 2) ^ l) & 15) << 2) + (k & 3));
}

// D8: d is a multiple of 8, so every 8-dimension unit below d is whole and
// the per-element guards drop out.
// VO (value only): the forward, the exchange of partial Q and S2, without W,
// the adjoint or G; the tensor-core value path for 256 < d <= 1024, K <= 64.
// The forward's MMAs release the stage, and w_full becomes the signal that
// every CTA of the cluster has reduced the tile (4 C arrivals), after which
// the inbox and the staging in W may be reused.
template <bool F16, bool D8, bool VO>
__global__ void __launch_bounds__(kGThreads, 1) k_tc_grad(GArgs a) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  const uint32_t base = smem_u32(smem_raw);
  if (base & 1023u) {   // identical in every CTA: the whole cluster leaves together
    if (threadIdx.x == 0) atomicOr(a.err, kErrBounds);
    return;
  }
  const int C = a.C, nr = kGM / C;    // CTAs of the cluster; rows of the tile each one reduces
  const uint32_t rank = cluster_rank();
  const uint32_t cl = cluster_id(), ncl = cluster_count();
  uint8_t* ring = smem_raw;
  uint8_t* ybuf = ring + kGStages * kGStageBytes;
  uint8_t* wbuf = ybuf + kGOpBytes;
  float* inbox = reinterpret_cast<float*>(wbuf + kGOpBytes);
  GSmem* sm = reinterpret_cast<GSmem*>(wbuf + 2 * kGOpBytes);
  const uint32_t sRing = base, sY = smem_u32(ybuf), sW = smem_u32(wbuf), sIn = smem_u32(inbox);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const LawArgs& la = a.la;
  const int d = la.d;
  constexpr uint32_t bslice = 2 * kGKp * 128;   // one 64-dimension block of the decision operand
  constexpr uint32_t wchunk = kGM * 128;        // W: the hi (or lo) half, 128 scenarios x 64 decisions
  volatile uint32_t* abort_flag = &sm->abort_flag;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kGStages; ++s) {
      mbar_init(smem_u32(&sm->a_full[s][0]), kGRngWarps / 2);
      mbar_init(smem_u32(&sm->a_full[s][1]), kGRngWarps / 2);
      mbar_init(smem_u32(&sm->a_empty[s]), 1);
    }
    for (int s = 0; s < 2; ++s) mbar_init(smem_u32(&sm->s_ready[s]), kGM / 32);
    mbar_init(smem_u32(&sm->y_full), 1);
    mbar_init(smem_u32(&sm->q_full), 1);
    mbar_init(smem_u32(&sm->q_empty), kGEpiWarps);
    mbar_init(smem_u32(&sm->x_full), kGEpiWarps);
    mbar_init(smem_u32(&sm->w_full), VO ? kGEpiWarps * C : kGEpiWarps);
    mbar_init(smem_u32(&sm->w_free), C);
    mbar_init(smem_u32(&sm->g_full), 1);
    mbar_init(smem_u32(&sm->g_empty), kGEpiWarps);
    mbar_init(smem_u32(&sm->drain), 1);
    mbar_init(smem_u32(&sm->drain_adj), 1);
    sm->abort_flag = 0u;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int k = threadIdx.x; k < kGKp; k += blockDim.x) {
    sm->gsc_f[k] = (k < a.K) ? (float)a.gaux[k] : 0.0f;
    sm->wsc_f[k] = (k < a.K) ? (float)a.gaux[a.K + k] : 0.0f;
  }
  // TMEM, 64 columns each: Q, (unused), the tile's G hi*hi and corrections,
  // G's running sum, its Kahan compensation
  constexpr uint32_t ncols = 512u;
  if (warp == kGMmaWarp) tmem_alloc(smem_u32(&sm->tmem_base), ncols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  cluster_sync();   // every CTA's barriers are initialised before any peer arrives on them
  const uint32_t tmem = sm->tmem_base;
  const uint32_t tq1 = tmem, tg1 = tmem + 128u, tg2 = tmem + 192u;
  const uint32_t tgs = tmem + 256u, tgc = tmem + 320u;
  const int my_tiles = (cl < (uint32_t)a.tiles) ? (int)((a.tiles - cl + ncl - 1) / ncl) : 0;
  const uint16_t cmask = (uint16_t)((1u << C) - 1u);
  float s2h[8], s2l[8];           // epilogue: S2 of this thread's 8 columns (float-float)
  float mh[8], ml[8];             // generator: m~ of this thread's 8 dimensions (float-float)
#pragma unroll
  for (int q = 0; q < 8; ++q) mh[q] = ml[q] = s2h[q] = s2l[q] = 0.0f;

  if (warp == kGMmaWarp) {
    // ------------------------------------------------------------ MMA ---
    if (lane == 0) {
      // this CTA's two 64-dimension blocks of the decision operand, resident
      const uint32_t yb = smem_u32(&sm->y_full);
      mbar_expect_tx(yb, 2 * bslice);
      bulk_g2s(sY, a.bimage + (size_t)(2 * rank) * bslice, 2 * bslice, yb);
      bool ok = mbar_wait(yb, 0, abort_flag, a.err);
      // One FP32 accumulator per tile: the corrections A_hi B_lo and A_lo
      // B_hi of both chunks first, then A_hi B_hi, so the small terms are
      // not added to the large running sum (the accumulator's rounding is
      // relative to it).  This thread issues only the forward; the adjoint
      // is issued by the epilogue once W is in place, so the next tile's
      // forward never waits on it.
      const uint32_t idf1 = idesc_f16(kGM, kGKp, F16);
      constexpr uint32_t bhalf = kGKp * 128;   // the lo half of a decision block follows its hi half
      int st = 0;
      uint32_t ph = 0;
      for (int tt = 0; ok && tt < my_tiles; ++tt) {
        ok = tt == 0 || mbar_wait(smem_u32(&sm->q_empty), (uint32_t)((tt - 1) & 1), abort_flag, a.err);
        if (!ok) break;
        const uint32_t stage = sRing + (uint32_t)(st * kGStageBytes);
        // forward: Q^(r) over this CTA's 128 dimensions, 16 per k step, each
        // 64-dimension chunk as soon as it is drawn
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          ok = mbar_wait(smem_u32(&sm->a_full[st][c]), ph, abort_flag, a.err);
          if (!ok) break;
          tc_fence_after();
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint32_t o = (uint32_t)(kk * 32);
            const uint32_t a_hi = stage + (uint32_t)(c * 2 * kGChunkBytes) + o, a_lo = a_hi + kGChunkBytes;
            const uint32_t b_hi = sY + (uint32_t)c * bslice + o;
            mma_bf16(tq1, desc_sw128(a_hi), desc_sw128(b_hi + bhalf), idf1, (c == 0 && kk == 0) ? 0u : 1u);
            mma_bf16(tq1, desc_sw128(a_lo), desc_sw128(b_hi), idf1, 1u);
          }
        }
        if (!ok) break;
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint32_t o = (uint32_t)(kk * 32);
            const uint32_t a_hi = stage + (uint32_t)(c * 2 * kGChunkBytes) + o;
            mma_bf16(tq1, desc_sw128(a_hi), desc_sw128(sY + (uint32_t)c * bslice + o), idf1, 1u);
          }
        mma_commit(smem_u32(&sm->q_full));
        if (VO) mma_commit(smem_u32(&sm->a_empty[st]));   // no adjoint reads the stage
        if (++st == kGStages) { st = 0; ph ^= 1u; }
      }
      // every forward MMA and the operand copy complete before TMEM and the stages are released
      mma_commit(smem_u32(&sm->drain));
      uint32_t never = 0u;
      mbar_wait(smem_u32(&sm->drain), 0, &never, a.err);
      mbar_wait(yb, 0, &never, a.err);
    }
    __syncwarp();
  } else if (warp < kGEpiWarps) {
    // ------------------------------------------------------- epilogue ---
    // Warp w reads TMEM lane quadrant w (rows / dimensions 32 w .. 32 w + 31).
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    const int row = warp * 32 + lane;                // forward: scenario of this TMEM lane; adjoint: dimension
    const int own = row / nr, lrow = row - own * nr;  // CTA that reduces this row, and its place there
    const int e = threadIdx.x;                       // 0 .. 127
    const int kq = e & 7;                            // reduce: this thread's columns 8 kq .. 8 kq + 7
    const int r0 = (int)rank * nr;                   // reduce: this CTA's rows r0 .. r0 + nr - 1
    const bool issuer = (threadIdx.x == 0);          // issues the adjoint MMAs
    const uint32_t ida2 = idesc_f16(kGDims, 2 * kGKp, F16) | kIdescAMajorMN | kIdescBMajorMN;
    const uint32_t ida1 = idesc_f16(kGDims, kGKp, F16) | kIdescAMajorMN | kIdescBMajorMN;
    bool adj_issued = false;
    // Kahan fold of the block of G (hi*hi + corrections) that ends with
    // tile tf (kGFoldTiles tiles, fewer at the end) into the running sum;
    // then the block's TMEM is free for the next adjoint
    auto fold = [&](int tf) {
      tc_fence_after();
#pragma unroll 1
      for (uint32_t c0 = 0; c0 < (uint32_t)kGKp; c0 += 8) {
        uint32_t rg[8], rh[8], rs[8], rc[8];
        tmem_ld8(tg1 + lane_base + c0, rg);
        tmem_ld8(tg2 + lane_base + c0, rh);
        if (tf >= kGFoldTiles) {
          tmem_ld8(tgs + lane_base + c0, rs);
          tmem_ld8(tgc + lane_base + c0, rc);
        }
        tmem_wait_ld();
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const float g = __uint_as_float(rg[q]) + __uint_as_float(rh[q]);
          if (tf < kGFoldTiles) {
            rc[q] = 0u;
            rg[q] = __float_as_uint(g);
          } else {
            const float s = __uint_as_float(rs[q]), c = __uint_as_float(rc[q]);
            const float y = g - c;
            const float t = s + y;
            rc[q] = __float_as_uint((t - s) - y);
            rg[q] = __float_as_uint(t);
          }
        }
        tmem_st8(tgs + lane_base + c0, rg);
        tmem_st8(tgc + lane_base + c0, rc);
        tmem_wait_st();
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&sm->g_empty));
    };
    int tt = 0;
    for (; tt < my_tiles; ++tt) {
      // ---- this CTA's partial Q of every row: its own rows straight into its
      // inbox, every other owner's rows staged in W (free: this CTA's last
      // adjoint is done) in the inbox's layout, then one bulk copy per half
      // block into the owner's inbox, completing bytes of its x_full
      if (!warp_wait(smem_u32(&sm->q_full), (uint32_t)(tt & 1), abort_flag, a.err)) break;
      if (tt > 0 && !warp_wait_cluster(smem_u32(&sm->w_full), (uint32_t)((tt - 1) & 1), abort_flag, a.err)) break;
      // the last tile's adjoint is done: W is free for the staging below, and
      // that tile's block of G is folded while the other CTAs' copies travel
      if (!VO && tt > 0 && !warp_wait(smem_u32(&sm->g_full), (uint32_t)((tt - 1) & 1), abort_flag, a.err)) break;
      tc_fence_after();
      const uint32_t half = (uint32_t)nr * 128u;   // bytes of half an owner's block
#pragma unroll 1
      for (uint32_t c0 = 0; c0 < (uint32_t)kGKp; c0 += 16) {
        uint32_t r1v[16];
        tmem_ld16(tq1 + lane_base + c0, r1v);
        tmem_wait_ld();
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float4 q = make_float4(__uint_as_float(r1v[4 * u + 0]), __uint_as_float(r1v[4 * u + 1]),
                                       __uint_as_float(r1v[4 * u + 2]), __uint_as_float(r1v[4 * u + 3]));
          const uint32_t off = inbox_off(0, nr, lrow, (int)c0 + 4 * u);   // float offset in the block
          if (own == (int)rank) {
            if (bc_ok((size_t)(own * nr * kGKp) + off + 3u, (size_t)kGM * kGKp, a.err))   // the 32 KB inbox
              *reinterpret_cast<float4*>(inbox + (uint32_t)(own * nr * kGKp) + off) = q;
          } else {
            const uint32_t bo = 4u * off;
            const uint32_t so = bo < half ? (uint32_t)own * half + bo : wchunk + (uint32_t)own * half + (bo - half);
            if (bc_ok(so + 15u, 2u * wchunk, a.err)) *reinterpret_cast<float4*>(wbuf + so) = q;
          }
        }
      }
      tc_fence_before();
      fence_proxy_async();   // staged partials: generic stores -> the bulk copies' reads
      __syncwarp();
      // This warp's 32 rows are whole halves of the blocks of one or two
      // owners (nr / 2 <= 32 rows per half): one lane per half copies it into
      // that owner's inbox.  Each warp then arrives on this CTA's x_full with
      // a quarter of the bytes the other C - 1 CTAs will send.
      if (C > 1 && lane < 2 * ((32 + nr - 1) / nr) && lane * (nr / 2) < 32) {
        const int hrow = warp * 32 + lane * (nr / 2);   // first row of this half
        const int q = hrow / nr, hs = (hrow - q * nr) / (nr / 2);   // its owner and which half
        if (q != (int)rank) {
          const uint32_t src = hs == 0 ? sW + (uint32_t)q * half : sW + wchunk + (uint32_t)q * half;
          const uint32_t dst = sIn + 4u * (uint32_t)((int)rank * nr * kGKp) + (uint32_t)hs * half;
          bulk_s2cluster(mapa(dst, (uint32_t)q), src, half, mapa(smem_u32(&sm->x_full), (uint32_t)q));
        }
      }
      if (lane == 0) {
        mbar_arrive(smem_u32(&sm->q_empty));
        mbar_expect_tx(smem_u32(&sm->x_full), (uint32_t)(C - 1) * (uint32_t)nr * 64u);
      }
      __syncwarp();
      if (!VO && tt > 0 && tt % kGFoldTiles == 0) fold(tt - 1);
      // ---- reduce this CTA's rows: the C partials in rank order, S2, and W into every CTA
      if (!warp_wait_cluster(smem_u32(&sm->x_full), (uint32_t)(tt & 1), abort_flag, a.err)) break;
      float s2t[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) s2t[q] = 0.0f;
      // warp w reduces rows w nr / 4 .. (w + 1) nr / 4 - 1 of this CTA's
      // (contiguous, so that it can copy its rows of W by itself)
      const int rpw = nr / kGEpiWarps;   // rows per warp: 32 / C
#pragma unroll 1
      for (int l = warp * rpw + (lane >> 3); l < (warp + 1) * rpw; l += 4) {
        float q[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) q[j] = 0.0f;
#pragma unroll
        for (int p = 0; p < kGMaxCluster; ++p) {   // rank order: the sum does not depend on timing
          if (p < C) {
            const float4 va = *reinterpret_cast<const float4*>(inbox + inbox_off(p, nr, l, 8 * kq));
            const float4 vb = *reinterpret_cast<const float4*>(inbox + inbox_off(p, nr, l, 8 * kq + 4));
            q[0] += va.x; q[1] += va.y; q[2] += va.z; q[3] += va.w;
            q[4] += vb.x; q[5] += vb.y; q[6] += vb.z; q[7] += vb.w;
          }
        }
        uint4 hv, lv;
        uint32_t* hp = &hv.x;
        uint32_t* lp = &lv.x;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          s2t[2 * u] = fmaf(q[2 * u], q[2 * u], s2t[2 * u]);
          s2t[2 * u + 1] = fmaf(q[2 * u + 1], q[2 * u + 1], s2t[2 * u + 1]);
        }
        if constexpr (!VO) {
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float wa = q[2 * u] * sm->wsc_f[8 * kq + 2 * u];   // powers of two: exact
            const float wb = q[2 * u + 1] * sm->wsc_f[8 * kq + 2 * u + 1];
            hp[u] = pack2<F16>(wa, wb);
            const float2 h = unpack2<F16>(hp[u]);
            lp[u] = pack2<F16>(wa - h.x, wb - h.y);
          }
          // decisions 8 kq .. 8 kq + 7 of scenario i: one 16-byte unit of W's row i, swizzled by i
          // (this CTA's own rows; the other CTAs' copies of them follow by bulk copy)
          const int i = r0 + l;
          const uint32_t woff = (uint32_t)(i * 128 + ((kq ^ (i & 7)) << 4));
          if (bc_ok(woff + 15u, wchunk, a.err)) {
            *reinterpret_cast<uint4*>(wbuf + woff) = hv;
            *reinterpret_cast<uint4*>(wbuf + wchunk + woff) = lv;
          }
        }
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) ff_add(s2h[q], s2l[q], s2t[q]);
      if (VO) {
        // this warp has read its rows of the inbox: tell every CTA of the cluster
        __syncwarp();
        if (lane < C) mbar_arrive_remote(mapa(smem_u32(&sm->w_full), (uint32_t)lane));
        continue;
      }
      fence_proxy_async();   // W: generic stores -> the MMAs' and the bulk copies' reads
      __syncwarp();
      // this warp's rows of W into every other CTA's W (lane p: CTA p), once
      // every CTA's adjoint of the last tile is done (the rows there also
      // held that CTA's staged partial for this CTA, read by now: x_full is
      // complete); then this warp's quarter of the bytes this CTA receives
      if (C > 1 && tt > 0 &&
          !warp_wait_cluster(smem_u32(&sm->w_free), (uint32_t)((tt - 1) & 1), abort_flag, a.err))
        break;
      if (C > 1 && lane < C && lane != (int)rank) {
        const uint32_t wo = (uint32_t)(r0 + warp * rpw) * 128u, wbytes = (uint32_t)rpw * 128u;
        const uint32_t wb = mapa(smem_u32(&sm->w_full), (uint32_t)lane);
        bulk_s2cluster(mapa(sW + wo, (uint32_t)lane), sW + wo, wbytes, wb);
        bulk_s2cluster(mapa(sW + wchunk + wo, (uint32_t)lane), sW + wchunk + wo, wbytes, wb);
      }
      if (lane == 0) mbar_expect_tx(smem_u32(&sm->w_full), (uint32_t)(C - 1) * (uint32_t)nr * 64u);
      __syncwarp();
      // ---- adjoint: G^(r) = A^(r)' W of the tile, once every row of W is in place and the
      // last tile's block is folded; the stage is read as an MN-major A (dimensions
      // contiguous, 64-dimension chunks 32 KB apart), W as an MN-major B (decisions
      // contiguous, the hi and lo halves 16 KB apart)
      if (issuer) {
        bool ok = mbar_wait_cluster(smem_u32(&sm->w_full), (uint32_t)(tt & 1), abort_flag, a.err) &&
                  (tt % kGFoldTiles != 0 || tt == 0 ||   // a new block waits for the last one's fold
                   mbar_wait(smem_u32(&sm->g_empty), (uint32_t)((tt / kGFoldTiles - 1) & 1), abort_flag, a.err));
        if (ok) {
          tc_fence_after();
          const uint32_t stage = sRing + (uint32_t)((tt % kGStages) * kGStageBytes);
#pragma unroll
          for (int kk = 0; kk < 8; ++kk) {   // 16 scenarios per k step
            const uint32_t at_hi = stage + (uint32_t)(kk * 2048), at_lo = at_hi + kGChunkBytes;
            const uint64_t bw = desc_mn_sw128(sW + (uint32_t)(kk * 2048), wchunk, 1024);
            mma_bf16(tg1, desc_mn_sw128(at_hi, 2 * kGChunkBytes, 1024), bw, ida2,
                     (kk == 0 && tt % kGFoldTiles == 0) ? 0u : 1u);
            mma_bf16(tg2, desc_mn_sw128(at_lo, 2 * kGChunkBytes, 1024), bw, ida1, 1u);
          }
          mma_commit(smem_u32(&sm->a_empty[tt % kGStages]));
          mma_commit(smem_u32(&sm->g_full));
          mma_commit_multicast(smem_u32(&sm->w_free), cmask);
          adj_issued = true;
        }
      }
      __syncwarp();
    }
    bool folded = false;   // every tile's block is in the running sum
    if (!VO && tt == my_tiles && my_tiles > 0 &&
        warp_wait(smem_u32(&sm->g_full), (uint32_t)((my_tiles - 1) & 1), abort_flag, a.err)) {
      fold(my_tiles - 1);
      folded = true;
    }
    if (tt < my_tiles && C > 1) {
      // the loop was abandoned (a bounded wait ran out): the bulk copies
      // already issued by the CTAs of the cluster carry no completion this
      // CTA can wait for, so give them a bounded pause to land
      const long long t0 = clock64();
      while (clock64() - t0 < 400000ll) {
      }
    }
    if (issuer && adj_issued) {   // every adjoint MMA complete before TMEM and the stages are released
      mma_commit(smem_u32(&sm->drain_adj));
      uint32_t never = 0u;
      mbar_wait(smem_u32(&sm->drain_adj), 0, &never, a.err);
    }
    // ---- this CTA's dimensions of G: running sum and its compensation
    const int j = (int)rank * kGDims + row;
    if (folded) {
      tc_fence_after();
#pragma unroll 1
      for (uint32_t c0 = 0; c0 < (uint32_t)kGKp; c0 += 8) {
        uint32_t rs[8], rc[8];
        tmem_ld8(tgs + lane_base + c0, rs);
        tmem_ld8(tgc + lane_base + c0, rc);
        tmem_wait_ld();
        if (j < d) {
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int k = (int)c0 + q;
            if (k < a.K) {
              const size_t o = ((size_t)cl * a.K + k) * d + j;
              const float g = sm->gsc_f[k];   // power of two: exact
              if (bc_ok(o, SAA_BOUND(a.n_g), a.err)) {
                a.part_g[o] = __uint_as_float(rs[q]) * g;
                a.part_gc[o] = __uint_as_float(rc[q]) * g;
              }
            }
          }
        }
      }
    } else if (!VO && my_tiles == 0 && j < d) {
      for (int k = 0; k < a.K; ++k) {
        const size_t o = ((size_t)cl * a.K + k) * d + j;
        if (bc_ok(o, SAA_BOUND(a.n_g), a.err)) {
          a.part_g[o] = 0.0f;
          a.part_gc[o] = 0.0f;
        }
      }
    }
  } else {
    // ------------------------------------------------------------ RNG ---
    const int rt = threadIdx.x - 32 * (kGMmaWarp + 1);   // 0 .. 511
    const int ch = rt >> 8;                               // 64-dimension chunk: warps 0..7 chunk 0, 8..15 chunk 1
    const int cu = rt & 7;                                // 16-byte unit (8 dimensions) of the chunk
    const int rbase = (rt >> 3) & 31;                     // rows rbase, rbase + 32, rbase + 64, rbase + 96
    const int j0 = (int)rank * kGDims + ch * 64 + cu * 8; // first dimension of this thread's unit
    uint32_t epoch = la.epoch;
    if (la.t_dev) epoch += (uint32_t)(*la.t_dev / la.M);
    const gen::Stream gs = gen::make_stream(la.seed, epoch, la.instance);
    const uint32_t half = la.N / 2u;
    const bool tlaw = la.law == SAA_LAW_STUDENT_T;
    const bool live_unit = j0 < d;
    int st = 0;
    uint32_t ph = 0;
    for (int tt = 0; tt < my_tiles; ++tt) {
      const uint32_t tile = cl + (uint32_t)tt * ncl;
      const uint32_t i0 = la.i_base + tile * (uint32_t)kGM;
      const int nrow = (int)min((uint32_t)kGM, la.rows_end() - i0);
      const int sb = tt & 1;
      const uint32_t s_bar = smem_u32(&sm->s_ready[sb]);
      if (!warp_wait(smem_u32(&sm->a_empty[st]), ph ^ 1u, abort_flag, a.err)) break;
      // Past this wait every generator warp has finished tile tt - 2, the
      // last user of this scale buffer, so two buffers suffice.
      if (tlaw && rt < kGM) {   // generator warps 0..3 draw the tile's scales
        sm->s_buf[sb][rt] = (rt < nrow) ? gen::t_scale_f(gs, i0 + (uint32_t)rt, la.nu) : 0.0f;
        __syncwarp();
        if (lane == 0) mbar_arrive(s_bar);
      }
      if (tlaw && !warp_wait(s_bar, (uint32_t)((tt >> 1) & 1), abort_flag, a.err)) break;
      uint8_t* chunk = ring + st * kGStageBytes + ch * 2 * kGChunkBytes;
      float msum[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) msum[q] = 0.0f;
#pragma unroll 1
      for (int r = rbase; r < kGM; r += 32) {
        float v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = 0.0f;
        if (r < nrow && live_unit) {
          const uint32_t i = i0 + (uint32_t)r;
          const bool logn = gen::is_lognormal(la.law, i, half);
          float z[4];
          gen::Gen<float>::block(gs, (uint32_t)(j0 >> 2), i, logn, z);
#pragma unroll
          for (int q = 0; q < 4; ++q) v[q] = (D8 || j0 + q < d) ? z[q] : 0.0f;
          if (D8 || j0 + 4 < d) {
            gen::Gen<float>::block(gs, (uint32_t)(j0 >> 2) + 1u, i, logn, z);
#pragma unroll
            for (int q = 0; q < 4; ++q) v[4 + q] = (D8 || j0 + 4 + q < d) ? z[q] : 0.0f;
          }
          if (tlaw) {
            const float s = sm->s_buf[sb][r];
#pragma unroll
            for (int q = 0; q < 8; ++q) v[q] *= s;
          }
        }
        uint32_t hi[4], lo[4];
#pragma unroll
        for (int q = 0; q < 8; q += 2) {
          msum[q] += v[q];
          msum[q + 1] += v[q + 1];
          hi[q / 2] = pack2<F16>(v[q], v[q + 1]);
          const float2 h = unpack2<F16>(hi[q / 2]);
          lo[q / 2] = pack2<F16>(v[q] - h.x, v[q + 1] - h.y);
        }
        const uint32_t off = sw_off(r, cu);
        if (bc_ok(off + 15u, (size_t)kGChunkBytes, a.err)) {   // one 16-byte unit of each half of the chunk
          *reinterpret_cast<uint4*>(chunk + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
          *reinterpret_cast<uint4*>(chunk + kGChunkBytes + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) ff_add(mh[q], ml[q], msum[q]);
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&sm->a_full[st][ch]));
      if (++st == kGStages) { st = 0; ph ^= 1u; }
    }
  }

  // ----------------------------------------------------- CTA reductions ---
  __syncthreads();   // MMAs and the copy drained, TMEM reads done: the stages are free
  double* red_m = reinterpret_cast<double*>(ring);        // [32 row groups][128 dims]
  double* red_s2 = red_m + 32 * kGDims;                   // [128 epilogue threads][8 columns]
  double* s2loc = red_s2 + kGEpiThreads * 8;              // [64]
  if (warp > kGMmaWarp) {
    const int rt = threadIdx.x - 32 * (kGMmaWarp + 1);
    const int jl = (rt >> 8) * 64 + (rt & 7) * 8;
#pragma unroll
    for (int q = 0; q < 8; ++q) red_m[((rt >> 3) & 31) * kGDims + jl + q] = (double)mh[q] + (double)ml[q];
  } else if (warp < kGEpiWarps) {
#pragma unroll
    for (int q = 0; q < 8; ++q) red_s2[threadIdx.x * 8 + q] = (double)s2h[q] + (double)s2l[q];
  }
  __syncthreads();
  if (threadIdx.x < kGDims) {   // m~ of this CTA's dimensions, row groups added in order
    const int j = (int)rank * kGDims + threadIdx.x;
    double s = 0.0;
    for (int g = 0; g < 32; ++g) s += red_m[g * kGDims + threadIdx.x];
    if (j < d && bc_ok((size_t)cl * d + j, SAA_BOUND(a.n_m), a.err)) a.part_m[(size_t)cl * d + j] = s;
  }
  if (threadIdx.x < kGKp) {     // S2 of this CTA's rows: the 16 threads of column k, in order
    const int kq = threadIdx.x >> 3, q = threadIdx.x & 7;
    double s = 0.0;
    for (int m = 0; m < kGEpiThreads / 8; ++m) s += red_s2[(kq + 8 * m) * 8 + q];
    s2loc[threadIdx.x] = s;
  }
  cluster_sync();   // every CTA's S2 is in place and every peer is done with this CTA's buffers
  if (rank == 0 && threadIdx.x < a.K) {   // the cluster's S2, CTAs added in rank order
    const uint32_t o = smem_u32(s2loc + threadIdx.x);
    double s = 0.0;
    for (int p = 0; p < C; ++p) s += ld_cluster_f64(mapa(o, (uint32_t)p));
    if (bc_ok((size_t)cl * a.K + threadIdx.x, SAA_BOUND(a.n_s2), a.err))
      a.part_s2[(size_t)cl * a.K + threadIdx.x] = s * a.scale2[threadIdx.x];
  }
  cluster_sync();   // rank 0 has read every peer's S2
  if (warp == kGMmaWarp) {
    tc_fence_after();
    tmem_dealloc(tmem, ncols);
  }
}

}  // namespace tc

bool tc_grad_supported(const saa_problem* p, int K) { return p->d <= tc::kGMaxDim && K <= tc::kGKp; }

// CTAs per cluster: the dimensions in 128-wide slices, rounded up to a power
// of two so that the 128 rows of a tile split evenly among them (a CTA whose
// slice lies past d draws nothing).
static int grad_cluster(int d) {
  const int c = (d + tc::kGDims - 1) / tc::kGDims;
  return c <= 1 ? 1 : c <= 2 ? 2 : c <= 4 ? 4 : 8;
}

// The decision operand in 64-dimension blocks, two per CTA of the cluster
// (blocks past d are zero), 64 decision rows each.
static size_t grad_image_bytes(int d) { return (size_t)(2 * grad_cluster(d)) * 2 * tc::kGKp * 128; }

template <bool F16, bool D8, bool VO = false>
static const void* grad_kernel() {
  return (const void*)tc::k_tc_grad<F16, D8, VO>;
}

// Clusters of C CTAs that fit on the device at once (one CTA per SM), per
// (device, C): the persistent grid.  Queried once and cached.
static int grad_max_clusters(const saa_ctx* ctx, int C, int smem) {
  static std::mutex mu;
  static int cache[64][tc::kGMaxCluster + 1];
  std::lock_guard<std::mutex> lock(mu);
  int& slot = cache[ctx->device & 63][C];
  if (slot > 0) return slot;
  int best = ctx->sm_count / C;
  const void* kern = grad_kernel<true, true>();
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) == cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)C);
    cfg.blockDim = dim3(tc::kGThreads);
    cfg.dynamicSmemBytes = (size_t)smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) == cudaSuccess && n > 0) best = n;
  }
  cudaGetLastError();   // a failed query leaves no sticky error
  slot = best;
  return best;
}

saa_status tc_grad_plan(const saa_ctx* ctx, const saa_problem* p, int K, Plan* plan) {
  const int C = grad_cluster(p->d);
  plan->bm = tc::kGM;
  plan->cluster = C;
  plan->tiles = (p->N + tc::kGM - 1) / tc::kGM;
  plan->smem = (int)tc::grad_smem_bytes();
  if (plan->smem > ctx->smem_optin) {
    set_error("tensor-core gradient tile does not fit in shared memory");
    return SAA_EUNSUPPORTED;
  }
  const int64_t cl = grad_max_clusters(ctx, C, plan->smem);
  plan->grid = (int)(plan->tiles < cl ? plan->tiles : cl);   // clusters; the partial slots are per cluster
  // operand image, then scale2[K], gaux[2K]
  plan->tc_bytes = grad_image_bytes(p->d) + (size_t)24 * K;
  return SAA_OK;
}

cudaError_t launch_tc_grad(const LawArgs& la, int K, int prec, const Plan& plan, const Workspace& ws, uint32_t* err,
                           cudaStream_t st, bool value_only) {
  const bool f16 = (prec == SAA_F16X3);
  tc::GArgs a;
  a.la = la;
  a.K = K;
  a.C = plan.cluster;
  a.tiles = plan.tiles;
  uint8_t* img = (uint8_t*)ws.tc;
  double* scale2 = (double*)(img + grad_image_bytes(la.d));
  double* gaux = scale2 + K;
  a.bimage = img;
  a.gaux = gaux;
  a.scale2 = scale2;
  a.part_s2 = ws.part_s2;
  a.part_m = ws.part_m;
  a.part_g = (float*)ws.part_g;
  a.part_gc = (float*)ws.part_gc;
#ifdef SAA_BOUNDS_CHECK
  a.n_s2 = ws.n_s2;
  a.n_m = ws.n_m;
  a.n_g = ws.n_g;
#endif
  a.err = err;
  cudaError_t e = launch_tc_image(la.d, K, tc::kGKp, 2 * a.C, f16, ws.Y64, scale2, gaux, img, st);
  if (e != cudaSuccess) return e;
  const bool d8 = (la.d & 7) == 0;
  const void* kern =
      value_only ? (f16 ? (d8 ? grad_kernel<true, true, true>() : grad_kernel<true, false, true>())
                        : (d8 ? grad_kernel<false, true, true>() : grad_kernel<false, false, true>()))
                 : (f16 ? (d8 ? grad_kernel<true, true>() : grad_kernel<true, false>())
                        : (d8 ? grad_kernel<false, true>() : grad_kernel<false, false>()));
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, plan.smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(plan.grid * a.C));
  cfg.blockDim = dim3(tc::kGThreads);
  cfg.dynamicSmemBytes = (size_t)plan.smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)a.C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  void* args[] = {&a};
  return cudaLaunchKernelExC(&cfg, kern, args);
}

}  // namespace saa
