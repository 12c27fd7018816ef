// internal.cuh -- host/device declarations shared by the libsaa translation
// units (not part of the public ABI).
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstddef>
#include <cstdint>
#include <string>

#include "../../include/saa.h"

namespace saa {

constexpr int kThreads = 256;   // threads per CTA of the SIMT kernels
constexpr int kDK = 32;         // dimensions per staged Y chunk
constexpr int kMaxDimSimt = 1024;

// Device error word bits (ctx->err).
enum : uint32_t { kErrBounds = 1u, kErrTimeout = 2u, kErrInput = 4u };

// Index checks of the SAA_BOUNDS_CHECK build (-DSAA_BOUNDS_CHECK; libsaa_bounds.so).
// There an index at or past its buffer's capacity raises kErrBounds in the
// error word and the caller skips the access, instead of faulting: a stand-in
// for a memory checker where none can run.  In the normal build the checks
// compile to nothing.
#ifdef SAA_BOUNDS_CHECK
constexpr bool kBoundsCheck = true;
#else
constexpr bool kBoundsCheck = false;
#endif
// A bound that exists only in the checked build (its kernel-argument fields
// are compiled in there alone, so the normal build's arguments and code stay
// as they are).
#ifdef SAA_BOUNDS_CHECK
#define SAA_BOUND(n) (n)
#else
#define SAA_BOUND(n) (~(size_t)0)
#endif
__device__ __forceinline__ bool bc_ok(size_t i, size_t n, uint32_t* err) {
  if (kBoundsCheck && i >= n) {
    atomicOr(err, kErrBounds);
    return false;
  }
  return true;
}

// Everything a sample-generating kernel needs to know about the law.
struct LawArgs {
  int d;
  int law;
  int nu;
  uint32_t N;
  uint64_t seed;
  uint32_t instance;
  uint32_t epoch;            // base resample index
  const int64_t* t_dev;      // optional: device iteration counter (Frank-Wolfe)
  int32_t M;                 // resample period when t_dev is set
  // Scenario range [i_base, i_base + n) of the sums (saa_partials); n = 0
  // means the whole set [0, N).  N itself stays the problem's (the mixed
  // law's split at N/2 and the counter words do not depend on the range).
  uint32_t i_base = 0;
  uint32_t n = 0;
  __host__ __device__ uint32_t rows_end() const { return n ? i_base + n : N; }
};

// Per-call workspace carve-up.  Partials are per CTA ("grid" of them) and are
// merged in CTA order by the finalize kernels, so results are deterministic.
struct Workspace {
  void* Y;            // [K][d] scalar (float or double): y_k = C' w_k
  double* Y64;        // [K][d] double copy (tensor paths build operands from it)
  double* c;          // [K] mu' w_k
  double* part_s1;    // [grid][K] sum_i Q_ik
  double* part_s2;    // [grid][K] sum_i Q_ik^2
  double* part_m;     // [grid][d] sum_i s_i zhat_i
  void* part_g;       // [grid][K][d] scalar: sum_i s_i zhat_i Q_ik  (grad)
  void* part_gc;      // [grid][K][d] scalar: Kahan compensation of part_g
  double* tot_s1;     // [K]
  double* tot_s2;     // [K]
  double* tot_m;      // [d]
  double* grad_tmp;   // [K][d] u_k of the gradient finalize
  double* grad_out;   // [K][d] (solve: gradient of the iterate)
  double* f_tmp;      // [K]    (solve)
  int64_t* t_dev;     // [1]    (solve: iteration counter)
  void* tc;           // tensor-path operand area
  float* q_dev;       // diagonal path: [N][K] Q_ik of the forward pass
  float* s_dev;       // diagonal path: [N] scales s_i
  double* part_gd;    // diagonal path: [slices][K][d] adjoint partials of G
  double* part_md;    // diagonal path: [slices][d] adjoint partials of m~
  float* zs;          // diagonal path, sample store: [N][round_up(d, 4)] FP32 normals
  size_t n_s2, n_m, n_g;   // elements of part_s2, part_m, part_g / part_gc (the bounds of the checked build)
  size_t bytes;       // total
};

struct Plan {
  int prec;       // saa_prec
  int bm;         // scenarios per tile
  int tn;         // SIMT: decisions per thread column group (K-chunk = 16 tn)
  int narrow;     // SIMT: K <= 4 kernel (dot products fused into the draw)
  int grid;       // CTAs of the main kernel
  int smem;       // dynamic shared memory of the main kernel
  int64_t tiles;  // scenario tiles
  size_t tc_bytes;
  int diag;       // diagonal covariance path (chol NULL, sd given)
  int nsplit;     // diagonal path: scenario slices of the adjoint
  int ablk;       // diagonal path: adjoint blocks over the dimensions
  int keep;       // diagonal path: the forward pass stores the normals for the adjoint
  int cluster;    // tensor-core gradient: CTAs per thread-block cluster (grid counts clusters)
};

}  // namespace saa

struct saa_ctx {
  int device;
  int sm_count;
  int smem_optin;
  uint32_t* err;                 // device error word
  // graph of the last saa_solve (kept until the next solve or destroy)
  cudaGraphExec_t fw_exec;
  cudaGraphExec_t* fw_more;      // graphs of the last saa_solve_adaptive (one per run of equal N)
  int fw_more_n;
  // kernel timing (saa_profile_*)
  int prof_on;
  int prof_n;                    // recorded event pairs
  cudaEvent_t prof_ev[2 * 256];  // (start, end) pairs, created on enable
  int64_t kernels;               // kernels launched since the last read
  // ragged batches: pinned staging buffer for the descriptor tables
  void* stage;
  size_t stage_bytes;
  cudaEvent_t stage_ready;       // the last upload from `stage` has completed
  int autotune;                  // time candidate tile shapes on a new batch shape
  size_t store_cap;              // diagonal path: most bytes of kept FP32 samples
};

namespace saa {

// NVTX range over one entry-point call (host side).  The NVTX v3 headers
// load no library unless a profiler injects one, so without a tool this is
// a pair of cheap no-op calls.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

void set_error(const std::string& msg);
saa_status cuda_status(cudaError_t e, const char* what);

// Plan and workspace for a problem (host).
saa_status make_plan(const saa_ctx* ctx, const saa_problem* p, int K, saa_prec prec, int want_grad, Plan* plan);
size_t carve(const saa_problem* p, int K, const Plan& plan, int want_grad, void* base, Workspace* ws);

// Launchers (host, one per translation unit).
cudaError_t launch_prologue(const saa_problem* p, int K, const double* X, int prec, const Workspace& ws,
                            uint32_t* err, cudaStream_t st);
cudaError_t launch_simt(const LawArgs& la, int K, int prec, int want_grad, const Plan& plan, const Workspace& ws,
                        cudaStream_t st);
cudaError_t launch_finalize(const saa_problem* p, int K, int prec, int want_grad, const Plan& plan,
                            const Workspace& ws, double* f, double* pbar, double* var, double* grad,
                            cudaStream_t st);
// saa_partials: the CTA partials of a scenario range, merged and mapped to
// [P1 | P2 | P3 = C m~ | P4 = C G (want_grad)] in `part`.
cudaError_t launch_partials_out(const saa_problem* p, int K, int prec, int want_grad, const Plan& plan,
                                const Workspace& ws, double* part, cudaStream_t st);
// saa_partials_merge: fixed-order compensated sum of R partial vectors.
cudaError_t launch_merge_partials(int R, int64_t len, const double* parts, double* total, cudaStream_t st);
// saa_finalize_partials: f, pbar, var, grad from the totals of the partials.
cudaError_t launch_finalize_partials(int64_t N, int d, int K, double lambda, const double* X, const double* mu,
                                     const double* part, double* f, double* pbar, double* var, double* grad,
                                     cudaStream_t st);
// grad_kj = sum_{l <= j} C_jl u_kl - mu_j (FP64, one warp per output).
cudaError_t launch_grad_out(int K, int d, const double* chol, const double* mu, const double* u, double* grad,
                            cudaStream_t st);
cudaError_t launch_generate(const LawArgs& la, int64_t i0, int64_t n, int prec, const double* mu,
                            const double* chol, void* z, void* s, void* xi, cudaStream_t st);
cudaError_t launch_fw_step(int d, const double* g, const double* f, double* w, const int64_t* t_dev,
                           int64_t t_base, double* f_trace, double* gap_trace, int64_t* t_next, cudaStream_t st);

// SIMT tile shape for (prec, d, K).
int simt_bm(int prec, int d);
int simt_tn(int K);
size_t simt_smem(int prec, int d, int bm, int tn);
int simt_occupancy(int prec, int bm, int tn, int smem);
size_t narrow_smem(int prec, int d, int bm);
int narrow_occupancy(int prec, int bm, int smem);

// Diagonal-covariance path of any dimension (large_d.cu).
saa_status diag_plan(const saa_ctx* ctx, const saa_problem* p, int K, saa_prec prec, int want_grad, Plan* plan);
size_t diag_carve(const saa_problem* p, int K, const Plan& plan, int want_grad, void* base, Workspace* ws);
cudaError_t launch_diag(const saa_problem* p, int K, const double* X, const LawArgs& la, int want_grad,
                        const Plan& plan, const Workspace& w, double* f, double* pbar, double* var, double* grad,
                        uint32_t* err, cudaStream_t st, cudaEvent_t ev0, cudaEvent_t ev1);

// Tensor-core (tcgen05, BF16 or FP16 hi/lo) value path.
inline bool is_tc(int prec) { return prec == SAA_BF16X3 || prec == SAA_F16X3; }
bool tc_supported(const saa_problem* p, int K, int want_grad);
saa_status tc_plan(const saa_ctx* ctx, const saa_problem* p, int K, Plan* plan);
cudaError_t launch_tc(const LawArgs& la, int K, int prec, const Plan& plan, const Workspace& ws, uint32_t* err,
                      cudaStream_t st);
cudaError_t launch_tc_image(int d, int K, int Kp, int nkb, bool f16, const double* Y64, double* scale2,
                            double* gaux, uint8_t* img, cudaStream_t st);

// Tensor-core path with the gradient (two passes over each tile).
bool tc_grad_supported(const saa_problem* p, int K);
saa_status tc_grad_plan(const saa_ctx* ctx, const saa_problem* p, int K, Plan* plan);
cudaError_t launch_tc_grad(const LawArgs& la, int K, int prec, const Plan& plan, const Workspace& ws, uint32_t* err,
                           cudaStream_t st,
                           bool value_only = false);

}  // namespace saa
