// saa_api.cu -- the C ABI declared in include/saa.h: argument validation,
// launch planning, workspace carve-up and the launch sequences of
// saa_eval / saa_grad / saa_solve / saa_generate.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "internal.cuh"

namespace saa {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

saa_status cuda_status(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return SAA_OK;
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return SAA_ECUDA;
}

cudaError_t launch_set_i64(int64_t* p, int64_t v, cudaStream_t st);
cudaError_t launch_selftest_timeout(uint32_t* err, uint32_t budget_us, cudaStream_t st);
cudaError_t launch_selftest_bounds(uint32_t* err, cudaStream_t st);

static saa_status fail(saa_status s, const std::string& msg) {
  set_error(msg);
  return s;
}

static saa_status check_problem(const saa_problem* p) {
  if (!p) return fail(SAA_EINVAL, "problem is NULL");
  if (p->d < 1) return fail(SAA_EINVAL, "d must be >= 1");
  if (p->N < 2) return fail(SAA_EINVAL, "N must be >= 2 (the variance divides by N-1)");
  if (p->N > 0xffffffffll) return fail(SAA_EINVAL, "N must be < 2^32 (scenario counter word)");
  if (p->law < SAA_LAW_GAUSS || p->law > SAA_LAW_MIX) return fail(SAA_EINVAL, "unknown law");
  if (p->law == SAA_LAW_STUDENT_T && (p->nu < 2 || (p->nu & 1) || p->nu > 64))
    return fail(SAA_EINVAL, "t law needs an even nu in [2, 64]");
  if (p->reserved != 0) return fail(SAA_EINVAL, "reserved field must be 0");
  if (!p->mu || (!p->chol && !p->sd)) return fail(SAA_EINVAL, "mu and chol (or sd) must be device pointers");
  return SAA_OK;
}

static size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

saa_status make_plan(const saa_ctx* ctx, const saa_problem* p, int K, saa_prec prec, int want_grad, Plan* plan) {
  std::memset(plan, 0, sizeof(*plan));
  plan->prec = prec;
  if (!p->chol) return diag_plan(ctx, p, K, prec, want_grad, plan);
  if (is_tc(prec) && want_grad) {
    if (!tc_grad_supported(p, K))
      return fail(SAA_EUNSUPPORTED, "tensor-core gradient path: needs d <= 1024 and K <= 64");
    return tc_grad_plan(ctx, p, K, plan);
  }
  if (is_tc(prec)) {
    if (tc_supported(p, K, want_grad)) return tc_plan(ctx, p, K, plan);
    // values above d = 256: the cluster kernel without its adjoint
    if (tc_grad_supported(p, K)) return tc_grad_plan(ctx, p, K, plan);
    return fail(SAA_EUNSUPPORTED, "tensor-core value path: needs d <= 256 (K <= 256) or d <= 1024 with K <= 64");
  }
  if (prec == SAA_FP8X)
    return fail(SAA_EUNSUPPORTED, "SAA_FP8X runs in the streamed mode only (saa_eval_samples)");
  if (prec != SAA_FP32 && prec != SAA_FP64) return fail(SAA_EUNSUPPORTED, "precision not built");
  if (p->d > kMaxDimSimt) return fail(SAA_EUNSUPPORTED, "d exceeds saa_max_dim for this precision");
  plan->bm = simt_bm(prec, p->d);
  plan->tn = simt_tn(K);
  plan->narrow = (K <= 4) ? 1 : 0;
  plan->smem = plan->narrow ? (int)narrow_smem(prec, p->d, plan->bm) : (int)simt_smem(prec, p->d, plan->bm, plan->tn);
  if (plan->smem > ctx->smem_optin) return fail(SAA_EUNSUPPORTED, "tile does not fit in shared memory");
  plan->tiles = (p->N + plan->bm - 1) / plan->bm;
  const int occ = plan->narrow ? narrow_occupancy(prec, plan->bm, plan->smem)
                               : simt_occupancy(prec, plan->bm, plan->tn, plan->smem);
  const int64_t cap = (int64_t)ctx->sm_count * occ;
  plan->grid = (int)(plan->tiles < cap ? plan->tiles : cap);
  return SAA_OK;
}

size_t carve(const saa_problem* p, int K, const Plan& plan, int want_grad, void* base, Workspace* ws) {
  if (plan.diag) return diag_carve(p, K, plan, want_grad, base, ws);
  const size_t d = (size_t)p->d, k = (size_t)K, g = (size_t)plan.grid;
  const size_t es = (plan.prec == SAA_FP64) ? 8 : 4;
  char* b = (char*)base;
  size_t off = 0;
  auto take = [&](size_t bytes) -> void* {
    void* r = b ? (void*)(b + off) : nullptr;
    off = align_up(off + bytes);
    return r;
  };
  Workspace w;
  std::memset(&w, 0, sizeof(w));
  w.Y = take(k * d * es);
  w.Y64 = (double*)take(k * d * 8);
  w.c = (double*)take(k * 8);
  w.part_s1 = (double*)take(g * k * 8);
  w.part_s2 = (double*)take(g * k * 8);
  w.part_m = (double*)take(g * d * 8);
  if (want_grad) {
    w.part_g = take(g * k * d * es);
    w.part_gc = take(g * k * d * es);
    w.grad_tmp = (double*)take(k * d * 8);
  }
  w.tot_s1 = (double*)take(k * 8);
  w.tot_s2 = (double*)take(k * 8);
  w.tot_m = (double*)take(d * 8);
  if (want_grad == 2) {
    w.f_tmp = (double*)take(k * 8);
    w.t_dev = (int64_t*)take(8);
    w.grad_out = (double*)take(k * d * 8);
  }
  if (plan.tc_bytes) w.tc = take(plan.tc_bytes);
  w.n_s2 = g * k;
  w.n_m = g * d;
  w.n_g = want_grad ? g * k * d : 0;
  w.bytes = off;
  if (ws) *ws = w;
  return off;
}

// Makes ctx->device current for the duration of a call.
struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

static LawArgs law_args(const saa_problem* p) {
  LawArgs la;
  la.d = p->d;
  la.law = p->law;
  la.nu = p->nu;
  la.N = (uint32_t)p->N;
  la.seed = p->seed;
  la.instance = p->instance;
  la.epoch = p->epoch;
  la.t_dev = nullptr;
  la.M = 1;
  return la;
}

// prologue -> main kernel -> finalize, all on `st`.
static saa_status run_estimator(saa_ctx* ctx, const saa_problem* p, int K, const double* X, saa_prec prec,
                                int want_grad, const Plan& plan, const Workspace& ws, const LawArgs& la, double* f,
                                double* pbar, double* var, double* grad, cudaStream_t st) {
  if (plan.diag) {
    const bool prof = ctx->prof_on && !la.t_dev && ctx->prof_n < 256;
    cudaEvent_t e0 = prof ? ctx->prof_ev[2 * ctx->prof_n] : nullptr;
    cudaEvent_t e1 = prof ? ctx->prof_ev[2 * ctx->prof_n + 1] : nullptr;
    if (prof) ++ctx->prof_n;
    const saa_status s = cuda_status(launch_diag(p, K, X, la, want_grad, plan, ws, f, pbar, var, grad, ctx->err, st,
                                                 e0, e1),
                                     "diagonal-covariance path launch");
    ctx->kernels += 3 + (want_grad ? 1 : 0) + ((want_grad && grad) ? 1 : 0);
    return s;
  }
  saa_status s = cuda_status(launch_prologue(p, K, X, prec, ws, ctx->err, st), "prologue launch");
  if (s != SAA_OK) return s;
  const bool prof = ctx->prof_on && !la.t_dev && ctx->prof_n < 256;
  if (prof) cudaEventRecord(ctx->prof_ev[2 * ctx->prof_n], st);
  if (is_tc(prec) && (want_grad || plan.cluster > 0))
    s = cuda_status(launch_tc_grad(la, K, prec, plan, ws, ctx->err, st, !want_grad),
                    "tensor-core gradient kernel launch");
  else if (is_tc(prec))
    s = cuda_status(launch_tc(la, K, prec, plan, ws, ctx->err, st), "tensor-core kernel launch");
  else
    s = cuda_status(launch_simt(la, K, prec, want_grad, plan, ws, st), "sample kernel launch");
  if (s != SAA_OK) return s;
  if (prof) cudaEventRecord(ctx->prof_ev[2 * ctx->prof_n++ + 1], st);
  s = cuda_status(launch_finalize(p, K, prec, want_grad, plan, ws, f, pbar, var, grad, st), "finalize launch");
  // prologue, main, reduce, value outputs, gradient (2); tensor path: operand
  // image + value outputs with S1 from m~ (always launched)
  ctx->kernels += 3 + ((want_grad && grad) ? 2 : 0) + (is_tc(prec) ? 2 : ((f || pbar || var) ? 1 : 0));
  return s;
}

// Frees the graphs of the previous solve (their replays may still be queued
// on another stream, hence the device-wide wait).
void release_fw_graphs(saa_ctx* ctx) {
  if (!ctx->fw_exec && ctx->fw_more_n == 0) return;
  cudaDeviceSynchronize();
  if (ctx->fw_exec) cudaGraphExecDestroy(ctx->fw_exec);
  ctx->fw_exec = nullptr;
  for (int i = 0; i < ctx->fw_more_n; ++i) cudaGraphExecDestroy(ctx->fw_more[i]);
  delete[] ctx->fw_more;
  ctx->fw_more = nullptr;
  ctx->fw_more_n = 0;
}

// T iterations of Algorithm 1 from global iteration t0 on the samples of
// prob (its N), starting from w_in (copied to w_out unless they are the
// same array): one iteration captured as a graph and replayed T times.  The
// instantiated graph is returned in *exec for the caller to keep alive.
saa_status solve_run(saa_ctx* ctx, const saa_problem* prob, const double* w_in, int32_t T, int32_t M,
                            int64_t t0, saa_prec prec, double* w_out, double* f_trace, double* gap_trace, void* ws,
                            size_t ws_bytes, cudaStream_t st, cudaGraphExec_t* exec) {
  *exec = nullptr;
  Plan plan;
  saa_status s = make_plan(ctx, prob, 1, prec, 1, &plan);
  if (s != SAA_OK) return s;
  Workspace w;
  const size_t need = carve(prob, 1, plan, 2, ws, &w);
  if (ws_bytes < need) return fail(SAA_ENOMEM, "workspace smaller than saa_workspace_size(..., want_grad=2)");
  const int d = prob->d;
  if (w_in != w_out) {
    s = cuda_status(cudaMemcpyAsync(w_out, w_in, sizeof(double) * d, cudaMemcpyDeviceToDevice, st), "copy w0");
    if (s != SAA_OK) return s;
  }
  s = cuda_status(launch_set_i64(w.t_dev, t0, st), "set iteration counter");
  if (s != SAA_OK || T == 0) return s;

  LawArgs la = law_args(prob);
  la.t_dev = w.t_dev;
  la.M = M;
  // Capture one iteration on a private stream, replay it T times on `st`.
  cudaStream_t cap;
  s = cuda_status(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "create capture stream");
  if (s != SAA_OK) return s;
  cudaGraph_t graph = nullptr;
  s = cuda_status(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal), "begin capture");
  if (s == SAA_OK) {
    saa_status r = run_estimator(ctx, prob, 1, w_out, prec, 1, plan, w, la, w.f_tmp, nullptr, nullptr, w.grad_out,
                                 cap);
    if (r == SAA_OK)
      r = cuda_status(launch_fw_step(d, w.grad_out, w.f_tmp, w_out, w.t_dev, t0, f_trace, gap_trace, w.t_dev, cap),
                      "Frank-Wolfe step launch");
    cudaError_t e = cudaStreamEndCapture(cap, &graph);
    s = (r != SAA_OK) ? r : cuda_status(e, "end capture");
  }
  if (s == SAA_OK) s = cuda_status(cudaGraphInstantiate(exec, graph, 0), "instantiate graph");
  for (int32_t it = 0; s == SAA_OK && it < T; ++it) s = cuda_status(cudaGraphLaunch(*exec, st), "graph launch");
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(cap);
  return s;
}

}  // namespace saa

using namespace saa;

extern "C" {

saa_status saa_ctx_create(saa_ctx** out, int device) {
  if (!out) return fail(SAA_EINVAL, "out is NULL");
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n)
    return fail(SAA_EINVAL, "no such CUDA device");
  DeviceGuard g(device);
  if (!g.ok) return fail(SAA_ECUDA, "cudaSetDevice failed");
  saa_ctx* c = new (std::nothrow) saa_ctx();
  if (!c) return fail(SAA_ENOMEM, "host allocation failed");
  std::memset(c, 0, sizeof(*c));
  c->device = device;
  cudaDeviceProp prop;
  saa_status s = cuda_status(cudaGetDeviceProperties(&prop, device), "cudaGetDeviceProperties");
  if (s == SAA_OK) {
    c->sm_count = prop.multiProcessorCount;
    c->smem_optin = (int)prop.sharedMemPerBlockOptin;
    if (prop.major != 10) s = fail(SAA_EUNSUPPORTED, "libsaa is built for sm_103a (Blackwell) only");
  }
  if (s == SAA_OK) s = cuda_status(cudaMalloc((void**)&c->err, sizeof(uint32_t)), "cudaMalloc(error word)");
  if (s == SAA_OK) s = cuda_status(cudaMemset(c->err, 0, sizeof(uint32_t)), "cudaMemset(error word)");
  if (s == SAA_OK)
    s = cuda_status(cudaEventCreateWithFlags(&c->stage_ready, cudaEventDisableTiming), "cudaEventCreate(stage)");
  if (s != SAA_OK) {
    if (c->err) cudaFree(c->err);
    delete c;
    return s;
  }
  c->autotune = 1;
  c->store_cap = (size_t)1 << 35;
  *out = c;
  return SAA_OK;
}

void saa_ctx_destroy(saa_ctx* ctx) {
  if (!ctx) return;
  DeviceGuard g(ctx->device);
  release_fw_graphs(ctx);
  if (ctx->prof_on)
    for (int i = 0; i < 2 * 256; ++i) cudaEventDestroy(ctx->prof_ev[i]);
  if (ctx->stage) {
    cudaEventSynchronize(ctx->stage_ready);
    cudaFreeHost(ctx->stage);
  }
  if (ctx->stage_ready) cudaEventDestroy(ctx->stage_ready);
  if (ctx->err) cudaFree(ctx->err);
  delete ctx;
}

saa_status saa_ctx_sync(saa_ctx* ctx, void* stream) {
  if (!ctx) return fail(SAA_EINVAL, "ctx is NULL");
  DeviceGuard g(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  saa_status s = cuda_status(cudaStreamSynchronize(st), "cudaStreamSynchronize");
  if (s != SAA_OK) return s;
  uint32_t w = 0;
  s = cuda_status(cudaMemcpy(&w, ctx->err, sizeof(w), cudaMemcpyDeviceToHost), "read error word");
  if (s != SAA_OK) return s;
  if (w) {
    cudaMemset(ctx->err, 0, sizeof(uint32_t));
    if (w & kErrTimeout) return fail(SAA_ETIMEOUT, "a bounded device wait gave up");
    return fail(SAA_EDEVICE, "a device-side check flagged an error");
  }
  return SAA_OK;
}

saa_status saa_selftest_timeout(saa_ctx* ctx, uint32_t budget_us, void* stream) {
  if (!ctx) return fail(SAA_EINVAL, "ctx is NULL");
  if (budget_us < 1 || budget_us > 100000) return fail(SAA_EINVAL, "budget must be in [1 us, 100 ms]");
  DeviceGuard g(ctx->device);
  return cuda_status(launch_selftest_timeout(ctx->err, budget_us, (cudaStream_t)stream), "self-test launch");
}

int32_t saa_bounds_check_enabled(void) { return kBoundsCheck ? 1 : 0; }

saa_status saa_selftest_bounds(saa_ctx* ctx, void* stream) {
  if (!ctx) return fail(SAA_EINVAL, "ctx is NULL");
  if (!kBoundsCheck)
    return fail(SAA_EUNSUPPORTED, "index checks are compiled out of this build (build with SAA_BOUNDS_CHECK)");
  DeviceGuard g(ctx->device);
  return cuda_status(launch_selftest_bounds(ctx->err, (cudaStream_t)stream), "self-test launch");
}

saa_status saa_ctx_set_autotune(saa_ctx* ctx, int enable) {
  if (!ctx) return fail(SAA_EINVAL, "ctx is NULL");
  ctx->autotune = enable ? 1 : 0;
  return SAA_OK;
}

saa_status saa_ctx_set_sample_store(saa_ctx* ctx, size_t max_bytes) {
  if (!ctx) return fail(SAA_EINVAL, "ctx is NULL");
  ctx->store_cap = max_bytes;
  return SAA_OK;
}

saa_status saa_profile_enable(saa_ctx* ctx, int enable) {
  if (!ctx) return fail(SAA_EINVAL, "ctx is NULL");
  DeviceGuard g(ctx->device);
  if (enable && !ctx->prof_on) {
    for (int i = 0; i < 2 * 256; ++i) {
      saa_status s = cuda_status(cudaEventCreate(&ctx->prof_ev[i]), "cudaEventCreate");
      if (s != SAA_OK) {
        for (int j = 0; j < i; ++j) cudaEventDestroy(ctx->prof_ev[j]);
        return s;
      }
    }
    ctx->prof_on = 1;
  } else if (!enable && ctx->prof_on) {
    for (int i = 0; i < 2 * 256; ++i) cudaEventDestroy(ctx->prof_ev[i]);
    ctx->prof_on = 0;
  }
  ctx->prof_n = 0;
  ctx->kernels = 0;
  return SAA_OK;
}

saa_status saa_profile_read(saa_ctx* ctx, double* main_ms, int64_t* main_launches, int64_t* kernels_launched) {
  if (!ctx) return fail(SAA_EINVAL, "ctx is NULL");
  DeviceGuard g(ctx->device);
  double total = 0.0;
  for (int i = 0; i < ctx->prof_n; ++i) {
    saa_status s = cuda_status(cudaEventSynchronize(ctx->prof_ev[2 * i + 1]), "cudaEventSynchronize");
    if (s != SAA_OK) return s;
    float ms = 0.f;
    s = cuda_status(cudaEventElapsedTime(&ms, ctx->prof_ev[2 * i], ctx->prof_ev[2 * i + 1]), "cudaEventElapsedTime");
    if (s != SAA_OK) return s;
    total += ms;
  }
  if (main_ms) *main_ms = total;
  if (main_launches) *main_launches = ctx->prof_n;
  if (kernels_launched) *kernels_launched = ctx->kernels;
  ctx->prof_n = 0;
  ctx->kernels = 0;
  return SAA_OK;
}

int32_t saa_max_dim(saa_prec prec) {
  switch (prec) {
    case SAA_FP64:
    case SAA_FP32: return kMaxDimSimt;
    case SAA_BF16X3:
    case SAA_F16X3: return 1024;
    default: return 0;
  }
}

saa_status saa_plan_info(const saa_ctx* ctx, const saa_problem* prob, int32_t K, saa_prec prec, int want_grad,
                         int32_t* grid, int32_t* cluster, int64_t* tiles) {
  if (!ctx) return fail(SAA_EINVAL, "ctx is NULL");
  saa_status s = check_problem(prob);
  if (s != SAA_OK) return s;
  if (K < 1 || K > 65535) return fail(SAA_EINVAL, "K must be in [1, 65535]");
  DeviceGuard g(ctx->device);
  Plan plan;
  s = make_plan(ctx, prob, K, prec, want_grad ? 1 : 0, &plan);
  if (s != SAA_OK) return s;
  const int c = plan.cluster > 0 ? plan.cluster : 1;
  if (grid) *grid = plan.grid * c;
  if (cluster) *cluster = c;
  if (tiles) *tiles = plan.tiles;
  return SAA_OK;
}

// Decisions per launch when one tensor-core launch cannot take all K (0:
// one launch, or not a tensor precision): saa_eval and saa_grad then run K
// as consecutive chunks of that size.  Each decision's estimate depends
// only on the scenarios, which every chunk redraws identically, and on its
// own x_k.
static int tc_chunk(const saa_problem* p, int K, saa_prec prec, int want_grad) {
  if (!is_tc(prec) || !p->chol) return 0;
  if (want_grad) return (!tc_grad_supported(p, K) && tc_grad_supported(p, 64)) ? 64 : 0;
  if (tc_supported(p, K, 0) || tc_grad_supported(p, K)) return 0;
  for (int k = 256; k >= 32; k /= 2)
    if (tc_supported(p, k, 0)) return k;
  return tc_grad_supported(p, 64) ? 64 : 0;
}

size_t saa_workspace_size(const saa_ctx* ctx, const saa_problem* prob, int32_t K, saa_prec prec, int want_grad) {
  if (!ctx || check_problem(prob) != SAA_OK || K < 1) return 0;
  if (want_grad == 2) K = 1;
  const int kc = want_grad == 2 ? 0 : tc_chunk(prob, K, prec, want_grad);
  if (kc > 0) K = kc;
  DeviceGuard g(ctx->device);
  Plan plan;
  if (make_plan(ctx, prob, K, prec, want_grad ? 1 : 0, &plan) != SAA_OK) return 0;
  return carve(prob, K, plan, want_grad, nullptr, nullptr);
}

static saa_status eval_impl(saa_ctx* ctx, const saa_problem* prob, int32_t K, const double* X, saa_prec prec,
                            int want_grad, double* f, double* pbar, double* var, double* grad, void* ws,
                            size_t ws_bytes, void* stream) {
  if (!ctx) return fail(SAA_EINVAL, "ctx is NULL");
  saa_status s = check_problem(prob);
  if (s != SAA_OK) return s;
  if (K < 1 || K > 65535) return fail(SAA_EINVAL, "K must be in [1, 65535]");
  if (!X) return fail(SAA_EINVAL, "X is NULL");
  if (want_grad ? !grad : !f) return fail(SAA_EINVAL, "output pointer is NULL");
  if (!ws) return fail(SAA_EINVAL, "workspace is NULL");
  if (((uintptr_t)ws) & 255u) return fail(SAA_EINVAL, "workspace must be 256-byte aligned");
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(SAA_ECUDA, "cudaSetDevice failed");
  const int kc = tc_chunk(prob, K, prec, want_grad);
  const int Kl = kc > 0 ? kc : K;   // decisions per launch
  Plan plan;
  s = make_plan(ctx, prob, Kl, prec, want_grad, &plan);
  if (s != SAA_OK) return s;
  Workspace w;
  const size_t need = carve(prob, Kl, plan, want_grad, ws, &w);
  if (ws_bytes < need) return fail(SAA_ENOMEM, "workspace smaller than saa_workspace_size()");
  const size_t d = (size_t)prob->d;
  for (int k0 = 0; k0 < K; k0 += Kl) {
    const int n = K - k0 < Kl ? K - k0 : Kl;
    Plan pc = plan;
    if (n != Kl) {   // the last, shorter chunk: its own plan in the same workspace
      s = make_plan(ctx, prob, n, prec, want_grad, &pc);
      if (s != SAA_OK) return s;
      if (carve(prob, n, pc, want_grad, ws, &w) > ws_bytes)
        return fail(SAA_ENOMEM, "workspace smaller than the last decision chunk needs");
    }
    s = run_estimator(ctx, prob, n, X + (size_t)k0 * d, prec, want_grad, pc, w, law_args(prob), f ? f + k0 : nullptr,
                      pbar ? pbar + k0 : nullptr, var ? var + k0 : nullptr, grad ? grad + (size_t)k0 * d : nullptr,
                      (cudaStream_t)stream);
    if (s != SAA_OK) return s;
  }
  return SAA_OK;
}

saa_status saa_eval(saa_ctx* ctx, const saa_problem* prob, int32_t K, const double* X, saa_prec prec, double* f,
                    double* pbar, double* var, void* ws, size_t ws_bytes, void* stream) {
  saa::NvtxRange nvtx_range("saa_eval");
  return eval_impl(ctx, prob, K, X, prec, 0, f, pbar, var, nullptr, ws, ws_bytes, stream);
}

// Host-buffer form: [saa_eval workspace][mu][chol or sd][X][f][pbar][var] in ws.
static size_t host_io_tail(const saa_problem* p, int32_t K) {
  const size_t d = (size_t)p->d, k = (size_t)K;
  return align_up(d * 8) + align_up((p->chol ? d * d : d) * 8) + align_up(k * d * 8) + 3 * align_up(k * 8);
}

size_t saa_eval_host_workspace_size(const saa_ctx* ctx, const saa_problem* prob, int32_t K, saa_prec prec) {
  const size_t base = saa_workspace_size(ctx, prob, K, prec, 0);
  return base ? align_up(base) + host_io_tail(prob, K) : 0;
}

saa_status saa_eval_host(saa_ctx* ctx, const saa_problem* prob, int32_t K, const double* X, saa_prec prec, double* f,
                         double* pbar, double* var, void* ws, size_t ws_bytes, void* stream) {
  saa::NvtxRange nvtx_range("saa_eval_host");
  if (!ctx) return fail(SAA_EINVAL, "ctx is NULL");
  saa_status s = check_problem(prob);
  if (s != SAA_OK) return s;
  if (K < 1 || K > 65535) return fail(SAA_EINVAL, "K must be in [1, 65535]");
  if (!X || !f) return fail(SAA_EINVAL, "X and f must be host pointers");
  if (!ws || (((uintptr_t)ws) & 255u)) return fail(SAA_EINVAL, "workspace must be non-NULL and 256-byte aligned");
  const size_t need = saa_eval_host_workspace_size(ctx, prob, K, prec);
  if (need == 0) return fail(SAA_EINVAL, std::string("no workspace for these arguments: ") + g_last_error);
  if (ws_bytes < need) return fail(SAA_ENOMEM, "workspace smaller than saa_eval_host_workspace_size()");
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(SAA_ECUDA, "cudaSetDevice failed");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t d = (size_t)prob->d, k = (size_t)K;
  const size_t base = align_up(saa_workspace_size(ctx, prob, K, prec, 0));
  char* b = (char*)ws + base;
  double* mu_d = (double*)b;
  b += align_up(d * 8);
  double* cov_d = (double*)b;
  const size_t cov_n = prob->chol ? d * d : d;
  b += align_up(cov_n * 8);
  double* X_d = (double*)b;
  b += align_up(k * d * 8);
  double* f_d = (double*)b;
  double* pbar_d = (double*)(b + align_up(k * 8));
  double* var_d = (double*)(b + 2 * align_up(k * 8));
  s = cuda_status(cudaMemcpyAsync(mu_d, prob->mu, d * 8, cudaMemcpyHostToDevice, st), "copy mu to the device");
  if (s == SAA_OK)
    s = cuda_status(cudaMemcpyAsync(cov_d, prob->chol ? prob->chol : prob->sd, cov_n * 8, cudaMemcpyHostToDevice, st),
                    "copy chol (or sd) to the device");
  if (s == SAA_OK)
    s = cuda_status(cudaMemcpyAsync(X_d, X, k * d * 8, cudaMemcpyHostToDevice, st), "copy X to the device");
  if (s != SAA_OK) return s;
  saa_problem p = *prob;
  p.mu = mu_d;
  if (prob->chol)
    p.chol = cov_d;
  else
    p.sd = cov_d;
  s = eval_impl(ctx, &p, K, X_d, prec, 0, f_d, pbar ? pbar_d : nullptr, var ? var_d : nullptr, nullptr, ws, base,
                stream);
  if (s != SAA_OK) return s;
  s = cuda_status(cudaMemcpyAsync(f, f_d, k * 8, cudaMemcpyDeviceToHost, st), "copy f to the host");
  if (s == SAA_OK && pbar)
    s = cuda_status(cudaMemcpyAsync(pbar, pbar_d, k * 8, cudaMemcpyDeviceToHost, st), "copy pbar to the host");
  if (s == SAA_OK && var)
    s = cuda_status(cudaMemcpyAsync(var, var_d, k * 8, cudaMemcpyDeviceToHost, st), "copy var to the host");
  if (s != SAA_OK) return s;
  return saa_ctx_sync(ctx, stream);
}

saa_status saa_grad(saa_ctx* ctx, const saa_problem* prob, int32_t K, const double* X, saa_prec prec, double* f,
                    double* grad, void* ws, size_t ws_bytes, void* stream) {
  saa::NvtxRange nvtx_range("saa_grad");
  return eval_impl(ctx, prob, K, X, prec, 1, f, nullptr, nullptr, grad, ws, ws_bytes, stream);
}

saa_status saa_solve(saa_ctx* ctx, const saa_problem* prob, const double* w0, int32_t T, int32_t M, int64_t t0,
                     saa_prec prec, double* w_out, double* f_trace, double* gap_trace, void* ws, size_t ws_bytes,
                     void* stream) {
  saa::NvtxRange nvtx_range("saa_solve");
  if (!ctx) return fail(SAA_EINVAL, "ctx is NULL");
  saa_status s = check_problem(prob);
  if (s != SAA_OK) return s;
  if (T < 0 || M < 1 || t0 < 0) return fail(SAA_EINVAL, "need T >= 0, M >= 1, t0 >= 0");
  if (!w0 || !w_out) return fail(SAA_EINVAL, "w0 and w_out must be device pointers");
  if (!ws || (((uintptr_t)ws) & 255u)) return fail(SAA_EINVAL, "workspace must be non-NULL and 256-byte aligned");
  if ((int64_t)prob->epoch + (t0 + T) / M > 0xffffffffll) return fail(SAA_EINVAL, "resample index overflows");
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(SAA_ECUDA, "cudaSetDevice failed");
  release_fw_graphs(ctx);
  cudaGraphExec_t exec = nullptr;
  s = solve_run(ctx, prob, w0, T, M, t0, prec, w_out, f_trace, gap_trace, ws, ws_bytes, (cudaStream_t)stream, &exec);
  ctx->fw_exec = exec;  // destroyed by the next solve or by saa_ctx_destroy
  return s;
}

size_t saa_solve_adaptive_workspace_size(const saa_ctx* ctx, const saa_problem* prob, const int64_t* N_sched,
                                         int32_t n_epochs, saa_prec prec) {
  if (!ctx || !prob || !N_sched || n_epochs < 1) return 0;
  size_t most = 0;
  for (int32_t k = 0; k < n_epochs; ++k) {
    saa_problem p = *prob;
    p.N = N_sched[k];
    const size_t need = saa_workspace_size(ctx, &p, 1, prec, 2);
    if (need == 0) return 0;
    most = need > most ? need : most;
  }
  return most;
}

saa_status saa_solve_adaptive(saa_ctx* ctx, const saa_problem* prob, const double* w0, const int64_t* N_sched,
                              int32_t n_epochs, int32_t M, int32_t k0, saa_prec prec, double* w_out,
                              double* f_trace, double* gap_trace, void* ws, size_t ws_bytes, void* stream) {
  saa::NvtxRange nvtx_range("saa_solve_adaptive");
  if (!ctx) return fail(SAA_EINVAL, "ctx is NULL");
  if (!N_sched || n_epochs < 1 || M < 1 || k0 < 0) return fail(SAA_EINVAL, "need N_sched, n_epochs >= 1, M >= 1, k0 >= 0");
  if (!w0 || !w_out) return fail(SAA_EINVAL, "w0 and w_out must be device pointers");
  if (!ws || (((uintptr_t)ws) & 255u)) return fail(SAA_EINVAL, "workspace must be non-NULL and 256-byte aligned");
  if ((int64_t)prob->epoch + (int64_t)k0 + n_epochs > 0xffffffffll) return fail(SAA_EINVAL, "resample index overflows");
  for (int32_t k = 0; k < n_epochs; ++k) {
    saa_problem p = *prob;
    p.N = N_sched[k];
    saa_status s = check_problem(&p);
    if (s != SAA_OK) return s;
  }
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(SAA_ECUDA, "cudaSetDevice failed");
  release_fw_graphs(ctx);
  // one graph per run of epochs with the same N, replayed over those epochs
  int runs = 0;
  for (int32_t k = 0; k < n_epochs; ++k)
    if (k == 0 || N_sched[k] != N_sched[k - 1]) ++runs;
  ctx->fw_more = new (std::nothrow) cudaGraphExec_t[runs];
  if (!ctx->fw_more) return fail(SAA_ENOMEM, "host allocation failed");
  saa_status s = SAA_OK;
  for (int32_t k = 0; s == SAA_OK && k < n_epochs;) {
    int32_t e = k + 1;
    while (e < n_epochs && N_sched[e] == N_sched[k]) ++e;
    saa_problem p = *prob;
    p.N = N_sched[k];
    const int64_t off = (int64_t)k * M;
    cudaGraphExec_t exec = nullptr;
    s = solve_run(ctx, &p, k == 0 ? w0 : w_out, (int32_t)((e - k) * M), M, (int64_t)(k0 + k) * M, prec, w_out,
                  f_trace ? f_trace + off : nullptr, gap_trace ? gap_trace + off : nullptr, ws, ws_bytes,
                  (cudaStream_t)stream, &exec);
    if (exec) ctx->fw_more[ctx->fw_more_n++] = exec;
    k = e;
  }
  return s;
}

// The plan of a scenario range: the problem with N = n sizes the grid and
// the workspace; the kernels still see the problem's own N (LawArgs).
static saa_status partials_plan(const saa_ctx* ctx, const saa_problem* prob, int64_t n, int32_t K, saa_prec prec,
                                int want_grad, Plan* plan) {
  saa_problem pr = *prob;
  pr.N = n < 2 ? 2 : n;
  return make_plan(ctx, &pr, K, prec, want_grad ? 1 : 0, plan);
}

size_t saa_partials_workspace_size(const saa_ctx* ctx, const saa_problem* prob, int64_t n, int32_t K, saa_prec prec,
                                   int want_grad) {
  if (!ctx || check_problem(prob) != SAA_OK || !prob->chol || K < 1 || n < 1 || n > prob->N) return 0;
  DeviceGuard g(ctx->device);
  Plan plan;
  if (partials_plan(ctx, prob, n, K, prec, want_grad, &plan) != SAA_OK) return 0;
  saa_problem pr = *prob;
  pr.N = n < 2 ? 2 : n;
  return carve(&pr, K, plan, want_grad ? 1 : 0, nullptr, nullptr);
}

saa_status saa_partials(saa_ctx* ctx, const saa_problem* prob, int64_t i0, int64_t n, int32_t K, const double* X,
                        saa_prec prec, int want_grad, double* part, void* ws, size_t ws_bytes, void* stream) {
  saa::NvtxRange nvtx_range("saa_partials");
  if (!ctx) return fail(SAA_EINVAL, "ctx is NULL");
  saa_status s = check_problem(prob);
  if (s != SAA_OK) return s;
  if (!prob->chol) return fail(SAA_EUNSUPPORTED, "saa_partials needs a dense chol (the diagonal form is not split)");
  if (i0 < 0 || n < 1 || i0 + n > prob->N) return fail(SAA_EINVAL, "scenario range outside [0, N) or empty");
  if (K < 1 || K > 65535) return fail(SAA_EINVAL, "K must be in [1, 65535]");
  if (!X || !part) return fail(SAA_EINVAL, "X and part must be device pointers");
  if (!ws || (((uintptr_t)ws) & 255u)) return fail(SAA_EINVAL, "workspace must be non-NULL and 256-byte aligned");
  want_grad = want_grad ? 1 : 0;
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(SAA_ECUDA, "cudaSetDevice failed");
  Plan plan;
  s = partials_plan(ctx, prob, n, K, prec, want_grad, &plan);
  if (s != SAA_OK) return s;
  saa_problem pr = *prob;
  pr.N = n < 2 ? 2 : n;
  Workspace w;
  const size_t need = carve(&pr, K, plan, want_grad, ws, &w);
  if (ws_bytes < need) return fail(SAA_ENOMEM, "workspace smaller than saa_partials_workspace_size()");
  LawArgs la = law_args(prob);
  la.i_base = (uint32_t)i0;
  la.n = (uint32_t)n;
  cudaStream_t st = (cudaStream_t)stream;
  s = cuda_status(launch_prologue(prob, K, X, prec, w, ctx->err, st), "prologue launch");
  if (s != SAA_OK) return s;
  if (is_tc(prec) && (want_grad || plan.cluster > 0))
    s = cuda_status(launch_tc_grad(la, K, prec, plan, w, ctx->err, st, !want_grad),
                    "tensor-core gradient kernel launch");
  else if (is_tc(prec))
    s = cuda_status(launch_tc(la, K, prec, plan, w, ctx->err, st), "tensor-core kernel launch");
  else
    s = cuda_status(launch_simt(la, K, prec, want_grad, plan, w, st), "sample kernel launch");
  if (s != SAA_OK) return s;
  return cuda_status(launch_partials_out(prob, K, prec, want_grad, plan, w, part, st), "partials launch");
}

saa_status saa_partials_merge(saa_ctx* ctx, int32_t R, int64_t len, const double* parts, double* total,
                              void* stream) {
  saa::NvtxRange nvtx_range("saa_partials_merge");
  if (!ctx) return fail(SAA_EINVAL, "ctx is NULL");
  if (R < 1 || len < 1 || !parts || !total) return fail(SAA_EINVAL, "need R >= 1, len >= 1 and device arrays");
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(SAA_ECUDA, "cudaSetDevice failed");
  return cuda_status(launch_merge_partials(R, len, parts, total, (cudaStream_t)stream), "merge launch");
}

saa_status saa_finalize_partials(saa_ctx* ctx, const saa_problem* prob, int32_t K, const double* X,
                                 const double* part, double* f, double* pbar, double* var, double* grad,
                                 void* stream) {
  saa::NvtxRange nvtx_range("saa_finalize_partials");
  if (!ctx) return fail(SAA_EINVAL, "ctx is NULL");
  saa_status s = check_problem(prob);
  if (s != SAA_OK) return s;
  if (K < 1 || K > 65535) return fail(SAA_EINVAL, "K must be in [1, 65535]");
  if (!X || !part) return fail(SAA_EINVAL, "X and part must be device pointers");
  if (!f && !pbar && !var && !grad) return fail(SAA_EINVAL, "no output requested");
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(SAA_ECUDA, "cudaSetDevice failed");
  return cuda_status(launch_finalize_partials(prob->N, prob->d, K, prob->lambda, X, prob->mu, part, f, pbar, var,
                                              grad, (cudaStream_t)stream),
                     "finalize-partials launch");
}

saa_status saa_generate(saa_ctx* ctx, const saa_problem* prob, int64_t i0, int64_t n, saa_prec prec, void* z_out,
                        void* s_out, void* xi_out, void* stream) {
  saa::NvtxRange nvtx_range("saa_generate");
  if (!ctx) return fail(SAA_EINVAL, "ctx is NULL");
  saa_status s = check_problem(prob);
  if (s != SAA_OK) return s;
  if (prec != SAA_FP32 && prec != SAA_FP64) return fail(SAA_EINVAL, "saa_generate takes SAA_FP32 or SAA_FP64");
  if (i0 < 0 || n < 0 || i0 + n > prob->N) return fail(SAA_EINVAL, "scenario range outside [0, N)");
  if (!z_out) return fail(SAA_EINVAL, "z_out is NULL");
  if (xi_out && !s_out) return fail(SAA_EINVAL, "xi_out needs s_out");
  if (xi_out && !prob->chol) return fail(SAA_EUNSUPPORTED, "xi_out needs a dense chol");
  if (n == 0) return SAA_OK;
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(SAA_ECUDA, "cudaSetDevice failed");
  return cuda_status(launch_generate(law_args(prob), i0, n, prec, prob->mu, prob->chol, z_out, s_out, xi_out,
                                     (cudaStream_t)stream),
                     "generate launch");
}

const char* saa_status_string(saa_status s) {
  switch (s) {
    case SAA_OK: return "SAA_OK";
    case SAA_EINVAL: return "SAA_EINVAL: invalid argument";
    case SAA_ENOMEM: return "SAA_ENOMEM: workspace too small or allocation failed";
    case SAA_ECUDA: return "SAA_ECUDA: CUDA runtime error";
    case SAA_ETIMEOUT: return "SAA_ETIMEOUT: bounded device wait gave up";
    case SAA_EDEVICE: return "SAA_EDEVICE: device-side check failed";
    case SAA_EUNSUPPORTED: return "SAA_EUNSUPPORTED: not supported by libsaa";
  }
  return "unknown saa_status";
}

const char* saa_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
