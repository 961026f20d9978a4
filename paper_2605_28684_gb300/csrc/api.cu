// Host side of librom: the C ABI declared in include/rom.h.
//
// The context owns every device buffer. All launches go to the context's
// stream; every entry point synchronises that stream once at the end and then
// reads the device status word (4 bytes), so the only host round trip per
// call is that status. The offline stage of Algorithm 1 is:
// w_init fine FOM steps -> per-variable scaling -> POD as a rank-growing iSVD
// with forgetting factor 1 (equal to the thin SVD of the training matrix
// while its numerical rank stays within kMaxR) -> initial reduced state ->
// first coarse correction state -> sampling points.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "rom_internal.cuh"
#include "rom_kernels.cuh"

using namespace rom;

namespace {

// Null-direction test while the POD grows (new direction kept only if
// rho > tol * max(|yhat|, sigma_1); singular values <= tol * sigma_1 dropped).
// A residual rho much below 1e-13 |yhat| is set by rounding and by the basis'
// own orthonormality error, not by the data: a direction normalised from it is
// not orthogonal to the basis, and the error compounds over the updates. The
// directions it drops lie far below the final truncation at rank_tol.
constexpr double kGrowRankTol = 1e-13;

#define RCK(call)                                  \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) {                       \
      if (ctx) ctx->poisoned = 1;                  \
      return ROM_ECUDA;                            \
    }                                              \
  } while (0)

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  return cudaMalloc((void**)p, count * sizeof(T));
}

int sm_count() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

bool device_ok() {
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess) return false;
  if (cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess) return false;
  return major == 10 && minor == 3;
}

int grid_for(int64_t n) {
  int64_t g = n / 64;
  if (g < 1) g = 1;
  int s = sm_count();
  return (int)(g < s ? g : s);
}

rom_status validate(const rom_config* c) {
  if (!c) return ROM_EINVAL;
  if (c->problem != ROM_BURGERS && c->problem != ROM_EULER) return ROM_EINVAL;
  if (c->precision != ROM_FP64 && c->precision != ROM_MIXED_FP32) return ROM_EINVAL;
  if (c->problem == ROM_BURGERS && c->n_var != 1) return ROM_EINVAL;
  if (c->problem == ROM_EULER && c->n_var != 3) return ROM_EINVAL;
  // DEIM-Galerkin Euler: the explicit form only (the paper's Galerkin-FGS ROM)
  if (c->problem == ROM_EULER && c->n_s > 0 && c->time_scheme != ROM_SSPRK43) return ROM_EINVAL;
  if (c->problem == ROM_EULER && c->n_cells > 128 * 256) return ROM_EINVAL;
  if (c->n_cells < 8 || c->n_cells > (int64_t)kMaxChunks * kMaxChunkRows) return ROM_EINVAL;
  int64_t N = c->n_cells * c->n_var;
  if (c->r < 1 || c->r > kMaxR || c->r >= N || c->r > c->w_init) return ROM_EINVAL;
  if (c->n_s < 0 || (c->n_s > 0 && (c->n_s < c->r || c->n_s > 256 || c->n_s > N))) return ROM_EINVAL;
  if (c->w_init < 1 || c->z < 1 || c->newton_max < 1) return ROM_EINVAL;
  if (c->n_s > 0) {   // the DEIM step stages the stencil mesh in shared memory
    size_t need = c->problem == ROM_EULER ? euler_hyper_smem(c->n_s, c->r)
                                          : (size_t)44 * c->n_s * c->r + (size_t)c->n_s * 44 + 33500;
    if (need > 220000) return ROM_EINVAL;
  }
  if (!(c->dt > 0.0) || !(c->nu >= 0.0) || !(c->lambda >= 0.0 && c->lambda <= 1.0)) return ROM_EINVAL;
  if (!(c->newton_tol > 0.0)) return ROM_EINVAL;
  if (c->projection != ROM_GALERKIN && c->projection != ROM_LSPG) return ROM_EINVAL;
  if (c->projection == ROM_LSPG && (c->problem != ROM_BURGERS || c->precision != ROM_FP64))
    return ROM_EINVAL;
  if (c->update_rule < ROM_UPDATE_ISVD || c->update_rule > ROM_UPDATE_GROUSE) return ROM_EINVAL;
  if ((c->update_rule == ROM_UPDATE_WINDOWED_SVD || c->update_rule == ROM_UPDATE_DIRECT) &&
      (c->precision != ROM_FP64 || c->window < 1 || c->window > c->w_init || c->window > kMaxR))
    return ROM_EINVAL;
  if (c->update_rule >= ROM_UPDATE_ONESTEP &&
      (c->precision != ROM_FP64 || c->n_s != 0 || c->time_scheme != ROM_BACKWARD_EULER ||
       !(c->learning_rate >= 0.0) || !std::isfinite(c->learning_rate)))
    return ROM_EINVAL;
  if (c->time_scheme != ROM_BACKWARD_EULER && c->time_scheme != ROM_SSPRK43) return ROM_EINVAL;
  if (c->time_scheme == ROM_SSPRK43 &&
      (c->projection != ROM_GALERKIN || c->precision != ROM_FP64 || c->update_rule != ROM_UPDATE_ISVD))
    return ROM_EINVAL;
  return ROM_OK;
}

rom_status status_to_rom(int st) {
  switch (st) {
    case 0: return ROM_OK;
    case kStNoConv: return ROM_ENOCONV;
    case kStNonFinite: return ROM_ENONFINITE;
    case kStTimeout: return ROM_ETIMEOUT;
    default: return ROM_ECUDA;
  }
}

// Synchronise, read and clear the device status word.
rom_status finish(rom_ctx* ctx) {
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e == cudaSuccess && ctx->fom_overlap) e = cudaStreamSynchronize(ctx->fom_stream);
  if (e != cudaSuccess) { ctx->poisoned = 1; return ROM_ECUDA; }
  int st = 0;
  e = cudaMemcpy(&st, ctx->d.status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) { ctx->poisoned = 1; return ROM_ECUDA; }
  if (st != 0) {
    cudaMemset(ctx->d.status, 0, sizeof(int));
    cudaMemset(ctx->d.bar, 0, sizeof(GridBarrier));
    cudaMemset(ctx->d.fom_bar, 0, sizeof(GridBarrier));
    if (st == kStTimeout) ctx->poisoned = 1;
  }
  return status_to_rom(st);
}

int km_of(const rom_ctx* ctx) { return km_bucket(ctx->cfg.r + 1); }

bool mixed(const rom_ctx* ctx) { return ctx->cfg.precision == ROM_MIXED_FP32; }
float* basis32(const rom_ctx* ctx) { return mixed(ctx) ? ctx->d.phi32 : nullptr; }

// Accumulate the recorded event pairs into the per-phase totals.
cudaError_t prof_flush(rom_ctx* ctx) {
  if (ctx->prof_n == 0) return cudaSuccess;
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e == cudaSuccess && ctx->fom_overlap) e = cudaStreamSynchronize(ctx->fom_stream);
  if (e != cudaSuccess) return e;
  for (int i = 0; i < ctx->prof_n; ++i) {
    float ms = 0.f;
    e = cudaEventElapsedTime(&ms, ctx->prof_ev[2 * i], ctx->prof_ev[2 * i + 1]);
    if (e != cudaSuccess) return e;
    ctx->prof_ms[ctx->prof_phase[i]] += ms;
    ctx->prof_cnt[ctx->prof_phase[i]] += 1;
  }
  ctx->prof_n = 0;
  return cudaSuccess;
}

// Record an event before (begin) / after (end) a phase launch when enabled.
cudaError_t prof_mark(rom_ctx* ctx, int phase, bool begin, cudaStream_t on = nullptr) {
  if (!ctx->prof_on) return cudaSuccess;
  if (begin && ctx->prof_n >= kMaxProfEvents) {
    cudaError_t e = prof_flush(ctx);
    if (e != cudaSuccess) return e;
  }
  int i = ctx->prof_n;
  if (begin) ctx->prof_phase[i] = phase;
  cudaError_t e = cudaEventRecord(ctx->prof_ev[2 * i + (begin ? 0 : 1)], on ? on : ctx->stream);
  if (!begin) ctx->prof_n += 1;
  return e;
}

FomParams fom_params(const rom_ctx* ctx, double h) {
  FomParams p;
  p.problem = ctx->cfg.problem;
  p.n_cells = ctx->cfg.n_cells;
  p.nu = ctx->cfg.nu;
  p.gamma = ctx->cfg.gamma;
  p.h = h;
  p.tol = ctx->cfg.newton_tol;
  p.max_iter = ctx->cfg.newton_max;
  return p;
}

FomScratch fom_scratch(const rom_ctx* ctx) {
  FomScratch s;
  s.chunk = ctx->d.fom_chunk;
  s.maxbuf = ctx->d.maxbuf;
  s.bar = ctx->d.fom_bar;
  s.status = ctx->d.status;
  s.iters = ctx->d.iters_fom;
  return s;
}

cudaError_t fom_step(rom_ctx* ctx, const double* q_prev, double* q, double h) {
  cudaError_t e = cudaMemsetAsync(ctx->d.maxbuf, 0, 4 * sizeof(unsigned long long), ctx->stream);
  if (e != cudaSuccess) return e;
  return launch_fom_step(fom_params(ctx, h), q_prev, q, fom_scratch(ctx), ctx->stream);
}

// The feature-guided candidates of a new correction snapshot y (hyper-reduced
// models only), on stream s (the stream that produced y).
cudaError_t select_features(rom_ctx* ctx, const double* y, cudaStream_t s, bool stage = true) {
  if (ctx->cfg.n_s <= 0) return cudaSuccess;
  cudaError_t e = prof_mark(ctx, 4, true, s);
  if (e == cudaSuccess)
    e = launch_fgs(y, ctx->N, ctx->cfg.n_var, ctx->cfg.gamma, fgs_list_length(ctx->N, ctx->cfg.r, ctx->cfg.n_s),
                   ctx->d.fgs_key, ctx->d.fgs_v, ctx->d.fgs_i, stage, s);
  if (e == cudaSuccess) e = prof_mark(ctx, 4, false, s);
  return e;
}

// The context's stream waits for a feature-guided selection still running
// on the coarse-FOM stream (see coarse_fom_fork).
cudaError_t wait_features(rom_ctx* ctx) {
  if (!ctx->fgs_pending) return cudaSuccess;
  ctx->fgs_pending = 0;
  return cudaStreamWaitEvent(ctx->stream, ctx->ev_fgs, 0);
}

EventArgs event_args(rom_ctx* ctx, const double* y, int preprocess, double lambda, double rank_tol,
                     int r_cap, int transfer, bool online = true) {
  EventArgs A;
  A.n = ctx->N;
  A.ld = ctx->N;
  A.r = r_cap;
  A.rank = ctx->d.rank;
  A.lambda = lambda;
  A.rank_tol = rank_tol;
  A.phi = ctx->d.phi;
  A.phi32 = online ? basis32(ctx) : nullptr;   // the offline POD runs in FP64
  A.gram = ctx->d.gram;
  A.sigma = ctx->d.sigma;
  A.a = transfer ? ctx->d.a : nullptr;
  A.transfer = transfer;
  A.y = y;
  A.q_ref = ctx->d.q_ref;
  A.drow = ctx->d.drow;
  A.preprocess = preprocess;
  A.yhat = ctx->d.yhat;
  A.qres = ctx->d.qres;
  A.partials = ctx->d.partials;
  A.core = ctx->d.core;
  A.ubar = ctx->d.ubar;
  A.rec = nullptr;
  A.bar = ctx->d.bar;
  A.status = ctx->d.status;
  return A;
}

SampleArgs sample_args(rom_ctx* ctx) {
  SampleArgs S;
  S.n = ctx->N;
  S.ld = ctx->N;
  S.r = ctx->cfg.r;
  S.n_s = ctx->cfg.n_s;
  S.n_var = ctx->cfg.n_var;
  S.rank = ctx->d.rank;
  S.phi = ctx->d.phi;
  S.phi32 = basis32(ctx);
  S.q_ref = ctx->d.q_ref;
  S.drow = ctx->d.drow;
  S.fgs_i = ctx->d.fgs_i;
  S.fgs_t = fgs_list_length(ctx->N, ctx->cfg.r, ctx->cfg.n_s);
  S.samples = ctx->d.samples;
  S.cand_v = ctx->d.cand_v;
  S.cand_f = ctx->d.cand_f;
  // every launch takes kMaxR fresh epochs (one per QDEIM step), so a word
  // left by an earlier launch never matches
  ctx->sample_epoch += (unsigned int)kMaxR;
  S.epoch = ctx->sample_epoch;
  S.qd_u = ctx->d.qd_u;
  S.mesh = ctx->d.mesh;
  S.minv = ctx->d.minv;
  S.bar = ctx->d.bar;
  S.status = ctx->d.status;
  return S;
}

StepArgs step_args(rom_ctx* ctx, int nsteps) {
  StepArgs A;
  A.n = ctx->N;
  A.ld = ctx->N;
  A.r = ctx->cfg.r;
  A.rank = ctx->d.rank;
  A.phi = ctx->d.phi;
  A.phi32 = basis32(ctx);
  A.q_ref = ctx->d.q_ref;
  A.drow = ctx->d.drow;
  A.dinv = ctx->d.dinv;
  A.a = ctx->d.a;
  A.nu = ctx->cfg.nu;
  A.gamma = ctx->cfg.gamma;
  A.dt = ctx->cfg.dt;
  A.tol = ctx->cfg.newton_tol;
  A.max_iter = ctx->cfg.newton_max;
  A.nsteps = nsteps;
  A.explicit_rk = ctx->cfg.time_scheme == ROM_SSPRK43 ? 1 : 0;
  A.partials = ctx->d.partials;
  A.jpartials = ctx->d.jpartials;
  A.jac = ctx->d.jac;
  A.n_s = ctx->cfg.n_s;
  A.samples = ctx->d.samples;
  A.mesh = ctx->d.mesh;
  A.minv = ctx->d.minv;
  A.npart = ctx->d.npart;
  A.bar = ctx->d.bar;
  A.status = ctx->d.status;
  A.iters = ctx->d.iters_rom;
  return A;
}

cudaError_t run_steps(rom_ctx* ctx, int nsteps) {
  StepArgs A = step_args(ctx, nsteps);
  cudaError_t e = prof_mark(ctx, 0, true);
  if (e != cudaSuccess) return e;
  if (ctx->cfg.n_s > 0 && ctx->cfg.problem == ROM_EULER) e = launch_euler_hyper_steps(A, ctx->stream);
  else if (ctx->cfg.n_s > 0) e = launch_hyper_steps(A, km_of(ctx), ctx->stream);
  else if (ctx->cfg.projection == ROM_LSPG) e = launch_lspg_steps(A, ctx->grid, ctx->stream);
  else if (ctx->cfg.problem == ROM_EULER) e = launch_euler_galerkin_steps(A, km_of(ctx), ctx->grid, ctx->stream);
  else e = launch_galerkin_steps(A, km_of(ctx), ctx->grid, ctx->stream);
  if (e != cudaSuccess) return e;
  return prof_mark(ctx, 0, false);
}

cudaError_t run_event_window(rom_ctx* ctx);

// The adaptation event of Algorithm 1 on the current y_corr.
cudaError_t run_event_instant(rom_ctx* ctx);
bool instant_rule(const rom_ctx* ctx) { return ctx->cfg.update_rule >= ROM_UPDATE_ONESTEP; }

cudaError_t run_event(rom_ctx* ctx) {
  if (instant_rule(ctx)) return run_event_instant(ctx);
  if (ctx->cfg.update_rule != ROM_UPDATE_ISVD) return run_event_window(ctx);
  EventArgs A = event_args(ctx, ctx->d.y_corr, 1, ctx->cfg.lambda, ctx->cfg.rank_tol, ctx->cfg.r, 1);
  cudaError_t e = prof_mark(ctx, 2, true);
  if (e == cudaSuccess) e = launch_event(A, km_of(ctx), ctx->grid, ctx->stream);
  if (e == cudaSuccess) e = prof_mark(ctx, 2, false);
  if (e != cudaSuccess) return e;
  if (ctx->cfg.n_s > 0) {
    e = wait_features(ctx);
    if (e == cudaSuccess) e = prof_mark(ctx, 3, true);
    if (e == cudaSuccess) e = launch_sampling(sample_args(ctx), km_of(ctx), ctx->grid, ctx->stream);
    if (e == cudaSuccess) e = prof_mark(ctx, 3, false);
  }
  return e;
}

// The comparison update rules (App. A) on the snapshot window: the lifted
// state is formed with the old basis, the new preprocessed snapshot replaces
// the oldest one in the window, the basis is rebuilt from an empty one by the
// rank-growing iSVD (forgetting factor 1) over the window (windowed SVD) or
// over the columns of Y V_c (Direct, V_c from the Jacobi SVD of Phi^T Y), and
// the state is transferred by projection, a = Phi_new^T D (q~ - q_ref).
cudaError_t run_event_window(rom_ctx* ctx) {
  const int64_t N = ctx->N;
  const int r = ctx->cfg.r, nw = ctx->cfg.window, G = ctx->grid;
  const int r_grow = ctx->cfg.w_init < kMaxR ? ctx->cfg.w_init : kMaxR;
  const int r_alloc = r_grow > r ? r_grow : r;
  cudaStream_t s = ctx->stream;
  DevState& d = ctx->d;
  cudaError_t e = prof_mark(ctx, 2, true);
  if (e != cudaSuccess) return e;
  LiftArgs L;
  L.n = N; L.ld = N; L.rank = d.rank; L.phi = d.phi; L.phi32 = nullptr; L.q_ref = d.q_ref;
  L.drow = d.drow; L.dinv = d.dinv; L.a = d.a; L.out = d.lifted;
  if ((e = launch_lift(L, km_of(ctx), s)) != cudaSuccess) return e;
  const int slot = ctx->win_head;
  e = launch_win_fill(d.y_corr, N, d.q_ref, d.drow, N, 1, d.win + (size_t)slot * N, s);
  if (e != cudaSuccess) return e;
  ctx->win_head = (slot + 1) % nw;
  double* C = d.dsm;
  double* Vc = d.dsm + kMaxR * kMaxR;
  double* sv = Vc + kMaxR * kMaxR;
  int* kc = reinterpret_cast<int*>(sv + kMaxR);
  int nfeed = nw, r_cap = nw < kMaxR ? nw : kMaxR;
  const bool direct = ctx->cfg.update_rule == ROM_UPDATE_DIRECT;
  if (direct) {
    if ((e = launch_tn(TnArgs{N, r, nw, d.phi, N, d.win, N, 1.0, d.dpart, C}, G, s)) != cudaSuccess) return e;
    if ((e = launch_direct_small(C, r, nw, d.rank, ctx->cfg.rank_tol, Vc, sv, kc, s)) != cudaSuccess) return e;
    int hkc = 0;
    if ((e = cudaMemcpyAsync(&hkc, kc, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    if (hkc < 1) return cudaErrorInvalidValue;
    e = launch_nn(NnArgs{N, nw, hkc, d.win, N, Vc, hkc, 1, 1.0, 0.0, d.dwork, N, d.dwork, N}, s);
    if (e != cudaSuccess) return e;
    nfeed = hkc;
    r_cap = hkc;
  }
  if ((e = cudaMemsetAsync(d.phi, 0, sizeof(double) * N * r_alloc, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(d.sigma, 0, sizeof(double) * (kMaxR + 1), s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(d.rank, 0, sizeof(int), s)) != cudaSuccess) return e;
  for (int j = 0; j < nfeed; ++j) {
    const double* col = direct ? d.dwork + (size_t)j * N : d.win + (size_t)((ctx->win_head + j) % nw) * N;
    EventArgs A = event_args(ctx, col, 0, 1.0, kGrowRankTol, r_cap, 0, false);
    if ((e = launch_event(A, km_bucket(r_cap + 1), G, s)) != cudaSuccess) return e;
  }
  if (direct) e = launch_set_sigma(sv, kc, d.sigma, d.rank, s);
  else e = launch_truncate(d.phi, N, d.sigma, d.rank, r, r_alloc, ctx->cfg.rank_tol, s);
  if (e != cudaSuccess) return e;
  ProjectArgs P;
  P.n = N; P.ld = N; P.r = r; P.rank = d.rank; P.phi = d.phi; P.phi32 = nullptr; P.v = d.lifted;
  P.q_ref = d.q_ref; P.drow = d.drow; P.a = d.a; P.partials = d.partials; P.bar = d.bar; P.status = d.status;
  if ((e = launch_project(P, km_of(ctx), G, s)) != cudaSuccess) return e;
  if ((e = prof_mark(ctx, 2, false)) != cudaSuccess) return e;
  if (ctx->cfg.n_s > 0) {
    e = wait_features(ctx);
    if (e == cudaSuccess) e = prof_mark(ctx, 3, true);
    if (e == cudaSuccess) e = launch_sampling(sample_args(ctx), km_of(ctx), G, s);
    if (e == cudaSuccess) e = prof_mark(ctx, 3, false);
  }
  return e;
}

// The instantaneous rules of App. A (one-step, Oja, GROUSE) on the live
// columns: the lifted state with the old basis, yhat = D (y_corr - q_ref)
// (the snapshot held, approximating the current time level), the products
// the rule needs (Phi^T yhat; for GROUSE the residual r by Gram-Schmidt twice
// and |r|^2), the rank-one update Phi += u v^T, CholQR twice for one-step and
// Oja, and the state transfer a = Phi_new^T D (q~ - q_ref). The caller
// advances the coarse FOM after this. The host reads the rank for the launch
// sizes (one synchronisation per event).
cudaError_t run_event_instant(rom_ctx* ctx) {
  const int64_t N = ctx->N;
  const int r = ctx->cfg.r, G = ctx->grid, rule = ctx->cfg.update_rule;
  cudaStream_t s = ctx->stream;
  DevState& d = ctx->d;
  cudaError_t e = prof_mark(ctx, 2, true);
  if (e != cudaSuccess) return e;
  int k = 0;
  if ((e = cudaMemcpyAsync(&k, d.rank, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  if (k > r) k = r;
  LiftArgs L;
  L.n = N; L.ld = N; L.rank = d.rank; L.phi = d.phi; L.phi32 = nullptr; L.q_ref = d.q_ref;
  L.drow = d.drow; L.dinv = d.dinv; L.a = d.a; L.out = d.lifted;
  if ((e = launch_lift(L, km_of(ctx), s)) != cudaSuccess) return e;
  if (k > 0) {
    double* Gm = d.dsm;                          // k x k Gram (ld k)
    double* Rinv = d.dsm + kMaxR * kMaxR;        // k x k (ld kMaxR)
    double* w1 = Rinv + kMaxR * kMaxR;
    double* w2 = w1 + kMaxR;
    double* g = w2 + kMaxR;
    double* v = g + kMaxR;
    double* coef = v + kMaxR;                    // c_y, c_r, |r|^2
    double* rr = coef + 2;
    if ((e = launch_win_fill(d.y_corr, N, d.q_ref, d.drow, N, 1, d.yhat, s)) != cudaSuccess) return e;
    if ((e = launch_tn(TnArgs{N, k, 1, d.phi, N, d.yhat, N, 1.0, d.dpart, w1}, G, s)) != cudaSuccess) return e;
    if (rule == ROM_UPDATE_GROUSE) {
      e = launch_nn(NnArgs{N, k, 1, d.phi, N, w1, 1, 1, -1.0, 1.0, d.yhat, N, d.qres, N}, s);
      if (e == cudaSuccess) e = launch_tn(TnArgs{N, k, 1, d.phi, N, d.qres, N, 1.0, d.dpart, w2}, G, s);
      if (e == cudaSuccess) e = launch_nn(NnArgs{N, k, 1, d.phi, N, w2, 1, 1, -1.0, 1.0, d.qres, N, d.qres, N}, s);
      if (e == cudaSuccess) e = launch_tn(TnArgs{N, 1, 1, d.qres, N, d.qres, N, 1.0, d.dpart, rr}, G, s);
    } else {
      e = cudaMemsetAsync(w2, 0, sizeof(double) * (kMaxR + 8 + 3 * kMaxR), s);
    }
    if (e != cudaSuccess) return e;
    e = launch_instant_coef(rule, d.rank, r, ctx->cfg.learning_rate, w1, w2, d.a, rr, coef, g, v, s);
    if (e == cudaSuccess) e = launch_rank1_update(d.phi, N, d.rank, r, d.yhat, d.qres, coef, g, v, s);
    for (int pass = 0; e == cudaSuccess && rule != ROM_UPDATE_GROUSE && pass < 2; ++pass) {
      e = launch_tn(TnArgs{N, k, k, d.phi, N, d.phi, N, 1.0, d.dpart, Gm}, G, s);
      if (e == cudaSuccess) e = launch_chol_inv(Gm, d.rank, r, Rinv, s);
      if (e == cudaSuccess)
        e = launch_nn(NnArgs{N, k, k, d.phi, N, Rinv, kMaxR, 1, 1.0, 0.0, d.dwork, N, d.dwork, N}, s);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(d.phi, d.dwork, sizeof(double) * N * k, cudaMemcpyDeviceToDevice, s);
    }
    if (e != cudaSuccess) return e;
  }
  ProjectArgs P;
  P.n = N; P.ld = N; P.r = r; P.rank = d.rank; P.phi = d.phi; P.phi32 = nullptr; P.v = d.lifted;
  P.q_ref = d.q_ref; P.drow = d.drow; P.a = d.a; P.partials = d.partials; P.bar = d.bar; P.status = d.status;
  if ((e = launch_project(P, km_of(ctx), G, s)) != cudaSuccess) return e;
  return prof_mark(ctx, 2, false);
}

// The coarse FOM step of a cycle on fom_stream, after everything queued on
// the context's stream so far; coarse_fom_join makes the stream wait for it
// and takes the new snapshot. The reduced steps queued in between run beside
// it: they read neither y_corr nor y_tmp, and the FOM kernel has its own
// grid barrier and scratch.
cudaError_t coarse_fom_fork(rom_ctx* ctx) {
  cudaStream_t fs = ctx->fom_stream;
  cudaError_t e = cudaEventRecord(ctx->ev_fork, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(fs, ctx->ev_fork, 0);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d.maxbuf, 0, 4 * sizeof(unsigned long long), fs);
  if (e == cudaSuccess) e = prof_mark(ctx, 1, true, fs);
  if (e == cudaSuccess)
    e = launch_fom_step(fom_params(ctx, ctx->cfg.z * ctx->cfg.dt), ctx->d.y_corr, ctx->d.y_tmp,
                        fom_scratch(ctx), fs);
  if (e == cudaSuccess) e = prof_mark(ctx, 1, false, fs);
  if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_join, fs);
  // the feature-guided selection of the new snapshot runs on, beside the
  // iSVD update (which needs only the snapshot); the sampling launch waits
  // for it. Its keys are read from global memory, so that its one CTA fits
  // beside a CTA of the cooperative update on the same SM
  if (e == cudaSuccess) e = select_features(ctx, ctx->d.y_tmp, fs, false);
  if (e == cudaSuccess && ctx->cfg.n_s > 0) {
    e = cudaEventRecord(ctx->ev_fgs, fs);
    ctx->fgs_pending = 1;
  }
  return e;
}

cudaError_t coarse_fom_join(rom_ctx* ctx) {
  cudaError_t e = cudaStreamWaitEvent(ctx->stream, ctx->ev_join, 0);
  if (e != cudaSuccess) return e;
  double* t = ctx->d.y_corr;
  ctx->d.y_corr = ctx->d.y_tmp;
  ctx->d.y_tmp = t;
  return cudaSuccess;
}

cudaError_t coarse_fom(rom_ctx* ctx) {
  cudaError_t e = cudaMemsetAsync(ctx->d.maxbuf, 0, 4 * sizeof(unsigned long long), ctx->stream);
  if (e == cudaSuccess) e = prof_mark(ctx, 1, true);
  if (e == cudaSuccess)
    e = launch_fom_step(fom_params(ctx, ctx->cfg.z * ctx->cfg.dt), ctx->d.y_corr, ctx->d.y_tmp,
                        fom_scratch(ctx), ctx->stream);
  if (e == cudaSuccess) e = prof_mark(ctx, 1, false);
  if (e == cudaSuccess) e = select_features(ctx, ctx->d.y_tmp, ctx->stream);
  if (e != cudaSuccess) return e;
  double* t = ctx->d.y_corr;
  ctx->d.y_corr = ctx->d.y_tmp;
  ctx->d.y_tmp = t;
  return cudaSuccess;
}

// per-variable mean square of the centred training data -> drow
__global__ void scale_partial_kernel(const double* Q, const double* q_ref, int64_t N, int w,
                                     int64_t n_cells, int n_var, double* partial) {
  __shared__ double red[32];
  for (int v = 0; v < n_var; ++v) {
    double s = 0.0;
    int64_t tot = n_cells * (int64_t)w;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
         e += (int64_t)gridDim.x * blockDim.x) {
      int64_t col = e / n_cells, cell = e % n_cells;
      int64_t i = v * n_cells + cell;
      double x = Q[col * N + i] - q_ref[i];
      s = fma(x, x, s);
    }
    s = block_sum(s, red);
    if (threadIdx.x == 0) partial[blockIdx.x * n_var + v] = s;
  }
}

__global__ void scale_final_kernel(const double* partial, int nb, int64_t n_cells, int n_var, int w,
                                   double* dvals) {
  if (threadIdx.x < n_var) {
    int v = threadIdx.x;
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += partial[b * n_var + v];
    double phi = s / ((double)n_cells * (double)w);
    if (phi < 1e-300) phi = 1.0;
    dvals[v] = 1.0 / phi;
  }
}

__global__ void to_fp32_kernel(const double* in, float* out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

__global__ void drow_kernel(const double* dvals, int64_t n_cells, int64_t N, double* drow,
                            double* dinv) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    drow[i] = dvals[i / n_cells];
    dinv[i] = 1.0 / dvals[i / n_cells];
  }
}

// true if every one of the n host values is finite
bool all_finite(const double* v, int64_t n) {
  for (int64_t i = 0; i < n; ++i)
    if (!std::isfinite(v[i])) return false;
  return true;
}

void free_state(rom_ctx* ctx) {
  DevState& d = ctx->d;
  void* ptrs[] = {d.q_ref, d.y_corr, d.y_tmp, d.yhat, d.qres, d.lifted, d.dvals, d.drow, d.dinv, d.phi,
                  d.phi32, d.gram, d.sigma, d.a, d.a_prev, d.rank, d.core, d.ubar, d.partials,
                  d.jpartials, d.jac, d.samples, d.qd_u, d.cand_v,
                  d.cand_f, d.fgs_key, d.fgs_v, d.fgs_i, d.mesh, d.minv, d.bar, d.fom_bar, d.status, d.iters_rom, d.iters_fom, d.maxbuf,
                  d.fom_chunk, d.npart, d.win, d.dwork, d.dsm, d.dpart, ctx->q_train};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  memset(&ctx->d, 0, sizeof(DevState));
  ctx->q_train = nullptr;
}

}  // namespace

extern "C" {

const char* rom_status_string(rom_status s) {
  switch (s) {
    case ROM_OK: return "ok";
    case ROM_EINVAL: return "invalid argument";
    case ROM_ENOMEM: return "device allocation failed";
    case ROM_ECUDA: return "CUDA error";
    case ROM_ENOCONV: return "Newton iteration did not converge";
    case ROM_ENONFINITE: return "non-finite value in the state";
    case ROM_ETIMEOUT: return "device-side wait timed out";
    case ROM_ESTATE: return "context poisoned by an earlier error";
  }
  return "unknown status";
}

void rom_destroy(rom_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  if (ctx->fom_overlap) {
    cudaStreamSynchronize(ctx->fom_stream);
    cudaStreamDestroy(ctx->fom_stream);
    cudaEventDestroy(ctx->ev_fork);
    cudaEventDestroy(ctx->ev_join);
    cudaEventDestroy(ctx->ev_fgs);
    ctx->fom_overlap = 0;
  }
  if (ctx->prof_ev_made)
    for (int i = 0; i < 2 * kMaxProfEvents; ++i) cudaEventDestroy(ctx->prof_ev[i]);
  free_state(ctx);
  delete ctx;
}

}  // extern "C"

namespace {

// rom_init; keep_train keeps the training matrix (N x w_init) on the device
// and computes the POD as a backward-stable thin SVD (pod_svd.cu) instead of
// the rank-growing iSVD, for the gradient pass, whose POD adjoint needs the
// basis fixed to rounding level.
rom_status init_ctx(const rom_config* cfg_in, const double* q0_host, void* stream, bool keep_train,
                    rom_ctx** out) {
  if (!out) return ROM_EINVAL;
  *out = nullptr;
  rom_status vs = validate(cfg_in);
  if (vs != ROM_OK) return vs;
  if (!q0_host) return ROM_EINVAL;
  if (!all_finite(q0_host, cfg_in->n_cells * cfg_in->n_var)) return ROM_ENONFINITE;
  if (!device_ok()) return ROM_ECUDA;
  rom_ctx* ctx = new rom_ctx;
  memset(&ctx->d, 0, sizeof(DevState));
  ctx->fom_overlap = 0;
  ctx->fgs_pending = 0;
  ctx->sample_epoch = 0u;
  ctx->q_train = nullptr;
  ctx->prof_on = 0;
  ctx->prof_n = 0;
  ctx->prof_ev_made = 0;
  for (int p = 0; p < kPhases; ++p) { ctx->prof_ms[p] = 0.0; ctx->prof_cnt[p] = 0; }
  ctx->cfg = *cfg_in;
  // numerical-rank tolerance: what the working precision of the projections
  // can resolve (FP64: 1e-10; FP32 projections of the mixed form: 1e-5)
  if (!(ctx->cfg.rank_tol > 0.0))
    ctx->cfg.rank_tol = (ctx->cfg.precision == ROM_MIXED_FP32) ? 1e-5 : 1e-10;
  ctx->stream = (cudaStream_t)stream;
  ctx->N = ctx->cfg.n_cells * ctx->cfg.n_var;
  ctx->step = 0;
  ctx->poisoned = 0;
  ctx->win_head = 0;
  ctx->grid = grid_for(ctx->N);
  if (ctx->cfg.n_s > 0) {
    // the DEIM steps are one CTA without a grid barrier, so the coarse FOM
    // step can run beside them on its own stream
    if (cudaStreamCreateWithFlags(&ctx->fom_stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      delete ctx;
      return ROM_ECUDA;
    }
    if (cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      cudaStreamDestroy(ctx->fom_stream);
      delete ctx;
      return ROM_ECUDA;
    }
    if (cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      cudaEventDestroy(ctx->ev_fork);
      cudaStreamDestroy(ctx->fom_stream);
      delete ctx;
      return ROM_ECUDA;
    }
    if (cudaEventCreateWithFlags(&ctx->ev_fgs, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      cudaEventDestroy(ctx->ev_join);
      cudaEventDestroy(ctx->ev_fork);
      cudaStreamDestroy(ctx->fom_stream);
      delete ctx;
      return ROM_ECUDA;
    }
    ctx->fom_overlap = 1;
  }
  const int64_t N = ctx->N;
  const int r = ctx->cfg.r;
  const int w = ctx->cfg.w_init;
  const int r_grow = w < kMaxR ? w : kMaxR;
  const int r_alloc = r_grow > r ? r_grow : r;
  const int G = ctx->grid;
  const int ns = ctx->cfg.n_s > 0 ? ctx->cfg.n_s : 1;
  DevState& d = ctx->d;
  cudaError_t e = cudaSuccess;
#define ALLOC(p, n) \
  if (e == cudaSuccess) e = dalloc(&(p), (size_t)(n))
  ALLOC(d.q_ref, N); ALLOC(d.y_corr, N); ALLOC(d.y_tmp, N); ALLOC(d.yhat, N); ALLOC(d.qres, N);
  ALLOC(d.lifted, N); ALLOC(d.dvals, 4); ALLOC(d.drow, N); ALLOC(d.dinv, N); ALLOC(d.phi, (size_t)N * r_alloc);
  ALLOC(d.sigma, kMaxR + 1); ALLOC(d.a, kMaxR + 1); ALLOC(d.a_prev, kMaxR + 1); ALLOC(d.rank, 1);
  ALLOC(d.core, core_ws_doubles()); ALLOC(d.ubar, kMaxCore * kMaxCore);
  ALLOC(d.partials, (size_t)3 * G * (kMaxCore + 2)); ALLOC(d.jpartials, (size_t)G * kMaxR * kMaxR);
  ALLOC(d.jac, kMaxR * kMaxR); ALLOC(d.samples, ns); ALLOC(d.cand_v, (size_t)G * kMaxNs);
  ALLOC(d.cand_f, (size_t)G * 2); ALLOC(d.mesh, (size_t)ns * 3 * ctx->cfg.n_var * kMeshStride);
  if (ctx->cfg.n_s > 0) {
    ALLOC(d.qd_u, (size_t)N * r); ALLOC(d.fgs_key, N);
    ALLOC(d.fgs_v, 2 * kMaxNs); ALLOC(d.fgs_i, 2 * kMaxNs);
  }
  ALLOC(d.minv, (size_t)kMaxR * ns); ALLOC(d.bar, 1); ALLOC(d.fom_bar, 1); ALLOC(d.status, 1); ALLOC(d.iters_rom, 1);
  ALLOC(d.iters_fom, 1); ALLOC(d.maxbuf, 4); ALLOC(d.fom_chunk, fom_chunk_floats());
  ALLOC(ctx->q_train, (size_t)N * w);
  if (ctx->cfg.precision == ROM_MIXED_FP32) {
    ALLOC(d.phi32, (size_t)N * r);
    ALLOC(d.gram, (size_t)G * kMaxR * kMaxR);
  }
  if (ctx->cfg.projection == ROM_LSPG) ALLOC(d.npart, lspg_partial_doubles(G));
  if (ctx->cfg.update_rule != ROM_UPDATE_ISVD) {
    ALLOC(d.win, (size_t)N * ctx->cfg.window);
    ALLOC(d.dwork, (size_t)N * kMaxR);
    ALLOC(d.dsm, 2 * kMaxR * kMaxR + 6 * kMaxR + 16);
    ALLOC(d.dpart, (size_t)G * kMaxR * kMaxR);
  }
#undef ALLOC
  if (e != cudaSuccess) {
    cudaGetLastError();
    free_state(ctx);
    delete ctx;
    return ROM_ENOMEM;
  }
  cudaStream_t s = ctx->stream;
  RCK(cudaMemsetAsync(d.bar, 0, sizeof(GridBarrier), s));
  RCK(cudaMemsetAsync(d.fom_bar, 0, sizeof(GridBarrier), s));
  RCK(cudaMemsetAsync(d.cand_f, 0, sizeof(unsigned long long) * G * 2, s));
  RCK(cudaMemsetAsync(d.status, 0, sizeof(int), s));
  RCK(cudaMemsetAsync(d.phi, 0, sizeof(double) * N * r_alloc, s));
  RCK(cudaMemsetAsync(d.sigma, 0, sizeof(double) * (kMaxR + 1), s));
  RCK(cudaMemsetAsync(d.a, 0, sizeof(double) * (kMaxR + 1), s));
  RCK(cudaMemsetAsync(d.rank, 0, sizeof(int), s));
  RCK(cudaMemcpyAsync(d.y_tmp, q0_host, sizeof(double) * N, cudaMemcpyHostToDevice, s));
  RCK(cudaMemcpyAsync(d.q_ref, d.y_tmp, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
  // training window: w_init fine FOM steps (backward Euler, or SSPRK(4,3) in
  // the explicit form with yhat, qres and lifted as its stage scratch)
  const double* prev = d.y_tmp;
  for (int j = 0; j < w; ++j) {
    double* cur = ctx->q_train + (size_t)j * N;
    if (ctx->cfg.time_scheme == ROM_SSPRK43)
      RCK(launch_fom_explicit_step(fom_params(ctx, ctx->cfg.dt), ctx->cfg.n_var, prev, cur, d.yhat, d.qres,
                                   d.lifted, s));
    else
      RCK(fom_step(ctx, prev, cur, ctx->cfg.dt));
    prev = cur;
  }
  rom_status st = finish(ctx);
  if (st != ROM_OK) { rom_destroy(ctx); return st; }
  // scaling D
  {
    int nb = 256;   // partial sums go to cand_v (grid * kMaxNs >= nb * n_var doubles)
    scale_partial_kernel<<<nb, 256, 0, s>>>(ctx->q_train, d.q_ref, N, w, ctx->cfg.n_cells,
                                            ctx->cfg.n_var, d.cand_v);
    RCK(cudaGetLastError());
    scale_final_kernel<<<1, 32, 0, s>>>(d.cand_v, nb, ctx->cfg.n_cells, ctx->cfg.n_var, w, d.dvals);
    RCK(cudaGetLastError());
    drow_kernel<<<256, 256, 0, s>>>(d.dvals, ctx->cfg.n_cells, N, d.drow, d.dinv);
    RCK(cudaGetLastError());
  }
  // POD for the gradient pass: thin SVD of D (Q_train - q_ref 1^T) by CGS2 QR and Jacobi
  if (keep_train) {
    double *X = nullptr, *Qm = nullptr, *Rm = nullptr, *Um = nullptr, *sv = nullptr, *wk = nullptr,
           *pt = nullptr;
    cudaError_t ae = dalloc(&X, (size_t)N * w);
    if (ae == cudaSuccess) ae = dalloc(&Qm, (size_t)N * w);
    if (ae == cudaSuccess) ae = dalloc(&Rm, (size_t)w * w);
    if (ae == cudaSuccess) ae = dalloc(&Um, (size_t)w * w);
    if (ae == cudaSuccess) ae = dalloc(&sv, (size_t)w);
    if (ae == cudaSuccess) ae = dalloc(&wk, 256);
    if (ae == cudaSuccess) ae = dalloc(&pt, (size_t)G * 16384);
    auto release = [&]() { cudaFree(X); cudaFree(Qm); cudaFree(Rm); cudaFree(Um); cudaFree(sv); cudaFree(wk); cudaFree(pt); };
    if (ae != cudaSuccess) { cudaGetLastError(); release(); rom_destroy(ctx); return ROM_ENOMEM; }
    ae = launch_win_fill(ctx->q_train, N, d.q_ref, d.drow, N, w, X, s);
    if (ae == cudaSuccess) ae = pod_thin_svd(X, N, w, Qm, Rm, Um, sv, wk, pt, G, s);
    std::vector<double> sg(w);
    if (ae == cudaSuccess) ae = cudaMemcpyAsync(sg.data(), sv, sizeof(double) * w, cudaMemcpyDeviceToHost, s);
    if (ae == cudaSuccess) ae = cudaStreamSynchronize(s);
    int k = 0;
    for (int j = 0; j < r && j < w; ++j)
      if (sg[0] > 0.0 && sg[j] > ctx->cfg.rank_tol * sg[0]) ++k;
    if (ae == cudaSuccess) ae = cudaMemsetAsync(d.phi, 0, sizeof(double) * N * r_alloc, s);
    if (ae == cudaSuccess) ae = cudaMemsetAsync(d.sigma, 0, sizeof(double) * (kMaxR + 1), s);
    if (ae == cudaSuccess && k > 0)
      ae = launch_nn(NnArgs{N, w, k, Qm, N, Um, w, 1, 1.0, 0.0, d.phi, N, d.phi, N}, s);
    if (ae == cudaSuccess && k > 0)
      ae = cudaMemcpyAsync(d.sigma, sv, sizeof(double) * k, cudaMemcpyDeviceToDevice, s);
    if (ae == cudaSuccess) ae = cudaMemcpyAsync(d.rank, &k, sizeof(int), cudaMemcpyHostToDevice, s);
    if (ae == cudaSuccess) ae = cudaStreamSynchronize(s);
    release();
    if (ae != cudaSuccess) { ctx->poisoned = 1; rom_destroy(ctx); return ROM_ECUDA; }
  } else {
    // POD: rank-growing iSVD of D (Q_train - q_ref 1^T), forgetting factor 1
    const int km = km_bucket(r_grow + 1);
    for (int j = 0; j < w; ++j) {
      EventArgs A = event_args(ctx, ctx->q_train + (size_t)j * N, 1, 1.0, kGrowRankTol, r_grow, 0, false);
      RCK(launch_event(A, km, G, s));
    }
    st = finish(ctx);
    if (st != ROM_OK) { rom_destroy(ctx); return st; }
    std::vector<double> sg(r_grow);
    RCK(cudaMemcpy(sg.data(), d.sigma, sizeof(double) * r_grow, cudaMemcpyDeviceToHost));
    int k = 0;
    for (int j = 0; j < r && j < r_grow; ++j)
      if (sg[0] > 0.0 && sg[j] > ctx->cfg.rank_tol * sg[0]) ++k;
    if (k < r_alloc) {
      RCK(cudaMemsetAsync(d.phi + (size_t)k * N, 0, sizeof(double) * N * (r_alloc - k), s));
      RCK(cudaMemsetAsync(d.sigma + k, 0, sizeof(double) * (kMaxR + 1 - k), s));
    }
    RCK(cudaMemcpyAsync(d.rank, &k, sizeof(int), cudaMemcpyHostToDevice, s));
    if (mixed(ctx)) {   // the online basis of the mixed form is the FP32 rounding of the POD
      to_fp32_kernel<<<512, 256, 0, s>>>(d.phi, d.phi32, (int64_t)N * r);
      RCK(cudaGetLastError());
    }
    RCK(cudaStreamSynchronize(s));
  }
  // the comparison rules' window: the last `window` training snapshots, preprocessed
  if (ctx->cfg.update_rule == ROM_UPDATE_WINDOWED_SVD || ctx->cfg.update_rule == ROM_UPDATE_DIRECT) {
    const int nw = ctx->cfg.window;
    RCK(launch_win_fill(ctx->q_train + (size_t)(w - nw) * N, N, d.q_ref, d.drow, N, nw, d.win, s));
  }
  // initial reduced state and first coarse correction state
  {
    const double* qlast = ctx->q_train + (size_t)(w - 1) * N;
    ProjectArgs P;
    P.n = N; P.ld = N; P.r = r; P.rank = d.rank; P.phi = d.phi; P.phi32 = basis32(ctx); P.v = qlast; P.q_ref = d.q_ref;
    P.drow = d.drow; P.a = d.a; P.partials = d.partials; P.bar = d.bar; P.status = d.status;
    RCK(launch_project(P, km_of(ctx), G, s));
    RCK(fom_step(ctx, qlast, d.y_corr, ctx->cfg.z * ctx->cfg.dt));
    RCK(select_features(ctx, d.y_corr, s));
    if (ctx->cfg.n_s > 0) RCK(launch_sampling(sample_args(ctx), km_of(ctx), G, s));
  }
  st = finish(ctx);
  if (st != ROM_OK) { rom_destroy(ctx); return st; }
  if (!keep_train) {
    cudaFree(ctx->q_train);
    ctx->q_train = nullptr;
  }
  ctx->step = w;
  *out = ctx;
  return ROM_OK;
}

}  // namespace

extern "C" {

rom_status rom_init(const rom_config* cfg_in, const double* q0_host, void* stream, rom_ctx** out) {
  return init_ctx(cfg_in, q0_host, stream, false, out);
}

rom_status rom_step(rom_ctx* ctx, int64_t n_steps) {
  if (!ctx || n_steps < 0) return ROM_EINVAL;
  if (ctx->poisoned) return ROM_ESTATE;
  const int64_t z = ctx->cfg.z, w = ctx->cfg.w_init;
  while (n_steps > 0) {
    int64_t m = (ctx->step - w) % z;
    if (m < 0) m += z;
    int64_t to_event = z - m;
    int64_t seg = n_steps < to_event ? n_steps : to_event;
    const bool event = seg == to_event;
    if (event && ctx->fom_overlap) {
      // the coarse FOM step depends only on the previous snapshot: it runs
      // beside the reduced steps of the interval
      RCK(coarse_fom_fork(ctx));
      RCK(run_steps(ctx, (int)seg));
      RCK(coarse_fom_join(ctx));
    } else {
      RCK(run_steps(ctx, (int)seg));
      if (event && !instant_rule(ctx)) RCK(coarse_fom(ctx));
    }
    ctx->step += seg;
    n_steps -= seg;
    if (event) {
      RCK(run_event(ctx));
      if (instant_rule(ctx)) RCK(coarse_fom(ctx));   // the instantaneous rules advance the snapshot last
    }
  }
  return finish(ctx);
}

rom_status rom_update_basis(rom_ctx* ctx, const double* y_host) {
  if (!ctx) return ROM_EINVAL;
  if (ctx->poisoned) return ROM_ESTATE;
  if (y_host && !all_finite(y_host, ctx->N)) return ROM_ENONFINITE;
  if (y_host) {
    RCK(cudaMemcpyAsync(ctx->d.y_corr, y_host, sizeof(double) * ctx->N, cudaMemcpyHostToDevice,
                        ctx->stream));
    RCK(select_features(ctx, ctx->d.y_corr, ctx->stream));
  } else if (!instant_rule(ctx)) {
    RCK(coarse_fom(ctx));
  }
  RCK(run_event(ctx));
  if (!y_host && instant_rule(ctx)) RCK(coarse_fom(ctx));
  return finish(ctx);
}

rom_status rom_state(rom_ctx* ctx, double* q_tilde, double* a, double* sigma, double* phi,
                     double* y_corr, int64_t* step) {
  if (!ctx) return ROM_EINVAL;
  if (ctx->poisoned) return ROM_ESTATE;
  const int64_t N = ctx->N;
  const int r = ctx->cfg.r;
  cudaStream_t s = ctx->stream;
  if (q_tilde) {
    LiftArgs L;
    L.n = N; L.ld = N; L.rank = ctx->d.rank; L.phi = ctx->d.phi; L.phi32 = basis32(ctx); L.q_ref = ctx->d.q_ref;
    L.drow = ctx->d.drow; L.dinv = ctx->d.dinv; L.a = ctx->d.a; L.out = ctx->d.lifted;
    RCK(launch_lift(L, km_of(ctx), s));
    RCK(cudaMemcpyAsync(q_tilde, ctx->d.lifted, sizeof(double) * N, cudaMemcpyDeviceToHost, s));
  }
  std::vector<double> ha(r), hphi;
  RCK(cudaMemcpyAsync(ha.data(), ctx->d.a, sizeof(double) * r, cudaMemcpyDeviceToHost, s));
  if (sigma) RCK(cudaMemcpyAsync(sigma, ctx->d.sigma, sizeof(double) * r, cudaMemcpyDeviceToHost, s));
  std::vector<float> phi32h;
  if (phi && mixed(ctx)) {
    phi32h.resize((size_t)N * r);
    RCK(cudaMemcpyAsync(phi32h.data(), ctx->d.phi32, sizeof(float) * N * r, cudaMemcpyDeviceToHost, s));
  } else if (phi) {
    RCK(cudaMemcpyAsync(phi, ctx->d.phi, sizeof(double) * N * r, cudaMemcpyDeviceToHost, s));
  }
  if (y_corr) RCK(cudaMemcpyAsync(y_corr, ctx->d.y_corr, sizeof(double) * N, cudaMemcpyDeviceToHost, s));
  rom_status st = finish(ctx);
  if (st != ROM_OK) return st;
  if (phi && mixed(ctx))
    for (size_t e = 0; e < phi32h.size(); ++e) phi[e] = (double)phi32h[e];
  // sign convention of the exported basis: largest-magnitude entry positive
  if (phi) {
    for (int j = 0; j < r; ++j) {
      double* col = phi + (size_t)j * N;
      int64_t im = 0;
      double best = -1.0;
      for (int64_t i = 0; i < N; ++i)
        if (fabs(col[i]) > best) { best = fabs(col[i]); im = i; }
      if (col[im] < 0.0) {
        for (int64_t i = 0; i < N; ++i) col[i] = -col[i];
        ha[j] = -ha[j];
      }
    }
  }
  if (a) memcpy(a, ha.data(), sizeof(double) * r);
  if (step) *step = ctx->step;
  return ROM_OK;
}

rom_status rom_load_state(rom_ctx* ctx, const double* phi, const double* sigma, const double* a,
                          const double* y_corr, int64_t step) {
  if (!ctx || !phi || !sigma || !a || !y_corr || step < ctx->cfg.w_init) return ROM_EINVAL;
  if (ctx->poisoned) return ROM_ESTATE;
  const int64_t N = ctx->N;
  const int r = ctx->cfg.r;
  if (!all_finite(phi, N * r) || !all_finite(sigma, r) || !all_finite(a, r) ||
      !all_finite(y_corr, N))
    return ROM_ENONFINITE;
  int k = 0;
  for (int j = 0; j < r; ++j)
    if (sigma[j] > 0.0) k = j + 1;
  cudaStream_t s = ctx->stream;
  std::vector<float> phi32h;
  if (mixed(ctx)) {
    phi32h.resize((size_t)N * r);
    for (size_t e = 0; e < phi32h.size(); ++e) phi32h[e] = (float)phi[e];
    RCK(cudaMemcpyAsync(ctx->d.phi32, phi32h.data(), sizeof(float) * N * r, cudaMemcpyHostToDevice, s));
  } else {
    RCK(cudaMemcpyAsync(ctx->d.phi, phi, sizeof(double) * N * r, cudaMemcpyHostToDevice, s));
  }
  RCK(cudaMemsetAsync(ctx->d.sigma, 0, sizeof(double) * (kMaxR + 1), s));
  RCK(cudaMemcpyAsync(ctx->d.sigma, sigma, sizeof(double) * r, cudaMemcpyHostToDevice, s));
  RCK(cudaMemsetAsync(ctx->d.a, 0, sizeof(double) * (kMaxR + 1), s));
  RCK(cudaMemcpyAsync(ctx->d.a, a, sizeof(double) * r, cudaMemcpyHostToDevice, s));
  RCK(cudaMemcpyAsync(ctx->d.y_corr, y_corr, sizeof(double) * N, cudaMemcpyHostToDevice, s));
  RCK(cudaMemcpyAsync(ctx->d.rank, &k, sizeof(int), cudaMemcpyHostToDevice, s));
  RCK(select_features(ctx, ctx->d.y_corr, s));
  if (ctx->cfg.n_s > 0) RCK(launch_sampling(sample_args(ctx), km_of(ctx), ctx->grid, s));
  rom_status st = finish(ctx);   // (also waits for the staged host copies above)
  if (st == ROM_OK) ctx->step = step;
  return st;
}

rom_status rom_samples(rom_ctx* ctx, int32_t* idx_host) {
  if (!ctx || !idx_host || ctx->cfg.n_s <= 0) return ROM_EINVAL;
  if (ctx->poisoned) return ROM_ESTATE;
  RCK(cudaMemcpyAsync(idx_host, ctx->d.samples, sizeof(int) * ctx->cfg.n_s, cudaMemcpyDeviceToHost,
                      ctx->stream));
  return finish(ctx);
}

rom_status rom_info(rom_ctx* ctx, int32_t* rank, int32_t* rom_iters, int32_t* fom_iters) {
  if (!ctx) return ROM_EINVAL;
  if (ctx->poisoned) return ROM_ESTATE;
  int v[3] = {0, 0, 0};
  RCK(cudaMemcpyAsync(&v[0], ctx->d.rank, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  RCK(cudaMemcpyAsync(&v[1], ctx->d.iters_rom, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  RCK(cudaMemcpyAsync(&v[2], ctx->d.iters_fom, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  rom_status st = finish(ctx);
  if (rank) *rank = v[0];
  if (rom_iters) *rom_iters = v[1];
  if (fom_iters) *fom_iters = v[2];
  return st;
}

rom_status rom_profile(rom_ctx* ctx, int32_t enable) {
  if (!ctx) return ROM_EINVAL;
  if (ctx->poisoned) return ROM_ESTATE;
  if (enable) {
    if (!ctx->prof_ev_made) {
      for (int i = 0; i < 2 * kMaxProfEvents; ++i) RCK(cudaEventCreate(&ctx->prof_ev[i]));
      ctx->prof_ev_made = 1;
    }
    RCK(cudaStreamSynchronize(ctx->stream));
    ctx->prof_n = 0;
    for (int p = 0; p < kPhases; ++p) { ctx->prof_ms[p] = 0.0; ctx->prof_cnt[p] = 0; }
    ctx->prof_on = 1;
  } else {
    RCK(prof_flush(ctx));
    ctx->prof_on = 0;
  }
  return ROM_OK;
}

rom_status rom_profile_read(rom_ctx* ctx, double* ms_total, int64_t* launches) {
  if (!ctx || !ms_total || !launches) return ROM_EINVAL;
  if (ctx->poisoned) return ROM_ESTATE;
  RCK(prof_flush(ctx));
  for (int p = 0; p < kPhases; ++p) {
    ms_total[p] = ctx->prof_ms[p];
    launches[p] = ctx->prof_cnt[p];
  }
  return ROM_OK;
}

// ---------------------------------------------------------------------------
// low-level entry points (caller-owned device buffers)
// ---------------------------------------------------------------------------

rom_status rom_fom_rhs_dev(int32_t problem, int64_t n_cells, double nu, double gamma,
                           const double* q_dev, double* f_dev, void* stream) {
  rom_ctx* ctx = nullptr;
  if (!q_dev || !f_dev || n_cells < 2 || (problem != ROM_BURGERS && problem != ROM_EULER))
    return ROM_EINVAL;
  if (!device_ok()) return ROM_ECUDA;
  FomParams p;
  p.problem = problem; p.n_cells = n_cells; p.nu = nu; p.gamma = gamma; p.h = 0; p.tol = 0; p.max_iter = 0;
  RCK(launch_fom_rhs(p, q_dev, f_dev, (cudaStream_t)stream));
  RCK(cudaStreamSynchronize((cudaStream_t)stream));
  return ROM_OK;
}

rom_status rom_fom_step_dev(int32_t problem, int64_t n_cells, double nu, double gamma, double h,
                            double newton_tol, int32_t newton_max, const double* q_prev_dev,
                            double* q_dev, int32_t* iters_host, void* stream) {
  if (!q_prev_dev || !q_dev || q_prev_dev == q_dev || n_cells < 2 || !(h > 0.0) ||
      newton_max < 1 || !(newton_tol > 0.0))
    return ROM_EINVAL;
  if (problem == ROM_BURGERS && n_cells > (int64_t)kMaxChunks * kMaxChunkRows) return ROM_EINVAL;
  if (problem == ROM_EULER && (n_cells < 8 || n_cells > 128 * 256)) return ROM_EINVAL;
  if (problem != ROM_BURGERS && problem != ROM_EULER) return ROM_EINVAL;
  if (!device_ok()) return ROM_ECUDA;
  cudaStream_t s = (cudaStream_t)stream;
  FomScratch sc;
  float* chunk = nullptr;
  unsigned long long* maxbuf = nullptr;
  GridBarrier* bar = nullptr;
  int* ints = nullptr;
  if (dalloc(&chunk, fom_chunk_floats()) != cudaSuccess || dalloc(&maxbuf, 4) != cudaSuccess ||
      dalloc(&bar, 1) != cudaSuccess || dalloc(&ints, 2) != cudaSuccess) {
    cudaFree(chunk); cudaFree(maxbuf); cudaFree(bar); cudaFree(ints);
    cudaGetLastError();
    return ROM_ENOMEM;
  }
  sc.chunk = chunk; sc.maxbuf = maxbuf; sc.bar = bar; sc.status = ints; sc.iters = ints + 1;
  FomParams p;
  p.problem = problem; p.n_cells = n_cells; p.nu = nu; p.gamma = gamma; p.h = h;
  p.tol = newton_tol; p.max_iter = newton_max;
  rom_status result = ROM_OK;
  cudaError_t e = cudaMemsetAsync(maxbuf, 0, 4 * sizeof(unsigned long long), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(bar, 0, sizeof(GridBarrier), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(ints, 0, 2 * sizeof(int), s);
  if (e == cudaSuccess) e = launch_fom_step(p, q_prev_dev, q_dev, sc, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  int hv[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpy(hv, ints, sizeof(hv), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) result = ROM_ECUDA;
  else result = status_to_rom(hv[0]);
  if (iters_host) *iters_host = hv[1];
  cudaFree(chunk); cudaFree(maxbuf); cudaFree(bar); cudaFree(ints);
  return result;
}

rom_status rom_debug_set_wait_limit(int64_t cycles) {
  const long long c = cycles > 0 ? (long long)cycles : kSpinLimitCycles;
  cudaError_t (*setters[])(long long) = {set_wait_limit_fom,      set_wait_limit_euler,
                                         set_wait_limit_isvd,     set_wait_limit_reduced,
                                         set_wait_limit_sampling, set_wait_limit_batch,
                                         set_wait_limit_adjoint,  set_wait_limit_lspg};
  for (auto f : setters)
    if (f(c) != cudaSuccess) return ROM_ECUDA;
  return ROM_OK;
}

rom_status rom_isvd_update_dev(int64_t n, int32_t r, double lambda, double rank_tol, double* phi_dev,
                               double* sigma_dev, const double* y_dev, double* ubar_host,
                               void* stream) {
  if (n < 2 || r < 1 || r > kMaxR || r >= n || !phi_dev || !sigma_dev || !y_dev ||
      !(lambda >= 0.0 && lambda <= 1.0))
    return ROM_EINVAL;
  if (!device_ok()) return ROM_ECUDA;
  if (!(rank_tol > 0.0)) rank_tol = 1e-10;
  cudaStream_t s = (cudaStream_t)stream;
  const int G = grid_for(n);
  std::vector<double> hs(r);
  if (cudaMemcpy(hs.data(), sigma_dev, sizeof(double) * r, cudaMemcpyDeviceToHost) != cudaSuccess)
    return ROM_ECUDA;
  int k = 0;
  for (int j = 0; j < r; ++j)
    if (hs[j] > 0.0) k = j + 1;
  double *qres = nullptr, *partials = nullptr, *core = nullptr, *ubar = nullptr;
  int* ints = nullptr;
  GridBarrier* bar = nullptr;
  if (dalloc(&qres, n) != cudaSuccess || dalloc(&partials, (size_t)3 * G * (kMaxCore + 2)) != cudaSuccess ||
      dalloc(&core, core_ws_doubles()) != cudaSuccess || dalloc(&ubar, kMaxCore * kMaxCore) != cudaSuccess ||
      dalloc(&ints, 2) != cudaSuccess || dalloc(&bar, 1) != cudaSuccess) {
    cudaFree(qres); cudaFree(partials); cudaFree(core); cudaFree(ubar); cudaFree(ints); cudaFree(bar);
    cudaGetLastError();
    return ROM_ENOMEM;
  }
  EventArgs A;
  A.n = n; A.ld = n; A.r = r; A.rank = ints + 1; A.lambda = lambda; A.rank_tol = rank_tol;
  A.phi = phi_dev; A.phi32 = nullptr; A.gram = nullptr; A.sigma = sigma_dev; A.a = nullptr;
  A.transfer = 0; A.y = y_dev;
  A.q_ref = nullptr; A.drow = nullptr; A.preprocess = 0; A.yhat = nullptr; A.qres = qres;
  A.partials = partials; A.core = core; A.ubar = ubar; A.rec = nullptr; A.bar = bar; A.status = ints;
  rom_status result = ROM_OK;
  cudaError_t e = cudaMemsetAsync(ints, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ints + 1, &k, sizeof(int), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(bar, 0, sizeof(GridBarrier), s);
  if (e == cudaSuccess) e = launch_event(A, km_bucket(r + 1), G, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  int st = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&st, ints, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && ubar_host) {
    const int nn = k + 1;
    std::vector<double> u((size_t)nn * nn);
    e = cudaMemcpy(u.data(), ubar, sizeof(double) * nn * nn, cudaMemcpyDeviceToHost);
    for (int c = 0; c < r + 1; ++c)
      for (int rr = 0; rr < r + 1; ++rr)
        ubar_host[(size_t)c * (r + 1) + rr] = (c < nn && rr < nn) ? u[(size_t)c * nn + rr] : 0.0;
  }
  result = (e != cudaSuccess) ? ROM_ECUDA : status_to_rom(st);
  cudaFree(qres); cudaFree(partials); cudaFree(core); cudaFree(ubar); cudaFree(ints); cudaFree(bar);
  return result;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Gradient of a terminal misfit (rom_adjoint)
// ---------------------------------------------------------------------------
//
// Forward: the offline stage (training matrix kept), then n_steps online
// steps of Algorithm 1 launched one step at a time, recording each step's
// root a^{n+1} and, at each event, the basis before the update with the
// residual q (N x (r+1)), yhat, the new coarse state, the core's U, its
// singular values, (rho, |yhat|, p), sigma and the ranks before and after.
// With ckpt_every < n_steps the first pass keeps only the online state every
// ckpt_every steps, and the reverse sweep re-runs each segment from its
// checkpoint to record it. Reverse: the event and step adjoints from the last
// step back to the first, then the offline adjoint (adjoint.cu).

namespace {

struct AdjSeg {          // records of one segment of the forward pass
  int max_ev = 0;
  double* a_hist = nullptr;    // steps x r
  double* B = nullptr;         // max_ev x N x (r+1)
  double* yhat = nullptr;      // max_ev x N
  double* ynew = nullptr;      // max_ev x N
  double* ubar = nullptr;      // max_ev x (r+1)^2
  double* sbar = nullptr;      // max_ev x (r+1)
  double* rec = nullptr;       // max_ev x (r+2)
  double* sig = nullptr;       // max_ev x r
  int* kold = nullptr;         // max_ev
  int* knew = nullptr;         // max_ev
  double* phi_end = nullptr;   // N x r
};

struct AdjBufs {
  std::vector<void*> owned;
  template <typename T>
  cudaError_t alloc(T** p, size_t count) {
    cudaError_t e = dalloc(p, count);
    if (e == cudaSuccess) owned.push_back(*p);
    return e;
  }
  ~AdjBufs() {
    for (void* p : owned) cudaFree(p);
  }
};

bool is_event_at(const rom_ctx* ctx, int64_t n) {
  return ((n + 1 - ctx->cfg.w_init) % ctx->cfg.z) == 0;
}

// One online step (and its event) with recording into seg at local index m.
cudaError_t record_step(rom_ctx* ctx, AdjSeg& sg, int m, int& ev, double* qT, double d) {
  const int64_t N = ctx->N;
  const int r = ctx->cfg.r;
  cudaStream_t s = ctx->stream;
  cudaError_t e = run_steps(ctx, 1);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(sg.a_hist + (size_t)m * r, ctx->d.a, sizeof(double) * r, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return e;
  if (qT && (e = launch_adj_lift(N, r, ctx->d.phi, ctx->d.a, ctx->d.q_ref, d, qT, s)) != cudaSuccess) return e;
  if (is_event_at(ctx, ctx->step)) {
    const int x = ev++;
    double* B = sg.B + (size_t)x * N * (r + 1);
#define ACP(dst, src, bytes) \
  if ((e = cudaMemcpyAsync((dst), (src), (bytes), cudaMemcpyDeviceToDevice, s)) != cudaSuccess) return e
    ACP(B, ctx->d.phi, sizeof(double) * N * r);
    ACP(sg.kold + x, ctx->d.rank, sizeof(int));
    ACP(sg.sig + (size_t)x * r, ctx->d.sigma, sizeof(double) * r);
    if ((e = coarse_fom(ctx)) != cudaSuccess) return e;
    EventArgs A = event_args(ctx, ctx->d.y_corr, 1, ctx->cfg.lambda, ctx->cfg.rank_tol, r, 1);
    A.rec = sg.rec + (size_t)x * (r + 2);
    if ((e = launch_event(A, km_of(ctx), ctx->grid, s)) != cudaSuccess) return e;
    ACP(B + (size_t)r * N, ctx->d.qres, sizeof(double) * N);
    ACP(sg.yhat + (size_t)x * N, ctx->d.yhat, sizeof(double) * N);
    ACP(sg.ynew + (size_t)x * N, ctx->d.y_corr, sizeof(double) * N);
    ACP(sg.ubar + (size_t)x * (r + 1) * (r + 1), ctx->d.ubar, sizeof(double) * (r + 1) * (r + 1));
    ACP(sg.sbar + (size_t)x * (r + 1), ctx->d.core + core_sbar_offset(), sizeof(double) * (r + 1));
    ACP(sg.knew + x, ctx->d.rank, sizeof(int));
#undef ACP
  }
  ctx->step += 1;
  return cudaSuccess;
}

// One online step without recording.
cudaError_t plain_step(rom_ctx* ctx, double* qT, double d) {
  cudaError_t e = run_steps(ctx, 1);
  if (e != cudaSuccess) return e;
  if (qT && (e = launch_adj_lift(ctx->N, ctx->cfg.r, ctx->d.phi, ctx->d.a, ctx->d.q_ref, d, qT,
                                 ctx->stream)) != cudaSuccess)
    return e;
  if (is_event_at(ctx, ctx->step)) {
    if ((e = coarse_fom(ctx)) != cudaSuccess) return e;
    if ((e = run_event(ctx)) != cudaSuccess) return e;
  }
  ctx->step += 1;
  return cudaSuccess;
}

}  // namespace

extern "C" rom_status rom_adjoint(const rom_config* cfg, const double* q0_host, const double* target_host,
                                  int64_t n_steps, int32_t ckpt_every, void* stream, double* J_out,
                                  double* dJ_dnu, double* dJ_dq0, double* q_final) {
  if (!cfg || !q0_host || !target_host || !J_out || !dJ_dnu || n_steps < 1 || ckpt_every < 1)
    return ROM_EINVAL;
  rom_status vs = validate(cfg);
  if (vs != ROM_OK) return vs;
  if (cfg->problem != ROM_BURGERS || cfg->precision != ROM_FP64 || cfg->n_s != 0 || cfg->w_init > 128 ||
      cfg->projection != ROM_GALERKIN || cfg->time_scheme != ROM_BACKWARD_EULER)
    return ROM_EINVAL;
  const int64_t N = cfg->n_cells;
  if (!all_finite(q0_host, N) || !all_finite(target_host, N)) return ROM_ENONFINITE;
  rom_ctx* ctx = nullptr;
  rom_status st = init_ctx(cfg, q0_host, stream, true, &ctx);
  if (st != ROM_OK) return st;
  struct Guard {
    rom_ctx* c;
    ~Guard() { rom_destroy(c); }
  } guard{ctx};
  cudaStream_t s = ctx->stream;
  const int r = cfg->r, w = cfg->w_init, z = cfg->z;
  const int G = ctx->grid;
  const double dt = ctx->cfg.dt, nu = ctx->cfg.nu, lam = ctx->cfg.lambda;
  const double hc = z * dt;
  double d = 0.0;
  RCK(cudaMemcpy(&d, ctx->d.dvals, sizeof(double), cudaMemcpyDeviceToHost));
  int k0 = 0;
  RCK(cudaMemcpy(&k0, ctx->d.rank, sizeof(int), cudaMemcpyDeviceToHost));
  if (k0 < 1) return ROM_EINVAL;

  AdjBufs ab;
  cudaError_t e = cudaSuccess;
#define AAL(p, n) \
  if (e == cudaSuccess) e = ab.alloc(&(p), (size_t)(n))
  // offline copies
  double *phi0, *sig0, *a0, *ycorr0;
  AAL(phi0, N * r); AAL(sig0, r); AAL(a0, r); AAL(ycorr0, N);
  // checkpoints
  const int64_t seg_len = ckpt_every < n_steps ? ckpt_every : n_steps;
  const int64_t n_seg = (n_steps + seg_len - 1) / seg_len;
  double *ck_phi = nullptr, *ck_sig = nullptr, *ck_a = nullptr, *ck_y = nullptr;
  int* ck_rank = nullptr;
  if (n_seg > 1) {
    AAL(ck_phi, (size_t)n_seg * N * r); AAL(ck_sig, (size_t)n_seg * r); AAL(ck_a, (size_t)n_seg * r);
    AAL(ck_y, (size_t)n_seg * N); AAL(ck_rank, n_seg);
  }
  AdjSeg sg;
  sg.max_ev = (int)(seg_len / z + 2);
  AAL(sg.a_hist, seg_len * r); AAL(sg.B, (size_t)sg.max_ev * N * (r + 1));
  AAL(sg.yhat, (size_t)sg.max_ev * N); AAL(sg.ynew, (size_t)sg.max_ev * N);
  AAL(sg.ubar, (size_t)sg.max_ev * (r + 1) * (r + 1)); AAL(sg.sbar, (size_t)sg.max_ev * (r + 1));
  AAL(sg.rec, (size_t)sg.max_ev * (r + 2)); AAL(sg.sig, (size_t)sg.max_ev * r);
  AAL(sg.kold, sg.max_ev); AAL(sg.knew, sg.max_ev); AAL(sg.phi_end, N * r);
  // reverse state and work
  double *phibar, *phibar2, *qtbar, *qrefbar, *ybar, *ybar2, *abar, *sigbar, *wv, *mpart, *vpart, *acc;
  double *small, *part, *pnb, *bbar, *tchunk, *qT, *target, *Jd, *dtot, *mpartial;
  GridBarrier* bar;
  int* status;
  AAL(phibar, N * r); AAL(phibar2, N * r); AAL(qtbar, N); AAL(qrefbar, N); AAL(ybar, N); AAL(ybar2, N);
  AAL(abar, r); AAL(sigbar, r); AAL(wv, kMaxR); AAL(mpart, (size_t)G * kMaxR * kMaxR);
  AAL(vpart, (size_t)G * kMaxR); AAL(acc, 2 * kAdjSlots); AAL(small, kAdjSmall);
  AAL(part, (size_t)G * 16384); AAL(pnb, N * r); AAL(bbar, N * (r + 1)); AAL(tchunk, kMaxChunks * 16);
  AAL(qT, N); AAL(target, N); AAL(Jd, 1); AAL(dtot, 1); AAL(mpartial, 256); AAL(bar, 1); AAL(status, 1);
  // offline reverse
  double *X, *Qf, *Uf, *Xbar, *Rw, *Uw, *sw, *Vw, *Vtmp, *wk, *Aw, *B1, *B2, *Am, *Ubar, *Uh;
  double *qlastbar, *qb0, *qb1;
  AAL(X, N * w); AAL(Qf, N * w); AAL(Uf, N * w); AAL(Xbar, N * w); AAL(Rw, w * w); AAL(Uw, w * w);
  AAL(sw, w); AAL(Vw, w * w); AAL(Vtmp, w * w); AAL(wk, 256); AAL(Aw, w * r); AAL(B1, w * w);
  AAL(B2, r * w); AAL(Am, r * r); AAL(Ubar, N * r); AAL(Uh, r * r);
  AAL(qlastbar, N); AAL(qb0, N); AAL(qb1, N);
#undef AAL
  if (e != cudaSuccess) {
    cudaGetLastError();
    return ROM_ENOMEM;
  }
  RCK(cudaMemcpyAsync(phi0, ctx->d.phi, sizeof(double) * N * r, cudaMemcpyDeviceToDevice, s));
  RCK(cudaMemcpyAsync(sig0, ctx->d.sigma, sizeof(double) * r, cudaMemcpyDeviceToDevice, s));
  RCK(cudaMemcpyAsync(a0, ctx->d.a, sizeof(double) * r, cudaMemcpyDeviceToDevice, s));
  RCK(cudaMemcpyAsync(ycorr0, ctx->d.y_corr, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
  RCK(cudaMemcpyAsync(target, target_host, sizeof(double) * N, cudaMemcpyHostToDevice, s));
  RCK(cudaMemsetAsync(acc, 0, sizeof(double) * 2 * kAdjSlots, s));
  RCK(cudaMemsetAsync(bar, 0, sizeof(GridBarrier), s));
  RCK(cudaMemsetAsync(status, 0, sizeof(int), s));
  const int64_t step0 = ctx->step;

  // ---- forward pass ----
  int ev_first = 0;
  for (int64_t m = 0; m < n_steps; ++m) {
    double* qt = (m == n_steps - 1) ? qT : nullptr;
    if (n_seg == 1) {
      RCK(record_step(ctx, sg, (int)m, ev_first, qt, d));
    } else {
      if (m % seg_len == 0) {
        const int64_t c = m / seg_len;
        RCK(cudaMemcpyAsync(ck_phi + (size_t)c * N * r, ctx->d.phi, sizeof(double) * N * r, cudaMemcpyDeviceToDevice, s));
        RCK(cudaMemcpyAsync(ck_sig + (size_t)c * r, ctx->d.sigma, sizeof(double) * r, cudaMemcpyDeviceToDevice, s));
        RCK(cudaMemcpyAsync(ck_a + (size_t)c * r, ctx->d.a, sizeof(double) * r, cudaMemcpyDeviceToDevice, s));
        RCK(cudaMemcpyAsync(ck_y + (size_t)c * N, ctx->d.y_corr, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
        RCK(cudaMemcpyAsync(ck_rank + c, ctx->d.rank, sizeof(int), cudaMemcpyDeviceToDevice, s));
      }
      RCK(plain_step(ctx, qt, d));
    }
  }
  st = finish(ctx);
  if (st != ROM_OK) return st;
  if (n_seg == 1)
    RCK(cudaMemcpyAsync(sg.phi_end, ctx->d.phi, sizeof(double) * N * r, cudaMemcpyDeviceToDevice, s));
  RCK(launch_adj_misfit(N, qT, target, qtbar, mpartial, Jd, s));
  RCK(cudaMemsetAsync(phibar, 0, sizeof(double) * N * r, s));
  RCK(cudaMemsetAsync(qrefbar, 0, sizeof(double) * N, s));
  RCK(cudaMemsetAsync(ybar, 0, sizeof(double) * N, s));
  RCK(cudaMemsetAsync(abar, 0, sizeof(double) * r, s));
  RCK(cudaMemsetAsync(sigbar, 0, sizeof(double) * r, s));

  // ---- reverse sweep, segment by segment ----
  for (int64_t c = n_seg - 1; c >= 0; --c) {
    const int64_t m0 = c * seg_len, m1 = (m0 + seg_len < n_steps) ? m0 + seg_len : n_steps;
    int n_ev = 0;
    if (n_seg == 1) {
      n_ev = ev_first;
    } else {
      RCK(cudaMemcpyAsync(ctx->d.phi, ck_phi + (size_t)c * N * r, sizeof(double) * N * r, cudaMemcpyDeviceToDevice, s));
      RCK(cudaMemcpyAsync(ctx->d.sigma, ck_sig + (size_t)c * r, sizeof(double) * r, cudaMemcpyDeviceToDevice, s));
      RCK(cudaMemcpyAsync(ctx->d.a, ck_a + (size_t)c * r, sizeof(double) * r, cudaMemcpyDeviceToDevice, s));
      RCK(cudaMemcpyAsync(ctx->d.y_corr, ck_y + (size_t)c * N, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
      RCK(cudaMemcpyAsync(ctx->d.rank, ck_rank + c, sizeof(int), cudaMemcpyDeviceToDevice, s));
      ctx->step = step0 + m0;
      for (int64_t m = m0; m < m1; ++m) RCK(record_step(ctx, sg, (int)(m - m0), n_ev, nullptr, d));
      RCK(cudaMemcpyAsync(sg.phi_end, ctx->d.phi, sizeof(double) * N * r, cudaMemcpyDeviceToDevice, s));
      st = finish(ctx);
      if (st != ROM_OK) return st;
    }
    // ranks of the segment's events and the rank at its end
    std::vector<int> kold(n_ev + 1), knew(n_ev + 1);
    if (n_ev > 0) {
      RCK(cudaMemcpy(kold.data(), sg.kold, sizeof(int) * n_ev, cudaMemcpyDeviceToHost));
      RCK(cudaMemcpy(knew.data(), sg.knew, sizeof(int) * n_ev, cudaMemcpyDeviceToHost));
    }
    int k_end = 0;
    RCK(cudaMemcpy(&k_end, ctx->d.rank, sizeof(int), cudaMemcpyDeviceToHost));
    // walk the segment backwards; ev = index of the next event at or after m
    int ev = n_ev - 1;
    // steps after the segment's last event use phi_end with rank k_end
    for (int64_t m = m1 - 1; m >= m0; --m) {
      const int64_t n_lvl = step0 + m;     // time level before the step
      const bool has_ev = is_event_at(ctx, n_lvl);
      const double* phi_step;
      int k_step;
      if (has_ev) {
        const int x = ev;
        const double* phinew = (x + 1 < n_ev) ? sg.B + (size_t)(x + 1) * N * (r + 1) : sg.phi_end;
        AdjEventArgs E;
        E.n = N; E.k = kold[x]; E.kn = knew[x]; E.r = r;
        E.B = sg.B + (size_t)x * N * (r + 1); E.phinew = phinew;
        E.a = sg.a_hist + (size_t)(m - m0) * r; E.q_ref = ctx->d.q_ref; E.d = d; E.lambda = lam;
        E.abar = abar; E.phibar = phibar; E.pnb = pnb; E.bbar = bbar;
        E.yhat = sg.yhat + (size_t)x * N; E.ynew = sg.ynew + (size_t)x * N;
        E.ybar = ybar; E.ybar_new = ybar2; E.phibar_out = phibar2; E.qtbar = qtbar; E.qrefbar = qrefbar;
        E.ubar = sg.ubar + (size_t)x * (r + 1) * (r + 1); E.sbar = sg.sbar + (size_t)x * (r + 1);
        E.sigma_old = sg.sig + (size_t)x * r; E.rec = sg.rec + (size_t)x * (r + 2);
        E.small = small; E.sigbar = sigbar; E.part = part; E.acc = acc;
        if (E.k < 1) return ROM_ECUDA;
        RCK(launch_adj_event(E, G, s));
        std::swap(phibar, phibar2);
        TbeArgs T;
        T.y = E.ynew; T.rhs1 = ybar2; T.rhs2 = nullptr; T.x = ybar; T.n = N; T.nu = nu; T.h = hc;
        T.chunk = tchunk; T.bar = bar; T.status = status; T.acc_nu = acc + kAdjSlots;
        RCK(launch_adj_tbe(T, s));
        RCK(cudaMemsetAsync(abar, 0, sizeof(double) * r, s));
        phi_step = E.B;
        k_step = E.k;
        --ev;
      } else if (ev + 1 < n_ev) {
        phi_step = sg.B + (size_t)(ev + 1) * N * (r + 1);
        k_step = kold[ev + 1];
      } else {
        phi_step = sg.phi_end;
        k_step = k_end;
      }
      AdjStepArgs S;
      S.n = N; S.k = k_step; S.phi = phi_step; S.q_ref = ctx->d.q_ref; S.d = d; S.nu = nu; S.dt = dt;
      S.a = sg.a_hist + (size_t)(m - m0) * r; S.w = wv; S.abar = abar; S.qtbar = qtbar; S.phibar = phibar;
      S.qrefbar = qrefbar; S.mpart = mpart; S.vpart = vpart; S.acc = acc;
      if (S.k < 1) return ROM_ECUDA;
      RCK(launch_adj_step(S, G, s));
    }
  }

  // ---- offline adjoint ----
  const double* Q = ctx->q_train;
  const double* qlast = Q + (size_t)(w - 1) * N;
  {
    TbeArgs T;
    T.y = ycorr0; T.rhs1 = ybar; T.rhs2 = nullptr; T.x = qlastbar; T.n = N; T.nu = nu; T.h = hc;
    T.chunk = tchunk; T.bar = bar; T.status = status; T.acc_nu = acc + kAdjSlots;
    RCK(launch_adj_tbe(T, s));
    AdjA0Args A0{N, k0, phi0, qlast, ctx->d.q_ref, d, abar, phibar, qlastbar, qrefbar, acc};
    RCK(launch_adj_a0(A0, G, s));
  }
  const int k = k0;
  // X = D (Q - q_ref 1^T) and its thin SVD with every triplet: the same
  // calls as the forward POD, so U[:, :k] and s[:k] are the forward's bits
  RCK(launch_win_fill(Q, N, ctx->d.q_ref, ctx->d.drow, N, w, X, s));
  RCK(pod_thin_svd(X, N, w, Qf, Rw, Uw, sw, wk, part, G, s, Vw, Vtmp));
  RCK(launch_nn(NnArgs{N, w, w, Qf, N, Uw, w, 1, 1.0, 0.0, Uf, N, Uf, N}, s));
  // Ubar = Phi-bar - U sym(U^T Phi-bar) (tangent part at the POD basis)
  RCK(launch_tn(TnArgs{N, k, k, phi0, N, phibar, N, 1.0, part, Am}, G, s));
  RCK(launch_adj_neg_sym(Am, Uh, k, s));
  RCK(launch_nn(NnArgs{N, k, k, phi0, N, Uh, k, 1, 1.0, 1.0, phibar, N, Ubar, N}, s));
  // A = U^T Ubar over all w columns of U; Xbar = U B1 + Ubar B2
  RCK(launch_tn(TnArgs{N, w, k, Uf, N, Ubar, N, 1.0, part, Aw}, G, s));
  {
    AdjPodArgs P{N, w, k, sw, sigbar, Aw, Vw, B1, B2};
    RCK(launch_adj_pod_full(P, s));
  }
  RCK(launch_nn(NnArgs{N, w, w, Uf, N, B1, w, 1, 1.0, 0.0, Xbar, N, Xbar, N}, s));
  RCK(launch_nn(NnArgs{N, k, w, Ubar, N, B2, w, 1, 1.0, 1.0, Xbar, N, Xbar, N}, s));
  // Qbar (into Qf's buffer) and q_ref-bar
  double* Qbar = Qf;
  {
    AdjXcArgs XA{N, w, Q, ctx->d.q_ref, d, Xbar, Qbar, qlastbar, qrefbar, acc, dtot};
    RCK(launch_adj_xc(XA, G, s));
  }
  // reversed training trajectory
  RCK(cudaMemsetAsync(qb0, 0, sizeof(double) * N, s));
  double* qcur = qb0;
  double* qnext = qb1;
  for (int j = w - 1; j >= 0; --j) {
    TbeArgs T;
    T.y = Q + (size_t)j * N; T.rhs1 = qcur; T.rhs2 = Qbar + (size_t)j * N; T.x = qnext; T.n = N;
    T.nu = nu; T.h = dt; T.chunk = tchunk; T.bar = bar; T.status = status; T.acc_nu = acc + kAdjSlots;
    RCK(launch_adj_tbe(T, s));
    std::swap(qcur, qnext);
  }
  RCK(launch_adj_add(N, qcur, qrefbar, qnext, s));       // q0-bar
  double* nubar_d = dtot;
  RCK(launch_adj_sum_slots(acc + kAdjSlots, nubar_d, 0, s));
  RCK(cudaStreamSynchronize(s));
  int dst = 0;
  RCK(cudaMemcpy(&dst, status, sizeof(int), cudaMemcpyDeviceToHost));
  if (dst != 0) return status_to_rom(dst);
  RCK(cudaMemcpy(J_out, Jd, sizeof(double), cudaMemcpyDeviceToHost));
  RCK(cudaMemcpy(dJ_dnu, nubar_d, sizeof(double), cudaMemcpyDeviceToHost));
  if (dJ_dq0) RCK(cudaMemcpy(dJ_dq0, qnext, sizeof(double) * N, cudaMemcpyDeviceToHost));
  if (q_final) RCK(cudaMemcpy(q_final, qT, sizeof(double) * N, cudaMemcpyDeviceToHost));
  return ROM_OK;
}
