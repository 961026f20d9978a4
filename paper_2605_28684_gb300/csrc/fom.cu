// Full-order model kernels: semi-discrete operator f(q) and the backward-Euler
// Newton step  q - q_prev - h f(q) = 0  (paper Eq. be_residual_rom_section,
// Eq. coarse_fom_backward_euler; Burgers setup of Sec. 5.1).
//
// Burgers: f_i = -(F_{i+1/2} - F_{i-1/2})/dx + nu (u_{i+1} - 2u_i + u_{i-1})/dx^2
// with the Godunov flux F(uL, uR) = max(max(uL,0)^2/2, min(uR,0)^2/2),
// periodic; the Jacobian takes the derivative of the selected branch (tie ->
// left).
//
// Newton solve, one cooperative launch per BE step. The residual is FP64; the
// periodic tridiagonal system (I - h J_f) delta = -r is solved in FP32 (it
// only steers the iteration; the converged root is fixed by the FP64
// residual). Partitioning: C chunks (power of two), one CTA each, one row per
// thread. The last row of every chunk is a separator s_c. The interior rows of
// chunk c are solved by parallel cyclic reduction (PCR) in shared memory for
// three right-hand sides, giving x_t = y_t + v_t s_{c-1} + w_t s_c. The
// separator equations then form a cyclic tridiagonal system of order C, which
// every CTA solves redundantly by cyclic PCR after one grid barrier.
#include <cmath>
#include <mutex>

#include "rom_internal.cuh"

namespace rom {

namespace {

struct BurgersRow {
  double f;                 // f_i
  double dl, dc, dr;        // df_i/du_{i-1}, df_i/du_i, df_i/du_{i+1}
};

__device__ __forceinline__ BurgersRow burgers_row(double ul, double u, double ur, double nu,
                                                  double inv_dx) {
  // interface i-1/2 between (ul, u)
  double Ll = 0.5 * fmax(ul, 0.0) * fmax(ul, 0.0);
  double Rl = 0.5 * fmin(u, 0.0) * fmin(u, 0.0);
  bool tl = Ll >= Rl;
  double Fl = tl ? Ll : Rl;
  double dFl_dl = tl ? fmax(ul, 0.0) : 0.0;
  double dFl_dc = tl ? 0.0 : fmin(u, 0.0);
  // interface i+1/2 between (u, ur)
  double Lr = 0.5 * fmax(u, 0.0) * fmax(u, 0.0);
  double Rr = 0.5 * fmin(ur, 0.0) * fmin(ur, 0.0);
  bool tr = Lr >= Rr;
  double Fr = tr ? Lr : Rr;
  double dFr_dc = tr ? fmax(u, 0.0) : 0.0;
  double dFr_dr = tr ? 0.0 : fmin(ur, 0.0);
  double inv_dx2 = inv_dx * inv_dx;
  BurgersRow o;
  o.f = -(Fr - Fl) * inv_dx + nu * (ur - 2.0 * u + ul) * inv_dx2;
  o.dl = dFl_dl * inv_dx + nu * inv_dx2;
  o.dc = (dFl_dc - dFr_dc) * inv_dx - 2.0 * nu * inv_dx2;
  o.dr = -dFr_dr * inv_dx + nu * inv_dx2;
  return o;
}

__global__ void burgers_rhs_kernel(const double* __restrict__ q, double* __restrict__ f,
                                   int64_t n, double nu) {
  double inv_dx = (double)n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double ul = q[(i - 1 + n) % n], u = q[i], ur = q[(i + 1) % n];
    f[i] = burgers_row(ul, u, ur, nu, inv_dx).f;
  }
}

__device__ __forceinline__ int64_t chunk_begin(int c, int C, int64_t n) {
  return (int64_t)c * n / C;
}

// Chunk summary published for the reduced (separator) system:
//  [0..3]  separator row (a, b, c, d) of  a x_{e-1} + b s + c x_{e+1} = d
//  [4..6]  (y, v, w) of the first interior row
//  [7..9]  (y, v, w) of the last interior row
constexpr int kChunkStride = 16;

struct BurgersNewtonArgs {
  const double* q_prev;
  double* q;
  int64_t n;
  double nu, h, tol;
  int max_iter, C;
  float* chunk;
  unsigned long long* maxbuf;
  GridBarrier* bar;
  int* status;
  int* iters;
};

__global__ void __launch_bounds__(kMaxChunkRows)
burgers_newton_kernel(BurgersNewtonArgs A) {
  __shared__ float sa[kMaxChunkRows], sb[kMaxChunkRows], sc[kMaxChunkRows];
  __shared__ float sd0[kMaxChunkRows], sd1[kMaxChunkRows], sd2[kMaxChunkRows];
  __shared__ double su[kMaxChunkRows];
  __shared__ float ra[kMaxChunks], rb[kMaxChunks], rc[kMaxChunks], rd[kMaxChunks];
  __shared__ float rs[kMaxChunks];
  __shared__ double red[32];

  const int C = A.C;
  const int c = blockIdx.x;
  const int t = threadIdx.x;
  const int64_t n = A.n;
  const int64_t beg = chunk_begin(c, C, n);
  const int m = (int)(chunk_begin(c + 1, C, n) - beg);
  const int mi = m - 1;                 // interior rows; row m-1 is the separator
  const bool active = t < m;
  const int64_t i = beg + t;
  const double inv_dx = (double)n;

  double u = active ? A.q_prev[i] : 0.0;
  const double un = u;
  if (active) A.q[i] = u;
  int it = 0;
  bool done = false;
  if (!grid_sync(A.bar, A.status)) return;

  for (it = 1; it <= A.max_iter && !done; ++it) {
    const int par = it & 1;
    // ---- phase A: residual (FP64), Jacobian row (FP32), interior PCR ----
    su[t] = u;
    __syncthreads();
    float a_t = 0.f, b_t = 1.f, c_t = 0.f, d0 = 0.f, d1 = 0.f, d2 = 0.f;
    if (active) {
      double ul = (t > 0) ? su[t - 1] : __ldcg(&A.q[(beg - 1 + n) % n]);
      double ur = (t < m - 1) ? su[t + 1] : __ldcg(&A.q[(beg + m) % n]);
      BurgersRow row = burgers_row(ul, u, ur, A.nu, inv_dx);
      double res = u - un - A.h * row.f;
      a_t = (float)(-A.h * row.dl);
      b_t = (float)(1.0 - A.h * row.dc);
      c_t = (float)(-A.h * row.dr);
      d0 = (float)(-res);
    }
    if (t == m - 1) {     // separator row: publish its equation
      float* ch = A.chunk + (size_t)c * kChunkStride;
      ch[0] = a_t; ch[1] = b_t; ch[2] = c_t; ch[3] = d0;
    }
    // interior system: rows 0..mi-1; couplings to the outside go to d1 / d2
    if (t < mi) {
      if (t == 0) { d1 = -a_t; a_t = 0.f; }
      if (t == mi - 1) { d2 = -c_t; c_t = 0.f; }
    } else {
      a_t = 0.f; b_t = 1.f; c_t = 0.f; d0 = d1 = d2 = 0.f;
    }
    sa[t] = a_t; sb[t] = b_t; sc[t] = c_t; sd0[t] = d0; sd1[t] = d1; sd2[t] = d2;
    __syncthreads();
    for (int s = 1; s < mi; s <<= 1) {
      float na = a_t, nb = b_t, nc = c_t, n0 = d0, n1 = d1, n2 = d2;
      if (t < mi) {
        int tm = t - s, tp = t + s;
        float am = 0.f, bm = 1.f, cm = 0.f, m0 = 0.f, m1 = 0.f, m2 = 0.f;
        float ap = 0.f, bp = 1.f, cp = 0.f, p0 = 0.f, p1 = 0.f, p2 = 0.f;
        if (tm >= 0) { am = sa[tm]; bm = sb[tm]; cm = sc[tm]; m0 = sd0[tm]; m1 = sd1[tm]; m2 = sd2[tm]; }
        if (tp < mi) { ap = sa[tp]; bp = sb[tp]; cp = sc[tp]; p0 = sd0[tp]; p1 = sd1[tp]; p2 = sd2[tp]; }
        float al = -a_t / bm, ga = -c_t / bp;
        na = al * am;
        nc = ga * cp;
        nb = b_t + al * cm + ga * ap;
        n0 = d0 + al * m0 + ga * p0;
        n1 = d1 + al * m1 + ga * p1;
        n2 = d2 + al * m2 + ga * p2;
      }
      __syncthreads();
      a_t = na; b_t = nb; c_t = nc; d0 = n0; d1 = n1; d2 = n2;
      sa[t] = a_t; sb[t] = b_t; sc[t] = c_t; sd0[t] = d0; sd1[t] = d1; sd2[t] = d2;
      __syncthreads();
    }
    float yv = 0.f, vv = 0.f, wv = 0.f;
    if (t < mi) { yv = d0 / b_t; vv = d1 / b_t; wv = d2 / b_t; }
    {
      float* ch = A.chunk + (size_t)c * kChunkStride;
      if (t == 0) { ch[4] = yv; ch[5] = vv; ch[6] = wv; }
      if (t == mi - 1) { ch[7] = yv; ch[8] = vv; ch[9] = wv; }
    }
    if (!grid_sync(A.bar, A.status)) return;

    // ---- phase B: separator system (cyclic, order C), every CTA ----
    // Every CTA has read the other parity's maxima (after the previous
    // iteration's second barrier) before arriving here, so it can be cleared.
    if (c == 0 && t == 0) {
      A.maxbuf[2 * (par ^ 1)] = 0ull;
      A.maxbuf[2 * (par ^ 1) + 1] = 0ull;
    }
    if (t < C) {
      const float* ch = A.chunk + (size_t)t * kChunkStride;
      const float* nx = A.chunk + (size_t)((t + 1) % C) * kChunkStride;
      float as_ = __ldcg(ch + 0), bs_ = __ldcg(ch + 1), cs_ = __ldcg(ch + 2), ds_ = __ldcg(ch + 3);
      float yL = __ldcg(ch + 7), vL = __ldcg(ch + 8), wL = __ldcg(ch + 9);
      float y0 = __ldcg(nx + 4), v0 = __ldcg(nx + 5), w0 = __ldcg(nx + 6);
      ra[t] = as_ * vL;
      rb[t] = bs_ + as_ * wL + cs_ * v0;
      rc[t] = cs_ * w0;
      rd[t] = ds_ - as_ * yL - cs_ * y0;
    }
    __syncthreads();
    for (int s = 1; s < C; s <<= 1) {
      float na = 0.f, nb = 0.f, nc = 0.f, nd = 0.f;
      if (t < C) {
        int tm = (t - s + C) % C, tp = (t + s) % C;
        float al = -ra[t] / rb[tm], ga = -rc[t] / rb[tp];
        na = al * ra[tm];
        nc = ga * rc[tp];
        nb = rb[t] + al * rc[tm] + ga * ra[tp];
        nd = rd[t] + al * rd[tm] + ga * rd[tp];
      }
      __syncthreads();
      if (t < C) { ra[t] = na; rb[t] = nb; rc[t] = nc; rd[t] = nd; }
      __syncthreads();
    }
    if (t < C) rs[t] = rd[t] / (ra[t] + rb[t] + rc[t]);
    __syncthreads();
    const float s_left = rs[(c - 1 + C) % C], s_self = rs[c];
    double delta = 0.0;
    if (t < mi) delta = (double)(yv + vv * s_left + wv * s_self);
    else if (t == m - 1) delta = (double)s_self;
    if (active) {
      u += delta;
      A.q[i] = u;
    }
    // maxima of |delta| (an FP32 value already) and |u| rounded to FP32 (it
    // only scales the tolerance), compared as integer keys; NaN/Inf map to
    // keys >= 0x7f800000
    unsigned int kdl = active ? (__float_as_uint(fabsf((float)delta))) : 0u;
    unsigned int kul = active ? (__float_as_uint(fabsf((float)u))) : 0u;
    if (active && !isfinite(u)) kul = 0x7fc00000u;
    kdl = block_max_u32(kdl, reinterpret_cast<unsigned int*>(red));
    kul = block_max_u32(kul, reinterpret_cast<unsigned int*>(red));
    if (t == 0) {
      atomicMax(&A.maxbuf[2 * par], (unsigned long long)kdl);
      atomicMax(&A.maxbuf[2 * par + 1], (unsigned long long)kul);
    }
    if (!grid_sync(A.bar, A.status)) return;
    unsigned int kd = (unsigned int)__ldcg(&A.maxbuf[2 * par]);
    unsigned int ku = (unsigned int)__ldcg(&A.maxbuf[2 * par + 1]);
    if (kd >= 0x7f800000u || ku >= 0x7f800000u) {
      if (c == 0 && t == 0) record_status(A.status, kStNonFinite);
      return;
    }
    if ((double)__uint_as_float(kd) <= A.tol * (1.0 + (double)__uint_as_float(ku))) done = true;
  }
  if (c == 0 && t == 0) {
    *A.iters = it - 1;
    if (!done) record_status(A.status, kStNoConv);
  }
}

int choose_chunks(int64_t n) {
  int C = 1;
  while (C * 2 <= kMaxChunks && n / (C * 2) >= 64) C *= 2;
  return C;
}

}  // namespace

size_t fom_chunk_floats() {
  size_t a = (size_t)kMaxChunks * kChunkStride, b = euler_chunk_floats();
  return a > b ? a : b;
}

cudaError_t launch_fom_rhs(const FomParams& p, const double* q, double* f, cudaStream_t s) {
  if (p.problem == ROM_EULER) return launch_euler_rhs(p.n_cells, p.gamma, q, f, s);
  if (p.problem != ROM_BURGERS) return cudaErrorInvalidValue;
  int64_t n = p.n_cells;
  int blocks = (int)((n + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  burgers_rhs_kernel<<<blocks, 256, 0, s>>>(q, f, n, p.nu);
  return cudaGetLastError();
}

cudaError_t launch_fom_step(const FomParams& p, const double* q_prev, double* q,
                            const FomScratch& sc, cudaStream_t s) {
  if (p.problem == ROM_EULER) return launch_euler_step(p, q_prev, q, sc, s);
  if (p.problem != ROM_BURGERS) return cudaErrorInvalidValue;
  int64_t n = p.n_cells;
  int C = choose_chunks(n);
  int64_t mmax = (n + C - 1) / C;
  if (mmax > kMaxChunkRows || n < 2) return cudaErrorInvalidValue;
  // one thread per row, and at least one per chunk for the separator system
  int threads = (int)((mmax + 31) / 32 * 32);
  if (threads < C) threads = C;
  BurgersNewtonArgs A;
  A.q_prev = q_prev; A.q = q; A.n = n; A.nu = p.nu; A.h = p.h; A.tol = p.tol;
  A.max_iter = p.max_iter; A.C = C; A.chunk = sc.chunk; A.maxbuf = sc.maxbuf;
  A.bar = sc.bar; A.status = sc.status; A.iters = sc.iters;
  void* args[] = {&A};
  return cudaLaunchCooperativeKernel((const void*)burgers_newton_kernel, dim3(C),
                                     dim3(threads), args, 0, s);
}

namespace {

// One stage of the four-stage, third-order SSP Runge-Kutta scheme (App. D)
// given f = f(x): out = x + h/2 f, or out = 2/3 u0 + 1/3 (x + h/2 f) in the
// third stage. Works on the whole state vector (n entries, any layout).
__global__ void rk_stage_kernel(const double* __restrict__ x, const double* __restrict__ f,
                                const double* __restrict__ u0, double* __restrict__ out, int64_t n,
                                double h2, int third) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double v = x[i] + h2 * f[i];
    if (third) v = (2.0 / 3.0) * u0[i] + (1.0 / 3.0) * v;
    out[i] = v;
  }
}

}  // namespace

cudaError_t launch_fom_explicit_step(const FomParams& p, int n_var, const double* q_prev, double* q,
                                     double* w1, double* w2, double* f, cudaStream_t s) {
  const int64_t n = p.n_cells * n_var;
  int blocks = (int)((n + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  const double h2 = 0.5 * p.h;
  const double* x[4] = {q_prev, w1, w2, w1};
  double* o[4] = {w1, w2, w1, q};
  for (int st = 0; st < 4; ++st) {
    cudaError_t e = launch_fom_rhs(p, x[st], f, s);
    if (e != cudaSuccess) return e;
    rk_stage_kernel<<<blocks, 256, 0, s>>>(x[st], f, q_prev, o[st], n, h2, st == 2 ? 1 : 0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Wait bound of this translation unit's kernels (see rom_internal.cuh).
cudaError_t set_wait_limit_fom(long long cycles) { return set_wait_limit_here(cycles); }

}  // namespace rom

// ---------------------------------------------------------------------------
// Allocation-free FOM step.
//
// Some callers cannot call cudaMalloc: for example a host application that
// owns all device memory through its own pool and forbids raw allocations, or
// a time-critical loop that cannot afford cudaMalloc/cudaFree (cudaFree waits
// for the whole device). rom_fom_step_noalloc_dev serves them: it runs the same
// Newton kernel as rom_fom_step_dev, but its scratch (separator-system chunk
// summaries, the two maxima per iteration parity, the grid barrier, the status
// and iteration words) lives in the fixed array below instead of memory
// allocated per call.
//
// The array is kNoAllocScratchBytes (8448 bytes, independent of n_cells); every
// GPU that loads the library holds it until the process exits. It is shared by
// all calls and keeps the contents of the last call, so each call first clears
// the parts that must start at zero. Calls whose work overlaps on the GPU (two
// host threads, or two streams, at the same time) race on it.
// ---------------------------------------------------------------------------

namespace {

constexpr size_t kNoAllocChunkBytes = sizeof(float) * rom::kMaxChunks * 16;   // 8 KiB
constexpr size_t kNoAllocMaxOff = kNoAllocChunkBytes;                           // 4 x u64
constexpr size_t kNoAllocBarOff = kNoAllocMaxOff + 4 * sizeof(unsigned long long);
constexpr size_t kNoAllocStatusOff = kNoAllocBarOff + sizeof(rom::GridBarrier);  // status, iters
constexpr size_t kNoAllocUsed = kNoAllocStatusOff + 2 * sizeof(int);
constexpr size_t kNoAllocScratchBytes = 8448;
static_assert(kNoAllocUsed <= kNoAllocScratchBytes, "scratch layout exceeds the array");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
unsigned char* g_noalloc_addr[kNoAllocMaxDevices] = {};

// Device address of the scratch array on the current device. Looked up once per
// device (with that device current) and cached; in host code the array's name
// is only a stand-in, not a device address.
cudaError_t noalloc_scratch(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_noalloc_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" rom_status rom_fom_step_noalloc_dev(int32_t problem, int64_t n_cells, double nu,
                                               double gamma, double h, double newton_tol,
                                               int32_t newton_max, const double* q_prev_dev,
                                               double* q_dev, int32_t* iters_host, void* stream) {
  const int64_t max_cells = (int64_t)rom::kMaxChunks * rom::kMaxChunkRows;
  if (!q_prev_dev || !q_dev || q_prev_dev == q_dev || problem != ROM_BURGERS || n_cells < 2 ||
      n_cells > max_cells || !(h > 0.0) || newton_max < 1 || !(newton_tol > 0.0))
    return ROM_EINVAL;
  unsigned char* base = nullptr;
  if (noalloc_scratch(&base) != cudaSuccess) return ROM_ECUDA;
  cudaStream_t s = (cudaStream_t)stream;
  rom::FomScratch sc;
  sc.chunk = reinterpret_cast<float*>(base);
  sc.maxbuf = reinterpret_cast<unsigned long long*>(base + kNoAllocMaxOff);
  sc.bar = reinterpret_cast<rom::GridBarrier*>(base + kNoAllocBarOff);
  sc.status = reinterpret_cast<int*>(base + kNoAllocStatusOff);
  sc.iters = sc.status + 1;
  rom::FomParams p;
  p.problem = problem; p.n_cells = n_cells; p.nu = nu; p.gamma = gamma; p.h = h;
  p.tol = newton_tol; p.max_iter = newton_max;
  // maxima, barrier, status and iteration count must start at zero
  cudaError_t e = cudaMemsetAsync(base + kNoAllocMaxOff, 0, kNoAllocUsed - kNoAllocMaxOff, s);
  if (e == cudaSuccess) e = rom::launch_fom_step(p, q_prev_dev, q_dev, sc, s);
  int hv[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(hv, sc.status, sizeof(hv), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return ROM_ECUDA;
  if (iters_host) *iters_host = hv[1];
  switch (hv[0]) {
    case rom::kStOK: return ROM_OK;
    case rom::kStNoConv: return ROM_ENOCONV;
    case rom::kStNonFinite: return ROM_ENONFINITE;
    case rom::kStTimeout: return ROM_ETIMEOUT;
    default: return ROM_ECUDA;
  }
}
