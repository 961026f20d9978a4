// Internal declarations of librom (not part of the ABI).
//
// Execution model. Work that scales with N runs in cooperative kernels whose
// CTAs are all resident (cudaLaunchCooperativeKernel), separated by a
// software grid barrier whose wait is bounded in time: when it runs out the
// kernel records ROM_ETIMEOUT in the status word and returns instead of
// spinning forever. Double precision is the bottleneck on this part (FP64 runs
// at about 1/70 of the FP32 rate), so every FP64 sum over N is spread over all
// CTAs, while Newton Jacobians and their linear solves, which only steer the
// iteration, run in FP32 against an FP64 residual.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/rom.h"

namespace rom {

constexpr int kMaxR = 64;            // maximum reduced dimension
constexpr int kMaxCore = kMaxR + 1;  // core matrix order
constexpr int kMaxNs = 512;          // maximum number of sampled cells
constexpr int kBlock = 256;          // threads of the generic cooperative kernels
constexpr int kMaxChunks = 128;      // FOM tridiagonal partitions (power of two)
constexpr int kMaxChunkRows = 1024;  // rows per partition (one thread each)
constexpr long long kSpinLimitCycles = 4000000000LL;  // ~2 s at 2 GHz

// Device status word values (same numbering as rom_status).
constexpr int kStOK = 0, kStNoConv = 4, kStNonFinite = 5, kStTimeout = 6;

struct GridBarrier {
  unsigned int count;
  unsigned int gen;
};

// Bound of every device-side wait, in SM clock cycles. Each translation unit
// holds its own copy (no relocatable device code), so each one exports a
// setter (set_wait_limit_<unit>) and rom_debug_set_wait_limit calls them all.
static __constant__ long long c_wait_limit = kSpinLimitCycles;
static inline cudaError_t set_wait_limit_here(long long cycles) {
  return cudaMemcpyToSymbol(c_wait_limit, &cycles, sizeof(cycles));
}
cudaError_t set_wait_limit_fom(long long cycles);
cudaError_t set_wait_limit_euler(long long cycles);
cudaError_t set_wait_limit_isvd(long long cycles);
cudaError_t set_wait_limit_reduced(long long cycles);
cudaError_t set_wait_limit_sampling(long long cycles);
cudaError_t set_wait_limit_batch(long long cycles);
cudaError_t set_wait_limit_adjoint(long long cycles);
cudaError_t set_wait_limit_lspg(long long cycles);

// ---------------------------------------------------------------- barrier --

// All CTAs of a cooperative launch call this the same number of times.
// Returns false (and records a timeout) if the other CTAs did not arrive within
// c_wait_limit cycles (kSpinLimitCycles unless a test lowered it); the caller
// must then return.
__device__ __forceinline__ bool grid_sync(GridBarrier* bar, int* status) {
  __syncthreads();
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    volatile unsigned int* vgen = &bar->gen;
    unsigned int g = *vgen;
    __threadfence();
    unsigned int arrived = atomicAdd(&bar->count, 1u);
    int ok = 1;
    if (arrived == gridDim.x - 1) {
      bar->count = 0;
      __threadfence();
      atomicAdd(&bar->gen, 1u);
    } else {
      const long long limit = c_wait_limit;
      long long t0 = clock64();
      while (*vgen == g) {
        if (clock64() - t0 > limit) {
          atomicExch(status, kStTimeout);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok;
}

// ------------------------------------------------------------- reductions --

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sumf(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide sum/max; every thread gets the result. scratch: >= 32 doubles.
__device__ __forceinline__ double block_sum(double v, double* scratch) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) scratch[wid] = v;
  __syncthreads();
  double t = (threadIdx.x < nw) ? scratch[threadIdx.x] : 0.0;
  if (wid == 0) t = warp_sum(t);
  if (threadIdx.x == 0) scratch[0] = t;
  __syncthreads();
  double r = scratch[0];
  __syncthreads();
  return r;
}
__device__ __forceinline__ double block_max(double v, double* scratch) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_max(v);
  __syncthreads();
  if (lane == 0) scratch[wid] = v;
  __syncthreads();
  double t = (threadIdx.x < nw) ? scratch[threadIdx.x] : -1.0e308;
  if (wid == 0) t = warp_max(t);
  if (threadIdx.x == 0) scratch[0] = t;
  __syncthreads();
  double r = scratch[0];
  __syncthreads();
  return r;
}

// Integer comparisons of non-negative floating-point values. On this part a
// dependent FP64 instruction costs tens of cycles, so maxima and argmax
// reductions compare the IEEE bit patterns (which order like the values for
// non-negative numbers) on the integer pipe instead.
__device__ __forceinline__ unsigned int warp_max_u32(unsigned int v) {
  return __reduce_max_sync(0xffffffffu, v);
}
__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}
// Block-wide maximum of a 32-bit key; every thread gets the result.
__device__ __forceinline__ unsigned int block_max_u32(unsigned int v, unsigned int* scratch) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_max_u32(v);
  __syncthreads();
  if (lane == 0) scratch[wid] = v;
  __syncthreads();
  unsigned int t = (threadIdx.x < nw) ? scratch[threadIdx.x] : 0u;
  if (wid == 0) t = warp_max_u32(t);
  if (threadIdx.x == 0) scratch[0] = t;
  __syncthreads();
  unsigned int r = scratch[0];
  __syncthreads();
  return r;
}

// Order-preserving key of a non-negative double for atomicMax.
__device__ __forceinline__ unsigned long long nonneg_key(double x) {
  return (unsigned long long)__double_as_longlong(x);
}
__device__ __forceinline__ double key_to_double(unsigned long long k) {
  return __longlong_as_double((long long)k);
}

// (value, index) packed so that a larger key = larger value, then lower index.
struct ArgMax {
  double v;
  int i;
};
// Larger value first, then lower index. Values are non-negative or negative
// sentinels; negative values map below every non-negative one. The test runs
// on integer keys (see above).
__device__ __forceinline__ long long argmax_key(double v) {
  long long b = __double_as_longlong(v);
  return b < 0 ? -1 - (b & 0x7fffffffffffffffLL) : b;
}
__device__ __forceinline__ bool argmax_better(double v1, int i1, double v2, int i2) {
  long long k1 = argmax_key(v1), k2 = argmax_key(v2);
  return (k1 > k2) || (k1 == k2 && i1 < i2);
}
__device__ __forceinline__ ArgMax warp_argmax(ArgMax a) {
  for (int o = 16; o > 0; o >>= 1) {
    double v = __shfl_xor_sync(0xffffffffu, a.v, o);
    int i = __shfl_xor_sync(0xffffffffu, a.i, o);
    if (argmax_better(v, i, a.v, a.i)) { a.v = v; a.i = i; }
  }
  return a;
}
__device__ __forceinline__ ArgMax block_argmax(ArgMax a, double* sv, int* si) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  a = warp_argmax(a);
  __syncthreads();
  if (lane == 0) { sv[wid] = a.v; si[wid] = a.i; }
  __syncthreads();
  ArgMax b{-1.0e308, 0x7fffffff};
  if (threadIdx.x < nw) { b.v = sv[threadIdx.x]; b.i = si[threadIdx.x]; }
  if (wid == 0) b = warp_argmax(b);
  if (threadIdx.x == 0) { sv[0] = b.v; si[0] = b.i; }
  __syncthreads();
  ArgMax r{sv[0], si[0]};
  __syncthreads();
  return r;
}

// out[j] = sum over CTAs b of partials[b * stride + j], j < k. Warps take
// columns, lanes take CTAs: the loads are independent (no chain of dependent
// L2 round trips) and the summation order is fixed (deterministic).
__device__ __forceinline__ void grid_reduce_cols(const double* partials, int G, int stride, int k,
                                                 double* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = wid; j < k; j += nw) {
    double s = 0.0;
    for (int b = lane; b < G; b += 32) s += __ldcg(&partials[(size_t)b * stride + j]);
    s = warp_sum(s);
    if (lane == 0) out[j] = s;
  }
  __syncthreads();
}

__device__ __forceinline__ void record_status(int* status, int code) {
  atomicCAS(status, kStOK, code);
}

// In-place LU with partial pivoting of a k x k FP32 matrix (row-major, ld
// kMaxR) by one block.
__device__ __forceinline__ void lu_factor(float* J, int* piv, int k) {
  __shared__ int s_p;
  for (int c = 0; c < k; ++c) {
    if (threadIdx.x == 0) {
      int p = c;
      float best = fabsf(J[c * kMaxR + c]);
      for (int r = c + 1; r < k; ++r) {
        float v = fabsf(J[r * kMaxR + c]);
        if (v > best) { best = v; p = r; }
      }
      piv[c] = p;
      s_p = p;
    }
    __syncthreads();
    int p = s_p;
    if (p != c)
      for (int j = threadIdx.x; j < k; j += blockDim.x) {
        float tmp = J[c * kMaxR + j];
        J[c * kMaxR + j] = J[p * kMaxR + j];
        J[p * kMaxR + j] = tmp;
      }
    __syncthreads();
    float inv = 1.0f / J[c * kMaxR + c];
    for (int r = c + 1 + threadIdx.x; r < k; r += blockDim.x) J[r * kMaxR + c] *= inv;
    __syncthreads();
    const int rem = k - c - 1;
    for (int e = threadIdx.x; e < rem * rem; e += blockDim.x) {
      int r = c + 1 + e / rem, j = c + 1 + e % rem;
      J[r * kMaxR + j] -= J[r * kMaxR + c] * J[c * kMaxR + j];
    }
    __syncthreads();
  }
}

// Inverse of a k x k FP32 matrix factorised by lu_factor, into Ji (row-major,
// ld kMaxR): thread l < k solves for column l (needs blockDim >= k). Newton
// loops that keep one factorisation for several iterations form it once, so
// that every iteration's solve is a k-thread matrix-vector product
// (inv_apply) instead of 2k dependent warp reductions.
__device__ __forceinline__ void lu_inverse(const float* J, const int* piv, float* Ji, int k) {
  const int l = threadIdx.x;
  if (l < k) {
    for (int i = 0; i < k; ++i) Ji[i * kMaxR + l] = (i == l) ? 1.f : 0.f;
    for (int c = 0; c < k; ++c) {        // the row swaps of the factorisation, in order
      const int p = piv[c];
      if (p != c) {
        const float tmp = Ji[c * kMaxR + l];
        Ji[c * kMaxR + l] = Ji[p * kMaxR + l];
        Ji[p * kMaxR + l] = tmp;
      }
    }
    for (int i = 0; i < k; ++i) {        // L y = P e_l (unit lower)
      float s = Ji[i * kMaxR + l];
      for (int m = 0; m < i; ++m) s = fmaf(-J[i * kMaxR + m], Ji[m * kMaxR + l], s);
      Ji[i * kMaxR + l] = s;
    }
    for (int i = k - 1; i >= 0; --i) {   // U x = y
      float s = Ji[i * kMaxR + l];
      for (int m = i + 1; m < k; ++m) s = fmaf(-J[i * kMaxR + m], Ji[m * kMaxR + l], s);
      Ji[i * kMaxR + l] = s / J[i * kMaxR + i];
    }
  }
  __syncthreads();
}

// x <- Ji x for a k-vector x in shared memory (block-level).
__device__ __forceinline__ void inv_apply(const float* Ji, float* x, int k) {
  const int j = threadIdx.x;
  float v = 0.f;
  if (j < k)
    for (int l = 0; l < k; ++l) v = fmaf(Ji[j * kMaxR + l], x[l], v);
  __syncthreads();
  if (j < k) x[j] = v;
  __syncthreads();
}

// Solve (LU) x = b for the RHS in x (FP32), by warp 0.
__device__ __forceinline__ void lu_solve(const float* J, const int* piv, float* x, int k) {
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    if (lane == 0)
      for (int c = 0; c < k; ++c) {
        int p = piv[c];
        if (p != c) { float tmp = x[c]; x[c] = x[p]; x[p] = tmp; }
      }
    __syncwarp();
    for (int i = 0; i < k; ++i) {          // L y = b (unit lower)
      float s = 0.f;
      for (int l = lane; l < i; l += 32) s += J[i * kMaxR + l] * x[l];
      s = warp_sumf(s);
      if (lane == 0) x[i] -= s;
      __syncwarp();
    }
    for (int i = k - 1; i >= 0; --i) {     // U x = y
      float s = 0.f;
      for (int l = i + 1 + lane; l < k; l += 32) s += J[i * kMaxR + l] * x[l];
      s = warp_sumf(s);
      if (lane == 0) x[i] = (x[i] - s) / J[i * kMaxR + i];
      __syncwarp();
    }
  }
  __syncthreads();
}


// ------------------------------------------------------------ FOM kernels --

struct FomParams {
  int problem;
  int64_t n_cells;
  double nu, gamma, h, tol;
  int max_iter;
};

// Scratch of a FOM Newton solve; owned by the caller (context or temporary).
struct FomScratch {
  float* chunk;                 // kMaxChunks * 16 (Burgers) or * 64 (Euler)
  unsigned long long* maxbuf;   // 4 keys: |delta|max and |q|max, two parities
  GridBarrier* bar;
  int* status;
  int* iters;
};

// Host launchers (fom.cu). q_dev receives the new state; q_prev_dev is read only.
cudaError_t launch_fom_rhs(const FomParams& p, const double* q, double* f, cudaStream_t s);
// One SSPRK(4,3) step of the FOM (App. D) over n_cells * n_var entries; w1,
// w2 and f are caller-owned scratch vectors of that length (fom.cu).
cudaError_t launch_fom_explicit_step(const FomParams& p, int n_var, const double* q_prev, double* q,
                                     double* w1, double* w2, double* f, cudaStream_t s);
cudaError_t launch_fom_step(const FomParams& p, const double* q_prev, double* q,
                            const FomScratch& sc, cudaStream_t s);
size_t fom_chunk_floats();
// Euler system (euler.cu)
cudaError_t launch_euler_rhs(int64_t n_cells, double gamma, const double* q, double* f,
                             cudaStream_t s);
cudaError_t launch_euler_step(const FomParams& p, const double* q_prev, double* q,
                              const FomScratch& sc, cudaStream_t s);
size_t euler_chunk_floats();

// ------------------------------------------------------------- ROM context --

struct DevState {
  // full-order vectors (N)
  double* q_ref;
  double* y_corr;
  double* y_tmp;
  double* yhat;
  double* qres;         // iSVD residual q (N)
  double* lifted;       // q~ (N)
  double* dvals;        // per-variable scaling D_v (n_var)
  double* drow;         // per-row scaling (N)
  double* dinv;         // 1 / drow (N)
  // basis
  double* phi;          // N x r (ld = N)
  float* phi32;         // FP32 basis, N x r (mixed precision only)
  double* gram;         // mixed precision: Gram partial sums (grid * kMaxR * kMaxR)
  double* sigma;        // r
  double* a;            // r
  double* a_prev;       // r
  int* rank;            // numerical rank k
  // iSVD core
  double* core;         // workspace for the core SVD (see isvd.cu)
  double* ubar;         // (r+1) x (r+1), column-major
  // projections
  double* partials;     // 2 * grid * (kMaxR + 1)
  float* jpartials;     // grid * kMaxR * kMaxR (FP32 Jacobian partial sums)
  float* jac;           // kMaxR * kMaxR
  // sampling (hyper-reduction)
  int* samples;         // n_s
  double* qd_u;         // N x r: row coordinates along the QDEIM residual directions
  double* cand_v;       // grid * kMaxNs candidate values
  unsigned long long* cand_f;  // grid * 2 QDEIM candidate words (epoch, index)
  unsigned long long* fgs_key;  // N: feature keys of the correction snapshot
  double* fgs_v;        // feature-guided candidates (values), best first
  int* fgs_i;           // their cell indices
  double* mesh;         // n_s * 3 * (kMaxR + 2): Phi rows, q_ref, d of the stencil
  double* minv;         // r x n_s  ((P^T Phi)^+, row-major r x n_s)
  // control
  GridBarrier* bar;
  GridBarrier* fom_bar;  // the coarse FOM step's own barrier (it may run beside a step kernel)
  int* status;
  int* iters_rom;
  int* iters_fom;
  unsigned long long* maxbuf;
  float* fom_chunk;
  double* npart;        // LSPG normal-equation partial sums
  // comparison update rules: snapshot window and Direct work space
  double* win;          // N x window (ring, oldest at win_head)
  double* dwork;        // N x kMaxR
  double* dsm;          // C (kMaxR^2), Vc (kMaxR^2), s (kMaxR), then the kc word
  double* dpart;        // grid x kMaxR^2 partial sums
};

}  // namespace rom

constexpr int kPhases = 5;
constexpr int kMaxProfEvents = 4096;

struct rom_ctx {
  rom_config cfg;
  // per-phase timing
  int prof_on;
  int prof_n;
  int prof_phase[kMaxProfEvents];
  cudaEvent_t prof_ev[2 * kMaxProfEvents];
  int prof_ev_made;
  double prof_ms[kPhases];
  long long prof_cnt[kPhases];
  cudaStream_t stream;
  // the coarse FOM step of an adaptation cycle runs on fom_stream beside the
  // reduced steps when those are the single-CTA DEIM kernel (fom_overlap)
  cudaStream_t fom_stream;
  cudaEvent_t ev_fork, ev_join, ev_fgs;   // ev_fgs: the feature-guided selection after the coarse step
  int fom_overlap;
  int fgs_pending;       // the context's stream has not yet waited for ev_fgs
  int64_t N;
  int64_t step;          // time level n
  int grid;              // CTAs of the generic cooperative kernels
  unsigned int sample_epoch;  // epoch of the next sampling launch's first QDEIM step
  int poisoned;
  int win_head;          // oldest slot of the snapshot window
  rom::DevState d;
  double* q_train;       // N x w_init (offline only, freed after init)
};
