// Sampling points of the DEIM-Galerkin model and the sampled-basis operators
// (paper Eq. qdeim_qr, Eq. fgs_selection, Eq. deim_galerkin_rom).
//
//  * Feature-guided candidates (fgs_key_kernel or fgs_key_euler_kernel, then
//    fgs_select_kernel): the T rows with the largest squared forward
//    difference of the feature of the correction snapshot, in decreasing
//    order, ties -> lowest index. Burgers: the feature is the state itself,
//    (y_{i+1} - y_i)^2, periodic. Euler: the feature is the cell pressure
//    (Sec. 5.3), (p_{i+1} - p_i)^2 with the zero-gradient ghost cell past the
//    right end, and each of a cell's three rows carries its cell's score.
//    They depend only on the snapshot, so they are computed right after the
//    coarse FOM step that produces it (beside the reduced steps of the
//    interval), by an exact radix selection on the IEEE bit patterns of the
//    squares.
//  * QDEIM (sampling_kernel): the first k pivots of a column-pivoted QR of
//    Phi^T, computed as greedy pivoting on the rows x_i of Phi: take the row
//    with the largest remaining squared norm (ties -> lowest index). The
//    remaining norms follow the pivoted Cholesky recursion of Phi Phi^T: with
//    the pivot p_s of step s and its remaining norm v_s,
//        c_i = x_i . x_{p_s} - sum_{l<s} c_i^(l) c_{p_s}^(l) / v_l,
//        res_i <- res_i - c_i^2 / v_s,
//    where c_i^(l) is row i's coordinate along the unnormalised residual
//    direction of pivot l (kept in a device array). This is the same
//    selection as Gram-Schmidt on the pivot directions, with one division
//    per pivot and no serial orthogonalisation.
//  * The remaining n_s - k points are the first feature-guided candidates
//    that are not QDEIM points.
//  * (P^T Phi)^+ = (A^T A)^{-1} A^T with A = P^T Phi (normal equations; the
//    symmetric positive definite A^T A inverted by Gauss-Jordan elimination in
//    FP64) and the stencil mesh used by the hyper-reduced step: Phi, q_ref
//    and D on the rows i-1, i, i+1 of every sampled cell (Burgers), or on the
//    three variable rows of the cells i-1, i, i+1 of every sampled row
//    (Euler).
#include <cfloat>
#include <cmath>

#include "rom_internal.cuh"
#include "rom_kernels.cuh"

namespace rom {

namespace {

constexpr int kFgsThreads = 512;   // threads of the feature-guided selection (one CTA)
constexpr int kFgsSort = 512;      // sort buffer of the selected candidates (T <= kFgsSort)
constexpr int kFgsStageKeys = 24576;  // keys staged in shared memory (192 KB)

// Bitonic sort (descending value, ascending index) of SIZE (value, index)
// pairs in shared memory, SIZE a power of two.
template <int SIZE>
__device__ void block_sort(double* v, int* idx) {
  for (int size = 2; size <= SIZE; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      __syncthreads();
      for (int t = threadIdx.x; t < SIZE / 2; t += blockDim.x) {
        int i = 2 * t - (t & (stride - 1));
        int j = i + stride;
        bool up = ((i & size) == 0);
        // "better" first when up
        bool jbetter = argmax_better(v[j], idx[j], v[i], idx[i]);
        if (jbetter == up) {
          double tv = v[i]; v[i] = v[j]; v[j] = tv;
          int ti = idx[i]; idx[i] = idx[j]; idx[j] = ti;
        }
      }
    }
  }
  __syncthreads();
}

// GPU-scope acquire load and release store of a 64-bit word.
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Exclusive prefix sum of one int per thread over the block; *total gets the
// sum. scratch: >= 33 ints.
__device__ __forceinline__ int block_scan_excl(int v, int* scratch, int* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  int x = v;
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  __syncthreads();
  if (lane == 31) scratch[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int w = (lane < nw) ? scratch[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < nw) scratch[lane] = w;      // inclusive warp totals
  }
  __syncthreads();
  const int before = (wid > 0) ? scratch[wid - 1] : 0;
  *total = scratch[nw - 1];
  __syncthreads();
  return before + x - v;
}

}  // namespace

// key_i = IEEE bits of (y_{i+1} - y_i)^2 (periodic). Squares are
// non-negative, so the keys order like the values.
__global__ void fgs_key_kernel(const double* __restrict__ y, int64_t n, unsigned long long* __restrict__ key) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double d = y[i + 1 == n ? 0 : i + 1] - y[i];
    key[i] = (unsigned long long)__double_as_longlong(d * d);
  }
}

// Cell pressure of the Euler state (App. B, floors included), every
// operation rounded on its own (no contraction into fused multiply-adds), so
// that the score is that of the plain expression.
__device__ __forceinline__ double cell_pressure(const double* __restrict__ y, int64_t nc, int64_t i,
                                                double gamma) {
  constexpr double kRhoFloor = 1e-10, kPFloor = 1e-10;
  const double rho = fmax(y[i], kRhoFloor);
  const double u = __ddiv_rn(y[nc + i], rho);
  const double ke = __dmul_rn(__dmul_rn(__dmul_rn(0.5, rho), u), u);
  return fmax(__dmul_rn(gamma - 1.0, __dsub_rn(y[2 * nc + i], ke)), kPFloor);
}

// Euler: key of the three rows of cell i = IEEE bits of (p_{i+1} - p_i)^2,
// p_nc = p_{nc-1} (zero-gradient ghost cell).
__global__ void fgs_key_euler_kernel(const double* __restrict__ y, int64_t nc, double gamma,
                                     unsigned long long* __restrict__ key) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += (int64_t)gridDim.x * blockDim.x) {
    const double p = cell_pressure(y, nc, i, gamma);
    const double pn = (i + 1 < nc) ? cell_pressure(y, nc, i + 1, gamma) : p;
    const double d = __dsub_rn(pn, p);
    const unsigned long long k = (unsigned long long)__double_as_longlong(__dmul_rn(d, d));
    key[i] = k;
    key[nc + i] = k;
    key[2 * nc + i] = k;
  }
}

// The T largest keys (ties -> lowest index), sorted, by one CTA: an MSB-first
// radix selection with 8-bit digits narrows the boundary until the entries
// above it and the whole boundary bin fit the sort buffer (or the full key
// is fixed), then an ordered compaction collects the entries above the
// boundary and those in it (all of them, or at full key the lowest-index
// ones), and a bitonic sort orders them; the first T are the result.
// With STAGE the keys are first copied to shared memory (n <= kFgsStageKeys),
// so that the passes read on-chip memory.
template <bool STAGE>
__global__ void __launch_bounds__(kFgsThreads) fgs_select_kernel(const unsigned long long* __restrict__ gkey,
                                                                 int64_t n, int T, double* out_v, int* out_i) {
  extern __shared__ __align__(16) unsigned long long s_keys[];
  const unsigned long long* key = STAGE ? s_keys : gkey;
  if (STAGE) {
#pragma unroll 8
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s_keys[i] = gkey[i];
  }
  __shared__ unsigned int hist[256];
  __shared__ unsigned long long s_prefix, s_mask;
  __shared__ long long s_need;
  __shared__ int s_all_eq;
  __shared__ int scan[33];
  __shared__ double sv[kFgsSort];
  __shared__ int si[kFgsSort];
  const int t = threadIdx.x, lane = t & 31;
  if (t == 0) {
    s_prefix = 0ull;
    s_mask = 0ull;
    s_need = T;
    s_all_eq = (n <= T) ? 1 : 0;      // fewer cells than T: every cell is a candidate
  }
  __syncthreads();
  for (int shift = 56; shift >= 0 && !s_all_eq; shift -= 8) {
    const unsigned long long prefix = s_prefix, mask = s_mask;
    for (int b = t; b < 256; b += blockDim.x) hist[b] = 0u;
    __syncthreads();
    for (int64_t base = 0; base < n; base += blockDim.x) {   // every lane runs every pass
      const int64_t i = base + t;
      unsigned int dg = 0xffffffffu;                           // not counted
      if (i < n) {
        const unsigned long long kk = key[i];
        if ((kk & mask) == prefix) dg = (unsigned int)((kk >> shift) & 255ull);
      }
      // one shared-memory atomic per distinct digit of the warp
      const unsigned int peers = __match_any_sync(0xffffffffu, dg);
      if (dg != 0xffffffffu && lane == __ffs(peers) - 1) atomicAdd(&hist[dg], (unsigned int)__popc(peers));
    }
    __syncthreads();
    if (t < 32) {
      // lane l holds the bins 255 - 8l ... 248 - 8l (descending)
      const long long need = s_need;     // read before any lane writes it (the shuffles order them)
      unsigned int c[8];
      unsigned int sum = 0u;
#pragma unroll
      for (int u = 0; u < 8; ++u) { c[u] = hist[255 - 8 * lane - u]; sum += c[u]; }
      unsigned int incl = sum;
      for (int o = 1; o < 32; o <<= 1) {
        unsigned int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      const unsigned int above = incl - sum;
      const bool mine = (long long)above < need && need <= (long long)incl;
      if (mine) {
        unsigned int acc = above;
        for (int u = 0; u < 8; ++u) {
          if ((long long)(acc + c[u]) >= need) {
            const unsigned long long d = (unsigned long long)(255 - 8 * lane - u);
            const long long left = need - (long long)acc;
            s_prefix = prefix | (d << shift);
            s_mask = mask | (255ull << shift);
            s_need = left;
            // the entries above this bin and the whole bin fit the sort
            // buffer: collect them all and let the sort decide (exact)
            s_all_eq = ((long long)T - left + (long long)c[u] <= (long long)kFgsSort) ? 1 : 0;
            break;
          }
          acc += c[u];
        }
      }
    }
    __syncthreads();
  }
  const unsigned long long prefix = s_prefix, mask = s_mask;
  const long long need = s_need;
  const bool all_eq = s_all_eq != 0;
  for (int e = t; e < kFgsSort; e += blockDim.x) { sv[e] = -1.0; si[e] = 0x7fffffff; }
  __syncthreads();
  int cnt;
  if (all_eq) {
    // every entry at or above the boundary prefix is collected (fewer than
    // kFgsSort); the order of collection is irrelevant, the sort fixes it.
    // Rows are strided over the threads (conflict-free shared-memory reads)
    // and appended through one warp-aggregated counter.
    __shared__ int s_cnt;
    if (t == 0) s_cnt = 0;
    __syncthreads();
    for (int64_t base = 0; base < n; base += blockDim.x) {   // every lane runs every pass
      const int64_t i = base + t;
      unsigned long long full = 0ull;
      bool sel = false;
      if (i < n) {
        full = key[i];
        sel = (full & mask) >= prefix;
      }
      const unsigned int bal = __ballot_sync(0xffffffffu, sel);
      int pos0 = 0;
      if (lane == 0 && bal) pos0 = atomicAdd(&s_cnt, __popc(bal));
      pos0 = __shfl_sync(0xffffffffu, pos0, 0);
      if (sel) {
        const int pos = pos0 + __popc(bal & ((1u << lane) - 1u));
        sv[pos] = __longlong_as_double((long long)full);
        si[pos] = (int)i;
      }
    }
    __syncthreads();
    cnt = s_cnt;
  } else {
    // the full key is fixed and more entries share it than are needed: an
    // ordered compaction (thread t takes the contiguous rows [t R, (t+1) R))
    // takes the entries above it and the lowest-index ones equal to it
    const int64_t R = (n + blockDim.x - 1) / blockDim.x;
    const int64_t r0 = (int64_t)t * R, r1 = (r0 + R < n) ? r0 + R : n;
    int n_above = 0, n_eq = 0;
    for (int64_t i = r0; i < r1; ++i) {
      const unsigned long long kk = key[i] & mask;
      n_above += (kk > prefix) ? 1 : 0;
      n_eq += (kk == prefix) ? 1 : 0;
    }
    int tot_above = 0, tot_eq = 0;
    const int off_above = block_scan_excl(n_above, scan, &tot_above);
    const int off_eq = block_scan_excl(n_eq, scan, &tot_eq);
    const int take_eq = (int)need;
    cnt = tot_above + take_eq;
    int pa = off_above, pe = off_eq;
    for (int64_t i = r0; i < r1; ++i) {
      const unsigned long long full = key[i];
      const unsigned long long kk = full & mask;
      if (kk > prefix) {
        sv[pa] = __longlong_as_double((long long)full); si[pa] = (int)i; ++pa;
      } else if (kk == prefix) {
        if (pe < take_eq) { sv[tot_above + pe] = __longlong_as_double((long long)full); si[tot_above + pe] = (int)i; }
        ++pe;
      }
    }
  }
  // the smallest power-of-two sort that holds the collected entries (the
  // rest of the buffer holds sentinels that sort last)
  if (cnt <= 128) block_sort<128>(sv, si);
  else if (cnt <= 256) block_sort<256>(sv, si);
  else block_sort<kFgsSort>(sv, si);
  for (int e = t; e < cnt && e < T; e += blockDim.x) {
    out_v[e] = sv[e];
    out_i[e] = si[e];
  }
}

namespace {

struct SampleSmem {
  double xp[kMaxR];      // basis row of the current pivot
  double up[kMaxR];      // its coordinates c_p^(l) / v_l, l < s
  double w[kMaxR];       // 1 / v_l
  double red[64];
  int redi[32];
  int scan[33];
  int piv[kMaxNs];       // QDEIM points, then the feature-guided points
  double G[kMaxR * kMaxR];   // A^T A, and the Gauss-Jordan steps (CTA 0) ...
  double G2[kMaxR * kMaxR];  // ... alternating with this buffer
  // followed by A = P^T Phi (n_s x k, row-major) on CTA 0
};

}  // namespace

template <typename TPhi>
__global__ void __launch_bounds__(kBlock) sampling_kernel(SampleArgs A) {
  const TPhi* phi = basis<TPhi>(A);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SampleSmem& sm = *reinterpret_cast<SampleSmem*>(smem_raw);
  double* X = reinterpret_cast<double*>(smem_raw + sizeof(SampleSmem));
  const int G = gridDim.x, b = blockIdx.x, t = threadIdx.x;
  const int64_t N = A.n, ld = A.ld;
  const int64_t beg = (int64_t)b * N / G, end = (int64_t)(b + 1) * N / G;
  const int k = *A.rank;
  const int kq = k < A.n_s ? k : A.n_s;
  const int lane = t & 31, wid = t >> 5, nw = blockDim.x >> 5;
  double* U = A.qd_u;   // c_i^(l): column l at U + l * N

  // ---- initial squared row norms and first local argmax ----
  // Each thread owns at most kRowsPerThread rows of this CTA's range and keeps
  // their remaining norms and chosen flags in registers across the pivots;
  // for its first row it also keeps the basis row and the coordinates c^(l)
  // in registers while k <= kRegK.
  constexpr int kRowsPerThread = 4;
  constexpr int kRegK = 8;
  const bool regs = k <= kRegK;
  double x0[kRegK], u0[kRegK];
#pragma unroll
  for (int j = 0; j < kRegK; ++j) { x0[j] = 0.0; u0[j] = 0.0; }
  double res[kRowsPerThread];
  bool taken[kRowsPerThread];
  ArgMax best{-1.0, 0x7fffffff};
#pragma unroll
  for (int r = 0; r < kRowsPerThread; ++r) {
    const int64_t i = beg + t + (int64_t)r * blockDim.x;
    res[r] = -1.0;
    taken[r] = false;
    if (i < end) {
      double s = 0.0;
      if (r == 0 && regs) {
#pragma unroll
        for (int j = 0; j < kRegK; ++j)
          if (j < k) x0[j] = (double)phi[j * ld + i];
#pragma unroll
        for (int j = 0; j < kRegK; ++j) s = fma(x0[j], x0[j], s);
      } else {
        for (int j = 0; j < k; ++j) { const double x = (double)phi[j * ld + i]; s = fma(x, x, s); }
      }
      res[r] = s;
      if (argmax_better(s, (int)i, best.v, best.i)) { best.v = s; best.i = (int)i; }
    }
  }

  // Exchange of the per-CTA candidates without a grid barrier: CTA b writes
  // the value of its candidate for step s to cand_v, fences, then writes the
  // word (epoch_s << 32 | index) to cand_f; readers wait for the word of every
  // CTA, then read the value. The slots are double-buffered by step parity:
  // a CTA writes a step's slot only after it has seen every CTA's word of the
  // step before, by which time every CTA has read the slot of two steps back.
  auto publish = [&](int step_w, const ArgMax& c) {
    if (t == 0) {
      const size_t sl = (size_t)b * 2 + (size_t)(step_w & 1);
      A.cand_v[sl] = c.v;
      const unsigned long long w = ((unsigned long long)(A.epoch + (unsigned int)step_w) << 32) |
                                   (unsigned long long)(unsigned int)c.i;
      st_release_u64(&A.cand_f[sl], w);   // orders the value (and the block's coordinates) before it
    }
  };
  // global argmax of step step_r over every CTA's candidate (fixed order);
  // false if the wait ran out (a timeout is recorded)
  auto gather = [&](int step_r, ArgMax& g) -> bool {
    g = ArgMax{-1.0, 0x7fffffff};
    bool late = false;
    const unsigned int ep = A.epoch + (unsigned int)step_r;
    for (int bb = t; bb < G; bb += blockDim.x) {
      const size_t sl = (size_t)bb * 2 + (size_t)(step_r & 1);
      const long long limit = c_wait_limit;
      const long long t0 = clock64();
      unsigned long long w = ld_acquire_u64(&A.cand_f[sl]);
      while ((unsigned int)(w >> 32) != ep) {
        if (clock64() - t0 > limit) { late = true; break; }
        __nanosleep(32);
        w = ld_acquire_u64(&A.cand_f[sl]);
      }
      if (late) break;
      const double v = __ldcg(&A.cand_v[sl]);
      const int i = (int)(unsigned int)(w & 0xffffffffull);
      if (argmax_better(v, i, g.v, g.i)) { g.v = v; g.i = i; }
    }
    if (__syncthreads_or(late)) {
      if (t == 0) record_status(A.status, kStTimeout);
      return false;
    }
    g = block_argmax(g, sm.red, sm.redi);
    return true;
  };

  if (kq > 0) {
    best = block_argmax(best, sm.red, sm.redi);
    publish(0, best);
  }
  for (int step = 0; step < kq; ++step) {
    ArgMax g;
    if (!gather(step, g)) return;
    const int p = g.i;
    if (t == 0) sm.piv[step] = p;
    if (step + 1 == kq) break;        // the last pivot needs no further update
    // the pivot row, its scaled coordinates along the earlier directions, and
    // 1 / v_s (independent loads and one division, issued together)
    if (t < k) sm.xp[t] = (double)phi[t * ld + p];
    if (t >= 64 && t - 64 < step) sm.up[t - 64] = __ldcg(&U[(size_t)(t - 64) * N + p]) * sm.w[t - 64];
    if (t == 128) sm.w[step] = (g.v > 0.0) ? 1.0 / g.v : 0.0;
    __syncthreads();
    const double ws = sm.w[step];
    best = ArgMax{-1.0, 0x7fffffff};
#pragma unroll
    for (int r = 0; r < kRowsPerThread; ++r) {
      const int64_t i = beg + t + (int64_t)r * blockDim.x;
      if (i < end) {
        double c = 0.0;
        if (r == 0 && regs) {
#pragma unroll
          for (int j = 0; j < kRegK; ++j)
            if (j < k) c = fma(x0[j], sm.xp[j], c);
#pragma unroll
          for (int l = 0; l < kRegK; ++l)
            if (l < step) c = fma(-u0[l], sm.up[l], c);
#pragma unroll
          for (int l = 0; l < kRegK; ++l)
            if (l == step) u0[l] = c;
        } else {
          for (int j = 0; j < k; ++j) c = fma((double)phi[j * ld + i], sm.xp[j], c);
          for (int l = 0; l < step; ++l) c = fma(-__ldcg(&U[(size_t)l * N + i]), sm.up[l], c);
        }
        U[(size_t)step * N + i] = c;
        res[r] = fma(-c * ws, c, res[r]);
        if (i == p) taken[r] = true;
        if (!taken[r] && argmax_better(res[r], (int)i, best.v, best.i)) { best.v = res[r]; best.i = (int)i; }
      }
    }
    best = block_argmax(best, sm.red, sm.redi);
    publish(step + 1, best);
  }

  // ---- feature-guided points: the first n_s - kq candidates that are not
  // QDEIM points (every CTA makes the same choice) ----
  const int ns = A.n_s;
  const int m = ns - kq;
  __syncthreads();
  {
    int off = 0;
    for (int base = 0; base < A.fgs_t && off < m; base += blockDim.x) {
      const int e = base + t;
      int ci = -1;
      if (e < A.fgs_t) {
        ci = __ldcg(&A.fgs_i[e]);
        for (int s = 0; s < kq; ++s) ci = (sm.piv[s] == ci) ? -1 : ci;
      }
      int tot = 0;
      const int pos = off + block_scan_excl(ci >= 0 ? 1 : 0, sm.scan, &tot);
      if (ci >= 0 && pos < m) sm.piv[kq + pos] = ci;
      off += tot;
    }
  }
  __syncthreads();
  if (b == 0)
    for (int s = t; s < ns; s += blockDim.x) A.samples[s] = sm.piv[s];

  // ---- stencil mesh: Phi, q_ref, D on the rows the sampled rows' f needs;
  // sample s by CTA s mod G (threads over its 3 n_var (kMaxR + 2) entries).
  // Burgers: rows i-1, i, i+1 (periodic). Euler, sampled row v nc + i: mesh
  // row 3 c + w is variable w of cell i - 1 + c (ends clamped: the
  // zero-gradient ghost cells) ----
  const int mrows = 3 * A.n_var;
  for (int s = b; s < ns; s += G) {
    const int64_t ic = sm.piv[s];
    for (int e = t; e < mrows * kMeshStride; e += blockDim.x) {
      const int o = e / kMeshStride, j = e % kMeshStride;
      int64_t i;
      if (A.n_var == 1) {
        i = ic + o - 1;
        i = (i < 0) ? i + N : ((i >= N) ? i - N : i);
      } else {
        const int64_t nc = N / 3;
        int64_t c = ic % nc + o / 3 - 1;
        c = (c < 0) ? 0 : ((c >= nc) ? nc - 1 : c);
        i = (int64_t)(o % 3) * nc + c;
      }
      double v;
      if (j < kMaxR) v = (j < k) ? (double)phi[j * ld + i] : 0.0;
      else if (j == kMaxR) v = A.q_ref[i];
      else v = A.drow[i];
      A.mesh[(size_t)(mrows * s + o) * kMeshStride + j] = v;
    }
  }
  if (b != 0) return;

  // ---- CTA 0: (P^T Phi)^+ = (A^T A)^{-1} A^T ----
  for (int e = t; e < ns * k; e += blockDim.x) {
    const int q = e / k, j = e % k;
    X[e] = (double)phi[j * ld + sm.piv[q]];
  }
  __syncthreads();
  // G = A^T A (upper triangle, one warp per entry, lanes over the samples)
  for (int e = wid; e < k * k; e += nw) {
    const int r = e / k, c = e % k;
    if (r > c) continue;
    double s = 0.0;
    for (int q = lane; q < ns; q += 32) s = fma(X[q * k + r], X[q * k + c], s);
    s = warp_sum(s);
    if (lane == 0) { sm.G[r * kMaxR + c] = s; sm.G[c * kMaxR + r] = s; }
  }
  __syncthreads();
  // Gauss-Jordan inversion (no pivoting: A^T A is symmetric positive
  // definite, so every leading pivot is positive), one elimination step per
  // barrier: step c reads Ga and writes Gb, then the two swap
  double* Ga = sm.G;
  double* Gb = sm.G2;
  for (int c = 0; c < k; ++c) {
    if (t < k * k) {
      const double inv = 1.0 / Ga[c * kMaxR + c];
      for (int e = t; e < k * k; e += blockDim.x) {
        const int i = e / k, j = e - i * k;
        const double aij = Ga[i * kMaxR + j], aic = Ga[i * kMaxR + c], acj = Ga[c * kMaxR + j];
        double v;
        if (i == c && j == c) v = inv;
        else if (i == c) v = acj * inv;
        else if (j == c) v = -aic * inv;
        else v = fma(-aic * inv, acj, aij);
        Gb[i * kMaxR + j] = v;
      }
    }
    __syncthreads();
    double* tmp = Ga; Ga = Gb; Gb = tmp;
  }
  // minv (r x n_s, row-major): rows j < k are (A^T A)^{-1} A^T, the rest zero
  for (int e = t; e < A.r * ns; e += blockDim.x) {
    const int j = e / ns, q = e % ns;
    double s = 0.0;
    if (j < k)
      for (int l = 0; l < k; ++l) s = fma(Ga[j * kMaxR + l], X[q * k + l], s);
    A.minv[e] = s;
  }
}

int fgs_list_length(int64_t n, int r, int n_s) {
  int64_t t = (int64_t)n_s + (r < n_s ? r : n_s);
  return (int)(t < n ? t : n);
}

template <typename TPhi>
static cudaError_t launch_sampling_t(const SampleArgs& A, int grid, cudaStream_t s) {
  size_t smem = sizeof(SampleSmem) + sizeof(double) * (size_t)A.n_s * (size_t)A.r;
  cudaError_t e = cudaFuncSetAttribute(sampling_kernel<TPhi>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  SampleArgs a = A;
  void* args[] = {&a};
  return cudaLaunchCooperativeKernel((const void*)sampling_kernel<TPhi>, dim3(grid), dim3(kBlock), args, smem, s);
}

cudaError_t launch_sampling(const SampleArgs& A, int /*km*/, int grid, cudaStream_t s) {
  // each thread keeps the QDEIM norms of at most 4 rows in registers; the
  // feature-guided list must leave n_s - k candidates after the QDEIM points
  if ((A.n + grid - 1) / grid > 4 * kBlock) return cudaErrorInvalidValue;
  if (A.n_s > 256 || A.n_s < A.r || A.r > kMaxR || A.fgs_t > kFgsSort ||
      !(A.n_var == 1 || (A.n_var == 3 && A.n % 3 == 0)) ||
      A.fgs_t < fgs_list_length(A.n, A.r, A.n_s))
    return cudaErrorInvalidValue;
  return A.phi32 ? launch_sampling_t<float>(A, grid, s) : launch_sampling_t<double>(A, grid, s);
}

cudaError_t launch_fgs(const double* y, int64_t n, int n_var, double gamma, int T, unsigned long long* key,
                       double* out_v, int* out_i, bool stage, cudaStream_t s) {
  if (T < 1 || T > kFgsSort || n < 1) return cudaErrorInvalidValue;
  if (!(n_var == 1 || (n_var == 3 && n % 3 == 0))) return cudaErrorInvalidValue;
  const int64_t cells = n / n_var;
  int blocks = (int)((cells + 255) / 256);
  if (blocks > 256) blocks = 256;
  if (n_var == 1) fgs_key_kernel<<<blocks, 256, 0, s>>>(y, n, key);
  else fgs_key_euler_kernel<<<blocks, 256, 0, s>>>(y, cells, gamma, key);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (stage && n <= kFgsStageKeys) {
    const int smem = (int)(sizeof(unsigned long long) * n);
    e = cudaFuncSetAttribute(fgs_select_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(unsigned long long) * kFgsStageKeys));
    if (e != cudaSuccess) return e;
    fgs_select_kernel<true><<<1, kFgsThreads, smem, s>>>(key, n, T, out_v, out_i);
  } else {
    fgs_select_kernel<false><<<1, kFgsThreads, 0, s>>>(key, n, T, out_v, out_i);
  }
  return cudaGetLastError();
}

// Wait bound of this translation unit's kernels (see rom_internal.cuh).
cudaError_t set_wait_limit_sampling(long long cycles) { return set_wait_limit_here(cycles); }

}  // namespace rom
