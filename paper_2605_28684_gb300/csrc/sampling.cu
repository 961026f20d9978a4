// Sampling points of the DEIM-Galerkin model and the sampled-basis operators
// (paper Eq. qdeim_qr, Eq. fgs_selection, Eq. deim_galerkin_rom), as one
// cooperative kernel.
//
//  * QDEIM: the first k pivots of a column-pivoted QR of Phi^T, computed as
//    greedy pivoting on the rows of Phi: take the row with the largest
//    remaining squared norm (ties -> lowest index), append its normalised
//    residual direction (classical Gram-Schmidt twice in R^k) to an
//    orthonormal set, and subtract the squared component along it from every
//    row's remaining norm.
//  * Feature-guided points: the remaining n_s - k points are the cells with
//    the largest squared forward difference (y_{i+1} - y_i)^2 of the
//    correction snapshot (the feature map is the state itself), skipping
//    cells already chosen, ties -> lowest index.
//  * (P^T Phi)^+ = (A^T A)^{-1} A^T with A = P^T Phi (normal equations,
//    Cholesky in FP64) and the stencil mesh (Phi, q_ref, D on the rows
//    i-1, i, i+1 of every sampled cell) used by the hyper-reduced step.
#include <cfloat>
#include <cmath>

#include "rom_internal.cuh"
#include "rom_kernels.cuh"

namespace rom {

namespace {

struct SampleSmem {
  double q[kMaxR * kMaxR];   // orthonormal pivot directions (row j: direction j)
  double v[kMaxR];
  double w[kMaxR];
  double red[64];
  int redi[32];
  double G[kMaxR * kMaxR];   // A^T A and its Cholesky factor
  double gdinv[kMaxR];       // 1 / L_jj
  int piv[kMaxNs];
  long long off;
  double cv[512];
  int ci[512];
  double X[256 * kMaxR];     // (P^T Phi)^+ columns being solved (n_s <= 256)
};

// Bitonic sort (descending value, ascending index) of SIZE (value, index)
// pairs in shared memory, SIZE a power of two <= 2 * blockDim.x.
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

}  // namespace

template <int KM, typename TPhi>
__global__ void __launch_bounds__(kBlock) sampling_kernel(SampleArgs A) {
  const TPhi* phi = basis<TPhi>(A);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SampleSmem& sm = *reinterpret_cast<SampleSmem*>(smem_raw);
  const int G = gridDim.x, b = blockIdx.x, t = threadIdx.x;
  const int64_t N = A.n, ld = A.ld;
  const int64_t beg = (int64_t)b * N / G, end = (int64_t)(b + 1) * N / G;
  const int k = *A.rank;
  const int kq = k < A.n_s ? k : A.n_s;
  const int lane = t & 31;

  // the merge counters (entries appended, CTAs done) are reset here, ahead of
  // the grid barriers that separate this from their first use
  if (b == 0 && t == 0) { A.merge_ctr[0] = 0u; A.merge_ctr[1] = 0u; }
  // ---- initial residual norms and first local argmax ----
  // Each thread owns at most kRowsPerThread rows of this CTA's range and keeps
  // their remaining norms and chosen flags in registers across the pivots.
  constexpr int kRowsPerThread = 4;
  // the first row of every thread is kept in registers across the pivots
  // (bucket size 9; larger buckets reload it)
  constexpr int KC = KM <= 9 ? KM : 1;
  double x0[KC];
#pragma unroll
  for (int j = 0; j < KC; ++j) x0[j] = 0.0;
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
      if (KM <= 9 && r == 0) {
#pragma unroll
        for (int j = 0; j < KC; ++j)
          if (j < k) x0[j] = (double)phi[j * ld + i];
#pragma unroll
        for (int j = 0; j < KC; ++j)
          if (j < k) s = fma(x0[j], x0[j], s);
      } else {
        for (int j = 0; j < k; ++j) { double x = (double)phi[j * ld + i]; s = fma(x, x, s); }
      }
      res[r] = s;
      if (argmax_better(s, (int)i, best.v, best.i)) { best.v = s; best.i = (int)i; }
    }
  }
  best = block_argmax(best, sm.red, sm.redi);
  if (t == 0) { A.cand_v[(size_t)b * kMaxNs] = best.v; A.cand_i[(size_t)b * kMaxNs] = best.i; }
  if (!grid_sync(A.bar, A.status)) return;

  // Candidate slots are double-buffered by step parity, so one grid barrier
  // per pivot suffices: step s reads slot s&1 and writes slot (s+1)&1.
  for (int step = 0; step < kq; ++step) {
    const size_t rd = (size_t)(step & 1), wr = (size_t)((step + 1) & 1);
    // global pivot (every CTA, same fixed-order reduction)
    ArgMax g{-1.0, 0x7fffffff};
    for (int bb = t; bb < G; bb += blockDim.x) {
      double v = __ldcg(&A.cand_v[(size_t)bb * kMaxNs + rd]);
      int i = __ldcg(&A.cand_i[(size_t)bb * kMaxNs + rd]);
      if (argmax_better(v, i, g.v, g.i)) { g.v = v; g.i = i; }
    }
    g = block_argmax(g, sm.red, sm.redi);
    const int p = g.i;
    if (t == 0) sm.piv[step] = p;
    // residual direction of row p against the previous directions: classical
    // Gram-Schmidt twice, by warp 0 alone (lanes over the k entries; no block
    // barriers between the dot products and the updates)
    if (t < 32) {
      for (int j = lane; j < k; j += 32) sm.v[j] = (double)phi[j * ld + p];
      __syncwarp();
      for (int pass = 0; pass < 2; ++pass) {
        for (int l = 0; l < step; ++l) {
          double s = 0.0;
          for (int j = lane; j < k; j += 32) s = fma(sm.v[j], sm.q[l * kMaxR + j], s);
          s = warp_sum(s);
          if (lane == 0) sm.w[l] = s;
        }
        __syncwarp();
        for (int j = lane; j < k; j += 32) {
          double x = sm.v[j];
          for (int l = 0; l < step; ++l) x = fma(-sm.w[l], sm.q[l * kMaxR + j], x);
          sm.v[j] = x;
        }
        __syncwarp();
      }
      double s = 0.0;
      for (int j = lane; j < k; j += 32) s = fma(sm.v[j], sm.v[j], s);
      s = warp_sum(s);
      double inv = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
      for (int j = lane; j < k; j += 32) sm.q[step * kMaxR + j] = sm.v[j] * inv;
    }
    __syncthreads();
    if (step + 1 == kq) break;        // the last pivot needs no further update
    // update residual norms, mark the pivot, next local argmax
    best = ArgMax{-1.0, 0x7fffffff};
#pragma unroll
    for (int r = 0; r < kRowsPerThread; ++r) {
      const int64_t i = beg + t + (int64_t)r * blockDim.x;
      if (i < end) {
        double c = 0.0;
        if (KM <= 9 && r == 0) {
#pragma unroll
          for (int j = 0; j < KC; ++j)
            if (j < k) c = fma(x0[j], sm.q[step * kMaxR + j], c);
        } else {
          for (int j = 0; j < k; ++j) c = fma((double)phi[j * ld + i], sm.q[step * kMaxR + j], c);
        }
        res[r] = fma(-c, c, res[r]);
        if (i == p) taken[r] = true;
        if (!taken[r] && argmax_better(res[r], (int)i, best.v, best.i)) { best.v = res[r]; best.i = (int)i; }
      }
    }
    best = block_argmax(best, sm.red, sm.redi);
    if (t == 0) { A.cand_v[(size_t)b * kMaxNs + wr] = best.v; A.cand_i[(size_t)b * kMaxNs + wr] = best.i; }
    if (!grid_sync(A.bar, A.status)) return;
  }

  // ---- feature-guided points: local top-m by (y_{i+1} - y_i)^2 ----
  // Every CTA sorts its candidates (passes of 256 merged into a running top
  // 256) and publishes its first min(m, 256) entries, their count and its
  // m-th value (-1 if it has fewer than m). CTA 0 then gathers the entries at
  // or above the largest published m-th value, lb: some list holds m
  // entries >= lb, so the global top m are among them.
  const int m = A.n_s - kq;
  if (kq > 0 && !grid_sync(A.bar, A.status)) return;   // all CTAs have read the last slot
  const int mm = m < 256 ? m : 256;
  if (m > 0) {
    for (int e = t; e < 512; e += blockDim.x) { sm.cv[e] = -1.0; sm.ci[e] = 0x7fffffff; }
    __syncthreads();
    const bool one_pass = (end - beg) <= 256;
    for (int64_t base = beg; base < end; base += 256) {
      int64_t i = base + t;
      double sc = -1.0;
      int ii = 0x7fffffff;
      if (i < end) {
        bool ch = false;
        for (int s = 0; s < kq; ++s) ch = ch || (sm.piv[s] == (int)i);
        if (!ch) {
          double dy = A.y[(i + 1) % N] - A.y[i];
          sc = dy * dy;
          ii = (int)i;
        }
      }
      if (one_pass) {
        sm.cv[t] = sc;
        sm.ci[t] = ii;
        block_sort<256>(sm.cv, sm.ci);
      } else {
        sm.cv[256 + t] = sc;
        sm.ci[256 + t] = ii;
        block_sort<512>(sm.cv, sm.ci);      // top 256 end up in [0, 256)
      }
    }
    int cnt = 0;                            // valid (non-negative) entries among the first mm
    for (int e = t; e < mm; e += blockDim.x) {
      A.cand_v[(size_t)b * kMaxNs + e] = sm.cv[e];
      A.cand_i[(size_t)b * kMaxNs + e] = sm.ci[e];
      cnt += (sm.cv[e] >= 0.0) ? 1 : 0;
    }
    cnt = (int)block_sum((double)cnt, sm.red);
    if (t == 0) {
      A.chosen[b] = cnt;
      A.resid[b] = (cnt >= m) ? sm.cv[m - 1] : -1.0;
    }
  }
  if (!grid_sync(A.bar, A.status)) return;

  // ---- top-m of the G sorted candidate lists ----
  // Every CTA finds lb (the largest published m-th value) and appends its own
  // entries >= lb to one compact array (some list holds m such entries, so
  // the global top m are among them; the order of appending does not matter:
  // CTA 0 sorts them by value, then index). CTA 0 waits for the G appends
  // (a bounded wait), sorts and keeps the first m.
  if (m > 0) {
    double lb = -1.0;
    for (int bb = t; bb < G; bb += blockDim.x) lb = fmax(lb, __ldcg(&A.resid[bb]));
    lb = block_max(lb, sm.red);
    int c = 0;                               // this CTA's entries >= lb (a prefix: sorted)
    for (int e = t; e < mm; e += blockDim.x) c += (sm.cv[e] >= lb && sm.cv[e] >= 0.0) ? 1 : 0;
    c = (int)block_sum((double)c, sm.red);
    if (t == 0) sm.off = (c > 0) ? (long long)atomicAdd(&A.merge_ctr[0], (unsigned int)c) : 0;
    __syncthreads();
    const long long off = sm.off;
    for (int e = t; e < c; e += blockDim.x) {
      A.merge_v[off + e] = sm.cv[e];
      A.merge_i[off + e] = sm.ci[e];
    }
    __threadfence();
    __syncthreads();
    if (t == 0) atomicAdd(&A.merge_ctr[1], 1u);
  }
  if (b != 0) return;
  if (m > 0) {
    __shared__ int s_ok;
    if (t == 0) {
      const volatile unsigned int* done = &A.merge_ctr[1];
      const long long limit = c_wait_limit;
      const long long t0 = clock64();
      int ok = 1;
      while (*done < (unsigned int)G) {
        if (clock64() - t0 > limit) {
          record_status(A.status, kStTimeout);
          ok = 0;
          break;
        }
      }
      __threadfence();
      s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) return;
    const int total = (int)__ldcg(&A.merge_ctr[0]);
    if (total <= 512) {
      for (int e = t; e < 512; e += blockDim.x) {
        sm.cv[e] = (e < total) ? __ldcg(&A.merge_v[e]) : -1.0;
        sm.ci[e] = (e < total) ? __ldcg(&A.merge_i[e]) : 0x7fffffff;
      }
      if (total <= 128) block_sort<128>(sm.cv, sm.ci);
      else if (total <= 256) block_sort<256>(sm.cv, sm.ci);
      else block_sort<512>(sm.cv, sm.ci);
      __syncthreads();
      for (int e = t; e < m; e += blockDim.x) sm.piv[kq + e] = sm.ci[e];
    } else {
      // more than 512 entries at or above lb: merge the lists one pick at a time
      __shared__ int head[1024];
      for (int bb = t; bb < G; bb += blockDim.x) head[bb] = 0;
      __syncthreads();
      for (int s = 0; s < m; ++s) {
        ArgMax g{-2.0, 0x7fffffff};
        int gb = -1;
        for (int bb = t; bb < G; bb += blockDim.x) {
          int h = head[bb];
          if (h < __ldcg(&A.chosen[bb])) {
            double v = A.cand_v[(size_t)bb * kMaxNs + h];
            int i = A.cand_i[(size_t)bb * kMaxNs + h];
            if (argmax_better(v, i, g.v, g.i)) { g.v = v; g.i = i; }
          }
        }
        g = block_argmax(g, sm.red, sm.redi);
        for (int bb = t; bb < G; bb += blockDim.x) {
          int h = head[bb];
          if (h < __ldcg(&A.chosen[bb]) && A.cand_i[(size_t)bb * kMaxNs + h] == g.i) gb = bb;
        }
        __syncthreads();
        if (gb >= 0) head[gb] += 1;
        if (t == 0) sm.piv[kq + s] = g.i;
        __syncthreads();
      }
    }
  }
  __syncthreads();
  const int ns = A.n_s;
  for (int s = t; s < ns; s += blockDim.x) A.samples[s] = sm.piv[s];

  // ---- stencil mesh: Phi, q_ref, D on rows i-1, i, i+1 of every sample ----
  // a warp takes kSpw samples per pass and issues all their loads (lanes over
  // the kMaxR basis entries of the three rows; lanes 0..2 q_ref and D) before
  // any store; the basis rows of the samples themselves (o = 1) are also
  // staged in shared memory (X) for the Gram matrix
  double* Ps = sm.X;                       // ns x k (row-major), rows of P^T Phi
  {
    constexpr int kSpw = 2;
    const int wid = t >> 5, nw = blockDim.x >> 5;
    for (int s0 = wid * kSpw; s0 < ns; s0 += nw * kSpw) {
      double v[kSpw][2][3], qv[kSpw], dv[kSpw];
#pragma unroll
      for (int u = 0; u < kSpw; ++u) {
        const int sidx = s0 + u;
        const bool ok = sidx < ns;
        const int64_t ic = ok ? (int64_t)sm.piv[sidx] : 0;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int j = lane + 32 * h;
#pragma unroll
          for (int o = 0; o < 3; ++o) {
            const int64_t i = (ic + (o - 1) + N) % N;
            v[u][h][o] = (ok && j < k) ? (double)phi[j * ld + i] : 0.0;
          }
        }
        const int64_t il = (ic + ((lane < 3 ? lane : 1) - 1) + N) % N;
        qv[u] = (ok && lane < 3) ? A.q_ref[il] : 0.0;
        dv[u] = (ok && lane < 3) ? A.drow[il] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < kSpw; ++u) {
        const int sidx = s0 + u;
        if (sidx >= ns) continue;
#pragma unroll
        for (int o = 0; o < 3; ++o) {
          double* row = A.mesh + (size_t)(3 * sidx + o) * kMeshStride;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int j = lane + 32 * h;
            if (j < kMaxR) row[j] = v[u][h][o];
            if (o == 1 && j < k) Ps[sidx * k + j] = v[u][h][o];
          }
        }
        if (lane < 3) {
          double* row = A.mesh + (size_t)(3 * sidx + lane) * kMeshStride;
          row[kMaxR] = qv[u];
          row[kMaxR + 1] = dv[u];
        }
      }
    }
  }
  __syncthreads();
  // ---- G = A^T A with A = P^T Phi (k x k), FP64: one warp per entry ----
  {
    const int wid = t >> 5, nw = blockDim.x >> 5;
    for (int e = wid; e < k * k; e += nw) {
      int r = e / k, c = e % k;
      double s = 0.0;
      for (int q = lane; q < ns; q += 32) s = fma(Ps[q * k + r], Ps[q * k + c], s);
      s = warp_sum(s);
      if (lane == 0) sm.G[r * kMaxR + c] = s;
    }
  }
  __syncthreads();
  // Cholesky (lower) by warp 0, one column at a time
  if (t < 32) {
    for (int j = 0; j < k; ++j) {
      double s = 0.0;
      for (int l = lane; l < j; l += 32) s += sm.G[j * kMaxR + l] * sm.G[j * kMaxR + l];
      s = warp_sum(s);
      if (lane == 0) {
        const double djj = sqrt(fmax(sm.G[j * kMaxR + j] - s, DBL_MIN));
        sm.G[j * kMaxR + j] = djj;
        sm.gdinv[j] = 1.0 / djj;       // one FP64 division per column
      }
      __syncwarp();
      const double rj = sm.gdinv[j];
      for (int i = j + 1 + lane; i < k; i += 32) {
        double v = sm.G[i * kMaxR + j];
        for (int l = 0; l < j; ++l) v -= sm.G[i * kMaxR + l] * sm.G[j * kMaxR + l];
        sm.G[i * kMaxR + j] = v * rj;
      }
      __syncwarp();
    }
  }
  __syncthreads();
  // M = G^{-1} A^T: each sample column q solves L L^T x = A(q, :)^T; the
  // solution overwrites the staged row q in shared memory
  for (int q = t; q < ns; q += blockDim.x) {
    double* x = Ps + q * k;
    for (int i = 0; i < k; ++i) {
      double s = x[i];
      for (int l = 0; l < i; ++l) s -= sm.G[i * kMaxR + l] * x[l];
      x[i] = s * sm.gdinv[i];
    }
    for (int i = k - 1; i >= 0; --i) {
      double s = x[i];
      for (int l = i + 1; l < k; ++l) s -= sm.G[l * kMaxR + i] * x[l];
      x[i] = s * sm.gdinv[i];
    }
  }
  __syncthreads();
  for (int e = t; e < A.r * ns; e += blockDim.x) {
    int i = e / ns, q = e % ns;
    A.minv[e] = (i < k) ? Ps[q * k + i] : 0.0;
  }
}

template <int KM, typename TPhi>
static cudaError_t launch_sampling_tt(const SampleArgs& A, int grid, cudaStream_t s) {
  size_t smem = sizeof(SampleSmem);
  cudaError_t e = cudaFuncSetAttribute(sampling_kernel<KM, TPhi>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  SampleArgs a = A;
  void* args[] = {&a};
  return cudaLaunchCooperativeKernel((const void*)sampling_kernel<KM, TPhi>, dim3(grid),
                                     dim3(kBlock), args, smem, s);
}

template <int KM>
static cudaError_t launch_sampling_t(const SampleArgs& A, int grid, cudaStream_t s) {
  return A.phi32 ? launch_sampling_tt<KM, float>(A, grid, s) : launch_sampling_tt<KM, double>(A, grid, s);
}

cudaError_t launch_sampling(const SampleArgs& A, int km, int grid, cudaStream_t s) {
  // each thread keeps the QDEIM norms of at most 4 rows in registers
  if ((A.n + grid - 1) / grid > 4 * kBlock) return cudaErrorInvalidValue;
  switch (km) {
    case 9: return launch_sampling_t<9>(A, grid, s);
    case 17: return launch_sampling_t<17>(A, grid, s);
    case 33: return launch_sampling_t<33>(A, grid, s);
    default: return launch_sampling_t<65>(A, grid, s);
  }
}

// Wait bound of this translation unit's kernels (see rom_internal.cuh).
cudaError_t set_wait_limit_sampling(long long cycles) { return set_wait_limit_here(cycles); }

}  // namespace rom
