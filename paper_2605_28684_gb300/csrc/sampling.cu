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
  int piv[kMaxNs];
  double cv[512];
  int ci[512];
  double X[256 * kMaxR];     // (P^T Phi)^+ columns being solved (n_s <= 256)
};

// Bitonic sort (descending value, ascending index) of 512 (value, index) pairs.
__device__ void block_sort512(double* v, int* idx) {
  for (int size = 2; size <= 512; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      __syncthreads();
      for (int t = threadIdx.x; t < 256; t += blockDim.x) {
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

  // ---- initial residual norms and first local argmax ----
  // Each thread owns at most kRowsPerThread rows of this CTA's range and keeps
  // their remaining norms and chosen flags in registers across the pivots.
  constexpr int kRowsPerThread = 4;
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
      for (int j = 0; j < k; ++j) { double x = (double)phi[j * ld + i]; s = fma(x, x, s); }
      res[r] = s;
      if (argmax_better(s, (int)i, best.v, best.i)) { best.v = s; best.i = (int)i; }
    }
  }
  best = block_argmax(best, sm.red, sm.redi);
  if (t == 0) { A.cand_v[(size_t)b * kMaxNs] = best.v; A.cand_i[(size_t)b * kMaxNs] = best.i; }
  if (!grid_sync(A.bar, A.status)) return;

  // Candidate slots are double-buffered by step parity, so one grid barrier
  // per pivot suffices: step s reads slot s&1 and writes slot (s+1)&1.
  const int wid = t >> 5, nwarp = blockDim.x >> 5;
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
    // Gram-Schmidt twice, the dot products of one pass computed by all warps
    for (int j = t; j < k; j += blockDim.x) sm.v[j] = (double)phi[j * ld + p];
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass) {
      for (int l = wid; l < step; l += nwarp) {
        double s = 0.0;
        for (int j = lane; j < k; j += 32) s = fma(sm.v[j], sm.q[l * kMaxR + j], s);
        s = warp_sum(s);
        if (lane == 0) sm.w[l] = s;
      }
      __syncthreads();
      for (int j = t; j < k; j += blockDim.x) {
        double x = sm.v[j];
        for (int l = 0; l < step; ++l) x = fma(-sm.w[l], sm.q[l * kMaxR + j], x);
        sm.v[j] = x;
      }
      __syncthreads();
    }
    if (t < 32) {
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
        for (int j = 0; j < k; ++j) c = fma((double)phi[j * ld + i], sm.q[step * kMaxR + j], c);
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
  const int m = A.n_s - kq;
  if (kq > 0 && !grid_sync(A.bar, A.status)) return;   // all CTAs have read the last slot
  if (m > 0) {
    for (int e = t; e < 512; e += blockDim.x) { sm.cv[e] = -1.0; sm.ci[e] = 0x7fffffff; }
    __syncthreads();
    // rows of this CTA in passes of 256 candidates merged with the current top
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
      sm.cv[256 + t] = sc;
      sm.ci[256 + t] = ii;
      block_sort512(sm.cv, sm.ci);      // top 256 end up in [0, 256)
    }
    const int mm = m < 256 ? m : 256;
    for (int e = t; e < mm; e += blockDim.x) {
      A.cand_v[(size_t)b * kMaxNs + e] = sm.cv[e];
      A.cand_i[(size_t)b * kMaxNs + e] = sm.ci[e];
    }
  }
  if (!grid_sync(A.bar, A.status)) return;
  if (b != 0) return;

  // ---- CTA 0: top-m of the G sorted candidate lists ----
  // lb = max over lists of their m-th entry: some list holds m entries >= lb,
  // so nothing below lb can be in the top m. The entries >= lb are gathered
  // and sorted in shared memory; if there are more than 512 of them the lists
  // are merged one pick at a time instead.
  if (m > 0) {
    __shared__ int s_len[1024];
    __shared__ int s_cnt[1024];
    __shared__ int s_off[1025];
    const int mm = m < 256 ? m : 256;
    double lb = -1.0;
    for (int bb = t; bb < G; bb += blockDim.x) {
      const double* lv = A.cand_v + (size_t)bb * kMaxNs;
      int lo = 0, hi = mm;                       // valid entries have value >= 0
      while (lo < hi) { int mid = (lo + hi) >> 1; if (__ldcg(lv + mid) >= 0.0) lo = mid + 1; else hi = mid; }
      s_len[bb] = lo;
      if (lo >= m) lb = fmax(lb, __ldcg(lv + m - 1));
    }
    lb = block_max(lb, sm.red);
    for (int bb = t; bb < G; bb += blockDim.x) {
      const double* lv = A.cand_v + (size_t)bb * kMaxNs;
      int lo = 0, hi = s_len[bb];
      while (lo < hi) { int mid = (lo + hi) >> 1; if (__ldcg(lv + mid) >= lb) lo = mid + 1; else hi = mid; }
      s_cnt[bb] = lo;
    }
    __syncthreads();
    if (t == 0) {
      int o = 0;
      for (int bb = 0; bb < G; ++bb) { s_off[bb] = o; o += s_cnt[bb]; }
      s_off[G] = o;
    }
    __syncthreads();
    const int total = s_off[G];
    if (total <= 512) {
      for (int e = t; e < 512; e += blockDim.x) { sm.cv[e] = -1.0; sm.ci[e] = 0x7fffffff; }
      __syncthreads();
      for (int bb = t; bb < G; bb += blockDim.x) {
        const int o = s_off[bb], c = s_cnt[bb];
#pragma unroll 4
        for (int e = 0; e < c; ++e) {
          sm.cv[o + e] = __ldcg(A.cand_v + (size_t)bb * kMaxNs + e);
          sm.ci[o + e] = __ldcg(A.cand_i + (size_t)bb * kMaxNs + e);
        }
      }
      block_sort512(sm.cv, sm.ci);
      for (int e = t; e < m; e += blockDim.x) sm.piv[kq + e] = sm.ci[e];
    } else {
      __shared__ int head[1024];
      for (int bb = t; bb < G; bb += blockDim.x) head[bb] = 0;
      __syncthreads();
      for (int s = 0; s < m; ++s) {
        ArgMax g{-2.0, 0x7fffffff};
        int gb = -1;
        for (int bb = t; bb < G; bb += blockDim.x) {
          int h = head[bb];
          if (h < s_len[bb]) {
            double v = A.cand_v[(size_t)bb * kMaxNs + h];
            int i = A.cand_i[(size_t)bb * kMaxNs + h];
            if (argmax_better(v, i, g.v, g.i)) { g.v = v; g.i = i; }
          }
        }
        g = block_argmax(g, sm.red, sm.redi);
        for (int bb = t; bb < G; bb += blockDim.x) {
          int h = head[bb];
          if (h < s_len[bb] && A.cand_i[(size_t)bb * kMaxNs + h] == g.i) gb = bb;
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
  for (int e = t; e < ns * 3; e += blockDim.x) {
    int s = e / 3, o = e % 3;
    int64_t i = ((int64_t)sm.piv[s] + (o - 1) + N) % N;
    double* row = A.mesh + (size_t)e * kMeshStride;
    for (int j = 0; j < kMaxR; ++j) row[j] = (j < k) ? (double)phi[j * ld + i] : 0.0;
    row[kMaxR] = A.q_ref[i];
    row[kMaxR + 1] = A.drow[i];
  }
  __syncthreads();
  // ---- G = A^T A with A = P^T Phi (k x k), FP64: one warp per entry ----
  {
    const int wid = t >> 5, nw = blockDim.x >> 5;
    for (int e = wid; e < k * k; e += nw) {
      int r = e / k, c = e % k;
      double s = 0.0;
      for (int q = lane; q < ns; q += 32)
        s = fma(A.mesh[(size_t)(3 * q + 1) * kMeshStride + r], A.mesh[(size_t)(3 * q + 1) * kMeshStride + c], s);
      s = warp_sum(s);
      if (lane == 0) sm.G[r * kMaxR + c] = s;
    }
  }
  __syncthreads();
  // Cholesky (lower), one column at a time
  for (int j = 0; j < k; ++j) {
    if (t < 32) {
      double s = 0.0;
      for (int l = lane; l < j; l += 32) s += sm.G[j * kMaxR + l] * sm.G[j * kMaxR + l];
      s = warp_sum(s);
      if (lane == 0) sm.G[j * kMaxR + j] = sqrt(fmax(sm.G[j * kMaxR + j] - s, DBL_MIN));
    }
    __syncthreads();
    for (int i = j + 1 + t; i < k; i += blockDim.x) {
      double s = sm.G[i * kMaxR + j];
      for (int l = 0; l < j; ++l) s -= sm.G[i * kMaxR + l] * sm.G[j * kMaxR + l];
      sm.G[i * kMaxR + j] = s / sm.G[j * kMaxR + j];
    }
    __syncthreads();
  }
  // M = G^{-1} A^T: each sample column q solves L L^T x = A(q, :)^T, with x in
  // shared memory (X[q * k + i])
  double* X = sm.X;
  for (int q = t; q < ns; q += blockDim.x) {
    for (int i = 0; i < k; ++i) {
      double s = A.mesh[(size_t)(3 * q + 1) * kMeshStride + i];
      for (int l = 0; l < i; ++l) s -= sm.G[i * kMaxR + l] * X[q * k + l];
      X[q * k + i] = s / sm.G[i * kMaxR + i];
    }
    for (int i = k - 1; i >= 0; --i) {
      double s = X[q * k + i];
      for (int l = i + 1; l < k; ++l) s -= sm.G[l * kMaxR + i] * X[q * k + l];
      X[q * k + i] = s / sm.G[i * kMaxR + i];
    }
  }
  __syncthreads();
  for (int e = t; e < A.r * ns; e += blockDim.x) {
    int i = e / ns, q = e % ns;
    A.minv[e] = (i < k) ? X[q * k + i] : 0.0;
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
