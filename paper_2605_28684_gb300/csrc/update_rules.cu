// Comparison basis-update rules of the paper (App. A) on the window of
// preprocessed correction snapshots: windowed SVD (Eqs. wsvd_window_matrix,
// wsvd_update) and the Direct method (Eqs. direct_optimization,
// direct_update). The host side (api.cu) drives them with the iSVD kernel in
// its rank-growing mode (forgetting factor 1), which reproduces the thin SVD
// of a column sequence:
//  * windowed SVD: an empty basis, the w window columns fed oldest first,
//    then the truncation to r at the rank tolerance (this file: the window
//    fill and the truncation);
//  * Direct: C = Phi^T Y (r x w), its right singular vectors V_c of the
//    singular values above the rank tolerance by one-sided Jacobi on C^T
//    (one CTA, FP64), then an orthonormal basis of span(Y V_c) =
//    span(Y (Phi^+ Y)^+) by the growing iSVD over the columns of Y V_c.
#include <cfloat>
#include <cmath>

#include "rom_internal.cuh"
#include "rom_kernels.cuh"

namespace rom {

namespace {

// win[:, j] = D (Q[:, j] - q_ref) for j < count
__global__ void win_fill_kernel(const double* Q, int64_t ldq, const double* q_ref, const double* drow,
                                int64_t n, int count, double* win) {
  const int64_t tot = n * (int64_t)count;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / n, i = e % n;
    win[j * n + i] = drow[i] * (Q[j * ldq + i] - q_ref[i]);
  }
}

// rank <- #{j < min(r, rank): sigma_j > tol sigma_0}; sigma_j <- 0 beyond it
__global__ void trunc_kernel(double* sigma, int* rank, int r, double tol) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const int k0 = *rank < r ? *rank : r;
    int k = 0;
    const double s0 = k0 > 0 ? sigma[0] : 0.0;
    for (int j = 0; j < k0; ++j)
      if (s0 > 0.0 && sigma[j] > tol * s0) ++k;
    for (int j = k; j <= kMaxR; ++j) sigma[j] = 0.0;
    *rank = k;
  }
}

// Phi[:, j] <- 0 for rank <= j < ncols
__global__ void zero_cols_kernel(double* phi, int64_t n, const int* rank, int ncols) {
  const int k = *rank;
  const int64_t tot = n * (int64_t)(ncols > k ? ncols - k : 0);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x)
    phi[(int64_t)k * n + e] = 0.0;
}

// One CTA: one-sided Jacobi on the k live rows of C (r x w, row-major), i.e.
// on the columns of C^T, until every pair is orthogonal to 1e-15; then the
// normalised rows sorted by norm are the right singular vectors of C. Writes
// Vc (w x kc, row-major, the kc vectors with singular value above tol times
// the largest), s (kc values, descending) and kc.
__global__ void __launch_bounds__(256) direct_small_kernel(const double* C, int r, int w, const int* rank,
                                                           double tol, double* Vc, double* s_out,
                                                           int* kc_out) {
  __shared__ double X[kMaxR * kMaxR];     // row j: vector j (length w <= kMaxR)
  __shared__ double nrm[kMaxR];
  __shared__ int order[kMaxR];
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5, nw = blockDim.x >> 5;
  const int k = *rank < r ? *rank : r;
  for (int e = t; e < k * w; e += blockDim.x) {
    const int j = e / w, c = e % w;
    X[j * kMaxR + c] = C[j * w + c];
  }
  __syncthreads();
  // cyclic-by-rows sweeps over the pairs (p, q) on warp 0 (lanes over the
  // vector length), at most 40 sweeps
  if (wid == 0) {
    for (int sweep = 0; sweep < 40 && k > 1; ++sweep) {
      bool rotated = false;
      for (int p = 0; p < k - 1; ++p)
        for (int q = p + 1; q < k; ++q) {
          double al = 0.0, be = 0.0, ga = 0.0;
          for (int c = lane; c < w; c += 32) {
            const double xp = X[p * kMaxR + c], xq = X[q * kMaxR + c];
            al = fma(xp, xp, al);
            be = fma(xq, xq, be);
            ga = fma(xp, xq, ga);
          }
          al = warp_sum(al);
          be = warp_sum(be);
          ga = warp_sum(ga);
          if (al > 0.0 && be > 0.0 && fabs(ga) > 1e-15 * sqrt(al * be)) {
            const double zeta = (be - al) / (2.0 * ga);
            const double tt = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
            const double cs = 1.0 / sqrt(1.0 + tt * tt), sn = cs * tt;
            for (int c = lane; c < w; c += 32) {
              const double xp = X[p * kMaxR + c], xq = X[q * kMaxR + c];
              X[p * kMaxR + c] = cs * xp - sn * xq;
              X[q * kMaxR + c] = sn * xp + cs * xq;
            }
            rotated = true;
          }
          __syncwarp();
        }
      if (!rotated) break;
    }
  }
  __syncthreads();
  for (int j = wid; j < k; j += nw) {
    double s2 = 0.0;
    for (int c = lane; c < w; c += 32) s2 = fma(X[j * kMaxR + c], X[j * kMaxR + c], s2);
    s2 = warp_sum(s2);
    if (lane == 0) nrm[j] = sqrt(s2);
  }
  __syncthreads();
  if (t == 0) {
    for (int j = 0; j < k; ++j) order[j] = j;
    for (int i = 1; i < k; ++i)            // insertion sort, descending, stable
      for (int j = i; j > 0 && nrm[order[j]] > nrm[order[j - 1]]; --j) {
        const int tmp = order[j]; order[j] = order[j - 1]; order[j - 1] = tmp;
      }
    int kc = 0;
    const double smax = k > 0 ? nrm[order[0]] : 0.0;
    for (int j = 0; j < k; ++j)
      if (smax > 0.0 && nrm[order[j]] > tol * smax) ++kc;
    *kc_out = kc;
    for (int j = 0; j < kc; ++j) s_out[j] = nrm[order[j]];
  }
  __syncthreads();
  const int kc = *kc_out;
  for (int e = t; e < w * kc; e += blockDim.x) {
    const int c = e / kc, j = e % kc;
    const int src = order[j];
    Vc[e] = X[src * kMaxR + c] / nrm[src];
  }
}

// sigma[0:k] <- s, zero beyond; rank <- k = min(kc, rank of the grown basis)
__global__ void set_sigma_kernel(const double* s, const int* kc, double* sigma, int* rank) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const int k = *kc < *rank ? *kc : *rank;
    for (int j = 0; j <= kMaxR; ++j) sigma[j] = (j < k) ? s[j] : 0.0;
    *rank = k;
  }
}

}  // namespace

cudaError_t launch_win_fill(const double* Q, int64_t ldq, const double* q_ref, const double* drow, int64_t n,
                            int count, double* win, cudaStream_t s) {
  win_fill_kernel<<<512, 256, 0, s>>>(Q, ldq, q_ref, drow, n, count, win);
  return cudaGetLastError();
}

cudaError_t launch_truncate(double* phi, int64_t n, double* sigma, int* rank, int r, int ncols, double tol,
                            cudaStream_t s) {
  trunc_kernel<<<1, 32, 0, s>>>(sigma, rank, r, tol);
  zero_cols_kernel<<<512, 256, 0, s>>>(phi, n, rank, ncols);
  return cudaGetLastError();
}

cudaError_t launch_direct_small(const double* C, int r, int w, const int* rank, double tol, double* Vc,
                                double* s_out, int* kc, cudaStream_t s) {
  if (r > kMaxR || w > kMaxR || w < 1) return cudaErrorInvalidValue;
  direct_small_kernel<<<1, 256, 0, s>>>(C, r, w, rank, tol, Vc, s_out, kc);
  return cudaGetLastError();
}

cudaError_t launch_set_sigma(const double* s_in, const int* kc, double* sigma, int* rank, cudaStream_t s) {
  set_sigma_kernel<<<1, 32, 0, s>>>(s_in, kc, sigma, rank);
  return cudaGetLastError();
}

}  // namespace rom
