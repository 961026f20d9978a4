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
//    span(Y (Phi^+ Y)^+) by the growing iSVD over the columns of Y V_c;
// and the instantaneous rules on the live columns of the basis (one-step,
// Oja, GROUSE: Eqs. onestep_update, oja_update, grouse_projection,
// grouse_update), all of the form Phi <- Phi + u v^T with
// u = c_y yhat + c_r r + Phi g, then (one-step, Oja) orthonormalisation by
// CholQR: G = Phi^T Phi, Phi <- Phi R^-1 with G = R^T R (FP64).
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

// Coefficients of the rank-one update of an instantaneous rule (one thread):
// in: w1 = Phi^T yhat, w2 = Phi^T q1 (GROUSE's second Gram-Schmidt pass),
// a (reduced state), rr = |r|^2; out: coef = (c_y, c_r), g (k), v (k).
__global__ void instant_coef_kernel(int rule, const int* rank, int r, double eta, const double* w1,
                                    const double* w2, const double* a, const double* rr, double* coef,
                                    double* g, double* v) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int k = *rank < r ? *rank : r;
  double cy = 0.0, cr = 0.0;
  for (int j = 0; j < k; ++j) { g[j] = 0.0; v[j] = 0.0; }
  if (rule == ROM_UPDATE_ONESTEP) {             // u = yhat - Phi a, v = a / |a|^2
    double nn = 0.0;
    for (int j = 0; j < k; ++j) nn = fma(a[j], a[j], nn);
    if (nn > 0.0) {
      cy = 1.0;
      for (int j = 0; j < k; ++j) { g[j] = -a[j]; v[j] = a[j] / nn; }
    }
  } else if (rule == ROM_UPDATE_OJA) {          // u = eta yhat, v = Phi^T yhat
    cy = eta;
    for (int j = 0; j < k; ++j) v[j] = w1[j];
  } else {                                      // GROUSE
    double ww = 0.0;
    for (int j = 0; j < k; ++j) { const double wj = w1[j] + w2[j]; ww = fma(wj, wj, ww); }
    const double np = sqrt(ww), nr = sqrt(*rr);  // |p| = |Phi w| = |w| for orthonormal Phi
    if (np > 0.0 && nr > 0.0) {
      const double al = eta * np * nr;
      cr = sin(al) / nr;
      const double cw = (cos(al) - 1.0) / np;   // u = cw Phi w + cr r, v = w / |w|
      for (int j = 0; j < k; ++j) {
        const double wj = w1[j] + w2[j];
        g[j] = cw * wj;
        v[j] = wj / np;
      }
    }
  }
  coef[0] = cy;
  coef[1] = cr;
}

// Phi[i, j] += u_i v_j (j < k) with u_i = c_y yhat_i + c_r res_i + sum_l Phi[i, l] g_l;
// each row is read whole before it is written, so the update is in place.
__global__ void rank1_update_kernel(double* phi, int64_t n, const int* rank, int r, const double* yhat,
                                    const double* res, const double* coef, const double* g, const double* v) {
  const int k = *rank < r ? *rank : r;
  __shared__ double sg[kMaxR], sv[kMaxR];
  for (int j = threadIdx.x; j < k; j += blockDim.x) { sg[j] = g[j]; sv[j] = v[j]; }
  __syncthreads();
  const double cy = coef[0], cr = coef[1];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double u = cy * yhat[i];
    if (cr != 0.0) u = fma(cr, res[i], u);
    for (int l = 0; l < k; ++l) u = fma(phi[l * n + i], sg[l], u);
    for (int j = 0; j < k; ++j) phi[j * n + i] = fma(u, sv[j], phi[j * n + i]);
  }
}

// R^-1 (k x k upper triangular, row-major, ld kMaxR) of the Cholesky factor
// G = R^T R of the Gram matrix G (k x k row-major, ld k), by one warp: the
// factor row by row (lanes over the row), then the inverse column by column
// (lane j back-substitutes column j).
__global__ void chol_inv_kernel(const double* G, const int* rank, int r, double* Rinv) {
  __shared__ double R[kMaxR * kMaxR];
  const int k = *rank < r ? *rank : r;
  const int lane = threadIdx.x;
  for (int e = lane; e < kMaxR * kMaxR; e += 32) R[e] = 0.0;
  __syncwarp();
  for (int c = 0; c < k; ++c) {
    double s = 0.0;
    for (int l = lane; l < c; l += 32) s = fma(R[l * kMaxR + c], R[l * kMaxR + c], s);
    s = warp_sum(s);
    const double d = sqrt(fmax(G[c * k + c] - s, DBL_MIN));
    const double id = 1.0 / d;
    for (int j = c + 1 + lane; j < k; j += 32) {
      double x = G[c * k + j];
      for (int l = 0; l < c; ++l) x = fma(-R[l * kMaxR + c], R[l * kMaxR + j], x);
      R[c * kMaxR + j] = x * id;
    }
    if (lane == 0) R[c * kMaxR + c] = d;
    __syncwarp();
  }
  for (int j = lane; j < k; j += 32) {
    for (int i = j; i >= 0; --i) {
      double x = (i == j) ? 1.0 : 0.0;
      for (int l = i + 1; l <= j; ++l) x = fma(-R[i * kMaxR + l], Rinv[l * kMaxR + j], x);
      Rinv[i * kMaxR + j] = x / R[i * kMaxR + i];
    }
    for (int i = j + 1; i < k; ++i) Rinv[i * kMaxR + j] = 0.0;
  }
}

}  // namespace

cudaError_t launch_instant_coef(int rule, const int* rank, int r, double eta, const double* w1, const double* w2,
                                const double* a, const double* rr, double* coef, double* g, double* v,
                                cudaStream_t s) {
  instant_coef_kernel<<<1, 32, 0, s>>>(rule, rank, r, eta, w1, w2, a, rr, coef, g, v);
  return cudaGetLastError();
}

cudaError_t launch_rank1_update(double* phi, int64_t n, const int* rank, int r, const double* yhat,
                                const double* res, const double* coef, const double* g, const double* v,
                                cudaStream_t s) {
  int blocks = (int)((n + 255) / 256);
  if (blocks > 1024) blocks = 1024;
  rank1_update_kernel<<<blocks, 256, 0, s>>>(phi, n, rank, r, yhat, res, coef, g, v);
  return cudaGetLastError();
}

cudaError_t launch_chol_inv(const double* G, const int* rank, int r, double* Rinv, cudaStream_t s) {
  chol_inv_kernel<<<1, 32, 0, s>>>(G, rank, r, Rinv);
  return cudaGetLastError();
}

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
