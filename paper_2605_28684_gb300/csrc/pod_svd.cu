// Thin SVD of the training matrix X = D (Q_train - q_ref 1^T) (N x w), for the
// gradient pass (Sec. 3.1: the POD is the leading left singular vectors of
// X). The gradient divides by gaps of the POD's singular values, so its basis
// must be fixed to rounding level, as a backward-stable SVD fixes it: the
// rank-growing iSVD of the plain forward path drops content below 1e-13 s_1
// while it grows, which moves the smallest kept vector by ~1e-12 s_1 / gap.
//
//  1. X = Q R by classical Gram-Schmidt applied twice, column by column
//     (the products with Q run on the tall-skinny kernels of adjoint.cu); a
//     column whose second residual is below 1e-14 of its norm is numerically
//     in the span and is dropped (zero column of Q, zero row of R).
//  2. R = U_R S V_R^T by one-sided Jacobi on the columns of R (one CTA, FP64,
//     round-robin order of disjoint pairs, one warp per pair), which resolves
//     the small singular values to high relative accuracy.
//  3. U = Q U_R (on the caller's side); V = the accumulated rotations when
//     asked for (the gradient pass needs every triplet).
#include <cfloat>
#include <cmath>

#include "rom_internal.cuh"
#include "rom_kernels.cuh"

namespace rom {

namespace {

// R_jj from the squared norms of the current residual and of the original
// column; scale = 1 / R_jj, or 0 when the column is numerically in the span.
__global__ void qr_diag_kernel(const double* nrm2_now, const double* nrm2_orig, double* Rjj, double* scale) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const double a = *nrm2_now, b = *nrm2_orig;
    const bool keep = a > 1e-28 * b && a > 0.0;
    const double r = keep ? sqrt(a) : 0.0;
    *Rjj = r;
    *scale = keep ? 1.0 / r : 0.0;
  }
}

__global__ void scale_col_kernel(double* v, int64_t n, const double* scale) {
  const double s = *scale;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[i] *= s;
}

// R[0:j, j] += c (R row-major w x w)
__global__ void add_rcol_kernel(double* R, int w, int j, const double* c) {
  for (int i = threadIdx.x; i < j; i += blockDim.x) R[i * w + j] += c[i];
}

constexpr int kJT = 1024;

// One-sided Jacobi SVD of the w x w matrix R (row-major, w <= 128): columns
// of R are rotated pairwise until orthogonal; their norms are the singular
// values and the normalised columns the left singular vectors. Output:
// U (w x w row-major, column c = c-th singular direction by descending
// singular value) and s (w). With Vw non-null the rotations are also applied
// to the columns of J = I (Vw, column-major, global memory): R J = U S, so
// V = J, written row-major to V_out in the same column order as U.
__global__ void __launch_bounds__(kJT) jacobi_svd_kernel(const double* R, int w, double* U, double* s_out,
                                                         double* Vw, double* V_out) {
  extern __shared__ __align__(16) double sm[];
  double* X = sm;                 // column-major: X[col * w + row]
  double* nrm = X + w * w;        // w
  int* order = reinterpret_cast<int*>(nrm + w);
  __shared__ int s_rot;
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5, nw = kJT / 32;
  for (int e = t; e < w * w; e += kJT) {
    const int row = e / w, col = e % w;
    X[col * w + row] = R[e];
    if (Vw) Vw[col * w + row] = (row == col) ? 1.0 : 0.0;
  }
  __syncthreads();
  const int m = (w % 2) ? w + 1 : w;       // players; an odd w has one idle player
  for (int sweep = 0; sweep < 60; ++sweep) {
    if (t == 0) s_rot = 0;
    __syncthreads();
    for (int round = 0; round < m - 1; ++round) {
      for (int pr = wid; pr < m / 2; pr += nw) {
        // circle method: position 0 holds player 0, position i >= 1 holds
        // player 1 + (i - 1 + round) mod (m - 1); pair pr is (pr, m - 1 - pr)
        const int i0 = pr, i1 = m - 1 - pr;
        const int pa = (i0 == 0) ? 0 : 1 + (i0 - 1 + round) % (m - 1);
        const int pb = 1 + (i1 - 1 + round) % (m - 1);
        const int p = pa < pb ? pa : pb, q = pa < pb ? pb : pa;
        if (q >= w) continue;               // the idle player of an odd w
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int c = lane; c < w; c += 32) {
          const double xp = X[p * w + c], xq = X[q * w + c];
          al = fma(xp, xp, al);
          be = fma(xq, xq, be);
          ga = fma(xp, xq, ga);
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        if (al > 0.0 && be > 0.0 && fabs(ga) > 2.0 * DBL_EPSILON * sqrt(al * be)) {
          const double zeta = (be - al) / (2.0 * ga);
          const double tt = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          const double cs = 1.0 / sqrt(1.0 + tt * tt), sn = cs * tt;
          for (int c = lane; c < w; c += 32) {
            const double xp = X[p * w + c], xq = X[q * w + c];
            X[p * w + c] = cs * xp - sn * xq;
            X[q * w + c] = sn * xp + cs * xq;
          }
          if (Vw)
            for (int c = lane; c < w; c += 32) {
              const double vp = Vw[p * w + c], vq = Vw[q * w + c];
              Vw[p * w + c] = cs * vp - sn * vq;
              Vw[q * w + c] = sn * vp + cs * vq;
            }
          if (lane == 0) s_rot = 1;
        }
      }
      __syncthreads();
    }
    const int any = s_rot;
    __syncthreads();
    if (!any) break;
  }
  for (int c = wid; c < w; c += nw) {
    double s2 = 0.0;
    for (int r = lane; r < w; r += 32) s2 = fma(X[c * w + r], X[c * w + r], s2);
    s2 = warp_sum(s2);
    if (lane == 0) nrm[c] = sqrt(s2);
  }
  __syncthreads();
  if (t == 0) {
    for (int c = 0; c < w; ++c) order[c] = c;
    for (int i = 1; i < w; ++i)
      for (int j = i; j > 0 && nrm[order[j]] > nrm[order[j - 1]]; --j) {
        const int tmp = order[j]; order[j] = order[j - 1]; order[j - 1] = tmp;
      }
    for (int c = 0; c < w; ++c) s_out[c] = nrm[order[c]];
  }
  __syncthreads();
  for (int e = t; e < w * w; e += kJT) {
    const int row = e / w, c = e % w;
    const int src = order[c];
    const double nn = nrm[src];
    U[e] = nn > 0.0 ? X[src * w + row] / nn : 0.0;
    if (Vw) V_out[e] = Vw[src * w + row];
  }
}

}  // namespace

cudaError_t pod_thin_svd(const double* X, int64_t n, int w, double* Q, double* R, double* U, double* s,
                         double* work, double* part, int grid, cudaStream_t st, double* V, double* Vwork) {
  if (w < 1 || w > 128 || (V == nullptr) != (Vwork == nullptr)) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(R, 0, sizeof(double) * w * w, st);
  if (e != cudaSuccess) return e;
  double* c = work;                 // w
  double* nrm_orig = work + 128;
  double* nrm_now = work + 129;
  double* scale = work + 130;
  for (int j = 0; j < w; ++j) {
    double* v = Q + (size_t)j * n;
    if ((e = cudaMemcpyAsync(v, X + (size_t)j * n, sizeof(double) * n, cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
      return e;
    if ((e = launch_tn(TnArgs{n, 1, 1, v, n, v, n, 1.0, part, nrm_orig}, grid, st)) != cudaSuccess) return e;
    if (j > 0) {
      for (int pass = 0; pass < 2; ++pass) {
        if ((e = launch_tn(TnArgs{n, j, 1, Q, n, v, n, 1.0, part, c}, grid, st)) != cudaSuccess) return e;
        if ((e = launch_nn(NnArgs{n, j, 1, Q, n, c, 1, 1, -1.0, 1.0, v, n, v, n}, st)) != cudaSuccess) return e;
        add_rcol_kernel<<<1, 128, 0, st>>>(R, w, j, c);
      }
    }
    if ((e = launch_tn(TnArgs{n, 1, 1, v, n, v, n, 1.0, part, nrm_now}, grid, st)) != cudaSuccess) return e;
    qr_diag_kernel<<<1, 32, 0, st>>>(nrm_now, nrm_orig, R + (size_t)j * w + j, scale);
    scale_col_kernel<<<256, 256, 0, st>>>(v, n, scale);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  const size_t smem = sizeof(double) * (w * w + w) + sizeof(int) * w;
  if ((e = cudaFuncSetAttribute(jacobi_svd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
      cudaSuccess)
    return e;
  jacobi_svd_kernel<<<1, kJT, smem, st>>>(R, w, U, s, Vwork, V);
  return cudaGetLastError();
}

}  // namespace rom
