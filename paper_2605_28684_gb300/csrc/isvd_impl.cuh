// Rank-one incremental SVD with forgetting (paper Algorithm 2, Eqs.
// isvd_residual ... isvd_truncation) as one cooperative kernel.
//
//  1. yhat = D (y - q_ref) (optional), p = Phi^T yhat, q = yhat - Phi p by
//     classical Gram-Schmidt applied twice (least squares for orthonormal Phi).
//  2. Core K = [[lam Sigma, p], [0, ||q||]] of order n = k+1. Its left singular
//     vectors are the eigenvectors of K K^T = diag(d)^2 + z z^T with
//     d = (lam sigma_1..lam sigma_k, 0) and z = (p, ||q||): a rank-one
//     modification of a diagonal matrix. After deflation (tiny |z_i|, close
//     d_i) the singular values are the roots of the secular equation
//     1 + sum_i z_i^2 / (d_i^2 - s^2) = 0 (Bunch, Nielsen and Sorensen 1978),
//     one root per CTA, each bracketed between consecutive poles and found by
//     safeguarded Newton in the shifted variable tau = s - d_origin. The
//     vectors use the z recomputed from the roots (Gu and Eisenstat 1995),
//     u_j ~ (zhat_i / (d_i^2 - s_j^2))_i, which keeps them orthogonal.
//  3. Phi <- [Phi, q/||q||] U(:, 1:k'), sigma <- s(1:k'), where k' <= r counts
//     the singular values above rank_tol * s_1; the other columns become zero.
//  4. Optional state transfer a <- Phi_new^T Phi_old a = U(1:k, 1:k')^T a
//     (exact because q/||q|| is orthogonal to Phi_old).
//
// This header holds the kernels as templates on the rank bucket KM; each
// bucket is compiled in its own object (isvd_bucket.cu built with
// -DROM_ISVD_KM=9, 17, 33, 65 and each basis type) so that they build in
// parallel, and
// isvd.cu dispatches to them.
#pragma once
#include <cfloat>
#include <cmath>
#include <type_traits>

#include "rom_internal.cuh"
#include "rom_kernels.cuh"
#include "secular.cuh"

namespace rom {

namespace {

// Workspace layout inside ctx->d.core (doubles):
constexpr int kWsTau = 0;                      // roots: tau_j       [kMaxCore]
constexpr int kWsOrig = kWsTau + kMaxCore;     // roots: origin o_j  [kMaxCore]
constexpr int kWsZhat = kWsOrig + kMaxCore;    // zhat_i             [kMaxCore]
constexpr int kWsSbar = kWsZhat + kMaxCore;    // sorted singular values [kMaxCore]
constexpr int kWsScal = kWsSbar + kMaxCore;    // scalars
constexpr int kWsSize = kWsScal + 16;

struct EventSmem {
  SecularSetup S;
  double d_desc[kMaxCore];
  double z[kMaxCore];
  double p1[kMaxCore];
  double p2[kMaxCore];
  double sc[8];
  double red[32 * kMaxCore];
  double U[kMaxCore * kMaxCore];    // U(:, 0:k') for the rotation
  double a_old[kMaxR];
  double a_new[kMaxR];
  int order[kMaxCore];              // position (descending value) of each eigenpair
  double val[kMaxCore];
  // mixed precision: FP32 copies of p1, p2 and U, the FP64 Gram matrix
  float p1f[kMaxCore];
  float p2f[kMaxCore];
  float Uf[kMaxCore * kMaxCore];
  double Gm[kMaxR * kMaxR];
};

}  // namespace

// --------------------------------------------------------------------------
// Row-parallel pieces (templated on the register budget KM >= k+1).
// --------------------------------------------------------------------------

// Calls f(std::integral_constant<int, KB>) with the smallest register budget
// KB in {9, 17, 33, 65} (capped at KM) that holds k+1 entries, so that loops
// over the rank are sized for the actual rank rather than the maximum.
template <int KM, typename F>
__device__ __forceinline__ void with_rank_bucket(int kp1, F&& f) {
  if (KM <= 9 || kp1 <= 9) f(std::integral_constant<int, (KM < 9 ? KM : 9)>{});
  else if (KM <= 17 || kp1 <= 17) f(std::integral_constant<int, (KM < 17 ? KM : 17)>{});
  else if (KM <= 33 || kp1 <= 33) f(std::integral_constant<int, (KM < 33 ? KM : 33)>{});
  else f(std::integral_constant<int, KM>{});
}

template <int KM>
__device__ __forceinline__ void block_reduce_vec(double (&acc)[KM], int k, double* red, double* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int j = 0; j < KM; ++j) {
    double v = warp_sum(acc[j]);
    if (lane == 0 && j < k) red[wid * KM + j] = v;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += red[w * KM + j];
    out[j] = s;
  }
  __syncthreads();
}

// Sum over CTAs of per-CTA partial vectors, in a fixed order (deterministic).
__device__ __forceinline__ void grid_reduce_vec(const double* partials, int G, int stride, int k,
                                                double* out) {
  grid_reduce_cols(partials, G, stride, k, out);
}

// TPhi is the storage type of the basis: double (FP64 form) or float (mixed
// form: FP32 projections with FP32 accumulation, FP64 core SVD, and an FP64
// CholQR re-orthonormalisation of the rotated basis).
template <int KM, typename TPhi>
__global__ void __launch_bounds__(kBlock) isvd_event_kernel(EventArgs A) {
  using Acc = TPhi;
  constexpr bool kMixed = std::is_same<TPhi, float>::value;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  EventSmem& sm = *reinterpret_cast<EventSmem*>(smem_raw);
  const TPhi* phi = basis<TPhi>(A);
  TPhi* phiw = const_cast<TPhi*>(phi);
  const int G = gridDim.x, b = blockIdx.x, t = threadIdx.x;
  const int64_t N = A.n, ld = A.ld;
  const int64_t beg = (int64_t)b * N / G, end = (int64_t)(b + 1) * N / G;
  const int k = *A.rank;
  const int n = k + 1;
  const int stride = KM + 2;
  double* part0 = A.partials;
  double* part1 = A.partials + (size_t)G * stride;
  double* part2 = A.partials + (size_t)2 * G * stride;
  double* ws = A.core;

  // ---- P1: yhat and p1 = Phi^T yhat, ||yhat||^2 ----
  with_rank_bucket<KM>(n, [&](auto kb) {
    constexpr int KB = decltype(kb)::value;
    Acc acc[KB];
#pragma unroll
    for (int j = 0; j < KB; ++j) acc[j] = Acc(0);
    double yy = 0.0;
    for (int64_t i = beg + t; i < end; i += blockDim.x) {
      double yh;
      if (A.preprocess) {
        yh = A.drow[i] * (A.y[i] - A.q_ref[i]);
        A.yhat[i] = yh;
      } else {
        yh = A.y[i];
      }
      yy = fma(yh, yh, yy);
      const Acc ya = (Acc)yh;
#pragma unroll
      for (int j = 0; j < KB; ++j)
        if (j < k) acc[j] = fma((Acc)phi[j * ld + i], ya, acc[j]);
    }
    if constexpr (kMixed) {
      double accd[KB];
#pragma unroll
      for (int j = 0; j < KB; ++j) accd[j] = (double)acc[j];
      block_reduce_vec<KB>(accd, k, sm.red, sm.p1);
    } else {
      block_reduce_vec<KB>(acc, k, sm.red, sm.p1);
    }
    double yys = block_sum(yy, sm.red);
    for (int j = t; j < k; j += blockDim.x) part0[(size_t)b * stride + j] = sm.p1[j];
    if (t == 0) part0[(size_t)b * stride + KM] = yys;
  });
  if (!grid_sync(A.bar, A.status)) return;
  grid_reduce_vec(part0, G, stride, k, sm.p1);
  grid_reduce_cols(part0 + KM, G, stride, 1, &sm.sc[0]);     // ||yhat||^2
  for (int j = t; j < k; j += blockDim.x) sm.p1f[j] = (float)sm.p1[j];
  __syncthreads();

  const double* yv = A.preprocess ? A.yhat : A.y;
  // ---- P2: q1 = yhat - Phi p1 ; p2 = Phi^T q1 ----
  with_rank_bucket<KM>(n, [&](auto kb) {
    constexpr int KB = decltype(kb)::value;
    Acc acc[KB];
#pragma unroll
    for (int j = 0; j < KB; ++j) acc[j] = Acc(0);
    for (int64_t i = beg + t; i < end; i += blockDim.x) {
      Acc x[KB];
#pragma unroll
      for (int j = 0; j < KB; ++j) x[j] = (j < k) ? (Acc)phi[j * ld + i] : Acc(0);
      Acc v = (Acc)yv[i];
#pragma unroll
      for (int j = 0; j < KB; ++j)
        if (j < k) v = fma(-x[j], kMixed ? (Acc)sm.p1f[j] : (Acc)sm.p1[j], v);
      A.qres[i] = (double)v;
#pragma unroll
      for (int j = 0; j < KB; ++j)
        if (j < k) acc[j] = fma(x[j], v, acc[j]);
    }
    if constexpr (kMixed) {
      double accd[KB];
#pragma unroll
      for (int j = 0; j < KB; ++j) accd[j] = (double)acc[j];
      block_reduce_vec<KB>(accd, k, sm.red, sm.p2);
    } else {
      block_reduce_vec<KB>(acc, k, sm.red, sm.p2);
    }
    for (int j = t; j < k; j += blockDim.x) part1[(size_t)b * stride + j] = sm.p2[j];
  });
  if (!grid_sync(A.bar, A.status)) return;
  grid_reduce_vec(part1, G, stride, k, sm.p2);
  for (int j = t; j < k; j += blockDim.x) sm.p2f[j] = (float)sm.p2[j];
  __syncthreads();
  // ---- P3: q = q1 - Phi p2, ||q||^2 ----
  {
    Acc qq = Acc(0);
    for (int64_t i = beg + t; i < end; i += blockDim.x) {
      Acc v = (Acc)A.qres[i];
      for (int j = 0; j < k; ++j)
        v = fma(-(Acc)phi[j * ld + i], kMixed ? (Acc)sm.p2f[j] : (Acc)sm.p2[j], v);
      A.qres[i] = (double)v;
      qq = fma(v, v, qq);
    }
    double qs = block_sum((double)qq, sm.red);
    if (t == 0) part2[(size_t)b * stride] = qs;
  }
  if (!grid_sync(A.bar, A.status)) return;

  // ---- core matrix and secular setup (every CTA, identical) ----
  grid_reduce_cols(part2, G, stride, 1, &sm.sc[3]);          // ||q||^2
  if (t == 0) {
    double rho = sqrt(sm.sc[3]);
    double ynorm = sqrt(sm.sc[0]);
    double s1 = (k > 0) ? A.sigma[0] : 0.0;
    bool keep_q = rho > A.rank_tol * fmax(ynorm, s1);
    if (!keep_q) rho = 0.0;
    sm.sc[1] = rho;
    sm.sc[2] = keep_q ? 1.0 / rho : 0.0;
    for (int j = 0; j < k; ++j) {
      sm.d_desc[j] = A.lambda * A.sigma[j];
      sm.z[j] = sm.p1[j] + sm.p2[j];
    }
    sm.d_desc[k] = 0.0;
    sm.z[k] = rho;
    if (A.rec && b == 0) {
      A.rec[0] = rho;
      A.rec[1] = ynorm;
      for (int j = 0; j < k; ++j) A.rec[2 + j] = sm.z[j];
    }
    secular_setup(sm.S, n, sm.d_desc, sm.z);
  }
  __syncthreads();
  const SecularSetup& S = sm.S;
  const int k2 = S.k2;

  // ---- roots: one per CTA (warp 0) ----
  if (t < 32) {
    for (int j = b; j < k2; j += G) {
      int o;
      double tau;
      secular_root(S, j, o, tau);
      if (t == 0) {
        ws[kWsTau + j] = tau;
        ws[kWsOrig + j] = (double)o;
      }
    }
  }
  if (!grid_sync(A.bar, A.status)) return;

  // ---- zhat_i (Loewner), one per CTA (warp 0) ----
  if (t < 32) {
    const int lane = t;
    for (int i = b; i < k2; i += G) {
      double pr = 1.0;
      for (int j = lane; j < k2; j += 32) {
        int o = (int)__ldcg(&ws[kWsOrig + j]);
        double tau = __ldcg(&ws[kWsTau + j]);
        double num = root_minus(S, o, tau, i) * root_plus(S, o, tau, i);   // s_j^2 - D_i^2
        double den;
        if (j == k2 - 1) den = 1.0;
        else if (j < i) den = (S.D[j] - S.D[i]) * (S.D[j] + S.D[i]);
        else den = (S.D[j + 1] - S.D[i]) * (S.D[j + 1] + S.D[i]);
        pr *= num / den;
      }
      pr = warp_prod(pr);
      if (lane == 0) ws[kWsZhat + i] = copysign(sqrt(fabs(pr)), S.Z[i]);
    }
  }
  if (!grid_sync(A.bar, A.status)) return;

  // ---- singular values, descending order, vectors ----
  // eigenpair e: e < k2 -> root e; e >= k2 -> deflated position (the
  // (e-k2)-th deflated position in ascending order).
  if (t == 0) {
    int c = 0;
    for (int e = 0; e < k2; ++e) {
      int o = (int)__ldcg(&ws[kWsOrig + e]);
      sm.val[e] = S.D[o] + __ldcg(&ws[kWsTau + e]);
    }
    c = k2;
    for (int p = 0; p < n; ++p)
      if (S.defl[p]) { sm.val[c] = S.dpos[p]; sm.order[c] = p; ++c; }
  }
  __syncthreads();
  // rank of each eigenpair in descending order (ties -> lower eigenpair index)
  __shared__ int s_pos[kMaxCore];
  __shared__ int s_defp[kMaxCore];
  if (t < n) {
    double v = sm.val[t];
    int pos = 0;
    for (int e = 0; e < n; ++e) {
      double w = sm.val[e];
      if (w > v || (w == v && e < t)) ++pos;
    }
    s_pos[t] = pos;
    s_defp[t] = (t >= k2) ? sm.order[t] : -1;
  }
  __syncthreads();
  // vectors: eigenpair e handled by CTA e mod G, warp 0; written as column
  // s_pos[e] of U (n x n, column-major, rows by original index).
  if (t < 32) {
    const int lane = t;
    for (int e = b; e < n; e += G) {
      double vec[kMaxCore / 32 + 1];   // by position, lanes own p = lane + 32 m
      const int nm = (n + 31) / 32;
      for (int m = 0; m < nm; ++m) vec[m] = 0.0;
      if (e < k2) {
        int o = (int)__ldcg(&ws[kWsOrig + e]);
        double tau = __ldcg(&ws[kWsTau + e]);
        double ss = 0.0;
        for (int m = 0; m < nm; ++m) {
          int ci = lane + 32 * m;     // compact index
          if (ci < k2) {
            double den = -(root_minus(S, o, tau, ci)) * root_plus(S, o, tau, ci);  // D_i^2 - s^2
            double u = __ldcg(&ws[kWsZhat + ci]) / den;
            vec[m] = u;
            ss += u * u;
          }
        }
        ss = warp_sum(ss);
        double inv = 1.0 / sqrt(ss);
        // scatter compact -> position: store in shared staging below
        for (int m = 0; m < nm; ++m) vec[m] *= inv;
      }
      // stage into a position-indexed array (shared, per CTA)
      __shared__ double pv[kMaxCore];
      for (int p = lane; p < n; p += 32) pv[p] = 0.0;
      __syncwarp();
      if (e < k2) {
        for (int m = 0; m < nm; ++m) {
          int ci = lane + 32 * m;
          if (ci < k2) pv[S.cidx[ci]] = vec[m];
        }
      } else if (lane == 0) {
        pv[s_defp[e]] = 1.0;
      }
      __syncwarp();
      // undo the deflating rotations (reverse order): x = G^T x'
      if (lane == 0) {
        for (int q = S.nrot - 1; q >= 0; --q) {
          int pa = S.rot_a[q], pb = S.rot_b[q];
          double c = S.rot_c[q], s = S.rot_s[q];
          double xa = pv[pa], xb = pv[pb];
          pv[pa] = c * xa + s * xb;
          pv[pb] = -s * xa + c * xb;
        }
      }
      __syncwarp();
      const int col = s_pos[e];
      for (int p = lane; p < n; p += 32) A.ubar[(size_t)col * n + (n - 1 - p)] = pv[p];
      if (lane == 0) ws[kWsSbar + col] = sm.val[e];
      __syncwarp();
    }
  }
  if (!grid_sync(A.bar, A.status)) return;

  // ---- rotation and truncation ----
  int knew = 0;
  {
    double s0 = __ldcg(&ws[kWsSbar + 0]);
    for (int j = 0; j < n && j < A.r; ++j) {
      double sj = __ldcg(&ws[kWsSbar + j]);
      if (s0 > 0.0 && sj > A.rank_tol * s0) ++knew;
    }
  }
  for (int e = t; e < n * knew; e += blockDim.x) {
    int col = e / n, row = e % n;
    double u = __ldcg(&A.ubar[(size_t)col * n + row]);
    sm.U[row * kMaxCore + col] = u;
    sm.Uf[row * kMaxCore + col] = (float)u;
  }
  if (b == 0)
    for (int j = t; j < k; j += blockDim.x) sm.a_old[j] = A.a ? A.a[j] : 0.0;
  __syncthreads();
  const double qinv = sm.sc[2];
  with_rank_bucket<KM>(n, [&](auto kb) {
    constexpr int KB = decltype(kb)::value;
    const Acc* Us = kMixed ? (const Acc*)(const void*)sm.Uf : (const Acc*)(const void*)sm.U;
    for (int64_t i = beg + t; i < end; i += blockDim.x) {
      Acc x[KB];
#pragma unroll
      for (int j = 0; j < KB; ++j) x[j] = (j < k) ? (Acc)phi[j * ld + i] : Acc(0);
      Acc qh = (Acc)(A.qres[i] * qinv);
#pragma unroll
      for (int c = 0; c < KB; ++c) {
        if (c < knew) {
          Acc v = qh * Us[k * kMaxCore + c];
#pragma unroll
          for (int j = 0; j < KB; ++j)
            if (j < k) v = fma(x[j], Us[j * kMaxCore + c], v);
          phiw[c * ld + i] = (TPhi)v;
        } else if (c < k) {
          phiw[c * ld + i] = TPhi(0);
        }
      }
    }
  });
  if constexpr (kMixed) {
    // ---- FP64 re-orthonormalisation of the FP32 basis (CholQR): G = Phi^T Phi
    // accumulated in FP64 (products of FP32 numbers are exact in FP64),
    // G = R^T R, Phi <- Phi R^-1, and a <- R a so that q~ is unchanged ----
    if (!grid_sync(A.bar, A.status)) return;
    const int kk = knew;
    for (int e = t; e < kk * kk; e += blockDim.x) {
      int j = e / kk, l = e % kk;
      double s = 0.0;
      if (l >= j)
        for (int64_t i = beg; i < end; ++i) s = fma((double)phi[j * ld + i], (double)phi[l * ld + i], s);
      A.gram[(size_t)b * kMaxR * kMaxR + j * kMaxR + l] = s;
    }
    if (!grid_sync(A.bar, A.status)) return;
    {
      const int lane = t & 31, wid = t >> 5, nw = blockDim.x >> 5;
      for (int e = wid; e < kk * kk; e += nw) {
        int j = e / kk, l = e % kk;
        double s = 0.0;
        if (l >= j)
          for (int bb = lane; bb < G; bb += 32) s += __ldcg(&A.gram[(size_t)bb * kMaxR * kMaxR + j * kMaxR + l]);
        s = warp_sum(s);
        if (lane == 0) sm.Gm[j * kMaxR + l] = s;
      }
    }
    __syncthreads();
    if (t == 0) {   // upper Cholesky factor R (in place, row-major, upper triangle)
      for (int j = 0; j < kk; ++j) {
        double d = sm.Gm[j * kMaxR + j];
        for (int l = 0; l < j; ++l) d -= sm.Gm[l * kMaxR + j] * sm.Gm[l * kMaxR + j];
        d = sqrt(fmax(d, DBL_MIN));
        sm.Gm[j * kMaxR + j] = d;
        const double inv = 1.0 / d;
        for (int c = j + 1; c < kk; ++c) {
          double v = sm.Gm[j * kMaxR + c];
          for (int l = 0; l < j; ++l) v -= sm.Gm[l * kMaxR + j] * sm.Gm[l * kMaxR + c];
          sm.Gm[j * kMaxR + c] = v * inv;
        }
      }
    }
    __syncthreads();
    for (int64_t i = beg + t; i < end; i += blockDim.x) {   // y R = x, row by row
      double y[kMaxR];
      for (int j = 0; j < kk; ++j) {
        double v = (double)phi[j * ld + i];
        for (int l = 0; l < j; ++l) v -= y[l] * sm.Gm[l * kMaxR + j];
        y[j] = v / sm.Gm[j * kMaxR + j];
      }
      for (int j = 0; j < kk; ++j) phiw[j * ld + i] = (TPhi)y[j];
    }
  }
  if (b == 0) {
    // sigma, state transfer and the new rank (other CTAs read none of these)
    if (t < A.r) {
      A.sigma[t] = (t < knew) ? __ldcg(&ws[kWsSbar + t]) : 0.0;
      if (A.a && A.transfer) {
        double v = 0.0;
        if (t < knew)
          for (int j = 0; j < k; ++j) v = fma(sm.U[j * kMaxCore + t], sm.a_old[j], v);
        sm.a_new[t] = v;               // staged: other threads still read a_old
      }
    }
    __syncthreads();
    if (t < A.r && A.a && A.transfer) {
      double v = sm.a_new[t];
      if constexpr (kMixed) {      // a <- R a
        if (t < knew) {
          double w = 0.0;
          for (int c = t; c < knew; ++c) w = fma(sm.Gm[t * kMaxR + c], sm.a_new[c], w);
          v = w;
        }
      }
      A.a[t] = v;
    }
    __syncthreads();
    if (t == 0) *A.rank = knew;
  }
}

// --------------------------------------------------------------------------
// Projection a = Phi^T D (v - q_ref) (offline initial state).
// --------------------------------------------------------------------------

template <int KM, typename TPhi>
__global__ void __launch_bounds__(kBlock) project_kernel(ProjectArgs A) {
  const TPhi* phi = basis<TPhi>(A);
  __shared__ double red[32 * KM];
  __shared__ double out[KM];
  const int G = gridDim.x, b = blockIdx.x, t = threadIdx.x;
  const int64_t N = A.n, ld = A.ld;
  const int64_t beg = (int64_t)b * N / G, end = (int64_t)(b + 1) * N / G;
  const int k = *A.rank;
  const int stride = KM + 2;
  double acc[KM];
#pragma unroll
  for (int j = 0; j < KM; ++j) acc[j] = 0.0;
  for (int64_t i = beg + t; i < end; i += blockDim.x) {
    double v = A.drow[i] * (A.v[i] - A.q_ref[i]);
#pragma unroll
    for (int j = 0; j < KM; ++j)
      if (j < k) acc[j] = fma((double)phi[j * ld + i], v, acc[j]);
  }
  block_reduce_vec<KM>(acc, k, red, out);
  for (int j = t; j < k; j += blockDim.x) A.partials[(size_t)b * stride + j] = out[j];
  if (!grid_sync(A.bar, A.status)) return;
  if (b == 0) {
    grid_reduce_vec(A.partials, G, stride, k, out);
    for (int j = t; j < A.r; j += blockDim.x) A.a[j] = (j < k) ? out[j] : 0.0;
  }
}

// --------------------------------------------------------------------------
// templated launchers (instantiated per rank bucket in isvd_bucket.cu)
// --------------------------------------------------------------------------

template <int KM, typename TPhi>
static cudaError_t launch_event_tt(const EventArgs& A, int grid, cudaStream_t s) {
  size_t smem = sizeof(EventSmem);
  cudaError_t e = cudaFuncSetAttribute(isvd_event_kernel<KM, TPhi>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  EventArgs a = A;
  void* args[] = {&a};
  return cudaLaunchCooperativeKernel((const void*)isvd_event_kernel<KM, TPhi>, dim3(grid),
                                     dim3(kBlock), args, smem, s);
}

template <int KM, typename TPhi>
static cudaError_t launch_project_tt(const ProjectArgs& A, int grid, cudaStream_t s) {
  ProjectArgs a = A;
  void* args[] = {&a};
  return cudaLaunchCooperativeKernel((const void*)project_kernel<KM, TPhi>, dim3(grid),
                                     dim3(kBlock), args, 0, s);
}

}  // namespace rom
