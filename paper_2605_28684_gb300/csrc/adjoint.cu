// Gradient of a terminal misfit of the plain-Galerkin Burgers ROM (reverse
// sweep in FP64). The paper states no adjoint; this is the reverse mode of
// the method as the forward path computes it (Algorithm 1 with the iSVD
// update of Algorithm 2, backward-Euler Galerkin steps, Eq.
// galerkin_continuous_rom; coarse backward-Euler FOM steps, Eq.
// coarse_fom_backward_euler; preprocessing and POD of Sec. 3.1).
//
//  * Reduced step a^{n+1} - a^n - dt Phi^T D f(q~) = 0 at its root: the
//    adjoint solves Jr^T w = abar + Phi^T qtbar / d with Jr = I - dt Phi^T J_f Phi
//    (D is a scalar d for Burgers), then scatters w into Phi-bar, q_ref-bar,
//    d-bar and nu-bar in one row pass (adj_jr_kernel, adj_solve_kernel,
//    adj_rows_kernel).
//  * Backward-Euler root y - y_prev - h f(y) = 0: y_prev-bar solves
//    (I - h J_f(y))^T x = y-bar, a periodic tridiagonal system whose row i
//    holds the upper band of cell i-1 and the lower band of cell i+1
//    (adj_tbe_kernel: chunked parallel cyclic reduction in FP64).
//  * iSVD update: adjoint of the core SVD (distinct singular values,
//    U^T dU = F o (P S + S P^T), F_ij = 1 / (s_j^2 - s_i^2)), of the rotation
//    [Phi, q/|q|] U and of the projection p = Phi^T yhat, q = yhat - Phi p,
//    with every basis adjoint projected onto the tangent space of orthonormal
//    bases (adj_event_*).
//  * POD of the training matrix X: the thin-SVD adjoint over all w singular
//    triplets of X (the backward-stable SVD of pod_svd.cu with V accumulated
//    from its rotations), so the gaps s_c^2 - s_i^2 come from the singular
//    values themselves (adj_pod_full_kernel and the generic tall-skinny
//    products).
// Scalar adjoints (d-bar, nu-bar) are summed per CTA into fixed slots and
// reduced in a fixed order, so the result does not depend on scheduling.
#include <cfloat>
#include <cmath>

#include "burgers_stencil.cuh"
#include "rom_internal.cuh"
#include "rom_kernels.cuh"

namespace rom {

namespace {

constexpr int kT = 256;   // threads of the row kernels

__device__ __forceinline__ int64_t wrap(int64_t i, int64_t n) {
  i %= n;
  return i < 0 ? i + n : i;
}

__device__ __forceinline__ double block_sum_d(double v, double* scratch) {
  return block_sum(v, scratch);
}

// LU with partial pivoting of the k x k FP64 matrix J (row-major, ld kMaxR) and
// solve J x = x in place, by one CTA (k <= kMaxR).
__device__ void lu_solve_fp64(double* J, double* x, int* piv, int k) {
  __shared__ int s_p;
  for (int c = 0; c < k; ++c) {
    if (threadIdx.x < 32) {
      // pivot: largest |J[r][c]|, r >= c, lowest index on ties
      double best = -1.0;
      int p = c;
      for (int r = c + threadIdx.x; r < k; r += 32) {
        double v = fabs(J[r * kMaxR + c]);
        if (v > best) { best = v; p = r; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        double bo = __shfl_xor_sync(0xffffffffu, best, o);
        int po = __shfl_xor_sync(0xffffffffu, p, o);
        if (bo > best || (bo == best && po < p)) { best = bo; p = po; }
      }
      if (threadIdx.x == 0) { piv[c] = p; s_p = p; }
    }
    __syncthreads();
    const int p = s_p;
    if (p != c) {
      for (int j = threadIdx.x; j < k; j += blockDim.x) {
        double t = J[c * kMaxR + j];
        J[c * kMaxR + j] = J[p * kMaxR + j];
        J[p * kMaxR + j] = t;
      }
      if (threadIdx.x == 0) { double t = x[c]; x[c] = x[p]; x[p] = t; }
    }
    __syncthreads();
    const double inv = 1.0 / J[c * kMaxR + c];
    for (int r = c + 1 + threadIdx.x; r < k; r += blockDim.x) J[r * kMaxR + c] *= inv;
    __syncthreads();
    const int rem = k - c - 1;
    for (int e = threadIdx.x; e < rem * rem; e += blockDim.x) {
      int r = c + 1 + e / rem, j = c + 1 + e % rem;
      J[r * kMaxR + j] -= J[r * kMaxR + c] * J[c * kMaxR + j];
    }
    for (int r = c + 1 + threadIdx.x; r < k; r += blockDim.x) x[r] -= J[r * kMaxR + c] * x[c];
    __syncthreads();
  }
  // back substitution by warp 0
  if (threadIdx.x < 32) {
    for (int i = k - 1; i >= 0; --i) {
      double s = 0.0;
      for (int l = i + 1 + threadIdx.x; l < k; l += 32) s += J[i * kMaxR + l] * x[l];
      s = warp_sum(s);
      if (threadIdx.x == 0) x[i] = (x[i] - s) / J[i * kMaxR + i];
      __syncwarp();
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// reduced step
// ---------------------------------------------------------------------------

// Partial sums of Phi^T J_f(q~) Phi (k x k) and Phi^T qtbar (k) over the CTA's
// rows, staged in chunks of 64 rows (Phi rows of the chunk and one halo row on
// each side in shared memory).
__global__ void __launch_bounds__(kT) adj_jr_kernel(AdjStepArgs A) {
  extern __shared__ __align__(16) double smem[];
  double* s_phi = smem;                          // 66 x kMaxR
  double* s_jphi = s_phi + 66 * kMaxR;           // 64 x kMaxR
  double* s_u = s_jphi + 64 * kMaxR;             // 66
  double* s_b = s_u + 66;                        // 3 x 64 bands
  const int G = gridDim.x, b = blockIdx.x, t = threadIdx.x;
  const int64_t N = A.n;
  const int k = A.k, kk = k * k;
  const int64_t beg = (int64_t)b * N / G, end = (int64_t)(b + 1) * N / G;
  const double inv_dx = (double)N, dinv = 1.0 / A.d;
  double macc[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) macc[q] = 0.0;
  double vacc = 0.0;
  for (int64_t c0 = beg; c0 < end; c0 += 64) {
    const int cr = (int)min((int64_t)64, end - c0);
    for (int e = t; e < (cr + 2) * k; e += kT) {
      const int rr = e / k, j = e % k;
      s_phi[rr * kMaxR + j] = A.phi[(size_t)j * N + wrap(c0 - 1 + rr, N)];
    }
    __syncthreads();
    for (int rr = t; rr < cr + 2; rr += kT) {
      double s = 0.0;
      for (int j = 0; j < k; ++j) s = fma(s_phi[rr * kMaxR + j], A.a[j], s);
      s_u[rr] = A.q_ref[wrap(c0 - 1 + rr, N)] + s * dinv;
    }
    __syncthreads();
    for (int rr = t; rr < cr; rr += kT) {
      StencilRow st = burgers_stencil(s_u[rr], s_u[rr + 1], s_u[rr + 2], A.nu, inv_dx);
      s_b[rr] = st.dl;
      s_b[64 + rr] = st.dc;
      s_b[128 + rr] = st.dr;
    }
    __syncthreads();
    for (int e = t; e < cr * k; e += kT) {
      const int rr = e / k, l = e % k;
      s_jphi[rr * kMaxR + l] = s_b[rr] * s_phi[rr * kMaxR + l] + s_b[64 + rr] * s_phi[(rr + 1) * kMaxR + l] +
                               s_b[128 + rr] * s_phi[(rr + 2) * kMaxR + l];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int e = t + q * kT;
      if (e < kk) {
        const int j = e / k, l = e % k;
        double s = 0.0;
        for (int rr = 0; rr < cr; ++rr) s = fma(s_phi[(rr + 1) * kMaxR + j], s_jphi[rr * kMaxR + l], s);
        macc[q] += s;
      }
    }
    if (t < k)
      for (int rr = 0; rr < cr; ++rr) vacc = fma(s_phi[(rr + 1) * kMaxR + t], A.qtbar[c0 + rr], vacc);
    __syncthreads();
  }
  double* mp = A.mpart + (size_t)b * kMaxR * kMaxR;
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int e = t + q * kT;
    if (e < kk) mp[e] = macc[q];
  }
  if (t < k) A.vpart[(size_t)b * kMaxR + t] = vacc;
}

// One CTA: Jr = I - dt M (M = sum of the partials), rhs = abar + v / d, and
// w = Jr^-T rhs; abar <- w.
__global__ void __launch_bounds__(kT) adj_solve_kernel(AdjStepArgs A, int G) {
  __shared__ double J[kMaxR * kMaxR];
  __shared__ double x[kMaxR];
  __shared__ int piv[kMaxR];
  const int k = A.k, kk = k * k, t = threadIdx.x;
  for (int e = t; e < kk; e += kT) {
    const int j = e / k, l = e % k;
    double s = 0.0;
    for (int b = 0; b < G; ++b) s += A.mpart[(size_t)b * kMaxR * kMaxR + e];
    // transposed: J[l][j] = Jr[j][l] = delta_jl - dt M_jl
    J[l * kMaxR + j] = (j == l ? 1.0 : 0.0) - A.dt * s;
  }
  if (t < k) {
    double s = 0.0;
    for (int b = 0; b < G; ++b) s += A.vpart[(size_t)b * kMaxR + t];
    x[t] = A.abar[t] + s / A.d;
  }
  __syncthreads();
  lu_solve_fp64(J, x, piv, k);
  if (t < k) {
    A.w[t] = x[t];
    A.abar[t] = x[t];
  }
}

// Row pass of the step adjoint: g = dt d Phi w, dqtp = qtbar + J_f^T g,
// q_ref-bar += dqtp, Phi-bar += dt d f w^T + dqtp a^T / d, and the d-bar and
// nu-bar sums. Each row reads Phi at rows i-2 .. i+2.
__global__ void __launch_bounds__(kT) adj_rows_kernel(AdjStepArgs A) {
  __shared__ double red[32];
  __shared__ double s_w[kMaxR], s_a[kMaxR];
  const int G = gridDim.x, b = blockIdx.x, t = threadIdx.x;
  const int64_t N = A.n;
  const int k = A.k;
  const int64_t beg = (int64_t)b * N / G, end = (int64_t)(b + 1) * N / G;
  const double d = A.d, dinv = 1.0 / d, inv_dx = (double)N;
  if (t < k) { s_w[t] = A.w[t]; s_a[t] = A.a[t]; }
  __syncthreads();
  double snu = 0.0, sd = 0.0;
  for (int64_t i = beg + t; i < end; i += kT) {
    double u[5], pw[5], pa = 0.0;
#pragma unroll
    for (int o = 0; o < 5; ++o) {
      const int64_t ii = wrap(i - 2 + o, N);
      double sa = 0.0, sw = 0.0;
      for (int j = 0; j < k; ++j) {
        const double ph = A.phi[(size_t)j * N + ii];
        sa = fma(ph, s_a[j], sa);
        sw = fma(ph, s_w[j], sw);
      }
      u[o] = A.q_ref[ii] + sa * dinv;
      pw[o] = sw;
      if (o == 2) pa = sa;
    }
    const StencilRow sm1 = burgers_stencil(u[0], u[1], u[2], A.nu, inv_dx);   // row i-1
    const StencilRow s0 = burgers_stencil(u[1], u[2], u[3], A.nu, inv_dx);    // row i
    const StencilRow sp1 = burgers_stencil(u[2], u[3], u[4], A.nu, inv_dx);   // row i+1
    const double gfac = A.dt * d;
    const double gm = gfac * pw[1], g0 = gfac * pw[2], gp = gfac * pw[3];
    const double dq = A.qtbar[i] + sp1.dl * gp + s0.dc * g0 + sm1.dr * gm;
    A.qrefbar[i] += dq;
    const double cf = A.dt * d * s0.f, ca = dq * dinv;
    for (int l = 0; l < k; ++l) A.phibar[(size_t)l * N + i] += cf * s_w[l] + ca * s_a[l];
    snu = fma(g0, s0.fnu, snu);
    sd += A.dt * pw[2] * s0.f - dq * pa * dinv * dinv;
    A.qtbar[i] = 0.0;
  }
  snu = block_sum_d(snu, red);
  sd = block_sum_d(sd, red);
  if (t == 0) {
    A.acc[b] += sd;
    A.acc[kAdjSlots + b] += snu;
  }
}

// ---------------------------------------------------------------------------
// transposed backward-Euler solve (FP64 chunked PCR, as the FOM Newton solve)
// ---------------------------------------------------------------------------

__device__ __forceinline__ int64_t chunk_begin_t(int c, int C, int64_t n) { return (int64_t)c * n / C; }

int choose_chunks_t(int64_t n) {
  int C = 1;
  while (C * 2 <= kMaxChunks && n / (C * 2) >= 64) C *= 2;
  return C;
}

constexpr int kTbeStride = 16;

__global__ void __launch_bounds__(kMaxChunkRows) adj_tbe_kernel(TbeArgs A, int C) {
  extern __shared__ __align__(16) double smem[];
  double* sa = smem;
  double* sb = sa + kMaxChunkRows;
  double* sc = sb + kMaxChunkRows;
  double* sd0 = sc + kMaxChunkRows;
  double* sd1 = sd0 + kMaxChunkRows;
  double* sd2 = sd1 + kMaxChunkRows;
  double* ra = sd2 + kMaxChunkRows;
  double* rb = ra + kMaxChunks;
  double* rc = rb + kMaxChunks;
  double* rd = rc + kMaxChunks;
  double* rs = rd + kMaxChunks;
  double* red = rs + kMaxChunks;   // 32
  const int c = blockIdx.x, t = threadIdx.x;
  const int64_t n = A.n;
  const int64_t beg = chunk_begin_t(c, C, n);
  const int m = (int)(chunk_begin_t(c + 1, C, n) - beg);
  const int mi = m - 1;
  const bool active = t < m;
  const int64_t i = beg + t;
  const double inv_dx = (double)n;
  double a_t = 0.0, b_t = 1.0, c_t = 0.0, d0 = 0.0, d1 = 0.0, d2 = 0.0, fnu = 0.0;
  if (active) {
    double y[5];
#pragma unroll
    for (int o = 0; o < 5; ++o) y[o] = A.y[wrap(i - 2 + o, n)];
    const StencilRow sm1 = burgers_stencil(y[0], y[1], y[2], A.nu, inv_dx);
    const StencilRow s0 = burgers_stencil(y[1], y[2], y[3], A.nu, inv_dx);
    const StencilRow sp1 = burgers_stencil(y[2], y[3], y[4], A.nu, inv_dx);
    a_t = -A.h * sm1.dr;          // coefficient of x_{i-1}
    b_t = 1.0 - A.h * s0.dc;
    c_t = -A.h * sp1.dl;          // coefficient of x_{i+1}
    d0 = A.rhs1[i] + (A.rhs2 ? A.rhs2[i] : 0.0);
    fnu = s0.fnu;
  }
  if (t == m - 1) {
    double* ch = A.chunk + (size_t)c * kTbeStride;
    ch[0] = a_t; ch[1] = b_t; ch[2] = c_t; ch[3] = d0;
  }
  if (t < mi) {
    if (t == 0) { d1 = -a_t; a_t = 0.0; }
    if (t == mi - 1) { d2 = -c_t; c_t = 0.0; }
  } else {
    a_t = 0.0; b_t = 1.0; c_t = 0.0; d0 = d1 = d2 = 0.0;
  }
  sa[t] = a_t; sb[t] = b_t; sc[t] = c_t; sd0[t] = d0; sd1[t] = d1; sd2[t] = d2;
  __syncthreads();
  for (int s = 1; s < mi; s <<= 1) {
    double na = a_t, nb = b_t, nc = c_t, n0 = d0, n1 = d1, n2 = d2;
    if (t < mi) {
      const int tm = t - s, tp = t + s;
      double am = 0.0, bm = 1.0, cm = 0.0, m0 = 0.0, m1 = 0.0, m2 = 0.0;
      double ap = 0.0, bp = 1.0, cp = 0.0, p0 = 0.0, p1 = 0.0, p2 = 0.0;
      if (tm >= 0) { am = sa[tm]; bm = sb[tm]; cm = sc[tm]; m0 = sd0[tm]; m1 = sd1[tm]; m2 = sd2[tm]; }
      if (tp < mi) { ap = sa[tp]; bp = sb[tp]; cp = sc[tp]; p0 = sd0[tp]; p1 = sd1[tp]; p2 = sd2[tp]; }
      const double al = -a_t / bm, ga = -c_t / bp;
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
  double yv = 0.0, vv = 0.0, wv = 0.0;
  if (t < mi) { yv = d0 / b_t; vv = d1 / b_t; wv = d2 / b_t; }
  {
    double* ch = A.chunk + (size_t)c * kTbeStride;
    if (t == 0) { ch[4] = yv; ch[5] = vv; ch[6] = wv; }
    if (t == mi - 1) { ch[7] = yv; ch[8] = vv; ch[9] = wv; }
  }
  if (!grid_sync(A.bar, A.status)) return;
  if (t < C) {
    const double* ch = A.chunk + (size_t)t * kTbeStride;
    const double* nx = A.chunk + (size_t)((t + 1) % C) * kTbeStride;
    const double as_ = __ldcg(ch + 0), bs_ = __ldcg(ch + 1), cs_ = __ldcg(ch + 2), ds_ = __ldcg(ch + 3);
    const double yL = __ldcg(ch + 7), vL = __ldcg(ch + 8), wL = __ldcg(ch + 9);
    const double y0 = __ldcg(nx + 4), v0 = __ldcg(nx + 5), w0 = __ldcg(nx + 6);
    ra[t] = as_ * vL;
    rb[t] = bs_ + as_ * wL + cs_ * v0;
    rc[t] = cs_ * w0;
    rd[t] = ds_ - as_ * yL - cs_ * y0;
  }
  __syncthreads();
  for (int s = 1; s < C; s <<= 1) {
    double na = 0.0, nb = 0.0, nc = 0.0, nd = 0.0;
    if (t < C) {
      const int tm = (t - s + C) % C, tp = (t + s) % C;
      const double al = -ra[t] / rb[tm], ga = -rc[t] / rb[tp];
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
  const double s_left = rs[(c - 1 + C) % C], s_self = rs[c];
  double xv = 0.0;
  if (t < mi) xv = yv + vv * s_left + wv * s_self;
  else if (t == m - 1) xv = s_self;
  if (active) A.x[i] = xv;
  double snu = active ? A.h * xv * fnu : 0.0;
  snu = block_sum_d(snu, red);
  if (t == 0) A.acc_nu[c] += snu;
}

// ---------------------------------------------------------------------------
// generic tall-skinny products
// ---------------------------------------------------------------------------

constexpr int kTnRows = 32;

__global__ void __launch_bounds__(kT) tn_part_kernel(TnArgs A) {
  extern __shared__ __align__(16) double smem[];
  double* sA = smem;                   // kTnRows x m
  double* sB = sA + kTnRows * A.m;     // kTnRows x nc
  const int G = gridDim.x, b = blockIdx.x, t = threadIdx.x;
  const int64_t N = A.n;
  const int m = A.m, nc = A.nc, E = m * nc;
  const int64_t beg = (int64_t)b * N / G, end = (int64_t)(b + 1) * N / G;
  double acc[64];
#pragma unroll
  for (int q = 0; q < 64; ++q) acc[q] = 0.0;
  for (int64_t r0 = beg; r0 < end; r0 += kTnRows) {
    const int rr = (int)min((int64_t)kTnRows, end - r0);
    for (int e = t; e < rr * m; e += kT) {
      const int r = e % rr, j = e / rr;
      sA[r * m + j] = A.A[(size_t)j * A.lda + r0 + r];
    }
    for (int e = t; e < rr * nc; e += kT) {
      const int r = e % rr, l = e / rr;
      sB[r * nc + l] = A.B[(size_t)l * A.ldb + r0 + r];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 64; ++q) {
      const int e = t + q * kT;
      if (e < E) {
        const int j = e / nc, l = e % nc;
        double s = 0.0;
        for (int r = 0; r < rr; ++r) s = fma(sA[r * m + j], sB[r * nc + l], s);
        acc[q] += s;
      }
    }
    __syncthreads();
  }
  double* p = A.part + (size_t)b * E;
#pragma unroll
  for (int q = 0; q < 64; ++q) {
    const int e = t + q * kT;
    if (e < E) p[e] = acc[q];
  }
}

__global__ void tn_reduce_kernel(TnArgs A, int G) {
  const int E = A.m * A.nc;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < G; ++b) s += A.part[(size_t)b * E + e];
    A.out[e] = A.alpha * s;
  }
}

constexpr int kNnCols = 16;

__global__ void __launch_bounds__(kT) nn_kernel(NnArgs A) {
  extern __shared__ __align__(16) double sM[];    // m x nc row-major
  const int m = A.m, nc = A.nc;
  for (int e = threadIdx.x; e < m * nc; e += blockDim.x) {
    const int j = e / nc, l = e % nc;
    sM[e] = A.M[(size_t)j * A.msj + (size_t)l * A.msl];
  }
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < A.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    for (int l0 = 0; l0 < nc; l0 += kNnCols) {
      double acc[kNnCols];
#pragma unroll
      for (int q = 0; q < kNnCols; ++q) acc[q] = 0.0;
      for (int j = 0; j < m; ++j) {
        const double a = A.A[(size_t)j * A.lda + i];
#pragma unroll
        for (int q = 0; q < kNnCols; ++q)
          if (l0 + q < nc) acc[q] = fma(a, sM[j * nc + l0 + q], acc[q]);
      }
#pragma unroll
      for (int q = 0; q < kNnCols; ++q) {
        const int l = l0 + q;
        if (l < nc) {
          const double c0 = (A.beta != 0.0) ? A.beta * A.Cin[(size_t)l * A.ldcin + i] : 0.0;
          A.C[(size_t)l * A.ldc + i] = c0 + A.alpha * acc[q];
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// event (iSVD update + state transfer)
// ---------------------------------------------------------------------------

// qhat into column k of B: B[:, k] = B[:, r] / rho (zero for an empty residual)
__global__ void adj_ev_qhat_kernel(AdjEventArgs A) {
  const double rho = A.rec[0];
  const double inv = rho > 0.0 ? 1.0 / rho : 0.0;
  const int64_t N = A.n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double q = A.B[(size_t)A.r * N + i];
    A.B[(size_t)A.k * N + i] = q * inv;
  }
}

// Transfer a_tr = Phi_new^T d (q~ - q_ref) reversed: Pnb = Phi-bar + d e abar^T,
// q~-bar += d Phi_new abar, q_ref-bar -= d Phi_new abar, d-bar += (Phi_new abar) . e,
// with e = Phi_old a / d.
__global__ void __launch_bounds__(kT) adj_ev1_kernel(AdjEventArgs A) {
  __shared__ double red[32];
  __shared__ double s_a[kMaxR], s_ab[kMaxR];
  const int G = gridDim.x, b = blockIdx.x, t = threadIdx.x;
  const int64_t N = A.n;
  const int k = A.k, kn = A.kn;
  const int64_t beg = (int64_t)b * N / G, end = (int64_t)(b + 1) * N / G;
  const double d = A.d;
  if (t < k) s_a[t] = A.a[t];
  if (t < kn) s_ab[t] = A.abar[t];
  __syncthreads();
  double sd = 0.0;
  for (int64_t i = beg + t; i < end; i += kT) {
    double pa = 0.0;
    for (int j = 0; j < k; ++j) pa = fma(A.B[(size_t)j * N + i], s_a[j], pa);
    const double e = pa / d;
    double we = 0.0;
    for (int l = 0; l < kn; ++l) {
      we = fma(A.phinew[(size_t)l * N + i], s_ab[l], we);
      A.pnb[(size_t)l * N + i] = A.phibar[(size_t)l * N + i] + d * e * s_ab[l];
    }
    sd = fma(we, e, sd);
    A.qtbar[i] += d * we;
    A.qrefbar[i] -= d * we;
  }
  sd = block_sum_d(sd, red);
  if (t == 0) A.acc[b] += sd;
}

// small[OFF_SYM]: -sym(A) of the kn x kn product at small[OFF_A]
__global__ void adj_ev_sym_kernel(const double* Am, double* M, int kn) {
  for (int e = threadIdx.x; e < kn * kn; e += blockDim.x) {
    const int j = e / kn, l = e % kn;
    M[e] = -0.5 * (Am[j * kn + l] + Am[l * kn + j]);
  }
}

// Offsets into the small device area of an event (doubles).
constexpr int kOffA = 0;                                  // kn x kn: Phi_new^T Pnb
constexpr int kOffSym = kOffA + kMaxCore * kMaxCore;      // kn x kn: -sym
constexpr int kOffUbb = kOffSym + kMaxCore * kMaxCore;    // n x kn: B^T Pbar
constexpr int kOffBtBb = kOffUbb + kMaxCore * kMaxCore;   // n: B^T qhat-bar
constexpr int kOffBtQ = kOffBtBb + kMaxCore;              // n: B^T qhat
constexpr int kOffPf = kOffBtQ + kMaxCore;                // k: final p-bar
constexpr int kOffCoef = kOffPf + kMaxCore;               // 1/rho, rho-bar total, empty

// One CTA: adjoint of the core SVD and of the projection, for n = k + 1.
//  G = F[:, :kn] o (U^T Ubb); P-bar[:, c] += G[:, c] s_c, P-bar[c, :] += G[:, c]^T s,
//  P-bar[c, c] += sigma-bar_c; K-bar = U P' W^T with W = K^T U and P' = P-bar / s
//  on the kept columns, P'[c, j] = G[j, c] on the others (their V column is
//  W_j / s_j and P-bar[c, j] = G[j, c] s_j). Then sigma_old-bar = lambda diag,
//  p-bar, rho-bar, and the projection terms.
__global__ void __launch_bounds__(kT) adj_core_kernel(AdjEventArgs A) {
  extern __shared__ __align__(16) double smem[];
  const int k = A.k, n = k + 1, kn = A.kn, t = threadIdx.x;
  double* U = smem;                  // n x n, U[row * n + col]
  double* W = U + n * n;             // n x n: W[row * n + col] = (K^T U)[row][col]
  double* Pp = W + n * n;            // n x n: P'
  double* T1 = Pp + n * n;           // n x n: U P'
  double* Kb = T1 + n * n;           // n x n: K-bar
  double* Gm = Kb + n * n;           // n x kn
  double* s = Gm + n * kMaxCore;     // n
  double* sm = A.small;
  const double lam = A.lambda, rho = A.rec[0];
  for (int e = t; e < n * n; e += kT) {
    const int row = e % n, col = e / n;
    U[row * n + col] = A.ubar[(size_t)col * n + row];
  }
  for (int j = t; j < n; j += kT) s[j] = A.sbar[j];
  __syncthreads();
  // W = K^T U: row r < k: lam sigma_r U[r][:]; row k: z^T U with z = [p; rho]
  // the core's last column. Row k of K K^T is rho z^T, so for a left singular
  // vector u_c, z^T u_c = s_c^2 u_c[k] / rho exactly; that form keeps the
  // relative accuracy of the small singular directions, where the dot
  // product p^T u + rho u[k] cancels terms of size |p| down to about s_c
  // (with lambda << 1 every direction but one is small). An empty new
  // direction (rho = 0) keeps the dot product.
  for (int e = t; e < n * n; e += kT) {
    const int row = e / n, col = e % n;
    double v;
    if (row < k) {
      v = lam * A.sigma_old[row] * U[row * n + col];
    } else if (rho > 0.0) {
      v = s[col] * s[col] * U[k * n + col] / rho;
    } else {
      v = rho * U[k * n + col];
      for (int m = 0; m < k; ++m) v = fma(A.rec[2 + m], U[m * n + col], v);
    }
    W[row * n + col] = v;
  }
  // G = F o (U^T Ubb) on the kept columns
  const double* Ubb = sm + kOffUbb;   // n x kn row-major
  for (int e = t; e < n * kn; e += kT) {
    const int i = e / kn, c = e % kn;
    double v = 0.0;
    for (int m = 0; m < n; ++m) v = fma(U[m * n + i], Ubb[m * kn + c], v);
    const double diff = s[c] * s[c] - s[i] * s[i];
    Gm[i * kMaxCore + c] = (i != c && diff != 0.0) ? v / diff : 0.0;
  }
  __syncthreads();
  for (int e = t; e < n * n; e += kT) {
    const int i = e / n, j = e % n;
    double v = 0.0;
    if (j < kn) {
      v = Gm[i * kMaxCore + j] * s[j];
      if (i < kn) v += Gm[j * kMaxCore + i] * s[j];
      if (i == j) v += A.sigbar[j];
      v /= s[j];
    } else if (i < kn) {
      v = Gm[j * kMaxCore + i];
    }
    Pp[i * n + j] = v;
  }
  __syncthreads();
  for (int e = t; e < n * n; e += kT) {
    const int i = e / n, j = e % n;
    double v = 0.0;
    for (int m = 0; m < n; ++m) v = fma(U[i * n + m], Pp[m * n + j], v);
    T1[i * n + j] = v;
  }
  __syncthreads();
  for (int e = t; e < n * n; e += kT) {
    const int i = e / n, j = e % n;
    double v = 0.0;
    for (int m = 0; m < n; ++m) v = fma(T1[i * n + m], W[j * n + m], v);
    Kb[i * n + j] = v;
  }
  __syncthreads();
  if (t == 0) {
    const bool empty = !(rho > 0.0);
    const double qq = sm[kOffBtBb + k];                // qhat . qhat-bar
    const double rbar = Kb[k * n + k];
    const double rtot = empty ? 0.0 : rbar - qq / rho;
    sm[kOffCoef + 0] = empty ? 0.0 : 1.0 / rho;
    sm[kOffCoef + 1] = rtot;
    sm[kOffCoef + 2] = empty ? 1.0 : 0.0;
  }
  __syncthreads();
  const bool empty = !(rho > 0.0);
  if (t < k) {
    const double pbar = Kb[t * n + k];
    double ptq = 0.0;
    if (!empty) ptq = sm[kOffBtBb + t] / rho + sm[kOffBtQ + t] * sm[kOffCoef + 1];
    sm[kOffPf + t] = pbar - ptq;
  }
  __syncthreads();
  for (int j = t; j < A.r; j += kT) A.sigbar[j] = (j < k) ? lam * Kb[j * n + j] : 0.0;
}

// Rows of the projection adjoint: qbar = qhat-bar / rho + qhat rho-bar,
// Phi_old-bar = Bbar[:, :k] - qbar p^T + yhat pbar^T, yhat-bar = qbar + Phi_old pbar,
// y-bar += d yhat-bar, d-bar += yhat-bar . (y_new - q_ref), q_ref-bar -= d yhat-bar.
__global__ void __launch_bounds__(kT) adj_ev2_kernel(AdjEventArgs A) {
  __shared__ double red[32];
  __shared__ double s_p[kMaxR], s_pf[kMaxR], s_c[4];
  const int G = gridDim.x, b = blockIdx.x, t = threadIdx.x;
  const int64_t N = A.n;
  const int k = A.k;
  const int64_t beg = (int64_t)b * N / G, end = (int64_t)(b + 1) * N / G;
  const double d = A.d;
  if (t < k) { s_p[t] = A.rec[2 + t]; s_pf[t] = A.small[kOffPf + t]; }
  if (t < 3) s_c[t] = A.small[kOffCoef + t];
  __syncthreads();
  const double inv_rho = s_c[0], rtot = s_c[1];
  const bool empty = s_c[2] != 0.0;
  double sd = 0.0;
  for (int64_t i = beg + t; i < end; i += kT) {
    const double qh = A.B[(size_t)k * N + i];
    const double qbar = empty ? 0.0 : A.bbar[(size_t)k * N + i] * inv_rho + qh * rtot;
    const double yh = A.yhat[i];
    double yb = qbar;
    for (int l = 0; l < k; ++l) {
      const double ph = A.B[(size_t)l * N + i];
      yb = fma(ph, s_pf[l], yb);
      A.phibar_out[(size_t)l * N + i] = A.bbar[(size_t)l * N + i] - qbar * s_p[l] + yh * s_pf[l];
    }
    A.ybar_new[i] = A.ybar[i] + d * yb;
    sd = fma(yb, A.ynew[i] - A.q_ref[i], sd);
    A.qrefbar[i] -= d * yb;
  }
  sd = block_sum_d(sd, red);
  if (t == 0) A.acc[b] += sd;
}

// ---------------------------------------------------------------------------
// offline pieces
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(kT) adj_a0_kernel(AdjA0Args A) {
  __shared__ double red[32];
  __shared__ double s_ab[kMaxR];
  const int G = gridDim.x, b = blockIdx.x, t = threadIdx.x;
  const int64_t N = A.n;
  const int k = A.k;
  const int64_t beg = (int64_t)b * N / G, end = (int64_t)(b + 1) * N / G;
  const double d = A.d;
  if (t < k) s_ab[t] = A.abar[t];
  __syncthreads();
  double sd = 0.0;
  for (int64_t i = beg + t; i < end; i += kT) {
    const double e = A.qlast[i] - A.q_ref[i];
    double we = 0.0;
    for (int l = 0; l < k; ++l) {
      we = fma(A.phi[(size_t)l * N + i], s_ab[l], we);
      A.phibar[(size_t)l * N + i] += d * e * s_ab[l];
    }
    sd = fma(we, e, sd);
    A.qlastbar[i] += d * we;
    A.qrefbar[i] -= d * we;
  }
  sd = block_sum_d(sd, red);
  if (t == 0) A.acc[b] += sd;
}

// The POD adjoint over every singular triplet of the thin SVD X = U S V^T
// (N x w, U = [u_1 ... u_w], descending s). Kept columns c < k carry
// Ubar_c and sbar_c; with A = U^T Ubar (w x k) and F_ic = 1 / (s_c^2 - s_i^2)
// (zero for i = c and for equal values):
//   Pbar_ic += F_ic A_ic s_c,  Pbar_ci += F_ic A_ic s_i,  Pbar_cc += sbar_c,
//   Xbar = U Pbar V^T + (Ubar - U A) S_k^-1 V_k^T
//        = U B1 + Ubar B2,  B1 = Pbar V^T - A S_k^-1 V_k^T,  B2 = S_k^-1 V_k^T.
// The gaps come from the singular values themselves, never from a Gram
// matrix of X, so singular values far below the rounding of X^T X (kept
// directions near the rank tolerance) keep their relative accuracy.
// One CTA: B1 (w x w row-major) and B2 (k x w row-major).
__global__ void __launch_bounds__(kT) adj_pod_full_kernel(AdjPodArgs A) {
  extern __shared__ __align__(16) double smem[];
  const int w = A.w, k = A.k, t = threadIdx.x;
  double* P = smem;                  // w x w: Pbar
  for (int e = t; e < w * w; e += kT) P[e] = 0.0;
  __syncthreads();
  // each entry of Pbar is written by exactly one thread: the (i, c) term goes
  // to P[i][c] (c < k) and its mirror to P[c][i]; both are summed per entry
  for (int e = t; e < w * w; e += kT) {
    const int i = e / w, j = e % w;
    double v = 0.0;
    if (j < k && i != j) {           // F_ij A_ij s_j
      const double diff = A.s[j] * A.s[j] - A.s[i] * A.s[i];
      if (diff != 0.0) v += A.A[i * k + j] / diff * A.s[j];
    }
    if (i < k && i != j) {           // F_ji A_ji s_j (mirror of the (j, i) term)
      const double diff = A.s[i] * A.s[i] - A.s[j] * A.s[j];
      if (diff != 0.0) v += A.A[j * k + i] / diff * A.s[j];
    }
    if (i == j && i < k) v += A.sbar[i];
    P[e] = v;
  }
  __syncthreads();
  for (int e = t; e < w * w; e += kT) {
    const int i = e / w, j = e % w;
    double v = 0.0;
    for (int l = 0; l < w; ++l) v = fma(P[i * w + l], A.V[j * w + l], v);
    for (int c = 0; c < k; ++c) v -= A.A[i * k + c] / A.s[c] * A.V[j * w + c];
    A.B1[e] = v;
  }
  for (int e = t; e < k * w; e += kT) {
    const int c = e / w, j = e % w;
    A.B2[e] = A.V[j * w + c] / A.s[c];
  }
}

// pass 0: acc[b] += sum Xbar o Xc; pass 1: Qbar = d Xbar - d^2 dtot (2 / (N w)) Xc,
// q_ref-bar -= row sums of Qbar, Qbar[:, w-1] += qlast-bar.
__global__ void __launch_bounds__(kT) adj_xc_kernel(AdjXcArgs A, int pass) {
  __shared__ double red[32];
  const int G = gridDim.x, b = blockIdx.x, t = threadIdx.x;
  const int64_t N = A.n;
  const int w = A.w;
  const int64_t beg = (int64_t)b * N / G, end = (int64_t)(b + 1) * N / G;
  const double d = A.d;
  if (pass == 0) {
    double s = 0.0;
    for (int64_t i = beg + t; i < end; i += kT) {
      const double qr = A.q_ref[i];
      for (int j = 0; j < w; ++j)
        s = fma(A.Xbar[(size_t)j * N + i], A.Q[(size_t)j * N + i] - qr, s);
    }
    s = block_sum_d(s, red);
    if (t == 0) A.acc[b] += s;
    return;
  }
  const double cf = d * d * (*A.dtot) * 2.0 / ((double)N * (double)w);
  for (int64_t i = beg + t; i < end; i += kT) {
    const double qr = A.q_ref[i];
    double rs = 0.0;
    for (int j = 0; j < w; ++j) {
      const double v = d * A.Xbar[(size_t)j * N + i] - cf * (A.Q[(size_t)j * N + i] - qr);
      rs += v;
      A.Qbar[(size_t)j * N + i] = v + (j == w - 1 ? A.qlastbar[i] : 0.0);
    }
    A.qrefbar[i] -= rs;
  }
}

__global__ void adj_sum_slots_kernel(const double* acc, double* out, int add) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = add ? *out : 0.0;
    for (int b = 0; b < kAdjSlots; ++b) s += acc[b];
    *out = s;
  }
}

__global__ void adj_add_kernel(int64_t n, const double* a, const double* b, double* y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a[i] + b[i];
}

__global__ void adj_lift_kernel(int64_t n, int k, const double* phi, const double* a,
                                const double* q_ref, double d, double* q) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < k; ++j) s = fma(phi[(size_t)j * n + i], a[j], s);
    q[i] = q_ref[i] + s / d;
  }
}

__global__ void adj_misfit_kernel(int64_t n, const double* q, const double* target, double* qtbar,
                                  double* part) {
  __shared__ double red[32];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double r = q[i] - target[i];
    qtbar[i] = r;
    s = fma(r, r, s);
  }
  s = block_sum_d(s, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void adj_misfit_final_kernel(const double* part, int nb, double* J) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += part[b];
    *J = 0.5 * s;
  }
}

int rows_grid(int64_t n, int grid) {
  int64_t g = n / 64;
  if (g < 1) g = 1;
  return (int)(g < grid ? g : grid);
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

cudaError_t launch_adj_step(const AdjStepArgs& A, int grid, cudaStream_t s) {
  if (A.k < 1 || A.k > kMaxR) return cudaErrorInvalidValue;
  const int G = rows_grid(A.n, grid);
  const size_t smem = sizeof(double) * (66 * kMaxR + 64 * kMaxR + 66 + 3 * 64);
  cudaError_t e = cudaFuncSetAttribute(adj_jr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  adj_jr_kernel<<<G, kT, smem, s>>>(A);
  adj_solve_kernel<<<1, kT, 0, s>>>(A, G);
  adj_rows_kernel<<<G, kT, 0, s>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_adj_tbe(const TbeArgs& A, cudaStream_t s) {
  const int C = choose_chunks_t(A.n);
  const int64_t mmax = (A.n + C - 1) / C;
  if (mmax > kMaxChunkRows || A.n < 2) return cudaErrorInvalidValue;
  int threads = (int)((mmax + 31) / 32 * 32);
  if (threads < C) threads = C;
  const size_t smem = sizeof(double) * (6 * kMaxChunkRows + 5 * kMaxChunks + 32);
  cudaError_t e = cudaFuncSetAttribute(adj_tbe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  TbeArgs a = A;
  int Cc = C;
  void* args[] = {&a, &Cc};
  return cudaLaunchCooperativeKernel((const void*)adj_tbe_kernel, dim3(C), dim3(threads), args, smem, s);
}

cudaError_t launch_tn(const TnArgs& A, int grid, cudaStream_t s) {
  if (A.m < 1 || A.nc < 1 || A.m > 128 || A.nc > 128 || A.m * A.nc > 64 * kT)
    return cudaErrorInvalidValue;
  const int G = rows_grid(A.n, grid);
  const size_t smem = sizeof(double) * kTnRows * (A.m + A.nc);
  cudaError_t e = cudaFuncSetAttribute(tn_part_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  tn_part_kernel<<<G, kT, smem, s>>>(A);
  const int E = A.m * A.nc;
  tn_reduce_kernel<<<(E + kT - 1) / kT, kT, 0, s>>>(A, G);
  return cudaGetLastError();
}

cudaError_t launch_nn(const NnArgs& A, cudaStream_t s) {
  if (A.m < 1 || A.nc < 1 || A.m * A.nc > 128 * 128) return cudaErrorInvalidValue;
  const size_t smem = sizeof(double) * A.m * A.nc;
  cudaError_t e = cudaFuncSetAttribute(nn_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int blocks = (int)((A.n + kT - 1) / kT);
  if (blocks > 1024) blocks = 1024;
  nn_kernel<<<blocks, kT, smem, s>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_adj_event(const AdjEventArgs& A, int grid, cudaStream_t s) {
  const int k = A.k, n = k + 1, kn = A.kn;
  if (k < 0 || k > kMaxR || kn < 1 || kn > kMaxR || kn > n) return cudaErrorInvalidValue;
  const int G = rows_grid(A.n, grid);
  double* sm = A.small;
  cudaError_t e;
  adj_ev_qhat_kernel<<<256, kT, 0, s>>>(A);
  adj_ev1_kernel<<<G, kT, 0, s>>>(A);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // stiefel projection of Pnb at Phi_new
  TnArgs t1{A.n, kn, kn, A.phinew, A.n, A.pnb, A.n, 1.0, A.part, sm + kOffA};
  if ((e = launch_tn(t1, grid, s)) != cudaSuccess) return e;
  adj_ev_sym_kernel<<<1, kT, 0, s>>>(sm + kOffA, sm + kOffSym, kn);
  NnArgs n1{A.n, kn, kn, A.phinew, A.n, sm + kOffSym, kn, 1, 1.0, 1.0, A.pnb, A.n, A.pnb, A.n};
  if ((e = launch_nn(n1, s)) != cudaSuccess) return e;
  // Bbar = Pbar U(:, :kn)^T: M(j, r) = U(r, j) = ubar[j * n + r]
  NnArgs n2{A.n, kn, n, A.pnb, A.n, A.ubar, n, 1, 1.0, 0.0, A.bbar, A.n, A.bbar, A.n};
  if ((e = launch_nn(n2, s)) != cudaSuccess) return e;
  // Ubb = B^T Pbar, B^T qhat-bar, B^T qhat
  TnArgs t2{A.n, n, kn, A.B, A.n, A.pnb, A.n, 1.0, A.part, sm + kOffUbb};
  if ((e = launch_tn(t2, grid, s)) != cudaSuccess) return e;
  TnArgs t3{A.n, n, 1, A.B, A.n, A.bbar + (size_t)k * A.n, A.n, 1.0, A.part, sm + kOffBtBb};
  if ((e = launch_tn(t3, grid, s)) != cudaSuccess) return e;
  TnArgs t4{A.n, n, 1, A.B, A.n, A.B + (size_t)k * A.n, A.n, 1.0, A.part, sm + kOffBtQ};
  if ((e = launch_tn(t4, grid, s)) != cudaSuccess) return e;
  const size_t csmem = sizeof(double) * (5 * n * n + n * kMaxCore + n);
  if ((e = cudaFuncSetAttribute(adj_core_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)csmem)) != cudaSuccess)
    return e;
  adj_core_kernel<<<1, kT, csmem, s>>>(A);
  adj_ev2_kernel<<<G, kT, 0, s>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_adj_neg_sym(const double* Am, double* M, int k, cudaStream_t s) {
  adj_ev_sym_kernel<<<1, kT, 0, s>>>(Am, M, k);
  return cudaGetLastError();
}

cudaError_t launch_adj_a0(const AdjA0Args& A, int grid, cudaStream_t s) {
  adj_a0_kernel<<<rows_grid(A.n, grid), kT, 0, s>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_adj_pod_full(const AdjPodArgs& A, cudaStream_t s) {
  if (A.w < 1 || A.w > 128 || A.k < 1 || A.k > A.w || A.k > kMaxR) return cudaErrorInvalidValue;
  const size_t smem = sizeof(double) * A.w * A.w;
  cudaError_t e = cudaFuncSetAttribute(adj_pod_full_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  adj_pod_full_kernel<<<1, kT, smem, s>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_adj_xc(const AdjXcArgs& A, int grid, cudaStream_t s) {
  const int G = rows_grid(A.n, grid);
  adj_xc_kernel<<<G, kT, 0, s>>>(A, 0);
  adj_sum_slots_kernel<<<1, 32, 0, s>>>(A.acc, A.dtot, 0);
  adj_xc_kernel<<<G, kT, 0, s>>>(A, 1);
  return cudaGetLastError();
}

cudaError_t launch_adj_sum_slots(const double* acc, double* out, int add, cudaStream_t s) {
  adj_sum_slots_kernel<<<1, 32, 0, s>>>(acc, out, add);
  return cudaGetLastError();
}

cudaError_t launch_adj_add(int64_t n, const double* a, const double* b, double* y, cudaStream_t s) {
  adj_add_kernel<<<256, kT, 0, s>>>(n, a, b, y);
  return cudaGetLastError();
}

cudaError_t launch_adj_lift(int64_t n, int k, const double* phi, const double* a, const double* q_ref,
                            double d, double* q, cudaStream_t s) {
  adj_lift_kernel<<<256, kT, 0, s>>>(n, k, phi, a, q_ref, d, q);
  return cudaGetLastError();
}

cudaError_t launch_adj_misfit(int64_t n, const double* q, const double* target, double* qtbar,
                              double* part, double* J, cudaStream_t s) {
  adj_misfit_kernel<<<256, kT, 0, s>>>(n, q, target, qtbar, part);
  adj_misfit_final_kernel<<<1, 32, 0, s>>>(part, 256, J);
  return cudaGetLastError();
}

// Wait bound of this translation unit's kernels (see rom_internal.cuh).
cudaError_t set_wait_limit_adjoint(long long cycles) { return set_wait_limit_here(cycles); }

}  // namespace rom
