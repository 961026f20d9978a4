// Reduced backward-Euler steps (Algorithm 1 line 10) and the lift of the
// reduced state (Eq. trial_approximation).
//
// Plain Galerkin (Eq. galerkin_continuous_rom discretised by backward Euler):
//   g(a) = a - a^n - dt Phi^T D f(q_ref + D^-1 Phi a) = 0.
// DEIM-Galerkin with U = Phi (Eq. deim_galerkin_rom):
//   g(a) = a - a^n - dt (P^T Phi)^+ P^T D f(q~(a)) = 0.
// Both are solved by Newton from a^n. The residual g is FP64 and fixes the
// root; the Jacobian  I - dt Phi^T D J_f D^-1 Phi  (or its sampled form) is
// formed in FP32 once per step at a^n and factorised by LU with partial
// pivoting in FP32 (a chord iteration). Stopping rule as the oracle:
// max|delta| <= tol (1 + max|a|).
#include <cfloat>
#include <cmath>

#include "rom_internal.cuh"
#include "rom_kernels.cuh"

namespace rom {

namespace {

struct RowF {
  double f;
  float dl, dc, dr;
};

__device__ __forceinline__ RowF burgers_f_row(double ul, double u, double ur, double nu,
                                              double inv_dx) {
  double Ll = 0.5 * fmax(ul, 0.0) * fmax(ul, 0.0);
  double Rl = 0.5 * fmin(u, 0.0) * fmin(u, 0.0);
  bool tl = Ll >= Rl;
  double Fl = tl ? Ll : Rl;
  double Lr = 0.5 * fmax(u, 0.0) * fmax(u, 0.0);
  double Rr = 0.5 * fmin(ur, 0.0) * fmin(ur, 0.0);
  bool tr = Lr >= Rr;
  double Fr = tr ? Lr : Rr;
  double inv_dx2 = inv_dx * inv_dx;
  RowF o;
  o.f = -(Fr - Fl) * inv_dx + nu * (ur - 2.0 * u + ul) * inv_dx2;
  double dFl_dl = tl ? fmax(ul, 0.0) : 0.0;
  double dFl_dc = tl ? 0.0 : fmin(u, 0.0);
  double dFr_dc = tr ? fmax(u, 0.0) : 0.0;
  double dFr_dr = tr ? 0.0 : fmin(ur, 0.0);
  o.dl = (float)(dFl_dl * inv_dx + nu * inv_dx2);
  o.dc = (float)((dFl_dc - dFr_dc) * inv_dx - 2.0 * nu * inv_dx2);
  o.dr = (float)(-dFr_dr * inv_dx + nu * inv_dx2);
  return o;
}

// In-place LU with partial pivoting of a k x k FP32 matrix (row-major, ld
// kMaxR) by one block.
__device__ void lu_factor(float* J, int* piv, int k) {
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

// Solve (LU) x = b for the RHS in x (FP32), by warp 0.
__device__ void lu_solve(const float* J, const int* piv, float* x, int k) {
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

}  // namespace

// ----------------------------------------------------------------------------
// Plain Galerkin: cooperative kernel over all rows.
// ----------------------------------------------------------------------------

template <int KM>
__global__ void __launch_bounds__(kBlock) galerkin_steps_kernel(StepArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int G = gridDim.x, b = blockIdx.x, t = threadIdx.x;
  const int64_t N = A.n, ld = A.ld;
  const int64_t beg = (int64_t)b * N / G, end = (int64_t)(b + 1) * N / G;
  const int rows = (int)(end - beg);
  const int k = *A.rank;
  const int stride = KM + 2;
  const double inv_dx = (double)N;

  // shared layout
  double* s_a = reinterpret_cast<double*>(smem_raw);          // KM
  double* s_ap = s_a + KM;                                     // KM
  double* s_g = s_ap + KM;                                     // KM
  double* red = s_g + KM;                                      // 32*KM
  double* s_sc = red + 32 * KM;                                // 8
  float* s_J = reinterpret_cast<float*>(s_sc + 8);             // kMaxR*kMaxR
  float* s_x = s_J + kMaxR * kMaxR;                            // kMaxR
  int* s_piv = reinterpret_cast<int*>(s_x + kMaxR);            // kMaxR
  double* s_qt = reinterpret_cast<double*>(s_piv + kMaxR);     // rows+2
  float* s_jl = reinterpret_cast<float*>(s_qt + (rows + 2));   // rows
  float* s_jc = s_jl + rows;
  float* s_jr = s_jc + rows;
  float* s_phi = s_jr + rows;                                  // 66 x KM  (FP32 tile)
  float* s_w = s_phi + 66 * KM;                                // 64 x KM

  for (int j = t; j < KM; j += blockDim.x) s_a[j] = (j < k) ? A.a[j] : 0.0;
  __syncthreads();
  int it_total = 0;
  for (int step = 0; step < A.nsteps; ++step) {
    for (int j = t; j < KM; j += blockDim.x) s_ap[j] = s_a[j];
    __syncthreads();
    bool conv = false;
    int it;
    for (it = 1; it <= A.max_iter; ++it) {
      const int par = it & 1;
      const bool jac_it = (it == 1);
      // lift q~ on rows beg-1 .. end (with the periodic halo)
      for (int e = t; e < rows + 2; e += blockDim.x) {
        int64_t i = (beg - 1 + e + N) % N;
        double s = 0.0;
#pragma unroll
        for (int j = 0; j < KM; ++j)
          if (j < k) s = fma(A.phi[j * ld + i], s_a[j], s);
        s_qt[e] = A.q_ref[i] + s * A.dinv[i];
      }
      __syncthreads();
      // f and D f, projected: partial g_j = sum_i Phi_ij d_i f_i
      double acc[KM];
#pragma unroll
      for (int j = 0; j < KM; ++j) acc[j] = 0.0;
      for (int e = t; e < rows; e += blockDim.x) {
        int64_t i = beg + e;
        RowF rf = burgers_f_row(s_qt[e], s_qt[e + 1], s_qt[e + 2], A.nu, inv_dx);
        double w = A.drow[i] * rf.f;
        s_jl[e] = rf.dl; s_jc[e] = rf.dc; s_jr[e] = rf.dr;
#pragma unroll
        for (int j = 0; j < KM; ++j)
          if (j < k) acc[j] = fma(A.phi[j * ld + i], w, acc[j]);
      }
      double* part = A.partials + (size_t)par * G * stride;
      {
        double* outv = s_g;
        // block reduction of acc
        const int lane = t & 31, wid = t >> 5, nw = blockDim.x >> 5;
#pragma unroll
        for (int j = 0; j < KM; ++j) {
          double v = warp_sum(acc[j]);
          if (lane == 0 && j < k) red[wid * KM + j] = v;
        }
        __syncthreads();
        for (int j = t; j < k; j += blockDim.x) {
          double s = 0.0;
          for (int w = 0; w < nw; ++w) s += red[w * KM + j];
          outv[j] = s;
          part[(size_t)b * stride + j] = s;
        }
        __syncthreads();
      }
      // FP32 Jacobian partial: sum_i Phi_ij d_i (J_f D^-1 Phi)_il over 64-row chunks
      if (jac_it) {
        float jacc[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) jacc[q] = 0.f;
        const int kk = k * k;
        for (int c0 = 0; c0 < rows; c0 += 64) {
          const int cr = min(64, rows - c0);
          for (int e = t; e < (cr + 2) * k; e += blockDim.x) {
            int rr = e / k, j = e % k;
            int64_t i = (beg + c0 - 1 + rr + N) % N;
            s_phi[rr * KM + j] = (float)A.phi[j * ld + i] * (float)A.dinv[i];
          }
          __syncthreads();
          for (int e = t; e < cr * k; e += blockDim.x) {
            int rr = e / k, l = e % k;
            int le = c0 + rr;
            float w = s_jl[le] * s_phi[rr * KM + l] + s_jc[le] * s_phi[(rr + 1) * KM + l] +
                      s_jr[le] * s_phi[(rr + 2) * KM + l];
            s_w[rr * KM + l] = w * (float)A.drow[beg + le];
          }
          __syncthreads();
          // s_phi row rr+1 holds Phi/d for row rr of the chunk: rescale by d
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            int e = t + q * kBlock;
            if (e < kk) {
              int j = e / k, l = e % k;
              float s = 0.f;
              for (int rr = 0; rr < cr; ++rr)
                s += s_phi[(rr + 1) * KM + j] * (float)A.drow[beg + c0 + rr] * s_w[rr * KM + l];
              jacc[q] += s;
            }
          }
          __syncthreads();
        }
        float* jp = A.jpartials + (size_t)b * kMaxR * kMaxR;
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          int e = t + q * kBlock;
          if (e < kk) jp[e] = jacc[q];
        }
      }
      if (!grid_sync(A.bar, A.status)) return;
      if (jac_it) {
        // distributed reduction of the Jacobian partials
        const int kk = k * k;
        const int e0 = (int)((int64_t)b * kk / G), e1 = (int)((int64_t)(b + 1) * kk / G);
        {
          const int lane = t & 31, wid = t >> 5, nw = blockDim.x >> 5;
          for (int e = e0 + wid; e < e1; e += nw) {
            float s = 0.f;
            for (int bb = lane; bb < G; bb += 32)
              s += __ldcg(&A.jpartials[(size_t)bb * kMaxR * kMaxR + e]);
            s = warp_sumf(s);
            if (lane == 0) A.jac[e] = s;
          }
        }
        if (!grid_sync(A.bar, A.status)) return;
        for (int e = t; e < kk; e += blockDim.x) {
          int j = e / k, l = e % k;
          s_J[j * kMaxR + l] = (j == l ? 1.0f : 0.0f) - (float)A.dt * __ldcg(&A.jac[e]);
        }
        __syncthreads();
        lu_factor(s_J, s_piv, k);
      }
      // residual g (every CTA, fixed-order sum) and Newton update
      grid_reduce_cols(part, G, stride, k, s_g);
      for (int j = t; j < k; j += blockDim.x) {
        double g = s_a[j] - s_ap[j] - A.dt * s_g[j];
        s_x[j] = (float)(-g);
      }
      __syncthreads();
      lu_solve(s_J, s_piv, s_x, k);
      if (t == 0) {
        double dm = 0.0, am = 0.0;
        bool bad = false;
        for (int j = 0; j < k; ++j) {
          double d = (double)s_x[j];
          s_a[j] += d;
          dm = fmax(dm, fabs(d));
          am = fmax(am, fabs(s_a[j]));
          bad = bad || !isfinite(s_a[j]);
        }
        s_sc[0] = bad ? -1.0 : ((dm <= A.tol * (1.0 + am)) ? 1.0 : 0.0);
      }
      __syncthreads();
      if (s_sc[0] < 0.0) {
        if (b == 0 && t == 0) record_status(A.status, kStNonFinite);
        return;
      }
      if (s_sc[0] > 0.0) { conv = true; break; }
    }
    it_total = conv ? it : A.max_iter;
    if (!conv) {
      if (b == 0 && t == 0) record_status(A.status, kStNoConv);
      return;
    }
  }
  if (b == 0) {
    for (int j = t; j < A.r; j += blockDim.x) A.a[j] = (j < k) ? s_a[j] : 0.0;
    if (t == 0) *A.iters = it_total;
  }
}

// ----------------------------------------------------------------------------
// DEIM-Galerkin: one CTA on the sample mesh.
// ----------------------------------------------------------------------------

template <int KM>
__global__ void __launch_bounds__(kBlock) hyper_steps_kernel(StepArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int t = threadIdx.x;
  const int k = *A.rank;
  const int ns = A.n_s;
  const double inv_dx = (double)A.n;
  double* s_a = reinterpret_cast<double*>(smem_raw);   // KM
  double* s_ap = s_a + KM;
  double* s_sc = s_ap + KM;                             // 8
  double* s_qt = s_sc + 8;                              // 3 ns
  double* s_f = s_qt + 3 * ns;                          // ns (d f at samples)
  float* s_J = reinterpret_cast<float*>(s_f + ns);      // kMaxR * kMaxR
  float* s_x = s_J + kMaxR * kMaxR;                     // kMaxR
  int* s_piv = reinterpret_cast<int*>(s_x + kMaxR);     // kMaxR
  float* s_jr3 = reinterpret_cast<float*>(s_piv + kMaxR);  // 3 ns  (J_f row)
  float* s_As = s_jr3 + 3 * ns;                         // ns x KM (FP32)
  double* s_dinv = reinterpret_cast<double*>(s_As + ns * KM + (ns * KM) % 2);  // 3 ns

  for (int e = t; e < 3 * ns; e += blockDim.x)
    s_dinv[e] = 1.0 / A.mesh[(size_t)e * kMeshStride + kMaxR + 1];
  for (int j = t; j < KM; j += blockDim.x) s_a[j] = (j < k) ? A.a[j] : 0.0;
  __syncthreads();
  int it_total = 0;
  for (int step = 0; step < A.nsteps; ++step) {
    for (int j = t; j < KM; j += blockDim.x) s_ap[j] = s_a[j];
    __syncthreads();
    bool conv = false;
    int it;
    for (it = 1; it <= A.max_iter; ++it) {
      // lift at the 3 stencil rows of every sample
      for (int e = t; e < 3 * ns; e += blockDim.x) {
        const double* row = A.mesh + (size_t)e * kMeshStride;
        double s = 0.0;
#pragma unroll
        for (int j = 0; j < KM; ++j)
          if (j < k) s = fma(row[j], s_a[j], s);
        s_qt[e] = row[kMaxR] + s * s_dinv[e];
      }
      __syncthreads();
      for (int q = t; q < ns; q += blockDim.x) {
        RowF rf = burgers_f_row(s_qt[3 * q], s_qt[3 * q + 1], s_qt[3 * q + 2], A.nu, inv_dx);
        const double dq = A.mesh[(size_t)(3 * q + 1) * kMeshStride + kMaxR + 1];
        s_f[q] = dq * rf.f;
        s_jr3[3 * q] = rf.dl; s_jr3[3 * q + 1] = rf.dc; s_jr3[3 * q + 2] = rf.dr;
      }
      __syncthreads();
      if (it == 1) {
        // sampled rows of D J_f D^-1 Phi (FP32)
        for (int e = t; e < ns * k; e += blockDim.x) {
          int q = e / k, l = e % k;
          float s = 0.f;
          for (int o = 0; o < 3; ++o) {
            const double* row = A.mesh + (size_t)(3 * q + o) * kMeshStride;
            s += s_jr3[3 * q + o] * (float)row[l] * (float)s_dinv[3 * q + o];
          }
          s_As[q * KM + l] = s * (float)A.mesh[(size_t)(3 * q + 1) * kMeshStride + kMaxR + 1];
        }
        __syncthreads();
        for (int e = t; e < k * k; e += blockDim.x) {
          int j = e / k, l = e % k;
          float s = 0.f;
          for (int q = 0; q < ns; ++q) s += (float)A.minv[(size_t)j * ns + q] * s_As[q * KM + l];
          s_J[j * kMaxR + l] = (j == l ? 1.0f : 0.0f) - (float)A.dt * s;
        }
        __syncthreads();
        lu_factor(s_J, s_piv, k);
      }
      for (int j = t; j < k; j += blockDim.x) {
        double s = 0.0;
        for (int q = 0; q < ns; ++q) s = fma(A.minv[(size_t)j * ns + q], s_f[q], s);
        double g = s_a[j] - s_ap[j] - A.dt * s;
        s_x[j] = (float)(-g);
      }
      __syncthreads();
      lu_solve(s_J, s_piv, s_x, k);
      if (t == 0) {
        double dm = 0.0, am = 0.0;
        bool bad = false;
        for (int j = 0; j < k; ++j) {
          double d = (double)s_x[j];
          s_a[j] += d;
          dm = fmax(dm, fabs(d));
          am = fmax(am, fabs(s_a[j]));
          bad = bad || !isfinite(s_a[j]);
        }
        s_sc[0] = bad ? -1.0 : ((dm <= A.tol * (1.0 + am)) ? 1.0 : 0.0);
      }
      __syncthreads();
      if (s_sc[0] < 0.0) {
        if (t == 0) record_status(A.status, kStNonFinite);
        return;
      }
      if (s_sc[0] > 0.0) { conv = true; break; }
    }
    it_total = conv ? it : A.max_iter;
    if (!conv) {
      if (t == 0) record_status(A.status, kStNoConv);
      return;
    }
  }
  for (int j = t; j < A.r; j += blockDim.x) A.a[j] = (j < k) ? s_a[j] : 0.0;
  if (t == 0) *A.iters = it_total;
}

// ----------------------------------------------------------------------------
// q~ = q_ref + D^-1 Phi a
// ----------------------------------------------------------------------------

template <int KM>
__global__ void lift_kernel(LiftArgs A) {
  const int k = *A.rank;
  __shared__ double s_a[KM];
  for (int j = threadIdx.x; j < KM; j += blockDim.x) s_a[j] = (j < k) ? A.a[j] : 0.0;
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < A.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < KM; ++j)
      if (j < k) s = fma(A.phi[j * A.ld + i], s_a[j], s);
    A.out[i] = A.q_ref[i] + s * A.dinv[i];
  }
}

// ----------------------------------------------------------------------------
// launchers
// ----------------------------------------------------------------------------

template <int KM>
static size_t galerkin_smem(int64_t n, int grid) {
  int rows = (int)((n + grid - 1) / grid) + 1;
  size_t bytes = sizeof(double) * (3 * KM + 32 * KM + 8) + sizeof(float) * (kMaxR * kMaxR + kMaxR) +
                 sizeof(int) * kMaxR + sizeof(double) * (rows + 2) + sizeof(float) * 3 * rows +
                 sizeof(float) * (66 * KM + 64 * KM) + 64;
  return bytes;
}

template <int KM>
static cudaError_t launch_galerkin_t(const StepArgs& A, int grid, cudaStream_t s) {
  size_t smem = galerkin_smem<KM>(A.n, grid);
  cudaError_t e = cudaFuncSetAttribute(galerkin_steps_kernel<KM>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  StepArgs a = A;
  void* args[] = {&a};
  return cudaLaunchCooperativeKernel((const void*)galerkin_steps_kernel<KM>, dim3(grid),
                                     dim3(kBlock), args, smem, s);
}

cudaError_t launch_galerkin_steps(const StepArgs& A, int km, int grid, cudaStream_t s) {
  switch (km) {
    case 9: return launch_galerkin_t<9>(A, grid, s);
    case 17: return launch_galerkin_t<17>(A, grid, s);
    case 33: return launch_galerkin_t<33>(A, grid, s);
    default: return launch_galerkin_t<65>(A, grid, s);
  }
}

template <int KM>
static cudaError_t launch_hyper_t(const StepArgs& A, cudaStream_t s) {
  int ns = A.n_s;
  size_t smem = sizeof(double) * (2 * KM + 8 + 3 * ns + ns) + sizeof(float) * (kMaxR * kMaxR + kMaxR) +
                sizeof(int) * kMaxR + sizeof(float) * (3 * ns + ns * KM + 1) + sizeof(double) * 3 * ns + 64;
  cudaError_t e = cudaFuncSetAttribute(hyper_steps_kernel<KM>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  hyper_steps_kernel<KM><<<1, kBlock, smem, s>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_hyper_steps(const StepArgs& A, int km, cudaStream_t s) {
  switch (km) {
    case 9: return launch_hyper_t<9>(A, s);
    case 17: return launch_hyper_t<17>(A, s);
    case 33: return launch_hyper_t<33>(A, s);
    default: return launch_hyper_t<65>(A, s);
  }
}

template <int KM>
static cudaError_t launch_lift_t(const LiftArgs& A, cudaStream_t s) {
  int blocks = (int)((A.n + 255) / 256);
  if (blocks > 1024) blocks = 1024;
  lift_kernel<KM><<<blocks, 256, 0, s>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_lift(const LiftArgs& A, int km, cudaStream_t s) {
  switch (km) {
    case 9: return launch_lift_t<9>(A, s);
    case 17: return launch_lift_t<17>(A, s);
    case 33: return launch_lift_t<33>(A, s);
    default: return launch_lift_t<65>(A, s);
  }
}

}  // namespace rom
