// Least-squares Petrov-Galerkin reduced steps (paper Sec. 3.1, Eq.
// lspg_minimization with the backward-Euler test basis of Eq.
// lspg_test_basis_be), Burgers, FP64.
//
// Each step minimises |D r(q~(a))| with r(q) = q - q~(a^n) - dt f(q) (Eq.
// be_residual_rom_section), i.e. D r = Phi (a - a^n) - dt D f(q~(a)), by
// Gauss-Newton: (Psi^T Psi) delta = -Psi^T D r with
// Psi = (I - dt D J_f D^-1) Phi, until max|delta| <= tol (1 + max|a|). The fixed
// point satisfies Eq. lspg_stationarity, Psi^T D r = 0.
//
// One cooperative launch runs nsteps steps. Per iteration every CTA stages its
// rows in chunks of 64 (Phi rows with one halo row on each side), forms the
// lifted state, f and the Jacobian row, the residual and the Psi rows, and
// accumulates Psi^T Psi and Psi^T D r (FP64); after one grid barrier every
// CTA sums the partials in CTA order and solves the k x k normal equations by
// Cholesky (FP64). Partials alternate between two buffers by iteration
// parity, so one barrier per iteration suffices.
//
// With hyper-reduction (n_s > 0) the hyper-reduced LSPG step of Eq.
// hyperreduced_lspg_stationarity, with the DEIM basis equal to Phi, has the
// DEIM-Galerkin root as its minimiser (see the API); this file covers n_s = 0.
#include <cfloat>
#include <cmath>

#include "burgers_stencil.cuh"
#include "rom_internal.cuh"
#include "rom_kernels.cuh"

namespace rom {

namespace {

constexpr int kCh = 64;   // rows per staged chunk

__device__ __forceinline__ int64_t wrapi(int64_t i, int64_t n) {
  i %= n;
  return i < 0 ? i + n : i;
}

__global__ void __launch_bounds__(kBlock) lspg_steps_kernel(StepArgs A) {
  extern __shared__ __align__(16) double smem[];
  double* s_phi = smem;                        // (kCh + 2) x kMaxR
  double* s_psi = s_phi + (kCh + 2) * kMaxR;   // kCh x kMaxR
  double* s_u = s_psi + kCh * kMaxR;           // kCh + 2
  double* s_di = s_u + (kCh + 2);              // kCh + 2: 1 / d
  double* s_res = s_di + (kCh + 2);            // kCh
  double* s_a = s_res + kCh;                   // kMaxR
  double* s_ap = s_a + kMaxR;                  // kMaxR
  double* s_x = s_ap + kMaxR;                  // kMaxR
  double* s_M = s_x + kMaxR;                   // kMaxR x kMaxR
  double* red = s_M + kMaxR * kMaxR;           // 32
  double* s_fl = red + 32;                     // 4
  const int G = gridDim.x, b = blockIdx.x, t = threadIdx.x;
  const int64_t N = A.n, ld = A.ld;
  const int64_t beg = (int64_t)b * N / G, end = (int64_t)(b + 1) * N / G;
  const int k = *A.rank, kk = k * k;
  const double inv_dx = (double)N, dt = A.dt;
  const size_t pstride = (size_t)kMaxR * kMaxR + kMaxR;
  for (int j = t; j < kMaxR; j += blockDim.x) s_a[j] = (j < k) ? A.a[j] : 0.0;
  __syncthreads();
  int gi = 0;            // iteration count over all steps (buffer parity)
  int it_last = 0;
  for (int step = 0; step < A.nsteps; ++step) {
    for (int j = t; j < kMaxR; j += blockDim.x) s_ap[j] = s_a[j];
    __syncthreads();
    bool conv = false;
    int it;
    for (it = 1; it <= A.max_iter; ++it) {
      const int par = (gi++) & 1;
      double macc[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) macc[q] = 0.0;
      double vacc = 0.0;
      for (int64_t c0 = beg; c0 < end; c0 += kCh) {
        const int cr = (int)min((int64_t)kCh, end - c0);
        for (int e = t; e < (cr + 2) * k; e += blockDim.x) {
          const int rr = e / k, j = e % k;
          s_phi[rr * kMaxR + j] = A.phi[(size_t)j * ld + wrapi(c0 - 1 + rr, N)];
        }
        __syncthreads();
        for (int rr = t; rr < cr + 2; rr += blockDim.x) {
          const int64_t i = wrapi(c0 - 1 + rr, N);
          double s = 0.0;
          for (int j = 0; j < k; ++j) s = fma(s_phi[rr * kMaxR + j], s_a[j], s);
          s_di[rr] = A.dinv[i];
          s_u[rr] = A.q_ref[i] + s * s_di[rr];
        }
        __syncthreads();
        for (int rr = t; rr < cr; rr += blockDim.x) {
          const int64_t i = c0 + rr;
          const StencilRow st = burgers_stencil(s_u[rr], s_u[rr + 1], s_u[rr + 2], A.nu, inv_dx);
          const double di = A.drow[i];
          double da = 0.0;
          for (int j = 0; j < k; ++j) da = fma(s_phi[(rr + 1) * kMaxR + j], s_a[j] - s_ap[j], da);
          s_res[rr] = da - dt * di * st.f;
          const double cl = dt * di * st.dl * s_di[rr], cc = dt * di * st.dc * s_di[rr + 1],
                       cr_ = dt * di * st.dr * s_di[rr + 2];
          for (int l = 0; l < k; ++l)
            s_psi[rr * kMaxR + l] = s_phi[(rr + 1) * kMaxR + l] -
                                    (cl * s_phi[rr * kMaxR + l] + cc * s_phi[(rr + 1) * kMaxR + l] +
                                     cr_ * s_phi[(rr + 2) * kMaxR + l]);
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int e = t + q * kBlock;
          if (e < kk) {
            const int j = e / k, l = e % k;
            if (l >= j) {
              double s = 0.0;
              for (int rr = 0; rr < cr; ++rr) s = fma(s_psi[rr * kMaxR + j], s_psi[rr * kMaxR + l], s);
              macc[q] += s;
            }
          }
        }
        if (t < k)
          for (int rr = 0; rr < cr; ++rr) vacc = fma(s_psi[rr * kMaxR + t], s_res[rr], vacc);
        __syncthreads();
      }
      double* part = A.npart + (size_t)par * G * pstride + (size_t)b * pstride;
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int e = t + q * kBlock;
        if (e < kk) part[e] = macc[q];
      }
      if (t < k) part[kMaxR * kMaxR + t] = vacc;
      if (!grid_sync(A.bar, A.status)) return;
      // normal equations, summed in CTA order by every CTA
      const double* p0 = A.npart + (size_t)par * G * pstride;
      for (int e = t; e < kk; e += blockDim.x) {
        const int j = e / k, l = e % k;
        const int es = (l >= j) ? e : l * k + j;    // upper triangle holds the sums
        double s = 0.0;
        for (int bb = 0; bb < G; ++bb) s += __ldcg(&p0[(size_t)bb * pstride + es]);
        s_M[j * kMaxR + l] = s;
      }
      for (int j = t; j < k; j += blockDim.x) {
        double s = 0.0;
        for (int bb = 0; bb < G; ++bb) s += __ldcg(&p0[(size_t)bb * pstride + kMaxR * kMaxR + j]);
        s_x[j] = -s;
      }
      __syncthreads();
      // Cholesky M = L L^T (lower, in place), then L L^T x = -Psi^T D r
      for (int j = 0; j < k; ++j) {
        if (t == 0) s_M[j * kMaxR + j] = sqrt(fmax(s_M[j * kMaxR + j], DBL_MIN));
        __syncthreads();
        const double djj = s_M[j * kMaxR + j];
        for (int i = j + 1 + t; i < k; i += blockDim.x) s_M[i * kMaxR + j] /= djj;
        __syncthreads();
        const int rem = k - j - 1;
        for (int e = t; e < rem * rem; e += blockDim.x) {
          const int i = j + 1 + e / rem, l = j + 1 + e % rem;
          if (l <= i) s_M[i * kMaxR + l] -= s_M[i * kMaxR + j] * s_M[l * kMaxR + j];
        }
        __syncthreads();
      }
      if (t < 32) {
        for (int i = 0; i < k; ++i) {
          double s = 0.0;
          for (int l = t; l < i; l += 32) s += s_M[i * kMaxR + l] * s_x[l];
          s = warp_sum(s);
          if (t == 0) s_x[i] = (s_x[i] - s) / s_M[i * kMaxR + i];
          __syncwarp();
        }
        for (int i = k - 1; i >= 0; --i) {
          double s = 0.0;
          for (int l = i + 1 + t; l < k; l += 32) s += s_M[l * kMaxR + i] * s_x[l];
          s = warp_sum(s);
          if (t == 0) s_x[i] = (s_x[i] - s) / s_M[i * kMaxR + i];
          __syncwarp();
        }
        // update and stopping rule (max|delta| <= tol (1 + max|a|)), NaN check
        double md = 0.0, ma = 0.0;
        bool bad = false;
        for (int j = t; j < k; j += 32) {
          const double an = s_a[j] + s_x[j];
          s_a[j] = an;
          md = fmax(md, fabs(s_x[j]));
          ma = fmax(ma, fabs(an));
          bad = bad || !isfinite(an);
        }
        md = warp_max(md);
        ma = warp_max(ma);
        bad = __any_sync(0xffffffffu, bad);
        if (t == 0) s_fl[0] = bad ? -1.0 : (md <= A.tol * (1.0 + ma) ? 1.0 : 0.0);
      }
      __syncthreads();
      if (s_fl[0] < 0.0) {
        if (b == 0 && t == 0) record_status(A.status, kStNonFinite);
        return;
      }
      if (s_fl[0] > 0.0) { conv = true; break; }
    }
    if (!conv) {
      if (b == 0 && t == 0) record_status(A.status, kStNoConv);
      return;
    }
    it_last = it;
  }
  if (b == 0) {
    for (int j = t; j < A.r; j += blockDim.x) A.a[j] = (j < k) ? s_a[j] : 0.0;
    if (t == 0) *A.iters = it_last;
  }
}

}  // namespace

size_t lspg_partial_doubles(int grid) { return (size_t)2 * grid * ((size_t)kMaxR * kMaxR + kMaxR); }

cudaError_t launch_lspg_steps(const StepArgs& A, int grid, cudaStream_t s) {
  if (!A.npart) return cudaErrorInvalidValue;
  const size_t smem = sizeof(double) * ((kCh + 2) * kMaxR + kCh * kMaxR + 2 * (kCh + 2) + kCh +
                                        3 * kMaxR + kMaxR * kMaxR + 36);
  cudaError_t e = cudaFuncSetAttribute(lspg_steps_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  StepArgs a = A;
  void* args[] = {&a};
  return cudaLaunchCooperativeKernel((const void*)lspg_steps_kernel, dim3(grid), dim3(kBlock), args,
                                     smem, s);
}

// Wait bound of this translation unit's kernels (see rom_internal.cuh).
cudaError_t set_wait_limit_lspg(long long cycles) { return set_wait_limit_here(cycles); }

}  // namespace rom
