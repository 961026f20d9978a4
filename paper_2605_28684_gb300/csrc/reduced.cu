// Reduced backward-Euler steps of the online loop of Algorithm 1 and the lift of the
// reduced state (Eq. trial_approximation).
//
// Plain Galerkin (Eq. galerkin_continuous_rom discretised by backward Euler):
//   g(a) = a - a^n - dt Phi^T D f(q_ref + D^-1 Phi a) = 0.
// DEIM-Galerkin with U = Phi (Eq. deim_galerkin_rom):
//   g(a) = a - a^n - dt (P^T Phi)^+ P^T D f(q~(a)) = 0.
// Both are solved by Newton from a^n. The residual g is FP64 and fixes the
// root; the Jacobian  I - dt Phi^T D J_f D^-1 Phi  (or its sampled form) is
// formed in FP32 once per step at a^n (the sampled form: once per launch, and
// again whenever a step needs more than three iterations) and factorised by
// LU with partial pivoting in FP32 (a chord iteration). Stopping rule as the oracle:
// max|delta| <= tol (1 + max|a|).
// The explicit form (App. D, the RDE solver's scheme) advances the same
// right-hand sides da/dt = Phi^T D f (or (P^T Phi)^+ P^T D f) by the
// four-stage, third-order SSP Runge-Kutta scheme: each of the four stages is
// one pass of the Newton loop's residual evaluation, x <- x + dt/2 rhs(x),
// with x <- 2/3 a^n + 1/3 x after the third; no Jacobian, no iteration.
#include <cfloat>
#include <cmath>
#include <type_traits>

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

}  // namespace

// ----------------------------------------------------------------------------
// Plain Galerkin: cooperative kernel over all rows.
// ----------------------------------------------------------------------------

template <int KM, typename TPhi>
__global__ void __launch_bounds__(kBlock) galerkin_steps_kernel(StepArgs A) {
  using Acc = TPhi;   // FP32 lift and projections with FP32 accumulation in the mixed form
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const TPhi* phi = basis<TPhi>(A);
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
  float* s_Ji = s_w + 64 * KM;                                 // kMaxR x kMaxR: inverse Jacobian

  for (int j = t; j < KM; j += blockDim.x) s_a[j] = (j < k) ? A.a[j] : 0.0;
  __syncthreads();
  int it_total = 0;
  for (int step = 0; step < A.nsteps; ++step) {
    for (int j = t; j < KM; j += blockDim.x) s_ap[j] = s_a[j];
    __syncthreads();
    bool conv = false;
    int it;
    const int nit = A.explicit_rk ? 4 : A.max_iter;
    for (it = 1; it <= nit; ++it) {
      const int par = it & 1;
      const bool jac_it = !A.explicit_rk && (it == 1);
      // lift q~ on rows beg-1 .. end (with the periodic halo)
      for (int e = t; e < rows + 2; e += blockDim.x) {
        int64_t i = (beg - 1 + e + N) % N;
        Acc s = Acc(0);
#pragma unroll
        for (int j = 0; j < KM; ++j)
          if (j < k) s = fma((Acc)phi[j * ld + i], (Acc)s_a[j], s);
        s_qt[e] = A.q_ref[i] + (double)s * A.dinv[i];
      }
      __syncthreads();
      // f and D f, projected: partial g_j = sum_i Phi_ij d_i f_i
      Acc acc[KM];
#pragma unroll
      for (int j = 0; j < KM; ++j) acc[j] = Acc(0);
      for (int e = t; e < rows; e += blockDim.x) {
        int64_t i = beg + e;
        RowF rf = burgers_f_row(s_qt[e], s_qt[e + 1], s_qt[e + 2], A.nu, inv_dx);
        Acc w = (Acc)(A.drow[i] * rf.f);
        s_jl[e] = rf.dl; s_jc[e] = rf.dc; s_jr[e] = rf.dr;
#pragma unroll
        for (int j = 0; j < KM; ++j)
          if (j < k) acc[j] = fma((Acc)phi[j * ld + i], w, acc[j]);
      }
      double* part = A.partials + (size_t)par * G * stride;
      {
        double* outv = s_g;
        // block reduction of acc
        const int lane = t & 31, wid = t >> 5, nw = blockDim.x >> 5;
#pragma unroll
        for (int j = 0; j < KM; ++j) {
          double v = warp_sum((double)acc[j]);
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
            s_phi[rr * KM + j] = (float)phi[j * ld + i] * (float)A.dinv[i];
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
        lu_inverse(s_J, s_piv, s_Ji, k);
      }
      // residual g (every CTA, fixed-order sum) and Newton update
      grid_reduce_cols(part, G, stride, k, s_g);
      if (A.explicit_rk) {
        int bad = 0;
        for (int j = t; j < k; j += blockDim.x) {
          double v = s_a[j] + 0.5 * A.dt * s_g[j];
          if (it == 3) v = (2.0 / 3.0) * s_ap[j] + (1.0 / 3.0) * v;
          s_a[j] = v;
          bad |= !isfinite(v);
        }
        if (__syncthreads_or(bad)) {
          if (b == 0 && t == 0) record_status(A.status, kStNonFinite);
          return;
        }
        if (it == 4) conv = true;
        continue;
      }
      for (int j = t; j < k; j += blockDim.x) {
        double g = s_a[j] - s_ap[j] - A.dt * s_g[j];
        s_x[j] = (float)(-g);
      }
      __syncthreads();
      inv_apply(s_Ji, s_x, k);
      if (t < 32) {
        unsigned int kd = 0u, ka = 0u;
        bool bad = false;
        for (int j = (t & 31); j < k; j += 32) {
          float d = s_x[j];
          double an = s_a[j] + (double)d;
          s_a[j] = an;
          kd = max(kd, __float_as_uint(fabsf(d)));
          ka = max(ka, __float_as_uint(fabsf((float)an)));
          bad = bad || !isfinite(an);
        }
        kd = warp_max_u32(kd);
        ka = warp_max_u32(ka);
        bad = __any_sync(0xffffffffu, bad);
        // the mixed form's residual carries FP32 rounding: stop at that level
        const double tol = std::is_same<TPhi, float>::value ? fmax(A.tol, 1e-7) : A.tol;
        if (t == 0)
          s_sc[0] = bad ? -1.0
                        : (((double)__uint_as_float(kd) <= tol * (1.0 + (double)__uint_as_float(ka))) ? 1.0 : 0.0);
      }
      __syncthreads();
      if (s_sc[0] < 0.0) {
        if (b == 0 && t == 0) record_status(A.status, kStNonFinite);
        return;
      }
      if (s_sc[0] > 0.0) { conv = true; break; }
    }
    it_total = A.explicit_rk ? 0 : (conv ? it : A.max_iter);
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
//
// The stencil mesh (3 n_s rows of Phi, q_ref and 1/D) is staged in shared
// memory once; every FP64 loop runs over the actual rank k with all lanes busy:
// the lift is one thread per mesh row, the residual M (D f) is one warp per
// reduced coordinate with lanes over the samples.
// ----------------------------------------------------------------------------

template <int KM>
__global__ void __launch_bounds__(kBlock) hyper_steps_kernel(StepArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5, nw = blockDim.x >> 5;
  const int k = *A.rank;
  const int ns = A.n_s;
  const int nm = 3 * ns;
  const double inv_dx = (double)A.n;
  double* s_mesh = reinterpret_cast<double*>(smem_raw);  // nm x k
  double* s_qr = s_mesh + (size_t)nm * k;                // nm
  double* s_di = s_qr + nm;                              // nm (1/d)
  double* s_qt = s_di + nm;                              // nm (lifted)
  double* s_f = s_qt + nm;                               // ns (d f at samples)
  double* s_dc = s_f + ns;                               // ns (d at samples)
  double* s_a = s_dc + ns;                               // KM
  double* s_ap = s_a + KM;                               // KM: a^n
  double* s_app = s_ap + KM;                             // KM: a^(n-1)
  double* s_sc = s_app + KM;                             // 8
  float* s_J = reinterpret_cast<float*>(s_sc + 8);       // kMaxR * kMaxR
  float* s_x = s_J + kMaxR * kMaxR;                      // kMaxR
  int* s_piv = reinterpret_cast<int*>(s_x + kMaxR);      // kMaxR
  float* s_jr3 = reinterpret_cast<float*>(s_piv + kMaxR);  // nm
  float* s_As = s_jr3 + nm;                              // ns x k (FP32)
  float* s_mf = s_As + ns * k;                           // nm x k: Phi row / d (FP32)
  float* s_Mf = s_mf + nm * k;                           // k x ns: (P^T Phi)^+ (FP32)
  float* s_dcf = s_Mf + k * ns;                          // ns: d at samples (FP32)
  float* s_Ji = s_dcf + ns;                              // kMaxR * kMaxR: inverse Jacobian (FP32)

  for (int e = t; e < nm * k; e += blockDim.x) {
    int row = e / k, j = e % k;
    s_mesh[e] = A.mesh[(size_t)row * kMeshStride + j];
  }
  for (int e = t; e < nm; e += blockDim.x) {
    s_qr[e] = A.mesh[(size_t)e * kMeshStride + kMaxR];
    s_di[e] = 1.0 / A.mesh[(size_t)e * kMeshStride + kMaxR + 1];
  }
  for (int q = t; q < ns; q += blockDim.x) s_dc[q] = A.mesh[(size_t)(3 * q + 1) * kMeshStride + kMaxR + 1];
  __syncthreads();
  // FP32 copies for the Jacobian, converted once per launch
  for (int e = t; e < nm * k; e += blockDim.x) s_mf[e] = (float)(s_mesh[e] * s_di[e / k]);
  for (int e = t; e < k * ns; e += blockDim.x) s_Mf[e] = (float)A.minv[e];
  for (int q = t; q < ns; q += blockDim.x) s_dcf[q] = (float)s_dc[q];
  for (int j = t; j < KM; j += blockDim.x) s_a[j] = (j < k) ? A.a[j] : 0.0;
  __syncthreads();
  int it_total = 0;
  // The sampled Jacobian (its FP32 inverse) is formed at the first iteration
  // of the launch and kept over its steps (the basis and samples are fixed
  // within a launch, and z dt is short); it is formed again at the next
  // iteration whenever a step has not converged after kChordIters.
  constexpr int kChordIters = 3;
  bool need_jac = true;
  for (int step = 0; step < A.nsteps; ++step) {
    // a^n; the backward-Euler iteration of a step starts from the polynomial
    // extrapolation of the launch's earlier steps: 2 a^n - a^(n-1) at the
    // second step (error O(dt^2)), 3 a^n - 3 a^(n-1) + a^(n-2) from the third
    // on (error O(dt^3)); the root is the same, reached in fewer iterations
    for (int j = t; j < k; j += blockDim.x) {
      const double an = s_a[j], an1 = s_ap[j];
      if (!A.explicit_rk) {
        if (step == 1) s_a[j] = 2.0 * an - an1;
        else if (step > 1) s_a[j] = fma(3.0, an - an1, s_app[j]);
      }
      s_app[j] = an1;
      s_ap[j] = an;
    }
    __syncthreads();
    bool conv = false;
    int it;
    const int nit = A.explicit_rk ? 4 : A.max_iter;
    for (it = 1; it <= nit; ++it) {
      // lift at the 3 stencil rows of every sample
      for (int e = t; e < nm; e += blockDim.x) {
        const double* row = s_mesh + (size_t)e * k;
        double s = 0.0;
        for (int j = 0; j < k; ++j) s = fma(row[j], s_a[j], s);
        s_qt[e] = s_qr[e] + s * s_di[e];
      }
      __syncthreads();
      for (int q = t; q < ns; q += blockDim.x) {
        RowF rf = burgers_f_row(s_qt[3 * q], s_qt[3 * q + 1], s_qt[3 * q + 2], A.nu, inv_dx);
        s_f[q] = s_dc[q] * rf.f;                          // d f at the sample
        s_jr3[3 * q] = rf.dl; s_jr3[3 * q + 1] = rf.dc; s_jr3[3 * q + 2] = rf.dr;
      }
      __syncthreads();
      if (need_jac && !A.explicit_rk) {
        need_jac = false;
        // sampled rows of D J_f D^-1 Phi (FP32), then J = I - dt M A (FP32)
        for (int e = t; e < ns * k; e += blockDim.x) {
          int q = e / k, l = e % k;
          float s = 0.f;
          for (int o = 0; o < 3; ++o) s += s_jr3[3 * q + o] * s_mf[(size_t)(3 * q + o) * k + l];
          s_As[q * k + l] = s * s_dcf[q];
        }
        __syncthreads();
        for (int e = wid; e < k * k; e += nw) {
          int j = e / k, l = e % k;
          float s = 0.f;
          for (int q = lane; q < ns; q += 32) s += s_Mf[(size_t)j * ns + q] * s_As[q * k + l];
          s = warp_sumf(s);
          if (lane == 0) s_J[j * kMaxR + l] = (j == l ? 1.0f : 0.0f) - (float)A.dt * s;
        }
        __syncthreads();
        lu_factor(s_J, s_piv, k);
        lu_inverse(s_J, s_piv, s_Ji, k);
      }
      if (A.explicit_rk) {
        // stage: a_j <- a_j + dt/2 sum_q M_jq (d f)_q (one warp per j; the
        // lift above read the old a, and a_j is written by its own warp only)
        int bad = 0;
        for (int j = wid; j < k; j += nw) {
          double s = 0.0;
          for (int q = lane; q < ns; q += 32) s = fma(A.minv[(size_t)j * ns + q], s_f[q], s);
          s = warp_sum(s);
          if (lane == 0) {
            double v = s_a[j] + 0.5 * A.dt * s;
            if (it == 3) v = (2.0 / 3.0) * s_ap[j] + (1.0 / 3.0) * v;
            s_a[j] = v;
            bad |= !isfinite(v);
          }
        }
        if (__syncthreads_or(bad)) {
          if (t == 0) record_status(A.status, kStNonFinite);
          return;
        }
        if (it == 4) conv = true;
        continue;
      }
      // residual g_j = a_j - a^n_j - dt sum_q M_jq (d f)_q: one warp per j
      for (int j = wid; j < k; j += nw) {
        double s = 0.0;
        for (int q = lane; q < ns; q += 32) s = fma(A.minv[(size_t)j * ns + q], s_f[q], s);
        s = warp_sum(s);
        if (lane == 0) s_x[j] = (float)(-(s_a[j] - s_ap[j] - A.dt * s));
      }
      __syncthreads();
      inv_apply(s_Ji, s_x, k);
      if (t < 32) {
        // max |delta| (an FP32 value) and max |a| rounded to FP32 (it only
        // scales the tolerance), compared as integer keys
        unsigned int kd = 0u, ka = 0u;
        bool bad = false;
        for (int j = lane; j < k; j += 32) {
          float d = s_x[j];
          double an = s_a[j] + (double)d;
          s_a[j] = an;
          kd = max(kd, __float_as_uint(fabsf(d)));
          ka = max(ka, __float_as_uint(fabsf((float)an)));
          bad = bad || !isfinite(an);
        }
        kd = warp_max_u32(kd);
        ka = warp_max_u32(ka);
        bad = __any_sync(0xffffffffu, bad);
        if (lane == 0)
          s_sc[0] = bad ? -1.0
                        : (((double)__uint_as_float(kd) <= A.tol * (1.0 + (double)__uint_as_float(ka))) ? 1.0 : 0.0);
      }
      __syncthreads();
      if (s_sc[0] < 0.0) {
        if (t == 0) record_status(A.status, kStNonFinite);
        return;
      }
      if (s_sc[0] > 0.0) { conv = true; break; }
      if (it >= kChordIters) need_jac = true;
    }
    it_total = A.explicit_rk ? 0 : (conv ? it : A.max_iter);
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

template <int KM, typename TPhi>
__global__ void lift_kernel(LiftArgs A) {
  const TPhi* phi = basis<TPhi>(A);
  const int k = *A.rank;
  __shared__ double s_a[KM];
  for (int j = threadIdx.x; j < KM; j += blockDim.x) s_a[j] = (j < k) ? A.a[j] : 0.0;
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < A.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < KM; ++j)
      if (j < k) s = fma((double)phi[j * A.ld + i], s_a[j], s);
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
                 sizeof(float) * (66 * KM + 64 * KM + kMaxR * kMaxR) + 64;
  return bytes;
}

template <int KM, typename TPhi>
static cudaError_t launch_galerkin_tt(const StepArgs& A, int grid, cudaStream_t s) {
  size_t smem = galerkin_smem<KM>(A.n, grid);
  cudaError_t e = cudaFuncSetAttribute(galerkin_steps_kernel<KM, TPhi>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  StepArgs a = A;
  void* args[] = {&a};
  return cudaLaunchCooperativeKernel((const void*)galerkin_steps_kernel<KM, TPhi>, dim3(grid),
                                     dim3(kBlock), args, smem, s);
}

template <int KM>
static cudaError_t launch_galerkin_t(const StepArgs& A, int grid, cudaStream_t s) {
  return A.phi32 ? launch_galerkin_tt<KM, float>(A, grid, s) : launch_galerkin_tt<KM, double>(A, grid, s);
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
  // sized for the largest rank the context can reach (k <= r <= KM - 1)
  const size_t ns = A.n_s, nm = 3 * ns, kmax = KM - 1;
  size_t smem = sizeof(double) * (nm * kmax + 3 * nm + 2 * ns + 3 * KM + 8) +
                sizeof(float) * (kMaxR * kMaxR + kMaxR) + sizeof(int) * kMaxR +
                sizeof(float) * (nm + ns * kmax + nm * kmax + kmax * ns + ns + kMaxR * kMaxR) + 64;
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
  if (A.phi32) lift_kernel<KM, float><<<blocks, 256, 0, s>>>(A);
  else lift_kernel<KM, double><<<blocks, 256, 0, s>>>(A);
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

// Wait bound of this translation unit's kernels (see rom_internal.cuh).
cudaError_t set_wait_limit_reduced(long long cycles) { return set_wait_limit_here(cycles); }

}  // namespace rom
