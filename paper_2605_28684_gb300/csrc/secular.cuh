// Secular-equation machinery of the core SVD of Algorithm 2 (internal).
//
// The core K = [[lam Sigma, p], [0, rho]] has left singular vectors equal to
// the eigenvectors of K K^T = diag(d)^2 + z z^T, a rank-one modification of a
// diagonal matrix (Bunch, Nielsen and Sorensen 1978). These helpers build the
// deflated, ascending-order problem and find one root per warp; the callers
// distribute the roots over warps or CTAs.
#pragma once

#include <cfloat>
#include <cmath>

#include "rom_internal.cuh"

namespace rom {
namespace {

struct SecularSetup {
  int n;                       // order of the core
  int k2;                      // non-deflated count
  int cidx[kMaxCore];          // compact -> position (ascending order)
  double D[kMaxCore];          // compact poles (ascending)
  double Z[kMaxCore];          // compact z (after deflating rotations)
  double dpos[kMaxCore];       // d by position (ascending)
  int defl[kMaxCore];          // 1 if position p is deflated
  int nrot;
  int rot_a[kMaxCore], rot_b[kMaxCore];
  double rot_c[kMaxCore], rot_s[kMaxCore];
  double znorm2;
};

// Builds the ascending-order secular problem from d (descending, by original
// index, d[n-1] = 0 for the new direction) and z. Run by one thread.
__device__ void secular_setup(SecularSetup& S, int n, const double* d_desc, const double* z_orig) {
  S.n = n;
  double dmax = 0.0, zn2 = 0.0;
  for (int p = 0; p < n; ++p) {
    S.dpos[p] = d_desc[n - 1 - p];
    dmax = fmax(dmax, fabs(S.dpos[p]));
    zn2 += z_orig[n - 1 - p] * z_orig[n - 1 - p];
  }
  double zp[kMaxCore];
  for (int p = 0; p < n; ++p) zp[p] = z_orig[n - 1 - p];
  const double tol = 8.0 * DBL_EPSILON * fmax(dmax, sqrt(zn2));
  S.nrot = 0;
  for (int p = 0; p < n; ++p) S.defl[p] = fabs(zp[p]) <= tol ? 1 : 0;
  int prev = -1;
  for (int p = 0; p < n; ++p) {
    if (S.defl[p]) continue;
    if (prev >= 0 && S.dpos[p] - S.dpos[prev] <= tol) {
      double rr = hypot(zp[prev], zp[p]);
      double c = zp[p] / rr, s = zp[prev] / rr;
      int q = S.nrot++;
      S.rot_a[q] = prev; S.rot_b[q] = p; S.rot_c[q] = c; S.rot_s[q] = s;
      zp[p] = rr;
      zp[prev] = 0.0;
      S.defl[prev] = 1;
    }
    prev = p;
  }
  int k2 = 0;
  double zz = 0.0;
  for (int p = 0; p < n; ++p) {
    if (S.defl[p]) continue;
    S.cidx[k2] = p;
    S.D[k2] = S.dpos[p];
    S.Z[k2] = zp[p];
    zz += zp[p] * zp[p];
    ++k2;
  }
  S.k2 = k2;
  S.znorm2 = zz;
}

// Root j (0-based, ascending) of the secular equation by one warp.
//
// Work in the shifted eigenvalue variable nu = s^2 - D_o^2 around the nearer
// pole D_o: f(nu) = 1 + sum_i z_i^2 / (Delta_i - nu), Delta_i = (D_i - D_o)(D_i + D_o),
// whose poles are all simple. Each update fits f ~ b - c/nu (the origin pole
// plus a constant) to f and f' at the current point, which is exact for one
// pole and converges fast near it; the bracket [lo, hi] between the poles
// guards every step (bisection otherwise). The iteration runs in FP32 on
// rescaled data first (cheap) and is finished by a few FP64 steps; a
// dependent FP64 operation costs tens of cycles on this part, so the
// number of FP64 steps is what sets the time.
__device__ void secular_root(const SecularSetup& S, int j, int& o_out, double& tau_out) {
  const int k2 = S.k2;
  const int lane = threadIdx.x & 31;
  int o;
  double lo, hi;
  if (j < k2 - 1) {
    double mid = 0.5 * (S.D[j] + S.D[j + 1]);
    double s = 0.0;
    for (int i = lane; i < k2; i += 32) s += S.Z[i] * S.Z[i] / ((S.D[i] - mid) * (S.D[i] + mid));
    double fm = 1.0 + warp_sum(s);
    if (fm >= 0.0) {
      o = j;
      lo = 0.0;
      hi = (mid - S.D[j]) * (mid + S.D[j]);
    } else {
      o = j + 1;
      lo = (mid - S.D[j + 1]) * (mid + S.D[j + 1]);
      hi = 0.0;
    }
  } else {
    o = k2 - 1;
    lo = 0.0;
    hi = S.znorm2;
  }
  const double Do = S.D[o];
  // per-lane terms (k2 <= 65: at most three per lane); the FP32 phase has
  // converged in at most a handful of steps and the FP64 finish in two or
  // three on the cores this method produces
  double dl[3], z2[3];
  int nt = 0;
  for (int i = lane; i < k2; i += 32, ++nt) {
    dl[nt] = (S.D[i] - Do) * (S.D[i] + Do);
    z2[nt] = S.Z[i] * S.Z[i];
  }
  // ---- FP32 phase on data scaled by 1 / ||z||^2 ----
  const double sc = 1.0 / S.znorm2;
  float dlf[3], z2f[3];
  for (int q = 0; q < nt; ++q) { dlf[q] = (float)(dl[q] * sc); z2f[q] = (float)(z2[q] * sc); }
  float flo = (float)(lo * sc), fhi = (float)(hi * sc);
  float nu = 0.5f * (flo + fhi);
  for (int it = 0; it < 60; ++it) {
    float f = 0.f, fp = 0.f, em = 0.f;
    for (int q = 0; q < nt; ++q) {
      float r = 1.0f / (dlf[q] - nu);
      float tq = z2f[q] * r;
      f += tq;
      fp += tq * r;
      em += fabsf(tq);
    }
    f = 1.0f + warp_sumf(f);
    fp = warp_sumf(fp);
    em = warp_sumf(em);
    if (fabsf(f) <= 8.0f * FLT_EPSILON * (1.0f + em)) break;   // root to working precision
    if (f < 0.f) flo = nu; else fhi = nu;
    // one-pole rational step, else Newton, else bisection (kept inside the bracket)
    float c = fp * nu * nu, bb = f + fp * nu;
    float nn = (bb != 0.f) ? c / bb : flo - 1.0f;
    if (!(nn > flo && nn < fhi)) nn = nu - f / fp;
    if (!(nn > flo && nn < fhi)) nn = 0.5f * (flo + fhi);
    bool stop = fabsf(nn - nu) <= 4.0f * FLT_EPSILON * fabsf(nn) || !(fhi > flo);
    nu = nn;
    if (stop) break;
  }
  // ---- FP64 finish ----
  double v = (double)nu / sc;
  if (!(v > lo && v < hi)) v = 0.5 * (lo + hi);
  for (int it = 0; it < 40; ++it) {
    double f = 0.0, fp = 0.0, em = 0.0;
    for (int q = 0; q < nt; ++q) {
      double r = 1.0 / (dl[q] - v);
      double tq = z2[q] * r;
      f += tq;
      fp += tq * r;
      em += fabs(tq);
    }
    f = 1.0 + warp_sum(f);
    fp = warp_sum(fp);
    em = warp_sum(em);
    // stop once f is at the level of its own rounding error
    if (fabs(f) <= 8.0 * DBL_EPSILON * (1.0 + em)) break;
    if (f < 0.0) lo = v; else hi = v;
    double c = fp * v * v, bb = f + fp * v;
    double nn = (bb != 0.0) ? c / bb : lo - 1.0;
    if (!(nn > lo && nn < hi)) nn = v - f / fp;
    if (!(nn > lo && nn < hi)) nn = 0.5 * (lo + hi);
    bool stop = fabs(nn - v) <= 2.0 * DBL_EPSILON * fabs(nn) ||
                (hi - lo) <= 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi));
    v = nn;
    if (stop) break;
  }
  // s = D_o + tau with tau (2 D_o + tau) = nu
  const double tau = v / (Do + sqrt(Do * Do + v));
  o_out = o;
  tau_out = tau;
}

// s_j - D_i and s_j + D_i for root j = (origin o, tau).
__device__ __forceinline__ double root_minus(const SecularSetup& S, int o, double tau, int i) {
  return (S.D[o] - S.D[i]) + tau;
}
__device__ __forceinline__ double root_plus(const SecularSetup& S, int o, double tau, int i) {
  return (S.D[o] + S.D[i]) + tau;
}

__device__ __forceinline__ double warp_prod(double v) {
  for (int o = 16; o > 0; o >>= 1) v *= __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace
}  // namespace rom
