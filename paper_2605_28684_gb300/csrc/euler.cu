// 1D Euler full-order model (paper App. B): conserved (rho, m, E), ideal gas,
// local Lax-Friedrichs (Rusanov) flux with s = max(|u_L|+c_L, |u_R|+c_R) (tie
// -> left), zero-gradient ghost cells, density and pressure floored at 1e-10
// when primitives are recovered. The state is variable-blocked:
// [rho_0..rho_{n-1}, m_0..m_{n-1}, E_0..E_{n-1}].
//
// Backward-Euler Newton step, one cooperative launch: the residual is FP64;
// the Jacobian of the discrete residual (3x3 blocks, the derivative of the
// selected branch of the max in s, floors' derivatives zero when active) is
// formed in FP32 and the block-tridiagonal system is solved in FP32 (it only
// steers the iteration). Partitioning as for the scalar solver: C chunks, one
// CTA each and one cell per thread; the last cell of every chunk is a
// separator; interior cells are eliminated by block parallel cyclic reduction
// in shared memory with seven right-hand-side columns
// (residual | coupling to the left separator | coupling to the right one),
// and the separators form a block-tridiagonal system of order C (not cyclic:
// the domain has two physical ends), solved by every CTA after one grid
// barrier.
#include <cmath>
#include <type_traits>

#include "rom_internal.cuh"
#include "rom_kernels.cuh"

namespace rom {

namespace {

constexpr double kRhoFloor = 1e-10, kPFloor = 1e-10;
constexpr int kEulerChunkCells = 256;       // cells per chunk (one thread each)
constexpr int kEulerChunkStride = 96;       // floats per published chunk summary

struct Cons { double r, m, e; };

__device__ __forceinline__ Cons load_cell(const double* U, int64_t n, int64_t i) {
  i = i < 0 ? 0 : (i >= n ? n - 1 : i);      // ghost cells copy the end states
  return Cons{U[i], U[n + i], U[2 * n + i]};
}

// FP64 Rusanov flux at the interface between L and R (App. B).
__device__ __forceinline__ void rusanov(const Cons& L, const Cons& R, double g, double F[3]) {
  double rl = fmax(L.r, kRhoFloor), ul = L.m / rl;
  double pl = fmax((g - 1.0) * (L.e - 0.5 * rl * ul * ul), kPFloor);
  double rr = fmax(R.r, kRhoFloor), ur = R.m / rr;
  double pr = fmax((g - 1.0) * (R.e - 0.5 * rr * ur * ur), kPFloor);
  double sl = fabs(ul) + sqrt(g * pl / rl), sr = fabs(ur) + sqrt(g * pr / rr);
  double s = sl >= sr ? sl : sr;
  F[0] = 0.5 * (L.m + R.m) - 0.5 * s * (R.r - L.r);
  F[1] = 0.5 * ((L.m * ul + pl) + (R.m * ur + pr)) - 0.5 * s * (R.m - L.m);
  F[2] = 0.5 * (ul * (L.e + pl) + ur * (R.e + pr)) - 0.5 * s * (R.e - L.e);
}

// FP32 per-cell derivatives: flux Jacobian dF[a][b] = dF_a/dU_b, the speed
// |u| + c and its gradient.
struct CellD { float dF[3][3]; float sp; float ds[3]; float U[3]; };

__device__ __forceinline__ CellD cell_derivs(const Cons& C, float g) {
  CellD o;
  float rraw = (float)C.r, m = (float)C.m, E = (float)C.e;
  o.U[0] = rraw; o.U[1] = m; o.U[2] = E;
  float rho = fmaxf(rraw, (float)kRhoFloor);
  float drho = rraw > (float)kRhoFloor ? 1.f : 0.f;
  float u = m / rho;
  float praw = (g - 1.f) * (E - 0.5f * rho * u * u);
  float p = fmaxf(praw, (float)kPFloor);
  float pact = praw > (float)kPFloor ? 1.f : 0.f;
  float g1 = g - 1.f;
  float du[3] = {-m / (rho * rho) * drho, 1.f / rho, 0.f};
  float dp[3] = {pact * g1 * 0.5f * m * m / (rho * rho) * drho, -pact * g1 * m / rho, pact * g1};
  for (int b = 0; b < 3; ++b) {
    o.dF[0][b] = (b == 1) ? 1.f : 0.f;
    o.dF[1][b] = m * du[b] + dp[b] + (b == 1 ? u : 0.f);
    o.dF[2][b] = du[b] * (E + p) + u * (dp[b] + (b == 2 ? 1.f : 0.f));
  }
  float c = sqrtf(g * p / rho);
  float drho_used[3] = {drho, 0.f, 0.f};
  float sgn = u >= 0.f ? 1.f : -1.f;
  for (int b = 0; b < 3; ++b) o.ds[b] = sgn * du[b] + 0.5f * c * (dp[b] / p - drho_used[b] / rho);
  o.sp = fabsf(u) + c;
  return o;
}

// dFhat/dU_L and dFhat/dU_R (FP32) at the interface between cells L and R.
__device__ __forceinline__ void rusanov_derivs(const CellD& L, const CellD& R, float dL[3][3],
                                               float dR[3][3]) {
  bool take_left = L.sp >= R.sp;
  float s = take_left ? L.sp : R.sp;
  float dU[3] = {R.U[0] - L.U[0], R.U[1] - L.U[1], R.U[2] - L.U[2]};
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      float eye = (a == b) ? 1.f : 0.f;
      float dsl = take_left ? L.ds[b] : 0.f, dsr = take_left ? 0.f : R.ds[b];
      dL[a][b] = 0.5f * L.dF[a][b] + 0.5f * s * eye - 0.5f * dU[a] * dsl;
      dR[a][b] = 0.5f * R.dF[a][b] - 0.5f * s * eye - 0.5f * dU[a] * dsr;
    }
}

// ---- 3x3 block helpers (FP32, row-major) ----
struct M3 { float v[9]; };
__device__ __forceinline__ M3 m3_zero() { M3 m; for (int e = 0; e < 9; ++e) m.v[e] = 0.f; return m; }
__device__ __forceinline__ M3 m3_eye() { M3 m = m3_zero(); m.v[0] = m.v[4] = m.v[8] = 1.f; return m; }
__device__ __forceinline__ M3 m3_mul(const M3& a, const M3& b) {
  M3 c;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      c.v[3 * i + j] = a.v[3 * i] * b.v[j] + a.v[3 * i + 1] * b.v[3 + j] + a.v[3 * i + 2] * b.v[6 + j];
  return c;
}
__device__ __forceinline__ M3 m3_add(const M3& a, const M3& b) {
  M3 c; for (int e = 0; e < 9; ++e) c.v[e] = a.v[e] + b.v[e]; return c;
}
__device__ __forceinline__ M3 m3_neg(const M3& a) { M3 c; for (int e = 0; e < 9; ++e) c.v[e] = -a.v[e]; return c; }
__device__ __forceinline__ M3 m3_inv(const M3& m) {
  const float* a = m.v;
  float c00 = a[4] * a[8] - a[5] * a[7], c01 = a[5] * a[6] - a[3] * a[8], c02 = a[3] * a[7] - a[4] * a[6];
  float det = a[0] * c00 + a[1] * c01 + a[2] * c02;
  float id = 1.f / det;
  M3 r;
  r.v[0] = c00 * id; r.v[1] = (a[2] * a[7] - a[1] * a[8]) * id; r.v[2] = (a[1] * a[5] - a[2] * a[4]) * id;
  r.v[3] = c01 * id; r.v[4] = (a[0] * a[8] - a[2] * a[6]) * id; r.v[5] = (a[2] * a[3] - a[0] * a[5]) * id;
  r.v[6] = c02 * id; r.v[7] = (a[1] * a[6] - a[0] * a[7]) * id; r.v[8] = (a[0] * a[4] - a[1] * a[3]) * id;
  return r;
}
// 3 x 7 right-hand side block: column 0 residual, 1-3 left coupling, 4-6 right coupling
struct R7 { float v[21]; };
__device__ __forceinline__ R7 r7_mul(const M3& a, const R7& b) {
  R7 c;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 7; ++j)
      c.v[7 * i + j] = a.v[3 * i] * b.v[j] + a.v[3 * i + 1] * b.v[7 + j] + a.v[3 * i + 2] * b.v[14 + j];
  return c;
}
__device__ __forceinline__ R7 r7_add(const R7& a, const R7& b) {
  R7 c; for (int e = 0; e < 21; ++e) c.v[e] = a.v[e] + b.v[e]; return c;
}

struct EulerNewtonArgs {
  const double* q_prev;
  double* q;
  int64_t n;          // cells
  double gamma, h, tol;
  int max_iter, C;
  float* chunk;       // C * kEulerChunkStride
  unsigned long long* maxbuf;
  GridBarrier* bar;
  int* status;
  int* iters;
};

__device__ __forceinline__ int64_t echunk_begin(int c, int C, int64_t n) { return (int64_t)c * n / C; }

// Shared layout: A, B, C blocks (9 floats each) and the 3x7 RHS (21) per cell.
constexpr int kCellFloats = 9 * 3 + 21;

__global__ void __launch_bounds__(kEulerChunkCells) euler_newton_kernel(EulerNewtonArgs A) {
  extern __shared__ __align__(16) float esm[];
  float* sA = esm;
  float* sB = sA + 9 * kEulerChunkCells;
  float* sC = sB + 9 * kEulerChunkCells;
  float* sD = sC + 9 * kEulerChunkCells;                 // 21 per cell
  __shared__ float rA[kMaxChunks * 9], rB[kMaxChunks * 9], rC[kMaxChunks * 9], rD[kMaxChunks * 3];
  __shared__ float rS[kMaxChunks * 3];
  __shared__ unsigned int red[32];

  const int Cn = A.C, c = blockIdx.x, t = threadIdx.x;
  const int64_t n = A.n;
  const int64_t beg = echunk_begin(c, Cn, n);
  const int m = (int)(echunk_begin(c + 1, Cn, n) - beg);
  const int mi = m - 1;
  const bool active = t < m;
  const int64_t i = beg + t;
  const float g32 = (float)A.gamma;
  const double inv_dx = (double)n;

  Cons u{0.0, 0.0, 0.0}, un{0.0, 0.0, 0.0};
  if (active) {
    u = Cons{A.q_prev[i], A.q_prev[n + i], A.q_prev[2 * n + i]};
    un = u;
    A.q[i] = u.r; A.q[n + i] = u.m; A.q[2 * n + i] = u.e;
  }
  int it = 0;
  bool done = false;
  if (!grid_sync(A.bar, A.status)) return;
  for (it = 1; it <= A.max_iter && !done; ++it) {
    const int par = it & 1;
    // ---- phase A: residual (FP64), Jacobian blocks (FP32), block PCR ----
    M3 a_t = m3_zero(), b_t = m3_eye(), c_t = m3_zero();
    R7 d_t;
    for (int e = 0; e < 21; ++e) d_t.v[e] = 0.f;
    if (active) {
      // neighbours (written by other threads/CTAs last iteration: read through
      // L2); the ghost cells beyond the ends copy the end states
      Cons ul = u, ur = u;
      if (i > 0) ul = Cons{__ldcg(&A.q[i - 1]), __ldcg(&A.q[n + i - 1]), __ldcg(&A.q[2 * n + i - 1])};
      if (i + 1 < n) ur = Cons{__ldcg(&A.q[i + 1]), __ldcg(&A.q[n + i + 1]), __ldcg(&A.q[2 * n + i + 1])};
      double Fl[3], Fr[3];
      rusanov(ul, u, A.gamma, Fl);
      rusanov(u, ur, A.gamma, Fr);
      double res[3];
      const double uu[3] = {u.r, u.m, u.e}, uun[3] = {un.r, un.m, un.e};
      for (int v = 0; v < 3; ++v) {
        double f = -(Fr[v] - Fl[v]) * inv_dx;
        res[v] = uu[v] - uun[v] - A.h * f;
        d_t.v[7 * v] = (float)(-res[v]);
      }
      // Jacobian blocks of the residual row
      CellD dl = cell_derivs(ul, g32), dc = cell_derivs(u, g32), dr = cell_derivs(ur, g32);
      float pL[3][3], pR[3][3], qL[3][3], qR[3][3];
      rusanov_derivs(dl, dc, pL, pR);     // interface i-1/2: (i-1, i)
      rusanov_derivs(dc, dr, qL, qR);     // interface i+1/2: (i, i+1)
      const float hx = (float)(A.h * inv_dx);
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          // df_i/dU_{i-1} = +pL/dx ; df_i/dU_i = -qL/dx + pR/dx ; df_i/dU_{i+1} = -qR/dx
          float lower = pL[a][b], diag = -qL[a][b] + pR[a][b], upper = -qR[a][b];
          if (i == 0) { diag += lower; lower = 0.f; }          // ghost = copy of cell 0
          if (i == n - 1) { diag += upper; upper = 0.f; }      // ghost = copy of cell n-1
          a_t.v[3 * a + b] = -hx * lower;
          b_t.v[3 * a + b] = (a == b ? 1.f : 0.f) - hx * diag;
          c_t.v[3 * a + b] = -hx * upper;
        }
    }
    if (t == m - 1) {   // separator cell: publish its equation (A, B, C, d)
      float* ch = A.chunk + (size_t)c * kEulerChunkStride;
      for (int e = 0; e < 9; ++e) { ch[e] = a_t.v[e]; ch[9 + e] = b_t.v[e]; ch[18 + e] = c_t.v[e]; }
      for (int v = 0; v < 3; ++v) ch[27 + v] = d_t.v[7 * v];
    }
    if (t < mi) {
      if (t == 0) {      // coupling to the left separator -> columns 1..3
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) d_t.v[7 * a + 1 + b] = -a_t.v[3 * a + b];
        a_t = m3_zero();
      }
      if (t == mi - 1) { // coupling to this chunk's separator -> columns 4..6
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) d_t.v[7 * a + 4 + b] = -c_t.v[3 * a + b];
        c_t = m3_zero();
      }
    } else {
      a_t = m3_zero(); b_t = m3_eye(); c_t = m3_zero();
      for (int e = 0; e < 21; ++e) d_t.v[e] = 0.f;
    }
    for (int e = 0; e < 9; ++e) { sA[9 * t + e] = a_t.v[e]; sB[9 * t + e] = b_t.v[e]; sC[9 * t + e] = c_t.v[e]; }
    for (int e = 0; e < 21; ++e) sD[21 * t + e] = d_t.v[e];
    __syncthreads();
    for (int s = 1; s < mi; s <<= 1) {
      M3 na = a_t, nb = b_t, nc = c_t;
      R7 nd = d_t;
      if (t < mi) {
        int tm = t - s, tp = t + s;
        M3 am = m3_zero(), bm = m3_eye(), cm = m3_zero(), ap = m3_zero(), bp = m3_eye(), cp = m3_zero();
        R7 dm, dp;
        for (int e = 0; e < 21; ++e) { dm.v[e] = 0.f; dp.v[e] = 0.f; }
        if (tm >= 0) {
          for (int e = 0; e < 9; ++e) { am.v[e] = sA[9 * tm + e]; bm.v[e] = sB[9 * tm + e]; cm.v[e] = sC[9 * tm + e]; }
          for (int e = 0; e < 21; ++e) dm.v[e] = sD[21 * tm + e];
        }
        if (tp < mi) {
          for (int e = 0; e < 9; ++e) { ap.v[e] = sA[9 * tp + e]; bp.v[e] = sB[9 * tp + e]; cp.v[e] = sC[9 * tp + e]; }
          for (int e = 0; e < 21; ++e) dp.v[e] = sD[21 * tp + e];
        }
        M3 al = m3_neg(m3_mul(a_t, m3_inv(bm)));
        M3 ga = m3_neg(m3_mul(c_t, m3_inv(bp)));
        na = m3_mul(al, am);
        nc = m3_mul(ga, cp);
        nb = m3_add(b_t, m3_add(m3_mul(al, cm), m3_mul(ga, ap)));
        nd = r7_add(d_t, r7_add(r7_mul(al, dm), r7_mul(ga, dp)));
      }
      __syncthreads();
      a_t = na; b_t = nb; c_t = nc; d_t = nd;
      for (int e = 0; e < 9; ++e) { sA[9 * t + e] = a_t.v[e]; sB[9 * t + e] = b_t.v[e]; sC[9 * t + e] = c_t.v[e]; }
      for (int e = 0; e < 21; ++e) sD[21 * t + e] = d_t.v[e];
      __syncthreads();
    }
    // x_t = B^-1 D: columns 0 (y), 1-3 (V), 4-6 (W)
    R7 x;
    if (t < mi) x = r7_mul(m3_inv(b_t), d_t);
    else for (int e = 0; e < 21; ++e) x.v[e] = 0.f;
    {
      float* ch = A.chunk + (size_t)c * kEulerChunkStride;
      if (t == 0) for (int e = 0; e < 21; ++e) ch[30 + e] = x.v[e];
      if (t == mi - 1) for (int e = 0; e < 21; ++e) ch[51 + e] = x.v[e];
    }
    if (!grid_sync(A.bar, A.status)) return;

    // ---- phase B: block-tridiagonal separator system (order C, not cyclic) ----
    if (c == 0 && t == 0) {
      A.maxbuf[2 * (par ^ 1)] = 0ull;
      A.maxbuf[2 * (par ^ 1) + 1] = 0ull;
    }
    if (t < Cn) {
      const float* ch = A.chunk + (size_t)t * kEulerChunkStride;
      M3 As, Bs, Cs, VL, WL, V0, W0;
      float ds[3], yL[3], y0[3];
      for (int e = 0; e < 9; ++e) { As.v[e] = __ldcg(ch + e); Bs.v[e] = __ldcg(ch + 9 + e); Cs.v[e] = __ldcg(ch + 18 + e); }
      for (int v = 0; v < 3; ++v) ds[v] = __ldcg(ch + 27 + v);
      for (int a = 0; a < 3; ++a) {
        yL[a] = __ldcg(ch + 51 + 7 * a);
        for (int b = 0; b < 3; ++b) { VL.v[3 * a + b] = __ldcg(ch + 51 + 7 * a + 1 + b); WL.v[3 * a + b] = __ldcg(ch + 51 + 7 * a + 4 + b); }
      }
      if (t + 1 < Cn) {
        const float* nx = A.chunk + (size_t)(t + 1) * kEulerChunkStride;
        for (int a = 0; a < 3; ++a) {
          y0[a] = __ldcg(nx + 30 + 7 * a);
          for (int b = 0; b < 3; ++b) { V0.v[3 * a + b] = __ldcg(nx + 30 + 7 * a + 1 + b); W0.v[3 * a + b] = __ldcg(nx + 30 + 7 * a + 4 + b); }
        }
      } else {          // last separator: no cell to its right (its C block is zero)
        V0 = m3_zero(); W0 = m3_zero();
        y0[0] = y0[1] = y0[2] = 0.f;
      }
      M3 ra = m3_mul(As, VL);
      M3 rb = m3_add(Bs, m3_add(m3_mul(As, WL), m3_mul(Cs, V0)));
      M3 rc = m3_mul(Cs, W0);
      for (int e = 0; e < 9; ++e) { rA[9 * t + e] = ra.v[e]; rB[9 * t + e] = rb.v[e]; rC[9 * t + e] = rc.v[e]; }
      for (int a = 0; a < 3; ++a) {
        float v = ds[a];
        for (int b = 0; b < 3; ++b) v -= As.v[3 * a + b] * yL[b] + Cs.v[3 * a + b] * y0[b];
        rD[3 * t + a] = v;
      }
    }
    __syncthreads();
    for (int s = 1; s < Cn; s <<= 1) {
      M3 na, nb, nc;
      float nd[3];
      if (t < Cn) {
        int tm = t - s, tp = t + s;
        M3 at, bt, ct, am = m3_zero(), bm = m3_eye(), cm = m3_zero(), ap = m3_zero(), bp = m3_eye(), cp = m3_zero();
        float dt_[3], dm[3] = {0.f, 0.f, 0.f}, dp[3] = {0.f, 0.f, 0.f};
        for (int e = 0; e < 9; ++e) { at.v[e] = rA[9 * t + e]; bt.v[e] = rB[9 * t + e]; ct.v[e] = rC[9 * t + e]; }
        for (int v = 0; v < 3; ++v) dt_[v] = rD[3 * t + v];
        if (tm >= 0) {
          for (int e = 0; e < 9; ++e) { am.v[e] = rA[9 * tm + e]; bm.v[e] = rB[9 * tm + e]; cm.v[e] = rC[9 * tm + e]; }
          for (int v = 0; v < 3; ++v) dm[v] = rD[3 * tm + v];
        }
        if (tp < Cn) {
          for (int e = 0; e < 9; ++e) { ap.v[e] = rA[9 * tp + e]; bp.v[e] = rB[9 * tp + e]; cp.v[e] = rC[9 * tp + e]; }
          for (int v = 0; v < 3; ++v) dp[v] = rD[3 * tp + v];
        }
        M3 al = m3_neg(m3_mul(at, m3_inv(bm)));
        M3 ga = m3_neg(m3_mul(ct, m3_inv(bp)));
        na = m3_mul(al, am);
        nc = m3_mul(ga, cp);
        nb = m3_add(bt, m3_add(m3_mul(al, cm), m3_mul(ga, ap)));
        for (int a = 0; a < 3; ++a) {
          float v = dt_[a];
          for (int b = 0; b < 3; ++b) v += al.v[3 * a + b] * dm[b] + ga.v[3 * a + b] * dp[b];
          nd[a] = v;
        }
      }
      __syncthreads();
      if (t < Cn) {
        for (int e = 0; e < 9; ++e) { rA[9 * t + e] = na.v[e]; rB[9 * t + e] = nb.v[e]; rC[9 * t + e] = nc.v[e]; }
        for (int v = 0; v < 3; ++v) rD[3 * t + v] = nd[v];
      }
      __syncthreads();
    }
    if (t < Cn) {
      M3 bt;
      for (int e = 0; e < 9; ++e) bt.v[e] = rB[9 * t + e];
      M3 bi = m3_inv(bt);
      for (int a = 0; a < 3; ++a)
        rS[3 * t + a] = bi.v[3 * a] * rD[3 * t] + bi.v[3 * a + 1] * rD[3 * t + 1] + bi.v[3 * a + 2] * rD[3 * t + 2];
    }
    __syncthreads();
    // delta of this cell
    float sl[3] = {0.f, 0.f, 0.f}, ss[3];
    if (c > 0) for (int a = 0; a < 3; ++a) sl[a] = rS[3 * (c - 1) + a];
    for (int a = 0; a < 3; ++a) ss[a] = rS[3 * c + a];
    float dlt[3] = {0.f, 0.f, 0.f};
    if (t < mi) {
      for (int a = 0; a < 3; ++a) {
        float v = x.v[7 * a];
        for (int b = 0; b < 3; ++b) v += x.v[7 * a + 1 + b] * sl[b] + x.v[7 * a + 4 + b] * ss[b];
        dlt[a] = v;
      }
    } else if (t == m - 1) {
      for (int a = 0; a < 3; ++a) dlt[a] = ss[a];
    }
    unsigned int kdl = 0u, kul = 0u;
    if (active) {
      u.r += (double)dlt[0]; u.m += (double)dlt[1]; u.e += (double)dlt[2];
      A.q[i] = u.r; A.q[n + i] = u.m; A.q[2 * n + i] = u.e;
      for (int a = 0; a < 3; ++a) kdl = max(kdl, __float_as_uint(fabsf(dlt[a])));
      kul = max(__float_as_uint(fabsf((float)u.r)), max(__float_as_uint(fabsf((float)u.m)),
                                                        __float_as_uint(fabsf((float)u.e))));
      if (!isfinite(u.r) || !isfinite(u.m) || !isfinite(u.e)) kul = 0x7fc00000u;
    }
    kdl = block_max_u32(kdl, red);
    kul = block_max_u32(kul, red);
    if (t == 0) {
      atomicMax(&A.maxbuf[2 * par], (unsigned long long)kdl);
      atomicMax(&A.maxbuf[2 * par + 1], (unsigned long long)kul);
    }
    if (!grid_sync(A.bar, A.status)) return;
    unsigned int kd = (unsigned int)__ldcg(&A.maxbuf[2 * par]);
    unsigned int ku = (unsigned int)__ldcg(&A.maxbuf[2 * par + 1]);
    if (kd >= 0x7f800000u || ku >= 0x7f800000u) {
      if (c == 0 && t == 0) record_status(A.status, kStNonFinite);
      return;
    }
    if ((double)__uint_as_float(kd) <= A.tol * (1.0 + (double)__uint_as_float(ku))) done = true;
  }
  if (c == 0 && t == 0) {
    *A.iters = it - 1;
    if (!done) record_status(A.status, kStNoConv);
  }
}

__global__ void euler_rhs_kernel(const double* __restrict__ U, double* __restrict__ f, int64_t n,
                                 double gamma) {
  const double inv_dx = (double)n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    Cons ul = load_cell(U, n, i - 1), uc = load_cell(U, n, i), ur = load_cell(U, n, i + 1);
    double Fl[3], Fr[3];
    rusanov(ul, uc, gamma, Fl);
    rusanov(uc, ur, gamma, Fr);
    for (int v = 0; v < 3; ++v) f[v * n + i] = -(Fr[v] - Fl[v]) * inv_dx;
  }
}

// ---------------------------------------------------------------------------
// DEIM-Galerkin reduced steps of the Euler system in the explicit form
// (Eq. deim_galerkin_rom continuous in time, advanced by the SSPRK(4,3)
// stages of App. D): one CTA on the sample mesh. The f of a sampled row
// (variable v of cell i) is the difference of its two Rusanov interface
// fluxes, which need the three variables of the cells i-1, i, i+1: nine mesh
// rows per sample (Phi, q_ref, 1/D), staged in shared memory once per launch.
// A stage lifts the mesh rows (one thread per row), evaluates D f at the
// samples (one thread per sample) and adds dt/2 (P^T Phi)^+ (D f) to the
// reduced state (one warp per coordinate, lanes over the samples).
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(kBlock) euler_hyper_kernel(StepArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5, nw = blockDim.x >> 5;
  const int k = *A.rank;
  const int ns = A.n_s, nm = 9 * ns, r = A.r;
  const int64_t ncell = A.n / 3;
  const double inv_dx = (double)ncell;
  double* s_mesh = reinterpret_cast<double*>(smem_raw);  // nm x k (room for nm x r)
  double* s_qr = s_mesh + (size_t)nm * r;                // nm
  double* s_di = s_qr + nm;                              // nm (1/d)
  double* s_qt = s_di + nm;                              // nm (lifted)
  double* s_f = s_qt + nm;                               // ns (d f at the samples)
  double* s_dc = s_f + ns;                               // ns (d at the samples)
  double* s_a = s_dc + ns;                               // r
  double* s_ap = s_a + r;                                // r: a^n
  int* s_var = reinterpret_cast<int*>(s_ap + r);         // ns: variable of each sampled row

  for (int e = t; e < nm * k; e += blockDim.x) {
    const int row = e / k, j = e % k;
    s_mesh[e] = A.mesh[(size_t)row * kMeshStride + j];
  }
  for (int e = t; e < nm; e += blockDim.x) {
    s_qr[e] = A.mesh[(size_t)e * kMeshStride + kMaxR];
    s_di[e] = 1.0 / A.mesh[(size_t)e * kMeshStride + kMaxR + 1];
  }
  for (int q = t; q < ns; q += blockDim.x) {
    const int v = (int)(A.samples[q] / ncell);
    s_var[q] = v;
    s_dc[q] = A.mesh[(size_t)(9 * q + 3 + v) * kMeshStride + kMaxR + 1];
  }
  for (int j = t; j < k; j += blockDim.x) s_a[j] = A.a[j];
  __syncthreads();
  for (int step = 0; step < A.nsteps; ++step) {
    for (int j = t; j < k; j += blockDim.x) s_ap[j] = s_a[j];
    for (int it = 1; it <= 4; ++it) {
      // lift the mesh rows at the stage value (the barrier before it also
      // orders the a^n copy above)
      __syncthreads();
      for (int e = t; e < nm; e += blockDim.x) {
        const double* row = s_mesh + (size_t)e * k;
        double s = 0.0;
        for (int j = 0; j < k; ++j) s = fma(row[j], s_a[j], s);
        s_qt[e] = s_qr[e] + s * s_di[e];
      }
      __syncthreads();
      for (int q = t; q < ns; q += blockDim.x) {
        const double* u = s_qt + 9 * q;
        const Cons L{u[0], u[1], u[2]}, C{u[3], u[4], u[5]}, R{u[6], u[7], u[8]};
        double Fl[3], Fr[3];
        rusanov(L, C, A.gamma, Fl);
        rusanov(C, R, A.gamma, Fr);
        const int v = s_var[q];
        const double fl = v == 0 ? Fl[0] : (v == 1 ? Fl[1] : Fl[2]);
        const double fr = v == 0 ? Fr[0] : (v == 1 ? Fr[1] : Fr[2]);
        s_f[q] = s_dc[q] * (-(fr - fl) * inv_dx);
      }
      __syncthreads();
      // stage: a_j <- a_j + dt/2 sum_q M_jq (d f)_q; after the third,
      // a_j <- 2/3 a^n_j + 1/3 a_j (a_j is written by its own warp only)
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
    }
  }
  for (int j = t; j < r; j += blockDim.x) A.a[j] = (j < k) ? s_a[j] : 0.0;
  if (t == 0) *A.iters = 0;
}

int euler_chunks(int64_t n) {
  int C = 1;
  while (C * 2 <= kMaxChunks && n / (C * 2) >= 32) C *= 2;
  return C;
}

}  // namespace

size_t euler_chunk_floats() { return (size_t)kMaxChunks * kEulerChunkStride; }

cudaError_t launch_euler_rhs(int64_t n_cells, double gamma, const double* q, double* f,
                             cudaStream_t s) {
  int blocks = (int)((n_cells + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  euler_rhs_kernel<<<blocks, 256, 0, s>>>(q, f, n_cells, gamma);
  return cudaGetLastError();
}

size_t euler_hyper_smem(int n_s, int r) {
  const size_t nm = 9 * (size_t)n_s;
  return sizeof(double) * (nm * (size_t)r + 3 * nm + 2 * (size_t)n_s + 2 * (size_t)r) +
         sizeof(int) * (size_t)n_s + 64;
}

cudaError_t launch_euler_hyper_steps(const StepArgs& A, cudaStream_t s) {
  if (A.n_s < 1 || A.n_s > 256 || A.r < 1 || A.r > kMaxR || A.n % 3 != 0 || !A.explicit_rk)
    return cudaErrorInvalidValue;
  const size_t smem = euler_hyper_smem(A.n_s, A.r);
  if (smem > 220000) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(euler_hyper_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  euler_hyper_kernel<<<1, kBlock, smem, s>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_euler_step(const FomParams& p, const double* q_prev, double* q,
                              const FomScratch& sc, cudaStream_t s) {
  const int64_t n = p.n_cells;
  const int C = euler_chunks(n);
  const int64_t mmax = (n + C - 1) / C;
  if (mmax > kEulerChunkCells || n < 4) return cudaErrorInvalidValue;
  // one thread per cell, and at least one per chunk for the separator system
  int threads = (int)((mmax + 31) / 32 * 32);
  if (threads < C) threads = C;
  const size_t smem = sizeof(float) * kCellFloats * kEulerChunkCells;
  cudaError_t e = cudaFuncSetAttribute(euler_newton_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  EulerNewtonArgs A;
  A.q_prev = q_prev; A.q = q; A.n = n; A.gamma = p.gamma; A.h = p.h; A.tol = p.tol;
  A.max_iter = p.max_iter; A.C = C; A.chunk = sc.chunk; A.maxbuf = sc.maxbuf; A.bar = sc.bar;
  A.status = sc.status; A.iters = sc.iters;
  void* args[] = {&A};
  return cudaLaunchCooperativeKernel((const void*)euler_newton_kernel, dim3(C), dim3(threads), args,
                                     smem, s);
}

namespace {

// ---------------------------------------------------------------------------
// Plain Galerkin reduced steps for the Euler system (Eq.
// galerkin_continuous_rom with backward Euler): cooperative over cells, each
// CTA owning a range of cells and their three variable rows. The residual
// (lift, Rusanov f, projection) is FP64 (FP32 projections in the mixed form);
// the reduced Jacobian Phi^T D J_f D^-1 Phi is assembled in FP32 from the 3x3
// blocks of J_f over 64-cell tiles, once per step (chord iteration).
// ---------------------------------------------------------------------------

constexpr int kTile = 64;

template <int KM, typename TPhi>
__global__ void __launch_bounds__(kBlock) euler_galerkin_kernel(StepArgs A) {
  using Acc = TPhi;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const TPhi* phi = basis<TPhi>(A);
  const int G = gridDim.x, b = blockIdx.x, t = threadIdx.x;
  const int64_t ncell = A.n / 3, ld = A.ld;
  const int64_t c0 = (int64_t)b * ncell / G, c1 = (int64_t)(b + 1) * ncell / G;
  const int cells = (int)(c1 - c0);
  const int k = *A.rank;
  const int stride = KM + 2;
  const double inv_dx = (double)ncell;
  const float g32 = (float)A.gamma;

  double* s_a = reinterpret_cast<double*>(smem_raw);          // KM
  double* s_ap = s_a + KM;
  double* s_g = s_ap + KM;
  double* red = s_g + KM;                                      // 32*KM
  double* s_sc = red + 32 * KM;                                // 8
  double* s_qt = s_sc + 8;                                     // 3 x (cells+2)
  float* s_J = reinterpret_cast<float*>(s_qt + 3 * (cells + 2));   // kMaxR^2
  float* s_x = s_J + kMaxR * kMaxR;
  int* s_piv = reinterpret_cast<int*>(s_x + kMaxR);
  float* s_blk = reinterpret_cast<float*>(s_piv + kMaxR);     // cells x 27 (J_f blocks)
  float* s_phi = s_blk + 27 * cells;                          // (kTile+2) x 3 x KM
  float* s_w = s_phi + (kTile + 2) * 3 * KM;                  // kTile x 3 x KM

  for (int j = t; j < KM; j += blockDim.x) s_a[j] = (j < k) ? A.a[j] : 0.0;
  __syncthreads();
  const int W2 = cells + 2;
  int it_total = 0;
  for (int step = 0; step < A.nsteps; ++step) {
    for (int j = t; j < KM; j += blockDim.x) s_ap[j] = s_a[j];
    __syncthreads();
    bool conv = false;
    int it;
    const int nit = A.explicit_rk ? 4 : A.max_iter;   // SSPRK(4,3): four stages (App. D)
    for (it = 1; it <= nit; ++it) {
      const int par = it & 1;
      const bool jac_it = !A.explicit_rk && (it == 1);
      // lift the three variables on cells c0-1 .. c1 (ends clamped: ghost cells)
      for (int e = t; e < 3 * W2; e += blockDim.x) {
        int v = e / W2, cc = e % W2;
        int64_t cell = c0 - 1 + cc;
        cell = cell < 0 ? 0 : (cell >= ncell ? ncell - 1 : cell);
        int64_t row = v * ncell + cell;
        Acc s = Acc(0);
        for (int j = 0; j < k; ++j) s = fma((Acc)phi[j * ld + row], (Acc)s_a[j], s);
        s_qt[e] = A.q_ref[row] + (double)s * A.dinv[row];
      }
      __syncthreads();
      double acc[KM];
#pragma unroll
      for (int j = 0; j < KM; ++j) acc[j] = 0.0;
      for (int e = t; e < cells; e += blockDim.x) {
        const int cc = e + 1;
        Cons ul{s_qt[cc - 1], s_qt[W2 + cc - 1], s_qt[2 * W2 + cc - 1]};
        Cons uc{s_qt[cc], s_qt[W2 + cc], s_qt[2 * W2 + cc]};
        Cons ur{s_qt[cc + 1], s_qt[W2 + cc + 1], s_qt[2 * W2 + cc + 1]};
        double Fl[3], Fr[3];
        rusanov(ul, uc, A.gamma, Fl);
        rusanov(uc, ur, A.gamma, Fr);
        const int64_t cell = c0 + e;
        for (int v = 0; v < 3; ++v) {
          const int64_t row = v * ncell + cell;
          const Acc w = (Acc)(A.drow[row] * (-(Fr[v] - Fl[v]) * inv_dx));
#pragma unroll
          for (int j = 0; j < KM; ++j)
            if (j < k) acc[j] = (double)fma((Acc)phi[j * ld + row], w, (Acc)acc[j]);
        }
        if (jac_it) {
          CellD dl = cell_derivs(ul, g32), dc = cell_derivs(uc, g32), dr = cell_derivs(ur, g32);
          float pL[3][3], pR[3][3], qL[3][3], qR[3][3];
          rusanov_derivs(dl, dc, pL, pR);
          rusanov_derivs(dc, dr, qL, qR);
          const float ix = (float)inv_dx;
          for (int a2 = 0; a2 < 3; ++a2)
            for (int b2 = 0; b2 < 3; ++b2) {
              float lower = pL[a2][b2], diag = -qL[a2][b2] + pR[a2][b2], upper = -qR[a2][b2];
              if (cell == 0) { diag += lower; lower = 0.f; }
              if (cell == ncell - 1) { diag += upper; upper = 0.f; }
              s_blk[27 * e + 3 * a2 + b2] = lower * ix;
              s_blk[27 * e + 9 + 3 * a2 + b2] = diag * ix;
              s_blk[27 * e + 18 + 3 * a2 + b2] = upper * ix;
            }
        }
      }
      double* part = A.partials + (size_t)par * G * stride;
      {
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
          s_g[j] = s;
          part[(size_t)b * stride + j] = s;
        }
        __syncthreads();
      }
      if (jac_it) {
        float jacc[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) jacc[q] = 0.f;
        const int kk = k * k;
        for (int t0 = 0; t0 < cells; t0 += kTile) {
          const int tc = min(kTile, cells - t0);
          // s_phi[cc][v][j] = Phi(v, cell) / d_v for cells t0-1 .. t0+tc (clamped)
          for (int e = t; e < (tc + 2) * 3 * k; e += blockDim.x) {
            int cc = e / (3 * k), rem = e % (3 * k), v = rem / k, j = rem % k;
            int64_t cell = c0 + t0 - 1 + cc;
            cell = cell < 0 ? 0 : (cell >= ncell ? ncell - 1 : cell);
            int64_t row = v * ncell + cell;
            s_phi[(cc * 3 + v) * KM + j] = (float)phi[j * ld + row] * (float)A.dinv[row];
          }
          __syncthreads();
          // W(cell, a, l) = d_a sum_b (L_ab Phi~(cell-1,b,l) + D_ab Phi~(cell,b,l) + U_ab Phi~(cell+1,b,l))
          for (int e = t; e < tc * 3 * k; e += blockDim.x) {
            int ce = e / (3 * k), rem = e % (3 * k), a2 = rem / k, l = rem % k;
            const float* bl = s_blk + 27 * (t0 + ce);
            float w = 0.f;
            for (int b2 = 0; b2 < 3; ++b2)
              w += bl[3 * a2 + b2] * s_phi[((ce) * 3 + b2) * KM + l] +
                   bl[9 + 3 * a2 + b2] * s_phi[((ce + 1) * 3 + b2) * KM + l] +
                   bl[18 + 3 * a2 + b2] * s_phi[((ce + 2) * 3 + b2) * KM + l];
            const int64_t row = a2 * ncell + c0 + t0 + ce;
            s_w[(ce * 3 + a2) * KM + l] = w * (float)A.drow[row];
          }
          __syncthreads();
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            int e = t + q * kBlock;
            if (e < kk) {
              int j = e / k, l = e % k;
              float s = 0.f;
              for (int ce = 0; ce < tc; ++ce)
                for (int a2 = 0; a2 < 3; ++a2) {
                  const int64_t row = a2 * ncell + c0 + t0 + ce;
                  s += s_phi[((ce + 1) * 3 + a2) * KM + j] * (float)A.drow[row] * s_w[(ce * 3 + a2) * KM + l];
                }
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
        const int kk = k * k;
        const int e0 = (int)((int64_t)b * kk / G), e1 = (int)((int64_t)(b + 1) * kk / G);
        {
          const int lane = t & 31, wid = t >> 5, nw = blockDim.x >> 5;
          for (int e = e0 + wid; e < e1; e += nw) {
            float s = 0.f;
            for (int bb = lane; bb < G; bb += 32) s += __ldcg(&A.jpartials[(size_t)bb * kMaxR * kMaxR + e]);
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
      grid_reduce_cols(part, G, stride, k, s_g);
      if (A.explicit_rk) {
        // stage: x <- x + dt/2 Phi^T D f(x); after the third, x <- 2/3 a^n + 1/3 x
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
        double gg = s_a[j] - s_ap[j] - A.dt * s_g[j];
        s_x[j] = (float)(-gg);
      }
      __syncthreads();
      lu_solve(s_J, s_piv, s_x, k);
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

}  // namespace

template <int KM, typename TPhi>
static cudaError_t launch_eg_tt(const StepArgs& A, int grid, cudaStream_t s) {
  const int64_t ncell = A.n / 3;
  const int cells = (int)((ncell + grid - 1) / grid) + 1;
  size_t smem = sizeof(double) * (3 * KM + 32 * KM + 8 + 3 * (cells + 2)) +
                sizeof(float) * (kMaxR * kMaxR + kMaxR) + sizeof(int) * kMaxR +
                sizeof(float) * (27 * cells + (kTile + 2) * 3 * KM + kTile * 3 * KM) + 64;
  cudaError_t e = cudaFuncSetAttribute(euler_galerkin_kernel<KM, TPhi>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  StepArgs a = A;
  void* args[] = {&a};
  return cudaLaunchCooperativeKernel((const void*)euler_galerkin_kernel<KM, TPhi>, dim3(grid),
                                     dim3(kBlock), args, smem, s);
}

template <int KM>
static cudaError_t launch_eg_t(const StepArgs& A, int grid, cudaStream_t s) {
  return A.phi32 ? launch_eg_tt<KM, float>(A, grid, s) : launch_eg_tt<KM, double>(A, grid, s);
}

cudaError_t launch_euler_galerkin_steps(const StepArgs& A, int km, int grid, cudaStream_t s) {
  switch (km) {
    case 9: return launch_eg_t<9>(A, grid, s);
    case 17: return launch_eg_t<17>(A, grid, s);
    case 33: return launch_eg_t<33>(A, grid, s);
    default: return launch_eg_t<65>(A, grid, s);
  }
}

// Wait bound of this translation unit's kernels (see rom_internal.cuh).
cudaError_t set_wait_limit_euler(long long cycles) { return set_wait_limit_here(cycles); }

}  // namespace rom
