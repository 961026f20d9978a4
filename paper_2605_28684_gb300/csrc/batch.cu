// Batched execution of many independent adaptive ROMs: Burgers instances of
// uneven size (N, r, nu, z, lambda per instance) in the mixed form (FP32 basis
// with FP32 lift, projections and rotation; FP64 coarse FOM, core SVD and
// re-orthonormalisation). Every instance runs the online loop of Algorithm 1
// with the plain Galerkin step and the iSVD of Algorithm 2.
//
// One launch serves every instance, so that the whole batch streams its FP32
// bases through the GPU together instead of running hundreds of small
// latency-bound solves one after another. Work is cut into row tiles
// (instance, first row, last row), and per-tile partial sums are combined per
// instance in tile order, so results do not depend on which CTA took which
// tile. Three persistent cooperative kernels:
//   batch_steps_kernel  BE Galerkin steps as dataflow: CTAs take the tiles of
//                       every instance's current Newton iteration from a work
//                       array (FP32 lift, FP32 difference-form residual, FP32
//                       projection, FP32 reduced Jacobian when due); the CTA
//                       that completes an instance's last tile runs its Newton
//                       update (inverse of the reduced Jacobian) and appends
//                       its next iteration, so instances advance
//                       independently, without a grid barrier per iteration.
//   batch_fom_kernel    the coarse FOM step (Eq. coarse_fom_backward_euler)
//                       of the instances that adapt now: Newton with FP64
//                       residuals over (instance, chunk) work items; the
//                       linear solve eliminates each thread's block of rows
//                       (Thomas), solves the block separators of a chunk by
//                       PCR and the chunk separators of an instance by PCR.
//   batch_event_kernel  Algorithm 2 for those instances: projections, one CTA
//                       per instance for the core SVD, rotation with a fused
//                       Gram matrix, FP64 Cholesky, basis <- basis R^-1.
//
// The reduced Jacobian I - dt Phi^T J_f Phi (D is a scalar for Burgers, so
// D and D^-1 cancel) is formed at the first step after every basis change
// and kept (a chord iteration); it is refreshed at the current iterate after
// every 8 iterations without convergence. The root is fixed by the residual.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <climits>
#include <cstddef>
#include <cstring>
#include <type_traits>
#include <vector>

#include "rom_internal.cuh"
#include "secular.cuh"

namespace rom {

namespace {

constexpr int kBT = 256;          // threads of the sweep kernels
constexpr int kFomT = 512;        // threads of the FOM kernel (two CTAs per SM)
constexpr int kFomR = 4;          // rows per thread of a FOM chunk
constexpr int kFomRows = kFomR * kFomT;   // rows per FOM chunk
constexpr int kFomMaxChunks = 256; // FOM chunks per instance (power of two)
constexpr int kFomItems = 256;     // FOM work items (chunks) per CTA
constexpr int kPS = kMaxR + 4;    // stride of the per-tile partial vectors
constexpr int kMaxBatch = 4096;   // instances per batch
constexpr int kTileRowsMin = 2048;  // smallest tile the autotuner tries (a multiple of every chunk)
constexpr int kTileCandidates[] = {2048, 4096, 8192, 16384};
constexpr int kChunkMax = 2048;   // rows per chunk of a sweep (256 threads x rows per thread)
constexpr int kFomChunkStride = 16;

// Per-instance constants (device array, written once at init).
struct Inst {
  long long phi_off;   // offset (floats) of the FP32 basis, N x r column-major
  long long vec_off;   // offset (doubles) of the N-vectors of this instance
  int n, r, z, maxit;
  int tile0, tile1;    // row tiles [tile0, tile1)
  int chunk0, nchunk;  // FOM chunks [chunk0, chunk0 + nchunk)
  double nu, dt, lam, d, dinv, tol, rank_tol;
};

struct BArgs {
  int count, ntiles, nchunks, nsteps, fom_maxit;
  const Inst* inst;
  const int* tile_inst;
  const int* tile_r0;
  const int* tile_r1;
  const int* order;        // queue order of the tiles (decreasing cost)
  const int4* qdesc;       // per queue slot: (tile, instance, first row, last row)
  const int* chunk_inst;
  const int* chunk_c;
  float* phi;
  const double* q_ref;
  float* qr32;             // q_ref rounded to FP32, packed like the N-vectors
  float* dq32;             // q_ref(i+1) - q_ref(i) (periodic), FP64 difference rounded
  float* lq32;             // q_ref(i+1) - 2 q_ref(i) + q_ref(i-1), likewise
  double* y_corr;          // correction snapshot (previous coarse FOM state)
  double* y_new;           // coarse FOM iterate / new snapshot
  double* dy;              // last snapshot increment y_new - y_corr (initial guess of the next solve)
  double* a;               // count x kMaxR: reduced state
  double* an;              // count x kMaxR: reduced state at the start of the step
  double* sigma;           // count x kMaxR
  int* rank;
  int* need_jac;
  int* iters_rom;
  int* iters_fom;
  long long* fom_its;      // count: coarse FOM Newton iterations since reset
  long long* sweeps;       // count: Newton iterations (sweeps over the basis) since reset
  long long* sweep_cols;   // count: basis columns streamed by those sweeps (rank each time)
  float* jlu;              // count x kMaxR x kMaxR: inverse of the reduced Jacobian (FP32)
  double* gpart;           // ntiles x kPS
  double* gpart2;          // ntiles x kPS
  float* mpart;            // ntiles x kMaxR x kMaxR: reduced Jacobian partials (FP32)
  double* gram_part;       // ntiles x kMaxR x kMaxR: Gram partials of the rotated basis (FP64)
  float* fom_row;          // 3 floats per row (PCR y, v, w)
  float* fom_chunk;        // nchunks x kFomChunkStride
  float* fom_sep;          // nchunks: separator values
  unsigned int* fom_keys;  // count x 4
  double* ev_p;            // count x kMaxCore: p1, then p = p1 + p2
  double* ev_p2;           // count x kMaxCore: p2 (second Gram-Schmidt pass)
  float* qres;             // q1 = yhat - Phi p1 per row (FP32), packed like the N-vectors
  float* yhat32;           // yhat = D (y - q_ref) per row, formed in FP64 and rounded
  double* ev_sc;           // count x 8: |yhat|^2, 1/rho, k', k
  float* ev_u;             // count x kMaxCore x kMaxR: rotation U(:, 0:k') (FP32)
  double* ev_anew;         // count x kMaxR: transferred state before a <- R a
  float* ev_r;             // count x kMaxR x kMaxR: Cholesky factor R (FP32 copy)
  unsigned int* ctl;       // [0..3] tile queues of the sweeps; steps kernel: [0] claimed
                           // entries, [1] appended entries, [2] instances done (host-zeroed)
  unsigned long long* wq;  // steps kernel work entries: epoch << 32 | tile
  long long wq_cap;        // entries of wq
  int* tcount;             // count: tiles of the current iteration counted in
  int* inst_it;            // count: Newton iteration of the current step
  int* inst_step;          // count: step of the launch
  unsigned int* epoch;     // launches of the steps kernel so far
  long long* M;            // online steps done by every instance
  GridBarrier* bar;
  int* status;
};

__device__ __forceinline__ bool is_event(const Inst& I, long long M) {
  return M > 0 && (M % I.z) == 0;
}

// ------------------------------------------------------------- Burgers ---

// Godunov flux F(uL, uR) = max(max(uL,0)^2, min(uR,0)^2) / 2 (tie -> left) as
// the selected state s (F = s^2 / 2). The branch is chosen on the magnitudes,
// which order the same way as the squares, using integer tests on the bit
// patterns; only the square is FP64 arithmetic.
struct Sel {
  double s;
  bool left;
};
__device__ __forceinline__ Sel godunov_sel(double uL, double uR) {
  const long long bl = __double_as_longlong(uL), br = __double_as_longlong(uR);
  const double lp = (bl > 0) ? uL : 0.0;     // max(uL, 0); a positive NaN stays
  const double rm = (br < 0) ? uR : 0.0;     // min(uR, 0); a negative NaN stays
  const long long ml = __double_as_longlong(lp) & 0x7fffffffffffffffLL;
  const long long mr = __double_as_longlong(rm) & 0x7fffffffffffffffLL;
  Sel o;
  o.left = ml >= mr;
  o.s = o.left ? lp : rm;
  return o;
}

// f_i = -(F_{i+1/2} - F_{i-1/2}) / dx + nu (u_{i+1} - 2 u_i + u_{i-1}) / dx^2.
__device__ __forceinline__ double burgers_f(double ul, double u, double ur, double nu, double inv_dx) {
  const Sel a = godunov_sel(ul, u), b = godunov_sel(u, ur);
  const double adv = (-0.5 * inv_dx) * (b.s * b.s - a.s * a.s);
  return fma(nu * inv_dx * inv_dx, fma(-2.0, u, ur + ul), adv);
}

// Tridiagonal row of J_f (FP32): df_i/du_{i-1}, df_i/du_i, df_i/du_{i+1}.
__device__ __forceinline__ void burgers_band(double ul, double u, double ur, float nu_f, float inv_dx_f,
                                             float& dl, float& dc, float& dr) {
  const Sel a = godunov_sel(ul, u), b = godunov_sel(u, ur);
  const float c2 = nu_f * inv_dx_f * inv_dx_f;
  const float sa = (float)a.s, sb = (float)b.s;
  dl = (a.left ? sa : 0.f) * inv_dx_f + c2;
  dc = ((a.left ? 0.f : sa) - (b.left ? sb : 0.f)) * inv_dx_f - 2.f * c2;
  dr = -(b.left ? 0.f : sb) * inv_dx_f + c2;
}

// FP32 form of f for the lifted state u = q_ref + delta (the mixed form's
// batched sweep). Differences of u are taken as differences of q_ref
// (computed in FP64 and rounded once) plus differences of delta: FP32
// subtraction of the nearly equal delta values is exact, so f carries the
// rounding of delta itself and one FP32 rounding, the same as evaluating f in
// FP64 on the FP32 lift and rounding it to FP32 for the FP32 projection.
//  qm, q0, qp: q_ref(i-1), q_ref(i), q_ref(i+1) (FP32); dm, d0, dp: delta;
//  em = q_ref(i) - q_ref(i-1), ep = q_ref(i+1) - q_ref(i);
//  lr = q_ref(i+1) - 2 q_ref(i) + q_ref(i-1).
__device__ __forceinline__ float burgers_f32(float qm, float q0, float qp, float dm, float d0, float dp,
                                             float em, float ep, float lr, float inv_dx, float c2) {
  const float um = qm + dm, u0 = q0 + d0, up = qp + dp;
  const float gm = em + (d0 - dm);          // u0 - um
  const float gp = ep + (dp - d0);          // up - u0
  // left interface (um, u0): 1 -> um, 2 -> u0, 0 -> zero; right (u0, up): 2 -> u0, 3 -> up
  const float lpL = um > 0.f ? um : 0.f, rmL = u0 < 0.f ? u0 : 0.f;
  const bool selL = fabsf(lpL) >= fabsf(rmL);
  const int iL = selL ? (um > 0.f ? 1 : 0) : (u0 < 0.f ? 2 : 0);
  const float sL = selL ? lpL : rmL;
  const float lpR = u0 > 0.f ? u0 : 0.f, rmR = up < 0.f ? up : 0.f;
  const bool selR = fabsf(lpR) >= fabsf(rmR);
  const int iR = selR ? (u0 > 0.f ? 2 : 0) : (up < 0.f ? 3 : 0);
  const float sR = selR ? lpR : rmR;
  float diff;                               // sR - sL without cancellation
  if (iL == 1 && iR == 2) diff = gm;
  else if (iL == 1 && iR == 3) diff = gm + gp;
  else if (iL == 2 && iR == 2) diff = 0.f;
  else if (iL == 2 && iR == 3) diff = gp;
  else diff = sR - sL;
  const float lap = lr + ((dp - d0) - (d0 - dm));
  return fmaf(c2, lap, -0.5f * inv_dx * diff * (sR + sL));
}

// Tridiagonal row of J_f in FP32 from FP32 states.
__device__ __forceinline__ void burgers_band32(float ul, float u, float ur, float inv_dx, float c2,
                                               float& dl, float& dc, float& dr) {
  const float lpL = ul > 0.f ? ul : 0.f, rmL = u < 0.f ? u : 0.f;
  const bool selL = fabsf(lpL) >= fabsf(rmL);
  const float lpR = u > 0.f ? u : 0.f, rmR = ur < 0.f ? ur : 0.f;
  const bool selR = fabsf(lpR) >= fabsf(rmR);
  dl = (selL ? lpL : 0.f) * inv_dx + c2;
  dc = ((selL ? 0.f : rmL) - (selR ? lpR : 0.f)) * inv_dx - 2.f * c2;
  dr = -(selR ? 0.f : rmR) * inv_dx + c2;
}

// --------------------------------------------------------- small helpers ---

// Rank bucket (register budget) of an instance: loops are sized for the
// bucket and guarded by the actual rank.
__host__ __device__ __forceinline__ int bucket_of(int r) {
  return r <= 8 ? 8 : r <= 16 ? 16 : r <= 32 ? 32 : r <= 48 ? 48 : 64;
}

// Calls f(integral_constant<KB>) for the bucket of r.
template <typename F>
__device__ __forceinline__ void with_bucket(int r, F&& f) {
  switch (bucket_of(r)) {
    case 8: f(std::integral_constant<int, 8>{}); break;
    case 16: f(std::integral_constant<int, 16>{}); break;
    case 32: f(std::integral_constant<int, 32>{}); break;
    case 48: f(std::integral_constant<int, 48>{}); break;
    default: f(std::integral_constant<int, 64>{}); break;
  }
}

// Rows per thread: keeps about 64 basis loads in flight per thread.
template <int KB>
struct Rpt {
  static constexpr int v = KB <= 8 ? 8 : KB <= 16 ? 4 : KB <= 32 ? 2 : 1;
};

// Next tile of a queue; -1 when empty. All threads call it.
__device__ __forceinline__ int next_tile(unsigned int* ctr, int ntiles, int* s_q) {
  __syncthreads();
  if (threadIdx.x == 0) *s_q = (int)atomicAdd(ctr, 1u);
  __syncthreads();
  const int q = *s_q;
  return q < ntiles ? q : -1;
}

// Runs body(q) for every queue slot q this CTA claims. The claim of the next
// slot goes out before the current tile is processed, so its round trip to
// L2 overlaps the work.
template <typename F>
__device__ __forceinline__ void for_each_tile(unsigned int* ctr, int ntiles, int* s_q, F&& body) {
  int q = next_tile(ctr, ntiles, s_q);
  while (q >= 0) {
    unsigned int qn = 0u;
    if (threadIdx.x == 0) qn = atomicAdd(ctr, 1u);
    body(q);
    __syncthreads();
    if (threadIdx.x == 0) *s_q = (int)qn;
    __syncthreads();
    q = *s_q;
    if (q >= ntiles) q = -1;
  }
}

// Sum of per-tile partial vectors of one instance, fixed order: warps over
// entries, lanes over tiles.
__device__ __forceinline__ void sum_tiles(const double* part, int tile0, int tile1, int nent, int off,
                                          double* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = wid; j < nent; j += nw) {
    double s = 0.0;
    for (int tt = tile0 + lane; tt < tile1; tt += 32) s += __ldcg(&part[(size_t)tt * kPS + off + j]);
    s = warp_sum(s);
    if (lane == 0) out[j] = s;
  }
}

// Block reduction of per-thread FP32 accumulators into FP64 per-tile partials.
template <int KB>
__device__ __forceinline__ void tile_reduce(const float (&acc)[KB], int k, float* red, double* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int j = 0; j < KB; ++j) {
    float v = warp_sumf(acc[j]);
    if (lane == 0) red[wid * KB + j] = v;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += (double)red[w * KB + j];
    out[j] = s;
  }
}

// Register-blocked accumulation of  M += sum_rows A_row^T B_row  for k x k
// (4 x 4 blocks per thread, rows split over groups of threads when the
// blocks are fewer than the threads). A, B: rows x KB, row-major in shared.
template <int KB>
struct Blk {
  static constexpr int nb = KB / 4;
  static constexpr int nblk = nb * nb;
  static constexpr int groups = kBT / nblk > 0 ? kBT / nblk : 1;
};

template <int KB>
__device__ __forceinline__ void blk_accum(const float* A, const float* B, int rows, float (&m)[16]) {
  const int t = threadIdx.x;
  const int g = t / Blk<KB>::nblk, bi = t % Blk<KB>::nblk;
  if (g >= Blk<KB>::groups) return;
  const int jb = bi / Blk<KB>::nb, lb = bi % Blk<KB>::nb;
  for (int rr = g; rr < rows; rr += Blk<KB>::groups) {
    const float4 av = *reinterpret_cast<const float4*>(A + rr * KB + 4 * jb);
    const float4 bv = *reinterpret_cast<const float4*>(B + rr * KB + 4 * lb);
    const float ar[4] = {av.x, av.y, av.z, av.w};
    const float br[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) m[p * 4 + q] = fmaf(ar[p], br[q], m[p * 4 + q]);
  }
}

// Adds the per-thread blocks into a k x k FP32 matrix (row-major, ld k) in
// shared memory that the caller zeroed.
template <int KB>
__device__ __forceinline__ void blk_flush(const float (&m)[16], int k, float* out) {
  const int t = threadIdx.x;
  const int g = t / Blk<KB>::nblk, bi = t % Blk<KB>::nblk;
  if (g >= Blk<KB>::groups) return;
  const int jb = bi / Blk<KB>::nb, lb = bi % Blk<KB>::nb;
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = 4 * jb + p, l = 4 * lb + q;
      if (j < k && l < k) atomicAdd(&out[j * k + l], m[p * 4 + q]);
    }
}

// ---------------------------------------------------- shared-memory plans ---

struct StepSmem {
  float sd[kChunkMax + 2];           // delta = D^-1 Phi a of a chunk (+ halo)
  float su[kChunkMax + 2];           // q_ref (FP32) of the same rows
  float sdq[kChunkMax + 2];          // q_ref(i+1) - q_ref(i), from row c0 - 1
  alignas(16) float P[66 * kMaxR];   // basis rows of a 64-row sub-chunk (+ halo)
  alignas(16) float W[64 * kMaxR];   // J_f Phi rows; tile Jacobian at the end
  float red[8 * kMaxR];
  float af[kMaxR];
  float hx[2 * kMaxR];               // basis rows of the chunk halo
  // instance phase
  float J[kMaxR * kMaxR];
  float Ji[kMaxR * kMaxR];           // inverse of the reduced Jacobian
  double g[kMaxR];
  float x[kMaxR];
  int piv[kMaxR];
  double sc[4];
  long long base;
  int q, act, cnt;
};

struct CoreSmem {
  SecularSetup S;
  double d_desc[kMaxCore], z[kMaxCore];
  double tau[kMaxCore], orig[kMaxCore], zhat[kMaxCore];
  double val[kMaxCore], sbar[kMaxCore];
  int order[kMaxCore], pos[kMaxCore], defp[kMaxCore];
  double pv[8][kMaxCore];
  double U[kMaxCore * kMaxCore];      // row-major [row][col], ld kMaxCore
  double aold[kMaxR];
  double sc[8];
};

struct SweepSmem {
  double dred[32];                   // FP64 block-reduction scratch
  alignas(16) float P[kBT * 64];     // new basis rows of a chunk (Gram)
  float U[kMaxCore * kMaxR];         // rotation (FP32), row-major [row][col]
  float R[kMaxR * kMaxR];            // Cholesky factor (FP32), row-major
  float Rd[kMaxR];                   // 1 / R_jj
  float pf[kMaxCore];
  float red[8 * kMaxR];
  double Gd[kBT * 16];               // per-thread FP64 Gram blocks (4 x 4 each)
  double sc[4];
  int q;
};

// float4 reads of the staged rows need 16-byte alignment
static_assert(offsetof(StepSmem, P) % 16 == 0 && offsetof(StepSmem, W) % 16 == 0, "alignment");
static_assert(offsetof(SweepSmem, P) % 16 == 0 && offsetof(SweepSmem, dred) % 8 == 0, "alignment");

struct CholSmem {
  double G[kMaxR * kMaxR];           // Gram, then R in its upper triangle
  double anew[kMaxR];
  double d;
};

// ======================================================== steps kernel ===

// Registers of one chunk of a sweep tile: the chunk's basis rows and
// reference-state data, and (warps 0 and 1) the two periodic halo rows.
template <int KB>
struct ChunkRegs {
  static constexpr int RPT = Rpt<KB>::v;
  float x[RPT][KB];
  float qr[RPT], dq[RPT], lq[RPT];
  float hv0, hv1, hq, hd;
};

struct TileCtx {
  const float* phi;
  const float* qr;
  const float* dq;
  const float* lq;
  int N, k, r1;
  float inv_dx, c2, d_f, dinv_f;
};

template <int KB>
__device__ __forceinline__ void load_chunk(const TileCtx& T, int c0, ChunkRegs<KB>& R) {
  constexpr int RPT = Rpt<KB>::v;
  constexpr int CR = kBT * RPT;
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const int rows = min(CR, T.r1 - c0);
  const int h = (wid == 0) ? (c0 - 1 + T.N) % T.N : (c0 + rows) % T.N;
  R.hv0 = R.hv1 = R.hq = R.hd = 0.f;
  if (wid < 2) {
    if (lane < T.k && lane < KB) R.hv0 = __ldg(&T.phi[(size_t)lane * T.N + h]);
    if (lane + 32 < T.k && lane + 32 < KB) R.hv1 = __ldg(&T.phi[(size_t)(lane + 32) * T.N + h]);
    if (lane == 0) { R.hq = T.qr[h]; R.hd = T.dq[h]; }
  }
#pragma unroll
  for (int rr = 0; rr < RPT; ++rr) {
    const int e = rr * kBT + t;
#pragma unroll
    for (int j = 0; j < KB; ++j) R.x[rr][j] = (e < rows && j < T.k) ? __ldg(&T.phi[(size_t)j * T.N + c0 + e]) : 0.f;
    R.qr[rr] = (e < rows) ? T.qr[c0 + e] : 0.f;
    R.dq[rr] = (e < rows) ? T.dq[c0 + e] : 0.f;
    R.lq[rr] = (e < rows) ? T.lq[c0 + e] : 0.f;
  }
}

// Lift, FP32 operator and projection of one chunk (and its part of the
// reduced Jacobian when due).
template <int KB>
__device__ __forceinline__ void compute_chunk(const TileCtx& T, int c0, const ChunkRegs<KB>& R, StepSmem& sm,
                                              bool jac, float (&acc)[KB], float (&m)[16]) {
  constexpr int RPT = Rpt<KB>::v;
  constexpr int CR = kBT * RPT;
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const int rows = min(CR, T.r1 - c0);
#pragma unroll
  for (int rr = 0; rr < RPT; ++rr) {
    const int e = rr * kBT + t;
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < KB; ++j) s = fmaf(R.x[rr][j], sm.af[j], s);
    if (e < rows) {
      sm.sd[1 + e] = T.dinv_f * s;
      sm.su[1 + e] = R.qr[rr];
      sm.sdq[1 + e] = R.dq[rr];
    }
  }
  if (wid < 2) {
    float s = 0.f;
    if (lane < KB) { sm.hx[wid * kMaxR + lane] = R.hv0; s = R.hv0 * sm.af[lane]; }
    if (lane + 32 < KB) { sm.hx[wid * kMaxR + lane + 32] = R.hv1; s = fmaf(R.hv1, sm.af[lane + 32], s); }
    s = warp_sumf(s);
    if (lane == 0) {
      const int e = (wid == 0) ? 0 : rows + 1;
      sm.sd[e] = T.dinv_f * s;
      sm.su[e] = R.hq;
      if (wid == 0) sm.sdq[0] = R.hd;   // q_ref(c0) - q_ref(c0 - 1)
    }
  }
  __syncthreads();
#pragma unroll
  for (int rr = 0; rr < RPT; ++rr) {
    const int e = rr * kBT + t;
    if (e < rows) {
      const float f = burgers_f32(sm.su[e], sm.su[e + 1], sm.su[e + 2], sm.sd[e], sm.sd[e + 1],
                                  sm.sd[e + 2], sm.sdq[e], sm.sdq[e + 1], R.lq[rr], T.inv_dx, T.c2);
      const float w = f * T.d_f;
#pragma unroll
      for (int j = 0; j < KB; ++j) acc[j] = fmaf(R.x[rr][j], w, acc[j]);
    }
  }
  if (jac) {
    // Phi^T J_f Phi over 64-row sub-chunks: stage basis rows (+ halo),
    // W = J_f Phi, then the blocked rank-64 update.
    for (int s0 = 0; s0 < rows; s0 += 64) {
      const int sr = min(64, rows - s0);
#pragma unroll
      for (int rr = 0; rr < RPT; ++rr) {
        const int e = rr * kBT + t;
        if (e < rows && e >= s0 - 1 && e <= s0 + sr) {
#pragma unroll
          for (int j = 0; j < KB; ++j) sm.P[(e - s0 + 1) * KB + j] = R.x[rr][j];
        }
      }
      if (s0 == 0)
        for (int j = t; j < KB; j += kBT) sm.P[j] = sm.hx[j];
      if (s0 + sr == rows)
        for (int j = t; j < KB; j += kBT) sm.P[(sr + 1) * KB + j] = sm.hx[kMaxR + j];
      __syncthreads();
      for (int e = t; e < sr * KB; e += kBT) {
        const int rl = e / KB, l = e % KB;
        const int ee = s0 + rl;
        float dl, dc, dr;
        burgers_band32(sm.su[ee] + sm.sd[ee], sm.su[ee + 1] + sm.sd[ee + 1], sm.su[ee + 2] + sm.sd[ee + 2],
                       T.inv_dx, T.c2, dl, dc, dr);
        sm.W[rl * KB + l] = dl * sm.P[rl * KB + l] + dc * sm.P[(rl + 1) * KB + l] + dr * sm.P[(rl + 2) * KB + l];
      }
      __syncthreads();
      blk_accum<KB>(sm.P + KB, sm.W, sr, m);
      __syncthreads();
    }
  }
  __syncthreads();
}

// Segments per warp pass of the barrier-free sweep: keeps about 32 basis
// loads in flight per lane.
template <int KB>
struct Useg {
  static constexpr int v = KB <= 8 ? 4 : KB <= 16 ? 2 : 1;
};

// Lift, FP32 operator and projection of the tile rows [r0, r1) without a
// block barrier: a warp takes 32 consecutive rows at a time (a segment);
// lanes 1..30 own one row each, and lanes 0 and 31 load the rows on either
// side, so the stencil's neighbours come from the adjacent lanes by warp
// shuffles (the tile's outer rows are read from the neighbouring rows,
// periodically at the instance's ends). Each row is evaluated by one lane,
// as in the staged form; only the partial sums' grouping differs.
template <int KB>
__device__ __forceinline__ void stream_tile(const TileCtx& T, int r0, int r1, const float* af,
                                            float (&acc)[KB]) {
  constexpr int U = Useg<KB>::v;
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int rows = r1 - r0;
  const int nseg = (rows + 29) / 30;
  float a[KB];
#pragma unroll
  for (int j = 0; j < KB; ++j) a[j] = af[j];
  for (int s0 = wid * U; s0 < nseg; s0 += nw * U) {
    float x[U][KB], q[U], dq[U], lq[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int rl = (s0 + u) * 30 + lane - 1;     // row in the tile, -1 .. rows
      const bool live = (s0 + u) < nseg && rl <= rows;
      int row = r0 + rl;
      if (row < 0) row += T.N;
      else if (row >= T.N) row -= T.N;
      if (!live) row = r0;                          // in bounds; nothing is read there
#pragma unroll
      for (int j = 0; j < KB; ++j) x[u][j] = (live && j < T.k) ? __ldg(&T.phi[(size_t)j * T.N + row]) : 0.f;
      q[u] = live ? __ldg(&T.qr[row]) : 0.f;
      dq[u] = live ? __ldg(&T.dq[row]) : 0.f;
      lq[u] = live ? __ldg(&T.lq[row]) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int rl = (s0 + u) * 30 + lane - 1;
      float sd = 0.f;
#pragma unroll
      for (int j = 0; j < KB; ++j) sd = fmaf(x[u][j], a[j], sd);
      const float d = T.dinv_f * sd;
      const float dm = __shfl_up_sync(full, d, 1), dp = __shfl_down_sync(full, d, 1);
      const float qm = __shfl_up_sync(full, q[u], 1), qp = __shfl_down_sync(full, q[u], 1);
      const float em = __shfl_up_sync(full, dq[u], 1);
      if (lane >= 1 && lane <= 30 && (s0 + u) < nseg && rl < rows) {
        const float f = burgers_f32(qm, q[u], qp, dm, d, dp, em, dq[u], lq[u], T.inv_dx, T.c2);
        const float w = f * T.d_f;
#pragma unroll
        for (int j = 0; j < KB; ++j) acc[j] = fmaf(x[u][j], w, acc[j]);
      }
    }
  }
}

// The tile context of instance i's tile `tile`.
__device__ __forceinline__ TileCtx tile_ctx(const BArgs& A, int tile, int i, int k) {
  const Inst I = A.inst[i];
  TileCtx T;
  T.phi = A.phi + I.phi_off;
  T.qr = A.qr32 + I.vec_off;
  T.dq = A.dq32 + I.vec_off;
  T.lq = A.lq32 + I.vec_off;
  T.N = I.n;
  T.k = k;
  T.r1 = A.tile_r1[tile];
  T.inv_dx = (float)I.n;
  T.c2 = (float)I.nu * T.inv_dx * T.inv_dx;
  T.d_f = (float)I.d;
  T.dinv_f = (float)I.dinv;
  return T;
}

// A tile whose iteration also forms the reduced Jacobian (the first after a
// basis change, and every eighth without convergence): rows staged in shared
// memory by chunks. Kept out of line so that its registers do not weigh on
// the barrier-free sweep of all other tiles.
template <int KB>
__device__ __noinline__ void step_tile_jac(const BArgs& A, StepSmem& sm, int tile, int i) {
  constexpr int RPT = Rpt<KB>::v;
  constexpr int CR = kBT * RPT;
  const int t = threadIdx.x;
  const int k = A.rank[i];
  const TileCtx T = tile_ctx(A, tile, i, k);
  const int r0 = A.tile_r0[tile], r1 = T.r1;
  for (int j = t; j < KB; j += kBT) sm.af[j] = (j < k) ? (float)__ldcg(&A.a[(size_t)i * kMaxR + j]) : 0.f;
  float acc[KB];
#pragma unroll
  for (int j = 0; j < KB; ++j) acc[j] = 0.f;
  float m[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) m[q] = 0.f;
  ChunkRegs<KB> ra;
  load_chunk<KB>(T, r0, ra);
  __syncthreads();
  for (int c0 = r0; c0 < r1; c0 += CR) {
    if (c0 > r0) load_chunk<KB>(T, c0, ra);
    compute_chunk<KB>(T, c0, ra, sm, true, acc, m);
  }
  tile_reduce<KB>(acc, k, sm.red, A.gpart + (size_t)tile * kPS);
  __syncthreads();
  for (int e = t; e < k * k; e += kBT) sm.W[e] = 0.f;
  __syncthreads();
  blk_flush<KB>(m, k, sm.W);
  __syncthreads();
  float* mp = A.mpart + (size_t)tile * kMaxR * kMaxR;
  for (int e = t; e < k * k; e += kBT) mp[e] = sm.W[e];
}

template <int KB>
__device__ void step_tile(const BArgs& A, StepSmem& sm, int tile, int i, bool jac) {
  if (jac) {
    step_tile_jac<KB>(A, sm, tile, i);
    return;
  }
  const int t = threadIdx.x;
  const int k = A.rank[i];
  const TileCtx T = tile_ctx(A, tile, i, k);
  const int r0 = A.tile_r0[tile], r1 = T.r1;
  for (int j = t; j < KB; j += kBT) sm.af[j] = (j < k) ? (float)__ldcg(&A.a[(size_t)i * kMaxR + j]) : 0.f;
  float acc[KB];
#pragma unroll
  for (int j = 0; j < KB; ++j) acc[j] = 0.f;
  __syncthreads();                        // sm.af written above
  stream_tile<KB>(T, r0, r1, sm.af, acc);
  tile_reduce<KB>(acc, k, sm.red, A.gpart + (size_t)tile * kPS);
}

// Newton update of instance i once every tile of its current iteration has
// reported (run by the CTA that completed the last one), then the instance's
// next work: the tiles of its next iteration, of its next step, or nothing
// when the last step of the launch has converged.
__device__ __noinline__ void update_instance(const BArgs& A, StepSmem& sm, int i, unsigned int epoch) {
  const Inst I = A.inst[i];
  const int t = threadIdx.x;
  const int k = A.rank[i];
  const int it = __ldcg(&A.inst_it[i]);
  const int jac = __ldcg(&A.need_jac[i]);
  sum_tiles(A.gpart, I.tile0, I.tile1, k, 0, sm.g);
  __syncthreads();
  float* J = sm.J;
  if (jac) {
    for (int e = t; e < k * k; e += blockDim.x) {
      float s = 0.f;
      for (int tt = I.tile0; tt < I.tile1; ++tt) s += __ldcg(&A.mpart[(size_t)tt * kMaxR * kMaxR + e]);
      const int j = e / k, l = e % k;
      J[j * kMaxR + l] = (j == l ? 1.f : 0.f) - (float)I.dt * s;
    }
    __syncthreads();
    lu_factor(J, sm.piv, k);
    lu_inverse(J, sm.piv, sm.Ji, k);
    float* jg = A.jlu + (size_t)i * kMaxR * kMaxR;
    for (int e = t; e < k * kMaxR; e += blockDim.x) jg[e] = sm.Ji[e];
    if (t == 0) A.need_jac[i] = 0;
  } else {
    const float* jg = A.jlu + (size_t)i * kMaxR * kMaxR;
    for (int e = t; e < k * kMaxR; e += blockDim.x) sm.Ji[e] = __ldcg(&jg[e]);
  }
  double* a = A.a + (size_t)i * kMaxR;
  const double* an = A.an + (size_t)i * kMaxR;
  for (int j = t; j < k; j += blockDim.x) sm.x[j] = (float)(-(__ldcg(&a[j]) - __ldcg(&an[j]) - I.dt * sm.g[j]));
  __syncthreads();
  inv_apply(sm.Ji, sm.x, k);
  // act: 0 stop (error recorded), 1 next iteration, 2 next step, 3 launch done
  if (t < 32) {
    unsigned int kd = 0u, ka = 0u;
    bool bad = false;
    for (int j = t; j < k; j += 32) {
      const float dlt = sm.x[j];
      const double v = __ldcg(&a[j]) + (double)dlt;
      a[j] = v;
      kd = max(kd, __float_as_uint(fabsf(dlt)));
      ka = max(ka, __float_as_uint(fabsf((float)v)));
      bad = bad || !isfinite(v);
    }
    kd = warp_max_u32(kd);
    ka = warp_max_u32(ka);
    bad = __any_sync(0xffffffffu, bad);
    // FP32 projections: stop at their rounding level
    const double tol = fmax(I.tol, 1e-7);
    if (t == 0) {
      const bool conv = (double)__uint_as_float(kd) <= tol * (1.0 + (double)__uint_as_float(ka));
      int act = 0;
      if (bad) {
        record_status(A.status, kStNonFinite);
      } else if (conv) {
        // per-instance state written by whichever CTA ran the last update:
        // read through L2
        A.iters_rom[i] = it;
        A.sweeps[i] = __ldcg(&A.sweeps[i]) + it;
        A.sweep_cols[i] = __ldcg(&A.sweep_cols[i]) + (long long)it * k;
        const int stp = __ldcg(&A.inst_step[i]) + 1;
        if (stp >= A.nsteps) {
          act = 3;
        } else {
          A.inst_step[i] = stp;
          A.inst_it[i] = 1;
          act = 2;
        }
      } else if (it >= I.maxit) {
        record_status(A.status, kStNoConv);
      } else {
        A.inst_it[i] = it + 1;
        if (it % 8 == 0) A.need_jac[i] = 1;    // stale Jacobian: refresh at this iterate
        act = 1;
      }
      sm.act = act;
    }
  }
  __syncthreads();
  const int act = sm.act;
  if (act >= 2) {
    // converged: the root becomes the next step's start value; within a launch
    // the basis is fixed, so the next step's Newton iteration starts from the
    // linear extrapolation 2 a^{n+1} - a^n (its error, O(dt^2), is below the
    // stopping level of the FP32 projections; the root is the same)
    for (int j = t; j < k; j += blockDim.x) {
      const double root = __ldcg(&a[j]);
      const double start = __ldcg(&an[j]);
      A.an[(size_t)i * kMaxR + j] = root;
      if (act == 2) a[j] = 2.0 * root - start;
    }
  }
  if (act == 0) return;
  if (t == 0) A.tcount[i] = 0;
  __threadfence();
  __syncthreads();
  if (act == 3) {
    if (t == 0) atomicAdd(&A.ctl[2], 1u);
    return;
  }
  // publish the next iteration's tiles: the state writes above are fenced
  // before the entries that let other CTAs read them
  const int n = I.tile1 - I.tile0;
  if (t == 0) sm.base = (long long)atomicAdd(&A.ctl[1], (unsigned int)n) + A.ntiles;
  __syncthreads();
  const long long base = sm.base;
  if (base + n > A.wq_cap) {       // cannot happen within the iteration limits
    if (t == 0) record_status(A.status, kStNoConv);
    return;
  }
  volatile unsigned long long* wq = A.wq;
  for (int e = t; e < n; e += blockDim.x)
    wq[base + e] = ((unsigned long long)epoch << 32) | (unsigned int)(I.tile0 + e);
}

// Tile of work entry h, or -1 once every instance is done, an error status is
// set, or the wait runs out (a timeout is recorded). Thread 0 waits; the
// result goes to every thread.
__device__ int wait_entry(const BArgs& A, long long h, unsigned int epoch, StepSmem& sm) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int tile = -1;
    const volatile unsigned long long* wq = A.wq;
    const volatile unsigned int* done = &A.ctl[2];
    const volatile int* st = A.status;
    const long long limit = c_wait_limit;
    const long long t0 = clock64();
    for (;;) {
      if (h < A.wq_cap) {
        const unsigned long long v = wq[h];
        if ((unsigned int)(v >> 32) == epoch) {
          tile = (int)(unsigned int)(v & 0xffffffffull);
          break;
        }
      }
      if (*done >= (unsigned int)A.count || *st != 0) break;
      if (clock64() - t0 > limit) {
        record_status(A.status, kStTimeout);
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
    sm.q = tile;
  }
  __syncthreads();
  return sm.q;
}

// Largest current rank over the batch (every CTA computes the same value).
__device__ int batch_max_rank(const BArgs& A) {
  __shared__ int s_m;
  if (threadIdx.x == 0) s_m = 0;
  __syncthreads();
  int m = 0;
  for (int i = threadIdx.x; i < A.count; i += blockDim.x) m = max(m, A.rank[i]);
  m = __reduce_max_sync(0xffffffffu, m);
  if ((threadIdx.x & 31) == 0) atomicMax(&s_m, m);
  __syncthreads();
  return s_m;
}

// Calls f(integral_constant<KB>) for the bucket of r, among the buckets up to
// MAXKB.
template <int MAXKB, typename F>
__device__ __forceinline__ void with_bucket_upto(int r, F&& f) {
  const int kb = bucket_of(r);
  if (kb <= 8) { f(std::integral_constant<int, 8>{}); return; }
  if constexpr (MAXKB >= 16) { if (kb <= 16) { f(std::integral_constant<int, 16>{}); return; } }
  if constexpr (MAXKB >= 32) { if (kb <= 32) { f(std::integral_constant<int, 32>{}); return; } }
  if constexpr (MAXKB >= 48) { if (kb <= 48) { f(std::integral_constant<int, 48>{}); return; } }
  if constexpr (MAXKB >= 64) { f(std::integral_constant<int, 64>{}); }
}

constexpr int kLowRank = 16;   // rank limit of the two-CTAs-per-SM instantiation

// Two instantiations are launched back to back for every segment of steps:
// MAXKB = kLowRank (two CTAs per SM; fewer registers) runs when every rank
// is at most kLowRank, MAXKB = kMaxR otherwise; the other one returns at once.
//
// Dataflow over a work array (wq): an entry names a row tile of one
// instance's current Newton iteration; the first iteration of the first step
// of every instance is filled in at the start. A CTA claims entries in order
// (the claim of the next one goes out before it works on the current one),
// computes the tile's partials, and counts the tile in; the CTA that counts
// an instance's last tile runs that instance's update at once and appends its
// next iteration's tiles. Instances therefore advance independently, and the
// small per-instance work overlaps the other instances' streaming; there is
// no grid-wide barrier per iteration. Entries carry the launch's epoch, so
// entries of an earlier launch are never taken for this one's. No CTA that
// appends waits for anything, and a CTA waits only for an entry that was
// claimed by it, so every wait ends: the entry is written, or every instance
// is done, or an error is recorded, or the bounded wait runs out.
template <int MAXKB>
__global__ void __launch_bounds__(kBT, MAXKB <= kLowRank ? 2 : 1) batch_steps_kernel(BArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  StepSmem& sm = *reinterpret_cast<StepSmem*>(smem_raw);
  const int G = gridDim.x, b = blockIdx.x, t = threadIdx.x;
  {
    const int mr = batch_max_rank(A);
    if (MAXKB < kMaxR ? (mr > MAXKB) : (mr <= kLowRank)) return;
  }
  const unsigned int epoch = __ldcg(A.epoch) + 1u;
  for (int i = b; i < A.count; i += G) {
    for (int j = t; j < kMaxR; j += blockDim.x) A.an[(size_t)i * kMaxR + j] = A.a[(size_t)i * kMaxR + j];
    if (t == 0) {
      A.tcount[i] = 0;
      A.inst_it[i] = 1;
      A.inst_step[i] = 0;
    }
  }
  for (long long q = (long long)b * blockDim.x + t; q < A.ntiles; q += (long long)G * blockDim.x)
    A.wq[q] = ((unsigned long long)epoch << 32) | (unsigned int)__ldg(&A.qdesc[q]).x;
  if (!grid_sync(A.bar, A.status)) return;
  if (b == 0 && t == 0) *A.epoch = epoch;
  long long h = 0;     // the claimed entry (thread 0)
  if (t == 0) h = (long long)atomicAdd(&A.ctl[0], 1u);
  for (;;) {
    const int tile = wait_entry(A, h, epoch, sm);
    if (tile < 0) break;
    if (t == 0) h = (long long)atomicAdd(&A.ctl[0], 1u);
    const int i = __ldg(&A.tile_inst[tile]);
    const bool jac = __ldcg(&A.need_jac[i]) != 0;
    with_bucket_upto<MAXKB>(A.rank[i], [&](auto kb) { step_tile<decltype(kb)::value>(A, sm, tile, i, jac); });
    __threadfence();
    __syncthreads();
    if (t == 0) sm.cnt = atomicAdd(&A.tcount[i], 1);
    __syncthreads();
    const int ntile_i = A.inst[i].tile1 - A.inst[i].tile0;
    if (sm.cnt == ntile_i - 1) {
      __threadfence();
      update_instance(A, sm, i, epoch);
    }
  }
  if (b == 0 && t == 0 && __ldcg(&A.ctl[2]) >= (unsigned int)A.count && __ldcg(A.status) == 0)
    *A.M += A.nsteps;
}

// One residual sweep over the tiles into the per-tile partials (scratch),
// without a Newton update: the tile autotuner times it.
template <int MAXKB>
__global__ void __launch_bounds__(kBT, MAXKB <= kLowRank ? 2 : 1) batch_sweep_kernel(BArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  StepSmem& sm = *reinterpret_cast<StepSmem*>(smem_raw);
  {
    const int mr = batch_max_rank(A);
    if (MAXKB < kMaxR ? (mr > MAXKB) : (mr <= kLowRank)) return;
  }
  for_each_tile(&A.ctl[0], A.ntiles, &sm.q, [&](int q) {
    const int4 dsc = __ldg(&A.qdesc[q]);
    with_bucket_upto<MAXKB>(A.rank[dsc.y], [&](auto kb) {
      step_tile<decltype(kb)::value>(A, sm, dsc.x, dsc.y, false);
    });
  });
}

// ========================================================== FOM kernel ===

__device__ __forceinline__ int64_t fchunk_begin(int c, int C, int64_t n) { return (int64_t)c * n / C; }

__global__ void __launch_bounds__(kFomT, 2) batch_fom_kernel(BArgs A) {
  __shared__ float sa[kFomT], sc[kFomT], sd0[kFomT], sd1[kFomT], sd2[kFomT], sib[kFomT];
  __shared__ float ra[kFomMaxChunks], rb[kFomMaxChunks], rc[kFomMaxChunks], rd[kFomMaxChunks];
  __shared__ double su[kFomRows + 2];
  __shared__ unsigned int redu[32];
  __shared__ unsigned char s_done[kMaxBatch];
  // this CTA's work items (chunks q = b + G j), read once per launch
  __shared__ int it_inst[kFomItems], it_c[kFomItems], it_C[kFomItems], it_beg[kFomItems], it_m[kFomItems];
  __shared__ int it_n[kFomItems], it_chunk0[kFomItems];
  __shared__ long long it_vec[kFomItems];
  __shared__ double it_nu[kFomItems], it_h[kFomItems];
  const int G = gridDim.x, b = blockIdx.x, t = threadIdx.x;
  const long long M = *A.M;
  const int nitems = (A.nchunks - b + G - 1) / G;
  for (int i = t; i < A.count; i += blockDim.x) s_done[i] = is_event(A.inst[i], M) ? 0 : 1;
  for (int j = t; j < nitems; j += blockDim.x) {
    const int q = b + G * j;
    const int i = A.chunk_inst[q];
    const Inst& I = A.inst[i];
    const int C = I.nchunk, c = A.chunk_c[q];
    const int64_t beg = fchunk_begin(c, C, I.n);
    it_inst[j] = i; it_c[j] = c; it_C[j] = C; it_beg[j] = (int)beg;
    it_m[j] = (int)(fchunk_begin(c + 1, C, I.n) - beg);
    it_n[j] = I.n; it_chunk0[j] = I.chunk0; it_vec[j] = I.vec_off;
    it_nu[j] = I.nu; it_h[j] = (double)I.z * I.dt;
  }
  if (b == 0)
    for (int e = t; e < 4 * A.count; e += blockDim.x) A.fom_keys[e] = 0u;
  __syncthreads();
  for (int it = 1; it <= A.fom_maxit; ++it) {
    const int par = it & 1;
    // ---- A: residual (FP64), Jacobian rows (FP32), two-level solve per chunk ----
    // Thread p owns rows [kFomR p, kFomR p + rt) of the chunk; the last of
    // them is its separator. Level 1: a Thomas sweep (three right-hand
    // sides) writes each of its other rows as x = y + v x_L + w x_s, x_L the
    // separator on its left (the previous thread's, or the previous chunk's
    // separator s_left for p = 0) and x_s its own. Level 2: the separators of
    // threads 0 .. nt-2 form a tridiagonal system between s_left and the
    // chunk's separator s_self (the last thread's), solved by PCR into
    // x_s = Y + V s_left + W s_self. The chunk separator's own row, and the
    // chunk's first and last-but-one rows in terms of (s_left, s_self), go to
    // the separator system across chunks (B). FP32: the solve only steers the
    // Newton iteration; the FP64 residual fixes the root.
    for (int j = 0; j < nitems; ++j) {
      const int i = it_inst[j];
      if (s_done[i]) continue;
      const int q = b + G * j;
      const int64_t n = it_n[j];
      const int64_t beg = it_beg[j];
      const int m = it_m[j];
      const int nt = (m + kFomR - 1) / kFomR;       // active threads
      const int r0 = kFomR * t;
      const int rt = max(0, min(kFomR, m - r0));    // rows of this thread
      const int ni = rt - 1;                        // its interior rows
      // iterate it-1: the previous snapshot extrapolated by the previous
      // increment (it == 1), else y_new
      const double* ucur = (it == 1 ? A.y_corr : A.y_new) + it_vec[j];
      const double* dy = A.dy + it_vec[j];
      const double* uprev = A.y_corr + it_vec[j];
      const double h = it_h[j];
      const double nu = it_nu[j];
      const double inv_dx = (double)n;
      const float nu_f = (float)nu, inv_dx_f = (float)n, h_f = (float)h;
      __syncthreads();
      double un[kFomR];
#pragma unroll
      for (int r = 0; r < kFomR; ++r) {
        un[r] = 0.0;
        if (r < rt) {
          double u = __ldcg(&ucur[beg + r0 + r]);
          if (it == 1) u += dy[beg + r0 + r];
          su[1 + r0 + r] = u;
          un[r] = uprev[beg + r0 + r];
        }
      }
      if (t == 0) {
        const int64_t il = (beg - 1 + n) % n, ir = (beg + m) % n;
        double hl = __ldcg(&ucur[il]), hr = __ldcg(&ucur[ir]);
        if (it == 1) { hl += dy[il]; hr += dy[ir]; }
        su[0] = hl;
        su[m + 1] = hr;
      }
      __syncthreads();
      float a_[kFomR], b_[kFomR], c_[kFomR], d_[kFomR];
#pragma unroll
      for (int r = 0; r < kFomR; ++r) {
        a_[r] = 0.f; b_[r] = 1.f; c_[r] = 0.f; d_[r] = 0.f;
        if (r < rt) {
          const int e = r0 + r;
          const double ul = su[e], u = su[e + 1], ur = su[e + 2];
          const double f = burgers_f(ul, u, ur, nu, inv_dx);
          const double res = u - un[r] - h * f;
          float dl, dc, dr;
          burgers_band(ul, u, ur, nu_f, inv_dx_f, dl, dc, dr);
          a_[r] = -h_f * dl;
          b_[r] = 1.f - h_f * dc;
          c_[r] = -h_f * dr;
          d_[r] = (float)(-res);
        }
      }
      float* ch = A.fom_chunk + (size_t)q * kFomChunkStride;
      float* rows3 = A.fom_row + 3 * (size_t)(it_vec[j] + beg);
      // level 1: Thomas over rows 0 .. ni-1 with x_{-1} = x_L, x_{ni} = x_s
      float Y[kFomR], V[kFomR], W[kFomR], g[kFomR];
#pragma unroll
      for (int r = 0; r < kFomR; ++r) { Y[r] = 0.f; V[r] = 0.f; W[r] = 0.f; g[r] = 0.f; }
#pragma unroll
      for (int r = 0; r < kFomR - 1; ++r) {
        if (r < ni) {
          const float am = (r > 0) ? a_[r] : 0.f;
          const float beta = b_[r] - ((r > 0) ? am * g[r - 1] : 0.f);
          const float ib = __frcp_rn(beta);
          g[r] = (r + 1 < ni) ? c_[r] * ib : 0.f;
          Y[r] = (d_[r] - ((r > 0) ? am * Y[r - 1] : 0.f)) * ib;
          V[r] = ((r == 0 ? -a_[0] : 0.f) - ((r > 0) ? am * V[r - 1] : 0.f)) * ib;
          W[r] = ((r + 1 == ni ? -c_[r] : 0.f) - ((r > 0) ? am * W[r - 1] : 0.f)) * ib;
        }
      }
#pragma unroll
      for (int r = kFomR - 3; r >= 0; --r) {
        if (r + 1 < ni) {
          Y[r] -= g[r] * Y[r + 1];
          V[r] -= g[r] * V[r + 1];
          W[r] -= g[r] * W[r + 1];
        }
      }
#pragma unroll
      for (int r = 0; r < kFomR - 1; ++r)
        if (r < ni) {
          float* rw = rows3 + 3 * (size_t)(r0 + r);
          rw[0] = Y[r]; rw[1] = V[r]; rw[2] = W[r];
        }
      // this thread's separator row and its interior ends
      float as_ = 0.f, bs_ = 1.f, cs_ = 0.f, ds_ = 0.f;
      float yF = 0.f, vF = 0.f, wF = 0.f, yL = 0.f, vL = 0.f, wL = 0.f;
#pragma unroll
      for (int r = 0; r < kFomR; ++r)
        if (r == rt - 1) { as_ = a_[r]; bs_ = b_[r]; cs_ = c_[r]; ds_ = d_[r]; }
#pragma unroll
      for (int r = 0; r < kFomR - 1; ++r)
        if (r == ni - 1) { yL = Y[r]; vL = V[r]; wL = W[r]; }
      if (ni >= 1) { yF = Y[0]; vF = V[0]; wF = W[0]; }
      if (t == nt - 1) { ch[0] = as_; ch[1] = bs_; ch[2] = cs_; ch[3] = ds_; }
      // publish the first interior row (coefficients of (x_L, x_s)) for the
      // thread on the left
      sd0[t] = yF; sd1[t] = vF; sd2[t] = wF; sib[t] = (ni >= 1) ? 1.f : 0.f;
      __syncthreads();
      // level 2: the reduced row of separator p in (x_{p-1}, x_p, x_{p+1})
      const int mi = nt - 1;
      float a2 = 0.f, b2 = 1.f, c2 = 0.f, e0 = 0.f, e1 = 0.f, e2 = 0.f;
      if (t < mi) {
        if (ni >= 1) { a2 = as_ * vL; b2 = bs_ + as_ * wL; e0 = ds_ - as_ * yL; }
        else { a2 = as_; b2 = bs_; e0 = ds_; }
        if (sib[t + 1] > 0.f) { b2 += cs_ * sd1[t + 1]; c2 = cs_ * sd2[t + 1]; e0 -= cs_ * sd0[t + 1]; }
        else { c2 = cs_; }
        if (t == 0) { e1 = -a2; a2 = 0.f; }
        if (t == mi - 1) { e2 = -c2; c2 = 0.f; }
      }
      __syncthreads();
      sa[t] = a2; sc[t] = c2; sd0[t] = e0; sd1[t] = e1; sd2[t] = e2; sib[t] = __frcp_rn(b2);
      __syncthreads();
      for (int s = 1; s < mi; s <<= 1) {
        float na = a2, nb = b2, nc = c2, n0 = e0, n1 = e1, n2 = e2;
        if (t < mi) {
          const int tm = t - s, tp = t + s;
          float am = 0.f, ibm = 1.f, cm = 0.f, m0 = 0.f, m1 = 0.f, m2 = 0.f;
          float ap = 0.f, ibp = 1.f, cp = 0.f, p0 = 0.f, p1 = 0.f, p2 = 0.f;
          if (tm >= 0) { am = sa[tm]; ibm = sib[tm]; cm = sc[tm]; m0 = sd0[tm]; m1 = sd1[tm]; m2 = sd2[tm]; }
          if (tp < mi) { ap = sa[tp]; ibp = sib[tp]; cp = sc[tp]; p0 = sd0[tp]; p1 = sd1[tp]; p2 = sd2[tp]; }
          const float al = -a2 * ibm, ga = -c2 * ibp;
          na = al * am;
          nc = ga * cp;
          nb = b2 + al * cm + ga * ap;
          n0 = e0 + al * m0 + ga * p0;
          n1 = e1 + al * m1 + ga * p1;
          n2 = e2 + al * m2 + ga * p2;
        }
        __syncthreads();
        a2 = na; b2 = nb; c2 = nc; e0 = n0; e1 = n1; e2 = n2;
        sa[t] = a2; sc[t] = c2; sd0[t] = e0; sd1[t] = e1; sd2[t] = e2; sib[t] = __frcp_rn(b2);
        __syncthreads();
      }
      // separator solutions x_p = Ys + Vs s_left + Ws s_self (threads < mi)
      float Ys = 0.f, Vs = 0.f, Ws = 0.f;
      if (t < mi) {
        const float ib = sib[t];
        Ys = e0 * ib; Vs = e1 * ib; Ws = e2 * ib;
        float* rw = rows3 + 3 * (size_t)(r0 + rt - 1);
        rw[0] = Ys; rw[1] = Vs; rw[2] = Ws;
      }
      __syncthreads();
      sd0[t] = Ys; sd1[t] = Vs; sd2[t] = Ws;
      __syncthreads();
      // the chunk's first row and its last-but-one row in (s_left, s_self)
      if (t == 0) {
        if (nt == 1) { ch[4] = yF; ch[5] = vF; ch[6] = wF; }          // x_s = s_self
        else if (ni >= 1) { ch[4] = yF + wF * Ys; ch[5] = vF + wF * Vs; ch[6] = wF * Ws; }
        else { ch[4] = Ys; ch[5] = Vs; ch[6] = Ws; }
      }
      if (t == nt - 1) {
        if (nt == 1) { ch[7] = yL; ch[8] = vL; ch[9] = wL; }          // x_L = s_left
        else if (ni >= 1) {
          const float yp = sd0[t - 1], vp = sd1[t - 1], wp = sd2[t - 1];
          ch[7] = yL + vL * yp; ch[8] = vL * vp; ch[9] = vL * wp + wL;
        } else {
          ch[7] = sd0[t - 1]; ch[8] = sd1[t - 1]; ch[9] = sd2[t - 1];
        }
      }
    }
    if (!grid_sync(A.bar, A.status)) return;
    // ---- B: cyclic separator system of each instance (order C) ----
    if (b == 0)   // every CTA read the other parity's keys before the barrier above
      for (int e = t; e < A.count; e += blockDim.x) {
        A.fom_keys[4 * e + 2 * (par ^ 1)] = 0u;
        A.fom_keys[4 * e + 2 * (par ^ 1) + 1] = 0u;
      }
    for (int i = b; i < A.count; i += G) {
      if (s_done[i]) continue;
      const Inst I = A.inst[i];
      const int C = I.nchunk;
      __syncthreads();
      if (t < C) {
        const float* ch = A.fom_chunk + (size_t)(I.chunk0 + t) * kFomChunkStride;
        const float* nx = A.fom_chunk + (size_t)(I.chunk0 + (t + 1) % C) * kFomChunkStride;
        const float as_ = __ldcg(ch + 0), bs_ = __ldcg(ch + 1), cs_ = __ldcg(ch + 2), ds_ = __ldcg(ch + 3);
        const float yL = __ldcg(ch + 7), vL = __ldcg(ch + 8), wL = __ldcg(ch + 9);
        const float y0 = __ldcg(nx + 4), v0 = __ldcg(nx + 5), w0 = __ldcg(nx + 6);
        ra[t] = as_ * vL;
        rb[t] = bs_ + as_ * wL + cs_ * v0;
        rc[t] = cs_ * w0;
        rd[t] = ds_ - as_ * yL - cs_ * y0;
      }
      __syncthreads();
      for (int s = 1; s < C; s <<= 1) {
        float na = 0.f, nb = 0.f, nc = 0.f, nd = 0.f;
        if (t < C) {
          const int tm = (t - s + C) % C, tp = (t + s) % C;
          const float al = -ra[t] / rb[tm], ga = -rc[t] / rb[tp];
          na = al * ra[tm];
          nc = ga * rc[tp];
          nb = rb[t] + al * rc[tm] + ga * ra[tp];
          nd = rd[t] + al * rd[tm] + ga * rd[tp];
        }
        __syncthreads();
        if (t < C) { ra[t] = na; rb[t] = nb; rc[t] = nc; rd[t] = nd; }
        __syncthreads();
      }
      if (t < C) A.fom_sep[I.chunk0 + t] = rd[t] / (ra[t] + rb[t] + rc[t]);
    }
    if (!grid_sync(A.bar, A.status)) return;
    // ---- C: update and per-instance maxima ----
    for (int j = 0; j < nitems; ++j) {
      const int i = it_inst[j];
      if (s_done[i]) continue;
      const int C = it_C[j], c = it_c[j];
      const int64_t beg = it_beg[j];
      const int m = it_m[j];
      const int nt = (m + kFomR - 1) / kFomR;
      const int r0 = kFomR * t;
      const int rt = max(0, min(kFomR, m - r0));
      const int ni = rt - 1;
      const long long vec_off = it_vec[j];
      const float s_left = __ldcg(&A.fom_sep[it_chunk0[j] + (c - 1 + C) % C]);
      const float s_self = __ldcg(&A.fom_sep[it_chunk0[j] + c]);
      const float* rows3 = A.fom_row + 3 * (size_t)(vec_off + beg);
      unsigned int kd = 0u, ku = 0u;
      if (rt > 0) {
        // this thread's separator and the one on its left (the previous
        // thread's, whose block has kFomR rows, or s_left)
        float xs = s_self, xl = s_left;
        if (t < nt - 1) {
          const float* rw = rows3 + 3 * (size_t)(r0 + rt - 1);
          xs = __ldcg(rw) + __ldcg(rw + 1) * s_left + __ldcg(rw + 2) * s_self;
        }
        if (t > 0) {
          const float* rw = rows3 + 3 * (size_t)(r0 - 1);
          xl = __ldcg(rw) + __ldcg(rw + 1) * s_left + __ldcg(rw + 2) * s_self;
        }
        const double* ucur = (it == 1 ? A.y_corr : A.y_new) + vec_off;
#pragma unroll
        for (int r = 0; r < kFomR; ++r) {
          if (r < rt) {
            float dl;
            if (r < ni) {
              const float* rw = rows3 + 3 * (size_t)(r0 + r);
              dl = __ldcg(rw) + __ldcg(rw + 1) * xl + __ldcg(rw + 2) * xs;
            } else {
              dl = xs;
            }
            double u = __ldcg(&ucur[beg + r0 + r]) + (double)dl;
            if (it == 1) u += A.dy[vec_off + beg + r0 + r];
            A.y_new[vec_off + beg + r0 + r] = u;
            kd = max(kd, isfinite(dl) ? __float_as_uint(fabsf(dl)) : 0x7fc00000u);
            ku = max(ku, isfinite(u) ? __float_as_uint(fabsf((float)u)) : 0x7fc00000u);
          }
        }
      }
      kd = block_max_u32(kd, redu);
      ku = block_max_u32(ku, redu);
      if (t == 0) {
        atomicMax(&A.fom_keys[4 * i + 2 * par], kd);
        atomicMax(&A.fom_keys[4 * i + 2 * par + 1], ku);
      }
    }
    if (!grid_sync(A.bar, A.status)) return;
    // ---- convergence (every CTA takes the same decisions from the same keys) ----
    int any = 0, fail = 0;
    for (int i = t; i < A.count; i += blockDim.x) {
      if (s_done[i]) continue;
      const Inst I = A.inst[i];
      const unsigned int kd = __ldcg(&A.fom_keys[4 * i + 2 * par]);
      const unsigned int ku = __ldcg(&A.fom_keys[4 * i + 2 * par + 1]);
      if (kd >= 0x7f800000u || ku >= 0x7f800000u) {
        if (b == 0) record_status(A.status, kStNonFinite);
        fail = 1;
      } else if ((double)__uint_as_float(kd) <= I.tol * (1.0 + (double)__uint_as_float(ku))) {
        s_done[i] = 1;
        if (b == 0) {
          A.iters_fom[i] = it;
          A.fom_its[i] += it;
        }
      } else if (it >= I.maxit) {
        if (b == 0) record_status(A.status, kStNoConv);
        fail = 1;
      } else {
        any = 1;
      }
    }
    fail = __syncthreads_or(fail);
    any = __syncthreads_or(any);
    if (fail || !any) return;
  }
}

// ======================================================== event kernel ===

// P1: yhat = d (y - q_ref) (and y_corr <- y), p1 partial = Phi^T yhat,
// |yhat|^2 partial.
template <int KB>
__device__ void ev_p1_tile(const BArgs& A, SweepSmem& sm, int tile, int i) {
  constexpr int RPT = Rpt<KB>::v;
  constexpr int CR = kBT * RPT;
  const Inst I = A.inst[i];
  const int t = threadIdx.x;
  const int k = A.rank[i];
  const int N = I.n;
  const float* phi = A.phi + I.phi_off;
  const int r0 = A.tile_r0[tile], r1 = A.tile_r1[tile];
  float acc[KB];
#pragma unroll
  for (int j = 0; j < KB; ++j) acc[j] = 0.f;
  float yy = 0.f;
  for (int c0 = r0; c0 < r1; c0 += CR) {
    const int rows = min(CR, r1 - c0);
#pragma unroll
    for (int rr = 0; rr < RPT; ++rr) {
      const int e = rr * kBT + t;
      if (e < rows) {
        const size_t gi = (size_t)I.vec_off + c0 + e;
        const double yn = __ldcg(&A.y_new[gi]);
        A.dy[gi] = yn - A.y_corr[gi];
        A.y_corr[gi] = yn;
        const float yf = (float)(I.d * (yn - A.q_ref[gi]));
        A.yhat32[gi] = yf;
        yy = fmaf(yf, yf, yy);
#pragma unroll
        for (int j = 0; j < KB; ++j)
          if (j < k) acc[j] = fmaf(__ldg(&phi[(size_t)j * N + c0 + e]), yf, acc[j]);
      }
    }
  }
  double* gp = A.gpart + (size_t)tile * kPS;
  tile_reduce<KB>(acc, k, sm.red, gp);
  __syncthreads();
  const double ys = block_sum((double)yy, sm.dred);
  if (t == 0) gp[kMaxR] = ys;
}

// P2: q1 = yhat - Phi p1, p2 partial = Phi^T q1, |q1|^2 partial.
template <int KB>
__device__ void ev_p2_tile(const BArgs& A, SweepSmem& sm, int tile, int i) {
  constexpr int RPT = Rpt<KB>::v;
  constexpr int CR = kBT * RPT;
  const Inst I = A.inst[i];
  const int t = threadIdx.x;
  const int k = A.rank[i];
  const int N = I.n;
  const float* phi = A.phi + I.phi_off;
  const int r0 = A.tile_r0[tile], r1 = A.tile_r1[tile];
  for (int j = t; j < KB; j += kBT) sm.pf[j] = (j < k) ? (float)__ldcg(&A.ev_p[(size_t)i * kMaxCore + j]) : 0.f;
  __syncthreads();
  float acc[KB];
#pragma unroll
  for (int j = 0; j < KB; ++j) acc[j] = 0.f;
  float qq = 0.f;
  for (int c0 = r0; c0 < r1; c0 += CR) {
    const int rows = min(CR, r1 - c0);
    float x[RPT][KB];
#pragma unroll
    for (int rr = 0; rr < RPT; ++rr) {
      const int e = rr * kBT + t;
#pragma unroll
      for (int j = 0; j < KB; ++j) x[rr][j] = (e < rows && j < k) ? __ldg(&phi[(size_t)j * N + c0 + e]) : 0.f;
    }
#pragma unroll
    for (int rr = 0; rr < RPT; ++rr) {
      const int e = rr * kBT + t;
      if (e < rows) {
        const size_t gi = (size_t)I.vec_off + c0 + e;
        float v = __ldcg(&A.yhat32[gi]);
#pragma unroll
        for (int j = 0; j < KB; ++j) v = fmaf(-x[rr][j], sm.pf[j], v);
        A.qres[gi] = v;
        qq = fmaf(v, v, qq);
#pragma unroll
        for (int j = 0; j < KB; ++j) acc[j] = fmaf(x[rr][j], v, acc[j]);
      }
    }
  }
  double* gp = A.gpart2 + (size_t)tile * kPS;
  tile_reduce<KB>(acc, k, sm.red, gp);
  __syncthreads();
  const double qs = block_sum((double)qq, sm.dred);
  if (t == 0) gp[kMaxR] = qs;
}

// Rotation Phi <- [Phi, q/rho] U(:, 0:k') with q = q1 - Phi p2 (the second
// pass of classical Gram-Schmidt, which keeps q orthogonal to Phi at the
// working precision even when yhat lies almost in span(Phi)), and the Gram
// partial of the rotated rows.
template <int KB>
__device__ void ev_rot_tile(const BArgs& A, SweepSmem& sm, int tile, int i) {
  constexpr int RPT = Rpt<KB>::v;
  constexpr int CR = kBT * RPT;
  const Inst I = A.inst[i];
  const int t = threadIdx.x;
  const double* esc = A.ev_sc + (size_t)i * 8;
  const float qinv = (float)__ldcg(&esc[1]);
  const int kn = (int)__ldcg(&esc[2]);
  const int k = (int)__ldcg(&esc[3]);
  const int N = I.n;
  float* phi = A.phi + I.phi_off;
  const int r0 = A.tile_r0[tile], r1 = A.tile_r1[tile];
  for (int j = t; j < KB; j += kBT) sm.pf[j] = (j < k) ? (float)__ldcg(&A.ev_p2[(size_t)i * kMaxCore + j]) : 0.f;
  const float* ug = A.ev_u + (size_t)i * kMaxCore * kMaxR;
  for (int e = t; e < (KB + 1) * KB; e += kBT) {     // rows 0..KB; rows past k are zero
    const int row = e / KB, col = e % KB;
    sm.U[row * KB + col] = (row <= k && col < kn) ? __ldcg(&ug[row * kMaxR + col]) : 0.f;
  }
  for (int q = 0; q < 16; ++q) sm.Gd[t * 16 + q] = 0.0;
  __syncthreads();
  for (int c0 = r0; c0 < r1; c0 += CR) {
    const int rows = min(CR, r1 - c0);
#pragma unroll
    for (int rr = 0; rr < RPT; ++rr) {
      const int e = rr * kBT + t;
      float x[KB];
#pragma unroll
      for (int j = 0; j < KB; ++j) x[j] = (e < rows && j < k) ? phi[(size_t)j * N + c0 + e] : 0.f;
      if (e < rows) {
        const size_t gi = (size_t)I.vec_off + c0 + e;
        float q = __ldcg(&A.qres[gi]);
#pragma unroll
        for (int j = 0; j < KB; ++j) q = fmaf(-x[j], sm.pf[j], q);
        const float qh = q * qinv;
#pragma unroll
        for (int c = 0; c < KB; ++c) {
          float v = qh * sm.U[k * KB + c];
#pragma unroll
          for (int j = 0; j < KB; ++j) v = fmaf(x[j], sm.U[j * KB + c], v);
          if (c < kn) {
            phi[(size_t)c * N + c0 + e] = v;
            sm.P[e * KB + c] = v;
          } else {
            if (c < k) phi[(size_t)c * N + c0 + e] = 0.f;
            sm.P[e * KB + c] = 0.f;
          }
        }
      }
    }
    __syncthreads();
    // FP32 sums over at most 64 of a thread's rows (its group takes every
    // groups-th row of a run of 64 * groups), added to the thread's FP64
    // slots: about eps * 8 relative error per run instead of
    // eps * sqrt(rows per tile), at 16 FP64 adds per 64 rows
    constexpr int kRun = 64 * Blk<KB>::groups;
    for (int s0 = 0; s0 < rows; s0 += kRun) {
      float m[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) m[q] = 0.f;
      blk_accum<KB>(sm.P + s0 * KB, sm.P + s0 * KB, min(kRun, rows - s0), m);
#pragma unroll
      for (int q = 0; q < 16; ++q) sm.Gd[t * 16 + q] += (double)m[q];
    }
    __syncthreads();
  }
  // fixed-order FP64 sum over the thread groups that share a 4 x 4 block
  double* gp = A.gram_part + (size_t)tile * kMaxR * kMaxR;
  for (int e = t; e < kn * kn; e += kBT) {
    const int j = e / kn, l = e % kn;
    const int bi = (j >> 2) * Blk<KB>::nb + (l >> 2), q = (j & 3) * 4 + (l & 3);
    double v = 0.0;
    for (int g = 0; g < Blk<KB>::groups; ++g) v += sm.Gd[(g * Blk<KB>::nblk + bi) * 16 + q];
    gp[e] = v;
  }
}

// Phi <- Phi R^-1: each row y solves y R = x (FP32, R from the FP64 Cholesky).
template <int KB>
__device__ void ev_apply_tile(const BArgs& A, SweepSmem& sm, int tile, int i) {
  constexpr int RPT = Rpt<KB>::v;
  constexpr int CR = kBT * RPT;
  const Inst I = A.inst[i];
  const int t = threadIdx.x;
  const int kn = (int)__ldcg(&A.ev_sc[(size_t)i * 8 + 2]);
  const int N = I.n;
  float* phi = A.phi + I.phi_off;
  const int r0 = A.tile_r0[tile], r1 = A.tile_r1[tile];
  const float* rg = A.ev_r + (size_t)i * kMaxR * kMaxR;
  for (int e = t; e < KB * KB; e += kBT) {
    const int j = e / KB, c = e % KB;
    sm.R[j * KB + c] = (j < kn && c < kn) ? __ldcg(&rg[j * kMaxR + c]) : 0.f;
  }
  for (int j = t; j < KB; j += kBT) sm.Rd[j] = (j < kn) ? 1.f / __ldcg(&rg[j * kMaxR + j]) : 0.f;
  __syncthreads();
  for (int c0 = r0; c0 < r1; c0 += CR) {
    const int rows = min(CR, r1 - c0);
#pragma unroll
    for (int rr = 0; rr < RPT; ++rr) {
      const int e = rr * kBT + t;
      if (e < rows) {
        float y[KB];
#pragma unroll
        for (int j = 0; j < KB; ++j) y[j] = (j < kn) ? __ldcg(&phi[(size_t)j * N + c0 + e]) : 0.f;
#pragma unroll
        for (int j = 0; j < KB; ++j) {
          float v = y[j];
#pragma unroll
          for (int l = 0; l < j; ++l) v = fmaf(-y[l], sm.R[l * KB + j], v);
          y[j] = v * sm.Rd[j];
        }
#pragma unroll
        for (int j = 0; j < KB; ++j)
          if (j < kn) phi[(size_t)j * N + c0 + e] = y[j];
      }
    }
  }
}

// Core SVD of instance i in one CTA: K = [[lam Sigma, p], [0, rho]], roots of
// the secular equation one per warp, zhat (Gu-Eisenstat), vectors, sorted;
// then truncation, sigma, and the transferred state U(0:k, 0:k')^T a.
__device__ void ev_core(const BArgs& A, CoreSmem& sm, int i) {
  const Inst I = A.inst[i];
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5, nw = blockDim.x >> 5;
  const int k = A.rank[i];
  const int n = k + 1;
  double* pv = A.ev_p + (size_t)i * kMaxCore;
  double* esc = A.ev_sc + (size_t)i * 8;
  // p2 and |q1|^2, then p = p1 + p2, rho^2 = |q1|^2 - |p2|^2
  sum_tiles(A.gpart2, I.tile0, I.tile1, k, 0, sm.z);   // p2
  __syncthreads();
  // |q1|^2 (offset kMaxR of each tile vector)
  sum_tiles(A.gpart2, I.tile0, I.tile1, 1, kMaxR, &sm.sc[0]);
  __syncthreads();
  if (t == 0) {
    double p2n = 0.0;
    for (int j = 0; j < k; ++j) p2n += sm.z[j] * sm.z[j];
    double rho2 = sm.sc[0] - p2n;
    double rho = sqrt(fmax(rho2, 0.0));
    const double ynorm = sqrt(__ldcg(&esc[0]));
    const double s1 = (k > 0) ? A.sigma[(size_t)i * kMaxR] : 0.0;
    const bool keep = rho > I.rank_tol * fmax(ynorm, s1);
    if (!keep) rho = 0.0;
    for (int j = 0; j < k; ++j) {
      const double p = __ldcg(&pv[j]) + sm.z[j];
      A.ev_p2[(size_t)i * kMaxCore + j] = sm.z[j];
      pv[j] = p;
      sm.z[j] = p;
      sm.d_desc[j] = I.lam * A.sigma[(size_t)i * kMaxR + j];
    }
    sm.d_desc[k] = 0.0;
    sm.z[k] = rho;
    esc[1] = keep ? 1.0 / rho : 0.0;
    secular_setup(sm.S, n, sm.d_desc, sm.z);
  }
  for (int j = t; j < k; j += blockDim.x) sm.aold[j] = A.a[(size_t)i * kMaxR + j];
  __syncthreads();
  const SecularSetup& S = sm.S;
  const int k2 = S.k2;
  for (int j = wid; j < k2; j += nw) {
    int o;
    double tau;
    secular_root(S, j, o, tau);
    if (lane == 0) { sm.tau[j] = tau; sm.orig[j] = (double)o; }
  }
  __syncthreads();
  for (int ii = wid; ii < k2; ii += nw) {
    double pr = 1.0;
    for (int j = lane; j < k2; j += 32) {
      const int o = (int)sm.orig[j];
      const double tau = sm.tau[j];
      const double num = root_minus(S, o, tau, ii) * root_plus(S, o, tau, ii);
      double den;
      if (j == k2 - 1) den = 1.0;
      else if (j < ii) den = (S.D[j] - S.D[ii]) * (S.D[j] + S.D[ii]);
      else den = (S.D[j + 1] - S.D[ii]) * (S.D[j + 1] + S.D[ii]);
      pr *= num / den;
    }
    pr = warp_prod(pr);
    if (lane == 0) sm.zhat[ii] = copysign(sqrt(fabs(pr)), S.Z[ii]);
  }
  if (t == 0) {
    for (int e = 0; e < k2; ++e) sm.val[e] = S.D[(int)sm.orig[e]] + sm.tau[e];
    int c = k2;
    for (int p = 0; p < n; ++p)
      if (S.defl[p]) { sm.val[c] = S.dpos[p]; sm.order[c] = p; ++c; }
  }
  __syncthreads();
  if (t < n) {
    const double v = sm.val[t];
    int ps = 0;
    for (int e = 0; e < n; ++e) {
      const double w = sm.val[e];
      if (w > v || (w == v && e < t)) ++ps;
    }
    sm.pos[t] = ps;
    sm.defp[t] = (t >= k2) ? sm.order[t] : -1;
  }
  __syncthreads();
  for (int e = wid; e < n; e += nw) {
    double* pw = sm.pv[wid];
    for (int p = lane; p < n; p += 32) pw[p] = 0.0;
    __syncwarp();
    if (e < k2) {
      const int o = (int)sm.orig[e];
      const double tau = sm.tau[e];
      double vec[3];
      double ss = 0.0;
      for (int mm = 0; mm < 3; ++mm) {
        const int ci = lane + 32 * mm;
        vec[mm] = 0.0;
        if (ci < k2) {
          const double den = -(root_minus(S, o, tau, ci)) * root_plus(S, o, tau, ci);
          const double u = sm.zhat[ci] / den;
          vec[mm] = u;
          ss += u * u;
        }
      }
      ss = warp_sum(ss);
      const double inv = 1.0 / sqrt(ss);
      for (int mm = 0; mm < 3; ++mm) {
        const int ci = lane + 32 * mm;
        if (ci < k2) pw[S.cidx[ci]] = vec[mm] * inv;
      }
    } else if (lane == 0) {
      pw[sm.defp[e]] = 1.0;
    }
    __syncwarp();
    if (lane == 0)
      for (int q = S.nrot - 1; q >= 0; --q) {
        const int pa = S.rot_a[q], pb = S.rot_b[q];
        const double c = S.rot_c[q], s = S.rot_s[q];
        const double xa = pw[pa], xb = pw[pb];
        pw[pa] = c * xa + s * xb;
        pw[pb] = -s * xa + c * xb;
      }
    __syncwarp();
    const int col = sm.pos[e];
    for (int p = lane; p < n; p += 32) sm.U[(n - 1 - p) * kMaxCore + col] = pw[p];
    if (lane == 0) sm.sbar[col] = sm.val[e];
    __syncwarp();
  }
  __syncthreads();
  // truncation: singular values above rank_tol * s_1, at most r
  int kn = 0;
  {
    const double s0 = sm.sbar[0];
    for (int j = 0; j < n && j < I.r; ++j)
      if (s0 > 0.0 && sm.sbar[j] > I.rank_tol * s0) ++kn;
  }
  float* ug = A.ev_u + (size_t)i * kMaxCore * kMaxR;
  for (int e = t; e < n * kn; e += blockDim.x) {
    const int row = e / kn, col = e % kn;
    ug[row * kMaxR + col] = (float)sm.U[row * kMaxCore + col];
  }
  if (t < I.r) {
    A.sigma[(size_t)i * kMaxR + t] = (t < kn) ? sm.sbar[t] : 0.0;
    double v = 0.0;
    if (t < kn)
      for (int j = 0; j < k; ++j) v = fma(sm.U[j * kMaxCore + t], sm.aold[j], v);
    A.ev_anew[(size_t)i * kMaxR + t] = v;
  }
  if (t == 0) { esc[2] = (double)kn; esc[3] = (double)k; }
  __syncthreads();
}

// Gram matrix of the rotated basis, FP64 Cholesky G = R^T R (R upper), the
// state a <- R a_new, rank and sigma bookkeeping.
__device__ void ev_chol(const BArgs& A, CholSmem& sm, int i) {
  const Inst I = A.inst[i];
  const int t = threadIdx.x;
  const int kn = (int)__ldcg(&A.ev_sc[(size_t)i * 8 + 2]);
  for (int e = t; e < kn * kn; e += blockDim.x) {
    double s = 0.0;
    for (int tt = I.tile0; tt < I.tile1; ++tt) s += __ldcg(&A.gram_part[(size_t)tt * kMaxR * kMaxR + e]);
    const int j = e / kn, l = e % kn;
    sm.G[j * kMaxR + l] = s;
  }
  for (int j = t; j < kn; j += blockDim.x) sm.anew[j] = __ldcg(&A.ev_anew[(size_t)i * kMaxR + j]);
  __syncthreads();
  // right-looking Cholesky on the upper triangle (row j of R = row j of G / d)
  for (int j = 0; j < kn; ++j) {
    if (t == 0) sm.d = sqrt(fmax(sm.G[j * kMaxR + j], DBL_MIN));
    __syncthreads();
    const double d = sm.d, inv = 1.0 / d;
    for (int c = j + t; c < kn; c += blockDim.x) sm.G[j * kMaxR + c] = (c == j) ? d : sm.G[j * kMaxR + c] * inv;
    __syncthreads();
    const int rem = kn - j - 1;
    for (int e = t; e < rem * rem; e += blockDim.x) {
      const int l = j + 1 + e / rem, c = j + 1 + e % rem;
      if (c >= l) sm.G[l * kMaxR + c] -= sm.G[j * kMaxR + l] * sm.G[j * kMaxR + c];
    }
    __syncthreads();
  }
  float* rg = A.ev_r + (size_t)i * kMaxR * kMaxR;
  for (int e = t; e < kn * kn; e += blockDim.x) {
    const int j = e / kn, c = e % kn;
    rg[j * kMaxR + c] = (c >= j) ? (float)sm.G[j * kMaxR + c] : 0.f;
  }
  if (t < I.r) {
    double v = 0.0;
    if (t < kn)
      for (int c = t; c < kn; ++c) v = fma(sm.G[t * kMaxR + c], sm.anew[c], v);
    A.a[(size_t)i * kMaxR + t] = v;
  }
  if (t == 0) {
    A.rank[i] = kn;
    A.need_jac[i] = 1;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kBT, 1) batch_event_kernel(BArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SweepSmem& sw = *reinterpret_cast<SweepSmem*>(smem_raw);
  CoreSmem& cs = *reinterpret_cast<CoreSmem*>(smem_raw);
  CholSmem& ch = *reinterpret_cast<CholSmem*>(smem_raw);
  const int G = gridDim.x, b = blockIdx.x;
  const long long M = *A.M;
  // ---- P1 ----
  for_each_tile(&A.ctl[0], A.ntiles, &sw.q, [&](int q) {
    const int4 dsc = __ldg(&A.qdesc[q]);
    const int tile = dsc.x, i = dsc.y;
    if (!is_event(A.inst[i], M)) return;
    with_bucket(A.rank[i], [&](auto kb) { ev_p1_tile<decltype(kb)::value>(A, sw, tile, i); });
  });
  if (!grid_sync(A.bar, A.status)) return;
  // ---- p1 and |yhat|^2 per instance ----
  for (int i = b; i < A.count; i += G) {
    const Inst I = A.inst[i];
    if (!is_event(I, M)) continue;
    __syncthreads();
    sum_tiles(A.gpart, I.tile0, I.tile1, A.rank[i], 0, A.ev_p + (size_t)i * kMaxCore);
    sum_tiles(A.gpart, I.tile0, I.tile1, 1, kMaxR, A.ev_sc + (size_t)i * 8);
  }
  if (!grid_sync(A.bar, A.status)) return;
  // ---- P2 ----
  for_each_tile(&A.ctl[1], A.ntiles, &sw.q, [&](int q) {
    const int4 dsc = __ldg(&A.qdesc[q]);
    const int tile = dsc.x, i = dsc.y;
    if (!is_event(A.inst[i], M)) return;
    with_bucket(A.rank[i], [&](auto kb) { ev_p2_tile<decltype(kb)::value>(A, sw, tile, i); });
  });
  if (!grid_sync(A.bar, A.status)) return;
  // ---- core SVD per instance ----
  for (int i = b; i < A.count; i += G) {
    if (!is_event(A.inst[i], M)) continue;
    __syncthreads();
    ev_core(A, cs, i);
  }
  if (!grid_sync(A.bar, A.status)) return;
  // ---- rotation + Gram ----
  for_each_tile(&A.ctl[2], A.ntiles, &sw.q, [&](int q) {
    const int4 dsc = __ldg(&A.qdesc[q]);
    const int tile = dsc.x, i = dsc.y;
    if (!is_event(A.inst[i], M)) return;
    const double* esc = A.ev_sc + (size_t)i * 8;   // k' and k of this update
    const int kb_cols = max((int)__ldcg(&esc[2]), (int)__ldcg(&esc[3]));
    with_bucket(kb_cols, [&](auto kb) { ev_rot_tile<decltype(kb)::value>(A, sw, tile, i); });
  });
  if (!grid_sync(A.bar, A.status)) return;
  // ---- Cholesky per instance ----
  for (int i = b; i < A.count; i += G) {
    if (!is_event(A.inst[i], M)) continue;
    __syncthreads();
    ev_chol(A, ch, i);
  }
  if (!grid_sync(A.bar, A.status)) return;
  // ---- Phi <- Phi R^-1 ----
  for_each_tile(&A.ctl[3], A.ntiles, &sw.q, [&](int q) {
    const int4 dsc = __ldg(&A.qdesc[q]);
    const int tile = dsc.x, i = dsc.y;
    if (!is_event(A.inst[i], M)) return;
    with_bucket((int)__ldcg(&A.ev_sc[(size_t)i * 8 + 2]), [&](auto kb) { ev_apply_tile<decltype(kb)::value>(A, sw, tile, i); });
  });
}

// FP32 copies of q_ref and of its first and second differences (periodic),
// differences taken in FP64.
__global__ void batch_qref_kernel(const double* q_ref, int n, float* qr, float* dq, float* lq) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double qm = q_ref[(i - 1 + n) % n], q0 = q_ref[i], qp = q_ref[(i + 1) % n];
    qr[i] = (float)q0;
    dq[i] = (float)(qp - q0);
    lq[i] = (float)((qp - q0) - (q0 - qm));
  }
}

// Lift of one instance: out = q_ref + d^-1 Phi a.
__global__ void batch_lift_kernel(const float* phi, const double* q_ref, const double* a, int n, int k,
                                  double dinv, double* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int j = 0; j < k; ++j) s = fmaf(phi[(size_t)j * n + i], (float)a[j], s);
    out[i] = fma(dinv, (double)s, q_ref[i]);
  }
}

}  // namespace
// Wait bound of this translation unit's kernels (see rom_internal.cuh).
cudaError_t set_wait_limit_batch(long long cycles) { return set_wait_limit_here(cycles); }

}  // namespace rom

// ============================================================= host side ===

using namespace rom;

struct rom_batch {
  int count;
  cudaStream_t stream;
  int grid_sweep, grid_fom, grid_lo;
  long long M;                 // online steps done by every instance
  int ntiles, nchunks, fom_maxit;
  int steps_per_launch;        // steps of one launch of the steps kernel
  int poisoned;
  std::vector<Inst> hinst;
  std::vector<rom_config> cfg;
  std::vector<long long> w_init;
  BArgs A;                     // device pointers
  double* lift;                // lifted state of one instance (max N)
  std::vector<void*> allocs;
  // tile tables (rebuilt by the autotuner) and their device copies
  Inst* d_inst;
  int *d_ti, *d_r0, *d_r1, *d_order;
  int4* d_qdesc;
  int tile_rows;
  float tune_ms[4];            // timed residual sweep per candidate tile size
  // one adaptation interval (steps + coarse FOM + iSVD) captured as a graph
  cudaGraphExec_t seg_graph;
  long long seg_len;
  int graph_state;             // 0 not tried, 1 captured, -1 unavailable
  // per-phase timing: 0 steps, 1 coarse FOM, 2 iSVD
  int prof_on;
  std::vector<cudaEvent_t> ev;
  std::vector<int> ev_phase;
  double prof_ms[3];
  long long prof_cnt[3];
};

namespace {

#define BCK(x)                                      \
  do {                                              \
    cudaError_t e_ = (x);                           \
    if (e_ != cudaSuccess) {                        \
      cudaGetLastError();                           \
      return ROM_ECUDA;                             \
    }                                               \
  } while (0)

template <typename T>
cudaError_t balloc(rom_batch* B, T** p, size_t n) {
  void* v = nullptr;
  cudaError_t e = cudaMalloc(&v, n * sizeof(T) > 0 ? n * sizeof(T) : 16);
  if (e != cudaSuccess) return e;
  B->allocs.push_back(v);
  *p = static_cast<T*>(v);
  return cudaSuccess;
}

void batch_free(rom_batch* B) {
  if (B->seg_graph) cudaGraphExecDestroy(B->seg_graph);
  B->seg_graph = nullptr;
  for (void* p : B->allocs) cudaFree(p);
  B->allocs.clear();
  for (cudaEvent_t e : B->ev) cudaEventDestroy(e);
  B->ev.clear();
}

rom_status batch_finish(rom_batch* B) {
  cudaError_t e = cudaStreamSynchronize(B->stream);
  if (e != cudaSuccess) { B->poisoned = 1; return ROM_ECUDA; }
  int st = 0;
  e = cudaMemcpy(&st, B->A.status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) { B->poisoned = 1; return ROM_ECUDA; }
  if (st != 0) {
    cudaMemset(B->A.status, 0, sizeof(int));
    cudaMemset(B->A.bar, 0, sizeof(GridBarrier));
    B->poisoned = 1;   // instances may have stopped mid-step
  }
  switch (st) {
    case 0: return ROM_OK;
    case kStNoConv: return ROM_ENOCONV;
    case kStNonFinite: return ROM_ENONFINITE;
    case kStTimeout: return ROM_ETIMEOUT;
    default: return ROM_ECUDA;
  }
}

cudaError_t prof_mark(rom_batch* B, int phase) {
  if (!B->prof_on) return cudaSuccess;
  cudaEvent_t e;
  cudaError_t r = cudaEventCreate(&e);
  if (r != cudaSuccess) return r;
  B->ev.push_back(e);
  B->ev_phase.push_back(phase);
  return cudaEventRecord(e, B->stream);
}

cudaError_t prof_collect(rom_batch* B) {
  cudaError_t r = cudaStreamSynchronize(B->stream);
  if (r != cudaSuccess) return r;
  for (size_t e = 0; e + 1 < B->ev.size(); e += 2) {
    float ms = 0.f;
    r = cudaEventElapsedTime(&ms, B->ev[e], B->ev[e + 1]);
    if (r != cudaSuccess) return r;
    B->prof_ms[B->ev_phase[e]] += ms;
    B->prof_cnt[B->ev_phase[e]] += 1;
  }
  for (cudaEvent_t e : B->ev) cudaEventDestroy(e);
  B->ev.clear();
  B->ev_phase.clear();
  return cudaSuccess;
}

cudaError_t launch_coop(const void* fn, int grid, int block, size_t smem, BArgs& A, cudaStream_t s) {
  void* args[] = {&A};
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(block), args, smem, s);
}

// nsteps steps of every instance, in launches of at most steps_per_launch
// steps (the bound that sizes the work array of the steps kernel).
cudaError_t run_steps(rom_batch* B, int nsteps) {
  for (int done = 0; done < nsteps;) {
    const int n = std::min(nsteps - done, B->steps_per_launch);
    cudaError_t e = cudaMemsetAsync(B->A.ctl, 0, 8 * sizeof(unsigned int), B->stream);
    if (e != cudaSuccess) return e;
    B->A.nsteps = n;
    if ((e = prof_mark(B, 0)) != cudaSuccess) return e;
    e = launch_coop((const void*)batch_steps_kernel<kLowRank>, B->grid_lo, kBT, sizeof(StepSmem), B->A, B->stream);
    if (e != cudaSuccess) return e;
    e = launch_coop((const void*)batch_steps_kernel<kMaxR>, B->grid_sweep, kBT, sizeof(StepSmem), B->A, B->stream);
    if (e != cudaSuccess) return e;
    if ((e = prof_mark(B, 0)) != cudaSuccess) return e;
    done += n;
  }
  return cudaSuccess;
}

cudaError_t run_event(rom_batch* B) {
  cudaError_t e = prof_mark(B, 1);
  if (e != cudaSuccess) return e;
  e = launch_coop((const void*)batch_fom_kernel, B->grid_fom, kFomT, 0, B->A, B->stream);
  if (e != cudaSuccess) return e;
  if ((e = prof_mark(B, 1)) != cudaSuccess) return e;
  e = cudaMemsetAsync(B->A.ctl, 0, 8 * sizeof(unsigned int), B->stream);
  if (e != cudaSuccess) return e;
  if ((e = prof_mark(B, 2)) != cudaSuccess) return e;
  size_t smem = std::max(sizeof(SweepSmem), std::max(sizeof(CoreSmem), sizeof(CholSmem)));
  e = launch_coop((const void*)batch_event_kernel, B->grid_sweep, kBT, smem, B->A, B->stream);
  if (e != cudaSuccess) return e;
  return prof_mark(B, 2);
}

size_t event_smem() { return std::max(sizeof(SweepSmem), std::max(sizeof(CoreSmem), sizeof(CholSmem))); }

// Captures the launches of one adaptation interval (seg steps, then the
// coarse FOM and the iSVD update) into a graph. Every launch reads the step
// counter and the ranks from device memory, so the same graph serves every
// interval of that length. Fails (and nothing runs) on a stream that cannot
// be captured, such as the legacy default stream.
cudaError_t capture_interval(rom_batch* B, long long seg) {
  cudaError_t e = cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t e1 = run_steps(B, (int)seg);
  if (e1 == cudaSuccess) e1 = run_event(B);
  cudaGraph_t g = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(B->stream, &g);
  if (e1 == cudaSuccess) e1 = e2;
  if (e1 == cudaSuccess) e1 = cudaGraphInstantiate(&B->seg_graph, g, 0);
  if (g) cudaGraphDestroy(g);
  return e1;
}

// Row tiles of tile_rows rows (the last one of an instance ragged), the queue
// ordered by decreasing cost (rows x (rank + 3), the live columns plus the
// reference data), uploaded with the instances' tile ranges.
cudaError_t set_tiles(rom_batch* B, int tile_rows, const std::vector<int>& rank) {
  std::vector<int> tinst, tr0, tr1;
  for (int i = 0; i < B->count; ++i) {
    Inst& I = B->hinst[i];
    I.tile0 = (int)tinst.size();
    for (int r0 = 0; r0 < I.n; r0 += tile_rows) {
      tinst.push_back(i);
      tr0.push_back(r0);
      tr1.push_back(std::min(I.n, r0 + tile_rows));
    }
    I.tile1 = (int)tinst.size();
  }
  const int nt = (int)tinst.size();
  std::vector<int> order(nt);
  for (int q = 0; q < nt; ++q) order[q] = q;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    const long long cx = (long long)(tr1[x] - tr0[x]) * (rank[tinst[x]] + 3);
    const long long cy = (long long)(tr1[y] - tr0[y]) * (rank[tinst[y]] + 3);
    return cx > cy;
  });
  std::vector<int4> qdesc(nt);
  for (int q = 0; q < nt; ++q) {
    const int tl = order[q];
    qdesc[q] = make_int4(tl, tinst[tl], tr0[tl], tr1[tl]);
  }
  cudaStream_t s = B->stream;
  cudaError_t e = cudaMemcpyAsync(B->d_ti, tinst.data(), sizeof(int) * nt, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(B->d_r0, tr0.data(), sizeof(int) * nt, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(B->d_r1, tr1.data(), sizeof(int) * nt, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(B->d_order, order.data(), sizeof(int) * nt, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(B->d_qdesc, qdesc.data(), sizeof(int4) * nt, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(B->d_inst, B->hinst.data(), sizeof(Inst) * B->count, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) {
    B->ntiles = nt;
    B->A.ntiles = nt;
    B->tile_rows = tile_rows;
  }
  return e;
}

// Device time of one residual sweep over all tiles (mean of three, after one
// untimed), without changing any state.
cudaError_t time_dry_sweep(rom_batch* B, float* ms) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  for (int r = -1; r < 3 && e == cudaSuccess; ++r) {
    if (r == 0) e = cudaEventRecord(e0, B->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(B->A.ctl, 0, 8 * sizeof(unsigned int), B->stream);
    if (e == cudaSuccess)
      e = launch_coop((const void*)batch_sweep_kernel<kLowRank>, B->grid_lo, kBT, sizeof(StepSmem), B->A, B->stream);
    if (e == cudaSuccess)
      e = launch_coop((const void*)batch_sweep_kernel<kMaxR>, B->grid_sweep, kBT, sizeof(StepSmem), B->A, B->stream);
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, B->stream);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  *ms = t / 3.f;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return e;
}

}  // namespace

extern "C" {

rom_status rom_batch_init(const rom_config* cfgs, const double* const* q0s, int32_t count, void* stream,
                          rom_batch** out) {
  if (!out) return ROM_EINVAL;
  *out = nullptr;
  if (!cfgs || !q0s || count < 1 || count > kMaxBatch) return ROM_EINVAL;
  for (int i = 0; i < count; ++i) {
    const rom_config& c = cfgs[i];
    if (c.problem != ROM_BURGERS || c.precision != ROM_MIXED_FP32 || c.n_s != 0 || c.n_var != 1 ||
        c.projection != ROM_GALERKIN || c.time_scheme != ROM_BACKWARD_EULER || c.r < 1 || c.r > kMaxR || c.n_cells < 256 ||
        c.n_cells > 131072 || c.z < 1 || !q0s[i])
      return ROM_EINVAL;
  }
  int dev = 0;
  BCK(cudaGetDevice(&dev));
  rom_batch* B = new rom_batch;
  B->count = count;
  B->stream = (cudaStream_t)stream;
  B->M = 0;
  B->poisoned = 0;
  B->prof_on = 0;
  B->seg_graph = nullptr;
  B->seg_len = 0;
  B->graph_state = 0;
  B->d_inst = nullptr;
  B->d_ti = B->d_r0 = B->d_r1 = B->d_order = nullptr;
  B->d_qdesc = nullptr;
  B->tile_rows = 0;
  for (int c = 0; c < 4; ++c) B->tune_ms[c] = 0.f;
  for (int p = 0; p < 3; ++p) { B->prof_ms[p] = 0.0; B->prof_cnt[p] = 0; }
  B->cfg.assign(cfgs, cfgs + count);
  memset(&B->A, 0, sizeof(BArgs));
  // ---- layout: packed bases and vectors, tiles, FOM chunks ----
  std::vector<int> cinst, cc;
  long long phi_tot = 0, vec_tot = 0, nmax = 1;
  int ntiles_max = 0;
  int fom_maxit = 1;
  B->hinst.resize(count);
  for (int i = 0; i < count; ++i) {
    const rom_config& c = cfgs[i];
    Inst& I = B->hinst[i];
    I.n = (int)c.n_cells;
    I.r = c.r;
    I.z = c.z;
    I.maxit = c.newton_max;
    I.nu = c.nu;
    I.dt = c.dt;
    I.lam = c.lambda;
    I.tol = c.newton_tol;
    I.rank_tol = c.rank_tol > 0.0 ? c.rank_tol : 1e-5;
    I.phi_off = phi_tot;
    nmax = std::max(nmax, (long long)I.n);
    I.vec_off = vec_tot;
    phi_tot += ((long long)I.n * I.r + 63) / 64 * 64;
    vec_tot += ((long long)I.n + 31) / 32 * 32;
    ntiles_max += (I.n + kTileRowsMin - 1) / kTileRowsMin;
    int C = 4;
    while ((I.n + C - 1) / C > kFomRows && C < kFomMaxChunks) C *= 2;
    if ((I.n + C - 1) / C > kFomRows) { delete B; return ROM_EINVAL; }
    I.chunk0 = (int)cinst.size();
    I.nchunk = C;
    for (int q = 0; q < C; ++q) { cinst.push_back(i); cc.push_back(q); }
    fom_maxit = std::max(fom_maxit, c.newton_max);
  }
  B->ntiles = ntiles_max;
  B->nchunks = (int)cinst.size();
  B->fom_maxit = fom_maxit;
  // work array of the steps kernel: the first iteration's tiles plus one
  // append of every tile per Newton iteration of every step of a launch
  // (fom_maxit is the largest Newton limit of the batch); at most 16 steps
  // a launch, fewer where the array would pass 4M entries
  {
    const long long budget = 4LL << 20;
    long long spl = (budget / std::max(1, ntiles_max) - 1) / std::max(1, fom_maxit);
    B->steps_per_launch = (int)std::max(1LL, std::min(16LL, spl));
  }
  const long long wq_cap = (long long)ntiles_max * (1 + (long long)B->steps_per_launch * fom_maxit);
  BArgs& A = B->A;
  A.count = count;
  A.ntiles = B->ntiles;
  A.nchunks = B->nchunks;
  A.fom_maxit = fom_maxit;
  cudaError_t e = cudaSuccess;
  Inst* d_inst = nullptr;
  int *d_ti = nullptr, *d_r0 = nullptr, *d_r1 = nullptr, *d_order = nullptr, *d_ci = nullptr, *d_cc = nullptr;
  int4* d_qdesc = nullptr;
#define BA(p, n) \
  if (e == cudaSuccess) e = balloc(B, &(p), (size_t)(n))
  BA(d_inst, count); BA(d_ti, B->ntiles); BA(d_r0, B->ntiles); BA(d_r1, B->ntiles); BA(d_order, B->ntiles);
  BA(d_ci, B->nchunks); BA(d_cc, B->nchunks); BA(d_qdesc, B->ntiles);
  BA(A.phi, phi_tot); BA(A.q_ref, vec_tot); BA(A.y_corr, vec_tot); BA(A.y_new, vec_tot); BA(A.dy, vec_tot);
  BA(A.a, (size_t)count * kMaxR); BA(A.an, (size_t)count * kMaxR); BA(A.sigma, (size_t)count * kMaxR);
  BA(A.sweeps, count); BA(A.sweep_cols, count); BA(A.rank, count); BA(A.need_jac, count); BA(A.iters_rom, count); BA(A.iters_fom, count); BA(A.fom_its, count);
  BA(A.jlu, (size_t)count * kMaxR * kMaxR);
  BA(A.gpart, (size_t)B->ntiles * kPS); BA(A.gpart2, (size_t)B->ntiles * kPS);
  BA(A.mpart, (size_t)B->ntiles * kMaxR * kMaxR); BA(A.gram_part, (size_t)B->ntiles * kMaxR * kMaxR);
  BA(A.fom_row, 3 * (size_t)vec_tot); BA(A.fom_chunk, (size_t)B->nchunks * kFomChunkStride);
  BA(A.fom_sep, B->nchunks); BA(A.fom_keys, 4 * (size_t)count);
  BA(A.ev_p, (size_t)count * kMaxCore); BA(A.ev_p2, (size_t)count * kMaxCore); BA(A.ev_sc, (size_t)count * 8);
  BA(A.qres, vec_tot); BA(A.yhat32, vec_tot); BA(A.qr32, vec_tot); BA(A.dq32, vec_tot); BA(A.lq32, vec_tot);
  BA(A.ev_u, (size_t)count * kMaxCore * kMaxR); BA(A.ev_anew, (size_t)count * kMaxR);
  BA(A.ev_r, (size_t)count * kMaxR * kMaxR); BA(A.ctl, 8); BA(A.M, 1); BA(A.bar, 1); BA(A.status, 1);
  BA(A.wq, wq_cap); BA(A.tcount, count); BA(A.inst_it, count); BA(A.inst_step, count); BA(A.epoch, 1);
  A.wq_cap = wq_cap;
  BA(B->lift, nmax);
#undef BA
  if (e != cudaSuccess) {
    cudaGetLastError();
    batch_free(B);
    delete B;
    return ROM_ENOMEM;
  }
  A.inst = d_inst;
  A.tile_inst = d_ti; A.tile_r0 = d_r0; A.tile_r1 = d_r1; A.order = d_order; A.qdesc = d_qdesc;
  A.chunk_inst = d_ci; A.chunk_c = d_cc;
  cudaStream_t s = B->stream;
  auto fail = [&](rom_status st) {
    cudaStreamSynchronize(s);
    cudaGetLastError();
    batch_free(B);
    delete B;
    return st;
  };
  const double* qref_d = A.q_ref;
  if (cudaMemsetAsync(A.phi, 0, sizeof(float) * phi_tot, s) != cudaSuccess ||
      cudaMemsetAsync(A.a, 0, sizeof(double) * count * kMaxR, s) != cudaSuccess ||
      cudaMemsetAsync(A.dy, 0, sizeof(double) * vec_tot, s) != cudaSuccess ||
      cudaMemsetAsync(A.sigma, 0, sizeof(double) * count * kMaxR, s) != cudaSuccess ||
      cudaMemsetAsync(A.need_jac, 0, sizeof(int) * count, s) != cudaSuccess ||
      cudaMemsetAsync(A.iters_rom, 0, sizeof(int) * count, s) != cudaSuccess ||
      cudaMemsetAsync(A.iters_fom, 0, sizeof(int) * count, s) != cudaSuccess ||
      cudaMemsetAsync(A.fom_its, 0, sizeof(long long) * count, s) != cudaSuccess ||
      cudaMemsetAsync(A.sweeps, 0, sizeof(long long) * count, s) != cudaSuccess ||
      cudaMemsetAsync(A.sweep_cols, 0, sizeof(long long) * count, s) != cudaSuccess ||
      cudaMemsetAsync(A.M, 0, sizeof(long long), s) != cudaSuccess ||
      cudaMemsetAsync(A.epoch, 0, sizeof(unsigned int), s) != cudaSuccess ||
      cudaMemsetAsync(A.wq, 0, sizeof(unsigned long long) * wq_cap, s) != cudaSuccess ||
      cudaMemsetAsync(A.bar, 0, sizeof(GridBarrier), s) != cudaSuccess ||
      cudaMemsetAsync(A.status, 0, sizeof(int), s) != cudaSuccess)
    return fail(ROM_ECUDA);
  // ---- offline stage of every instance (training FOM, POD, initial state,
  //      first correction snapshot) through the single-instance path ----
  B->w_init.resize(count);
  for (int i = 0; i < count; ++i) {
    rom_ctx* ctx = nullptr;
    rom_status st = rom_init(&cfgs[i], q0s[i], stream, &ctx);
    if (st != ROM_OK) return fail(st);
    Inst& I = B->hinst[i];
    const size_t N = (size_t)I.n;
    double dv = 1.0;
    bool ok = cudaMemcpyAsync(A.phi + I.phi_off, ctx->d.phi32, sizeof(float) * N * I.r, cudaMemcpyDeviceToDevice, s) == cudaSuccess &&
              cudaMemcpyAsync(const_cast<double*>(qref_d) + I.vec_off, ctx->d.q_ref, sizeof(double) * N, cudaMemcpyDeviceToDevice, s) == cudaSuccess &&
              cudaMemcpyAsync(A.y_corr + I.vec_off, ctx->d.y_corr, sizeof(double) * N, cudaMemcpyDeviceToDevice, s) == cudaSuccess &&
              cudaMemcpyAsync(A.a + (size_t)i * kMaxR, ctx->d.a, sizeof(double) * I.r, cudaMemcpyDeviceToDevice, s) == cudaSuccess &&
              cudaMemcpyAsync(A.sigma + (size_t)i * kMaxR, ctx->d.sigma, sizeof(double) * I.r, cudaMemcpyDeviceToDevice, s) == cudaSuccess &&
              cudaMemcpyAsync(A.rank + i, ctx->d.rank, sizeof(int), cudaMemcpyDeviceToDevice, s) == cudaSuccess &&
              cudaMemcpyAsync(&dv, ctx->d.dvals, sizeof(double), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
              cudaStreamSynchronize(s) == cudaSuccess;
    I.rank_tol = ctx->cfg.rank_tol;
    B->w_init[i] = ctx->step;
    batch_qref_kernel<<<64, 256, 0, s>>>(qref_d + I.vec_off, I.n, A.qr32 + I.vec_off, A.dq32 + I.vec_off,
                                         A.lq32 + I.vec_off);
    ok = ok && cudaGetLastError() == cudaSuccess;
    rom_destroy(ctx);
    if (!ok) return fail(ROM_ECUDA);
    I.d = dv;
    I.dinv = 1.0 / dv;
  }
  B->d_inst = d_inst; B->d_ti = d_ti; B->d_r0 = d_r0; B->d_r1 = d_r1; B->d_order = d_order;
  B->d_qdesc = d_qdesc;
  std::vector<int> rank0(count, 1);
  {
    std::vector<int> ones(count, 1);
    if (cudaMemcpyAsync(A.need_jac, ones.data(), sizeof(int) * count, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(rank0.data(), A.rank, sizeof(int) * count, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(d_ci, cinst.data(), sizeof(int) * B->nchunks, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(d_cc, cc.data(), sizeof(int) * B->nchunks, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess ||
        set_tiles(B, kTileCandidates[0], rank0) != cudaSuccess)
      return fail(ROM_ECUDA);
  }
  // ---- cooperative grids ----
  int sms = 0, nb = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return fail(ROM_ECUDA);
  if (cudaFuncSetAttribute((const void*)batch_steps_kernel<kMaxR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sizeof(StepSmem)) != cudaSuccess ||
      cudaFuncSetAttribute((const void*)batch_steps_kernel<kLowRank>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sizeof(StepSmem)) != cudaSuccess ||
      cudaFuncSetAttribute((const void*)batch_sweep_kernel<kMaxR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sizeof(StepSmem)) != cudaSuccess ||
      cudaFuncSetAttribute((const void*)batch_sweep_kernel<kLowRank>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sizeof(StepSmem)) != cudaSuccess ||
      cudaFuncSetAttribute((const void*)batch_event_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)event_smem()) != cudaSuccess)
    return fail(ROM_ECUDA);
  int g1 = 0, g2 = 0, g3 = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (const void*)batch_steps_kernel<kMaxR>, kBT, sizeof(StepSmem)) != cudaSuccess) return fail(ROM_ECUDA);
  g1 = nb;
  int g4 = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g4, (const void*)batch_steps_kernel<kLowRank>, kBT, sizeof(StepSmem)) != cudaSuccess) return fail(ROM_ECUDA);
  if (g4 < 1) return fail(ROM_ECUDA);
  B->grid_lo = sms * g4;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (const void*)batch_event_kernel, kBT, event_smem()) != cudaSuccess) return fail(ROM_ECUDA);
  g2 = nb;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (const void*)batch_fom_kernel, kFomT, 0) != cudaSuccess) return fail(ROM_ECUDA);
  g3 = nb;
  if (g1 < 1 || g2 < 1 || g3 < 1) return fail(ROM_ECUDA);
  B->grid_sweep = sms * std::min(g1, g2);
  B->grid_fom = sms * g3;
  // every CTA of the FOM kernel keeps a table of its chunks in shared memory
  if ((B->nchunks + B->grid_fom - 1) / B->grid_fom > kFomItems) return fail(ROM_EINVAL);
  // tile autotuning: time a residual sweep over the actual bases for each
  // candidate tile size and keep the fastest
  {
    int best = kTileCandidates[0];
    float best_ms = 0.f;
    for (int c = 0; c < (int)(sizeof(kTileCandidates) / sizeof(int)); ++c) {
      float ms = 0.f;
      if (set_tiles(B, kTileCandidates[c], rank0) != cudaSuccess || time_dry_sweep(B, &ms) != cudaSuccess)
        return fail(ROM_ECUDA);
      B->tune_ms[c] = ms;
      if (c == 0 || ms < best_ms) { best = kTileCandidates[c]; best_ms = ms; }
    }
    if (set_tiles(B, best, rank0) != cudaSuccess) return fail(ROM_ECUDA);
  }
  *out = B;
  return ROM_OK;
}

rom_status rom_batch_step(rom_batch* B, int64_t n_steps) {
  if (!B || n_steps < 0) return ROM_EINVAL;
  if (B->poisoned) return ROM_ESTATE;
  while (n_steps > 0) {
    long long to_event = LLONG_MAX;
    for (int i = 0; i < B->count; ++i) {
      const long long z = B->hinst[i].z;
      to_event = std::min(to_event, z - (B->M % z));
    }
    // whole adaptation intervals replay one captured graph (not while the
    // per-phase timer is on)
    if (!B->prof_on && B->graph_state >= 0 && to_event <= n_steps) {
      if (B->graph_state == 0) {
        if (capture_interval(B, to_event) == cudaSuccess) {
          B->graph_state = 1;
          B->seg_len = to_event;
        } else {
          cudaGetLastError();
          B->graph_state = -1;
        }
      }
      if (B->graph_state == 1 && to_event == B->seg_len) {
        if (cudaGraphLaunch(B->seg_graph, B->stream) != cudaSuccess) {
          B->poisoned = 1;
          cudaGetLastError();
          return ROM_ECUDA;
        }
        B->M += to_event;
        n_steps -= to_event;
        continue;
      }
    }
    const long long seg = std::min<long long>(n_steps, to_event);
    if (run_steps(B, (int)seg) != cudaSuccess) { B->poisoned = 1; cudaGetLastError(); return ROM_ECUDA; }
    B->M += seg;
    n_steps -= seg;
    bool any = false;
    for (int i = 0; i < B->count && !any; ++i) any = (B->M % B->hinst[i].z) == 0;
    if (any && run_event(B) != cudaSuccess) { B->poisoned = 1; cudaGetLastError(); return ROM_ECUDA; }
  }
  rom_status st = batch_finish(B);
  if (st == ROM_OK && B->prof_on && prof_collect(B) != cudaSuccess) return ROM_ECUDA;
  return st;
}

rom_status rom_batch_state(rom_batch* B, int32_t i, double* q_tilde, double* a, double* sigma, double* phi,
                           double* y_corr, int64_t* step) {
  if (!B || i < 0 || i >= B->count) return ROM_EINVAL;
  if (B->poisoned) return ROM_ESTATE;
  const Inst& I = B->hinst[i];
  const size_t N = (size_t)I.n;
  cudaStream_t s = B->stream;
  int k = 0;
  BCK(cudaMemcpyAsync(&k, B->A.rank + i, sizeof(int), cudaMemcpyDeviceToHost, s));
  BCK(cudaStreamSynchronize(s));
  std::vector<double> ha(I.r);
  BCK(cudaMemcpyAsync(ha.data(), B->A.a + (size_t)i * kMaxR, sizeof(double) * I.r, cudaMemcpyDeviceToHost, s));
  if (q_tilde) {
    batch_lift_kernel<<<256, 256, 0, s>>>(B->A.phi + I.phi_off, B->A.q_ref + I.vec_off, B->A.a + (size_t)i * kMaxR,
                                          I.n, k, I.dinv, B->lift);
    BCK(cudaGetLastError());
    BCK(cudaMemcpyAsync(q_tilde, B->lift, sizeof(double) * N, cudaMemcpyDeviceToHost, s));
  }
  if (sigma) BCK(cudaMemcpyAsync(sigma, B->A.sigma + (size_t)i * kMaxR, sizeof(double) * I.r, cudaMemcpyDeviceToHost, s));
  std::vector<float> p32;
  if (phi) {
    p32.resize(N * I.r);
    BCK(cudaMemcpyAsync(p32.data(), B->A.phi + I.phi_off, sizeof(float) * N * I.r, cudaMemcpyDeviceToHost, s));
  }
  if (y_corr) BCK(cudaMemcpyAsync(y_corr, B->A.y_corr + I.vec_off, sizeof(double) * N, cudaMemcpyDeviceToHost, s));
  BCK(cudaStreamSynchronize(s));
  if (phi) {
    for (size_t e = 0; e < p32.size(); ++e) phi[e] = (double)p32[e];
    for (int j = 0; j < I.r; ++j) {   // sign convention: largest-magnitude entry positive
      double* col = phi + (size_t)j * N;
      size_t im = 0;
      double best = -1.0;
      for (size_t r = 0; r < N; ++r)
        if (fabs(col[r]) > best) { best = fabs(col[r]); im = r; }
      if (col[im] < 0.0) {
        for (size_t r = 0; r < N; ++r) col[r] = -col[r];
        ha[j] = -ha[j];
      }
    }
  }
  if (a) memcpy(a, ha.data(), sizeof(double) * I.r);
  if (step) *step = B->w_init[i] + B->M;
  return ROM_OK;
}

rom_status rom_batch_info(rom_batch* B, int32_t i, int32_t* rank, int32_t* rom_iters, int32_t* fom_iters) {
  if (!B || i < 0 || i >= B->count) return ROM_EINVAL;
  if (B->poisoned) return ROM_ESTATE;
  int v[3] = {0, 0, 0};
  BCK(cudaMemcpyAsync(&v[0], B->A.rank + i, sizeof(int), cudaMemcpyDeviceToHost, B->stream));
  BCK(cudaMemcpyAsync(&v[1], B->A.iters_rom + i, sizeof(int), cudaMemcpyDeviceToHost, B->stream));
  BCK(cudaMemcpyAsync(&v[2], B->A.iters_fom + i, sizeof(int), cudaMemcpyDeviceToHost, B->stream));
  BCK(cudaStreamSynchronize(B->stream));
  if (rank) *rank = v[0];
  if (rom_iters) *rom_iters = v[1];
  if (fom_iters) *fom_iters = v[2];
  return ROM_OK;
}

rom_status rom_batch_layout(rom_batch* B, int64_t* basis_bytes, int64_t* rows, int32_t* tiles,
                            int32_t* tile_rows, int32_t* grid, int32_t* graph) {
  if (!B) return ROM_EINVAL;
  if (graph) *graph = B->graph_state;
  if (tile_rows) *tile_rows = B->tile_rows;
  long long bb = 0, nr = 0;
  for (const Inst& I : B->hinst) {
    bb += (long long)I.n * I.r * (long long)sizeof(float);
    nr += I.n;
  }
  if (basis_bytes) *basis_bytes = bb;
  if (rows) *rows = nr;
  if (tiles) *tiles = B->ntiles;
  if (grid) *grid = B->grid_sweep;
  return ROM_OK;
}

rom_status rom_batch_profile(rom_batch* B, int32_t enable) {
  if (!B) return ROM_EINVAL;
  if (B->poisoned) return ROM_ESTATE;
  B->prof_on = enable ? 1 : 0;
  for (int p = 0; p < 3; ++p) { B->prof_ms[p] = 0.0; B->prof_cnt[p] = 0; }
  BCK(cudaMemsetAsync(B->A.sweeps, 0, sizeof(long long) * B->count, B->stream));
  BCK(cudaMemsetAsync(B->A.sweep_cols, 0, sizeof(long long) * B->count, B->stream));
  BCK(cudaMemsetAsync(B->A.fom_its, 0, sizeof(long long) * B->count, B->stream));
  BCK(cudaStreamSynchronize(B->stream));
  return ROM_OK;
}

rom_status rom_batch_fom_work(rom_batch* B, int64_t* row_iterations, double* fom_bytes) {
  if (!B) return ROM_EINVAL;
  if (B->poisoned) return ROM_ESTATE;
  std::vector<long long> it(B->count);
  BCK(cudaMemcpyAsync(it.data(), B->A.fom_its, sizeof(long long) * B->count, cudaMemcpyDeviceToHost,
                      B->stream));
  BCK(cudaStreamSynchronize(B->stream));
  long long rows = 0;
  for (int i = 0; i < B->count; ++i) rows += (long long)B->hinst[i].n * it[i];
  if (row_iterations) *row_iterations = rows;
  // a Newton iteration of backward Euler reads the iterate and the previous
  // state and writes the update: three FP64 words per row
  if (fom_bytes) *fom_bytes = 24.0 * (double)rows;
  return ROM_OK;
}

rom_status rom_batch_work(rom_batch* B, int64_t* newton_iters, double* sweep_bytes) {
  if (!B) return ROM_EINVAL;
  if (B->poisoned) return ROM_ESTATE;
  std::vector<long long> sw(B->count), sc(B->count);
  BCK(cudaMemcpyAsync(sw.data(), B->A.sweeps, sizeof(long long) * B->count, cudaMemcpyDeviceToHost, B->stream));
  BCK(cudaMemcpyAsync(sc.data(), B->A.sweep_cols, sizeof(long long) * B->count, cudaMemcpyDeviceToHost, B->stream));
  BCK(cudaStreamSynchronize(B->stream));
  long long it = 0;
  double by = 0.0;
  for (int i = 0; i < B->count; ++i) {
    const Inst& I = B->hinst[i];
    it += sw[i];
    // a sweep reads the k live FP32 basis columns (zero columns are not
    // read) and three FP32 words of q_ref data per row
    by += (double)I.n * (4.0 * (double)sc[i] + 12.0 * (double)sw[i]);
  }
  if (newton_iters) *newton_iters = it;
  if (sweep_bytes) *sweep_bytes = by;
  return ROM_OK;
}

rom_status rom_batch_profile_read(rom_batch* B, double* ms_total, int64_t* launches) {
  if (!B || !ms_total || !launches) return ROM_EINVAL;
  for (int p = 0; p < 3; ++p) { ms_total[p] = B->prof_ms[p]; launches[p] = B->prof_cnt[p]; }
  return ROM_OK;
}

void rom_batch_destroy(rom_batch* B) {
  if (!B) return;
  cudaStreamSynchronize(B->stream);
  batch_free(B);
  delete B;
}

}  // extern "C"
