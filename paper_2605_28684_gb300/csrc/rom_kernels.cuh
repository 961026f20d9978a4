// Argument blocks and launchers of the librom kernels (internal).
#pragma once

#include "rom_internal.cuh"

namespace rom {

// iSVD update (isvd.cu).
struct EventArgs {
  int64_t n, ld;
  int r;
  int* rank;
  double lambda, rank_tol;
  double* phi;
  float* phi32;         // FP32 basis (mixed precision); null in the FP64 form
  double* gram;         // mixed precision: grid * kMaxR * kMaxR Gram partial sums
  double* sigma;
  double* a;            // reduced state to transfer (may be null)
  int transfer;
  const double* y;      // raw snapshot (preprocess = 1) or preprocessed
  const double* q_ref;
  const double* drow;
  int preprocess;
  double* yhat;
  double* qres;
  double* partials;     // >= 3 * grid * (KM + 2)
  double* core;         // core_ws_doubles()
  double* ubar;         // (r+1)^2
  double* rec;          // null, or receives (rho, ||yhat||, p_0 .. p_{k-1}) of the core
                        // (rho = 0 for an empty residual), for the gradient pass
  GridBarrier* bar;
  int* status;
};

struct ProjectArgs {
  int64_t n, ld;
  int r;
  const int* rank;
  const double* phi;
  const float* phi32;
  const double* v;
  const double* q_ref;
  const double* drow;
  double* a;
  double* partials;
  GridBarrier* bar;
  int* status;
};

cudaError_t launch_event(const EventArgs& A, int km, int grid, cudaStream_t s);
cudaError_t launch_project(const ProjectArgs& A, int km, int grid, cudaStream_t s);
size_t event_smem_bytes();
size_t core_ws_doubles();
int km_bucket(int kplus1);

// Reduced steps (reduced.cu).
struct StepArgs {
  int64_t n, ld;
  int r;
  const int* rank;
  const double* phi;
  const float* phi32;
  const double* q_ref;
  const double* drow;
  const double* dinv;
  double* a;
  double nu, gamma, dt, tol;
  int max_iter;
  int nsteps;
  int explicit_rk;      // 1: SSPRK(4,3) stages instead of backward-Euler Newton (App. D)
  double* partials;     // 2 * grid * (KM + 2)
  float* jpartials;     // grid * kMaxR * kMaxR
  float* jac;           // kMaxR * kMaxR
  // hyper-reduction
  int n_s;
  const int* samples;
  const double* mesh;   // n_s x 3 n_var x (kMaxR + 2): Phi rows (k), then q_ref, d
  const double* minv;   // k x n_s row-major
  double* npart;        // LSPG: lspg_partial_doubles(grid) partial sums
  GridBarrier* bar;
  int* status;
  int* iters;           // Newton iterations of the last step
};

cudaError_t launch_galerkin_steps(const StepArgs& A, int km, int grid, cudaStream_t s);
cudaError_t launch_euler_galerkin_steps(const StepArgs& A, int km, int grid, cudaStream_t s);
cudaError_t launch_hyper_steps(const StepArgs& A, int km, cudaStream_t s);
// DEIM-Galerkin steps of the Euler system, explicit form (euler.cu), and the
// shared memory they stage (n_s samples of nine mesh rows, rank <= r)
cudaError_t launch_euler_hyper_steps(const StepArgs& A, cudaStream_t s);
size_t euler_hyper_smem(int n_s, int r);
// LSPG steps (lspg.cu), FP64 Burgers, n_s = 0
cudaError_t launch_lspg_steps(const StepArgs& A, int grid, cudaStream_t s);
size_t lspg_partial_doubles(int grid);

struct LiftArgs {
  int64_t n, ld;
  const int* rank;
  const double* phi;
  const float* phi32;
  const double* q_ref;
  const double* drow;
  const double* dinv;
  const double* a;
  double* out;
};
cudaError_t launch_lift(const LiftArgs& A, int km, cudaStream_t s);

// Sampling (sampling.cu).
struct SampleArgs {
  int64_t n, ld;
  int r, n_s;
  int n_var;            // 1 (Burgers: rows are cells) or 3 (Euler: variable-blocked rows)
  const int* rank;
  const double* phi;
  const float* phi32;
  const double* q_ref;
  const double* drow;
  const int* fgs_i;     // feature-guided candidates, best first (launch_fgs)
  int fgs_t;            // their number (>= fgs_list_length(n, r, n_s))
  int* samples;
  double* cand_v;       // grid * 2: per-CTA QDEIM candidate values (two step parities)
  unsigned long long* cand_f;  // grid * 2: (epoch << 32 | index) of those candidates
  unsigned int epoch;   // first step epoch of this launch (the caller advances it by kMaxR per launch)
  double* qd_u;         // n x r: coordinates of the rows along the QDEIM residual directions
  double* mesh;         // n_s x 3 n_var x (kMaxR + 2)
  double* minv;         // r x n_s
  GridBarrier* bar;
  int* status;
};
cudaError_t launch_sampling(const SampleArgs& A, int km, int grid, cudaStream_t s);
// Length of the feature-guided candidate list: n_s + min(r, n_s) (at most n).
int fgs_list_length(int64_t n, int r, int n_s);
// The fgs_list_length best feature-guided candidates of the snapshot y of n
// rows (fgs_key_kernel or fgs_key_euler_kernel, then fgs_select_kernel):
// values out_v, row indices out_i, best first; key is n words of scratch.
// n_var 1: the feature is y itself; n_var 3: the cell pressures (gamma).
// stage: copy the keys to shared memory first (when they fit); otherwise
// they are read from global memory.
cudaError_t launch_fgs(const double* y, int64_t n, int n_var, double gamma, int T, unsigned long long* key,
                       double* out_v, int* out_i, bool stage, cudaStream_t s);

constexpr int kMeshStride = kMaxR + 2;   // per stencil row: k basis entries, q_ref, d

// Basis pointer of the storage type a kernel instance was compiled for.
template <typename TPhi, typename Args>
__device__ __forceinline__ const TPhi* basis(const Args& A);
template <>
__device__ __forceinline__ const double* basis<double>(const EventArgs& A) { return A.phi; }
template <>
__device__ __forceinline__ const float* basis<float>(const EventArgs& A) { return A.phi32; }
template <>
__device__ __forceinline__ const double* basis<double>(const ProjectArgs& A) { return A.phi; }
template <>
__device__ __forceinline__ const float* basis<float>(const ProjectArgs& A) { return A.phi32; }
template <>
__device__ __forceinline__ const double* basis<double>(const StepArgs& A) { return A.phi; }
template <>
__device__ __forceinline__ const float* basis<float>(const StepArgs& A) { return A.phi32; }
template <>
__device__ __forceinline__ const double* basis<double>(const LiftArgs& A) { return A.phi; }
template <>
__device__ __forceinline__ const float* basis<float>(const LiftArgs& A) { return A.phi32; }
template <>
__device__ __forceinline__ const double* basis<double>(const SampleArgs& A) { return A.phi; }
template <>
__device__ __forceinline__ const float* basis<float>(const SampleArgs& A) { return A.phi32; }

}  // namespace rom

// ---------------------------------------------------------------------------
// Gradient pass (adjoint.cu): reverse sweep of the plain-Galerkin Burgers ROM
// in FP64. All matrices are column-major with the leading dimension given;
// small results of reductions are row-major m x nc.
// ---------------------------------------------------------------------------
namespace rom {

constexpr int kAdjSlots = 256;   // per-CTA accumulator slots of the scalar adjoints

// Adjoint of one reduced backward-Euler step with no event (three launches:
// Jacobian partials, one-CTA transposed solve, row pass).
struct AdjStepArgs {
  int64_t n;
  int k;                  // live rank of the basis in effect
  const double* phi;      // N x k, leading dimension n
  const double* q_ref;
  double d, nu, dt;
  const double* a;        // k: the step's root a^{n+1}
  double* w;              // k: adjoint of the step's residual (written)
  double* abar;           // k: adjoint of a; in: after the step, out: before it
  double* qtbar;          // N: adjoint at the step's lifted state (read, then zeroed)
  double* phibar;         // N x k, accumulated
  double* qrefbar;        // N, accumulated
  double* mpart;          // grid x kMaxR^2 partial sums
  double* vpart;          // grid x kMaxR partial sums
  double* acc;            // [0, kAdjSlots): d-bar slots; [kAdjSlots, 2 kAdjSlots): nu-bar slots
};
cudaError_t launch_adj_step(const AdjStepArgs& A, int grid, cudaStream_t s);

// x = (I - h J_f(y))^{-T} (rhs1 + rhs2) for periodic Burgers (FP64, chunked
// PCR); acc_nu[cta] += h x . f_nu(y).
struct TbeArgs {
  const double* y;
  const double* rhs1;
  const double* rhs2;     // may be null
  double* x;
  int64_t n;
  double nu, h;
  double* chunk;          // kMaxChunks * 16 doubles
  GridBarrier* bar;
  int* status;
  double* acc_nu;         // kAdjSlots slots
};
cudaError_t launch_adj_tbe(const TbeArgs& A, cudaStream_t s);

// out (m x nc, row-major) = alpha A^T B over N rows (m, nc <= 128, m*nc <= 16384);
// part holds grid * m * nc doubles.
struct TnArgs {
  int64_t n;
  int m, nc;
  const double* A;
  int64_t lda;
  const double* B;
  int64_t ldb;
  double alpha;
  double* part;
  double* out;
};
cudaError_t launch_tn(const TnArgs& A, int grid, cudaStream_t s);

// C = beta Cin + alpha A M over N rows; A is N x m, M(j, l) = M[j * msj + l * msl]
// (device, m x nc with m, nc <= 128, m * nc <= 16384); C may alias Cin.
struct NnArgs {
  int64_t n;
  int m, nc;
  const double* A;
  int64_t lda;
  const double* M;
  int64_t msj, msl;
  double alpha, beta;
  const double* Cin;
  int64_t ldcin;
  double* C;
  int64_t ldc;
};
cudaError_t launch_nn(const NnArgs& A, cudaStream_t s);

// Event pieces (rows of the iSVD adjoint and of the state transfer).
struct AdjEventArgs {
  int64_t n;
  int k, kn, r;           // rank before and after the event; capacity
  double* B;              // N x (k+1): Phi_old, then qhat in column k (finalised from column r)
  const double* phinew;   // N x kn
  const double* a;        // k: the step's root in the old basis
  const double* q_ref;
  double d, lambda;
  const double* abar;     // kn
  const double* phibar;   // N x kn
  double* pnb;            // N x kn work
  double* bbar;           // N x (k+1) work
  const double* yhat;
  const double* ynew;
  const double* ybar;     // N in
  double* ybar_new;       // N out
  double* phibar_out;     // N x k out
  double* qtbar;
  double* qrefbar;
  const double* ubar;     // (k+1)^2 column-major
  const double* sbar;     // k+1
  const double* sigma_old;
  const double* rec;      // rho, ||yhat||, p (k)
  double* small;          // device work for the small matrices (kAdjSmall doubles)
  double* sigbar;         // r: in sigma_new-bar (kn), out sigma_old-bar (k)
  double* part;           // partials for launch_tn
  double* acc;
};
constexpr int kAdjSmall = 12 * kMaxCore * kMaxCore;
cudaError_t launch_adj_event(const AdjEventArgs& A, int grid, cudaStream_t s);

// Offline stage: the a0 transfer rows, the POD adjoint and the reversed
// training trajectory are driven from api.cu through these pieces.
struct AdjA0Args {
  int64_t n;
  int k;
  const double* phi;      // N x k (POD basis)
  const double* qlast;
  const double* q_ref;
  double d;
  const double* abar;     // k
  double* phibar;         // N x k (accumulated)
  double* qlastbar;       // N (accumulated)
  double* qrefbar;
  double* acc;
};
cudaError_t launch_adj_a0(const AdjA0Args& A, int grid, cudaStream_t s);
// small dense pieces of the POD adjoint over all w triplets (see adjoint.cu)
struct AdjPodArgs {
  int64_t n;
  int w, k;
  const double* s;        // w singular values, descending
  const double* sbar;     // k
  const double* A;        // w x k row-major: U^T Ubar
  const double* V;        // w x w row-major: right singular vectors (columns)
  double* B1;             // w x w row-major out
  double* B2;             // k x w row-major out
};
cudaError_t launch_adj_pod_full(const AdjPodArgs& A, cudaStream_t s);
// Qbar from Xbar (two passes around the reduction of d-bar), see adjoint.cu
struct AdjXcArgs {
  int64_t n;
  int w;
  const double* Q;
  const double* q_ref;
  double d;
  const double* Xbar;     // N x w
  double* Qbar;           // N x w out
  const double* qlastbar;
  double* qrefbar;
  double* acc;            // d-bar slots (pass 1 adds sum Xbar o Xc)
  double* dtot;           // device scalar: total d-bar (written between the passes)
};
cudaError_t launch_adj_xc(const AdjXcArgs& A, int grid, cudaStream_t s);
// sum of the kAdjSlots slots at acc (fixed order) into *out (+ *out if add)
cudaError_t launch_adj_sum_slots(const double* acc, double* out, int add, cudaStream_t s);
// M = -(A + A^T) / 2 for a k x k row-major A (one CTA)
cudaError_t launch_adj_neg_sym(const double* Am, double* M, int k, cudaStream_t s);
// y = a + b (N)
cudaError_t launch_adj_add(int64_t n, const double* a, const double* b, double* y, cudaStream_t s);
// lift q = q_ref + Phi a / d (N)
cudaError_t launch_adj_lift(int64_t n, int k, const double* phi, const double* a, const double* q_ref,
                            double d, double* q, cudaStream_t s);
// J = 1/2 |q - target|^2 and qtbar = q - target
cudaError_t launch_adj_misfit(int64_t n, const double* q, const double* target, double* qtbar,
                              double* part, double* J, cudaStream_t s);
size_t core_sbar_offset();
// thin SVD of an N x w matrix (w <= 128) by CGS2 QR and one-sided Jacobi on R
// (pod_svd.cu): U (w x w row-major) and s (w, descending) of R; Q (N x w) the
// orthonormal factor; work >= 256 doubles; part as launch_tn's. With V and
// Vwork (w x w each) non-null, V (row-major) gets the right singular vectors
// from the accumulated rotations; U and s do not depend on it.
cudaError_t pod_thin_svd(const double* X, int64_t n, int w, double* Q, double* R, double* U, double* s,
                         double* work, double* part, int grid, cudaStream_t st, double* V = nullptr,
                         double* Vwork = nullptr);
// comparison update rules (update_rules.cu)
cudaError_t launch_win_fill(const double* Q, int64_t ldq, const double* q_ref, const double* drow, int64_t n,
                            int count, double* win, cudaStream_t s);
cudaError_t launch_truncate(double* phi, int64_t n, double* sigma, int* rank, int r, int ncols, double tol,
                            cudaStream_t s);
cudaError_t launch_direct_small(const double* C, int r, int w, const int* rank, double tol, double* Vc,
                                double* s_out, int* kc, cudaStream_t s);
cudaError_t launch_set_sigma(const double* s_in, const int* kc, double* sigma, int* rank, cudaStream_t s);
// Instantaneous rules (one-step, Oja, GROUSE): coefficients of the rank-one
// update, the update itself, and the inverse Cholesky factor of a Gram matrix.
cudaError_t launch_instant_coef(int rule, const int* rank, int r, double eta, const double* w1, const double* w2,
                                const double* a, const double* rr, double* coef, double* g, double* v,
                                cudaStream_t s);
cudaError_t launch_rank1_update(double* phi, int64_t n, const int* rank, int r, const double* yhat,
                                const double* res, const double* coef, const double* g, const double* v,
                                cudaStream_t s);
cudaError_t launch_chol_inv(const double* G, const int* rank, int r, double* Rinv, cudaStream_t s);

}  // namespace rom
