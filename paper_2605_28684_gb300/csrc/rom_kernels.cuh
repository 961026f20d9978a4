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
  double* partials;     // 2 * grid * (KM + 2)
  float* jpartials;     // grid * kMaxR * kMaxR
  float* jac;           // kMaxR * kMaxR
  // hyper-reduction
  int n_s;
  const int* samples;
  const double* mesh;   // n_s x 3 x (kMaxR + 2): Phi rows (k), then q_ref, d
  const double* minv;   // k x n_s row-major
  GridBarrier* bar;
  int* status;
  int* iters;           // Newton iterations of the last step
};

cudaError_t launch_galerkin_steps(const StepArgs& A, int km, int grid, cudaStream_t s);
cudaError_t launch_euler_galerkin_steps(const StepArgs& A, int km, int grid, cudaStream_t s);
cudaError_t launch_hyper_steps(const StepArgs& A, int km, cudaStream_t s);

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
  const int* rank;
  const double* phi;
  const float* phi32;
  const double* y;      // correction snapshot (feature-guided points)
  const double* q_ref;
  const double* drow;
  int* samples;
  int* chosen;          // n flags
  double* resid;        // n
  double* cand_v;       // grid * kMaxNs
  int* cand_i;          // grid * kMaxNs
  double* qdir;         // kMaxR * kMaxR
  double* mesh;         // n_s x 3 x (kMaxR + 2)
  double* minv;         // r x n_s
  GridBarrier* bar;
  int* status;
};
cudaError_t launch_sampling(const SampleArgs& A, int km, int grid, cudaStream_t s);

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
