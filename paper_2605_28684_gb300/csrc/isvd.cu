// Dispatch of the iSVD update and projection kernels (isvd_impl.cuh) to the
// objects that instantiate them, one per rank bucket (isvd_bucket.cu).
#include "isvd_impl.cuh"

namespace rom {

#define ROM_ISVD_DECLARE(KM, SFX)                                                            \
  cudaError_t launch_event_b##KM##SFX(const EventArgs& A, int grid, cudaStream_t s);       \
  cudaError_t launch_project_b##KM##SFX(const ProjectArgs& A, int grid, cudaStream_t s);   \
  cudaError_t set_wait_limit_isvd_b##KM##SFX(long long cycles);
#define ROM_ISVD_DECLARE_BOTH(KM) ROM_ISVD_DECLARE(KM, _f64) ROM_ISVD_DECLARE(KM, _f32)
ROM_ISVD_DECLARE_BOTH(9)
ROM_ISVD_DECLARE_BOTH(17)
ROM_ISVD_DECLARE_BOTH(33)
ROM_ISVD_DECLARE_BOTH(65)
#undef ROM_ISVD_DECLARE_BOTH
#undef ROM_ISVD_DECLARE

// The FP32 basis of the mixed form selects the f32 objects.
#define ROM_ISVD_PICK(fn, KM, A) ((A).phi32 ? fn##KM##_f32 : fn##KM##_f64)

size_t event_smem_bytes() { return sizeof(EventSmem); }
size_t core_ws_doubles() { return kWsSize; }
size_t core_sbar_offset() { return kWsSbar; }

cudaError_t launch_event(const EventArgs& A, int km, int grid, cudaStream_t s) {
  switch (km) {
    case 9: return ROM_ISVD_PICK(launch_event_b, 9, A)(A, grid, s);
    case 17: return ROM_ISVD_PICK(launch_event_b, 17, A)(A, grid, s);
    case 33: return ROM_ISVD_PICK(launch_event_b, 33, A)(A, grid, s);
    default: return ROM_ISVD_PICK(launch_event_b, 65, A)(A, grid, s);
  }
}

cudaError_t launch_project(const ProjectArgs& A, int km, int grid, cudaStream_t s) {
  switch (km) {
    case 9: return ROM_ISVD_PICK(launch_project_b, 9, A)(A, grid, s);
    case 17: return ROM_ISVD_PICK(launch_project_b, 17, A)(A, grid, s);
    case 33: return ROM_ISVD_PICK(launch_project_b, 33, A)(A, grid, s);
    default: return ROM_ISVD_PICK(launch_project_b, 65, A)(A, grid, s);
  }
}

int km_bucket(int kplus1) {
  if (kplus1 <= 9) return 9;
  if (kplus1 <= 17) return 17;
  if (kplus1 <= 33) return 33;
  return 65;
}

// Wait bound of the iSVD kernels: every bucket object holds its own copy.
cudaError_t set_wait_limit_isvd(long long cycles) {
  cudaError_t (*setters[])(long long) = {
      set_wait_limit_isvd_b9_f64,  set_wait_limit_isvd_b9_f32,  set_wait_limit_isvd_b17_f64,
      set_wait_limit_isvd_b17_f32, set_wait_limit_isvd_b33_f64, set_wait_limit_isvd_b33_f32,
      set_wait_limit_isvd_b65_f64, set_wait_limit_isvd_b65_f32};
  for (auto f : setters) {
    cudaError_t e = f(cycles);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace rom
