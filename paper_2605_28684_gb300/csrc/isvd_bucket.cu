// One rank bucket and basis type of the iSVD update and projection kernels
// (isvd_impl.cuh). The build compiles this file once per pair with
// -DROM_ISVD_KM=<KM> (9, 17, 33, 65) and -DROM_ISVD_F32=<0|1> (FP64 basis,
// or the FP32 basis of the mixed form).
#include "isvd_impl.cuh"

#if !defined(ROM_ISVD_KM) || !defined(ROM_ISVD_F32)
#error "compile with -DROM_ISVD_KM=9|17|33|65 -DROM_ISVD_F32=0|1"
#endif

#define ROM_PASTE3(a, b, c) a##b##c
#define ROM_NAME(a, b, c) ROM_PASTE3(a, b, c)
#if ROM_ISVD_F32
#define ROM_ISVD_T float
#define ROM_ISVD_SFX _f32
#else
#define ROM_ISVD_T double
#define ROM_ISVD_SFX _f64
#endif

namespace rom {

cudaError_t ROM_NAME(launch_event_b, ROM_ISVD_KM, ROM_ISVD_SFX)(const EventArgs& A, int grid,
                                                                cudaStream_t s) {
  return launch_event_tt<ROM_ISVD_KM, ROM_ISVD_T>(A, grid, s);
}

cudaError_t ROM_NAME(launch_project_b, ROM_ISVD_KM, ROM_ISVD_SFX)(const ProjectArgs& A, int grid,
                                                                  cudaStream_t s) {
  return launch_project_tt<ROM_ISVD_KM, ROM_ISVD_T>(A, grid, s);
}

cudaError_t ROM_NAME(set_wait_limit_isvd_b, ROM_ISVD_KM, ROM_ISVD_SFX)(long long cycles) {
  return set_wait_limit_here(cycles);
}

}  // namespace rom
