// spd_detect_f32.cu -- detect kernels for f32 planes (one translation unit
// per storage type so that the instantiations compile in parallel).
#include "spd_detect_kernel.cuh"

namespace spd {
template cudaError_t launch_detect_dt<SPD_F32>(const Launch &, int, bool, bool, size_t, int,
                                          cudaStream_t);
}  // namespace spd
