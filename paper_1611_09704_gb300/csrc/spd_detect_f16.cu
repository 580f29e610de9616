// spd_detect_f16.cu -- detect kernels for f16 planes (one translation unit
// per storage type so that the instantiations compile in parallel).
#include "spd_detect_kernel.cuh"

namespace spd {
template cudaError_t launch_detect_dt<SPD_F16>(const Launch &, int, bool, bool, size_t, int,
                                          cudaStream_t);
}  // namespace spd
