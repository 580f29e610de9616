// spd_search_bf16.cu -- candidate search kernels for bf16 planes (one translation
// unit per storage type so that the instantiations compile in parallel).
#include "spd_search_kernel.cuh"

namespace spd {
template cudaError_t launch_search_dt<SPD_BF16>(const Launch &, int, bool, size_t, int, int,
                                                  cudaStream_t);
}  // namespace spd
