// spd_detect.cu -- dispatch by storage type of the search kernel
// (spd_search_kernel.cuh): candidate search and plane output.
#include "spd_internal.cuh"

namespace spd {

template <int DT>
cudaError_t launch_search_dt(const Launch &L, int G, bool multi_block, size_t smem,
                             int ctas_per_sm, int threads, cudaStream_t s);

cudaError_t launch_search(const Launch &L, int dtype, int G, bool multi_block, size_t smem,
                          int ctas_per_sm, int threads, cudaStream_t s) {
    if (L.n_tiles <= 0) return cudaSuccess;
    switch (dtype) {
        case SPD_F32:
            return launch_search_dt<SPD_F32>(L, G, multi_block, smem, ctas_per_sm, threads, s);
        case SPD_F16:
            return launch_search_dt<SPD_F16>(L, G, multi_block, smem, ctas_per_sm, threads, s);
        default:
            return launch_search_dt<SPD_BF16>(L, G, multi_block, smem, ctas_per_sm, threads, s);
    }
}

}  // namespace spd
