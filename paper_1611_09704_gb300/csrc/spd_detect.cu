// spd_detect.cu -- dispatch by storage type of the detect kernels: plane
// output (spd_detect_kernel.cuh) and the candidate search
// (spd_search_kernel.cuh).
#include "spd_internal.cuh"

namespace spd {

template <int DT>
cudaError_t launch_detect_dt(const Launch &L, int G, bool plane_out, bool multi_block,
                             size_t smem, int ctas_per_sm, cudaStream_t s);

cudaError_t launch_detect(const Launch &L, int dtype, int G, bool plane_out, bool multi_block,
                          size_t smem, int ctas_per_sm, cudaStream_t s) {
    if (L.n_tiles <= 0) return cudaSuccess;
    switch (dtype) {
        case SPD_F32: return launch_detect_dt<SPD_F32>(L, G, plane_out, multi_block, smem, ctas_per_sm, s);
        case SPD_F16: return launch_detect_dt<SPD_F16>(L, G, plane_out, multi_block, smem, ctas_per_sm, s);
        default: return launch_detect_dt<SPD_BF16>(L, G, plane_out, multi_block, smem, ctas_per_sm, s);
    }
}

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
