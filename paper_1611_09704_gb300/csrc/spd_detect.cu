// spd_detect.cu -- dispatch of the fused detect kernel by storage type; the
// kernel itself is in spd_detect_kernel.cuh.
#include "spd_internal.cuh"

namespace spd {

template <int DT>
cudaError_t launch_detect_dt(const DetectArgs &a, const Program &prog, bool plane_out,
                             size_t smem, cudaStream_t s);

cudaError_t launch_detect(const DetectArgs &a, const Program &prog, int dtype, bool plane_out,
                          size_t smem, cudaStream_t s) {
    if (a.n_dm * a.tiles_per_row <= 0) return cudaSuccess;
    switch (dtype) {
        case SPD_F32: return launch_detect_dt<SPD_F32>(a, prog, plane_out, smem, s);
        case SPD_F16: return launch_detect_dt<SPD_F16>(a, prog, plane_out, smem, s);
        default: return launch_detect_dt<SPD_BF16>(a, prog, plane_out, smem, s);
    }
}

}  // namespace spd
