// spd_dedisperse.cu -- incoherent de-dispersion: the DM x time plane the
// detector searches (Sec. 1), made from a filterbank of channel rows by
// summing each channel shifted by its dispersion delay for every DM trial.
// A producer for the streaming search: it can write DM trials straight into
// a push workspace's chunk view, so the search reads them in place (the
// coupling Sec. 3 names as future work).
#include "spd_internal.cuh"

namespace spd {
void note_cuda_error(int e);
}

using namespace spd;

namespace {

constexpr int kDdThreads = 256;
constexpr int kDdPer = 4;                      // outputs per thread
constexpr int kDdSpan = kDdThreads * kDdPer;   // outputs per CTA

template <int DT>
__device__ __forceinline__ float fb_value(const typename Elem<DT>::T *p, bool has_sc, float sc,
                                          float of) {
    const float x = Elem<DT>::cvt(*p);
    return has_sc ? fmaf(sc, x, of) : x;
}

__device__ __forceinline__ void store_out(void *out, int dt, int64_t idx, float v) {
    if (dt == SPD_F32) static_cast<float *>(out)[idx] = v;
    else if (dt == SPD_F16) static_cast<__half *>(out)[idx] = __float2half_rn(v);
    else static_cast<__nv_bfloat16 *>(out)[idx] = __float2bfloat16_rn(v);
}

// One CTA: kDdSpan consecutive outputs of one DM trial (grid.y walks the DM
// trials).  Thread t sums outputs t0 + t + 256 j, j < 4: at every channel the
// warp reads consecutive samples, and the channel's delay is one broadcast.
template <int DT>
__global__ void __launch_bounds__(kDdThreads) dedisperse_kernel(
    const typename Elem<DT>::T *fb, int64_t n_chan, int64_t n_samp, int64_t fb_stride,
    const float *scale, const float *offset, const int32_t *delays, int64_t n_dm, void *out,
    int out_dt, int64_t n_out, int64_t out_stride, spd_result *status) {
    using T = typename Elem<DT>::T;
    const int64_t t0 = (int64_t)blockIdx.x * kDdSpan + threadIdx.x;
    const int64_t max_delay = n_samp - n_out;
    const bool has_sc = scale != nullptr;
    for (int64_t d = blockIdx.y; d < n_dm; d += gridDim.y) {
        const int32_t *dl = delays + d * n_chan;
        float acc[kDdPer];
#pragma unroll
        for (int j = 0; j < kDdPer; ++j) acc[j] = 0.f;
        bool bad = false;
        for (int64_t c = 0; c < n_chan; ++c) {
            const int64_t dc = __ldg(dl + c);
            if (dc < 0 || dc > max_delay) {   // no read outside the row
                bad = true;
#pragma unroll
                for (int j = 0; j < kDdPer; ++j) acc[j] = __int_as_float(0x7fc00000);
                continue;
            }
            const float sc = has_sc ? __ldg(scale + c) : 1.f;
            const float of = (has_sc && offset) ? __ldg(offset + c) : 0.f;
            const T *row = fb + c * fb_stride + dc;
#pragma unroll
            for (int j = 0; j < kDdPer; ++j) {
                const int64_t t = t0 + (int64_t)kDdThreads * j;
                if (t < n_out) acc[j] = __fadd_rn(acc[j], fb_value<DT>(row + t, has_sc, sc, of));
            }
        }
        if (bad && status && threadIdx.x == 0 && blockIdx.x == 0)
            atomicExch(&status->status, (int)SPD_ERR_INVALID_ARG);
#pragma unroll
        for (int j = 0; j < kDdPer; ++j) {
            const int64_t t = t0 + (int64_t)kDdThreads * j;
            if (t < n_out) store_out(out, out_dt, d * out_stride + t, acc[j]);
        }
    }
}

}  // namespace

extern "C" spd_status spd_dedisperse(const spd_plane *fb, const int32_t *delays, int64_t n_dm,
                                     void *out, int32_t out_dtype, int64_t n_out,
                                     int64_t out_stride, spd_result *status_dev, void *stream) {
    if (!fb || fb->dtype < SPD_F32 || fb->dtype > SPD_BF16) return SPD_ERR_INVALID_ARG;
    if (out_dtype < SPD_F32 || out_dtype > SPD_BF16) return SPD_ERR_INVALID_ARG;
    const int64_t n_chan = fb->n_dm, n_samp = fb->n_samp;
    if (n_chan < 0 || n_samp < 0 || n_dm < 0 || n_out < 0 || n_out > n_samp) return SPD_ERR_INVALID_ARG;
    if (n_dm == 0 || n_out == 0) return SPD_OK;
    if (n_chan == 0 || !fb->data || fb->row_stride < n_samp || !delays || !out ||
        out_stride < n_out)
        return SPD_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(fb->data) % elem_bytes(fb->dtype) ||
        reinterpret_cast<uintptr_t>(out) % elem_bytes(out_dtype) ||
        reinterpret_cast<uintptr_t>(delays) % 4)
        return SPD_ERR_INVALID_ARG;
    if (fb->row_offset && !fb->row_scale) return SPD_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t gx = (n_out + kDdSpan - 1) / kDdSpan;
    if (gx > INT32_MAX) return SPD_ERR_INVALID_ARG;
    const dim3 grid((unsigned)gx, (unsigned)(n_dm < 65535 ? n_dm : 65535));
    switch (fb->dtype) {
        case SPD_F32:
            dedisperse_kernel<SPD_F32><<<grid, kDdThreads, 0, st>>>(
                static_cast<const float *>(fb->data), n_chan, n_samp, fb->row_stride,
                fb->row_scale, fb->row_offset, delays, n_dm, out, out_dtype, n_out, out_stride,
                status_dev);
            break;
        case SPD_F16:
            dedisperse_kernel<SPD_F16><<<grid, kDdThreads, 0, st>>>(
                static_cast<const __half *>(fb->data), n_chan, n_samp, fb->row_stride,
                fb->row_scale, fb->row_offset, delays, n_dm, out, out_dtype, n_out, out_stride,
                status_dev);
            break;
        default:
            dedisperse_kernel<SPD_BF16><<<grid, kDdThreads, 0, st>>>(
                static_cast<const __nv_bfloat16 *>(fb->data), n_chan, n_samp, fb->row_stride,
                fb->row_scale, fb->row_offset, delays, n_dm, out, out_dtype, n_out, out_stride,
                status_dev);
            break;
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        note_cuda_error((int)e);
        return SPD_ERR_CUDA;
    }
    return SPD_OK;
}
