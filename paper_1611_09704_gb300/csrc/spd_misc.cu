// spd_misc.cu -- step (d) on a stored SNR plane (Sec. 2.4) and the raw boxcar
// sums test aid.
#include "spd_internal.cuh"

#include <math.h>

namespace spd {

namespace {

constexpr int kThrThreads = 256;
constexpr int kThrPer = 8;                        // samples per thread
constexpr int kThrTile = kThrThreads * kThrPer;   // samples per CTA

// Every (dm, t) with snr >= thr becomes a record.  One atomicAdd per CTA on
// the global count (block-aggregated); records past `capacity` are counted
// but not written.
__global__ void __launch_bounds__(kThrThreads) threshold_kernel(
    const float *snr, const uint16_t *width, int64_t n_samp, int64_t stride,
    int64_t tiles_per_row, float thr, spd_candidate *out, int64_t capacity,
    spd_result *result) {
    __shared__ int s_wsum[kThrThreads / 32];
    __shared__ unsigned long long s_base;
    const int tid = threadIdx.x;
    const int64_t row = blockIdx.x / tiles_per_row;
    const int64_t t0 = (blockIdx.x - row * tiles_per_row) * (int64_t)kThrTile;
    const int64_t i0 = t0 + (int64_t)tid * kThrPer;
    const float *sp = snr + row * stride;
    const uint16_t *wp = width + row * stride;

    float v[kThrPer];
    int w[kThrPer];
    const bool vec = i0 + kThrPer <= n_samp &&
                     ((reinterpret_cast<uintptr_t>(sp + i0) & 15) == 0) &&
                     ((reinterpret_cast<uintptr_t>(wp + i0) & 15) == 0);
    if (vec) {
        const float4 a = __ldcs(reinterpret_cast<const float4 *>(sp + i0));
        const float4 b = __ldcs(reinterpret_cast<const float4 *>(sp + i0) + 1);
        const uint4 u = __ldcs(reinterpret_cast<const uint4 *>(wp + i0));
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
        w[0] = u.x & 0xffff; w[1] = u.x >> 16; w[2] = u.y & 0xffff; w[3] = u.y >> 16;
        w[4] = u.z & 0xffff; w[5] = u.z >> 16; w[6] = u.w & 0xffff; w[7] = u.w >> 16;
    } else {
#pragma unroll
        for (int k = 0; k < kThrPer; ++k) {
            const bool ok = i0 + k < n_samp;
            v[k] = ok ? sp[i0 + k] : -INFINITY;
            w[k] = ok ? wp[i0 + k] : 0;
        }
    }
    uint32_t mask = 0;
#pragma unroll
    for (int k = 0; k < kThrPer; ++k)
        if (i0 + k < n_samp && v[k] >= thr) mask |= 1u << k;
    const int cnt = __popc(mask);
    const int lane = tid & 31, warp = tid >> 5;
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int x = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += x;
    }
    if (lane == 31) s_wsum[warp] = incl;
    __syncthreads();
    if (tid < 32) {
        const int wv = (lane < kThrThreads / 32) ? s_wsum[lane] : 0;
        int wi = wv;
#pragma unroll
        for (int o = 1; o < kThrThreads / 32; o <<= 1) {
            const int x = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += x;
        }
        if (lane < kThrThreads / 32) s_wsum[lane] = wi - wv;
        const int total = __shfl_sync(0xffffffffu, wi, kThrThreads / 32 - 1);
        if (lane == 0)
            s_base = total ? atomicAdd(reinterpret_cast<unsigned long long *>(&result->count),
                                       (unsigned long long)total)
                           : 0ull;
    }
    __syncthreads();
    if (cnt) {
        unsigned long long idx = s_base + (unsigned long long)(s_wsum[warp] + incl - cnt);
#pragma unroll
        for (int k = 0; k < kThrPer; ++k) {
            if (mask & (1u << k)) {
                if (idx < (unsigned long long)capacity) {
                    int4 rec;
                    rec.x = (int)row;
                    rec.y = (int)(i0 + k);
                    rec.z = __float_as_int(v[k]);
                    rec.w = w[k];
                    reinterpret_cast<int4 *>(out)[idx] = rec;
                }
                ++idx;
            }
        }
    }
}

// Raw boxcar sum of one width per output sample, compensated FP32 summation.
template <int DT>
__global__ void boxcar_sums_kernel(const spd_plane p, int w, float *out, int64_t out_stride) {
    using T = typename Elem<DT>::T;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t r = blockIdx.y;
    if (i >= p.n_samp) return;
    float *o = out + r * out_stride + i;
    if (i + w > p.n_samp) {
        *o = __int_as_float(0x7fc00000);
        return;
    }
    const T *x = static_cast<const T *>(p.data) + r * p.row_stride + i;
    const bool has_sc = p.row_scale != nullptr;
    const float sc = has_sc ? p.row_scale[r] : 1.f;
    const float of = (has_sc && p.row_offset) ? p.row_offset[r] : 0.f;
    float s = 0.f, c = 0.f;
    for (int k = 0; k < w; ++k) {
        float v = Elem<DT>::cvt(x[k]);
        if (has_sc) v = fmaf(sc, v, of);
        const float y = v - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    *o = s;
}

}  // namespace

cudaError_t launch_threshold(const float *snr, const uint16_t *width, int64_t n_dm,
                             int64_t n_samp, int64_t stride, float thr, spd_candidate *out,
                             int64_t capacity, spd_result *result, cudaStream_t s) {
    const int64_t tpr = (n_samp + kThrTile - 1) / kThrTile;
    const int64_t tiles = n_dm * tpr;
    if (tiles <= 0) return cudaSuccess;
    threshold_kernel<<<(unsigned)tiles, kThrThreads, 0, s>>>(snr, width, n_samp, stride, tpr,
                                                             thr, out, capacity, result);
    return cudaGetLastError();
}

cudaError_t launch_boxcar_sums(const spd_plane &p, int w, float *out, int64_t out_stride,
                               cudaStream_t s) {
    if (p.n_dm <= 0 || p.n_samp <= 0) return cudaSuccess;
    const dim3 grid((unsigned)((p.n_samp + 255) / 256), (unsigned)p.n_dm);
    switch (p.dtype) {
        case SPD_F32: boxcar_sums_kernel<SPD_F32><<<grid, 256, 0, s>>>(p, w, out, out_stride); break;
        case SPD_F16: boxcar_sums_kernel<SPD_F16><<<grid, 256, 0, s>>>(p, w, out, out_stride); break;
        default: boxcar_sums_kernel<SPD_BF16><<<grid, 256, 0, s>>>(p, w, out, out_stride); break;
    }
    return cudaGetLastError();
}

}  // namespace spd
