// spd_misc.cu -- step (d) on a stored SNR plane (Sec. 2.4), the per-DM
// clustering of its candidates, and the raw boxcar sums test aid.
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

// Per-DM clustering of the candidates (snr >= thr) in time: one warp scans
// one row, 32 samples per step, kClusterSteps steps of loads in flight.  In
// sample order a candidate joins the open cluster when it lies at most `gap`
// samples after the previous candidate, else the open cluster is written and
// a new one starts.  A step is taken a segment at a time, not a candidate at a
// time: each lane finds its previous candidate (in the step's ballot mask, or
// the open cluster's last), the lanes that start a cluster form a second mask,
// and each segment between starts is absorbed with a popcount, its highest
// set bit, and one warp max (redux) over order-preserving keys of its SNRs.
// Every lane holds the same cluster state, so lane 0 alone writes records.
constexpr int kClusterWarps = 8;   // rows per CTA
constexpr int kClusterSteps = 8;   // 32-sample steps loaded at once per warp

struct ClusterState {
    int64_t first, last, peak_t, members;
    float peak;
    unsigned peak_key;
    int peak_w;
};

// Monotone map of a non-NaN float to an unsigned key (larger float, larger
// key; -0.0 and +0.0 compare equal, so they share one key); every key is
// > 0, so 0 stands for "no member".
__device__ __forceinline__ unsigned order_key(float f) {
    unsigned u = __float_as_uint(f);
    if (u == 0x80000000u) u = 0u;
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ void emit_cluster(const ClusterState &c, int64_t row,
                                             spd_cluster *out, int64_t capacity,
                                             spd_result *result, int lane) {
    if (lane != 0) return;
    const unsigned long long idx =
        atomicAdd(reinterpret_cast<unsigned long long *>(&result->count), 1ull);
    if (idx < (unsigned long long)capacity) {
        spd_cluster r;
        r.dm = (int32_t)row;
        r.first = (int32_t)c.first;
        r.last = (int32_t)c.last;
        r.peak_sample = (int32_t)c.peak_t;
        r.peak_snr = c.peak;
        r.peak_width = c.peak_w;
        r.members = (int32_t)c.members;
        r.reserved0 = 0;
        out[idx] = r;
    }
}

// The members M (a lane mask of this step, starting at sample t0) join the
// open cluster: count, last sample, and the peak (strict: an earlier equal
// peak stays; within M the lowest lane of the maximum).
__device__ __forceinline__ void absorb(ClusterState &c, unsigned M, int64_t t0, unsigned key,
                                       float v, int w, int lane) {
    c.members += __popc(M);
    c.last = t0 + (31 - __clz(M));
    const unsigned mine = ((M >> lane) & 1u) ? key : 0u;
    const unsigned kmax = __reduce_max_sync(0xffffffffu, mine);
    if (kmax > c.peak_key) {
        const int pl = __ffs(__ballot_sync(0xffffffffu, mine == kmax)) - 1;
        c.peak_key = kmax;
        c.peak = __shfl_sync(0xffffffffu, v, pl);
        c.peak_w = __shfl_sync(0xffffffffu, w, pl);
        c.peak_t = t0 + pl;
    }
}

__global__ void __launch_bounds__(32 * kClusterWarps) cluster_kernel(
    const float *snr, const uint16_t *width, int64_t n_dm, int64_t n_samp, int64_t stride,
    float thr, int64_t gap, spd_cluster *out, int64_t capacity, spd_result *result) {
    const int lane = threadIdx.x & 31;
    const int64_t row = (int64_t)blockIdx.x * kClusterWarps + (threadIdx.x >> 5);
    if (row >= n_dm) return;   // the whole warp
    const float *sp = snr + row * stride;
    const uint16_t *wp = width + row * stride;
    bool open = false;
    ClusterState c{0, 0, 0, 0, 0.f, 0u, 0};
    for (int64_t base = 0; base < n_samp; base += 32 * kClusterSteps) {
        float v[kClusterSteps];
        int w[kClusterSteps];
#pragma unroll
        for (int k = 0; k < kClusterSteps; ++k) {
            const int64_t t = base + 32 * k + lane;
            v[k] = t < n_samp ? __ldcs(sp + t) : -INFINITY;
            w[k] = t < n_samp ? (int)__ldcs(wp + t) : 0;
        }
#pragma unroll
        for (int k = 0; k < kClusterSteps; ++k) {
            const bool cand = v[k] >= thr;   // NaN: not a candidate
            const unsigned m = __ballot_sync(0xffffffffu, cand);
            if (!m) continue;
            const int64_t t0 = base + 32 * k;
            // does this lane's candidate start a cluster?
            const unsigned below = m & ((1u << lane) - 1u);
            const bool has_prev = below != 0u || open;
            const int64_t prev = below ? t0 + (31 - __clz(below)) : c.last;
            const bool start = cand && (!has_prev || (t0 + lane) - prev > gap);
            unsigned S = __ballot_sync(0xffffffffu, start);
            const unsigned key = cand ? order_key(v[k]) : 0u;
            // members before the first start continue the open cluster
            const int fs = S ? __ffs(S) - 1 : 32;
            const unsigned cont = fs == 32 ? m : (m & ((1u << fs) - 1u));
            if (cont) absorb(c, cont, t0, key, v[k], w[k], lane);
            while (S) {
                const int s0 = __ffs(S) - 1;
                S &= S - 1u;
                const int e = S ? __ffs(S) - 1 : 32;
                const unsigned seg = m & (0xffffffffu << s0) & (e == 32 ? 0xffffffffu : ((1u << e) - 1u));
                if (open) emit_cluster(c, row, out, capacity, result, lane);
                open = true;
                c.first = t0 + s0;
                c.members = 0;
                c.peak_key = 0u;
                absorb(c, seg, t0, key, v[k], w[k], lane);
            }
        }
    }
    if (open) emit_cluster(c, row, out, capacity, result, lane);
}

}  // namespace

// Thresholding of Sec. 2.4 on the plane, in place: 8 samples per thread,
// 128-bit accesses where the row allows.
__global__ void __launch_bounds__(256) threshold_plane_kernel(float *snr, uint16_t *width,
                                                              int64_t n_samp, int64_t stride,
                                                              float thr) {
    const int64_t row = blockIdx.y;
    const int64_t i0 = ((int64_t)blockIdx.x * 256 + threadIdx.x) * 8;
    if (i0 >= n_samp) return;
    float *sp = snr + row * stride;
    uint16_t *wp = width ? width + row * stride : nullptr;
    const bool vec = i0 + 8 <= n_samp && ((reinterpret_cast<uintptr_t>(sp + i0) & 15) == 0) &&
                     (!wp || (reinterpret_cast<uintptr_t>(wp + i0) & 15) == 0);
    if (vec) {
        float4 a = reinterpret_cast<float4 *>(sp + i0)[0];
        float4 b = reinterpret_cast<float4 *>(sp + i0)[1];
        const bool k[8] = {a.x >= thr, a.y >= thr, a.z >= thr, a.w >= thr,
                           b.x >= thr, b.y >= thr, b.z >= thr, b.w >= thr};
        a.x = k[0] ? a.x : 0.f; a.y = k[1] ? a.y : 0.f; a.z = k[2] ? a.z : 0.f;
        a.w = k[3] ? a.w : 0.f; b.x = k[4] ? b.x : 0.f; b.y = k[5] ? b.y : 0.f;
        b.z = k[6] ? b.z : 0.f; b.w = k[7] ? b.w : 0.f;
        reinterpret_cast<float4 *>(sp + i0)[0] = a;
        reinterpret_cast<float4 *>(sp + i0)[1] = b;
        if (wp) {
            uint4 u = reinterpret_cast<uint4 *>(wp + i0)[0];
            uint32_t *uw = reinterpret_cast<uint32_t *>(&u);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint32_t lo = k[2 * q] ? (uw[q] & 0xffffu) : 0u;
                const uint32_t hi = k[2 * q + 1] ? (uw[q] & 0xffff0000u) : 0u;
                uw[q] = lo | hi;
            }
            reinterpret_cast<uint4 *>(wp + i0)[0] = u;
        }
        return;
    }
    for (int q = 0; q < 8 && i0 + q < n_samp; ++q) {
        const bool keep = sp[i0 + q] >= thr;
        if (!keep) {
            sp[i0 + q] = 0.f;
            if (wp) wp[i0 + q] = 0;
        }
    }
}

cudaError_t launch_threshold_plane(float *snr, uint16_t *width, int64_t n_dm, int64_t n_samp,
                                   int64_t stride, float thr, cudaStream_t s) {
    if (n_dm <= 0 || n_samp <= 0) return cudaSuccess;
    const int64_t per = 256 * 8;
    int64_t y = n_dm;
    for (int64_t r0 = 0; r0 < n_dm; r0 += 65535) {   // grid.y limit
        y = n_dm - r0 < 65535 ? n_dm - r0 : 65535;
        const dim3 grid((unsigned)((n_samp + per - 1) / per), (unsigned)y);
        threshold_plane_kernel<<<grid, 256, 0, s>>>(snr + r0 * stride,
                                                    width ? width + r0 * stride : nullptr,
                                                    n_samp, stride, thr);
    }
    return cudaGetLastError();
}

// Decimation in time by 2: dst[r][j] = x[r][2j] + x[r][2j+1] in FP32 (x the
// dequantised source), for j < n_out.  Four outputs per thread.
template <int DT>
__global__ void __launch_bounds__(256) decimate2_kernel(const typename Elem<DT>::T *src,
                                                        int64_t src_stride, const float *scale,
                                                        const float *offset, int64_t n_out,
                                                        float *dst, int64_t dst_stride) {
    const int64_t row = blockIdx.y;
    const int64_t j0 = ((int64_t)blockIdx.x * 256 + threadIdx.x) * 4;
    if (j0 >= n_out) return;
    const typename Elem<DT>::T *sp = src + row * src_stride + 2 * j0;
    const float sc = scale ? scale[row] : 1.f;
    const float of = (scale && offset) ? offset[row] : 0.f;
    float o[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (j0 + q < n_out) {
            float a = Elem<DT>::cvt(sp[2 * q]), b = Elem<DT>::cvt(sp[2 * q + 1]);
            if (scale) { a = fmaf(sc, a, of); b = fmaf(sc, b, of); }
            o[q] = __fadd_rn(a, b);
        }
    }
    float *dp = dst + row * dst_stride + j0;
    if (j0 + 4 <= n_out && (reinterpret_cast<uintptr_t>(dp) & 15) == 0) {
        *reinterpret_cast<float4 *>(dp) = make_float4(o[0], o[1], o[2], o[3]);
    } else {
        for (int q = 0; q < 4 && j0 + q < n_out; ++q) dp[q] = o[q];
    }
}

cudaError_t launch_decimate2(const spd_plane &p, float *dst, int64_t n_out, int64_t dst_stride,
                             cudaStream_t s) {
    if (p.n_dm <= 0 || n_out <= 0) return cudaSuccess;
    for (int64_t r0 = 0; r0 < p.n_dm; r0 += 65535) {   // grid.y limit
        const int64_t y = p.n_dm - r0 < 65535 ? p.n_dm - r0 : 65535;
        const dim3 grid((unsigned)((n_out + 1023) / 1024), (unsigned)y);
        const float *sc = p.row_scale ? p.row_scale + r0 : nullptr;
        const float *of = p.row_offset ? p.row_offset + r0 : nullptr;
        float *d = dst + r0 * dst_stride;
        switch (p.dtype) {
            case SPD_F32:
                decimate2_kernel<SPD_F32><<<grid, 256, 0, s>>>(
                    static_cast<const float *>(p.data) + r0 * p.row_stride, p.row_stride, sc, of,
                    n_out, d, dst_stride);
                break;
            case SPD_F16:
                decimate2_kernel<SPD_F16><<<grid, 256, 0, s>>>(
                    static_cast<const __half *>(p.data) + r0 * p.row_stride, p.row_stride, sc, of,
                    n_out, d, dst_stride);
                break;
            default:
                decimate2_kernel<SPD_BF16><<<grid, 256, 0, s>>>(
                    static_cast<const __nv_bfloat16 *>(p.data) + r0 * p.row_stride, p.row_stride,
                    sc, of, n_out, d, dst_stride);
                break;
        }
    }
    return cudaGetLastError();
}

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

cudaError_t launch_cluster(const float *snr, const uint16_t *width, int64_t n_dm,
                           int64_t n_samp, int64_t stride, float thr, int64_t gap,
                           spd_cluster *out, int64_t capacity, spd_result *result,
                           cudaStream_t s) {
    const int64_t blocks = (n_dm + kClusterWarps - 1) / kClusterWarps;
    if (blocks <= 0 || n_samp <= 0) return cudaSuccess;
    cluster_kernel<<<(unsigned)blocks, 32 * kClusterWarps, 0, s>>>(
        snr, width, n_dm, n_samp, stride, thr, gap, out, capacity, result);
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
