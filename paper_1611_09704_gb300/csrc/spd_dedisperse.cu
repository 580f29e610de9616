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
constexpr int kDdPer = 2;                        // outputs per thread and DM trial
constexpr int kDdSpan = kDdThreads * kDdPer;     // output samples per CTA
constexpr int kDdDms = 16;                       // DM trials per CTA
constexpr int kDdChunk = 256;                    // channels whose delays are staged at once
constexpr int kDdSpread = 1024;                  // delay spread of a DM block held in shared memory
constexpr int kDdWin = kDdSpan + kDdSpread;      // staged window of one channel
constexpr int kDdLoads = kDdWin / kDdThreads;    // staging loads per thread (register path)
constexpr int kDdRing = 4;                       // channel windows in flight (FP32)

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

// 4-byte asynchronous copy global -> shared; with valid false nothing is read
// and the word is zero-filled.
__device__ __forceinline__ void cp_async4(float *dst, const float *src, bool valid) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src),
                 "r"(valid ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// One CTA: kDdSpan consecutive outputs t0 .. of kDdDms consecutive DM trials
// d0 ...  For every channel c the trials of the block read the one window
// x[c][t0 + lo_c, t0 + kDdSpan + hi_c) (lo_c, hi_c: the smallest and largest
// delay of the block at c), staged in shared memory; thread t sums outputs
// t0 + t + 256 j, j < 2, of every trial from it.  FP32 rows arrive by
// asynchronous copies kDdRing - 1 channels ahead of the channel being summed
// (a ring of windows, one barrier per channel); FP16 / BF16 rows are loaded
// one channel ahead into registers, decoded and stored (double buffer).
// Channels are summed in order c = 0, 1, ... for every output.  A block whose
// spread at some channel exceeds kDdSpread reads that channel from global
// memory instead.  A delay outside [0, n_samp - n_out] makes its trial's
// outputs NaN and sets the status (no read outside the row).
template <int DT>
__global__ void __launch_bounds__(kDdThreads) dedisperse_kernel(
    const typename Elem<DT>::T *fb, int64_t n_chan, int64_t n_samp, int64_t fb_stride,
    const float *scale, const float *offset, const int32_t *delays, int64_t n_dm, void *out,
    int out_dt, int64_t n_out, int64_t out_stride, spd_result *status) {
    using T = typename Elem<DT>::T;
    __shared__ __align__(16) float s_x[kDdRing][kDdWin];
    __shared__ __align__(16) int32_t s_dl[kDdChunk][kDdDms];
    __shared__ int32_t s_lo[kDdChunk], s_hi[kDdChunk];
    __shared__ uint32_t s_bad;                   // bit d: trial d0 + d has a bad delay
    const int tid = threadIdx.x;
    // block b: DM block b % n_dmb of time tile b / n_dmb, so the DM blocks of
    // one time tile run side by side and read its channel windows from L2
    const int64_t n_dmb = (n_dm + kDdDms - 1) / kDdDms;
    const int64_t b = blockIdx.x;
    const int64_t t0 = (b / n_dmb) * kDdSpan;
    const int64_t max_delay = n_samp - n_out;
    const bool has_sc = scale != nullptr;
    {
        const int64_t d0 = (b % n_dmb) * kDdDms;
        const int nd = (int)min((int64_t)kDdDms, n_dm - d0);
        // the thread's two outputs t0 + tid and t0 + tid + 256 of trial d as
        // one packed pair (two IEEE adds per packed add)
        static_assert(kDdPer == 2, "outputs per thread are one float2");
        float2 acc[kDdDms];
#pragma unroll
        for (int d = 0; d < kDdDms; ++d) acc[d] = make_float2(0.f, 0.f);
        if (tid == 0) s_bad = 0u;
        for (int64_t c0 = 0; c0 < n_chan; c0 += kDdChunk) {
            const int nc = (int)min((int64_t)kDdChunk, n_chan - c0);
            __syncthreads();   // the last chunk's delays and windows are no longer read
            // the chunk's delays; a bad one is replaced by the smallest good
            // delay of its channel (its trial's result is NaN anyway)
            for (int i = tid; i < nc * kDdDms; i += kDdThreads) {
                const int c = i / kDdDms, d = i - c * kDdDms;
                int32_t v = 0;
                if (d < nd) {
                    v = __ldg(delays + (d0 + d) * n_chan + c0 + c);
                    if (v < 0 || (int64_t)v > max_delay) {
                        atomicOr(&s_bad, 1u << d);
                        v = -1;
                    }
                }
                s_dl[c][d] = d < nd ? v : -1;
            }
            __syncthreads();
            for (int c = tid; c < nc; c += kDdThreads) {
                int lo = INT32_MAX, hi = -1;
                for (int d = 0; d < nd; ++d) {
                    const int v = s_dl[c][d];
                    if (v >= 0) {
                        lo = min(lo, v);
                        hi = max(hi, v);
                    }
                }
                if (hi < 0) lo = hi = 0;
                // delays relative to the channel's smallest; a bad delay and
                // the trials past the block's last read offset 0 (their sums
                // are never stored)
#pragma unroll
                for (int d = 0; d < kDdDms; ++d) {
                    const int v = s_dl[c][d];
                    s_dl[c][d] = (d < nd && v >= 0) ? v - lo : 0;
                }
                s_lo[c] = lo;
                s_hi[c] = hi;
            }
            __syncthreads();
            // channel c into the accumulators, from its staged window w
            auto sum_channel = [&](int c, const float *w) {
                const int lo = s_lo[c];
                if (s_hi[c] - lo <= kDdSpread) {
                    const int4 *dv = reinterpret_cast<const int4 *>(s_dl[c]);
#pragma unroll
                    for (int q = 0; q < kDdDms / 4; ++q) {
                        const int4 d4 = dv[q];   // four trials' delays, one broadcast load
                        const int dls[4] = {d4.x, d4.y, d4.z, d4.w};
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const float *p = w + tid + dls[e];
                            acc[4 * q + e] =
                                __fadd2_rn(acc[4 * q + e], make_float2(p[0], p[kDdThreads]));
                        }
                    }
                } else {   // a wide spread: this channel straight from global memory
                    const T *row = fb + (c0 + c) * fb_stride;
                    const float sc = has_sc ? __ldg(scale + c0 + c) : 1.f;
                    const float of = (has_sc && offset) ? __ldg(offset + c0 + c) : 0.f;
#pragma unroll
                    for (int d = 0; d < kDdDms; ++d) {
                        if (d >= nd) break;
                        const int64_t dl = (int64_t)lo + s_dl[c][d];
                        const int64_t t = t0 + tid;
                        if (t < n_out)
                            acc[d].x = __fadd_rn(acc[d].x, fb_value<DT>(row + t + dl, has_sc, sc, of));
                        if (t + kDdThreads < n_out)
                            acc[d].y = __fadd_rn(acc[d].y,
                                                 fb_value<DT>(row + t + kDdThreads + dl, has_sc, sc, of));
                    }
                }
            };
            // positions of channel c's window that are staged (none for a
            // channel read from global memory)
            auto need_of = [&](int c) {
                const int sp = s_hi[c] - s_lo[c];
                return sp <= kDdSpread ? kDdSpan + sp : 0;
            };
            if constexpr (DT == SPD_F32) {
                auto stage = [&](int c) {   // one copy group per channel, empty ones too
                    if (c < nc) {
                        const int64_t base = t0 + s_lo[c];
                        const float *row = reinterpret_cast<const float *>(fb) + (c0 + c) * fb_stride;
                        const int need = need_of(c);
                        float *w = s_x[c % kDdRing];
                        for (int i = tid; i < need; i += kDdThreads) {
                            const int64_t q = base + i;
                            const bool ok = q < n_samp;   // past the row end: zeros, never read
                            cp_async4(w + i, ok ? row + q : row, ok);
                        }
                    }
                    cp_async_commit();
                };
#pragma unroll
                for (int c = 0; c < kDdRing - 1; ++c) stage(c);
                for (int c = 0; c < nc; ++c) {
                    cp_async_wait<kDdRing - 2>();   // this thread's copies of channel c landed
                    __syncthreads();                // everyone's; channel c - 1 is summed
                    stage(c + kDdRing - 1);         // into the slot channel c - 1 used
                    sum_channel(c, s_x[c % kDdRing]);
                }
                cp_async_wait<0>();
            } else {
                float pre[kDdLoads];
                auto fetch = [&](int c) {
                    const int64_t base = t0 + s_lo[c];
                    const T *row = fb + (c0 + c) * fb_stride;
                    const float sc = has_sc ? __ldg(scale + c0 + c) : 1.f;
                    const float of = (has_sc && offset) ? __ldg(offset + c0 + c) : 0.f;
                    const int need = need_of(c);
#pragma unroll
                    for (int u = 0; u < kDdLoads; ++u) {
                        const int i = tid + u * kDdThreads;
                        const int64_t q = base + i;
                        pre[u] = (i < need && q < n_samp) ? fb_value<DT>(row + q, has_sc, sc, of)
                                                          : 0.f;
                    }
                };
                auto put = [&](int b) {
#pragma unroll
                    for (int u = 0; u < kDdLoads; ++u) s_x[b][tid + u * kDdThreads] = pre[u];
                };
                fetch(0);
                put(0);
                for (int c = 0; c < nc; ++c) {
                    const int b = c & 1;
                    const bool next = c + 1 < nc;
                    if (next) fetch(c + 1);   // in flight while channel c is summed
                    __syncthreads();          // window c staged; window c - 1 no longer read
                    sum_channel(c, s_x[b]);
                    if (next) put(b ^ 1);
                }
            }
        }
        __syncthreads();
        const uint32_t bad = s_bad;
        if (bad && status && tid == 0)
            atomicExch(&status->status, (int)SPD_ERR_INVALID_ARG);
#pragma unroll
        for (int d = 0; d < kDdDms; ++d) {
            if (d >= nd) break;
            const float nan = __int_as_float(0x7fc00000);
#pragma unroll
            for (int j = 0; j < kDdPer; ++j) {
                const int64_t t = t0 + tid + j * kDdThreads;
                if (t < n_out)
                    store_out(out, out_dt, (d0 + d) * out_stride + t,
                              ((bad >> d) & 1u) ? nan : (j ? acc[d].y : acc[d].x));
            }
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
    const int64_t n_tt = (n_out + kDdSpan - 1) / kDdSpan;
    const int64_t n_dmb = (n_dm + kDdDms - 1) / kDdDms;
    if (n_tt > INT32_MAX / n_dmb) return SPD_ERR_INVALID_ARG;
    const dim3 grid((unsigned)(n_tt * n_dmb));
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
