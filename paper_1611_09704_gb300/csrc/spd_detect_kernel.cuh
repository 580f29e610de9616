// spd_detect_kernel.cuh -- steps (b), (c), (d): boxcar filters, SNR, max over widths
// with the winning width, and thresholding with compaction (Sec. 2.3-2.4,
// Algorithm 1), in one kernel per DM-row tile.
//
// A CTA of 256 threads owns kTile = 4096 consecutive samples of one DM row and
// stages them, plus the (wmax - 1)-sample halo to their right, once in shared
// memory as centred values y = x - mu.  Each thread owns kX = 16 consecutive
// start samples and keeps their running boxcar sums B[k] in registers; the
// sums grow one step at a time as in Algorithm 1 (B = B + x[...]) from either
// a single sample y or a precomputed G-sample window sum S_G (for width lists
// that step by G), so B_w carries no large-prefix cancellation.  For every
// listed width: SNR = B * (1/sigma_w) and a running max.
//
// The winning width travels with the max: the low 6 mantissa bits of each SNR
// are replaced by a code (63 - index within a group of 64 widths) before a
// plain float max, so one max instruction keeps both, and among SNRs equal to
// 2^-17 relative the smallest width wins -- the strict ">" of Algorithm 1 at
// that resolution.  Widths past the row end see y = -inf, which packs to NaN
// and is ignored by max.
//
// Shared arrays are stored transposed ([16][R], position p at
// (p % 16) * R + p / 16) so that the 32 lanes of a warp, each reading
// "its own start + the same offset", hit 32 consecutive words.
#pragma once
#include "spd_internal.cuh"

#include <math.h>

namespace spd {

namespace {

__device__ __forceinline__ float packw(float s, uint32_t code) {
    return __uint_as_float((__float_as_uint(s) & 0xFFFFFFC0u) | code);
}

__device__ __forceinline__ float fmax3(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

__device__ __forceinline__ float ld_t(const float *base_t, int R, int off) {
    return base_t[(off & (kX - 1)) * R + (off >> 4)];
}

template <int DT>
__device__ __forceinline__ void load4v(const typename Elem<DT>::T *p, float &a, float &b,
                                       float &c, float &d);
template <>
__device__ __forceinline__ void load4v<SPD_F32>(const float *p, float &a, float &b, float &c,
                                                float &d) {
    const float4 v = __ldcs(reinterpret_cast<const float4 *>(p));
    a = v.x; b = v.y; c = v.z; d = v.w;
}
template <>
__device__ __forceinline__ void load4v<SPD_F16>(const __half *p, float &a, float &b, float &c,
                                                float &d) {
    const uint2 v = __ldcs(reinterpret_cast<const uint2 *>(p));
    const float2 lo = __half22float2(*reinterpret_cast<const __half2 *>(&v.x));
    const float2 hi = __half22float2(*reinterpret_cast<const __half2 *>(&v.y));
    a = lo.x; b = lo.y; c = hi.x; d = hi.y;
}
template <>
__device__ __forceinline__ void load4v<SPD_BF16>(const __nv_bfloat16 *p, float &a, float &b,
                                                 float &c, float &d) {
    const uint2 v = __ldcs(reinterpret_cast<const uint2 *>(p));
    const float2 lo = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&v.x));
    const float2 hi = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&v.y));
    a = lo.x; b = lo.y; c = hi.x; d = hi.y;
}

// Running state of one thread: kX boxcar sums and kX packed maxima.
struct State {
    float B[kX];
    float best[kX];
};

// d = 1 run from y: widths c0 + cc use W[k + cc].
__device__ __forceinline__ void run_fine(State &st, const float *sy_t, int R, const Run &r,
                                         const float *s_inv) {
    const bool eval = (r.flags & kRunEval) != 0;
    float W[2 * kX];
#pragma unroll
    for (int m = 0; m < kX; ++m) W[m] = ld_t(sy_t, R, r.off + m);
    for (int c0 = 0; c0 < r.count; c0 += kX) {
#pragma unroll
        for (int m = 0; m < kX; ++m) W[kX + m] = ld_t(sy_t, R, r.off + c0 + kX + m);
        if (eval) {
#pragma unroll
            for (int cc = 0; cc < kX; cc += 2) {
                const int c = c0 + cc;
                if (c + 1 < r.count) {
                    const int wi = r.widx0 + c;
                    const float i0 = s_inv[wi], i1 = s_inv[wi + 1];
                    const uint32_t k0 = 63u - (uint32_t)(wi & 63);
                    const uint32_t k1 = 63u - (uint32_t)((wi + 1) & 63);
#pragma unroll
                    for (int k = 0; k < kX; ++k) {
                        st.B[k] += W[k + cc];
                        const float s0 = st.B[k] * i0;
                        st.B[k] += W[k + cc + 1];
                        const float s1 = st.B[k] * i1;
                        st.best[k] = fmax3(st.best[k], packw(s0, k0), packw(s1, k1));
                    }
                } else if (c < r.count) {
                    const int wi = r.widx0 + c;
                    const float i0 = s_inv[wi];
                    const uint32_t k0 = 63u - (uint32_t)(wi & 63);
#pragma unroll
                    for (int k = 0; k < kX; ++k) {
                        st.B[k] += W[k + cc];
                        st.best[k] = fmaxf(st.best[k], packw(st.B[k] * i0, k0));
                    }
                }
            }
        } else {
#pragma unroll
            for (int cc = 0; cc < kX; ++cc) {
                if (c0 + cc < r.count) {
#pragma unroll
                    for (int k = 0; k < kX; ++k) st.B[k] += W[k + cc];
                }
            }
        }
#pragma unroll
        for (int m = 0; m < kX; ++m) W[m] = W[kX + m];
    }
}

// d = G run from S_G: width c uses S_G at offsets off + c*G + k, k < 16.
// Segments of G values live in a ring of NS = 16/G + 1 slots.
template <int G>
__device__ __forceinline__ void run_coarse(State &st, const float *sg_t, int R, const Run &r,
                                           const float *s_inv) {
    const bool eval = (r.flags & kRunEval) != 0;
    constexpr int SEG = kX / G;
    constexpr int NS = SEG + 1;
    float Wr[NS * G];
#pragma unroll
    for (int s = 0; s < SEG - 1; ++s)
#pragma unroll
        for (int e = 0; e < G; ++e) Wr[s * G + e] = ld_t(sg_t, R, r.off + s * G + e);

    for (int c0 = 0; c0 < r.count; c0 += 2 * NS) {
#pragma unroll
        for (int u = 0; u < 2 * NS; u += 2) {
            const int c = c0 + u;
            if (c >= r.count) break;
            const bool two = (c + 1 < r.count);
            // segment c + SEG - 1 -> slot (u + SEG - 1) % NS
#pragma unroll
            for (int e = 0; e < G; ++e)
                Wr[((u + SEG - 1) % NS) * G + e] = ld_t(sg_t, R, r.off + (c + SEG - 1) * G + e);
            if (two) {
#pragma unroll
                for (int e = 0; e < G; ++e)
                    Wr[((u + SEG) % NS) * G + e] = ld_t(sg_t, R, r.off + (c + SEG) * G + e);
            }
            if (eval) {
                const int wi = r.widx0 + c;
                const float i0 = s_inv[wi];
                const uint32_t k0 = 63u - (uint32_t)(wi & 63);
                if (two) {
                    const float i1 = s_inv[wi + 1];
                    const uint32_t k1 = 63u - (uint32_t)((wi + 1) & 63);
#pragma unroll
                    for (int k = 0; k < kX; ++k) {
                        st.B[k] += Wr[((u + k / G) % NS) * G + (k % G)];
                        const float s0 = st.B[k] * i0;
                        st.B[k] += Wr[((u + 1 + k / G) % NS) * G + (k % G)];
                        const float s1 = st.B[k] * i1;
                        st.best[k] = fmax3(st.best[k], packw(s0, k0), packw(s1, k1));
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < kX; ++k) {
                        st.B[k] += Wr[((u + k / G) % NS) * G + (k % G)];
                        st.best[k] = fmaxf(st.best[k], packw(st.B[k] * i0, k0));
                    }
                }
            } else {
#pragma unroll
                for (int k = 0; k < kX; ++k) st.B[k] += Wr[((u + k / G) % NS) * G + (k % G)];
                if (two) {
#pragma unroll
                    for (int k = 0; k < kX; ++k)
                        st.B[k] += Wr[((u + 1 + k / G) % NS) * G + (k % G)];
                }
            }
        }
    }
}

// Build S_G over all positions of the tile's shared window: chunk c holds
// positions 16c .. 16c+15; S_G[p] = y[p] + ... + y[p+G-1] by pairwise levels.
template <int G>
__device__ __forceinline__ void build_sg(const float *s_y, float *s_g, int R) {
    for (int c = threadIdx.x; c < R - 1; c += kThreads) {
        float v[kX + G - 1];
#pragma unroll
        for (int m = 0; m < kX + G - 1; ++m) v[m] = s_y[(m & (kX - 1)) * R + c + (m >> 4)];
#pragma unroll
        for (int len = 1; len < G; len *= 2) {
#pragma unroll
            for (int m = 0; m < kX + G - 1 - len; ++m) v[m] = v[m] + v[m + len];
        }
#pragma unroll
        for (int m = 0; m < kX; ++m) s_g[m * R + c] = v[m];
    }
    // last column: positions past the window are never read by an evaluated
    // width; fill with -inf for determinism.
    if (threadIdx.x < kX) s_g[threadIdx.x * R + (R - 1)] = -INFINITY;
}

template <int DT, int G, bool PLANE, bool MG>
__global__ void __launch_bounds__(kThreads, 2) detect_kernel(const DetectArgs a,
                                                             const __grid_constant__ Program prog) {
    using T = typename Elem<DT>::T;
    extern __shared__ __align__(16) float smem[];
    const int R = a.R;
    float *s_y = smem;
    float *s_g = s_y + kX * R;
    float *s_inv = s_y + (G > 1 ? 2 : 1) * kX * R;
    __shared__ int s_wsum[kThreads / 32];
    __shared__ unsigned long long s_base;

    const int tid = threadIdx.x;
    const int64_t row = blockIdx.x / a.tiles_per_row;
    const int64_t t0 = (blockIdx.x - row * a.tiles_per_row) * (int64_t)kTile;
    const int entry = a.per_row ? (int)row : 0;
    const int64_t i0 = t0 + (int64_t)tid * kX;   // first start sample of this thread

    if (a.flags[entry]) {
        if (PLANE) {
            for (int k = 0; k < kX; ++k) {
                if (i0 + k < a.n_samp) {
                    a.snr_out[row * a.out_stride + i0 + k] = __int_as_float(0x7fc00000);
                    a.width_out[row * a.out_stride + i0 + k] = 0;
                }
            }
        }
        return;
    }

    for (int k = tid; k < prog.n_eval; k += kThreads)
        s_inv[k] = a.inv_tab[(int64_t)entry * prog.n_eval + k];
    const float2 mu = a.mu_tab[entry];
    const bool has_sc = a.scale != nullptr;
    const float sc = has_sc ? a.scale[row] : 1.f;
    const float of = (has_sc && a.offset) ? a.offset[row] : 0.f;
    const T *rowp = static_cast<const T *>(a.data) + row * a.stride;
    const int span = kTile + prog.wmax - 1;   // positions [0, span) of the window are needed

    // Stage centred samples; -inf past the row end (and past the window).
    for (int q = tid; q < (kX * R) / 4; q += kThreads) {
        const int p = 4 * q;
        const int64_t gt = t0 + p;
        float x[4];
        if (a.vec_ok && gt + 3 < a.n_samp && p + 3 < span) {
            load4v<DT>(rowp + gt, x[0], x[1], x[2], x[3]);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if (has_sc) x[e] = fmaf(sc, x[e], of);
                x[e] = (x[e] - mu.x) - mu.y;
            }
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if (gt + e < a.n_samp && p + e < span) {
                    float v = Elem<DT>::cvt(rowp[gt + e]);
                    if (has_sc) v = fmaf(sc, v, of);
                    x[e] = (v - mu.x) - mu.y;
                } else {
                    x[e] = -INFINITY;
                }
            }
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) s_y[((p + e) & (kX - 1)) * R + ((p + e) >> 4)] = x[e];
    }
    __syncthreads();
    if (G > 1) {
        build_sg<(G > 1 ? G : 2)>(s_y, s_g, R);
        __syncthreads();
    }

    State st;
    float obest[MG ? kX : 1];
    int ogrp[MG ? kX : 1];
#pragma unroll
    for (int k = 0; k < kX; ++k) {
        st.B[k] = 0.f;
        st.best[k] = -INFINITY;
    }
    if (MG) {
#pragma unroll
        for (int k = 0; k < kX; ++k) { obest[k] = -INFINITY; ogrp[k] = 0; }
    }
    const float *sy_t = s_y + tid;
    const float *sg_t = s_g + tid;
    for (int ri = 0; ri < prog.n_runs; ++ri) {
        const Run r = prog.runs[ri];
        if (G > 1 && (r.flags & kRunSrcG))
            run_coarse<(G > 1 ? G : 2)>(st, sg_t, R, r, s_inv);
        else
            run_fine(st, sy_t, R, r, s_inv);
        if (MG && (r.flags & kRunEndGroup)) {
            const int g = r.widx0 >> 6;
#pragma unroll
            for (int k = 0; k < kX; ++k) {
                if (st.best[k] > obest[k]) { obest[k] = st.best[k]; ogrp[k] = g; }
                st.best[k] = -INFINITY;
            }
        }
    }

    // Decode (value, width) and emit.
    float snr[kX];
    int wdt[kX];
#pragma unroll
    for (int k = 0; k < kX; ++k) {
        const float bv = MG ? obest[k] : st.best[k];
        const uint32_t bits = __float_as_uint(bv);
        const int g = MG ? ogrp[k] : 0;
        const int wi = g * 64 + (63 - (int)(bits & 63u));
        snr[k] = __uint_as_float(bits & 0xFFFFFFC0u);
        wdt[k] = (wi < prog.n_eval) ? (int)prog.eval_w[wi] : 0;
    }

    if (PLANE) {
        float *so = a.snr_out + row * a.out_stride;
        uint16_t *wo = a.width_out + row * a.out_stride;
        const bool full = i0 + kX <= a.n_samp;
        const bool al = ((reinterpret_cast<uintptr_t>(so + i0) & 15) == 0) &&
                        ((reinterpret_cast<uintptr_t>(wo + i0) & 15) == 0);
        if (full && al) {
#pragma unroll
            for (int v = 0; v < kX / 4; ++v)
                reinterpret_cast<float4 *>(so + i0)[v] =
                    make_float4(snr[4 * v], snr[4 * v + 1], snr[4 * v + 2], snr[4 * v + 3]);
#pragma unroll
            for (int v = 0; v < kX / 8; ++v) {
                uint4 u;
                u.x = (uint32_t)wdt[8 * v] | ((uint32_t)wdt[8 * v + 1] << 16);
                u.y = (uint32_t)wdt[8 * v + 2] | ((uint32_t)wdt[8 * v + 3] << 16);
                u.z = (uint32_t)wdt[8 * v + 4] | ((uint32_t)wdt[8 * v + 5] << 16);
                u.w = (uint32_t)wdt[8 * v + 6] | ((uint32_t)wdt[8 * v + 7] << 16);
                reinterpret_cast<uint4 *>(wo + i0)[v] = u;
            }
        } else {
#pragma unroll
            for (int k = 0; k < kX; ++k) {
                if (i0 + k < a.n_samp) {
                    so[i0 + k] = snr[k];
                    wo[i0 + k] = (uint16_t)wdt[k];
                }
            }
        }
        return;
    }

    // Threshold (Sec. 2.4, inclusive) and block-aggregated compaction.
    uint32_t mask = 0;
#pragma unroll
    for (int k = 0; k < kX; ++k)
        if (i0 + k < a.n_samp && snr[k] >= a.threshold) mask |= 1u << k;
    const int cnt = __popc(mask);
    const int lane = tid & 31, warp = tid >> 5;
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) s_wsum[warp] = incl;
    __syncthreads();
    if (tid < 32) {
        const int wv = (lane < kThreads / 32) ? s_wsum[lane] : 0;
        int wi = wv;
#pragma unroll
        for (int o = 1; o < kThreads / 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += v;
        }
        if (lane < kThreads / 32) s_wsum[lane] = wi - wv;   // exclusive
        const int total = __shfl_sync(0xffffffffu, wi, kThreads / 32 - 1);
        if (lane == 0)
            s_base = total ? atomicAdd(reinterpret_cast<unsigned long long *>(&a.result->count),
                                       (unsigned long long)total)
                           : 0ull;
    }
    __syncthreads();
    if (cnt) {
        unsigned long long idx = s_base + (unsigned long long)(s_wsum[warp] + incl - cnt);
#pragma unroll
        for (int k = 0; k < kX; ++k) {
            if (mask & (1u << k)) {
                if (idx < (unsigned long long)a.capacity) {
                    int4 rec;
                    rec.x = (int)row;
                    rec.y = (int)(i0 + k);
                    rec.z = __float_as_int(snr[k]);
                    rec.w = wdt[k];
                    reinterpret_cast<int4 *>(a.out)[idx] = rec;
                }
                ++idx;
            }
        }
    }
}

template <int DT, int G>
cudaError_t launch_dg(const DetectArgs &a, const Program &prog, bool plane_out, bool mg,
                      size_t smem, cudaStream_t s) {
    const int64_t tiles = a.n_dm * a.tiles_per_row;
    const dim3 grid((unsigned)tiles);
    void (*k)(const DetectArgs, const Program);
    if (plane_out)
        k = mg ? detect_kernel<DT, G, true, true> : detect_kernel<DT, G, true, false>;
    else
        k = mg ? detect_kernel<DT, G, false, true> : detect_kernel<DT, G, false, false>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, kThreads, smem, s>>>(a, prog);
    return cudaGetLastError();
}

}  // namespace

template <int DT>
cudaError_t launch_detect_dt(const DetectArgs &a, const Program &prog, bool plane_out, size_t smem,
                     cudaStream_t s) {
    const bool mg = prog.n_eval > 64;
    switch (prog.G) {
        case 4: return launch_dg<DT, 4>(a, prog, plane_out, mg, smem, s);
        case 8: return launch_dg<DT, 8>(a, prog, plane_out, mg, smem, s);
        case 16: return launch_dg<DT, 16>(a, prog, plane_out, mg, smem, s);
        default: return launch_dg<DT, 1>(a, prog, plane_out, mg, smem, s);
    }
}


}  // namespace spd
