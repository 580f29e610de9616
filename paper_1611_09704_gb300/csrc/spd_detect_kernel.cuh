// spd_detect_kernel.cuh -- steps (b) and (c) over every sample: the plane
// output of spd_boxcar_snr, each start's best SNR over the widths and the
// winning width (Sec. 2.3, Algorithm 1).  The candidate search, which prunes
// with bounds and writes records, is the search kernel (spd_search_kernel.cuh).
//
// Persistent CTAs of 256 threads walk the plane's tiles (kTile = 4096
// consecutive samples of one DM row).  Each tile's window -- the tile plus the
// (wmax - 1)-sample halo to its right -- arrives in shared memory by a 1-D
// bulk (TMA) copy issued one tile ahead, so the copy of tile k+1 overlaps the
// arithmetic of tile k.  The window is then staged as centred values
// y = x - mu, G-sample window sums S_G, and per 16-position block a
// compensated (hi + lo) prefix sum of y.
//
// Each thread owns kX = 16 consecutive start samples and keeps their running
// boxcar sums B in registers as eight pairs of adjacent samples (one packed
// f32x2 add or multiply serves two samples).  Widths are taken in groups: a
// group's sums start from the prefix sums (B_off = C[i+off] - C[i]) and grow
// one step per width as in Algorithm 1 (B = B + x[...]); SNR = B * (1/sigma_w).
// The low 6 mantissa bits of each SNR are replaced by a code (63 - index
// within a block of 64 widths) before a float max, so one max keeps value and
// width; among SNRs equal to 2^-17 relative the smallest width wins -- the
// strict ">" of Algorithm 1 at that resolution.
//
// Widths past the row end see y = -inf (sums -inf or NaN), ignored by max.
// Shared arrays hold 16 positions in 20 words (4 padding words per block of
// 16): lane t reads "16 t + offset", so 32 lanes hit distinct banks and
// 128-bit loads are conflict-free within each quarter warp.
#pragma once
#include "spd_device.cuh"

namespace spd {

namespace {

constexpr int kPad = 20;             // shared words per 16 positions
constexpr int kMaxLevel = 5;         // sparse max table: windows up to 2^5 blocks

__device__ __forceinline__ int padr(int p) { return (p & 15) + kPad * (p >> 4); }

// ------------------------------------------------------------ width sinks

// Plane output: packed (SNR, width code) max per sample.
struct PackSink {
    float best[kX];
    __device__ __forceinline__ void two(int j, int wi, float2 sa, float2 sb) {
        const uint32_t ka = 63u - (uint32_t)(wi & 63), kb = 63u - (uint32_t)((wi + 1) & 63);
        best[2 * j] = fmax3(best[2 * j], packw(sa.x, ka), packw(sb.x, kb));
        best[2 * j + 1] = fmax3(best[2 * j + 1], packw(sa.y, ka), packw(sb.y, kb));
    }
    __device__ __forceinline__ void one(int j, int wi, float2 sa) {
        const uint32_t ka = 63u - (uint32_t)(wi & 63);
        best[2 * j] = fmaxf(best[2 * j], packw(sa.x, ka));
        best[2 * j + 1] = fmaxf(best[2 * j + 1], packw(sa.y, ka));
    }
};

// Two consecutive widths (eval indices wi, wi+1) with step values Va, Vb.
template <class Sink>
__device__ __forceinline__ void eval2(float2 *B, Sink &sk, const float2 *Va, const float2 *Vb,
                                      int wi, const float *s_inv) {
    const float ia = s_inv[wi], ib = s_inv[wi + 1];
    const float2 ia2 = make_float2(ia, ia), ib2 = make_float2(ib, ib);
#pragma unroll
    for (int j = 0; j < kX / 2; ++j) {
        B[j] = add2(B[j], Va[j]);
        const float2 sa = mul2(B[j], ia2);
        B[j] = add2(B[j], Vb[j]);
        const float2 sb = mul2(B[j], ib2);
        sk.two(j, wi, sa, sb);
    }
}

template <class Sink>
__device__ __forceinline__ void eval1(float2 *B, Sink &sk, const float2 *Va, int wi,
                                      const float *s_inv) {
    const float ia = s_inv[wi];
    const float2 ia2 = make_float2(ia, ia);
#pragma unroll
    for (int j = 0; j < kX / 2; ++j) {
        B[j] = add2(B[j], Va[j]);
        sk.one(j, wi, mul2(B[j], ia2));
    }
}

// Fine group (step 1) whose start is a multiple of 16.  For 16 widths c0 + cc
// the steps are y[16t + q0 + cc + k], k < 16, q0 = off + c0: even cc read the
// pairs E[q] = positions (2q, 2q+1), odd cc the pairs O[q] = (2q+1, 2q+2).
template <class Sink>
__device__ __forceinline__ void run_fine_aligned(float2 *B, Sink &sk, const float *bt,
                                                 const Group &g, const float *s_inv) {
    for (int c0 = 0; c0 < g.count; c0 += 16) {
        const float *blk = bt + kPad * ((g.off + c0) >> 4);
        float2 E[16], O[15];
        // widths cc < 8 read E[0..11) and O[0..11); the rest is loaded after
#pragma unroll
        for (int v = 0; v < 6; ++v) {
            const float4 f = *reinterpret_cast<const float4 *>(blk + (v >> 2) * kPad + (v & 3) * 4);
            E[2 * v] = make_float2(f.x, f.y);
            E[2 * v + 1] = make_float2(f.z, f.w);
        }
#pragma unroll
        for (int q = 0; q < 11; ++q) O[q] = make_float2(blk[padr(2 * q + 1)], blk[padr(2 * q + 2)]);
#pragma unroll
        for (int cc = 0; cc < 16; cc += 2) {
            if (cc == 8) {
#pragma unroll
                for (int v = 6; v < 8; ++v) {
                    const float4 f =
                        *reinterpret_cast<const float4 *>(blk + (v >> 2) * kPad + (v & 3) * 4);
                    E[2 * v] = make_float2(f.x, f.y);
                    E[2 * v + 1] = make_float2(f.z, f.w);
                }
#pragma unroll
                for (int q = 11; q < 15; ++q)
                    O[q] = make_float2(blk[padr(2 * q + 1)], blk[padr(2 * q + 2)]);
            }
            const int c = c0 + cc;
            if (c + 1 < g.count)
                eval2(B, sk, E + cc / 2, O + cc / 2, g.widx0 + c, s_inv);
            else if (c < g.count)
                eval1(B, sk, E + cc / 2, g.widx0 + c, s_inv);
        }
    }
}

// Coarse group (step G = 8 or 16) whose start is a multiple of 16.  Width c
// reads S_G at 16t + off + cG + k, k < 16: SEG = 16/G segments of G positions,
// kept in a ring of SEG + 1 slots so each segment is loaded once; 2 (SEG + 1)
// widths per iteration keep every offset a compile-time constant.
template <int G, class Sink>
__device__ __forceinline__ void run_coarse_aligned(float2 *B, Sink &sk, const float *bt,
                                                   const Group &g, const float *s_inv) {
    constexpr int SEG = 16 / G;
    constexpr int NS = SEG + 1;
    constexpr int U = 2 * NS;
    constexpr int PV = G / 2;          // float2 per segment
    float2 ring[NS][PV];
    const float *b0 = bt + kPad * (g.off >> 4);
#pragma unroll
    for (int m = 0; m < SEG - 1; ++m) {
#pragma unroll
        for (int v = 0; v < G / 4; ++v) {
            const float4 f = *reinterpret_cast<const float4 *>(
                b0 + kPad * (m / SEG) + G * (m % SEG) + 4 * v);
            ring[m][2 * v] = make_float2(f.x, f.y);
            ring[m][2 * v + 1] = make_float2(f.z, f.w);
        }
    }
    for (int c0 = 0; c0 < g.count; c0 += U) {
        const float *bi = b0 + kPad * (c0 / SEG);
#pragma unroll
        for (int u = 0; u < U; u += 2) {
            const int c = c0 + u;
            if (c >= g.count) break;
            const bool two = c + 1 < g.count;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (h == 1 && !two) break;
                const int m = u + h + SEG - 1;           // segment to bring in
#pragma unroll
                for (int v = 0; v < G / 4; ++v) {
                    const float4 f = *reinterpret_cast<const float4 *>(
                        bi + kPad * (m / SEG) + G * (m % SEG) + 4 * v);
                    ring[m % NS][2 * v] = make_float2(f.x, f.y);
                    ring[m % NS][2 * v + 1] = make_float2(f.z, f.w);
                }
            }
            float2 Va[kX / 2], Vb[kX / 2];
#pragma unroll
            for (int j = 0; j < kX / 2; ++j) {
                Va[j] = ring[(u + j / PV) % NS][j % PV];
                Vb[j] = ring[(u + 1 + j / PV) % NS][j % PV];
            }
            if (two)
                eval2(B, sk, Va, Vb, g.widx0 + c, s_inv);
            else
                eval1(B, sk, Va, g.widx0 + c, s_inv);
        }
    }
}

// Any group, one width at a time with per-step loads (start not a multiple of
// 16, or the compact recovery pass).  The running sums see the same additions
// in the same order as in the unrolled paths, so the SNRs are bitwise equal.
template <class Sink>
__device__ __forceinline__ void run_generic(float2 *B, Sink &sk, const float *bt, const Group &g,
                                            int d, const float *s_inv) {
#pragma unroll 1
    for (int c = 0; c < g.count; ++c) {
        const int p0 = g.off + c * d;
        float2 V[kX / 2];
#pragma unroll
        for (int j = 0; j < kX / 2; ++j)
            V[j] = make_float2(bt[padr(p0 + 2 * j)], bt[padr(p0 + 2 * j + 1)]);
        eval1(B, sk, V, g.widx0 + c, s_inv);
    }
}

// Sum of the block sums of blocks b0 .. b1-1, Kahan-compensated in block order.
__device__ __forceinline__ float blocks_sum(const float *s_bs, int b0, int b1) {
    float sum = 0.f, comp = 0.f;
    for (int b = b0; b < b1; ++b) {
        const float y = __fsub_rn(s_bs[b], comp);
        const float t = __fadd_rn(sum, y);
        comp = __fsub_rn(__fsub_rn(t, sum), y);
        sum = t;
    }
    return sum;
}

// Sum of the first q samples of block b.
__device__ __forceinline__ float block_part(const float *s_y, int b, int q) {
    float part = 0.f;
    for (int i = 0; i < q; ++i) part = __fadd_rn(part, s_y[kPad * b + i]);
    return part;
}

// Start sums of a group for the thread's 16 samples (thread t, samples 16t+k):
// B_off(16t + k) = y[16t + k] + ... + y[16t + k + off - 1], taken as the sum
// of whole blocks between the two positions plus the partial sums inside the
// blocks at each end.
__device__ __forceinline__ void group_start(float2 *B, const float *s_y, const float *s_bs,
                                            int t, int off) {
    if (off == 0) {
#pragma unroll
        for (int j = 0; j < kX / 2; ++j) B[j] = make_float2(0.f, 0.f);
    } else if ((off & 15) == 0) {
        const int ta = t + (off >> 4);
        const float d = blocks_sum(s_bs, t, ta);
        const float *ya = s_y + kPad * ta;
        const float *y0 = s_y + kPad * t;
        float pa = 0.f, p0 = 0.f;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const float4 fa = *reinterpret_cast<const float4 *>(ya + 4 * v);
            const float4 f0 = *reinterpret_cast<const float4 *>(y0 + 4 * v);
            float2 r;
            r.x = __fadd_rn(d, __fsub_rn(pa, p0));
            pa = __fadd_rn(pa, fa.x); p0 = __fadd_rn(p0, f0.x);
            r.y = __fadd_rn(d, __fsub_rn(pa, p0));
            pa = __fadd_rn(pa, fa.y); p0 = __fadd_rn(p0, f0.y);
            B[2 * v] = r;
            r.x = __fadd_rn(d, __fsub_rn(pa, p0));
            pa = __fadd_rn(pa, fa.z); p0 = __fadd_rn(p0, f0.z);
            r.y = __fadd_rn(d, __fsub_rn(pa, p0));
            pa = __fadd_rn(pa, fa.w); p0 = __fadd_rn(p0, f0.w);
            B[2 * v + 1] = r;
        }
    } else {
#pragma unroll
        for (int j = 0; j < kX / 2; ++j) {
            float v2x, v2y;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int p = 16 * t + 2 * j + h, q = p + off;
                const float whole = blocks_sum(s_bs, p >> 4, q >> 4);
                const float v = __fadd_rn(whole, __fsub_rn(block_part(s_y, q >> 4, q & 15),
                                                           block_part(s_y, p >> 4, p & 15)));
                if (h == 0) v2x = v; else v2y = v;
            }
            B[j] = make_float2(v2x, v2y);
        }
    }
}

template <int G, class Sink>
__device__ __forceinline__ void run_group(float2 *B, Sink &sk, const float *sy_t,
                                          const float *sg_t, const Group &g, const float *s_inv) {
    const bool aligned = (g.off & 15) == 0;
    if (G > 1 && (g.flags & kGroupCoarse)) {
        if (aligned)
            run_coarse_aligned<(G > 1 ? G : 8)>(B, sk, sg_t, g, s_inv);
        else
            run_generic(B, sk, sg_t, g, G, s_inv);
    } else {
        if (aligned)
            run_fine_aligned(B, sk, sy_t, g, s_inv);
        else
            run_generic(B, sk, sy_t, g, 1, s_inv);
    }
}

// Compact evaluation of a group (recovery of the winning width).
template <int G, class Sink>
__device__ __forceinline__ void run_group_compact(float2 *B, Sink &sk, const float *sy_t,
                                                  const float *sg_t, const Group &g,
                                                  const float *s_inv) {
    if (G > 1 && (g.flags & kGroupCoarse))
        run_generic(B, sk, sg_t, g, G, s_inv);
    else
        run_generic(B, sk, sy_t, g, 1, s_inv);
}

template <int G>
__device__ __forceinline__ int group_step(const Group &g) {
    return (G > 1 && (g.flags & kGroupCoarse)) ? G : 1;
}

// One pass over the window's 16-position blocks: S_G[p] = y[p] + ... + y[p+G-1]
// (when G > 1; the first of a block by pairwise sums, the next 15 by sliding
// the window one sample), and per block b its sum s_bs[b] and the largest /
// smallest prefix C over its 16 positions (s_mx / s_mn, FP32, used only for
// bounds; C from an FP32 scan of the block sums).  Ends with a barrier.
template <int G>
__device__ void build_stats(const float *s_y, float *s_g, float *s_bs, float *s_mx, float *s_mn,
                            float *s_wt, int R) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
#pragma unroll 1
    for (int r = 0; r * kThreads < R; ++r) {
        const int c = r * kThreads + tid;
        float sum = 0.f, hi = 0.f, lo = 0.f;
        if (c < R) {
            float v[32];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4 f = *reinterpret_cast<const float4 *>(s_y + kPad * c + 4 * q);
                v[4 * q] = f.x; v[4 * q + 1] = f.y; v[4 * q + 2] = f.z; v[4 * q + 3] = f.w;
            }
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                if (q) { hi = fmaxf(hi, sum); lo = fminf(lo, sum); }
                sum = __fadd_rn(sum, v[q]);
            }
            if (G > 1) {
                if (c < R - 1) {
#pragma unroll
                    for (int q = 4; q < 8; ++q) {
                        const float4 f =
                            *reinterpret_cast<const float4 *>(s_y + kPad * (c + 1) + 4 * (q - 4));
                        v[4 * q] = f.x; v[4 * q + 1] = f.y; v[4 * q + 2] = f.z; v[4 * q + 3] = f.w;
                    }
                    float w[G];
#pragma unroll
                    for (int q = 0; q < G; ++q) w[q] = v[q];
#pragma unroll
                    for (int len = 1; len < G; len *= 2) {
#pragma unroll
                        for (int q = 0; q + len < G; q += 2 * len) w[q] = __fadd_rn(w[q], w[q + len]);
                    }
                    float o[16];
                    o[0] = w[0];
#pragma unroll
                    for (int q = 1; q < 16; ++q)
                        o[q] = __fadd_rn(__fsub_rn(o[q - 1], v[q - 1]), v[q - 1 + G]);
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        *reinterpret_cast<float4 *>(s_g + kPad * c + 4 * q) =
                            make_float4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
                } else {
#pragma unroll
                    for (int q = 0; q < 16; ++q) s_g[kPad * c + q] = -INFINITY;
                }
            }
            s_bs[c] = sum;
            s_mx[c] = hi;   // relative to the block start until the scan below
            s_mn[c] = lo;
        }
        // inclusive warp scan of the block sums (FP32, for bounds only)
        float x = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const float u = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += u;
        }
        if (lane == 31) s_wt[r * (kThreads / 32) + warp] = x;
        const float xe = __shfl_up_sync(0xffffffffu, x, 1);
        if (c < R) s_wt[3 * (kThreads / 32) + c] = lane ? xe : 0.f;   // exclusive in warp
    }
    __syncthreads();
#pragma unroll 1
    for (int c = tid; c < R; c += kThreads) {
        float before = 0.f;
        const int chunk = c >> 5;   // warp chunk of 32 blocks
        for (int w = 0; w < chunk; ++w) before += s_wt[w];
        const float P = before + s_wt[3 * (kThreads / 32) + c];   // C at the block start
        s_mx[c] += P;
        s_mn[c] += P;
    }
    __syncthreads();
}

// Per-range constants in shared memory: 1/sigma_w per eval index, the width
// of each eval index, and (candidate search) per group the blocks its bound
// looks at: the prefix maxima over blocks [t + a, t + b] of a unit t, read as
// the maximum of two windows of 2^k blocks, [t + a, ...) and [t + bk, ...),
// of the sparse max table (k = -1: a plain loop, for spans over 64 blocks),
// with the group's largest 1/sigma_w.  *s_kmax = the highest level any group
// reads.
__device__ __forceinline__ void load_range_consts(const RangeDesc &rd, int entry, float *s_inv,
                                                  uint16_t *s_ew, int4 *s_gb, Group *s_grp,
                                                  int *s_kmax, bool bounds) {
    const RangeProg &rp = rd.prog;
    for (int gi = threadIdx.x; gi < rp.n_groups; gi += kThreads) s_grp[gi] = rp.groups[gi];
    for (int q = threadIdx.x; q < rp.n_eval; q += kThreads)
        s_inv[q] = rd.inv_tab[(int64_t)entry * rp.n_eval + q];
    if (threadIdx.x == 0) *s_kmax = 0;
    __syncthreads();
    for (int gi = threadIdx.x; gi < rp.n_groups; gi += kThreads) {
        const Group g = s_grp[gi];
        const int d = (g.flags & kGroupCoarse) ? rp.G : 1;
        float mxv = 0.f;
        for (int c = 0; c < g.count; ++c) {
            s_ew[g.widx0 + c] = (uint16_t)(g.off + (c + 1) * d);
            if (bounds) mxv = fmaxf(mxv, rd.inv_tab[(int64_t)entry * rp.n_eval + g.widx0 + c]);
        }
        if (bounds) {
            const int a = (g.off + d) >> 4, b = (15 + g.off + g.count * d) >> 4;
            const int len = b - a + 1;
            int k = -1, bk = b;
            if (len <= 2 << kMaxLevel) {
                k = 31 - __clz(len);
                if (k > kMaxLevel) k = kMaxLevel;
                bk = b - (1 << k) + 1;
                atomicMax(s_kmax, k);
            }
            s_gb[gi] = make_int4(a, bk, k, __float_as_int(mxv));
        }
    }
}

template <int DT, int G, bool PLANE, bool MG>
__global__ void __launch_bounds__(kThreads, 512 / kThreads) detect_kernel(const __grid_constant__ Launch L) {
    using T = typename Elem<DT>::T;
    extern __shared__ __align__(16) unsigned char smem[];
    const int RM = L.R;
    uint64_t *s_bar = reinterpret_cast<uint64_t *>(smem);
    unsigned char *s_raw0 = smem + 16;
    float *s_y = reinterpret_cast<float *>(s_raw0 + 2 * L.raw_bytes);
    float *s_g = s_y + kPad * RM;
    float *s_bs = s_y + (G > 1 ? 2 : 1) * kPad * RM;
    float *s_mx = s_bs + RM;
    float *s_mn = s_mx + RM;
    float *s_st = s_mn + RM;                       // kMaxLevel levels of RM
    float *s_inv = s_st + kMaxLevel * RM;
    int4 *s_gb = reinterpret_cast<int4 *>(
        (reinterpret_cast<uintptr_t>(s_inv + L.max_eval) + 15) & ~(uintptr_t)15);
    uint16_t *s_ew = reinterpret_cast<uint16_t *>(s_gb + kMaxCodeGroups);
    __shared__ int s_kmax;
    __shared__ Group s_grp[kMaxCodeGroups];   // the range's width groups
    __shared__ float s_wt[3 * (kThreads / 32) + 3 * kThreads];

    const int tid = threadIdx.x;
    const int64_t n_tiles = L.n_tiles;
    const int64_t esz = (int64_t)sizeof(T);

    // all ranges of a launch agree on bulk copies (the host checks)
    const bool tma = L.rng[0].vec_ok != 0;
    if (tma) {
        if (tid == 0) {
            mbar_init(s_bar);
            mbar_init(s_bar + 1);
            fence_mbar_init();
        }
        __syncthreads();
    }
    auto range_of = [&](int64_t tile, int from) {
        int r = from;
        while (r + 1 < L.n_ranges && tile >= L.rng[r + 1].tile0) ++r;
        return r;
    };
    // bulk copy of tile `tile`'s window into raw buffer `buf` (thread 0 only)
    auto issue = [&](int64_t tile, int ri, int buf) {
        const RangeDesc &rd = L.rng[ri];
        const int64_t lt = tile - rd.tile0;
        const int64_t row = lt / rd.tiles_per_row;
        const int64_t t0 = (lt - row * rd.tiles_per_row) * (int64_t)kTile;
        const int64_t have = min((int64_t)rd.span, rd.n_samp - t0);
        const uint32_t nb = (uint32_t)((have * esz) & ~(int64_t)15);
        uint64_t *bar = s_bar + buf;
        fence_proxy_async();
        mbar_expect(bar, nb + L.extra_tx);
        if (nb) {
            const T *src = static_cast<const T *>(rd.data) + row * rd.stride + t0;
            bulk_load(s_raw0 + buf * L.raw_bytes, src, nb, bar);
        }
    };
    if (tma && tid == 0 && (int64_t)blockIdx.x < n_tiles)
        issue(blockIdx.x, range_of(blockIdx.x, 0), 0);

    int k = 0, ri = 0, cur_ri = -1;
    int64_t key = -1;   // (range, scope entry) whose constants are in shared memory
    int64_t row = 0, col = 0;   // the tile's row and tile column within its range
    int64_t step_rows = 0, step_cols = 0;   // gridDim.x tiles as rows + columns of the range
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++k) {
        const int buf = k & 1;
        ri = range_of(tile, ri);
        const RangeDesc &rd = L.rng[ri];
        const RangeProg &rp = rd.prog;
        const int R = rd.R;
        if (ri != cur_ri) {   // first tile of a range: divisions once
            const int64_t lt = tile - rd.tile0;
            row = lt / rd.tiles_per_row;
            col = lt - row * rd.tiles_per_row;
            step_rows = (int64_t)gridDim.x / rd.tiles_per_row;
            step_cols = (int64_t)gridDim.x - step_rows * rd.tiles_per_row;
            cur_ri = ri;
        } else {              // the next tile of this CTA: gridDim.x tiles on
            row += step_rows;
            col += step_cols;
            if (col >= rd.tiles_per_row) {
                col -= rd.tiles_per_row;
                ++row;
            }
        }
        const int64_t t0 = col * (int64_t)kTile;
        const int entry = rd.per_row ? (int)row : 0;
        const int64_t i0 = t0 + (int64_t)tid * kX;   // first start sample of this thread
        const T *rowp = static_cast<const T *>(rd.data) + row * rd.stride;

        if (tma) {
            // thread 0 waits for the copy; the barrier then orders every
            // thread's reads after it.  If the copy did not land in time the
            // whole CTA reports it, gives the copy (the only one in flight)
            // one more bounded wait, and leaves.
            const bool ok =
                tid != 0 || mbar_wait(s_bar + buf, (uint32_t)((k >> 1) & 1), L.wait_ns);
            if (__syncthreads_or(!ok)) {
                if (tid == 0) {
                    if (L.result) atomicExch(&L.result->status, (int)SPD_ERR_TIMEOUT);
                    mbar_wait(s_bar + buf, (uint32_t)((k >> 1) & 1), L.wait_ns);
                }
                return;
            }
        }

        const bool deg = rd.flags[entry] != 0;
        const float2 mu = rd.mu_tab[entry];
        const bool has_sc = rd.scale != nullptr;
        const float sc = has_sc ? rd.scale[row] : 1.f;
        const float of = (has_sc && rd.offset) ? rd.offset[row] : 0.f;
        const int have = (int)min((int64_t)rd.span, rd.n_samp - t0);   // window samples in the row
        const int nraw = tma ? (int)((((int64_t)have * esz) & ~(int64_t)15) / esz) : 0;
        const T *raw = reinterpret_cast<const T *>(s_raw0 + buf * L.raw_bytes);

        if (!deg) {
            const int64_t nk = ((int64_t)ri << 32) | (uint32_t)entry;
            if (nk != key) {
                load_range_consts(rd, entry, s_inv, s_ew, s_gb, s_grp, &s_kmax, !PLANE);
                key = nk;
            }
            // Stage centred samples; -inf past the row end and past the window.
            for (int q = tid; q < 4 * R; q += kThreads) {
                const int p = 4 * q;
                float x[4];
                if (p + 3 < nraw) {   // the common case: four copied samples
                    load4v<DT>(raw + p, x[0], x[1], x[2], x[3]);
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        if (has_sc) x[e] = fmaf(sc, x[e], of);
                        x[e] = __fsub_rn(__fsub_rn(x[e], mu.x), mu.y);
                    }
                    *reinterpret_cast<float4 *>(s_y + padr(p)) =
                        make_float4(x[0], x[1], x[2], x[3]);
                    continue;
                } else {
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        x[e] = (p + e < nraw)  ? Elem<DT>::cvt(raw[p + e])
                               : (p + e < have) ? Elem<DT>::cvt(rowp[t0 + p + e])
                                                : -INFINITY;
                }
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    if (p + e < have) {
                        if (has_sc) x[e] = fmaf(sc, x[e], of);
                        x[e] = __fsub_rn(__fsub_rn(x[e], mu.x), mu.y);
                    } else {
                        x[e] = -INFINITY;
                    }
                }
                *reinterpret_cast<float4 *>(s_y + padr(p)) = make_float4(x[0], x[1], x[2], x[3]);
            }
        }
        __syncthreads();
        // the raw buffer is free again: prefetch the window of the tile after
        if (tma && tid == 0 && tile + gridDim.x < n_tiles)
            issue(tile + gridDim.x, range_of(tile + gridDim.x, ri), buf ^ 1);

        if (deg) {
            if (PLANE) {
                for (int q = 0; q < kX; ++q) {
                    if (i0 + q < rd.n_samp) {
                        L.snr_out[row * L.out_stride + i0 + q] = __int_as_float(0x7fc00000);
                        L.width_out[row * L.out_stride + i0 + q] = 0;
                    }
                }
            }
            continue;   // uniform across the CTA
        }

        build_stats<G>(s_y, s_g, s_bs, s_mx, s_mn, s_wt, R);   // ends with a barrier

        const float *sy_t = s_y + kPad * tid;
        const float *sg_t = s_g + kPad * tid;
        float2 B[kX / 2];
        float snr[kX];
        int wdt[kX];
        if (PLANE) {
            float obest[MG ? kX : 1];
            int ogrp[MG ? kX : 1];
            if (MG) {
#pragma unroll
                for (int q = 0; q < kX; ++q) { obest[q] = -INFINITY; ogrp[q] = 0; }
            }
            PackSink sk;
            float *best = sk.best;
#pragma unroll
            for (int q = 0; q < kX; ++q) best[q] = -INFINITY;
            int cur = 0;   // block of 64 eval indices being packed
            for (int gi = 0; gi < rp.n_groups; ++gi) {
                const Group g = s_grp[gi];
                if (MG && (g.widx0 >> 6) != cur) {
                    // blocks of 64 widths: a later block wins only with a larger
                    // value (its code bits say nothing about earlier blocks)
#pragma unroll
                    for (int q = 0; q < kX; ++q) {
                        if (trunc17(best[q]) > trunc17(obest[q]) || obest[q] != obest[q]) {
                            obest[q] = best[q];
                            ogrp[q] = cur;
                        }
                        best[q] = -INFINITY;
                    }
                    cur = g.widx0 >> 6;
                }
                group_start(B, s_y, s_bs, tid, g.off);
                run_group<G>(B, sk, sy_t, sg_t, g, s_inv);
            }
            if (MG) {
#pragma unroll
                for (int q = 0; q < kX; ++q)
                    if (trunc17(best[q]) > trunc17(obest[q]) || obest[q] != obest[q]) {
                        obest[q] = best[q];
                        ogrp[q] = cur;
                    }
            }
#pragma unroll
            for (int q = 0; q < kX; ++q) {
                const float bv = MG ? obest[q] : best[q];
                const uint32_t bits = __float_as_uint(bv);
                const int wi = (MG ? ogrp[q] : 0) * 64 + (63 - (int)(bits & 63u));
                snr[q] = __uint_as_float(bits & 0xFFFFFFC0u);
                wdt[q] = (wi < rp.n_eval) ? (int)s_ew[wi] : 0;
            }
            float *so = L.snr_out + row * L.out_stride;
            uint16_t *wo = L.width_out + row * L.out_stride;
            const bool full = i0 + kX <= rd.n_samp;
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
                for (int q = 0; q < kX; ++q) {
                    if (i0 + q < rd.n_samp) {
                        so[i0 + q] = snr[q];
                        wo[i0 + q] = (uint16_t)wdt[q];
                    }
                }
            }
            __syncthreads();   // shared arrays are rewritten by the next tile
            continue;
        }

    }
}

template <int DT, int G>
cudaError_t launch_dg(const Launch &L, bool plane_out, bool mg, size_t smem, int ctas_per_sm,
                      cudaStream_t s) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (!plane_out) return cudaErrorInvalidValue;   // candidates: the search kernel
    void (*k)(const Launch) = mg ? detect_kernel<DT, G, true, true> : detect_kernel<DT, G, true, false>;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if (ctas_per_sm > 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
    const int64_t grid = L.n_tiles < (int64_t)sms * per_sm ? L.n_tiles : (int64_t)sms * per_sm;
    k<<<(unsigned)grid, kThreads, smem, s>>>(L);
    return cudaGetLastError();
}

}  // namespace

template <int DT>
cudaError_t launch_detect_dt(const Launch &L, int G, bool plane_out, bool multi_block,
                             size_t smem, int ctas_per_sm, cudaStream_t s) {
    switch (G) {
        case 8: return launch_dg<DT, 8>(L, plane_out, multi_block, smem, ctas_per_sm, s);
        case 16: return launch_dg<DT, 16>(L, plane_out, multi_block, smem, ctas_per_sm, s);
        default: return launch_dg<DT, 1>(L, plane_out, multi_block, smem, ctas_per_sm, s);
    }
}

}  // namespace spd
