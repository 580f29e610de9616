// spd_msd.cu -- step (a): mean and standard deviation of the DM x time plane
// (Sec. 2.1).  Two kernels, as the paper splits them:
//   msd_partial_kernel: every block reduces one equal-sized unit of a row
//     (kMsdUnit samples) to (n, T, S).  Each thread applies Eq. 1 to groups of
//     four consecutive samples and Eq. 2 to fold each group into its running
//     (n, T, S); lanes, then warps, are folded with Eq. 2.  FP32 throughout,
//     with T carried as an unevaluated hi + lo pair (compensated summation).
//   msd_merge_*: Eq. 2 over the unit partials in FP64 in a fixed tree order
//     (deterministic), giving mu = T/n and sigma = sqrt(S/n) (population sd).
// Plus the per-width constant kernel of step (c): 1/sigma_w from Eq. 4 / 5.
#include "spd_internal.cuh"

#include <math.h>

namespace spd {

namespace {

// Running (n, T, S) of one thread in FP32; T = Th + Tl.
struct Acc {
    float m, Th, Tl, S, lo, hi;

    __device__ __forceinline__ Acc()
        : m(0.f), Th(0.f), Tl(0.f), S(0.f), lo(INFINITY), hi(-INFINITY) {}

    __device__ __forceinline__ void range4(float a, float b, float c, float d) {
        lo = fminf(lo, fminf(fminf(a, b), fminf(c, d)));
        hi = fmaxf(hi, fmaxf(fmaxf(a, b), fmaxf(c, d)));
    }

    // TwoSum: Th + v exactly as (Th, error) -> error folded into Tl.
    __device__ __forceinline__ void add_T(float v) {
        const float s = Th + v;
        const float bb = s - Th;
        const float e = (Th - (s - bb)) + (v - bb);
        Th = s;
        Tl += e;
    }

    // Eq. 2 with the second set holding n = 4 samples of sum tb and S sb.
    __device__ __forceinline__ void fold4(float tb, float sb) {
        if (m == 0.f) {
            Th = tb; Tl = 0.f; S = sb; m = 4.f;
            return;
        }
        const float ta = Th + Tl;
        const float q = __fdividef(1.f, m * (m + 4.f));
        const float f = (4.f * (m + 4.f) * q) * ta - tb;         // (n/m) T_a - T_b
        S += sb + (0.25f * m * m * q) * f * f;                   // m/(n(m+n)) (...)^2
        add_T(tb);
        m += 4.f;
    }

    // Eq. 1 over four consecutive samples (j = 1..4), then fold with Eq. 2.
    __device__ __forceinline__ void add4(float a, float b, float c, float d) {
        const float t2 = a + b;
        const float d2 = fmaf(2.f, b, -t2);
        float s = 0.5f * d2 * d2;
        const float t3 = t2 + c;
        const float d3 = fmaf(3.f, c, -t3);
        s = fmaf(d3 * d3, 1.f / 6.f, s);
        const float t4 = t3 + d;
        const float d4 = fmaf(4.f, d, -t4);
        s = fmaf(d4 * d4, 1.f / 12.f, s);
        fold4(t4, s);
    }

    // Eq. 1 for a single further sample x_j, j = m + 1.
    __device__ __forceinline__ void add1(float x) {
        lo = fminf(lo, x);
        hi = fmaxf(hi, x);
        const float j = m + 1.f;
        add_T(x);
        if (j > 1.f) {
            const float d = fmaf(j, x, -(Th + Tl));
            S += d * d / (j * (j - 1.f));
        }
        m = j;
    }

    // Eq. 2 for two arbitrary sets (general m, n).
    __device__ __forceinline__ void merge(float mb, float Thb, float Tlb, float Sb) {
        if (mb == 0.f) return;
        if (m == 0.f) {
            m = mb; Th = Thb; Tl = Tlb; S = Sb;
            return;
        }
        const float ta = Th + Tl, tb = Thb + Tlb;
        const float f = (mb / m) * ta - tb;
        S = S + Sb + (m / (mb * (m + mb))) * f * f;
        const float s = Th + Thb;
        const float bb = s - Th;
        const float e = (Th - (s - bb)) + (Thb - bb);
        Th = s;
        Tl = Tl + Tlb + e;
        m += mb;
    }

    __device__ __forceinline__ void merge_down(int off) {
        const float mb = __shfl_down_sync(0xffffffffu, m, off);
        const float th = __shfl_down_sync(0xffffffffu, Th, off);
        const float tl = __shfl_down_sync(0xffffffffu, Tl, off);
        const float sb = __shfl_down_sync(0xffffffffu, S, off);
        lo = fminf(lo, __shfl_down_sync(0xffffffffu, lo, off));
        hi = fmaxf(hi, __shfl_down_sync(0xffffffffu, hi, off));
        merge(mb, th, tl, sb);
    }
};

template <int DT>
__device__ __forceinline__ void load4(const typename Elem<DT>::T *p, float &a, float &b,
                                      float &c, float &d);

template <>
__device__ __forceinline__ void load4<SPD_F32>(const float *p, float &a, float &b, float &c,
                                               float &d) {
    const float4 v = __ldcs(reinterpret_cast<const float4 *>(p));
    a = v.x; b = v.y; c = v.z; d = v.w;
}

template <>
__device__ __forceinline__ void load4<SPD_F16>(const __half *p, float &a, float &b, float &c,
                                               float &d) {
    const uint2 v = __ldcs(reinterpret_cast<const uint2 *>(p));
    const float2 lo = __half22float2(*reinterpret_cast<const __half2 *>(&v.x));
    const float2 hi = __half22float2(*reinterpret_cast<const __half2 *>(&v.y));
    a = lo.x; b = lo.y; c = hi.x; d = hi.y;
}

template <>
__device__ __forceinline__ void load4<SPD_BF16>(const __nv_bfloat16 *p, float &a, float &b,
                                                float &c, float &d) {
    const uint2 v = __ldcs(reinterpret_cast<const uint2 *>(p));
    const float2 lo = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&v.x));
    const float2 hi = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&v.y));
    a = lo.x; b = lo.y; c = hi.x; d = hi.y;
}

template <int DT>
__global__ void __launch_bounds__(kMsdThreads) msd_partial_kernel(const MsdArgs a) {
    using T = typename Elem<DT>::T;
    const int tid = threadIdx.x;
    const int64_t unit = blockIdx.x;
    const int64_t row = unit / a.units_per_row;
    const int64_t t_begin = (unit - row * a.units_per_row) * kMsdUnit;
    const int64_t len = min((int64_t)kMsdUnit, a.n_samp - t_begin);
    const T *p = static_cast<const T *>(a.data) + row * a.stride + t_begin;
    const bool has_sc = a.scale != nullptr;
    const float sc = has_sc ? a.scale[row] : 1.f;
    const float of = (has_sc && a.offset) ? a.offset[row] : 0.f;

    Acc acc;
    const int64_t ngrp = len >> 2;
    for (int64_t g = tid; g < ngrp; g += kMsdThreads) {
        float x0, x1, x2, x3;
        if (a.vec_ok) {
            load4<DT>(p + 4 * g, x0, x1, x2, x3);
        } else {
            x0 = Elem<DT>::cvt(p[4 * g]);
            x1 = Elem<DT>::cvt(p[4 * g + 1]);
            x2 = Elem<DT>::cvt(p[4 * g + 2]);
            x3 = Elem<DT>::cvt(p[4 * g + 3]);
        }
        if (has_sc) {
            x0 = fmaf(sc, x0, of); x1 = fmaf(sc, x1, of);
            x2 = fmaf(sc, x2, of); x3 = fmaf(sc, x3, of);
        }
        acc.range4(x0, x1, x2, x3);
        acc.add4(x0, x1, x2, x3);
    }
    for (int64_t t = 4 * ngrp + tid; t < len; t += kMsdThreads) {
        float x = Elem<DT>::cvt(p[t]);
        if (has_sc) x = fmaf(sc, x, of);
        acc.add1(x);
    }

    // Eq. 2 across lanes (fixed pairing), then across the block's warps.
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc.merge_down(off);
    __shared__ float4 s_w[kMsdThreads / 32];
    __shared__ float2 s_r[kMsdThreads / 32];
    const int lane = tid & 31, warp = tid >> 5;
    if (lane == 0) {
        s_w[warp] = make_float4(acc.m, acc.Th, acc.Tl, acc.S);
        s_r[warp] = make_float2(acc.lo, acc.hi);
    }
    __syncthreads();
    if (warp == 0) {
        Acc b;
        if (lane < kMsdThreads / 32) {
            const float4 v = s_w[lane];
            b.m = v.x; b.Th = v.y; b.Tl = v.z; b.S = v.w;
            b.lo = s_r[lane].x; b.hi = s_r[lane].y;
        }
#pragma unroll
        for (int off = 4; off > 0; off >>= 1) b.merge_down(off);
        if (lane == 0) {
            MsdPart out;
            out.n = (double)b.m;
            out.T = (double)b.Th + (double)b.Tl;
            out.S = (double)b.S;
            out.lo = (double)b.lo;
            out.hi = (double)b.hi;
            a.parts[unit] = out;
        }
    }
}

// Eq. 2 in FP64, the paper's form.
__device__ __forceinline__ void dmerge(MsdPart &a, const MsdPart &b) {
    if (b.n == 0.0) return;
    if (a.n == 0.0) { a = b; return; }
    a.lo = fmin(a.lo, b.lo);
    a.hi = fmax(a.hi, b.hi);
    const double d = (b.n / a.n) * a.T - b.T;
    a.S = a.S + b.S + a.n / (b.n * (a.n + b.n)) * d * d;
    a.T = a.T + b.T;
    a.n = a.n + b.n;
}

// Block-wide Eq. 2 over parts[lo, hi): thread t folds lo+t, lo+t+256, ... in
// order, then a halving tree in shared memory.  Result valid in thread 0.
__device__ MsdPart block_merge(const MsdPart *parts, int64_t lo, int64_t hi) {
    __shared__ MsdPart s_p[kMsdThreads];
    MsdPart acc{0.0, 0.0, 0.0, 0.0, 0.0};
    for (int64_t k = lo + threadIdx.x; k < hi; k += kMsdThreads) dmerge(acc, parts[k]);
    s_p[threadIdx.x] = acc;
    __syncthreads();
    for (int s = kMsdThreads / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) dmerge(s_p[threadIdx.x], s_p[threadIdx.x + s]);
        __syncthreads();
    }
    return s_p[0];
}

__device__ void write_msd(spd_msd_stats *o, const MsdPart &p) {
    spd_msd_stats r;
    r.n = (int64_t)p.n;
    r.nmax = 0;
    r.sd_nmax = 0.0;
    if (p.n > 0.0) {
        r.mean = p.T / p.n;
        r.sd = p.lo == p.hi ? 0.0 : sqrt(p.S / p.n);
    } else {
        r.mean = nan("");
        r.sd = nan("");
    }
    const bool ok = p.n > 0.0 && isfinite(r.mean) && isfinite(r.sd) && r.sd > 0.0;
    r.status = ok ? SPD_OK : SPD_ERR_DEGENERATE_SIGMA;
    *o = r;
}

__global__ void __launch_bounds__(kMsdThreads) msd_merge_l1_kernel(const MsdPart *parts,
                                                                   int64_t n_parts, int64_t per,
                                                                   MsdPart *scratch) {
    const int64_t lo = blockIdx.x * per;
    const int64_t hi = min(n_parts, lo + per);
    const MsdPart r = block_merge(parts, lo, hi);
    if (threadIdx.x == 0) scratch[blockIdx.x] = r;
}

__global__ void __launch_bounds__(kMsdThreads) msd_merge_final_kernel(const MsdPart *scratch,
                                                                      int n, spd_msd_stats *out) {
    const MsdPart r = block_merge(scratch, 0, n);
    if (threadIdx.x == 0) write_msd(out, r);
}

__global__ void __launch_bounds__(kMsdThreads) msd_merge_rows_kernel(const MsdPart *parts,
                                                                     int64_t n_dm, int64_t upr,
                                                                     spd_msd_stats *out) {
    const int64_t r = blockIdx.x * (int64_t)kMsdThreads + threadIdx.x;
    if (r >= n_dm) return;
    MsdPart acc{0.0, 0.0, 0.0, 0.0, 0.0};
    for (int64_t u = 0; u < upr; ++u) dmerge(acc, parts[r * upr + u]);
    write_msd(out + r, acc);
}

// Width of eval index k: member k - widx0 of the group holding k.
__device__ __forceinline__ int eval_width(const RangeProg &prog, int k) {
    for (int gi = 0; gi < prog.n_groups; ++gi) {
        const Group g = prog.groups[gi];
        if (k >= g.widx0 && k < g.widx0 + g.count) {
            const int d = (g.flags & kGroupCoarse) ? prog.G : 1;
            return g.off + (k - g.widx0 + 1) * d;
        }
    }
    return 0;
}

// Step (c) constants: per scope entry e and eval index k, 1/sigma_w in FP32
// (sigma_w in FP64 from Eq. 4 or Eq. 5), and the mean split as hi + lo FP32.
__global__ void __launch_bounds__(256) consts_kernel(const ConstArgs a,
                                                     const __grid_constant__ RangeProg prog) {
    const int e = blockIdx.x;
    const spd_msd_stats m = a.msd[e];
    bool deg = m.status != SPD_OK || !(m.sd > 0.0) || !isfinite(m.sd) || !isfinite(m.mean);
    // Eq. 5 uses the Nmax at which sigma_Nmax was measured (recorded in the MSD).
    const double nm = (double)m.nmax;
    if (a.sigma_mode != SPD_SIGMA_SQRTN && (m.nmax < 2 || !(m.sd_nmax > 0.0) || !isfinite(m.sd_nmax)))
        deg = true;
    for (int k = threadIdx.x; k < prog.n_eval; k += blockDim.x) {
        const double w = (double)eval_width(prog, k);
        double sw = sqrt(w) * m.sd;
        if (a.sigma_mode == SPD_SIGMA_LINEAR)
            sw += (w - 1.0) * m.sd_nmax / (nm - 1.0);
        else if (a.sigma_mode == SPD_SIGMA_LINEAR_EXCESS)
            sw += (w - 1.0) * (m.sd_nmax - sqrt(nm) * m.sd) / (nm - 1.0);
        const bool bad = !(sw > 0.0) || !isfinite(sw);
        // a NaN 1/sigma makes every SNR of that width NaN, which no max keeps
        a.inv_tab[(int64_t)e * prog.n_eval + k] =
            (a.skip_w1 && k == 0) ? __int_as_float(0x7fc00000) : bad ? 0.f : (float)(1.0 / sw);
        if (bad) deg = true;
    }
    deg = __syncthreads_or(deg);
    if (threadIdx.x == 0) {
        const float hi = (float)m.mean;
        const float lo = (float)(m.mean - (double)hi);
        a.mu_tab[e] = make_float2(hi, lo);
        a.flags[e] = deg ? 1 : 0;
        if (deg && a.result) atomicExch(&a.result->status, (int)SPD_ERR_DEGENERATE_SIGMA);
    }
}

// ----------------------------------------------------- sigma_Nmax (Eq. 5)

constexpr int kNmaxTile = 4096;        // start samples of one tile
constexpr int kNmaxPer = kNmaxTile / kMsdThreads;   // 16 consecutive starts per thread
constexpr int kNmaxTilesPerCta = 8;    // consecutive tiles of one row per CTA (one partial)

// Sec. 2.2, Eq. 5 needs sigma_Nmax, the measured sd of the boxcar series
// B_Nmax(i) = x[i] + ... + x[i+Nmax-1] over full windows.  Each CTA walks up
// to kNmaxTilesPerCta consecutive tiles of one row; per tile it stages the
// centred samples plus an (Nmax - 1)-sample halo and forms B for its 16
// consecutive starts per thread (whole-block sums plus partial sums for the
// first start, then sliding one sample), adding them with Eq. 1 to the
// thread's running (n, T, S).  At the end Eq. 2 merges across lanes and warps
// into the CTA's one partial.  The sd does not depend on the centring.
template <int DT>
__global__ void __launch_bounds__(kMsdThreads) nmax_partial_kernel(const NmaxArgs a) {
    using T = typename Elem<DT>::T;
    // centred samples, 16 positions in 20 words (lane t reading 16t + k with
    // 128-bit loads hits distinct banks within each quarter warp)
    extern __shared__ __align__(16) float s_y[];   // [nb * 20]
    float *s_bs = s_y + 20 * a.nb;                 // [nb] block sums
    const int tid = threadIdx.x;
    const int64_t row = blockIdx.x / a.tiles_per_row;   // tiles_per_row: partials per row
    const int64_t part = blockIdx.x - row * a.tiles_per_row;
    const int64_t tiles_in_row = (a.n_samp + kNmaxTile - 1) / kNmaxTile;
    const int64_t tl0 = part * kNmaxTilesPerCta;
    const int64_t tl1 = min(tl0 + kNmaxTilesPerCta, tiles_in_row);
    const int entry = a.per_row ? (int)row : 0;
    const double mu = a.msd[entry].mean;
    const float mh = (float)mu, ml = (float)(mu - (double)mh);
    const T *rp = static_cast<const T *>(a.data) + row * a.stride;
    const bool has_sc = a.scale != nullptr;
    const float sc = has_sc ? a.scale[row] : 1.f;
    const float of = (has_sc && a.offset) ? a.offset[row] : 0.f;
    const int nmax = a.nmax;
    const int p0 = tid * kNmaxPer;                 // first start of this thread (tile-local)
    const int qe = p0 + nmax;
    Acc acc;
    for (int64_t tl = tl0; tl < tl1; ++tl) {
        const int64_t t0 = tl * (int64_t)kNmaxTile;
        __syncthreads();   // the previous tile's reads of s_y / s_bs are done
        for (int q4 = tid; q4 < 4 * a.nb; q4 += kMsdThreads) {
            const int p = 4 * q4;
            float x[4];
            if (a.vec_ok && t0 + p + 3 < a.n_samp) {
                load4<DT>(rp + t0 + p, x[0], x[1], x[2], x[3]);
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    x[e] = t0 + p + e < a.n_samp ? Elem<DT>::cvt(rp[t0 + p + e]) : 0.f;
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if (has_sc) x[e] = fmaf(sc, x[e], of);
                x[e] = t0 + p + e < a.n_samp ? (x[e] - mh) - ml : 0.f;
            }
            *reinterpret_cast<float4 *>(s_y + (p & 15) + 20 * (p >> 4)) =
                make_float4(x[0], x[1], x[2], x[3]);
        }
        __syncthreads();
        for (int b = tid; b < a.nb; b += kMsdThreads) {
            float sum = 0.f;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4 f = *reinterpret_cast<const float4 *>(s_y + 20 * b + 4 * q);
                sum += (f.x + f.y) + (f.z + f.w);
            }
            s_bs[b] = sum;
        }
        __syncthreads();

        // B at p0: whole blocks from p0 to p0 + nmax (Kahan), plus the partial
        // block at the end (p0 is a multiple of 16)
        float whole = 0.f, comp = 0.f;
        for (int b = p0 >> 4; b < (qe >> 4); ++b) {
            const float y = s_bs[b] - comp;
            const float t = whole + y;
            comp = (t - whole) - y;
            whole = t;
        }
        float tail = 0.f;
        for (int q = (qe & ~15); q < qe; ++q) tail += s_y[(q & 15) + 20 * (q >> 4)];
        float B = whole + tail;
        // the thread's 16 samples and the 16 that enter the window as it slides
        float lo[16], hi[16];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 f = *reinterpret_cast<const float4 *>(s_y + 20 * tid + 4 * q);
            lo[4 * q] = f.x; lo[4 * q + 1] = f.y; lo[4 * q + 2] = f.z; lo[4 * q + 3] = f.w;
        }
        if ((nmax & 15) == 0) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4 f =
                    *reinterpret_cast<const float4 *>(s_y + 20 * (tid + (nmax >> 4)) + 4 * q);
                hi[4 * q] = f.x; hi[4 * q + 1] = f.y; hi[4 * q + 2] = f.z; hi[4 * q + 3] = f.w;
            }
        } else {
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const int q = p0 + k + nmax;
                hi[k] = s_y[(q & 15) + 20 * (q >> 4)];
            }
        }
        float bw[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            bw[k] = B;
            B = (B - lo[k]) + hi[k];
        }
        // starts t0 + p0 + k are full windows while t0 + p0 + k + nmax <= n_samp
        const int64_t nvalid = a.n_samp - nmax - (t0 + p0) + 1;
        if (nvalid >= 16) {
#pragma unroll
            for (int k = 0; k < 16; k += 4) acc.add4(bw[k], bw[k + 1], bw[k + 2], bw[k + 3]);
        } else {
#pragma unroll
            for (int k = 0; k < 16; ++k)
                if (k < nvalid) acc.add1(bw[k]);
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc.merge_down(off);
    __shared__ float4 s_w[kMsdThreads / 32];
    const int lane = tid & 31, warp = tid >> 5;
    if (lane == 0) s_w[warp] = make_float4(acc.m, acc.Th, acc.Tl, acc.S);
    __syncthreads();
    if (warp == 0) {
        Acc b;
        if (lane < kMsdThreads / 32) {
            const float4 v = s_w[lane];
            b.m = v.x; b.Th = v.y; b.Tl = v.z; b.S = v.w;
        }
#pragma unroll
        for (int off = 4; off > 0; off >>= 1) b.merge_down(off);
        if (lane == 0) {
            MsdPart out;
            out.n = (double)b.m;
            out.T = (double)b.Th + (double)b.Tl;
            out.S = (double)b.S;
            out.lo = out.hi = 0.0;
            a.parts[blockIdx.x] = out;
        }
    }
}

__device__ void write_nmax(spd_msd_stats *o, const MsdPart &p, int nmax) {
    o->nmax = nmax;
    o->sd_nmax = p.n > 0.0 ? sqrt(p.S / p.n) : 0.0;
}

__global__ void __launch_bounds__(kMsdThreads) nmax_merge_final_kernel(const MsdPart *scratch,
                                                                       int n, int nmax,
                                                                       spd_msd_stats *out) {
    const MsdPart r = block_merge(scratch, 0, n);
    if (threadIdx.x == 0) write_nmax(out, r, nmax);
}

__global__ void __launch_bounds__(kMsdThreads) nmax_merge_rows_kernel(const MsdPart *parts,
                                                                      int64_t n_dm, int64_t tpr,
                                                                      int nmax, spd_msd_stats *out) {
    const int64_t r = blockIdx.x * (int64_t)kMsdThreads + threadIdx.x;
    if (r >= n_dm) return;
    MsdPart acc{0.0, 0.0, 0.0, 0.0, 0.0};
    for (int64_t u = 0; u < tpr; ++u) dmerge(acc, parts[r * tpr + u]);
    write_nmax(out + r, acc, nmax);
}

// ------------------------------------------------------------ shard partials

// One block: fold n parts into one with the block tree (as the final merge).
__global__ void __launch_bounds__(kMsdThreads) fold_final_kernel(const MsdPart *scratch, int n,
                                                                 MsdPart *out) {
    const MsdPart r = block_merge(scratch, 0, n);
    if (threadIdx.x == 0) *out = r;
}

// Shard partials merged with Eq. 2 in shard order (one thread: the order, and
// so every bit of the result, is the same on every rank).  what = 0: mean and
// sd into out; what = 1: sd_nmax of the B_Nmax series.
__global__ void merge_shards_kernel(const MsdPart *parts, int n, int what, int nmax,
                                    spd_msd_stats *out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    MsdPart acc{0.0, 0.0, 0.0, 0.0, 0.0};
    for (int k = 0; k < n; ++k) dmerge(acc, parts[k]);
    if (what == 0)
        write_msd(out, acc);
    else
        write_nmax(out, acc, nmax);
}

// ------------------------------------------------------------ streaming MSD

// Running MSD of a stream: state[e] holds (n, T, S, min, max) of every sample
// pushed so far for scope entry e.  The new chunk's unit partials are added
// with Eq. 2 (state first, then the chunk in unit order) and the result is
// written back and as spd_msd_stats.  Global scope: one CTA; per row: one
// thread per row.
__global__ void __launch_bounds__(kMsdThreads) stream_msd_global_kernel(const MsdPart *parts,
                                                                       int64_t n_parts,
                                                                       MsdPart *state,
                                                                       spd_msd_stats *out) {
    const MsdPart c = block_merge(parts, 0, n_parts);
    if (threadIdx.x == 0) {
        MsdPart s = *state;
        dmerge(s, c);
        *state = s;
        write_msd(out, s);
    }
}

__global__ void __launch_bounds__(kMsdThreads) stream_msd_rows_kernel(const MsdPart *parts,
                                                                     int64_t n_dm, int64_t upr,
                                                                     MsdPart *state,
                                                                     spd_msd_stats *out) {
    const int64_t r = blockIdx.x * (int64_t)kMsdThreads + threadIdx.x;
    if (r >= n_dm) return;
    MsdPart s = state[r];
    for (int64_t u = 0; u < upr; ++u) dmerge(s, parts[r * upr + u]);
    state[r] = s;
    write_msd(out + r, s);
}

__global__ void zero_parts_kernel(MsdPart *p, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) p[i] = MsdPart{0.0, 0.0, 0.0, 0.0, 0.0};
}

}  // namespace

cudaError_t launch_msd_partial(const MsdArgs &a, int dtype, cudaStream_t s) {
    const int64_t units = a.n_dm * a.units_per_row;
    if (units <= 0) return cudaSuccess;
    const dim3 grid((unsigned)units);
    switch (dtype) {
        case SPD_F32: msd_partial_kernel<SPD_F32><<<grid, kMsdThreads, 0, s>>>(a); break;
        case SPD_F16: msd_partial_kernel<SPD_F16><<<grid, kMsdThreads, 0, s>>>(a); break;
        default: msd_partial_kernel<SPD_BF16><<<grid, kMsdThreads, 0, s>>>(a); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_msd_merge(const MsdPart *parts, int64_t n_dm, int64_t upr, int64_t n_samp,
                             int per_row, MsdPart *scratch, int n_scratch, spd_msd_stats *out,
                             cudaStream_t s) {
    (void)n_samp;
    if (per_row) {
        const unsigned g = (unsigned)((n_dm + kMsdThreads - 1) / kMsdThreads);
        msd_merge_rows_kernel<<<g, kMsdThreads, 0, s>>>(parts, n_dm, upr, out);
        return cudaGetLastError();
    }
    const int64_t n_parts = n_dm * upr;
    int64_t n1 = (n_parts + kMsdThreads - 1) / kMsdThreads;
    if (n1 > n_scratch) n1 = n_scratch;
    if (n1 < 1) n1 = 1;
    const int64_t per = (n_parts + n1 - 1) / n1;
    msd_merge_l1_kernel<<<(unsigned)n1, kMsdThreads, 0, s>>>(parts, n_parts, per, scratch);
    msd_merge_final_kernel<<<1, kMsdThreads, 0, s>>>(scratch, (int)n1, out);
    return cudaGetLastError();
}

int nmax_blocks(int nmax) { return (kNmaxTile + nmax + 15) / 16 + 1; }
int64_t nmax_tiles_per_row(int64_t n_samp) {
    const int64_t tiles = (n_samp + kNmaxTile - 1) / kNmaxTile;
    return (tiles + kNmaxTilesPerCta - 1) / kNmaxTilesPerCta;   // partials per row
}

cudaError_t launch_nmax_partial(const NmaxArgs &a, int dtype, cudaStream_t s) {
    const int64_t tiles = a.n_dm * a.tiles_per_row;
    if (tiles <= 0) return cudaSuccess;
    const size_t smem = (size_t)a.nb * 21 * sizeof(float);
    switch (dtype) {
        case SPD_F32: nmax_partial_kernel<SPD_F32><<<(unsigned)tiles, kMsdThreads, smem, s>>>(a); break;
        case SPD_F16: nmax_partial_kernel<SPD_F16><<<(unsigned)tiles, kMsdThreads, smem, s>>>(a); break;
        default: nmax_partial_kernel<SPD_BF16><<<(unsigned)tiles, kMsdThreads, smem, s>>>(a); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_fold_parts(const MsdPart *parts, int64_t n_parts, MsdPart *scratch,
                              int n_scratch, MsdPart *out, cudaStream_t s) {
    int64_t n1 = (n_parts + kMsdThreads - 1) / kMsdThreads;
    if (n1 > n_scratch) n1 = n_scratch;
    if (n1 < 1) n1 = 1;
    const int64_t per = (n_parts + n1 - 1) / n1;
    msd_merge_l1_kernel<<<(unsigned)n1, kMsdThreads, 0, s>>>(parts, n_parts, per, scratch);
    fold_final_kernel<<<1, kMsdThreads, 0, s>>>(scratch, (int)n1, out);
    return cudaGetLastError();
}

cudaError_t launch_merge_shards(const MsdPart *parts, int n, int what, int nmax,
                                spd_msd_stats *out, cudaStream_t s) {
    merge_shards_kernel<<<1, 32, 0, s>>>(parts, n, what, nmax, out);
    return cudaGetLastError();
}

cudaError_t launch_nmax(const NmaxArgs &a, int dtype, MsdPart *scratch, int n_scratch,
                        spd_msd_stats *out, cudaStream_t s) {
    const int64_t tiles = a.n_dm * a.tiles_per_row;
    {
        cudaError_t e = launch_nmax_partial(a, dtype, s);
        if (e != cudaSuccess) return e;
    }
    if (a.per_row) {
        const unsigned g = (unsigned)((a.n_dm + kMsdThreads - 1) / kMsdThreads);
        nmax_merge_rows_kernel<<<g, kMsdThreads, 0, s>>>(a.parts, a.n_dm, a.tiles_per_row, a.nmax, out);
        return cudaGetLastError();
    }
    int64_t n1 = (tiles + kMsdThreads - 1) / kMsdThreads;
    if (n1 > n_scratch) n1 = n_scratch;
    if (n1 < 1) n1 = 1;
    const int64_t per = (tiles + n1 - 1) / n1;
    msd_merge_l1_kernel<<<(unsigned)n1, kMsdThreads, 0, s>>>(a.parts, tiles, per, scratch);
    nmax_merge_final_kernel<<<1, kMsdThreads, 0, s>>>(scratch, (int)n1, a.nmax, out);
    return cudaGetLastError();
}

cudaError_t launch_stream_msd(const MsdPart *parts, int64_t n_dm, int64_t upr, int per_row,
                              MsdPart *state, spd_msd_stats *out, cudaStream_t s) {
    if (per_row) {
        const unsigned g = (unsigned)((n_dm + kMsdThreads - 1) / kMsdThreads);
        if (g) stream_msd_rows_kernel<<<g, kMsdThreads, 0, s>>>(parts, n_dm, upr, state, out);
    } else {
        stream_msd_global_kernel<<<1, kMsdThreads, 0, s>>>(parts, n_dm * upr, state, out);
    }
    return cudaGetLastError();
}

cudaError_t launch_zero_parts(MsdPart *p, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    zero_parts_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, n);
    return cudaGetLastError();
}

cudaError_t launch_consts(const ConstArgs &a, const RangeProg &prog, cudaStream_t s) {
    consts_kernel<<<a.entries, 256, 0, s>>>(a, prog);
    return cudaGetLastError();
}

}  // namespace spd
