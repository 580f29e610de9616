// spd_msd.cu -- step (a): mean and standard deviation of the DM x time plane
// (Sec. 2.1).  Two kernels, as the paper splits them:
//   msd_partial_kernel: every block reduces one equal-sized unit of a row
//     (kMsdUnit samples) to (n, T, S).  Each thread takes 16 consecutive
//     samples at a time as two sets of 8 (even and odd positions) in the two
//     lanes of packed f32x2 arithmetic, applies Eq. 1 to each set and Eq. 2 to
//     fold it into the lane's running (n, T, S); the two lanes, then lanes of
//     the warp, then warps, are folded with Eq. 2.  FP32 throughout, with T
//     carried as an unevaluated hi + lo pair (compensated summation).
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

    // TwoSum: Th + v exactly as (Th, error) -> error folded into Tl.
    __device__ __forceinline__ void add_T(float v) {
        const float s = Th + v;
        const float bb = s - Th;
        const float e = (Th - (s - bb)) + (v - bb);
        Th = s;
        Tl += e;
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

__device__ __forceinline__ float fmin3(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ float fmax3(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }

// Running (n, T, S) of two disjoint sets of equal size n, one per lane of a
// float2, updated with packed f32x2 arithmetic; T = Th + Tl per lane.
struct Acc2 {
    float m;
    float2 Th, Tl, S;

    __device__ __forceinline__ Acc2() : m(0.f), Th(f2(0.f)), Tl(f2(0.f)), S(f2(0.f)) {}

    // Eq. 1 over v[0..7] (one set of 8 per lane): returns U = -T_8 and S_8.
    // The j-th term uses (j - 1) x_j - T_{j-1}, which equals j x_j - T_j.
    static __device__ __forceinline__ void eq1_8(const float2 *v, float2 &U, float2 &S8) {
        const float2 m1 = f2(-1.f);
        U = __fmul2_rn(v[0], m1);
        float2 d = __fadd2_rn(v[1], U);
        S8 = __fmul2_rn(__fmul2_rn(d, f2(1.f / 2.f)), d);
        U = __ffma2_rn(v[1], m1, U);
#pragma unroll
        for (int j = 3; j <= 8; ++j) {
            d = __ffma2_rn(v[j - 1], f2((float)(j - 1)), U);
            S8 = __ffma2_rn(__fmul2_rn(d, f2(1.f / (float)(j * (j - 1)))), d, S8);
            U = __ffma2_rn(v[j - 1], m1, U);
        }
    }

    // (T, S) of v[0..7] per lane by their definition: the sum, then the
    // squared deviations from the group mean.  Returns U = -T and S8.
    static __device__ __forceinline__ void direct_8(const float2 *v, float2 &U, float2 &S8) {
        const float2 t = __fadd2_rn(__fadd2_rn(__fadd2_rn(v[0], v[1]), __fadd2_rn(v[2], v[3])),
                                    __fadd2_rn(__fadd2_rn(v[4], v[5]), __fadd2_rn(v[6], v[7])));
        const float2 nm = __fmul2_rn(t, f2(-0.125f));   // minus the mean
        float2 d = __fadd2_rn(v[0], nm);
        S8 = __fmul2_rn(d, d);
#pragma unroll
        for (int k = 1; k < 8; ++k) {
            d = __fadd2_rn(v[k], nm);
            S8 = __ffma2_rn(d, d, S8);
        }
        U = __fmul2_rn(t, f2(-1.f));
    }

    // Eq. 2: fold a set of 8 per lane (sum -U, S8) into the running sets.
    __device__ __forceinline__ void fold8(float2 U, float2 S8) {
        const float2 m1 = f2(-1.f);
        if (m == 0.f) {
            Th = __fmul2_rn(U, m1);
            Tl = f2(0.f);
            S = S8;
            m = 8.f;
            return;
        }
        const float q = __fdividef(1.f, m * (m + 8.f));
        const float r = 8.f * (m + 8.f) * q;          // n / m
        const float k = 0.125f * m * m * q;           // m / (n (m + n))
        const float2 ta = __fadd2_rn(Th, Tl);
        const float2 f = __ffma2_rn(f2(r), ta, U);    // (n/m) T_a - T_b
        S = __ffma2_rn(__fmul2_rn(f, f), f2(k), __fadd2_rn(S, S8));
        // TwoSum: Th + T_b exactly as (s, e), T_b = -U
        const float2 sm = __ffma2_rn(U, m1, Th);
        const float2 bb = __ffma2_rn(Th, m1, sm);
        const float2 t2 = __ffma2_rn(__ffma2_rn(bb, m1, sm), m1, Th);
        const float2 e = __ffma2_rn(__fadd2_rn(U, bb), m1, t2);
        Th = sm;
        Tl = __fadd2_rn(Tl, e);
        m += 8.f;
    }

    // Eq. 2: the two lanes as one scalar accumulator.
    __device__ __forceinline__ Acc lanes() const {
        Acc a, b;
        a.m = m; a.Th = Th.x; a.Tl = Tl.x; a.S = S.x;
        b.m = m; b.Th = Th.y; b.Tl = Tl.y; b.S = S.y;
        a.merge(b.m, b.Th, b.Tl, b.S);
        return a;
    }
};

// 16 consecutive samples as 8 float2: v[k] = (x[2k], x[2k+1]).
template <int DT>
__device__ __forceinline__ void load16(const typename Elem<DT>::T *p, bool vec, float2 *v) {
    if (vec) {
        if constexpr (DT == SPD_F32) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4 f = __ldcs(reinterpret_cast<const float4 *>(p) + q);
                v[2 * q] = make_float2(f.x, f.y);
                v[2 * q + 1] = make_float2(f.z, f.w);
            }
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint2 u = __ldcs(reinterpret_cast<const uint2 *>(p) + q);
                if constexpr (DT == SPD_F16) {
                    v[2 * q] = __half22float2(*reinterpret_cast<const __half2 *>(&u.x));
                    v[2 * q + 1] = __half22float2(*reinterpret_cast<const __half2 *>(&u.y));
                } else {
                    v[2 * q] = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u.x));
                    v[2 * q + 1] =
                        __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u.y));
                }
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < 8; ++k)
            v[k] = make_float2(Elem<DT>::cvt(p[2 * k]), Elem<DT>::cvt(p[2 * k + 1]));
    }
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

    // 16 samples per thread and step: Eq. 1 on the even and on the odd eight
    // (one per f32x2 lane), Eq. 2 into the lane's running partial
    Acc2 acc2;
    float lo = INFINITY, hi = -INFINITY;
    const int64_t ngrp = len >> 4;
    for (int64_t g = tid; g < ngrp; g += kMsdThreads) {
        float2 v[8];
        load16<DT>(p + 16 * g, a.vec_ok != 0, v);
        if (has_sc) {
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] = __ffma2_rn(f2(sc), v[k], f2(of));
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            lo = fmin3(lo, v[k].x, v[k].y);
            hi = fmax3(hi, v[k].x, v[k].y);
        }
        float2 U, S8;
        Acc2::eq1_8(v, U, S8);
        acc2.fold8(U, S8);
    }
    Acc acc = acc2.lanes();
    acc.lo = lo;
    acc.hi = hi;
    for (int64_t t = 16 * ngrp + tid; t < len; t += kMsdThreads) {
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

constexpr int kNmaxThreads = 128;
constexpr int kNmaxPer = 64;                                // consecutive starts per thread
constexpr int kNmaxTile = kNmaxThreads * kNmaxPer;          // 8192 starts per tile
constexpr int kNmaxTilesPerCta = 4;    // consecutive tiles of one row per CTA (one partial)

// Four stored samples as one load, and their values as two float2.
template <int DT> struct Quad;
template <> struct Quad<SPD_F32> {
    using V = float4;
    static constexpr int kInFlight = 9;   // loads in flight per thread while staging
    static __device__ __forceinline__ V ld(const float *p) {
        return __ldcs(reinterpret_cast<const float4 *>(p));
    }
    static __device__ __forceinline__ void cvt(V v, float2 &a, float2 &b) {
        a = make_float2(v.x, v.y);
        b = make_float2(v.z, v.w);
    }
};
template <> struct Quad<SPD_F16> {
    using V = uint2;
    static constexpr int kInFlight = 17;
    static __device__ __forceinline__ V ld(const __half *p) {
        return __ldcs(reinterpret_cast<const uint2 *>(p));
    }
    static __device__ __forceinline__ void cvt(V v, float2 &a, float2 &b) {
        a = __half22float2(*reinterpret_cast<const __half2 *>(&v.x));
        b = __half22float2(*reinterpret_cast<const __half2 *>(&v.y));
    }
};
template <> struct Quad<SPD_BF16> {
    using V = uint2;
    static constexpr int kInFlight = 17;
    static __device__ __forceinline__ V ld(const __nv_bfloat16 *p) {
        return __ldcs(reinterpret_cast<const uint2 *>(p));
    }
    static __device__ __forceinline__ void cvt(V v, float2 &a, float2 &b) {
        a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&v.x));
        b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&v.y));
    }
};

// Shared layout of the staged window: position p at word p + 4 (p / 64), so
// 16-position blocks are contiguous and 64-position runs start 68 words apart.
__host__ __device__ __forceinline__ int npad(int p) { return p + 4 * (p >> 6); }
__host__ __device__ __forceinline__ int nmax_ywords(int nb) {
    return (npad(16 * nb) + 3) & ~3;   // block sums follow, 16-byte aligned
}
size_t nmax_smem_bytes(int nb) { return ((size_t)nmax_ywords(nb) + nb) * sizeof(float); }

__device__ __forceinline__ float block_sum(const float *s_y, int b) {
    float sum = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float4 f = *reinterpret_cast<const float4 *>(s_y + npad(16 * b) + 4 * q);
        sum += (f.x + f.y) + (f.z + f.w);
    }
    return sum;
}

// Sec. 2.2, Eq. 5 needs sigma_Nmax, the measured sd of the boxcar series
// B_Nmax(i) = x[i] + ... + x[i+Nmax-1] over full windows.  Each CTA walks up
// to kNmaxTilesPerCta consecutive tiles of one row; per tile it stages the
// centred samples plus an (Nmax - 1)-sample halo, with 16-sample block sums.
// A thread owns 64 consecutive starts: B0 = B at the first, from the whole
// blocks of its window (four interleaved sums) plus the partial block; then
// d = B - B0 slides one sample at a time, and the thread sums d and d^2 over
// its starts with full windows (even and odd starts in the two f32x2 lanes).
// Its run's (n, T, S) -- n, n B0 + sum d, sum d^2 - (sum d)^2 / n -- goes
// into the thread's running (n, T, S) by Eq. 2 once per tile.  At the end
// Eq. 2 merges the lanes of the warp and the warps into the CTA's one
// partial.  The sd does not depend on the centring.
template <int DT>
__global__ void __launch_bounds__(kNmaxThreads, 5) nmax_partial_kernel(const NmaxArgs a) {
    using T = typename Elem<DT>::T;
    // centred samples, 64 positions in 68 words: lane t reading its own
    // 64-position run (or the run nmax later) with 128-bit loads hits distinct
    // banks within each quarter warp
    extern __shared__ __align__(16) float s_y[];   // [nmax_ywords(nb)]
    float *s_bs = s_y + nmax_ywords(a.nb);         // [nb] block sums
    const int tid = threadIdx.x;
    const int64_t row = blockIdx.x / a.tiles_per_row;   // tiles_per_row: partials per row
    const int64_t part = blockIdx.x - row * a.tiles_per_row;
    const int64_t tiles_in_row = (a.n_samp + kNmaxTile - 1) / kNmaxTile;
    const int64_t tl0 = part * kNmaxTilesPerCta;
    const int64_t tl1 = min(tl0 + kNmaxTilesPerCta, tiles_in_row);
    const int entry = a.per_row ? (int)row : 0;
    const T *rp = static_cast<const T *>(a.data) + row * a.stride;
    const bool has_sc = a.scale != nullptr;
    const float sc = has_sc ? a.scale[row] : 1.f;
    const float of = (has_sc && a.offset) ? a.offset[row] : 0.f;
    // centring shift, rounded once: a constant error in it moves every B of
    // the row alike, which the sd does not see
    const float cy = (float)((double)of - a.msd[entry].mean);
    const float2 sc2 = f2(sc), c2 = f2(cy);
    constexpr int kQ = Quad<DT>::kInFlight;
    const int nmax = a.nmax;
    const int b0 = tid * (kNmaxPer / 16);          // the thread's first block (tile-local)
    const int qe = 16 * b0 + nmax;                 // end of its first window
    Acc run_acc;    // the thread's runs: one Eq. 2 merge per tile
    for (int64_t tl = tl0; tl < tl1; ++tl) {
        const int64_t t0 = tl * (int64_t)kNmaxTile;
        __syncthreads();   // the previous tile's reads of s_y / s_bs are done
        // Stage the window, kQ groups of 4 samples per thread at a time: all
        // loads of a round are issued before any is used, so a tile waits for
        // memory once per round.  y = scale x + (offset - mu), one rounding;
        // positions past the row end hold 0.
        const int nq = 4 * a.nb;
        for (int c0 = 0; c0 < nq; c0 += kQ * kNmaxThreads) {
            const int cq = min(c0 + kQ * kNmaxThreads, nq);   // this round's end
            if (a.vec_ok && t0 + 4 * (int64_t)cq <= a.n_samp) {
                typename Quad<DT>::V r[kQ];
#pragma unroll
                for (int u = 0; u < kQ; ++u) {
                    const int q4 = c0 + u * kNmaxThreads + tid;
                    if (q4 < cq) r[u] = Quad<DT>::ld(rp + t0 + 4 * q4);
                }
#pragma unroll
                for (int u = 0; u < kQ; ++u) {
                    const int q4 = c0 + u * kNmaxThreads + tid;
                    if (q4 < cq) {
                        float2 v0, v1;
                        Quad<DT>::cvt(r[u], v0, v1);
                        v0 = __ffma2_rn(sc2, v0, c2);
                        v1 = __ffma2_rn(sc2, v1, c2);
                        const int p = 4 * q4;
                        *reinterpret_cast<float4 *>(s_y + npad(p)) =
                            make_float4(v0.x, v0.y, v1.x, v1.y);
                    }
                }
            } else {
                for (int q4 = c0 + tid; q4 < cq; q4 += kNmaxThreads) {
                    const int p = 4 * q4;
                    float y[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int64_t t = t0 + p + e;
                        y[e] = t < a.n_samp ? fmaf(sc, Elem<DT>::cvt(rp[t]), cy) : 0.f;
                    }
                    *reinterpret_cast<float4 *>(s_y + npad(p)) =
                        make_float4(y[0], y[1], y[2], y[3]);
                }
            }
        }
        __syncthreads();
        // block sums: the thread's own four blocks, then the halo blocks
        {
            float bs4[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) bs4[c] = block_sum(s_y, b0 + c);
            *reinterpret_cast<float4 *>(s_bs + b0) = make_float4(bs4[0], bs4[1], bs4[2], bs4[3]);
            for (int b = kNmaxTile / 16 + tid; b < a.nb; b += kNmaxThreads)
                s_bs[b] = block_sum(s_y, b);
        }
        __syncthreads();

        // B at the thread's first start: whole blocks of the window (four
        // interleaved sums), plus the partial block at its end
        float w0 = 0.f, w1 = 0.f, w2 = 0.f, w3 = 0.f;
        int b = b0;                      // a multiple of 4: 128-bit loads
        const int be = qe >> 4;
        for (; b + 3 < be; b += 4) {
            const float4 f = *reinterpret_cast<const float4 *>(s_bs + b);
            w0 += f.x;
            w1 += f.y;
            w2 += f.z;
            w3 += f.w;
        }
        for (; b < be; ++b) w0 += s_bs[b];
        float tail = 0.f;
        for (int q = (qe & ~15); q < qe; ++q) tail += s_y[npad(q)];
        const float B0 = ((w0 + w1) + (w2 + w3)) + tail;
        // B slides as its difference d = B - B0 from the thread's first start:
        // over its full-window starts the thread keeps sums of d and d^2 (even
        // and odd starts in the two packed lanes), so that (n, T, S) of its run
        // is n, n B0 + sum d and sum d^2 - (sum d)^2 / n, merged once per
        // tile.  d stays near 0 within a run of 64 starts, so the difference
        // of sums loses little.
        float Bd = 0.f;
        float2 Td = f2(0.f), Sd = f2(0.f);
        int nrun = 0;
        // starts t0 + 16 b0 + k are full windows while k < nvalid
        const int64_t nvalid = a.n_samp - nmax - (t0 + 16 * b0) + 1;
#pragma unroll 1
        for (int c = 0; c < kNmaxPer / 16; ++c) {
            // the unit's 16 samples and the 16 that enter the window as it slides
            const int bl = b0 + c;
            float lo[16], hi[16];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4 f = *reinterpret_cast<const float4 *>(s_y + npad(16 * bl) + 4 * q);
                lo[4 * q] = f.x; lo[4 * q + 1] = f.y; lo[4 * q + 2] = f.z; lo[4 * q + 3] = f.w;
            }
            if ((nmax & 15) == 0) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float4 f =
                        *reinterpret_cast<const float4 *>(s_y + npad(16 * bl + nmax) + 4 * q);
                    hi[4 * q] = f.x; hi[4 * q + 1] = f.y; hi[4 * q + 2] = f.z; hi[4 * q + 3] = f.w;
                }
            } else {
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const int q = 16 * bl + k + nmax;
                    hi[k] = s_y[npad(q)];
                }
            }
            // d slides by hi - lo per start (the differences as f32x2 pairs)
            float2 bw[8];   // bw[k] = (d at unit start + 2k, d at unit start + 2k + 1)
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const float2 dl = __ffma2_rn(make_float2(lo[2 * k], lo[2 * k + 1]), f2(-1.f),
                                             make_float2(hi[2 * k], hi[2 * k + 1]));
                bw[k].x = Bd;
                Bd += dl.x;
                bw[k].y = Bd;
                Bd += dl.y;
            }
            const int64_t nv = nvalid - 16 * c;
            if (nv >= 16) {
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    Td = __fadd2_rn(Td, bw[k]);
                    Sd = __ffma2_rn(bw[k], bw[k], Sd);
                }
                nrun += 16;
            } else if (nv > 0) {   // near the row end: the starts with full windows
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const float2 dm = make_float2(2 * k < nv ? bw[k].x : 0.f,
                                                  2 * k + 1 < nv ? bw[k].y : 0.f);
                    Td = __fadd2_rn(Td, dm);
                    Sd = __ffma2_rn(dm, dm, Sd);
                }
                nrun += (int)nv;
            }
        }
        if (nrun) {   // the run's (n, T, S), T with the product n B0 kept exactly
            const float n = (float)nrun;
            const float td = Td.x + Td.y;
            const float sr = fmaf(-td, td / n, Sd.x + Sd.y);
            const float th = n * B0;
            const float tlo = fmaf(n, B0, -th) + td;
            run_acc.merge(n, th, tlo, fmaxf(sr, 0.f));
        }
    }
    Acc acc = run_acc;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc.merge_down(off);
    __shared__ float4 s_w[kNmaxThreads / 32];
    const int lane = tid & 31, warp = tid >> 5;
    if (lane == 0) s_w[warp] = make_float4(acc.m, acc.Th, acc.Tl, acc.S);
    __syncthreads();
    if (warp == 0) {
        Acc b;
        if (lane < kNmaxThreads / 32) {
            const float4 v = s_w[lane];
            b.m = v.x; b.Th = v.y; b.Tl = v.z; b.S = v.w;
        }
#pragma unroll
        for (int off = kNmaxThreads / 64; off > 0; off >>= 1) b.merge_down(off);
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
    const size_t smem = nmax_smem_bytes(a.nb);
    // above 48 KB (Nmax >= 2705) the kernel opts in to the larger window,
    // on the current device, before each such launch
    if (smem > 48 * 1024) {
        const void *fn = dtype == SPD_F32   ? (const void *)nmax_partial_kernel<SPD_F32>
                         : dtype == SPD_F16 ? (const void *)nmax_partial_kernel<SPD_F16>
                                            : (const void *)nmax_partial_kernel<SPD_BF16>;
        const cudaError_t e =
            cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    switch (dtype) {
        case SPD_F32: nmax_partial_kernel<SPD_F32><<<(unsigned)tiles, kNmaxThreads, smem, s>>>(a); break;
        case SPD_F16: nmax_partial_kernel<SPD_F16><<<(unsigned)tiles, kNmaxThreads, smem, s>>>(a); break;
        default: nmax_partial_kernel<SPD_BF16><<<(unsigned)tiles, kNmaxThreads, smem, s>>>(a); break;
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
