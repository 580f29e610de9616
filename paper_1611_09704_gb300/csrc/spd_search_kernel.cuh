// spd_search_kernel.cuh -- the candidate search: steps (b), (c) and (d) fused
// (boxcar filters, SNR with the max over widths and the winning width, and
// thresholding with compaction; Sec. 2.3-2.4, Algorithm 1) over one or more
// DM ranges in one persistent launch.
//
// CTAs of 256 (or 128) threads walk tiles of 16 U consecutive start samples
// of one DM row, U = the threads less the halo's blocks, so that every thread
// stages one block of the window (U = the threads for halos of more than 64
// blocks, staged in several rounds).  A tile's window (the tile plus the
// (wmax - 1)-sample halo) arrives in
// shared memory by one 1-D bulk (TMA) copy, issued for the next tile as soon
// as the current one has been staged, so it overlaps the whole search of the
// current tile.
//
// Staging (one thread per block of 16 window positions): the centred samples
// y = x - mu, the in-block prefix sums P (for the start of a width group at
// any block offset), the G-sample window sums S_G, and per block its sum, its
// energy sum(y^2) and its largest and smallest prefix value.  Warp scans and
// the warp totals then give the tile's prefix C at every block start (FP32,
// used only for bounds), the prefix maxima with a small sparse max table,
// and the energy prefix.
//
// Search (thread t owns starts 16t .. 16t+15, a "unit"): the widths form
// groups (runs of consecutive widths of step 1, or of step G through S_G).
// Groups are visited from the widest down.  Before a group is evaluated two
// upper bounds of its SNRs over the unit are compared with
// lim = max(threshold, the smallest current best of the unit):
//   prefix:  B_w(i) = C[i+w] - C[i] <= max C over the blocks the windows end
//            in - min C at the unit's starts, times the largest 1/sigma_w;
//   energy:  B_w(i) <= sqrt(w * sum of y^2 over the window) (Cauchy-Schwarz),
//            so SNR^2 <= (energy of the blocks the windows lie in) * max w/sigma_w^2.
// A group that cannot reach lim cannot change any candidate and is skipped.
// The group of widths 1..16 is first tested per sample (the energy of each
// start's own 16-sample window against its own best).
//
// Evaluation follows Algorithm 1: a group's running sums start at B_off (the
// sum of whole blocks plus the difference of in-block prefixes) and grow by
// one sample (step 1) or one window sum (step G) per width, two samples per
// packed f32x2 add and multiply.  Each SNR is packed with a code (63 minus the
// eval index within its block of 64) in its low 6 mantissa bits before a
// float max, so one max keeps value and width; among SNRs equal to 2^-17
// relative the smallest width wins -- the strict ">" of Algorithm 1 at that
// resolution.  With more than 64 evaluated widths the bests of successive
// blocks of 64 are merged by value, ties to the smaller widths.
//
// Candidates (best truncated to 2^-17 >= threshold, Sec. 2.4) are compacted
// with one atomic per tile and written as 16-byte records.
//
// Widths past the row end see y = -inf (sums -inf or NaN), which no max keeps
// and which no bound prunes wrongly (NaN bounds never prune).
#pragma once
#include "spd_device.cuh"

namespace spd {

namespace {

__device__ __forceinline__ int sadr(int p) { return (p & 15) + kSPad * (p >> 4); }

// Centred values y = (x - mu.hi) - mu.lo of window positions p .. p+N-1
// (x = fmaf(scale, q, offset) for scaled storage), -inf at and past `have`.
// Elements below nraw come from the raw staging buffer, the rest of the row
// from global memory.
template <int DT, int N>
__device__ __forceinline__ void load_centred(float *v, const typename Elem<DT>::T *raw,
                                             const typename Elem<DT>::T *gsrc, int p, int nraw,
                                             int have, bool has_sc, float sc, float of, float2 mu) {
    const float2 mh = make_float2(-mu.x, -mu.x), ml = make_float2(-mu.y, -mu.y);
    if (p + N <= nraw) {
#pragma unroll
        for (int u = 0; u < N / 4; ++u) {
            float a, b, c, d;
            load4v<DT>(raw + p + 4 * u, a, b, c, d);
            float2 x0 = make_float2(a, b), x1 = make_float2(c, d);
            if (has_sc) {
                const float2 s2 = make_float2(sc, sc), o2 = make_float2(of, of);
                x0 = fma2(s2, x0, o2);
                x1 = fma2(s2, x1, o2);
            }
            x0 = add2(add2(x0, mh), ml);
            x1 = add2(add2(x1, mh), ml);
            v[4 * u] = x0.x; v[4 * u + 1] = x0.y; v[4 * u + 2] = x1.x; v[4 * u + 3] = x1.y;
        }
    } else {
#pragma unroll
        for (int e = 0; e < N; ++e) {
            const int q = p + e;
            float x = 0.f;
            if (q < nraw) x = Elem<DT>::cvt(raw[q]);
            else if (q < have) x = Elem<DT>::cvt(gsrc[q]);
            if (has_sc) x = fmaf(sc, x, of);
            x = __fsub_rn(__fsub_rn(x, mu.x), mu.y);
            v[e] = q < have ? x : -INFINITY;
        }
    }
}

// --------------------------------------------------------- group evaluation

// Packed max of two widths (codes ka, ka - 1) of a pair of samples.
__device__ __forceinline__ void pmax2(float &m0, float &m1, float2 sa, float2 sb, uint32_t ka) {
    m0 = fmax3(m0, packw(sa.x, ka), packw(sb.x, ka - 1));
    m1 = fmax3(m1, packw(sa.y, ka), packw(sb.y, ka - 1));
}
__device__ __forceinline__ void pmax1(float &m0, float &m1, float2 sa, uint32_t ka) {
    m0 = fmaxf(m0, packw(sa.x, ka));
    m1 = fmaxf(m1, packw(sa.y, ka));
}

// Step-1 group, pairs of samples (k, k + 8): B[j] = (B(16t + j), B(16t + j + 8)).
// The step of width c for pair j is (y[off + c + j], y[off + c + j + 8])
// (positions relative to 16t), held in ring slot (j + c) & 7: from one width
// to the next, pair j takes pair j + 1's slot, and the slot pair 0 leaves
// becomes pair 7's, (y[off + c + 8], y[off + c + 16]) -- one new sample per
// width.
template <bool AL>
__device__ __forceinline__ void eval_fine(float (&cb)[kX], float2 (&B)[8], const float *yb,
                                          const Group &g, const float *s_inv) {
    const int off = g.off;
    float2 R[8];
    if (AL) {
        const float *p = yb + kSPad * (off >> 4);
        const float4 a0 = *reinterpret_cast<const float4 *>(p);
        const float4 a1 = *reinterpret_cast<const float4 *>(p + 4);
        const float4 a2 = *reinterpret_cast<const float4 *>(p + 8);
        const float4 a3 = *reinterpret_cast<const float4 *>(p + 12);
        R[0] = make_float2(a0.x, a2.x); R[1] = make_float2(a0.y, a2.y);
        R[2] = make_float2(a0.z, a2.z); R[3] = make_float2(a0.w, a2.w);
        R[4] = make_float2(a1.x, a3.x); R[5] = make_float2(a1.y, a3.y);
        R[6] = make_float2(a1.z, a3.z); R[7] = make_float2(a1.w, a3.w);
    } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) R[j] = make_float2(yb[sadr(off + j)], yb[sadr(off + j + 8)]);
    }
    const float *ynext = AL ? yb + kSPad * ((off >> 4) + 1) : yb;   // y[off + 16 + c]
    for (int c0 = 0; c0 < g.count; c0 += 8) {
#pragma unroll
        for (int cc = 0; cc < 8; cc += 2) {
            const int c = c0 + cc;
            if (c >= g.count) break;
            const int wi = g.widx0 + c;
            const uint32_t ka = 63u - (uint32_t)(wi & 63);
            const float ia = s_inv[wi];
            const float2 ia2 = make_float2(ia, ia);
            float2 sa[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                B[j] = add2(B[j], R[(j + cc) & 7]);
                sa[j] = mul2(B[j], ia2);
            }
            R[cc].x = R[cc].y;
            R[cc].y = AL ? ynext[kSPad * (c >> 4) + (c & 15)] : yb[sadr(off + c + 16)];
            if (c + 1 < g.count) {
                const float ib = s_inv[wi + 1];
                const float2 ib2 = make_float2(ib, ib);
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    B[j] = add2(B[j], R[(j + cc + 1) & 7]);
                    pmax2(cb[j], cb[j + 8], sa[j], mul2(B[j], ib2), ka);
                }
                R[cc + 1].x = R[cc + 1].y;
                R[cc + 1].y = AL ? ynext[kSPad * ((c + 1) >> 4) + ((c + 1) & 15)]
                                 : yb[sadr(off + c + 17)];
            } else {
#pragma unroll
                for (int j = 0; j < 8; ++j) pmax1(cb[j], cb[j + 8], sa[j], ka);
            }
        }
    }
}

// Step-G group (G = 8 or 16) starting at a block boundary, pairs (2j, 2j + 1).
// Member c adds S_G at positions off + cG + k, k < 16: four float4 segments,
// of which (G = 8) two carry over to the next member through a ring.
template <int G>
__device__ __forceinline__ void eval_coarse(float (&cb)[kX], float2 (&B)[8], const float *gb,
                                            const Group &g, const float *s_inv) {
    const float *base = gb + kSPad * (g.off >> 4);
    if (G == 8) {
        float4 r0 = *reinterpret_cast<const float4 *>(base);
        float4 r1 = *reinterpret_cast<const float4 *>(base + 4);
        for (int c = 0; c < g.count; c += 2) {
            const float *pb = base + kSPad * (c >> 1);
            const float4 r2 = *reinterpret_cast<const float4 *>(pb + 8);
            const float4 r3 = *reinterpret_cast<const float4 *>(pb + 12);
            const int wi = g.widx0 + c;
            const uint32_t ka = 63u - (uint32_t)(wi & 63);
            const float ia = s_inv[wi];
            const float2 ia2 = make_float2(ia, ia);
            const float2 va[8] = {make_float2(r0.x, r0.y), make_float2(r0.z, r0.w),
                                  make_float2(r1.x, r1.y), make_float2(r1.z, r1.w),
                                  make_float2(r2.x, r2.y), make_float2(r2.z, r2.w),
                                  make_float2(r3.x, r3.y), make_float2(r3.z, r3.w)};
            float2 sa[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                B[j] = add2(B[j], va[j]);
                sa[j] = mul2(B[j], ia2);
            }
            if (c + 1 < g.count) {
                r0 = *reinterpret_cast<const float4 *>(pb + kSPad);
                r1 = *reinterpret_cast<const float4 *>(pb + kSPad + 4);
                const float ib = s_inv[wi + 1];
                const float2 ib2 = make_float2(ib, ib);
                const float2 vb[8] = {make_float2(r2.x, r2.y), make_float2(r2.z, r2.w),
                                      make_float2(r3.x, r3.y), make_float2(r3.z, r3.w),
                                      make_float2(r0.x, r0.y), make_float2(r0.z, r0.w),
                                      make_float2(r1.x, r1.y), make_float2(r1.z, r1.w)};
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    B[j] = add2(B[j], vb[j]);
                    pmax2(cb[2 * j], cb[2 * j + 1], sa[j], mul2(B[j], ib2), ka);
                }
            } else {
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    pmax1(cb[2 * j], cb[2 * j + 1], sa[j], ka);
            }
        }
    } else {
        for (int c = 0; c < g.count; c += 2) {
            const int wi = g.widx0 + c;
            const uint32_t ka = 63u - (uint32_t)(wi & 63);
            const float ia = s_inv[wi];
            const float2 ia2 = make_float2(ia, ia);
            const float *pa = base + kSPad * c;
            float2 sa[8];
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const float4 f = *reinterpret_cast<const float4 *>(pa + 4 * v);
                B[2 * v] = add2(B[2 * v], make_float2(f.x, f.y));
                B[2 * v + 1] = add2(B[2 * v + 1], make_float2(f.z, f.w));
                sa[2 * v] = mul2(B[2 * v], ia2);
                sa[2 * v + 1] = mul2(B[2 * v + 1], ia2);
            }
            if (c + 1 < g.count) {
                const float ib = s_inv[wi + 1];
                const float2 ib2 = make_float2(ib, ib);
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const float4 f = *reinterpret_cast<const float4 *>(pa + kSPad + 4 * v);
                    B[2 * v] = add2(B[2 * v], make_float2(f.x, f.y));
                    B[2 * v + 1] = add2(B[2 * v + 1], make_float2(f.z, f.w));
                    pmax2(cb[4 * v], cb[4 * v + 1], sa[2 * v], mul2(B[2 * v], ib2), ka);
                    pmax2(cb[4 * v + 2], cb[4 * v + 3], sa[2 * v + 1], mul2(B[2 * v + 1], ib2), ka);
                }
            } else {
#pragma unroll
                for (int j = 0; j < 8; ++j) pmax1(cb[2 * j], cb[2 * j + 1], sa[j], ka);
            }
        }
    }
}

// Any group (start not at a block boundary, or any step d), one width at a
// time with per-sample loads, pairs (2j, 2j + 1).
__device__ __forceinline__ void eval_generic(float (&cb)[kX], float2 (&B)[8], const float *sb,
                                             const Group &g, int d, const float *s_inv) {
#pragma unroll 1
    for (int c = 0; c < g.count; ++c) {
        const int p0 = g.off + c * d;
        const int wi = g.widx0 + c;
        const uint32_t ka = 63u - (uint32_t)(wi & 63);
        const float ia = s_inv[wi];
        const float2 ia2 = make_float2(ia, ia);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            B[j] = add2(B[j], make_float2(sb[sadr(p0 + 2 * j)], sb[sadr(p0 + 2 * j + 1)]));
            pmax1(cb[2 * j], cb[2 * j + 1], mul2(B[j], ia2), ka);
        }
    }
}

// Per-sample test of the group of widths 1..16 (off 0): can any start of the
// unit reach its own bar max(threshold, best)?  Energy of each start's
// 16-sample window, e_k = sum y^2 over [16t + k, 16t + k + 16), bounds every
// SNR of widths <= 16 by sqrt(e_k * max w / sigma_w^2).
__device__ __forceinline__ bool refine16(const float *yb, const float (&best)[kX], float thr,
                                         float m2) {
    float sq[32];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const float4 f = *reinterpret_cast<const float4 *>(yb + kSPad * (u >> 2) + 4 * (u & 3));
        sq[4 * u] = f.x * f.x; sq[4 * u + 1] = f.y * f.y;
        sq[4 * u + 2] = f.z * f.z; sq[4 * u + 3] = f.w * f.w;
    }
    float ps[33];   // ps[m] = sq[0] + ... + sq[m-1]
    ps[0] = 0.f;
#pragma unroll
    for (int m = 0; m < 32; ++m) ps[m + 1] = ps[m] + sq[m];
    // rounding of the prefix and of the difference: a few ulp of ps[32]
    const float slack = 4e-6f * ps[32] + 1e-30f;
    bool need = false;
#pragma unroll
    for (int k = 0; k < kX; ++k) {
        const float eu = (ps[k + 16] - ps[k]) + slack;
        const float lim = fmaxf(thr, trunc17(best[k]));
        const float ll = lim * (1.f - 2e-5f);
        // NaN (a window past the row end) never rules the group out
        need |= !(lim > 0.f && eu * m2 < ll * ll);
    }
    return need;
}

// In-block part of B_off(16t + k), k < 16, for a group starting at a block
// boundary (off = 16 o): D + P_{t+o}[k] - P_t[k], with D the sum of the whole
// blocks t .. t + o - 1 and P the in-block prefix sums.
__device__ __forceinline__ void start_aligned(float (&v)[kX], const float *s_p, int t, int o,
                                              float D) {
    const float *pa = s_p + kSPad * (t + o), *p0 = s_p + kSPad * t;
    const float2 d2 = make_float2(D, D);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const float4 a = *reinterpret_cast<const float4 *>(pa + 4 * u);
        const float4 z = *reinterpret_cast<const float4 *>(p0 + 4 * u);
        const float2 lo = add2(d2, add2(make_float2(a.x, a.y), make_float2(-z.x, -z.y)));
        const float2 hi = add2(d2, add2(make_float2(a.z, a.w), make_float2(-z.z, -z.w)));
        v[4 * u] = lo.x; v[4 * u + 1] = lo.y; v[4 * u + 2] = hi.x; v[4 * u + 3] = hi.y;
    }
}

// B_off(16t + k) for any other offset: the sum over [16t, 16t + off), then
// one slide per start.
__device__ __forceinline__ void start_generic(float (&v)[kX], const float *s_y, const float *s_bs,
                                              int t, int off) {
    const float *yt = s_y + kSPad * t;
    const int o = off >> 4;
    float s = 0.f;
    for (int b = 0; b < o; ++b) s = __fadd_rn(s, s_bs[t + b]);
    for (int j = 16 * o; j < off; ++j) s = __fadd_rn(s, yt[sadr(j)]);
    v[0] = s;
#pragma unroll
    for (int k = 1; k < kX; ++k) {
        s = __fadd_rn(s, __fsub_rn(yt[sadr(off + k - 1)], yt[sadr(k - 1)]));
        v[k] = s;
    }
}

// Per-group data in shared memory (two int4 per group):
//   a = {off | count << 16, widx0 | flags << 16, q1, q2}
//   b = {qe, level, bits of the largest 1/sigma_w (margin folded in),
//        bits of the largest w / sigma_w^2 (margin folded in)}
// q1, q2: offsets from the table base (level 0 = the block prefix maxima) of
// the two table windows the prefix bound reads (level -1: first and last
// block of a plain loop); qe: blocks of the energy bound.
__device__ __forceinline__ void load_search_consts(const RangeDesc &rd, int entry, int RM,
                                                   float *s_inv, int4 *s_gr, uint16_t *s_ew) {
    const RangeProg &rp = rd.prog;
    for (int q = threadIdx.x; q < rp.n_eval; q += blockDim.x)
        s_inv[q] = rd.inv_tab[(int64_t)entry * rp.n_eval + q];
    __syncthreads();
    for (int gi = threadIdx.x; gi < rp.n_groups; gi += blockDim.x) {
        const Group g = rp.groups[gi];
        const int d = (g.flags & kGroupCoarse) ? rp.G : 1;
        float imax = 0.f, m2 = 0.f;
        for (int c = 0; c < g.count; ++c) {
            const int w = g.off + (c + 1) * d;
            const float inv = s_inv[g.widx0 + c];
            s_ew[g.widx0 + c] = (uint16_t)w;
            imax = fmaxf(imax, inv);              // a NaN 1/sigma (no SNR) is ignored
            m2 = fmaxf(m2, (float)w * inv * inv);
        }
        const GroupGeom q = group_geom(g.off, g.count, d);
        const int base = q.lvl > 0 ? RM * q.lvl : 0;
        s_gr[2 * gi] = make_int4((int)(uint16_t)g.off | ((int)g.count << 16),
                                 (int)(uint16_t)g.widx0 | ((int)g.flags << 16), base + q.a,
                                 base + q.bk);
        // margins for the rounding of the computed SNRs (a few ulp)
        s_gr[2 * gi + 1] = make_int4(q.e, q.lvl, __float_as_int(imax * 1.00002f),
                                     __float_as_int(m2 * 1.00004f));
    }
    __syncthreads();
    // energy factor of a group and of every narrower one (a running max from
    // the narrowest group up): once it rules a group out, it rules out all
    // the narrower ones too (their windows lie inside the same blocks)
    if (threadIdx.x == 0) {
        float run = 0.f;
        for (int gi = 0; gi < rp.n_groups; ++gi) {
            run = fmaxf(run, __int_as_float(s_gr[2 * gi + 1].w));
            s_gr[2 * gi + 1].w = __float_as_int(run);
        }
    }
    __syncthreads();
}

// Position of a tile in the launch: range, row, tile column.
struct TilePos {
    int ri;
    int64_t row, col;
};

template <int DT, int G, bool MG, int NT, bool PL>
__global__ void __launch_bounds__(NT, 512 / NT) search_kernel(const __grid_constant__ Launch L) {
    constexpr int kThreads = NT;
    // units of 16 starts per tile: NT less the halo blocks when the whole
    // window then fits one block per thread (one staging round), else NT
    const int U = L.units;
    const int64_t kTile = (int64_t)kX * U;   // starts of one tile
    using T = typename Elem<DT>::T;
    extern __shared__ __align__(16) unsigned char smem[];
    const int RM = L.R;          // multiple of 4
    const int KM = L.kmax;
    const SearchSmem sm = search_smem(RM, L.raw_bytes, L.max_eval, KM, G);
    uint64_t *s_bar = reinterpret_cast<uint64_t *>(smem);
    unsigned char *s_raw = smem + sm.raw;
    float *s_y = reinterpret_cast<float *>(smem + sm.y);
    float *s_p = reinterpret_cast<float *>(smem + sm.p);
    float *s_g = reinterpret_cast<float *>(smem + sm.g);
    float *s_bs = reinterpret_cast<float *>(smem + sm.bs);
    float *s_mx = reinterpret_cast<float *>(smem + sm.mx);     // table level 0, then 1 .. KM
    float *s_mn = reinterpret_cast<float *>(smem + sm.mn);
    float *s_pq = reinterpret_cast<float *>(smem + sm.pq);
    float *s_ex = reinterpret_cast<float *>(smem + sm.ex);
    float *s_eq = reinterpret_cast<float *>(smem + sm.eq);
    float *s_rh = reinterpret_cast<float *>(smem + sm.rh);
    float *s_rl = reinterpret_cast<float *>(smem + sm.rl);
    float *s_inv = reinterpret_cast<float *>(smem + sm.inv);
    int4 *s_gr = reinterpret_cast<int4 *>(smem + sm.gr);
    uint16_t *s_ew = reinterpret_cast<uint16_t *>(smem + sm.ew);
    __shared__ float s_wt[48], s_wq[48];       // warp totals per chunk of 32 blocks
    __shared__ int s_wsum[kThreads / 32];
    __shared__ unsigned long long s_wbase[kThreads / 32];
    __shared__ float2 s_mu;
    __shared__ int s_deg;
    __shared__ int s_mag;      // bits of the tile's largest finite |prefix| (non-negative float)

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t esz = (int64_t)sizeof(T);
    // Tiles go in chunks of L.chunk consecutive tiles.  CTA b starts with
    // chunk b, then takes chunk gridDim.x + v for v from an atomic counter,
    // claimed one chunk ahead of need: CTAs that meet costly tiles (wide
    // width lists, dense candidates) take fewer of them.  The chunks in
    // flight at one time are neighbours, so a window's halo is still in L2.
    // The counter (the result word's reserved field) is 0 at launch; the CTA
    // that gets the last claim of all sets it back to 0.  Plane output (PL),
    // where every tile costs the same, takes one fixed run of tiles per CTA
    // instead, without a counter.
    auto counter = [&]() { return reinterpret_cast<unsigned *>(&L.result->reserved0); };
    // the host launches at most n_chunks CTAs (PL: at most n_tiles)
    int64_t tile = PL ? (int64_t)blockIdx.x * L.n_tiles / gridDim.x
                      : (int64_t)blockIdx.x * L.chunk;
    // the launch's tile count (PL: the end of the CTA's run) and chunk length,
    // read from shared memory where needed (kept out of registers through the
    // search)
    __shared__ long long s_ntiles;
    __shared__ int s_chunk;
    if (tid == 0) {
        s_ntiles = PL ? (int64_t)(blockIdx.x + 1) * L.n_tiles / gridDim.x : L.n_tiles;
        s_chunk = L.chunk;
    }
    __syncthreads();
    // chunks are aligned and a power of two long: a tile is its chunk's last
    // when the next one starts a chunk
    auto chunk_ends = [&]() {
        if (PL) return tile + 1 >= s_ntiles;
        return (((uint32_t)tile + 1u) & (uint32_t)(s_chunk - 1)) == 0u || tile + 1 == s_ntiles;
    };
    __shared__ long long s_next;                // first tile of the next chunk, or -1
    __shared__ unsigned s_claim;                // thread 0's claim for the chunk after this one
    unsigned claim = 0;                         // thread 0, until it parks it in s_claim
    bool claimed = !PL && tid == 0;
    if (claimed) claim = atomicAdd(counter(), 1u);

    const bool tma = L.rng[0].vec_ok != 0;   // all ranges of a launch agree (the host checks)
    if (tma) {
        if (tid == 0) {
            mbar_init(s_bar);
            fence_mbar_init();
        }
        __syncthreads();
    }
    auto pos_of = [&](int64_t t) {
        TilePos p;
        int r = 0;
        while (r + 1 < L.n_ranges && t >= L.rng[r + 1].tile0) ++r;
        const int64_t lt = t - L.rng[r].tile0;
        p.ri = r;
        p.row = lt / L.rng[r].tiles_per_row;
        p.col = lt - p.row * L.rng[r].tiles_per_row;
        return p;
    };
    TilePos pos = pos_of(tile);
    auto advance = [&](TilePos p) {
        if (++p.col == L.rng[p.ri].tiles_per_row) {
            p.col = 0;
            if (++p.row == L.rng[p.ri].n_dm) {
                p.row = 0;
                ++p.ri;
            }
        }
        return p;
    };
    // bulk copy of the window of the tile at p into the raw buffer (thread 0)
    auto issue = [&](const TilePos &p) {
        const RangeDesc &rd = L.rng[p.ri];
        const int64_t t0 = p.col * (int64_t)kTile;
        const int64_t have = min((int64_t)rd.span, rd.n_samp - t0);
        const uint32_t nb = (uint32_t)((have * esz) & ~(int64_t)15);
        fence_proxy_async();
        mbar_expect(s_bar, nb + L.extra_tx);
        if (nb) {
            const T *src = static_cast<const T *>(rd.data) + p.row * rd.stride + t0;
            bulk_load(s_raw, src, nb, s_bar);
        }
    };
    if (tma && tid == 0) issue(pos);
    // thread 0, once the current window is staged: the next tile's window into
    // the raw buffer, and at a chunk's last tile the next chunk for everyone
    auto issue_next = [&]() {
        int64_t nt = -1;
        if (!chunk_ends()) {
            nt = tile + 1;
        } else {
            if (!PL) {
                const unsigned v = s_claim;
                const int64_t ch = s_chunk;
                const int64_t n_chunks = (s_ntiles + ch - 1) / ch;
                const int64_t nc = (int64_t)gridDim.x + (int64_t)v;
                if (nc < n_chunks) nt = nc * ch;
                else if ((int64_t)v == n_chunks - 1) atomicExch(counter(), 0u);   // the last claim
            }
            s_next = nt;
        }
        if (tma && nt >= 0) issue(nt == tile + 1 ? advance(pos) : pos_of(nt));
    };

    int64_t key = -1;                       // (range, scope entry) of the constants loaded
    int64_t skey = -1;                      // (range, row) whose scale and offset are held
    float sc = 1.f, of = 0.f;
    // The candidates of a tile are written during the next tile: its first
    // barrier publishes the warps' counts, one thread reserves the tile's
    // slice of the list while the others stage, and after the staging barrier
    // each warp writes its records.  Until then they wait in registers: SNR
    // bits, widths (two per word), sample and row fields.
    constexpr int kAtomicThread = kThreads - 32;   // lane 0 of the last warp
    uint32_t pmask = 0, pbits[kX], pobk[MG ? kX / 4 : 1];
    int pdm = 0, psb = 0, psh = 0, pwtot = 0;
    // kAtomicThread: one atomic reserves the last tile's records; the warps'
    // slices are published from its result only after this thread's staging,
    // so that the round trip of the atomic (L2, possibly on the other die)
    // overlaps the staging instead of delaying this warp at the next barrier
    auto reserve = [&]() -> unsigned long long {
        int tot = 0;
#pragma unroll
        for (int w = 0; w < kThreads / 32; ++w) tot += s_wsum[w];
        return tot ? atomicAdd(reinterpret_cast<unsigned long long *>(&L.result->count),
                               (unsigned long long)tot)
                   : 0ull;
    };
    auto publish = [&](unsigned long long base) {   // s_wsum unchanged since reserve()
#pragma unroll
        for (int w = 0; w < kThreads / 32; ++w) {
            s_wbase[w] = base;
            base += (unsigned long long)s_wsum[w];
        }
    };
    auto flush = [&]() {     // a warp writes the last tile's records
        if (!pwtot) return;   // warp-uniform
        // records start index by start index: for start q the lanes holding a
        // candidate there write consecutive slots (rank among them by
        // ballot), so each store instruction is one coalesced run
        // unsigned: whatever the count word held before, no slot lies
        // outside out[0, capacity)
        const unsigned long long wb = s_wbase[warp];
        const unsigned long long cap = (unsigned long long)L.capacity;
        const unsigned long long room = wb >= cap ? 0ull : cap - wb;
        const int nroom = room < (unsigned long long)pwtot ? (int)room : pwtot;
        int4 *dst = reinterpret_cast<int4 *>(L.out) + wb;
        const uint32_t ltm = (1u << lane) - 1u;
        int off = 0;
#pragma unroll
        for (int q = 0; q < kX; ++q) {
            const bool has = (pmask >> q) & 1u;
            const uint32_t bal = __ballot_sync(0xffffffffu, has);
            const int slot = off + __popc(bal & ltm);
            if (has && slot < nroom) {
                // packed best: SNR truncated to 2^-17 and the width's code
                const int eb = MG ? 64 * (int)((pobk[q >> 2] >> (8 * (q & 3))) & 0xffu) : 0;
                dst[slot] = make_int4(pdm, psb + (q << psh), (int)(pbits[q] & 0xFFFFFFC0u),
                                      (int)s_ew[eb + 63 - (int)(pbits[q] & 63u)] << psh);
            }
            off += __popc(bal);
        }
        pwtot = 0;
    };
    for (int64_t k = 0;; ++k) {
        if (k) {   // the next tile: within the chunk, else the next chunk's first
            if (!chunk_ends()) {
                ++tile;
                pos = advance(pos);
            } else {
                const int64_t nt = s_next;   // written before the last barrier
                if (nt < 0) break;
                tile = nt;
                pos = pos_of(tile);
                claimed = !PL && tid == 0;
                if (claimed) claim = atomicAdd(counter(), 1u);
            }
        }
        const int ri = pos.ri;
        const RangeDesc &rd = L.rng[ri];
        const RangeProg &rp = rd.prog;
        const int R = rd.R;
        const int64_t row = pos.row;
        const int64_t t0 = pos.col * (int64_t)kTile;
        const int entry = rd.per_row ? (int)row : 0;
        const T *rowp = static_cast<const T *>(rd.data) + row * rd.stride + t0;

        // (A) the window has landed; every thread is done with the last tile
        if (tma) {
            const bool ok = tid != 0 || mbar_wait(s_bar, (uint32_t)(k & 1), L.wait_ns);
            if (__syncthreads_or(!ok)) {
                if (tid == 0) {
                    if (L.result) atomicExch(&L.result->status, (int)SPD_ERR_TIMEOUT);
                    mbar_wait(s_bar, (uint32_t)(k & 1), L.wait_ns);
                }
                return;
            }
        } else {
            __syncthreads();
        }
        bool held = !PL && k && tid == kAtomicThread;   // a reservation not yet published
        unsigned long long rbase = 0;
        if (held) rbase = reserve();
        {
            const int64_t nk = ((int64_t)ri << 32) | (uint32_t)entry;
            if (nk != key) {
                // the last tile's records read the widths it was searched with
                if (k) {
                    if (held) publish(rbase);
                    held = false;
                    __syncthreads();
                    flush();
                }
                if (tid == 0) {
                    s_mu = rd.mu_tab[entry];
                    s_deg = rd.flags[entry];
                }
                load_search_consts(rd, entry, RM, s_inv, s_gr, s_ew);   // barriers inside
                key = nk;
            }
        }
        if (s_deg) {   // degenerate sigma: no candidates (uniform across the CTA)
            if (held) publish(rbase);
            __syncthreads();
            if (claimed) s_claim = claim;
            claimed = false;
            if (tid == 0) issue_next();
            flush();
            if (PL && tid < U) {   // no SNR: NaN, width 0
                const int64_t i0 = t0 + (int64_t)tid * kX;
#pragma unroll
                for (int q = 0; q < kX; ++q) {
                    if (i0 + q < rd.n_samp) {
                        L.snr_out[row * L.out_stride + i0 + q] = __int_as_float(0x7fc00000);
                        L.width_out[row * L.out_stride + i0 + q] = 0;
                    }
                }
            }
            __syncthreads();   // every warp has read its slice before the counts change
            if (lane == 0) s_wsum[warp] = 0;
            continue;
        }
        if (rd.scale && (((int64_t)ri << 40 | row) != skey)) {
            sc = rd.scale[row];
            of = rd.offset ? rd.offset[row] : 0.f;
            skey = (int64_t)ri << 40 | row;
        }
        const bool has_sc = rd.scale != nullptr;
        const float2 mu = s_mu;
        const int have = (int)min((int64_t)rd.span, rd.n_samp - t0);
        const int nraw = tma ? (int)((((int64_t)have * esz) & ~(int64_t)15) / esz) : 0;
        const T *raw = reinterpret_cast<const T *>(s_raw);
        if (tid == 0) s_mag = 0;

        // ---- staging: one thread per block of 16 window positions
        for (int r = 0; r * kThreads < R; ++r) {
            const int c = r * kThreads + tid;
            if (r * kThreads + warp * 32 >= R) break;   // warp-uniform: the warp has no block
            float sum = 0.f, en = 0.f;
            if (c < R) {
                constexpr int NX = G > 1 ? 16 + G : 16;
                float v[NX];
                load_centred<DT, 16>(v, raw, rowp, 16 * c, nraw, have, has_sc, sc, of, mu);
                if (G > 1) load_centred<DT, G>(v + 16, raw, rowp, 16 * c + 16, nraw, have, has_sc,
                                               sc, of, mu);
                float Cp[NX + 1];      // in-block prefix: Cp[k] = v[0] + ... + v[k-1]
                Cp[0] = 0.f;
#pragma unroll
                for (int q = 0; q < NX; ++q) Cp[q + 1] = __fadd_rn(Cp[q], v[q]);
                sum = Cp[16];
                float hi = fmax3(Cp[0], Cp[1], Cp[2]), lo = fmin3(Cp[0], Cp[1], Cp[2]);
#pragma unroll
                for (int q = 3; q < 15; q += 2) {
                    hi = fmax3(hi, Cp[q], Cp[q + 1]);
                    lo = fmin3(lo, Cp[q], Cp[q + 1]);
                }
                hi = fmaxf(hi, Cp[15]);
                lo = fminf(lo, Cp[15]);
                if (16 * c + 16 <= have) {
                    float2 e2 = make_float2(0.f, 0.f);
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const float2 y2 = make_float2(v[2 * q], v[2 * q + 1]);
                        e2 = fma2(y2, y2, e2);
                    }
                    en = e2.x + e2.y;
                } else {   // the energy of the positions inside the row
#pragma unroll
                    for (int q = 0; q < 16; ++q) en += 16 * c + q < have ? v[q] * v[q] : 0.f;
                }
                float *yd = s_y + kSPad * c, *pd = s_p + kSPad * c;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    *reinterpret_cast<float4 *>(yd + 4 * u) =
                        make_float4(v[4 * u], v[4 * u + 1], v[4 * u + 2], v[4 * u + 3]);
                    *reinterpret_cast<float4 *>(pd + 4 * u) =
                        make_float4(Cp[4 * u], Cp[4 * u + 1], Cp[4 * u + 2], Cp[4 * u + 3]);
                }
                if (G > 1) {
                    float *gd = s_g + kSPad * c;
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const float2 a = add2(make_float2(Cp[4 * u + G], Cp[4 * u + 1 + G]),
                                              make_float2(-Cp[4 * u], -Cp[4 * u + 1]));
                        const float2 b = add2(make_float2(Cp[4 * u + 2 + G], Cp[4 * u + 3 + G]),
                                              make_float2(-Cp[4 * u + 2], -Cp[4 * u + 3]));
                        *reinterpret_cast<float4 *>(gd + 4 * u) = make_float4(a.x, a.y, b.x, b.y);
                    }
                }
                s_bs[c] = sum;
                s_rh[c] = hi;
                s_rl[c] = lo;
            }
            // inclusive warp scans of the block sums and energies; exclusive
            // values by shuffle (the block holding the window's end has sum
            // -inf, yet the prefix at its start is finite)
            float xs = sum, xq = en;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const float us = __shfl_up_sync(0xffffffffu, xs, o);
                const float uq = __shfl_up_sync(0xffffffffu, xq, o);
                if (lane >= o) {
                    xs += us;
                    xq += uq;
                }
            }
            const float es = __shfl_up_sync(0xffffffffu, xs, 1);
            const float eqv = __shfl_up_sync(0xffffffffu, xq, 1);
            if (lane == 31) {
                s_wt[c >> 5] = xs;
                s_wq[c >> 5] = xq;
            }
            if (c < R) {
                s_ex[c] = lane ? es : 0.f;
                s_eq[c] = lane ? eqv : 0.f;
            }
        }
        if (held) publish(rbase);
        if (claimed) s_claim = claim;   // the atomic's round trip overlapped the staging
        claimed = false;
        __syncthreads();   // (B)
        // the raw buffer is free: fetch the next tile's window
        if (tid == 0) issue_next();
        flush();           // the last tile's records, into the slice reserved above

        if (!PL) {   // the bounds' data (plane output evaluates every group)
            // ---- prefix values at block starts, their maxima, energy prefix
            {
                // prefix of the chunk totals, by a warp scan (at most 32 chunks)
                const int nch = (R + 31) >> 5;
                float ws = lane < nch ? s_wt[lane] : 0.f, wq = lane < nch ? s_wq[lane] : 0.f;
    #pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const float us = __shfl_up_sync(0xffffffffu, ws, o);
                    const float uq = __shfl_up_sync(0xffffffffu, wq, o);
                    if (lane >= o) {
                        ws += us;
                        wq += uq;
                    }
                }
                const int kl = KM < 3 ? KM : 3;
                float mag = 0.f;
                for (int r = 0; r * kThreads < R; ++r) {
                    const int c = r * kThreads + tid;
                    if (r * kThreads + warp * 32 >= R) break;   // warp-uniform
                    const int chunk = c >> 5;   // the same for the whole warp
                    // exclusive prefix of chunk `chunk` and of the next one
                    const float pre = __shfl_sync(0xffffffffu, ws, (chunk - 1) & 31);
                    const float pre_n = __shfl_sync(0xffffffffu, ws, chunk & 31);
                    const float preq = __shfl_sync(0xffffffffu, wq, (chunk - 1) & 31);
                    const float preq_n = __shfl_sync(0xffffffffu, wq, chunk & 31);
                    if (c >= R) continue;
                    const float P = (chunk ? pre : 0.f) + s_ex[c];
                    const float mx = P + s_rh[c];
                    const float mn = P + s_rl[c];
                    s_mx[c] = mx;
                    s_mn[c] = mn;
                    if (fabsf(mx) < INFINITY) mag = fmaxf(mag, fabsf(mx));
                    if (fabsf(mn) < INFINITY) mag = fmaxf(mag, fabsf(mn));
                    s_pq[c] = (chunk ? preq : 0.f) + s_eq[c];
                    if (c == R - 1) s_pq[R] = preq_n;
                    if (kl > 0) {
                        float m = mx;
    #pragma unroll
                        for (int j = 1; j < 8; ++j) {
                            if (j >= (1 << kl)) break;
                            const int b = min(c + j, R - 1);
                            const float Pb = ((b >> 5) == chunk ? (chunk ? pre : 0.f) : pre_n) + s_ex[b];
                            m = fmaxf(m, Pb + s_rh[b]);
                            if (j == 1) s_mx[RM + c] = m;
                            if (j == 3) s_mx[2 * RM + c] = m;
                            if (j == 7) s_mx[3 * RM + c] = m;
                        }
                    }
                }
    #pragma unroll
                for (int o = 16; o; o >>= 1) mag = fmaxf(mag, __shfl_xor_sync(0xffffffffu, mag, o));
                if (lane == 0) atomicMax(&s_mag, __float_as_int(mag));
            }
            __syncthreads();   // (C)
            for (int lv = 4; lv <= KM; ++lv) {
                const float *lo = s_mx + (lv - 1) * RM;
                const int h = 1 << (lv - 1);
                for (int c = tid; c < R; c += kThreads)
                    s_mx[lv * RM + c] = fmaxf(lo[c], lo[min(c + h, R - 1)]);
                __syncthreads();
            }
        }

        // ---- search of the unit's 16 starts (widest group first)
        const float thr = rd.threshold;
        const float minC = s_mn[tid];
        // the FP32 prefix values are off by at most ~30 roundings of the
        // tile's largest partial sum: the prefix bound adds twice that
        const float cslack = fmaf(8e-6f, __int_as_float(s_mag), 1e-30f) - minC;
        const float pq0 = s_pq[tid];
        const float *yb = s_y + kSPad * tid;
        float cb[kX];
        float ob[MG ? kX : 1];
        uint32_t obk[MG ? kX / 4 : 1];
#pragma unroll
        for (int q = 0; q < kX; ++q) cb[q] = -INFINITY;
        if (MG) {
#pragma unroll
            for (int q = 0; q < kX; ++q) ob[q] = -INFINITY;
#pragma unroll
            for (int q = 0; q < kX / 4; ++q) obk[q] = 0;
        }
        int cur_blk = -1;
        bool any = false;
        int lastO = -1;          // block offset of the last aligned group start, and its sum
        float lastD = 0.f;
        // bars of the bounds: lim with a relative margin, and its square (-1:
        // the energy bound cannot rule anything out when lim <= 0)
        float limv = thr;
        float lim_lo = thr - 1e-5f * fabsf(thr);
        float lim2 = thr > 0.f ? lim_lo * lim_lo : -1.f;
        auto merge_block = [&]() {
            // the block just searched holds smaller widths than every block
            // merged before: ties go to it
#pragma unroll
            for (int q = 0; q < kX; ++q) {
                if (trunc17(cb[q]) >= trunc17(ob[q])) {
                    ob[q] = cb[q];
                    obk[q >> 2] = (obk[q >> 2] & ~(0xffu << (8 * (q & 3)))) |
                                  ((uint32_t)cur_blk << (8 * (q & 3)));
                }
            }
        };
        // threads past the tile's units only stage (the halo blocks)
        for (int gi = tid < U ? rp.n_groups - 1 : -1; gi >= 0; --gi) {
            const int4 ga = s_gr[2 * gi];
            const int4 gb = s_gr[2 * gi + 1];
            if (!PL) {
                float rmax;
                if (gb.y >= 0) {
                    rmax = fmaxf(s_mx[tid + ga.z], s_mx[tid + ga.w]);
                } else {
                    rmax = -INFINITY;
                    for (int jb = tid + ga.z; jb <= tid + ga.w; ++jb) rmax = fmaxf(rmax, s_mx[jb]);
                }
                // prefix bound, with the margin for the rounding of the FP32
                // prefix; a non-positive bound caps every SNR at 0; NaN stays NaN
                const float pbound = fmaxf(rmax + cslack, 0.f) * __int_as_float(gb.z);
                // energy bound (squared); the prefix of energies is non-negative
                // and rounds by a few ulp of its larger end.  The factor covers
                // this group and all narrower ones, whose windows lie in the
                // same blocks
                const float ebound2 =
                    fmaf(s_pq[tid + gb.x], 1.000008f, -pq0) * __int_as_float(gb.w);
                if (ebound2 < lim2) break;
                // NaN bounds (windows past the row end) never prune
                if (pbound < lim_lo) continue;
            }
            Group g;
            g.off = (int16_t)(ga.x & 0xffff);
            g.count = (int16_t)(ga.x >> 16);
            g.widx0 = (int16_t)(ga.y & 0xffff);
            g.flags = (uint16_t)(ga.y >> 16);
            if (MG) {
                const int blk = g.widx0 >> 6;
                if (blk != cur_blk) {
                    if (cur_blk >= 0) merge_block();
#pragma unroll
                    for (int q = 0; q < kX; ++q) cb[q] = -INFINITY;
                    cur_blk = blk;
                }
            }
            if (!PL && (g.flags & kGroupRefine)) {
                float bq[kX];
#pragma unroll
                for (int q = 0; q < kX; ++q) bq[q] = MG ? fmaxf(cb[q], ob[q]) : cb[q];
                if (!refine16(yb, bq, thr, __int_as_float(gb.w))) continue;
            }
            any = true;
            float2 B[8];
            const bool coarse = G > 1 && (g.flags & kGroupCoarse);
            if (g.off == 0) {
#pragma unroll
                for (int j = 0; j < 8; ++j) B[j] = make_float2(0.f, 0.f);
            } else {
                float v[kX];
                if ((g.off & 15) == 0) {
                    const int o = g.off >> 4;
                    float D;
                    // widest group first: take off the blocks between.  Not
                    // from a sum that met the row end (-inf): the blocks of
                    // this group may all lie inside the row
                    if (lastO >= o && lastO - o <= 16 && lastD > -INFINITY) {
                        D = lastD;
                        for (int b = o; b < lastO; ++b) D = __fsub_rn(D, s_bs[tid + b]);
                    } else {
                        D = 0.f;
                        if (o <= 16) {
                            for (int b = 0; b < o; ++b) D = __fadd_rn(D, s_bs[tid + b]);
                        } else {   // Kahan-compensated in block order
                            float comp = 0.f;
                            for (int b = 0; b < o; ++b) {
                                const float y = __fsub_rn(s_bs[tid + b], comp);
                                const float sn = __fadd_rn(D, y);
                                comp = __fsub_rn(__fsub_rn(sn, D), y);
                                D = sn;
                            }
                        }
                    }
                    lastO = o;
                    lastD = D;
                    start_aligned(v, s_p, tid, o, D);
                } else {
                    start_generic(v, s_y, s_bs, tid, g.off);
                }
                const bool fine_al = !coarse && (g.off & 15) == 0;
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    B[j] = fine_al ? make_float2(v[j], v[j + 8]) : make_float2(v[2 * j], v[2 * j + 1]);
            }
            if (coarse) {
                if ((g.off & 15) == 0)
                    eval_coarse<(G > 1 ? G : 8)>(cb, B, s_g + kSPad * tid, g, s_inv);
                else
                    eval_generic(cb, B, s_g + kSPad * tid, g, G, s_inv);
            } else if ((g.off & 15) == 0) {
                eval_fine<true>(cb, B, yb, g, s_inv);
            } else {
                eval_generic(cb, B, yb, g, 1, s_inv);
            }
            // the bar rises to the smallest best of the unit
            if (PL) continue;
            float mb;
            if (MG) {
                mb = fmaxf(cb[0], ob[0]);
#pragma unroll
                for (int q = 1; q < kX; ++q) mb = fminf(mb, fmaxf(cb[q], ob[q]));
            } else {
                mb = fmin3(cb[0], cb[1], cb[2]);
#pragma unroll
                for (int q = 3; q < kX - 1; q += 2) mb = fmin3(mb, cb[q], cb[q + 1]);
                mb = fminf(mb, cb[kX - 1]);
            }
            mb = trunc17(mb);
            if (mb > limv) {
                limv = mb;
                lim_lo = mb - 1e-5f * fabsf(mb);
                lim2 = lim_lo * lim_lo;   // mb > thr: positive here when thr >= 0
                if (!(mb > 0.f)) lim2 = -1.f;
            }
        }
        if (MG && cur_blk >= 0) merge_block();

        if (PL) {   // every sample's best SNR (truncated to 2^-17) and its width
            const int64_t i0 = t0 + (int64_t)tid * kX;
            if (tid < U && i0 < rd.n_samp) {
                float snr[kX];
                int wdt[kX];
#pragma unroll
                for (int q = 0; q < kX; ++q) {
                    const uint32_t bits = __float_as_uint(MG ? ob[q] : cb[q]);
                    const int eb = MG ? 64 * (int)((obk[q >> 2] >> (8 * (q & 3))) & 0xffu) : 0;
                    const int wi = eb + 63 - (int)(bits & 63u);
                    snr[q] = __uint_as_float(bits & 0xFFFFFFC0u);
                    wdt[q] = wi < rp.n_eval ? (int)s_ew[wi] : 0;
                }
                float *so = L.snr_out + row * L.out_stride + i0;
                uint16_t *wo = L.width_out + row * L.out_stride + i0;
                const bool al = ((reinterpret_cast<uintptr_t>(so) | reinterpret_cast<uintptr_t>(wo)) &
                                 15) == 0;
                if (al && i0 + kX <= rd.n_samp) {
#pragma unroll
                    for (int v = 0; v < kX / 4; ++v)
                        reinterpret_cast<float4 *>(so)[v] =
                            make_float4(snr[4 * v], snr[4 * v + 1], snr[4 * v + 2], snr[4 * v + 3]);
#pragma unroll
                    for (int v = 0; v < kX / 8; ++v) {
                        uint4 u;
                        u.x = (uint32_t)wdt[8 * v] | ((uint32_t)wdt[8 * v + 1] << 16);
                        u.y = (uint32_t)wdt[8 * v + 2] | ((uint32_t)wdt[8 * v + 3] << 16);
                        u.z = (uint32_t)wdt[8 * v + 4] | ((uint32_t)wdt[8 * v + 5] << 16);
                        u.w = (uint32_t)wdt[8 * v + 6] | ((uint32_t)wdt[8 * v + 7] << 16);
                        reinterpret_cast<uint4 *>(wo)[v] = u;
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < kX; ++q) {
                        if (i0 + q < rd.n_samp) {
                            so[q] = snr[q];
                            wo[q] = (uint16_t)wdt[q];
                        }
                    }
                }
            }
            if (lane == 0) s_wsum[warp] = 0;
            continue;
        }

        // ---- threshold (Sec. 2.4, inclusive); the records wait for the next tile
        uint32_t mask = 0;
        if (any) {
            const int64_t ne = rd.n_emit - (t0 + (int64_t)tid * kX);
            const int lim = ne <= 0 ? 0 : (ne >= kX ? kX : (int)ne);
#pragma unroll
            for (int q = 0; q < kX; ++q) {
                const float bv = MG ? ob[q] : cb[q];
                if (trunc17(bv) >= thr) mask |= 1u << q;
            }
            if (lim < kX) mask &= (1u << lim) - 1u;
        }
        pmask = mask;
#pragma unroll
        for (int q = 0; q < kX; ++q) pbits[q] = __float_as_uint(MG ? ob[q] : cb[q]);
        if (MG) {
#pragma unroll
            for (int q = 0; q < kX / 4; ++q) pobk[q] = obk[q];
        }
        pdm = rd.dm_offset + (int)row;
        psh = rd.sample_shift;
        psb = (int)(rd.sample_base + ((t0 + (int64_t)tid * kX) << psh));
        pwtot = __reduce_add_sync(0xffffffffu, __popc(mask));
        if (lane == 0) s_wsum[warp] = pwtot;
    }
    if (PL) return;
    // the last tile's records
    __syncthreads();
    if (tid == kAtomicThread) publish(reserve());
    __syncthreads();
    flush();
}

template <int DT, int G, int NT, bool PL>
cudaError_t launch_sgn(const Launch &L, bool mg, size_t smem, int ctas_per_sm, cudaStream_t s) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    void (*k)(const Launch) =
        mg ? search_kernel<DT, G, true, NT, PL> : search_kernel<DT, G, false, NT, PL>;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, NT, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if (ctas_per_sm > 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
    // chunks of 1 to 16 tiles (a power of two), about 8 per CTA at least;
    // plane output: one run of tiles per CTA
    const int64_t gmax = (int64_t)sms * per_sm;
    int64_t ch = 16;
    while (ch > 1 && L.n_tiles < 8 * gmax * ch) ch >>= 1;
    if (PL) ch = 1;
    Launch Lc = L;
    Lc.chunk = (int32_t)ch;
    const int64_t n_chunks = (L.n_tiles + ch - 1) / ch;
    const int64_t grid = n_chunks < gmax ? n_chunks : gmax;
    if (grid < 1) return cudaSuccess;
    k<<<(unsigned)grid, NT, smem, s>>>(Lc);
    return cudaGetLastError();
}

template <int DT, int G>
cudaError_t launch_sg(const Launch &L, bool mg, size_t smem, int ctas_per_sm, int threads,
                      cudaStream_t s) {
    if (L.snr_out) return launch_sgn<DT, G, 256, true>(L, mg, smem, ctas_per_sm, s);
    return threads == 128 ? launch_sgn<DT, G, 128, false>(L, mg, smem, ctas_per_sm, s)
                          : launch_sgn<DT, G, 256, false>(L, mg, smem, ctas_per_sm, s);
}

}  // namespace

template <int DT>
cudaError_t launch_search_dt(const Launch &L, int G, bool multi_block, size_t smem,
                             int ctas_per_sm, int threads, cudaStream_t s) {
    switch (G) {
        case 8: return launch_sg<DT, 8>(L, multi_block, smem, ctas_per_sm, threads, s);
        case 16: return launch_sg<DT, 16>(L, multi_block, smem, ctas_per_sm, threads, s);
        default: return launch_sg<DT, 1>(L, multi_block, smem, ctas_per_sm, threads, s);
    }
}

}  // namespace spd
