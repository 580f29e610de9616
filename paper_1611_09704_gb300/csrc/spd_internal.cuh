// spd_internal.cuh -- device-side structures and launchers shared by the
// translation units of libspd.  Not part of the public ABI (include/spd.h).
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "spd.h"

namespace spd {

// ---------------------------------------------------------------- elements

// Value of a stored element as FP32: the raw value, or fmaf(scale, q, offset)
// when a per-row scale is given (FP16 / BF16 storage, Sec. "precision form").
template <int DT> struct Elem;
template <> struct Elem<SPD_F32> {
    using T = float;
    static __device__ __forceinline__ float cvt(T v) { return v; }
};
template <> struct Elem<SPD_F16> {
    using T = __half;
    static __device__ __forceinline__ float cvt(T v) { return __half2float(v); }
};
template <> struct Elem<SPD_BF16> {
    using T = __nv_bfloat16;
    static __device__ __forceinline__ float cvt(T v) { return __bfloat162float(v); }
};

inline size_t elem_bytes(int dt) { return dt == SPD_F32 ? 4 : 2; }

// ------------------------------------------------------------------- MSD

constexpr int kMsdThreads = 256;
constexpr int kMsdUnit = 65536;   // samples of one row per block-partial unit

// (n, T, S) of a piece of the data, Sec. 2.1, written per unit in FP64, plus
// the piece's smallest and largest value: sigma is exactly 0 iff they agree,
// a test that does not depend on how S was rounded.
struct MsdPart {
    double n, T, S, lo, hi;
};

struct MsdArgs {
    const void *data;
    int64_t n_dm, n_samp, stride;
    const float *scale, *offset;
    int64_t units_per_row;
    int vec_ok;          // 16-byte aligned rows: vector loads allowed
    MsdPart *parts;      // [n_dm * units_per_row]
};

// Arguments of the sigma_Nmax pass (Eq. 5): tiles of 4096 starts per row.
struct NmaxArgs {
    const void *data;
    int64_t n_dm, n_samp, stride;
    const float *scale, *offset;
    const spd_msd_stats *msd;   // mean used for centring, per scope entry
    int per_row;
    int vec_ok;                 // rows aligned for 4-element vector loads
    int nmax;
    int nb;                     // staged blocks of 16 samples per tile
    int64_t tiles_per_row;      // partials per row (each covers up to 8 tiles of 4096 starts)
    MsdPart *parts;             // [n_dm * tiles_per_row]
};

// ------------------------------------------------------------------ detect

constexpr int kX = 16;              // consecutive samples owned by one thread

// One group of evaluated widths (host-compiled from the width list).  The
// running boxcar sum B of every start sample i starts as
// B_off(i) = y[i] + ... + y[i+off-1] (read from the tile's compensated prefix
// sums) and then grows one step per member, as in Algorithm 1: from the
// centred samples y (step 1, positions off, off+1, ...) or from the G-sample
// window sums S_G (step G, positions off, off+G, ...).  Member c is the width
// off + (c+1) * step with eval index widx0 + c.  Groups are evaluated in any
// order; in the candidate search a group whose upper bound cannot reach the
// threshold or the current best is skipped.
struct Group {
    int16_t off;
    int16_t count;
    int16_t widx0;
    uint16_t flags;   // bit 0: step G (window sums), else step 1
};
constexpr uint16_t kGroupCoarse = 1;
constexpr uint16_t kGroupRefine = 2;   // widths 1..16 from off 0: per-sample energy test first

constexpr int kMaxCodeGroups = 64;          // groups a packed max can tell apart
constexpr int kMaxEval = SPD_MAX_WIDTHS + 1;
constexpr int kMaxRanges = 8;               // DM ranges searched by one launch

// The width groups of one range.  Member c of group g is the width
// g.off + (c + 1) * step (step G for coarse groups, else 1) with eval index
// g.widx0 + c; eval index 0 is width 1.
struct RangeProg {
    int32_t n_groups;
    int32_t n_eval;     // evaluated widths: width 1 first, then the listed ones
    int32_t wmax;
    int32_t G;          // step of the coarse window sums, 0 if unused
    Group groups[kMaxCodeGroups];
};

// One DM range (a plane with its own widths, MSD and threshold) of a launch.
struct RangeDesc {
    const void *data;
    int64_t n_dm, n_samp, stride;
    const float *scale, *offset;
    const float *inv_tab;       // [entries][n_eval]: 1 / sigma_w, FP32
    const float2 *mu_tab;       // [entries]: mean split into hi + lo FP32
    const int32_t *flags;       // [entries]: nonzero = degenerate sigma
    int64_t tile0;              // first launch-wide tile index of this range
    int64_t tiles_per_row;
    int32_t vec_ok;             // 16-byte aligned rows: bulk (TMA) copies allowed
    int32_t per_row;            // MSD scope entry = row (else entry 0)
    int32_t R;                  // blocks of 16 positions staged per tile
    int32_t span;               // positions of one tile's window (tile + wmax - 1)
    int32_t dm_offset;          // added to the row index in candidate records
    float threshold;
    int64_t n_emit;             // only starts < n_emit become candidates (n_samp normally)
    int64_t sample_base;        // added to the start sample in candidate records
    int32_t sample_shift;       // records carry start << shift and width << shift
    int32_t reserved0;
    RangeProg prog;
};

// Everything one detect launch needs, passed by value as a __grid_constant__
// kernel parameter (no host-to-device copy of its own, so it can be captured
// in a CUDA graph).
struct Launch {
    int32_t n_ranges;
    int32_t R;                  // shared arrays sized for the widest range
    int32_t raw_bytes;          // bytes of one raw staging buffer (multiple of 16)
    int32_t max_eval;
    int64_t n_tiles;
    spd_candidate *out;
    int64_t capacity;
    spd_result *result;
    float *snr_out;             // plane output (single range) or null
    uint16_t *width_out;
    int64_t out_stride;
    uint64_t wait_ns;           // bound of a wait for a bulk copy
    uint32_t extra_tx;          // test aid: bytes expected beyond each copy (0 in use)
    int32_t kmax;               // search kernel: levels of the block max table
    int32_t units;              // search kernel: units of 16 starts per tile (<= threads)
    int32_t chunk;              // search kernel: tiles per scheduling chunk (set at launch)
    RangeDesc rng[kMaxRanges];
};

// ------------------------------------------------------------ search kernel

constexpr int kSPad = 20;          // shared words per 16 positions (4 padding words)
constexpr int kSLevels = 5;        // block max table: windows of up to 2^5 blocks

// Bound geometry of one width group (Group) of step d, for the unit of 16
// starts 16t .. 16t+15: its windows end in blocks t + a .. t + b and lie in
// blocks t .. t + e - 1.  The largest block prefix over [t + a, t + b] is
// read as the max of two table windows of 2^lvl blocks at t + a and t + bk
// (lvl = -1: a plain loop over the blocks, for spans longer than the table).
struct GroupGeom {
    int a, bk, lvl, e;
};
__host__ __device__ inline GroupGeom group_geom(int off, int count, int d) {
    GroupGeom q;
    q.a = (off + d) >> 4;
    const int b = (15 + off + count * d) >> 4;
    const int len = b - q.a + 1;
    q.lvl = -1;
    q.bk = b;
    if (len <= (2 << kSLevels)) {
        int k = 0;
        while ((2 << k) <= len) ++k;   // floor(log2(len))
        if (k > kSLevels) k = kSLevels;
        q.lvl = k;
        q.bk = b - (1 << k) + 1;
    }
    q.e = 1 + ((14 + off + count * d) >> 4);
    return q;
}

// Shared memory of one search CTA, in the order the kernel lays it out:
// mbarrier (16 B), one raw staging buffer, then FP32 arrays -- centred samples
// y, in-block prefix sums P and (G > 1) G-sample window sums, each 20 words
// per 16 positions; per block: sums, prefix maxima (level 0 of the table) and
// kmax table levels, prefix minima, energy prefix (RM + 4), four scan
// temporaries; 1/sigma_w per eval index -- then per group two int4 of
// evaluation and bound data, and the width per eval index (uint16).
// RM is a multiple of 4.
struct SearchSmem {
    size_t raw, y, p, g, bs, mx, mn, pq, ex, eq, rh, rl, inv, gr, ew, total;
};
__host__ __device__ inline SearchSmem search_smem(int RM, int raw_bytes, int max_eval, int kmax,
                                                  int G) {
    SearchSmem m;
    const size_t blk = (size_t)kSPad * RM * sizeof(float);
    const size_t arr = (size_t)RM * sizeof(float);
    m.raw = 16;
    m.y = m.raw + (size_t)raw_bytes;
    m.p = m.y + blk;
    m.g = m.p + blk;
    m.bs = m.g + (G > 1 ? blk : 0);
    m.mx = m.bs + arr;                       // level 0; levels 1..kmax follow
    m.mn = m.mx + (size_t)(1 + kmax) * arr;
    m.pq = m.mn + arr;
    m.ex = m.pq + arr + 16;
    m.eq = m.ex + arr;
    m.rh = m.eq + arr;
    m.rl = m.rh + arr;
    m.inv = m.rl + arr;
    m.gr = m.inv + (((size_t)max_eval * sizeof(float) + 15) & ~(size_t)15);
    m.ew = m.gr + (size_t)kMaxCodeGroups * 32;
    m.total = (m.ew + (size_t)max_eval * sizeof(uint16_t) + 15) & ~(size_t)15;
    return m;
}
inline size_t search_smem_bytes(int RM, int raw_bytes, int max_eval, int kmax, int G) {
    return search_smem(RM, raw_bytes, max_eval, kmax, G).total;
}

struct ConstArgs {
    const spd_msd_stats *msd;   // [entries]
    int entries;
    int sigma_mode;
    float *inv_tab;
    float2 *mu_tab;
    int32_t *flags;
    spd_result *result;   // may be null: status set on a degenerate entry (count untouched)
    int skip_w1;          // eval index 0 (the width-1 start) takes no part: 1/sigma = NaN
};

// Launchers (return cudaGetLastError() of the launch).
cudaError_t launch_msd_partial(const MsdArgs &a, int dtype, cudaStream_t s);
cudaError_t launch_msd_merge(const MsdPart *parts, int64_t n_dm, int64_t units_per_row,
                             int64_t n_samp, int per_row, MsdPart *scratch, int n_scratch,
                             spd_msd_stats *out, cudaStream_t s);
cudaError_t launch_consts(const ConstArgs &a, const RangeProg &prog, cudaStream_t s);
cudaError_t launch_stream_msd(const MsdPart *parts, int64_t n_dm, int64_t upr, int per_row,
                              MsdPart *state, spd_msd_stats *out, cudaStream_t s);
cudaError_t launch_zero_parts(MsdPart *p, int64_t n, cudaStream_t s);
int nmax_blocks(int nmax);
// sigma_Nmax partials per row (CTAs of the partial kernel per row).
int64_t nmax_tiles_per_row(int64_t n_samp);
cudaError_t launch_nmax_partial(const NmaxArgs &a, int dtype, cudaStream_t s);
// Fold n_parts partials into *out (the block tree of the final merge).
cudaError_t launch_fold_parts(const MsdPart *parts, int64_t n_parts, MsdPart *scratch,
                              int n_scratch, MsdPart *out, cudaStream_t s);
// Shard partials in shard order -> mean/sd (what 0) or sd_nmax (what 1).
cudaError_t launch_merge_shards(const MsdPart *parts, int n, int what, int nmax,
                                spd_msd_stats *out, cudaStream_t s);
cudaError_t launch_nmax(const NmaxArgs &a, int dtype, MsdPart *scratch, int n_scratch,
                        spd_msd_stats *out, cudaStream_t s);
// The candidate search (search kernel): same launch description with the
// ranges' tiles of 16 * threads starts (threads = 128 or 256), kmax set.
cudaError_t launch_search(const Launch &L, int dtype, int G, bool multi_block, size_t smem,
                          int ctas_per_sm, int threads, cudaStream_t s);
constexpr int kSearchThreads = 256;   // threads of a search CTA by default
// x[2j] + x[2j+1] of a plane (dequantised) into an FP32 plane, j < n_out.
cudaError_t launch_decimate2(const spd_plane &p, float *dst, int64_t n_out, int64_t dst_stride,
                             cudaStream_t s);
cudaError_t launch_threshold_plane(float *snr, uint16_t *width, int64_t n_dm, int64_t n_samp,
                                   int64_t stride, float thr, cudaStream_t s);
cudaError_t launch_threshold(const float *snr, const uint16_t *width, int64_t n_dm,
                             int64_t n_samp, int64_t stride, float thr, spd_candidate *out,
                             int64_t capacity, spd_result *result, cudaStream_t s);
// Per-DM clustering of the candidates of an SNR plane (one warp per row).
cudaError_t launch_cluster(const float *snr, const uint16_t *width, int64_t n_dm,
                           int64_t n_samp, int64_t stride, float thr, int64_t gap,
                           spd_cluster *out, int64_t capacity, spd_result *result,
                           cudaStream_t s);
cudaError_t launch_boxcar_sums(const spd_plane &p, int w, float *out, int64_t out_stride,
                               cudaStream_t s);

}  // namespace spd
