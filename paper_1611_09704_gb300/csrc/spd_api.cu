// spd_api.cu -- host side of the C ABI declared in include/spd.h: argument
// validation, the width program (how the running boxcar sums grow from one
// listed width to the next), workspace layout and kernel launches.
#include "spd_internal.cuh"

#include <math.h>
#include <stdint.h>
#include <string.h>

#include <vector>

using namespace spd;

static_assert(sizeof(spd_msd_part) == sizeof(spd::MsdPart), "spd_msd_part layout");
static_assert(sizeof(spd_cluster) == 32, "spd_cluster layout");

namespace {

thread_local int g_last_cuda_error = 0;

spd_status cuda_fail(cudaError_t e) {
    g_last_cuda_error = (int)e;
    return SPD_ERR_CUDA;
}

#define SPD_CK(x)                                        \
    do {                                                 \
        cudaError_t e_ = (x);                            \
        if (e_ != cudaSuccess) return cuda_fail(e_);     \
    } while (0)

#define SPD_TRY(x)                                       \
    do {                                                 \
        spd_status s_ = (x);                             \
        if (s_ != SPD_OK) return s_;                     \
    } while (0)

constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

bool plane_empty(const spd_plane *p) { return p->n_dm == 0 || p->n_samp == 0; }

spd_status check_plane(const spd_plane *p) {
    if (!p) return SPD_ERR_INVALID_ARG;
    if (p->dtype < SPD_F32 || p->dtype > SPD_BF16) return SPD_ERR_INVALID_ARG;
    if (p->n_dm < 0 || p->n_samp < 0) return SPD_ERR_INVALID_ARG;
    if (p->n_dm > INT32_MAX || p->n_samp > INT32_MAX) return SPD_ERR_INVALID_ARG;
    if (plane_empty(p)) return SPD_OK;
    if (!p->data || p->row_stride < p->n_samp) return SPD_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(p->data) % elem_bytes(p->dtype)) return SPD_ERR_INVALID_ARG;
    if (p->row_offset && !p->row_scale) return SPD_ERR_INVALID_ARG;
    return SPD_OK;
}

int plane_vec_ok(const spd_plane *p) {
    const size_t eb = elem_bytes(p->dtype);
    const size_t need = 4 * eb;   // four elements per vector load
    return (reinterpret_cast<uintptr_t>(p->data) % need == 0) &&
           ((size_t)p->row_stride * eb) % need == 0;
}

int64_t entries_of(const spd_plane *p, int scope) { return scope == SPD_MSD_PER_ROW ? p->n_dm : 1; }

bool scope_ok(int scope) { return scope == SPD_MSD_GLOBAL || scope == SPD_MSD_PER_ROW; }

// ------------------------------------------------------------ MSD workspace

struct MsdLayout {
    int64_t upr;           // units per row
    int64_t ntpr;          // sigma_Nmax tiles per row (0 when not measured)
    size_t parts_off, scratch_off, nmax_off, total;
};
constexpr int kMergeScratch = 256;

MsdLayout msd_layout(const spd_plane *p, int nmax = 0) {
    MsdLayout l;
    l.upr = p->n_samp > 0 ? (p->n_samp + kMsdUnit - 1) / kMsdUnit : 0;
    l.ntpr = nmax >= 2 ? nmax_tiles_per_row(p->n_samp) : 0;
    const size_t parts = (size_t)(p->n_dm * l.upr) * sizeof(MsdPart);
    l.parts_off = 0;
    l.scratch_off = align_up(parts);
    l.nmax_off = l.scratch_off + align_up(kMergeScratch * sizeof(MsdPart));
    l.total = l.nmax_off + align_up((size_t)(p->n_dm * l.ntpr) * sizeof(MsdPart));
    return l;
}

// ----------------------------------------------------------- width program

// Evaluated widths are width 1 (the starting value of Algorithm 1) followed
// by the listed widths.  They are cut into groups of consecutive widths that
// step by 1 (the running sum adds one sample per width) or by G (it adds one
// G-sample window sum); a group's sums start from the block sums at `off`.
// Groups hold at most 16 (step 1) widths times `scale`, and at most
// 4 (16/G + 1) (step G; plane output) or 4 (candidate search, where each group
// has its own bound) widths times `scale`; `scale` doubles until there are at
// most 64 groups, and groups never cross a multiple of 64 in eval index.  G is
// the most frequent step of 8 or 16, if any.  In the candidate search the
// group of widths 1..16 is marked for the per-sample energy test.
spd_status compile_program(const int32_t *widths, int32_t n, RangeProg &prog, int scale0 = 1,
                           bool search = false) {
    if (!widths || n < 1 || n > SPD_MAX_WIDTHS) return SPD_ERR_INVALID_ARG;
    for (int k = 0; k < n; ++k) {
        if (widths[k] < 1 || widths[k] > SPD_MAX_WIDTH) return SPD_ERR_INVALID_ARG;
        if (k && widths[k] <= widths[k - 1]) return SPD_ERR_INVALID_ARG;
    }
    std::vector<int> E;
    if (widths[0] != 1) E.push_back(1);
    for (int k = 0; k < n; ++k) E.push_back(widths[k]);
    const int ne = (int)E.size();

    int n8 = 0, n16 = 0;
    for (int k = 1; k < ne; ++k) {
        n8 += E[k] - E[k - 1] == 8;
        n16 += E[k] - E[k - 1] == 16;
    }
    const int G = (n8 || n16) ? (n8 >= n16 ? 8 : 16) : 0;

    std::vector<Group> groups;
    for (int scale = scale0 < 1 ? 1 : scale0;; scale *= 2) {
        // coarse groups hold 4 (16 / G + 1) widths at scale 1: their start and
        // merge cost more than a fine group's relative to their widths
        const int max_fine = 16 * scale;
        const int max_coarse = (G ? (search ? 4 : 4 * (16 / G + 1)) : 1) * scale;
        groups.clear();
        for (int k = 0; k < ne; ++k) {
            const int step = k ? E[k] - E[k - 1] : 1;
            if (!groups.empty()) {
                Group &g = groups.back();
                const bool coarse = g.flags & kGroupCoarse;
                const bool fits = coarse ? (G && step == G && g.count < max_coarse)
                                         : (step == 1 && g.count < max_fine);
                if (fits && (k >> 6) == (g.widx0 >> 6)) {
                    g.count++;
                    continue;
                }
            }
            Group g;
            const bool coarse = G && step == G;
            g.off = (int16_t)(E[k] - (coarse ? G : 1));
            g.count = 1;
            g.widx0 = (int16_t)k;
            g.flags = coarse ? kGroupCoarse : 0;
            groups.push_back(g);
        }
        if ((int)groups.size() <= kMaxCodeGroups) break;
        if (max_fine > SPD_MAX_WIDTHS) return SPD_ERR_UNSUPPORTED;   // irregular lists
    }

    memset(&prog, 0, sizeof(prog));
    prog.n_groups = (int)groups.size();
    prog.n_eval = ne;
    prog.wmax = E.back();
    prog.G = G;
    for (size_t i = 0; i < groups.size(); ++i) {
        Group g = groups[i];
        if (search && !(g.flags & kGroupCoarse) && g.off == 0 && g.count == 16)
            g.flags |= kGroupRefine;
        prog.groups[i] = g;
    }
    return SPD_OK;
}

// Highest block max table level any group of a program reads (0: none).
int prog_kmax(const RangeProg &prog) {
    int k = 0;
    for (int i = 0; i < prog.n_groups; ++i) {
        const Group &g = prog.groups[i];
        const int d = (g.flags & kGroupCoarse) ? prog.G : 1;
        const GroupGeom q = group_geom(g.off, g.count, d);
        if (q.lvl > k) k = q.lvl;
    }
    return k;
}

// Bytes of the raw staging buffer for a window of `span` positions (whole
// 16-byte pieces).
int raw_bytes_of(int span, int dtype) { return (int)((span * elem_bytes(dtype) + 15) / 16 * 16); }

// --------------------------------------------------------- detect workspace

struct DetLayout {
    size_t inv_off, mu_off, flags_off, total;
};

DetLayout det_layout(int64_t entries, int n_eval) {
    DetLayout l;
    l.inv_off = 0;
    l.mu_off = align_up((size_t)entries * n_eval * sizeof(float));
    l.flags_off = l.mu_off + align_up((size_t)entries * sizeof(float2));
    l.total = l.flags_off + align_up((size_t)entries * sizeof(int32_t));
    return l;
}

spd_status check_ws(const void *ws, size_t have, size_t need) {
    if (need == 0) return SPD_OK;
    if (!ws) return SPD_ERR_NO_MEMORY;
    if (reinterpret_cast<uintptr_t>(ws) % kAlign) return SPD_ERR_INVALID_ARG;
    if (have < need) return SPD_ERR_NO_MEMORY;
    return SPD_OK;
}

spd_status check_params(const spd_search_params *q) {
    if (!q) return SPD_ERR_INVALID_ARG;
    if (!isfinite(q->threshold)) return SPD_ERR_INVALID_ARG;
    if (q->sigma_mode < SPD_SIGMA_SQRTN || q->sigma_mode > SPD_SIGMA_LINEAR_EXCESS)
        return SPD_ERR_INVALID_ARG;
    if (!scope_ok(q->msd_scope)) return SPD_ERR_INVALID_ARG;
    if (q->nmax_sigma < 0 || q->nmax_sigma == 1 || q->nmax_sigma > SPD_MAX_WIDTH)
        return SPD_ERR_INVALID_ARG;
    return SPD_OK;
}

int nmax_of(const spd_search_params *q) {
    if (q->sigma_mode == SPD_SIGMA_SQRTN) return 0;
    if (q->nmax_sigma) return q->nmax_sigma;
    return q->widths && q->n_widths > 0 ? q->widths[q->n_widths - 1] : 0;
}

// Constants kernel for one range: 1/sigma_w per entry and width, mean, flags.
spd_status range_consts(const spd_plane *p, const RangeProg &prog, const spd_msd_stats *msd_dev,
                        int scope, int sigma_mode, spd_result *result, void *ws,
                        cudaStream_t st, RangeDesc &rd, int skip_w1 = 0) {
    const int64_t entries = entries_of(p, scope);
    const DetLayout L = det_layout(entries, prog.n_eval);
    char *base = static_cast<char *>(ws);
    ConstArgs c;
    c.msd = msd_dev;
    c.entries = (int)entries;
    c.sigma_mode = sigma_mode;
    c.inv_tab = reinterpret_cast<float *>(base + L.inv_off);
    c.mu_tab = reinterpret_cast<float2 *>(base + L.mu_off);
    c.flags = reinterpret_cast<int32_t *>(base + L.flags_off);
    c.result = result;
    c.skip_w1 = skip_w1;
    SPD_CK(launch_consts(c, prog, st));

    memset(&rd, 0, sizeof(rd));
    rd.data = p->data;
    rd.n_dm = p->n_dm;
    rd.n_samp = p->n_samp;
    rd.stride = p->row_stride;
    rd.scale = p->row_scale;
    rd.offset = p->row_offset;
    rd.inv_tab = c.inv_tab;
    rd.mu_tab = c.mu_tab;
    rd.flags = c.flags;
    rd.tiles_per_row = 0;   // the tile geometry is set by run_launch
    rd.vec_ok = plane_vec_ok(p);
    rd.per_row = scope == SPD_MSD_PER_ROW;
    rd.R = 0;
    rd.span = 0;
    rd.n_emit = p->n_samp;
    rd.sample_base = 0;
    rd.sample_shift = 0;
    rd.prog = prog;
    return SPD_OK;
}

// Bound of a wait for a bulk copy, and bytes expected beyond each copy (a
// test aid that makes the waits run out); set by spd_debug_set_copy_wait.
thread_local uint64_t g_wait_ns = 2000000000ull;
thread_local uint32_t g_extra_tx = 0;

// One search-kernel launch over ranges rd[0 .. n) (same storage type and G):
// candidates, or with snr_out the plane output (every group evaluated).
// Tiles of 16 starts per unit, units = the threads (128 or 256, 0 = the
// default; plane output 256) less the halo's blocks.
spd_status run_launch(const RangeDesc *rd, int n, int dtype, spd_candidate *out, int64_t cap,
                      spd_result *result, float *snr_out, uint16_t *width_out,
                      int64_t out_stride, int ctas_per_sm, cudaStream_t st, int threads = 0) {
    static thread_local Launch L;
    memset(&L, 0, sizeof(L));
    const int nt = !snr_out && (threads == 128 || threads == 256) ? threads : kSearchThreads;
    // candidate search: U units of 16 starts per tile, the threads less the
    // widest range's halo blocks when that leaves one block per thread
    int halo = 0;
    for (int i = 0; i < n; ++i) {
        const int h = (rd[i].prog.wmax + 32 + 15) / 16 + 1;
        halo = h > halo ? h : halo;
    }
    const int units = halo <= 64 ? nt - halo : nt;
    int64_t tiles = 0;
    int R = 0, raw = 0, max_eval = 0, G = rd[0].prog.G;
    for (int i = 0; i < n; ++i) {
        L.rng[i] = rd[i];
        const int tile = kX * units;
        L.rng[i].tiles_per_row = (rd[i].n_samp + tile - 1) / tile;
        L.rng[i].R = (tile + rd[i].prog.wmax + 32 + 15) / 16 + 1;
        // the window rounded up to whole 16-byte pieces: one bulk copy brings
        // all of it (a tail fetched by plain loads would put a global-memory
        // latency into every tile's staging); the extra samples lie in no
        // evaluated window
        const int per16 = 16 / (int)elem_bytes(dtype);
        L.rng[i].span = (tile + rd[i].prog.wmax - 1 + per16 - 1) / per16 * per16;
        L.rng[i].tile0 = tiles;
        tiles += L.rng[i].n_dm * L.rng[i].tiles_per_row;
        R = L.rng[i].R > R ? L.rng[i].R : R;
        const int rb = raw_bytes_of(L.rng[i].span, dtype);
        raw = rb > raw ? rb : raw;
        max_eval = rd[i].prog.n_eval > max_eval ? rd[i].prog.n_eval : max_eval;
    }
    L.n_ranges = n;
    L.R = R;
    L.raw_bytes = raw;
    L.max_eval = max_eval;
    L.n_tiles = tiles;
    L.out = out;
    L.capacity = cap;
    L.result = result;
    L.snr_out = snr_out;
    L.width_out = width_out;
    L.out_stride = out_stride;
    L.wait_ns = g_wait_ns;
    L.extra_tx = g_extra_tx;
    // plane output (every sample's best SNR and width) evaluates every group
    // and needs no bound tables
    int kmax = 0;
    for (int i = 0; i < n && !snr_out; ++i) {
        const int k = prog_kmax(rd[i].prog);
        kmax = k > kmax ? k : kmax;
    }
    L.R = (R + 3) & ~3;
    L.kmax = kmax;
    L.units = units;
    const size_t smem = search_smem_bytes(L.R, raw, max_eval, kmax, G);
    if (smem > 227 * 1024) return SPD_ERR_UNSUPPORTED;
    SPD_CK(launch_search(L, dtype, G, max_eval > 64, smem, ctas_per_sm, nt, st));
    return SPD_OK;
}

// Constants + one detect launch over one plane (plane output or candidates).
spd_status run_detect(const spd_plane *p, const RangeProg &prog, const spd_msd_stats *msd_dev,
                      int scope, int sigma_mode, float thr, spd_candidate *out, int64_t cap,
                      spd_result *result, float *snr_out, uint16_t *width_out,
                      int64_t out_stride, void *ws, cudaStream_t st) {
    RangeDesc rd;
    SPD_TRY(range_consts(p, prog, msd_dev, scope, sigma_mode, result, ws, st, rd));
    rd.threshold = thr;
    return run_launch(&rd, 1, p->dtype, out, cap, result, snr_out, width_out, out_stride, 0, st);
}

}  // namespace

namespace spd {
// Records a CUDA error for spd_last_cuda_error from other translation units.
void note_cuda_error(int e) { g_last_cuda_error = e; }
}  // namespace spd

extern "C" {

int32_t spd_version(void) { return SPD_VERSION; }

const char *spd_status_string(int32_t s) {
    switch (s) {
        case SPD_OK: return "ok";
        case SPD_ERR_INVALID_ARG: return "invalid argument";
        case SPD_ERR_CUDA: return "CUDA error";
        case SPD_ERR_NO_MEMORY: return "workspace too small";
        case SPD_ERR_OVERFLOW: return "more candidates than capacity";
        case SPD_ERR_DEGENERATE_SIGMA: return "degenerate standard deviation";
        case SPD_ERR_TIMEOUT: return "device wait timed out";
        case SPD_ERR_UNSUPPORTED: return "unsupported request";
        default: return "unknown status";
    }
}

int32_t spd_last_cuda_error(void) { return g_last_cuda_error; }

size_t spd_msd_workspace_bytes(const spd_plane *plane, int32_t scope, int32_t nmax_sigma) {
    if (check_plane(plane) != SPD_OK || !scope_ok(scope)) return 0;
    if (nmax_sigma < 0 || nmax_sigma == 1 || nmax_sigma > SPD_MAX_WIDTH) return 0;
    return msd_layout(plane, nmax_sigma).total;
}

spd_status spd_msd(const spd_plane *plane, int32_t scope, int32_t nmax_sigma,
                   spd_msd_stats *out_dev, void *workspace, size_t workspace_bytes, void *stream) {
    SPD_TRY(check_plane(plane));
    if (!scope_ok(scope) || !out_dev) return SPD_ERR_INVALID_ARG;
    if (nmax_sigma < 0 || nmax_sigma == 1 || nmax_sigma > SPD_MAX_WIDTH)
        return SPD_ERR_INVALID_ARG;
    const MsdLayout L = msd_layout(plane, nmax_sigma);
    SPD_TRY(check_ws(workspace, workspace_bytes, L.total));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char *base = static_cast<char *>(workspace);
    MsdPart *parts = reinterpret_cast<MsdPart *>(base + L.parts_off);
    MsdPart *scratch = reinterpret_cast<MsdPart *>(base + L.scratch_off);
    if (!plane_empty(plane)) {
        MsdArgs a;
        a.data = plane->data;
        a.n_dm = plane->n_dm;
        a.n_samp = plane->n_samp;
        a.stride = plane->row_stride;
        a.scale = plane->row_scale;
        a.offset = plane->row_offset;
        a.units_per_row = L.upr;
        a.vec_ok = plane_vec_ok(plane);
        a.parts = parts;
        SPD_CK(launch_msd_partial(a, plane->dtype, st));
    }
    if (scope == SPD_MSD_PER_ROW && plane->n_dm == 0) return SPD_OK;
    SPD_CK(launch_msd_merge(parts, plane->n_dm, L.upr, plane->n_samp,
                            scope == SPD_MSD_PER_ROW, scratch, kMergeScratch, out_dev, st));
    if (nmax_sigma >= 2 && !plane_empty(plane)) {
        // sigma_Nmax of Eq. 5, centred on the mean just merged
        NmaxArgs n;
        n.data = plane->data;
        n.n_dm = plane->n_dm;
        n.n_samp = plane->n_samp;
        n.stride = plane->row_stride;
        n.scale = plane->row_scale;
        n.offset = plane->row_offset;
        n.msd = out_dev;
        n.per_row = scope == SPD_MSD_PER_ROW;
        n.vec_ok = plane_vec_ok(plane);
        n.nmax = nmax_sigma;
        n.nb = nmax_blocks(nmax_sigma);
        n.tiles_per_row = L.ntpr;
        n.parts = reinterpret_cast<MsdPart *>(base + L.nmax_off);
        SPD_CK(launch_nmax(n, plane->dtype, scratch, kMergeScratch, out_dev, st));
    }
    return SPD_OK;
}

spd_status spd_msd_shard_partial(const spd_plane *plane, spd_msd_part *part_dev, void *workspace,
                                 size_t workspace_bytes, void *stream) {
    SPD_TRY(check_plane(plane));
    if (!part_dev) return SPD_ERR_INVALID_ARG;
    const MsdLayout L = msd_layout(plane, 0);
    SPD_TRY(check_ws(workspace, workspace_bytes, L.total));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char *base = static_cast<char *>(workspace);
    MsdPart *parts = reinterpret_cast<MsdPart *>(base + L.parts_off);
    MsdPart *scratch = reinterpret_cast<MsdPart *>(base + L.scratch_off);
    MsdPart *out = reinterpret_cast<MsdPart *>(part_dev);
    if (plane_empty(plane)) {
        SPD_CK(launch_zero_parts(out, 1, st));
        return SPD_OK;
    }
    MsdArgs a;
    a.data = plane->data;
    a.n_dm = plane->n_dm;
    a.n_samp = plane->n_samp;
    a.stride = plane->row_stride;
    a.scale = plane->row_scale;
    a.offset = plane->row_offset;
    a.units_per_row = L.upr;
    a.vec_ok = plane_vec_ok(plane);
    a.parts = parts;
    SPD_CK(launch_msd_partial(a, plane->dtype, st));
    SPD_CK(launch_fold_parts(parts, plane->n_dm * L.upr, scratch, kMergeScratch, out, st));
    return SPD_OK;
}

spd_status spd_msd_merge_partials(const spd_msd_part *parts_dev, int32_t n_shards,
                                  spd_msd_stats *out_dev, void *stream) {
    if (!parts_dev || !out_dev || n_shards < 1) return SPD_ERR_INVALID_ARG;
    SPD_CK(launch_merge_shards(reinterpret_cast<const MsdPart *>(parts_dev), n_shards, 0, 0,
                               out_dev, static_cast<cudaStream_t>(stream)));
    return SPD_OK;
}

spd_status spd_sd_nmax_shard_partial(const spd_plane *plane, int32_t nmax_sigma,
                                     const spd_msd_stats *msd_dev, spd_msd_part *part_dev,
                                     void *workspace, size_t workspace_bytes, void *stream) {
    SPD_TRY(check_plane(plane));
    if (!part_dev || !msd_dev || nmax_sigma < 2 || nmax_sigma > SPD_MAX_WIDTH)
        return SPD_ERR_INVALID_ARG;
    const MsdLayout L = msd_layout(plane, nmax_sigma);
    SPD_TRY(check_ws(workspace, workspace_bytes, L.total));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char *base = static_cast<char *>(workspace);
    MsdPart *scratch = reinterpret_cast<MsdPart *>(base + L.scratch_off);
    MsdPart *out = reinterpret_cast<MsdPart *>(part_dev);
    if (plane_empty(plane)) {
        SPD_CK(launch_zero_parts(out, 1, st));
        return SPD_OK;
    }
    NmaxArgs n;
    n.data = plane->data;
    n.n_dm = plane->n_dm;
    n.n_samp = plane->n_samp;
    n.stride = plane->row_stride;
    n.scale = plane->row_scale;
    n.offset = plane->row_offset;
    n.msd = msd_dev;
    n.per_row = 0;
    n.vec_ok = plane_vec_ok(plane);
    n.nmax = nmax_sigma;
    n.nb = nmax_blocks(nmax_sigma);
    n.tiles_per_row = L.ntpr;
    n.parts = reinterpret_cast<MsdPart *>(base + L.nmax_off);
    SPD_CK(launch_nmax_partial(n, plane->dtype, st));
    SPD_CK(launch_fold_parts(n.parts, plane->n_dm * L.ntpr, scratch, kMergeScratch, out, st));
    return SPD_OK;
}

spd_status spd_sd_nmax_merge_partials(const spd_msd_part *parts_dev, int32_t n_shards,
                                      int32_t nmax_sigma, spd_msd_stats *out_dev, void *stream) {
    if (!parts_dev || !out_dev || n_shards < 1 || nmax_sigma < 2 || nmax_sigma > SPD_MAX_WIDTH)
        return SPD_ERR_INVALID_ARG;
    SPD_CK(launch_merge_shards(reinterpret_cast<const MsdPart *>(parts_dev), n_shards, 1,
                               nmax_sigma, out_dev, static_cast<cudaStream_t>(stream)));
    return SPD_OK;
}

size_t spd_boxcar_snr_workspace_bytes(const spd_plane *plane, int32_t scope,
                                      const int32_t *widths, int32_t n_widths) {
    if (check_plane(plane) != SPD_OK || !scope_ok(scope)) return 0;
    RangeProg prog;
    if (compile_program(widths, n_widths, prog) != SPD_OK) return 0;
    return det_layout(entries_of(plane, scope), prog.n_eval).total;
}

spd_status spd_boxcar_snr(const spd_plane *plane, const spd_msd_stats *msd_dev, int32_t scope,
                          const int32_t *widths, int32_t n_widths, int32_t sigma_mode,
                          float *snr_out, uint16_t *width_out, int64_t out_stride,
                          void *workspace, size_t workspace_bytes, void *stream) {
    SPD_TRY(check_plane(plane));
    if (!scope_ok(scope)) return SPD_ERR_INVALID_ARG;
    if (sigma_mode < SPD_SIGMA_SQRTN || sigma_mode > SPD_SIGMA_LINEAR_EXCESS)
        return SPD_ERR_INVALID_ARG;
    static thread_local RangeProg prog;
    SPD_TRY(compile_program(widths, n_widths, prog));
    if (plane_empty(plane)) return SPD_OK;
    if (!msd_dev || !snr_out || !width_out || out_stride < plane->n_samp)
        return SPD_ERR_INVALID_ARG;
    const size_t need = det_layout(entries_of(plane, scope), prog.n_eval).total;
    SPD_TRY(check_ws(workspace, workspace_bytes, need));
    return run_detect(plane, prog, msd_dev, scope, sigma_mode, 0.f, nullptr, 0, nullptr,
                      snr_out, width_out, out_stride, workspace,
                      static_cast<cudaStream_t>(stream));
}

spd_status spd_threshold_plane(float *snr, uint16_t *width, int64_t n_dm, int64_t n_samp,
                               int64_t stride, float threshold, void *stream) {
    if (n_dm < 0 || n_samp < 0 || n_dm > INT32_MAX || n_samp > INT32_MAX) return SPD_ERR_INVALID_ARG;
    if (n_dm == 0 || n_samp == 0) return SPD_OK;
    if (!snr || stride < n_samp || !isfinite(threshold)) return SPD_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(snr) % 4 || reinterpret_cast<uintptr_t>(width) % 2)
        return SPD_ERR_INVALID_ARG;
    SPD_CK(launch_threshold_plane(snr, width, n_dm, n_samp, stride, threshold,
                                  static_cast<cudaStream_t>(stream)));
    return SPD_OK;
}

spd_status spd_threshold_candidates(const float *snr, const uint16_t *width, int64_t n_dm,
                                    int64_t n_samp, int64_t stride, float threshold,
                                    spd_candidate *out, int64_t capacity,
                                    spd_result *result_dev, void *stream) {
    if (n_dm < 0 || n_samp < 0 || n_dm > INT32_MAX || n_samp > INT32_MAX)
        return SPD_ERR_INVALID_ARG;
    if (!result_dev || capacity < 0 || (capacity > 0 && !out) || !isfinite(threshold))
        return SPD_ERR_INVALID_ARG;
    if (out && reinterpret_cast<uintptr_t>(out) % 16) return SPD_ERR_INVALID_ARG;
    const bool empty = n_dm == 0 || n_samp == 0;
    if (!empty && (!snr || !width || stride < n_samp)) return SPD_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    SPD_CK(cudaMemsetAsync(result_dev, 0, sizeof(spd_result), st));
    if (empty) return SPD_OK;
    SPD_CK(launch_threshold(snr, width, n_dm, n_samp, stride, threshold, out, capacity,
                            result_dev, st));
    return SPD_OK;
}

spd_status spd_cluster_rows(const float *snr, const uint16_t *width, int64_t n_dm,
                            int64_t n_samp, int64_t stride, float threshold, int32_t max_gap,
                            spd_cluster *out, int64_t capacity, spd_result *result_dev,
                            void *stream) {
    if (n_dm < 0 || n_samp < 0 || n_dm > INT32_MAX || n_samp > INT32_MAX)
        return SPD_ERR_INVALID_ARG;
    if (!result_dev || capacity < 0 || (capacity > 0 && !out) || !isfinite(threshold) ||
        max_gap < 1)
        return SPD_ERR_INVALID_ARG;
    if (out && reinterpret_cast<uintptr_t>(out) % 16) return SPD_ERR_INVALID_ARG;
    const bool empty = n_dm == 0 || n_samp == 0;
    if (!empty && (!snr || !width || stride < n_samp)) return SPD_ERR_INVALID_ARG;
    if (!empty && (reinterpret_cast<uintptr_t>(snr) % 4 || reinterpret_cast<uintptr_t>(width) % 2))
        return SPD_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    SPD_CK(cudaMemsetAsync(result_dev, 0, sizeof(spd_result), st));
    if (empty) return SPD_OK;
    SPD_CK(launch_cluster(snr, width, n_dm, n_samp, stride, threshold, max_gap, out, capacity,
                          result_dev, st));
    return SPD_OK;
}

size_t spd_detect_workspace_bytes(const spd_plane *plane, const spd_search_params *params) {
    if (check_plane(plane) != SPD_OK || check_params(params) != SPD_OK) return 0;
    RangeProg prog;
    if (compile_program(params->widths, params->n_widths, prog) != SPD_OK) return 0;
    return det_layout(entries_of(plane, params->msd_scope), prog.n_eval).total;
}

spd_status spd_detect(const spd_plane *plane, const spd_search_params *params,
                      const spd_msd_stats *msd_dev, spd_candidate *out, int64_t capacity,
                      spd_result *result_dev, void *workspace, size_t workspace_bytes,
                      void *stream) {
    SPD_TRY(check_plane(plane));
    SPD_TRY(check_params(params));
    static thread_local RangeProg prog;
    SPD_TRY(compile_program(params->widths, params->n_widths, prog, 1, true));
    if (!result_dev || capacity < 0 || (capacity > 0 && !out)) return SPD_ERR_INVALID_ARG;
    if (out && reinterpret_cast<uintptr_t>(out) % 16) return SPD_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (plane_empty(plane)) {
        SPD_CK(cudaMemsetAsync(result_dev, 0, sizeof(spd_result), st));
        return SPD_OK;
    }
    if (!msd_dev) return SPD_ERR_INVALID_ARG;
    const size_t need = det_layout(entries_of(plane, params->msd_scope), prog.n_eval).total;
    SPD_TRY(check_ws(workspace, workspace_bytes, need));
    SPD_CK(cudaMemsetAsync(result_dev, 0, sizeof(spd_result), st));
    return run_detect(plane, prog, msd_dev, params->msd_scope, params->sigma_mode,
                      params->threshold, out, capacity, result_dev, nullptr, nullptr, 0,
                      workspace, st);
}

size_t spd_search_workspace_bytes(const spd_plane *plane, const spd_search_params *params) {
    if (check_plane(plane) != SPD_OK || check_params(params) != SPD_OK) return 0;
    RangeProg prog;
    if (compile_program(params->widths, params->n_widths, prog) != SPD_OK) return 0;
    const int64_t entries = entries_of(plane, params->msd_scope);
    return msd_layout(plane, nmax_of(params)).total +
           align_up((size_t)entries * sizeof(spd_msd_stats)) + det_layout(entries, prog.n_eval).total;
}

spd_status spd_search(const spd_plane *plane, const spd_search_params *params,
                      spd_candidate *out, int64_t capacity, spd_result *result_dev,
                      spd_msd_stats *msd_out_dev, void *workspace, size_t workspace_bytes,
                      void *stream) {
    SPD_TRY(check_plane(plane));
    SPD_TRY(check_params(params));
    static thread_local RangeProg prog;
    SPD_TRY(compile_program(params->widths, params->n_widths, prog, 1, true));
    if (!result_dev || capacity < 0 || (capacity > 0 && !out)) return SPD_ERR_INVALID_ARG;
    if (out && reinterpret_cast<uintptr_t>(out) % 16) return SPD_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (plane_empty(plane)) {
        SPD_CK(cudaMemsetAsync(result_dev, 0, sizeof(spd_result), st));
        return SPD_OK;
    }
    const int64_t entries = entries_of(plane, params->msd_scope);
    const MsdLayout ML = msd_layout(plane, nmax_of(params));
    const size_t msd_bytes = align_up((size_t)entries * sizeof(spd_msd_stats));
    const size_t need = ML.total + msd_bytes + det_layout(entries, prog.n_eval).total;
    SPD_TRY(check_ws(workspace, workspace_bytes, need));
    char *base = static_cast<char *>(workspace);
    spd_msd_stats *msd = msd_out_dev ? msd_out_dev : reinterpret_cast<spd_msd_stats *>(base + ML.total);
    SPD_TRY(spd_msd(plane, params->msd_scope, nmax_of(params), msd, base, ML.total, stream));
    SPD_CK(cudaMemsetAsync(result_dev, 0, sizeof(spd_result), st));
    return run_detect(plane, prog, msd, params->msd_scope, params->sigma_mode,
                      params->threshold, out, capacity, result_dev, nullptr, nullptr, 0,
                      base + ML.total + msd_bytes, st);
}

}  // extern "C"

namespace {

struct BatchLayout {
    size_t msd_off[kMaxRanges], stats_off[kMaxRanges], det_off[kMaxRanges], total;
    size_t msd_bytes[kMaxRanges];
};

spd_status batch_plan(const spd_range *ranges, int n, const spd_tuning *tuning,
                      RangeProg *progs, BatchLayout &L) {
    if (!ranges || n < 1 || n > kMaxRanges) return SPD_ERR_INVALID_ARG;
    const int scale = tuning && tuning->group_scale > 0 ? tuning->group_scale : 1;
    if (tuning && (tuning->ctas_per_sm < 0 || tuning->group_scale < 0)) return SPD_ERR_INVALID_ARG;
    if (tuning && tuning->tile_threads != 0 && tuning->tile_threads != 128 &&
        tuning->tile_threads != 256)
        return SPD_ERR_INVALID_ARG;
    size_t off = 0;
    for (int i = 0; i < n; ++i) {
        const spd_range &r = ranges[i];
        SPD_TRY(check_plane(&r.plane));
        SPD_TRY(check_params(&r.params));
        if (r.dm_offset < 0 || r.decimation < 0) return SPD_ERR_INVALID_ARG;
        SPD_TRY(compile_program(r.params.widths, r.params.n_widths, progs[i], scale, true));
        const int64_t entries = entries_of(&r.plane, r.params.msd_scope);
        L.msd_off[i] = off;
        L.msd_bytes[i] = msd_layout(&r.plane, nmax_of(&r.params)).total;
        off += align_up(L.msd_bytes[i]);
        L.stats_off[i] = off;
        off += align_up((size_t)entries * sizeof(spd_msd_stats));
        L.det_off[i] = off;
        off += align_up(det_layout(entries, progs[i].n_eval).total);
    }
    L.total = off;
    return SPD_OK;
}

spd_status batched_impl(const spd_range *ranges, int32_t n_ranges, const spd_tuning *tuning,
                        const int *shifts, spd_candidate *out, int64_t capacity,
                        spd_result *result_dev, spd_msd_stats *msd_out_dev, void *workspace,
                        size_t workspace_bytes, void *stream);

}  // namespace

extern "C" {

size_t spd_search_batched_workspace_bytes(const spd_range *ranges, int32_t n_ranges,
                                          const spd_tuning *tuning) {
    RangeProg progs[kMaxRanges];
    BatchLayout L;
    if (batch_plan(ranges, n_ranges, tuning, progs, L) != SPD_OK) return 0;
    return L.total;
}

spd_status spd_search_batched(const spd_range *ranges, int32_t n_ranges,
                              const spd_tuning *tuning, spd_candidate *out, int64_t capacity,
                              spd_result *result_dev, spd_msd_stats *msd_out_dev,
                              void *workspace, size_t workspace_bytes, void *stream) {
    return batched_impl(ranges, n_ranges, tuning, nullptr, out, capacity, result_dev,
                        msd_out_dev, workspace, workspace_bytes, stream);
}

}  // extern "C"

namespace {

// The batched search; shifts (NULL = none): per range, records carry
// start << shift and width << shift.
spd_status batched_impl(const spd_range *ranges, int32_t n_ranges, const spd_tuning *tuning,
                        const int *shifts, spd_candidate *out, int64_t capacity,
                        spd_result *result_dev, spd_msd_stats *msd_out_dev, void *workspace,
                        size_t workspace_bytes, void *stream) {
    static thread_local RangeProg progs[kMaxRanges];
    BatchLayout L;
    SPD_TRY(batch_plan(ranges, n_ranges, tuning, progs, L));
    if (!result_dev || capacity < 0 || (capacity > 0 && !out)) return SPD_ERR_INVALID_ARG;
    if (out && reinterpret_cast<uintptr_t>(out) % 16) return SPD_ERR_INVALID_ARG;
    SPD_TRY(check_ws(workspace, workspace_bytes, L.total));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char *base = static_cast<char *>(workspace);
    SPD_CK(cudaMemsetAsync(result_dev, 0, sizeof(spd_result), st));

    // (a) per range, and the constants of (c)
    RangeDesc rds[kMaxRanges];
    int live[kMaxRanges], n_live = 0;
    int64_t msd_pos = 0;
    for (int i = 0; i < n_ranges; ++i) {
        const spd_range &r = ranges[i];
        const int64_t entries = entries_of(&r.plane, r.params.msd_scope);
        spd_msd_stats *msd = msd_out_dev ? msd_out_dev + msd_pos
                                         : reinterpret_cast<spd_msd_stats *>(base + L.stats_off[i]);
        msd_pos += entries;
        if (plane_empty(&r.plane)) continue;
        SPD_TRY(spd_msd(&r.plane, r.params.msd_scope, nmax_of(&r.params), msd,
                        base + L.msd_off[i], L.msd_bytes[i], stream));
        // a decimated level evaluates only its listed widths
        const int skip_w1 = shifts && shifts[i] > 0 && r.params.widths[0] != 1;
        SPD_TRY(range_consts(&r.plane, progs[i], msd, r.params.msd_scope, r.params.sigma_mode,
                             result_dev, base + L.det_off[i], st, rds[i], skip_w1));
        rds[i].threshold = r.params.threshold;
        rds[i].dm_offset = r.dm_offset;
        rds[i].sample_shift = shifts ? shifts[i] : 0;
        live[n_live++] = i;
    }
    // (b, c, d): one persistent launch per class of ranges with equal G,
    // storage type and bulk-copy eligibility
    bool done[kMaxRanges] = {false};
    for (int a = 0; a < n_live; ++a) {
        const int i = live[a];
        if (done[i]) continue;
        RangeDesc grp[kMaxRanges];
        int m = 0;
        for (int b = a; b < n_live; ++b) {
            const int j = live[b];
            if (done[j] || rds[j].prog.G != rds[i].prog.G || rds[j].vec_ok != rds[i].vec_ok ||
                ranges[j].plane.dtype != ranges[i].plane.dtype)
                continue;
            grp[m++] = rds[j];
            done[j] = true;
        }
        SPD_TRY(run_launch(grp, m, ranges[i].plane.dtype, out, capacity, result_dev, nullptr,
                           nullptr, 0, tuning ? tuning->ctas_per_sm : 0, st,
                           tuning ? tuning->tile_threads : 0));
    }
    return SPD_OK;
}

// Decimated search: level planes (FP32, rows 16-byte aligned), then the
// batched workspace of the levels' ranges.
constexpr int kMaxDecLevel = 12;
struct DecLayout {
    int lmax;
    int64_t n[kMaxDecLevel + 1], stride[kMaxDecLevel + 1];
    size_t plane_off[kMaxDecLevel + 1];
    size_t batch_off, batch_bytes, total;
};

spd_status dec_plan(const spd_plane *plane, const spd_level *levels, int32_t n_levels,
                    float threshold, spd_range *ranges, int *shifts, DecLayout &D,
                    char *ws_base) {
    SPD_TRY(check_plane(plane));
    if (!levels || n_levels < 1 || n_levels > SPD_MAX_LEVELS || !isfinite(threshold))
        return SPD_ERR_INVALID_ARG;
    int prev_level = -1, prev_wmax = 0;
    for (int k = 0; k < n_levels; ++k) {
        const spd_level &lv = levels[k];
        if (lv.level <= prev_level || lv.level < 0 || lv.level > kMaxDecLevel) return SPD_ERR_INVALID_ARG;
        if (!lv.widths || lv.n_widths < 1) return SPD_ERR_INVALID_ARG;
        // native widths of the levels strictly ascending: a record's width
        // tells its level
        if (((int64_t)lv.widths[0] << lv.level) <= prev_wmax && k > 0) return SPD_ERR_INVALID_ARG;
        prev_level = lv.level;
        prev_wmax = (int)((int64_t)lv.widths[lv.n_widths - 1] << lv.level);
    }
    D.lmax = levels[n_levels - 1].level;
    size_t off = 0;
    D.n[0] = plane->n_samp;
    D.stride[0] = plane->row_stride;
    for (int l = 1; l <= D.lmax; ++l) {
        D.n[l] = plane->n_samp >> l;
        D.stride[l] = (D.n[l] + 7) / 8 * 8;
        D.plane_off[l] = off;
        off += align_up((size_t)plane->n_dm * D.stride[l] * sizeof(float));
    }
    for (int k = 0; k < n_levels; ++k) {
        const int l = levels[k].level;
        spd_range &r = ranges[k];
        memset(&r, 0, sizeof(r));
        if (l == 0) {
            r.plane = *plane;
        } else {
            r.plane.data = ws_base ? ws_base + D.plane_off[l] : reinterpret_cast<void *>(256);
            r.plane.dtype = SPD_F32;
            r.plane.n_dm = plane->n_dm;
            r.plane.n_samp = D.n[l];
            r.plane.row_stride = D.stride[l];
        }
        r.params.widths = levels[k].widths;
        r.params.n_widths = levels[k].n_widths;
        r.params.threshold = threshold;
        r.params.sigma_mode = SPD_SIGMA_SQRTN;
        r.params.msd_scope = SPD_MSD_GLOBAL;
        r.dm_offset = 0;
        r.decimation = 1 << l;
        shifts[k] = l;
    }
    RangeProg progs[kMaxRanges];
    BatchLayout B;
    SPD_TRY(batch_plan(ranges, n_levels, nullptr, progs, B));
    D.batch_off = off;
    D.batch_bytes = B.total;
    D.total = off + align_up(B.total);
    return SPD_OK;
}

}  // namespace

extern "C" {

size_t spd_search_decimated_workspace_bytes(const spd_plane *plane, const spd_level *levels,
                                            int32_t n_levels) {
    spd_range ranges[SPD_MAX_LEVELS];
    int shifts[SPD_MAX_LEVELS];
    DecLayout D;
    if (dec_plan(plane, levels, n_levels, 1.f, ranges, shifts, D, nullptr) != SPD_OK) return 0;
    return D.total;
}

spd_status spd_search_decimated(const spd_plane *plane, const spd_level *levels, int32_t n_levels,
                                float threshold, spd_candidate *out, int64_t capacity,
                                spd_result *result_dev, spd_msd_stats *msd_out_dev,
                                void *workspace, size_t workspace_bytes, void *stream) {
    spd_range ranges[SPD_MAX_LEVELS];
    int shifts[SPD_MAX_LEVELS];
    DecLayout D;
    char *base = static_cast<char *>(workspace);
    SPD_TRY(dec_plan(plane, levels, n_levels, threshold, ranges, shifts, D, base));
    SPD_TRY(check_ws(workspace, workspace_bytes, D.total));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // level l from level l - 1 (the input plane for l = 1)
    for (int l = 1; l <= D.lmax; ++l) {
        spd_plane src;
        if (l == 1) {
            src = *plane;
        } else {
            memset(&src, 0, sizeof(src));
            src.data = base + D.plane_off[l - 1];
            src.dtype = SPD_F32;
            src.n_dm = plane->n_dm;
            src.n_samp = D.n[l - 1];
            src.row_stride = D.stride[l - 1];
        }
        if (!plane_empty(&src))
            SPD_CK(launch_decimate2(src, reinterpret_cast<float *>(base + D.plane_off[l]), D.n[l],
                                    D.stride[l], st));
    }
    return batched_impl(ranges, n_levels, nullptr, shifts, out, capacity, result_dev, msd_out_dev,
                        base + D.batch_off, D.batch_bytes, stream);
}

}  // extern "C"

namespace {

// Stream state: [entries] MsdPart running MSD, the halo [n_dm][halo_cap], and
// the beam's per-row scale and offset (copied from its first push).
struct StreamLayout {
    int64_t entries;
    int halo_cap;
    size_t msd_off, halo_off, scale_off, offset_off, total;
};

spd_status stream_layout(int64_t n_dm, int32_t dtype, const spd_search_params *params,
                         RangeProg &prog, StreamLayout &L) {
    if (n_dm < 1 || n_dm > INT32_MAX || dtype < SPD_F32 || dtype > SPD_BF16)
        return SPD_ERR_INVALID_ARG;
    SPD_TRY(check_params(params));
    if (params->sigma_mode != SPD_SIGMA_SQRTN) return SPD_ERR_UNSUPPORTED;
    SPD_TRY(compile_program(params->widths, params->n_widths, prog, 1, true));
    L.entries = params->msd_scope == SPD_MSD_PER_ROW ? n_dm : 1;
    L.halo_cap = ((prog.wmax - 1) + 7) / 8 * 8;
    L.msd_off = 0;
    L.halo_off = align_up((size_t)L.entries * sizeof(MsdPart));
    L.scale_off = L.halo_off + align_up((size_t)n_dm * L.halo_cap * elem_bytes(dtype));
    L.offset_off = L.scale_off + align_up((size_t)n_dm * sizeof(float));
    L.total = L.offset_off + align_up((size_t)n_dm * sizeof(float));
    return SPD_OK;
}

// Push workspace: combined [n_dm][cstride] buffer, chunk MSD workspace,
// msd stats, detect constants.
struct PushLayout {
    int64_t cstride;
    size_t comb_off, msd_off, msd_bytes, stats_off, det_off, total;
};

PushLayout push_layout(int64_t n_dm, int64_t max_chunk, int32_t dtype, const StreamLayout &S,
                       const RangeProg &prog) {
    PushLayout L;
    const size_t eb = elem_bytes(dtype);
    L.cstride = (S.halo_cap + max_chunk + 7) / 8 * 8;
    L.comb_off = 0;
    L.msd_off = align_up((size_t)n_dm * L.cstride * eb);
    spd_plane probe;
    memset(&probe, 0, sizeof(probe));
    probe.n_dm = n_dm;
    probe.n_samp = max_chunk > 0 ? max_chunk : 1;
    L.msd_bytes = msd_layout(&probe).total;
    L.stats_off = L.msd_off + align_up(L.msd_bytes);
    L.det_off = L.stats_off + align_up((size_t)S.entries * sizeof(spd_msd_stats));
    L.total = L.det_off + align_up(det_layout(S.entries, prog.n_eval).total);
    return L;
}

spd_status check_info(const spd_stream_info *info, const StreamLayout &S, int32_t dtype,
                      const spd_search_params *params) {
    if (!info || info->dtype != dtype || info->msd_scope != params->msd_scope) return SPD_ERR_INVALID_ARG;
    if (info->halo_cap != S.halo_cap || info->halo < 0 || info->halo > S.halo_cap)
        return SPD_ERR_INVALID_ARG;
    return SPD_OK;
}

// Search the combined buffer [halo | chunk] (n = halo + chunk samples per row)
// with the running MSD in `stats`; emit starts below n_emit.
spd_status stream_search(const spd_stream_info *info, const RangeProg &prog,
                         const spd_search_params *params, const void *comb, int64_t cstride,
                         int64_t n, int64_t n_emit, const float *scale, const float *offset,
                         const spd_msd_stats *stats, spd_candidate *out, int64_t cap,
                         spd_result *result, void *det_ws, cudaStream_t st) {
    spd_plane cp;
    memset(&cp, 0, sizeof(cp));
    cp.data = comb;
    cp.dtype = info->dtype;
    cp.n_dm = info->n_dm;
    cp.n_samp = n;
    cp.row_stride = cstride;
    cp.row_scale = scale;
    cp.row_offset = offset;
    RangeDesc rd;
    SPD_TRY(range_consts(&cp, prog, stats, params->msd_scope, params->sigma_mode, result, det_ws,
                         st, rd));
    rd.threshold = params->threshold;
    rd.n_emit = n_emit;
    rd.sample_base = info->seen - info->halo;
    return run_launch(&rd, 1, info->dtype, out, cap, result, nullptr, nullptr, 0, 0, st);
}

}  // namespace

extern "C" {

size_t spd_stream_state_bytes(int64_t n_dm, int32_t dtype, const spd_search_params *params) {
    RangeProg prog;
    StreamLayout S;
    if (stream_layout(n_dm, dtype, params, prog, S) != SPD_OK) return 0;
    return S.total;
}

size_t spd_stream_workspace_bytes(int64_t n_dm, int64_t max_chunk, int32_t dtype,
                                  const spd_search_params *params) {
    RangeProg prog;
    StreamLayout S;
    if (max_chunk < 0 || max_chunk > INT32_MAX) return 0;
    if (stream_layout(n_dm, dtype, params, prog, S) != SPD_OK) return 0;
    return push_layout(n_dm, max_chunk, dtype, S, prog).total;
}

spd_status spd_stream_reset(spd_stream_info *info, void *state_dev, int64_t n_dm, int32_t dtype,
                            const spd_search_params *params, void *stream) {
    RangeProg prog;
    StreamLayout S;
    SPD_TRY(stream_layout(n_dm, dtype, params, prog, S));
    if (!info || !state_dev || reinterpret_cast<uintptr_t>(state_dev) % kAlign)
        return SPD_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    SPD_CK(launch_zero_parts(reinterpret_cast<MsdPart *>(static_cast<char *>(state_dev) + S.msd_off),
                             S.entries, st));
    memset(info, 0, sizeof(*info));
    info->n_dm = n_dm;
    info->dtype = dtype;
    info->msd_scope = params->msd_scope;
    info->wmax = prog.wmax;
    info->halo_cap = S.halo_cap;
    return SPD_OK;
}

spd_status spd_stream_push(spd_stream_info *info, void *state_dev, const spd_plane *chunk,
                           const spd_search_params *params, spd_candidate *out,
                           int64_t capacity, spd_result *result_dev, spd_msd_stats *msd_out_dev,
                           void *workspace, size_t workspace_bytes, void *stream) {
    RangeProg prog;
    StreamLayout S;
    if (!info || !chunk) return SPD_ERR_INVALID_ARG;
    SPD_TRY(stream_layout(info->n_dm, info->dtype, params, prog, S));
    SPD_TRY(check_info(info, S, chunk->dtype, params));
    SPD_TRY(check_plane(chunk));
    if (chunk->n_dm != info->n_dm || !state_dev) return SPD_ERR_INVALID_ARG;
    // every chunk of a beam carries a per-row scale / offset, or none does
    if (info->seen > 0 && ((chunk->row_scale != nullptr) != (info->has_scale != 0) ||
                           (chunk->row_offset != nullptr) != (info->has_offset != 0)))
        return SPD_ERR_INVALID_ARG;
    if (!result_dev || capacity < 0 || (capacity > 0 && !out)) return SPD_ERR_INVALID_ARG;
    if (out && reinterpret_cast<uintptr_t>(out) % 16) return SPD_ERR_INVALID_ARG;
    const int64_t L = chunk->n_samp;
    const size_t eb = elem_bytes(info->dtype);
    const PushLayout P = push_layout(info->n_dm, L, info->dtype, S, prog);
    SPD_TRY(check_ws(workspace, workspace_bytes, P.total));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char *ws = static_cast<char *>(workspace);
    char *state = static_cast<char *>(state_dev);
    MsdPart *run = reinterpret_cast<MsdPart *>(state + S.msd_off);
    char *halo = state + S.halo_off;
    char *comb = ws + P.comb_off;
    const int64_t H = info->halo;
    SPD_CK(cudaMemsetAsync(result_dev, 0, sizeof(spd_result), st));
    if (L == 0) return SPD_OK;
    if (info->seen == 0) {
        // the flush has no chunk: keep the beam's scale / offset in the state
        const size_t rb = (size_t)info->n_dm * sizeof(float);
        if (chunk->row_scale)
            SPD_CK(cudaMemcpyAsync(state + S.scale_off, chunk->row_scale, rb,
                                   cudaMemcpyDeviceToDevice, st));
        if (chunk->row_offset)
            SPD_CK(cudaMemcpyAsync(state + S.offset_off, chunk->row_offset, rb,
                                   cudaMemcpyDeviceToDevice, st));
        info->has_scale = chunk->row_scale != nullptr;
        info->has_offset = chunk->row_offset != nullptr;
    }
    // [halo | chunk] into the combined buffer
    if (H > 0)
        SPD_CK(cudaMemcpy2DAsync(comb, P.cstride * eb, halo, S.halo_cap * eb, H * eb, info->n_dm,
                                 cudaMemcpyDeviceToDevice, st));
    const char *src = static_cast<const char *>(chunk->data);
    if (src == comb + H * eb && chunk->row_stride == P.cstride) {
        // written in place through spd_stream_chunk_view
    } else if (src < ws + workspace_bytes && src + (size_t)chunk->n_dm * chunk->row_stride * eb > ws) {
        return SPD_ERR_INVALID_ARG;  // inside the workspace but not at the view
    } else {
        // device or page-locked host memory (unified addressing decides)
        SPD_CK(cudaMemcpy2DAsync(comb + H * eb, P.cstride * eb, src, chunk->row_stride * eb,
                                 L * eb, info->n_dm, cudaMemcpyDefault, st));
    }
    // running MSD: the chunk's unit partials (read from its place in the
    // combined buffer) added to the state
    spd_plane in_place = *chunk;
    in_place.data = comb + H * eb;
    in_place.row_stride = P.cstride;
    const MsdLayout ML = msd_layout(&in_place);
    MsdArgs ma;
    ma.data = in_place.data;
    ma.n_dm = chunk->n_dm;
    ma.n_samp = L;
    ma.stride = P.cstride;
    ma.scale = chunk->row_scale;
    ma.offset = chunk->row_offset;
    ma.units_per_row = ML.upr;
    ma.vec_ok = plane_vec_ok(&in_place);
    MsdPart *parts = reinterpret_cast<MsdPart *>(ws + P.msd_off);
    ma.parts = parts;
    SPD_CK(launch_msd_partial(ma, chunk->dtype, st));
    spd_msd_stats *stats =
        msd_out_dev ? msd_out_dev : reinterpret_cast<spd_msd_stats *>(ws + P.stats_off);
    SPD_CK(launch_stream_msd(parts, info->n_dm, ML.upr, params->msd_scope == SPD_MSD_PER_ROW,
                             run, stats, st));
    // search every start with a full window; hold the last wmax - 1 back
    const int64_t n = H + L;
    const int64_t hold = n < (int64_t)(prog.wmax - 1) ? n : (int64_t)(prog.wmax - 1);
    const int64_t n_emit = n - hold;
    SPD_TRY(stream_search(info, prog, params, comb, P.cstride, n, n_emit, chunk->row_scale,
                          chunk->row_offset, stats, out, capacity, result_dev, ws + P.det_off, st));
    if (hold > 0)
        SPD_CK(cudaMemcpy2DAsync(halo, S.halo_cap * eb, comb + n_emit * eb, P.cstride * eb,
                                 hold * eb, info->n_dm, cudaMemcpyDeviceToDevice, st));
    info->seen += L;
    info->halo = hold;
    info->chunks += 1;
    return SPD_OK;
}

spd_status spd_stream_chunk_view(const spd_stream_info *info, const spd_search_params *params,
                                 int64_t n_samp, void *workspace, size_t workspace_bytes,
                                 void **data, int64_t *row_stride) {
    RangeProg prog;
    StreamLayout S;
    if (!info || !data || !row_stride || n_samp < 0 || n_samp > INT32_MAX)
        return SPD_ERR_INVALID_ARG;
    SPD_TRY(stream_layout(info->n_dm, info->dtype, params, prog, S));
    SPD_TRY(check_info(info, S, info->dtype, params));
    const PushLayout P = push_layout(info->n_dm, n_samp, info->dtype, S, prog);
    SPD_TRY(check_ws(workspace, workspace_bytes, P.total));
    *data = static_cast<char *>(workspace) + P.comb_off + info->halo * elem_bytes(info->dtype);
    *row_stride = P.cstride;
    return SPD_OK;
}

spd_status spd_stream_flush(spd_stream_info *info, void *state_dev,
                            const spd_search_params *params, spd_candidate *out,
                            int64_t capacity, spd_result *result_dev, void *workspace,
                            size_t workspace_bytes, void *stream) {
    RangeProg prog;
    StreamLayout S;
    if (!info) return SPD_ERR_INVALID_ARG;
    SPD_TRY(stream_layout(info->n_dm, info->dtype, params, prog, S));
    SPD_TRY(check_info(info, S, info->dtype, params));
    if (!state_dev || !result_dev || capacity < 0 || (capacity > 0 && !out))
        return SPD_ERR_INVALID_ARG;
    const PushLayout P = push_layout(info->n_dm, 0, info->dtype, S, prog);
    SPD_TRY(check_ws(workspace, workspace_bytes, P.total));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    SPD_CK(cudaMemsetAsync(result_dev, 0, sizeof(spd_result), st));
    const int64_t H = info->halo;
    if (H == 0) return SPD_OK;
    const size_t eb = elem_bytes(info->dtype);
    char *ws = static_cast<char *>(workspace);
    char *state = static_cast<char *>(state_dev);
    SPD_CK(cudaMemcpy2DAsync(ws + P.comb_off, P.cstride * eb, state + S.halo_off,
                             S.halo_cap * eb, H * eb, info->n_dm, cudaMemcpyDeviceToDevice, st));
    spd_msd_stats *stats = reinterpret_cast<spd_msd_stats *>(ws + P.stats_off);
    SPD_CK(launch_stream_msd(reinterpret_cast<MsdPart *>(ws + P.msd_off), info->n_dm, 0,
                             info->msd_scope == SPD_MSD_PER_ROW,
                             reinterpret_cast<MsdPart *>(state + S.msd_off), stats, st));
    const float *scale = info->has_scale ? reinterpret_cast<const float *>(state + S.scale_off)
                                         : nullptr;
    const float *offset = info->has_offset
                              ? reinterpret_cast<const float *>(state + S.offset_off)
                              : nullptr;
    SPD_TRY(stream_search(info, prog, params, ws + P.comb_off, P.cstride, H, H, scale, offset,
                          stats, out, capacity, result_dev, ws + P.det_off, st));
    info->halo = 0;
    return SPD_OK;
}

spd_status spd_debug_set_copy_wait(uint64_t limit_ns, uint32_t extra_bytes) {
    if (limit_ns < 1000000ull || limit_ns > 10000000000ull || extra_bytes > 4096u ||
        (extra_bytes & 15u))
        return SPD_ERR_INVALID_ARG;
    g_wait_ns = limit_ns;
    g_extra_tx = extra_bytes;
    return SPD_OK;
}

spd_status spd_boxcar_sums(const spd_plane *plane, int32_t w, float *out, int64_t out_stride,
                           void *stream) {
    SPD_TRY(check_plane(plane));
    if (w < 1 || w > SPD_MAX_WIDTH) return SPD_ERR_INVALID_ARG;
    if (plane_empty(plane)) return SPD_OK;
    if (!out || out_stride < plane->n_samp || plane->n_dm > 65535) return SPD_ERR_INVALID_ARG;
    SPD_CK(launch_boxcar_sums(*plane, w, out, out_stride, static_cast<cudaStream_t>(stream)));
    return SPD_OK;
}

}  // extern "C"

// ------------------------------------------------- the host-buffer search

namespace {

// Workspace of spd_search_host: the plane (rows padded to 16 bytes), its
// scale and offset, spd_search's own workspace (MSD part, then the detect
// constants), the result word, the MSD and the records.
struct HostLayout {
    int64_t dstride;
    size_t plane_off, scale_off, offset_off, search_off, msd_ws_bytes, result_off, msd_off,
        out_off, total;
};

spd_status host_layout(const spd_plane *hp, const spd_search_params *q, int64_t capacity,
                       HostLayout &H) {
    const size_t eb = elem_bytes(hp->dtype);
    const int64_t per = (int64_t)(16 / eb);
    H.dstride = (hp->n_samp + per - 1) / per * per;
    spd_plane dp = *hp;
    dp.data = reinterpret_cast<void *>(256);   // any aligned address: sizes only
    dp.row_stride = H.dstride;
    const size_t search_bytes = spd_search_workspace_bytes(&dp, q);
    if (!search_bytes) return SPD_ERR_INVALID_ARG;
    H.msd_ws_bytes = msd_layout(&dp, nmax_of(q)).total;
    const int64_t entries = entries_of(hp, q->msd_scope);
    H.plane_off = 0;
    H.scale_off = align_up((size_t)hp->n_dm * H.dstride * eb);
    H.offset_off = H.scale_off + align_up((size_t)hp->n_dm * sizeof(float));
    H.search_off = H.offset_off + align_up((size_t)hp->n_dm * sizeof(float));
    H.result_off = H.search_off + align_up(search_bytes);
    H.msd_off = H.result_off + kAlign;
    H.out_off = H.msd_off + align_up((size_t)entries * sizeof(spd_msd_stats));
    H.total = H.out_off + align_up((size_t)capacity * sizeof(spd_candidate));
    return SPD_OK;
}

constexpr int kHostBlocks = 16;   // most row blocks of one call

// Per host thread: the copy-out stream and the events of the row blocks (on
// the device current when they were made), and page-locked result words.
// Released when the thread exits (errors ignored: at process exit the
// runtime may already be gone), and the stream and events when the thread
// moves to another device.
struct HostAux {
    int dev = -1;
    cudaStream_t cs = nullptr;
    cudaEvent_t ev[kHostBlocks] = {};
    spd_result *pin = nullptr;

    void release_device_objects() {
        for (int b = 0; b < kHostBlocks; ++b) {
            if (ev[b]) (void)cudaEventDestroy(ev[b]);
            ev[b] = nullptr;
        }
        if (cs) (void)cudaStreamDestroy(cs);
        cs = nullptr;
        dev = -1;
    }
    ~HostAux() {
        release_device_objects();
        if (pin) (void)cudaFreeHost(pin);
    }
};
thread_local HostAux g_aux;

cudaError_t host_aux(HostAux **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    HostAux &a = g_aux;
    if (!a.pin) {
        e = cudaHostAlloc(reinterpret_cast<void **>(&a.pin), sizeof(spd_result) * kHostBlocks,
                          cudaHostAllocPortable);
        if (e != cudaSuccess) return e;
    }
    if (a.dev != dev) {
        a.release_device_objects();
        e = cudaStreamCreateWithFlags(&a.cs, cudaStreamNonBlocking);
        if (e != cudaSuccess) return e;
        for (int b = 0; b < kHostBlocks; ++b) {
            e = cudaEventCreateWithFlags(&a.ev[b], cudaEventDisableTiming);
            if (e != cudaSuccess) return e;
        }
        a.dev = dev;
    }
    *out = &a;
    return cudaSuccess;
}

}  // namespace

extern "C" {

size_t spd_search_host_workspace_bytes(const spd_plane *plane, const spd_search_params *params,
                                       int64_t capacity) {
    if (check_plane(plane) != SPD_OK || check_params(params) != SPD_OK || capacity < 0) return 0;
    HostLayout H;
    if (host_layout(plane, params, capacity, H) != SPD_OK) return 0;
    return H.total;
}

spd_status spd_search_host(const spd_plane *host_plane, const spd_search_params *params,
                           spd_candidate *host_out, int64_t capacity, spd_result *host_result,
                           spd_msd_stats *host_msd, void *workspace, size_t workspace_bytes,
                           void *stream) {
    SPD_TRY(check_plane(host_plane));
    SPD_TRY(check_params(params));
    if (!host_result || capacity < 0 || (capacity > 0 && !host_out)) return SPD_ERR_INVALID_ARG;
    static thread_local RangeProg prog;
    SPD_TRY(compile_program(params->widths, params->n_widths, prog, 1, true));
    HostLayout H;
    SPD_TRY(host_layout(host_plane, params, capacity, H));
    SPD_TRY(check_ws(workspace, workspace_bytes, H.total));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char *base = static_cast<char *>(workspace);
    spd_result *res = reinterpret_cast<spd_result *>(base + H.result_off);
    spd_msd_stats *msd = reinterpret_cast<spd_msd_stats *>(base + H.msd_off);
    spd_candidate *dev_out = reinterpret_cast<spd_candidate *>(base + H.out_off);
    const int64_t n_dm = host_plane->n_dm;
    const size_t eb = elem_bytes(host_plane->dtype);
    if (plane_empty(host_plane)) {
        memset(host_result, 0, sizeof(spd_result));
        return SPD_OK;
    }

    // the plane and its scale / offset into device memory
    void *dplane = base + H.plane_off;
    spd_plane dp = *host_plane;
    dp.data = dplane;
    dp.row_stride = H.dstride;
    SPD_CK(cudaMemcpy2DAsync(dplane, (size_t)H.dstride * eb, host_plane->data,
                             (size_t)host_plane->row_stride * eb, (size_t)host_plane->n_samp * eb,
                             (size_t)n_dm, cudaMemcpyHostToDevice, st));
    if (host_plane->row_scale) {
        float *sc = reinterpret_cast<float *>(base + H.scale_off);
        SPD_CK(cudaMemcpyAsync(sc, host_plane->row_scale, n_dm * sizeof(float),
                               cudaMemcpyHostToDevice, st));
        dp.row_scale = sc;
    }
    if (host_plane->row_offset) {
        float *of = reinterpret_cast<float *>(base + H.offset_off);
        SPD_CK(cudaMemcpyAsync(of, host_plane->row_offset, n_dm * sizeof(float),
                               cudaMemcpyHostToDevice, st));
        dp.row_offset = of;
    }

    // (a) the MSD of the whole plane, the result word zeroed, then the
    // constants of every row once
    char *sws = base + H.search_off;
    SPD_TRY(spd_msd(&dp, params->msd_scope, nmax_of(params), msd, sws, H.msd_ws_bytes, stream));
    SPD_CK(cudaMemsetAsync(res, 0, sizeof(spd_result), st));
    RangeDesc rd;
    SPD_TRY(range_consts(&dp, prog, msd, params->msd_scope, params->sigma_mode, res,
                         sws + H.msd_ws_bytes, st, rd));
    rd.threshold = params->threshold;

    // (b, c, d) by blocks of rows; block b's records go out while b + 1 runs
    HostAux *aux = nullptr;
    SPD_CK(host_aux(&aux));
    int nb = (int)(n_dm / 256);
    nb = nb < 1 ? 1 : (nb > kHostBlocks ? kHostBlocks : nb);
    for (int b = 0; b < nb; ++b) {
        const int64_t r0 = n_dm * b / nb, r1 = n_dm * (b + 1) / nb;
        RangeDesc rb = rd;
        rb.data = static_cast<const char *>(dp.data) + r0 * H.dstride * (int64_t)eb;
        rb.n_dm = r1 - r0;
        if (rb.scale) rb.scale += r0;
        if (rb.offset) rb.offset += r0;
        if (rd.per_row) {
            rb.inv_tab += r0 * prog.n_eval;
            rb.mu_tab += r0;
            rb.flags += r0;
        }
        rb.dm_offset = (int32_t)r0;
        SPD_TRY(run_launch(&rb, 1, dp.dtype, dev_out, capacity, res, nullptr, nullptr, 0, 0, st));
        SPD_CK(cudaMemcpyAsync(aux->pin + b, res, sizeof(spd_result), cudaMemcpyDeviceToHost, st));
        SPD_CK(cudaEventRecord(aux->ev[b], st));
    }
    uint64_t done = 0;
    for (int b = 0; b < nb; ++b) {
        SPD_CK(cudaEventSynchronize(aux->ev[b]));
        const uint64_t c = aux->pin[b].count < (uint64_t)capacity ? aux->pin[b].count
                                                                 : (uint64_t)capacity;
        if (c > done) {
            SPD_CK(cudaStreamWaitEvent(aux->cs, aux->ev[b], 0));
            SPD_CK(cudaMemcpyAsync(host_out + done, dev_out + done,
                                   (size_t)(c - done) * sizeof(spd_candidate),
                                   cudaMemcpyDeviceToHost, aux->cs));
            done = c;
        }
    }
    if (host_msd)
        SPD_CK(cudaMemcpyAsync(host_msd, msd,
                               (size_t)entries_of(&dp, params->msd_scope) * sizeof(spd_msd_stats),
                               cudaMemcpyDeviceToHost, aux->cs));
    SPD_CK(cudaStreamSynchronize(aux->cs));
    *host_result = aux->pin[nb - 1];
    return SPD_OK;
}

}  // extern "C"
