/*
 * spd.h -- C ABI of libspd, a GB300 (sm_103a) single-pulse search over
 * de-dispersed data laid out as DM trials x time samples, after Adamek &
 * Armour, "A Real-time Single Pulse Detection Algorithm for GPUs"
 * (arXiv:1611.09704).
 *
 * The search has four steps:
 *   (a) mean mu and standard deviation sigma of the data with Chan's streaming
 *       update (Eq. 1) and pairwise merge (Eq. 2), as a block-partial kernel
 *       followed by a merge kernel (Sec. 2.1);
 *   (b) boxcar filters of the listed widths at every sample (Sec. 2.3);
 *   (c) SNR = (B_w - w mu) / sigma_w with sigma_w from Eq. 4 or Eq. 5
 *       (Sec. 2.2), keeping per sample the highest SNR and its width
 *       (Algorithm 1, strict ">" so the smallest width wins ties);
 *   (d) candidates with SNR >= threshold, compacted into an unordered list of
 *       (DM, sample, SNR, width) records (Sec. 2.4).
 *
 * Conventions shared by every call:
 *   - Pointers named *_dev, and plane data, are device pointers; everything
 *     else (structs passed by pointer, width lists) lives on the host and is
 *     read before the call returns.  The caller owns all memory; the library
 *     never allocates device memory and keeps no pointer after a call returns.
 *   - Every call is asynchronous on `stream` (a cudaStream_t passed as void*;
 *     NULL means the legacy default stream).  Arguments are validated on the
 *     host before anything is launched; a failed validation launches nothing.
 *   - Results that depend on data (degenerate sigma, number of candidates)
 *     are written to device memory and become visible after the caller
 *     synchronises the stream.  Nothing is thrown across the ABI.
 *   - Sample windows are forward: B_w(i) = x[i] + ... + x[i+w-1].  Near the
 *     end of a row only widths w <= n_samp - i are evaluated; width 1 is always
 *     evaluated.  Candidates carry the start sample i.
 *   - Widths: strictly ascending, 1 <= w <= SPD_MAX_WIDTH, at most
 *     SPD_MAX_WIDTHS of them.
 */
#ifndef SPD_H
#define SPD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SPD_VERSION 100
#define SPD_MAX_WIDTH 4096
#define SPD_MAX_WIDTHS 4096

typedef enum {
    SPD_OK = 0,
    SPD_ERR_INVALID_ARG = 1,      /* bad pointer, size, width list or mode */
    SPD_ERR_CUDA = 2,             /* a CUDA call or launch failed; see spd_last_cuda_error */
    SPD_ERR_NO_MEMORY = 3,        /* the workspace passed is smaller than required */
    SPD_ERR_OVERFLOW = 4,         /* more candidates than capacity (reported by the host) */
    SPD_ERR_DEGENERATE_SIGMA = 5, /* sigma <= 0 or not finite: no SNR is defined */
    SPD_ERR_TIMEOUT = 6,          /* a bounded device-side wait gave up */
    SPD_ERR_UNSUPPORTED = 7       /* valid request this build cannot serve */
} spd_status;

typedef enum { SPD_F32 = 0, SPD_F16 = 1, SPD_BF16 = 2 } spd_dtype;

/* sigma_w after a w-sample boxcar (Sec. 2.2):
 *   SQRTN          Eq. 4: sqrt(w) sigma
 *   LINEAR         Eq. 5 as printed: sqrt(w) sigma + (w-1) sigma_Nmax/(Nmax-1)
 *   LINEAR_EXCESS  Eq. 5 read as the linear excess over Eq. 4, exact at w = 1
 *                  and w = Nmax: sqrt(w) sigma
 *                                + (w-1)(sigma_Nmax - sqrt(Nmax) sigma)/(Nmax-1)
 * sigma_Nmax is the measured standard deviation of the Nmax-sample boxcar
 * series over full windows (Sec. 2.2). */
typedef enum {
    SPD_SIGMA_SQRTN = 0,
    SPD_SIGMA_LINEAR = 1,
    SPD_SIGMA_LINEAR_EXCESS = 2
} spd_sigma_mode;

/* Which samples one (mu, sigma) describes: the whole plane of the call, as in
 * Sec. 2.1 ("for the dataset"), or each DM row on its own. */
typedef enum { SPD_MSD_GLOBAL = 0, SPD_MSD_PER_ROW = 1 } spd_msd_scope;

/* A DM x time plane in device memory, row-major: element (r, t) is at
 * data + (r * row_stride + t) * sizeof(element), 0 <= t < n_samp <= row_stride.
 * F16 / BF16 data may carry an FP32 per-row scale and offset (device arrays of
 * n_dm floats, either may be NULL); the value searched is
 * fmaf(scale[r], q, offset[r]) computed in FP32 (scale NULL: q itself). */
typedef struct {
    const void *data;
    int32_t dtype;            /* spd_dtype */
    int32_t reserved0;
    int64_t n_dm;
    int64_t n_samp;
    int64_t row_stride;       /* in elements */
    const float *row_scale;   /* device, n_dm entries, or NULL */
    const float *row_offset;  /* device, n_dm entries, or NULL */
} spd_plane;

/* Result of step (a) for one scope entry (40 bytes).  n: samples described;
 * sd_nmax: sigma_Nmax of Eq. 5 (0 when not measured); status: SPD_OK or
 * SPD_ERR_DEGENERATE_SIGMA. */
typedef struct {
    double mean;
    double sd;
    double sd_nmax;
    int64_t n;
    int32_t nmax;
    int32_t status;
} spd_msd_stats;

/* One candidate (16 bytes): DM row, start sample, highest SNR, its width. */
typedef struct {
    int32_t dm;
    int32_t sample;
    float snr;
    int32_t width;
} spd_candidate;

/* One cluster of a DM row's candidates (32 bytes), from spd_cluster_rows. */
typedef struct {
    int32_t dm;
    int32_t first;        /* sample of the cluster's first candidate */
    int32_t last;         /* sample of its last candidate */
    int32_t peak_sample;  /* sample of its highest SNR (the earliest among equals) */
    float peak_snr;
    int32_t peak_width;   /* the width at peak_sample */
    int32_t members;      /* candidates in the cluster */
    int32_t reserved0;
} spd_cluster;

/* Device-side summary written by the record-producing calls (16 bytes).
 * count: the exact number of records the call produced, even when it exceeds
 * the capacity (then only `capacity` records are written, which ones is
 * unspecified).  For the search and threshold calls (spd_search, spd_detect,
 * spd_search_batched, spd_search_decimated, spd_stream_push/flush,
 * spd_threshold_candidates) that is the number of candidates, samples with
 * SNR >= threshold; for spd_cluster_rows the number of clusters.
 * status: SPD_OK, SPD_ERR_DEGENERATE_SIGMA, or SPD_ERR_TIMEOUT (a tile's bulk
 * copy did not land within the kernel's wait bound, 2 s: the kernel stopped
 * instead of waiting on; see spd_debug_set_copy_wait).
 * reserved0: the candidate search's work counter while its kernels run (the
 * calls zero the whole word first); 0 again once they have finished, unless
 * one stopped on SPD_ERR_TIMEOUT. */
typedef struct {
    uint64_t count;
    int32_t status;
    int32_t reserved0;
} spd_result;

/* Parameters of the search (host struct; `widths` is a host array). */
typedef struct {
    const int32_t *widths;
    int32_t n_widths;
    float threshold;          /* f_T of Sec. 2.4, in SNR units */
    int32_t sigma_mode;       /* spd_sigma_mode */
    int32_t msd_scope;        /* spd_msd_scope */
    int32_t nmax_sigma;       /* Nmax of Eq. 5; 0 = last listed width */
    int32_t reserved0;
} spd_search_params;

/* ------------------------------------------------------------------------ */

int32_t spd_version(void);
const char *spd_status_string(int32_t status);
/* cudaError_t of the most recent SPD_ERR_CUDA on the calling thread (0 if none). */
int32_t spd_last_cuda_error(void);

/* Bytes of device workspace spd_msd needs (256-byte aligned base). */
size_t spd_msd_workspace_bytes(const spd_plane *plane, int32_t scope, int32_t nmax_sigma);

/* Step (a), Sec. 2.1, Eq. 1-2 (and the sigma_Nmax of Sec. 2.2 when
 * nmax_sigma >= 2).  A block-partial kernel gives (n, T, S) of equal-sized
 * pieces of each row (Eq. 1 per thread in FP32 with compensated sums, Eq. 2
 * across lanes, warps and the block); a merge kernel adds the pieces with
 * Eq. 2 in FP64 in a fixed order, so the result is deterministic.
 *   out_dev: device array of 1 (GLOBAL) or n_dm (PER_ROW) spd_msd_stats.
 *   nmax_sigma: 0 skips sigma_Nmax; >= 2 also measures the sd of the
 *     nmax-sample boxcar series over full windows (rows shorter than nmax
 *     contribute nothing).
 * Errors: SPD_ERR_INVALID_ARG (bad plane/scope/nmax), SPD_ERR_NO_MEMORY
 * (workspace too small), SPD_ERR_CUDA.  An empty plane (n_dm or n_samp 0)
 * yields n = 0 and status SPD_ERR_DEGENERATE_SIGMA; so does sigma <= 0. */
spd_status spd_msd(const spd_plane *plane, int32_t scope, int32_t nmax_sigma,
                   spd_msd_stats *out_dev, void *workspace, size_t workspace_bytes,
                   void *stream);

/* The same MSD as spd_msd, for callers that cannot give the library a
 * workspace.  The paper has no counterpart: this is a deployment aid.
 * Some callers must not allocate device memory once they run -- a real-time
 * backend that fixes its memory at start-up because a later cudaMalloc can
 * stall the device, or a plain C caller that holds only its plane and output
 * and has no allocator to size a workspace with.  They pass the plane and
 * out_dev (1 or n_dm spd_msd_stats, device) as for spd_msd, and the block
 * partials go to a static array of 1,320,960 bytes that the library declares
 * in device memory; every GPU that loads the library keeps it until the
 * process exits.  Limit: n_dm * ceil(n_samp / SPD_MSD_UNIT_SAMPLES) must not
 * exceed SPD_MSD_NOALLOC_MAX_UNITS (e.g. 4096 x 524288), else the call returns
 * SPD_ERR_NO_MEMORY and launches nothing.  Every call made outside stream
 * capture looks up the array's device address on the current device (a CUDA
 * runtime query), so a device reset, after which the array may sit elsewhere,
 * is handled; a call during stream capture uses the address found by the last
 * call outside capture on that device, so make one call outside capture
 * first (else SPD_ERR_CUDA).  All calls share the one array: calls whose
 * kernels overlap on the GPU (different streams, or different host threads)
 * race and give wrong results; calls ordered on one stream do not.  Nothing in
 * the array needs clearing between calls -- each call writes every entry it
 * reads.  Errors: as spd_msd. */
#define SPD_MSD_UNIT_SAMPLES 65536
#define SPD_MSD_NOALLOC_MAX_UNITS 32768
spd_status spd_msd_noalloc(const spd_plane *plane, int32_t scope, spd_msd_stats *out_dev,
                           void *stream);

/* ------------------------------------------------------ DM-row shards
 * A plane split by DM rows over several GPUs (one shard per rank) shares one
 * MSD of the whole plane (Sec. 2.1 defines it for the dataset).  Eq. 2 makes
 * the merge of partials order-free up to rounding, so each rank reduces its
 * shard to one partial, the ranks exchange partials (an all-gather of
 * sizeof(spd_msd_part) bytes per rank; the exchange is the caller's), and
 * every rank merges the gathered array in shard order, which gives every rank
 * the same bits.  Global scope only: per-row statistics need no exchange.
 * With one shard the result equals spd_msd's bit for bit. */
typedef struct {
    double n;      /* samples */
    double T;      /* sum */
    double S;      /* sum of squared deviations from T / n */
    double lo, hi; /* min and max value (exact constancy test) */
} spd_msd_part;

/* The shard's partial of the samples (Eq. 1 per thread, Eq. 2 up to one
 * record) into *part_dev (device, one record).  Workspace: as
 * spd_msd_workspace_bytes(plane, SPD_MSD_GLOBAL, 0).  Errors: as spd_msd. */
spd_status spd_msd_shard_partial(const spd_plane *plane, spd_msd_part *part_dev, void *workspace,
                                 size_t workspace_bytes, void *stream);
/* Eq. 2 over parts_dev[0 .. n_shards) in that order -> out_dev (one
 * spd_msd_stats: mean, sd, n, status as spd_msd; sd_nmax 0). */
spd_status spd_msd_merge_partials(const spd_msd_part *parts_dev, int32_t n_shards,
                                  spd_msd_stats *out_dev, void *stream);
/* Eq. 5's sigma_Nmax needs a second exchange: the partial of the shard's
 * B_Nmax series (full windows within each row), centred on the merged mean
 * in msd_dev.  Workspace: as spd_msd_workspace_bytes(plane, SPD_MSD_GLOBAL,
 * nmax_sigma). */
spd_status spd_sd_nmax_shard_partial(const spd_plane *plane, int32_t nmax_sigma,
                                     const spd_msd_stats *msd_dev, spd_msd_part *part_dev,
                                     void *workspace, size_t workspace_bytes, void *stream);
/* Eq. 2 over the gathered B_Nmax partials in shard order -> sd_nmax and nmax
 * of out_dev (its other fields are left as they are). */
spd_status spd_sd_nmax_merge_partials(const spd_msd_part *parts_dev, int32_t n_shards,
                                      int32_t nmax_sigma, spd_msd_stats *out_dev, void *stream);

/* Bytes of device workspace spd_boxcar_snr needs. */
size_t spd_boxcar_snr_workspace_bytes(const spd_plane *plane, int32_t scope,
                                      const int32_t *widths, int32_t n_widths);

/* Steps (b)+(c), Sec. 2.3, Algorithm 1: for every sample of every row, the
 * highest SNR over width 1 and the listed widths and the width that gave it.
 *   msd_dev: the spd_msd_stats array of `scope` (from spd_msd, or filled by the
 *     caller; sd_nmax is used by the LINEAR modes, with nmax_sigma = its nmax).
 *   snr_out: float [n_dm][out_stride]; width_out: uint16 [n_dm][out_stride]
 *     (device; columns >= n_samp are not written).
 * SNRs are exact up to FP32 rounding plus a relative 2^-17 quantisation used
 * to carry the width index through the max; widths whose SNRs differ by less
 * than that are treated as ties.  A degenerate MSD entry leaves its rows'
 * outputs at NaN / 0.
 * Errors: SPD_ERR_INVALID_ARG, SPD_ERR_NO_MEMORY, SPD_ERR_CUDA. */
spd_status spd_boxcar_snr(const spd_plane *plane, const spd_msd_stats *msd_dev, int32_t scope,
                          const int32_t *widths, int32_t n_widths, int32_t sigma_mode,
                          float *snr_out, uint16_t *width_out, int64_t out_stride,
                          void *workspace, size_t workspace_bytes, void *stream);

/* Step (d), Sec. 2.4: every (dm, t) with snr[dm][t] >= threshold becomes a
 * record; records are appended in no particular order with warp- and
 * block-aggregated atomics.  snr, width: device planes [n_dm][stride].
 * out: device array of `capacity` records (may be NULL when capacity is 0).
 * result_dev->count is set to the exact number found (the call zeroes it
 * first).  Errors: SPD_ERR_INVALID_ARG, SPD_ERR_CUDA. */
spd_status spd_threshold_candidates(const float *snr, const uint16_t *width, int64_t n_dm,
                                    int64_t n_samp, int64_t stride, float threshold,
                                    spd_candidate *out, int64_t capacity,
                                    spd_result *result_dev, void *stream);

/* Step (d) as the thresholding of Sec. 2.4 writes it, on the plane: in place,
 * snr[dm][t] keeps its value where snr >= threshold and becomes 0 elsewhere
 * (a NaN SNR, from a degenerate MSD, is not >= threshold and becomes 0);
 * width[dm][t] (may be NULL) keeps the width where the SNR is kept, else 0.
 * The kept entries are exactly the records of spd_threshold_candidates.
 * snr, width: device planes [n_dm][stride].  Errors: SPD_ERR_INVALID_ARG,
 * SPD_ERR_CUDA. */
spd_status spd_threshold_plane(float *snr, uint16_t *width, int64_t n_dm, int64_t n_samp,
                               int64_t stride, float threshold, void *stream);

/* An extension after step (d): per-DM clustering of the candidates in time.
 * Sec. 2.4 leaves the list unordered and does no clustering; this groups it.
 * A row's candidates are its samples with snr >= threshold (exactly the
 * records of spd_threshold_candidates). Taken in sample order, a candidate
 * joins the previous candidate's cluster when it lies at most max_gap samples
 * after it, and otherwise starts a new cluster. Equivalently, a cluster is a
 * connected component of the graph that links any two candidates at most
 * max_gap samples apart. Each cluster becomes one spd_cluster record;
 * records are appended in no particular order.
 *   snr, width: device planes [n_dm][stride] (e.g. spd_boxcar_snr's output);
 *     a NaN SNR is never a candidate.
 *   max_gap: >= 1 (1 groups only adjacent samples).
 *   out: device array of `capacity` records, 16-byte aligned (may be NULL when
 *     capacity is 0); result_dev->count is set to the exact number of
 *     clusters (the call zeroes it first), and only the first `capacity`
 *     records are written.
 * One warp scans one row.  Errors: SPD_ERR_INVALID_ARG, SPD_ERR_CUDA. */
spd_status spd_cluster_rows(const float *snr, const uint16_t *width, int64_t n_dm,
                            int64_t n_samp, int64_t stride, float threshold, int32_t max_gap,
                            spd_cluster *out, int64_t capacity, spd_result *result_dev,
                            void *stream);

/* Bytes of device workspace spd_detect / spd_search need. */
size_t spd_detect_workspace_bytes(const spd_plane *plane, const spd_search_params *params);
size_t spd_search_workspace_bytes(const spd_plane *plane, const spd_search_params *params);

/* Steps (b)+(c)+(d) fused in one kernel given the MSD (msd_dev as for
 * spd_boxcar_snr): boxcars, SNR, max over widths and thresholding happen in
 * registers and shared memory; only candidate records leave the SM.  The
 * candidate set equals thresholding spd_boxcar_snr's output.
 * Errors: as spd_boxcar_snr, plus result semantics as spd_threshold_candidates. */
spd_status spd_detect(const spd_plane *plane, const spd_search_params *params,
                      const spd_msd_stats *msd_dev, spd_candidate *out, int64_t capacity,
                      spd_result *result_dev, void *workspace, size_t workspace_bytes,
                      void *stream);

/* The whole path: spd_msd (a) then spd_detect (b, c, d) on one stream.
 *   msd_out_dev: optional device array (1 or n_dm entries) receiving the MSD;
 *     NULL keeps it inside the workspace.
 * The plane is read twice from HBM: once for the MSD, once for the search,
 * because no SNR is known before the dataset's sigma is (Sec. 2.1 -> 2.3). */
spd_status spd_search(const spd_plane *plane, const spd_search_params *params,
                      spd_candidate *out, int64_t capacity, spd_result *result_dev,
                      spd_msd_stats *msd_out_dev, void *workspace, size_t workspace_bytes,
                      void *stream);

/* The whole path for a plane held in HOST memory, the call an application
 * with a host-side DM x time plane makes.  Blocking: it returns when the
 * records are in host memory.  The plane (host data and, if given, host
 * per-row scale / offset) is copied into the workspace, the MSD (a) is
 * computed there, and the search (b, c, d) runs in blocks of rows.  Each
 * block's records are copied to host_out on a second stream while the next
 * block is searched.  Page-locked host memory makes the copies asynchronous;
 * pageable memory works, with slower synchronous copies.
 *   host_out: host array of `capacity` records (the first min(count,
 *     capacity) written, in no stated order); host_result: host summary
 *     (semantics as spd_search); host_msd: optional host array (1 or n_dm
 *     entries) receiving the MSD.
 *   workspace: device, spd_search_host_workspace_bytes(plane, params,
 *     capacity) bytes, 256-byte aligned; it holds the plane, the records and
 *     the search's own workspace.
 * Two host threads may call this at once with their own workspaces and
 * streams; one plane's copies in then overlap the other's copies out.
 * Errors: as spd_search, SPD_ERR_CUDA on a failed copy. */
size_t spd_search_host_workspace_bytes(const spd_plane *plane, const spd_search_params *params,
                                       int64_t capacity);
spd_status spd_search_host(const spd_plane *host_plane, const spd_search_params *params,
                           spd_candidate *host_out, int64_t capacity, spd_result *host_result,
                           spd_msd_stats *host_msd, void *workspace, size_t workspace_bytes,
                           void *stream);

/* One DM range of a batched search: a plane with its own search parameters.
 * dm_offset is added to the row index in the range's candidate records, so
 * that ranges can share one record list; decimation records the time
 * decimation the caller applied to this range (sample and width are in
 * decimated samples; it does not change the search). */
typedef struct {
    spd_plane plane;
    spd_search_params params;
    int32_t dm_offset;
    int32_t decimation;
} spd_range;

/* Launch shape of the candidate search kernel (what the autotuner chooses).
 * ctas_per_sm: persistent CTAs per SM, 0 = as many as fit.
 * group_scale: widths per group are 16 (step 1) or 4 (step G) times this
 *   factor (>= 1): larger groups mean fewer bounds and group starts, smaller
 *   groups a finer pruning.
 * tile_threads: threads per CTA, 128 or 256 (0 = 256); a CTA searches tiles
 *   of 16 * tile_threads consecutive starts of a row, each staged once with
 *   its (wmax - 1)-sample halo.  Other values: SPD_ERR_INVALID_ARG. */
typedef struct {
    int32_t ctas_per_sm;
    int32_t group_scale;
    int32_t tile_threads;
    int32_t reserved1;
} spd_tuning;

#define SPD_MAX_RANGES 8

/* Bytes of device workspace spd_search_batched needs. */
size_t spd_search_batched_workspace_bytes(const spd_range *ranges, int32_t n_ranges,
                                          const spd_tuning *tuning);

/* The whole path over up to SPD_MAX_RANGES DM ranges of uneven length, width
 * set and decimation: per range the MSD (a) and its constants, then ONE
 * persistent detect launch (b, c, d) whose CTAs walk the tiles of all ranges
 * -- per launch, ranges whose width lists step by the same G (8, 16 or 1) and
 * that share storage type and row alignment.  Every call is a fixed sequence of
 * asynchronous launches with no host synchronisation and no allocation, so it
 * can be captured in a CUDA graph and replayed.
 *   tuning: NULL for the defaults.
 *   out / capacity / result_dev: one record list for all ranges (records carry
 *     dm_offset + row).
 *   msd_out_dev: optional; the ranges' spd_msd_stats concatenated in order
 *     (1 or n_dm entries each); NULL keeps them in the workspace.
 * Each range's records are the records spd_search gives for that range alone
 * (with dm_offset added).  Errors: as spd_search; SPD_ERR_INVALID_ARG for
 * n_ranges outside 1..SPD_MAX_RANGES. */
spd_status spd_search_batched(const spd_range *ranges, int32_t n_ranges,
                              const spd_tuning *tuning, spd_candidate *out, int64_t capacity,
                              spd_result *result_dev, spd_msd_stats *msd_out_dev,
                              void *workspace, size_t workspace_bytes, void *stream);

/* ------------------------------------------------------------- streaming
 * A beam delivers its DM x time data in chunks (all chunks of a beam: same
 * n_dm, storage type and per-row scale/offset).  The caller owns a device
 * state buffer (spd_stream_state_bytes) and a host spd_stream_info the calls
 * keep up to date.  The state holds the running MSD of every sample pushed so
 * far (Eq. 2 adds each chunk to it, so mu and sigma are those of all data seen,
 * as Sec. 2.1 defines them for the dataset) and the last wmax - 1 samples of
 * each row (the halo).  A push searches every start whose full window is
 * available -- the halo's starts first, then the chunk's -- with the MSD
 * including that chunk, and holds the last wmax - 1 starts back for the next
 * push; spd_stream_flush searches the held-back starts at the end of the
 * stream with the row-end truncation of the one-shot calls.  The first push
 * with data copies the per-row scale / offset into the state (for the flush);
 * every chunk of the beam must carry the same values.  Candidate
 * samples count from the first sample of the stream.  sigma modes other than
 * SQRTN are unsupported in streaming. */
typedef struct {
    int64_t n_dm;
    int32_t dtype;
    int32_t msd_scope;
    int64_t seen;       /* samples per row pushed so far */
    int64_t halo;       /* samples per row held in the state, not yet searched */
    int64_t chunks;     /* pushes so far */
    int32_t wmax;
    int32_t halo_cap;   /* halo capacity per row in the state (>= wmax - 1) */
    int32_t has_scale;  /* the beam's chunks carry row_scale (set by the first push) */
    int32_t has_offset; /* ... row_offset */
} spd_stream_info;

size_t spd_stream_state_bytes(int64_t n_dm, int32_t dtype, const spd_search_params *params);
size_t spd_stream_workspace_bytes(int64_t n_dm, int64_t max_chunk, int32_t dtype,
                                  const spd_search_params *params);
/* Start a stream: zero the running MSD, empty the halo, fill *info. */
spd_status spd_stream_reset(spd_stream_info *info, void *state_dev, int64_t n_dm, int32_t dtype,
                            const spd_search_params *params, void *stream);
/* Search one chunk (n_samp <= the max_chunk the workspace was sized for).
 * chunk->data may be device memory or page-locked host memory (the chunk is
 * first copied into the workspace on `stream`; pageable host memory makes
 * that copy synchronous); row_scale / row_offset are device pointers.  msd_out_dev: optional device spd_msd_stats (1 or n_dm) receiving
 * the running MSD used.  Result semantics as spd_search. */
spd_status spd_stream_push(spd_stream_info *info, void *state_dev, const spd_plane *chunk,
                           const spd_search_params *params, spd_candidate *out,
                           int64_t capacity, spd_result *result_dev, spd_msd_stats *msd_out_dev,
                           void *workspace, size_t workspace_bytes, void *stream);
/* Where in a push workspace the caller may write a chunk of n_samp samples per
 * row ([n_dm] rows, *row_stride elements apart, 16-byte aligned rows not
 * guaranteed) so that the next spd_stream_push of this stream, given a plane
 * with exactly that data pointer and row_stride and the same workspace, reads
 * it in place instead of copying it.  Valid until that push. */
spd_status spd_stream_chunk_view(const spd_stream_info *info, const spd_search_params *params,
                                 int64_t n_samp, void *workspace, size_t workspace_bytes,
                                 void **data, int64_t *row_stride);
/* Search the held-back starts (end of stream); the state stays valid. */
spd_status spd_stream_flush(spd_stream_info *info, void *state_dev,
                            const spd_search_params *params, spd_candidate *out,
                            int64_t capacity, spd_result *result_dev, void *workspace,
                            size_t workspace_bytes, void *stream);

/* ------------------------------------------------- decimation in time
 * Wide boxcars on data decimated in time, which Sec. 3 names as the way to
 * widen the search; the paper gives no details, so this is this library's
 * scheme.  Level l searches the series x_l[j] = x[2^l j] + ... + x[2^l j +
 * 2^l - 1] (complete groups only, FP32) with its own listed widths (in level
 * samples) and its own measured MSD (Sec. 2.1 on x_l, global scope, Eq. 4),
 * thresholded like the plain search.  A level-l boxcar of w samples at j is
 * the plain B_{w 2^l}(j 2^l), so level l evaluates native widths w 2^l at
 * starts that are multiples of 2^l only: a variant of the plain search, not
 * equal to it.  Records carry native units: sample j 2^l, width w 2^l; the
 * levels' native widths must ascend strictly from level to level, so a
 * record's width tells its level.  msd_out_dev (optional): one spd_msd_stats
 * per level.  Errors: as spd_search_batched. */
#define SPD_MAX_LEVELS 8
typedef struct {
    int32_t level;           /* 0 .. 12, strictly ascending over the array */
    int32_t n_widths;
    const int32_t *widths;   /* host, ascending, in samples of the level */
} spd_level;

size_t spd_search_decimated_workspace_bytes(const spd_plane *plane, const spd_level *levels,
                                            int32_t n_levels);
spd_status spd_search_decimated(const spd_plane *plane, const spd_level *levels, int32_t n_levels,
                                float threshold, spd_candidate *out, int64_t capacity,
                                spd_result *result_dev, spd_msd_stats *msd_out_dev,
                                void *workspace, size_t workspace_bytes, void *stream);

/* Test aid, for the calling host thread's later searches: every wait of the
 * fused kernel for a bulk copy of a tile gives up after limit_ns (1 ms ..
 * 10 s; default 2 s), and extra_bytes (a multiple of 16, at most 4096; 0 in
 * use) more bytes than the copy delivers are expected, so that with
 * extra_bytes > 0 every wait runs out: the kernel sets SPD_ERR_TIMEOUT in the
 * result word and its CTAs leave (each copy itself has landed, so nothing is
 * left in flight).  spd_debug_set_copy_wait(2000000000, 0) restores the
 * default.  Errors: SPD_ERR_INVALID_ARG. */
spd_status spd_debug_set_copy_wait(uint64_t limit_ns, uint32_t extra_bytes);

/* ------------------------------------------------------ de-dispersion
 * The detector runs on de-dispersed data (Sec. 1: the DM x time plane that
 * the pipeline's de-dispersion step produces; Sec. 3 names coupling the
 * search to that step as future work).  This is the plain incoherent
 * de-dispersion that produces such a plane, so that a producer can write DM
 * trials straight into a streaming search's chunk view
 * (spd_stream_chunk_view) and the push reads them in place:
 *   out[d][t] = sum over channels c of x[c][t + delays[d * n_chan + c]],
 * t < n_out, summed in FP32 in channel order.
 * fb: the filterbank as a plane of n_chan = fb->n_dm channel rows of
 * fb->n_samp samples (any storage type, with optional per-channel scale and
 * offset as for the search).  delays: device int32 [n_dm][n_chan] in samples,
 * each in 0 .. fb->n_samp - n_out; a delay outside that range makes the
 * channel add NaN to the output sample (nothing is read outside the row) and
 * sets status_dev->status (optional, device) to SPD_ERR_INVALID_ARG.
 * out: device plane [n_dm][out_stride] of out_dtype (FP32, or FP16 / BF16
 * rounded from the FP32 sum), out_stride >= n_out.  Errors:
 * SPD_ERR_INVALID_ARG (bad sizes or pointers), SPD_ERR_CUDA. */
spd_status spd_dedisperse(const spd_plane *fb, const int32_t *delays, int64_t n_dm, void *out,
                          int32_t out_dtype, int64_t n_out, int64_t out_stride,
                          spd_result *status_dev, void *stream);

/* Test aid: raw boxcar sums B_w(i) (no centring, no scaling) for one width,
 * NaN where i + w > n_samp.  out: float [n_dm][out_stride] (device). */
spd_status spd_boxcar_sums(const spd_plane *plane, int32_t w, float *out,
                           int64_t out_stride, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* SPD_H */
