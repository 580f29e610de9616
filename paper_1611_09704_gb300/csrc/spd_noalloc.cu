// spd_noalloc.cu -- spd_msd_noalloc: the MSD of spd_msd computed with scratch
// memory that the library owns statically, for callers that cannot hand the
// library a workspace.
//
// Who needs it: a caller that must not allocate device memory once it is
// running -- a real-time telescope backend that fixes its memory at start-up
// and treats any later allocation as a latency hazard, code running where a
// cudaMalloc would synchronise the device or is not allowed, or a plain C
// caller that owns only the plane and the output and has no allocator to
// size a workspace with.  Such a caller passes its input plane and its
// output array; the block partials live in a fixed array in device memory
// that this library declares at file scope.
//
// The array is loaded with the library on every GPU that uses it and stays
// allocated until the process exits.  Host code must not use the array's name
// as a device address (it is a host-side stand-in): the address comes from
// cudaGetSymbolAddress with the device current.  Every call made outside
// stream capture looks it up again, so a device reset (after which the array
// may sit elsewhere) is handled; a call during stream capture uses the
// address found by the last call outside capture on that device, so one call
// outside capture must come first.
#include "spd_internal.cuh"

#include <mutex>

namespace spd {
void note_cuda_error(int e);
}

constexpr int kMergeSlots = 256;

// One partial per (row, 65536-sample unit) plus the merge kernel's level-1
// slots; (32768 + 256) * 40 bytes = 1,320,960 bytes.
static __device__ __align__(256) spd::MsdPart g_msd_scratch[SPD_MSD_NOALLOC_MAX_UNITS + kMergeSlots];

namespace {

constexpr int kMaxDevices = 64;

std::mutex g_mu;
void *g_addr[kMaxDevices] = {nullptr};

// Device address of g_msd_scratch on the current device: looked up on every
// call outside stream capture (and remembered), the remembered one during
// capture.
cudaError_t scratch_address(cudaStream_t st, void **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_mu);
    if (cs == cudaStreamCaptureStatusNone) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_msd_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    } else if (!g_addr[dev]) {
        return cudaErrorStreamCaptureUnsupported;   // no call outside capture yet
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" spd_status spd_msd_noalloc(const spd_plane *plane, int32_t scope,
                                      spd_msd_stats *out_dev, void *stream) {
    if (!plane || !out_dev) return SPD_ERR_INVALID_ARG;
    if (scope != SPD_MSD_GLOBAL && scope != SPD_MSD_PER_ROW) return SPD_ERR_INVALID_ARG;
    if (plane->dtype < SPD_F32 || plane->dtype > SPD_BF16) return SPD_ERR_INVALID_ARG;
    if (plane->n_dm < 0 || plane->n_samp < 0 || plane->n_dm > INT32_MAX ||
        plane->n_samp > INT32_MAX)
        return SPD_ERR_INVALID_ARG;
    const bool empty = plane->n_dm == 0 || plane->n_samp == 0;
    if (!empty) {
        if (!plane->data || plane->row_stride < plane->n_samp) return SPD_ERR_INVALID_ARG;
        if (reinterpret_cast<uintptr_t>(plane->data) % spd::elem_bytes(plane->dtype))
            return SPD_ERR_INVALID_ARG;
        if (plane->row_offset && !plane->row_scale) return SPD_ERR_INVALID_ARG;
    }
    const int64_t upr = plane->n_samp > 0 ? (plane->n_samp + spd::kMsdUnit - 1) / spd::kMsdUnit : 0;
    const int64_t units = plane->n_dm * upr;
    if (units > SPD_MSD_NOALLOC_MAX_UNITS) return SPD_ERR_NO_MEMORY;   // beyond the static array
    if (scope == SPD_MSD_PER_ROW && plane->n_dm == 0) return SPD_OK;

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    void *base = nullptr;
    cudaError_t e = scratch_address(st, &base);
    if (e != cudaSuccess) { spd::note_cuda_error((int)e); return SPD_ERR_CUDA; }
    spd::MsdPart *parts = static_cast<spd::MsdPart *>(base);
    spd::MsdPart *slots = parts + SPD_MSD_NOALLOC_MAX_UNITS;

    // Every partial and slot read below is written earlier in this call, so
    // nothing left in the array by a previous call is used.
    if (!empty) {
        spd::MsdArgs a;
        a.data = plane->data;
        a.n_dm = plane->n_dm;
        a.n_samp = plane->n_samp;
        a.stride = plane->row_stride;
        a.scale = plane->row_scale;
        a.offset = plane->row_offset;
        a.units_per_row = upr;
        const size_t need = 4 * spd::elem_bytes(plane->dtype);
        a.vec_ok = (reinterpret_cast<uintptr_t>(plane->data) % need == 0) &&
                   ((size_t)plane->row_stride * spd::elem_bytes(plane->dtype)) % need == 0;
        a.parts = parts;
        e = spd::launch_msd_partial(a, plane->dtype, st);
        if (e != cudaSuccess) { spd::note_cuda_error((int)e); return SPD_ERR_CUDA; }
    }
    e = spd::launch_msd_merge(parts, plane->n_dm, upr, plane->n_samp, scope == SPD_MSD_PER_ROW,
                              slots, kMergeSlots, out_dev, st);
    if (e != cudaSuccess) { spd::note_cuda_error((int)e); return SPD_ERR_CUDA; }
    return SPD_OK;
}
