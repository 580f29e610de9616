"""GB300 (sm_103a) single-pulse search over de-dispersed DM x time planes,
after Adamek & Armour, arXiv:1611.09704.

The search runs in the CUDA kernels of ``_build/libspd.so`` behind the C ABI
of ``include/spd.h``; :mod:`.binding` marshals torch tensors into those calls.
Build the library with :func:`build`.
"""
from .builder import build, LIB as LIBRARY_PATH  # noqa: F401
from .binding import (  # noqa: F401
    BF16, F16, F32, MSD_GLOBAL, MSD_PER_ROW, SIGMA_LINEAR, SIGMA_LINEAR_EXCESS, SIGMA_SQRTN,
    CAND_DTYPE, MSD_DTYPE, Plane, SpdError, boxcar_snr, boxcar_sums, candidates_to_numpy,
    detect, load, msd, msd_to_numpy, read_result, search, search_workspace_bytes,
    threshold_candidates, threshold_plane, widths_to_numpy, RangeSpec, BatchedSearch, search_batched,
    search_batched_workspace_bytes, SpdTuning, BeamStream, search_decimated,
    search_decimated_workspace_bytes, cluster_rows, clusters_to_numpy, CLUSTER_DTYPE, dedisperse,
    search_host, search_host_workspace_bytes)
