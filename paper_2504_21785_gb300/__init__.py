"""Frozen Gaussian reconstruction on GB300: Python binding of libfgr (include/fgr.h).

The computation lives in the CUDA library ``libfgr.so`` (sources in csrc/);
``fgr`` marshals arguments to its C ABI.  Build the library with
``paper_2504_21785_gb300._build.build()`` (``__graft_entry__.build()`` does it).
"""

from . import fgr  # noqa: F401
from .fgr import (  # noqa: F401
    Context, FgrError, make_grid, make_options, make_packets, make_potential,
    fgr_create, fgr_destroy, fgr_propagate, fgr_decompose, fgr_fggc_multistep, fgr_decompose_tensor,
    fgr_fggc_multistep_tensor, make_axes, fgr_reconstruct_direct, fgr_reconstruct_direct_batch,
    fgr_reconstruct_fggc, fgr_fggc_plan_create, fgr_reconstruct_fggc_planned, fgr_reconstruct_fggc_batch,
    fgr_fggc_plan_overflow,
    fgr_fggc_plan_info, fgr_fggc_plan_destroy,
    fgr_get_info, fgr_set_timing, fgr_get_stats, fgr_last_error, fgr_autotune, fgr_get_tuning,
    fgr_set_tuning,
    fgr_server_create, fgr_server_destroy, fgr_server_set_max_batch, fgr_register_packets, fgr_release_packets,
    fgr_submit, fgr_poll, fgr_cancel, make_request, FGR_FP64, FGR_FP32, FGR_FLAG_FFT_GRID, FGR_FLAG_SNAP_CP, FGR_FLAG_DIRECT_FMA,
)
