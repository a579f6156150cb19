"""GB300 (sm_103a) pentago retrograde library: Python binding of the C ABI.

The binding only marshals arguments: every step of the computation runs in
the CUDA kernels of ``libpentago_gb300.so`` (see ``include/pentago_gb300.h``).
If the library is missing, every call raises; there is no CPU fallback.

Device buffers are PyTorch CUDA tensors, passed by pointer together with the
current CUDA stream.  Super values are ``int64`` tensors of shape ``[n, 8]``
(words 0-3 win table, 4-7 not-lose table, bit beta(g) = g0 + 4 g1 + 16 g2 +
64 g3 at word beta >> 6, bit beta & 63; int64 holds the uint64 bit pattern).
"""
from __future__ import annotations

from ._native import (  # noqa: F401
    autotune_cache_clear,
    autotune_cache_load,
    autotune_cache_save,
    autotune_cache_stats,
    PentagoError,
    SECTION_DTYPE,
    Server,
    Stager,
    SlicePlan,
    MidgamePlan,
    five_masks,
    init,
    launch_count,
    lib,
    library_path,
    midgame_solve,
    midgame_solve_host,
    midgame_parity_workspace_bytes,
    midgame_solve_noalloc,
    midgame_solve_parity,
    midgame_workspace_bytes,
    prepare_children,
    prepare_children_ready,
    quadrant_states,
    rmax,
    section_compute,
    selftest_barrier_timeout,
    set_barrier_poll_limit,
    shift,
    PP_ABSENT,
    compact_offsets,
    section_count,
    slice_children,
    slice_sections,
    slice_step_sparse,
    slice_step,
    super_digest,
    symmetry_board,
    symmetry_info,
    symmetry_transform,
)
