"""GB300-native boxcar single-pulse detection (Adamek & Armour, arXiv:1910.08324).

This package is a thin ctypes binding over ``libspd.so`` (CUDA, sm_103a), whose C
ABI is declared in ``include/spd.h``.  Every step of the search runs in the
library's kernels; Python only marshals arguments.  PyTorch is used for device
memory and streams.  There is no CPU fallback: if the library cannot be built
or loaded, importing the binding functions raises.

Entry points (same names as the C ABI): ``spd_plan_create``,
``spd_plan_destroy``, ``spd_plan_widths``, ``spd_workspace_size``,
``spd_execute``, ``spd_candidates``, ``spd_candidates_static``, ``spd_search``,
``spd_noise_stats``, ``spd_plan_set_segment``, the batch calls
(``spd_batch_create``, ``spd_batch_execute``, ``spd_batch_status``,
``spd_batch_candidates``; ``Batch`` for the rest), ``spd_sync_status``,
``spd_status_string``, ``spd_version``.  Convenience wrappers taking torch
tensors: ``execute``, ``candidates``, ``search``, ``noise_stats``,
``batch_execute``.
"""
from ._binding import (  # noqa: F401
    CANDIDATE_DTYPE,
    SPD_ALGO_BOXDIT,
    SPD_ALGO_EXHAUSTIVE,
    SPD_ALGO_IGRID,
    SPD_BF16,
    SPD_F16,
    SPD_F32,
    SPD_U8,
    Batch,
    Plan,
    SpdError,
    batch_execute,
    candidates,
    execute,
    library_path,
    load_library,
    net_adam,
    net_decimate,
    net_gather,
    net_select,
    net_forward,
    net_gradient,
    net_gradient_ordered,
    spd_net_gradient_workspace_size,
    noise_stats,
    records,
    search,
    spd_batch_candidates,
    spd_batch_create,
    spd_batch_execute,
    spd_batch_status,
    spd_candidates,
    spd_candidates_static,
    spd_candidates_status,
    spd_execute,
    spd_net_param_count,
    spd_noise_stats,
    spd_plan_create,
    spd_plan_set_segment,
    spd_plan_set_starts,
    spd_plan_create_grid,
    spd_plan_destroy,
    spd_plan_widths,
    spd_search,
    spd_status_string,
    spd_sync_status,
    spd_version,
    spd_workspace_size,
)
