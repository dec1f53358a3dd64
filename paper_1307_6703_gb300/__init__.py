"""GB300 (sm_103a) lattice Boltzmann solver for the van der Waals liquid-vapour
fluid under a periodic potential and shear (arXiv:1307.6703).

The computation runs in the CUDA library ``_build/liblb.so`` (C ABI in
``include/lb.h``); :mod:`paper_1307_6703_gb300.lb` is a thin ctypes binding
with the same names.  There is no CPU fallback.
"""
from .lb import (Batch, LB_BF16DEV, LB_DTYPE_F32, LB_DTYPE_F64, LB_ERR_ARG, LB_ERR_CUDA,
                 LB_ERR_OOM, LB_ERR_STATE, LB_ERR_TIMEOUT, LB_ERR_UNSTABLE, LB_FP16DEV,
                 LB_FP32, LB_FP64, LBError, Solver, lb_create, lb_destroy, lb_get_state,
                 lb_autotune, lb_batch_autotune, lb_batch_create, lb_batch_destroy,
                 lb_batch_handle, lb_batch_last_error, lb_batch_step, lb_get_step, lb_init, lb_last_error, lb_moments, lb_params, lb_reduce,
                 lb_monitor, lb_reduce_async, lb_reduce_noalloc, lb_set_seg_h, lb_get_tiling, lb_set_tiling, lb_set_state, lb_step, lb_sweep_dependencies,
                 load_library)

__all__ = [n for n in dir() if n.startswith(("lb_", "LB_"))] + ["Solver", "Batch", "LBError", "load_library"]
