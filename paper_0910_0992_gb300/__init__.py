"""GB300-native temporally preconditioned anisotropic Wilson solver (arXiv 0910.0992).

The compute path is the C-ABI library ``libwf.so`` (hand-written CUDA for sm_103a,
declared in ``include/wf.h``); this package is a thin ctypes binding with the same
entry-point names. It does argument marshalling only: every step of an apply or a
solve runs in the library's kernels. There is no CPU fallback: importing the
binding fails loudly if the library has not been built (``build_lib.build()``).

Arrays are complex128, C-contiguous, in the layouts of ``include/wf.h``; they may
be torch tensors (CUDA or CPU) or NumPy arrays (host).
"""

from ._lib import (  # noqa: F401
    WF_OK, WF_EINVAL, WF_ENOMEM, WF_ECUDA, WF_ESINGULAR, WF_ENOCONV, WF_ENAN, WF_ETIMEOUT,
    WF_UNPREC, WF_EO4D, WF_TEMPORAL, WF_TEMPORAL_SCHUR, WF_TEMPORAL_ILU, WF_FP64, WF_FP32, WF_FP16MIX, WF_X0, WF_MAX_SOLVE_RHS,
    WFError, lib, lib_path, exported_symbols,
    wf_create, wf_destroy, wf_set_stream, wf_last_error, wf_set_gauge_frame, wf_field_elems, wf_half_elems,
    wf_load_gauge, wf_load_gauge_clover, wf_apply_clover, wf_apply_ilu, wf_apply_ilu_f32, wf_apply_M, wf_apply_M_f32, wf_apply_Tinv, wf_apply_Tinv_f32, wf_apply_C,
    wf_apply_schur, wf_apply_schur_f32, wf_apply_schur_f16, wf_apply_schur_noalloc, wf_apply_eo4d, wf_apply_eo4d_f32, wf_apply_Qinv, wf_apply_Qinv_f32, wf_apply_schur_full_sw, wf_apply_schur_full_sw_f32, wf_solve_full_sw, wf_solve, wf_solve_many, wf_force, wf_temporal_logdet, wf_launch_count, wf_check_tables, wf_hop_config, wf_hop_pipe_config, wf_set_max_iterations, wf_profile, wf_profile_get,
    Wilson,
)
