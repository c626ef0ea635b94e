"""Stein ICP on GB300: the data-parallel hot path of Stein ICP (Afzal Maken,
Ramos, Ott) as hand-written sm_103a CUDA kernels behind a C ABI
(include/steinicp.h, libsteinicp.so), with this thin Python binding."""
from .binding import (  # noqa: F401
    EXPORTS, SICP_EINVAL, SICP_ENOMEM, SICP_ENOREF, SICP_ENOSURROGATE, SICP_ECUDA, SICP_ETIMEOUT,
    SICP_NN_BRUTE_BF16, SICP_NN_BRUTE_FP32, SICP_NN_GRID, SICP_NN_SURROGATE, SICP_OK, SicpError,
    LIB_PATH, lib, sicp_create, sicp_default_params, sicp_destroy, sicp_icp_grad, sicp_last_error,
    sicp_minibatch, sicp_moments, sicp_moments_circular, sicp_nn, sicp_params, sicp_profile, sicp_register,
    sicp_set_reference,
    sicp_stats, sicp_stein_adam, sicp_icp_grad_noalloc, sicp_register_batched, sicp_autotune_batched, pack_batch,
    SURROGATE_NPARAM, sicp_surrogate_train, sicp_surrogate_params, sicp_surrogate_loss_grad, sicp_surrogate_infer,
    sicp_register_continue, sicp_surrogate_save, sicp_surrogate_load, sicp_reference_normals, SICP_POINT_TO_PLANE,
    SICP_INDEPENDENT, sicp_gaussian_kl, sicp_gaussian_ovl, sicp_pose_distribution, sicp_compound, chain_odometry,
    sicp_export_state, sicp_import_state, sicp_resume, sicp_set_memory_limit, sicp_set_wait_check,
    sicp_trace_batched, sicp_read_batched_trace, sicp_surrogate_train_run, sicp_set_telemetry,
    sicp_read_telemetry, TELEMETRY_FIELDS, sicp_check_status,
)
