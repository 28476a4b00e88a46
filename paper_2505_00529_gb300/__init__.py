"""GB300-native (sm_103a) exact gradient and Hessian of the discrete
quantum-optimal-control cost by the first- and second-order adjoint method
(Bhat, arXiv 2505.00529), behind the C ABI declared in include/qoc.h.

``inputs`` draws the seeded synthetic problems; ``_lib`` binds libqoc.so
(build it with ``build.build()``)."""
from . import inputs
from ._lib import (  # noqa: F401
    Problem, QocError, TrOptions, TrReport, lib, qoc_create_problem, qoc_destroy_problem,
    qoc_enable_timing, qoc_eval_grad, qoc_eval_grad_hess, qoc_eval_grad_hess_dev, qoc_eval_J,
    qoc_get_diagnostics, qoc_read_buffer, qoc_set_eig_method, qoc_set_hess_method,
    qoc_sync_status, qoc_trust_region_solve, qoc_set_block_steps, qoc_device_bytes, qoc_max_basis_size, qoc_version,
    MLP, qoc_set_target, qoc_mlp_param_count, Batch, qoc_batch_create, qoc_batch_destroy,
    qoc_batch_eval_grad_hess, qoc_batch_eval_grad_hess_dev, qoc_batch_set_graph,
    qoc_assemble_grad_hess_noalloc, qoc_assemble_noalloc_scratch_doubles, qoc_get_phase_times, qoc_get_eig_stats, qoc_set_panel_columns,
    qoc_get_precision, QOC_MIXED_FP32_ALWAYS, qoc_measure_fp64_rate, qoc_batch_trust_region_solve, qoc_tr_subproblem,
    qoc_eval_grad_hess_model, qoc_set_refine_sweeps, qoc_selftest_bounded_wait, qoc_set_pipeline, qoc_get_tr_phase_times, qoc_set_mu_split,
    QOC_FP64, QOC_MIXED_FP32, QOC_HESS_SECOND_ORDER_ADJOINT, QOC_HESS_TANGENT, QOC_EIG_REFINED,
    QOC_EIG_JACOBI_FP64,
)
