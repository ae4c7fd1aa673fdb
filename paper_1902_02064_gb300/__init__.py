"""GB300 thick-restart block Lanczos for M-scheme shell-model Hamiltonians.

Thin Python binding of the C-ABI library libtrbl.so (declared in
include/trbl.h): argument marshalling only.  Every step of the computation
runs in the library's CUDA kernels; there is no CPU fallback.  PyTorch is
used for device memory and streams.

Method: Shimizu, Mizusaki, Utsuno, Tsunoda, arXiv 1902.02064 -- the
thick-restart block Lanczos method (Sec. III D, Alg. 4) with the on-the-fly
block product H V on a proton-neutron factorised M-scheme basis (App. A,
App. B).
"""
from ._lib import (  # noqa: F401
    TRBL_OK, TRBL_ERR_ARG, TRBL_ERR_CUDA, TRBL_ERR_OOM, TRBL_ERR_BREAKDOWN, TRBL_ERR_NOCONV,
    TRBL_F32, TRBL_F64, TRBL_PREC_F64, TRBL_PREC_MIXED, TRBL_PROJ_TENSOR, TRBL_PROJ_CUDA_CORE, TRBL_REORTH_SELECTIVE, TRBL_REORTH_TWICE,
    TRBL_NOALLOC_SCRATCH_BYTES,
    TRBL_APPLY_GROUPED, TRBL_APPLY_FAST, TRBL_APPLY_GROUPED_X2, TRBL_APPLY_SPLIT, TRBL_APPLY_SPLIT_X4, TRBL_APPLY_SPLIT_TMA, TRBL_TUNE_CANDIDATES, TrblError,
    lib, library_path,
    trbl_basis_create, trbl_basis_destroy, trbl_basis_info, trbl_basis_export,
    trbl_basis_export_jumps, trbl_hamiltonian_create, trbl_hamiltonian_destroy,
    trbl_apply_block, trbl_solve, trbl_last_error, trbl_kernel_launches, trbl_block_dot, block_dot,
    trbl_block_dot_noalloc, trbl_block_dot_tc, trbl_block_update, block_update,
    trbl_solver_create, trbl_solver_step, trbl_solver_step_host, trbl_solver_block,
    trbl_solver_stats, trbl_solver_destroy, trbl_solver_state_bytes, trbl_solver_save, trbl_solver_load,
    trbl_param_count, trbl_grad, arrays_from_theta, clusters_of, hf_gradient, hf_gradient_clusters, LowestEigenvalues,
    solve_batch, apply_autotune, apply_set_rows, apply_set_shape, apply_get_shape, apply_set_compensated,
    Basis, Hamiltonian, Solver, HostBuffer, shard_plan, shard_sources, solve,
)
