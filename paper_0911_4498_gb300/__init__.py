"""GB300-native fast Basic SSA (arXiv:0911.4498): FFT-based trajectory-matrix
products driving a thick-restart Golub-Kahan-Lanczos truncated SVD, and
FFT-based grouped Hankelization, in hand-written CUDA for sm_103a.

The compute lives in ``libssa_gb300.so`` (C ABI in ``include/ssa.h``);
``paper_0911_4498_gb300._lib`` is its ctypes binding and
``paper_0911_4498_gb300.build`` compiles it.  ``synth`` holds the seeded
synthetic workloads.
"""
from ._lib import (ssa_batch_destroy, ssa_batch_get, ssa_batch_info, ssa_batch_plan, ssa_batch_reconstruct,
                   ssa_batch_run, ssa_batch_wait, ssa_decompose_batch,  # noqa: F401
                   SSA_ENOCONV, SSA_ENOMEM, SSA_OK, SSA_PREC_F32C, SSA_PREC_F64, SSA_REFINE_OFF, SSA_REFINE_ON, SSA_REORTH_FULL, SSA_REORTH_NONE, SSA_REORTH_PRO,
                   SSAError, groups_csr, lib, make_opts,
                   ssa_decomp_destroy, ssa_decomp_get, ssa_decomp_info, ssa_decompose, ssa_default_opts,
                   ssa_embed_plan, ssa_fft_threads, ssa_fft_tiling, ssa_get_spectrum, ssa_hankelize, ssa_hmatrix, ssa_last_error, ssa_matvec, ssa_matvec_noalloc,
                   ssa_plan_destroy,
                   ssa_plan_info, ssa_reconstruct, ssa_set_series, ssa_stats_enable, ssa_stats_get,
                   ssa_kernel_launches, ssa_fault_inject_alloc, ssa_cw_filter, ssa_strerror, SSA_SERVE_VECTORS, make_serve_opts, ssa_serve_create,
                   ssa_serve_default_opts, ssa_serve_destroy, ssa_serve_poll, ssa_serve_stats, ssa_serve_submit,
                   ssa_serve_take)
