"""GB300 (sm_103a) randomized PCA: the hot path of Szlam, Kluger & Tygert (2014).

The compute is in librpca.so (hand-written CUDA behind the C ABI of
include/rpca.h); ``rpca`` holds the Python binding with the same entry-point
names.  ``build.build()`` compiles the library in-tree.
"""
from .rpca import (RpcaError, rpca_dense, rpca_dense_workspace_size, rpca_gaussian_omega,  # noqa: F401
                   rpca_resid_norm, rpca_dense_pass, rpca_csr, rpca_resid_norm_csr, Batch, rpca_batched,
                   rpca_launch_count, rpca_philox4x64_10, rpca_read_status, make_opts,
                   read_status_block, workspace, rpca_timing_enable, rpca_timing_reset,
                   rpca_timing_read, rpca_timing_select, rpca_sketch_features, rpca_batched_features, batch_col_offsets,
                   rpca_mlp_pack, rpca_mlp_forward, rpca_mlp_loss_grad, rpca_mlp_adam, rpca_leverage_target,
                   rpca_dense_learned, weights_table, rpca_batched_tune, rpca_sym, rpca_nystrom, rpca_small_svd,
                   rpca_batched_learned)
