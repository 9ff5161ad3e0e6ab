"""GB300 (sm_103a) randomized PCA: the hot path of Szlam, Kluger & Tygert (2014).

The compute is in librpca.so (hand-written CUDA behind the C ABI of
include/rpca.h); ``rpca`` holds the Python binding with the same entry-point
names.  ``build.build()`` compiles the library in-tree.
"""
from .rpca import (RpcaError, rpca_dense, rpca_dense_workspace_size, rpca_gaussian_omega,  # noqa: F401
                   rpca_launch_count, rpca_philox4x64_10, rpca_read_status, make_opts,
                   read_status_block, workspace)
