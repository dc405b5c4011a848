"""GB300-native screened Fock exchange (Challacombe & Bock, "An N-Body
Solution to the Problem of Fock Exchange").

The library ``libkx.so`` (CUDA, sm_103a) exposes the C ABI of
``include/kx.h``; this package is its Python binding (``_binding``) and
build script (``build``).  There is no CPU path: without the built library
the binding raises.
"""
from ._binding import (  # noqa: F401
    EXPORTS, KX_ECAPACITY, KX_ECUDA, KX_EINVAL, KX_ENOMEM, KX_ENOTIMPL, KX_ESTATE, KX_ETIMEOUT,
    KX_FP64, KX_MIXED, KX_MIXED_DW, NSTREAM, KX_OK, BatchExchange, Exchange, KxError, kx_basis, kx_build_schwarz, kx_build_tree,
    kx_create, kx_default_opts, kx_destroy, kx_exchange, kx_exchange_host, kx_count, kx_get_leaves,
    kx_get_norms, kx_get_order, kx_get_profile, kx_get_worklist, kx_peak_probe, kx_traverse_level_noalloc, KX_NOALLOC_MAX_TASKS,
    kx_traverse, kx_leaf_features, kx_cull_kept, kx_evaluate_kept, kx_exchange_leaves, kx_block_norms,
    kx_mlp_infer_bf16, kx_mlp_loss_grad, kx_mlp_adam, KX_NFEAT, KX_MLP_HIDDEN, KX_MLP_NPARAM, kx_last_error, kx_n_functions, kx_opts,
    kx_stats, library_path, load, kx_create_batch, kx_exchange_batch, kx_exchange_batch_host, kx_packed_size,
    kx_autotune, kx_get_launch_shapes, kx_set_launch_shape, kx_graph_plan, kx_graph_launch, KX_PROBE_FP64_MMA, KX_PROBE_DW,
    kx_row_work, kx_shard_bounds, kx_split_plan, kx_class_flops,
)
