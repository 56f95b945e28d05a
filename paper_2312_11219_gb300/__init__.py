"""GB300-native three-way ACA for convolution-quadrature boundary elements.

Python binding of the C ABI (include/g3aca.h) of the CUDA library built in
`lib/libg3aca.so`.  Importing this package loads the library; if it has not
been built the import fails (there is no CPU fallback).

Entry points (same names as the C ABI):
  build_cluster_tree, assemble_near, aca3_compress, apply_gcq
plus the tree of element-local linear shape functions (build_p1_tree) for the
hypersingular operator and the adjoint double layer, frequency sets (g3_freqs_bdf2, g3_freqs_gcq, g3_freqs_from_array), diagnostic entries
(g3_entries), a separable-tensor compression used by the tests, and the
block predictor (Mlp, mlp_create, mlp_train, block_features) whose rank and
first-frequency predictions size the factor pool, order the queue and seed k1.
"""
from ._binding import (  # noqa: F401
    EXPORTED, LIB_PATH, Context, Factors, Freqs, G3Error, Near, Tree, aca3_compress, aca3_compress_batch, autotune,
    aca3_compress_separable, apply_gcq, apply_gcq_noalloc, gcq_history, assemble_near, build_cluster_tree, build_p1_tree, freqs_from_spec,
    g3_entries, shard_rows, tree_subset, tree_partition_host, g3_freqs_bdf2, g3_freqs_gcq, g3_freqs_from_array, MLP_NF, MLP_NP, Mlp, block_features, mlp_create, mlp_train,
)
