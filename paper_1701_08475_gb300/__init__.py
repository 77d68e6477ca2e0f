"""GB300 (sm_103a) kNN-graph construction by two-means trees
(Zhao, Yang, Deng, arXiv 1701.08475, Sec. 3.1, Alg. 1) with neighbour-of-
neighbour refinement, the enhanced hill-climbing search over the graph
(Sec. 3.2, Alg. 2), and the residue-quantisation inverted index that seeds it
(Sec. 4).

A thin binding of the C ABI declared in include/knng.h: every function has
the name of its C entry point, marshals tensors to plain pointers and sizes,
and calls the CUDA library.  No step of the method runs in Python.
"""
from ._lib import (  # noqa: F401
    KNNG_BF16,
    KNNG_FP16,
    KNNG_FP32,
    KNNG_FP8,
    KNNG_JOIN_FWD,
    KNNG_JOIN_FWD_REV,
    KNNG_JOIN_SAMPLED,
    KnngError,
    Params,
    default_params,
    knng_build,
    knng_build_ex,
    knng_build_batched,
    BuildPlan,
    BatchedPlan,
    knng_exact,
    knng_search,
    knng_rvq_train,
    knng_rvq_index,
    knng_rvq_seeds,
    knng_exact_noalloc,
    knng_leaf_dhat,
    knng_leaf_update,
    knng_partition,
    knng_recall,
    knng_refine,
    knng_tree_depth,
    knng_workspace_bytes,
    library_path,
    load,
    stats,
    stats_enable,
    stats_reset,
)
