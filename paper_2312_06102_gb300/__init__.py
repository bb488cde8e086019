"""GB300 oct-tree builder: Python binding of the C ABI in include/tb.h.

Argument marshalling only -- every step of the build runs in the CUDA
library ``_build/libtb.so`` (compiled by ``compile_lib.py`` for sm_103a).  PyTorch
supplies device memory and the current stream.  There is no CPU fallback:
importing the binding without the library raises.

    import torch, paper_2312_06102_gb300 as tb
    tree = tb.build(pos_cuda_f32_n3, n_crit=16)
    tb.moments(tree, pos, mass)
    tree.ckey, tree.level, tree.parent ...   # torch CUDA tensors (views)
"""
from __future__ import annotations

from ._lib import (  # noqa: F401
    KEYS_HILBERT,
    KEYS_MORTON,
    LEVELS,
    MOM_FP32_COMP,
    MOM_FP32_PLAIN,
    MOM_FP64,
    STATUS,
    TbError,
    Tree,
    build,
    build_batched,
    NOALLOC_MAX_N,
    kernel_launches,
    keys_sorted_noalloc,
    reorder,
    walk,
    walk_counts,
    lib,
    library_path,
    moments,
    selftest_wait,
    set_wait_limit,
    sort_variants,
    status_string,
)
