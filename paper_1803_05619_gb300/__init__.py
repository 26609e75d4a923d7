"""Fast end-to-end trainable guided filter (Wu et al.) on sm_103a.

The layer runs in libdgf.so (hand-written CUDA kernels behind the C ABI of
include/dgf.h); this package is its Python binding.
"""
from . import _lib  # noqa: F401
from .layer import (GuidedFilter, GuidedFilterFn, GuidedFilterTransformFn,  # noqa: F401
                    GuidedFilterWithTransform, gf_backward, gf_backward_batched, gf_forward,
                    gf_forward_batched)
