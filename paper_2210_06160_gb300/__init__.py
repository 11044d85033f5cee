"""GB300 (sm_103a) implementation of the RTSDF hot path (arxiv 2210.06160).

`rtsdf` is the Python binding of librtsdf (include/rtsdf.h); `scenes` generates
seeded synthetic inputs; `build` compiles the CUDA library in-tree.
"""
__all__ = ["rtsdf", "scenes", "build"]
