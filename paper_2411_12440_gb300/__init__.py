"""GB300-native (sm_103a) rasterizer for 3D Linear Splatting (arxiv 2411.12440).

The compute path is a C-ABI library of hand-written CUDA kernels (libls.so,
declared in include/ls.h); this package only marshals arguments to it.  The
native library is loaded on first use and its absence is an error: there is
no CPU fallback.
"""
__all__ = ["scenes"]
