"""GB300-native block-based volume renderer after City-on-Web (arXiv 2312.16457).

The renderer is libcow.so (CUDA kernels for sm_103a behind the C ABI in
include/cow.h); ``cow`` is its ctypes binding, ``synth`` the seeded input
generator and ``build`` the in-tree nvcc build.
"""
__all__ = ["cow", "synth", "build"]
