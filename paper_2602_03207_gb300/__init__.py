"""GB300-native (sm_103a) 3D Gaussian Splatting render path of WebSplatter
(arXiv 2602.03207): C-ABI library ``libwebsplat.so`` plus a thin binding.

Modules:
    capi       ctypes binding of include/websplat.h (same names as the C ABI)
    render     Renderer: buffers + the four calls of a frame
    batch      BatchRenderer: many views of one scene, forward + backward
    autotune   tile size x digit width search for the batched step
    ply        3DGS scenes from / to PLY files
    synthetic  seeded input generators (no render arithmetic)
    build      nvcc build of the library
"""
__all__ = ["capi", "render", "batch", "autotune", "ply", "synthetic", "build"]
