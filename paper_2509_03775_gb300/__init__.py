"""GB300-native codebook Gaussian-splatting rasterizer (the differentiable
renderer of ContraGS, arXiv 2509.03775), behind the C ABI of include/cg.h.

The CUDA library libcg.so is built in-tree by ``_build.build()``; ``cg``
holds the ctypes binding, the workspace-owning ``Renderer`` and the
``CodebookRender`` autograd Function; ``scenes`` draws seeded synthetic
inputs.
"""
__all__ = ["cg", "scenes"]
