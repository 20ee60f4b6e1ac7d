"""GB300 (sm_103a) wavelet rasterizer: the differentiable rendering path of WIPES
(wavelet-based visual primitives, ICCV 2025) behind a C ABI (``include/wipes.h``).

Importing the package does not load the CUDA library; the first call does, and fails loudly if
``libwipes.so`` has not been built (``paper_2508_12615_gb300.build.build()``).
"""
from .render import (Context, Deform6D, DeformMLP, Render2D, Render3D, State, backward, deform6d, deform_field,
                     deform_mlp, deform_mlp_backward, deform_mlp_param_count, forward2d, forward3d, l2_loss,
                     make_opts, render2d, render3d, sort_pairs)

__all__ = ["Context", "State", "Render2D", "Render3D", "Deform6D", "DeformMLP", "render2d", "render3d", "deform6d",
           "deform_field", "deform_mlp", "deform_mlp_backward", "deform_mlp_param_count", "forward2d", "forward3d",
           "backward", "l2_loss", "make_opts", "sort_pairs"]
