"""GB300-native differentiable splatting of rectangular plane primitives.

PlanarSplatting (arxiv 2412.03451) renders 3D rectangles (center, quaternion,
four one-sided radii) into per-view depth and normal maps with a soft
rectangle-boundary weight and front-to-back compositing, and fits them to
depth/normal supervision with Adam.  This package holds the sm_103a CUDA
library that runs every step of that hot path (``csrc/``), its ctypes
binding (``binding``), the PyTorch-side driver of one optimisation step
(``splat``), batched multi-scene fitting (``batch``, ``autotune``), the
seed-proposal network (``seednet``, ``seed_train``), the multi-rank helpers
(``ranks``) and the seeded synthetic room generator (``scenes``).  Nothing here falls back to the CPU: if the
compiled library is missing the binding raises.
"""
__all__ = ["scenes"]
