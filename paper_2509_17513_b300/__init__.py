"""B300-native differentiable tile rasterizer for hierarchical 4D Gaussians.

The compute path is libgc4d.so (hand-written sm_103a CUDA behind the C ABI of
include/gc4d.h); this package only marshals PyTorch tensors into it.
"""
from ._abi import GCError, lib  # noqa: F401
from .render import BatchGraph, GaussianSet, LevelsGraph, MotionField, MotionFrame, Renderer, Saved, camera_struct, render  # noqa: F401

__all__ = ["Renderer", "BatchGraph", "LevelsGraph", "GaussianSet", "MotionField", "MotionFrame", "Saved", "render", "camera_struct", "lib",
           "GCError"]
