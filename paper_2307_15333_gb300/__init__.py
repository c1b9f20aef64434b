"""GB300-native Dynamic PlenOctree (DOT, arXiv 2307.15333) hot path.

The CUDA library ``libdot.so`` (C ABI in include/dot.h) renders rays through a sparse octree of
(density, SH) leaves (Eq. 1-2), differentiates the render, accumulates the training signal of
Sec. 3.1, selects leaves (Sec. 3.2, Algorithm 1) and applies the prune / sample operations
(Eq. 3-4).  ``dot`` is the ctypes binding with the same entry-point names; ``autograd`` wraps
forward and backward in a ``torch.autograd.Function``.
"""
from . import dot
from .dot import (DotError, Octree, build_desc, cameras_tensor, dot_accumulate_signal,
                  dot_octree_build, dot_refine_plan, dot_refine_prune, dot_render_backward,
                  dot_render_forward, dot_render_stats, dot_select_masks, dot_tree_import,
                  dot_tree_status, dot_version, lib, rays_buffer, rays_cameras, render_opts,
                  select_opts)

__all__ = ["dot", "DotError", "Octree", "build_desc", "cameras_tensor", "dot_accumulate_signal",
           "dot_octree_build", "dot_refine_plan", "dot_refine_prune", "dot_render_backward",
           "dot_render_forward", "dot_render_stats", "dot_select_masks", "dot_tree_import",
           "dot_tree_status", "dot_version", "lib", "rays_buffer", "rays_cameras", "render_opts",
           "select_opts", "octree_from_scene"]


def octree_from_scene(scene, stream=None, allocator=None) -> Octree:
    """Builds the octree of a scene description (any object with center, half_size, max_depth,
    sh_degree, storage, prims, density_lo/hi, sh_std, sh_dc, seed attributes); `allocator`
    (dot.TorchAllocator) backs the tree's arrays with torch's caching allocator."""
    d = build_desc(scene.center, scene.half_size, scene.max_depth, scene.sh_degree,
                   scene.storage, scene.prims, (scene.density_lo, scene.density_hi),
                   scene.sh_std, scene.sh_dc, scene.seed)
    return dot_octree_build(d, stream, allocator)
