"""Host-buffer convenience calls on top of the C ABI (what an application calls)."""
from __future__ import annotations

from typing import Optional

import torch

from . import dot


def render_views(tree: dot.Octree, cams_host: torch.Tensor, width: int, height: int,
                 opts: Optional[dot.dot_render_opts] = None,
                 out_host: Optional[torch.Tensor] = None, stream=None,
                 view_order: bool = True, T_host: Optional[torch.Tensor] = None,
                 workspace: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Renders every camera of `cams_host` (float32 [n, 18] dot_camera records in host memory)
    and returns the images in host memory ([n, H, W, 3] float32, pinned when `out_host` is not
    given), through dot_render_views_host: into page-locked host images (the default here) one
    launch writes every image in place; into other host buffers the views are rendered in chunks
    and each finished chunk is copied to the host while the next ones render.  With `view_order`
    the views are rendered in a nearest-neighbour chain (dot_camera_order) so that consecutive
    views reuse the leaves in L2; the images do not change.  Pass a device `workspace` (uint8, at
    least dot_render_views_host_workspace bytes) to reuse one across calls.  The call returns
    after the images have arrived."""
    if opts is None:
        opts = dot.render_opts()
    n = cams_host.shape[0]
    order = dot.dot_camera_order(cams_host.numpy()) if view_order else None
    if out_host is None:
        out_host = torch.empty(n, height, width, 3, dtype=torch.float32, pin_memory=True)
    dot.dot_render_views_host(tree, cams_host, width, height, opts, out_host, T_host=T_host,
                              view_order=order, workspace=workspace, stream=stream)
    return out_host
