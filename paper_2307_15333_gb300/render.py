"""Host-buffer convenience calls on top of the C ABI (what an application calls)."""
from __future__ import annotations

from typing import Optional

import torch

from . import dot


def render_views(tree: dot.Octree, cams_host: torch.Tensor, width: int, height: int,
                 opts: Optional[dot.dot_render_opts] = None,
                 out_host: Optional[torch.Tensor] = None, stream=None,
                 view_order: bool = True) -> torch.Tensor:
    """Renders every camera of `cams_host` (float32 [n, 18] dot_camera records in host memory,
    ideally pinned) and returns the images in host memory ([n, H, W, 3] float32, pinned when
    `out_host` is not given).  With `view_order` the views are rendered in a nearest-neighbour
    chain (dot_camera_order) so that consecutive views reuse the leaves in L2; the images do not
    change.  The host-to-device copies of the cameras and the order, the render and the
    device-to-host copy of the images are queued on one stream; the call returns after the
    images have arrived."""
    if opts is None:
        opts = dot.render_opts()
    s = stream if stream is not None else torch.cuda.current_stream()
    n = cams_host.shape[0]
    order = torch.from_numpy(dot.dot_camera_order(cams_host.numpy())) if view_order else None
    with torch.cuda.stream(s):
        cams = cams_host.to("cuda", non_blocking=True)
        order_d = order.to("cuda", non_blocking=True) if order is not None else None
        rgb = torch.empty(n * height * width, 3, dtype=torch.float32, device="cuda")
        dot.dot_render_forward(tree, dot.rays_cameras(cams, width, height, order_d), opts, rgb,
                               stream=s)
        if out_host is None:
            out_host = torch.empty(n, height, width, 3, dtype=torch.float32, pin_memory=True)
        out_host.view(-1, 3).copy_(rgb, non_blocking=True)
    s.synchronize()
    return out_host
