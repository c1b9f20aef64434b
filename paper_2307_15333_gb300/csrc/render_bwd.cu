// render_bwd.cu -- backward kernels: recompute the march and scatter leaf gradients.
#include "march_launch.cuh"

namespace dot {
cudaError_t launch_march_bwd(int storage, int deg, bool exact, const TreeView &tv,
                             const RaySource &rs, const RenderParams &rp, const RenderIO &io,
                             cudaStream_t stream) {
    return launch_march_mode<kBwd>(storage, deg, exact, tv, rs, rp, io, stream);
}
}  // namespace dot
