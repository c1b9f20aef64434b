// render_fwdbwd.cu -- the fused training pass: forward (Eq. 1-2), MSE gradient and backward of
// each ray in one kernel, the backward scattering from the ray's recorded occupied segments.
#include "march_launch.cuh"

namespace dot {
cudaError_t launch_march_fwdbwd(int storage, int deg, bool exact, const TreeView &tv,
                                const RaySource &rs, const RenderParams &rp, const RenderIO &io,
                                cudaStream_t stream) {
    return launch_march_mode<kFwdBwd>(storage, deg, exact, tv, rs, rp, io, stream);
}
}  // namespace dot
