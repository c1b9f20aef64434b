// render_fwd.cu -- forward render kernels (Eq. 1-2), every storage type and SH degree.
#include "march_launch.cuh"

namespace dot {
cudaError_t launch_march_fwd_comp(int storage, int deg, bool exact, const TreeView &tv,
                                  const RaySource &rs, const RenderParams &rp, const RenderIO &io,
                                  cudaStream_t stream);

cudaError_t launch_march_fwd(int storage, int deg, bool exact, const TreeView &tv,
                             const RaySource &rs, const RenderParams &rp, const RenderIO &io,
                             cudaStream_t stream) {
    if (tv.rec != nullptr) return launch_march_fwd_comp(storage, deg, exact, tv, rs, rp, io, stream);
    return launch_march_mode<kFwd>(storage, deg, exact, tv, rs, rp, io, stream);
}
}  // namespace dot
