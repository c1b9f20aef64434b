// render_fwd_comp.cu -- forward render kernels of compressed trees (16-bit storage; density and
// palette row read from one 32-bit record per leaf), every SH degree.
#include "march_launch.cuh"

namespace dot {

namespace {
template <typename S>
cudaError_t comp_s(int deg, bool exact, const TreeView &tv, const RaySource &rs,
                   const RenderParams &rp, const RenderIO &io, cudaStream_t stream) {
    switch (deg) {
        case 0: return launch_sk<S, 1, kFwd, true>(exact, tv, rs, rp, io, stream);
        case 1: return launch_sk<S, 4, kFwd, true>(exact, tv, rs, rp, io, stream);
        case 2: return launch_sk<S, 9, kFwd, true>(exact, tv, rs, rp, io, stream);
        case 3: return launch_sk<S, 16, kFwd, true>(exact, tv, rs, rp, io, stream);
    }
    return cudaErrorInvalidValue;
}
}  // namespace

cudaError_t launch_march_fwd_comp(int storage, int deg, bool exact, const TreeView &tv,
                                  const RaySource &rs, const RenderParams &rp, const RenderIO &io,
                                  cudaStream_t stream) {
    switch (storage) {
        case DOT_STORAGE_F16: return comp_s<__half>(deg, exact, tv, rs, rp, io, stream);
        case DOT_STORAGE_BF16: return comp_s<__nv_bfloat16>(deg, exact, tv, rs, rp, io, stream);
    }
    return cudaErrorInvalidValue;
}

}  // namespace dot
