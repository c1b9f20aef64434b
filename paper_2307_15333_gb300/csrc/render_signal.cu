// render_signal.cu -- density-only marches: the training signal of Sec. 3.1 and march counts.
#include "march_launch.cuh"

namespace dot {
cudaError_t launch_march_signal(int storage, bool exact, const TreeView &tv, const RaySource &rs,
                                const RenderParams &rp, const RenderIO &io, cudaStream_t stream) {
    return launch_march_mode<kSignal>(storage, 0, exact, tv, rs, rp, io, stream);
}
cudaError_t launch_march_stats(int storage, bool exact, const TreeView &tv, const RaySource &rs,
                               const RenderParams &rp, const RenderIO &io, cudaStream_t stream) {
    return launch_march_mode<kStats>(storage, 0, exact, tv, rs, rp, io, stream);
}

// DOT_SIGNAL_SIGMA: S_v = max(sigma_v, 0), no march
template <typename S>
__global__ void sigma_signal_kernel(const S *__restrict__ sigma, int64_t n, float *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = fmaxf(Storage<S>::load(sigma + i), 0.f);
}

cudaError_t launch_sigma_signal(int storage, const void *sigma, int64_t n, float *signal,
                                cudaStream_t stream) {
    if (n == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    switch (storage) {
        case DOT_STORAGE_F32: sigma_signal_kernel<<<blocks, 256, 0, stream>>>((const float *)sigma, n, signal); break;
        case DOT_STORAGE_F16: sigma_signal_kernel<<<blocks, 256, 0, stream>>>((const __half *)sigma, n, signal); break;
        default: sigma_signal_kernel<<<blocks, 256, 0, stream>>>((const __nv_bfloat16 *)sigma, n, signal); break;
    }
    return cudaGetLastError();
}
}  // namespace dot
