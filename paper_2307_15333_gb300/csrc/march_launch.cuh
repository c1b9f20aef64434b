// march_launch.cuh -- grid shapes and template dispatch of the march kernel for one mode.
#pragma once

#include "march.cuh"

namespace dot {

inline dim3 march_grid(const RaySource &rs) {
    if (rs.kind == DOT_RAYS_CAMERAS) {
        const int ty = (rs.height + 15) / 16;
        return dim3((unsigned)(rs.tiles_x * ty), (unsigned)rs.n_cams);
    }
    return dim3((unsigned)((rs.n_rays + kMarchThreads - 1) / kMarchThreads));
}

// Blocks above which a forward launch uses the occupancy build: two full waves of 4 blocks on
// every SM of the current device (152 SMs on a GB300).
inline int64_t occupancy_blocks() {
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return 2 * 4 * (int64_t)sms;
}

template <typename S, int K, int MODE>
cudaError_t launch_sk(bool exact, const TreeView &tv, const RaySource &rs, const RenderParams &rp,
                      const RenderIO &io, cudaStream_t stream) {
    const dim3 grid = march_grid(rs);
    if (grid.x == 0 || grid.y == 0) return cudaSuccess;
    const bool occ = MODE == kFwd && (int64_t)grid.x * grid.y >= occupancy_blocks();
    if constexpr (MODE == kFwd) {
        if (occ) {
            if (exact)
                march_kernel<S, K, MODE, true, 4><<<grid, kMarchThreads, 0, stream>>>(tv, rs, rp, io);
            else
                march_kernel<S, K, MODE, false, 4><<<grid, kMarchThreads, 0, stream>>>(tv, rs, rp, io);
            return cudaGetLastError();
        }
    }
    if (exact)
        march_kernel<S, K, MODE, true, 1><<<grid, kMarchThreads, 0, stream>>>(tv, rs, rp, io);
    else
        march_kernel<S, K, MODE, false, 1><<<grid, kMarchThreads, 0, stream>>>(tv, rs, rp, io);
    return cudaGetLastError();
}

template <typename S, int MODE>
cudaError_t launch_s(int deg, bool exact, const TreeView &tv, const RaySource &rs,
                     const RenderParams &rp, const RenderIO &io, cudaStream_t stream) {
    if constexpr (MODE == kSignal || MODE == kStats) {
        return launch_sk<S, 1, MODE>(exact, tv, rs, rp, io, stream);
    } else {
        switch (deg) {
            case 0: return launch_sk<S, 1, MODE>(exact, tv, rs, rp, io, stream);
            case 1: return launch_sk<S, 4, MODE>(exact, tv, rs, rp, io, stream);
            case 2: return launch_sk<S, 9, MODE>(exact, tv, rs, rp, io, stream);
            case 3: return launch_sk<S, 16, MODE>(exact, tv, rs, rp, io, stream);
        }
        return cudaErrorInvalidValue;
    }
}

template <int MODE>
cudaError_t launch_march_mode(int storage, int deg, bool exact, const TreeView &tv,
                              const RaySource &rs, const RenderParams &rp, const RenderIO &io,
                              cudaStream_t stream) {
    switch (storage) {
        case DOT_STORAGE_F32: return launch_s<float, MODE>(deg, exact, tv, rs, rp, io, stream);
        case DOT_STORAGE_F16: return launch_s<__half, MODE>(deg, exact, tv, rs, rp, io, stream);
        case DOT_STORAGE_BF16: return launch_s<__nv_bfloat16, MODE>(deg, exact, tv, rs, rp, io, stream);
    }
    return cudaErrorInvalidValue;
}

}  // namespace dot
