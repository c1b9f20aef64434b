// march_launch.cuh -- grid shapes and template dispatch of the march kernel for one mode.
#pragma once

#include "march.cuh"

// Build-time launch shapes (measured on a GB300 on the 64 M-ray workloads; -D to override):
// threads per block of large forward launches, and blocks per SM of large backward launches.
#ifndef DOT_FWD_NT
#define DOT_FWD_NT 128
#endif
#ifndef DOT_BWD_MINB
#define DOT_BWD_MINB 6
#endif

namespace dot {

// threads per block of large forward launches, and the blocks per SM they are built for (8 of
// 128 threads: 9.82 ms on the 800^2 workload against 10.10 / 10.65 ms for 7 / 6)
#ifndef DOT_FWD_MINB
#define DOT_FWD_MINB (1024 / DOT_FWD_NT)
#endif
constexpr int kFwdThreads = DOT_FWD_NT;
constexpr int kFwdMinBlocks = DOT_FWD_MINB;

template <int NT>
inline dim3 march_grid(const RaySource &rs) {
    if (rs.kind == DOT_RAYS_CAMERAS) {
        const int tx = (rs.width + CamTile<NT>::kW - 1) / CamTile<NT>::kW;
        const int ty = (rs.height + CamTile<NT>::kH - 1) / CamTile<NT>::kH;
        return dim3((unsigned)(tx * ty), (unsigned)rs.n_cams);
    }
    return dim3((unsigned)((rs.n_rays + NT - 1) / NT));
}

// Forward launches of at least two full waves of the occupancy build on every SM of the current
// device (152 SMs on a GB300) use that build.
inline int64_t occupancy_threads() {
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return 2 * 1024 * (int64_t)sms;
}

template <typename S, int K, int MODE, int MINB, int NT, bool DEFER, bool COMP = false>
cudaError_t launch_nt(bool exact, const TreeView &tv, const RaySource &rs0, const RenderParams &rp,
                      const RenderIO &io, cudaStream_t stream) {
    RaySource rs = rs0;
    rs.tiles_x = (rs.width + CamTile<NT>::kW - 1) / CamTile<NT>::kW;
    const dim3 grid = march_grid<NT>(rs);
    if (grid.x == 0 || grid.y == 0) return cudaSuccess;
    if (exact)
        march_kernel<S, K, MODE, true, MINB, NT, DEFER, COMP><<<grid, NT, 0, stream>>>(tv, rs, rp, io);
    else
        march_kernel<S, K, MODE, false, MINB, NT, DEFER, COMP><<<grid, NT, 0, stream>>>(tv, rs, rp, io);
    return cudaGetLastError();
}

// COMP: forward renders of a compressed tree (density and palette row from the leaf records)
template <typename S, int K, int MODE, bool COMP = false>
cudaError_t launch_sk(bool exact, const TreeView &tv, const RaySource &rs, const RenderParams &rp,
                      const RenderIO &io, cudaStream_t stream) {
    if (rs.n_rays <= 0) return cudaSuccess;
    if constexpr (MODE == kFwd) {
        if (rs.n_rays >= occupancy_threads())
            return launch_nt<S, K, MODE, kFwdMinBlocks, kFwdThreads, false, COMP>(exact, tv, rs, rp, io, stream);
    }
    // large backward launches: 128-thread blocks built for 6 per SM (80 registers, 24 warps)
    if constexpr ((MODE == kBwd || MODE == kFwdBwd) && DOT_BWD_MINB > 0) {
        if (rs.n_rays >= occupancy_threads())
            return launch_nt<S, K, MODE, DOT_BWD_MINB, 128, false, COMP>(exact, tv, rs, rp, io, stream);
    }
    constexpr bool defer = MODE == kFwd || MODE == kBwd || MODE == kFwdBwd;
    return launch_nt<S, K, MODE, 1, kMarchThreads, defer, COMP>(exact, tv, rs, rp, io, stream);
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
