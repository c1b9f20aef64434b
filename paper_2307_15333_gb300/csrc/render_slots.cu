// render_slots.cu -- one persistent launch rendering many camera requests (mixed resolutions,
// several resident trees) from a device slot table.
//
// Every request is cut into 16x8 pixel tiles (four warps of 8x4 pixels, the tiles of the large
// forward launches); tile t of the launch belongs to the slot whose tile_begin is the largest one
// <= t.  A grid of (SMs x resident blocks) blocks pulls tiles from one device counter until it
// passes total_tiles, then exits: there is no waiting on flags.  Each pixel runs the same march
// as dot_render_forward, so a request's image does not depend on what else shares the launch.
#include "march.cuh"

namespace dot {

namespace {

struct SlotTrees {
    TreeView t[DOT_MAX_SERVE_TREES];
    int32_t n;
};

struct SlotHeader {
    int32_t n_slots;
    int32_t pad_;
    int64_t total_tiles;
};

constexpr int kSlotThreads = 128;

template <typename S, int K, bool EXACT, bool COMP>
__global__ void __launch_bounds__(kSlotThreads, 8)
slots_kernel(SlotTrees trees, const char *__restrict__ table, int32_t max_slots, RenderParams rp,
             unsigned long long *__restrict__ counter, uint32_t *status) {
    __shared__ long long s_tile;
    const SlotHeader *hdr = reinterpret_cast<const SlotHeader *>(table);
    const dot_slot *slots = reinterpret_cast<const dot_slot *>(table + sizeof(SlotHeader));
    const int n = min(hdr->n_slots, max_slots);
    const long long total = hdr->total_tiles;
    RenderIO io{};
    io.status = status;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (n <= 0) return;
    while (true) {
        if (threadIdx.x == 0) s_tile = (long long)atomicAdd(counter, 1ull);
        __syncthreads();
        const long long tile = s_tile;
        __syncthreads();
        if (tile >= total) break;
        // the slot holding this tile: largest s with tile_begin[s] <= tile
        int lo = 0, hi = n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (slots[mid].tile_begin <= tile) lo = mid;
            else hi = mid - 1;
        }
        const dot_slot *sl = slots + lo;
        const int W = sl->camera.width, H = sl->camera.height;
        const int tx_n = (W + 15) / 16, ty_n = (H + 7) / 8;
        const long long local = tile - sl->tile_begin;
        const int tr = sl->tree;
        if (local < 0 || local >= (long long)tx_n * ty_n || tr < 0 || tr >= trees.n) continue;
        const int tx = (int)(local % tx_n), ty = (int)(local / tx_n);
        const int px = tx * 16 + (warp & 1) * 8 + (lane & 7);
        const int py = ty * 8 + (warp >> 1) * 4 + (lane >> 3);
        if (px < W && py < H) {
            float ow[3], dw[3];
            camera_ray(&sl->camera, px, py, ow, dw);
            RayOut out;
            march_ray<S, K, kFwd, EXACT, false, COMP>(trees.t[tr], rp, io, 0, ow, dw, out);
            float *dst = sl->out + ((int64_t)py * W + px) * 3;
#pragma unroll
            for (int ch = 0; ch < 3; ch++) dst[ch] = out.rgb[ch];
        }
    }
}

template <typename S, int K, bool EXACT, bool COMP>
cudaError_t launch_slots_sk(const SlotTrees &trees, const void *table, int32_t max_slots,
                            const RenderParams &rp, unsigned long long *counter, uint32_t *status,
                            int grid, cudaStream_t s) {
    if (grid <= 0) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, slots_kernel<S, K, EXACT, COMP>,
                                                      kSlotThreads, 0);
        grid = sms * (per_sm > 0 ? per_sm : 1);
    }
    slots_kernel<S, K, EXACT, COMP><<<grid, kSlotThreads, 0, s>>>(
        trees, reinterpret_cast<const char *>(table), max_slots, rp, counter, status);
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_slots_s(int deg, bool exact, bool comp, const SlotTrees &trees, const void *table,
                           int32_t max_slots, const RenderParams &rp, unsigned long long *counter,
                           uint32_t *status, int grid, cudaStream_t s) {
#define DOT_SLOTS_CASE(D, KK)                                                                    \
    case D:                                                                                      \
        if (comp)                                                                                \
            return exact ? launch_slots_sk<S, KK, true, true>(trees, table, max_slots, rp, counter, status, grid, s) \
                         : launch_slots_sk<S, KK, false, true>(trees, table, max_slots, rp, counter, status, grid, s); \
        return exact ? launch_slots_sk<S, KK, true, false>(trees, table, max_slots, rp, counter, status, grid, s) \
                     : launch_slots_sk<S, KK, false, false>(trees, table, max_slots, rp, counter, status, grid, s);
    switch (deg) {
        DOT_SLOTS_CASE(0, 1)
        DOT_SLOTS_CASE(1, 4)
        DOT_SLOTS_CASE(2, 9)
        DOT_SLOTS_CASE(3, 16)
    }
#undef DOT_SLOTS_CASE
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_render_slots(int storage, int deg, bool exact, const TreeView *views,
                                int n_trees, const void *table, int32_t max_slots,
                                const RenderParams &rp, unsigned long long *counter,
                                uint32_t *status, int grid, cudaStream_t s) {
    SlotTrees trees{};
    const bool comp = n_trees > 0 && views[0].rec != nullptr;
    for (int i = 0; i < n_trees; i++) trees.t[i] = views[i];
    trees.n = n_trees;
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    switch (storage) {
        case DOT_STORAGE_F32: return launch_slots_s<float>(deg, exact, false, trees, table, max_slots, rp, counter, status, grid, s);
        case DOT_STORAGE_F16: return launch_slots_s<__half>(deg, exact, comp, trees, table, max_slots, rp, counter, status, grid, s);
        case DOT_STORAGE_BF16: return launch_slots_s<__nv_bfloat16>(deg, exact, comp, trees, table, max_slots, rp, counter, status, grid, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace dot
