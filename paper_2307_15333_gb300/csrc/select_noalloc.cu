// select_noalloc.cu -- dot_select_masks_noalloc: the prune / sample selection computed without
// allocating device memory, for callers that cannot call cudaMalloc (see include/dot.h).
//
// The working memory lives in one file-scope __device__ array of fixed size.  It holds the
// radix-select histogram and state and one equal-key count per tile of 4096 leaves, so trees of
// up to 2^26 leaves fit in about 66 KB.  Instead of flag and rank arrays as long as the tree, the
// ranks of the keys equal to the selected key are rebuilt tile by tile: each tile counts its
// equal keys, the counts are scanned in place, and each tile re-derives its local ranks.
#include <mutex>

#include "internal.cuh"

namespace dot {

namespace {

constexpr int64_t kNoAllocMaxLeaves = (int64_t)1 << 26;
constexpr int kTileThreads = 256;
constexpr int kTileItems = 16;
constexpr int kTile = kTileThreads * kTileItems;                  // 4096 leaves per tile
constexpr int kMaxTiles = (int)(kNoAllocMaxLeaves / kTile);       // 16384

struct NaState {
    unsigned prefix;
    unsigned mask;
    long long krem;  // 1-based rank still to find among keys matching prefix / mask
};

struct NaScratch {
    unsigned hist[256];
    NaState st;
    int32_t pad[60];
    int32_t tile_count[kMaxTiles];
};

// The scratch every call of dot_select_masks_noalloc on this device shares.
static __device__ __align__(256) NaScratch g_select_scratch;

__device__ __forceinline__ unsigned na_key(float s, bool largest_first) {
    unsigned u = __float_as_uint(s);
    if ((u & 0x7fffffffu) > 0x7f800000u) return 0xffffffffu;  // NaN: after every number
    if (u == 0x80000000u) u = 0u;                             // -0 is the same value as +0
    const unsigned a = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    return largest_first ? ~a : a;  // a number's key never reaches 0xffffffff
}

__global__ void na_init_kernel(NaScratch *sc, long long k) {
    sc->hist[threadIdx.x] = 0u;
    if (threadIdx.x == 0) {
        sc->st.prefix = 0u;
        sc->st.mask = 0u;
        sc->st.krem = k;
    }
}

__global__ void na_hist_kernel(const float *__restrict__ sig, int64_t n, bool largest_first,
                               NaScratch *sc, int shift) {
    __shared__ unsigned sh[256];
    sh[threadIdx.x] = 0u;
    __syncthreads();
    const unsigned prefix = sc->st.prefix, mask = sc->st.mask;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned k = na_key(__ldg(sig + i), largest_first);
        if ((k & mask) == prefix) atomicAdd(&sh[(k >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (sh[threadIdx.x]) atomicAdd(&sc->hist[threadIdx.x], sh[threadIdx.x]);
}

__global__ void na_pick_kernel(NaScratch *sc, int shift) {
    __shared__ long long cum[256];
    const unsigned c = sc->hist[threadIdx.x];
    cum[threadIdx.x] = c;
    __syncthreads();
    for (int off = 1; off < 256; off <<= 1) {
        const long long v = threadIdx.x >= (unsigned)off ? cum[threadIdx.x - off] : 0;
        __syncthreads();
        cum[threadIdx.x] += v;
        __syncthreads();
    }
    const long long incl = cum[threadIdx.x];
    const long long excl = incl - c;
    const long long krem = sc->st.krem;
    __syncthreads();
    if (c > 0 && excl < krem && krem <= incl) {
        sc->st.prefix |= (unsigned)threadIdx.x << shift;
        sc->st.mask |= 255u << shift;
        sc->st.krem = krem - excl;
    }
    sc->hist[threadIdx.x] = 0u;
}

// exclusive scan of one int per thread over a 256-thread block
__device__ __forceinline__ int32_t na_block_scan(int32_t v, int32_t *total) {
    __shared__ int32_t warp_sum[kTileThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t inc = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int32_t o = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += o;
    }
    if (lane == 31) warp_sum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int32_t w = lane < kTileThreads / 32 ? warp_sum[lane] : 0;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int32_t o = __shfl_up_sync(0xffffffffu, w, off);
            if (lane >= off) w += o;
        }
        if (lane < kTileThreads / 32) warp_sum[lane] = w;
    }
    __syncthreads();
    const int32_t base = warp ? warp_sum[warp - 1] : 0;
    *total = warp_sum[kTileThreads / 32 - 1];
    __syncthreads();
    return base + inc - v;
}

// marks keys below the selected key (and equal to it with ties, quantile mode); counts the
// tile's keys equal to it
__global__ void __launch_bounds__(kTileThreads)
na_mark_lt_kernel(const float *__restrict__ sig, int64_t n, bool largest_first, bool ties,
                  NaScratch *sc, uint8_t *__restrict__ mark) {
    const unsigned v = sc->st.prefix;
    const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kTileItems;
    int32_t eq = 0;
#pragma unroll
    for (int i = 0; i < kTileItems; i++) {
        const int64_t idx = base + i;
        if (idx < n) {
            const unsigned k = na_key(__ldg(sig + idx), largest_first);
            mark[idx] = (k < v || (ties && k == v)) ? 1 : 0;
            eq += k == v;
        }
    }
    int32_t tot;
    na_block_scan(eq, &tot);
    if (threadIdx.x == 0) sc->tile_count[blockIdx.x] = tot;
}

// in-place exclusive scan of the tile counts (one block)
__global__ void __launch_bounds__(kTileThreads) na_scan_tiles_kernel(NaScratch *sc, int n_tiles) {
    int32_t carry = 0;
    for (int b0 = 0; b0 < n_tiles; b0 += kTileThreads) {
        const int b = b0 + threadIdx.x;
        const int32_t v = b < n_tiles ? sc->tile_count[b] : 0;
        int32_t tot;
        const int32_t ex = na_block_scan(v, &tot);
        if (b < n_tiles) sc->tile_count[b] = carry + ex;
        carry += tot;
    }
}

// takes the keys equal to the selected key in leaf-id order, up to the remaining count
__global__ void __launch_bounds__(kTileThreads)
na_mark_eq_kernel(const float *__restrict__ sig, int64_t n, bool largest_first, NaScratch *sc,
                  uint8_t *__restrict__ mark) {
    const unsigned v = sc->st.prefix;
    const long long krem = sc->st.krem;
    const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kTileItems;
    uint32_t eqbits = 0;
    int32_t eq = 0;
#pragma unroll
    for (int i = 0; i < kTileItems; i++) {
        const int64_t idx = base + i;
        if (idx < n && na_key(__ldg(sig + idx), largest_first) == v) {
            eqbits |= 1u << i;
            eq++;
        }
    }
    int32_t tot;
    long long r = (long long)na_block_scan(eq, &tot) + sc->tile_count[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kTileItems; i++) {
        if (eqbits & (1u << i)) {
            if (r < krem) mark[base + i] = 1;
            r++;
        }
    }
}

__global__ void na_threshold_kernel(const float *__restrict__ sig, int64_t n, bool prune, float thr,
                                    uint8_t *__restrict__ mark) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float s = __ldg(sig + i);
    mark[i] = prune ? (s <= thr) : (s > thr);
}

__global__ void na_fill_kernel(uint8_t *__restrict__ mark, int64_t n, uint8_t value) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) mark[i] = value;
}

// Device address of the scratch.  Outside stream capture it is looked up on every call with the
// calling device current, so a context destroyed and created again (cudaDeviceReset) never
// leaves a stale address behind; the last address seen on each device is kept for calls made
// while their stream is being captured, where the lookup is not repeated.
std::mutex g_addr_mutex;
NaScratch *g_addr[64] = {nullptr};

cudaError_t scratch_address(cudaStream_t s, NaScratch **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    if (cap == cudaStreamCaptureStatusNone) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_select_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = reinterpret_cast<NaScratch *>(p);
    } else if (!g_addr[dev]) {
        return cudaErrorStreamCaptureUnsupported;  // no call on this device before the capture
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

cudaError_t na_one_mask(NaScratch *sc, const float *sig, int64_t n, int mode, double value,
                        bool prune, uint8_t *mark, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    if (mode == DOT_SELECT_NONE) {
        na_fill_kernel<<<blocks, 256, 0, s>>>(mark, n, 0);
        return cudaGetLastError();
    }
    if (mode == DOT_SELECT_THRESHOLD) {
        na_threshold_kernel<<<blocks, 256, 0, s>>>(sig, n, prune, (float)value, mark);
        return cudaGetLastError();
    }
    const double kk = ceil(value * (double)n);
    const int64_t k = kk < 0 ? 0 : (kk > (double)n ? n : (int64_t)kk);
    if (k <= 0 || k >= n) {
        na_fill_kernel<<<blocks, 256, 0, s>>>(mark, n, k <= 0 ? 0 : 1);
        return cudaGetLastError();
    }
    const bool largest_first = !prune;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (n + 255) / 256;
    const unsigned grid = (unsigned)(want < (int64_t)sms * 8 ? want : (int64_t)sms * 8);
    na_init_kernel<<<1, 256, 0, s>>>(sc, (long long)k);
    for (int shift = 24; shift >= 0; shift -= 8) {
        na_hist_kernel<<<grid, 256, 0, s>>>(sig, n, largest_first, sc, shift);
        na_pick_kernel<<<1, 256, 0, s>>>(sc, shift);
    }
    const int n_tiles = (int)((n + kTile - 1) / kTile);
    const bool ties = mode == DOT_SELECT_QUANTILE;
    na_mark_lt_kernel<<<n_tiles, kTileThreads, 0, s>>>(sig, n, largest_first, ties, sc, mark);
    if (!ties) {
        na_scan_tiles_kernel<<<1, kTileThreads, 0, s>>>(sc, n_tiles);
        na_mark_eq_kernel<<<n_tiles, kTileThreads, 0, s>>>(sig, n, largest_first, sc, mark);
    }
    return cudaGetLastError();
}

}  // namespace

int64_t select_noalloc_max_leaves() { return kNoAllocMaxLeaves; }

cudaError_t select_masks_noalloc(const float *signal, int64_t n, int prune_mode,
                                 double prune_value, int sample_mode, double sample_value,
                                 uint8_t *prune_mark, uint8_t *sample_mark, cudaStream_t s) {
    NaScratch *sc = nullptr;
    cudaError_t e = scratch_address(s, &sc);
    if (e != cudaSuccess) return e;
    e = na_one_mask(sc, signal, n, prune_mode, prune_value, true, prune_mark, s);
    if (e != cudaSuccess) return e;
    return na_one_mask(sc, signal, n, sample_mode, sample_value, false, sample_mark, s);
}

}  // namespace dot
