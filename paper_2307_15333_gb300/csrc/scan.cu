// scan.cu -- device-wide exclusive prefix sum of int32 values (three passes: block totals, a
// scan of the totals in one block, then block-local scans offset by the totals).
#include "internal.cuh"

namespace dot {

namespace {
constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int32_t warp_incl_scan(int32_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int32_t o = __shfl_up_sync(0xffffffffu, v, off);
        if (lane >= off) v += o;
    }
    return v;
}

// exclusive scan of one value per thread across the block; returns the block total in *total
__device__ __forceinline__ int32_t block_excl_scan(int32_t v, int32_t *total) {
    __shared__ int32_t s_warp[kScanThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int32_t inc = warp_incl_scan(v);
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int32_t w = lane < kScanThreads / 32 ? s_warp[lane] : 0;
        w = warp_incl_scan(w);
        if (lane < kScanThreads / 32) s_warp[lane] = w;
    }
    __syncthreads();
    const int32_t base = warp ? s_warp[warp - 1] : 0;
    *total = s_warp[kScanThreads / 32 - 1];
    __syncthreads();
    return base + inc - v;
}

__global__ void __launch_bounds__(kScanThreads)
scan_reduce_kernel(const int32_t *__restrict__ in, int64_t n, int32_t *__restrict__ part) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    int32_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        const int64_t idx = base + (int64_t)i * kScanThreads + threadIdx.x;
        if (idx < n) s += in[idx];
    }
    int32_t tot;
    block_excl_scan(s, &tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads)
scan_parts_kernel(int32_t *__restrict__ part, int64_t nb, int32_t *__restrict__ total) {
    int32_t carry = 0;
    for (int64_t b0 = 0; b0 < nb; b0 += kScanThreads) {
        const int64_t b = b0 + threadIdx.x;
        const int32_t v = b < nb ? part[b] : 0;
        int32_t tot;
        const int32_t ex = block_excl_scan(v, &tot);
        if (b < nb) part[b] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void __launch_bounds__(kScanThreads)
scan_down_kernel(const int32_t *__restrict__ in, int64_t n, const int32_t *__restrict__ part,
                 int32_t *__restrict__ out) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int32_t v[kScanItems];
    int32_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        const int64_t idx = base + i;
        v[i] = idx < n ? in[idx] : 0;
        s += v[i];
    }
    int32_t tot;
    int32_t run = block_excl_scan(s, &tot) + part[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        const int64_t idx = base + i;
        if (idx < n) out[idx] = run;
        run += v[i];
    }
}
}  // namespace

size_t scan_scratch_bytes(int64_t n) {
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    return (size_t)((nb + 1) * sizeof(int32_t) + 255) / 256 * 256;
}

cudaError_t scan_exclusive_i32(const int32_t *in, int32_t *out, int64_t n, int32_t *total,
                               void *scratch, cudaStream_t stream) {
    if (n <= 0) return cudaMemsetAsync(total, 0, sizeof(int32_t), stream);
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    int32_t *part = reinterpret_cast<int32_t *>(scratch);
    scan_reduce_kernel<<<(unsigned)nb, kScanThreads, 0, stream>>>(in, n, part);
    scan_parts_kernel<<<1, kScanThreads, 0, stream>>>(part, nb, total);
    scan_down_kernel<<<(unsigned)nb, kScanThreads, 0, stream>>>(in, n, part, out);
    return cudaGetLastError();
}

}  // namespace dot
