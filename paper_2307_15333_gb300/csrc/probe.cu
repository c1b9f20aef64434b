// probe.cu -- the L2 read bandwidth that the two-level roofline of the march kernels divides
// their per-segment bytes by (compulsory bytes at HBM speed against sample bytes at L2 speed).
//
// A grid of whole waves streams one device buffer `passes` times with 16-byte loads that are
// cached in L2 only (ld.global.cg: no L1 allocation, so every pass is served by L2 once the
// buffer fits there) and folds every word into one per-thread value; a thread writes its value
// only if it equals a key no input can produce, so the loads cannot be dropped and nothing is
// written in practice.
#include "internal.cuh"

namespace dot {

namespace {

constexpr int kProbeThreads = 512;

__global__ void __launch_bounds__(kProbeThreads)
l2_read_kernel(const uint4 *__restrict__ buf, int64_t n_vec, int32_t passes,
               unsigned long long *__restrict__ sink) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned acc = 0u;
    for (int32_t p = 0; p < passes; p++) {
        int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        // four independent loads in flight per thread
        for (; i + 3 * stride < n_vec; i += 4 * stride) {
            const uint4 a = __ldcg(buf + i), b = __ldcg(buf + i + stride);
            const uint4 c = __ldcg(buf + i + 2 * stride), d = __ldcg(buf + i + 3 * stride);
            acc ^= (a.x + b.y) ^ (c.z + d.w) ^ (a.w + b.z) ^ (c.y + d.x) ^ (a.y + b.x) ^ (c.w + d.z) ^
                   (a.z + b.w) ^ (c.x + d.y);
        }
        for (; i < n_vec; i += stride) {
            const uint4 a = __ldcg(buf + i);
            acc ^= a.x ^ a.y ^ a.z ^ a.w;
        }
        acc = acc * 0x9E3779B9u + (unsigned)p;
    }
    if (acc == 0xFFFFFFFFu && sink) atomicAdd(sink, 1ull);
}

}  // namespace

cudaError_t launch_l2_read(const void *buf, int64_t bytes, int32_t passes,
                           unsigned long long *sink, cudaStream_t s) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, l2_read_kernel, kProbeThreads, 0);
    const int grid = sms * (per_sm > 0 ? per_sm : 1);
    l2_read_kernel<<<grid, kProbeThreads, 0, s>>>(reinterpret_cast<const uint4 *>(buf), bytes / 16,
                                                  passes, sink);
    return cudaGetLastError();
}

}  // namespace dot
