// select.cu -- prune / sample marks from the per-leaf signal (Sec. 3.2; Algorithm 1).
//
// Threshold mode is elementwise.  Rank mode selects the k = ceil(f L) smallest (prune) or largest
// (sample) signals with ties broken by ascending leaf id: the k-th key is found by a 4-pass radix
// select over order-preserving 32-bit keys (256-bin histograms, all on the device), then keys
// below it are taken and keys equal to it are taken in id order up to the remaining count (an
// exclusive scan of the equality flags).  Quantile mode takes every key up to and including the
// k-th (no scan).
#include "internal.cuh"
#include "tree.cuh"

namespace dot {

namespace {

struct SelState {
    unsigned prefix;
    unsigned mask;
    long long krem;  // 1-based rank still to find within the keys matching prefix/mask
};

// order-preserving key: smaller key = earlier in the selection order
__device__ __forceinline__ unsigned sel_key(float s, bool largest_first) {
    unsigned u = __float_as_uint(s);
    if ((u & 0x7fffffffu) > 0x7f800000u) return 0xffffffffu;  // NaN: after every number
    if (u == 0x80000000u) u = 0u;                             // -0 is the same value as +0
    const unsigned a = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    return largest_first ? ~a : a;  // a number's key never reaches 0xffffffff
}

__global__ void hist_kernel(const float *__restrict__ sig, int64_t n, bool largest_first,
                            const SelState *__restrict__ st, int shift,
                            unsigned *__restrict__ hist) {
    __shared__ unsigned sh[256];
    sh[threadIdx.x] = 0;
    __syncthreads();
    const unsigned prefix = st->prefix, mask = st->mask;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned k = sel_key(__ldg(sig + i), largest_first);
        if ((k & mask) == prefix) atomicAdd(&sh[(k >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (sh[threadIdx.x]) atomicAdd(&hist[threadIdx.x], sh[threadIdx.x]);
}

// one block of 256 threads: pick the digit holding rank krem, refine the prefix, clear hist
__global__ void pick_kernel(unsigned *__restrict__ hist, SelState *__restrict__ st, int shift) {
    __shared__ long long cum[256];
    const unsigned c = hist[threadIdx.x];
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
    const long long krem = st->krem;
    __syncthreads();
    if (c > 0 && excl < krem && krem <= incl) {
        st->prefix |= (unsigned)threadIdx.x << shift;
        st->mask |= 255u << shift;
        st->krem = krem - excl;
    }
    hist[threadIdx.x] = 0;
}

// ties: every key equal to the selected one is taken too (quantile mode; eq is not written)
__global__ void mark_lt_kernel(const float *__restrict__ sig, int64_t n, bool largest_first,
                               const SelState *__restrict__ st, bool ties,
                               uint8_t *__restrict__ mark, int32_t *__restrict__ eq) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned k = sel_key(__ldg(sig + i), largest_first);
    const unsigned v = st->prefix;
    mark[i] = (k < v || (ties && k == v)) ? 1 : 0;
    if (!ties) eq[i] = k == v ? 1 : 0;
}

__global__ void mark_eq_kernel(const int32_t *__restrict__ eq, const int32_t *__restrict__ rank,
                               int64_t n, const SelState *__restrict__ st,
                               uint8_t *__restrict__ mark) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (eq[i] && (long long)rank[i] < st->krem) mark[i] = 1;
}

__global__ void init_state_kernel(SelState *st, unsigned *hist, long long k) {
    hist[threadIdx.x] = 0;
    if (threadIdx.x == 0) {
        st->prefix = 0u;
        st->mask = 0u;
        st->krem = k;
    }
}

__global__ void threshold_kernel(const float *__restrict__ sig, int64_t n, bool prune, float thr,
                                 uint8_t *__restrict__ mark) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float s = __ldg(sig + i);
    mark[i] = prune ? (s <= thr) : (s > thr);
}

#define SEL_CK(x)                              \
    do {                                       \
        cudaError_t e_ = (x);                  \
        if (e_ != cudaSuccess) return e_;      \
    } while (0)

cudaError_t rank_select(const float *sig, int64_t n, int64_t k, bool largest_first, bool ties,
                        uint8_t *mark, cudaStream_t s) {
    if (k <= 0) return cudaMemsetAsync(mark, 0, (size_t)n, s);
    if (k >= n) return cudaMemsetAsync(mark, 1, (size_t)n, s);
    // scratch: histogram, state, equality flags, their ranks, scan partials
    const size_t off_state = 256 * sizeof(unsigned);           // 1024: after the histogram
    const size_t off_eq = off_state + 256;                      // state occupies 16 bytes
    const size_t off_rank = off_eq + ((size_t)n * 4 + 255) / 256 * 256;
    const size_t off_scan = off_rank + ((size_t)n * 4 + 255) / 256 * 256;
    const size_t off_total = off_scan + scan_scratch_bytes(n);
    const size_t bytes = off_total + 256;
    char *scratch = nullptr;
    SEL_CK(cudaMallocAsync((void **)&scratch, bytes, s));
    unsigned *hist = (unsigned *)scratch;
    SelState *st = (SelState *)(scratch + off_state);
    int32_t *eq = (int32_t *)(scratch + off_eq);
    int32_t *rank = (int32_t *)(scratch + off_rank);
    init_state_kernel<<<1, 256, 0, s>>>(st, hist, (long long)k);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (n + 255) / 256;
    const unsigned grid = (unsigned)(want < (int64_t)sms * 8 ? want : (int64_t)sms * 8);
    for (int shift = 24; shift >= 0; shift -= 8) {
        hist_kernel<<<grid, 256, 0, s>>>(sig, n, largest_first, st, shift, hist);
        pick_kernel<<<1, 256, 0, s>>>(hist, st, shift);
    }
    const unsigned blocks = (unsigned)((n + 255) / 256);
    mark_lt_kernel<<<blocks, 256, 0, s>>>(sig, n, largest_first, st, ties, mark, eq);
    cudaError_t err = cudaGetLastError();
    if (err == cudaSuccess && !ties)
        err = scan_exclusive_i32(eq, rank, n, (int32_t *)(scratch + off_total), scratch + off_scan, s);
    if (err == cudaSuccess && !ties) {
        mark_eq_kernel<<<blocks, 256, 0, s>>>(eq, rank, n, st, mark);
        err = cudaGetLastError();
    }
    // the scratch goes back on every path once it is allocated; the first error is reported
    const cudaError_t ef = cudaFreeAsync(scratch, s);
    return err != cudaSuccess ? err : ef;
}

cudaError_t one_mask(const float *sig, int64_t n, int mode, double value, bool prune,
                     uint8_t *mark, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    if (mode == DOT_SELECT_NONE) return cudaMemsetAsync(mark, 0, (size_t)n, s);
    if (mode == DOT_SELECT_THRESHOLD) {
        threshold_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(sig, n, prune, (float)value, mark);
        return cudaGetLastError();
    }
    double kk = ceil(value * (double)n);
    int64_t k = kk < 0 ? 0 : (kk > (double)n ? n : (int64_t)kk);
    return rank_select(sig, n, k, !prune, mode == DOT_SELECT_QUANTILE, mark, s);
}

}  // namespace

cudaError_t select_masks(const float *signal, int64_t n, int prune_mode, double prune_value,
                         int sample_mode, double sample_value, uint8_t *prune_mark,
                         uint8_t *sample_mark, cudaStream_t s) {
    if (prune_mark) SEL_CK(one_mask(signal, n, prune_mode, prune_value, true, prune_mark, s));
    if (sample_mark) SEL_CK(one_mask(signal, n, sample_mode, sample_value, false, sample_mark, s));
    return cudaSuccess;
}

}  // namespace dot
