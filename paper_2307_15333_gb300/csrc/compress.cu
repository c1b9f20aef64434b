// compress.cu -- compressed models (Sec. 4.1): every leaf's SH coefficient row is replaced by one
// of 2^bits palette rows found by median cut (Heckbert 1982) over the leaves' coefficient vectors,
// and the leaf keeps a 16-bit palette index next to its 16-bit density in one 32-bit record, so a
// rendered segment reads 4 bytes per leaf plus a palette row that stays resident in L2
// (2^16 rows x 96 bytes = 6.3 MB at SH degree 3).
//
// Median cut rules: each of the bits rounds splits every box of two or more vectors at the median
// of its longest axis (largest max - min, computed in double; ties to the lowest axis), the
// members ordered by (value on that axis, leaf id), floor(m/2) of them to child 2b and the rest
// to child 2b + 1 (a box of fewer than two keeps its members in child 2b); a palette row is the
// mean of its box (zeros if empty), rounded to the storage type.
//
// On the GPU every leaf carries its box number, and a permutation of the leaves keeps every box's
// members contiguous (split stably after each round).  A round:
//   1. per box and axis, the min and max of the members (order-preserving 32-bit keys, atomics
//      aggregated over the lanes of a warp that share a box, and in the first rounds, with few
//      boxes, over a block in shared memory), and the member count;
//   2. per box, the longest axis;
//   3. per box, the member of rank floor(m/2) in (value, id) order: a radix select over the
//      64-bit keys (value key << 32 | leaf id), unique per leaf, in 8 histogram passes of 8 bits;
//   4. every leaf moves to child 2b, or 2b + 1 if its key is at or above that member's.
// The palette is then the per-box mean of FP64 sums.
#include <algorithm>
#include <type_traits>

#include "internal.cuh"
#include "tree.cuh"

namespace dot {

namespace {

constexpr int kMcThreads = 256;

// order-preserving key of a float (a smaller float has a smaller key)
__device__ __forceinline__ unsigned mc_key(float f) {
    const unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float mc_val(unsigned k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

template <typename S>
__device__ __forceinline__ float mc_coef(const S *rows, int64_t v, int stride, int d) {
    return Storage<S>::to_f32(rows[v * stride + d]);
}

struct McBox {
    int32_t count;
    int32_t axis;              // -1: fewer than two members, not split
    unsigned long long prefix; // radix select: key bits fixed so far
    unsigned long long mask;
    long long krem;            // 1-based rank still to find among keys matching prefix / mask
};

__global__ void mc_clear_kernel(unsigned *lo, unsigned *hi, McBox *box, int64_t n_boxes, int dim) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_boxes * dim) {
        lo[i] = 0xffffffffu;
        hi[i] = 0u;
    }
    if (i < n_boxes) box[i].count = 0;
}

// min / max per (box, axis) and the member counts; lanes of a warp with the same box combine
// their values before the atomic
template <typename S>
__global__ void __launch_bounds__(kMcThreads)
mc_minmax_kernel(const S *__restrict__ rows, int stride, int dim, int64_t L,
                 const int32_t *__restrict__ box_of, const int32_t *__restrict__ perm, unsigned *lo,
                 unsigned *hi, McBox *box) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool ok = i < L;
    const int64_t v = ok ? perm[i] : 0;
    const int b = ok ? box_of[v] : -1;
    const unsigned grp = __match_any_sync(0xffffffffu, b);
    const bool leader = (threadIdx.x & 31) == (__ffs(grp) - 1);
    if (ok && leader) atomicAdd(&box[b].count, __popc(grp));
    for (int d = 0; d < dim; d++) {
        const unsigned k = ok ? mc_key(mc_coef(rows, v, stride, d)) : 0u;
        const unsigned kmin = __reduce_min_sync(grp, k), kmax = __reduce_max_sync(grp, k);
        if (ok && leader) {
            atomicMin(lo + (int64_t)b * dim + d, kmin);
            atomicMax(hi + (int64_t)b * dim + d, kmax);
        }
    }
}

// The same for rounds of at most kMcSharedBoxes boxes, where every box has tens of thousands of
// members and the atomics above would queue on a few addresses: a resident grid walks the leaves,
// each block keeps its min / max per (box, axis) and its member counts in shared memory (only its
// own lanes contend there, after the warp's aggregation), then adds them to the global ones with
// one atomic per (box, axis).  Min and max are exact in any order, so the result is the same.
constexpr int kMcSharedBoxes = 64;
constexpr int kMcMaxDim = 48;  // 3 x 16 coefficients at SH degree 3
template <typename S>
__global__ void __launch_bounds__(kMcThreads)
mc_minmax_shared_kernel(const S *__restrict__ rows, int stride, int dim, int64_t L,
                        const int32_t *__restrict__ box_of, const int32_t *__restrict__ perm,
                        unsigned *lo, unsigned *hi, McBox *box, int nb) {
    __shared__ unsigned s_lo[kMcSharedBoxes * kMcMaxDim], s_hi[kMcSharedBoxes * kMcMaxDim];
    __shared__ int s_cnt[kMcSharedBoxes];
    const int n = nb * dim;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        s_lo[i] = 0xffffffffu;
        s_hi[i] = 0u;
    }
    for (int i = threadIdx.x; i < nb; i += blockDim.x) s_cnt[i] = 0;
    __syncthreads();
    for (int64_t b0 = (int64_t)blockIdx.x * blockDim.x; b0 < L; b0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = b0 + threadIdx.x;
        const bool ok = i < L;
        const int64_t v = ok ? perm[i] : 0;
        const int b = ok ? box_of[v] : -1;
        const unsigned grp = __match_any_sync(0xffffffffu, b);
        const bool leader = (threadIdx.x & 31) == (__ffs(grp) - 1);
        if (ok && leader) atomicAdd(&s_cnt[b], __popc(grp));
        for (int d = 0; d < dim; d++) {
            const unsigned k = ok ? mc_key(mc_coef(rows, v, stride, d)) : 0u;
            const unsigned kmin = __reduce_min_sync(grp, k), kmax = __reduce_max_sync(grp, k);
            if (ok && leader) {
                atomicMin(&s_lo[b * dim + d], kmin);
                atomicMax(&s_hi[b * dim + d], kmax);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        if (s_lo[i] != 0xffffffffu) atomicMin(lo + i, s_lo[i]);
        if (s_hi[i] != 0u) atomicMax(hi + i, s_hi[i]);
    }
    for (int i = threadIdx.x; i < nb; i += blockDim.x)
        if (s_cnt[i]) atomicAdd(&box[i].count, s_cnt[i]);
}

// longest axis of every box; the radix select starts at rank floor(m/2) + 1 (1-based)
__global__ void mc_axis_kernel(const unsigned *lo, const unsigned *hi, McBox *box, int64_t n_boxes,
                               int dim) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n_boxes) return;
    McBox &x = box[b];
    x.prefix = 0ull;
    x.mask = 0ull;
    if (x.count < 2) {
        x.axis = -1;
        return;
    }
    int axis = 0;
    double best = -1.0;
    for (int d = 0; d < dim; d++) {
        const double range = (double)mc_val(hi[b * dim + d]) - (double)mc_val(lo[b * dim + d]);
        if (range > best) {
            best = range;
            axis = d;
        }
    }
    x.axis = axis;
    x.krem = x.count / 2 + 1;
}

template <typename S>
__device__ __forceinline__ unsigned long long mc_select_key(const S *rows, int stride, int64_t v,
                                                            int axis) {
    return ((unsigned long long)mc_key(mc_coef(rows, v, stride, axis)) << 32) | (unsigned long long)v;
}

// one radix-select pass: per box, the histogram of the digit at `shift` of the keys that match the
// box's prefix so far
template <typename S>
__global__ void __launch_bounds__(kMcThreads)
mc_hist_kernel(const S *__restrict__ rows, int stride, int64_t L, const int32_t *__restrict__ box_of,
               const McBox *__restrict__ box, int shift, unsigned *hist) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= L) return;
    const int b = box_of[v];
    const McBox x = box[b];
    if (x.axis < 0) return;
    const unsigned long long k = mc_select_key(rows, stride, v, x.axis);
    if ((k & x.mask) != x.prefix) return;
    atomicAdd(hist + (int64_t)b * 256 + ((k >> shift) & 255u), 1u);
}

// one warp per box: the digit holding rank krem; the histogram is cleared for the next pass
__global__ void mc_pick_kernel(unsigned *hist, McBox *box, int64_t n_boxes, int shift) {
    const int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (b >= n_boxes) return;
    McBox &x = box[b];
    unsigned *h = hist + b * 256;
    if (x.axis < 0) return;  // never histogrammed
    unsigned c[8];
    long long sum = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) {
        c[i] = h[lane * 8 + i];
        sum += c[i];
    }
    long long incl = sum;  // inclusive scan of the lanes' sums
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const long long o = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += o;
    }
    const long long krem = x.krem;
    long long base = incl - sum;
    int digit = -1;
    long long below = 0;
    if (base < krem && krem <= incl) {
        for (int i = 0; i < 8; i++) {
            if (base + c[i] >= krem) {
                digit = lane * 8 + i;
                below = base;
                break;
            }
            base += c[i];
        }
    }
    const unsigned found = __ballot_sync(0xffffffffu, digit >= 0);
    const int src = __ffs(found) - 1;
    const int d = __shfl_sync(0xffffffffu, digit, src < 0 ? 0 : src);
    const long long bl = __shfl_sync(0xffffffffu, below, src < 0 ? 0 : src);
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 8; i++) h[lane * 8 + i] = 0u;
    if (lane == 0 && src >= 0) {
        x.prefix |= (unsigned long long)d << shift;
        x.mask |= 255ull << shift;
        x.krem = krem - bl;
    }
}

// split: below the selected member's key -> child 2b, at or above -> child 2b + 1
template <typename S>
__global__ void mc_assign_kernel(const S *__restrict__ rows, int stride, int64_t L,
                                 int32_t *box_of, const McBox *__restrict__ box) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= L) return;
    const int b = box_of[v];
    const McBox x = box[b];
    int child = 2 * b;
    if (x.axis >= 0 && mc_select_key(rows, stride, v, x.axis) >= x.prefix) child += 1;
    box_of[v] = child;
}

__global__ void mc_init_kernel(int32_t *box_of, int32_t *perm, int64_t L) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < L) {
        box_of[v] = 0;
        perm[v] = (int32_t)v;
    }
}

// The members of every box are kept contiguous in perm (box b at [start[b], start[b] + m_b)), so
// that the min / max pass meets each box's members together and a warp's lanes mostly share one
// box.  After a round's assignment each segment is split, stably, into its child 2b (the first
// lower(m_b) entries) and 2b + 1; up[i] flags the entries that moved to the upper child and its
// exclusive scan ranks them within their segment.
__device__ __forceinline__ int64_t mc_lower(const McBox &x) {
    return x.count < 2 ? x.count : x.count / 2;
}
__global__ void mc_flag_kernel(const int32_t *__restrict__ perm, const int32_t *__restrict__ box_of,
                               int64_t L, int32_t *__restrict__ up) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < L) up[i] = box_of[perm[i]] & 1;
}
__global__ void mc_partition_kernel(const int32_t *__restrict__ perm, const int32_t *__restrict__ box_of,
                                    const int32_t *__restrict__ up_before,
                                    const int32_t *__restrict__ start, const McBox *__restrict__ box,
                                    int64_t L, int32_t *__restrict__ perm_next) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= L) return;
    const int32_t v = perm[i];
    const int c = box_of[v];
    const int b = c >> 1;
    const int64_t s0 = start[b];
    const int64_t ups = up_before[i] - up_before[s0];  // entries of the segment before i that went up
    const int64_t pos = (c & 1) ? s0 + mc_lower(box[b]) + ups : s0 + (i - s0) - ups;
    if (pos >= 0 && pos < L) perm_next[pos] = v;
}
__global__ void mc_starts_kernel(const int32_t *__restrict__ start, const McBox *__restrict__ box,
                                 int64_t n_boxes, int32_t *__restrict__ start_next) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n_boxes) return;
    start_next[2 * b] = start[b];
    start_next[2 * b + 1] = (int32_t)(start[b] + mc_lower(box[b]));
}

// FP64 sums of every final box's members, and their counts
template <typename S>
__global__ void __launch_bounds__(kMcThreads)
mc_sum_kernel(const S *__restrict__ rows, int stride, int dim, int64_t L,
              const int32_t *__restrict__ box_of, double *sum, int32_t *count) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= L) return;
    const int b = box_of[v];
    atomicAdd(count + b, 1);
    for (int d = 0; d < dim; d++)
        atomicAdd(sum + (int64_t)b * dim + d, (double)mc_coef(rows, v, stride, d));
}

template <typename S>
__global__ void mc_palette_kernel(const double *sum, const int32_t *count, int64_t P, int dim,
                                  int stride, S *palette) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P * stride) return;
    const int64_t b = i / stride;
    const int d = (int)(i - b * stride);
    double m = 0.0;
    if (d < dim && count[b] > 0) m = sum[b * dim + d] / (double)count[b];
    if constexpr (std::is_same<S, __half>::value) palette[i] = __double2half(m);
    else palette[i] = __double2bfloat16(m);
}

template <typename S>
__global__ void mc_record_kernel(const S *sigma, const int32_t *box_of, int64_t L, uint32_t *rec) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= L) return;
    unsigned short bits;
    if constexpr (std::is_same<S, __half>::value) bits = __half_as_ushort(sigma[v]);
    else bits = __bfloat16_as_ushort(sigma[v]);
    rec[v] = (uint32_t)bits | ((uint32_t)box_of[v] << 16);
}

#define MC_CK(x)                             \
    do {                                     \
        cudaError_t e_ = (x);                \
        if (e_ != cudaSuccess) return e_;    \
    } while (0)

inline unsigned blocks_of(int64_t n, int t = kMcThreads) { return (unsigned)((n + t - 1) / t); }

template <typename S>
cudaError_t median_cut(const S *rows, const S *sigma, int64_t L, int dim, int stride, int bits,
                       S *palette, uint32_t *rec, char *scratch, cudaStream_t s) {
    const int64_t P = int64_t(1) << bits, half = P / 2;
    // scratch layout (256-byte aligned pieces)
    auto up = [](size_t x) { return (x + 255) / 256 * 256; };
    int32_t *box_of = reinterpret_cast<int32_t *>(scratch);
    size_t off = up((size_t)L * 4);
    unsigned *lo = reinterpret_cast<unsigned *>(scratch + off);
    off += up((size_t)half * dim * 4);
    unsigned *hi = reinterpret_cast<unsigned *>(scratch + off);
    off += up((size_t)half * dim * 4);
    McBox *box = reinterpret_cast<McBox *>(scratch + off);
    off += up((size_t)half * sizeof(McBox));
    unsigned *hist = reinterpret_cast<unsigned *>(scratch + off);
    off += up((size_t)half * 256 * 4);
    double *sum = reinterpret_cast<double *>(scratch + off);
    off += up((size_t)P * dim * 8);
    int32_t *count = reinterpret_cast<int32_t *>(scratch + off);
    off += up((size_t)P * 4);
    int32_t *perm = reinterpret_cast<int32_t *>(scratch + off);
    off += up((size_t)L * 4);
    int32_t *perm2 = reinterpret_cast<int32_t *>(scratch + off);
    off += up((size_t)L * 4);
    int32_t *upf = reinterpret_cast<int32_t *>(scratch + off);
    off += up((size_t)L * 4);
    int32_t *upscan = reinterpret_cast<int32_t *>(scratch + off);
    off += up((size_t)L * 4);
    int32_t *start = reinterpret_cast<int32_t *>(scratch + off);
    off += up((size_t)P * 4);
    int32_t *start2 = reinterpret_cast<int32_t *>(scratch + off);
    off += up((size_t)P * 4);
    int32_t *total = reinterpret_cast<int32_t *>(scratch + off);
    off += up(4);
    void *scan_scr = scratch + off;

    if (L == 0) return cudaMemsetAsync(palette, 0, (size_t)P * stride * sizeof(S), s);
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    MC_CK(cudaMemsetAsync(hist, 0, (size_t)half * 256 * 4, s));
    mc_init_kernel<<<blocks_of(L), kMcThreads, 0, s>>>(box_of, perm, L);
    MC_CK(cudaMemsetAsync(start, 0, sizeof(int32_t), s));  // round 0: one box, from entry 0
    for (int r = 0; r < bits; r++) {
        const int64_t nb = int64_t(1) << r;
        mc_clear_kernel<<<blocks_of(nb * dim), kMcThreads, 0, s>>>(lo, hi, box, nb, dim);
        if (nb <= kMcSharedBoxes && dim <= kMcMaxDim) {
            const unsigned grid = std::min<unsigned>(blocks_of(L), (unsigned)(4 * sms));
            mc_minmax_shared_kernel<S><<<grid, kMcThreads, 0, s>>>(rows, stride, dim, L, box_of, perm,
                                                                   lo, hi, box, (int)nb);
        } else {
            mc_minmax_kernel<S><<<blocks_of(L), kMcThreads, 0, s>>>(rows, stride, dim, L, box_of, perm,
                                                                    lo, hi, box);
        }
        mc_axis_kernel<<<blocks_of(nb), kMcThreads, 0, s>>>(lo, hi, box, nb, dim);
        for (int shift = 56; shift >= 0; shift -= 8) {
            mc_hist_kernel<S><<<blocks_of(L), kMcThreads, 0, s>>>(rows, stride, L, box_of, box, shift, hist);
            mc_pick_kernel<<<blocks_of(nb * 32), kMcThreads, 0, s>>>(hist, box, nb, shift);
        }
        mc_assign_kernel<S><<<blocks_of(L), kMcThreads, 0, s>>>(rows, stride, L, box_of, box);
        if (r + 1 < bits) {  // the next round's segments
            mc_flag_kernel<<<blocks_of(L), kMcThreads, 0, s>>>(perm, box_of, L, upf);
            MC_CK(scan_exclusive_i32(upf, upscan, L, total, scan_scr, s));
            mc_partition_kernel<<<blocks_of(L), kMcThreads, 0, s>>>(perm, box_of, upscan, start, box,
                                                                    L, perm2);
            mc_starts_kernel<<<blocks_of(nb), kMcThreads, 0, s>>>(start, box, nb, start2);
            std::swap(perm, perm2);
            std::swap(start, start2);
        }
    }
    MC_CK(cudaMemsetAsync(sum, 0, (size_t)P * dim * 8, s));
    MC_CK(cudaMemsetAsync(count, 0, (size_t)P * 4, s));
    mc_sum_kernel<S><<<blocks_of(L), kMcThreads, 0, s>>>(rows, stride, dim, L, box_of, sum, count);
    mc_palette_kernel<S><<<blocks_of(P * stride), kMcThreads, 0, s>>>(sum, count, P, dim, stride, palette);
    mc_record_kernel<S><<<blocks_of(L), kMcThreads, 0, s>>>(sigma, box_of, L, rec);
    return cudaGetLastError();
}

size_t median_cut_scratch(int64_t L, int dim, int bits) {
    const int64_t P = int64_t(1) << bits, half = P / 2;
    auto up = [](size_t x) { return (x + 255) / 256 * 256; };
    return up((size_t)L * 4) + 2 * up((size_t)half * dim * 4) + up((size_t)half * sizeof(McBox)) +
           up((size_t)half * 256 * 4) + up((size_t)P * dim * 8) + up((size_t)P * 4) +
           4 * up((size_t)L * 4) + 2 * up((size_t)P * 4) + up(4) + scan_scratch_bytes(L);
}

}  // namespace

cudaError_t compress_tree(TreeArrays &a, int bits, const DevAlloc &al, cudaStream_t s) {
    const int64_t L = a.n_leaves, P = int64_t(1) << bits;
    const int dim = 3 * a.K, rs = a.row_stride;
    void *palette = al.alloc((size_t)P * rs * 2, s);
    uint32_t *leaf_rec = (uint32_t *)al.alloc((size_t)std::max<int64_t>(L, 1) * 4, s);
    char *scratch = nullptr;
    cudaError_t e = (palette && leaf_rec) ? cudaSuccess : cudaErrorMemoryAllocation;
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&scratch, median_cut_scratch(L, dim, bits), s);
    if (e == cudaSuccess) {
        if (a.storage == DOT_STORAGE_F16)
            e = median_cut<__half>((const __half *)a.sh, (const __half *)a.sigma, L, dim, rs, bits,
                                   (__half *)palette, leaf_rec, scratch, s);
        else
            e = median_cut<__nv_bfloat16>((const __nv_bfloat16 *)a.sh, (const __nv_bfloat16 *)a.sigma,
                                          L, dim, rs, bits, (__nv_bfloat16 *)palette, leaf_rec,
                                          scratch, s);
    }
    if (scratch) {
        const cudaError_t ef = cudaFreeAsync(scratch, s);
        if (e == cudaSuccess) e = ef;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        al.release(palette, s);
        al.release(leaf_rec, s);
        return e;
    }
    al.release(a.sh, s);
    a.sh = nullptr;
    a.palette = palette;
    a.leaf_rec = leaf_rec;
    a.palette_bits = bits;
    return cudaSuccess;
}

}  // namespace dot
