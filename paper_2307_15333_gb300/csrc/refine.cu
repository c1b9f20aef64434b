// refine.cu -- prune (Eq. 3) and sample (Eq. 4) as flag kernels, exclusive scans and scatters.
//
// Plan: merge[p] for parents (not the root) whose 8 children are prune-marked leaves with no
// sample mark; sampled[v] for sample-marked leaves above the depth cap; survive[v] for leaves
// neither merged away nor sampled.  Exclusive scans of these flags number the new tree:
//   leaves: survivors | merged parents | 8 children per sampled leaf,
//   nodes:  surviving nodes | sampled leaves.
// Apply: one thread per old node writes its new node (or merged leaf), one thread per old leaf
// writes its survivor (or new node and 8 children); parameters are copied row by row as 16-byte
// vectors, merged means are pairwise FP32 sums times 1/8 rounded once to the storage type.
#include "internal.cuh"
#include "tree.cuh"

namespace dot {

namespace {

__device__ __forceinline__ int key_level(uint64_t key) { return (63 - __clzll((long long)key)) / 3; }

__global__ void merge_flags_kernel(const int32_t *__restrict__ child, int64_t N,
                                   const uint8_t *__restrict__ prune,
                                   const uint8_t *__restrict__ sample, int32_t *__restrict__ merge,
                                   int32_t *__restrict__ keep) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    bool m = p != 0;
#pragma unroll
    for (int j = 0; j < 8; j++) {
        const int32_t c = child[8 * p + j];
        if (c >= 0) {
            m = false;
        } else {
            const int32_t v = -1 - c;
            m = m && prune[v] && !sample[v];
        }
    }
    merge[p] = m ? 1 : 0;
    keep[p] = m ? 0 : 1;
}

__global__ void leaf_flags_kernel(const uint64_t *__restrict__ leaf_key,
                                  const int32_t *__restrict__ leaf_parent, int64_t L,
                                  const uint8_t *__restrict__ sample,
                                  const int32_t *__restrict__ merge, int d_cap,
                                  int32_t *__restrict__ sampled, int32_t *__restrict__ survive,
                                  unsigned long long *__restrict__ capped) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= L) return;
    const bool pm = merge[leaf_parent[v]] != 0;
    const bool sm = sample[v] != 0;
    const bool deep = key_level(leaf_key[v]) >= d_cap;
    const bool sp = sm && !deep && !pm;
    sampled[v] = sp ? 1 : 0;
    survive[v] = (!pm && !sp) ? 1 : 0;
    if (sm && deep) atomicAdd(capped, 1ull);
}

struct Ranks {
    const int32_t *merge, *keep, *sampled, *survive;  // flags
    const int32_t *m_idx, *n_idx, *c_idx, *s_idx;     // exclusive scans
    int64_t S, M, NS;                                  // totals
};

template <typename S>
__device__ __forceinline__ void copy_row(const S *__restrict__ src, S *__restrict__ dst, int stride) {
    const uint4 *a = reinterpret_cast<const uint4 *>(src);
    uint4 *b = reinterpret_cast<uint4 *>(dst);
    const int nv = stride * (int)sizeof(S) / 16;
    for (int i = 0; i < nv; i++) b[i] = a[i];
}

__device__ __forceinline__ float pairwise8(const float x[8]) {
    return ((x[0] + x[1]) + (x[2] + x[3])) + ((x[4] + x[5]) + (x[6] + x[7]));
}

__global__ void apply_nodes_kernel(const int32_t *__restrict__ child,
                                   const int32_t *__restrict__ node_parent,
                                   const uint64_t *__restrict__ node_key, int64_t N, Ranks R,
                                   int32_t *__restrict__ n_child, int32_t *__restrict__ n_parent,
                                   uint64_t *__restrict__ n_key) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N || !R.keep[p]) return;
    const int64_t q = R.n_idx[p];
    const int32_t par = node_parent[p];
    n_parent[q] = par >= 0 ? R.n_idx[par] : -1;
    n_key[q] = node_key[p];
#pragma unroll
    for (int j = 0; j < 8; j++) {
        const int32_t c = child[8 * p + j];
        int32_t nc;
        if (c >= 0) {
            nc = R.merge[c] ? (int32_t)(-1 - (R.S + R.m_idx[c])) : R.n_idx[c];
        } else {
            const int32_t v = -1 - c;
            nc = R.sampled[v] ? (int32_t)(R.NS + R.c_idx[v]) : (int32_t)(-1 - R.s_idx[v]);
        }
        n_child[8 * q + j] = nc;
    }
}

template <typename S>
__global__ void apply_merged_kernel(const int32_t *__restrict__ child,
                                    const int32_t *__restrict__ node_parent,
                                    const uint64_t *__restrict__ node_key, int64_t N, Ranks R,
                                    const S *__restrict__ sigma, const S *__restrict__ sh,
                                    int row_stride, int ncomp, int32_t *__restrict__ l_parent,
                                    uint64_t *__restrict__ l_key, S *__restrict__ n_sigma,
                                    S *__restrict__ n_sh, int32_t *__restrict__ leaf_map) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N || !R.merge[p]) return;
    const int64_t u = R.S + R.m_idx[p];
    l_parent[u] = R.n_idx[node_parent[p]];
    l_key[u] = node_key[p];
    leaf_map[u] = (int32_t)(-1 - p);
    int32_t v[8];
#pragma unroll
    for (int j = 0; j < 8; j++) v[j] = -1 - child[8 * p + j];
    float x[8];
#pragma unroll
    for (int j = 0; j < 8; j++) x[j] = Storage<S>::to_f32(sigma[v[j]]);
    n_sigma[u] = Storage<S>::from_f32(pairwise8(x) * 0.125f);
    S *dst = n_sh + u * row_stride;
    for (int i = 0; i < row_stride; i++) {
        if (i < ncomp) {
#pragma unroll
            for (int j = 0; j < 8; j++) x[j] = Storage<S>::to_f32(sh[(int64_t)v[j] * row_stride + i]);
            dst[i] = Storage<S>::from_f32(pairwise8(x) * 0.125f);
        } else {
            dst[i] = Storage<S>::from_f32(0.f);
        }
    }
}

template <typename S>
__global__ void apply_leaves_kernel(const uint64_t *__restrict__ leaf_key,
                                    const int32_t *__restrict__ leaf_parent, int64_t L, Ranks R,
                                    const S *__restrict__ sigma, const S *__restrict__ sh,
                                    int row_stride, int32_t *__restrict__ n_child,
                                    int32_t *__restrict__ n_parent, uint64_t *__restrict__ n_key,
                                    int32_t *__restrict__ l_parent, uint64_t *__restrict__ l_key,
                                    S *__restrict__ n_sigma, S *__restrict__ n_sh,
                                    int32_t *__restrict__ leaf_map) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= L) return;
    if (R.survive[v]) {
        const int64_t u = R.s_idx[v];
        l_parent[u] = R.n_idx[leaf_parent[v]];
        l_key[u] = leaf_key[v];
        leaf_map[u] = (int32_t)v;
        n_sigma[u] = sigma[v];
        copy_row(sh + v * row_stride, n_sh + u * row_stride, row_stride);
    } else if (R.sampled[v]) {
        const int64_t q = R.NS + R.c_idx[v];
        const int64_t base = R.S + R.M + 8 * (int64_t)R.c_idx[v];
        n_parent[q] = R.n_idx[leaf_parent[v]];
        n_key[q] = leaf_key[v];
        const S sv = sigma[v];
        for (int j = 0; j < 8; j++) {
            const int64_t u = base + j;
            n_child[8 * q + j] = (int32_t)(-1 - u);
            l_parent[u] = (int32_t)q;
            l_key[u] = (leaf_key[v] << 3) | (uint64_t)j;
            leaf_map[u] = (int32_t)v;
            n_sigma[u] = sv;
            copy_row(sh + v * row_stride, n_sh + u * row_stride, row_stride);
        }
    }
}

// extra per-leaf FP32 arrays carried through the refine
__global__ void remap_aux_kernel(const int32_t *__restrict__ leaf_map, int64_t L_new,
                                 const int32_t *__restrict__ old_child,
                                 const float *__restrict__ src, float *__restrict__ dst, int width,
                                 int merge) {
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= L_new) return;
    const int32_t m = leaf_map[u];
    if (m >= 0) {
        for (int i = 0; i < width; i++) dst[u * width + i] = src[(int64_t)m * width + i];
        return;
    }
    const int64_t p = -1 - (int64_t)m;
    for (int i = 0; i < width; i++) {
        float x[8];
#pragma unroll
        for (int j = 0; j < 8; j++) x[j] = src[(int64_t)(-1 - old_child[8 * p + j]) * width + i];
        float r;
        if (merge == DOT_MERGE_MAX) {
            r = x[0];
#pragma unroll
            for (int j = 1; j < 8; j++) r = fmaxf(r, x[j]);
        } else {
            r = pairwise8(x);
            if (merge == DOT_MERGE_MEAN) r *= 0.125f;
        }
        dst[u * width + i] = r;
    }
}

__global__ void max_level_kernel(const uint64_t *__restrict__ key, int64_t n, int *__restrict__ out) {
    int best = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        best = max(best, key_level(key[i]));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) best = max(best, __shfl_down_sync(0xffffffffu, best, off));
    if ((threadIdx.x & 31) == 0) atomicMax(out, best);
}

#define RF_CK(x)                               \
    do {                                       \
        cudaError_t e_ = (x);                  \
        if (e_ != cudaSuccess) {               \
            cleanup();                         \
            return e_;                         \
        }                                      \
    } while (0)

template <typename S>
void launch_apply(const TreeArrays &old, const Ranks &R, TreeArrays &nw, int32_t *leaf_map,
                  cudaStream_t s) {
    const int64_t N = old.n_nodes, L = old.n_leaves;
    const int ncomp = 3 * old.K;
    if (N > 0) {
        const unsigned b = (unsigned)((N + 255) / 256);
        apply_nodes_kernel<<<b, 256, 0, s>>>(old.child, old.node_parent, old.node_key, N, R,
                                             nw.child, nw.node_parent, nw.node_key);
        apply_merged_kernel<S><<<b, 256, 0, s>>>(old.child, old.node_parent, old.node_key, N, R,
                                                 (const S *)old.sigma, (const S *)old.sh,
                                                 old.row_stride, ncomp, nw.leaf_parent, nw.leaf_key,
                                                 (S *)nw.sigma, (S *)nw.sh, leaf_map);
    }
    if (L > 0) {
        const unsigned b = (unsigned)((L + 255) / 256);
        apply_leaves_kernel<S><<<b, 256, 0, s>>>(old.leaf_key, old.leaf_parent, L, R,
                                                 (const S *)old.sigma, (const S *)old.sh,
                                                 old.row_stride, nw.child, nw.node_parent,
                                                 nw.node_key, nw.leaf_parent, nw.leaf_key,
                                                 (S *)nw.sigma, (S *)nw.sh, leaf_map);
    }
}

}  // namespace

cudaError_t refine_tree(const TreeArrays &old, const uint8_t *prune, const uint8_t *sample,
                        int d_cap, bool apply, TreeArrays *out, const DevAlloc &alloc,
                        int32_t *leaf_map, const dot_leaf_array *aux, int n_aux,
                        RefinePlan *plan, cudaStream_t s) {
    const int64_t N = old.n_nodes, L = old.n_leaves;
    // scratch: 4 flag arrays + 4 scans (int32) + scan partials + totals + capped counter
    const size_t aN = ((size_t)N * 4 + 255) / 256 * 256, aL = ((size_t)L * 4 + 255) / 256 * 256;
    const size_t sc = scan_scratch_bytes(N > L ? N : L);
    const size_t bytes = 4 * aN + 4 * aL + sc + 256;
    char *scratch = nullptr;
    auto cleanup = [&]() {
        if (scratch) cudaFreeAsync(scratch, s);
        scratch = nullptr;
    };
    RF_CK(cudaMallocAsync((void **)&scratch, bytes, s));
    int32_t *merge = (int32_t *)scratch, *keep = (int32_t *)(scratch + aN);
    int32_t *m_idx = (int32_t *)(scratch + 2 * aN), *n_idx = (int32_t *)(scratch + 3 * aN);
    char *lb = scratch + 4 * aN;
    int32_t *sampled = (int32_t *)lb, *survive = (int32_t *)(lb + aL);
    int32_t *c_idx = (int32_t *)(lb + 2 * aL), *s_idx = (int32_t *)(lb + 3 * aL);
    char *scan_tmp = lb + 4 * aL;
    int32_t *totals = (int32_t *)(scan_tmp + sc);                 // [4]
    unsigned long long *capped = (unsigned long long *)(totals + 4);
    RF_CK(cudaMemsetAsync(totals, 0, 64, s));
    if (N > 0)
        merge_flags_kernel<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(old.child, N, prune, sample,
                                                                       merge, keep);
    if (L > 0)
        leaf_flags_kernel<<<(unsigned)((L + 255) / 256), 256, 0, s>>>(
            old.leaf_key, old.leaf_parent, L, sample, merge, d_cap, sampled, survive, capped);
    RF_CK(cudaGetLastError());
    RF_CK(scan_exclusive_i32(merge, m_idx, N, totals + 0, scan_tmp, s));
    RF_CK(scan_exclusive_i32(keep, n_idx, N, totals + 1, scan_tmp, s));
    RF_CK(scan_exclusive_i32(sampled, c_idx, L, totals + 2, scan_tmp, s));
    RF_CK(scan_exclusive_i32(survive, s_idx, L, totals + 3, scan_tmp, s));
    struct {
        int32_t t[4];
        unsigned long long capped;
    } h;
    RF_CK(cudaMemcpyAsync(&h, totals, sizeof(h), cudaMemcpyDeviceToHost, s));
    RF_CK(cudaStreamSynchronize(s));
    const int64_t M = h.t[0], NS = h.t[1], C = h.t[2], Sv = h.t[3];
    plan->n_merged = M;
    plan->n_keep = NS;
    plan->n_sampled = C;
    plan->n_survive = Sv;
    plan->n_capped = (int64_t)h.capped;
    plan->n_nodes = NS + C;
    plan->n_leaves = Sv + M + 8 * C;
    if (!apply) {
        cleanup();
        return cudaSuccess;
    }
    TreeArrays nw;
    nw.n_nodes = plan->n_nodes;
    nw.n_leaves = plan->n_leaves;
    nw.sh_degree = old.sh_degree;
    nw.storage = old.storage;
    nw.K = old.K;
    nw.row_stride = old.row_stride;
    RF_CK(alloc_tree_arrays(nw, alloc, s));
    Ranks R{merge, keep, sampled, survive, m_idx, n_idx, c_idx, s_idx, Sv, M, NS};
    switch (old.storage) {
        case DOT_STORAGE_F32: launch_apply<float>(old, R, nw, leaf_map, s); break;
        case DOT_STORAGE_F16: launch_apply<__half>(old, R, nw, leaf_map, s); break;
        default: launch_apply<__nv_bfloat16>(old, R, nw, leaf_map, s); break;
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = build_ropes(nw, s);
    for (int i = 0; e == cudaSuccess && i < n_aux; i++) {
        if (nw.n_leaves == 0) break;
        remap_aux_kernel<<<(unsigned)((nw.n_leaves + 255) / 256), 256, 0, s>>>(
            leaf_map, nw.n_leaves, old.child, aux[i].src, aux[i].dst, aux[i].width, aux[i].merge);
        e = cudaGetLastError();
    }
    int *d_lvl = (int *)(totals + 2);
    int h_lvl = 0;
    if (e == cudaSuccess) e = cudaMemsetAsync(d_lvl, 0, sizeof(int), s);
    if (e == cudaSuccess && nw.n_leaves > 0) {
        const int64_t want = (nw.n_leaves + 255) / 256;
        max_level_kernel<<<(unsigned)(want < 1024 ? want : 1024), 256, 0, s>>>(nw.leaf_key, nw.n_leaves, d_lvl);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_lvl, d_lvl, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        free_tree_arrays(nw, alloc, s);
        cleanup();
        return e;
    }
    nw.max_level = h_lvl;
    cleanup();
    *out = nw;
    return cudaSuccess;
}

}  // namespace dot
