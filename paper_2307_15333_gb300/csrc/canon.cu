// canon.cu -- canonical renumbering of a tree: nodes and leaves in the build's order (breadth
// first, Morton order within a level, which is ascending key order).  Refines append new leaves
// and nodes at the end of the arrays, so after many refines neighbouring cells drift apart in
// memory; renumbering puts each level's cells back in Morton order.
//
// Level-synchronous walk from the root: the internal nodes of level l are known in canonical
// order; their 8 n_l child slots are flagged internal / leaf and one exclusive scan of the flags
// numbers the level-(l + 1) nodes (the rank) and leaves (slot index minus the rank), in parent
// order then slot order, which is Morton order.  One host sync per level reads the count.
#include <algorithm>

#include "internal.cuh"
#include "tree.cuh"

namespace dot {

namespace {

#define CN_CK(x)                                    \
    do {                                            \
        cudaError_t e_ = (x);                       \
        if (e_ != cudaSuccess) {                    \
            cleanup();                              \
            return e_;                              \
        }                                           \
    } while (0)

// node records of the current level, and the flag (internal child) of each of its slots
__global__ void level_nodes_kernel(const int32_t *__restrict__ cur, const int32_t *__restrict__ cur_parent,
                                   int64_t n_cur, int64_t cur_base,
                                   const int32_t *__restrict__ old_child,
                                   const uint64_t *__restrict__ old_key, uint64_t *__restrict__ new_key,
                                   int32_t *__restrict__ new_parent, int32_t *__restrict__ flags) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= 8 * n_cur) return;
    const int64_t i = s >> 3;
    const int j = (int)(s & 7);
    const int32_t o = cur[i];
    flags[s] = old_child[(int64_t)o * 8 + j] >= 0 ? 1 : 0;
    if (j == 0) {
        new_key[cur_base + i] = old_key[o];
        new_parent[cur_base + i] = cur_parent[i];
    }
}

// child pointers of the current level; the next level's nodes; leaf ranks and records
__global__ void level_scatter_kernel(const int32_t *__restrict__ cur, int64_t n_cur, int64_t cur_base,
                                     int64_t next_base, int64_t leaf_base,
                                     const int32_t *__restrict__ old_child,
                                     const int32_t *__restrict__ rank,
                                     const uint64_t *__restrict__ old_leaf_key,
                                     int32_t *__restrict__ new_child, int32_t *__restrict__ next,
                                     int32_t *__restrict__ next_parent, int32_t *__restrict__ perm,
                                     uint64_t *__restrict__ new_leaf_key,
                                     int32_t *__restrict__ new_leaf_parent) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= 8 * n_cur) return;
    const int64_t i = s >> 3;
    const int j = (int)(s & 7);
    const int32_t c = old_child[(int64_t)cur[i] * 8 + j];
    const int64_t r = rank[s];
    if (c >= 0) {
        next[r] = c;
        next_parent[r] = (int32_t)(cur_base + i);
        new_child[(cur_base + i) * 8 + j] = (int32_t)(next_base + r);
    } else {
        const int64_t u = leaf_base + (s - r);
        const int32_t v = -1 - c;
        perm[u] = v;
        new_leaf_key[u] = old_leaf_key[v];
        new_leaf_parent[u] = (int32_t)(cur_base + i);
        new_child[(cur_base + i) * 8 + j] = (int32_t)(-1 - u);
    }
}

template <typename S>
__global__ void gather_leaves_kernel(const int32_t *__restrict__ perm, int64_t L,
                                     const S *__restrict__ sigma, S *__restrict__ nsigma,
                                     const uint4 *__restrict__ sh, uint4 *__restrict__ nsh,
                                     int row_vec, const uint32_t *__restrict__ rec,
                                     uint32_t *__restrict__ nrec) {
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= L) return;
    const int64_t v = perm[u];
    nsigma[u] = sigma[v];
    if (sh)
        for (int q = 0; q < row_vec; q++) nsh[u * row_vec + q] = sh[v * row_vec + q];
    if (rec) nrec[u] = rec[v];
}

__global__ void gather_aux_kernel(const int32_t *__restrict__ perm, int64_t L,
                                  const float *__restrict__ src, float *__restrict__ dst, int width) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= L * width) return;
    const int64_t u = i / width;
    const int k = (int)(i - u * width);
    dst[i] = src[(int64_t)perm[u] * width + k];
}

unsigned blocks_for(int64_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace

cudaError_t canonicalize_tree(const TreeArrays &old, TreeArrays *out, const DevAlloc &alloc,
                              int32_t *perm, const dot_leaf_array *aux, int n_aux, cudaStream_t s) {
    TreeArrays nw;
    nw.n_nodes = old.n_nodes;
    nw.n_leaves = old.n_leaves;
    nw.max_level = old.max_level;
    nw.sh_degree = old.sh_degree;
    nw.storage = old.storage;
    nw.K = old.K;
    nw.row_stride = old.row_stride;
    nw.palette_bits = old.palette_bits;
    const int64_t N = old.n_nodes, L = old.n_leaves;
    const size_t sb = (size_t)storage_bytes(old.storage);
    const size_t row_bytes = (size_t)old.row_stride * sb;

    int32_t *cur = nullptr, *cur_parent = nullptr, *flags = nullptr, *rank = nullptr;
    int32_t *total = nullptr, *next = nullptr, *next_parent = nullptr;
    void *scratch = nullptr;
    bool owned_new = false;
    auto cleanup = [&]() {
        for (void *p : {(void *)cur, (void *)cur_parent, (void *)flags, (void *)rank,
                        (void *)total, (void *)next, (void *)next_parent, scratch})
            if (p) cudaFreeAsync(p, s);
        cur = cur_parent = flags = rank = total = next = next_parent = nullptr;
        scratch = nullptr;
        if (owned_new) free_tree_arrays(nw, alloc, s);
    };

    // arrays of the new tree (SH rows only when the tree has them; palette copied as is)
    nw.child = (int32_t *)alloc.alloc((size_t)N * 8 * 4, s);
    nw.node_parent = (int32_t *)alloc.alloc((size_t)N * 4, s);
    nw.node_key = (uint64_t *)alloc.alloc((size_t)N * 8, s);
    nw.leaf_parent = (int32_t *)alloc.alloc((size_t)L * 4, s);
    nw.leaf_key = (uint64_t *)alloc.alloc((size_t)L * 8, s);
    nw.sigma = alloc.alloc((size_t)L * sb, s);
    nw.rope = (int32_t *)alloc.alloc((size_t)L * 6 * sizeof(int32_t), s);
    if (old.sh) nw.sh = alloc.alloc((size_t)L * row_bytes, s);
    if (old.leaf_rec) {
        nw.leaf_rec = (uint32_t *)alloc.alloc((size_t)L * 4, s);
        nw.palette = alloc.alloc(((size_t)1 << old.palette_bits) * row_bytes, s);
    }
    owned_new = true;
    if (!nw.child || !nw.node_parent || !nw.node_key || !nw.leaf_parent || !nw.leaf_key ||
        !nw.sigma || !nw.rope || (old.sh && !nw.sh) ||
        (old.leaf_rec && (!nw.leaf_rec || !nw.palette))) {
        cleanup();
        return cudaErrorMemoryAllocation;
    }

    CN_CK(cudaMallocAsync(&total, sizeof(int32_t), s));
    CN_CK(cudaMallocAsync(&cur, sizeof(int32_t), s));
    CN_CK(cudaMallocAsync(&cur_parent, sizeof(int32_t), s));
    {
        const int32_t root = 0, none = -1;
        CN_CK(cudaMemcpyAsync(cur, &root, 4, cudaMemcpyHostToDevice, s));
        CN_CK(cudaMemcpyAsync(cur_parent, &none, 4, cudaMemcpyHostToDevice, s));
    }
    int64_t n_cur = N > 0 ? 1 : 0, cur_base = 0, leaf_base = 0;
    while (n_cur > 0) {
        const int64_t slots = 8 * n_cur;
        CN_CK(cudaMallocAsync(&flags, (size_t)slots * 4, s));
        CN_CK(cudaMallocAsync(&rank, (size_t)slots * 4, s));
        CN_CK(cudaMallocAsync(&scratch, scan_scratch_bytes(slots), s));
        level_nodes_kernel<<<blocks_for(slots), 256, 0, s>>>(cur, cur_parent, n_cur, cur_base,
                                                             old.child, old.node_key, nw.node_key,
                                                             nw.node_parent, flags);
        CN_CK(cudaGetLastError());
        CN_CK(scan_exclusive_i32(flags, rank, slots, total, scratch, s));
        int32_t n_next = 0;
        CN_CK(cudaMemcpyAsync(&n_next, total, 4, cudaMemcpyDeviceToHost, s));
        CN_CK(cudaStreamSynchronize(s));
        const int64_t next_base = cur_base + n_cur;
        if (next_base + n_next > N || leaf_base + (slots - n_next) > L) {  // inconsistent table
            cleanup();
            return cudaErrorInvalidValue;
        }
        CN_CK(cudaMallocAsync(&next, (size_t)std::max<int64_t>(n_next, 1) * 4, s));
        CN_CK(cudaMallocAsync(&next_parent, (size_t)std::max<int64_t>(n_next, 1) * 4, s));
        level_scatter_kernel<<<blocks_for(slots), 256, 0, s>>>(
            cur, n_cur, cur_base, next_base, leaf_base, old.child, rank, old.leaf_key, nw.child,
            next, next_parent, perm, nw.leaf_key, nw.leaf_parent);
        CN_CK(cudaGetLastError());
        CN_CK(cudaFreeAsync(flags, s));
        CN_CK(cudaFreeAsync(rank, s));
        CN_CK(cudaFreeAsync(scratch, s));
        CN_CK(cudaFreeAsync(cur, s));
        CN_CK(cudaFreeAsync(cur_parent, s));
        flags = rank = nullptr;
        scratch = nullptr;
        cur = next;
        cur_parent = next_parent;
        next = next_parent = nullptr;
        leaf_base += slots - n_next;
        cur_base = next_base;
        n_cur = n_next;
    }
    if (cur_base != N || leaf_base != L) {  // a node or leaf unreachable from the root
        cleanup();
        return cudaErrorInvalidValue;
    }
    if (L > 0) {
        const int row_vec = (int)(row_bytes / 16);
        switch (old.storage) {
            case DOT_STORAGE_F32:
                gather_leaves_kernel<float><<<blocks_for(L), 256, 0, s>>>(
                    perm, L, (const float *)old.sigma, (float *)nw.sigma, (const uint4 *)old.sh,
                    (uint4 *)nw.sh, row_vec, old.leaf_rec, nw.leaf_rec);
                break;
            default:
                gather_leaves_kernel<uint16_t><<<blocks_for(L), 256, 0, s>>>(
                    perm, L, (const uint16_t *)old.sigma, (uint16_t *)nw.sigma,
                    (const uint4 *)old.sh, (uint4 *)nw.sh, row_vec, old.leaf_rec, nw.leaf_rec);
        }
        CN_CK(cudaGetLastError());
        for (int i = 0; i < n_aux; i++) {
            gather_aux_kernel<<<blocks_for(L * aux[i].width), 256, 0, s>>>(
                perm, L, (const float *)aux[i].src, (float *)aux[i].dst, aux[i].width);
            CN_CK(cudaGetLastError());
        }
    }
    if (old.leaf_rec)
        CN_CK(cudaMemcpyAsync(nw.palette, old.palette, ((size_t)1 << old.palette_bits) * row_bytes,
                              cudaMemcpyDeviceToDevice, s));
    CN_CK(build_ropes(nw, s));
    if (cur) CN_CK(cudaFreeAsync(cur, s));
    if (cur_parent) CN_CK(cudaFreeAsync(cur_parent, s));
    CN_CK(cudaFreeAsync(total, s));
    cur = cur_parent = total = nullptr;
    owned_new = false;
    *out = nw;
    return cudaSuccess;
}

}  // namespace dot
