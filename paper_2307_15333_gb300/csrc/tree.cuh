// tree.cuh -- the arrays a tree owns, and the allocator they come from.
#pragma once

#include "internal.cuh"

namespace dot {

// Allocator of tree-owned arrays: the caller's dot_allocator when given, else cudaMallocAsync.
struct DevAlloc {
    dot_allocator user{};
    bool has_user = false;
    void *alloc(size_t bytes, cudaStream_t s) const {
        if (bytes == 0) bytes = 16;
        if (has_user) {
            void *p = user.alloc(user.ctx, bytes, (void *)s);
            if (p && (reinterpret_cast<uintptr_t>(p) & 15u)) {  // rows are read as 16-byte vectors
                user.free(user.ctx, p, (void *)s);
                return nullptr;
            }
            return p;
        }
        void *p = nullptr;
        if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return p;
    }
    void release(void *p, cudaStream_t s) const {
        if (!p) return;
        if (has_user) user.free(user.ctx, p, (void *)s);
        else cudaFreeAsync(p, s);
    }
};

struct TreeArrays {
    int64_t n_nodes = 0, n_leaves = 0;
    int max_level = 0, sh_degree = 0, storage = 0, K = 1, row_stride = 4;
    int32_t *child = nullptr;
    int32_t *node_parent = nullptr;
    uint64_t *node_key = nullptr;
    int32_t *leaf_parent = nullptr;
    uint64_t *leaf_key = nullptr;
    void *sigma = nullptr;
    void *sh = nullptr;            // [L][row_stride]; null once the SH rows are compressed
    // compressed SH (16-bit storage only): palette [2^palette_bits][row_stride] and one 32-bit
    // record per leaf, the density's 16 bits in the low half and the palette row in the high half
    void *palette = nullptr;
    uint32_t *leaf_rec = nullptr;
    int palette_bits = 0;
    // ropes [L][6]: across face 2 axis + upper of a leaf, the node id at the leaf's level (>= 0),
    // or -1 - (v << kRopeLevelBits | levels coarser) for a leaf v, or INT32_MIN outside the root;
    // built by build_ropes
    int32_t *rope = nullptr;
};

inline void free_tree_arrays(TreeArrays &a, const DevAlloc &al, cudaStream_t s) {
    al.release(a.child, s);
    al.release(a.node_parent, s);
    al.release(a.node_key, s);
    al.release(a.leaf_parent, s);
    al.release(a.leaf_key, s);
    al.release(a.sigma, s);
    al.release(a.sh, s);
    al.release(a.palette, s);
    al.release(a.leaf_rec, s);
    al.release(a.rope, s);
    a.palette = nullptr;
    a.leaf_rec = nullptr;
    a.rope = nullptr;
    a.palette_bits = 0;
    a.child = a.node_parent = a.leaf_parent = nullptr;
    a.node_key = a.leaf_key = nullptr;
    a.sigma = a.sh = nullptr;
}

// allocates every array for the counts already set in a; all or nothing
inline cudaError_t alloc_tree_arrays(TreeArrays &a, const DevAlloc &al, cudaStream_t s) {
    const size_t sb = (size_t)storage_bytes(a.storage);
    a.child = (int32_t *)al.alloc((size_t)a.n_nodes * 8 * sizeof(int32_t), s);
    a.node_parent = (int32_t *)al.alloc((size_t)a.n_nodes * sizeof(int32_t), s);
    a.node_key = (uint64_t *)al.alloc((size_t)a.n_nodes * sizeof(uint64_t), s);
    a.leaf_parent = (int32_t *)al.alloc((size_t)a.n_leaves * sizeof(int32_t), s);
    a.leaf_key = (uint64_t *)al.alloc((size_t)a.n_leaves * sizeof(uint64_t), s);
    a.sigma = al.alloc((size_t)a.n_leaves * sb, s);
    a.sh = al.alloc((size_t)a.n_leaves * (size_t)a.row_stride * sb, s);
    a.rope = (int32_t *)al.alloc((size_t)a.n_leaves * 6 * sizeof(int32_t), s);
    if (!a.child || !a.node_parent || !a.node_key || !a.leaf_parent || !a.leaf_key || !a.sigma ||
        !a.sh || !a.rope) {
        free_tree_arrays(a, al, s);
        return cudaErrorMemoryAllocation;
    }
    return cudaSuccess;
}

cudaError_t build_tree(const dot_build_desc &desc, TreeArrays &out, const DevAlloc &alloc,
                       cudaStream_t s);

// ropes.cu: fills a.rope from a.child and a.leaf_key (after every change of the structure)
cudaError_t build_ropes(const TreeArrays &a, cudaStream_t s);

struct RefinePlan {
    int64_t n_nodes, n_leaves, n_merged, n_sampled, n_capped, n_survive, n_keep;
};

// refine.cu
cudaError_t refine_tree(const TreeArrays &old, const uint8_t *prune, const uint8_t *sample,
                        int d_cap, bool apply, TreeArrays *out, const DevAlloc &alloc,
                        int32_t *leaf_map, const dot_leaf_array *aux, int n_aux, RefinePlan *plan,
                        cudaStream_t s);

// select.cu
cudaError_t select_masks(const float *signal, int64_t n, int prune_mode, double prune_value,
                         int sample_mode, double sample_value, uint8_t *prune_mark,
                         uint8_t *sample_mark, cudaStream_t s);

}  // namespace dot
