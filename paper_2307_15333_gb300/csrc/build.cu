// build.cu -- octree construction from seeded primitives (level by level) and the seeded leaf
// parameter fill.
//
// Per level l the cells (in canonical order) are classified (internal iff the cell meets a
// primitive and l < D; the root always), ranked by an exclusive scan, and scattered: internal
// cells become nodes and emit their 8 children (slot order) as the next level's cells, the
// others become leaves.  Because parents are in Morton order and children are emitted in slot
// order, every level stays in Morton order and the numbering is breadth-first.
#include <vector>

#include "internal.cuh"
#include "tree.cuh"

namespace dot {

namespace {

__device__ __forceinline__ void key_corner(uint64_t key, int level, int64_t k[3]) {
    k[0] = k[1] = k[2] = 0;
    for (int i = level - 1; i >= 0; i--) {
        const unsigned tri = (unsigned)(key >> (3 * i)) & 7u;
        k[0] = (k[0] << 1) | ((tri >> 2) & 1u);
        k[1] = (k[1] << 1) | ((tri >> 1) & 1u);
        k[2] = (k[2] << 1) | (tri & 1u);
    }
}

// open interior of the cell [A, B] meets primitive p (integer units of 2^-24 of the root edge)
__device__ __forceinline__ bool meets(const int64_t *__restrict__ p, const int64_t A[3],
                                      const int64_t B[3]) {
    const int64_t type = __ldg(p);
    if (type == DOT_PRIM_SPHERE) {
        int64_t d2 = 0;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const int64_t c = __ldg(p + 1 + a);
            const int64_t e = c < A[a] ? A[a] - c : (c > B[a] ? c - B[a] : 0);
            d2 += e * e;
        }
        const int64_t r = __ldg(p + 4);
        return d2 < r * r;
    }
    if (type == DOT_PRIM_BOX) {
#pragma unroll
        for (int a = 0; a < 3; a++)
            if (!(A[a] < __ldg(p + 4 + a) && __ldg(p + 1 + a) < B[a])) return false;
        return true;
    }
    if (type == DOT_PRIM_CYLINDER) {
        const int64_t cx = __ldg(p + 1), cz = __ldg(p + 2), r = __ldg(p + 3);
        const int64_t ex = cx < A[0] ? A[0] - cx : (cx > B[0] ? cx - B[0] : 0);
        const int64_t ez = cz < A[2] ? A[2] - cz : (cz > B[2] ? cz - B[2] : 0);
        if (!(ex * ex + ez * ez < r * r)) return false;
        return A[1] < __ldg(p + 5) && __ldg(p + 4) < B[1];
    }
    return false;
}

__global__ void classify_kernel(const uint64_t *__restrict__ cell_key, int64_t n, int level,
                                int max_depth, const int64_t *__restrict__ prims, int n_prims,
                                int32_t *__restrict__ internal, uint8_t *__restrict__ inside) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    int64_t k[3], A[3], B[3];
    key_corner(cell_key[c], level, k);
    const int64_t sz = (int64_t)1 << (24 - level);
#pragma unroll
    for (int a = 0; a < 3; a++) {
        A[a] = k[a] * sz;
        B[a] = A[a] + sz;
    }
    bool m = false;
    for (int i = 0; i < n_prims && !m; i++) m = meets(prims + 8 * (int64_t)i, A, B);
    internal[c] = (level == 0 || (m && level < max_depth)) ? 1 : 0;
    inside[c] = m ? 1 : 0;
}

__global__ void scatter_kernel(const uint64_t *__restrict__ cell_key,
                               const int32_t *__restrict__ cell_parent, int64_t n,
                               const int32_t *__restrict__ internal,
                               const int32_t *__restrict__ rank,
                               const uint8_t *__restrict__ inside, int64_t node_base,
                               int64_t leaf_base, int32_t *__restrict__ prev_child,
                               int64_t prev_base, uint64_t *__restrict__ node_key,
                               int32_t *__restrict__ node_parent, uint64_t *__restrict__ leaf_key,
                               int32_t *__restrict__ leaf_parent, uint8_t *__restrict__ leaf_inside,
                               uint64_t *__restrict__ next_key, int32_t *__restrict__ next_parent) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const uint64_t key = cell_key[c];
    const int32_t P = cell_parent[c];
    const int slot = (int)(key & 7u);
    const int64_t r = rank[c];
    if (internal[c]) {
        const int32_t id = (int32_t)(node_base + r);
        node_key[r] = key;
        node_parent[r] = P;
        if (P >= 0) prev_child[(P - prev_base) * 8 + slot] = id;
#pragma unroll
        for (int j = 0; j < 8; j++) {
            next_key[8 * r + j] = (key << 3) | (uint64_t)j;
            next_parent[8 * r + j] = id;
        }
    } else {
        const int64_t lr = c - r;
        const int32_t v = (int32_t)(leaf_base + lr);
        leaf_key[lr] = key;
        leaf_parent[lr] = P;
        leaf_inside[lr] = inside[c];
        prev_child[(P - prev_base) * 8 + slot] = -1 - v;
    }
}

// SplitMix64 output number n for the given seed: mix(seed + (n + 1) gamma), gamma the golden
// ratio constant, mix the variant-13 finaliser (Steele, Lea, Flood 2014).
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t n) {
    uint64_t z = seed + (n + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

template <typename S>
__global__ void fill_params_kernel(const uint64_t *__restrict__ leaf_key,
                                   const uint8_t *__restrict__ inside, int64_t L, int K,
                                   int row_stride, uint64_t seed, float dlo, float dhi,
                                   float s_eff, float dc, S *__restrict__ sigma, S *__restrict__ sh) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= L) return;
    const uint64_t base = leaf_key[v] * 64ull;
    // density: lo + (hi - lo) u, u = (h >> 40) 2^-24, float32 products and sums
    const uint64_t h0 = splitmix64_at(seed, base);
    const float u = (float)(h0 >> 40) * (1.f / 16777216.f);
    const float s = __fadd_rn(dlo, __fmul_rn(__fsub_rn(dhi, dlo), u));
    sigma[v] = Storage<S>::from_f32(inside[v] ? s : 0.f);
    // SH: centred Irwin-Hall (n = 4) of the four 16-bit fields, scaled in float32
    S *row = sh + v * (int64_t)row_stride;
    for (int i = 0; i < 3 * K; i++) {
        const uint64_t h = splitmix64_at(seed, base + 1ull + (uint64_t)i);
        const int64_t sum = (int64_t)(h & 0xFFFFull) + (int64_t)((h >> 16) & 0xFFFFull) +
                            (int64_t)((h >> 32) & 0xFFFFull) + (int64_t)((h >> 48) & 0xFFFFull);
        const float z = (float)(2 * sum - 4 * 65535);
        float val = __fmul_rn(z, s_eff);
        if (i % K == 0) val = __fadd_rn(val, dc);
        row[i] = Storage<S>::from_f32(val);
    }
    for (int i = 3 * K; i < row_stride; i++) row[i] = Storage<S>::from_f32(0.f);
}

template <typename T>
cudaError_t dalloc(T **p, size_t count, cudaStream_t s) {
    *p = nullptr;
    if (count == 0) return cudaSuccess;
    return cudaMallocAsync((void **)p, count * sizeof(T), s);
}

struct LevelPiece {
    int64_t n_int = 0, n_leaf = 0;
    uint64_t *node_key = nullptr;
    int32_t *node_parent = nullptr;
    int32_t *child = nullptr;
    uint64_t *leaf_key = nullptr;
    int32_t *leaf_parent = nullptr;
    uint8_t *leaf_inside = nullptr;
};

}  // namespace

#define DOT_CK(x)                              \
    do {                                       \
        cudaError_t e_ = (x);                  \
        if (e_ != cudaSuccess) return e_;      \
    } while (0)

cudaError_t build_tree(const dot_build_desc &desc, TreeArrays &out, const DevAlloc &alloc,
                       cudaStream_t s) {
    const int D = desc.max_depth;
    const int K = (desc.sh_degree + 1) * (desc.sh_degree + 1);
    int64_t *d_prims = nullptr;
    const int np = desc.n_primitives;
    if (np > 0) {
        DOT_CK(dalloc(&d_prims, (size_t)np * 8, s));
        DOT_CK(cudaMemcpyAsync(d_prims, desc.primitives, (size_t)np * 8 * sizeof(int64_t),
                               cudaMemcpyHostToDevice, s));
    }
    std::vector<LevelPiece> pieces;
    uint64_t *cell_key = nullptr;
    int32_t *cell_parent = nullptr;
    int64_t n_cells = 1;
    {
        const uint64_t one = 1;
        const int32_t none = -1;
        DOT_CK(dalloc(&cell_key, 1, s));
        DOT_CK(dalloc(&cell_parent, 1, s));
        DOT_CK(cudaMemcpyAsync(cell_key, &one, sizeof(one), cudaMemcpyHostToDevice, s));
        DOT_CK(cudaMemcpyAsync(cell_parent, &none, sizeof(none), cudaMemcpyHostToDevice, s));
        DOT_CK(cudaStreamSynchronize(s));
    }
    int32_t *d_total = nullptr;
    DOT_CK(dalloc(&d_total, 1, s));
    int64_t node_base = 0, leaf_base = 0, prev_base = 0;
    int32_t *prev_child = nullptr;
    int max_level = 0;
    for (int l = 0; l <= D && n_cells > 0; l++) {
        const int64_t n = n_cells;
        int32_t *flags = nullptr, *rank = nullptr;
        uint8_t *inside = nullptr;
        void *scratch = nullptr;
        DOT_CK(dalloc(&flags, (size_t)n, s));
        DOT_CK(dalloc(&rank, (size_t)n, s));
        DOT_CK(dalloc(&inside, (size_t)n, s));
        DOT_CK(cudaMallocAsync(&scratch, scan_scratch_bytes(n), s));
        const unsigned blocks = (unsigned)((n + 255) / 256);
        classify_kernel<<<blocks, 256, 0, s>>>(cell_key, n, l, D, d_prims, np, flags, inside);
        DOT_CK(cudaGetLastError());
        DOT_CK(scan_exclusive_i32(flags, rank, n, d_total, scratch, s));
        int32_t h_total = 0;
        DOT_CK(cudaMemcpyAsync(&h_total, d_total, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        DOT_CK(cudaStreamSynchronize(s));
        LevelPiece pc;
        pc.n_int = h_total;
        pc.n_leaf = n - h_total;
        if (pc.n_leaf > 0) max_level = l;
        DOT_CK(dalloc(&pc.node_key, (size_t)pc.n_int, s));
        DOT_CK(dalloc(&pc.node_parent, (size_t)pc.n_int, s));
        DOT_CK(dalloc(&pc.child, (size_t)pc.n_int * 8, s));
        DOT_CK(dalloc(&pc.leaf_key, (size_t)pc.n_leaf, s));
        DOT_CK(dalloc(&pc.leaf_parent, (size_t)pc.n_leaf, s));
        DOT_CK(dalloc(&pc.leaf_inside, (size_t)pc.n_leaf, s));
        uint64_t *next_key = nullptr;
        int32_t *next_parent = nullptr;
        DOT_CK(dalloc(&next_key, (size_t)pc.n_int * 8, s));
        DOT_CK(dalloc(&next_parent, (size_t)pc.n_int * 8, s));
        scatter_kernel<<<blocks, 256, 0, s>>>(cell_key, cell_parent, n, flags, rank, inside,
                                              node_base, leaf_base, prev_child, prev_base,
                                              pc.node_key, pc.node_parent, pc.leaf_key,
                                              pc.leaf_parent, pc.leaf_inside, next_key, next_parent);
        DOT_CK(cudaGetLastError());
        DOT_CK(cudaFreeAsync(flags, s));
        DOT_CK(cudaFreeAsync(rank, s));
        DOT_CK(cudaFreeAsync(inside, s));
        DOT_CK(cudaFreeAsync(scratch, s));
        DOT_CK(cudaFreeAsync(cell_key, s));
        DOT_CK(cudaFreeAsync(cell_parent, s));
        cell_key = next_key;
        cell_parent = next_parent;
        n_cells = pc.n_int * 8;
        prev_child = pc.child;
        prev_base = node_base;
        node_base += pc.n_int;
        leaf_base += pc.n_leaf;
        pieces.push_back(pc);
    }
    if (cell_key) DOT_CK(cudaFreeAsync(cell_key, s));
    if (cell_parent) DOT_CK(cudaFreeAsync(cell_parent, s));
    DOT_CK(cudaFreeAsync(d_total, s));
    if (d_prims) DOT_CK(cudaFreeAsync(d_prims, s));

    // final arrays (owned by the tree) and concatenation of the per-level pieces
    out.n_nodes = node_base;
    out.n_leaves = leaf_base;
    out.max_level = max_level;
    out.sh_degree = desc.sh_degree;
    out.storage = desc.storage;
    out.K = K;
    out.row_stride = row_stride_elems(desc.storage, K);
    cudaError_t e = alloc_tree_arrays(out, alloc, s);
    if (e != cudaSuccess) return e;
    uint8_t *inside_all = nullptr;
    DOT_CK(dalloc(&inside_all, (size_t)leaf_base, s));
    int64_t no = 0, lo = 0;
    for (auto &pc : pieces) {
        if (pc.n_int) {
            DOT_CK(cudaMemcpyAsync(out.node_key + no, pc.node_key, pc.n_int * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
            DOT_CK(cudaMemcpyAsync(out.node_parent + no, pc.node_parent, pc.n_int * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
            DOT_CK(cudaMemcpyAsync(out.child + 8 * no, pc.child, pc.n_int * 8 * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
        }
        if (pc.n_leaf) {
            DOT_CK(cudaMemcpyAsync(out.leaf_key + lo, pc.leaf_key, pc.n_leaf * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
            DOT_CK(cudaMemcpyAsync(out.leaf_parent + lo, pc.leaf_parent, pc.n_leaf * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
            DOT_CK(cudaMemcpyAsync(inside_all + lo, pc.leaf_inside, pc.n_leaf, cudaMemcpyDeviceToDevice, s));
        }
        no += pc.n_int;
        lo += pc.n_leaf;
        for (void *p : {(void *)pc.node_key, (void *)pc.node_parent, (void *)pc.child,
                        (void *)pc.leaf_key, (void *)pc.leaf_parent, (void *)pc.leaf_inside})
            if (p) DOT_CK(cudaFreeAsync(p, s));
    }
    // seeded parameters
    const double s_ih = 2.0 * sqrt(4.0 * (65536.0 * 65536.0 - 1.0) / 12.0);
    const float s_eff = (float)((double)desc.sh_std / s_ih);
    if (leaf_base > 0) {
        const unsigned blocks = (unsigned)((leaf_base + 255) / 256);
        switch (desc.storage) {
            case DOT_STORAGE_F32:
                fill_params_kernel<float><<<blocks, 256, 0, s>>>(out.leaf_key, inside_all, leaf_base, K, out.row_stride, desc.seed, desc.density_lo, desc.density_hi, s_eff, desc.sh_dc, (float *)out.sigma, (float *)out.sh);
                break;
            case DOT_STORAGE_F16:
                fill_params_kernel<__half><<<blocks, 256, 0, s>>>(out.leaf_key, inside_all, leaf_base, K, out.row_stride, desc.seed, desc.density_lo, desc.density_hi, s_eff, desc.sh_dc, (__half *)out.sigma, (__half *)out.sh);
                break;
            default:
                fill_params_kernel<__nv_bfloat16><<<blocks, 256, 0, s>>>(out.leaf_key, inside_all, leaf_base, K, out.row_stride, desc.seed, desc.density_lo, desc.density_hi, s_eff, desc.sh_dc, (__nv_bfloat16 *)out.sigma, (__nv_bfloat16 *)out.sh);
                break;
        }
        DOT_CK(cudaGetLastError());
    }
    DOT_CK(build_ropes(out, s));
    if (inside_all) DOT_CK(cudaFreeAsync(inside_all, s));
    return cudaSuccess;
}

}  // namespace dot
