// ropes.cu -- the face-neighbour table of the leaves (ropes): for each leaf and each of its six
// faces, the node on the other side of that face at the leaf's level, or the leaf covering that
// place when the tree is coarser there.  The march follows a rope when a step leaves a leaf
// through one face, so that it finds the next leaf with one load (and a descent only into a
// neighbour subdivided finer) instead of re-descending from the deepest common ancestor.  The
// table depends on the structure only (child table and leaf keys) and is rebuilt after every
// call that changes the structure.
#include "internal.cuh"
#include "tree.cuh"

namespace dot {
namespace {

// one thread per (leaf, face); face f = 2 axis + (1 for the upper face)
__global__ void ropes_kernel(const int32_t *__restrict__ child, const uint64_t *__restrict__ leaf_key,
                             int64_t L, int32_t *__restrict__ rope) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 6 * L) return;
    const int64_t v = i / 6;
    const int f = (int)(i - 6 * v);
    const int axis = f >> 1;
    const uint64_t key = leaf_key[v];
    const int level = (63 - __clzll((long long)key)) / 3;  // key = 1 << 3 level | coordinates
    int c[3] = {0, 0, 0};
    for (int b = 0; b < level; b++) {  // x is the most significant bit of each triple
        const int tri = (int)((key >> (3 * (level - 1 - b))) & 7u);
        c[0] = (c[0] << 1) | (tri >> 2);
        c[1] = (c[1] << 1) | ((tri >> 1) & 1);
        c[2] = (c[2] << 1) | (tri & 1);
    }
    const int cs = 1 << (kGridBits - level);
    int g[3];
#pragma unroll
    for (int a = 0; a < 3; a++) g[a] = c[a] << (kGridBits - level);  // corner on the 2^16 grid
    g[axis] += (f & 1) ? cs : -cs;                                   // the neighbour's corner
    int32_t out = INT32_MIN;                                         // outside the root
    if (g[axis] >= 0 && g[axis] < (1 << kGridBits)) {
        int32_t node = 0;
        for (int l = 0; l < level; l++) {
            const int sh = kGridBits - 1 - l;
            const int j = (((g[0] >> sh) & 1) << 2) | (((g[1] >> sh) & 1) << 1) | ((g[2] >> sh) & 1);
            const int32_t ch = child[(int64_t)node * 8 + j];
            if (ch < 0) {  // a leaf at level l + 1: its id and how many levels coarser it is
                out = -1 - (((-1 - ch) << kRopeLevelBits) | (level - (l + 1)));
                break;
            }
            if (l + 1 == level) {  // the node at the leaf's level: the neighbour is finer
                out = ch;
                break;
            }
            node = ch;
        }
    }
    rope[i] = out;
}

}  // namespace

cudaError_t build_ropes(const TreeArrays &a, cudaStream_t s) {
    if (a.n_leaves == 0) return cudaSuccess;
    if (a.n_leaves > kMaxRopeLeaves) return cudaErrorNotSupported;
    const int64_t n = 6 * a.n_leaves;
    ropes_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a.child, a.leaf_key, a.n_leaves, a.rope);
    return cudaGetLastError();
}

}  // namespace dot
