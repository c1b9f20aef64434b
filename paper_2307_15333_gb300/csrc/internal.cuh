// internal.cuh -- types and helpers shared by the CUDA translation units of libdot.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/dot.h"

namespace dot {

constexpr int kGridBits = 16;              // finest addressable level: cells of 2^-16 root edge
constexpr int kRopeLevelBits = 4;          // a rope to a leaf holds its id and level difference
constexpr int64_t kMaxRopeLeaves = (int64_t)1 << (31 - kRopeLevelBits);  // leaves a tree may hold
constexpr int kMaxLevels = 16;
#ifndef DOT_SMALL_NT
#define DOT_SMALL_NT 256
#endif
constexpr int kMarchThreads = DOT_SMALL_NT;  // threads per block of launches below two waves
constexpr int kMaxPrimitives = 4096;

// ---------------------------------------------------------------------------------------------
// tree and launch descriptors passed by value to kernels
// ---------------------------------------------------------------------------------------------

struct TreeView {
    const int32_t *child;
    const void *sigma;
    const void *sh;            // SH rows, or the palette rows of a compressed tree
    const uint32_t *rec;       // compressed tree: per-leaf (density bits | palette row << 16)
    const int32_t *rope;       // [L][6] face neighbours (see ropes.cu)
    int64_t n_nodes, n_leaves;
    int32_t row_stride;        // storage elements per SH row
    int32_t max_level;
    float lo[3];               // root low corner (world)
    float size;                // root edge 2h (world)
    float scale;               // 1 / size
};

struct RaySource {
    int32_t kind;              // DOT_RAYS_*
    int32_t n_cams, width, height;
    int32_t tiles_x;           // ceil(width / 16)
    const dot_camera *cams;
    const int32_t *order;      // CAMERAS: view rendered by block row y, or null (identity)
    const float *origins, *dirs;
    int64_t n_rays;
};

struct RenderParams {
    float bg[3];
    float eps_T;
    int32_t color_act;
    int32_t signal_mode;
    int32_t max_steps;
};

struct RenderIO {
    float *rgb;                // FWD [R][3]
    float *T_final;            // FWD [R] or null
    float *signal;             // [L] or null
    const float *grad_rgb;     // BWD [R][3]
    const float *rgb_fwd;      // BWD [R][3]
    float *grad_sigma;         // BWD [L]
    float *grad_sh;            // BWD [L][3K]
    unsigned long long *stats; // STATS [4]
    uint32_t *status;          // device status word
    int32_t grad_vec;          // BWD: grad_sh rows may use 16-byte vector atomics
    uint8_t *touched;          // BWD: [L] or null; set to 1 for every leaf given a gradient
    const float *target;       // FWDBWD [R][3]: MSE target
    float *grad_out;           // FWDBWD [R][3]: dL/dC written (read back by the overflow re-march)
    double *loss_sum;          // FWDBWD: += sum (rgb - target)^2 * inv3R (or null)
    float inv3R;               // FWDBWD: 1 / (3 R)
};

// kFwdBwd: forward, MSE gradient and backward of each ray in one pass -- the occupied segments are
// recorded during the forward march and the gradients scattered from the record, so the
// backward needs no second traversal (rays with more occupied segments than the record holds
// march again in the backward mode).
enum MarchMode : int { kFwd = 0, kBwd = 1, kSignal = 2, kStats = 3, kFwdBwd = 4 };
// occupied segments a ray of the fused pass records (32 bytes each, local memory); the rays that
// overflow it are the longest ones, so it is sized above the 99.9th percentile of training rays
// (build-time tunable: -DDOT_RECORD_SEGMENTS=n)
#ifndef DOT_RECORD_SEGMENTS
#define DOT_RECORD_SEGMENTS 48
#endif
constexpr int kRecordSegments = DOT_RECORD_SEGMENTS;

// ---------------------------------------------------------------------------------------------
// host-side launchers (defined in the .cu files)
// ---------------------------------------------------------------------------------------------

cudaError_t launch_sigma_signal(int storage, const void *sigma, int64_t n, float *signal,
                                cudaStream_t stream);

// scans (scan.cu): exclusive prefix sum of int32 values, with the total written to *total.
size_t scan_scratch_bytes(int64_t n);
cudaError_t scan_exclusive_i32(const int32_t *in, int32_t *out, int64_t n, int32_t *total,
                               void *scratch, cudaStream_t stream);

// sizes of a row of SH coefficients in the storage type, padded to 16 bytes
inline int storage_bytes(int storage) { return storage == DOT_STORAGE_F32 ? 4 : 2; }
inline int row_stride_elems(int storage, int K) {
    int b = storage_bytes(storage);
    int bytes = 3 * K * b;
    bytes = (bytes + 15) / 16 * 16;
    return bytes / b;
}

// ---------------------------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------------------------

template <typename S> struct Storage;
template <> struct Storage<float> {
    static __device__ __forceinline__ float load(const float *p) { return __ldg(p); }
    static __device__ __forceinline__ float from_bits16(uint32_t) { return 0.f; }  // no 16-bit form
    static __device__ __forceinline__ float from_f32(float x) { return x; }
    static __device__ __forceinline__ float to_f32(float x) { return x; }
};
template <> struct Storage<__half> {
    static __device__ __forceinline__ float load(const __half *p) { return __half2float(__ldg(p)); }
    static __device__ __forceinline__ float from_bits16(uint32_t b) {
        return __half2float(__ushort_as_half((unsigned short)(b & 0xffffu)));
    }
    static __device__ __forceinline__ __half from_f32(float x) { return __float2half_rn(x); }
    static __device__ __forceinline__ float to_f32(__half x) { return __half2float(x); }
};
template <> struct Storage<__nv_bfloat16> {
    static __device__ __forceinline__ float load(const __nv_bfloat16 *p) {
        return __bfloat162float(__ldg(p));
    }
    static __device__ __forceinline__ float from_bits16(uint32_t b) {
        return __bfloat162float(__ushort_as_bfloat16((unsigned short)(b & 0xffffu)));
    }
    static __device__ __forceinline__ __nv_bfloat16 from_f32(float x) { return __float2bfloat16_rn(x); }
    static __device__ __forceinline__ float to_f32(__nv_bfloat16 x) { return __bfloat162float(x); }
};

}  // namespace dot
