// train.cu -- the optimisation step of the training loop (Algorithm 1, optimization):
//   * the MSE loss over stochastic ray samples (Sec. 4.1) and its gradient dL/dC, the input of
//     the backward march;
//   * one RMSProp update of every leaf's density and SH coefficients (Sec. 3.3; learning rates of
//     Sec. 4.1), fused with zeroing the FP32 gradients for the next step.
// Both are HBM-bound streams: RMSProp moves 4 + 4 + 4 (+ 4 + 4 + 4 written) bytes of FP32
// gradient and mean-square state and 2 x storage bytes of parameter per coefficient.
#include "internal.cuh"

namespace dot {

namespace {

constexpr int kTrainThreads = 256;

// lanes that update one touched leaf in the sparse RMSProp step (4, 8 or 16); 16 measured fastest
// on a degree-3 tree (a 49-coefficient row in four coalesced 16-byte passes)
#ifndef DOT_SPARSE_GROUP
#define DOT_SPARSE_GROUP 16
#endif
// leaves a group updates per pass of the sparse RMSProp step, and the blocks per SM its register
// budget is built for (0: no bound)
#ifndef DOT_SPARSE_UNROLL
#define DOT_SPARSE_UNROLL 2
#endif
#ifndef DOT_SPARSE_MINB
#define DOT_SPARSE_MINB 4
#endif
// 1: the optimiser state rows stream through L2 with evict-first loads and stores, so that the
// tree's nodes, ropes and densities stay in L2 for the next step's march (258.6 -> 252.2 us per
// training step)
#ifndef DOT_SPARSE_STREAM
#define DOT_SPARSE_STREAM 1
#endif

// grad[r][c] = 2 (rgb - target) / (3 R); loss_sum += sum (rgb - target)^2 / (3 R)
__global__ void __launch_bounds__(kTrainThreads)
mse_grad_kernel(const float *__restrict__ rgb, const float *__restrict__ target, int64_t n,
                float inv, float *__restrict__ grad, double *__restrict__ loss_sum) {
    __shared__ float s_part[kTrainThreads / 32];
    float acc = 0.f;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float e = rgb[i] - target[i];
        grad[i] = 2.f * e * inv;
        acc = fmaf(e, e, acc);
    }
    if (!loss_sum) return;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float b = 0.f;
        for (int w = 0; w < kTrainThreads / 32; w++) b += s_part[w];
        atomicAdd(loss_sum, (double)b * (double)inv);
    }
}

struct Rms {
    float lr, rho, one_minus_rho, eps;
    int zero_grad;
};

__device__ __forceinline__ float rms_update(float p, float g, float &ms, const Rms &o) {
    ms = fmaf(o.rho, ms, o.one_minus_rho * (g * g));
    return p - __fdiv_rn(o.lr * g, sqrtf(ms) + o.eps);
}

// one coefficient per thread: entry i of a [rows][width] FP32 array, parameter at
// row * pstride + column in the storage type
template <typename S>
__global__ void __launch_bounds__(kTrainThreads)
rmsprop_scalar_kernel(S *__restrict__ param, int64_t pstride, float *__restrict__ grad,
                      float *__restrict__ ms, int64_t rows, int width, Rms o) {
    const int64_t n = rows * width;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int64_t r = i / width;
        const int c = (int)(i - r * width);
        S *pp = param + r * pstride + c;
        const float g = grad[i];
        float m = ms[i];
        const float p = rms_update(Storage<S>::to_f32(*pp), g, m, o);
        ms[i] = m;
        *pp = Storage<S>::from_f32(p);
        if (o.zero_grad) grad[i] = 0.f;
    }
}

// four consecutive coefficients per thread (width % 4 == 0 and 16-byte aligned arrays)
template <typename S> struct Vec4;
template <> struct Vec4<float> {
    using T = float4;
    static __device__ __forceinline__ void get(const T &v, float x[4]) { x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w; }
    static __device__ __forceinline__ T make(const float x[4]) { return make_float4(x[0], x[1], x[2], x[3]); }
};
template <> struct Vec4<__half> {
    using T = uint2;
    static __device__ __forceinline__ void get(const T &v, float x[4]) {
        const __half2 a = *reinterpret_cast<const __half2 *>(&v.x), b = *reinterpret_cast<const __half2 *>(&v.y);
        const float2 fa = __half22float2(a), fb = __half22float2(b);
        x[0] = fa.x; x[1] = fa.y; x[2] = fb.x; x[3] = fb.y;
    }
    static __device__ __forceinline__ T make(const float x[4]) {
        const __half2 a = __halves2half2(__float2half_rn(x[0]), __float2half_rn(x[1]));
        const __half2 b = __halves2half2(__float2half_rn(x[2]), __float2half_rn(x[3]));
        T v;
        v.x = *reinterpret_cast<const unsigned *>(&a);
        v.y = *reinterpret_cast<const unsigned *>(&b);
        return v;
    }
};
template <> struct Vec4<__nv_bfloat16> {
    using T = uint2;
    static __device__ __forceinline__ void get(const T &v, float x[4]) {
        const __nv_bfloat162 a = *reinterpret_cast<const __nv_bfloat162 *>(&v.x);
        const __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162 *>(&v.y);
        const float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
        x[0] = fa.x; x[1] = fa.y; x[2] = fb.x; x[3] = fb.y;
    }
    static __device__ __forceinline__ T make(const float x[4]) {
        const __nv_bfloat162 a = __halves2bfloat162(__float2bfloat16_rn(x[0]), __float2bfloat16_rn(x[1]));
        const __nv_bfloat162 b = __halves2bfloat162(__float2bfloat16_rn(x[2]), __float2bfloat16_rn(x[3]));
        T v;
        v.x = *reinterpret_cast<const unsigned *>(&a);
        v.y = *reinterpret_cast<const unsigned *>(&b);
        return v;
    }
};

template <typename S>
__global__ void __launch_bounds__(kTrainThreads)
rmsprop_vec4_kernel(S *__restrict__ param, int64_t pstride, float *__restrict__ grad,
                    float *__restrict__ ms, int64_t rows, int width, Rms o) {
    using V = Vec4<S>;
    const int q = width / 4;
    const int64_t n = rows * q;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int64_t r = i / q;
        const int c = (int)(i - r * q) * 4;
        float4 *g4 = reinterpret_cast<float4 *>(grad) + i;
        float4 *m4 = reinterpret_cast<float4 *>(ms) + i;
        typename V::T *pv = reinterpret_cast<typename V::T *>(param + r * pstride + c);
        const float4 g = *g4;
        float4 m = *m4;
        float p[4];
        V::get(*pv, p);
        p[0] = rms_update(p[0], g.x, m.x, o);
        p[1] = rms_update(p[1], g.y, m.y, o);
        p[2] = rms_update(p[2], g.z, m.z, o);
        p[3] = rms_update(p[3], g.w, m.w, o);
        *m4 = m;
        *pv = V::make(p);
        if (o.zero_grad) *g4 = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

int grid_for(int64_t n) {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (n + kTrainThreads - 1) / kTrainThreads;
    const int64_t cap = (int64_t)sms * 8;  // 8 resident blocks of 256 per SM, grid-stride beyond
    return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

// blocks of kTrainThreads for n threads' worth of work, at most one resident wave of KERNEL
template <auto KERNEL>
int resident_grid(int64_t n) {
    static const int per_sm = [] {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, KERNEL, kTrainThreads, 0) != cudaSuccess)
            cudaGetLastError();
        return b > 0 ? b : 1;
    }();
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (n + kTrainThreads - 1) / kTrainThreads;
    const int64_t cap = (int64_t)sms * per_sm;
    return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

template <typename S>
cudaError_t rmsprop_array(S *param, int64_t pstride, float *grad, float *ms, int64_t rows,
                          int width, const Rms &o, cudaStream_t s) {
    if (rows == 0 || width == 0) return cudaSuccess;
    const bool vec = width % 4 == 0 && pstride % 4 == 0 && aligned16(grad) && aligned16(ms) &&
                     (reinterpret_cast<uintptr_t>(param) % (4 * sizeof(S))) == 0;
    if (vec) {
        const int64_t n = rows * (width / 4);
        rmsprop_vec4_kernel<S><<<grid_for(n), kTrainThreads, 0, s>>>(param, pstride, grad, ms, rows, width, o);
    } else {
        const int64_t n = rows * width;
        rmsprop_scalar_kernel<S><<<grid_for(n), kTrainThreads, 0, s>>>(param, pstride, grad, ms, rows, width, o);
    }
    return cudaGetLastError();
}

template <typename S>
cudaError_t rmsprop_s(void *sigma, void *sh, int64_t L, int K, int row_stride, float *grad_sigma,
                      float *grad_sh, float *ms_sigma, float *ms_sh, const dot_rmsprop_opts &op,
                      cudaStream_t s) {
    Rms o;
    o.rho = op.rho;
    o.one_minus_rho = 1.f - op.rho;
    o.eps = op.eps;
    o.zero_grad = op.zero_grad;
    o.lr = op.lr_sigma;
    // the density vector [L] walked as rows of 4096 contiguous entries plus one shorter row
    cudaError_t e = cudaSuccess;
    const int64_t W = 4096;
    const int64_t full = L / W, rest = L - full * W;
    S *sg = reinterpret_cast<S *>(sigma);
    if (full) e = rmsprop_array<S>(sg, W, grad_sigma, ms_sigma, full, (int)W, o, s);
    if (e == cudaSuccess && rest)
        e = rmsprop_array<S>(sg + full * W, W, grad_sigma + full * W, ms_sigma + full * W, 1,
                             (int)rest, o, s);
    if (e != cudaSuccess) return e;
    o.lr = op.lr_sh;
    return rmsprop_array<S>(reinterpret_cast<S *>(sh), row_stride, grad_sh, ms_sh, L, 3 * K, o, s);
}

// ---- sparse RMSProp: only the leaves touched since the last step, with deferred decay ----------

// list[count++] = v for every touched leaf (order irrelevant: leaves update independently)
__global__ void __launch_bounds__(kTrainThreads)
compact_touched_kernel(const uint8_t *__restrict__ touched, int64_t L, int32_t *__restrict__ list,
                       int32_t *__restrict__ count) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < L; base += stride) {
        const int64_t v = base + threadIdx.x;
        const bool f = v < L && touched[v] != 0;
        const unsigned m = __ballot_sync(0xffffffffu, f);
        int32_t pos = 0;
        if (lane == 0 && m) pos = atomicAdd(count, __popc(m));
        pos = __shfl_sync(0xffffffffu, pos, 0);
        if (f) list[pos + __popc(m & ((1u << lane) - 1u))] = (int32_t)v;
    }
}

// The same list, sixteen flags per thread (one 16-byte load) and one counter atomic per block of
// 4096 flags: the per-warp atomics above contend on the single counter.  touched must be 16-byte
// aligned; the flags past L are read from the last chunk with bounds checks.
__global__ void __launch_bounds__(kTrainThreads)
compact_touched16_kernel(const uint8_t *__restrict__ touched, int64_t L, int32_t *__restrict__ list,
                         int32_t *__restrict__ count) {
    __shared__ int32_t s_warp[kTrainThreads / 32];
    __shared__ int32_t s_base;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t per_block = (int64_t)kTrainThreads * 16;
    for (int64_t b0 = (int64_t)blockIdx.x * per_block; b0 < L; b0 += (int64_t)gridDim.x * per_block) {
        const int64_t v0 = b0 + (int64_t)threadIdx.x * 16;
        uint32_t bits = 0;  // bit j: flag of leaf v0 + j
        if (v0 + 16 <= L) {
            const uint4 q = *reinterpret_cast<const uint4 *>(touched + v0);
            const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int k = 0; k < 4; k++)
#pragma unroll
                for (int j = 0; j < 4; j++)
                    if ((w[k] >> (8 * j)) & 0xffu) bits |= 1u << (4 * k + j);
        } else {
            for (int j = 0; j < 16 && v0 + j < L; j++)
                if (touched[v0 + j]) bits |= 1u << j;
        }
        const int n = __popc(bits);
        int inc = n;  // inclusive warp scan of the counts
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int o = __shfl_up_sync(0xffffffffu, inc, off);
            if (lane >= off) inc += o;
        }
        if (lane == 31) s_warp[warp] = inc;
        __syncthreads();
        if (threadIdx.x == 0) {
            int run = 0;
            for (int w = 0; w < kTrainThreads / 32; w++) {
                const int c = s_warp[w];
                s_warp[w] = run;
                run += c;
            }
            s_base = run ? atomicAdd(count, run) : 0;
        }
        __syncthreads();
        int32_t pos = s_base + s_warp[warp] + inc - n;
        while (bits) {
            const int j = __ffs(bits) - 1;
            bits &= bits - 1;
            list[pos++] = (int32_t)(v0 + j);
        }
        __syncthreads();  // s_warp and s_base are rewritten by the next chunk
    }
}

// rho^k by binary powering in FP32 (k >= 0)
__device__ __forceinline__ float rho_pow(float rho, int k) {
    float r = 1.f, b = rho;
    while (k > 0) {
        if (k & 1) r *= b;
        b *= b;
        k >>= 1;
    }
    return r;
}

// G lanes per touched leaf: lane 0 updates the density, the lanes walk the coefficient row four
// at a time (16-byte gradient and mean-square loads, coalesced across the lanes).  A group takes U
// leaves of the list per pass.  Each pass issues all its loads (the leaves' last-update steps,
// densities and first row chunks) before any arithmetic, and the list entries of the next pass
// are loaded one pass ahead, so a pass costs one memory round trip instead of three (list, then
// last step, then the rows behind the decay's loop).
template <typename S, bool VEC, int G, int U>
__global__ void __launch_bounds__(kTrainThreads, DOT_SPARSE_MINB)
rmsprop_sparse_kernel(const int32_t *__restrict__ list, const int32_t *__restrict__ count,
                      S *__restrict__ sigma, S *__restrict__ sh, int row_stride, int width,
                      float *__restrict__ grad_sigma, float *__restrict__ grad_sh,
                      float *__restrict__ ms_sigma, float *__restrict__ ms_sh,
                      uint8_t *__restrict__ touched, int32_t *__restrict__ last, int32_t step,
                      float lr_sigma, float lr_sh, Rms o) {
    static_assert(G == 4 || G == 8 || G == 16, "group of 4, 8 or 16 lanes");
    constexpr int LOG_G = G == 4 ? 2 : (G == 8 ? 3 : 4);
    using V = Vec4<S>;
    const int64_t n = *count;
    const int gl = threadIdx.x & (G - 1);
    const unsigned gmask = ((1u << G) - 1u) << (threadIdx.x & 31 & ~(G - 1));
    const int64_t groups = ((int64_t)gridDim.x * blockDim.x) >> LOG_G;
    const int64_t per_pass = groups * U;
    const int q4 = width / 4;
    int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> LOG_G;
    int32_t vn[U];  // list entries of the next pass
#pragma unroll
    for (int u = 0; u < U; u++) vn[u] = i0 + u * groups < n ? list[i0 + u * groups] : 0;
    for (; i0 < n; i0 += per_pass) {
        int32_t v[U], lv[U];
        bool ok[U];
        float ps[U], gs[U], ms[U];
        float4 g[U], m[U];
        typename V::T pv[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            ok[u] = i0 + u * groups < n;
            v[u] = vn[u];
            lv[u] = ok[u] ? last[v[u]] : step - 1;
        }
        if (gl == 0) {
#pragma unroll
            for (int u = 0; u < U; u++) {
                if (ok[u]) {
                    ps[u] = Storage<S>::to_f32(sigma[v[u]]);
                    gs[u] = grad_sigma[v[u]];
                    ms[u] = ms_sigma[v[u]];
                }
            }
        }
        auto load_chunk = [&](int q) {  // four coefficients of every leaf of the pass
#pragma unroll
            for (int u = 0; u < U; u++) {
                if (ok[u]) {
#if DOT_SPARSE_STREAM
                    g[u] = __ldcs(reinterpret_cast<const float4 *>(grad_sh + (int64_t)v[u] * width) + q);
                    m[u] = __ldcs(reinterpret_cast<const float4 *>(ms_sh + (int64_t)v[u] * width) + q);
#else
                    g[u] = reinterpret_cast<const float4 *>(grad_sh + (int64_t)v[u] * width)[q];
                    m[u] = reinterpret_cast<const float4 *>(ms_sh + (int64_t)v[u] * width)[q];
#endif
                    pv[u] = *reinterpret_cast<const typename V::T *>(sh + (int64_t)v[u] * row_stride + 4 * q);
                }
            }
        };
        if constexpr (VEC) {
            if (gl < q4) load_chunk(gl);
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int64_t j = i0 + per_pass + u * groups;
            vn[u] = j < n ? list[j] : 0;
        }
        float decay[U];
#pragma unroll
        for (int u = 0; u < U; u++) decay[u] = ok[u] ? rho_pow(o.rho, step - lv[u] - 1) : 0.f;  // steps sat out
        if (gl == 0) {
            o.lr = lr_sigma;
#pragma unroll
            for (int u = 0; u < U; u++) {
                if (ok[u]) {
                    float mm = decay[u] * ms[u];
                    const float p = rms_update(ps[u], gs[u], mm, o);
                    ms_sigma[v[u]] = mm;
                    sigma[v[u]] = Storage<S>::from_f32(p);
                    if (o.zero_grad) grad_sigma[v[u]] = 0.f;
                }
            }
        }
        o.lr = lr_sh;
        if constexpr (VEC) {
            for (int q = gl; q < q4; q += G) {
                if (q != gl) load_chunk(q);
#pragma unroll
                for (int u = 0; u < U; u++) {
                    if (!ok[u]) continue;
                    float4 mm = m[u];
                    mm.x *= decay[u];
                    mm.y *= decay[u];
                    mm.z *= decay[u];
                    mm.w *= decay[u];
                    float p[4];
                    V::get(pv[u], p);
                    p[0] = rms_update(p[0], g[u].x, mm.x, o);
                    p[1] = rms_update(p[1], g[u].y, mm.y, o);
                    p[2] = rms_update(p[2], g[u].z, mm.z, o);
                    p[3] = rms_update(p[3], g[u].w, mm.w, o);
#if DOT_SPARSE_STREAM
                    __stcs(reinterpret_cast<float4 *>(ms_sh + (int64_t)v[u] * width) + q, mm);
#else
                    reinterpret_cast<float4 *>(ms_sh + (int64_t)v[u] * width)[q] = mm;
#endif
                    *reinterpret_cast<typename V::T *>(sh + (int64_t)v[u] * row_stride + 4 * q) = V::make(p);
                    if (o.zero_grad)
#if DOT_SPARSE_STREAM
                        __stcs(reinterpret_cast<float4 *>(grad_sh + (int64_t)v[u] * width) + q,
                               make_float4(0.f, 0.f, 0.f, 0.f));
#else
                        reinterpret_cast<float4 *>(grad_sh + (int64_t)v[u] * width)[q] = make_float4(0.f, 0.f, 0.f, 0.f);
#endif
                }
            }
        } else {
#pragma unroll
            for (int u = 0; u < U; u++) {
                if (!ok[u]) continue;
                for (int c = gl; c < width; c += G) {
                    float *gp = grad_sh + (int64_t)v[u] * width + c;
                    float *mp = ms_sh + (int64_t)v[u] * width + c;
                    S *pp = sh + (int64_t)v[u] * row_stride + c;
                    float mm = decay[u] * *mp;
                    const float p = rms_update(Storage<S>::to_f32(*pp), *gp, mm, o);
                    *mp = mm;
                    *pp = Storage<S>::from_f32(p);
                    if (o.zero_grad) *gp = 0.f;
                }
            }
        }
        __syncwarp(gmask);  // every lane has read last[v]
        if (gl == 0) {
#pragma unroll
            for (int u = 0; u < U; u++) {
                if (ok[u]) {
                    touched[v[u]] = 0;
                    last[v[u]] = step;
                }
            }
        }
    }
}

// ms <- rho^(step - last) ms over the flat [L][width] array (one entry per thread, coalesced);
// last is only read here and advanced by rmsprop_flush_last_kernel afterwards
__global__ void __launch_bounds__(kTrainThreads)
rmsprop_flush_kernel(int64_t L, int width, float *__restrict__ ms_sigma, float *__restrict__ ms_sh,
                     const int32_t *__restrict__ last, int32_t step, float rho) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t n = L * width;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n + L; i += stride) {
        const int64_t v = i < n ? i / width : i - n;
        const int k = step - last[v];
        if (k <= 0) continue;
        const float d = rho_pow(rho, k);
        if (i < n) ms_sh[i] *= d;
        else ms_sigma[v] *= d;
    }
}

__global__ void __launch_bounds__(kTrainThreads)
rmsprop_flush_last_kernel(int64_t L, int32_t *__restrict__ last, int32_t step) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < L; v += stride)
        last[v] = step;
}

}  // namespace

cudaError_t launch_rmsprop_sparse(int storage, void *sigma, void *sh, int64_t L, int K,
                                  int row_stride, float *grad_sigma, float *grad_sh,
                                  float *ms_sigma, float *ms_sh, uint8_t *touched, int32_t *last,
                                  int32_t step, int32_t *work, const dot_rmsprop_opts &op,
                                  cudaStream_t s) {
    if (L == 0) return cudaSuccess;
    int32_t *count = work + L;
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    if ((reinterpret_cast<uintptr_t>(touched) & 15) == 0) {
        const int64_t chunks = (L + (int64_t)kTrainThreads * 16 - 1) / ((int64_t)kTrainThreads * 16);
        const int grid = (int)(chunks < (int64_t)grid_for(L) ? chunks : grid_for(L));
        compact_touched16_kernel<<<grid, kTrainThreads, 0, s>>>(touched, L, work, count);
    } else {
        compact_touched_kernel<<<grid_for(L), kTrainThreads, 0, s>>>(touched, L, work, count);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    Rms o;
    o.rho = op.rho;
    o.one_minus_rho = 1.f - op.rho;
    o.eps = op.eps;
    o.zero_grad = op.zero_grad;
    o.lr = 0.f;
    const int width = 3 * K;
    const bool vec = width % 4 == 0 && row_stride % 4 == 0 &&
                     (reinterpret_cast<uintptr_t>(grad_sh) & 15) == 0 &&
                     (reinterpret_cast<uintptr_t>(ms_sh) & 15) == 0;
    constexpr int G = DOT_SPARSE_GROUP;
    constexpr int U = DOT_SPARSE_UNROLL;
    // one resident wave: the list length is known only on the device
#define DOT_SPARSE_LAUNCH(T)                                                                     \
    if (vec)                                                                                     \
        rmsprop_sparse_kernel<T, true, G, U>                                                     \
            <<<resident_grid<rmsprop_sparse_kernel<T, true, G, U>>(L * G), kTrainThreads, 0, s>>>( \
                work, count, (T *)sigma, (T *)sh, row_stride, width, grad_sigma, grad_sh,        \
                ms_sigma, ms_sh, touched, last, step, op.lr_sigma, op.lr_sh, o);                 \
    else                                                                                         \
        rmsprop_sparse_kernel<T, false, G, U>                                                    \
            <<<resident_grid<rmsprop_sparse_kernel<T, false, G, U>>(L * G), kTrainThreads, 0, s>>>( \
                work, count, (T *)sigma, (T *)sh, row_stride, width, grad_sigma, grad_sh,        \
                ms_sigma, ms_sh, touched, last, step, op.lr_sigma, op.lr_sh, o);
    switch (storage) {
        case DOT_STORAGE_F32: DOT_SPARSE_LAUNCH(float) break;
        case DOT_STORAGE_F16: DOT_SPARSE_LAUNCH(__half) break;
        default: DOT_SPARSE_LAUNCH(__nv_bfloat16) break;
    }
#undef DOT_SPARSE_LAUNCH
    return cudaGetLastError();
}

cudaError_t launch_rmsprop_flush(int64_t L, int K, float *ms_sigma, float *ms_sh, int32_t *last,
                                 int32_t step, float rho, cudaStream_t s) {
    if (L == 0) return cudaSuccess;
    rmsprop_flush_kernel<<<grid_for(L * (3 * K + 1)), kTrainThreads, 0, s>>>(L, 3 * K, ms_sigma,
                                                                             ms_sh, last, step, rho);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    rmsprop_flush_last_kernel<<<grid_for(L), kTrainThreads, 0, s>>>(L, last, step);
    return cudaGetLastError();
}

cudaError_t launch_mse_grad(const float *rgb, const float *target, int64_t n_rays, float *grad,
                            double *loss_sum, cudaStream_t s) {
    if (n_rays == 0) return cudaSuccess;
    const int64_t n = 3 * n_rays;
    const float inv = (float)(1.0 / (3.0 * (double)n_rays));
    mse_grad_kernel<<<grid_for(n), kTrainThreads, 0, s>>>(rgb, target, n, inv, grad, loss_sum);
    return cudaGetLastError();
}

cudaError_t launch_rmsprop(int storage, void *sigma, void *sh, int64_t L, int K, int row_stride,
                           float *grad_sigma, float *grad_sh, float *ms_sigma, float *ms_sh,
                           const dot_rmsprop_opts &op, cudaStream_t s) {
    switch (storage) {
        case DOT_STORAGE_F32: return rmsprop_s<float>(sigma, sh, L, K, row_stride, grad_sigma, grad_sh, ms_sigma, ms_sh, op, s);
        case DOT_STORAGE_F16: return rmsprop_s<__half>(sigma, sh, L, K, row_stride, grad_sigma, grad_sh, ms_sigma, ms_sh, op, s);
        case DOT_STORAGE_BF16: return rmsprop_s<__nv_bfloat16>(sigma, sh, L, K, row_stride, grad_sigma, grad_sh, ms_sigma, ms_sh, op, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace dot
