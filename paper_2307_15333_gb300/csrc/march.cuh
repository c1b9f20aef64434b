// march.cuh -- one ray's march through the octree, shared by the forward, backward, signal and
// statistics kernels so that every mode sees bit-identical segments and transmittance.
//
// Per ray (Sec. 3 Preliminaries; Eq. 1-2):
//   1. slab test against the root cube, entry t0 >= 0;
//   2. the current cell is kept as integer coordinates g on the 2^16 grid; a step that leaves a
//      leaf through one face follows that face's rope (the neighbour at the leaf's level, or the
//      coarser leaf there) and descends from it only if the neighbour is subdivided finer; a step
//      across an edge or a corner descends from the root;
//   3. the leaf's exit time is the nearest of its three exit faces; delta = t_exit - t;
//   4. occupied segments (sigma > 0) are shaded: SH colour, alpha = 1 - exp(-sigma delta),
//      w = T alpha, C += w c, T *= exp(-sigma delta); the march stops once T < eps_T;
//   5. the next cell steps across every exit face hit at t_exit (edges and corners included) and
//      keeps the other coordinates of the exit point clamped into the old cell.
// Plane times are computed from the plane's exact coordinate, never accumulated, so neighbouring
// cells agree bit for bit on shared faces and segment lengths telescope.  In exact mode they are
// float-float values (about 44 bits), in fast mode float32.
#pragma once

#include <type_traits>

#include "internal.cuh"

// 1: forward launches store their images with evict-first stores (8.670 -> 8.648 ms on the
// 800^2 workload)
#ifndef DOT_STREAM_OUT
#define DOT_STREAM_OUT 1
#endif

namespace dot {

// ---------------------------------------------------------------------------------------------
// real spherical-harmonic constants from their closed forms, evaluated at compile time
// ---------------------------------------------------------------------------------------------
namespace cexpr {
constexpr double newton_sqrt(double x, double g, int n) {
    return n == 0 ? g : newton_sqrt(x, 0.5 * (g + x / g), n - 1);
}
constexpr double sqrt(double x) { return newton_sqrt(x, x < 1.0 ? 1.0 : x, 80); }
constexpr double pi = 3.14159265358979323846264338327950288;
}  // namespace cexpr

constexpr float kY00 = float(1.0 / (2.0 * cexpr::sqrt(cexpr::pi)));          // 1 / (2 sqrt(pi))
constexpr float kY1 = float(cexpr::sqrt(3.0 / (4.0 * cexpr::pi)));            // sqrt(3 / 4pi)
constexpr float kY2a = float(cexpr::sqrt(15.0 / cexpr::pi) / 2.0);            // sqrt(15/pi) / 2
constexpr float kY2b = float(cexpr::sqrt(5.0 / cexpr::pi) / 4.0);             // sqrt(5/pi) / 4
constexpr float kY2c = float(cexpr::sqrt(15.0 / cexpr::pi) / 4.0);            // sqrt(15/pi) / 4
constexpr float kY3p = float(cexpr::sqrt(35.0 / (2.0 * cexpr::pi)) / 4.0);    // sqrt(35/2pi) / 4
constexpr float kY3q = float(cexpr::sqrt(105.0 / cexpr::pi) / 2.0);           // sqrt(105/pi) / 2
constexpr float kY3s = float(cexpr::sqrt(21.0 / (2.0 * cexpr::pi)) / 4.0);    // sqrt(21/2pi) / 4
constexpr float kY3u = float(cexpr::sqrt(7.0 / cexpr::pi) / 4.0);             // sqrt(7/pi) / 4
constexpr float kY3v = float(cexpr::sqrt(105.0 / cexpr::pi) / 4.0);           // sqrt(105/pi) / 4

// real SH basis Y_k (k = l^2 + l + m) at the unit direction (x, y, z), degrees 0..deg(K)
template <int K>
__device__ __forceinline__ void sh_basis(float x, float y, float z, float *Y) {
    Y[0] = kY00;
    if constexpr (K > 1) {
        Y[1] = -kY1 * y;
        Y[2] = kY1 * z;
        Y[3] = -kY1 * x;
    }
    if constexpr (K > 4) {
        const float xx = x * x, yy = y * y, zz = z * z;
        Y[4] = kY2a * (x * y);
        Y[5] = -kY2a * (y * z);
        Y[6] = kY2b * (2.f * zz - xx - yy);
        Y[7] = -kY2a * (x * z);
        Y[8] = kY2c * (xx - yy);
        if constexpr (K > 9) {
            Y[9] = -kY3p * y * (3.f * xx - yy);
            Y[10] = kY3q * (x * y) * z;
            Y[11] = -kY3s * y * (4.f * zz - xx - yy);
            Y[12] = kY3u * z * (2.f * zz - 3.f * xx - 3.f * yy);
            Y[13] = -kY3s * x * (4.f * zz - xx - yy);
            Y[14] = kY3v * z * (xx - yy);
            Y[15] = -kY3p * x * (xx - 3.f * yy);
        }
    }
}

// ---------------------------------------------------------------------------------------------
// L2 eviction policies of small launches: the traversal data (ropes, densities, child rows) is
// loaded evict-last and the SH rows evict-first, so that a batch's stream of rows does not push
// the next steps' ropes and densities out of L2 (2^16-ray batches: forward 122.8 -> 116.5 us,
// fused pass 164.3 -> 156.6 us; the full-size launches, whose L2 holds other rays' leaves, are
// slower with it, 8.71 -> 9.25 ms, and keep plain loads)
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ uint64_t l2_policy_last() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t l2_policy_first() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ int32_t ld_hint(const int32_t *a, uint64_t pol) {
    int32_t v;
    asm volatile("ld.global.nc.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ uint32_t ld_hint(const uint32_t *a, uint64_t pol) {
    uint32_t v;
    asm volatile("ld.global.nc.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ uint4 ld_hint(const uint4 *a, uint64_t pol) {
    uint4 v;
    asm volatile("ld.global.nc.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(a), "l"(pol));
    return v;
}
template <typename S> __device__ __forceinline__ float ld_hint_storage(const S *a, uint64_t pol) {
    if constexpr (sizeof(S) == 2) {
        unsigned short h;
        asm volatile("ld.global.nc.L2::cache_hint.b16 %0, [%1], %2;" : "=h"(h) : "l"(a), "l"(pol));
        if constexpr (std::is_same<S, __half>::value) return __half2float(__ushort_as_half(h));
        else return __bfloat162float(__ushort_as_bfloat16(h));
    } else {
        float f;
        asm volatile("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(f) : "l"(a), "l"(pol));
        return f;
    }
}

// ---------------------------------------------------------------------------------------------
// SH rows: [3][K] coefficients in the storage type, padded to 16-byte vectors
// ---------------------------------------------------------------------------------------------
template <typename S, int K> struct Row {
    static constexpr int kBytes = ((3 * K * (int)sizeof(S) + 15) / 16) * 16;
    static constexpr int kVec = kBytes / 16;
};

// z[ch] = sum_k row[ch][k] Y_k in FP32, one 16-byte vector of the row at a time (each channel's
// terms summed in k order); HINT: the row is loaded with L2 policy `pol`
template <typename S, int K, bool HINT = false>
__device__ __forceinline__ void leaf_z(const S *row, const float *Y, float z[3], uint64_t pol = 0) {
    constexpr int E = 16 / (int)sizeof(S);
    const uint4 *p = reinterpret_cast<const uint4 *>(row);
    float acc[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 0; i < Row<S, K>::kVec; i++) {
        uint4 v;
        if constexpr (HINT) v = ld_hint(p + i, pol);
        else v = __ldg(p + i);
        const S *e = reinterpret_cast<const S *>(&v);
#pragma unroll
        for (int j = 0; j < E; j++) {
            const int idx = i * E + j;
            if (idx < 3 * K) acc[idx / K] = fmaf(Storage<S>::to_f32(e[j]), Y[idx % K], acc[idx / K]);
        }
    }
#pragma unroll
    for (int ch = 0; ch < 3; ch++) z[ch] = acc[ch];
}

// requests the 16-byte-aligned SH row into L1 ahead of its use (both ends: a row may straddle
// two 128-byte lines)
template <typename S, int K>
__device__ __forceinline__ void prefetch_row(const S *row) {
    const char *b = reinterpret_cast<const char *>(row);
    asm volatile("prefetch.global.L1 [%0];" ::"l"(b));
    asm volatile("prefetch.global.L1 [%0];" ::"l"(b + Row<S, K>::kBytes - 1));
}

template <bool EXACT> __device__ __forceinline__ float ex(float x) {
    if constexpr (EXACT) return expf(x);
    else return __expf(x);
}

template <bool EXACT> __device__ __forceinline__ float sigmoid(float z) {
    if constexpr (EXACT) return 1.f / (1.f + expf(-z));
    else return __fdividef(1.f, 1.f + __expf(-z));
}

// ---------------------------------------------------------------------------------------------
// plane times
// ---------------------------------------------------------------------------------------------
struct FF {
    float hi, lo;
};
__device__ __forceinline__ bool lt(float a, float b) { return a < b; }
__device__ __forceinline__ bool lt(FF a, FF b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool eq(float a, float b) { return a == b; }
__device__ __forceinline__ bool eq(FF a, FF b) { return a.hi == b.hi && a.lo == b.lo; }
__device__ __forceinline__ float val(float a) { return a; }
__device__ __forceinline__ float val(FF a) { return a.hi + a.lo; }
__device__ __forceinline__ float diff(float a, float b) { return a - b; }
// a - b for close a, b: the high parts subtract exactly (Sterbenz), the low parts add the rest
__device__ __forceinline__ float diff(FF a, FF b) { return (a.hi - b.hi) + (a.lo - b.lo); }
template <typename P> __device__ __forceinline__ P pinf();
template <> __device__ __forceinline__ float pinf<float>() { return __int_as_float(0x7f800000); }
template <> __device__ __forceinline__ FF pinf<FF>() { return FF{__int_as_float(0x7f800000), 0.f}; }
template <typename P> __device__ __forceinline__ P pzero();
template <> __device__ __forceinline__ float pzero<float>() { return 0.f; }
template <> __device__ __forceinline__ FF pzero<FF>() { return FF{0.f, 0.f}; }

// Ray state for plane-time evaluation.  Fast: t(x) = x * inv + c on normalised coordinates.
// Exact: t(x) = (lo + x size - o) / d in world units, as a float-float (error-free product and
// sums, one Newton-corrected quotient).
struct RayAxes {
    float on[3], dn[3];      // normalised origin and direction (root = [0,1]^3)
    int sg[3];               // direction signs
    // fast mode on the 2^16 grid: t(g) = g inv16 + c16 (inv16 = 0, c16 = +inf for a zero
    // direction, so that axis never exits; inv16 > 0 when the exit face is the upper one); grid
    // position at t: t dn16 + on16
    float inv16[3], c16[3], on16[3], dn16[3];
    int upm[3];              // fast mode: -1 where the exit face is the upper one, else 0
    float ow[3], dw[3], invw[3], lo[3], size;  // exact mode
};

template <bool EXACT>
__device__ __forceinline__ typename std::conditional<EXACT, FF, float>::type
plane_t(const RayAxes &r, int a, float x) {
    if constexpr (!EXACT) {
        return fmaf(x * 65536.f, r.inv16[a], r.c16[a]);  // = x inv + c exactly (power-of-2 scaling)
    } else {
        const float p = x * r.size;
        const float pe = fmaf(x, r.size, -p);            // x size = p + pe exactly
        float s = r.lo[a] + p;                            // two-sum(lo, p)
        float bb = s - r.lo[a];
        float e = (r.lo[a] - (s - bb)) + (p - bb);
        e += pe;
        const float m = -r.ow[a];
        float n = s + m;                                   // two-sum(s, -o)
        float b2 = n - s;
        float ne = (s - (n - b2)) + (m - b2);
        ne += e;
        const float q = n * r.invw[a];
        const float rem = fmaf(-q, r.dw[a], n) + ne;      // remainder of the quotient
        const float q2 = rem * r.invw[a];
        const float hi = q + q2;
        return FF{hi, q2 - (hi - q)};
    }
}

// ---------------------------------------------------------------------------------------------
// the march
// ---------------------------------------------------------------------------------------------
struct RayOut {
    float rgb[3];
    float T;
    float loss = 0.f;       // FWDBWD: the ray's squared error summed over channels
    bool overflow = false;  // FWDBWD: more occupied segments than the record holds
    float g[3], rgbf[3];    // BWD in: dL/dC and the forward colour; FWDBWD out: dL/dC
    unsigned long long st[4];  // STATS: hit, steps, occupied, child loads
};

// DEFER: shade each occupied segment one occupied segment later, after prefetching its SH row
// into L1, so that the row's latency overlaps the traversal in between (a gain for launches too
// small to hide latency by occupancy).  COMP: the tree is compressed -- density and palette row
// come from one 32-bit record per leaf and the rows are palette rows.
template <typename S, int K, int MODE, bool EXACT, bool DEFER = false, bool COMP = false>
__device__ __forceinline__ void march_ray(const TreeView &tv, const RenderParams &rp,
                                          const RenderIO &io, int64_t ray, const float ow[3],
                                          const float dw[3], RayOut &out) {
    using PT = typename std::conditional<EXACT, FF, float>::type;
    RayAxes r;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        r.on[a] = (ow[a] - tv.lo[a]) * tv.scale;
        r.dn[a] = dw[a] * tv.scale;
        r.sg[a] = r.dn[a] > 0.f ? 1 : (r.dn[a] < 0.f ? -1 : 0);
        if constexpr (!EXACT) {
            const float inv = 1.f / r.dn[a];
            // scaling by powers of two is exact: plane times equal x inv + c to the bit
            r.inv16[a] = r.sg[a] != 0 ? inv * (1.f / 65536.f) : 0.f;
            r.c16[a] = r.sg[a] != 0 ? -r.on[a] * inv : pinf<float>();
            r.on16[a] = r.on[a] * 65536.f;
            r.dn16[a] = r.dn[a] * 65536.f;
            r.upm[a] = r.sg[a] > 0 ? -1 : 0;
        } else {
            r.ow[a] = ow[a];
            r.dw[a] = dw[a];
            r.invw[a] = 1.f / dw[a];
            r.lo[a] = tv.lo[a];
        }
    }
    if constexpr (EXACT) r.size = tv.size;

    float T = 1.f;
    float C[3] = {0.f, 0.f, 0.f};
    out.T = 1.f;

    // ---- root slab ----
    PT tn = pzero<PT>(), tf = pinf<PT>();
    bool hit = true;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        if (r.sg[a] == 0) {
            if (!(r.on[a] >= 0.f && r.on[a] <= 1.f)) hit = false;
        } else {
            const PT t0 = plane_t<EXACT>(r, a, r.sg[a] > 0 ? 0.f : 1.f);
            const PT t1 = plane_t<EXACT>(r, a, r.sg[a] > 0 ? 1.f : 0.f);
            if (lt(tn, t0)) tn = t0;
            if (lt(t1, tf)) tf = t1;
        }
    }
    if (!hit || !lt(tn, tf)) {
#pragma unroll
        for (int ch = 0; ch < 3; ch++) out.rgb[ch] = rp.bg[ch];
        if constexpr (MODE == kFwdBwd) {
            float loss = 0.f;
#pragma unroll
            for (int ch = 0; ch < 3; ch++) {
                const float e = out.rgb[ch] - __ldg(io.target + 3 * ray + ch);
                out.g[ch] = 2.f * e * io.inv3R;
                loss = fmaf(e, e, loss);
            }
            out.loss = loss;
        }
        return;
    }
    if constexpr (MODE == kStats) out.st[0] += 1;

    constexpr bool SHADE = MODE == kFwd || MODE == kBwd || MODE == kFwdBwd;
    float Y[K];
    if constexpr (SHADE) sh_basis<K>(dw[0], dw[1], dw[2], Y);
    // POST (small forward and fused launches, SH degree 2 and 3): the occupied segments are
    // recorded during the march and shaded after it, in march order, so the lock-step traversal
    // loop carries no shading; the record holds (row, w, Tn, delta), and for the fused pass also
    // each segment's colour.  Rows of degree 0 and 1 are cheap enough to shade in the loop (the
    // tiny degree-1 scene's 2^16-ray fused pass: 36.97 us with the record, 32.85 us without)
    constexpr bool POST = DEFER && (MODE == kFwd || MODE == kFwdBwd) && K >= 9;
    constexpr int RS = MODE == kFwdBwd ? 2 : 1;  // float4 per record entry
    float4 rec[MODE == kFwdBwd ? 2 * kRecordSegments : (POST ? kRecordSegments : 1)];
    int nrec = 0;
    int nshaded = 0;  // POST: record entries shaded so far
    float g[3], rgbf[3];
    if constexpr (MODE == kBwd) {
#pragma unroll
        for (int ch = 0; ch < 3; ch++) {
            g[ch] = out.g[ch];
            rgbf[ch] = out.rgbf[ch];
        }
    }

    // ---- first cell ----
    int gc[3];
    {
        const float t0 = val(tn);
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const float p = fmaf(t0, r.dn[a], r.on[a]);
            const int gi = (int)floorf(p * 65536.f);
            gc[a] = min(max(gi, 0), 65535);
        }
    }

    const S *sigma = reinterpret_cast<const S *>(tv.sigma);
    const S *shp = reinterpret_cast<const S *>(tv.sh);
    // small launches (DEFER): L2 policies of the traversal loads and of the SH rows
    uint64_t pol_keep = 0, pol_stream = 0;
    if constexpr (DEFER) {
        pol_keep = l2_policy_last();
        pol_stream = l2_policy_first();
    }

    // descend from (node, level) to the leaf holding gc.  Table indices fit 32 bits: a tree holds
    // at most 2^27 leaves (the rope encoding) and fewer than 2^28 nodes (import checks the child
    // table), so leaf * 6 + face and node * 8 + slot are formed in 32-bit arithmetic.
    auto descend = [&](int32_t node, int level, int32_t &leaf_out, int &level_out) -> bool {
        int32_t c;
        const int g0 = gc[0] << 2, g1 = gc[1] << 1, g2 = gc[2];  // slot bits land at 4, 2, 1
        while (true) {
            const int sh = kGridBits - 1 - level;
            const int j = ((g0 >> sh) & 4) | ((g1 >> sh) & 2) | ((g2 >> sh) & 1);
            if constexpr (DEFER) c = ld_hint(tv.child + (uint32_t)(node * 8 + j), pol_keep);
            else c = __ldg(tv.child + (uint32_t)(node * 8 + j));
            ++level;
            if constexpr (MODE == kStats) out.st[3] += 1;
            if (c < 0 || level >= tv.max_level) break;
            node = c;
        }
        leaf_out = -1 - c;
        level_out = level;
        return c < 0;  // false: deeper than the tree claims (corrupted table)
    };

    // colour of one occupied segment (weight w, transmittance after it Tn, length delta):
    // C += w c; the backward also scatters dL/dsigma and dL/dSH for it.  Segments are shaded in
    // march order, so C is the prefix sum C_{<=i} the backward needs.
    // gradient of one occupied segment given C = C_{<=i} (colour up to and including it), the
    // ray's dL/dC g and its rendered colour rgbf: dL/dsigma and dL/dSH scattered into the leaf
    auto scatter = [&](int32_t lf, float w, float Tn, float delta, const float col[3]) {
        float acc = 0.f;
        float dz[3];
#pragma unroll
        for (int ch = 0; ch < 3; ch++) {
            const float suffix = rgbf[ch] - C[ch];
            acc = fmaf(g[ch], Tn * col[ch] - suffix, acc);
            const float ag = rp.color_act == DOT_ACT_LINEAR ? 1.f : col[ch] * (1.f - col[ch]);
            dz[ch] = g[ch] * w * ag;
        }
        atomicAdd(io.grad_sigma + lf, delta * acc);
        if (io.touched) io.touched[lf] = 1;
        float *gr = io.grad_sh + (int64_t)lf * (3 * K);
        if constexpr ((3 * K) % 4 == 0) {
            if (io.grad_vec) {
                float4 *g4 = reinterpret_cast<float4 *>(gr);
#pragma unroll
                for (int q = 0; q < 3 * K / 4; q++) {
                    float4 v;
                    v.x = dz[(4 * q + 0) / K] * Y[(4 * q + 0) % K];
                    v.y = dz[(4 * q + 1) / K] * Y[(4 * q + 1) % K];
                    v.z = dz[(4 * q + 2) / K] * Y[(4 * q + 2) % K];
                    v.w = dz[(4 * q + 3) / K] * Y[(4 * q + 3) % K];
                    atomicAdd(g4 + q, v);
                }
            } else {
#pragma unroll
                for (int i = 0; i < 3 * K; i++) atomicAdd(gr + i, dz[i / K] * Y[i % K]);
            }
        } else {
#pragma unroll
            for (int i = 0; i < 3 * K; i++) atomicAdd(gr + i, dz[i / K] * Y[i % K]);
        }
    };

    // colour of one occupied segment (weight w, transmittance after it Tn, length delta):
    // C += w c; the backward also scatters dL/dsigma and dL/dSH for it, the fused mode records
    // it.  Segments are shaded in march order, so C is the prefix sum C_{<=i} the backward needs.
    auto shade = [&](int32_t lf, int64_t row, float w, float Tn, float delta) {
        if constexpr (SHADE) {
            float z[3], col[3];
            leaf_z<S, K, DEFER>(shp + row * tv.row_stride, Y, z, pol_stream);
#pragma unroll
            for (int ch = 0; ch < 3; ch++)
                col[ch] = rp.color_act == DOT_ACT_LINEAR ? z[ch] : sigmoid<EXACT>(z[ch]);
#pragma unroll
            for (int ch = 0; ch < 3; ch++) C[ch] = fmaf(w, col[ch], C[ch]);
            if constexpr (MODE == kBwd) scatter(lf, w, Tn, delta, col);
            if constexpr (MODE == kFwdBwd) {
                if (nrec < kRecordSegments) {
                    rec[2 * nrec] = make_float4(__int_as_float(lf), w, Tn, delta);
                    rec[2 * nrec + 1] = make_float4(col[0], col[1], col[2], 0.f);
                }
                ++nrec;
            }
        }
    };
    // POST: shades record entries [nshaded, upto) in order (their rows were prefetched into L1 when
    // they were recorded)
    auto post_shade = [&](int upto) {
        if constexpr (POST) {
            for (int i = nshaded; i < upto; i++) {
                const float4 a = rec[RS * i];
                float z[3], col[3];
                leaf_z<S, K, DEFER>(shp + (int64_t)__float_as_int(a.x) * tv.row_stride, Y, z, pol_stream);
#pragma unroll
                for (int ch = 0; ch < 3; ch++)
                    col[ch] = rp.color_act == DOT_ACT_LINEAR ? z[ch] : sigmoid<EXACT>(z[ch]);
#pragma unroll
                for (int ch = 0; ch < 3; ch++) C[ch] = fmaf(a.y, col[ch], C[ch]);
                if constexpr (MODE == kFwdBwd) rec[RS * i + 1] = make_float4(col[0], col[1], col[2], 0.f);
            }
            nshaded = upto > nshaded ? upto : nshaded;
        }
    };
    int32_t p_leaf = -1;  // deferred occupied segment (DEFER)
    int64_t p_row = 0;
    float p_w = 0.f, p_Tn = 0.f, p_delta = 0.f;

    PT t = tn;
    int32_t leaf;
    int level;
    int steps = 0;
    if (!descend(0, 0, leaf, level)) {
        atomicOr(io.status, DOT_STATUS_STEP_LIMIT);
        level = -1;
    }
    // Two-stage pipeline per step: the current leaf's density is requested first; the exit face,
    // the next cell and the next leaf's descent are computed while that load is in flight; then
    // the current segment is shaded.
    while (level >= 0) {
        if (steps >= rp.max_steps) {
            atomicOr(io.status, DOT_STATUS_STEP_LIMIT);
            break;
        }
        ++steps;
        float sv;
        int64_t row;  // SH row of the leaf: its own, or its palette entry
        if constexpr (COMP) {
            uint32_t w;
            if constexpr (DEFER) w = ld_hint(tv.rec + leaf, pol_keep);
            else w = __ldg(tv.rec + leaf);
            sv = Storage<S>::from_bits16(w);
            row = w >> 16;
        } else {
            if constexpr (DEFER) sv = ld_hint_storage<S>(sigma + leaf, pol_keep);
            else sv = Storage<S>::load(sigma + leaf);
            row = leaf;
        }
        const int cs = 1 << (kGridBits - level);
        int lo_g[3], bnd[3];
        PT te[3];
        PT tout = pinf<PT>();
        bool outside = false;
        if constexpr (!EXACT) {
            // exit: the nearest of the three faces ahead (a zero direction gives +inf)
            const int msk = -cs;
#pragma unroll
            for (int a = 0; a < 3; a++) {
                lo_g[a] = gc[a] & msk;
                bnd[a] = lo_g[a] + (cs & r.upm[a]);  // the exit plane on this axis
                te[a] = fmaf((float)bnd[a], r.inv16[a], r.c16[a]);
            }
            tout = fminf(fminf(te[0], te[1]), te[2]);
        } else {
#pragma unroll
            for (int a = 0; a < 3; a++) {
                lo_g[a] = gc[a] & ~(cs - 1);
                if (r.sg[a] != 0) {
                    const int f = r.sg[a] > 0 ? lo_g[a] + cs : lo_g[a];
                    te[a] = plane_t<EXACT>(r, a, (float)f * (1.f / 65536.f));
                    if (lt(te[a], tout)) tout = te[a];
                } else {
                    te[a] = pinf<PT>();
                }
            }
        }
        if (!(val(tout) < pinf<float>())) break;  // only for a zero direction
        const float delta = diff(tout, t);

        // ---- next cell and its leaf ----
        const float toutv = val(tout);
        int crossed = 0, face = 0;  // faces crossed at tout; the last one (2 axis + upper)
        if constexpr (!EXACT) {
#pragma unroll
            for (int a = 0; a < 3; a++) {
                // across every face hit at tout (the plane itself upwards, the cell below it
                // downwards); on the other axes the exit point, clamped into the old cell
                const bool x = te[a] == tout;
                const int gi = (int)floorf(fmaf(toutv, r.dn16[a], r.on16[a]));
                const int in = min(max(gi, lo_g[a]), lo_g[a] + cs - 1);
                gc[a] = x ? bnd[a] + ~r.upm[a] : in;
                crossed += x ? 1 : 0;
                face = x ? 2 * a + (r.upm[a] & 1) : face;
            }
            outside = ((gc[0] | gc[1] | gc[2]) & ~65535) != 0;
        } else {
#pragma unroll
            for (int a = 0; a < 3; a++) {
                if (r.sg[a] != 0 && eq(te[a], tout)) {
                    gc[a] = r.sg[a] > 0 ? lo_g[a] + cs : lo_g[a] - 1;
                    outside |= (gc[a] < 0) | (gc[a] > 65535);
                    ++crossed;
                    face = 2 * a + (r.sg[a] > 0 ? 1 : 0);
                } else {
                    const float p = fmaf(toutv, r.dn[a], r.on[a]);
                    const int gi = (int)floorf(p * 65536.f);
                    gc[a] = min(max(gi, lo_g[a]), lo_g[a] + cs - 1);
                }
            }
        }
        int32_t next_leaf = 0;
        int next_level = -1;
        if (!outside) {
            bool found;
            if (crossed == 1) {  // across one face: its rope
                int32_t rp;
                if constexpr (DEFER) rp = ld_hint(tv.rope + (uint32_t)(leaf * 6 + face), pol_keep);
                else rp = __ldg(tv.rope + (uint32_t)(leaf * 6 + face));
                if constexpr (MODE == kStats) out.st[3] += 1;
                if (rp >= 0) {  // the node at this leaf's level: descend into the finer neighbour
                    found = rp < tv.n_nodes && descend(rp, level, next_leaf, next_level);
                } else {        // a leaf at this level or coarser (INT32_MIN, outside, fails here)
                    const int32_t code = -1 - rp;
                    next_leaf = code >> kRopeLevelBits;
                    next_level = level - (code & ((1 << kRopeLevelBits) - 1));
                    found = next_leaf < tv.n_leaves && rp != INT32_MIN;
                }
            } else {  // across an edge or a corner: from the root
                found = descend(0, 0, next_leaf, next_level);
            }
            if (!found) {
                atomicOr(io.status, DOT_STATUS_STEP_LIMIT);
                next_level = -1;
            }
        }

        // ---- the current segment: density now, colour now or one occupied segment later ----
        if constexpr (MODE == kStats) out.st[1] += 1;
        bool stop = false;
        if (delta > 0.f && sv > 0.f) {
            if constexpr (MODE == kStats) out.st[2] += 1;
            const float e = ex<EXACT>(-(sv * delta));
            const float alpha = 1.f - e;
            const float w = T * alpha;
            if constexpr (SHADE) {
                if constexpr (POST) {
                    if (nrec < kRecordSegments) {
                        prefetch_row<S, K>(shp + row * tv.row_stride);
                        rec[RS * nrec] = make_float4(__int_as_float((int32_t)row), w, T * e, delta);
                        ++nrec;
                    } else {  // record full: shade it now, in order, then this segment in place
                        if (nshaded < kRecordSegments) post_shade(kRecordSegments);
                        shade(leaf, row, w, T * e, delta);
                    }
                } else if constexpr (DEFER) {
                    prefetch_row<S, K>(shp + row * tv.row_stride);
                    if (p_leaf >= 0) shade(p_leaf, p_row, p_w, p_Tn, p_delta);
                    p_leaf = leaf;
                    p_row = row;
                    p_w = w;
                    p_Tn = T * e;
                    p_delta = delta;
                } else {
                    shade(leaf, row, w, T * e, delta);
                }
            }
            if (MODE != kStats && io.signal != nullptr) {
                if (rp.signal_mode == DOT_SIGNAL_SUM_ALPHA) atomicAdd(io.signal + leaf, alpha);
                else if (rp.signal_mode == DOT_SIGNAL_MAX_WEIGHT)
                    atomicMax(reinterpret_cast<int *>(io.signal) + leaf, __float_as_int(w));
            }
            T = T * e;
            stop = T < rp.eps_T;
        }
        if (stop || outside) break;
        if (lt(t, tout)) t = tout;
        leaf = next_leaf;
        level = next_level;
    }
    if constexpr (POST) {
        post_shade(nrec < kRecordSegments ? nrec : kRecordSegments);
    } else if constexpr (DEFER && SHADE) {
        if (p_leaf >= 0) shade(p_leaf, p_row, p_w, p_Tn, p_delta);
    }
#pragma unroll
    for (int ch = 0; ch < 3; ch++) out.rgb[ch] = fmaf(T, rp.bg[ch], C[ch]);
    out.T = T;
    if constexpr (MODE == kFwdBwd) {
        // MSE gradient of this ray, then the backward from the record of its occupied segments
        float loss = 0.f;
#pragma unroll
        for (int ch = 0; ch < 3; ch++) {
            rgbf[ch] = out.rgb[ch];
            const float e = rgbf[ch] - __ldg(io.target + 3 * ray + ch);
            g[ch] = 2.f * e * io.inv3R;
            loss = fmaf(e, e, loss);
            out.g[ch] = g[ch];
        }
        out.loss = loss;
        if (nrec <= kRecordSegments) {
#pragma unroll
            for (int ch = 0; ch < 3; ch++) C[ch] = 0.f;
            // the record is read kScatterAhead entries at a time, all loads issued before the
            // first of them is used (one record round trip per group, not per segment: 173.6 ->
            // 165.7 us per 2^16-ray pass; 2 entries 168.3)
            constexpr int kScatterAhead = 4;
            for (int i0 = 0; i0 < nrec; i0 += kScatterAhead) {
                float4 a[kScatterAhead], b[kScatterAhead];
#pragma unroll
                for (int u = 0; u < kScatterAhead; u++) {
                    if (i0 + u < nrec) {
                        a[u] = rec[2 * (i0 + u)];
                        b[u] = rec[2 * (i0 + u) + 1];
                    }
                }
#pragma unroll
                for (int u = 0; u < kScatterAhead; u++) {
                    if (i0 + u < nrec) {
                        const float col[3] = {b[u].x, b[u].y, b[u].z};
#pragma unroll
                        for (int ch = 0; ch < 3; ch++) C[ch] = fmaf(a[u].y, col[ch], C[ch]);
                        scatter(__float_as_int(a[u].x), a[u].y, a[u].z, a[u].w, col);
                    }
                }
            }
        } else {
            out.overflow = true;  // the caller re-marches this ray in the backward mode
        }
    }
}

// ray of a thread: pinhole pixel (bit-exact float32 recipe of dot_camera) or a buffer entry
__device__ __forceinline__ void camera_ray(const dot_camera *cam, int i, int j, float o[3], float d[3]) {
    const float fx = __ldg(&cam->fx), fy = __ldg(&cam->fy), cx = __ldg(&cam->cx), cy = __ldg(&cam->cy);
    const float xc = __fdiv_rn(__fsub_rn(__fadd_rn((float)i, 0.5f), cx), fx);
    const float yc = -__fdiv_rn(__fsub_rn(__fadd_rn((float)j, 0.5f), cy), fy);
    float e[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const float r0 = __ldg(&cam->c2w[4 * a + 0]), r1 = __ldg(&cam->c2w[4 * a + 1]);
        const float r2 = __ldg(&cam->c2w[4 * a + 2]);
        e[a] = __fsub_rn(__fadd_rn(__fmul_rn(r0, xc), __fmul_rn(r1, yc)), r2);
        o[a] = __ldg(&cam->c2w[4 * a + 3]);
    }
    const float n2 = __fadd_rn(__fadd_rn(__fmul_rn(e[0], e[0]), __fmul_rn(e[1], e[1])), __fmul_rn(e[2], e[2]));
    const float inv = __fdiv_rn(1.f, __fsqrt_rn(n2));
#pragma unroll
    for (int a = 0; a < 3; a++) d[a] = __fmul_rn(e[a], inv);
}

// Tile of pixels covered by a block of NT threads in camera mode: warps of 8x4 pixels, two
// warps side by side when there are several (8 warps: 16x16, 4: 16x8, 2: 16x4, 1: 8x4).
template <int NT> struct CamTile {
    static constexpr int kWarps = NT / 32;
    static constexpr int kW = kWarps >= 2 ? 16 : 8;
    static constexpr int kH = kWarps >= 2 ? 4 * (kWarps / 2) : 4;
};

// MINB: minimum resident blocks per SM requested from the register allocator (MINB x NT = 1024
// threads: at most 64 registers, 32 warps per SM, for launches large enough to fill the GPU
// several times over; a single block's worth for small launches, whose time is the longest
// ray's latency).
template <typename S, int K, int MODE, bool EXACT, int MINB, int NT = kMarchThreads,
          bool DEFER = false, bool COMP = false>
__global__ void __launch_bounds__(NT, MINB)
march_kernel(TreeView tv, RaySource rs, RenderParams rp, RenderIO io) {

    int64_t ray;
    bool valid;
    float ow[3], dw[3];
    if (rs.kind == DOT_RAYS_CAMERAS) {
        using TL = CamTile<NT>;
        const int tx = blockIdx.x % rs.tiles_x, ty = blockIdx.x / rs.tiles_x;
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const int px = tx * TL::kW + (warp % (TL::kW / 8)) * 8 + (lane & 7);
        const int py = ty * TL::kH + (warp / (TL::kW / 8)) * 4 + (lane >> 3);
        valid = px < rs.width && py < rs.height;
        int v = blockIdx.y;
        if (rs.order) {
            v = __ldg(rs.order + blockIdx.y);
            if (v < 0 || v >= rs.n_cams) {
                if (threadIdx.x == 0) atomicOr(io.status, DOT_STATUS_BAD_INPUT);
                return;
            }
        }
        ray = ((int64_t)v * rs.height + py) * rs.width + px;
        if (valid) camera_ray(rs.cams + v, px, py, ow, dw);
    } else {
        ray = (int64_t)blockIdx.x * NT + threadIdx.x;
        valid = ray < rs.n_rays;
        if (valid) {
#pragma unroll
            for (int a = 0; a < 3; a++) {
                ow[a] = __ldg(rs.origins + 3 * ray + a);
                dw[a] = __ldg(rs.dirs + 3 * ray + a);
            }
        }
    }
    RayOut out;
    out.st[0] = out.st[1] = out.st[2] = out.st[3] = 0;
    if (valid) {
        if constexpr (MODE == kBwd) {
#pragma unroll
            for (int ch = 0; ch < 3; ch++) {
                out.g[ch] = __ldg(io.grad_rgb + 3 * ray + ch);
                out.rgbf[ch] = __ldg(io.rgb_fwd + 3 * ray + ch);
            }
        }
        march_ray<S, K, MODE, EXACT, DEFER, COMP>(tv, rp, io, ray, ow, dw, out);
        if constexpr (MODE == kFwd && DOT_STREAM_OUT) {
            // the images are written once and not read here: evict-first keeps L2 for the tree
#pragma unroll
            for (int ch = 0; ch < 3; ch++) __stcs(io.rgb + 3 * ray + ch, out.rgb[ch]);
            if (io.T_final) __stcs(io.T_final + ray, out.T);
        } else if constexpr (MODE == kFwd || MODE == kFwdBwd) {
#pragma unroll
            for (int ch = 0; ch < 3; ch++) io.rgb[3 * ray + ch] = out.rgb[ch];
            if (io.T_final) io.T_final[ray] = out.T;
        }
        if constexpr (MODE == kFwdBwd) {
#pragma unroll
            for (int ch = 0; ch < 3; ch++) io.grad_out[3 * ray + ch] = out.g[ch];
            if (out.overflow) {  // too many occupied segments to record: march again backward
                RayOut b;
#pragma unroll
                for (int ch = 0; ch < 3; ch++) {
                    b.g[ch] = out.g[ch];
                    b.rgbf[ch] = out.rgb[ch];
                }
                RenderParams rb = rp;
                rb.signal_mode = DOT_SIGNAL_NONE;
                RenderIO ib = io;
                ib.signal = nullptr;
                march_ray<S, K, kBwd, EXACT, DEFER, COMP>(tv, rb, ib, ray, ow, dw, b);
            }
        }
    }
    if constexpr (MODE == kFwdBwd) {
        if (io.loss_sum) {  // block sum of the squared errors, one double atomic per block
            __shared__ double s_loss[NT / 32];
            float l = valid ? out.loss : 0.f;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) l += __shfl_down_sync(0xffffffffu, l, off);
            if ((threadIdx.x & 31) == 0) s_loss[threadIdx.x >> 5] = (double)l * io.inv3R;
            __syncthreads();
            if (threadIdx.x == 0) {
                double b = 0.0;
#pragma unroll
                for (int w = 0; w < NT / 32; w++) b += s_loss[w];
                if (b != 0.0) atomicAdd(io.loss_sum, b);
            }
        }
    }
    if constexpr (MODE == kStats) {
#pragma unroll
        for (int i = 0; i < 4; i++) {
            unsigned long long v = out.st[i];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
            if ((threadIdx.x & 31) == 0 && v) atomicAdd(io.stats + i, v);
        }
    }
}

}  // namespace dot
