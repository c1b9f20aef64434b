// compress.cu -- compressed models (Sec. 4.1): every leaf's SH coefficient row is replaced by one
// of 2^bits palette rows found by median cut (Heckbert 1982) over the leaves' coefficient vectors,
// and the leaf keeps a 16-bit palette index next to its 16-bit density in one 32-bit record, so a
// rendered segment reads 4 bytes per leaf plus a palette row that stays resident in L2
// (2^16 rows x 96 bytes = 6.3 MB at SH degree 3).
//
// The quantiser is an offline step and runs on the host: copy the rows out, median cut, write the
// palette and the records back.  Median cut rules: each of the bits rounds splits every box of two
// or more vectors at the median of its longest axis (largest max - min, computed in double; ties
// to the lowest axis), the members ordered by (value on that axis, leaf id), floor(m/2) of them
// to child 2b and the rest to child 2b + 1; a palette row is the mean of its box (zeros if empty),
// rounded to the storage type.
#include <algorithm>
#include <thread>
#include <vector>

#include "internal.cuh"
#include "tree.cuh"

namespace dot {

namespace {

float bits_to_float(uint16_t b, int storage) {
    if (storage == DOT_STORAGE_F16) {
        __half_raw r;
        r.x = b;
        return __half2float(__half(r));
    }
    __nv_bfloat16_raw r;
    r.x = b;
    return __bfloat162float(__nv_bfloat16(r));
}

uint16_t double_to_bits(double v, int storage) {
    if (storage == DOT_STORAGE_F16) {
        __half_raw r = __double2half(v);
        return r.x;
    }
    __nv_bfloat16_raw r = __double2bfloat16(v);
    return r.x;
}

template <typename F>
void parallel_for(int64_t n, F &&f) {
    const int64_t hw = std::max(1u, std::thread::hardware_concurrency());
    const int64_t nt = std::min<int64_t>(hw, n);
    if (nt <= 1) {
        for (int64_t i = 0; i < n; i++) f(i);
        return;
    }
    std::vector<std::thread> th;
    for (int64_t t = 0; t < nt; t++)
        th.emplace_back([&, t] {
            for (int64_t i = t; i < n; i += nt) f(i);
        });
    for (auto &x : th) x.join();
}

// x: n vectors of dim floats (exact copies of 16-bit values); index[n] and palette[P][dim]
void median_cut(int64_t n, int dim, const float *x, int bits, std::vector<int32_t> &index,
                std::vector<double> &palette) {
    const int64_t P = int64_t(1) << bits;
    std::vector<int64_t> order(n);
    for (int64_t i = 0; i < n; i++) order[i] = i;
    std::vector<int64_t> start{0, n}, next;
    for (int r = 0; r < bits; r++) {
        const int64_t boxes = (int64_t)start.size() - 1;
        next.assign(2 * boxes + 1, 0);
        parallel_for(boxes, [&](int64_t b) {
            const int64_t s = start[b], e = start[b + 1], m = e - s;
            next[2 * b] = s;
            if (m < 2) {
                next[2 * b + 1] = e;
                return;
            }
            std::vector<float> lo(x + order[s] * dim, x + order[s] * dim + dim), hi = lo;
            for (int64_t k = s + 1; k < e; k++) {
                const float *v = x + order[k] * dim;
                for (int d = 0; d < dim; d++) {
                    lo[d] = std::min(lo[d], v[d]);
                    hi[d] = std::max(hi[d], v[d]);
                }
            }
            int axis = 0;
            double best = -1.0;
            for (int d = 0; d < dim; d++) {
                const double range = (double)hi[d] - (double)lo[d];
                if (range > best) {
                    best = range;
                    axis = d;
                }
            }
            std::nth_element(order.begin() + s, order.begin() + s + m / 2, order.begin() + e,
                             [&](int64_t i, int64_t j) {
                                 const float u = x[i * dim + axis], w = x[j * dim + axis];
                                 return u < w || (u == w && i < j);
                             });
            next[2 * b + 1] = s + m / 2;
        });
        next[2 * boxes] = n;
        start.swap(next);
    }
    index.assign(n, 0);
    palette.assign(P * dim, 0.0);
    parallel_for(P, [&](int64_t b) {
        const int64_t s = start[b], e = start[b + 1];
        double *row = palette.data() + b * dim;
        for (int64_t k = s; k < e; k++) {
            index[order[k]] = (int32_t)b;
            const float *v = x + order[k] * dim;
            for (int d = 0; d < dim; d++) row[d] += (double)v[d];
        }
        if (e > s)
            for (int d = 0; d < dim; d++) row[d] /= (double)(e - s);
    });
}

}  // namespace

cudaError_t compress_tree(TreeArrays &a, int bits, const DevAlloc &al, cudaStream_t s) {
    const int64_t L = a.n_leaves, P = int64_t(1) << bits;
    const int dim = 3 * a.K, rs = a.row_stride;
    std::vector<uint16_t> rows((size_t)L * rs), sig((size_t)L);
    cudaError_t e = cudaSuccess;
    if (L > 0) {
        e = cudaMemcpyAsync(rows.data(), a.sh, (size_t)L * rs * 2, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(sig.data(), a.sigma, (size_t)L * 2, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return e;
    }
    std::vector<float> x((size_t)L * dim);
    parallel_for(L, [&](int64_t v) {
        for (int d = 0; d < dim; d++) x[v * dim + d] = bits_to_float(rows[v * rs + d], a.storage);
    });
    std::vector<int32_t> index;
    std::vector<double> pal;
    median_cut(L, dim, x.data(), bits, index, pal);
    std::vector<uint16_t> prow((size_t)P * rs, 0);
    for (int64_t b = 0; b < P; b++)
        for (int d = 0; d < dim; d++) prow[b * rs + d] = double_to_bits(pal[b * dim + d], a.storage);
    std::vector<uint32_t> rec((size_t)L);
    for (int64_t v = 0; v < L; v++) rec[v] = (uint32_t)sig[v] | ((uint32_t)index[v] << 16);

    void *palette = al.alloc((size_t)P * rs * 2, s);
    uint32_t *leaf_rec = (uint32_t *)al.alloc((size_t)std::max<int64_t>(L, 1) * 4, s);
    if (!palette || !leaf_rec) {
        al.release(palette, s);
        al.release(leaf_rec, s);
        return cudaErrorMemoryAllocation;
    }
    e = cudaMemcpyAsync(palette, prow.data(), (size_t)P * rs * 2, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && L > 0)
        e = cudaMemcpyAsync(leaf_rec, rec.data(), (size_t)L * 4, cudaMemcpyHostToDevice, s);
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
