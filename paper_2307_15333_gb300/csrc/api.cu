// api.cu -- the extern "C" entry points of libdot (include/dot.h): argument checks on the host,
// tree lifecycle, import / export, and dispatch to the kernels.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "internal.cuh"
#include "tree.cuh"

struct dot_tree {
    int device = 0;
    dot::DevAlloc alloc;
    dot::TreeArrays a;
    float center[3] = {0, 0, 0};
    float half_size = 1.f;
    uint32_t *status = nullptr;
};

namespace dot {
cudaError_t launch_march_fwd(int storage, int deg, bool exact, const TreeView &tv,
                             const RaySource &rs, const RenderParams &rp, const RenderIO &io,
                             cudaStream_t stream);
cudaError_t launch_march_bwd(int storage, int deg, bool exact, const TreeView &tv,
                             const RaySource &rs, const RenderParams &rp, const RenderIO &io,
                             cudaStream_t stream);
cudaError_t launch_march_signal(int storage, bool exact, const TreeView &tv, const RaySource &rs,
                                const RenderParams &rp, const RenderIO &io, cudaStream_t stream);
cudaError_t launch_march_fwdbwd(int storage, int deg, bool exact, const TreeView &tv,
                                const RaySource &rs, const RenderParams &rp, const RenderIO &io,
                                cudaStream_t stream);
cudaError_t launch_march_stats(int storage, bool exact, const TreeView &tv, const RaySource &rs,
                               const RenderParams &rp, const RenderIO &io, cudaStream_t stream);
cudaError_t compress_tree(TreeArrays &a, int bits, const DevAlloc &al, cudaStream_t s);
cudaError_t launch_rmsprop_sparse(int storage, void *sigma, void *sh, int64_t L, int K,
                                  int row_stride, float *grad_sigma, float *grad_sh,
                                  float *ms_sigma, float *ms_sh, uint8_t *touched, int32_t *last,
                                  int32_t step, int32_t *work, const dot_rmsprop_opts &op,
                                  cudaStream_t s);
cudaError_t launch_rmsprop_flush(int64_t L, int K, float *ms_sigma, float *ms_sh, int32_t *last,
                                 int32_t step, float rho, cudaStream_t s);
cudaError_t canonicalize_tree(const TreeArrays &old, TreeArrays *out, const DevAlloc &alloc,
                              int32_t *perm, const dot_leaf_array *aux, int n_aux, cudaStream_t s);
cudaError_t launch_mse_grad(const float *rgb, const float *target, int64_t n_rays, float *grad,
                            double *loss_sum, cudaStream_t s);
cudaError_t launch_rmsprop(int storage, void *sigma, void *sh, int64_t L, int K, int row_stride,
                           float *grad_sigma, float *grad_sh, float *ms_sigma, float *ms_sh,
                           const dot_rmsprop_opts &op, cudaStream_t s);
}  // namespace dot

namespace {

thread_local std::string g_err;

int fail(int code, const std::string &msg) {
    g_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *where) {
    cudaGetLastError();
    if (e == cudaErrorNotSupported) {  // the library's own capacity limits
        g_err = std::string(where) + ": the tree would exceed 2^27 leaves";
        return DOT_ERR_UNSUPPORTED;
    }
    g_err = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return e == cudaErrorMemoryAllocation ? DOT_ERR_OOM : DOT_ERR_CUDA;
}

#define API_CK(call, where)                                   \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(e_, where);   \
    } while (0)

cudaStream_t S(void *stream) { return reinterpret_cast<cudaStream_t>(stream); }

int check_tree(const dot_tree *t) {
    if (!t) return fail(DOT_ERR_INVALID_ARG, "tree is NULL");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return cuda_fail(cudaGetLastError(), "cudaGetDevice");
    if (dev != t->device) return fail(DOT_ERR_INVALID_ARG, "the current device is not the tree's device");
    return DOT_OK;
}

// calls that read or write per-leaf SH rows do not apply to a compressed tree
int check_uncompressed(const dot_tree *t, const char *what) {
    if (t->a.leaf_rec)
        return fail(DOT_ERR_UNSUPPORTED, std::string(what) + ": the tree's SH rows are compressed "
                                         "(rendering only)");
    return DOT_OK;
}

int make_alloc(const dot_allocator *alloc, dot::DevAlloc &out) {
    if (alloc) {
        if (!alloc->alloc || !alloc->free)
            return fail(DOT_ERR_INVALID_ARG, "allocator needs both alloc and free");
        out.user = *alloc;
        out.has_user = true;
    }
    return DOT_OK;
}

int new_tree(const dot::DevAlloc &al, cudaStream_t s, dot_tree **out) {
    dot_tree *t = new dot_tree();
    if (cudaGetDevice(&t->device) != cudaSuccess) {
        delete t;
        return cuda_fail(cudaGetLastError(), "cudaGetDevice");
    }
    t->alloc = al;
    t->status = (uint32_t *)al.alloc(16, s);
    if (!t->status) {
        delete t;
        return fail(DOT_ERR_OOM, "could not allocate the tree status word");
    }
    cudaError_t e = cudaMemsetAsync(t->status, 0, 16, s);
    if (e != cudaSuccess) {
        al.release(t->status, s);
        delete t;
        return cuda_fail(e, "cudaMemsetAsync");
    }
    *out = t;
    return DOT_OK;
}

void destroy_tree(dot_tree *t) {
    cudaDeviceSynchronize();
    dot::free_tree_arrays(t->a, t->alloc, 0);
    t->alloc.release(t->status, 0);
    cudaStreamSynchronize(0);
    delete t;
}

dot::TreeView view_of(const dot_tree *t) {
    dot::TreeView tv;
    tv.child = t->a.child;
    tv.sigma = t->a.sigma;
    tv.sh = t->a.leaf_rec ? t->a.palette : t->a.sh;
    tv.rec = t->a.leaf_rec;
    tv.rope = t->a.rope;
    tv.n_nodes = t->a.n_nodes;
    tv.n_leaves = t->a.n_leaves;
    tv.row_stride = t->a.row_stride;
    tv.max_level = t->a.max_level;
    for (int a = 0; a < 3; a++) tv.lo[a] = t->center[a] - t->half_size;
    tv.size = 2.f * t->half_size;
    tv.scale = 1.f / tv.size;
    return tv;
}

int make_rays(const dot_rays *rays, dot::RaySource &rs, int64_t &n_rays) {
    if (!rays) return fail(DOT_ERR_INVALID_ARG, "rays is NULL");
    std::memset(&rs, 0, sizeof(rs));
    rs.kind = rays->kind;
    if (rays->kind == DOT_RAYS_BUFFER) {
        if (rays->n_rays < 0) return fail(DOT_ERR_INVALID_ARG, "n_rays < 0");
        if (rays->n_rays > 0 && (!rays->origins || !rays->dirs))
            return fail(DOT_ERR_INVALID_ARG, "ray buffers are NULL");
        if (rays->n_rays > ((int64_t)1 << 40)) return fail(DOT_ERR_INVALID_ARG, "too many rays");
        rs.origins = rays->origins;
        rs.dirs = rays->dirs;
        rs.n_rays = rays->n_rays;
        n_rays = rays->n_rays;
        return DOT_OK;
    }
    if (rays->kind == DOT_RAYS_CAMERAS) {
        if (rays->n_cameras < 0 || rays->n_cameras > 65535)
            return fail(DOT_ERR_INVALID_ARG, "n_cameras must be in [0, 65535]");
        if (rays->n_cameras > 0 && !rays->cameras) return fail(DOT_ERR_INVALID_ARG, "cameras is NULL");
        if (rays->width <= 0 || rays->height <= 0 || rays->width > 65536 || rays->height > 65536)
            return fail(DOT_ERR_INVALID_ARG, "camera width / height out of range");
        rs.cams = rays->cameras;
        rs.order = rays->view_order;
        rs.n_cams = rays->n_cameras;
        rs.width = rays->width;
        rs.height = rays->height;
        rs.tiles_x = (rays->width + 15) / 16;
        n_rays = (int64_t)rays->n_cameras * rays->width * rays->height;
        rs.n_rays = n_rays;
        return DOT_OK;
    }
    return fail(DOT_ERR_INVALID_ARG, "unknown rays kind");
}

int make_params(const dot_tree *t, const dot_render_opts *o, dot::RenderParams &rp, bool &exact) {
    if (!o) return fail(DOT_ERR_INVALID_ARG, "opts is NULL");
    if (!(o->eps_T >= 0.f && o->eps_T < 1.f)) return fail(DOT_ERR_INVALID_ARG, "eps_T must be in [0, 1)");
    if (o->color_act != DOT_ACT_SIGMOID && o->color_act != DOT_ACT_LINEAR)
        return fail(DOT_ERR_INVALID_ARG, "unknown color_act");
    if (o->signal_mode < DOT_SIGNAL_NONE || o->signal_mode > DOT_SIGNAL_MAX_WEIGHT)
        return fail(DOT_ERR_INVALID_ARG, "signal_mode of a render call must be NONE, SUM_ALPHA or MAX_WEIGHT");
    if (o->precision < DOT_PRECISION_AUTO || o->precision > DOT_PRECISION_EXACT)
        return fail(DOT_ERR_INVALID_ARG, "unknown precision");
    if (o->max_steps < 0) return fail(DOT_ERR_INVALID_ARG, "max_steps < 0");
    for (int c = 0; c < 3; c++) {
        if (!std::isfinite(o->background[c])) return fail(DOT_ERR_INVALID_ARG, "background not finite");
        rp.bg[c] = o->background[c];
    }
    rp.eps_T = o->eps_T;
    rp.color_act = o->color_act;
    rp.signal_mode = o->signal_mode;
    rp.max_steps = o->max_steps ? o->max_steps : 3 * (1 << t->a.max_level) + 64;
    exact = o->precision == DOT_PRECISION_EXACT ||
            (o->precision == DOT_PRECISION_AUTO && t->a.storage == DOT_STORAGE_F32);
    return DOT_OK;
}

int key_level_host(uint64_t key) {
    int b = -1;
    while (key) {
        key >>= 1;
        b++;
    }
    return b / 3;
}

}  // namespace

extern "C" {

const char *dot_last_error(void) { return g_err.c_str(); }

int dot_version(void) { return 100; }

int dot_octree_build(const dot_build_desc *desc, const dot_allocator *alloc, void *stream,
                     dot_tree **out) {
    if (!desc || !out) return fail(DOT_ERR_INVALID_ARG, "desc and out must not be NULL");
    if (desc->max_depth < 1 || desc->max_depth > dot::kMaxLevels)
        return fail(DOT_ERR_INVALID_ARG, "max_depth must be in [1, 16]");
    if (desc->sh_degree < 0 || desc->sh_degree > 3)
        return fail(DOT_ERR_UNSUPPORTED, "sh_degree must be in [0, 3]");
    if (desc->storage < DOT_STORAGE_F32 || desc->storage > DOT_STORAGE_BF16)
        return fail(DOT_ERR_INVALID_ARG, "unknown storage type");
    if (desc->n_primitives < 0 || desc->n_primitives > dot::kMaxPrimitives)
        return fail(DOT_ERR_INVALID_ARG, "n_primitives must be in [0, 4096]");
    if (desc->n_primitives > 0 && !desc->primitives)
        return fail(DOT_ERR_INVALID_ARG, "primitives is NULL");
    if (!(desc->half_size > 0.f) || !std::isfinite(desc->half_size))
        return fail(DOT_ERR_INVALID_ARG, "half_size must be positive and finite");
    for (int a = 0; a < 3; a++)
        if (!std::isfinite(desc->center[a])) return fail(DOT_ERR_INVALID_ARG, "center not finite");
    if (!std::isfinite(desc->density_lo) || !std::isfinite(desc->density_hi) ||
        !std::isfinite(desc->sh_std) || !std::isfinite(desc->sh_dc))
        return fail(DOT_ERR_INVALID_ARG, "parameter distribution not finite");
    for (int i = 0; i < desc->n_primitives; i++) {
        const dot_primitive &p = desc->primitives[i];
        if (p.type < DOT_PRIM_SPHERE || p.type > DOT_PRIM_CYLINDER)
            return fail(DOT_ERR_INVALID_ARG, "unknown primitive type");
        for (int k = 0; k < 7; k++)
            if (p.p[k] < -((int64_t)1 << 30) || p.p[k] > ((int64_t)1 << 30))
                return fail(DOT_ERR_INVALID_ARG, "primitive parameter out of range (|p| <= 2^30)");
    }
    dot::DevAlloc al;
    int rc = make_alloc(alloc, al);
    if (rc) return rc;
    dot_tree *t = nullptr;
    rc = new_tree(al, S(stream), &t);
    if (rc) return rc;
    for (int a = 0; a < 3; a++) t->center[a] = desc->center[a];
    t->half_size = desc->half_size;
    cudaError_t e = dot::build_tree(*desc, t->a, al, S(stream));
    if (e != cudaSuccess) {
        int r = cuda_fail(e, "dot_octree_build");
        destroy_tree(t);
        return r;
    }
    *out = t;
    return DOT_OK;
}

int dot_tree_free(dot_tree *tree) {
    if (!tree) return DOT_OK;
    destroy_tree(tree);
    return DOT_OK;
}

int dot_tree_get_info(const dot_tree *t, dot_tree_info *info) {
    if (!t || !info) return fail(DOT_ERR_INVALID_ARG, "tree and info must not be NULL");
    std::memset(info, 0, sizeof(*info));
    info->n_nodes = t->a.n_nodes;
    info->n_leaves = t->a.n_leaves;
    info->max_level = t->a.max_level;
    info->sh_degree = t->a.sh_degree;
    info->n_coeffs = t->a.K;
    info->storage = t->a.storage;
    info->sh_row_stride = t->a.row_stride;
    for (int a = 0; a < 3; a++) info->center[a] = t->center[a];
    info->half_size = t->half_size;
    info->child = t->a.child;
    info->node_parent = t->a.node_parent;
    info->node_key = t->a.node_key;
    info->leaf_parent = t->a.leaf_parent;
    info->leaf_key = t->a.leaf_key;
    info->sigma = t->a.sigma;
    info->sh = t->a.sh;
    info->palette_bits = t->a.palette_bits;
    info->palette = t->a.palette;
    info->leaf_record = t->a.leaf_rec;
    info->rope = t->a.rope;
    return DOT_OK;
}

int dot_tree_export(const dot_tree *t, void *stream, int32_t *child, int32_t *node_parent,
                    uint64_t *node_key, int32_t *leaf_parent, uint64_t *leaf_key, void *sigma,
                    void *sh) {
    int rc = check_tree(t);
    if (rc) return rc;
    cudaStream_t s = S(stream);
    const auto &a = t->a;
    const size_t sb = (size_t)dot::storage_bytes(a.storage);
    auto cp = [&](void *dst, const void *src, size_t bytes) -> cudaError_t {
        if (!dst || bytes == 0) return cudaSuccess;
        return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s);
    };
    API_CK(cp(child, a.child, (size_t)a.n_nodes * 8 * 4), "export child");
    API_CK(cp(node_parent, a.node_parent, (size_t)a.n_nodes * 4), "export node_parent");
    API_CK(cp(node_key, a.node_key, (size_t)a.n_nodes * 8), "export node_key");
    API_CK(cp(leaf_parent, a.leaf_parent, (size_t)a.n_leaves * 4), "export leaf_parent");
    API_CK(cp(leaf_key, a.leaf_key, (size_t)a.n_leaves * 8), "export leaf_key");
    API_CK(cp(sigma, a.sigma, (size_t)a.n_leaves * sb), "export sigma");
    if (sh && a.n_leaves > 0 && !a.leaf_rec)
        API_CK(cudaMemcpy2DAsync(sh, 3 * a.K * sb, a.sh, (size_t)a.row_stride * sb, 3 * a.K * sb,
                                 (size_t)a.n_leaves, cudaMemcpyDeviceToHost, s),
               "export sh");
    if (sh && a.n_leaves > 0 && a.leaf_rec) {
        // compressed: every leaf's coefficients are its palette row
        const int64_t P = int64_t(1) << a.palette_bits;
        std::vector<uint16_t> pal((size_t)P * a.row_stride);
        std::vector<uint32_t> rec((size_t)a.n_leaves);
        API_CK(cudaMemcpyAsync(pal.data(), a.palette, pal.size() * 2, cudaMemcpyDeviceToHost, s),
               "export palette");
        API_CK(cudaMemcpyAsync(rec.data(), a.leaf_rec, rec.size() * 4, cudaMemcpyDeviceToHost, s),
               "export records");
        API_CK(cudaStreamSynchronize(s), "export sync");
        uint16_t *out = static_cast<uint16_t *>(sh);
        for (int64_t v = 0; v < a.n_leaves; v++)
            std::memcpy(out + v * 3 * a.K, pal.data() + (size_t)(rec[v] >> 16) * a.row_stride,
                        (size_t)3 * a.K * 2);
    }
    API_CK(cudaStreamSynchronize(s), "export sync");
    return DOT_OK;
}

int dot_tree_import(const dot_host_tree *h, const dot_allocator *alloc, void *stream,
                    dot_tree **out) {
    if (!h || !out) return fail(DOT_ERR_INVALID_ARG, "host tree and out must not be NULL");
    const int64_t N = h->n_nodes, L = h->n_leaves;
    if (N < 1 || L < 1 || N > (int64_t)INT32_MAX / 8 || L > (int64_t)INT32_MAX)
        return fail(DOT_ERR_INVALID_ARG, "node / leaf counts out of range");
    if (h->sh_degree < 0 || h->sh_degree > 3) return fail(DOT_ERR_UNSUPPORTED, "sh_degree must be in [0, 3]");
    if (h->storage < DOT_STORAGE_F32 || h->storage > DOT_STORAGE_BF16)
        return fail(DOT_ERR_INVALID_ARG, "unknown storage type");
    if (!h->child || !h->node_parent || !h->node_key || !h->leaf_parent || !h->leaf_key ||
        !h->sigma || !h->sh)
        return fail(DOT_ERR_INVALID_ARG, "host arrays must not be NULL");
    if (!(h->half_size > 0.f)) return fail(DOT_ERR_INVALID_ARG, "half_size must be positive");
    // structural validation: every node but the root and every leaf referenced once, parents
    // and keys consistent, levels <= 16
    std::vector<uint8_t> seen_n((size_t)N, 0), seen_l((size_t)L, 0);
    if (h->node_key[0] != 1 || h->node_parent[0] != -1)
        return fail(DOT_ERR_INVALID_ARG, "node 0 must be the root (key 1, parent -1)");
    int max_level = 0;
    for (int64_t p = 0; p < N; p++) {
        if (key_level_host(h->node_key[p]) >= dot::kMaxLevels)
            return fail(DOT_ERR_INVALID_ARG, "internal node below level 15");
        for (int j = 0; j < 8; j++) {
            const int32_t c = h->child[8 * p + j];
            const uint64_t ck = (h->node_key[p] << 3) | (uint64_t)j;
            if (c >= 0) {
                if (c == 0 || c >= N || seen_n[c]) return fail(DOT_ERR_INVALID_ARG, "bad internal child pointer");
                seen_n[c] = 1;
                if (h->node_parent[c] != p || h->node_key[c] != ck)
                    return fail(DOT_ERR_INVALID_ARG, "node parent / key inconsistent with child table");
            } else {
                const int64_t v = -1 - (int64_t)c;
                if (v >= L || seen_l[v]) return fail(DOT_ERR_INVALID_ARG, "bad leaf child pointer");
                seen_l[v] = 1;
                if (h->leaf_parent[v] != p || h->leaf_key[v] != ck)
                    return fail(DOT_ERR_INVALID_ARG, "leaf parent / key inconsistent with child table");
                const int lv = key_level_host(ck);
                if (lv > max_level) max_level = lv;
            }
        }
    }
    for (int64_t p = 1; p < N; p++)
        if (!seen_n[p]) return fail(DOT_ERR_INVALID_ARG, "unreferenced internal node");
    for (int64_t v = 0; v < L; v++)
        if (!seen_l[v]) return fail(DOT_ERR_INVALID_ARG, "unreferenced leaf");
    dot::DevAlloc al;
    int rc = make_alloc(alloc, al);
    if (rc) return rc;
    cudaStream_t s = S(stream);
    dot_tree *t = nullptr;
    rc = new_tree(al, s, &t);
    if (rc) return rc;
    for (int a = 0; a < 3; a++) t->center[a] = h->center[a];
    t->half_size = h->half_size;
    t->a.n_nodes = N;
    t->a.n_leaves = L;
    t->a.max_level = max_level;
    t->a.sh_degree = h->sh_degree;
    t->a.storage = h->storage;
    t->a.K = (h->sh_degree + 1) * (h->sh_degree + 1);
    t->a.row_stride = dot::row_stride_elems(h->storage, t->a.K);
    cudaError_t e = dot::alloc_tree_arrays(t->a, al, s);
    const size_t sb = (size_t)dot::storage_bytes(h->storage);
    if (e == cudaSuccess) e = cudaMemcpyAsync(t->a.child, h->child, (size_t)N * 32, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(t->a.node_parent, h->node_parent, (size_t)N * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(t->a.node_key, h->node_key, (size_t)N * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(t->a.leaf_parent, h->leaf_parent, (size_t)L * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(t->a.leaf_key, h->leaf_key, (size_t)L * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(t->a.sigma, h->sigma, (size_t)L * sb, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(t->a.sh, 0, (size_t)L * t->a.row_stride * sb, s);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(t->a.sh, (size_t)t->a.row_stride * sb, h->sh, 3 * t->a.K * sb,
                              3 * t->a.K * sb, (size_t)L, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = dot::build_ropes(t->a, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        int r = cuda_fail(e, "dot_tree_import");
        destroy_tree(t);
        return r;
    }
    *out = t;
    return DOT_OK;
}

int dot_tree_status(dot_tree *t, void *stream, uint32_t *status) {
    int rc = check_tree(t);
    if (rc) return rc;
    if (!status) return fail(DOT_ERR_INVALID_ARG, "status is NULL");
    uint32_t h = 0;
    API_CK(cudaMemcpyAsync(&h, t->status, 4, cudaMemcpyDeviceToHost, S(stream)), "status read");
    API_CK(cudaMemsetAsync(t->status, 0, 4, S(stream)), "status clear");
    API_CK(cudaStreamSynchronize(S(stream)), "status sync");
    *status = h;
    return DOT_OK;
}

int dot_render_forward(const dot_tree *t, const dot_rays *rays, const dot_render_opts *opts,
                       float *rgb, float *T_final, float *signal, void *stream) {
    int rc = check_tree(t);
    if (rc) return rc;
    dot::RaySource rs;
    int64_t R = 0;
    if ((rc = make_rays(rays, rs, R))) return rc;
    dot::RenderParams rp;
    bool exact = false;
    if ((rc = make_params(t, opts, rp, exact))) return rc;
    if (R > 0 && !rgb) return fail(DOT_ERR_INVALID_ARG, "rgb is NULL");
    if (rp.signal_mode != DOT_SIGNAL_NONE && !signal)
        return fail(DOT_ERR_INVALID_ARG, "signal_mode set but signal is NULL");
    dot::RenderIO io{};
    io.rgb = rgb;
    io.T_final = T_final;
    io.signal = rp.signal_mode != DOT_SIGNAL_NONE ? signal : nullptr;
    io.status = t->status;
    if (R == 0) return DOT_OK;
    API_CK(dot::launch_march_fwd(t->a.storage, t->a.sh_degree, exact, view_of(t), rs, rp, io, S(stream)),
           "dot_render_forward");
    return DOT_OK;
}

int dot_render_backward(const dot_tree *t, const dot_rays *rays, const dot_render_opts *opts,
                        const float *grad_rgb, const float *rgb, float *grad_sigma,
                        float *grad_sh, float *signal, uint8_t *touched, void *stream) {
    int rc = check_tree(t);
    if (rc) return rc;
    dot::RaySource rs;
    int64_t R = 0;
    if ((rc = make_rays(rays, rs, R))) return rc;
    dot::RenderParams rp;
    bool exact = false;
    if ((rc = make_params(t, opts, rp, exact))) return rc;
    if ((rc = check_uncompressed(t, "dot_render_backward"))) return rc;
    if (R > 0 && (!grad_rgb || !rgb || !grad_sigma || !grad_sh))
        return fail(DOT_ERR_INVALID_ARG, "grad_rgb, rgb, grad_sigma and grad_sh must not be NULL");
    if (rp.signal_mode != DOT_SIGNAL_NONE && !signal)
        return fail(DOT_ERR_INVALID_ARG, "signal_mode set but signal is NULL");
    dot::RenderIO io{};
    io.grad_rgb = grad_rgb;
    io.rgb_fwd = rgb;
    io.grad_sigma = grad_sigma;
    io.grad_sh = grad_sh;
    io.signal = rp.signal_mode != DOT_SIGNAL_NONE ? signal : nullptr;
    io.status = t->status;
    io.grad_vec = ((reinterpret_cast<uintptr_t>(grad_sh) & 15u) == 0) ? 1 : 0;
    io.touched = touched;
    if (R == 0) return DOT_OK;
    API_CK(dot::launch_march_bwd(t->a.storage, t->a.sh_degree, exact, view_of(t), rs, rp, io, S(stream)),
           "dot_render_backward");
    return DOT_OK;
}

int dot_accumulate_signal(const dot_tree *t, const dot_rays *rays, const dot_render_opts *opts,
                          int32_t mode, float *signal, void *stream) {
    int rc = check_tree(t);
    if (rc) return rc;
    if (!signal) return fail(DOT_ERR_INVALID_ARG, "signal is NULL");
    if (mode == DOT_SIGNAL_SIGMA) {
        API_CK(dot::launch_sigma_signal(t->a.storage, t->a.sigma, t->a.n_leaves, signal, S(stream)),
               "dot_accumulate_signal");
        return DOT_OK;
    }
    if (mode != DOT_SIGNAL_SUM_ALPHA && mode != DOT_SIGNAL_MAX_WEIGHT)
        return fail(DOT_ERR_INVALID_ARG, "mode must be SUM_ALPHA, MAX_WEIGHT or SIGMA");
    dot::RaySource rs;
    int64_t R = 0;
    if ((rc = make_rays(rays, rs, R))) return rc;
    dot::RenderParams rp;
    bool exact = false;
    if ((rc = make_params(t, opts, rp, exact))) return rc;
    rp.signal_mode = mode;
    dot::RenderIO io{};
    io.signal = signal;
    io.status = t->status;
    if (R == 0) return DOT_OK;
    API_CK(dot::launch_march_signal(t->a.storage, exact, view_of(t), rs, rp, io, S(stream)),
           "dot_accumulate_signal");
    return DOT_OK;
}

int dot_select_masks(const dot_tree *t, const float *signal, const dot_select_opts *opts,
                     uint8_t *prune_mark, uint8_t *sample_mark, void *stream) {
    int rc = check_tree(t);
    if (rc) return rc;
    if (!opts) return fail(DOT_ERR_INVALID_ARG, "opts is NULL");
    const int64_t L = t->a.n_leaves;
    for (int m : {opts->prune_mode, opts->sample_mode})
        if (m < DOT_SELECT_NONE || m > DOT_SELECT_QUANTILE)
            return fail(DOT_ERR_INVALID_ARG, "unknown selection mode");
    if ((opts->prune_mode >= DOT_SELECT_FRACTION && !(opts->prune_value >= 0.0 && opts->prune_value <= 1.0)) ||
        (opts->sample_mode >= DOT_SELECT_FRACTION && !(opts->sample_value >= 0.0 && opts->sample_value <= 1.0)))
        return fail(DOT_ERR_INVALID_ARG, "selection fraction must be in [0, 1]");
    if (L > 0 && (!signal || !prune_mark || !sample_mark))
        return fail(DOT_ERR_INVALID_ARG, "signal and masks must not be NULL");
    API_CK(dot::select_masks(signal, L, opts->prune_mode, opts->prune_value, opts->sample_mode,
                             opts->sample_value, prune_mark, sample_mark, S(stream)),
           "dot_select_masks");
    return DOT_OK;
}

int dot_refine_plan(const dot_tree *t, const uint8_t *prune_mark, const uint8_t *sample_mark,
                    int32_t depth_cap, dot_refine_counts *out, void *stream) {
    int rc = check_tree(t);
    if (rc) return rc;
    if ((rc = check_uncompressed(t, "dot_refine_plan"))) return rc;
    if (!prune_mark || !sample_mark || !out) return fail(DOT_ERR_INVALID_ARG, "masks and out must not be NULL");
    if (depth_cap < 1 || depth_cap > dot::kMaxLevels) return fail(DOT_ERR_INVALID_ARG, "depth_cap must be in [1, 16]");
    dot::RefinePlan plan{};
    API_CK(dot::refine_tree(t->a, prune_mark, sample_mark, depth_cap, false, nullptr, t->alloc,
                            nullptr, nullptr, 0, &plan, S(stream)),
           "dot_refine_plan");
    out->n_nodes = plan.n_nodes;
    out->n_leaves = plan.n_leaves;
    out->n_pruned_groups = plan.n_merged;
    out->n_sampled = plan.n_sampled;
    out->n_capped = plan.n_capped;
    return DOT_OK;
}

int dot_refine_prune(dot_tree *t, const uint8_t *prune_mark, const uint8_t *sample_mark,
                     int32_t depth_cap, int32_t *leaf_map, const dot_leaf_array *aux, int32_t n_aux,
                     void *stream) {
    int rc = check_tree(t);
    if (rc) return rc;
    if ((rc = check_uncompressed(t, "dot_refine_prune"))) return rc;
    if (!prune_mark || !sample_mark || !leaf_map) return fail(DOT_ERR_INVALID_ARG, "masks and leaf_map must not be NULL");
    if (depth_cap < 1 || depth_cap > dot::kMaxLevels) return fail(DOT_ERR_INVALID_ARG, "depth_cap must be in [1, 16]");
    if (n_aux < 0 || (n_aux > 0 && !aux)) return fail(DOT_ERR_INVALID_ARG, "bad aux arrays");
    for (int i = 0; i < n_aux; i++) {
        if (!aux[i].src || !aux[i].dst || aux[i].width < 1)
            return fail(DOT_ERR_INVALID_ARG, "aux array needs src, dst and width >= 1");
        if (aux[i].merge < DOT_MERGE_MEAN || aux[i].merge > DOT_MERGE_MAX)
            return fail(DOT_ERR_INVALID_ARG, "unknown aux merge");
    }
    dot::RefinePlan plan{};
    dot::TreeArrays nw;
    API_CK(dot::refine_tree(t->a, prune_mark, sample_mark, depth_cap, true, &nw, t->alloc, leaf_map,
                            aux, n_aux, &plan, S(stream)),
           "dot_refine_prune");
    dot::free_tree_arrays(t->a, t->alloc, S(stream));
    t->a = nw;
    return DOT_OK;
}

int dot_render_stats(const dot_tree *t, const dot_rays *rays, const dot_render_opts *opts,
                     int64_t out[4], void *stream) {
    int rc = check_tree(t);
    if (rc) return rc;
    if (!out) return fail(DOT_ERR_INVALID_ARG, "out is NULL");
    dot::RaySource rs;
    int64_t R = 0;
    if ((rc = make_rays(rays, rs, R))) return rc;
    dot::RenderParams rp;
    bool exact = false;
    if ((rc = make_params(t, opts, rp, exact))) return rc;
    cudaStream_t s = S(stream);
    unsigned long long *d = nullptr;
    API_CK(cudaMallocAsync((void **)&d, 4 * sizeof(unsigned long long), s), "stats alloc");
    dot::RenderIO io{};
    io.stats = d;
    io.status = t->status;
    cudaError_t e = cudaMemsetAsync(d, 0, 4 * sizeof(unsigned long long), s);
    if (e == cudaSuccess && R > 0) e = dot::launch_march_stats(t->a.storage, exact, view_of(t), rs, rp, io, s);
    unsigned long long h[4] = {0, 0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(d, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "dot_render_stats");
    for (int i = 0; i < 4; i++) out[i] = (int64_t)h[i];
    return DOT_OK;
}

}  // extern "C"

namespace dot {
int64_t select_noalloc_max_leaves();
cudaError_t select_masks_noalloc(const float *signal, int64_t n, int prune_mode,
                                 double prune_value, int sample_mode, double sample_value,
                                 uint8_t *prune_mark, uint8_t *sample_mark, cudaStream_t s);
}  // namespace dot

extern "C" int dot_select_masks_noalloc(const dot_tree *t, const float *signal,
                                        const dot_select_opts *opts, uint8_t *prune_mark,
                                        uint8_t *sample_mark, void *stream) {
    int rc = check_tree(t);
    if (rc) return rc;
    if (!opts) return fail(DOT_ERR_INVALID_ARG, "opts is NULL");
    const int64_t L = t->a.n_leaves;
    if (L > dot::select_noalloc_max_leaves())
        return fail(DOT_ERR_INVALID_ARG,
                    "dot_select_masks_noalloc handles at most 2^26 leaves; use dot_select_masks");
    for (int m : {opts->prune_mode, opts->sample_mode})
        if (m < DOT_SELECT_NONE || m > DOT_SELECT_QUANTILE)
            return fail(DOT_ERR_INVALID_ARG, "unknown selection mode");
    if ((opts->prune_mode >= DOT_SELECT_FRACTION && !(opts->prune_value >= 0.0 && opts->prune_value <= 1.0)) ||
        (opts->sample_mode >= DOT_SELECT_FRACTION && !(opts->sample_value >= 0.0 && opts->sample_value <= 1.0)))
        return fail(DOT_ERR_INVALID_ARG, "selection fraction must be in [0, 1]");
    if (L > 0 && (!signal || !prune_mark || !sample_mark))
        return fail(DOT_ERR_INVALID_ARG, "signal and masks must not be NULL");
    API_CK(dot::select_masks_noalloc(signal, L, opts->prune_mode, opts->prune_value,
                                     opts->sample_mode, opts->sample_value, prune_mark,
                                     sample_mark, S(stream)),
           "dot_select_masks_noalloc");
    return DOT_OK;
}

namespace dot {
cudaError_t launch_l2_read(const void *buf, int64_t bytes, int32_t passes,
                           unsigned long long *sink, cudaStream_t s);
cudaError_t launch_render_slots(int storage, int deg, bool exact, const TreeView *views,
                                int n_trees, const void *table, int32_t max_slots,
                                const RenderParams &rp, unsigned long long *counter,
                                uint32_t *status, int grid, cudaStream_t s);
}  // namespace dot

extern "C" int dot_render_slots(dot_tree *const *trees, int32_t n_trees, const void *table,
                                int32_t max_slots, const dot_render_opts *opts,
                                unsigned long long *work_counter, void *stream) {
    if (!trees || n_trees < 1 || n_trees > DOT_MAX_SERVE_TREES)
        return fail(DOT_ERR_INVALID_ARG, "n_trees must be in [1, DOT_MAX_SERVE_TREES]");
    if (!table || !work_counter || max_slots < 1)
        return fail(DOT_ERR_INVALID_ARG, "table, work_counter and max_slots >= 1 are required");
    dot::TreeView views[DOT_MAX_SERVE_TREES];
    int max_level = 0;
    for (int i = 0; i < n_trees; i++) {
        int rc = check_tree(trees[i]);
        if (rc) return rc;
        if (trees[i]->a.storage != trees[0]->a.storage || trees[i]->a.sh_degree != trees[0]->a.sh_degree)
            return fail(DOT_ERR_INVALID_ARG, "served trees must share storage type and SH degree");
        if ((trees[i]->a.leaf_rec != nullptr) != (trees[0]->a.leaf_rec != nullptr))
            return fail(DOT_ERR_INVALID_ARG, "served trees must be all compressed or none");
        views[i] = view_of(trees[i]);
        if (trees[i]->a.max_level > max_level) max_level = trees[i]->a.max_level;
    }
    dot::RenderParams rp;
    bool exact = false;
    int rc = make_params(trees[0], opts, rp, exact);
    if (rc) return rc;
    if (rp.signal_mode != DOT_SIGNAL_NONE) return fail(DOT_ERR_INVALID_ARG, "signal_mode must be NONE");
    if (opts->max_steps == 0) rp.max_steps = 3 * (1 << max_level) + 64;
    API_CK(dot::launch_render_slots(trees[0]->a.storage, trees[0]->a.sh_degree, exact, views,
                                    n_trees, table, max_slots, rp, work_counter, trees[0]->status,
                                    0, S(stream)),
           "dot_render_slots");
    return DOT_OK;
}

extern "C" int dot_mse_grad(const float *rgb, const float *target, int64_t n_rays,
                            float *grad_rgb, double *loss_sum, void *stream) {
    if (n_rays < 0) return fail(DOT_ERR_INVALID_ARG, "n_rays < 0");
    if (n_rays == 0) return DOT_OK;
    if (!rgb || !target || !grad_rgb) return fail(DOT_ERR_INVALID_ARG, "rgb, target and grad_rgb are required");
    if (grad_rgb == rgb || grad_rgb == target)
        return fail(DOT_ERR_INVALID_ARG, "grad_rgb must not alias rgb or target");
    API_CK(dot::launch_mse_grad(rgb, target, n_rays, grad_rgb, loss_sum, S(stream)), "dot_mse_grad");
    return DOT_OK;
}

extern "C" int dot_rmsprop_step(dot_tree *t, float *grad_sigma, float *grad_sh, float *ms_sigma,
                                float *ms_sh, const dot_rmsprop_opts *opts, void *stream) {
    int rc = check_tree(t);
    if (rc) return rc;
    if (!opts) return fail(DOT_ERR_INVALID_ARG, "opts is NULL");
    if ((rc = check_uncompressed(t, "dot_rmsprop_step"))) return rc;
    if (t->a.n_leaves == 0) return DOT_OK;
    if (!grad_sigma || !grad_sh || !ms_sigma || !ms_sh)
        return fail(DOT_ERR_INVALID_ARG, "gradients and mean-square arrays are required");
    if (!(opts->rho >= 0.f && opts->rho < 1.f)) return fail(DOT_ERR_INVALID_ARG, "rho must be in [0, 1)");
    if (!(opts->eps >= 0.f) || !std::isfinite(opts->lr_sigma) || !std::isfinite(opts->lr_sh))
        return fail(DOT_ERR_INVALID_ARG, "eps must be >= 0 and learning rates finite");
    API_CK(dot::launch_rmsprop(t->a.storage, t->a.sigma, t->a.sh, t->a.n_leaves, t->a.K,
                               t->a.row_stride, grad_sigma, grad_sh, ms_sigma, ms_sh, *opts,
                               S(stream)),
           "dot_rmsprop_step");
    return DOT_OK;
}

extern "C" int dot_compress_sh(dot_tree *t, int32_t bits, void *stream) {
    int rc = check_tree(t);
    if (rc) return rc;
    if (bits < 1 || bits > 16) return fail(DOT_ERR_INVALID_ARG, "bits must be in [1, 16]");
    if (t->a.storage == DOT_STORAGE_F32)
        return fail(DOT_ERR_UNSUPPORTED, "compression needs 16-bit leaf storage");
    if ((rc = check_uncompressed(t, "dot_compress_sh"))) return rc;
    API_CK(dot::compress_tree(t->a, bits, t->alloc, S(stream)), "dot_compress_sh");
    return DOT_OK;
}

extern "C" int dot_tree_canonicalize(dot_tree *t, int32_t *leaf_perm, const dot_leaf_array *aux,
                                     int32_t n_aux, void *stream) {
    int rc = check_tree(t);
    if (rc) return rc;
    if (!leaf_perm && t->a.n_leaves > 0) return fail(DOT_ERR_INVALID_ARG, "leaf_perm is NULL");
    if (n_aux < 0 || (n_aux > 0 && !aux)) return fail(DOT_ERR_INVALID_ARG, "bad aux arrays");
    for (int i = 0; i < n_aux; i++)
        if (!aux[i].src || !aux[i].dst || aux[i].width < 1 || aux[i].src == aux[i].dst)
            return fail(DOT_ERR_INVALID_ARG, "aux array needs distinct src and dst and width >= 1");
    dot::TreeArrays nw;
    cudaError_t e = dot::canonicalize_tree(t->a, &nw, t->alloc, leaf_perm, aux, n_aux, S(stream));
    if (e == cudaErrorInvalidValue)
        return fail(DOT_ERR_INVALID_ARG, "the node table does not reach every node and leaf once");
    API_CK(e, "dot_tree_canonicalize");
    dot::free_tree_arrays(t->a, t->alloc, S(stream));
    t->a = nw;
    return DOT_OK;
}

namespace {
int check_rms_opts(const dot_rmsprop_opts *opts) {
    if (!opts) return fail(DOT_ERR_INVALID_ARG, "opts is NULL");
    if (!(opts->rho >= 0.f && opts->rho < 1.f)) return fail(DOT_ERR_INVALID_ARG, "rho must be in [0, 1)");
    if (!(opts->eps >= 0.f) || !std::isfinite(opts->lr_sigma) || !std::isfinite(opts->lr_sh))
        return fail(DOT_ERR_INVALID_ARG, "eps must be >= 0 and learning rates finite");
    return DOT_OK;
}
}  // namespace

extern "C" int dot_rmsprop_step_sparse(dot_tree *t, float *grad_sigma, float *grad_sh,
                                       float *ms_sigma, float *ms_sh, uint8_t *touched,
                                       int32_t *last_step, int32_t step, int32_t *work,
                                       const dot_rmsprop_opts *opts, void *stream) {
    int rc = check_tree(t);
    if (rc) return rc;
    if ((rc = check_rms_opts(opts))) return rc;
    if ((rc = check_uncompressed(t, "dot_rmsprop_step_sparse"))) return rc;
    if (t->a.n_leaves == 0) return DOT_OK;
    if (!grad_sigma || !grad_sh || !ms_sigma || !ms_sh || !touched || !last_step || !work)
        return fail(DOT_ERR_INVALID_ARG, "gradients, mean squares, touched, last_step and work are required");
    if (step < 1) return fail(DOT_ERR_INVALID_ARG, "step must be >= 1");
    API_CK(dot::launch_rmsprop_sparse(t->a.storage, t->a.sigma, t->a.sh, t->a.n_leaves, t->a.K,
                                      t->a.row_stride, grad_sigma, grad_sh, ms_sigma, ms_sh,
                                      touched, last_step, step, work, *opts, S(stream)),
           "dot_rmsprop_step_sparse");
    return DOT_OK;
}

extern "C" int dot_rmsprop_flush(dot_tree *t, float *ms_sigma, float *ms_sh, int32_t *last_step,
                                 int32_t step, const dot_rmsprop_opts *opts, void *stream) {
    int rc = check_tree(t);
    if (rc) return rc;
    if ((rc = check_rms_opts(opts))) return rc;
    if (t->a.n_leaves == 0) return DOT_OK;
    if (!ms_sigma || !ms_sh || !last_step)
        return fail(DOT_ERR_INVALID_ARG, "mean squares and last_step are required");
    API_CK(dot::launch_rmsprop_flush(t->a.n_leaves, t->a.K, ms_sigma, ms_sh, last_step, step,
                                     opts->rho, S(stream)),
           "dot_rmsprop_flush");
    return DOT_OK;
}

extern "C" int dot_render_forward_backward_mse(const dot_tree *t, const dot_rays *rays,
                                               const dot_render_opts *opts, const float *target,
                                               float *rgb, float *grad_rgb, double *loss_sum,
                                               float *grad_sigma, float *grad_sh, float *signal,
                                               uint8_t *touched, void *stream) {
    int rc = check_tree(t);
    if (rc) return rc;
    if ((rc = check_uncompressed(t, "dot_render_forward_backward_mse"))) return rc;
    dot::RaySource rs;
    int64_t R = 0;
    if ((rc = make_rays(rays, rs, R))) return rc;
    dot::RenderParams rp;
    bool exact = false;
    if ((rc = make_params(t, opts, rp, exact))) return rc;
    if (R > 0 && (!target || !rgb || !grad_rgb || !grad_sigma || !grad_sh))
        return fail(DOT_ERR_INVALID_ARG, "target, rgb, grad_rgb, grad_sigma and grad_sh are required");
    if (grad_rgb == rgb || grad_rgb == target || rgb == target)
        return fail(DOT_ERR_INVALID_ARG, "target, rgb and grad_rgb must be distinct buffers");
    if (rp.signal_mode != DOT_SIGNAL_NONE && !signal)
        return fail(DOT_ERR_INVALID_ARG, "signal_mode set but signal is NULL");
    dot::RenderIO io{};
    io.rgb = rgb;
    io.target = target;
    io.grad_out = grad_rgb;
    io.loss_sum = loss_sum;
    io.inv3R = R > 0 ? (float)(1.0 / (3.0 * (double)R)) : 0.f;
    io.grad_sigma = grad_sigma;
    io.grad_sh = grad_sh;
    io.signal = rp.signal_mode != DOT_SIGNAL_NONE ? signal : nullptr;
    io.touched = touched;
    io.status = t->status;
    io.grad_vec = ((reinterpret_cast<uintptr_t>(grad_sh) & 15u) == 0) ? 1 : 0;
    if (R == 0) return DOT_OK;
    API_CK(dot::launch_march_fwdbwd(t->a.storage, t->a.sh_degree, exact, view_of(t), rs, rp, io,
                                    S(stream)),
           "dot_render_forward_backward_mse");
    return DOT_OK;
}

extern "C" int dot_camera_order(const dot_camera *cams, int32_t n, int32_t *order) {
    if (n < 0) return fail(DOT_ERR_INVALID_ARG, "n < 0");
    if (n == 0) return DOT_OK;
    if (!cams || !order) return fail(DOT_ERR_INVALID_ARG, "cameras and order are required");
    std::vector<char> used((size_t)n, 0);
    int32_t cur = 0;
    used[0] = 1;
    order[0] = 0;
    for (int32_t k = 1; k < n; k++) {
        const float *a = cams[cur].c2w;
        double best = -1.0;
        int32_t bi = -1;
        for (int32_t j = 0; j < n; j++) {
            if (used[(size_t)j]) continue;
            const float *b = cams[j].c2w;
            const double dx = (double)b[3] - a[3], dy = (double)b[7] - a[7], dz = (double)b[11] - a[11];
            const double d2 = dx * dx + dy * dy + dz * dz;
            if (bi < 0 || d2 < best) {
                best = d2;
                bi = j;
            }
        }
        used[(size_t)bi] = 1;
        order[k] = bi;
        cur = bi;
    }
    return DOT_OK;
}

// ---------------------------------------------------------------------------------------------
// whole views to host memory: chunked march on the caller's stream (and a second render stream),
// device-to-host copies of the finished chunks on a copy stream
// ---------------------------------------------------------------------------------------------
// 1: page-locked, mapped host images are written in place by one launch (no copies): 100 views of
// 800x800 to host memory in 8.66 ms against 9.07 ms through the chunked copies (8.65 ms on the
// device alone)
#ifndef DOT_VIEWS_DIRECT
#define DOT_VIEWS_DIRECT 1
#endif
// log2 of the rays per chunk, about
#ifndef DOT_VIEWS_CHUNK_LOG2
#define DOT_VIEWS_CHUNK_LOG2 23
#endif
// render streams the chunks alternate over (1 or 2): with 2, a chunk's launch starts while the
// previous chunk's last blocks still run
#ifndef DOT_VIEWS_STREAMS
#define DOT_VIEWS_STREAMS 2
#endif
// 1: the views left after the full chunks go in halving chunks down to one view, so the copy
// that cannot overlap any march (the last chunk's) is one view.  100 views of 800x800 on a
// 2.9 M-leaf tree, 9.81 ms in one launch: 10.90 ms to host memory with one stream and no taper,
// 10.31 with two streams, 10.14 with two streams and the taper (chunks of 2^22 rays: 10.20).
#ifndef DOT_VIEWS_TAPER
#define DOT_VIEWS_TAPER 1
#endif

namespace {

constexpr int kViewSlots = 3;  // chunk buffers in the ring
constexpr int64_t kChunkRays = (int64_t)1 << DOT_VIEWS_CHUNK_LOG2;
static_assert(DOT_VIEWS_STREAMS == 1 || DOT_VIEWS_STREAMS == 2, "one or two render streams");

// Workspace layout: the cameras in render order, then the ring of chunk buffers (rgb, then T when
// requested), every part 256-byte aligned.
struct ViewsPlan {
    int64_t per_view = 0;     // pixels of one view
    int32_t chunk_views = 0;  // views of a full chunk (the capacity of a ring buffer)
    int32_t slots = 0;
    std::vector<int32_t> first;  // the chunks: first view (in render order) of each, then n
    int64_t cams_bytes = 0, order_bytes = 0, rgb_bytes = 0, T_bytes = 0, total = 0;
};

int64_t align256(int64_t x) { return (x + 255) / 256 * 256; }

bool plan_views(int32_t n, int32_t W, int32_t H, bool with_T, ViewsPlan &p) {
    if (n < 0 || n > 65535 || W <= 0 || H <= 0 || W > 65536 || H > 65536) return false;
    p = ViewsPlan{};
    p.per_view = (int64_t)W * H;
    if (n == 0) return true;
    const int64_t want = std::min<int64_t>(n, std::max<int64_t>(1, (p.per_view * n + kChunkRays - 1) / kChunkRays));
    p.chunk_views = (int32_t)((n + want - 1) / want);
    int32_t v = 0;
    while (n - v > p.chunk_views) {  // full chunks
        p.first.push_back(v);
        v += p.chunk_views;
    }
    while (v < n) {  // the rest: one chunk, or halving chunks after a full one
        p.first.push_back(v);
        const int32_t rem = n - v;
        v += (DOT_VIEWS_TAPER && v > 0 && rem > 1) ? (rem + 1) / 2 : rem;
    }
    p.first.push_back(n);
    p.slots = std::min<int32_t>(kViewSlots, (int32_t)p.first.size() - 1);
    p.cams_bytes = align256((int64_t)n * (int64_t)sizeof(dot_camera));
    p.order_bytes = align256((int64_t)n * (int64_t)sizeof(int32_t));
    p.rgb_bytes = align256(p.chunk_views * p.per_view * 3 * (int64_t)sizeof(float));
    p.T_bytes = with_T ? align256(p.chunk_views * p.per_view * (int64_t)sizeof(float)) : 0;
    p.total = p.cams_bytes + p.order_bytes + p.slots * (p.rgb_bytes + p.T_bytes);
    return true;
}

// The streams and per-slot events of one call; on every exit the work already queued finishes
// before the host buffers and the workspace are handed back.
struct ViewsPipe {
    cudaStream_t render[2] = {nullptr, nullptr}, copy = nullptr;
    bool own_render1 = false;
    cudaEvent_t ready = nullptr, rendered[kViewSlots] = {}, copied[kViewSlots] = {};
    ~ViewsPipe() {
        if (copy) {
            cudaStreamSynchronize(copy);
            cudaStreamDestroy(copy);
        }
        if (own_render1) {
            cudaStreamSynchronize(render[1]);
            cudaStreamDestroy(render[1]);
        }
        cudaStreamSynchronize(render[0]);
        if (ready) cudaEventDestroy(ready);
        for (int i = 0; i < kViewSlots; i++) {
            if (rendered[i]) cudaEventDestroy(rendered[i]);
            if (copied[i]) cudaEventDestroy(copied[i]);
        }
    }
};

// The device address of host buffer [p, p + bytes) when all of it lies in one page-locked
// allocation mapped into the device's address space, else null (pageable or foreign memory).
float *mapped_device_ptr(float *p, size_t bytes) {
    cudaPointerAttributes a0{}, a1{};
    if (cudaPointerGetAttributes(&a0, p) != cudaSuccess ||
        cudaPointerGetAttributes(&a1, reinterpret_cast<char *>(p) + bytes - 1) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a0.type != cudaMemoryTypeHost || a1.type != cudaMemoryTypeHost || !a0.devicePointer ||
        !a1.devicePointer)
        return nullptr;
    if (static_cast<char *>(a1.devicePointer) - static_cast<char *>(a0.devicePointer) !=
        static_cast<ptrdiff_t>(bytes - 1))
        return nullptr;
    return static_cast<float *>(a0.devicePointer);
}

// device-to-host copies of `cnt` views of one chunk: view j of the chunk goes to host view
// order[j]; runs of consecutive views go in one copy
cudaError_t copy_views_out(float *host, const float *dev, const int32_t *order, int32_t cnt,
                           int64_t floats_per_view, cudaStream_t s) {
    const size_t bytes = (size_t)floats_per_view * sizeof(float);
    for (int32_t j = 0; j < cnt;) {
        int32_t e = j + 1;
        while (e < cnt && order[e] == order[e - 1] + 1) e++;
        cudaError_t err = cudaMemcpyAsync(host + (int64_t)order[j] * floats_per_view,
                                          dev + (int64_t)j * floats_per_view, bytes * (size_t)(e - j),
                                          cudaMemcpyDeviceToHost, s);
        if (err != cudaSuccess) return err;
        j = e;
    }
    return cudaSuccess;
}

}  // namespace

extern "C" int64_t dot_render_views_host_workspace(int32_t n_cameras, int32_t width, int32_t height,
                                                   int32_t with_T) {
    ViewsPlan p;
    return plan_views(n_cameras, width, height, with_T != 0, p) ? p.total : -1;
}

extern "C" int dot_render_views_host(const dot_tree *t, const dot_camera *cameras, int32_t n,
                                     int32_t width, int32_t height, const int32_t *view_order,
                                     const dot_render_opts *opts, float *rgb, float *T_final,
                                     void *workspace, int64_t workspace_bytes, void *stream) {
    int rc = check_tree(t);
    if (rc) return rc;
    ViewsPlan p;
    if (!plan_views(n, width, height, T_final != nullptr, p))
        return fail(DOT_ERR_INVALID_ARG, "n_cameras must be in [0, 65535] and width, height in [1, 65536]");
    dot::RenderParams rp;
    bool exact = false;
    if ((rc = make_params(t, opts, rp, exact))) return rc;
    if (rp.signal_mode != DOT_SIGNAL_NONE)
        return fail(DOT_ERR_INVALID_ARG, "dot_render_views_host: signal_mode must be NONE");
    if (n == 0) return DOT_OK;
    if (!cameras || !rgb) return fail(DOT_ERR_INVALID_ARG, "cameras and rgb are required");
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255))
        return fail(DOT_ERR_INVALID_ARG, "workspace must be a 256-byte aligned device buffer");
    if (workspace_bytes < p.total)
        return fail(DOT_ERR_INVALID_ARG, "workspace is smaller than dot_render_views_host_workspace");
    std::vector<int32_t> order((size_t)n);
    if (view_order) {
        std::vector<char> seen((size_t)n, 0);
        for (int32_t i = 0; i < n; i++) {
            const int32_t v = view_order[i];
            if (v < 0 || v >= n || seen[(size_t)v])
                return fail(DOT_ERR_INVALID_ARG, "view_order is not a permutation of 0..n_cameras-1");
            seen[(size_t)v] = 1;
            order[(size_t)i] = v;
        }
    } else {
        for (int32_t i = 0; i < n; i++) order[(size_t)i] = i;
    }
    char *ws = static_cast<char *>(workspace);
    dot_camera *d_cams = reinterpret_cast<dot_camera *>(ws);
    const dot::TreeView tv = view_of(t);
    const char *where = "dot_render_views_host";

    // page-locked, mapped host images: one launch writes every view in place, no copies
    float *rgb_dev = DOT_VIEWS_DIRECT ? mapped_device_ptr(rgb, (size_t)(n * p.per_view * 3) * sizeof(float)) : nullptr;
    float *T_dev = (rgb_dev && T_final) ? mapped_device_ptr(T_final, (size_t)(n * p.per_view) * sizeof(float)) : nullptr;
    if (rgb_dev && (!T_final || T_dev)) {
        int32_t *d_order = reinterpret_cast<int32_t *>(ws + p.cams_bytes);
        std::vector<dot_camera> cams_in(cameras, cameras + n);  // alive until the call returns
        cudaStream_t s = S(stream);
        API_CK(cudaMemcpyAsync(d_cams, cams_in.data(), (size_t)n * sizeof(dot_camera),
                               cudaMemcpyHostToDevice, s), where);
        API_CK(cudaMemcpyAsync(d_order, order.data(), (size_t)n * sizeof(int32_t),
                               cudaMemcpyHostToDevice, s), where);
        dot_rays r{};
        r.kind = DOT_RAYS_CAMERAS;
        r.n_cameras = n;
        r.cameras = d_cams;
        r.width = width;
        r.height = height;
        r.view_order = d_order;
        dot::RaySource rs;
        int64_t R = 0;
        if ((rc = make_rays(&r, rs, R))) return rc;
        dot::RenderIO io{};
        io.rgb = rgb_dev;
        io.T_final = T_dev;
        io.status = t->status;
        API_CK(dot::launch_march_fwd(t->a.storage, t->a.sh_degree, exact, tv, rs, rp, io, s), where);
        API_CK(cudaStreamSynchronize(s), where);
        return DOT_OK;
    }

    std::vector<dot_camera> cams((size_t)n);  // in render order; alive until the call returns
    for (int32_t i = 0; i < n; i++) cams[(size_t)i] = cameras[order[(size_t)i]];
    ViewsPipe pipe;
    pipe.render[0] = pipe.render[1] = S(stream);
    API_CK(cudaStreamCreateWithFlags(&pipe.copy, cudaStreamNonBlocking), where);
    API_CK(cudaEventCreateWithFlags(&pipe.ready, cudaEventDisableTiming), where);
    for (int i = 0; i < p.slots; i++) {
        API_CK(cudaEventCreateWithFlags(&pipe.rendered[i], cudaEventDisableTiming), where);
        API_CK(cudaEventCreateWithFlags(&pipe.copied[i], cudaEventDisableTiming), where);
    }
    API_CK(cudaMemcpyAsync(d_cams, cams.data(), (size_t)n * sizeof(dot_camera), cudaMemcpyHostToDevice,
                           pipe.render[0]),
           where);
    if (DOT_VIEWS_STREAMS == 2 && p.first.size() > 2) {
        API_CK(cudaStreamCreateWithFlags(&pipe.render[1], cudaStreamNonBlocking), where);
        pipe.own_render1 = true;
        API_CK(cudaEventRecord(pipe.ready, pipe.render[0]), where);  // the cameras have arrived
        API_CK(cudaStreamWaitEvent(pipe.render[1], pipe.ready, 0), where);
    }
    const int32_t n_chunks = (int32_t)p.first.size() - 1;
    for (int32_t k = 0; k < n_chunks; k++) {
        const int slot = k % p.slots;
        cudaStream_t rs_k = pipe.render[k & 1];
        const int32_t first = p.first[(size_t)k];
        const int32_t cnt = p.first[(size_t)k + 1] - first;
        float *d_rgb = reinterpret_cast<float *>(ws + p.cams_bytes + p.order_bytes +
                                                 slot * (p.rgb_bytes + p.T_bytes));
        float *d_T = T_final ? reinterpret_cast<float *>(reinterpret_cast<char *>(d_rgb) + p.rgb_bytes) : nullptr;
        if (k >= p.slots)  // the slot's previous chunk has left for the host
            API_CK(cudaStreamWaitEvent(rs_k, pipe.copied[slot], 0), where);
        dot_rays r{};
        r.kind = DOT_RAYS_CAMERAS;
        r.n_cameras = cnt;
        r.cameras = d_cams + first;
        r.width = width;
        r.height = height;
        dot::RaySource rs;
        int64_t R = 0;
        if ((rc = make_rays(&r, rs, R))) return rc;
        dot::RenderIO io{};
        io.rgb = d_rgb;
        io.T_final = d_T;
        io.status = t->status;
        API_CK(dot::launch_march_fwd(t->a.storage, t->a.sh_degree, exact, tv, rs, rp, io, rs_k), where);
        API_CK(cudaEventRecord(pipe.rendered[slot], rs_k), where);
        API_CK(cudaStreamWaitEvent(pipe.copy, pipe.rendered[slot], 0), where);
        API_CK(copy_views_out(rgb, d_rgb, order.data() + first, cnt, p.per_view * 3, pipe.copy), where);
        if (T_final)
            API_CK(copy_views_out(T_final, d_T, order.data() + first, cnt, p.per_view, pipe.copy), where);
        API_CK(cudaEventRecord(pipe.copied[slot], pipe.copy), where);
    }
    API_CK(cudaStreamSynchronize(pipe.copy), where);
    if (pipe.own_render1) API_CK(cudaStreamSynchronize(pipe.render[1]), where);
    API_CK(cudaStreamSynchronize(pipe.render[0]), where);
    return DOT_OK;
}

extern "C" int dot_probe_l2_read(const void *buf, int64_t bytes, int32_t passes,
                                 unsigned long long *sink, void *stream) {
    if (!buf || bytes <= 0 || bytes % 16 != 0 || (reinterpret_cast<uintptr_t>(buf) & 15) != 0)
        return fail(DOT_ERR_INVALID_ARG, "buf must be 16-byte aligned and bytes a positive multiple of 16");
    if (passes < 1) return fail(DOT_ERR_INVALID_ARG, "passes must be >= 1");
    API_CK(dot::launch_l2_read(buf, bytes, passes, sink, S(stream)), "dot_probe_l2_read");
    return DOT_OK;
}
