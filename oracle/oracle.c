/*
 * oracle.c -- plain, slow, FP64 reference of the Dynamic PlenOctree (DOT) hot path.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).  Every function follows the plain definition of what
 * it computes, step by step, with no blocking, fusion or reordering:
 *   build      -- the PlenOctree structure (Sec. 3 Preliminaries): a cube root subdivided 8-way;
 *                 a cell is subdivided while it meets the scene and is above the maximum depth.
 *   segments   -- the ray's intersections with the leaves, in ray order (Sec. 3 Preliminaries).
 *   render     -- Eq. 1-2: C = sum_i T_i Q_i c_i, Q_i = 1 - exp(-sigma_i delta_i),
 *                 T_i = exp(-sum_{j<i} sigma_j delta_j), plus the background term.
 *   backward   -- the analytic derivative of the render with respect to sigma and SH.
 *   signal     -- Sec. 3.1: per-leaf sum over rays of Q_i (and the max-weight variant).
 *   select     -- Sec. 3.2 thresholds {Q <= tau}, {Q > gamma} and the top-k of Algorithm 1.
 *   refine     -- Eq. 3 (prune: children averaged into the parent) and Eq. 4 (sample: the
 *                 parent's values copied to 8 new children).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define QB 24 /* primitive parameters are integers in units of 2^-24 of the root edge */

/* ------------------------------------------------------------------------------------------ */
/* keys                                                                                        */
/* ------------------------------------------------------------------------------------------ */

static int key_level(uint64_t key) {
    int b = -1;
    while (key) { key >>= 1; b++; }
    return b / 3;
}

static void key_corner(uint64_t key, int64_t k[3]) {
    int l = key_level(key);
    k[0] = k[1] = k[2] = 0;
    for (int i = l - 1; i >= 0; i--) {
        unsigned tri = (unsigned)((key >> (3 * i)) & 7u);
        k[0] = (k[0] << 1) | ((tri >> 2) & 1);
        k[1] = (k[1] << 1) | ((tri >> 1) & 1);
        k[2] = (k[2] << 1) | (tri & 1);
    }
}

/* ------------------------------------------------------------------------------------------ */
/* build                                                                                       */
/* ------------------------------------------------------------------------------------------ */

/* does the open interior of the cell [A, B] (integer units) meet primitive p? */
static int prim_meets(const int64_t *p, const int64_t A[3], const int64_t B[3]) {
    int64_t type = p[0];
    const int64_t *q = p + 1;
    if (type == 0) { /* sphere (cx, cy, cz, r): distance from centre to the box below r */
        int64_t d2 = 0;
        for (int a = 0; a < 3; a++) {
            int64_t e = 0;
            if (q[a] < A[a]) e = A[a] - q[a];
            else if (q[a] > B[a]) e = q[a] - B[a];
            d2 += e * e;
        }
        return d2 < q[3] * q[3];
    }
    if (type == 1) { /* box (lo xyz, hi xyz): open intervals overlap on every axis */
        for (int a = 0; a < 3; a++)
            if (!(A[a] < q[3 + a] && q[a] < B[a])) return 0;
        return 1;
    }
    if (type == 2) { /* vertical cylinder (cx, cz, r, y0, y1) */
        int64_t ex = 0, ez = 0;
        if (q[0] < A[0]) ex = A[0] - q[0]; else if (q[0] > B[0]) ex = q[0] - B[0];
        if (q[1] < A[2]) ez = A[2] - q[1]; else if (q[1] > B[2]) ez = q[1] - B[2];
        if (!(ex * ex + ez * ez < q[2] * q[2])) return 0;
        return A[1] < q[4] && q[3] < B[1];
    }
    return 0;
}

static int cell_meets(const int64_t *prims, int32_t n, uint64_t key) {
    int l = key_level(key);
    int64_t k[3], A[3], B[3];
    key_corner(key, k);
    int64_t sz = (int64_t)1 << (QB - l);
    for (int a = 0; a < 3; a++) { A[a] = k[a] * sz; B[a] = A[a] + sz; }
    for (int i = 0; i < n; i++)
        if (prim_meets(prims + 8 * (int64_t)i, A, B)) return 1;
    return 0;
}

typedef struct { uint64_t key; int32_t parent; int32_t slot; } qcell;

static void *grow(void *p, int64_t *cap, int64_t need, size_t elem) {
    if (need <= *cap) return p;
    int64_t c = *cap ? *cap : 64;
    while (c < need) c *= 2;
    *cap = c;
    return realloc(p, (size_t)c * elem);
}

int oracle_build(const int64_t *prims, int32_t n_prims, int32_t D, otree *out) {
    memset(out, 0, sizeof(*out));
    if (D < 1 || D > 16) return -1;
    int64_t cap_n = 0, cap_l = 0, cap_cur = 0, cap_nxt = 0;
    qcell *cur = NULL, *nxt = NULL;
    int64_t n_cur = 1, n_nxt = 0;
    cur = grow(cur, &cap_cur, 1, sizeof(qcell));
    cur[0].key = 1; cur[0].parent = -1; cur[0].slot = 0;
    for (int l = 0; l <= D && n_cur > 0; l++) {
        n_nxt = 0;
        for (int64_t c = 0; c < n_cur; c++) {
            int m = cell_meets(prims, n_prims, cur[c].key);
            int internal = (l == 0) || (m && l < D); /* the root is always subdivided */
            if (internal) {
                int64_t id = out->n_nodes++;
                out->child = grow(out->child, &cap_n, out->n_nodes, 8 * sizeof(int32_t));
                out->node_parent = realloc(out->node_parent, (size_t)cap_n * sizeof(int32_t));
                out->node_key = realloc(out->node_key, (size_t)cap_n * sizeof(uint64_t));
                out->node_parent[id] = cur[c].parent;
                out->node_key[id] = cur[c].key;
                if (cur[c].parent >= 0) out->child[8 * (int64_t)cur[c].parent + cur[c].slot] = (int32_t)id;
                nxt = grow(nxt, &cap_nxt, n_nxt + 8, sizeof(qcell));
                for (int j = 0; j < 8; j++) {
                    nxt[n_nxt].key = (cur[c].key << 3) | (uint64_t)j;
                    nxt[n_nxt].parent = (int32_t)id;
                    nxt[n_nxt].slot = j;
                    n_nxt++;
                }
            } else {
                int64_t v = out->n_leaves++;
                int64_t oc = cap_l;
                out->leaf_key = grow(out->leaf_key, &cap_l, out->n_leaves, sizeof(uint64_t));
                if (cap_l != oc) {
                    out->leaf_parent = realloc(out->leaf_parent, (size_t)cap_l * sizeof(int32_t));
                    out->leaf_inside = realloc(out->leaf_inside, (size_t)cap_l);
                }
                out->leaf_key[v] = cur[c].key;
                out->leaf_parent[v] = cur[c].parent;
                out->leaf_inside[v] = (uint8_t)m;
                out->child[8 * (int64_t)cur[c].parent + cur[c].slot] = -1 - (int32_t)v;
            }
        }
        qcell *tmp = cur; cur = nxt; nxt = tmp;
        int64_t tc = cap_cur; cap_cur = cap_nxt; cap_nxt = tc;
        n_cur = n_nxt;
    }
    free(cur);
    free(nxt);
    return 0;
}

void oracle_tree_free(otree *t) {
    free(t->child); free(t->node_parent); free(t->node_key);
    free(t->leaf_parent); free(t->leaf_key); free(t->leaf_inside);
    memset(t, 0, sizeof(*t));
}

void oracle_free(void *p) { free(p); }

/* ------------------------------------------------------------------------------------------ */
/* segments: recursive ray-box descent                                                         */
/* ------------------------------------------------------------------------------------------ */

typedef struct { int32_t leaf; double t0, t1; } oseg;
typedef struct { oseg *s; int64_t n, cap; } segvec;

/* interval of the ray inside the box [lo, hi] (normalised).  On an axis with zero direction the
 * box contains the ray iff lo <= o < hi, with the upper face closed where it is the root's. */
static int slab(const double o[3], const double d[3], const double lo[3], const double hi[3],
                double *t0, double *t1) {
    double tn = -INFINITY, tf = INFINITY;
    for (int a = 0; a < 3; a++) {
        if (d[a] == 0.0) {
            int in = lo[a] <= o[a] && (hi[a] == 1.0 ? o[a] <= hi[a] : o[a] < hi[a]);
            if (!in) return 0;
        } else {
            double ta = (lo[a] - o[a]) / d[a], tb = (hi[a] - o[a]) / d[a];
            if (ta > tb) { double x = ta; ta = tb; tb = x; }
            if (ta > tn) tn = ta;
            if (tb < tf) tf = tb;
        }
    }
    *t0 = tn; *t1 = tf;
    return 1;
}

static void push_seg(segvec *v, int32_t leaf, double t0, double t1) {
    v->s = grow(v->s, &v->cap, v->n + 1, sizeof(oseg));
    v->s[v->n].leaf = leaf; v->s[v->n].t0 = t0; v->s[v->n].t1 = t1;
    v->n++;
}

static void descend(const otree *t, int32_t node, int l, const int64_t k[3], const double o[3],
                    const double d[3], segvec *out) {
    double cand_t0[8], cand_t1[8];
    int cand_j[8], nc = 0;
    double sz = ldexp(1.0, -(l + 1));
    for (int j = 0; j < 8; j++) {
        int64_t ck[3] = {2 * k[0] + ((j >> 2) & 1), 2 * k[1] + ((j >> 1) & 1), 2 * k[2] + (j & 1)};
        double lo[3], hi[3], t0, t1;
        for (int a = 0; a < 3; a++) { lo[a] = (double)ck[a] * sz; hi[a] = lo[a] + sz; }
        if (!slab(o, d, lo, hi, &t0, &t1)) continue;
        if (t0 < 0.0) t0 = 0.0;
        if (!(t1 > t0)) continue; /* empty or zero-length: dropped */
        /* insertion by (t0, slot) */
        int p = nc;
        while (p > 0 && cand_t0[p - 1] > t0) {
            cand_t0[p] = cand_t0[p - 1]; cand_t1[p] = cand_t1[p - 1]; cand_j[p] = cand_j[p - 1];
            p--;
        }
        cand_t0[p] = t0; cand_t1[p] = t1; cand_j[p] = j;
        nc++;
    }
    for (int c = 0; c < nc; c++) {
        int j = cand_j[c];
        int32_t ch = t->child[8 * (int64_t)node + j];
        if (ch >= 0) {
            int64_t ck[3] = {2 * k[0] + ((j >> 2) & 1), 2 * k[1] + ((j >> 1) & 1), 2 * k[2] + (j & 1)};
            descend(t, ch, l + 1, ck, o, d, out);
        } else {
            push_seg(out, -1 - ch, cand_t0[c], cand_t1[c]);
        }
    }
}

static void ray_segments(const otree *t, const oopts *op, const float *of, const float *df,
                         segvec *out) {
    double o[3], d[3];
    for (int a = 0; a < 3; a++) {
        o[a] = ((double)of[a] - op->root_lo[a]) / op->root_size;
        d[a] = (double)df[a] / op->root_size;
    }
    out->n = 0;
    double lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1}, t0, t1;
    if (!slab(o, d, lo, hi, &t0, &t1)) return;
    if (t0 < 0.0) t0 = 0.0;
    if (!(t1 > t0)) return;
    int64_t k[3] = {0, 0, 0};
    descend(t, 0, 0, k, o, d, out);
}

int64_t oracle_segments(const otree *t, const oopts *op, const float *o, const float *d,
                        int64_t cap, int32_t *leaf, double *t_in, double *t_out) {
    segvec v = {0};
    ray_segments(t, op, o, d, &v);
    int64_t n = v.n;
    if (n > cap) { free(v.s); return -n; }
    for (int64_t i = 0; i < n; i++) { leaf[i] = v.s[i].leaf; t_in[i] = v.s[i].t0; t_out[i] = v.s[i].t1; }
    free(v.s);
    return n;
}

/* ------------------------------------------------------------------------------------------ */
/* real spherical harmonics, degree 0..3, evaluated at the unit direction d                     */
/* ------------------------------------------------------------------------------------------ */

void oracle_sh_basis(int32_t deg, const double *dir, double *Y) {
    const double pi = acos(-1.0);
    double x = dir[0], y = dir[1], z = dir[2];
    Y[0] = 1.0 / (2.0 * sqrt(pi));
    if (deg < 1) return;
    double c1 = sqrt(3.0 / (4.0 * pi));
    Y[1] = -c1 * y; Y[2] = c1 * z; Y[3] = -c1 * x;
    if (deg < 2) return;
    double a = sqrt(15.0 / pi) / 2.0, b = sqrt(5.0 / pi) / 4.0, c = sqrt(15.0 / pi) / 4.0;
    Y[4] = a * x * y;
    Y[5] = -a * y * z;
    Y[6] = b * (2.0 * z * z - x * x - y * y);
    Y[7] = -a * x * z;
    Y[8] = c * (x * x - y * y);
    if (deg < 3) return;
    double p = sqrt(35.0 / (2.0 * pi)) / 4.0, q = sqrt(105.0 / pi) / 2.0;
    double s = sqrt(21.0 / (2.0 * pi)) / 4.0, u = sqrt(7.0 / pi) / 4.0, v = sqrt(105.0 / pi) / 4.0;
    Y[9] = -p * y * (3.0 * x * x - y * y);
    Y[10] = q * x * y * z;
    Y[11] = -s * y * (4.0 * z * z - x * x - y * y);
    Y[12] = u * z * (2.0 * z * z - 3.0 * x * x - 3.0 * y * y);
    Y[13] = -s * x * (4.0 * z * z - x * x - y * y);
    Y[14] = v * z * (x * x - y * y);
    Y[15] = -p * x * (x * x - 3.0 * y * y);
}

static double act(int mode, double zv) { return mode == 1 ? zv : 1.0 / (1.0 + exp(-zv)); }
static double act_grad(int mode, double cv) { return mode == 1 ? 1.0 : cv * (1.0 - cv); }

/* colour of leaf v seen along unit direction d: c = act(sum_k sh[v][ch][k] Y_k(d)) */
static void leaf_color(const oopts *op, const double *sh, int32_t v, const double *Y, double z[3],
                       double c[3]) {
    int K = (op->sh_degree + 1) * (op->sh_degree + 1);
    for (int ch = 0; ch < 3; ch++) {
        double acc = 0.0;
        for (int k = 0; k < K; k++) acc += sh[((int64_t)v * 3 + ch) * K + k] * Y[k];
        z[ch] = acc;
        c[ch] = act(op->color_act, acc);
    }
}

/* ------------------------------------------------------------------------------------------ */
/* render (Eq. 1-2) and signal (Sec. 3.1)                                                       */
/* ------------------------------------------------------------------------------------------ */

static void render_one(const otree *t, const oopts *op, const double *sigma, const double *sh,
                       const float *of, const float *df, double rgb[3], double *Tf,
                       double *signal, int32_t signal_mode, int32_t *nseg, double *margin) {
    segvec v = {0};
    ray_segments(t, op, of, df, &v);
    double dir[3] = {df[0], df[1], df[2]};
    double Y[16], z[3], c[3];
    oracle_sh_basis(op->sh_degree, dir, Y);
    double T = 1.0, C[3] = {0, 0, 0};
    double mg = INFINITY; /* closest approach of T_{i+1} to eps_T, relative to eps_T */
    int64_t i;
    for (i = 0; i < v.n; i++) {
        int32_t leaf = v.s[i].leaf;
        double delta = v.s[i].t1 - v.s[i].t0;
        double s = sigma[leaf] > 0.0 ? sigma[leaf] : 0.0;
        double alpha = 1.0 - exp(-s * delta);
        double w = T * alpha;
        leaf_color(op, sh, leaf, Y, z, c);
        for (int ch = 0; ch < 3; ch++) C[ch] += w * c[ch];
        if (signal) {
            if (signal_mode == 1) signal[leaf] += alpha;
            else if (signal_mode == 2 && w > signal[leaf]) signal[leaf] = w;
        }
        T = T * (1.0 - alpha);
        if (op->eps_T > 0.0) {
            double m = fabs(T - op->eps_T) / op->eps_T;
            if (m < mg) mg = m;
            if (T < op->eps_T) { i++; break; }
        }
    }
    for (int ch = 0; ch < 3; ch++) rgb[ch] = C[ch] + T * op->bg[ch];
    *Tf = T;
    if (nseg) *nseg = (int32_t)i;
    if (margin) *margin = mg;
    free(v.s);
}

int oracle_render(const otree *t, const oopts *op, const double *sigma, const double *sh,
                  int64_t n_rays, const float *o, const float *d, double *rgb, double *T_final,
                  double *signal, int32_t signal_mode, int32_t *n_seg, double *margin,
                  int32_t n_threads) {
    if (signal) { /* the signal is a shared accumulator: plain serial loop */
        for (int64_t r = 0; r < n_rays; r++)
            render_one(t, op, sigma, sh, o + 3 * r, d + 3 * r, rgb + 3 * r, T_final + r, signal,
                       signal_mode, n_seg ? n_seg + r : 0, margin ? margin + r : 0);
        return 0;
    }
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16) num_threads(n_threads > 0 ? n_threads : 1)
#endif
    for (int64_t r = 0; r < n_rays; r++)
        render_one(t, op, sigma, sh, o + 3 * r, d + 3 * r, rgb + 3 * r, T_final + r, 0, 0,
                   n_seg ? n_seg + r : 0, margin ? margin + r : 0);
    (void)n_threads;
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* backward: dL/dsh and dL/dsigma for L = sum_ch g_ch C_ch                                      */
/* ------------------------------------------------------------------------------------------ */

int oracle_backward(const otree *t, const oopts *op, const double *sigma, const double *sh,
                    int64_t n_rays, const float *o, const float *d, const double *grad_rgb,
                    double *grad_sigma, double *grad_sh, double *abs_sigma, double *abs_sh) {
    int K = (op->sh_degree + 1) * (op->sh_degree + 1);
    segvec v = {0};
    double *wv = NULL, *cv = NULL, *Tn = NULL, *dl = NULL;
    int64_t cap = 0;
    for (int64_t r = 0; r < n_rays; r++) {
        ray_segments(t, op, o + 3 * r, d + 3 * r, &v);
        if (v.n > cap) {
            cap = v.n;
            wv = realloc(wv, cap * sizeof(double));
            cv = realloc(cv, cap * 3 * sizeof(double));
            Tn = realloc(Tn, cap * sizeof(double));
            dl = realloc(dl, cap * sizeof(double));
        }
        double dir[3] = {d[3 * r], d[3 * r + 1], d[3 * r + 2]};
        double Y[16], z[3];
        oracle_sh_basis(op->sh_degree, dir, Y);
        /* forward, keeping per-segment values */
        double T = 1.0, C[3] = {0, 0, 0};
        int64_t n = 0;
        for (int64_t i = 0; i < v.n; i++) {
            int32_t leaf = v.s[i].leaf;
            double delta = v.s[i].t1 - v.s[i].t0;
            double s = sigma[leaf] > 0.0 ? sigma[leaf] : 0.0;
            double alpha = 1.0 - exp(-s * delta);
            double w = T * alpha;
            leaf_color(op, sh, leaf, Y, z, cv + 3 * i);
            for (int ch = 0; ch < 3; ch++) C[ch] += w * cv[3 * i + ch];
            T = T * (1.0 - alpha);
            wv[i] = w; Tn[i] = T; dl[i] = delta;
            n = i + 1;
            if (op->eps_T > 0.0 && T < op->eps_T) break;
        }
        for (int ch = 0; ch < 3; ch++) C[ch] += T * op->bg[ch]; /* C includes the background */
        const double *g = grad_rgb + 3 * r;
        double Cle[3] = {0, 0, 0};
        for (int64_t i = 0; i < n; i++) {
            int32_t leaf = v.s[i].leaf;
            const double *c = cv + 3 * i;
            for (int ch = 0; ch < 3; ch++) Cle[ch] += wv[i] * c[ch];
            /* dC/dsh[ch][k] = w act'(z) Y_k */
            for (int ch = 0; ch < 3; ch++) {
                double dz = g[ch] * wv[i] * act_grad(op->color_act, c[ch]);
                for (int k = 0; k < K; k++) {
                    double term = dz * Y[k];
                    grad_sh[((int64_t)leaf * 3 + ch) * K + k] += term;
                    if (abs_sh) abs_sh[((int64_t)leaf * 3 + ch) * K + k] += fabs(term);
                }
            }
            /* dC/dsigma = delta (T_{i+1} c_i - (C - C_{<=i})) where sigma > 0 */
            if (sigma[leaf] > 0.0) {
                double acc = 0.0;
                for (int ch = 0; ch < 3; ch++) acc += g[ch] * (Tn[i] * c[ch] - (C[ch] - Cle[ch]));
                double term = dl[i] * acc;
                grad_sigma[leaf] += term;
                if (abs_sigma) abs_sigma[leaf] += fabs(term);
            }
        }
    }
    free(v.s); free(wv); free(cv); free(Tn); free(dl);
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* selection                                                                                   */
/* ------------------------------------------------------------------------------------------ */

static const float *g_sort_sig;
/* Selection order of two signals: numeric order, with -0 and +0 equal (IEEE comparison) and a
 * NaN after every number in either direction; equal keys fall back to the leaf id. */
static int sig_order(float x, float y, int desc) {
    int nx = isnan(x), ny = isnan(y);
    if (nx || ny) return nx - ny;
    if (x < y) return desc ? 1 : -1;
    if (x > y) return desc ? -1 : 1;
    return 0;
}
static int cmp_desc(const void *a, const void *b) {
    int64_t i = *(const int64_t *)a, j = *(const int64_t *)b;
    int c = sig_order(g_sort_sig[i], g_sort_sig[j], 1);
    if (c) return c;
    return (i > j) - (i < j);
}
static int cmp_asc(const void *a, const void *b) {
    int64_t i = *(const int64_t *)a, j = *(const int64_t *)b;
    int c = sig_order(g_sort_sig[i], g_sort_sig[j], 0);
    if (c) return c;
    return (i > j) - (i < j);
}

/* the k = ceil(frac n) first leaves in the selection order; with ties, also every leaf whose
 * signal compares equal to the k-th (a threshold at the k-th value) */
static void rank_select(const float *s, int64_t n, double frac, int desc, int ties, uint8_t *mark) {
    int64_t k = (int64_t)ceil(frac * (double)n);
    if (k > n) k = n;
    if (k < 0) k = 0;
    int64_t *idx = malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    for (int64_t i = 0; i < n; i++) idx[i] = i;
    g_sort_sig = s;
    if (n > 1) qsort(idx, (size_t)n, sizeof(int64_t), desc ? cmp_desc : cmp_asc);
    for (int64_t i = 0; i < n; i++) mark[i] = 0;
    for (int64_t i = 0; i < k; i++) mark[idx[i]] = 1;
    if (ties && k > 0) {
        float kth = s[idx[k - 1]];
        for (int64_t i = 0; i < n; i++)
            if (sig_order(s[i], kth, desc) == 0) mark[i] = 1;
    }
    free(idx);
}

int oracle_select(const float *s, int64_t n, int32_t prune_mode, double prune_value,
                  int32_t sample_mode, double sample_value, uint8_t *prune_mark,
                  uint8_t *sample_mark) {
    if (prune_mode == 0) memset(prune_mark, 0, (size_t)n);
    else if (prune_mode == 1) { float thr = (float)prune_value; for (int64_t i = 0; i < n; i++) prune_mark[i] = s[i] <= thr; }
    else rank_select(s, n, prune_value, 0, prune_mode == 3, prune_mark);
    if (sample_mode == 0) memset(sample_mark, 0, (size_t)n);
    else if (sample_mode == 1) { float thr = (float)sample_value; for (int64_t i = 0; i < n; i++) sample_mark[i] = s[i] > thr; }
    else rank_select(s, n, sample_value, 1, sample_mode == 3, sample_mark);
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* refine: prune (Eq. 3) and sample (Eq. 4)                                                    */
/* ------------------------------------------------------------------------------------------ */

/* Eq. 3 with M = 8, summed pairwise so that 8 identical values average exactly */
static double mean8(const double x[8]) {
    return (((x[0] + x[1]) + (x[2] + x[3])) + ((x[4] + x[5]) + (x[6] + x[7]))) / 8.0;
}

int oracle_refine(const otree *t, const double *sigma, const double *sh, int32_t n_sh,
                  const uint8_t *prune, const uint8_t *sample, int32_t d_cap, otree *out,
                  int32_t **leaf_map_out, double **sigma_out, double **sh_out,
                  orefine_counts *cnt) {
    int64_t N = t->n_nodes, L = t->n_leaves;
    uint8_t *prunable = calloc((size_t)(N > 0 ? N : 1), 1);
    uint8_t *sampled = calloc((size_t)(L > 0 ? L : 1), 1);
    int64_t *node_new = malloc((size_t)(N > 0 ? N : 1) * sizeof(int64_t));
    int64_t *leaf_new = malloc((size_t)(L > 0 ? L : 1) * sizeof(int64_t));   /* survivors */
    int64_t *merged_new = malloc((size_t)(N > 0 ? N : 1) * sizeof(int64_t)); /* merged parents */
    int64_t *inner_new = malloc((size_t)(L > 0 ? L : 1) * sizeof(int64_t));  /* sampled leaves */
    int64_t *child_base = malloc((size_t)(L > 0 ? L : 1) * sizeof(int64_t)); /* first new child */
    memset(cnt, 0, sizeof(*cnt));

    /* 1. a parent (never the root) is merged iff its 8 children are leaves, all prune-marked
     *    and none sample-marked */
    for (int64_t p = 1; p < N; p++) {
        int ok = 1;
        for (int j = 0; j < 8; j++) {
            int32_t ch = t->child[8 * p + j];
            if (ch >= 0) { ok = 0; break; }
            int32_t v = -1 - ch;
            if (!prune[v] || sample[v]) { ok = 0; break; }
        }
        prunable[p] = (uint8_t)ok;
    }
    /* 2. a leaf is subdivided iff sample-marked, above the depth cap and its parent survives */
    for (int64_t v = 0; v < L; v++) {
        if (!sample[v]) continue;
        if (key_level(t->leaf_key[v]) >= d_cap) { cnt->n_capped++; continue; }
        if (prunable[t->leaf_parent[v]]) continue;
        sampled[v] = 1;
    }
    /* 3. numbering: leaves = survivors (old order), merged parents (old node order), children
     *    of sampled leaves (old leaf order x slot); nodes = surviving nodes (old order), then
     *    sampled leaves (old leaf order) */
    int64_t nl = 0, nn = 0;
    for (int64_t v = 0; v < L; v++) {
        leaf_new[v] = -1;
        if (!prunable[t->leaf_parent[v]] && !sampled[v]) leaf_new[v] = nl++;
    }
    for (int64_t p = 0; p < N; p++) {
        merged_new[p] = -1;
        if (prunable[p]) { merged_new[p] = nl++; cnt->n_pruned_groups++; }
    }
    for (int64_t v = 0; v < L; v++) {
        child_base[v] = -1;
        if (sampled[v]) { child_base[v] = nl; nl += 8; cnt->n_sampled++; }
    }
    for (int64_t p = 0; p < N; p++) {
        node_new[p] = -1;
        if (!prunable[p]) node_new[p] = nn++;
    }
    for (int64_t v = 0; v < L; v++) {
        inner_new[v] = -1;
        if (sampled[v]) inner_new[v] = nn++;
    }
    cnt->n_nodes = nn;
    cnt->n_leaves = nl;

    memset(out, 0, sizeof(*out));
    out->n_nodes = nn;
    out->n_leaves = nl;
    out->child = malloc((size_t)(nn > 0 ? nn : 1) * 8 * sizeof(int32_t));
    out->node_parent = malloc((size_t)(nn > 0 ? nn : 1) * sizeof(int32_t));
    out->node_key = malloc((size_t)(nn > 0 ? nn : 1) * sizeof(uint64_t));
    out->leaf_parent = malloc((size_t)(nl > 0 ? nl : 1) * sizeof(int32_t));
    out->leaf_key = malloc((size_t)(nl > 0 ? nl : 1) * sizeof(uint64_t));
    out->leaf_inside = calloc((size_t)(nl > 0 ? nl : 1), 1);
    int32_t *lm = malloc((size_t)(nl > 0 ? nl : 1) * sizeof(int32_t));
    double *so = malloc((size_t)(nl > 0 ? nl : 1) * sizeof(double));
    double *sho = malloc((size_t)(nl > 0 ? nl : 1) * (size_t)n_sh * sizeof(double));

    /* 4. surviving internal nodes and their child pointers */
    for (int64_t p = 0; p < N; p++) {
        if (prunable[p]) continue;
        int64_t q = node_new[p];
        out->node_parent[q] = t->node_parent[p] >= 0 ? (int32_t)node_new[t->node_parent[p]] : -1;
        out->node_key[q] = t->node_key[p];
        for (int j = 0; j < 8; j++) {
            int32_t ch = t->child[8 * p + j];
            int32_t nc;
            if (ch >= 0) nc = prunable[ch] ? -1 - (int32_t)merged_new[ch] : (int32_t)node_new[ch];
            else {
                int32_t v = -1 - ch;
                nc = sampled[v] ? (int32_t)inner_new[v] : -1 - (int32_t)leaf_new[v];
            }
            out->child[8 * q + j] = nc;
        }
    }
    /* 5. sampled leaves become internal nodes with 8 new leaf children (Eq. 4: exact copies) */
    for (int64_t v = 0; v < L; v++) {
        if (!sampled[v]) continue;
        int64_t q = inner_new[v];
        out->node_parent[q] = (int32_t)node_new[t->leaf_parent[v]];
        out->node_key[q] = t->leaf_key[v];
        for (int j = 0; j < 8; j++) {
            int64_t u = child_base[v] + j;
            out->child[8 * q + j] = -1 - (int32_t)u;
            out->leaf_parent[u] = (int32_t)q;
            out->leaf_key[u] = (t->leaf_key[v] << 3) | (uint64_t)j;
            lm[u] = (int32_t)v;
            so[u] = sigma[v];
            for (int c = 0; c < n_sh; c++) sho[u * n_sh + c] = sh[v * n_sh + c];
        }
    }
    /* 6. survivors keep their values */
    for (int64_t v = 0; v < L; v++) {
        if (leaf_new[v] < 0) continue;
        int64_t u = leaf_new[v];
        out->leaf_parent[u] = (int32_t)node_new[t->leaf_parent[v]];
        out->leaf_key[u] = t->leaf_key[v];
        lm[u] = (int32_t)v;
        so[u] = sigma[v];
        for (int c = 0; c < n_sh; c++) sho[u * n_sh + c] = sh[v * n_sh + c];
    }
    /* 7. merged parents become leaves holding the mean of their 8 children (Eq. 3, M = 8) */
    for (int64_t p = 0; p < N; p++) {
        if (!prunable[p]) continue;
        int64_t u = merged_new[p];
        out->leaf_parent[u] = (int32_t)node_new[t->node_parent[p]];
        out->leaf_key[u] = t->node_key[p];
        lm[u] = -1 - (int32_t)p;
        double x[8];
        for (int j = 0; j < 8; j++) x[j] = sigma[-1 - t->child[8 * p + j]];
        so[u] = mean8(x);
        for (int c = 0; c < n_sh; c++) {
            for (int j = 0; j < 8; j++) x[j] = sh[(int64_t)(-1 - t->child[8 * p + j]) * n_sh + c];
            sho[u * n_sh + c] = mean8(x);
        }
    }
    *leaf_map_out = lm;
    *sigma_out = so;
    *sh_out = sho;
    free(prunable); free(sampled); free(node_new); free(leaf_new); free(merged_new);
    free(inner_new); free(child_base);
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* optimisation step (Algorithm 1, optimization; Sec. 3.3; Sec. 4.1)                           */
/* ------------------------------------------------------------------------------------------ */

/* Mean squared error of the prediction against the target over n rays x 3 channels (Algorithm 1
 * computes loss = MSE(pred, GT) on stochastic image samples, Sec. 4.1):
 * loss = (1 / 3n) sum (rgb - target)^2, and its gradient 2 (rgb - target) / 3n. */
double oracle_mse(int64_t n, const double *rgb, const double *target, double *grad) {
    double loss = 0.0;
    const double inv = n > 0 ? 1.0 / (3.0 * (double)n) : 0.0;
    for (int64_t i = 0; i < 3 * n; i++) {
        const double e = rgb[i] - target[i];
        loss += e * e;
        if (grad) grad[i] = 2.0 * e * inv;
    }
    return loss * inv;
}

/* One RMSProp update of n parameters (Sec. 3.3 optimises the cached coefficients with RMSProp;
 * Sec. 4.1 gives learning rates 0.1 for sigma and 0.01 for the SH colour):
 *   ms <- rho ms + (1 - rho) g^2,   p <- p - lr g / (sqrt(ms) + eps). */
void oracle_rmsprop(int64_t n, double *param, double *ms, const double *grad, double lr,
                    double rho, double eps) {
    for (int64_t i = 0; i < n; i++) {
        ms[i] = rho * ms[i] + (1.0 - rho) * grad[i] * grad[i];
        param[i] = param[i] - lr * grad[i] / (sqrt(ms[i]) + eps);
    }
}

/* ------------------------------------------------------------------------------------------ */
/* compressed models: median-cut quantisation of the SH coefficient vectors (Sec. 4.1)          */
/* ------------------------------------------------------------------------------------------ */

static const double *mc_x;   /* the vectors being sorted (qsort has no context argument) */
static int mc_dim, mc_axis;

static int mc_cmp(const void *a, const void *b) {
    const int64_t i = *(const int64_t *)a, j = *(const int64_t *)b;
    const double u = mc_x[i * mc_dim + mc_axis], v = mc_x[j * mc_dim + mc_axis];
    if (u < v) return -1;
    if (u > v) return 1;
    return (i > j) - (i < j);
}

/* Median cut (Heckbert 1982, the quantiser Sec. 4.1 applies to the SH coefficients): n vectors of
 * dimension dim go into 2^bits boxes.  Starting from one box holding every vector, each of the
 * bits rounds splits every box of two or more vectors at the median of its longest side: the
 * axis of largest (max - min) (ties to the lowest axis), members ordered by (value on that axis,
 * vector id), the first floor(m/2) to child 2b and the rest to child 2b+1 (a box of fewer than two
 * keeps its members in child 2b).  The palette entry of a box is the mean of its members (zeros
 * for an empty box).  index[n] receives each vector's box; palette is [2^bits][dim]. */
int oracle_median_cut(int64_t n, int32_t dim, const double *x, int32_t bits, int32_t *index,
                      double *palette) {
    const int64_t P = (int64_t)1 << bits;
    int64_t *order = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    int64_t *start = (int64_t *)calloc((size_t)P + 1, sizeof(int64_t));
    int64_t *nstart = (int64_t *)calloc((size_t)P + 1, sizeof(int64_t));
    if (!order || !start || !nstart) return -1;
    for (int64_t i = 0; i < n; i++) order[i] = i;
    int64_t boxes = 1;
    start[0] = 0;
    start[1] = n;
    mc_x = x;
    mc_dim = dim;
    for (int r = 0; r < bits; r++) {
        for (int64_t b = 0; b < boxes; b++) {
            const int64_t s = start[b], e = start[b + 1], m = e - s;
            nstart[2 * b] = s;
            if (m < 2) {
                nstart[2 * b + 1] = e;
                continue;
            }
            int axis = 0;
            double best = -1.0;
            for (int d = 0; d < dim; d++) {
                double lo = x[order[s] * dim + d], hi = lo;
                for (int64_t k = s + 1; k < e; k++) {
                    const double v = x[order[k] * dim + d];
                    if (v < lo) lo = v;
                    if (v > hi) hi = v;
                }
                if (hi - lo > best) {
                    best = hi - lo;
                    axis = d;
                }
            }
            mc_axis = axis;
            qsort(order + s, (size_t)m, sizeof(int64_t), mc_cmp);
            nstart[2 * b + 1] = s + m / 2;
        }
        nstart[2 * boxes] = n;
        boxes *= 2;
        for (int64_t b = 0; b <= boxes; b++) start[b] = nstart[b];
    }
    for (int64_t b = 0; b < P; b++) {
        for (int d = 0; d < dim; d++) palette[b * dim + d] = 0.0;
        const int64_t s = start[b], e = start[b + 1];
        for (int64_t k = s; k < e; k++) {
            index[order[k]] = (int32_t)b;
            for (int d = 0; d < dim; d++) palette[b * dim + d] += x[order[k] * dim + d];
        }
        if (e > s)
            for (int d = 0; d < dim; d++) palette[b * dim + d] /= (double)(e - s);
    }
    free(order);
    free(start);
    free(nstart);
    return 0;
}
