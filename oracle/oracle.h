/*
 * oracle.h -- FP64 CPU oracle of the Dynamic PlenOctree (DOT) hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's CPU-baseline leg
 * load this library; the product path (the CUDA library) never calls it, and the two share no
 * source, header, table or constant.
 *
 * Coordinates: the root cube [lo, lo + size]^3 is mapped to [0,1]^3.  A cell at level l with
 * integer corner k covers [k 2^-l, (k+1) 2^-l).  Keys are Morton codes with a leading 1 bit:
 * key = (1 << 3l) | interleave(kx, ky, kz) with x the most significant bit of each triple, so the
 * child in slot j = 4 bx + 2 by + bz of a cell has key (key << 3) | j.
 * Child pointers: >= 0 internal node id, < 0 leaf id v encoded as -1 - v.
 */
#ifndef DOT_ORACLE_H
#define DOT_ORACLE_H
#include <stdint.h>

typedef struct {
    int64_t n_nodes, n_leaves;
    int32_t *child;        /* [n_nodes][8] */
    int32_t *node_parent;  /* [n_nodes], -1 for the root */
    uint64_t *node_key;    /* [n_nodes] */
    int32_t *leaf_parent;  /* [n_leaves] */
    uint64_t *leaf_key;    /* [n_leaves] */
    uint8_t *leaf_inside;  /* [n_leaves]: the leaf's cell meets a primitive (build only) */
} otree;

typedef struct {
    double root_lo[3];
    double root_size;      /* edge length 2h of the root cube */
    int32_t sh_degree;     /* 0..3 */
    int32_t color_act;     /* 0 sigmoid, 1 linear */
    double bg[3];
    double eps_T;          /* stop after the segment that takes T below eps_T; 0 disables */
} oopts;

/* build: returns 0 on success; allocates the arrays of *out (free with oracle_tree_free) */
int oracle_build(const int64_t *prims, int32_t n_prims, int32_t max_depth, otree *out);
void oracle_tree_free(otree *t);

/* segment list of one ray: returns the count (or -needed if cap is too small) */
int64_t oracle_segments(const otree *t, const oopts *op, const float *o, const float *d,
                        int64_t cap, int32_t *leaf, double *t_in, double *t_out);

void oracle_sh_basis(int32_t deg, const double *d, double *Y);

/* forward render (Eq. 1-2).  sigma [L], sh [L][3][K] raw (pre-activation) values.
 * signal (nullable): accumulated in place with mode 1 = sum of alpha, 2 = max of weight.
 * margin (nullable): per ray, min over segments of |T_{i+1} - eps_T| / eps_T (infinity when
 * eps_T = 0): how close the early-termination decision came to going the other way. */
int oracle_render(const otree *t, const oopts *op, const double *sigma, const double *sh,
                  int64_t n_rays, const float *o, const float *d, double *rgb, double *T_final,
                  double *signal, int32_t signal_mode, int32_t *n_seg, double *margin,
                  int32_t n_threads);

/* gradient of sum(grad_rgb . rgb) with respect to sigma and sh, accumulated (+=) in place;
 * abs_sigma / abs_sh (nullable) accumulate the magnitudes of the summed terms. */
int oracle_backward(const otree *t, const oopts *op, const double *sigma, const double *sh,
                    int64_t n_rays, const float *o, const float *d, const double *grad_rgb,
                    double *grad_sigma, double *grad_sh, double *abs_sigma, double *abs_sh);

/* selection: mode 1 threshold (prune: S <= thr, sample: S > thr), mode 2 rank fraction
 * (prune: the ceil(f L) smallest by (S asc, id asc); sample: the ceil(f L) largest by
 * (S desc, id asc)), mode 3 quantile (mode 2 plus every leaf whose signal equals the last one
 * taken).  Signals compare as IEEE floats (-0 equals +0); a NaN is never marked by a
 * threshold and comes after every number in both rank orders. */
int oracle_select(const float *signal, int64_t n, int32_t prune_mode, double prune_value,
                  int32_t sample_mode, double sample_value, uint8_t *prune_mark,
                  uint8_t *sample_mark);

typedef struct {
    int64_t n_nodes, n_leaves, n_pruned_groups, n_sampled, n_capped;
} orefine_counts;

/* prune (Eq. 3) and sample (Eq. 4) given masks; allocates *out and the returned arrays */
int oracle_refine(const otree *t, const double *sigma, const double *sh, int32_t n_sh,
                  const uint8_t *prune_mark, const uint8_t *sample_mark, int32_t d_cap,
                  otree *out, int32_t **leaf_map, double **sigma_out, double **sh_out,
                  orefine_counts *counts);

/* MSE over n rays x 3 channels (Algorithm 1, optimization): returns (1/3n) sum (rgb - target)^2
 * and writes its gradient 2 (rgb - target) / 3n to grad (nullable). */
double oracle_mse(int64_t n, const double *rgb, const double *target, double *grad);

/* RMSProp (Sec. 3.3) in place over n entries: ms <- rho ms + (1 - rho) g^2,
 * p <- p - lr g / (sqrt(ms) + eps). */
void oracle_rmsprop(int64_t n, double *param, double *ms, const double *grad, double lr,
                    double rho, double eps);

/* Median cut (Heckbert 1982; Sec. 4.1 compressed models) of n vectors of dimension dim into
 * 2^bits boxes, every round splitting every box of >= 2 members at the median of its longest
 * axis (ties: lowest axis; order (value, id); floor(m/2) members to the lower child).  Writes each
 * vector's box to index[n] and the box means (zeros when empty) to palette[2^bits][dim]. */
int oracle_median_cut(int64_t n, int32_t dim, const double *x, int32_t bits, int32_t *index,
                      double *palette);

void oracle_free(void *p);

#endif
