/*
 * dot.h -- C ABI of the GB300 Dynamic PlenOctree (DOT) hot path.
 *
 * The library renders rays through a sparse octree whose leaves hold a density sigma and
 * degree-0..3 real spherical-harmonic colour coefficients (Sec. 3, Preliminaries, Eq. 1-2),
 * differentiates that render, accumulates the per-leaf training signal of Sec. 3.1, selects
 * leaves by threshold or rank (Sec. 3.2, Algorithm 1), and restructures the tree by the prune
 * (Eq. 3) and sample (Eq. 4) operations.  Every call runs hand-written sm_103a CUDA kernels.
 *
 * Conventions shared by every call
 *  - Every call returns an int status: DOT_OK (0) or a negative DOT_ERR_* code; the message of
 *    the last failure on the calling thread is returned by dot_last_error().
 *  - Argument errors (null pointers, sizes out of range, unsupported degrees or modes) are
 *    detected on the host before any launch; nothing is launched then and outputs are untouched.
 *  - "stream" is a cudaStream_t passed as void* (NULL = the legacy default stream).  Calls are
 *    asynchronous on it unless stated otherwise.
 *  - Device pointers passed in are owned by the caller; the library never frees them.  The
 *    library owns the opaque dot_tree and the arrays it holds; those are allocated through the
 *    caller's dot_allocator when one is given, else with cudaMallocAsync on the call's stream.
 *  - Anomalies seen inside kernels (a ray exceeding the step cap) set bits of a per-tree device
 *    status word, read and cleared by dot_tree_status().
 *  - Besides the arrays of dot_tree_info, a tree keeps a face-neighbour table (24 bytes per
 *    leaf) that the renders follow from leaf to leaf; every call that changes the structure
 *    rebuilds it.  A tree holds at most 2^27 leaves: a build, import, refine or renumbering that
 *    would exceed that fails with DOT_ERR_UNSUPPORTED.
 *
 * Geometry
 *  - The root cube is [c - h, c + h]^3 (world units).  A cell at level l (root = 0) with
 *    integer corner k covers [k, k + 1) * 2^-l of the root in each axis.  Levels go up to 16.
 *  - Keys: key = (1 << 3l) | interleave(kx, ky, kz) with x the most significant bit of each
 *    triple; the child in slot j = 4 bx + 2 by + bz of a cell has key (key << 3) | j.
 *  - Child table child[n][8]: >= 0 internal node id, < 0 leaf id v stored as -1 - v.  Node 0 is
 *    the root; the root is always internal.
 *  - Leaf parameters: sigma[L] and sh[L][row] in the storage type, where a row holds the SH
 *    coefficients [3 channels][K] (K = (degree + 1)^2) padded to a multiple of 16 bytes
 *    (row = sh_row_stride elements).  Colour c = act(sum_k sh[ch][k] Y_k(d)) with the real SH
 *    basis Y_k evaluated at the unit ray direction d; density max(sigma, 0).
 */
#ifndef DOT_H
#define DOT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DOT_OK 0
#define DOT_ERR_INVALID_ARG (-1)
#define DOT_ERR_OOM (-2)
#define DOT_ERR_CUDA (-3)
#define DOT_ERR_STEP_LIMIT (-4)
#define DOT_ERR_UNSUPPORTED (-5)

#define DOT_STORAGE_F32 0
#define DOT_STORAGE_F16 1
#define DOT_STORAGE_BF16 2

#define DOT_PRIM_SPHERE 0   /* p = (cx, cy, cz, r) */
#define DOT_PRIM_BOX 1      /* p = (lox, loy, loz, hix, hiy, hiz) */
#define DOT_PRIM_CYLINDER 2 /* p = (cx, cz, r, y0, y1): axis along +y */

#define DOT_ACT_SIGMOID 0
#define DOT_ACT_LINEAR 1

#define DOT_SIGNAL_NONE 0
#define DOT_SIGNAL_SUM_ALPHA 1  /* S_v += 1 - exp(-sigma delta) over every segment in v (Sec. 3.1) */
#define DOT_SIGNAL_MAX_WEIGHT 2 /* S_v = max(S_v, T alpha) */
#define DOT_SIGNAL_SIGMA 3      /* S_v = max(sigma_v, 0) (the density signal of Sec. 3.1) */

#define DOT_SELECT_NONE 0
#define DOT_SELECT_THRESHOLD 1 /* prune: S <= value; sample: S > value (Sec. 3.2) */
#define DOT_SELECT_FRACTION 2  /* prune: ceil(value L) smallest by (S asc, id asc);
                                  sample: ceil(value L) largest by (S desc, id asc) (Algorithm 1) */
#define DOT_SELECT_QUANTILE 3  /* the FRACTION selection widened to every leaf whose signal equals
                                  the last one taken: prune S <= the ceil(value L)-th smallest, sample
                                  S >= the ceil(value L)-th largest (a threshold at a quantile) */

#define DOT_MERGE_MEAN 0
#define DOT_MERGE_SUM 1
#define DOT_MERGE_MAX 2

#define DOT_RAYS_BUFFER 0
#define DOT_RAYS_CAMERAS 1

#define DOT_PRECISION_AUTO 0  /* F32 storage -> exact-t, 16-bit storage -> fast */
#define DOT_PRECISION_FAST 1  /* float32 plane times and fast exponentials */
#define DOT_PRECISION_EXACT 2 /* float-float plane times and full-precision exponentials */

#define DOT_STATUS_STEP_LIMIT 1u /* a ray hit the step cap; its output is truncated */
#define DOT_STATUS_BAD_INPUT 2u  /* a device-side input was out of range and was skipped */

typedef struct dot_tree dot_tree;

/* Caller-supplied allocator for the arrays the tree owns.  alloc returns NULL on failure, else a
 * block of at least `bytes` bytes, 16-byte aligned, usable in stream order on `stream`; a
 * misaligned block is handed back to free at once and counts as a failed allocation
 * (DOT_ERR_OOM).  free receives the stream of the call that releases the block. */
typedef struct {
    void *ctx;
    void *(*alloc)(void *ctx, size_t bytes, void *stream);
    void (*free)(void *ctx, void *ptr, void *stream);
} dot_allocator;

/* One primitive; parameters are integers in units of 2^-24 of the root edge, measured from the
 * root's low corner (the layout of an int64 [n][8] array). */
typedef struct {
    int64_t type;
    int64_t p[7];
} dot_primitive;

typedef struct {
    float center[3];
    float half_size;
    int32_t max_depth;  /* D, 1..16 */
    int32_t sh_degree;  /* 0..3 */
    int32_t storage;    /* DOT_STORAGE_* */
    int32_t n_primitives;
    const dot_primitive *primitives; /* HOST pointer, n_primitives entries (<= 4096) */
    float density_lo, density_hi;    /* sigma ~ U(lo, hi) in finest cells meeting the scene */
    float sh_std, sh_dc;             /* SH ~ N(0, std) (Irwin-Hall n = 4), DC term + dc */
    uint64_t seed;
} dot_build_desc;

typedef struct {
    int64_t n_nodes, n_leaves;
    int32_t max_level;     /* deepest level holding a leaf */
    int32_t sh_degree;
    int32_t n_coeffs;      /* K */
    int32_t storage;
    int32_t sh_row_stride; /* elements per SH row (>= 3K, row bytes a multiple of 16) */
    int32_t pad_;
    float center[3];
    float half_size;
    int32_t *child;        /* device [n_nodes][8] */
    int32_t *node_parent;  /* device [n_nodes] (-1 for the root) */
    uint64_t *node_key;    /* device [n_nodes] */
    int32_t *leaf_parent;  /* device [n_leaves] */
    uint64_t *leaf_key;    /* device [n_leaves] */
    void *sigma;           /* device [n_leaves], storage type */
    void *sh;              /* device [n_leaves][sh_row_stride], storage type; NULL if compressed */
    int32_t palette_bits;  /* 0, or the palette of a compressed tree has 2^palette_bits rows */
    int32_t pad2_;
    void *palette;         /* device [2^palette_bits][sh_row_stride], storage type, or NULL */
    uint32_t *leaf_record; /* device [n_leaves]: density bits | palette row << 16, or NULL */
    int32_t *rope;         /* device [n_leaves][6], read-only: across face 2 axis + (1 for the upper
                              face) of leaf v, the node id (>= 0) at v's level when the tree is
                              finer there, else -1 - (u << 4 | d) for the leaf u covering that
                              place, d levels coarser than v, or INT32_MIN outside the root */
} dot_tree_info;

/* Host copy of a tree (checkpoint / import).  sh is [n_leaves][3K] without row padding. */
typedef struct {
    int64_t n_nodes, n_leaves;
    int32_t sh_degree, storage;
    float center[3];
    float half_size;
    const int32_t *child;
    const int32_t *node_parent;
    const uint64_t *node_key;
    const int32_t *leaf_parent;
    const uint64_t *leaf_key;
    const void *sigma;
    const void *sh;
} dot_host_tree;

/* Pinhole camera: c2w row-major 3x4 (columns right, up, back, position); looks down -z.
 * Pixel (i, j) (column, row from the top) has the ray built by these float32 round-to-nearest
 * operations: xc = ((i + .5) - cx) / fx, yc = -(((j + .5) - cy) / fy),
 * e_a = ((R[a][0] xc) + (R[a][1] yc)) - R[a][2], d = e * (1 / sqrt((e0 e0 + e1 e1) + e2 e2)). */
typedef struct {
    float c2w[12];
    float fx, fy, cx, cy;
    int32_t width, height;
} dot_camera;

typedef struct {
    int32_t kind;      /* DOT_RAYS_BUFFER or DOT_RAYS_CAMERAS */
    int32_t n_cameras; /* CAMERAS */
    const dot_camera *cameras; /* CAMERAS: device [n_cameras] */
    int32_t width, height;     /* CAMERAS: shared by every camera; ray id = (cam H + j) W + i */
    int64_t n_rays;            /* BUFFER */
    const float *origins;      /* BUFFER: device [n_rays][3] */
    const float *dirs;         /* BUFFER: device [n_rays][3], unit length */
    const int32_t *view_order; /* CAMERAS: device [n_cameras] or NULL -- the order in which the
                                  views are rendered (a permutation; ray ids are unchanged).  A
                                  locality-friendly order (dot_camera_order) lets consecutive views
                                  reuse the leaves left in L2.  Entries out of range are skipped
                                  and set DOT_STATUS_BAD_INPUT */
} dot_rays;

#define DOT_MAX_SERVE_TREES 8

/* One admitted request of a slot table (96 bytes): a camera (its own width and height), the
 * index of the tree it looks at, its first work tile, and its device output [height][width][3]. */
typedef struct {
    dot_camera camera;
    int32_t tree;
    int32_t pad_;
    int64_t tile_begin; /* sum of ceil(W/16) ceil(H/8) over the slots before this one */
    float *out;
} dot_slot;

/* A slot table in device memory is this header followed by max_slots dot_slot records. */
typedef struct {
    int32_t n_slots;
    int32_t pad_;
    int64_t total_tiles; /* tile_begin of the last slot plus its tile count */
} dot_slot_table_header;

typedef struct {
    float background[3];  /* added as T_final * background */
    float eps_T;          /* stop after the segment that takes T below eps_T; 0 disables; < 1 */
    int32_t color_act;    /* DOT_ACT_* */
    int32_t signal_mode;  /* fused signal in render calls: NONE, SUM_ALPHA or MAX_WEIGHT */
    int32_t precision;    /* DOT_PRECISION_* */
    int32_t max_steps;    /* per-ray cell-step cap; 0 = 3 * 2^max_level + 64 */
} dot_render_opts;

typedef struct {
    int32_t prune_mode;  /* DOT_SELECT_* */
    int32_t sample_mode;
    double prune_value;  /* tau, or the fraction of leaves */
    double sample_value; /* gamma, or the fraction of leaves */
} dot_select_opts;

typedef struct {
    int64_t n_nodes, n_leaves;  /* after the refine */
    int64_t n_pruned_groups;    /* parents merged (Eq. 3) */
    int64_t n_sampled;          /* leaves subdivided (Eq. 4) */
    int64_t n_capped;           /* sample marks ignored at the depth cap */
} dot_refine_counts;

/* A per-leaf FP32 array carried through a refine: dst[new][width] from src[old][width]. */
typedef struct {
    const float *src;
    float *dst;
    int32_t width;
    int32_t merge; /* DOT_MERGE_*: how the 8 children of a merged parent combine */
} dot_leaf_array;

/* Message of the last failure on this thread ("" if none). */
const char *dot_last_error(void);

/* ABI version (major * 100 + minor). */
int dot_version(void);

/*
 * dot_octree_build -- the octree of the primitive union (Sec. 3 Preliminaries: POT's octree,
 * here carved from seeded primitives in place of a trained NeRF-SH, Sec. 4.1).
 * The root is always subdivided; a cell is subdivided while its open interior meets a primitive
 * (integer-exact tests) and its level is below max_depth.  Numbering is canonical: nodes and
 * leaves each in breadth-first order, by Morton key within a level.  Leaves at max_depth meeting
 * the scene get sigma ~ U(density_lo, density_hi), others sigma = 0; every leaf gets SH
 * coefficients; values are drawn by SplitMix64(seed) at counter 64 key + component and rounded
 * to the storage type.  Synchronises the stream once per level.  *out receives a new tree.
 */
int dot_octree_build(const dot_build_desc *desc, const dot_allocator *alloc, void *stream,
                     dot_tree **out);

/* Frees the tree and its arrays (stream-ordered on the stream of the last call). */
int dot_tree_free(dot_tree *tree);

/* Sizes and device pointers of the tree (valid until the next refine or free). */
int dot_tree_get_info(const dot_tree *tree, dot_tree_info *info);

/* Copies the tree to host buffers sized from dot_tree_get_info (sh without row padding: [L][3K]).
 * Any pointer may be NULL to skip that array.  Synchronises the stream. */
int dot_tree_export(const dot_tree *tree, void *stream, int32_t *child, int32_t *node_parent,
                    uint64_t *node_key, int32_t *leaf_parent, uint64_t *leaf_key, void *sigma,
                    void *sh);

/* Creates a tree from host arrays after checking that they describe a valid octree (child
 * pointers in range, each node and leaf referenced once, keys consistent with parents). */
int dot_tree_import(const dot_host_tree *host, const dot_allocator *alloc, void *stream,
                    dot_tree **out);

/* Synchronises the stream, returns the tree's device status bits (DOT_STATUS_*) and clears
 * them. */
int dot_tree_status(dot_tree *tree, void *stream, uint32_t *status);

/*
 * dot_camera_order -- a rendering order for n cameras (HOST array) in which consecutive views are
 * close: a greedy nearest-neighbour chain over the camera positions starting at camera 0.  Written
 * to order[n] (host); pass it (copied to the device) as dot_rays.view_order.
 */
int dot_camera_order(const dot_camera *cameras, int32_t n, int32_t *order);

/*
 * dot_render_forward -- Eq. 1-2 per ray: the ray's segments through the leaves in order,
 * alpha_i = 1 - exp(-max(sigma,0) delta_i), w_i = T_i alpha_i, C = sum_i w_i c_i + T bg,
 * stopping after the segment that takes T below eps_T.
 * rgb: device [R][3] float (written); T_final: device [R] or NULL; signal: device [L] or NULL,
 * accumulated with opts->signal_mode (the caller initialises it).
 */
int dot_render_forward(const dot_tree *tree, const dot_rays *rays, const dot_render_opts *opts,
                       float *rgb, float *T_final, float *signal, void *stream);

/*
 * dot_render_views_host -- dot_render_forward over n_cameras whole camera views whose cameras and
 * images live in HOST memory (Eq. 1-2 per pixel; every value equals dot_render_forward's for the
 * same camera).  The views are rendered in view_order when given, so that consecutive views
 * reuse the leaves left in L2.  When rgb (and T_final) lie in page-locked host memory mapped into
 * the device's address space (cudaHostAlloc, or cudaHostRegister with mapping; with unified
 * addressing every page-locked allocation is), one launch writes every image in place.
 * Otherwise the views are rendered in chunks of about 2^23 rays (the views left after the full
 * chunks in halving chunks down to one view), alternately on `stream` and on a second render
 * stream, into a ring of three chunk buffers in the workspace, and each finished chunk is copied
 * to the host on a copy stream while the next chunks render.  The work is ordered after what
 * `stream` already holds; the call returns after every image is in rgb (and T_final).
 * cameras: host [n_cameras] dot_camera (copied to the workspace by this call).  width, height: the
 * resolution shared by every camera.  view_order: host [n_cameras] or NULL -- the render order, a
 * permutation of 0..n_cameras-1 (anything else fails with DOT_ERR_INVALID_ARG before any work).
 * rgb: host [n_cameras][height][width][3] float (written); T_final: host [n_cameras][height][width]
 * float or NULL.  Page-locked host buffers (cudaHostAlloc, cudaHostRegister) let the copies run
 * asynchronously at the link's speed; pageable ones work, through the driver's staging copies.
 * workspace: device buffer owned by the caller, 256-byte aligned, of at least
 * dot_render_views_host_workspace(n_cameras, width, height, T_final != NULL) bytes; no other work
 * may use it until this call returns.  opts->signal_mode must be NONE.
 */
int dot_render_views_host(const dot_tree *tree, const dot_camera *cameras, int32_t n_cameras,
                          int32_t width, int32_t height, const int32_t *view_order,
                          const dot_render_opts *opts, float *rgb, float *T_final,
                          void *workspace, int64_t workspace_bytes, void *stream);

/* Workspace bytes dot_render_views_host needs (host arithmetic only; -1 for invalid sizes). */
int64_t dot_render_views_host_workspace(int32_t n_cameras, int32_t width, int32_t height,
                                        int32_t with_T);

/*
 * dot_render_slots -- renders every request of a device slot table in one persistent launch
 * (Eq. 1-2 per pixel, as dot_render_forward): the requests may differ in resolution and in the
 * tree they look at.  Blocks take 16x8 tiles from a work counter until the table's tiles run out;
 * each pixel's value does not depend on the other requests in the table.
 * trees[n_trees] (1..DOT_MAX_SERVE_TREES, host array of handles): resident trees sharing one
 * storage type and SH degree.  table: device dot_slot_table_header + max_slots dot_slot (read by
 * the kernel, so it may be rewritten between launches).  work_counter: device uint64, zeroed by
 * this call on the stream.  opts->signal_mode must be NONE.
 */
int dot_render_slots(dot_tree *const *trees, int32_t n_trees, const void *table,
                     int32_t max_slots, const dot_render_opts *opts,
                     unsigned long long *work_counter, void *stream);

/*
 * dot_render_backward -- gradient of L = sum_r grad_rgb[r] . rgb[r] with respect to the leaf
 * parameters (the differentiable render of Sec. 3 Preliminaries, Eq. 1-2), by recomputing each
 * ray's march (no per-sample state from the forward):
 *   dL/dsh[v][ch][k] += g_ch w_i act'(z_ch) Y_k,
 *   dL/dsigma[v]     += [sigma_v > 0] delta_i sum_ch g_ch (T_{i+1} c_ch - (C_ch - C_{<=i,ch})).
 * grad_rgb, rgb: device [R][3] (rgb = this tree's forward output for the same rays and opts);
 * grad_sigma: device [L] float (+=); grad_sh: device [L][3][K] float (+=); signal as forward;
 * touched: device [L] uint8 or NULL -- set to 1 for every leaf the backward gives a gradient
 * (an occupied segment of some ray), for dot_rmsprop_step_sparse.
 */
int dot_render_backward(const dot_tree *tree, const dot_rays *rays, const dot_render_opts *opts,
                        const float *grad_rgb, const float *rgb, float *grad_sigma,
                        float *grad_sh, float *signal, uint8_t *touched, void *stream);

/*
 * dot_render_forward_backward_mse -- one training pass over a batch of rays in one launch: the
 * forward render (Eq. 1-2, as dot_render_forward, with its fused signal), the MSE gradient
 * grad_rgb = 2 (rgb - target) / (3R) (as dot_mse_grad; loss_sum += the MSE), and the backward
 * (as dot_render_backward with that gradient).  Each ray records its occupied segments (weight,
 * transmittance, length, colour) while marching forward and scatters the gradients from that
 * record, so the backward takes no second traversal; a ray with more than 48 occupied segments
 * marches again in the backward mode.  Results equal the three separate calls up to the order
 * of the FP32 atomic sums.
 * target, rgb, grad_rgb: device [R][3] float (rgb and grad_rgb written, all distinct);
 * loss_sum: device double or NULL; grad_sigma [L], grad_sh [L][3][K]: accumulated (+=); signal
 * and touched as in dot_render_forward / dot_render_backward.  Not for compressed trees.
 */
int dot_render_forward_backward_mse(const dot_tree *tree, const dot_rays *rays,
                                    const dot_render_opts *opts, const float *target, float *rgb,
                                    float *grad_rgb, double *loss_sum, float *grad_sigma,
                                    float *grad_sh, float *signal, uint8_t *touched, void *stream);

/*
 * dot_accumulate_signal -- the per-leaf training signal of Sec. 3.1 (Algorithm 1, optimization
 * step): SUM_ALPHA or MAX_WEIGHT by marching the rays (densities only), or SIGMA (no rays).
 * signal: device [L] float, accumulated (SIGMA: written).
 */
int dot_accumulate_signal(const dot_tree *tree, const dot_rays *rays, const dot_render_opts *opts,
                          int32_t mode, float *signal, void *stream);

/*
 * dot_select_masks -- prune and sample marks from the signal (Sec. 3.2; Algorithm 1 pruning
 * and sampling).  Rank selections break ties by leaf id.  Signals compare as floats: -0 equals
 * +0, and a NaN is never marked by a threshold and comes after every number in both rank orders
 * (taken only when k exceeds the count of numbers).  signal: device [L] float;
 * prune_mark, sample_mark: device [L] uint8 (written 0/1).
 */
int dot_select_masks(const dot_tree *tree, const float *signal, const dot_select_opts *opts,
                     uint8_t *prune_mark, uint8_t *sample_mark, void *stream);

/*
 * dot_select_masks_noalloc -- the same prune and sample marks as dot_select_masks, computed
 * without allocating any device memory.  The paper has no counterpart to this call.
 *
 * It exists for applications that cannot have the library allocate while it works: a process
 * that reserves its whole device-memory budget at start-up (an engine or renderer that owns the
 * memory pool, or a serving loop that admits work by free memory and must not see hidden
 * allocations shift that figure), or a caller whose allocation path may block or fail while the
 * device is under memory pressure.  dot_select_masks takes its working memory from
 * cudaMallocAsync; this call never calls cudaMalloc, cudaMallocAsync, cudaFree or any other
 * allocating routine.
 *
 * Its working memory is one fixed array of about 66 KB in the library's device memory (the
 * radix-select histogram and state, and one count per tile of 4096 leaves), which every GPU
 * that loads the library keeps until the process exits.  Limits and behaviour:
 *  - trees of at most 2^26 (67,108,864) leaves; larger trees return DOT_ERR_INVALID_ARG;
 *  - a call made outside stream capture looks up the array's device address with the calling
 *    device current; a call made while its stream is being captured reuses the address the last
 *    call on that device found (DOT_ERR_CUDA if there was none), so make one call on each device
 *    before any stream capture;
 *  - every call on a device shares the array and leaves its last contents there (the call clears
 *    what must start at zero itself); calls whose work overlaps on the GPU, for example on two
 *    streams without ordering, race on it and can return wrong marks, so order such calls.
 * Arguments, modes, tie-breaking and results are those of dot_select_masks.
 */
int dot_select_masks_noalloc(const dot_tree *tree, const float *signal,
                             const dot_select_opts *opts, uint8_t *prune_mark,
                             uint8_t *sample_mark, void *stream);

/*
 * dot_refine_plan -- the sizes dot_refine_prune will produce for these marks (the merges of Eq. 3
 * and the subdivisions of Eq. 4; synchronises).
 */
int dot_refine_plan(const dot_tree *tree, const uint8_t *prune_mark, const uint8_t *sample_mark,
                    int32_t depth_cap, dot_refine_counts *out, void *stream);

/*
 * dot_refine_prune -- applies prune (Eq. 3) and sample (Eq. 4) in place on the tree.
 *  - A parent other than the root whose 8 children are leaves, all prune-marked and none
 *    sample-marked, becomes a leaf holding their mean (pairwise FP32 sum x 1/8, rounded to the
 *    storage type).
 *  - A sample-marked leaf above depth_cap becomes an internal node with 8 leaf children holding
 *    exact copies of its values.
 *  - New numbering: leaves = survivors (old order), merged parents (old node order), children of
 *    sampled leaves (old leaf order x slot); nodes = surviving nodes (old order), then the
 *    sampled leaves (old leaf order).
 * leaf_map: device [n_leaves after] int32 (written): the old leaf id, or -1 - old parent id for
 * merged leaves.  aux[n_aux]: extra per-leaf arrays remapped the same way (dst sized by the
 * plan).  Frees the old arrays; previous dot_tree_get_info pointers become invalid.
 */
int dot_refine_prune(dot_tree *tree, const uint8_t *prune_mark, const uint8_t *sample_mark,
                     int32_t depth_cap, int32_t *leaf_map, const dot_leaf_array *aux,
                     int32_t n_aux, void *stream);

/* RMSProp hyper-parameters (Sec. 3.3 names RMSProp; Sec. 4.1 gives lr 0.1 for sigma and 0.01
 * for the SH colour; the decay rho and eps are not given: the usual 0.9 and 1e-8 are defaults of
 * the Python binding). */
typedef struct {
    float lr_sigma, lr_sh;
    float rho;          /* decay of the mean square, in [0, 1) */
    float eps;          /* added to sqrt(mean square), >= 0 */
    int32_t zero_grad;  /* 1: write zeros to the gradients after reading them */
} dot_rmsprop_opts;

/*
 * dot_mse_grad -- the MSE loss of Algorithm 1 (optimization) over R rays x 3 channels of
 * stochastic samples (Sec. 4.1): grad_rgb = 2 (rgb - target) / (3R), the input of
 * dot_render_backward, and loss_sum += sum (rgb - target)^2 / (3R).
 * rgb, target, grad_rgb: device [R][3] float (grad_rgb may alias neither input); loss_sum: device
 * double (accumulated; may be NULL).  R = 0 is a no-op.
 */
int dot_mse_grad(const float *rgb, const float *target, int64_t n_rays, float *grad_rgb,
                 double *loss_sum, void *stream);

/*
 * dot_rmsprop_step -- one RMSProp update of every leaf's density and SH coefficients in place
 * (Sec. 3.3), FP32 arithmetic, parameters rounded to the storage type:
 *   ms <- rho ms + (1 - rho) g^2,   p <- p - lr g / (sqrt(ms) + eps)
 * with lr = lr_sigma for sigma and lr_sh for the SH coefficients; with zero_grad the gradients are
 * zeroed in the same pass (ready for the next dot_render_backward).
 * grad_sigma, ms_sigma: device [L] float; grad_sh, ms_sh: device [L][3][K] float.  The tree's
 * parameters change; its structure does not.
 */
int dot_rmsprop_step(dot_tree *tree, float *grad_sigma, float *grad_sh, float *ms_sigma,
                     float *ms_sh, const dot_rmsprop_opts *opts, void *stream);

/*
 * dot_rmsprop_step_sparse -- dot_rmsprop_step (RMSProp, Sec. 3.3) restricted to the leaves whose
 * `touched` flag is set (dot_render_backward sets it for every leaf it gives a gradient), with
 * the same results up to FP32 rounding.  A leaf nobody touched has zero gradients, so the dense update would only
 * multiply its mean squares by rho; that decay is deferred and applied as rho^k for the k steps
 * it sat out, the next time the leaf is touched or by dot_rmsprop_flush.
 * touched: device [L] uint8, read and cleared; last_step: device [L] int32, the step up to which
 * each leaf's mean squares are current (zeros before the first step); step: this step's number
 * (1, 2, ...; increasing by one per call); work: device int32 [L + 1] scratch owned by the
 * caller (the list of touched leaves and its count).  Gradients of touched leaves are zeroed
 * when zero_grad is set; the others are zero already.
 */
int dot_rmsprop_step_sparse(dot_tree *tree, float *grad_sigma, float *grad_sh, float *ms_sigma,
                            float *ms_sh, uint8_t *touched, int32_t *last_step, int32_t step,
                            int32_t *work, const dot_rmsprop_opts *opts, void *stream);

/*
 * dot_rmsprop_flush -- applies every deferred RMSProp decay (Sec. 3.3) up to step `step`:
 * ms <- rho^(step - last_step) ms and last_step <- step for every leaf (before reading the mean
 * squares, refining the tree or switching to dot_rmsprop_step).
 */
int dot_rmsprop_flush(dot_tree *tree, float *ms_sigma, float *ms_sh, int32_t *last_step,
                      int32_t step, const dot_rmsprop_opts *opts, void *stream);

/*
 * dot_compress_sh -- the compressed model of Sec. 4.1: every leaf's SH coefficient row is replaced
 * by one of 2^bits palette rows, found by median cut (Heckbert 1982) over the leaves' coefficient
 * vectors: each of the bits rounds splits every box of two or more vectors at the median of its
 * longest axis (largest max - min; ties to the lowest axis; members ordered by (value, leaf id),
 * floor(m/2) to the lower child); a palette row is the mean of its box rounded to the storage
 * type.  Each leaf then keeps one 32-bit record, its 16-bit density in the low half and its
 * palette row in the high half, so rendering reads 4 bytes per segment plus a palette row.
 * bits: 1..16; 16-bit storage only (DOT_ERR_UNSUPPORTED for FP32).  The quantiser runs on the
 * GPU (each round: per-box ranges by atomics over a permutation that keeps every box's members
 * contiguous, the median member by a per-box radix select over (value, leaf id) keys, then a
 * stable split of every box's segment) and the call synchronises the stream.  Afterwards forward
 * renders, signals, statistics and slot tables read the records; dot_render_backward,
 * dot_rmsprop_step, dot_refine_plan and dot_refine_prune return DOT_ERR_UNSUPPORTED;
 * dot_tree_export writes the expanded coefficients.
 */
int dot_compress_sh(dot_tree *tree, int32_t bits, void *stream);

/*
 * dot_tree_canonicalize -- renumbers the tree's nodes and leaves into the build's canonical order
 * (breadth first, Morton order within a level: ascending key order).  Refines (Eq. 3-4) append
 * new cells at the end of the arrays; renumbering restores memory locality between neighbouring
 * cells.  The cells and their values do not change, so renders are bit-identical.
 * leaf_perm: device [L] int32 (written): the old id of each new leaf (compose with a refine's
 * leaf_map as leaf_map[leaf_perm[u]]).  aux[n_aux]: per-leaf FP32 arrays [L][width] permuted the
 * same way from src into dst (distinct buffers).  Works on compressed trees too.  Synchronises
 * once per level; frees the old arrays (previous dot_tree_get_info pointers become invalid).
 */
int dot_tree_canonicalize(dot_tree *tree, int32_t *leaf_perm, const dot_leaf_array *aux,
                          int32_t n_aux, void *stream);

/*
 * dot_render_stats -- counts of the march for these rays (not part of any hot path): out[0] =
 * rays entering the root, out[1] = segments (cell steps), out[2] = occupied segments
 * (sigma > 0, delta > 0), out[3] = child-table loads.  Synchronises the stream.
 */
int dot_render_stats(const dot_tree *tree, const dot_rays *rays, const dot_render_opts *opts,
                     int64_t out[4], void *stream);

/*
 * dot_probe_l2_read -- a measurement helper with no counterpart in the paper: streams `bytes`
 * of the device buffer `buf` `passes` times with 16-byte loads cached in L2 only, one grid of
 * whole waves, asynchronous on `stream`.  Timed by the caller (events around the call) on a
 * buffer that fits in L2, it gives the L2 read bandwidth that the two-level roofline of the
 * march kernels divides their per-segment bytes by.  buf: device, 16-byte aligned, bytes a
 * multiple of 16 and > 0; passes >= 1; sink: device uint64 or NULL (written only if the folded
 * data hits an impossible key, i.e. never in practice).  DOT_ERR_INVALID_ARG otherwise.
 */
int dot_probe_l2_read(const void *buf, int64_t bytes, int32_t passes, unsigned long long *sink,
                      void *stream);

#ifdef __cplusplus
}
#endif
#endif /* DOT_H */
