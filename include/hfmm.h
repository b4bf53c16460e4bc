/*
 * hfmm.h -- C ABI of the GB300 heterogeneous FMM (H-FMM) for the 2-D
 * Helmholtz equation in a half-space with an impedance boundary, a two-layer
 * or a three-layer medium (Cho, Huang, Chen, Cai: "A Heterogeneous FMM for
 * 2-D Layered Media Helmholtz Equation I: Two & Three Layers Cases").
 *
 * The library computes the matrix-vector product of Sec. 2.4,
 *
 *     y_i = sum_j A_ij q_j,   A_ij = u_{x_j}(x_i)           (Sec. 2.4)
 *         = sum_{j != i} (i/4) H0^(1)(k1 |x_i - x_j|) q_j   (Eq. (eq:freeGreen))
 *         + sum_j        G^s(x_i - x_j, y_i + y_j)     q_j   (Eq. (eq:multisommer), (eq:multitop))
 *
 *     G^s(X, Y) = 1/(4 pi) int_R e^{-s1 Y} / s1  e^{i lambda X} sigma(lambda) dlambda,
 *     s_j = -i sqrt(k_j^2 - lambda^2)  (principal root, Re s_j >= 0),
 *
 * for N points that are both sources and targets, all in the top layer
 * y > 0.  The free-space self term (i = j) is omitted; the reaction self term
 * G^s(0, 2 y_i) is included.  sigma is
 *     impedance:    (s1 + i alpha) / (s1 - i alpha)                       (Sec. 2.2)
 *     two layers:   (s1 - s2) / (s1 + s2)                                 (Sec. 2.3, d -> inf)
 *     three layers: (r12 + r23 e^{-2 s2 d}) / (1 + r12 r23 e^{-2 s2 d}),
 *                   r_ij = (s_i - s_j) / (s_i + s_j)                      (Sec. 2.3, 4x4 system)
 * The impedance condition du/dn - i alpha u = 0 (Eq. (impedBC)) is taken with
 * the normal pointing out of the upper half-plane (n = -y_hat); time factor
 * e^{-i omega t}.
 *
 * Algorithm (Algorithm 1, Sec. 3-5): uniform quadtree over the smallest
 * bounding square; free-space P2M (Eq. (multi_coeff)), M2M, L2L, L2P and
 * Graf M2L; heterogeneous M2L with the matrix A_{p,m} of Eq. (eq:m2loperator)
 * (sigma generalised as in Sec. 5) built at plan time by FP64 quadrature on
 * the GPU; direct free-space H0 sums over neighbouring leaves.
 *
 * Memory and ownership.  All array arguments are plain pointers that may
 * point to host memory or to device memory of the current CUDA device (the
 * library asks the driver which).  The caller owns them; the library never
 * frees or keeps them past the call.  The plan owns all of its device memory
 * (tree, tables, expansion buffers) and releases it in hfmm_plan_destroy.
 * Complex arrays are interleaved (re, im).  Multi-RHS arrays are column-major
 * [nrhs][n]: right-hand side r occupies elements r*n .. r*n+n-1, in the
 * caller's point order.
 *
 * Streams.  `stream` is a cudaStream_t passed as void* (NULL = legacy
 * default stream).  Host inputs/outputs make the call synchronous on that
 * stream; with device pointers the call only enqueues work.
 *
 * Errors.  Every function returns an hfmm_status; no C++ exception crosses
 * the ABI.  hfmm_last_error() returns a thread-local message describing the
 * most recent failure on the calling thread.  A failed call leaves the plan
 * usable.
 */
#ifndef HFMM_H
#define HFMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hfmm_plan_s* hfmm_plan_t;

typedef enum {
    HFMM_OK = 0,
    HFMM_ERR_INVALID_ARG = 1,   /* bad pointer, size, point below y = 0, non-finite input */
    HFMM_ERR_UNSUPPORTED = 2,   /* valid request the library does not handle (e.g. alpha < 0) */
    HFMM_ERR_OOM = 3,           /* device or host allocation failed */
    HFMM_ERR_CUDA = 4,          /* a CUDA runtime call failed */
    HFMM_ERR_NUMERICS = 5,      /* a table quadrature did not reach its tolerance */
    HFMM_ERR_TIMEOUT = 6        /* a bounded device wait gave up */
} hfmm_status;

typedef enum {
    HFMM_IMPEDANCE = 0,         /* y > 0 over the impedance line y = 0 */
    HFMM_TWO_LAYER = 1,         /* k[0] for y > 0, k[1] for y < 0 */
    HFMM_THREE_LAYER = 2        /* k[0] for y > 0, k[1] for -d < y < 0, k[2] for y < -d */
} hfmm_medium_kind;

typedef enum {
    HFMM_FP64 = 0,              /* complex128 in/out, FP64 arithmetic everywhere */
    HFMM_MIXED = 1              /* complex64 in/out, FP32 P2P/P2M/L2P, tensor-core M2L */
} hfmm_precision;

typedef struct {
    int32_t kind;               /* hfmm_medium_kind */
    int32_t reserved;
    double k[3];                /* real wavenumbers, k[0] > 0 */
    double d;                   /* three layers: middle-layer thickness > 0 */
    double alpha;               /* impedance: real alpha >= 0 */
} hfmm_medium;

typedef struct {
    double tol;                 /* target relative accuracy; selects the expansion order */
    int32_t p;                  /* > 0: fixed low-frequency order instead of the tol rule */
    int32_t leaf_size;          /* mean points per leaf that sets the leaf level */
    int32_t levels;             /* > 0: force the leaf level L */
    int32_t precision;          /* hfmm_precision */
    int32_t max_rhs;            /* largest nrhs of later apply calls (buffers sized for it) */
    int32_t flags;              /* HFMM_FLAG_* bits, 0 = none */
    int64_t spin_limit;         /* polls of each bounded device wait (each suspends <= ~1 us);
                                   0 = default (2e6, about 2 s).  A wait that gives up sets
                                   device_error; host-buffer applies then return HFMM_ERR_TIMEOUT */
    double quad_scale;          /* scale of the panel counts of every table quadrature rule
                                   (0 = 1).  Each reaction table entry and each directly summed
                                   block is also computed on the rule with twice the panels;
                                   hfmm_plan_create returns HFMM_ERR_NUMERICS when the two differ
                                   by more than 1e-12 (relative, weighted by what the normalised
                                   expansions can reach; see hfmm_plan_info.table_check).
                                   Values below 1 coarsen the rules (a test of that check). */
    int32_t small_rhs;          /* HFMM_MIXED: applies with nrhs <= small_rhs run on warp-level
                                   SIMT kernels (one warp per box and coefficient chunk, a few
                                   right-hand sides per pass) instead of the tensor-core tiles,
                                   whose 128-row tiles hold 64 right-hand sides; 0 = default
                                   (HFMM_SMALL_RHS_DEFAULT), -1 = never */
} hfmm_options;

#define HFMM_SMALL_RHS_DEFAULT 4

/* Option flags. */
#define HFMM_FLAG_PROFILE 1     /* record CUDA events around every stage of each apply */
#define HFMM_FLAG_SIMT_M2L 2    /* HFMM_MIXED: keep the downward pass on FP32 SIMT cores
                                   instead of the tcgen05 tensor-core pass */
#define HFMM_FLAG_AUTOTUNE 4    /* build the plan at the leaf levels L-1, L, L+1 around the
                                   leaf_size choice, time max_rhs-wide applies on the device
                                   and keep the fastest (hfmm_plan_info.tune_*); mixed plans
                                   with tensor-core state and small_rhs = 0 then time both
                                   engines at nrhs = 1, 2, 4, ... and set small_rhs to the
                                   largest nrhs where the warp-level kernels are faster */
#define HFMM_FLAG_PERSISTENT 8  /* batches: mixed-precision applies with nrhs <= small_rhs run as
                                   one persistent kernel over a device work queue (see
                                   hfmm_batch_device_error) instead of one graph branch per
                                   instance */
#define HFMM_FLAG_ADAPTIVE 32   /* HFMM_FP64: adaptive tree (Sec. 3.1): boxes with more than
                                   leaf_size points are split (down to level 16), empty children
                                   pruned, so leaves sit on many levels; U/V/W/X lists (W: a small
                                   box's multipole evaluated at a leaf's points, X: a leaf's points
                                   into a small box's local expansion), and the reaction pairs of
                                   the uniform tree's recursion, summed directly below a leaf.  The
                                   tree and lists are built on the host at plan time.  FP64, or
                                   HFMM_MIXED as FP32 passes over plan-time FP32 bases of the points
                                   (no tensor cores, no persistent batches).  Not with
                                   HFMM_FLAG_AUTOTUNE (HFMM_ERR_UNSUPPORTED); no position gradients
                                   (hfmm_apply_grad returns UNSUPPORTED) */
#define HFMM_FLAG_DENSE_M2L 16  /* HFMM_FP64: keep the dense (2p+1)^2 translations on every level.
                                   Without it the plan tries the diagonal form of the free and
                                   reaction translations (their matrices depend on m - p only,
                                   Sec. 3.3, so a circulant embedding of length Q >= 4p + 1 makes
                                   each translation an O(Q) pointwise product between one FFT per
                                   source box and one inverse FFT per target box) on each level
                                   and keeps it where it reproduces the dense product on random
                                   expansions to 1e-12 (weighted as in table_check); that holds
                                   only on levels whose boxes are large against the wavelength
                                   (hfmm_plan_info.diag_levels) */

/* Stages reported by hfmm_plan_get_stage_times (milliseconds of the last apply). */
#define HFMM_STAGE_GATHER   0   /* caller order -> leaf order */
#define HFMM_STAGE_P2M      1
#define HFMM_STAGE_M2M      2
#define HFMM_STAGE_DOWN     3   /* L2L + free-space M2L + reaction M2L, all levels */
#define HFMM_STAGE_L2P      4
#define HFMM_STAGE_P2P      5
#define HFMM_STAGE_DIRECT   6   /* directly summed reaction */
#define HFMM_STAGE_SCATTER  7
#define HFMM_NUM_STAGES     8

/* Plan summary for callers and tests. */
#define HFMM_MAX_LEVELS 24
typedef struct {
    int64_t n;
    int32_t levels;             /* leaf level L */
    int32_t lmin;               /* coarsest level with translation work */
    int32_t p[HFMM_MAX_LEVELS]; /* expansion order per level (2p+1 coefficients) */
    int64_t nonempty_leaves;
    int64_t v_pairs;            /* free-space M2L pairs, all levels */
    int64_t r_pairs;            /* reaction M2L pairs, all levels */
    int64_t direct_leaf_pairs;  /* leaf pairs whose reaction is summed directly */
    int64_t u_pairs;            /* neighbouring non-empty leaf pairs (P2P) */
    double x0, y0, size;        /* root square [x0, x0+size] x [y0, y0+size] */
    double table_bytes;         /* device bytes of translation tables */
    double buffer_bytes;        /* device bytes of expansion buffers */
    double plan_ms;             /* wall time of hfmm_plan_create */
    int32_t precision;
    int32_t max_rhs;
    int64_t launches_last_apply;  /* kernels launched by the last apply call */
    double flops_last_apply[HFMM_NUM_STAGES];  /* algorithmic real flops per stage, last apply */
    double bytes_last_apply[HFMM_NUM_STAGES];  /* algorithmic DRAM bytes per stage, last apply */
    int32_t device_error;       /* nonzero if a bounded device wait gave up (results invalid) */
    int32_t tensor_levels;      /* levels whose downward pass runs on tcgen05 tensor cores */
    int32_t tune_levels[3];     /* HFMM_FLAG_AUTOTUNE: leaf levels tried (0 = not tried) */
    double tune_ms[3];          /* and the apply time measured for each */
    int64_t near_tc_blocks;     /* HFMM_MIXED: four-leaf blocks of the tensor-core near field */
    int64_t near_simt_leaves;   /*             leaves of wider blocks, on the SIMT kernel */
    int32_t leaf_l2p_fused;     /* HFMM_MIXED: 1 if the leaves' L2P runs in the tensor-core downward
                                   epilogue, 0 if on the SIMT kernel */
    int32_t leaf_tc_width;      /* HFMM_MIXED: column-block width (MMA N) of the leaf-level
                                   tensor-core pass, 0 without one */
    double table_check;         /* largest difference between a quadrature table entry (reaction
                                   A_n, weighted by s(|m|) s(|p|) of the translations it feeds,
                                   or a directly summed G^s block) and its node-doubled value,
                                   relative to the entry's largest weighted value (<= 1e-12) */
    int32_t small_rhs;          /* HFMM_MIXED: applies with nrhs <= small_rhs run on the warp-level
                                   kernels (0 for FP64 plans) */
    int32_t diag_levels;        /* HFMM_FP64: bit l set if level l translates in diagonal form
                                   (see HFMM_FLAG_DENSE_M2L) */
    double diag_check;          /* largest plan-time difference of a level kept in diagonal form */
    int32_t adaptive;           /* 1 for HFMM_FLAG_ADAPTIVE plans (levels = deepest level,
                                   nonempty_leaves = leaves, direct_leaf_pairs = leaf pairs of
                                   the directly summed reaction) */
    int32_t tc_run_levels;      /* HFMM_MIXED, tensor-core pass: number of the finest levels with
                                   level-wide f16 scales, whose free and reaction steps (and the
                                   M2M from them) accumulate in tensor memory with one drain */
    int64_t w_pairs;            /* adaptive: (leaf, box) M2P pairs */
    int64_t x_pairs;            /* adaptive: (box, leaf) P2L pairs */
} hfmm_plan_info;

/* Bits of `parts` in hfmm_apply_parts (sum of the selected terms). */
#define HFMM_PART_NEAR_FREE   1  /* H0 sums over neighbouring leaves (Algorithm 1, step 5) */
#define HFMM_PART_FAR_FREE    2  /* free-space M2L through the tree (steps 2-4) */
#define HFMM_PART_FAR_REACT   4  /* reaction M2L with A_{p,m} (steps 3-4) */
#define HFMM_PART_NEAR_REACT  8  /* directly summed reaction (step 5) */
#define HFMM_PART_ALL        15

/* Defaults: tol 1e-6, p 0, leaf_size 32, levels 0, FP64, max_rhs 1. */
void hfmm_options_default(hfmm_options* opts);

/*
 * Build a plan for n points xy[n][2] (x, y interleaved, FP64; host or device
 * pointer).  Builds the quadtree on the device (Morton sort, leaf binning,
 * interaction lists), chooses the expansion order per level and computes the
 * translation tables (Sec. 3.3, Eq. (eq:m2loperator); "precompute tables" of
 * Algorithm 1, step 1).  Synchronises `stream` before returning.
 * Errors: INVALID_ARG for n < 1, a null pointer, non-finite coordinates or
 * y <= 0; UNSUPPORTED for alpha < 0, k <= 0 or d <= 0 (three layers);
 * OOM / CUDA / NUMERICS as named.  *out is NULL on failure.
 */
hfmm_status hfmm_plan_create(hfmm_plan_t* out, int64_t n, const double* xy,
                             const hfmm_medium* medium, const hfmm_options* opts,
                             void* stream);

/*
 * y = A q for nrhs right-hand sides (1 <= nrhs <= max_rhs).  q, y: [nrhs][n]
 * complex, complex128 for HFMM_FP64 plans, complex64 for HFMM_MIXED plans,
 * in the caller's point order.  q and y must not overlap.  Device buffers:
 * stream-ordered, no host synchronisation.  Page-locked (registered) host
 * buffers are read and written in place by the permutation kernels; other
 * host buffers are staged through plan-owned device buffers.  With any host
 * buffer the call synchronises `stream` before returning.
 */
hfmm_status hfmm_apply(hfmm_plan_t plan, int32_t nrhs, const void* q, void* y, void* stream);

/* As hfmm_apply but only the terms selected by `parts` (HFMM_PART_*). */
hfmm_status hfmm_apply_parts(hfmm_plan_t plan, int32_t nrhs, const void* q, void* y,
                             int32_t parts, void* stream);

/*
 * w = A^H v: the transposed tree pass (L2P^T, L2L^T, M2L^T with transposed
 * tables, M2M^T, P2M^T, P2P^T) applied to conj(v), conjugated.  Same layout
 * and dtype rules as hfmm_apply.
 */
hfmm_status hfmm_apply_adjoint(hfmm_plan_t plan, int32_t nrhs, const void* v, void* w, void* stream);

/*
 * Position gradient of a real loss L(y), y = A(x) q, through the matrix of
 * Sec. 2.4 (A_ij = u_{x_j}(x_i)).  Given g = dL/dRe(y) + i dL/dIm(y)
 * ([nrhs][n] complex, caller order) writes gxy[2j], gxy[2j+1] = dL/dx_j, dL/dy_j:
 *     dL/dx_j = Re sum_r [ conj(g_rj) grad u_r(x_j) + q_rj grad w_r(x_j) ],
 *     u_r = sum_k G(., x_k) q_rk,   w_r = sum_k G(., x_k) conj(g_rk),
 * which uses the reciprocity G(a, b) = G(b, a) of the domain Green's function.
 * Field gradients come from the derivative of the local expansion
 * ((d/dx +- i d/dy) J_p e^{ip theta} = -+k J_{p+-1} e^{i(p+-1) theta}), of the
 * free-space kernel ((i/4)(-k H1(kr)) (x - x_j)/r) and of the Sommerfeld
 * integrand (factors i lambda and -s1) for directly summed reaction pairs.
 * Strength gradients are hfmm_apply_adjoint(g).  q, g: the plan's complex type
 * (complex128, or complex64 for HFMM_MIXED); gxy: [n][2] doubles; host or
 * device pointers.  A mixed plan widens q and g to complex128 and runs the FP64
 * tree pass with its FP64 translation tables; its first call allocates the FP64
 * expansions (2 x boxes x max_rhs x (2p+1) complex128 per level) and three
 * n x max_rhs complex128 buffers, held until hfmm_plan_destroy.
 */
hfmm_status hfmm_apply_grad(hfmm_plan_t plan, int32_t nrhs, const void* q, const void* g, double* gxy,
                            void* stream);

/*
 * Batches of independent problems of uneven sizes (same medium and options),
 * e.g. many scatterers or many inverse-problem instances.  One plan per
 * instance; hfmm_batch_apply applies all of them: the first call with a given
 * set of buffers runs them once eagerly on `stream` (lazily initialised
 * state is set up outside capture; `stream` is synchronised), then records
 * all instances' applies into one CUDA graph on a private stream of the
 * batch (one branch per instance, or one persistent launch with
 * HFMM_FLAG_PERSISTENT) and launches it on `stream`; later calls
 * with the same buffers only launch the graph.  q[i], y[i]: device buffers
 * [nrhs][n_i] of instance i (dtype as for hfmm_apply); adjoint != 0 applies
 * A_i^H instead.  Changing any buffer pointer, nrhs or adjoint re-records the
 * graph.  Errors: HFMM_ERR_INVALID_ARG for host buffers or nrhs outside
 * 1..max_rhs, HFMM_ERR_CUDA if capture or instantiation fails.  The batch
 * owns its plans; calls on one batch must not overlap.
 */
typedef struct hfmm_batch_s* hfmm_batch_t;
hfmm_status hfmm_batch_create(hfmm_batch_t* out, int32_t ninst, const int64_t* n, const double* const* xy,
                              const hfmm_medium* medium, const hfmm_options* opts, void* stream);
hfmm_status hfmm_batch_apply(hfmm_batch_t batch, int32_t nrhs, const void* const* q, void* const* y,
                             int32_t adjoint, void* stream);
/*
 * Batches created with HFMM_FLAG_PERSISTENT whose mixed-precision applies have
 * nrhs <= the plans' small_rhs run as one persistent kernel: a device queue
 * of work items over every stage and level of every instance; an item waits
 * for the items it depends on with a bounded wait (options.spin_limit polls).  A wait that gave up sets a flag of the
 * batch and the results of that apply are invalid.  hfmm_batch_device_error
 * synchronises the device and returns that flag of the last apply in
 * *device_error (0 = none; always 0 for batches on the per-instance graph).
 */
hfmm_status hfmm_batch_device_error(hfmm_batch_t batch, int32_t* device_error);
/*
 * Position gradients of every instance of a batch (hfmm_apply_grad per
 * instance, in order, on `stream`): gxy[i] = dL/dx, dL/dy of instance i for a
 * real loss of y_i = A_i q_i, given g[i] = dL/dRe(y_i) + i dL/dIm(y_i).
 * Strength gradients are the adjoint (hfmm_batch_apply with adjoint != 0).
 * Same buffer rules and errors as hfmm_apply_grad (Sec. 2.4: A_ij =
 * u_{x_j}(x_i); the derivative acts on both arguments of G).
 */
hfmm_status hfmm_batch_apply_grad(hfmm_batch_t batch, int32_t nrhs, const void* const* q, const void* const* g,
                                  double* const* gxy, void* stream);
/* Plan of instance i (owned by the batch; for introspection and single applies). */
hfmm_status hfmm_batch_get_plan(hfmm_batch_t batch, int32_t i, hfmm_plan_t* plan);
hfmm_status hfmm_batch_destroy(hfmm_batch_t batch);

/*
 * HFMM_FLAG_PROFILE plans, mixed path: event time (ms) of the leaf-level
 * tensor-core downward launch of the last apply (L2L + free and reaction
 * M2L of the leaves, plus their L2P when info.leaf_l2p_fused) and its
 * algorithmic real flops (8 nrhs per complex multiply-add, the per-level
 * counts of flops_last_apply); both 0 when the last apply had no such launch.
 */
hfmm_status hfmm_plan_get_leaf_down(hfmm_plan_t plan, double* ms, double* flops);

/* Fill *info (host pointer). */
hfmm_status hfmm_plan_get_info(hfmm_plan_t plan, hfmm_plan_info* info);

/*
 * Copy the plan's tree to host arrays: perm[n] (caller index of the i-th
 * point in leaf order, int64) and leaf_ix[n], leaf_iy[n] (leaf column / row
 * of each caller-order point, int32).  Any pointer may be NULL.
 */
hfmm_status hfmm_plan_get_tree(hfmm_plan_t plan, int64_t* perm, int32_t* leaf_ix, int32_t* leaf_iy);

/*
 * Copy the interaction pairs of level `level` to host arrays of the given
 * capacity: kind 0 = free-space M2L (V list), 1 = reaction M2L, 2 = direct
 * reaction leaf pairs, 3 = neighbouring leaf pairs (U list).  Each pair is
 * (target ix, target iy, source ix, source iy) in out[4*i .. 4*i+3].
 * *count receives the number of pairs (also when cap is too small, in
 * which case INVALID_ARG is returned).
 */
hfmm_status hfmm_plan_get_pairs(hfmm_plan_t plan, int32_t kind, int32_t level,
                                int32_t* out, int64_t cap, int64_t* count);

/*
 * Adaptive plans (HFMM_FLAG_ADAPTIVE): the boxes of the tree, by level and in
 * Morton order within a level, as out[6*i .. 6*i+5] = (level, ix, iy, first
 * sorted point, end, leaf flag) (the sorted order is hfmm_plan_get_tree's
 * perm).  *count receives the number of boxes; out may be NULL to ask for it;
 * INVALID_ARG if cap is smaller, UNSUPPORTED for uniform plans.
 */
hfmm_status hfmm_plan_get_boxes(hfmm_plan_t plan, int32_t* out, int64_t cap, int64_t* count);

/*
 * Adaptive plans: the pairs of one list as (target box, source box) indices
 * into hfmm_plan_get_boxes in out[2*i], out[2*i+1]: kind 0 U (leaf, leaf),
 * 1 V, 2 W (leaf, box: M2P), 3 X (box, leaf: P2L), 4 reaction M2L (same-level
 * boxes), 5 directly summed reaction (box pairs with a leaf on one side; the
 * sum runs over the leaf pairs below them).  Count / capacity as above.
 */
hfmm_status hfmm_plan_get_lists(hfmm_plan_t plan, int32_t kind, int32_t* out, int64_t cap, int64_t* count);

/*
 * Stage times of the last apply of a plan created with HFMM_FLAG_PROFILE:
 * ms[HFMM_NUM_STAGES] (host array), measured with CUDA events recorded on
 * the apply's stream around each stage.  Synchronises that stream.
 * INVALID_ARG if the plan was created without the flag.
 */
hfmm_status hfmm_plan_get_stage_times(hfmm_plan_t plan, double* ms);

/*
 * Leaf ordering that allocates nothing.  The paper has no counterpart: this
 * is a service for callers that cannot let a library allocate device memory,
 * e.g. an application that has reserved the GPU's memory for its own pool
 * allocator, or one whose other streams must not be stalled by the implicit
 * device synchronisation of cudaMalloc / cudaFree.
 *
 * Computes what hfmm_plan_create's tree build computes for `levels` leaf
 * levels: the smallest bounding square of xy, the Morton index of every
 * point's leaf, a stable sort by leaf, and the leaf ranges.
 *   xy          device pointer, [n][2] doubles (x, y), all y > 0;
 *   perm        device pointer, [n] int64 out: caller index of the i-th point
 *               in leaf order (equal to hfmm_plan_get_tree's perm for a plan
 *               built with the same leaf level);
 *   leaf_begin  device pointer, [4^levels + 1] int32 out: the points of the
 *               leaf with Morton index b are perm[leaf_begin[b] .. leaf_begin[b+1]).
 * Limits: 1 <= n <= HFMM_NOALLOC_MAX_POINTS and 2 <= levels <=
 * HFMM_NOALLOC_MAX_LEVELS; anything larger returns INVALID_ARG with a message
 * naming the limit.  Non-finite coordinates or y <= 0 return INVALID_ARG.
 * Every call synchronises `stream` once, after the bounding-box pass, to read
 * that input check back to the host; the remaining work is queued on `stream`
 * without waiting.
 *
 * All temporaries live in one static device array of about 6 MB that every
 * GPU loading this library holds until the process exits.  The first call on
 * a device looks up that array's device address (with that device current);
 * make that first call before any stream capture.  Every call shares the
 * array and it keeps the last call's contents: calls whose work overlaps on
 * the GPU (other streams, other host threads) race and must be serialised by
 * the caller.
 */
#define HFMM_NOALLOC_MAX_POINTS (1 << 18)
#define HFMM_NOALLOC_MAX_LEVELS 9
hfmm_status hfmm_leaf_order_noalloc(int64_t n, const double* xy, int32_t levels, int64_t* perm,
                                    int32_t* leaf_begin, void* stream);

/*
 * Solve (sigma I + A) x = b for one right-hand side by restarted GMRES, with
 * A_ij = u_{x_j}(x_i) the plan's matrix (Sec. 2.4: the discretised layer or
 * volume potential of a second-kind integral equation).  Each iteration is
 * one apply of the plan plus Krylov updates on the device (dot products
 * accumulated in FP64); the Hessenberg least-squares problem is solved on the
 * host, so every iteration synchronises `stream`.
 *   sigma    host pointer to (re, im) of the shift;
 *   b, x     device buffers of n complex values (complex128 for HFMM_FP64,
 *            complex64 for HFMM_MIXED) in the caller's point order; x holds
 *            the initial guess on entry and the solution on return;
 *   tol      relative residual ||b - (sigma I + A) x|| / ||b|| to reach (the
 *            mixed path's apply carries a few 1e-6 relative error: ask >= 1e-5);
 *   restart  Krylov dimension between restarts (1..1000), maxit the total
 *            number of applies; *iters, *relres report them (the true
 *            residual of the returned x).
 * Returns HFMM_ERR_NUMERICS (x still holds the last iterate) when tol was not
 * reached, HFMM_ERR_INVALID_ARG for host buffers or bad parameters.  The
 * first call allocates (restart + 2) n complex values of Krylov vectors,
 * held by the plan.
 */
hfmm_status hfmm_solve(hfmm_plan_t plan, const double* sigma, const void* b, void* x, double tol, int32_t restart,
                       int32_t maxit, int32_t* iters, double* relres, void* stream);

/* Release the plan (NULL is accepted).  Synchronises the device. */
hfmm_status hfmm_plan_destroy(hfmm_plan_t plan);

/* Static description of a status code. */
const char* hfmm_status_string(hfmm_status s);

/* Thread-local message of the last failure on this thread ("" if none). */
const char* hfmm_last_error(void);

/*
 * Host reference of the library's own Bessel code (no GPU needed): for x > 0
 * writes J_n(x) to j[0..nmax] and H_n^(1)(x) to h[2*(0..nmax)] (re, im).
 * Used by tests to compare the library's Bessel evaluation with other
 * implementations.
 */
/*
 * One bounded device wait, as the tensor-core kernels wait on their
 * mbarriers: on a barrier whose phase completes only when `arrive` is nonzero
 * (the arrival precedes the wait).  HFMM_ERR_TIMEOUT when the wait gave up
 * after `spin` polls (each suspends at most ~1 us), HFMM_OK when it completed.
 * Exercises the timeout path without any fault; needs a GPU.
 */
hfmm_status hfmm_debug_wait_timeout(int64_t spin, int32_t arrive);

hfmm_status hfmm_debug_bessel(double x, int32_t nmax, double* j, double* h);

/*
 * Host copy of the FP32 free-space kernel used by the HFMM_MIXED near field:
 * g[2i], g[2i+1] = (i/4) H0^(1)(z[i]) (re, im) evaluated in single precision
 * from the library's piecewise polynomial tables of J0 and of the smooth part
 * Y0 - (2/pi) ln(z/2) J0, for 0 < z < 16 (NaN outside).  No GPU needed.
 */
hfmm_status hfmm_debug_green_f32(int32_t n, const double* z, float* g);

#ifdef __cplusplus
}
#endif

#endif /* HFMM_H */
