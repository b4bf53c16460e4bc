// Internal plan layout of the H-FMM library.
//
// Boxes.  The quadtree has uniform depth: level l holds 4^l boxes of side
// h_l = S / 2^l over the root square [x0, x0 + S] x [y0, y0 + S].  A box is
// addressed by its Morton index b (bits of ix in even, bits of iy in odd
// positions), so the children of b are 4b .. 4b + 3 and the leaves below b
// form the contiguous range [b 4^(L-l), (b+1) 4^(L-l)).  Points are sorted by
// leaf Morton index (ties by caller index), so every box owns a contiguous
// range of sorted points: [leaf_begin[b 4^(L-l)], leaf_begin[(b+1) 4^(L-l)]).
//
// Expansions.  Level l stores for each box, each right-hand side r and each
// order n = -p_l .. p_l one complex coefficient at
//     buf_l[(b * max_rhs + r) * (2 p_l + 1) + n + p_l].
#pragma once

#include <vector>

#include <cuda_fp16.h>

#include "common.cuh"

struct LevelInfo {
    int p = 0;
    int ncoef = 1;          // 2p + 1
    double h = 0.0;
    int64_t nbox = 1;       // 4^l
    // free-space M2L (V list), CSR over target boxes
    int32_t* v_begin = nullptr;   // [nbox + 1]
    int32_t* v_src = nullptr;     // [nv]
    int32_t* v_off = nullptr;     // [nv] offset index (dx + 3) * 7 + (dy + 3)
    int64_t nv = 0;
    // reaction M2L, CSR over target boxes
    int32_t* r_begin = nullptr;   // [nbox + 1]
    int32_t* r_src = nullptr;     // [nr]
    int32_t* r_tab = nullptr;     // [nr] index of the A_n table entry
    int64_t nr = 0;
    int32_t* r_tgt = nullptr;     // [n_rtgt] target boxes with a nonempty reaction list, increasing
    int64_t n_rtgt = 0;
    // tensor-core pass with level-wide scales: this level's multipole rows are
    // written with the exponent of the bound 2 max|q_r| tc_gain, and its free and
    // reaction tables share one factor (a tile's steps accumulate in TMEM)
    bool tc_runs = false;
    float tc_gain = 0.0f;
    // tables
    cd* t_free = nullptr;         // [49][4p + 1]  C_n(dx h, dy h), n = -2p .. 2p
    cd* t_m2m = nullptr;          // [4][2(p + p_child) + 1] J_n(parent - child_c)  (this level = parent)
    cd* t_l2l = nullptr;          // [4][2(p + p_child) + 1] J_n(child_c - parent)
    cd* t_react = nullptr;        // [nentries][4p + 1] A_n(X, Y), n = -2p .. 2p
    int n_react_entries = 0;
    int react_dx_max = 0;         // entries indexed (dx + dxmax) * 3 + ysum
    // expansion buffers (FP64 path)
    cd* mult = nullptr;
    cd* loc = nullptr;
    // mixed path: scaled expansions a~_n = a_n / s(|n|), b~_n = b_n s(|n|) with
    // s(n) = min(1, (k R_l / 2)^n / n!), R_l = h_l / sqrt(2) (|J_n(k rho)| <= s(n) for
    // rho <= R_l), and full scaled translation matrices in FP32
    std::vector<double> log_s;    // log s(n), n = 0 .. p
    cf* mult32 = nullptr;
    cf* loc32 = nullptr;
    cf* t_free32 = nullptr;       // [49][m][p] (input coefficient m outer)
    cf* t_react32 = nullptr;      // [nentries][m][p] (image reflection folded in)
    cf* t_m2m32 = nullptr;        // [4][m child][j parent]   (this level = parent)
    cf* t_l2l32 = nullptr;        // [4][n parent][m child]   (this level = parent)
    double* d_log_s = nullptr;    // [p + 1] log s(n) on the device
    // tensor-core passes (m2l_tc.cu): real GEMM width tc_np = tc_nb column blocks
    // of tc_nbw, K chunks of this level (tc_kc) and of the parent (tc_kc2),
    // pre-split f16 operator chunks with one power-of-two factor per matrix,
    // target-pair tiles and their source steps for the downward pass (L2L +
    // M2L) and for M2M into this level
    int tc_np = 0, tc_nb = 0, tc_nbw = 0, tc_kc = 0, tc_kc2 = 0;
    __half* tc_bfree = nullptr;
    __half* tc_breact = nullptr;
    __half* tc_bl2l = nullptr;
    __half* tc_bm2m = nullptr;
    float* tc_sfree = nullptr;    // 2^-e of each operator matrix (undoes its scaling)
    float* tc_sreact = nullptr;
    float* tc_sl2l = nullptr;
    float* tc_sm2m = nullptr;
    void* tc_tiles = nullptr;
    void* tc_steps = nullptr;
    int64_t tc_ntiles = 0;
    void* tc_mtiles = nullptr;
    void* tc_msteps = nullptr;
    int64_t tc_nmtiles = 0;
    int tc_maxsteps = 0, tc_mmaxsteps = 0;   // longest step list of a tile (downward, M2M)
    // MMA-ready expansions (f16 hi / lo) and the 2^-e factor of every
    // (box, RHS block, column block, row) that undoes their scaling
    __half* tc_amma = nullptr;    // multipoles of this level
    float* tc_asc = nullptr;
    __half* tc_pmma = nullptr;    // local expansions of the parent level
    float* tc_psc = nullptr;
    // diagonal form of the FP64 translations (diag.cu): circulant length 2^diag_logq
    // (0: dense), twiddles, spectra of the free / reaction table rows, spectra of
    // the level's multipoles [nbox][max_rhs][Q], and the plan-time check's result
    int diag_logq = 0;
    cd* diag_tw = nullptr;
    cd* diag_ofree = nullptr;
    cd* diag_oreact = nullptr;
    cd* diag_spec = nullptr;
    double diag_err = -1.0;
    int64_t nonempty = 0;         // non-empty boxes (set by the diagonal-form check)
};

// Diagonal form: kept on a level when its weighted difference to the dense
// product on random expansions is at most DIAG_RTOL; spectra capped per level.
constexpr double DIAG_RTOL = 1e-12;
constexpr size_t DIAG_MAX_BYTES = (size_t)8 << 30;

// Power-of-two scale of the stored near-field Green's function tiles (f16).
constexpr int NT_GSCALE_EXP = 10;

// Near field on tensor cores: one K chunk of a block (the four leaves of a
// parent box at level L - 1): up to 8 consecutive sorted points of one source
// leaf of the 4 x 4 neighbourhood.  The pre-split B tile of the chunk (rows =
// the padded targets of the adjacent leaves, in leaf order) starts at half
// offset boff of the plan's tile store: hi rows x 16, then lo.
struct NtChunk {
    int32_t src;     // first source point (sorted index)
    int32_t cnt;     // sources in the chunk (1 .. 8)
    int32_t mask;    // target leaves the tile covers (bit c = child c)
    int32_t rows;    // rows of the tile (sum of their padded widths)
    int64_t boff;
    int32_t par;     // parent box (level L - 1)
    int32_t aux;     // source leaf code (sx + 1) + 4 (sy + 1)
    int32_t nrun;    // runs of consecutive covered leaves (1 or 2)
    int32_t run[2];  // each: width | first column << 8 | first tile row << 16
    int32_t pad;
};

// Adaptive trees (adaptive.cu): deepest level, and the host / device tree.
constexpr int AD_MAX_LEVEL = 16;
struct AdaptiveTree;

struct hfmm_plan_s {
    int64_t n = 0;
    AdaptiveTree* ad = nullptr;     // HFMM_FLAG_ADAPTIVE plans
    int L = 0;
    int lmin = 0;
    int lstar = 0;                // first level whose bottom-row pairs are admissible
    int precision = HFMM_FP64;
    int max_rhs = 1;
    hfmm_medium med{};
    double k = 0.0;
    double x0 = 0.0, y0 = 0.0, S = 1.0;
    double tol = 1e-6;
    std::vector<LevelInfo> lev;

    // sorted points
    double2* xy_sorted = nullptr;   // [n]
    int64_t* perm = nullptr;        // [n] caller index of sorted point i
    int32_t* leaf_begin = nullptr;  // [4^L + 1]
    std::vector<int32_t> h_leaf_begin;

    // directly summed reaction: leaf pairs (CSR over target leaves)
    int32_t* d_begin = nullptr;     // [4^L + 1]
    int32_t* d_src = nullptr;       // [nd]
    int64_t* d_blk = nullptr;       // [nd] offset of the n_T x n_S block in d_vals
    cd* d_vals = nullptr;
    int64_t nd = 0;
    int64_t nd_vals = 0;

    // work buffers
    cd* q_sorted = nullptr;         // [max_rhs][n]
    cd* y_sorted = nullptr;         // [max_rhs][n]
    cd* io_q = nullptr;             // staging for host pointers
    cd* io_y = nullptr;
    double* io_gxy = nullptr;
    // mixed path
    cf* q32 = nullptr;              // [n][nrhs] (point-major)
    cf* y32 = nullptr;              // [n][nrhs]
    int32_t* iperm32 = nullptr;     // [n] sorted position of caller index j
    // near field on tensor cores (p2p_tc.cu): blocks (parent box, first chunk,
    // end, 0), their chunks, the pre-split tile store, and the leaves of blocks
    // too wide for the kernel (SIMT kernel)
    int32_t* nt_blocks = nullptr;
    int64_t nt_nblocks = 0;
    NtChunk* nt_chunks = nullptr;
    __half* nt_tiles = nullptr;     // f16 hi / lo tiles of (i/4) H0 x 2^NT_GSCALE_EXP
    unsigned* qmax = nullptr;       // per right-hand side: largest |Re q|, |Im q| (float bits), each apply
    int32_t* nt_fallback = nullptr;
    int64_t nt_nfallback = 0;
    int32_t* nt_leaves = nullptr;   // non-empty leaves of the tensor-core blocks (separate L2P)
    int64_t nt_nleaves = 0;
    cf* d_vals32 = nullptr;
    float2* xl32 = nullptr;         // [n] point offsets from their own leaf centre (FP32)
    cf* basis32 = nullptr;          // [n][2 p_L + 1] scaled P2M basis of each sorted point
                                    // (J_|m| e^{-i m theta} / s(|m|), sign of Graf's addition
                                    // theorem folded in); its conjugate is the L2P basis
    // position gradients (FP64): field-gradient buffers and d/dX, d/dY of the
    // directly summed reaction blocks
    // FP64 near field: (i/4) H0 blocks of every target leaf's U list, built
    // at plan time (fmm64.cu), and their offsets per leaf; null above the budget
    int64_t* near64_off = nullptr;
    cd* near64_vals = nullptr;
    void* krylov = nullptr;         // hfmm_solve: Krylov vectors (first call; grows with restart)
    size_t krylov_bytes = 0;
    double* krylov_part = nullptr;  // partial sums of its dot products
    cd* near64g_x = nullptr;        // d/dx, d/dy of the same blocks (first gradient request)
    cd* near64g_y = nullptr;
    cd* grad_buf = nullptr;         // [5][max_rhs][n]
    cd* grad_q = nullptr;           // mixed plans: widened strengths / loss gradient
    cd* grad_g = nullptr;
    cd* d_gvals = nullptr;          // [2][nd_vals]
    void* dj_jobs = nullptr;        // direct-block quadrature jobs and segments (tables.cu)
    void* dj_segs = nullptr;
    int64_t dj_njobs = 0;
    bool tc_on = false;             // every level lmin..L has tensor-core M2M / downward state
    bool tc_l2p = false;            // leaf L2P fused into the tensor-core downward epilogue
    // leaf level with level-wide scales: every leaf multipole row r written with
    // the exponent of the bound 2 qmax_r p2m_gain (p2m_gain = largest sum over a
    // leaf's points of |basis|), one factor for all free and reaction tables, so
    // the leaf-level V and reaction steps of a tile accumulate in TMEM (one drain)
    bool tc_leaf_runs = false;
    float p2m_gain = 0.0f;
    // concurrent near field: the far-field chain on a high-priority stream, the
    // near field on a low-priority one, both forked from and joined back into the
    // caller's stream (created on first use)
    cudaStream_t far_st = nullptr, near_st = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_near_done = nullptr, ev_far_done = nullptr;
    int* tc_err = nullptr;          // set by the tensor-core pass when a bounded wait gave up
    long tc_spin = 0;               // polls of a bounded device wait (options.spin_limit or the default)
    __half* tc_zero = nullptr;      // 4 KB of zeros: the A half of a missing source box
    float* tc_part = nullptr;       // partial sums of split launches (levels with few tiles)
    size_t tc_part_floats = 0;

    // table quadrature: panel-count scale (hfmm_options.quad_scale) and the
    // node-doubling check's largest weighted relative difference and where
    // (level, dx, ysum; level -1 for a directly summed block)
    double quad_scale = 1.0;
    int small_rhs = 0;              // HFMM_MIXED: applies with nrhs <= small_rhs run on small.cu
    double table_check = 0.0;
    int table_check_where[3] = {0, 0, 0};
    int diag_levels = 0;            // bit l: level l translates in diagonal form (diag.cu)
    double diag_check = 0.0;        // largest plan-time difference of a kept level

    // info
    int64_t u_pairs = 0;
    double table_bytes = 0.0;
    double buffer_bytes = 0.0;
    double plan_ms = 0.0;
    int64_t p2p_point_pairs = 0;    // sum over leaves T of n_T * sum_{S in U(T)} n_S
    std::vector<void*> allocations;

    // autotuning record (HFMM_FLAG_AUTOTUNE)
    int tune_levels[3] = {0, 0, 0};
    double tune_ms[3] = {0.0, 0.0, 0.0};

    // profiling (HFMM_FLAG_PROFILE)
    int flags = 0;
    bool events_ready = false;
    cudaEvent_t ev[HFMM_NUM_STAGES][2];
    cudaEvent_t ev_leaf[2];         // around the leaf-level tensor-core downward launch
    bool ev_leaf_used = false;
    double leaf_flops = 0.0;        // its algorithmic flops in the last apply
    bool ev_used[HFMM_NUM_STAGES] = {};
    cudaStream_t last_stream = nullptr;
    int64_t launches = 0;
    double st_flops[HFMM_NUM_STAGES] = {};
    double st_bytes[HFMM_NUM_STAGES] = {};
};

// Stage timing helper: records events on the apply stream when profiling.
struct StageTimer {
    hfmm_plan_s* P;
    cudaStream_t st;
    void begin(int s) {
        if (P->events_ready) { cudaEventRecord(P->ev[s][0], st); P->ev_used[s] = true; }
    }
    void end(int s) {
        if (P->events_ready) cudaEventRecord(P->ev[s][1], st);
    }
};

// allocation helper that records the pointer in the plan
hfmm_status plan_alloc(hfmm_plan_s* P, void** ptr, size_t bytes);

// tree.cu
hfmm_status build_tree(hfmm_plan_s* P, const double* d_xy, cudaStream_t st);
hfmm_status build_lists(hfmm_plan_s* P, cudaStream_t st);
// tables.cu
hfmm_status build_tables(hfmm_plan_s* P, cudaStream_t st);
// a directly summed reaction block: target / source point ranges (sorted
// indices) and the |X| bound and Y range of its point pairs
struct DirectSpec {
    int32_t t_lo, t_n, s_lo, s_n;
    double xmax, ymin, ymax;
};
hfmm_status build_direct_blocks(hfmm_plan_s* P, const std::vector<DirectSpec>& specs, std::vector<int64_t>& blk,
                                cudaStream_t st);
hfmm_status build_tables32(hfmm_plan_s* P, cudaStream_t st);
hfmm_status build_direct_grad(hfmm_plan_s* P, cudaStream_t st);
hfmm_status apply_grad_fp64(hfmm_plan_s* P, int nrhs, const cd* q, const cd* g, double* gxy, cudaStream_t st);
// fmm64.cu
constexpr double NEAR64_MAX_BYTES = 32e9;   // plan-time FP64 near-field blocks up to this size
hfmm_status build_near64(hfmm_plan_s* P, cudaStream_t st);
hfmm_status build_diag(hfmm_plan_s* P, cudaStream_t st);
hfmm_status build_adaptive_tree(hfmm_plan_s* P, const double* d_xy, int leaf_size, cudaStream_t st);
hfmm_status build_adaptive_lists(hfmm_plan_s* P, cudaStream_t st);
hfmm_status apply_adaptive(hfmm_plan_s* P, int nrhs, int parts, cudaStream_t st);
hfmm_status build_adaptive32(hfmm_plan_s* P, cudaStream_t st);
hfmm_status apply_adaptive32(hfmm_plan_s* P, int nrhs, int parts, cudaStream_t st);
hfmm_status adaptive_boxes(const hfmm_plan_s* P, int64_t* count, int32_t* out);
hfmm_status adaptive_pairs(const hfmm_plan_s* P, int kind, int64_t* count, int32_t* out);
int64_t adaptive_count(const hfmm_plan_s* P, int kind);
void adaptive_destroy(AdaptiveTree* T);
hfmm_status diag_src(hfmm_plan_s* P, int l, int nrhs, cudaStream_t st);
hfmm_status diag_m2l(hfmm_plan_s* P, int l, int nrhs, int parts, cudaStream_t st);
double diag_flops(const hfmm_plan_s* P, int l, int nrhs, int parts);
hfmm_status build_near64_grad(hfmm_plan_s* P, cudaStream_t st);
hfmm_status apply_fp64(hfmm_plan_s* P, int nrhs, const cd* q, cd* y, int parts, bool adjoint,
                       cudaStream_t st);
// fmm32.cu
hfmm_status apply_mixed(hfmm_plan_s* P, int nrhs, const cf* q, cf* y, int parts, bool adjoint,
                        cudaStream_t st);
hfmm_status init_h0_table(cudaStream_t st);
const float* h0_table_host();        // [2][64][6]: J0 then R0 = Y0 - (2/pi) ln(z/2) J0 pieces
// Persistent batch kernel (small.cu): segments of work items, instances and levels.
struct PSeg {
    int kind, inst, level, nchunk;   // stage, instance, level, coefficient chunks per box
    int item0, nitems;               // first global item number, item count
    int dep0, dep1;                  // segments that must be complete first (-1: none)
    int wpb;                         // 1 = eight boxes per item, one per warp (P2M, near field, and M2M /
                                     // downward levels with at most 32 coefficients), 0 = one (box,
                                     // coefficient chunk) per item
    int idep, irel;                  // segment whose items covering this item's boxes must be done first:
                                     // irel 0 the same boxes, 1 their children, 2 their parents
    int pad;
};
struct PLev {                        // one level of one instance (mixed-path buffers and tables)
    int p, pp, pc;                   // order of this level, of its parent and of its children
    cf* mult;
    cf* loc;
    const cf* cmult;                 // children's multipoles (M2M into this level)
    const cf* ploc;                  // parent's locals (null at the coarsest level)
    const cf *Tl2l, *Tfree, *Treact, *Tm2m;
    const int32_t *v_begin, *v_src, *v_off, *r_begin, *r_src, *r_tab;
};
struct PInst {
    const int32_t* lb;
    int L, lmin, lev0, nc;           // leaf level, coarsest level, first PLev, leaf coefficients
    int64_t n;
    float k, h;                      // wavenumber, leaf side
    const float2* xl;
    const cf* basis;
    cf *q32, *y32;
    const int32_t* iperm;
    const int32_t *d_begin, *d_src;
    const int64_t* d_blk;
    const cf* d_vals;
    const cf* q;                     // caller buffers the batch graph was recorded for
    cf* y;
};
struct PersistBatch;
hfmm_status persist_create(const std::vector<hfmm_plan_s*>& plans, PersistBatch** out);
hfmm_status persist_set_buffers(PersistBatch* B, const void* const* q, void* const* y, cudaStream_t st);
hfmm_status persist_launch(PersistBatch* B, int nrhs, bool adjoint, cudaStream_t st);
hfmm_status persist_device_error(PersistBatch* B, int* err);
void persist_destroy(PersistBatch* B);

// small.cu: the small-nrhs mixed path (warp-level SIMT kernels, no tensor cores)
hfmm_status init_small(hfmm_plan_s* P, cudaStream_t st);
// P2M, M2M, downward pass and near field + L2P of one apply on the sorted q32 / y32
hfmm_status apply_small(hfmm_plan_s* P, int nrhs, int parts, cudaStream_t st);
// forks P->near_st (low priority) and P->far_st (high priority) from st
hfmm_status fork_near_far(hfmm_plan_s* P, cudaStream_t st);
hfmm_status build_local_coords(hfmm_plan_s* P, cudaStream_t st);
hfmm_status fill_near_tiles(hfmm_plan_s* P, int64_t nchunks, int64_t total_rows, cudaStream_t st);
// p2p_tc.cu
hfmm_status build_p2p_tc(hfmm_plan_s* P, cudaStream_t st);
hfmm_status launch_p2p_tc(hfmm_plan_s* P, int nrhs, cudaStream_t st);
// m2l_tc.cu
hfmm_status build_tc(hfmm_plan_s* P, cudaStream_t st);
hfmm_status launch_m2l_tc(hfmm_plan_s* P, int l, int nrhs, bool fp32_out, bool l2p, cudaStream_t st);
hfmm_status launch_m2m_tc(hfmm_plan_s* P, int l, int nrhs, bool fp32_out, cudaStream_t st);
hfmm_status tc_wait_probe(long spin, int arrive, int* timed_out);

// Morton helpers
HD uint32_t spread_bits(uint32_t v) {
    v &= 0xFFFFu;
    v = (v | (v << 8)) & 0x00FF00FFu;
    v = (v | (v << 4)) & 0x0F0F0F0Fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
}
HD uint32_t compact_bits(uint32_t v) {
    v &= 0x55555555u;
    v = (v | (v >> 1)) & 0x33333333u;
    v = (v | (v >> 2)) & 0x0F0F0F0Fu;
    v = (v | (v >> 4)) & 0x00FF00FFu;
    v = (v | (v >> 8)) & 0x0000FFFFu;
    return v;
}
HD uint32_t morton(uint32_t ix, uint32_t iy) { return spread_bits(ix) | (spread_bits(iy) << 1); }
HD uint32_t morton_x(uint32_t b) { return compact_bits(b); }
HD uint32_t morton_y(uint32_t b) { return compact_bits(b >> 1); }

// Points of box b at level l.
HD void box_range(const int32_t* leaf_begin, int L, int l, int64_t b, int32_t* lo, int32_t* hi) {
    const int64_t span = (int64_t)1 << (2 * (L - l));
    *lo = leaf_begin[b * span];
    *hi = leaf_begin[(b + 1) * span];
}

// Reaction admissibility at level l (image box one box below the target box):
// y_T + y_S >= 2 h_l  <=>  iyT + iyS >= 1  or  2 y0 >= h_l.
HD bool reaction_admissible(int iyT, int iyS, double y0, double hl) {
    return (iyT + iyS >= 1) || (2.0 * y0 >= hl);
}
