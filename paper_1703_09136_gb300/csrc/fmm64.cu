// FP64 apply path: y = G q through the H-FMM (Algorithm 1, steps 2-5).
//
// Conventions (unscaled expansions, C_n(D) = H_n(k|D|) e^{i n angle D},
// J_n(v) = J_n(k|v|) e^{i n angle v}):
//   P2M  alpha_m   = sum_j q_j e^{-i m theta_j} J_m(k rho_j)              (Eq. (multi_coeff))
//   M2M  alpha^P_j = sum_m alpha^c_m J_{m-j}(P - c)
//   M2L  beta_p   += sum_m alpha_m C_{m-p}(x_T - x_S)                    (Sec. 3.3)
//   react beta_p  += sum_m (-1)^m alpha_m A_{-m-p}(x_T - x_S, y_T + y_S)  (Eq. (m2l), (eq:m2loperator);
//                    image coefficients alpha^im_m = (-1)^m alpha_{-m})
//   L2L  beta^c_m  = sum_n beta^P_n J_{n-m}(c - P)
//   L2P  y_i      += (i/4) sum_p beta_p J_p(k rho_i) e^{i p theta_i}
//   P2P  y_i      += sum_{j in U, j != i} (i/4) H0(k r_ij) q_j            (Eq. (eq:direct), free part)
//   direct reaction for leaf pairs whose images are not separated from the target leaf.
#include <algorithm>
#include <vector>

#include "bessel.cuh"
#include "plan.cuh"

namespace {

constexpr int TB = 128;

// CTAs per box for the per-box translation kernels: enough to spread a level
// with few boxes over the GPU (FP64 throughput is per SM), one where the
// level alone fills it.
inline unsigned box_split(int64_t nbox, int items) {
    if (nbox >= 2048) return 1;
    const int64_t by_items = (items + TB - 1) / TB;
    const int64_t by_grid = (2048 + nbox - 1) / nbox;
    return (unsigned)std::max<int64_t>(1, std::min(by_items, by_grid));
}

__global__ void gather_q(const cd* q, const int64_t* perm, int64_t n, int nrhs, bool conj_in,
                         cd* qs) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t j = perm[i];
    for (int r = 0; r < nrhs; ++r) {
        cd v = q[(int64_t)r * n + j];
        qs[(int64_t)r * n + i] = conj_in ? cconj(v) : v;
    }
}

__global__ void scatter_y(const cd* ys, const int64_t* perm, int64_t n, int nrhs, bool conj_out,
                          cd* y) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t j = perm[i];
    for (int r = 0; r < nrhs; ++r) {
        cd v = ys[(int64_t)r * n + i];
        y[(int64_t)r * n + j] = conj_out ? cconj(v) : v;
    }
}

// basis of one point about centre (cx, cy): B[m + p] = J_m(k rho) e^{sgn i m theta},
// m = -p .. p, using J_{-m} = (-1)^m J_m.  Jt: scratch of p + 1 doubles.
__device__ void point_basis(double px, double py, double cx, double cy, double k, int p, int sgn,
                            double* Jt, cd* B) {
    const double dx = px - cx, dy = py - cy;
    const double rho = hypot(dx, dy);
    bessel_j_seq(k * rho, p, Jt);
    const double th = atan2(dy, dx);
    const cd e1 = cexpi(sgn * th);
    cd e = cmk(1.0, 0.0);
    B[p] = cmk(Jt[0], 0.0);
    for (int m = 1; m <= p; ++m) {
        e = cmul(e, e1);
        const double sg = (m & 1) ? -1.0 : 1.0;
        B[p + m] = cscale(e, Jt[m]);
        B[p - m] = cscale(cconj(e), sg * Jt[m]);
    }
}

// P2M: one CTA per leaf.  Dynamic smem: chunk * (ncoef cd + (p+1) double).
__global__ void p2m_kernel(const int32_t* lb, const double2* xs, const cd* qs, int64_t n, int nrhs,
                           double x0, double y0, double h, int L, double k, int p, int chunk,
                           cd* mult) {
    extern __shared__ double smem[];
    const int64_t b = blockIdx.x;
    const int ncoef = 2 * p + 1;
    cd* B = (cd*)smem;
    double* Jt = (double*)(B + (size_t)chunk * ncoef);
    const int32_t lo = lb[b], hi = lb[b + 1];
    const double cx = x0 + (morton_x((uint32_t)b) + 0.5) * h;
    const double cy = y0 + (morton_y((uint32_t)b) + 0.5) * h;
    cd* out = mult + (int64_t)b * nrhs * ncoef;
    const int items = nrhs * ncoef;
    for (int it = threadIdx.x; it < items; it += blockDim.x) out[it] = cmk(0.0, 0.0);
    for (int32_t c0 = lo; c0 < hi; c0 += chunk) {
        const int cnt = min(chunk, hi - c0);
        __syncthreads();
        for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
            const double2 pt = xs[c0 + t];
            point_basis(pt.x, pt.y, cx, cy, k, p, -1, Jt + (size_t)t * (p + 1), B + (size_t)t * ncoef);
        }
        __syncthreads();
        for (int it = threadIdx.x; it < items; it += blockDim.x) {
            const int r = it / ncoef, m = it % ncoef;
            cd acc = out[it];
            const cd* qr = qs + (int64_t)r * n + c0;
            for (int t = 0; t < cnt; ++t) cfma(acc, qr[t], B[(size_t)t * ncoef + m]);
            out[it] = acc;
        }
    }
}

// M2M: parent b at level l from children at level l + 1.
__global__ void m2m_kernel(const cd* child, const cd* T, int pc, int pp, int nrhs, cd* parent) {
    const int64_t b = blockIdx.x;
    const int nc = 2 * pc + 1, np = 2 * pp + 1, nmax = pc + pp, w = 2 * nmax + 1;
    const int items = nrhs * np;
    // blockIdx.y splits a box's outputs over several CTAs (coarse levels have few boxes)
    for (int it = blockIdx.y * blockDim.x + threadIdx.x; it < items; it += gridDim.y * blockDim.x) {
        const int r = it / np, j = it % np - pp;
        cd acc = cmk(0.0, 0.0);
        for (int c = 0; c < 4; ++c) {
            const cd* a = child + ((4 * b + c) * nrhs + r) * (int64_t)nc;
            const cd* Tc = T + (int64_t)c * w + nmax;
            for (int m = -pc; m <= pc; ++m) cfma(acc, a[m + pc], Tc[m - j]);
        }
        parent[(b * nrhs + r) * (int64_t)np + j + pp] = acc;
    }
}

// Downward pass at level l, one CTA per non-empty box:
// L2L from the parent, free-space M2L over the V list, reaction M2L over the R list.
__global__ void downward_kernel(const int32_t* lb, int L, int l, int lmin, int nrhs, int p,
                                int pp, const cd* ploc, const cd* Tl2l, const cd* mult,
                                const int32_t* v_begin, const int32_t* v_src,
                                const int32_t* v_off, const cd* Tfree, const int32_t* r_begin,
                                const int32_t* r_src, const int32_t* r_tab, const cd* Treact,
                                int parts, cd* loc) {
    const int64_t b = blockIdx.x;
    int32_t lo, hi;
    box_range(lb, L, l, b, &lo, &hi);
    if (hi <= lo) return;
    const int nc = 2 * p + 1;
    const int items = nrhs * nc;
    const int wf = 4 * p + 1;
    for (int it = blockIdx.y * blockDim.x + threadIdx.x; it < items; it += gridDim.y * blockDim.x) {
        const int r = it / nc, q = it % nc - p;
        cd acc = cmk(0.0, 0.0);
        if (l > lmin && ploc) {
            const int64_t P = b >> 2;
            const int c = (int)(b & 3);
            const int npp = 2 * pp + 1, nmax = p + pp, w = 2 * nmax + 1;
            const cd* beta = ploc + (P * nrhs + r) * (int64_t)npp;
            const cd* Tc = Tl2l + (int64_t)c * w + nmax;
            for (int n = -pp; n <= pp; ++n) cfma(acc, beta[n + pp], Tc[n - q]);
        }
        if ((parts & HFMM_PART_FAR_FREE) && v_begin) {
            for (int32_t e = v_begin[b]; e < v_begin[b + 1]; ++e) {
                const cd* a = mult + ((int64_t)v_src[e] * nrhs + r) * nc;
                const cd* F = Tfree + (int64_t)v_off[e] * wf + 2 * p;
                for (int m = -p; m <= p; ++m) cfma(acc, a[m + p], F[m - q]);
            }
        }
        if ((parts & HFMM_PART_FAR_REACT) && r_begin) {
            for (int32_t e = r_begin[b]; e < r_begin[b + 1]; ++e) {
                const cd* a = mult + ((int64_t)r_src[e] * nrhs + r) * nc;
                const cd* A = Treact + (int64_t)r_tab[e] * wf + 2 * p;
                for (int m = -p; m <= p; ++m) {
                    cd v = a[m + p];
                    if (m & 1) v = cneg(v);
                    cfma(acc, v, A[-m - q]);
                }
            }
        }
        loc[(b * nrhs + r) * (int64_t)nc + q + p] = acc;
    }
}

// L2P: one CTA per non-empty leaf.
__global__ void l2p_kernel(const int32_t* lb, const double2* xs, const cd* loc, int64_t n, int nrhs,
                           double x0, double y0, double h, double k, int p, int chunk, cd* ys) {
    extern __shared__ double smem[];
    const int64_t b = blockIdx.x;
    const int32_t lo = lb[b], hi = lb[b + 1];
    if (hi <= lo) return;
    const int ncoef = 2 * p + 1;
    cd* B = (cd*)smem;
    double* Jt = (double*)(B + (size_t)chunk * ncoef);
    const double cx = x0 + (morton_x((uint32_t)b) + 0.5) * h;
    const double cy = y0 + (morton_y((uint32_t)b) + 0.5) * h;
    const cd* beta = loc + (int64_t)b * nrhs * ncoef;
    for (int32_t c0 = lo; c0 < hi; c0 += chunk) {
        const int cnt = min(chunk, hi - c0);
        __syncthreads();
        for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
            const double2 pt = xs[c0 + t];
            point_basis(pt.x, pt.y, cx, cy, k, p, +1, Jt + (size_t)t * (p + 1), B + (size_t)t * ncoef);
        }
        __syncthreads();
        const int items = nrhs * cnt;
        for (int it = threadIdx.x; it < items; it += blockDim.x) {
            const int r = it / cnt, t = it % cnt;
            cd acc = cmk(0.0, 0.0);
            const cd* br = beta + (int64_t)r * ncoef;
            for (int m = 0; m < ncoef; ++m) cfma(acc, br[m], B[(size_t)t * ncoef + m]);
            cd* yy = ys + (int64_t)r * n + c0 + t;
            *yy = cadd(*yy, cmuli(cscale(acc, 0.25)));
        }
    }
}

// P2P free-space part: one CTA per non-empty target leaf; kernel blocks of
// 32 x 32 (i/4) H0 values in shared memory reused across right-hand sides.
constexpr int PT = 32;
constexpr int P2P_THREADS = 256;
constexpr int P2P_RHS = 64;
constexpr int P2P_ITEMS = P2P_RHS * PT / P2P_THREADS;   // 8

__global__ void __launch_bounds__(P2P_THREADS) p2p_kernel(const int32_t* lb, int L, const double2* xs, const cd* qs,
                                                          int64_t n, int nrhs, double k, cd* ys) {
    __shared__ cd G[PT][PT + 1];
    __shared__ double2 sp[PT];
    __shared__ double2 tp[PT];
    const int64_t b = blockIdx.x;
    const int32_t tlo = lb[b], thi = lb[b + 1];
    if (thi <= tlo) return;
    const int m = 1 << L;
    const int ix = (int)morton_x((uint32_t)b), iy = (int)morton_y((uint32_t)b);
    for (int r0 = 0; r0 < nrhs; r0 += P2P_RHS) {
        const int nr = min(P2P_RHS, nrhs - r0);
        for (int32_t t0 = tlo; t0 < thi; t0 += PT) {
            const int tn = min(PT, thi - t0);
            cd acc[P2P_ITEMS];
            for (int u = 0; u < P2P_ITEMS; ++u) acc[u] = cmk(0.0, 0.0);
            __syncthreads();
            if (threadIdx.x < tn) tp[threadIdx.x] = xs[t0 + threadIdx.x];
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const int sx = ix + dx, sy = iy + dy;
                    if (sx < 0 || sy < 0 || sx >= m || sy >= m) continue;
                    const uint32_t s = morton((uint32_t)sx, (uint32_t)sy);
                    const int32_t slo = lb[s], shi = lb[s + 1];
                    for (int32_t s0 = slo; s0 < shi; s0 += PT) {
                        const int sn = min(PT, shi - s0);
                        __syncthreads();
                        if (threadIdx.x < sn) sp[threadIdx.x] = xs[s0 + threadIdx.x];
                        __syncthreads();
                        for (int e = threadIdx.x; e < PT * PT; e += blockDim.x) {
                            const int i = e / PT, j = e % PT;
                            cd g = cmk(0.0, 0.0);
                            if (i < tn && j < sn && (t0 + i) != (s0 + j)) {
                                const double r = hypot(tp[i].x - sp[j].x, tp[i].y - sp[j].y);
                                cd h0 = hankel0(k * r);
                                g = cmk(-0.25 * h0.y, 0.25 * h0.x);
                            }
                            G[i][j] = g;
                        }
                        __syncthreads();
                        for (int u = 0; u < P2P_ITEMS; ++u) {
                            const int it = u * P2P_THREADS + threadIdx.x;
                            const int rr = it / PT, i = it % PT;
                            if (rr >= nr || i >= tn) continue;
                            const cd* qr = qs + (int64_t)(r0 + rr) * n + s0;
                            cd a = acc[u];
                            for (int j = 0; j < sn; ++j) cfma(a, G[i][j], qr[j]);
                            acc[u] = a;
                        }
                    }
                }
            for (int u = 0; u < P2P_ITEMS; ++u) {
                const int it = u * P2P_THREADS + threadIdx.x;
                const int rr = it / PT, i = it % PT;
                if (rr >= nr || i >= tn) continue;
                cd* yy = ys + (int64_t)(r0 + rr) * n + t0 + i;
                *yy = cadd(*yy, acc[u]);
            }
        }
    }
}

// Directly summed reaction: one CTA per target leaf with direct pairs.
__global__ void direct_react_kernel(const int32_t* lb, const int32_t* d_begin, const int32_t* d_src,
                                    const int64_t* d_blk, const cd* vals, const cd* qs, int64_t n,
                                    int nrhs, cd* ys) {
    const int64_t b = blockIdx.x;
    const int32_t e0 = d_begin[b], e1 = d_begin[b + 1];
    if (e1 <= e0) return;
    const int32_t tlo = lb[b], tn = lb[b + 1] - tlo;
    const int items = nrhs * tn;
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
        const int r = it / tn, i = it % tn;
        cd acc = cmk(0.0, 0.0);
        for (int32_t e = e0; e < e1; ++e) {
            const int32_t s = d_src[e];
            const int32_t slo = lb[s], sn = lb[s + 1] - slo;
            const cd* G = vals + d_blk[e] + (int64_t)i * sn;
            const cd* qr = qs + (int64_t)r * n + slo;
            for (int j = 0; j < sn; ++j) cfma(acc, G[j], qr[j]);
        }
        cd* yy = ys + (int64_t)r * n + tlo + i;
        *yy = cadd(*yy, acc);
    }
}

// Near field from per-plan blocks (FP64 plans): for every target leaf T the
// values (i/4) H0(k |x_t - x_s|) of all its U-list sources s (the 3 x 3
// neighbourhood in dy, dx order, each leaf's points in order; 0 for s = t),
// stored source-major, G[off[T] + j * n_T + i], so that the lanes (targets)
// of a warp read consecutive values.  The plan computes each H0 once; an
// apply streams the blocks.
__global__ void near64_fill_kernel(const int32_t* __restrict__ lb, int L, const double2* __restrict__ xs, double k,
                                   const int64_t* __restrict__ off, cd* __restrict__ G) {
    const int64_t b = blockIdx.x;
    const int32_t tlo = lb[b], tn = lb[b + 1] - tlo;
    if (tn <= 0) return;
    const int m = 1 << L;
    const int ix = (int)morton_x((uint32_t)b), iy = (int)morton_y((uint32_t)b);
    int64_t j0 = 0;
    for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
            const int sx = ix + dx, sy = iy + dy;
            if (sx < 0 || sy < 0 || sx >= m || sy >= m) continue;
            const uint32_t s = morton((uint32_t)sx, (uint32_t)sy);
            const int32_t slo = lb[s], sn = lb[s + 1] - slo;
            for (int e = threadIdx.x; e < sn * tn; e += blockDim.x) {
                const int j = e / tn, i = e % tn;
                cd g = cmk(0.0, 0.0);
                if (tlo + i != slo + j) {
                    const double2 a = xs[tlo + i], c = xs[slo + j];
                    const cd h0 = hankel0(k * hypot(a.x - c.x, a.y - c.y));
                    g = cmk(-0.25 * h0.y, 0.25 * h0.x);
                }
                G[off[b] + (j0 + j) * tn + i] = g;
            }
            j0 += sn;
        }
}

// y[r][t] += sum over the U-list sources s of G[s][t] q[r][s]: a warp per
// target leaf (four per CTA), lane = target (passes of 32).
__global__ void __launch_bounds__(128) near64_kernel(const int32_t* __restrict__ lb, int L, int64_t nleaf,
                                                     const int64_t* __restrict__ off, const cd* __restrict__ G,
                                                     const cd* __restrict__ qs, int64_t n, int nrhs,
                                                     cd* __restrict__ ys) {
    const int64_t b = (int64_t)blockIdx.x * 4 + (threadIdx.x >> 5);
    if (b >= nleaf) return;
    const int lane = threadIdx.x & 31;
    const int32_t tlo = lb[b], tn = lb[b + 1] - tlo;
    if (tn <= 0) return;
    const int m = 1 << L;
    const int ix = (int)morton_x((uint32_t)b), iy = (int)morton_y((uint32_t)b);
    const cd* Gb = G + off[b];
    for (int r = 0; r < nrhs; ++r)
        for (int i0 = 0; i0 < tn; i0 += 32) {
            const int i = i0 + lane;
            const bool live = i < tn;
            cd acc = cmk(0.0, 0.0);
            int64_t j = 0;
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const int sx = ix + dx, sy = iy + dy;
                    if (sx < 0 || sy < 0 || sx >= m || sy >= m) continue;
                    const uint32_t s = morton((uint32_t)sx, (uint32_t)sy);
                    const int32_t slo = lb[s], shi = lb[s + 1];
                    const cd* qr = qs + (int64_t)r * n;
#pragma unroll 4
                    for (int32_t js = slo; js < shi; ++js, ++j)
                        if (live) cfma(acc, Gb[j * tn + i], qr[js]);
                }
            if (live) {
                cd* yy = ys + (int64_t)r * n + tlo + i;
                *yy = cadd(*yy, acc);
            }
        }
}

int pick_chunk(int p) {
    const int ncoef = 2 * p + 1;
    int c = (int)(40000 / (ncoef * 16 + (p + 1) * 8));
    return std::max(1, std::min(32, c));
}

}  // namespace

// Dense free + reaction translations of level l alone (no L2L) from mult into
// loc (used by the plan-time check of the diagonal form).
hfmm_status down64_lists(hfmm_plan_s* P, int l, int nrhs, const cd* mult, cd* loc, cudaStream_t st) {
    LevelInfo& lv = P->lev[l];
    downward_kernel<<<dim3((unsigned)lv.nbox, box_split(lv.nbox, nrhs * lv.ncoef)), TB, 0, st>>>(P->leaf_begin, P->L, l, l, nrhs, lv.p, 0, nullptr, nullptr, mult,
                                                     lv.nv ? lv.v_begin : nullptr, lv.v_src, lv.v_off, lv.t_free,
                                                     lv.nr ? lv.r_begin : nullptr, lv.r_src, lv.r_tab, lv.t_react,
                                                     HFMM_PART_ALL, loc);
    HFMM_CUDA_TRY(cudaGetLastError());
    return HFMM_OK;
}

hfmm_status apply_fp64(hfmm_plan_s* P, int nrhs, const cd* q, cd* y, int parts, bool adjoint,
                       cudaStream_t st) {
    const int64_t n = P->n;
    const int L = P->L;
    const int nb = ceil_div(n, 256);
    StageTimer tm{P, st};
    P->launches = 0;
    for (int s = 0; s < HFMM_NUM_STAGES; ++s) { P->st_flops[s] = 0.0; P->st_bytes[s] = 0.0; P->ev_used[s] = false; }
    const double C = 16.0 * nrhs;      // bytes of one complex128 value per right-hand side
    const double MAC = 8.0 * nrhs;     // real flops of one complex multiply-add per right-hand side
    tm.begin(HFMM_STAGE_GATHER);
    gather_q<<<nb, 256, 0, st>>>(q, P->perm, n, nrhs, adjoint, P->q_sorted);
    ++P->launches;
    HFMM_CUDA_TRY(cudaMemsetAsync(P->y_sorted, 0, sizeof(cd) * n * nrhs, st));
    tm.end(HFMM_STAGE_GATHER);
    P->st_bytes[HFMM_STAGE_GATHER] = 2.0 * C * n + 8.0 * n;
    if (P->ad) HFMM_TRY(apply_adaptive(P, nrhs, parts, st));
    else {
        const bool far = (parts & (HFMM_PART_FAR_FREE | HFMM_PART_FAR_REACT)) != 0;
        if (far) {
            // step 2: upward pass
            {
                LevelInfo& lv = P->lev[L];
                const int chunk = pick_chunk(lv.p);
                const size_t sm = (size_t)chunk * ((2 * lv.p + 1) * sizeof(cd) + (lv.p + 1) * sizeof(double));
                tm.begin(HFMM_STAGE_P2M);
                p2m_kernel<<<(unsigned)lv.nbox, TB, sm, st>>>(P->leaf_begin, P->xy_sorted, P->q_sorted, n, nrhs,
                                                             P->x0, P->y0, lv.h, L, P->k, lv.p, chunk, lv.mult);
                ++P->launches;
                HFMM_CUDA_TRY(cudaGetLastError());
                if (lv.diag_logq) HFMM_TRY(diag_src(P, L, nrhs, st));
                tm.end(HFMM_STAGE_P2M);
                P->st_flops[HFMM_STAGE_P2M] = MAC * n * lv.ncoef;
                P->st_bytes[HFMM_STAGE_P2M] = C * n + 16.0 * n + C * lv.nbox * lv.ncoef;
            }
            tm.begin(HFMM_STAGE_M2M);
            for (int l = L - 1; l >= P->lmin; --l) {
                LevelInfo& lv = P->lev[l];
                m2m_kernel<<<dim3((unsigned)lv.nbox, box_split(lv.nbox, nrhs * lv.ncoef)), TB, 0, st>>>(P->lev[l + 1].mult, lv.t_m2m, P->lev[l + 1].p, lv.p,
                                                            nrhs, lv.mult);
                ++P->launches;
                HFMM_CUDA_TRY(cudaGetLastError());
                if (lv.diag_logq) HFMM_TRY(diag_src(P, l, nrhs, st));
                P->st_flops[HFMM_STAGE_M2M] += MAC * 4.0 * lv.nbox * lv.ncoef * P->lev[l + 1].ncoef;
                P->st_bytes[HFMM_STAGE_M2M] += C * (4.0 * lv.nbox * P->lev[l + 1].ncoef + lv.nbox * lv.ncoef);
            }
            tm.end(HFMM_STAGE_M2M);
            // step 3: downward pass
            tm.begin(HFMM_STAGE_DOWN);
            for (int l = P->lmin; l <= L; ++l) {
                LevelInfo& lv = P->lev[l];
                const bool has_parent = l > P->lmin;
                const bool dg = lv.diag_logq > 0;   // translations in diagonal form after the L2L
                downward_kernel<<<dim3((unsigned)lv.nbox, box_split(lv.nbox, nrhs * lv.ncoef)), TB, 0, st>>>(
                    P->leaf_begin, L, l, P->lmin, nrhs, lv.p, has_parent ? P->lev[l - 1].p : 0,
                    has_parent ? P->lev[l - 1].loc : nullptr, has_parent ? P->lev[l - 1].t_l2l : nullptr,
                    lv.mult, lv.nv && !dg ? lv.v_begin : nullptr, lv.v_src, lv.v_off, lv.t_free,
                    lv.nr && !dg ? lv.r_begin : nullptr, lv.r_src, lv.r_tab, lv.t_react, parts, lv.loc);
                ++P->launches;
                HFMM_CUDA_TRY(cudaGetLastError());
                if (dg) HFMM_TRY(diag_m2l(P, l, nrhs, parts, st));
                double pairs = 0.0;
                if (parts & HFMM_PART_FAR_FREE) pairs += (double)lv.nv;
                if (parts & HFMM_PART_FAR_REACT) pairs += (double)lv.nr;
                if (dg) P->st_flops[HFMM_STAGE_DOWN] += diag_flops(P, l, nrhs, parts);
                else P->st_flops[HFMM_STAGE_DOWN] += MAC * pairs * lv.ncoef * lv.ncoef;
                if (has_parent) P->st_flops[HFMM_STAGE_DOWN] += MAC * lv.nbox * lv.ncoef * P->lev[l - 1].ncoef;
                P->st_bytes[HFMM_STAGE_DOWN] += C * lv.nbox * lv.ncoef * 2.0 +
                                                (has_parent ? C * P->lev[l - 1].nbox * P->lev[l - 1].ncoef : 0.0);
            }
            tm.end(HFMM_STAGE_DOWN);
            // step 4: local expansions at the targets
            {
                LevelInfo& lv = P->lev[L];
                const int chunk = pick_chunk(lv.p);
                const size_t sm = (size_t)chunk * ((2 * lv.p + 1) * sizeof(cd) + (lv.p + 1) * sizeof(double));
                tm.begin(HFMM_STAGE_L2P);
                l2p_kernel<<<(unsigned)lv.nbox, TB, sm, st>>>(P->leaf_begin, P->xy_sorted, lv.loc, n, nrhs, P->x0,
                                                             P->y0, lv.h, P->k, lv.p, chunk, P->y_sorted);
                ++P->launches;
                HFMM_CUDA_TRY(cudaGetLastError());
                tm.end(HFMM_STAGE_L2P);
                P->st_flops[HFMM_STAGE_L2P] = MAC * n * lv.ncoef;
                P->st_bytes[HFMM_STAGE_L2P] = C * lv.nbox * lv.ncoef + 16.0 * n + 2.0 * C * n;
            }
        }
        // step 5: direct interactions
        if (parts & HFMM_PART_NEAR_FREE) {
            tm.begin(HFMM_STAGE_P2P);
            if (P->near64_vals)
                near64_kernel<<<(unsigned)ceil_div(P->lev[L].nbox, 4), 128, 0, st>>>(
                    P->leaf_begin, L, P->lev[L].nbox, P->near64_off, P->near64_vals, P->q_sorted, n, nrhs, P->y_sorted);
            else
                p2p_kernel<<<(unsigned)P->lev[L].nbox, P2P_THREADS, 0, st>>>(P->leaf_begin, L, P->xy_sorted,
                                                                             P->q_sorted, n, nrhs, P->k, P->y_sorted);
            ++P->launches;
            HFMM_CUDA_TRY(cudaGetLastError());
            tm.end(HFMM_STAGE_P2P);
            P->st_flops[HFMM_STAGE_P2P] = MAC * (double)P->p2p_point_pairs;
            P->st_bytes[HFMM_STAGE_P2P] = C * n + 2.0 * C * n + 16.0 * n +
                                          (P->near64_vals ? 16.0 * (double)P->p2p_point_pairs : 0.0);
        }
        if ((parts & HFMM_PART_NEAR_REACT) && P->nd > 0) {
            tm.begin(HFMM_STAGE_DIRECT);
            direct_react_kernel<<<(unsigned)P->lev[L].nbox, TB, 0, st>>>(P->leaf_begin, P->d_begin, P->d_src,
                                                                         P->d_blk, P->d_vals, P->q_sorted, n,
                                                                         nrhs, P->y_sorted);
            ++P->launches;
            HFMM_CUDA_TRY(cudaGetLastError());
            tm.end(HFMM_STAGE_DIRECT);
            P->st_flops[HFMM_STAGE_DIRECT] = MAC * (double)P->nd_vals;
            P->st_bytes[HFMM_STAGE_DIRECT] = 16.0 * (double)P->nd_vals;
        }
    }
    tm.begin(HFMM_STAGE_SCATTER);
    scatter_y<<<nb, 256, 0, st>>>(P->y_sorted, P->perm, n, nrhs, adjoint, y);
    ++P->launches;
    HFMM_CUDA_TRY(cudaGetLastError());
    tm.end(HFMM_STAGE_SCATTER);
    P->st_bytes[HFMM_STAGE_SCATTER] = 2.0 * C * n + 8.0 * n;
    P->last_stream = st;
    return HFMM_OK;
}

// ---------------------------------------------------------------------------
// Field gradients (FP64) for position gradients of a loss through y = A(x) q.
// For Z_n e^{in theta} of any cylinder function,
//   (d/dx + i d/dy) Z_n e^{in th} = -k Z_{n+1} e^{i(n+1) th},
//   (d/dx - i d/dy) Z_n e^{in th} =  k Z_{n-1} e^{i(n-1) th},
// so the local expansion (i/4) sum_p b_p J_p(x - c) has
//   d/dx = (i/4)(k/2) sum_p b_p (J_{p-1} - J_{p+1}),
//   d/dy = (i/4)(i k/2) sum_p b_p (J_{p-1} + J_{p+1}),
// and the free kernel d/dx (i/4) H0(k r) = (i/4)(-k H1(k r)) (x - x_j) / r.
// ---------------------------------------------------------------------------
namespace {

// Bx, By [2p+1]: gradient bases of one point; E scratch [2p+3], Jt [p+2]
__device__ void point_basis_grad(double px, double py, double cx, double cy, double k, int p, double* Jt,
                                 cd* E, cd* Bx, cd* By) {
    const double dx = px - cx, dy = py - cy;
    const double rho = hypot(dx, dy);
    bessel_j_seq(k * rho, p + 1, Jt);
    const double th = atan2(dy, dx);
    const cd e1 = cexpi(th);
    cd e = cmk(1.0, 0.0);
    E[p + 1] = cmk(Jt[0], 0.0);                 // E[n + p + 1] = J_n(k rho) e^{i n th}
    for (int m = 1; m <= p + 1; ++m) {
        e = cmul(e, e1);
        const double sg = (m & 1) ? -1.0 : 1.0;
        E[p + 1 + m] = cscale(e, Jt[m]);
        E[p + 1 - m] = cscale(cconj(e), sg * Jt[m]);
    }
    const cd cx_ = cmk(0.0, 0.125 * k);         // (i/4)(k/2)
    const cd cy_ = cmk(-0.125 * k, 0.0);        // (i/4)(i k/2)
    for (int q = -p; q <= p; ++q) {
        const cd lo = E[p + 1 + q - 1], hi = E[p + 1 + q + 1];
        Bx[q + p] = cmul(cx_, csub(lo, hi));
        By[q + p] = cmul(cy_, cadd(lo, hi));
    }
}

__global__ void l2p_grad_kernel(const int32_t* lb, const double2* xs, const cd* loc, int64_t n, int nrhs,
                                double x0, double y0, double h, double k, int p, int chunk, cd* fx, cd* fy) {
    extern __shared__ double smem[];
    const int64_t b = blockIdx.x;
    const int32_t lo = lb[b], hi = lb[b + 1];
    if (hi <= lo) return;
    const int nc = 2 * p + 1;
    cd* Bx = (cd*)smem;
    cd* By = Bx + (size_t)chunk * nc;
    cd* E = By + (size_t)chunk * nc;
    double* Jt = (double*)(E + (size_t)chunk * (nc + 2));
    const double cx = x0 + (morton_x((uint32_t)b) + 0.5) * h;
    const double cy = y0 + (morton_y((uint32_t)b) + 0.5) * h;
    const cd* beta = loc + (int64_t)b * nrhs * nc;
    for (int32_t c0 = lo; c0 < hi; c0 += chunk) {
        const int cnt = min(chunk, hi - c0);
        __syncthreads();
        for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
            const double2 pt = xs[c0 + t];
            point_basis_grad(pt.x, pt.y, cx, cy, k, p, Jt + (size_t)t * (p + 2), E + (size_t)t * (nc + 2),
                             Bx + (size_t)t * nc, By + (size_t)t * nc);
        }
        __syncthreads();
        for (int it = threadIdx.x; it < nrhs * cnt; it += blockDim.x) {
            const int r = it / cnt, t = it % cnt;
            cd ax = cmk(0.0, 0.0), ay = cmk(0.0, 0.0);
            const cd* br = beta + (int64_t)r * nc;
            for (int m = 0; m < nc; ++m) {
                cfma(ax, br[m], Bx[(size_t)t * nc + m]);
                cfma(ay, br[m], By[(size_t)t * nc + m]);
            }
            const int64_t o = (int64_t)r * n + c0 + t;
            fx[o] = cadd(fx[o], ax);
            fy[o] = cadd(fy[o], ay);
        }
    }
}

constexpr int GPT = 32;
__global__ void __launch_bounds__(256) p2p_grad_kernel(const int32_t* lb, int L, const double2* xs, const cd* qs,
                                                       int64_t n, int nrhs, double k, cd* fx, cd* fy) {
    __shared__ cd Gx[GPT][GPT + 1];
    __shared__ cd Gy[GPT][GPT + 1];
    __shared__ double2 sp[GPT];
    __shared__ double2 tp[GPT];
    const int64_t b = blockIdx.x;
    const int32_t tlo = lb[b], thi = lb[b + 1];
    if (thi <= tlo) return;
    const int m = 1 << L;
    const int ix = (int)morton_x((uint32_t)b), iy = (int)morton_y((uint32_t)b);
    for (int32_t t0 = tlo; t0 < thi; t0 += GPT) {
        const int tn = min(GPT, thi - t0);
        __syncthreads();
        if (threadIdx.x < tn) tp[threadIdx.x] = xs[t0 + threadIdx.x];
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const int sx = ix + dx, sy = iy + dy;
                if (sx < 0 || sy < 0 || sx >= m || sy >= m) continue;
                const uint32_t s = morton((uint32_t)sx, (uint32_t)sy);
                const int32_t slo = lb[s], shi = lb[s + 1];
                for (int32_t s0 = slo; s0 < shi; s0 += GPT) {
                    const int sn = min(GPT, shi - s0);
                    __syncthreads();
                    if (threadIdx.x < sn) sp[threadIdx.x] = xs[s0 + threadIdx.x];
                    __syncthreads();
                    for (int e = threadIdx.x; e < GPT * GPT; e += blockDim.x) {
                        const int i = e / GPT, j = e % GPT;
                        cd gx = cmk(0.0, 0.0), gy = cmk(0.0, 0.0);
                        if (i < tn && j < sn && (t0 + i) != (s0 + j)) {
                            const double ddx = tp[i].x - sp[j].x, ddy = tp[i].y - sp[j].y;
                            const double r = hypot(ddx, ddy);
                            cd h0, h1;
                            hankel01(k * r, &h0, &h1);
                            const cd c = cscale(cmuli(h1), -0.25 * k / r);   // (i/4)(-k H1) / r
                            gx = cscale(c, ddx);
                            gy = cscale(c, ddy);
                        }
                        Gx[i][j] = gx;
                        Gy[i][j] = gy;
                    }
                    __syncthreads();
                    for (int it = threadIdx.x; it < nrhs * GPT; it += blockDim.x) {
                        const int rr = it / GPT, i = it % GPT;
                        if (i >= tn) continue;
                        const cd* qr = qs + (int64_t)rr * n + s0;
                        cd ax = cmk(0.0, 0.0), ay = cmk(0.0, 0.0);
                        for (int j = 0; j < sn; ++j) {
                            cfma(ax, Gx[i][j], qr[j]);
                            cfma(ay, Gy[i][j], qr[j]);
                        }
                        const int64_t o = (int64_t)rr * n + t0 + i;
                        fx[o] = cadd(fx[o], ax);
                        fy[o] = cadd(fy[o], ay);
                    }
                }
            }
    }
}

__global__ void direct_grad_kernel(const int32_t* lb, const int32_t* d_begin, const int32_t* d_src,
                                   const int64_t* d_blk, const cd* gvx, const cd* gvy, const cd* qs, int64_t n,
                                   int nrhs, cd* fx, cd* fy) {
    const int64_t b = blockIdx.x;
    const int32_t e0 = d_begin[b], e1 = d_begin[b + 1];
    if (e1 <= e0) return;
    const int32_t tlo = lb[b], tn = lb[b + 1] - tlo;
    for (int it = threadIdx.x; it < nrhs * tn; it += blockDim.x) {
        const int r = it / tn, i = it % tn;
        cd ax = cmk(0.0, 0.0), ay = cmk(0.0, 0.0);
        for (int32_t e = e0; e < e1; ++e) {
            const int32_t s = d_src[e];
            const int32_t slo = lb[s], sn = lb[s + 1] - slo;
            const int64_t o = d_blk[e] + (int64_t)i * sn;
            const cd* qr = qs + (int64_t)r * n + slo;
            for (int j = 0; j < sn; ++j) {
                cfma(ax, gvx[o + j], qr[j]);
                cfma(ay, gvy[o + j], qr[j]);
            }
        }
        const int64_t o = (int64_t)r * n + tlo + i;
        fx[o] = cadd(fx[o], ax);
        fy[o] = cadd(fy[o], ay);
    }
}

// gxy[perm[i]] = Re sum_r conj(g) d u + q d w  (sorted inputs)
__global__ void grad_combine_kernel(const cd* qs, const cd* gs_conj, const cd* ux, const cd* uy, const cd* wx,
                                    const cd* wy, const int64_t* perm, int64_t n, int nrhs, double* gxy) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double ax = 0.0, ay = 0.0;
    for (int r = 0; r < nrhs; ++r) {
        const int64_t o = (int64_t)r * n + i;
        const cd g = gs_conj[o];             // conj(g) in sorted order
        const cd q = qs[o];
        ax += cmul(g, ux[o]).x + cmul(q, wx[o]).x;
        ay += cmul(g, uy[o]).x + cmul(q, wy[o]).x;
    }
    const int64_t j = perm[i];
    gxy[2 * j] = ax;
    gxy[2 * j + 1] = ay;
}

// Near-field gradient blocks (built on a plan's first position-gradient
// request): d/dx and d/dy of (i/4) H0(k |x_t - x_s|) at the target,
// (i/4)(-k H1(k r)) (x_t - x_s) / r, for the same pairs and layout as the
// near-field blocks above (0 for s = t).
__global__ void near64_grad_fill_kernel(const int32_t* __restrict__ lb, int L, const double2* __restrict__ xs,
                                        double k, const int64_t* __restrict__ off, cd* __restrict__ Gx,
                                        cd* __restrict__ Gy) {
    const int64_t b = blockIdx.x;
    const int32_t tlo = lb[b], tn = lb[b + 1] - tlo;
    if (tn <= 0) return;
    const int m = 1 << L;
    const int ix = (int)morton_x((uint32_t)b), iy = (int)morton_y((uint32_t)b);
    int64_t j0 = 0;
    for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
            const int sx = ix + dx, sy = iy + dy;
            if (sx < 0 || sy < 0 || sx >= m || sy >= m) continue;
            const uint32_t s = morton((uint32_t)sx, (uint32_t)sy);
            const int32_t slo = lb[s], sn = lb[s + 1] - slo;
            for (int e = threadIdx.x; e < sn * tn; e += blockDim.x) {
                const int j = e / tn, i = e % tn;
                cd gx = cmk(0.0, 0.0), gy = cmk(0.0, 0.0);
                if (tlo + i != slo + j) {
                    const double2 a = xs[tlo + i], c = xs[slo + j];
                    const double ddx = a.x - c.x, ddy = a.y - c.y;
                    const double r = hypot(ddx, ddy);
                    cd h0, h1;
                    hankel01(k * r, &h0, &h1);
                    const cd cc = cscale(cmuli(h1), -0.25 * k / r);
                    gx = cscale(cc, ddx);
                    gy = cscale(cc, ddy);
                }
                const int64_t o = off[b] + (j0 + j) * tn + i;
                Gx[o] = gx;
                Gy[o] = gy;
            }
            j0 += sn;
        }
}

// fx[r][t] += sum_s Gx[s][t] v[r][s], fy likewise: a warp per target leaf.
__global__ void __launch_bounds__(128) near64_grad_kernel(const int32_t* __restrict__ lb, int L, int64_t nleaf,
                                                          const int64_t* __restrict__ off, const cd* __restrict__ Gx,
                                                          const cd* __restrict__ Gy, const cd* __restrict__ qs,
                                                          int64_t n, int nrhs, cd* __restrict__ fx,
                                                          cd* __restrict__ fy) {
    const int64_t b = (int64_t)blockIdx.x * 4 + (threadIdx.x >> 5);
    if (b >= nleaf) return;
    const int lane = threadIdx.x & 31;
    const int32_t tlo = lb[b], tn = lb[b + 1] - tlo;
    if (tn <= 0) return;
    const int m = 1 << L;
    const int ix = (int)morton_x((uint32_t)b), iy = (int)morton_y((uint32_t)b);
    for (int r = 0; r < nrhs; ++r)
        for (int i0 = 0; i0 < tn; i0 += 32) {
            const int i = i0 + lane;
            const bool live = i < tn;
            cd ax = cmk(0.0, 0.0), ay = cmk(0.0, 0.0);
            int64_t j = 0;
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const int sx = ix + dx, sy = iy + dy;
                    if (sx < 0 || sy < 0 || sx >= m || sy >= m) continue;
                    const uint32_t s = morton((uint32_t)sx, (uint32_t)sy);
                    const int32_t slo = lb[s], shi = lb[s + 1];
                    const cd* qr = qs + (int64_t)r * n;
                    for (int32_t js = slo; js < shi; ++js, ++j)
                        if (live) {
                            const cd v = qr[js];
                            const int64_t o = off[b] + j * tn + i;
                            cfma(ax, Gx[o], v);
                            cfma(ay, Gy[o], v);
                        }
                }
            if (live) {
                const int64_t o = (int64_t)r * n + tlo + i;
                fx[o] = cadd(fx[o], ax);
                fy[o] = cadd(fy[o], ay);
            }
        }
}

int pick_chunk_grad(int p) {
    const int nc = 2 * p + 1;
    int c = (int)(40000 / ((3 * nc + 2) * 16 + (p + 2) * 8));
    return std::max(1, std::min(32, c));
}

// Field gradient of v (already in sorted order in P->q_sorted) into fx, fy.
hfmm_status field_grad_fp64(hfmm_plan_s* P, int nrhs, cd* fx, cd* fy, cudaStream_t st) {
    const int64_t n = P->n;
    const int L = P->L;
    HFMM_CUDA_TRY(cudaMemsetAsync(fx, 0, sizeof(cd) * n * nrhs, st));
    HFMM_CUDA_TRY(cudaMemsetAsync(fy, 0, sizeof(cd) * n * nrhs, st));
    {
        LevelInfo& lv = P->lev[L];
        const int chunk = pick_chunk(lv.p);
        const size_t sm = (size_t)chunk * ((2 * lv.p + 1) * sizeof(cd) + (lv.p + 1) * sizeof(double));
        p2m_kernel<<<(unsigned)lv.nbox, TB, sm, st>>>(P->leaf_begin, P->xy_sorted, P->q_sorted, n, nrhs, P->x0,
                                                     P->y0, lv.h, L, P->k, lv.p, chunk, lv.mult);
        HFMM_CUDA_TRY(cudaGetLastError());
        if (lv.diag_logq) HFMM_TRY(diag_src(P, L, nrhs, st));
    }
    for (int l = L - 1; l >= P->lmin; --l) {
        LevelInfo& lv = P->lev[l];
        m2m_kernel<<<dim3((unsigned)lv.nbox, box_split(lv.nbox, nrhs * lv.ncoef)), TB, 0, st>>>(P->lev[l + 1].mult, lv.t_m2m, P->lev[l + 1].p, lv.p, nrhs, lv.mult);
        HFMM_CUDA_TRY(cudaGetLastError());
        if (lv.diag_logq) HFMM_TRY(diag_src(P, l, nrhs, st));
    }
    for (int l = P->lmin; l <= L; ++l) {
        LevelInfo& lv = P->lev[l];
        const bool has_parent = l > P->lmin;
        const bool dg = lv.diag_logq > 0;
        downward_kernel<<<dim3((unsigned)lv.nbox, box_split(lv.nbox, nrhs * lv.ncoef)), TB, 0, st>>>(
            P->leaf_begin, L, l, P->lmin, nrhs, lv.p, has_parent ? P->lev[l - 1].p : 0,
            has_parent ? P->lev[l - 1].loc : nullptr, has_parent ? P->lev[l - 1].t_l2l : nullptr, lv.mult,
            lv.nv && !dg ? lv.v_begin : nullptr, lv.v_src, lv.v_off, lv.t_free, lv.nr && !dg ? lv.r_begin : nullptr,
            lv.r_src, lv.r_tab, lv.t_react, HFMM_PART_ALL, lv.loc);
        HFMM_CUDA_TRY(cudaGetLastError());
        if (dg) HFMM_TRY(diag_m2l(P, l, nrhs, HFMM_PART_ALL, st));
    }
    {
        LevelInfo& lv = P->lev[L];
        const int chunk = pick_chunk_grad(lv.p);
        const int nc = 2 * lv.p + 1;
        const size_t sm = (size_t)chunk * ((3 * nc + 2) * sizeof(cd) + (lv.p + 2) * sizeof(double));
        l2p_grad_kernel<<<(unsigned)lv.nbox, TB, sm, st>>>(P->leaf_begin, P->xy_sorted, lv.loc, n, nrhs, P->x0,
                                                          P->y0, lv.h, P->k, lv.p, chunk, fx, fy);
        HFMM_CUDA_TRY(cudaGetLastError());
    }
    if (P->near64g_x)
        near64_grad_kernel<<<(unsigned)ceil_div(P->lev[L].nbox, 4), 128, 0, st>>>(
            P->leaf_begin, L, P->lev[L].nbox, P->near64_off, P->near64g_x, P->near64g_y, P->q_sorted, n, nrhs, fx, fy);
    else
        p2p_grad_kernel<<<(unsigned)P->lev[L].nbox, 256, 0, st>>>(P->leaf_begin, L, P->xy_sorted, P->q_sorted, n,
                                                                  nrhs, P->k, fx, fy);
    HFMM_CUDA_TRY(cudaGetLastError());
    if (P->nd > 0) {
        direct_grad_kernel<<<(unsigned)P->lev[L].nbox, TB, 0, st>>>(P->leaf_begin, P->d_begin, P->d_src, P->d_blk,
                                                                    P->d_gvals, P->d_gvals + P->nd_vals,
                                                                    P->q_sorted, n, nrhs, fx, fy);
        HFMM_CUDA_TRY(cudaGetLastError());
    }
    return HFMM_OK;
}

}  // namespace

hfmm_status apply_grad_fp64(hfmm_plan_s* P, int nrhs, const cd* q, const cd* g, double* gxy, cudaStream_t st) {
    const int64_t n = P->n;
    const int nb = ceil_div(n, 256);
    const size_t bytes = sizeof(cd) * (size_t)n * P->max_rhs;
    if (!P->grad_buf) {
        HFMM_TRY(plan_alloc(P, (void**)&P->grad_buf, 5 * bytes));
        HFMM_TRY(build_direct_grad(P, st));
        HFMM_TRY(build_near64_grad(P, st));
    }
    cd* ux = P->grad_buf;
    cd* uy = ux + (size_t)n * P->max_rhs;
    cd* wx = uy + (size_t)n * P->max_rhs;
    cd* wy = wx + (size_t)n * P->max_rhs;
    cd* gsc = wy + (size_t)n * P->max_rhs;
    // u = field of q
    gather_q<<<nb, 256, 0, st>>>(q, P->perm, n, nrhs, false, P->q_sorted);
    HFMM_CUDA_TRY(cudaGetLastError());
    HFMM_TRY(field_grad_fp64(P, nrhs, ux, uy, st));
    // w = field of conj(g)
    gather_q<<<nb, 256, 0, st>>>(g, P->perm, n, nrhs, true, gsc);
    HFMM_CUDA_TRY(cudaGetLastError());
    gather_q<<<nb, 256, 0, st>>>(g, P->perm, n, nrhs, true, P->q_sorted);
    HFMM_CUDA_TRY(cudaGetLastError());
    HFMM_TRY(field_grad_fp64(P, nrhs, wx, wy, st));
    // sorted q again for the combination
    gather_q<<<nb, 256, 0, st>>>(q, P->perm, n, nrhs, false, P->q_sorted);
    grad_combine_kernel<<<nb, 256, 0, st>>>(P->q_sorted, gsc, ux, uy, wx, wy, P->perm, n, nrhs, gxy);
    HFMM_CUDA_TRY(cudaGetLastError());
    return HFMM_OK;
}

// Offsets of the near-field blocks (every target leaf's U-list pairs) on
// the device, once per plan; returns the number of pairs in *pairs.
static hfmm_status near64_offsets(hfmm_plan_s* P, int64_t* pairs, bool alloc, cudaStream_t st) {
    const int L = P->L;
    const int64_t nleaf = P->lev[L].nbox;
    const auto& lb = P->h_leaf_begin;
    const int m = 1 << L;
    std::vector<int64_t> off(nleaf + 1, 0);
    for (int64_t b = 0; b < nleaf; ++b) {
        const int64_t tn = lb[b + 1] - lb[b];
        int64_t ns = 0;
        if (tn > 0) {
            const int ix = (int)morton_x((uint32_t)b), iy = (int)morton_y((uint32_t)b);
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const int sx = ix + dx, sy = iy + dy;
                    if (sx < 0 || sy < 0 || sx >= m || sy >= m) continue;
                    const uint32_t s = morton((uint32_t)sx, (uint32_t)sy);
                    ns += lb[s + 1] - lb[s];
                }
        }
        off[b + 1] = off[b] + tn * ns;
    }
    *pairs = off[nleaf];
    if (alloc && !P->near64_off) {
        HFMM_TRY(plan_alloc(P, (void**)&P->near64_off, sizeof(int64_t) * (nleaf + 1)));
        HFMM_CUDA_TRY(cudaMemcpyAsync(P->near64_off, off.data(), sizeof(int64_t) * (nleaf + 1),
                                      cudaMemcpyHostToDevice, st));
        HFMM_CUDA_TRY(cudaStreamSynchronize(st));
    }
    return HFMM_OK;
}

// Near-field gradient blocks, on a plan's first position-gradient request
// (skipped above the byte budget: the gradient then evaluates H1 per pair).
hfmm_status build_near64_grad(hfmm_plan_s* P, cudaStream_t st) {
    int64_t pairs = 0;
    HFMM_TRY(near64_offsets(P, &pairs, false, st));
    if (32.0 * (double)pairs > NEAR64_MAX_BYTES) return HFMM_OK;
    HFMM_TRY(near64_offsets(P, &pairs, true, st));
    HFMM_TRY(plan_alloc(P, (void**)&P->near64g_x, sizeof(cd) * std::max<int64_t>(pairs, 1)));
    HFMM_TRY(plan_alloc(P, (void**)&P->near64g_y, sizeof(cd) * std::max<int64_t>(pairs, 1)));
    near64_grad_fill_kernel<<<(unsigned)P->lev[P->L].nbox, 128, 0, st>>>(P->leaf_begin, P->L, P->xy_sorted, P->k,
                                                                          P->near64_off, P->near64g_x, P->near64g_y);
    HFMM_CUDA_TRY(cudaGetLastError());
    return HFMM_OK;
}

// Plan-time near-field blocks of an FP64 plan (skipped above the byte budget:
// the apply then evaluates H0 per pair).
hfmm_status build_near64(hfmm_plan_s* P, cudaStream_t st) {
    const int L = P->L;
    const int64_t nleaf = P->lev[L].nbox;
    const auto& lb = P->h_leaf_begin;
    const int m = 1 << L;
    std::vector<int64_t> off(nleaf + 1, 0);
    for (int64_t b = 0; b < nleaf; ++b) {
        const int64_t tn = lb[b + 1] - lb[b];
        int64_t ns = 0;
        if (tn > 0) {
            const int ix = (int)morton_x((uint32_t)b), iy = (int)morton_y((uint32_t)b);
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const int sx = ix + dx, sy = iy + dy;
                    if (sx < 0 || sy < 0 || sx >= m || sy >= m) continue;
                    const uint32_t s = morton((uint32_t)sx, (uint32_t)sy);
                    ns += lb[s + 1] - lb[s];
                }
        }
        off[b + 1] = off[b] + tn * ns;
    }
    const double bytes = 16.0 * (double)off[nleaf];
    if (bytes > NEAR64_MAX_BYTES) return HFMM_OK;
    HFMM_TRY(plan_alloc(P, (void**)&P->near64_off, sizeof(int64_t) * (nleaf + 1)));
    HFMM_TRY(plan_alloc(P, (void**)&P->near64_vals, sizeof(cd) * std::max<int64_t>(off[nleaf], 1)));
    HFMM_CUDA_TRY(cudaMemcpyAsync(P->near64_off, off.data(), sizeof(int64_t) * (nleaf + 1), cudaMemcpyHostToDevice, st));
    near64_fill_kernel<<<(unsigned)nleaf, 128, 0, st>>>(P->leaf_begin, L, P->xy_sorted, P->k, P->near64_off,
                                                        P->near64_vals);
    HFMM_CUDA_TRY(cudaGetLastError());
    P->table_bytes += bytes;
    HFMM_CUDA_TRY(cudaStreamSynchronize(st));
    return HFMM_OK;
}
