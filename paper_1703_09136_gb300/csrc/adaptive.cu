// Adaptive quadtree for FP64 plans (Sec. 3.1; HFMM_FLAG_ADAPTIVE).
//
// Tree: the root is the smallest bounding square of the points; a box that
// holds more than leaf_size points is split into its four children (down to
// level AD_MAX_LEVEL) and empty children are pruned, so leaves sit on many
// levels.  Points are sorted by their Morton key at AD_MAX_LEVEL (ties by
// caller index), so every box owns a contiguous range of sorted points.  The
// tree and its lists are built on the host at plan time (Algorithm 1, step 1);
// every step of an apply runs on the device.
//
// Lists, the usual ones of an adaptive FMM (the paper names only the
// interaction list and the neighbouring boxes):
//   V(B)  children of the colleagues of B's parent not adjacent to B    (M2L)
//   U(B)  leaves adjacent to a leaf B, of any level                     (P2P)
//   W(B)  boxes below the colleagues of a leaf B that are not adjacent
//         to B while their parent is: multipoles evaluated at B's points (M2P)
//   X(B)  leaves C with B in W(C): C's points into B's local expansion  (P2L)
// Reaction part: the pair recursion of the uniform tree from (root, root).
// An admissible pair (image box one box below the target box) goes through
// the reaction M2L of its level (same tables, indexed (dx, ysum)); an
// inadmissible pair splits into its children's pairs while both boxes have
// children; otherwise (a leaf on either side) it is summed directly, over the
// leaf pairs below it, with plan-time G^s blocks.
//
// With the multipole about c, u(x) = (i/4) sum_m a_m C_m(x - c), and the
// local expansion about l, u(x) = (i/4) sum_p b_p J_p(x - l) (C_n, J_n as in
// the uniform path), M2P and P2L are the M2L into / from an expansion of
// radius zero:
//   M2P  u(x) += (i/4) sum_m a_m H_m(k|x - c|) e^{i m angle(x - c)}
//   P2L  b_p  += q_j H_{-p}(k|l - x_j|) e^{-i p angle(l - x_j)}.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <unordered_map>
#include <vector>

#include "bessel.cuh"
#include "plan.cuh"

namespace {

constexpr int AD_TB = 128;

struct AdBox {
    int32_t level, ix, iy, lo, hi, parent, leaf, lidx;   // lidx: index within its level
    int32_t child[4];                                    // by child position (ix & 1) + 2 (iy & 1); -1: none
};

// per-level expansion pointers and orders, passed by value
struct AdLevels {
    cd* mult[AD_MAX_LEVEL + 1];
    cd* loc[AD_MAX_LEVEL + 1];
    int p[AD_MAX_LEVEL + 1];
    double h[AD_MAX_LEVEL + 1];
};

__device__ __forceinline__ void ad_centre(double x0, double y0, double h, int ix, int iy, double* cx, double* cy) {
    *cx = x0 + (ix + 0.5) * h;
    *cy = y0 + (iy + 0.5) * h;
}

// B[(m + p) sm] = J_m(k rho) e^{sgn i m theta}, m = -p .. p, (rho, theta) of
// (dx, dy); Jt: p + 1 scratch; sm: elements between consecutive orders.
__device__ void ad_jbasis(double dx, double dy, double k, int p, int sgn, double* Jt, cd* B, int sm) {
    const double rho = hypot(dx, dy);
    bessel_j_seq(k * rho, p, Jt);
    const cd e1 = cexpi(sgn * atan2(dy, dx));
    cd e = cmk(1.0, 0.0);
    B[p * sm] = cmk(Jt[0], 0.0);
    for (int m = 1; m <= p; ++m) {
        e = cmul(e, e1);
        const double sg = (m & 1) ? -1.0 : 1.0;
        B[(p + m) * sm] = cscale(e, Jt[m]);
        B[(p - m) * sm] = cscale(cconj(e), sg * Jt[m]);
    }
}

// M2P basis B[(m + p) sm] = H_m(k r) e^{i m theta} and, with p2l = true, the
// P2L basis B[(q + p) sm] = H_{-q}(k r) e^{-i q theta}; (r, theta) of (dx,
// dy), r > 0; Ht: p + 1 scratch.  H_{-m} = (-1)^m H_m.
__device__ void ad_hbasis(double dx, double dy, double k, int p, bool p2l, cd* Ht, cd* B, int sm) {
    hankel_seq(k * hypot(dx, dy), p, Ht);
    const cd e1 = cexpi(atan2(dy, dx));
    cd e = cmk(1.0, 0.0);
    B[p * sm] = Ht[0];
    for (int m = 1; m <= p; ++m) {
        e = cmul(e, e1);                                   // e^{i m theta}
        const double sg = (m & 1) ? -1.0 : 1.0;
        const cd pos = cmul(Ht[m], e);                     // H_m e^{i m theta}
        const cd neg = cscale(cmul(Ht[m], cconj(e)), sg);  // H_{-m} e^{-i m theta}
        B[(p + m) * sm] = p2l ? neg : pos;
        B[(p - m) * sm] = p2l ? pos : neg;
    }
}

// P2M at the listed leaves, one warp per leaf: per pass of up to `chunk`
// points each lane builds its point's basis (row layout B[t][m]), then the
// lanes split the (RHS, order) outputs.  Dynamic smem: chunk * ((2 pmax + 1)
// + pmax + 1) cd.
__global__ void __launch_bounds__(32) ad_p2m_kernel(const AdBox* __restrict__ boxes, const int32_t* __restrict__ list,
                                                    const double2* __restrict__ xs, const cd* __restrict__ qs, int64_t n,
                                                    int nrhs, double x0, double y0, double k, AdLevels lv, int chunk) {
    extern __shared__ double smem[];
    const AdBox b = boxes[list[blockIdx.x]];
    const int lane = threadIdx.x;
    const int l = b.level, p = lv.p[l], nc = 2 * p + 1;
    cd* B = (cd*)smem;
    cd* scr = B + (size_t)chunk * nc;
    double cx, cy;
    ad_centre(x0, y0, lv.h[l], b.ix, b.iy, &cx, &cy);
    cd* out = lv.mult[l] + (int64_t)b.lidx * nrhs * nc;
    const int items = nrhs * nc;
    for (int it = lane; it < items; it += 32) out[it] = cmk(0.0, 0.0);
    for (int32_t c0 = b.lo; c0 < b.hi; c0 += chunk) {
        const int cnt = min(chunk, b.hi - c0);
        __syncwarp();
        if (lane < cnt) {
            const double2 pt = xs[c0 + lane];
            ad_jbasis(pt.x - cx, pt.y - cy, k, p, -1, (double*)(scr + (size_t)lane * (p + 1)), B + (size_t)lane * nc, 1);
        }
        __syncwarp();
        for (int it = lane; it < items; it += 32) {
            const int r = it / nc, m = it % nc;
            cd acc = out[it];
            const cd* qr = qs + (int64_t)r * n + c0;
            for (int t = 0; t < cnt; ++t) cfma(acc, qr[t], B[(size_t)t * nc + m]);
            out[it] = acc;
        }
    }
}

// M2M into the non-leaf boxes of level l (grid: boxes of the level).
__global__ void __launch_bounds__(AD_TB) ad_m2m_kernel(const AdBox* __restrict__ boxes, int64_t off, int l,
                                                       const cd* __restrict__ T, AdLevels lv, int nrhs) {
    const AdBox b = boxes[off + blockIdx.x];
    if (b.leaf) return;
    const int pc = lv.p[l + 1], pp = lv.p[l];
    const int nc = 2 * pc + 1, np = 2 * pp + 1, nmax = pc + pp, w = 2 * nmax + 1;
    const int items = nrhs * np;
    for (int it = blockIdx.y * blockDim.x + threadIdx.x; it < items; it += gridDim.y * blockDim.x) {
        const int r = it / np, j = it % np - pp;
        cd acc = cmk(0.0, 0.0);
        for (int c = 0; c < 4; ++c) {
            if (b.child[c] < 0) continue;
            const cd* a = lv.mult[l + 1] + ((int64_t)boxes[b.child[c]].lidx * nrhs + r) * nc;
            const cd* Tc = T + (int64_t)c * w + nmax;
            for (int m = -pc; m <= pc; ++m) cfma(acc, a[m + pc], Tc[m - j]);
        }
        lv.mult[l][((int64_t)b.lidx * nrhs + r) * np + j + pp] = acc;
    }
}

// Downward pass at level l (grid: boxes of the level): L2L from the parent,
// V-list M2L, reaction M2L (sources by index within the level), then P2L of
// the X-list leaves' points.  Dynamic smem: chunk * ((2 pmax + 1) + pmax + 1) cd.
__global__ void __launch_bounds__(AD_TB) ad_down_kernel(
    const AdBox* __restrict__ boxes, int64_t off, int l, int lmin, int nrhs, AdLevels lv, const cd* __restrict__ Tl2l,
    const int32_t* __restrict__ v_beg, const int32_t* __restrict__ v_src, const int32_t* __restrict__ v_off,
    const cd* __restrict__ Tfree, const int32_t* __restrict__ r_beg, const int32_t* __restrict__ r_src,
    const int32_t* __restrict__ r_tab, const cd* __restrict__ Treact, const int32_t* __restrict__ x_beg,
    const int32_t* __restrict__ x_src, const double2* __restrict__ xs, const cd* __restrict__ qs, int64_t n,
    double x0, double y0, double k, int parts, int chunk) {
    extern __shared__ double smem[];
    const int64_t bi = off + blockIdx.x;
    const AdBox b = boxes[bi];
    const int p = lv.p[l], nc = 2 * p + 1, wf = 4 * p + 1;
    const int items = nrhs * nc;
    cd* out = lv.loc[l] + (int64_t)b.lidx * nrhs * nc;
    const bool ff = (parts & HFMM_PART_FAR_FREE) != 0, fr = (parts & HFMM_PART_FAR_REACT) != 0;
    // blockIdx.y splits the box's outputs over several CTAs (coarse levels have few
    // boxes); each thread keeps the same outputs in both phases
    for (int it = blockIdx.y * blockDim.x + threadIdx.x; it < items; it += gridDim.y * blockDim.x) {
        const int r = it / nc, q = it % nc - p;
        cd acc = cmk(0.0, 0.0);
        if (l > lmin && b.parent >= 0) {
            const AdBox P = boxes[b.parent];
            const int pp = lv.p[l - 1], npp = 2 * pp + 1, nmax = p + pp, w = 2 * nmax + 1;
            const int c = (b.ix & 1) + 2 * (b.iy & 1);
            const cd* beta = lv.loc[l - 1] + ((int64_t)P.lidx * nrhs + r) * npp;
            const cd* Tc = Tl2l + (int64_t)c * w + nmax;
            for (int m = -pp; m <= pp; ++m) cfma(acc, beta[m + pp], Tc[m - q]);
        }
        if (ff)
            for (int32_t e = v_beg[bi]; e < v_beg[bi + 1]; ++e) {
                const cd* a = lv.mult[l] + ((int64_t)v_src[e] * nrhs + r) * nc;
                const cd* F = Tfree + (int64_t)v_off[e] * wf + 2 * p;
                for (int m = -p; m <= p; ++m) cfma(acc, a[m + p], F[m - q]);
            }
        if (fr)
            for (int32_t e = r_beg[bi]; e < r_beg[bi + 1]; ++e) {
                const cd* a = lv.mult[l] + ((int64_t)r_src[e] * nrhs + r) * nc;
                const cd* A = Treact + (int64_t)r_tab[e] * wf + 2 * p;
                for (int m = -p; m <= p; ++m) {
                    cd v = a[m + p];
                    if (m & 1) v = cneg(v);
                    cfma(acc, v, A[-m - q]);
                }
            }
        out[it] = acc;
    }
    if (!ff || x_beg[bi] == x_beg[bi + 1]) return;
    // P2L: each thread keeps the items it wrote above
    cd* B = (cd*)smem;
    cd* Ht = B + (size_t)chunk * nc;
    double cx, cy;
    ad_centre(x0, y0, lv.h[l], b.ix, b.iy, &cx, &cy);
    for (int32_t e = x_beg[bi]; e < x_beg[bi + 1]; ++e) {
        const AdBox C = boxes[x_src[e]];
        for (int32_t c0 = C.lo; c0 < C.hi; c0 += chunk) {
            const int cnt = min(chunk, C.hi - c0);
            __syncthreads();
            for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
                const double2 pt = xs[c0 + t];
                ad_hbasis(cx - pt.x, cy - pt.y, k, p, true, Ht + (size_t)t * (p + 1), B + (size_t)t * nc, 1);
            }
            __syncthreads();
            for (int it = blockIdx.y * blockDim.x + threadIdx.x; it < items; it += gridDim.y * blockDim.x) {
                const int r = it / nc, q = it % nc;
                cd acc = out[it];
                const cd* qr = qs + (int64_t)r * n + c0;
                for (int t = 0; t < cnt; ++t) cfma(acc, qr[t], B[(size_t)t * nc + q]);
                out[it] = acc;
            }
        }
    }
}

// Far field at the points of every leaf, one warp per leaf (lane = point,
// passes of up to `chunk` points): L2P of its local expansion (levels >=
// lmin) and M2P of its W-list multipoles.  Each lane builds its point's basis
// in the column layout B[m][lane] and sums it against the broadcast
// coefficients.  Dynamic smem: chunk * ((2 pmax + 1) + pmax + 1) cd.
__global__ void __launch_bounds__(32) ad_leaf_far_kernel(
    const AdBox* __restrict__ boxes, const int32_t* __restrict__ leaves, const int32_t* __restrict__ w_beg,
    const int32_t* __restrict__ w_src, const double2* __restrict__ xs, int64_t n, int nrhs, double x0, double y0,
    double k, AdLevels lv, int lmin, int parts, int chunk, cd* __restrict__ ys) {
    extern __shared__ double smem[];
    const int li = blockIdx.x, lane = threadIdx.x;
    const AdBox b = boxes[leaves[li]];
    const bool l2p = b.level >= lmin;
    const int nw = (parts & HFMM_PART_FAR_FREE) ? w_beg[li + 1] - w_beg[li] : 0;
    if (!l2p && nw == 0) return;
    cd* B = (cd*)smem;
    for (int32_t c0 = b.lo; c0 < b.hi; c0 += chunk) {
        const int cnt = min(chunk, b.hi - c0);
        const bool live = lane < cnt;
        const double2 pt = live ? xs[c0 + lane] : make_double2(0.0, 0.0);
        for (int s = l2p ? 0 : 1; s <= nw; ++s) {
            int sl;
            double cx, cy;
            const cd* coef;
            if (s == 0) {
                sl = b.level;
                ad_centre(x0, y0, lv.h[sl], b.ix, b.iy, &cx, &cy);
                coef = lv.loc[sl] + (int64_t)b.lidx * nrhs * (2 * lv.p[sl] + 1);
            } else {
                const AdBox D = boxes[w_src[w_beg[li] + s - 1]];
                sl = D.level;
                ad_centre(x0, y0, lv.h[sl], D.ix, D.iy, &cx, &cy);
                coef = lv.mult[sl] + (int64_t)D.lidx * nrhs * (2 * lv.p[sl] + 1);
            }
            const int sp = lv.p[sl], nc = 2 * sp + 1;
            cd* scr = B + (size_t)chunk * nc + (size_t)lane * (sp + 1);
            __syncwarp();
            if (live) {
                if (s == 0) ad_jbasis(pt.x - cx, pt.y - cy, k, sp, +1, (double*)scr, B + lane, chunk);
                else ad_hbasis(pt.x - cx, pt.y - cy, k, sp, false, scr, B + lane, chunk);
                for (int r = 0; r < nrhs; ++r) {
                    cd acc = cmk(0.0, 0.0);
                    const cd* cr = coef + (int64_t)r * nc;
                    for (int m = 0; m < nc; ++m) cfma(acc, cr[m], B[(size_t)m * chunk + lane]);
                    cd* yy = ys + (int64_t)r * n + c0 + lane;
                    *yy = cadd(*yy, cmuli(cscale(acc, 0.25)));
                }
            }
        }
    }
}

// Plan time: (i/4) H0(k r) of every U-list pair of every leaf, source-major
// G[blk + j n_T + i] (0 where the source is the target itself).
__global__ void ad_near_fill_kernel(const AdBox* __restrict__ boxes, const int32_t* __restrict__ leaves,
                                    const int32_t* __restrict__ u_beg, const int32_t* __restrict__ u_src,
                                    const int64_t* __restrict__ u_blk, const double2* __restrict__ xs, double k,
                                    cd* __restrict__ G) {
    const int li = blockIdx.x;
    const AdBox b = boxes[leaves[li]];
    const int tn = b.hi - b.lo;
    for (int32_t e = u_beg[li]; e < u_beg[li + 1]; ++e) {
        const AdBox S = boxes[u_src[e]];
        const int sn = S.hi - S.lo;
        for (int idx = threadIdx.x; idx < tn * sn; idx += blockDim.x) {
            const int j = idx / tn, i = idx % tn;
            cd g = cmk(0.0, 0.0);
            if (b.lo + i != S.lo + j) {
                const double2 a = xs[b.lo + i], c = xs[S.lo + j];
                g = cmuli(cscale(hankel0(k * hypot(a.x - c.x, a.y - c.y)), 0.25));
            }
            G[u_blk[e] + (int64_t)j * tn + i] = g;
        }
    }
}

// Near field of every leaf, one warp per leaf (four per CTA), lane = target
// point (passes of 32): (i/4) H0 over its U list, from the plan's blocks when
// they exist (else evaluated here), and its directly summed reaction blocks.
__global__ void __launch_bounds__(128) ad_near_kernel(
    const AdBox* __restrict__ boxes, const int32_t* __restrict__ leaves, int64_t nleaf,
    const int32_t* __restrict__ u_beg, const int32_t* __restrict__ u_src, const int64_t* __restrict__ u_blk,
    const cd* __restrict__ G, const int32_t* __restrict__ d_beg, const int32_t* __restrict__ d_src,
    const int64_t* __restrict__ d_blk, const cd* __restrict__ dvals, const double2* __restrict__ xs,
    const cd* __restrict__ qs, int64_t n, int nrhs, double k, int parts, cd* __restrict__ ys) {
    const int64_t li = (int64_t)blockIdx.x * 4 + (threadIdx.x >> 5);
    if (li >= nleaf) return;
    const int lane = threadIdx.x & 31;
    const AdBox b = boxes[leaves[li]];
    const int tn = b.hi - b.lo;
    const bool nf = (parts & HFMM_PART_NEAR_FREE) != 0, nr = (parts & HFMM_PART_NEAR_REACT) != 0;
    for (int r = 0; r < nrhs; ++r) {
        const cd* qr = qs + (int64_t)r * n;
        for (int i0 = 0; i0 < tn; i0 += 32) {
            const int i = i0 + lane;
            if (i >= tn) continue;
            cd acc = cmk(0.0, 0.0);
            if (nf)
                for (int32_t e = u_beg[li]; e < u_beg[li + 1]; ++e) {
                    const AdBox S = boxes[u_src[e]];
                    if (G) {
                        const cd* Ge = G + u_blk[e] + i;
                        for (int32_t j = 0; j < S.hi - S.lo; ++j) cfma(acc, Ge[(int64_t)j * tn], qr[S.lo + j]);
                    } else {
                        const double2 a = xs[b.lo + i];
                        for (int32_t j = S.lo; j < S.hi; ++j) {
                            if (j == b.lo + i) continue;
                            const double2 c = xs[j];
                            cfma(acc, cmuli(cscale(hankel0(k * hypot(a.x - c.x, a.y - c.y)), 0.25)), qr[j]);
                        }
                    }
                }
            if (nr)
                for (int32_t e = d_beg[li]; e < d_beg[li + 1]; ++e) {
                    const AdBox S = boxes[d_src[e]];
                    const int sn = S.hi - S.lo;
                    const cd* Gr = dvals + d_blk[e] + (int64_t)i * sn;
                    for (int j = 0; j < sn; ++j) cfma(acc, Gr[j], qr[S.lo + j]);
                }
            cd* yy = ys + (int64_t)r * n + b.lo + i;
            *yy = cadd(*yy, acc);
        }
    }
}

// ---------------------------------------------------------------------------
// Mixed precision (HFMM_MIXED): expansions scaled per level as in the uniform
// mixed path (a~_m = a_m / s(|m|), b~_p = b_p s(|p|), s(n) = min(1, (k R /
// 2)^n / n!)) in FP32, the scaled FP32 translation matrices of the uniform
// path, and plan-time FP32 copies of every point's basis, computed in FP64:
//   P2M / L2P   B[m]  = J_m(k rho) e^{-i m theta} / s_l(|m|)   (L2P: conj(B))
//   P2L (X)     P[q]  = s_l(|q|) H_{-q}(k r) e^{-i q theta},  (r, theta) of l - x_j
//   M2P (W)     M[m]  = s_D(|m|) H_m(k r) e^{i m theta},      (r, theta) of x - c_D
// all bounded by one (|J_m| <= s(m) over the box; |s H_m| ~ (R / r)^m / m with
// r > R), so the apply is plain FP32 arithmetic on point-major strengths.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cfma_f(cf& acc, cf a, cf b) {
    acc.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x));
    acc.y = fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y));
}

// Plan time: scaled P2M basis of every point of the listed leaves (one CTA
// per leaf, a thread per point; Jt scratch of p + 1 doubles per thread in
// dynamic shared memory).
__global__ void ad32_basis_p2m_kernel(const AdBox* __restrict__ boxes, const int32_t* __restrict__ leaves,
                                      const int64_t* __restrict__ boff, int lup, const double2* __restrict__ xs,
                                      double x0, double y0, double k, AdLevels lv,
                                      const double* const* __restrict__ log_s, cf* __restrict__ out) {
    extern __shared__ double jt[];
    const AdBox b = boxes[leaves[blockIdx.x]];
    if (b.level < lup) return;   // no expansions at this level: no basis (and no range in out)
    const int l = b.level, p = lv.p[l], nc = 2 * p + 1;
    const double* ls = log_s[l];
    double cx, cy;
    ad_centre(x0, y0, lv.h[l], b.ix, b.iy, &cx, &cy);
    double* Jt = jt + (size_t)threadIdx.x * (p + 1);
    for (int32_t i = b.lo + threadIdx.x; i < b.hi; i += blockDim.x) {
        const double dx = xs[i].x - cx, dy = xs[i].y - cy;
        bessel_j_seq(k * hypot(dx, dy), p, Jt);
        const cd e1 = cexpi(-atan2(dy, dx));
        cf* B = out + boff[blockIdx.x] + (int64_t)(i - b.lo) * nc;
        cd e = cmk(1.0, 0.0);
        B[p] = cfmk((float)(Jt[0] * exp(-ls[0])), 0.0f);
        for (int m = 1; m <= p; ++m) {
            e = cmul(e, e1);
            const double a = Jt[m] * exp(-ls[m]);
            const double sg = (m & 1) ? -a : a;
            B[p + m] = cfmk((float)(e.x * a), (float)(e.y * a));
            B[p - m] = cfmk((float)(e.x * sg), (float)(-e.y * sg));
        }
    }
}

// Plan time: scaled M2P (m2p = true: pair = (leaf, W box), points of the
// leaf) or P2L (pair = (box, X leaf), points of the leaf, about the box)
// basis of every point of every pair.  One CTA per pair, a thread per point;
// Ht scratch of p + 1 complex values per thread in dynamic shared memory.
__global__ void ad32_basis_pair_kernel(const AdBox* __restrict__ boxes, const int32_t* __restrict__ tgt,
                                       const int32_t* __restrict__ src, const int64_t* __restrict__ boff, bool m2p,
                                       const double2* __restrict__ xs, double x0, double y0, double k, AdLevels lv,
                                       const double* const* __restrict__ log_s, cf* __restrict__ out) {
    extern __shared__ double hsm[];
    const int64_t e = blockIdx.x;
    const AdBox T = boxes[tgt[e]], S = boxes[src[e]];
    // the expansion box (its centre, order and scaling) and the box holding the points
    const AdBox& E = m2p ? S : T;
    const AdBox& X = m2p ? T : S;
    const int l = E.level, p = lv.p[l], nc = 2 * p + 1;
    const double* ls = log_s[l];
    double cx, cy;
    ad_centre(x0, y0, lv.h[l], E.ix, E.iy, &cx, &cy);
    cd* Ht = (cd*)hsm + (size_t)threadIdx.x * (p + 1);
    for (int32_t i = X.lo + threadIdx.x; i < X.hi; i += blockDim.x) {
        // M2P: (r, theta) of x - c; P2L: of c - x
        const double dx = m2p ? xs[i].x - cx : cx - xs[i].x, dy = m2p ? xs[i].y - cy : cy - xs[i].y;
        hankel_seq(k * hypot(dx, dy), p, Ht);
        const cd e1 = cexpi(atan2(dy, dx));
        cf* B = out + boff[e] + (int64_t)(i - X.lo) * nc;
        cd ee = cmk(1.0, 0.0);
        B[p] = cfmk((float)Ht[0].x, (float)Ht[0].y);
        for (int m = 1; m <= p; ++m) {
            ee = cmul(ee, e1);
            const double sc = exp(ls[m]);
            const double sg = (m & 1) ? -sc : sc;
            const cd pos = cscale(cmul(Ht[m], ee), sc);          // s H_m e^{i m theta}
            const cd neg = cscale(cmul(Ht[m], cconj(ee)), sg);   // s H_{-m} e^{-i m theta}
            const cd hi = m2p ? pos : neg, lo = m2p ? neg : pos;
            B[p + m] = cfmk((float)hi.x, (float)hi.y);
            B[p - m] = cfmk((float)lo.x, (float)lo.y);
        }
    }
}

// Plan time: (i/4) H0 of every U pair in FP32 (source-major, as the FP64 blocks).
__global__ void ad32_near_fill_kernel(const AdBox* __restrict__ boxes, const int32_t* __restrict__ leaves,
                                      const int32_t* __restrict__ u_beg, const int32_t* __restrict__ u_src,
                                      const int64_t* __restrict__ u_blk, const double2* __restrict__ xs, double k,
                                      cf* __restrict__ G) {
    const int li = blockIdx.x;
    const AdBox b = boxes[leaves[li]];
    const int tn = b.hi - b.lo;
    for (int32_t e = u_beg[li]; e < u_beg[li + 1]; ++e) {
        const AdBox S = boxes[u_src[e]];
        const int sn = S.hi - S.lo;
        for (int idx = threadIdx.x; idx < tn * sn; idx += blockDim.x) {
            const int j = idx / tn, i = idx % tn;
            cf g = cfmk(0.f, 0.f);
            if (b.lo + i != S.lo + j) {
                const double2 a = xs[b.lo + i], c = xs[S.lo + j];
                const cd h = cmuli(cscale(hankel0(k * hypot(a.x - c.x, a.y - c.y)), 0.25));
                g = cfmk((float)h.x, (float)h.y);
            }
            G[u_blk[e] + (int64_t)j * tn + i] = g;
        }
    }
}

// per-level FP32 expansion pointers
struct AdLevels32 {
    cf* mult[AD_MAX_LEVEL + 1];
    cf* loc[AD_MAX_LEVEL + 1];
    int p[AD_MAX_LEVEL + 1];
};

// P2M (scaled) at the listed leaves, one warp per leaf: lanes over (RHS, order).
__global__ void __launch_bounds__(32) ad32_p2m_kernel(const AdBox* __restrict__ boxes, const int32_t* __restrict__ leaves,
                                                      const int32_t* __restrict__ list, const int64_t* __restrict__ boff,
                                                      const cf* __restrict__ basis, const cf* __restrict__ qs, int nrhs,
                                                      AdLevels32 lv) {
    const int li = list[blockIdx.x];
    const AdBox b = boxes[leaves[li]];
    const int l = b.level, nc = 2 * lv.p[l] + 1;
    const cf* B = basis + boff[li];
    cf* out = lv.mult[l] + (int64_t)b.lidx * nrhs * nc;
    for (int it = threadIdx.x; it < nrhs * nc; it += 32) {
        const int r = it / nc, m = it % nc;
        cf acc = cfmk(0.f, 0.f);
        for (int32_t j = b.lo; j < b.hi; ++j) cfma_f(acc, qs[(int64_t)j * nrhs + r], B[(int64_t)(j - b.lo) * nc + m]);
        out[it] = acc;
    }
}

// M2M (scaled) into the non-leaf boxes of level l: a~_j += sum_c sum_m T~[c][m][j] a~^c_m.
__global__ void __launch_bounds__(AD_TB) ad32_m2m_kernel(const AdBox* __restrict__ boxes, int64_t off, int l,
                                                         const cf* __restrict__ T, AdLevels32 lv, int nrhs) {
    const AdBox b = boxes[off + blockIdx.x];
    if (b.leaf) return;
    const int nc = 2 * lv.p[l + 1] + 1, np = 2 * lv.p[l] + 1;
    for (int it = blockIdx.y * blockDim.x + threadIdx.x; it < nrhs * np; it += gridDim.y * blockDim.x) {
        const int r = it / np, j = it % np;
        cf acc = cfmk(0.f, 0.f);
        for (int c = 0; c < 4; ++c) {
            if (b.child[c] < 0) continue;
            const cf* a = lv.mult[l + 1] + ((int64_t)boxes[b.child[c]].lidx * nrhs + r) * nc;
            const cf* Tc = T + (int64_t)c * nc * np + j;
            for (int m = 0; m < nc; ++m) cfma_f(acc, a[m], Tc[(int64_t)m * np]);
        }
        lv.mult[l][((int64_t)b.lidx * nrhs + r) * np + j] = acc;
    }
}

// Downward pass (scaled) at level l: L2L, V-list and reaction M2L, then P2L of
// the X-list leaves' points with their plan-time bases.
__global__ void __launch_bounds__(AD_TB) ad32_down_kernel(
    const AdBox* __restrict__ boxes, int64_t off, int l, int lmin, int nrhs, AdLevels32 lv,
    const cf* __restrict__ Tl2l, const int32_t* __restrict__ v_beg, const int32_t* __restrict__ v_src,
    const int32_t* __restrict__ v_off, const cf* __restrict__ Tfree, const int32_t* __restrict__ r_beg,
    const int32_t* __restrict__ r_src, const int32_t* __restrict__ r_tab, const cf* __restrict__ Treact,
    const int32_t* __restrict__ x_beg, const int32_t* __restrict__ x_src, const int64_t* __restrict__ x_boff,
    const cf* __restrict__ p2l, const cf* __restrict__ qs, int parts) {
    const int64_t bi = off + blockIdx.x;
    const AdBox b = boxes[bi];
    const int nc = 2 * lv.p[l] + 1;
    const bool ff = (parts & HFMM_PART_FAR_FREE) != 0, fr = (parts & HFMM_PART_FAR_REACT) != 0;
    const bool l2l = l > lmin && b.parent >= 0;
    const int c = (b.ix & 1) + 2 * (b.iy & 1);
    for (int it = blockIdx.y * blockDim.x + threadIdx.x; it < nrhs * nc; it += gridDim.y * blockDim.x) {
        const int r = it / nc, q = it % nc;
        cf acc = cfmk(0.f, 0.f);
        if (l2l) {
            const int npp = 2 * lv.p[l - 1] + 1;
            const cf* beta = lv.loc[l - 1] + ((int64_t)boxes[b.parent].lidx * nrhs + r) * npp;
            const cf* Tc = Tl2l + (int64_t)c * npp * nc + q;
            for (int n = 0; n < npp; ++n) cfma_f(acc, beta[n], Tc[(int64_t)n * nc]);
        }
        if (ff)
            for (int32_t e = v_beg[bi]; e < v_beg[bi + 1]; ++e) {
                const cf* a = lv.mult[l] + ((int64_t)v_src[e] * nrhs + r) * nc;
                const cf* F = Tfree + (int64_t)v_off[e] * nc * nc + q;
                for (int m = 0; m < nc; ++m) cfma_f(acc, a[m], F[(int64_t)m * nc]);
            }
        if (fr)
            for (int32_t e = r_beg[bi]; e < r_beg[bi + 1]; ++e) {
                const cf* a = lv.mult[l] + ((int64_t)r_src[e] * nrhs + r) * nc;
                const cf* H = Treact + (int64_t)r_tab[e] * nc * nc + q;
                for (int m = 0; m < nc; ++m) cfma_f(acc, a[m], H[(int64_t)m * nc]);
            }
        if (ff)
            for (int32_t e = x_beg[bi]; e < x_beg[bi + 1]; ++e) {
                const AdBox C = boxes[x_src[e]];
                const cf* Pb = p2l + x_boff[e] + q;
                for (int32_t j = C.lo; j < C.hi; ++j) cfma_f(acc, qs[(int64_t)j * nrhs + r], Pb[(int64_t)(j - C.lo) * nc]);
            }
        lv.loc[l][((int64_t)b.lidx * nrhs + r) * nc + q] = acc;
    }
}

// Far field (scaled) at the points of every leaf, one warp per leaf, lane =
// point: L2P (conj of the P2M basis) and M2P of the W list.
__global__ void __launch_bounds__(32) ad32_leaf_far_kernel(
    const AdBox* __restrict__ boxes, const int32_t* __restrict__ leaves, const int64_t* __restrict__ boff,
    const cf* __restrict__ basis, const int32_t* __restrict__ w_beg, const int32_t* __restrict__ w_src,
    const int64_t* __restrict__ w_boff, const cf* __restrict__ m2p, int nrhs, AdLevels32 lv, int lmin, int parts,
    cf* __restrict__ ys) {
    const int li = blockIdx.x, lane = threadIdx.x;
    const AdBox b = boxes[leaves[li]];
    const bool l2p = b.level >= lmin;
    const int nw = (parts & HFMM_PART_FAR_FREE) ? w_beg[li + 1] - w_beg[li] : 0;
    const int ncl = 2 * lv.p[b.level] + 1;
    for (int32_t i = b.lo + lane; i < b.hi; i += 32) {
        for (int r = 0; r < nrhs; ++r) {
            cf acc = cfmk(0.f, 0.f);
            if (l2p) {
                const cf* beta = lv.loc[b.level] + ((int64_t)b.lidx * nrhs + r) * ncl;
                const cf* B = basis + boff[li] + (int64_t)(i - b.lo) * ncl;
                for (int m = 0; m < ncl; ++m) cfma_f(acc, beta[m], cfmk(B[m].x, -B[m].y));
            }
            for (int s = 0; s < nw; ++s) {
                const int32_t e = w_beg[li] + s;
                const AdBox D = boxes[w_src[e]];
                const int ncd = 2 * lv.p[D.level] + 1;
                const cf* a = lv.mult[D.level] + ((int64_t)D.lidx * nrhs + r) * ncd;
                const cf* M = m2p + w_boff[e] + (int64_t)(i - b.lo) * ncd;
                for (int m = 0; m < ncd; ++m) cfma_f(acc, a[m], M[m]);
            }
            cf* yy = ys + (int64_t)i * nrhs + r;
            *yy = cfmk(yy->x - 0.25f * acc.y, yy->y + 0.25f * acc.x);
        }
    }
}

// Near field (FP32) of every leaf, one warp per leaf (four per CTA), lane =
// target: plan-time (i/4) H0 blocks of the U list and the directly summed
// reaction blocks.
__global__ void __launch_bounds__(128) ad32_near_kernel(
    const AdBox* __restrict__ boxes, const int32_t* __restrict__ leaves, int64_t nleaf,
    const int32_t* __restrict__ u_beg, const int32_t* __restrict__ u_src, const int64_t* __restrict__ u_blk,
    const cf* __restrict__ G, const int32_t* __restrict__ d_beg, const int32_t* __restrict__ d_src,
    const int64_t* __restrict__ d_blk, const cf* __restrict__ dvals, const cf* __restrict__ qs, int nrhs, int parts,
    cf* __restrict__ ys) {
    const int64_t li = (int64_t)blockIdx.x * 4 + (threadIdx.x >> 5);
    if (li >= nleaf) return;
    const int lane = threadIdx.x & 31;
    const AdBox b = boxes[leaves[li]];
    const int tn = b.hi - b.lo;
    const bool nf = (parts & HFMM_PART_NEAR_FREE) != 0, nr = (parts & HFMM_PART_NEAR_REACT) != 0;
    for (int i = lane; i < tn; i += 32)
        for (int r = 0; r < nrhs; ++r) {
            cf acc = cfmk(0.f, 0.f);
            if (nf)
                for (int32_t e = u_beg[li]; e < u_beg[li + 1]; ++e) {
                    const AdBox S = boxes[u_src[e]];
                    const cf* Ge = G + u_blk[e] + i;
                    for (int32_t j = 0; j < S.hi - S.lo; ++j)
                        cfma_f(acc, Ge[(int64_t)j * tn], qs[(int64_t)(S.lo + j) * nrhs + r]);
                }
            if (nr)
                for (int32_t e = d_beg[li]; e < d_beg[li + 1]; ++e) {
                    const AdBox S = boxes[d_src[e]];
                    const int sn = S.hi - S.lo;
                    const cf* Gr = dvals + d_blk[e] + (int64_t)i * sn;
                    for (int j = 0; j < sn; ++j) cfma_f(acc, Gr[j], qs[(int64_t)(S.lo + j) * nrhs + r]);
                }
            cf* yy = ys + (int64_t)(b.lo + i) * nrhs + r;
            *yy = cfmk(yy->x + acc.x, yy->y + acc.y);
        }
}

int ad_chunk(int pmax, int cap) {
    // (2p + 1) basis values + (p + 1) scratch values of 16 bytes per point in ~45 KB
    const int per = (2 * pmax + 1) * (int)sizeof(cd) + (pmax + 1) * (int)sizeof(cd);
    return std::max(1, std::min(cap, 45000 / per));
}

// CTAs per box for a level of nbox boxes with `items` outputs each (see the
// uniform FP64 kernels): spread levels with few boxes over the GPU.
unsigned ad_split(int64_t nbox, int items) {
    if (nbox >= 2048) return 1;
    const int64_t by_items = (items + AD_TB - 1) / AD_TB;
    const int64_t by_grid = (2048 + nbox - 1) / nbox;
    return (unsigned)std::max<int64_t>(1, std::min(by_items, by_grid));
}

size_t ad_smem(int chunk, int pmax) {
    return (size_t)chunk * ((2 * pmax + 1) + (pmax + 1)) * sizeof(cd);
}

uint64_t ad_key(int level, int ix, int iy) {
    return ((uint64_t)level << 42) | ((uint64_t)(uint32_t)ix << 21) | (uint64_t)(uint32_t)iy;
}

bool ad_adjacent(const AdBox& A, const AdBox& B) {
    const int l = std::max(A.level, B.level);
    const int sa = l - A.level, sb = l - B.level;
    const int64_t ax0 = (int64_t)A.ix << sa, ax1 = (int64_t)(A.ix + 1) << sa;
    const int64_t ay0 = (int64_t)A.iy << sa, ay1 = (int64_t)(A.iy + 1) << sa;
    const int64_t bx0 = (int64_t)B.ix << sb, bx1 = (int64_t)(B.ix + 1) << sb;
    const int64_t by0 = (int64_t)B.iy << sb, by1 = (int64_t)(B.iy + 1) << sb;
    return ax0 <= bx1 && bx0 <= ax1 && ay0 <= by1 && by0 <= ay1;
}

uint64_t morton16(uint32_t x, uint32_t y) {
    uint64_t k = 0;
    for (int i = 0; i < AD_MAX_LEVEL; ++i) {
        k |= (uint64_t)((x >> i) & 1u) << (2 * i);
        k |= (uint64_t)((y >> i) & 1u) << (2 * i + 1);
    }
    return k;
}

}  // namespace

// Host-side tree, lists and their device copies.
struct AdaptiveTree {
    std::vector<AdBox> boxes;                 // by level, then Morton order within the level
    std::vector<int64_t> lev_off;             // first box of each level, [L + 2]
    std::vector<int32_t> leaves;              // leaf box indices (box order)
    std::unordered_map<uint64_t, int32_t> index;
    // CSR lists: V and R over boxes (sources as index within the level), X over
    // boxes (source leaf boxes), W, U and direct over leaves (source boxes)
    std::vector<int32_t> v_beg, v_src, v_off, r_beg, r_src, r_tab, x_beg, x_src;
    std::vector<int32_t> w_beg, w_src, u_beg, u_src, d_beg, d_src;
    std::vector<int64_t> d_blk;
    std::vector<std::pair<int32_t, int32_t>> r_pairs_box, direct_pairs_box;   // (target, source) boxes
    int lup = 0;                              // coarsest level of the upward pass
    int pmax = 0;                             // largest order of any level
    int pmax_leaf = 0;                        // largest order of a leaf's level or a W box's level
    std::vector<int64_t> u_blk;               // offset of each U pair's H0 block
    cd* near_G = nullptr;                     // plan-time H0 blocks (null above the budget)
    int64_t* du_blk = nullptr;
    // mixed precision: plan-time FP32 bases (P2M / L2P per leaf point, M2P per W
    // pair and point, P2L per X pair and point) with their offsets, FP32 H0 blocks
    cf *basis32 = nullptr, *m2p32 = nullptr, *p2l32 = nullptr, *near_G32 = nullptr;
    int64_t *d_boff = nullptr, *d_wboff = nullptr, *d_xboff = nullptr;
    int32_t* d_p2m_li = nullptr;              // leaf ordinals of the P2M list
    // device
    AdBox* d_boxes = nullptr;
    int32_t *dv_beg = nullptr, *dv_src = nullptr, *dv_off = nullptr, *dr_beg = nullptr, *dr_src = nullptr,
            *dr_tab = nullptr, *dx_beg = nullptr, *dx_src = nullptr, *dw_beg = nullptr, *dw_src = nullptr,
            *du_beg = nullptr, *du_src = nullptr, *dd_beg = nullptr, *dd_src = nullptr, *d_leaves = nullptr,
            *d_p2m = nullptr;
    int64_t n_p2m = 0;
    int64_t* dd_blk = nullptr;
};

void adaptive_destroy(AdaptiveTree* T) { delete T; }

namespace {

template <class V>
hfmm_status ad_upload(hfmm_plan_s* P, const std::vector<V>& h, V** d, cudaStream_t st) {
    HFMM_TRY(plan_alloc(P, (void**)d, sizeof(V) * std::max<size_t>(h.size(), 1)));
    if (!h.empty()) HFMM_CUDA_TRY(cudaMemcpyAsync(*d, h.data(), sizeof(V) * h.size(), cudaMemcpyHostToDevice, st));
    return HFMM_OK;
}

}  // namespace

// Tree of the points (host), sorted points and permutation (device).
hfmm_status build_adaptive_tree(hfmm_plan_s* P, const double* d_xy, int leaf_size, cudaStream_t st) {
    const int64_t n = P->n;
    std::vector<double> xy((size_t)2 * n);
    HFMM_CUDA_TRY(cudaMemcpyAsync(xy.data(), d_xy, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost, st));
    HFMM_CUDA_TRY(cudaStreamSynchronize(st));
    double xmin = INFINITY, ymin = INFINITY, xmax = -INFINITY, ymax = -INFINITY;
    for (int64_t i = 0; i < n; ++i) {
        const double x = xy[2 * i], y = xy[2 * i + 1];
        if (!std::isfinite(x) || !std::isfinite(y)) { hfmm_set_error("point %lld is not finite", (long long)i); return HFMM_ERR_INVALID_ARG; }
        if (!(y > 0.0)) { hfmm_set_error("point %lld has y <= 0 (sources must lie in the top layer)", (long long)i); return HFMM_ERR_INVALID_ARG; }
        xmin = std::min(xmin, x); ymin = std::min(ymin, y);
        xmax = std::max(xmax, x); ymax = std::max(ymax, y);
    }
    double S = std::max(xmax - xmin, ymax - ymin);
    if (!(S > 0.0)) S = 1.0;
    P->x0 = xmin;
    P->y0 = ymin;
    P->S = S;
    const int D = AD_MAX_LEVEL;
    const int64_t m = (int64_t)1 << D;
    const double scale = (double)m / S;
    std::vector<uint32_t> qx(n), qy(n);
    std::vector<uint64_t> key(n);
    for (int64_t i = 0; i < n; ++i) {
        qx[i] = (uint32_t)std::min<double>(std::floor((xy[2 * i] - xmin) * scale), (double)(m - 1));
        qy[i] = (uint32_t)std::min<double>(std::floor((xy[2 * i + 1] - ymin) * scale), (double)(m - 1));
        key[i] = morton16(qx[i], qy[i]);
    }
    std::vector<int64_t> perm(n);
    std::iota(perm.begin(), perm.end(), 0);
    std::stable_sort(perm.begin(), perm.end(), [&](int64_t a, int64_t b) { return key[a] < key[b]; });
    std::vector<uint64_t> skey(n);
    std::vector<double2> xs(n);
    for (int64_t i = 0; i < n; ++i) {
        skey[i] = key[perm[i]];
        xs[i] = make_double2(xy[2 * perm[i]], xy[2 * perm[i] + 1]);
    }
    // boxes, breadth first: each level's boxes in Morton order
    AdaptiveTree* T = new (std::nothrow) AdaptiveTree();
    if (!T) { hfmm_set_error("host allocation failed"); return HFMM_ERR_OOM; }
    P->ad = T;
    AdBox root{0, 0, 0, 0, (int32_t)n, -1, 1, 0, {-1, -1, -1, -1}};
    T->boxes.push_back(root);
    T->lev_off.push_back(0);
    int64_t lbeg = 0, lend = 1;
    int level = 0;
    while (lbeg < lend) {
        T->lev_off.push_back(lend);   // provisional end of this level
        for (int64_t bi = lbeg; bi < lend; ++bi) {
            T->boxes[bi].lidx = (int32_t)(bi - lbeg);
            const AdBox b = T->boxes[bi];   // a copy: children are appended below
            if (b.hi - b.lo <= leaf_size || level >= D) continue;
            // children by the two key bits of level + 1
            const int sh = 2 * (D - level - 1);
            int32_t lo = b.lo;
            for (int c = 0; c < 4; ++c) {
                int32_t hi = lo;
                while (hi < b.hi && (int)((skey[hi] >> sh) & 3u) == c) ++hi;
                if (hi > lo) {
                    AdBox ch{level + 1, 2 * b.ix + (c & 1), 2 * b.iy + (c >> 1), lo, hi, (int32_t)bi, 1, 0,
                             {-1, -1, -1, -1}};
                    T->boxes[bi].child[c] = (int32_t)T->boxes.size();
                    T->boxes[bi].leaf = 0;
                    T->boxes.push_back(ch);
                }
                lo = hi;
            }
        }
        lbeg = lend;
        lend = (int64_t)T->boxes.size();
        if (lbeg < lend) ++level;
    }
    T->lev_off.resize(level + 2);
    T->lev_off[level + 1] = (int64_t)T->boxes.size();
    P->L = level;
    for (size_t i = 0; i < T->boxes.size(); ++i) {
        const AdBox& b = T->boxes[i];
        T->index[ad_key(b.level, b.ix, b.iy)] = (int32_t)i;
        if (b.leaf) T->leaves.push_back((int32_t)i);
    }
    HFMM_TRY(plan_alloc(P, (void**)&P->xy_sorted, sizeof(double2) * n));
    HFMM_TRY(plan_alloc(P, (void**)&P->perm, sizeof(int64_t) * n));
    HFMM_CUDA_TRY(cudaMemcpyAsync(P->xy_sorted, xs.data(), sizeof(double2) * n, cudaMemcpyHostToDevice, st));
    HFMM_CUDA_TRY(cudaMemcpyAsync(P->perm, perm.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice, st));
    HFMM_CUDA_TRY(cudaStreamSynchronize(st));
    return HFMM_OK;
}

// Lists (host) and their device copies; per-level box counts and pair counts.
hfmm_status build_adaptive_lists(hfmm_plan_s* P, cudaStream_t st) {
    AdaptiveTree* T = P->ad;
    const int L = P->L;
    auto& bx = T->boxes;
    const int64_t nb = (int64_t)bx.size();
    auto find = [&](int l, int ix, int iy) -> int32_t {
        if (ix < 0 || iy < 0 || ix >= (1 << l) || iy >= (1 << l)) return -1;
        auto it = T->index.find(ad_key(l, ix, iy));
        return it == T->index.end() ? -1 : it->second;
    };
    auto colleagues = [&](int32_t b, std::vector<int32_t>& out) {
        out.clear();
        const AdBox& B = bx[b];
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const int32_t c = find(B.level, B.ix + dx, B.iy + dy);
                if (c >= 0) out.push_back(c);
            }
    };
    std::vector<std::vector<int32_t>> V(nb), X(nb), R(nb), Rt(nb);
    std::vector<int32_t> col, stack;
    // V lists (level >= 2)
    for (int32_t b = 0; b < nb; ++b) {
        const AdBox& B = bx[b];
        if (B.level < 2) continue;
        colleagues(B.parent, col);
        for (int32_t c : col)
            for (int a = 0; a < 4; ++a) {
                const int32_t d = bx[c].child[a];
                if (d >= 0 && !ad_adjacent(bx[d], B)) V[b].push_back(d);
            }
        std::sort(V[b].begin(), V[b].end());
    }
    // U and W lists of the leaves; X by inverting W
    const int64_t nl = (int64_t)T->leaves.size();
    std::vector<std::vector<int32_t>> U(nl), Wl(nl), Dl(nl);
    for (int64_t li = 0; li < nl; ++li) {
        const int32_t b = T->leaves[li];
        const AdBox& B = bx[b];
        stack.assign(1, 0);
        while (!stack.empty()) {
            const int32_t c = stack.back();
            stack.pop_back();
            if (!ad_adjacent(bx[c], B)) continue;
            if (bx[c].leaf) U[li].push_back(c);
            else
                for (int a = 0; a < 4; ++a)
                    if (bx[c].child[a] >= 0) stack.push_back(bx[c].child[a]);
        }
        std::sort(U[li].begin(), U[li].end());
        colleagues(b, col);
        stack.clear();
        for (int32_t c : col)
            if (c != b)
                for (int a = 0; a < 4; ++a)
                    if (bx[c].child[a] >= 0) stack.push_back(bx[c].child[a]);
        while (!stack.empty()) {
            const int32_t d = stack.back();
            stack.pop_back();
            if (ad_adjacent(bx[d], B)) {
                for (int a = 0; a < 4; ++a)
                    if (bx[d].child[a] >= 0) stack.push_back(bx[d].child[a]);
            } else {
                Wl[li].push_back(d);
                X[d].push_back(b);
            }
        }
        std::sort(Wl[li].begin(), Wl[li].end());
    }
    for (auto& x : X) std::sort(x.begin(), x.end());
    // reaction pairs from (root, root)
    std::vector<std::pair<int32_t, int32_t>> pst(1, {0, 0});
    while (!pst.empty()) {
        const auto pr = pst.back();
        pst.pop_back();
        const AdBox& A = bx[pr.first];
        const AdBox& S = bx[pr.second];
        const int l = A.level;
        if (reaction_admissible(A.iy, S.iy, P->y0, P->S / (double)(1 << l))) {
            R[pr.first].push_back(pr.second);
            T->r_pairs_box.push_back(pr);
        } else if (A.leaf || S.leaf) {
            T->direct_pairs_box.push_back(pr);
        } else {
            for (int a = 0; a < 4; ++a)
                for (int c = 0; c < 4; ++c)
                    if (A.child[a] >= 0 && S.child[c] >= 0) pst.push_back({A.child[a], S.child[c]});
        }
    }
    for (auto& r : R) std::sort(r.begin(), r.end());
    // direct pairs over the leaf pairs below them
    std::vector<int32_t> leaf_ord(nb, -1);
    for (int64_t li = 0; li < nl; ++li) leaf_ord[T->leaves[li]] = (int32_t)li;
    auto leaves_below = [&](int32_t b, std::vector<int32_t>& out) {
        out.clear();
        std::vector<int32_t> s2(1, b);
        while (!s2.empty()) {
            const int32_t c = s2.back();
            s2.pop_back();
            if (bx[c].leaf) out.push_back(c);
            else
                for (int a = 0; a < 4; ++a)
                    if (bx[c].child[a] >= 0) s2.push_back(bx[c].child[a]);
        }
    };
    struct DPair { int32_t t, s; double xmax, h; };
    std::vector<std::vector<DPair>> DP(nl);
    std::vector<int32_t> lt, ls;
    for (const auto& pr : T->direct_pairs_box) {
        const AdBox& A = bx[pr.first];
        const AdBox& S = bx[pr.second];
        const double h = P->S / (double)(1 << A.level);
        const double xm = (std::abs(A.ix - S.ix) + 1) * h;
        leaves_below(pr.first, lt);
        leaves_below(pr.second, ls);
        for (int32_t a : lt)
            for (int32_t c : ls) DP[leaf_ord[a]].push_back({a, c, xm, h});
    }
    // CSR and per-level counts
    auto csr = [](const std::vector<std::vector<int32_t>>& lists, std::vector<int32_t>& beg, std::vector<int32_t>& src) {
        beg.assign(lists.size() + 1, 0);
        for (size_t i = 0; i < lists.size(); ++i) beg[i + 1] = beg[i] + (int32_t)lists[i].size();
        src.clear();
        src.reserve(beg.back());
        for (const auto& v : lists) src.insert(src.end(), v.begin(), v.end());
    };
    csr(V, T->v_beg, T->v_src);
    csr(R, T->r_beg, T->r_src);
    csr(X, T->x_beg, T->x_src);
    csr(U, T->u_beg, T->u_src);
    csr(Wl, T->w_beg, T->w_src);
    T->v_off.resize(T->v_src.size());
    T->r_tab.resize(T->r_src.size());
    for (int32_t b = 0; b < nb; ++b) {
        const AdBox& B = bx[b];
        for (int32_t e = T->v_beg[b]; e < T->v_beg[b + 1]; ++e) {
            const AdBox& S = bx[T->v_src[e]];
            T->v_off[e] = (B.ix - S.ix + 3) * 7 + (B.iy - S.iy + 3);
            T->v_src[e] = S.lidx;
        }
        const int dxmax = B.level == 0 ? 0 : (1 << B.level) - 1;
        for (int32_t e = T->r_beg[b]; e < T->r_beg[b + 1]; ++e) {
            const AdBox& S = bx[T->r_src[e]];
            T->r_tab[e] = (B.ix - S.ix + dxmax) * 3 + (B.iy + S.iy);
            T->r_src[e] = S.lidx;
        }
    }
    T->d_beg.assign(nl + 1, 0);
    std::vector<DirectSpec> specs;
    for (int64_t li = 0; li < nl; ++li) {
        T->d_beg[li + 1] = T->d_beg[li] + (int32_t)DP[li].size();
        for (const DPair& d : DP[li]) {
            T->d_src.push_back(d.s);
            const AdBox& A = bx[d.t];
            const AdBox& S = bx[d.s];
            specs.push_back({A.lo, A.hi - A.lo, S.lo, S.hi - S.lo, d.xmax, 2.0 * P->y0, 2.0 * P->y0 + 2.0 * d.h});
        }
    }
    // levels: box counts, pair counts (the tables are built for the levels
    // with reaction pairs), the coarsest levels of the passes
    int lmin = L, lup = L;
    for (int l = 0; l <= L; ++l) {
        LevelInfo& lv = P->lev[l];
        lv.nbox = T->lev_off[l + 1] - T->lev_off[l];
        lv.nv = T->v_beg[T->lev_off[l + 1]] - T->v_beg[T->lev_off[l]];
        lv.nr = T->r_beg[T->lev_off[l + 1]] - T->r_beg[T->lev_off[l]];
        const int64_t nx = T->x_beg[T->lev_off[l + 1]] - T->x_beg[T->lev_off[l]];
        if (lv.nv + lv.nr + nx > 0) lmin = std::min(lmin, l);
    }
    lup = lmin;
    for (int32_t d : T->w_src) lup = std::min(lup, (int)bx[d].level);
    P->lmin = lup;   // tables and buffers from the upward pass's coarsest level
    T->lup = lup;
    int lstar = L + 1;
    for (int l = 0; l <= L; ++l)
        if (2.0 * P->y0 >= P->S / (double)(1 << l)) { lstar = l; break; }
    P->lstar = lstar;
    for (int l = 0; l <= L; ++l) T->pmax = std::max(T->pmax, P->lev[l].p);
    for (int32_t b : T->leaves) T->pmax_leaf = std::max(T->pmax_leaf, P->lev[bx[b].level].p);
    for (int32_t d : T->w_src) T->pmax_leaf = std::max(T->pmax_leaf, P->lev[bx[d].level].p);
    // leaves needing P2M: those of levels >= lup
    std::vector<int32_t> p2m;
    for (int32_t b : T->leaves)
        if (bx[b].level >= lup) p2m.push_back(b);
    T->n_p2m = (int64_t)p2m.size();
    int64_t up = 0, pp = 0;
    for (int64_t li = 0; li < nl; ++li) {
        const AdBox& B = bx[T->leaves[li]];
        for (int32_t e = T->u_beg[li]; e < T->u_beg[li + 1]; ++e) {
            ++up;
            pp += (int64_t)(B.hi - B.lo) * (bx[T->u_src[e]].hi - bx[T->u_src[e]].lo);
        }
    }
    P->u_pairs = up;
    P->p2p_point_pairs = pp;
    // offsets of the U pairs' H0 blocks (n_T x n_S each, source-major)
    T->u_blk.assign(T->u_src.size(), 0);
    {
        int64_t o = 0;
        for (int64_t li = 0; li < nl; ++li) {
            const AdBox& B = bx[T->leaves[li]];
            for (int32_t e = T->u_beg[li]; e < T->u_beg[li + 1]; ++e) {
                T->u_blk[e] = o;
                o += (int64_t)(B.hi - B.lo) * (bx[T->u_src[e]].hi - bx[T->u_src[e]].lo);
            }
        }
    }
    P->nd = (int64_t)T->d_src.size();
    // every index the kernels follow stays inside its array (checked before any upload)
    {
        bool ok = true;
        for (int32_t b = 0; b < nb && ok; ++b) {
            const AdBox& B = bx[b];
            const int64_t nbl = T->lev_off[B.level + 1] - T->lev_off[B.level];
            const int dxmax = B.level == 0 ? 0 : (1 << B.level) - 1;
            ok = B.lo >= 0 && B.hi <= P->n && B.lo < B.hi && B.lidx >= 0 && B.lidx < nbl &&
                 (B.parent < 0 ? b == 0 : B.parent < nb);
            for (int a = 0; a < 4; ++a) ok = ok && B.child[a] < nb;
            for (int32_t e = T->v_beg[b]; e < T->v_beg[b + 1] && ok; ++e)
                ok = T->v_src[e] >= 0 && T->v_src[e] < nbl && T->v_off[e] >= 0 && T->v_off[e] < 49;
            for (int32_t e = T->r_beg[b]; e < T->r_beg[b + 1] && ok; ++e)
                ok = T->r_src[e] >= 0 && T->r_src[e] < nbl && T->r_tab[e] >= 0 && T->r_tab[e] < (2 * dxmax + 1) * 3;
            for (int32_t e = T->x_beg[b]; e < T->x_beg[b + 1] && ok; ++e)
                ok = T->x_src[e] >= 0 && T->x_src[e] < nb && bx[T->x_src[e]].leaf;
        }
        for (int32_t v : T->w_src) ok = ok && v >= 0 && v < nb && bx[v].level >= lup;
        for (int32_t v : T->u_src) ok = ok && v >= 0 && v < nb && bx[v].leaf;
        for (int32_t v : T->d_src) ok = ok && v >= 0 && v < nb && bx[v].leaf;
        for (int32_t v : p2m) ok = ok && bx[v].level >= lup;
        if (!ok) {
            hfmm_set_error("adaptive tree: internal list check failed");
            return HFMM_ERR_CUDA;
        }
    }
    // device copies
    HFMM_TRY(ad_upload(P, bx, &T->d_boxes, st));
    HFMM_TRY(ad_upload(P, T->leaves, &T->d_leaves, st));
    HFMM_TRY(ad_upload(P, p2m, &T->d_p2m, st));
    HFMM_TRY(ad_upload(P, T->v_beg, &T->dv_beg, st));
    HFMM_TRY(ad_upload(P, T->v_src, &T->dv_src, st));
    HFMM_TRY(ad_upload(P, T->v_off, &T->dv_off, st));
    HFMM_TRY(ad_upload(P, T->r_beg, &T->dr_beg, st));
    HFMM_TRY(ad_upload(P, T->r_src, &T->dr_src, st));
    HFMM_TRY(ad_upload(P, T->r_tab, &T->dr_tab, st));
    HFMM_TRY(ad_upload(P, T->x_beg, &T->dx_beg, st));
    HFMM_TRY(ad_upload(P, T->x_src, &T->dx_src, st));
    HFMM_TRY(ad_upload(P, T->w_beg, &T->dw_beg, st));
    HFMM_TRY(ad_upload(P, T->w_src, &T->dw_src, st));
    HFMM_TRY(ad_upload(P, T->u_beg, &T->du_beg, st));
    HFMM_TRY(ad_upload(P, T->u_src, &T->du_src, st));
    HFMM_TRY(ad_upload(P, T->d_beg, &T->dd_beg, st));
    HFMM_TRY(ad_upload(P, T->d_src, &T->dd_src, st));
    HFMM_TRY(ad_upload(P, T->u_blk, &T->du_blk, st));
    // the near field's (i/4) H0 blocks, computed once (within the same budget as
    // the uniform tree's FP64 blocks)
    if (P->precision == HFMM_FP64 && 16.0 * (double)pp <= NEAR64_MAX_BYTES && pp > 0) {
        HFMM_TRY(plan_alloc(P, (void**)&T->near_G, sizeof(cd) * (size_t)pp));
        ad_near_fill_kernel<<<(unsigned)nl, 128, 0, st>>>(T->d_boxes, T->d_leaves, T->du_beg, T->du_src, T->du_blk,
                                                          P->xy_sorted, P->k, T->near_G);
        HFMM_CUDA_TRY(cudaGetLastError());
        P->table_bytes += 16.0 * (double)pp;
    }
    // the specs are kept for the table stage (direct blocks need the sorted points)
    T->d_blk.clear();
    if (!specs.empty()) {
        // checked against their node-doubled rule with the other tables (build_tables)
        HFMM_TRY(build_direct_blocks(P, specs, T->d_blk, st));
    } else {
        P->nd_vals = 0;
        HFMM_TRY(plan_alloc(P, (void**)&P->d_vals, sizeof(cd)));
    }
    HFMM_TRY(ad_upload(P, T->d_blk, &T->dd_blk, st));
    HFMM_CUDA_TRY(cudaStreamSynchronize(st));
    return HFMM_OK;
}

// The adaptive apply between the gather and the scatter (FP64).
hfmm_status apply_adaptive(hfmm_plan_s* P, int nrhs, int parts, cudaStream_t st) {
    AdaptiveTree* T = P->ad;
    const int L = P->L;
    const int64_t n = P->n;
    StageTimer tm{P, st};
    AdLevels lv{};
    for (int l = 0; l <= L; ++l) {
        lv.mult[l] = P->lev[l].mult;
        lv.loc[l] = P->lev[l].loc;
        lv.p[l] = P->lev[l].p;
        lv.h[l] = P->lev[l].h;
    }
    const int chunk = ad_chunk(T->pmax, 32);             // P2L passes in the downward kernel
    const size_t sm = ad_smem(chunk, T->pmax);
    const int lchunk = ad_chunk(T->pmax_leaf, 32);       // the warp-per-leaf kernels
    const size_t lsm = ad_smem(lchunk, T->pmax_leaf);
    const double MAC = 8.0 * nrhs;
    const bool far = (parts & (HFMM_PART_FAR_FREE | HFMM_PART_FAR_REACT)) != 0;
    const int lmin = T->lup;
    if (far) {
        tm.begin(HFMM_STAGE_P2M);
        if (T->n_p2m > 0) {
            ad_p2m_kernel<<<(unsigned)T->n_p2m, 32, lsm, st>>>(T->d_boxes, T->d_p2m, P->xy_sorted, P->q_sorted, n,
                                                              nrhs, P->x0, P->y0, P->k, lv, lchunk);
            ++P->launches;
            HFMM_CUDA_TRY(cudaGetLastError());
        }
        tm.end(HFMM_STAGE_P2M);
        tm.begin(HFMM_STAGE_M2M);
        for (int l = L - 1; l >= lmin; --l) {
            const LevelInfo& v = P->lev[l];
            ad_m2m_kernel<<<dim3((unsigned)v.nbox, ad_split(v.nbox, nrhs * v.ncoef)), AD_TB, 0, st>>>(
                T->d_boxes, T->lev_off[l], l, v.t_m2m, lv, nrhs);
            ++P->launches;
            HFMM_CUDA_TRY(cudaGetLastError());
            P->st_flops[HFMM_STAGE_M2M] += MAC * 4.0 * v.nbox * v.ncoef * P->lev[l + 1].ncoef;
        }
        tm.end(HFMM_STAGE_M2M);
        tm.begin(HFMM_STAGE_DOWN);
        for (int l = lmin; l <= L; ++l) {
            const LevelInfo& v = P->lev[l];
            ad_down_kernel<<<dim3((unsigned)v.nbox, ad_split(v.nbox, nrhs * v.ncoef)), AD_TB, sm, st>>>(
                T->d_boxes, T->lev_off[l], l, lmin, nrhs, lv, l > lmin ? P->lev[l - 1].t_l2l : nullptr, T->dv_beg,
                T->dv_src, T->dv_off, v.t_free, T->dr_beg, T->dr_src, T->dr_tab, v.t_react, T->dx_beg, T->dx_src,
                P->xy_sorted, P->q_sorted, n, P->x0, P->y0, P->k, parts, chunk);
            ++P->launches;
            HFMM_CUDA_TRY(cudaGetLastError());
            double pairs = 0.0;
            if (parts & HFMM_PART_FAR_FREE) pairs += (double)v.nv;
            if (parts & HFMM_PART_FAR_REACT) pairs += (double)v.nr;
            P->st_flops[HFMM_STAGE_DOWN] += MAC * pairs * v.ncoef * v.ncoef;
        }
        tm.end(HFMM_STAGE_DOWN);
        tm.begin(HFMM_STAGE_L2P);
        ad_leaf_far_kernel<<<(unsigned)T->leaves.size(), 32, lsm, st>>>(
            T->d_boxes, T->d_leaves, T->dw_beg, T->dw_src, P->xy_sorted, n, nrhs, P->x0, P->y0, P->k, lv, lmin, parts,
            lchunk, P->y_sorted);
        ++P->launches;
        HFMM_CUDA_TRY(cudaGetLastError());
        tm.end(HFMM_STAGE_L2P);
    }
    if (parts & (HFMM_PART_NEAR_FREE | HFMM_PART_NEAR_REACT)) {
        tm.begin(HFMM_STAGE_P2P);
        const int64_t nleaf = (int64_t)T->leaves.size();
        ad_near_kernel<<<(unsigned)ceil_div(nleaf, 4), 128, 0, st>>>(
            T->d_boxes, T->d_leaves, nleaf, T->du_beg, T->du_src, T->du_blk, T->near_G, T->dd_beg, T->dd_src, T->dd_blk,
            P->d_vals, P->xy_sorted, P->q_sorted, n, nrhs, P->k, parts, P->y_sorted);
        ++P->launches;
        HFMM_CUDA_TRY(cudaGetLastError());
        tm.end(HFMM_STAGE_P2P);
        P->st_flops[HFMM_STAGE_P2P] = MAC * (double)P->p2p_point_pairs;
        P->st_flops[HFMM_STAGE_DIRECT] = MAC * (double)P->nd_vals;
    }
    return HFMM_OK;
}

namespace {

__global__ void ad_iperm_kernel(const int64_t* __restrict__ perm, int64_t n, int32_t* __restrict__ iperm) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) iperm[perm[i]] = (int32_t)i;
}

}  // namespace

// Mixed-precision state of an adaptive plan (after build_tables32): the
// inverse permutation, the plan-time FP32 bases and FP32 near-field blocks.
hfmm_status build_adaptive32(hfmm_plan_s* P, cudaStream_t st) {
    AdaptiveTree* T = P->ad;
    const auto& bx = T->boxes;
    const int64_t nl = (int64_t)T->leaves.size();
    const int lup = T->lup;
    HFMM_TRY(plan_alloc(P, (void**)&P->iperm32, sizeof(int32_t) * P->n));
    ad_iperm_kernel<<<(unsigned)ceil_div(P->n, 256), 256, 0, st>>>(P->perm, P->n, P->iperm32);
    HFMM_CUDA_TRY(cudaGetLastError());
    AdLevels lv{};
    std::vector<const double*> lsp(AD_MAX_LEVEL + 1, nullptr);
    for (int l = 0; l <= P->L; ++l) {
        lv.p[l] = P->lev[l].p;
        lv.h[l] = P->lev[l].h;
        lsp[l] = P->lev[l].d_log_s;
    }
    const double** d_lsp = nullptr;
    HFMM_TRY(ad_upload(P, lsp, &d_lsp, st));
    auto nc = [&](int l) { return (int64_t)(2 * P->lev[l].p + 1); };
    // P2M / L2P bases of the leaves at levels >= lup
    std::vector<int64_t> boff(nl, 0), wboff(T->w_src.size(), 0), xboff(T->x_src.size(), 0);
    std::vector<int32_t> p2m_li;
    int64_t nb = 0;
    for (int64_t li = 0; li < nl; ++li) {
        const AdBox& B = bx[T->leaves[li]];
        boff[li] = nb;
        if (B.level >= lup) {
            nb += (int64_t)(B.hi - B.lo) * nc(B.level);
            p2m_li.push_back((int32_t)li);
        }
    }
    std::vector<int32_t> w_tgt(T->w_src.size()), x_tgt(T->x_src.size());
    int64_t nw = 0;
    for (int64_t li = 0; li < nl; ++li) {
        const AdBox& B = bx[T->leaves[li]];
        for (int32_t e = T->w_beg[li]; e < T->w_beg[li + 1]; ++e) {
            w_tgt[e] = T->leaves[li];
            wboff[e] = nw;
            nw += (int64_t)(B.hi - B.lo) * nc(bx[T->w_src[e]].level);
        }
    }
    int64_t nx = 0;
    for (size_t b = 0; b < bx.size(); ++b)
        for (int32_t e = T->x_beg[b]; e < T->x_beg[b + 1]; ++e) {
            x_tgt[e] = (int32_t)b;
            xboff[e] = nx;
            const AdBox& C = bx[T->x_src[e]];
            nx += (int64_t)(C.hi - C.lo) * nc(bx[b].level);
        }
    HFMM_TRY(ad_upload(P, boff, &T->d_boff, st));
    HFMM_TRY(ad_upload(P, wboff, &T->d_wboff, st));
    HFMM_TRY(ad_upload(P, xboff, &T->d_xboff, st));
    HFMM_TRY(ad_upload(P, p2m_li, &T->d_p2m_li, st));
    int32_t *d_wt = nullptr, *d_xt = nullptr;
    HFMM_TRY(ad_upload(P, w_tgt, &d_wt, st));
    HFMM_TRY(ad_upload(P, x_tgt, &d_xt, st));
    HFMM_TRY(plan_alloc(P, (void**)&T->basis32, sizeof(cf) * std::max<int64_t>(nb, 1)));
    HFMM_TRY(plan_alloc(P, (void**)&T->m2p32, sizeof(cf) * std::max<int64_t>(nw, 1)));
    HFMM_TRY(plan_alloc(P, (void**)&T->p2l32, sizeof(cf) * std::max<int64_t>(nx, 1)));
    P->buffer_bytes += sizeof(cf) * (double)(nb + nw + nx);
    const int pm = T->pmax;
    const int thr = std::max(1, std::min(128, 6000 / (pm + 1)));
    if (nl > 0) {
        ad32_basis_p2m_kernel<<<(unsigned)nl, thr, (size_t)thr * (pm + 1) * sizeof(double), st>>>(
            T->d_boxes, T->d_leaves, T->d_boff, lup, P->xy_sorted, P->x0, P->y0, P->k, lv, d_lsp, T->basis32);
        HFMM_CUDA_TRY(cudaGetLastError());
    }
    const int thr2 = std::max(1, std::min(128, 3000 / (pm + 1)));
    if (!T->w_src.empty()) {
        ad32_basis_pair_kernel<<<(unsigned)T->w_src.size(), thr2, (size_t)thr2 * (pm + 1) * sizeof(cd), st>>>(
            T->d_boxes, d_wt, T->dw_src, T->d_wboff, true, P->xy_sorted, P->x0, P->y0, P->k, lv, d_lsp, T->m2p32);
        HFMM_CUDA_TRY(cudaGetLastError());
    }
    if (!T->x_src.empty()) {
        ad32_basis_pair_kernel<<<(unsigned)T->x_src.size(), thr2, (size_t)thr2 * (pm + 1) * sizeof(cd), st>>>(
            T->d_boxes, d_xt, T->dx_src, T->d_xboff, false, P->xy_sorted, P->x0, P->y0, P->k, lv, d_lsp, T->p2l32);
        HFMM_CUDA_TRY(cudaGetLastError());
    }
    // FP32 near-field blocks
    const double pp = (double)P->p2p_point_pairs;
    if (pp > 0 && 8.0 * pp <= NEAR64_MAX_BYTES) {
        HFMM_TRY(plan_alloc(P, (void**)&T->near_G32, sizeof(cf) * (size_t)P->p2p_point_pairs));
        ad32_near_fill_kernel<<<(unsigned)nl, 128, 0, st>>>(T->d_boxes, T->d_leaves, T->du_beg, T->du_src, T->du_blk,
                                                            P->xy_sorted, P->k, T->near_G32);
        HFMM_CUDA_TRY(cudaGetLastError());
        P->table_bytes += 8.0 * pp;
    } else if (pp > 0) {
        hfmm_set_error("adaptive mixed plan: near-field blocks of %.3g GB exceed the budget", 8.0 * pp / 1e9);
        return HFMM_ERR_OOM;
    }
    HFMM_CUDA_TRY(cudaStreamSynchronize(st));
    return HFMM_OK;
}

// The adaptive apply of a mixed plan between its gather and scatter (FP32
// strengths and fields, point-major).
hfmm_status apply_adaptive32(hfmm_plan_s* P, int nrhs, int parts, cudaStream_t st) {
    AdaptiveTree* T = P->ad;
    const int L = P->L;
    StageTimer tm{P, st};
    AdLevels32 lv{};
    for (int l = 0; l <= L; ++l) {
        lv.mult[l] = P->lev[l].mult32;
        lv.loc[l] = P->lev[l].loc32;
        lv.p[l] = P->lev[l].p;
    }
    const double MAC = 8.0 * nrhs;
    const int lmin = T->lup;
    const int64_t nl = (int64_t)T->leaves.size();
    const bool far = (parts & (HFMM_PART_FAR_FREE | HFMM_PART_FAR_REACT)) != 0;
    if (far) {
        tm.begin(HFMM_STAGE_P2M);
        if (T->n_p2m > 0) {
            ad32_p2m_kernel<<<(unsigned)T->n_p2m, 32, 0, st>>>(T->d_boxes, T->d_leaves, T->d_p2m_li, T->d_boff,
                                                               T->basis32, P->q32, nrhs, lv);
            ++P->launches;
            HFMM_CUDA_TRY(cudaGetLastError());
        }
        tm.end(HFMM_STAGE_P2M);
        tm.begin(HFMM_STAGE_M2M);
        for (int l = L - 1; l >= lmin; --l) {
            const LevelInfo& v = P->lev[l];
            ad32_m2m_kernel<<<dim3((unsigned)v.nbox, ad_split(v.nbox, nrhs * v.ncoef)), AD_TB, 0, st>>>(
                T->d_boxes, T->lev_off[l], l, v.t_m2m32, lv, nrhs);
            ++P->launches;
            HFMM_CUDA_TRY(cudaGetLastError());
            P->st_flops[HFMM_STAGE_M2M] += MAC * 4.0 * v.nbox * v.ncoef * P->lev[l + 1].ncoef;
        }
        tm.end(HFMM_STAGE_M2M);
        tm.begin(HFMM_STAGE_DOWN);
        for (int l = lmin; l <= L; ++l) {
            const LevelInfo& v = P->lev[l];
            ad32_down_kernel<<<dim3((unsigned)v.nbox, ad_split(v.nbox, nrhs * v.ncoef)), AD_TB, 0, st>>>(
                T->d_boxes, T->lev_off[l], l, lmin, nrhs, lv, l > lmin ? P->lev[l - 1].t_l2l32 : nullptr, T->dv_beg,
                T->dv_src, T->dv_off, v.t_free32, T->dr_beg, T->dr_src, T->dr_tab, v.t_react32, T->dx_beg, T->dx_src,
                T->d_xboff, T->p2l32, P->q32, parts);
            ++P->launches;
            HFMM_CUDA_TRY(cudaGetLastError());
            double pairs = 0.0;
            if (parts & HFMM_PART_FAR_FREE) pairs += (double)v.nv;
            if (parts & HFMM_PART_FAR_REACT) pairs += (double)v.nr;
            P->st_flops[HFMM_STAGE_DOWN] += MAC * pairs * v.ncoef * v.ncoef;
        }
        tm.end(HFMM_STAGE_DOWN);
        tm.begin(HFMM_STAGE_L2P);
        ad32_leaf_far_kernel<<<(unsigned)nl, 32, 0, st>>>(T->d_boxes, T->d_leaves, T->d_boff, T->basis32, T->dw_beg,
                                                          T->dw_src, T->d_wboff, T->m2p32, nrhs, lv, lmin, parts,
                                                          P->y32);
        ++P->launches;
        HFMM_CUDA_TRY(cudaGetLastError());
        tm.end(HFMM_STAGE_L2P);
    }
    if (parts & (HFMM_PART_NEAR_FREE | HFMM_PART_NEAR_REACT)) {
        tm.begin(HFMM_STAGE_P2P);
        ad32_near_kernel<<<(unsigned)ceil_div(nl, 4), 128, 0, st>>>(
            T->d_boxes, T->d_leaves, nl, T->du_beg, T->du_src, T->du_blk, T->near_G32, T->dd_beg, T->dd_src, T->dd_blk,
            P->d_vals32, P->q32, nrhs, parts, P->y32);
        ++P->launches;
        HFMM_CUDA_TRY(cudaGetLastError());
        tm.end(HFMM_STAGE_P2P);
        P->st_flops[HFMM_STAGE_P2P] = MAC * (double)P->p2p_point_pairs;
        P->st_flops[HFMM_STAGE_DIRECT] = MAC * (double)P->nd_vals;
    }
    return HFMM_OK;
}

// Introspection: boxes (level, ix, iy, first sorted point, end, leaf) and
// list pairs (target box, source box) of kind 0 U, 1 V, 2 W, 3 X, 4 reaction
// M2L, 5 directly summed reaction (box pairs before the expansion to leaves).
hfmm_status adaptive_boxes(const hfmm_plan_s* P, int64_t* count, int32_t* out) {
    const AdaptiveTree* T = P->ad;
    *count = (int64_t)T->boxes.size();
    if (out)
        for (size_t i = 0; i < T->boxes.size(); ++i) {
            const AdBox& b = T->boxes[i];
            int32_t* o = out + 6 * i;
            o[0] = b.level; o[1] = b.ix; o[2] = b.iy; o[3] = b.lo; o[4] = b.hi; o[5] = b.leaf;
        }
    return HFMM_OK;
}

hfmm_status adaptive_pairs(const hfmm_plan_s* P, int kind, int64_t* count, int32_t* out) {
    const AdaptiveTree* T = P->ad;
    std::vector<std::pair<int32_t, int32_t>> pr;
    const auto& bx = T->boxes;
    auto level_box = [&](int l, int32_t lidx) { return (int32_t)(T->lev_off[l] + lidx); };
    switch (kind) {
        case 0:
            for (size_t li = 0; li < T->leaves.size(); ++li)
                for (int32_t e = T->u_beg[li]; e < T->u_beg[li + 1]; ++e) pr.push_back({T->leaves[li], T->u_src[e]});
            break;
        case 1:
            for (size_t b = 0; b < bx.size(); ++b)
                for (int32_t e = T->v_beg[b]; e < T->v_beg[b + 1]; ++e)
                    pr.push_back({(int32_t)b, level_box(bx[b].level, T->v_src[e])});
            break;
        case 2:
            for (size_t li = 0; li < T->leaves.size(); ++li)
                for (int32_t e = T->w_beg[li]; e < T->w_beg[li + 1]; ++e) pr.push_back({T->leaves[li], T->w_src[e]});
            break;
        case 3:
            for (size_t b = 0; b < bx.size(); ++b)
                for (int32_t e = T->x_beg[b]; e < T->x_beg[b + 1]; ++e) pr.push_back({(int32_t)b, T->x_src[e]});
            break;
        case 4: pr = T->r_pairs_box; break;
        case 5: pr = T->direct_pairs_box; break;
        default: hfmm_set_error("unknown list kind %d", kind); return HFMM_ERR_INVALID_ARG;
    }
    *count = (int64_t)pr.size();
    if (out)
        for (size_t i = 0; i < pr.size(); ++i) {
            out[2 * i] = pr[i].first;
            out[2 * i + 1] = pr[i].second;
        }
    return HFMM_OK;
}

int64_t adaptive_count(const hfmm_plan_s* P, int kind) {
    const AdaptiveTree* T = P->ad;
    switch (kind) {
        case 0: return (int64_t)T->leaves.size();
        case 2: return (int64_t)T->w_src.size();
        case 3: return (int64_t)T->x_src.size();
        case 5: return (int64_t)T->direct_pairs_box.size();
        default: return 0;
    }
}
