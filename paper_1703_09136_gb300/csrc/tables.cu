// Plan-time translation tables, FP64 on the GPU (Algorithm 1, step 1:
// "precompute tables"; the paper used Mathematica, here quadrature kernels).
//
//  * free-space M2L:  C_n(D) = H_n(k|D|) e^{i n angle D}, n = -2p .. 2p, for the
//    49 offsets D = (dx, dy) h_l, |dx|, |dy| <= 3 (Graf, Sec. 3.3);
//  * M2M / L2L:       J_n(v) = J_n(k|v|) e^{i n angle v} for the four child
//    offsets v = +-(h_{l+1}/2, h_{l+1}/2);
//  * reaction M2L:    A_n(X, Y) of Eq. (eq:m2loperator) with sigma of the
//    medium (Sec. 5), n = -2p .. 2p, for every (dx, ysum) used by the
//    reaction lists, X = dx h_l, Y = 2 y0 + (ysum + 1) h_l;
//  * direct reaction: G^s(x_i - x_j, y_i + y_j) = (i/4) A_0 per point pair of
//    the leaf pairs whose images are not separated from the target leaf.
//
// Quadrature (written for this library): the propagating part is integrated
// over tau in [0, pi] with composite 16-point Gauss-Legendre panels; the
// evanescent part over t >= 0, where for layered media the path first dips
// below the real axis on [0, tb] (t = u - i c 4 u (tb - u) / tb^2) to pass
// the branch points of s2, s3 and the guided-mode poles on the radiating side,
// then follows the real axis to the point where the integrand envelope
// e^{-tY} ((xi + t)/k1)^nmax / xi has decayed by e^{-38}.
#include <algorithm>
#include <cmath>
#include <vector>

#include "bessel.cuh"
#include "plan.cuh"

namespace {

constexpr int GLN = 16;
// Largest accepted difference between a table and its node-doubled rule
// (weighted as in react_check_kernel).  Converged FP64 rules agree to a few
// 1e-14; the bound sits well above that and ten times below the FP64 path's
// 1e-11 parity bound.
constexpr double TABLE_RTOL = 1e-12;
__constant__ double c_glx[GLN];
__constant__ double c_glw[GLN];
double h_glx[GLN], h_glw[GLN];
bool gl_ready = false;

// Gauss-Legendre nodes on [-1, 1] by Newton's method on P_n.
void gauss_legendre(int n, double* x, double* w) {
    for (int i = 0; i < n; ++i) {
        double z = std::cos(HFMM_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = 0.0;
            for (int j = 1; j <= n; ++j) {
                double p2 = p1;
                p1 = p0;
                p0 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p2) / j;
            }
            dp = n * (z * p0 - p1) / (z * z - 1.0);
            const double dz = p0 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        // derivative at the converged node
        double p0 = 1.0, p1 = 0.0;
        for (int j = 1; j <= n; ++j) {
            double p2 = p1;
            p1 = p0;
            p0 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p2) / j;
        }
        dp = n * (z * p0 - p1) / (z * z - 1.0);
        x[i] = -z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

hfmm_status ensure_gl() {
    if (!gl_ready) {
        gauss_legendre(GLN, h_glx, h_glw);
        gl_ready = true;
    }
    HFMM_CUDA_TRY(cudaMemcpyToSymbol(c_glx, h_glx, sizeof(h_glx)));
    HFMM_CUDA_TRY(cudaMemcpyToSymbol(c_glw, h_glw, sizeof(h_glw)));
    return HFMM_OK;
}

// quadrature segment: kind 0 tau (real panels on [a, b] in [0, pi]), 1 deformed
// t on [a, b] = [0, tb] with depth c, 2 real t on [a, b]
struct Seg {
    double a, b, c, tb;
    int kind, npan;
    int64_t node0;
};

struct Entry {
    double X, Y;
    int nmax;
    int seg0, seg1;
    int64_t nodes;
    int64_t out;      // offset of A_{-nmax} in the output
    int64_t wofs;     // offset of this level's weights w_n in the check's weight array
    int level, dx, ysum;
};

// real t >= 0 where sigma is not analytic (branch points of s_j, k_j > k1;
// guided-mode poles lie below the largest of them)
void singular_t(const hfmm_medium& m, std::vector<double>& out) {
    const double k1 = m.k[0];
    int nl = m.kind == HFMM_TWO_LAYER ? 1 : (m.kind == HFMM_THREE_LAYER ? 2 : 0);
    for (int j = 1; j <= nl; ++j) {
        double kj = m.k[j];
        if (kj > k1) out.push_back(std::sqrt(kj * kj - k1 * k1));
    }
}

void tau_kinks(const hfmm_medium& m, std::vector<double>& out) {
    const double k1 = m.k[0];
    int nl = m.kind == HFMM_TWO_LAYER ? 1 : (m.kind == HFMM_THREE_LAYER ? 2 : 0);
    for (int j = 1; j <= nl; ++j) {
        double kj = m.k[j];
        if (kj < k1) {
            out.push_back(std::acos(kj / k1));
            out.push_back(std::acos(-kj / k1));
        }
    }
}

double log_env(double t, double k1, double Y, int nmax) {
    double xi = std::sqrt(t * t + k1 * k1);
    return -t * Y + nmax * std::log((xi + t) / k1) - std::log(xi);
}

// end of the evanescent integral
double t_end(double k1, double Y, int nmax) {
    // peak of the envelope: derivative -Y + nmax / xi - t / xi^2 = 0
    double lo = 0.0, hi = std::max(1.0, (nmax + 1.0) / Y) * 4.0;
    auto d = [&](double t) {
        double xi = std::sqrt(t * t + k1 * k1);
        return -Y + nmax / xi - t / (xi * xi);
    };
    double tp = 0.0;
    if (d(0.0) > 0.0) {
        for (int it = 0; it < 200; ++it) {
            double mid = 0.5 * (lo + hi);
            if (d(mid) > 0.0) lo = mid; else hi = mid;
        }
        tp = 0.5 * (lo + hi);
    }
    const double target = log_env(tp, k1, Y, nmax) - 38.0;
    double a = tp, b = std::max(2.0 * tp, tp + 1.0);
    while (log_env(b, k1, Y, nmax) > target) b *= 2.0;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (a + b);
        if (log_env(mid, k1, Y, nmax) > target) a = mid; else b = mid;
    }
    return b;
}

// Build the segments of one integral; returns the number of nodes.
// `scale` multiplies every panel count: 1 is the table's rule, 2 its
// node-doubled check, other values come from hfmm_options.quad_scale.
int64_t make_rule(const hfmm_medium& m, double xmax, double ymin, double ymax, int nmax,
                  std::vector<Seg>& segs, double scale) {
    const double k1 = m.k[0];
    const bool three = m.kind == HFMM_THREE_LAYER;
    const double dd = three ? m.d : 0.0;
    int64_t nodes = 0;
    auto push = [&](double a, double b, int kind, int npan, double c, double tb) {
        Seg s{a, b, c, tb, kind, std::max((int)std::ceil(npan * scale), 1), nodes};
        nodes += (int64_t)s.npan * GLN;
        segs.push_back(s);
    };
    // propagating part
    double rate = k1 * (std::fabs(xmax) + std::fabs(ymax)) + nmax + 1.0;
    if (three) rate += 2.0 * dd * std::max(m.k[1], k1);
    std::vector<double> brk{0.0};
    tau_kinks(m, brk);
    brk.push_back(HFMM_PI);
    std::sort(brk.begin(), brk.end());
    // impedance: sigma has a pole at s1 = i alpha, i.e. sin tau = -alpha / k1; for
    // 0 < alpha < k1 it lies on the real tau axis at -delta and pi + delta,
    // delta = asin(alpha / k1), so the panels near both ends are graded: no
    // panel is wider than 1.5 times its distance to the pole
    const bool imp_pole = m.kind == HFMM_IMPEDANCE && m.alpha > 0.0;
    const double delta = (imp_pole && m.alpha < k1) ? std::asin(m.alpha / k1) : -1.0;
    const double wu = 4.0 / rate;
    for (size_t i = 0; i + 1 < brk.size(); ++i) {
        const double A = brk[i], B = brk[i + 1];
        if (delta <= 0.0 || 1.5 * delta >= wu) {
            push(A, B, 0, (int)std::ceil((B - A) * rate / 4.0) + 1, 0.0, 0.0);
            continue;
        }
        const double M = 0.5 * (A + B);
        std::vector<std::pair<double, double>> right;
        for (double a = A; a < M;) {
            const double w = std::min(wu, 1.5 * (a + delta));
            const double b = w >= wu ? M : std::min(M, std::max(a + 8.0 * w, 2.0 * a + delta));
            push(a, b, 0, (int)std::ceil((b - a) / w), 0.0, 0.0);
            a = b;
        }
        for (double b = B; b > M;) {
            const double dist = HFMM_PI + delta - b;
            const double w = std::min(wu, 1.5 * dist);
            const double a = w >= wu ? M : std::max(M, std::min(b - 8.0 * w, b - dist));
            right.push_back({a, b});
            b = a;
        }
        for (auto it = right.rbegin(); it != right.rend(); ++it) {
            const double w = std::min(wu, 1.5 * (HFMM_PI + delta - it->second));
            push(it->first, it->second, 0, (int)std::ceil((it->second - it->first) / w), 0.0, 0.0);
        }
    }
    // evanescent part
    const double xa = std::max(std::fabs(xmax), 1e-12);
    double T = t_end(k1, ymin, nmax);
    std::vector<double> sing;
    singular_t(m, sing);
    double t0 = 0.0;
    if (!sing.empty()) {
        double ts = *std::max_element(sing.begin(), sing.end());
        double tb = 1.3 * ts + 0.1 * k1;
        double c = std::min(0.2 * tb, 0.8 / xa);
        double w = std::min({0.7 * c, 3.0 / std::max(ymax, 1e-12), 3.0 / xa});
        if (three && dd > 0) w = std::min(w, 1.5 / dd);
        push(0.0, tb, 1, (int)std::ceil(tb / w) + 2, c, tb);
        t0 = tb;
        T = std::max(T, tb + 1.0);
    }
    double wc = std::min(4.0 / std::max(ymin, 1e-300), 4.0 / xa);
    if (three && dd > 0) wc = std::min(wc, 2.0 / dd);
    const double wmin = wc / 16.0;
    double a = t0;
    while (a < T) {
        double wl = nmax > 0 ? 3.0 * a / nmax : wc;
        double w = std::min(wc, std::max(wmin, wl));
        // impedance pole at t = i alpha: panel width <= 1.5 x its distance
        if (imp_pole) w = std::min(w, 1.5 * std::sqrt(a * a + m.alpha * m.alpha));
        // branch points of 1/xi, xi = sqrt(t^2 + k1^2), at t = +-i k1 (close to
        // t = 0 at low frequency): the same grading
        w = std::min(w, 1.5 * std::sqrt(a * a + k1 * k1));
        double b = (w < wc) ? std::min(T, std::max(a + 16.0 * w, 2.0 * a)) : T;
        push(a, b, 2, (int)std::ceil((b - a) / w), 0.0, 0.0);
        a = b;
    }
    return nodes;
}

struct MedDev {
    int kind;
    double k1, k2sq, k3sq, d, alpha;
};

MedDev make_med(const hfmm_medium& m) {
    MedDev d;
    d.kind = m.kind;
    d.k1 = m.k[0];
    d.k2sq = m.k[1] * m.k[1];
    d.k3sq = m.k[2] * m.k[2];
    d.d = m.d;
    d.alpha = m.alpha;
    return d;
}

// s = -i sqrt(k^2 - lambda^2), principal root (Re s >= 0)
__device__ __forceinline__ cd s_branch(double kk, cd lam2) {
    cd r = csqrtz(cmk(kk - lam2.x, -lam2.y));
    return cmk(r.y, -r.x);
}

__device__ cd sigma_dev(const MedDev& m, cd lam2, cd s1) {
    if (m.kind == HFMM_IMPEDANCE) {
        return cdiv(cmk(s1.x, s1.y + m.alpha), cmk(s1.x, s1.y - m.alpha));
    }
    cd s2 = s_branch(m.k2sq, lam2);
    cd r12 = cdiv(csub(s1, s2), cadd(s1, s2));
    if (m.kind == HFMM_TWO_LAYER) return r12;
    cd s3 = s_branch(m.k3sq, lam2);
    cd r23 = cdiv(csub(s2, s3), cadd(s2, s3));
    cd e = cexpz(cscale(s2, -2.0 * m.d));
    cd re = cmul(r23, e);
    return cdiv(cadd(r12, re), cadd(cmk(1.0, 0.0), cmul(r12, re)));
}

struct Node {
    int kind;        // 0 tau, 1 t
    cd base;         // tau: w e^{i k1 (Y sin - X cos)} sigma ; t: unused
    double tau;
    cd lp, lm;       // t: log(w dt sigma / xi) - tY +- i xi X
    cd lzp, lzm;     // t: log zp, log zm
    cd xi, t;        // t: xi = sqrt(t^2 + k1^2) and t
};

__device__ Node eval_node(const MedDev& m, const Seg* segs, int s0, int s1, int64_t nu, double X,
                          double Y) {
    int s = s0;
    while (s + 1 < s1 && segs[s + 1].node0 <= nu) ++s;
    const Seg sg = segs[s];
    const int64_t local = nu - sg.node0;
    const int pan = (int)(local / GLN), g = (int)(local % GLN);
    const double w = (sg.b - sg.a) / sg.npan;
    const double u = sg.a + (pan + 0.5 + 0.5 * c_glx[g]) * w;
    const double wu = 0.5 * w * c_glw[g];
    Node nd;
    const double k1 = m.k1;
    if (sg.kind == 0) {
        double st, ct;
        sincos(u, &st, &ct);
        cd lam2 = cmk(k1 * k1 * ct * ct, 0.0);
        cd sg1 = sigma_dev(m, lam2, cmk(0.0, -k1 * st));
        nd.kind = 0;
        nd.tau = u;
        nd.base = cscale(cmul(cexpi(k1 * (Y * st - X * ct)), sg1), wu);
        return nd;
    }
    cd t, dt;
    if (sg.kind == 1) {
        double tb = sg.tb;
        t = cmk(u, -sg.c * 4.0 * u * (tb - u) / (tb * tb));
        dt = cmk(1.0, -sg.c * 4.0 * (tb - 2.0 * u) / (tb * tb));
    } else {
        t = cmk(u, 0.0);
        dt = cmk(1.0, 0.0);
    }
    cd lam2 = cadd(cmul(t, t), cmk(k1 * k1, 0.0));
    cd xi = csqrtz(lam2);
    cd sg1 = sigma_dev(m, lam2, t);
    cd common = cdiv(cmul(cscale(dt, wu), sg1), xi);
    cd lc = clogz(common);
    cd ixX = cmuli(cscale(xi, X));            // i xi X
    cd mtY = cscale(t, -Y);                   // -t Y
    nd.kind = 1;
    nd.xi = xi;
    nd.t = t;
    nd.lp = cadd(cadd(lc, mtY), ixX);
    nd.lm = csub(cadd(lc, mtY), ixX);
    cd xpt = cadd(xi, t);
    cd lx = clogz(xpt);
    double lk = log(k1);
    nd.lzp = cmk(lk - lx.x, -lx.y);
    nd.lzm = cmk(lx.x - lk, lx.y + HFMM_PI);
    return nd;
}

constexpr int CH = 8;   // orders per chunk

// One CTA per table entry.  Writes A_n, n = -nmax .. nmax, scaled by `scale`.
__global__ void react_table_kernel(MedDev m, const Entry* ents, const Seg* segs, cd* out,
                                   double scale) {
    const Entry e = ents[blockIdx.x];
    const int nn = 2 * e.nmax + 1;
    __shared__ cd red[CH][2][32];
    for (int n0 = -e.nmax; n0 <= e.nmax; n0 += CH) {
        cd at[CH], ae[CH];
        for (int j = 0; j < CH; ++j) { at[j] = cmk(0, 0); ae[j] = cmk(0, 0); }
        for (int64_t nu = threadIdx.x; nu < e.nodes; nu += blockDim.x) {
            Node nd = eval_node(m, segs, e.seg0, e.seg1, nu, e.X, e.Y);
            if (nd.kind == 0) {
                cd v = cmul(nd.base, cexpi(-(double)n0 * nd.tau));
                cd st = cexpi(-nd.tau);
                for (int j = 0; j < CH; ++j) { at[j] = cadd(at[j], v); v = cmul(v, st); }
            } else {
                cd vp = cexpz(cadd(nd.lp, cscale(nd.lzp, (double)n0)));
                cd vm = cexpz(cadd(nd.lm, cscale(nd.lzm, (double)n0)));
                cd zp = cexpz(nd.lzp), zm = cexpz(nd.lzm);
                for (int j = 0; j < CH; ++j) {
                    ae[j] = cadd(ae[j], cadd(vp, vm));
                    vp = cmul(vp, zp);
                    vm = cmul(vm, zm);
                }
            }
        }
        // block reduction (warp shuffles, then one warp over the warps)
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        for (int j = 0; j < CH; ++j) {
            for (int o = 16; o > 0; o >>= 1) {
                at[j].x += __shfl_down_sync(0xffffffffu, at[j].x, o);
                at[j].y += __shfl_down_sync(0xffffffffu, at[j].y, o);
                ae[j].x += __shfl_down_sync(0xffffffffu, ae[j].x, o);
                ae[j].y += __shfl_down_sync(0xffffffffu, ae[j].y, o);
            }
            if (lane == 0) { red[j][0][wid] = at[j]; red[j][1][wid] = ae[j]; }
        }
        __syncthreads();
        if (wid == 0) {
            const int nw = blockDim.x >> 5;
            for (int j = 0; j < CH; ++j) {
                cd a = lane < nw ? red[j][0][lane] : cmk(0, 0);
                cd b = lane < nw ? red[j][1][lane] : cmk(0, 0);
                for (int o = 16; o > 0; o >>= 1) {
                    a.x += __shfl_down_sync(0xffffffffu, a.x, o);
                    a.y += __shfl_down_sync(0xffffffffu, a.y, o);
                    b.x += __shfl_down_sync(0xffffffffu, b.x, o);
                    b.y += __shfl_down_sync(0xffffffffu, b.y, o);
                }
                const int n = n0 + j;
                if (lane == 0 && n <= e.nmax) {
                    // i^n / pi * tau-sum + (-i)^n / (i pi) * t-sum
                    int r = ((n % 4) + 4) % 4;
                    cd in = (r == 0) ? cmk(1, 0) : (r == 1) ? cmk(0, 1) : (r == 2) ? cmk(-1, 0) : cmk(0, -1);
                    cd mi = cconj(in);                  // (-i)^n
                    cd v = cadd(cscale(cmul(in, a), 1.0 / HFMM_PI),
                                cscale(cmul(mi, cmk(b.y, -b.x)), 1.0 / HFMM_PI));  // b / i = -i b
                    out[e.out + (n + e.nmax)] = cscale(v, scale);
                }
            }
        }
        __syncthreads();
        (void)nn;
    }
}

// Direct reaction blocks: one thread per point pair (i in T, j in S).
struct DirectJob {
    int32_t t_lo, t_n, s_lo, s_n;
    int seg0, seg1;
    int64_t nodes;
    int64_t blk;
};

__global__ void direct_block_kernel(MedDev m, const DirectJob* jobs, const Seg* segs,
                                    const double2* xs, cd* vals) {
    const DirectJob jb = jobs[blockIdx.x];
    for (int idx = threadIdx.x; idx < jb.t_n * jb.s_n; idx += blockDim.x) {
    const int i = idx / jb.s_n, j = idx % jb.s_n;
    const double2 pi_ = xs[jb.t_lo + i], pj = xs[jb.s_lo + j];
    const double X = pi_.x - pj.x, Y = pi_.y + pj.y;
    cd at = cmk(0, 0), ae = cmk(0, 0);
    for (int64_t nu = 0; nu < jb.nodes; ++nu) {
        Node nd = eval_node(m, segs, jb.seg0, jb.seg1, nu, X, Y);
        if (nd.kind == 0) at = cadd(at, nd.base);
        else ae = cadd(ae, cadd(cexpz(nd.lp), cexpz(nd.lm)));
    }
    // A_0 = tau-sum / pi + t-sum / (i pi);  G^s = (i/4) A_0
    cd a0 = cadd(cscale(at, 1.0 / HFMM_PI), cscale(cmk(ae.y, -ae.x), 1.0 / HFMM_PI));
    vals[jb.blk + idx] = cmuli(cscale(a0, 0.25));
    }
}

// d/dX and d/dY (target point) of the directly summed reaction blocks: the
// target factor e^{-s1 Y + i lambda X} of the integrand contributes i lambda
// and -s1 (tau part: lambda = -k1 cos tau, s1 = -i k1 sin tau; t part:
// lambda = +-xi, s1 = t).
__global__ void direct_grad_block_kernel(MedDev m, const DirectJob* jobs, const Seg* segs, const double2* xs,
                                         cd* gx, cd* gy) {
    const DirectJob jb = jobs[blockIdx.x];
    for (int idx = threadIdx.x; idx < jb.t_n * jb.s_n; idx += blockDim.x) {
        const int i = idx / jb.s_n, j = idx % jb.s_n;
        const double2 pi_ = xs[jb.t_lo + i], pj = xs[jb.s_lo + j];
        const double X = pi_.x - pj.x, Y = pi_.y + pj.y;
        cd tx = cmk(0, 0), ty = cmk(0, 0), ex = cmk(0, 0), ey = cmk(0, 0);
        for (int64_t nu = 0; nu < jb.nodes; ++nu) {
            Node nd = eval_node(m, segs, jb.seg0, jb.seg1, nu, X, Y);
            if (nd.kind == 0) {
                double s_, c_;
                sincos(nd.tau, &s_, &c_);
                tx = cadd(tx, cmul(nd.base, cmk(0.0, -m.k1 * c_)));
                ty = cadd(ty, cmul(nd.base, cmk(0.0, m.k1 * s_)));
            } else {
                const cd vp = cexpz(nd.lp), vm = cexpz(nd.lm);
                ex = cadd(ex, cmul(cmuli(nd.xi), csub(vp, vm)));
                ey = cadd(ey, cmul(cneg(nd.t), cadd(vp, vm)));
            }
        }
        // A = tau-sum / pi + t-sum / (i pi); G^s derivatives = (i/4) A
        const cd ax = cadd(cscale(tx, 1.0 / HFMM_PI), cscale(cmk(ex.y, -ex.x), 1.0 / HFMM_PI));
        const cd ay = cadd(cscale(ty, 1.0 / HFMM_PI), cscale(cmk(ey.y, -ey.x), 1.0 / HFMM_PI));
        gx[jb.blk + idx] = cmuli(cscale(ax, 0.25));
        gy[jb.blk + idx] = cmuli(cscale(ay, 0.25));
    }
}

// Node-doubling check of the tables.  The reaction entry A_n feeds the
// translation entries s(|m|) s(|p|) A_n (m + p = -n) that act on the
// normalised expansions (|J_m(k rho)| <= s(|m|) inside a box); its weight w_n
// is the largest such product, so a difference that no translated field can
// see (the tiny coefficients the expansions never reach) does not count.
// One CTA per entry: max_n w_n |A_n - A2_n| / max_n w_n |A2_n|.
__device__ double block_max(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    v = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

__global__ void react_check_kernel(const Entry* ents, const cd* a1, const cd* a2, const double* w,
                                   double* ratio) {
    __shared__ double red[32];
    const Entry e = ents[blockIdx.x];
    double dm = 0.0, am = 0.0;
    for (int i = threadIdx.x; i < 2 * e.nmax + 1; i += blockDim.x) {
        const cd x = a1[e.out + i], y = a2[e.out + i];
        const double wi = w[e.wofs + i];
        dm = fmax(dm, wi * hypot(x.x - y.x, x.y - y.y));
        am = fmax(am, wi * hypot(y.x, y.y));
    }
    dm = block_max(dm, red);
    am = block_max(am, red);
    if (threadIdx.x == 0) ratio[blockIdx.x] = am > 0.0 ? dm / am : (dm > 0.0 ? INFINITY : 0.0);
}

// Directly summed blocks: max |G - G2| / max |G2| over the block's point pairs.
__global__ void direct_check_kernel(const DirectJob* jobs, const cd* v1, const cd* v2, double* ratio) {
    __shared__ double red[32];
    const DirectJob jb = jobs[blockIdx.x];
    double dm = 0.0, am = 0.0;
    for (int64_t i = threadIdx.x; i < (int64_t)jb.t_n * jb.s_n; i += blockDim.x) {
        const cd x = v1[jb.blk + i], y = v2[jb.blk + i];
        dm = fmax(dm, hypot(x.x - y.x, x.y - y.y));
        am = fmax(am, hypot(y.x, y.y));
    }
    dm = block_max(dm, red);
    am = block_max(am, red);
    if (threadIdx.x == 0) ratio[blockIdx.x] = am > 0.0 ? dm / am : (dm > 0.0 ? INFINITY : 0.0);
}

// Mirrored reaction entries: out[dst + nmax + n] = out[src + nmax - n].
struct int64_t3 {
    int64_t dst, src, nmax;
};

__global__ void mirror_kernel(const int64_t3* mir, cd* out) {
    const int64_t3 m = mir[blockIdx.x];
    for (int64_t i = threadIdx.x; i <= 2 * m.nmax; i += blockDim.x) out[m.dst + i] = out[m.src + 2 * m.nmax - i];
}

// free-space M2L: one thread per (offset) of one level
__global__ void free_table_kernel(double k, double h, int p, cd* out) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= 49) return;
    const int dx = o / 7 - 3, dy = o % 7 - 3;
    const int w = 4 * p + 1;
    cd* T = out + (int64_t)o * w;
    if (abs(dx) < 2 && abs(dy) < 2) {
        for (int i = 0; i < w; ++i) T[i] = cmk(0, 0);
        return;
    }
    const double X = dx * h, Y = dy * h;
    const double r = hypot(X, Y), th = atan2(Y, X);
    const double x = k * r;
    cd h0, h1;
    hankel01(x, &h0, &h1);
    cd hm = h0, hn = h1;
    T[2 * p] = h0;
    for (int n = 1; n <= 2 * p; ++n) {
        cd ph = cexpi(n * th);
        double sg = (n & 1) ? -1.0 : 1.0;
        T[2 * p + n] = cmul(hn, ph);
        T[2 * p - n] = cscale(cmul(hn, cconj(ph)), sg);
        cd hx = csub(cscale(hn, 2.0 * n / x), hm);
        hm = hn;
        hn = hx;
    }
}

// M2M (P - c) and L2L (c - P) tables of parent level l: thread per child
__global__ void shift_table_kernel(double k, double hc, int nmax, double* scratch, cd* m2m,
                                   cd* l2l) {
    const int c = threadIdx.x;
    if (c >= 4) return;
    const int w = 2 * nmax + 1;
    const double vx = (0.5 - (c & 1)) * hc, vy = (0.5 - (c >> 1)) * hc;   // P - c
    const double r = hypot(vx, vy), th = atan2(vy, vx);
    double* J = scratch + (int64_t)c * (nmax + 1);
    bessel_j_seq(k * r, nmax, J);
    for (int n = 0; n <= nmax; ++n) {
        cd ph = cexpi(n * th);
        double sg = (n & 1) ? -1.0 : 1.0;
        cd vp = cscale(ph, J[n]);                  // J_n(v) e^{i n th}
        cd vn = cscale(cconj(ph), sg * J[n]);      // J_{-n} e^{-i n th}
        m2m[(int64_t)c * w + nmax + n] = vp;
        m2m[(int64_t)c * w + nmax - n] = vn;
        // c - P = -v: J_n(-v) = (-1)^n J_n(v)
        l2l[(int64_t)c * w + nmax + n] = cscale(vp, sg);
        l2l[(int64_t)c * w + nmax - n] = cscale(vn, sg);
    }
}

}  // namespace

// G^s blocks of directly summed point-range pairs (target range x source
// range, row-major in the target) by quadrature on the panel rule for the
// pair's largest |X| and its range of Y, each block checked against the
// node-doubled rule (table_check).  Sets d_vals, nd_vals and the job list;
// blk[i] = offset of pair i's block.
hfmm_status build_direct_blocks(hfmm_plan_s* P, const std::vector<DirectSpec>& specs, std::vector<int64_t>& blk,
                                cudaStream_t st) {
    HFMM_TRY(ensure_gl());
    const MedDev md = make_med(P->med);
    const double qs = P->quad_scale;
    std::vector<Seg> dsg, dsg2;
    std::vector<DirectJob> jobs, jobs2;
    blk.assign(specs.size(), 0);
    int64_t off = 0;
    int64_t maxpairs = 0;
    for (size_t i = 0; i < specs.size(); ++i) {
        const DirectSpec& sp = specs[i];
        DirectJob jb;
        jb.t_lo = sp.t_lo; jb.t_n = sp.t_n;
        jb.s_lo = sp.s_lo; jb.s_n = sp.s_n;
        jb.blk = off;
        DirectJob jb2 = jb;
        jb.seg0 = (int)dsg.size();
        std::vector<Seg> tmp;
        jb.nodes = make_rule(P->med, sp.xmax, sp.ymin, sp.ymax, 0, tmp, qs);
        for (auto& sgm : tmp) dsg.push_back(sgm);
        jb.seg1 = (int)dsg.size();
        tmp.clear();
        jb2.seg0 = (int)dsg2.size();
        jb2.nodes = make_rule(P->med, sp.xmax, sp.ymin, sp.ymax, 0, tmp, 2.0 * qs);
        for (auto& sgm : tmp) dsg2.push_back(sgm);
        jb2.seg1 = (int)dsg2.size();
        blk[i] = off;
        off += (int64_t)jb.t_n * jb.s_n;
        maxpairs = std::max<int64_t>(maxpairs, (int64_t)jb.t_n * jb.s_n);
        jobs.push_back(jb);
        jobs2.push_back(jb2);
    }
    P->nd_vals = off;
    HFMM_TRY(plan_alloc(P, (void**)&P->d_vals, sizeof(cd) * std::max<int64_t>(off, 1)));
    if (jobs.empty()) return HFMM_OK;
    Seg* dsegs = nullptr;
    DirectJob* djobs = nullptr;
    HFMM_TRY(plan_alloc(P, (void**)&dsegs, sizeof(Seg) * std::max<size_t>(dsg.size(), 1)));
    HFMM_TRY(plan_alloc(P, (void**)&djobs, sizeof(DirectJob) * jobs.size()));
    if (!dsg.empty())
        HFMM_CUDA_TRY(cudaMemcpyAsync(dsegs, dsg.data(), sizeof(Seg) * dsg.size(), cudaMemcpyHostToDevice, st));
    HFMM_CUDA_TRY(cudaMemcpyAsync(djobs, jobs.data(), sizeof(DirectJob) * jobs.size(), cudaMemcpyHostToDevice, st));
    if (maxpairs > 0) {
        direct_block_kernel<<<(unsigned)jobs.size(), 128, 0, st>>>(md, djobs, dsegs, P->xy_sorted, P->d_vals);
        HFMM_CUDA_TRY(cudaGetLastError());
        // node-doubled blocks for the check
        cd* vals2 = nullptr;
        Seg* dsegs2 = nullptr;
        DirectJob* djobs2 = nullptr;
        double* dratio = nullptr;
        HFMM_TRY(plan_alloc(P, (void**)&vals2, sizeof(cd) * off));
        HFMM_TRY(plan_alloc(P, (void**)&dsegs2, sizeof(Seg) * std::max<size_t>(dsg2.size(), 1)));
        HFMM_TRY(plan_alloc(P, (void**)&djobs2, sizeof(DirectJob) * jobs2.size()));
        HFMM_TRY(plan_alloc(P, (void**)&dratio, sizeof(double) * jobs.size()));
        if (!dsg2.empty())
            HFMM_CUDA_TRY(cudaMemcpyAsync(dsegs2, dsg2.data(), sizeof(Seg) * dsg2.size(), cudaMemcpyHostToDevice, st));
        HFMM_CUDA_TRY(cudaMemcpyAsync(djobs2, jobs2.data(), sizeof(DirectJob) * jobs2.size(), cudaMemcpyHostToDevice, st));
        direct_block_kernel<<<(unsigned)jobs2.size(), 128, 0, st>>>(md, djobs2, dsegs2, P->xy_sorted, vals2);
        direct_check_kernel<<<(unsigned)jobs.size(), 128, 0, st>>>(djobs, P->d_vals, vals2, dratio);
        HFMM_CUDA_TRY(cudaGetLastError());
        std::vector<double> ratio(jobs.size());
        HFMM_CUDA_TRY(cudaMemcpyAsync(ratio.data(), dratio, sizeof(double) * ratio.size(), cudaMemcpyDeviceToHost, st));
        HFMM_CUDA_TRY(cudaStreamSynchronize(st));
        for (size_t i = 0; i < ratio.size(); ++i) {
            if (!(ratio[i] <= P->table_check)) {
                P->table_check = std::isnan(ratio[i]) ? INFINITY : ratio[i];
                P->table_check_where[0] = -1;      // a directly summed pair
                P->table_check_where[1] = (int)i;
                P->table_check_where[2] = 0;
            }
        }
    }
    P->dj_jobs = djobs;
    P->dj_segs = dsegs;
    P->dj_njobs = (int64_t)jobs.size();
    P->table_bytes += sizeof(cd) * (double)off;
    return HFMM_OK;
}

hfmm_status build_tables(hfmm_plan_s* P, cudaStream_t st) {
    HFMM_TRY(ensure_gl());
    const int L = P->L;
    const double k = P->k;
    const MedDev md = make_med(P->med);
    // free M2L and shift tables
    for (int l = 0; l <= L; ++l) {
        LevelInfo& lv = P->lev[l];
        if (l >= 2 && l >= P->lmin) {
            HFMM_TRY(plan_alloc(P, (void**)&lv.t_free, sizeof(cd) * 49 * (4 * lv.p + 1)));
            free_table_kernel<<<1, 64, 0, st>>>(k, lv.h, lv.p, lv.t_free);
            HFMM_CUDA_TRY(cudaGetLastError());
            P->table_bytes += sizeof(cd) * 49.0 * (4 * lv.p + 1);
        }
        if (l < L && l >= P->lmin) {
            const int nmax = lv.p + P->lev[l + 1].p;
            const int w = 2 * nmax + 1;
            double* scratch = nullptr;
            HFMM_TRY(plan_alloc(P, (void**)&scratch, sizeof(double) * 4 * (nmax + 1)));
            HFMM_TRY(plan_alloc(P, (void**)&lv.t_m2m, sizeof(cd) * 4 * w));
            HFMM_TRY(plan_alloc(P, (void**)&lv.t_l2l, sizeof(cd) * 4 * w));
            shift_table_kernel<<<1, 32, 0, st>>>(k, P->lev[l + 1].h, nmax, scratch, lv.t_m2m, lv.t_l2l);
            HFMM_CUDA_TRY(cudaGetLastError());
            P->table_bytes += sizeof(cd) * 8.0 * w;
        }
    }
    // reaction tables (on the panel rule, and on the node-doubled rule for the check)
    const double qs = P->quad_scale;
    std::vector<Seg> segs, segs2;
    std::vector<Entry> ents, ents2;
    std::vector<int64_t3> mirrors;   // (destination, source, nmax) of mirrored entries
    std::vector<double> wts;
    int64_t total = 0;
    std::vector<int64_t> lev_off(L + 1, 0);
    for (int l = 0; l <= L; ++l) {
        LevelInfo& lv = P->lev[l];
        if (lv.nr == 0) continue;
        const int m = 1 << l;
        const int dxmax = l == 0 ? 0 : m - 1;
        lv.react_dx_max = dxmax;
        lv.n_react_entries = (2 * dxmax + 1) * 3;
        const int nmax = 2 * lv.p;
        lev_off[l] = total;
        // weights w_n = max over m + p = -n (|m|, |p| <= p_l) of s(|m|) s(|p|),
        // s(n) = min(1, (k R_l / 2)^n / n!)
        const int64_t wofs = (int64_t)wts.size();
        {
            const double kR = P->k * lv.h / std::sqrt(2.0);
            std::vector<double> ls(lv.p + 1);
            for (int j = 0; j <= lv.p; ++j)
                ls[j] = std::min(0.0, j * std::log(0.5 * kR) - std::lgamma(j + 1.0));
            for (int n = -nmax; n <= nmax; ++n) {
                double best = -1e300;
                for (int mm = -lv.p; mm <= lv.p; ++mm) {
                    const int pp = -n - mm;
                    if (pp < -lv.p || pp > lv.p) continue;
                    best = std::max(best, ls[std::abs(mm)] + ls[std::abs(pp)]);
                }
                wts.push_back(std::exp(std::max(best, -700.0)));
            }
        }
        for (int dx = -dxmax; dx <= dxmax; ++dx)
            for (int ys = 0; ys < 3; ++ys) {
                const int64_t idx = (int64_t)(dx + dxmax) * 3 + ys;
                bool used = (l == 0) ? (dx == 0 && ys == 0)
                                     : (ys <= 2 && reaction_admissible(ys, 0, P->y0, lv.h) && !(ys == 2 && m < 2));
                if (l == 0) used = used && P->lstar == 0;
                if (!used) continue;
                if (dx < 0) {
                    // sigma is even in lambda: A_n(-X, Y) = A_{-n}(X, Y), a copy of the dx > 0 entry
                    mirrors.push_back({total + idx * (2 * nmax + 1), total + ((int64_t)(-dx + dxmax) * 3 + ys) * (2 * nmax + 1),
                                       (int64_t)nmax});
                    continue;
                }
                Entry e;
                e.X = dx * lv.h;
                e.Y = 2.0 * P->y0 + (ys + 1) * lv.h;
                e.nmax = nmax;
                e.out = total + idx * (2 * nmax + 1);
                e.wofs = wofs;
                e.level = l;
                e.dx = dx;
                e.ysum = ys;
                Entry e2 = e;
                std::vector<Seg> tmp;
                e.seg0 = (int)segs.size();
                e.nodes = make_rule(P->med, e.X, e.Y, e.Y, nmax, tmp, qs);
                for (auto& sg : tmp) segs.push_back(sg);
                e.seg1 = (int)segs.size();
                ents.push_back(e);
                tmp.clear();
                e2.seg0 = (int)segs2.size();
                e2.nodes = make_rule(P->med, e2.X, e2.Y, e2.Y, nmax, tmp, 2.0 * qs);
                for (auto& sg : tmp) segs2.push_back(sg);
                e2.seg1 = (int)segs2.size();
                ents2.push_back(e2);
            }
        total += (int64_t)lv.n_react_entries * (2 * nmax + 1);
    }
    if (!ents.empty()) {
        cd* tab = nullptr;
        HFMM_TRY(plan_alloc(P, (void**)&tab, sizeof(cd) * total));
        HFMM_CUDA_TRY(cudaMemsetAsync(tab, 0, sizeof(cd) * total, st));
        for (int l = 0; l <= L; ++l)
            if (P->lev[l].nr > 0) P->lev[l].t_react = tab + lev_off[l];
        Seg* dsegs = nullptr;
        Entry* dents = nullptr;
        HFMM_TRY(plan_alloc(P, (void**)&dsegs, sizeof(Seg) * segs.size()));
        HFMM_TRY(plan_alloc(P, (void**)&dents, sizeof(Entry) * ents.size()));
        HFMM_CUDA_TRY(cudaMemcpyAsync(dsegs, segs.data(), sizeof(Seg) * segs.size(), cudaMemcpyHostToDevice, st));
        HFMM_CUDA_TRY(cudaMemcpyAsync(dents, ents.data(), sizeof(Entry) * ents.size(), cudaMemcpyHostToDevice, st));
        react_table_kernel<<<(unsigned)ents.size(), 256, 0, st>>>(md, dents, dsegs, tab, 1.0);
        HFMM_CUDA_TRY(cudaGetLastError());
        if (!mirrors.empty()) {
            int64_t3* dmir = nullptr;
            HFMM_TRY(plan_alloc(P, (void**)&dmir, sizeof(int64_t3) * mirrors.size()));
            HFMM_CUDA_TRY(cudaMemcpyAsync(dmir, mirrors.data(), sizeof(int64_t3) * mirrors.size(),
                                          cudaMemcpyHostToDevice, st));
            mirror_kernel<<<(unsigned)mirrors.size(), 128, 0, st>>>(dmir, tab);
            HFMM_CUDA_TRY(cudaGetLastError());
        }
        P->table_bytes += sizeof(cd) * (double)total;
        // the same entries on the node-doubled rule, compared entry by entry
        cd* tab2 = nullptr;
        Seg* dsegs2 = nullptr;
        Entry* dents2 = nullptr;
        double *dw = nullptr, *dratio = nullptr;
        HFMM_TRY(plan_alloc(P, (void**)&tab2, sizeof(cd) * total));
        HFMM_TRY(plan_alloc(P, (void**)&dsegs2, sizeof(Seg) * segs2.size()));
        HFMM_TRY(plan_alloc(P, (void**)&dents2, sizeof(Entry) * ents2.size()));
        HFMM_TRY(plan_alloc(P, (void**)&dw, sizeof(double) * wts.size()));
        HFMM_TRY(plan_alloc(P, (void**)&dratio, sizeof(double) * ents.size()));
        HFMM_CUDA_TRY(cudaMemcpyAsync(dsegs2, segs2.data(), sizeof(Seg) * segs2.size(), cudaMemcpyHostToDevice, st));
        HFMM_CUDA_TRY(cudaMemcpyAsync(dents2, ents2.data(), sizeof(Entry) * ents2.size(), cudaMemcpyHostToDevice, st));
        HFMM_CUDA_TRY(cudaMemcpyAsync(dw, wts.data(), sizeof(double) * wts.size(), cudaMemcpyHostToDevice, st));
        HFMM_CUDA_TRY(cudaMemsetAsync(tab2, 0, sizeof(cd) * total, st));
        react_table_kernel<<<(unsigned)ents2.size(), 256, 0, st>>>(md, dents2, dsegs2, tab2, 1.0);
        react_check_kernel<<<(unsigned)ents.size(), 128, 0, st>>>(dents, tab, tab2, dw, dratio);
        HFMM_CUDA_TRY(cudaGetLastError());
        std::vector<double> ratio(ents.size());
        HFMM_CUDA_TRY(cudaMemcpyAsync(ratio.data(), dratio, sizeof(double) * ratio.size(), cudaMemcpyDeviceToHost, st));
        HFMM_CUDA_TRY(cudaStreamSynchronize(st));
        for (size_t i = 0; i < ratio.size(); ++i) {
            if (!(ratio[i] <= P->table_check)) {       // also catches NaN
                P->table_check = std::isnan(ratio[i]) ? INFINITY : ratio[i];
                P->table_check_where[0] = ents[i].level;
                P->table_check_where[1] = ents[i].dx;
                P->table_check_where[2] = ents[i].ysum;
            }
        }
    }
    // direct reaction blocks: leaf pairs of the bottom row (adaptive trees build theirs with their lists)
    if (P->nd > 0 && !P->ad) {
        const double h = P->lev[L].h;
        std::vector<int32_t> dbeg((size_t)P->lev[L].nbox + 1), dsrc(P->nd);
        HFMM_CUDA_TRY(cudaMemcpyAsync(dbeg.data(), P->d_begin, sizeof(int32_t) * dbeg.size(), cudaMemcpyDeviceToHost, st));
        HFMM_CUDA_TRY(cudaMemcpyAsync(dsrc.data(), P->d_src, sizeof(int32_t) * P->nd, cudaMemcpyDeviceToHost, st));
        HFMM_CUDA_TRY(cudaStreamSynchronize(st));
        const auto& lb = P->h_leaf_begin;
        std::vector<DirectSpec> specs;
        specs.reserve(P->nd);
        for (int64_t b = 0; b < P->lev[L].nbox; ++b)
            for (int32_t e = dbeg[b]; e < dbeg[b + 1]; ++e) {
                const int64_t s = dsrc[e];
                const int dx = (int)morton_x((uint32_t)b) - (int)morton_x((uint32_t)s);
                specs.push_back({lb[b], lb[b + 1] - lb[b], lb[s], lb[s + 1] - lb[s], (std::abs(dx) + 1) * h,
                                 2.0 * P->y0, 2.0 * P->y0 + 2.0 * h});
            }
        std::vector<int64_t> blk;
        HFMM_TRY(build_direct_blocks(P, specs, blk, st));
        HFMM_TRY(plan_alloc(P, (void**)&P->d_blk, sizeof(int64_t) * P->nd));
        HFMM_CUDA_TRY(cudaMemcpyAsync(P->d_blk, blk.data(), sizeof(int64_t) * P->nd, cudaMemcpyHostToDevice, st));
    }
    HFMM_CUDA_TRY(cudaStreamSynchronize(st));
    if (!(P->table_check <= TABLE_RTOL)) {
        if (P->table_check_where[0] >= 0)
            hfmm_set_error("reaction table quadrature not converged: level %d, dx %d, ysum %d differs from its "
                           "node-doubled rule by %.3g (bound %.1g)", P->table_check_where[0],
                           P->table_check_where[1], P->table_check_where[2], P->table_check, TABLE_RTOL);
        else
            hfmm_set_error("direct reaction quadrature not converged: leaf-pair block %d differs from its "
                           "node-doubled rule by %.3g (bound %.1g)", P->table_check_where[1], P->table_check,
                           TABLE_RTOL);
        return HFMM_ERR_NUMERICS;
    }
    return HFMM_OK;
}

// ---------------------------------------------------------------------------
// Mixed path: scaled FP32 translation matrices from the FP64 tables.
//   a~_n = a_n / s_l(|n|), b~_n = b_n s_l(|n|),  s_l(n) = min(1, (k R_l / 2)^n / n!)
// so that every stored matrix entry is O(1) or smaller (FP32 range).
// ---------------------------------------------------------------------------
namespace {

__device__ __forceinline__ cf to_cf(cd v) { return cfmk((float)v.x, (float)v.y); }

// Matrices are stored column-major (input coefficient outer, output inner),
// so that threads over output coefficients read consecutive entries.
// free-space M2L: F~[off][m][p] = s(p) s(m) C_{m-p}(off)
__global__ void free32_kernel(const cd* T, const double* ls, int p, cf* out) {
    const int nc = 2 * p + 1, w = 4 * p + 1;
    const int64_t total = (int64_t)49 * nc * nc;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int off = (int)(e / (nc * nc));
        const int r = (int)(e % (nc * nc));
        const int pp = r / nc - p, m = r % nc - p;
        const double sc = exp(ls[abs(pp)] + ls[abs(m)]);
        out[(int64_t)off * nc * nc + (int64_t)(m + p) * nc + (pp + p)] =
            to_cf(cscale(T[(int64_t)off * w + (m - pp) + 2 * p], sc));
    }
}

// reaction M2L on a (not a^im): H~[e][m][p] = s(p) s(m) (-1)^m A_{-m-p}
__global__ void react32_kernel(const cd* T, int nent, const double* ls, int p, cf* out) {
    const int nc = 2 * p + 1, w = 4 * p + 1;
    const int64_t total = (int64_t)nent * nc * nc;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int ent = (int)(e / (nc * nc));
        const int r = (int)(e % (nc * nc));
        const int pp = r / nc - p, m = r % nc - p;
        double sc = exp(ls[abs(pp)] + ls[abs(m)]);
        if (m & 1) sc = -sc;
        out[(int64_t)ent * nc * nc + (int64_t)(m + p) * nc + (pp + p)] =
            to_cf(cscale(T[(int64_t)ent * w + (-m - pp) + 2 * p], sc));
    }
}

// M2M child (level l+1, order pc) -> parent (level l, order pp):
//   T~[c][m][j] = J_{m-j}(P - c) s_{l+1}(m) / s_l(j)
// L2L parent -> child: L~[c][n][m] = J_{n-m}(c - P) s_{l+1}(m) / s_l(n)
__global__ void shift32_kernel(const cd* m2m, const cd* l2l, const double* lsp, const double* lsc,
                               int pp, int pc, cf* om2m, cf* ol2l) {
    const int np = 2 * pp + 1, nc = 2 * pc + 1, nmax = pp + pc, w = 2 * nmax + 1;
    const int64_t total = (int64_t)4 * np * nc;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e / (np * nc));
        const int r = (int)(e % (np * nc));
        // M2M: row j (parent), column m (child)
        {
            const int j = r / nc - pp, m = r % nc - pc;
            const double sc = exp(lsc[abs(m)] - lsp[abs(j)]);
            om2m[(int64_t)c * np * nc + (int64_t)(m + pc) * np + (j + pp)] =
                to_cf(cscale(m2m[(int64_t)c * w + nmax + (m - j)], sc));
        }
        // L2L: row m (child), column n (parent)
        {
            const int m = r / np - pc, n = r % np - pp;
            const double sc = exp(lsc[abs(m)] - lsp[abs(n)]);
            ol2l[(int64_t)c * np * nc + (int64_t)(n + pp) * nc + (m + pc)] =
                to_cf(cscale(l2l[(int64_t)c * w + nmax + (n - m)], sc));
        }
    }
}

__global__ void vals32_kernel(const cd* v, int64_t n, cf* out) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        out[e] = to_cf(v[e]);
}

}  // namespace

hfmm_status build_tables32(hfmm_plan_s* P, cudaStream_t st) {
    const int L = P->L;
    const int grid = 4 * 152, tb = 256;
    for (int l = P->lmin; l <= L; ++l) {
        LevelInfo& lv = P->lev[l];
        const double kR = P->k * lv.h / std::sqrt(2.0);
        lv.log_s.assign(lv.p + 1, 0.0);
        for (int n = 0; n <= lv.p; ++n) {
            double v = n * std::log(0.5 * kR) - std::lgamma(n + 1.0);
            lv.log_s[n] = std::max(-690.0, std::min(0.0, v));
        }
        HFMM_TRY(plan_alloc(P, (void**)&lv.d_log_s, sizeof(double) * (lv.p + 1)));
        HFMM_CUDA_TRY(cudaMemcpyAsync(lv.d_log_s, lv.log_s.data(), sizeof(double) * (lv.p + 1), cudaMemcpyHostToDevice, st));
    }
    for (int l = P->lmin; l <= L; ++l) {
        LevelInfo& lv = P->lev[l];
        const int nc = lv.ncoef;
        if (lv.t_free) {
            HFMM_TRY(plan_alloc(P, (void**)&lv.t_free32, sizeof(cf) * 49 * nc * nc));
            free32_kernel<<<grid, tb, 0, st>>>(lv.t_free, lv.d_log_s, lv.p, lv.t_free32);
            HFMM_CUDA_TRY(cudaGetLastError());
            P->table_bytes += sizeof(cf) * 49.0 * nc * nc;
        }
        if (lv.t_react && lv.n_react_entries > 0) {
            HFMM_TRY(plan_alloc(P, (void**)&lv.t_react32, sizeof(cf) * (size_t)lv.n_react_entries * nc * nc));
            react32_kernel<<<grid, tb, 0, st>>>(lv.t_react, lv.n_react_entries, lv.d_log_s, lv.p, lv.t_react32);
            HFMM_CUDA_TRY(cudaGetLastError());
            P->table_bytes += sizeof(cf) * (double)lv.n_react_entries * nc * nc;
        }
        if (l < L && lv.t_m2m) {
            const int ncc = P->lev[l + 1].ncoef;
            HFMM_TRY(plan_alloc(P, (void**)&lv.t_m2m32, sizeof(cf) * 4 * nc * ncc));
            HFMM_TRY(plan_alloc(P, (void**)&lv.t_l2l32, sizeof(cf) * 4 * nc * ncc));
            shift32_kernel<<<grid, tb, 0, st>>>(lv.t_m2m, lv.t_l2l, lv.d_log_s, P->lev[l + 1].d_log_s, lv.p,
                                                P->lev[l + 1].p, lv.t_m2m32, lv.t_l2l32);
            HFMM_CUDA_TRY(cudaGetLastError());
            P->table_bytes += sizeof(cf) * 8.0 * nc * ncc;
        }
    }
    if (P->nd_vals > 0) {
        HFMM_TRY(plan_alloc(P, (void**)&P->d_vals32, sizeof(cf) * P->nd_vals));
        vals32_kernel<<<grid, tb, 0, st>>>(P->d_vals, P->nd_vals, P->d_vals32);
        HFMM_CUDA_TRY(cudaGetLastError());
    }
    HFMM_CUDA_TRY(cudaStreamSynchronize(st));
    return HFMM_OK;
}

// Gradient blocks of the directly summed reaction (built on the first
// position-gradient request).
hfmm_status build_direct_grad(hfmm_plan_s* P, cudaStream_t st) {
    if (P->nd == 0 || P->nd_vals == 0) return HFMM_OK;
    HFMM_TRY(ensure_gl());
    HFMM_TRY(plan_alloc(P, (void**)&P->d_gvals, sizeof(cd) * 2 * P->nd_vals));
    const MedDev md = make_med(P->med);
    direct_grad_block_kernel<<<(unsigned)P->dj_njobs, 128, 0, st>>>(md, (const DirectJob*)P->dj_jobs,
                                                                     (const Seg*)P->dj_segs, P->xy_sorted,
                                                                     P->d_gvals, P->d_gvals + P->nd_vals);
    HFMM_CUDA_TRY(cudaGetLastError());
    return HFMM_OK;
}
