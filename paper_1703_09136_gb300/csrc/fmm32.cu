// Mixed-precision apply path (HFMM_MIXED): complex64 in/out, FP32 storage and
// arithmetic for expansions and direct sums; FP64 only where the method needs
// it (Bessel recurrences of the point bases, plan-time tables).
//
// Expansions are scaled so that FP32 never over- or underflows:
//   a~_m = a_m / s_l(|m|),  b~_p = b_p s_l(|p|),  s_l(n) = min(1, (k R_l / 2)^n / n!)
// and the translation matrices are the scaled full matrices of tables.cu.
// Near field: H0 by a piecewise degree-5 polynomial table for J0 and for the
// smooth part R0 = Y0 - (2/pi) ln(z/2) J0 (coefficients fitted at library
// initialisation from the FP64 Bessel code by Chebyshev interpolation).
#include <algorithm>
#include <cmath>
#include <vector>

#include "bessel.cuh"
#include "plan.cuh"

namespace {

// ---------------------------------------------------------------------------
// FP32 H0 table
// ---------------------------------------------------------------------------
constexpr int H0_DEG = 5;
constexpr int H0_NI = 64;              // intervals on [0, 16]
constexpr float H0_ZMAX = 16.0f;
constexpr float H0_INV_DZ = 4.0f;      // 1 / interval width
__constant__ float c_h0j[H0_NI][H0_DEG + 1];
__constant__ float c_h0r[H0_NI][H0_DEG + 1];
float h_h0j[H0_NI][H0_DEG + 1], h_h0r[H0_NI][H0_DEG + 1];
bool h0_ready = false;

void fit_h0_table() {
    const int n = H0_DEG + 1;
    double tn[n], cheb[n][n];   // Chebyshev -> monomial coefficients
    for (int i = 0; i < n; ++i) for (int j = 0; j < n; ++j) cheb[i][j] = 0.0;
    cheb[0][0] = 1.0;
    cheb[1][1] = 1.0;
    for (int j = 2; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            double v = -cheb[j - 2][i];
            if (i > 0) v += 2.0 * cheb[j - 1][i - 1];
            cheb[j][i] = v;
        }
    for (int iv = 0; iv < H0_NI; ++iv) {
        const double half = 0.5 / H0_INV_DZ, mid = (iv + 0.5) / H0_INV_DZ;
        double fj[n], fr[n];
        for (int k = 0; k < n; ++k) {
            tn[k] = std::cos(HFMM_PI * (k + 0.5) / n);
            const double z = mid + half * tn[k];
            double j0, y0;
            if (z <= 5.0) bessel_01_series(z, &j0, &y0);
            else bessel_miller(z, 1, nullptr, &j0, nullptr, &y0, nullptr);
            fj[k] = j0;
            fr[k] = y0 - HFMM_2_OVER_PI * std::log(0.5 * z) * j0;
        }
        double cj[n], cr[n];
        for (int j = 0; j < n; ++j) {
            double sj = 0.0, sr = 0.0;
            for (int k = 0; k < n; ++k) {
                const double T = std::cos(j * HFMM_PI * (k + 0.5) / n);
                sj += fj[k] * T;
                sr += fr[k] * T;
            }
            cj[j] = (j == 0 ? 1.0 : 2.0) * sj / n;
            cr[j] = (j == 0 ? 1.0 : 2.0) * sr / n;
        }
        for (int i = 0; i < n; ++i) {
            double aj = 0.0, ar = 0.0;
            for (int j = 0; j < n; ++j) { aj += cj[j] * cheb[j][i]; ar += cr[j] * cheb[j][i]; }
            h_h0j[iv][i] = (float)aj;
            h_h0r[iv][i] = (float)ar;
        }
    }
}

// (i/4) H0(z) in FP32 for 0 < z < 16
__device__ __forceinline__ cf green_free_f32(float z) {
    const int iv = min((int)(z * H0_INV_DZ), H0_NI - 1);
    const float t = (z - ((float)iv + 0.5f) / H0_INV_DZ) * (2.0f * H0_INV_DZ);
    float j = c_h0j[iv][H0_DEG], r = c_h0r[iv][H0_DEG];
#pragma unroll
    for (int d = H0_DEG - 1; d >= 0; --d) {
        j = fmaf(j, t, c_h0j[iv][d]);
        r = fmaf(r, t, c_h0r[iv][d]);
    }
    const float y = fmaf(0.63661977236758134f * logf(0.5f * z), j, r);
    return cfmk(-0.25f * y, 0.25f * j);
}

HD void cfma32(cf& acc, cf a, cf b) {
    acc.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x));
    acc.y = fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y));
}

__global__ void gather_q32(const cf* q, const int64_t* perm, int64_t n, int nrhs, bool conj_in, cf* qs) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t j = perm[i];
    for (int r = 0; r < nrhs; ++r) {
        cf v = q[(int64_t)r * n + j];
        if (conj_in) v.y = -v.y;
        qs[(int64_t)r * n + i] = v;
    }
}

__global__ void scatter_y32(const cf* ys, const int64_t* perm, int64_t n, int nrhs, bool conj_out, cf* y) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t j = perm[i];
    for (int r = 0; r < nrhs; ++r) {
        cf v = ys[(int64_t)r * n + i];
        if (conj_out) v.y = -v.y;
        y[(int64_t)r * n + j] = v;
    }
}

// scaled point basis B[m + p] = J_m(k rho) e^{sgn i m theta} / s(|m|), FP64 then FP32
__device__ void point_basis32(double px, double py, double cx, double cy, double k, int p, int sgn,
                              const double* log_s, double* Jt, cf* B) {
    const double dx = px - cx, dy = py - cy;
    const double rho = hypot(dx, dy);
    bessel_j_seq(k * rho, p, Jt);
    const double th = atan2(dy, dx);
    const cd e1 = cexpi(sgn * th);
    cd e = cmk(1.0, 0.0);
    B[p] = cfmk((float)(Jt[0] * exp(-log_s[0])), 0.0f);
    for (int m = 1; m <= p; ++m) {
        e = cmul(e, e1);
        const double a = Jt[m] * exp(-log_s[m]);
        const double sg = (m & 1) ? -a : a;
        B[p + m] = cfmk((float)(e.x * a), (float)(e.y * a));
        B[p - m] = cfmk((float)(e.x * sg), (float)(-e.y * sg));
    }
}

__global__ void p2m32_kernel(const int32_t* lb, const double2* xs, const cf* qs, int64_t n, int nrhs,
                             double x0, double y0, double h, double k, int p, const double* log_s,
                             int chunk, cf* mult) {
    extern __shared__ double smem[];
    const int64_t b = blockIdx.x;
    const int ncoef = 2 * p + 1;
    double* Jt = smem;
    cf* B = (cf*)(Jt + (size_t)chunk * (p + 1));
    const int32_t lo = lb[b], hi = lb[b + 1];
    const double cx = x0 + (morton_x((uint32_t)b) + 0.5) * h;
    const double cy = y0 + (morton_y((uint32_t)b) + 0.5) * h;
    cf* out = mult + (int64_t)b * nrhs * ncoef;
    const int items = nrhs * ncoef;
    for (int it = threadIdx.x; it < items; it += blockDim.x) out[it] = cfmk(0.f, 0.f);
    for (int32_t c0 = lo; c0 < hi; c0 += chunk) {
        const int cnt = min(chunk, hi - c0);
        __syncthreads();
        for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
            const double2 pt = xs[c0 + t];
            point_basis32(pt.x, pt.y, cx, cy, k, p, -1, log_s, Jt + (size_t)t * (p + 1), B + (size_t)t * ncoef);
        }
        __syncthreads();
        for (int it = threadIdx.x; it < items; it += blockDim.x) {
            const int r = it / ncoef, m = it % ncoef;
            cf acc = out[it];
            const cf* qr = qs + (int64_t)r * n + c0;
            for (int t = 0; t < cnt; ++t) cfma32(acc, qr[t], B[(size_t)t * ncoef + m]);
            out[it] = acc;
        }
    }
}

// M2M (scaled): a~^P[r][j] = sum_c sum_m T~[c][m][j] a~^c[r][m]
__global__ void m2m32_kernel(const cf* child, const cf* T, int pc, int pp, int nrhs, cf* parent) {
    const int64_t b = blockIdx.x;
    const int nc = 2 * pc + 1, np = 2 * pp + 1;
    const int nq = (np + 3) / 4;            // groups of 4 parent coefficients
    const int items = nrhs * nq;
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
        const int r = it / nq, j0 = 4 * (it % nq);
        const int nj = min(4, np - j0);
        cf acc[4] = {cfmk(0.f, 0.f), cfmk(0.f, 0.f), cfmk(0.f, 0.f), cfmk(0.f, 0.f)};
        for (int c = 0; c < 4; ++c) {
            const cf* a = child + ((4 * b + c) * nrhs + r) * (int64_t)nc;
            const cf* Tc = T + (int64_t)c * nc * np + j0;
            for (int m = 0; m < nc; ++m) {
                const cf av = a[m];
                const cf* Tm = Tc + (int64_t)m * np;
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (u < nj) cfma32(acc[u], av, Tm[u]);
            }
        }
        for (int u = 0; u < nj; ++u) parent[(b * nrhs + r) * (int64_t)np + j0 + u] = acc[u];
    }
}

// Downward pass (scaled): one CTA per non-empty box, right-hand sides staged
// in shared memory per source box, matrices read column-major.
constexpr int DOWN_THREADS = 256;

__global__ void __launch_bounds__(DOWN_THREADS) down32_kernel(
    const int32_t* lb, int L, int l, int lmin, int nrhs, int p, int pp, const cf* ploc, const cf* Tl2l,
    const cf* mult, const int32_t* v_begin, const int32_t* v_src, const int32_t* v_off, const cf* Tfree,
    const int32_t* r_begin, const int32_t* r_src, const int32_t* r_tab, const cf* Treact, int parts,
    int rc, cf* loc) {
    extern __shared__ float sm32[];
    cf* as = (cf*)sm32;                         // [rc][nsrc coef]
    const int64_t b = blockIdx.x;
    int32_t lo, hi;
    box_range(lb, L, l, b, &lo, &hi);
    if (hi <= lo) return;
    const int nc = 2 * p + 1, npp = 2 * pp + 1;
    const bool has_parent = (l > lmin) && ploc;
    const int64_t P = b >> 2;
    const int cchild = (int)(b & 3);
    const int nv0 = ((parts & HFMM_PART_FAR_FREE) && v_begin) ? v_begin[b] : 0;
    const int nv1 = ((parts & HFMM_PART_FAR_FREE) && v_begin) ? v_begin[b + 1] : 0;
    const int nr0 = ((parts & HFMM_PART_FAR_REACT) && r_begin) ? r_begin[b] : 0;
    const int nr1 = ((parts & HFMM_PART_FAR_REACT) && r_begin) ? r_begin[b + 1] : 0;
    const int nsrc = (has_parent ? 1 : 0) + (nv1 - nv0) + (nr1 - nr0);
    for (int r0 = 0; r0 < nrhs; r0 += rc) {
        const int nr = min(rc, nrhs - r0);
        const int items = nr * nc;
        constexpr int MAXI = 8;
        cf acc[MAXI];
        for (int u = 0; u < MAXI; ++u) acc[u] = cfmk(0.f, 0.f);
        for (int s = 0; s < nsrc; ++s) {
            const cf* src;
            const cf* M;
            int ncs;
            if (has_parent && s == 0) {
                src = ploc + (P * nrhs + r0) * (int64_t)npp;
                M = Tl2l + (int64_t)cchild * npp * nc;
                ncs = npp;
            } else {
                int e = s - (has_parent ? 1 : 0);
                if (e < nv1 - nv0) {
                    src = mult + ((int64_t)v_src[nv0 + e] * nrhs + r0) * nc;
                    M = Tfree + (int64_t)v_off[nv0 + e] * nc * nc;
                } else {
                    e -= nv1 - nv0;
                    src = mult + ((int64_t)r_src[nr0 + e] * nrhs + r0) * nc;
                    M = Treact + (int64_t)r_tab[nr0 + e] * nc * nc;
                }
                ncs = nc;
            }
            __syncthreads();
            for (int i = threadIdx.x; i < nr * ncs; i += blockDim.x) as[i] = src[i];
            __syncthreads();
            for (int u = 0; u < MAXI; ++u) {
                const int it = u * DOWN_THREADS + threadIdx.x;
                if (it >= items) break;
                const int r = it / nc, q = it % nc;
                const cf* ar = as + r * ncs;
                const cf* Mq = M + q;
                cf a = acc[u];
                for (int m = 0; m < ncs; ++m) cfma32(a, ar[m], Mq[(int64_t)m * nc]);
                acc[u] = a;
            }
        }
        for (int u = 0; u < MAXI; ++u) {
            const int it = u * DOWN_THREADS + threadIdx.x;
            if (it >= items) break;
            const int r = it / nc, q = it % nc;
            loc[(b * nrhs + r0 + r) * (int64_t)nc + q] = acc[u];
        }
    }
}

__global__ void l2p32_kernel(const int32_t* lb, const double2* xs, const cf* loc, int64_t n, int nrhs,
                             double x0, double y0, double h, double k, int p, const double* log_s, int chunk,
                             cf* ys) {
    extern __shared__ double smem[];
    const int64_t b = blockIdx.x;
    const int32_t lo = lb[b], hi = lb[b + 1];
    if (hi <= lo) return;
    const int ncoef = 2 * p + 1;
    double* Jt = smem;
    cf* B = (cf*)(Jt + (size_t)chunk * (p + 1));
    const double cx = x0 + (morton_x((uint32_t)b) + 0.5) * h;
    const double cy = y0 + (morton_y((uint32_t)b) + 0.5) * h;
    const cf* beta = loc + (int64_t)b * nrhs * ncoef;
    for (int32_t c0 = lo; c0 < hi; c0 += chunk) {
        const int cnt = min(chunk, hi - c0);
        __syncthreads();
        for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
            const double2 pt = xs[c0 + t];
            point_basis32(pt.x, pt.y, cx, cy, k, p, +1, log_s, Jt + (size_t)t * (p + 1), B + (size_t)t * ncoef);
        }
        __syncthreads();
        const int items = nrhs * cnt;
        for (int it = threadIdx.x; it < items; it += blockDim.x) {
            const int r = it / cnt, t = it % cnt;
            cf acc = cfmk(0.f, 0.f);
            const cf* br = beta + (int64_t)r * ncoef;
            for (int m = 0; m < ncoef; ++m) cfma32(acc, br[m], B[(size_t)t * ncoef + m]);
            cf* yy = ys + (int64_t)r * n + c0 + t;
            yy->x += -0.25f * acc.y;
            yy->y += 0.25f * acc.x;
        }
    }
}

// point offsets from their own leaf centre, FP32 (near-field geometry without FP64)
__global__ void local_coords_kernel(const int32_t* lb, const double2* xs, int64_t nleaf, double x0,
                                    double y0, double h, float2* xl) {
    const int64_t b = blockIdx.x;
    if (b >= nleaf) return;
    const double cx = x0 + (morton_x((uint32_t)b) + 0.5) * h;
    const double cy = y0 + (morton_y((uint32_t)b) + 0.5) * h;
    for (int32_t i = lb[b] + threadIdx.x; i < lb[b + 1]; i += blockDim.x)
        xl[i] = make_float2((float)(xs[i].x - cx), (float)(xs[i].y - cy));
}

// P2P free-space part, FP32 (Algorithm 1, step 5): one CTA per non-empty
// target leaf, 32 x 32 blocks of (i/4) H0 values in shared memory, source
// strengths of 64 right-hand sides staged beside them, 2 targets x 4 RHS
// accumulators per thread.
constexpr int P2T = 32;            // targets / sources per block
constexpr int P2R = 64;            // right-hand sides per pass
constexpr int P2_THREADS = 256;

__global__ void __launch_bounds__(P2_THREADS) p2p32b_kernel(const int32_t* lb, int L, const float2* xl,
                                                            const cf* qs, int64_t n, int nrhs, float k,
                                                            float h, cf* ys) {
    __shared__ cf G[P2T][P2T + 1];
    __shared__ cf Q[P2R][P2T + 1];
    __shared__ float2 sp[P2T];
    __shared__ float2 tp[P2T];
    __shared__ float tj[H0_NI][H0_DEG + 1];
    __shared__ float tr[H0_NI][H0_DEG + 1];
    const int64_t b = blockIdx.x;
    const int32_t tlo = lb[b], thi = lb[b + 1];
    if (thi <= tlo) return;
    for (int e = threadIdx.x; e < H0_NI * (H0_DEG + 1); e += blockDim.x) {
        tj[e / (H0_DEG + 1)][e % (H0_DEG + 1)] = c_h0j[e / (H0_DEG + 1)][e % (H0_DEG + 1)];
        tr[e / (H0_DEG + 1)][e % (H0_DEG + 1)] = c_h0r[e / (H0_DEG + 1)][e % (H0_DEG + 1)];
    }
    const int m = 1 << L;
    const int ix = (int)morton_x((uint32_t)b), iy = (int)morton_y((uint32_t)b);
    const int tpair = threadIdx.x & 15, rg = threadIdx.x >> 4;   // targets 2*tpair(+1), rhs 4*rg..4*rg+3
    for (int r0 = 0; r0 < nrhs; r0 += P2R) {
        const int nr = min(P2R, nrhs - r0);
        for (int32_t t0 = tlo; t0 < thi; t0 += P2T) {
            const int tn = min(P2T, thi - t0);
            cf acc[2][4];
            for (int a = 0; a < 2; ++a)
                for (int c = 0; c < 4; ++c) acc[a][c] = cfmk(0.f, 0.f);
            __syncthreads();
            if (threadIdx.x < tn) tp[threadIdx.x] = xl[t0 + threadIdx.x];
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const int sx = ix + dx, sy = iy + dy;
                    if (sx < 0 || sy < 0 || sx >= m || sy >= m) continue;
                    const uint32_t s = morton((uint32_t)sx, (uint32_t)sy);
                    const int32_t slo = lb[s], shi = lb[s + 1];
                    const float ox = (float)(-dx) * h, oy = (float)(-dy) * h;   // c_T - c_S
                    for (int32_t s0 = slo; s0 < shi; s0 += P2T) {
                        const int sn = min(P2T, shi - s0);
                        __syncthreads();
                        if (threadIdx.x < sn) sp[threadIdx.x] = xl[s0 + threadIdx.x];
                        for (int e = threadIdx.x; e < P2R * P2T; e += blockDim.x) {
                            const int rr = e / P2T, j = e % P2T;
                            Q[rr][j] = (rr < nr && j < sn) ? qs[(int64_t)(r0 + rr) * n + s0 + j] : cfmk(0.f, 0.f);
                        }
                        __syncthreads();
                        for (int e = threadIdx.x; e < P2T * P2T; e += blockDim.x) {
                            const int i = e / P2T, j = e % P2T;
                            cf g = cfmk(0.f, 0.f);
                            if (i < tn && j < sn && (t0 + i) != (s0 + j)) {
                                const float ddx = ox + (tp[i].x - sp[j].x);
                                const float ddy = oy + (tp[i].y - sp[j].y);
                                const float z = k * sqrtf(ddx * ddx + ddy * ddy);
                                if (z < H0_ZMAX) {
                                    const int iv = min((int)(z * H0_INV_DZ), H0_NI - 1);
                                    const float t = (z - ((float)iv + 0.5f) / H0_INV_DZ) * (2.0f * H0_INV_DZ);
                                    float jj = tj[iv][H0_DEG], rr2 = tr[iv][H0_DEG];
#pragma unroll
                                    for (int d = H0_DEG - 1; d >= 0; --d) {
                                        jj = fmaf(jj, t, tj[iv][d]);
                                        rr2 = fmaf(rr2, t, tr[iv][d]);
                                    }
                                    const float y = fmaf(0.63661977236758134f * logf(0.5f * z), jj, rr2);
                                    g = cfmk(-0.25f * y, 0.25f * jj);
                                } else {
                                    cd h0 = hankel0((double)z);
                                    g = cfmk((float)(-0.25 * h0.y), (float)(0.25 * h0.x));
                                }
                            }
                            G[i][j] = g;
                        }
                        __syncthreads();
#pragma unroll 4
                        for (int j = 0; j < P2T; ++j) {
                            const cf g0 = G[2 * tpair][j], g1 = G[2 * tpair + 1][j];
#pragma unroll
                            for (int c = 0; c < 4; ++c) {
                                const cf qv = Q[4 * rg + c][j];
                                cfma32(acc[0][c], g0, qv);
                                cfma32(acc[1][c], g1, qv);
                            }
                        }
                    }
                }
            for (int a = 0; a < 2; ++a) {
                const int i = 2 * tpair + a;
                if (i >= tn) continue;
                for (int c = 0; c < 4; ++c) {
                    const int rr = 4 * rg + c;
                    if (rr >= nr) continue;
                    cf* yy = ys + (int64_t)(r0 + rr) * n + t0 + i;
                    yy->x += acc[a][c].x;
                    yy->y += acc[a][c].y;
                }
            }
        }
    }
}

// P2P free-space part in FP32
constexpr int PT = 32;
constexpr int P2P_THREADS = 256;
constexpr int P2P_RHS = 64;
constexpr int P2P_ITEMS = P2P_RHS * PT / P2P_THREADS;   // 8

__global__ void __launch_bounds__(P2P_THREADS) p2p32_kernel(const int32_t* lb, int L, const double2* xs,
                                                            const cf* qs, int64_t n, int nrhs, double k,
                                                            cf* ys) {
    __shared__ cf G[PT][PT + 1];
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
            cf acc[P2P_ITEMS];
            for (int u = 0; u < P2P_ITEMS; ++u) acc[u] = cfmk(0.f, 0.f);
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
                            cf g = cfmk(0.f, 0.f);
                            if (i < tn && j < sn && (t0 + i) != (s0 + j)) {
                                // coordinates differences in FP64, distance rounded to FP32
                                const double r = hypot(tp[i].x - sp[j].x, tp[i].y - sp[j].y);
                                const double z = k * r;
                                if (z < (double)H0_ZMAX) {
                                    g = green_free_f32((float)z);
                                } else {
                                    cd h0 = hankel0(z);
                                    g = cfmk((float)(-0.25 * h0.y), (float)(0.25 * h0.x));
                                }
                            }
                            G[i][j] = g;
                        }
                        __syncthreads();
                        for (int u = 0; u < P2P_ITEMS; ++u) {
                            const int it = u * P2P_THREADS + threadIdx.x;
                            const int rr = it / PT, i = it % PT;
                            if (rr >= nr || i >= tn) continue;
                            const cf* qr = qs + (int64_t)(r0 + rr) * n + s0;
                            cf a = acc[u];
                            for (int j = 0; j < sn; ++j) cfma32(a, G[i][j], qr[j]);
                            acc[u] = a;
                        }
                    }
                }
            for (int u = 0; u < P2P_ITEMS; ++u) {
                const int it = u * P2P_THREADS + threadIdx.x;
                const int rr = it / PT, i = it % PT;
                if (rr >= nr || i >= tn) continue;
                cf* yy = ys + (int64_t)(r0 + rr) * n + t0 + i;
                yy->x += acc[u].x;
                yy->y += acc[u].y;
            }
        }
    }
}

__global__ void direct32_kernel(const int32_t* lb, const int32_t* d_begin, const int32_t* d_src,
                                const int64_t* d_blk, const cf* vals, const cf* qs, int64_t n, int nrhs,
                                cf* ys) {
    const int64_t b = blockIdx.x;
    const int32_t e0 = d_begin[b], e1 = d_begin[b + 1];
    if (e1 <= e0) return;
    const int32_t tlo = lb[b], tn = lb[b + 1] - tlo;
    const int items = nrhs * tn;
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
        const int r = it / tn, i = it % tn;
        cf acc = cfmk(0.f, 0.f);
        for (int32_t e = e0; e < e1; ++e) {
            const int32_t s = d_src[e];
            const int32_t slo = lb[s], sn = lb[s + 1] - slo;
            const cf* G = vals + d_blk[e] + (int64_t)i * sn;
            const cf* qr = qs + (int64_t)r * n + slo;
            for (int j = 0; j < sn; ++j) cfma32(acc, G[j], qr[j]);
        }
        cf* yy = ys + (int64_t)r * n + tlo + i;
        yy->x += acc.x;
        yy->y += acc.y;
    }
}

int pick_chunk32(int p) {
    const int ncoef = 2 * p + 1;
    int c = (int)(40000 / (ncoef * 8 + (p + 1) * 8));
    return std::max(1, std::min(32, c));
}

}  // namespace

hfmm_status init_h0_table(cudaStream_t st) {
    if (!h0_ready) {
        fit_h0_table();
        h0_ready = true;
    }
    HFMM_CUDA_TRY(cudaMemcpyToSymbolAsync(c_h0j, h_h0j, sizeof(h_h0j), 0, cudaMemcpyHostToDevice, st));
    HFMM_CUDA_TRY(cudaMemcpyToSymbolAsync(c_h0r, h_h0r, sizeof(h_h0r), 0, cudaMemcpyHostToDevice, st));
    return HFMM_OK;
}

hfmm_status build_local_coords(hfmm_plan_s* P, cudaStream_t st) {
    HFMM_TRY(plan_alloc(P, (void**)&P->xl32, sizeof(float2) * P->n));
    const LevelInfo& lv = P->lev[P->L];
    local_coords_kernel<<<(unsigned)lv.nbox, 128, 0, st>>>(P->leaf_begin, P->xy_sorted, lv.nbox, P->x0, P->y0, lv.h,
                                                           P->xl32);
    HFMM_CUDA_TRY(cudaGetLastError());
    return HFMM_OK;
}

extern "C" hfmm_status hfmm_debug_green_f32(int32_t n, const double* z, float* g) {
    if (n < 0 || (n > 0 && (!z || !g))) { hfmm_set_error("bad arguments"); return HFMM_ERR_INVALID_ARG; }
    if (!h0_ready) { fit_h0_table(); h0_ready = true; }
    for (int i = 0; i < n; ++i) {
        const float zz = (float)z[i];
        if (!(zz > 0.0f) || zz >= H0_ZMAX) { g[2 * i] = NAN; g[2 * i + 1] = NAN; continue; }
        const int iv = std::min((int)(zz * H0_INV_DZ), H0_NI - 1);
        const float t = (zz - ((float)iv + 0.5f) / H0_INV_DZ) * (2.0f * H0_INV_DZ);
        float j = h_h0j[iv][H0_DEG], r = h_h0r[iv][H0_DEG];
        for (int d = H0_DEG - 1; d >= 0; --d) {
            j = std::fma(j, t, h_h0j[iv][d]);
            r = std::fma(r, t, h_h0r[iv][d]);
        }
        const float y = std::fma(0.63661977236758134f * std::log(0.5f * zz), j, r);
        g[2 * i] = -0.25f * y;
        g[2 * i + 1] = 0.25f * j;
    }
    return HFMM_OK;
}

hfmm_status apply_mixed(hfmm_plan_s* P, int nrhs, const cf* q, cf* y, int parts, bool adjoint,
                        cudaStream_t st) {
    const int64_t n = P->n;
    const int L = P->L;
    const int nb = ceil_div(n, 256);
    StageTimer tm{P, st};
    P->launches = 0;
    for (int s = 0; s < HFMM_NUM_STAGES; ++s) { P->st_flops[s] = 0.0; P->st_bytes[s] = 0.0; P->ev_used[s] = false; }
    const double C = 8.0 * nrhs;
    const double MAC = 8.0 * nrhs;
    tm.begin(HFMM_STAGE_GATHER);
    gather_q32<<<nb, 256, 0, st>>>(q, P->perm, n, nrhs, adjoint, P->q32);
    ++P->launches;
    HFMM_CUDA_TRY(cudaMemsetAsync(P->y32, 0, sizeof(cf) * n * nrhs, st));
    tm.end(HFMM_STAGE_GATHER);
    P->st_bytes[HFMM_STAGE_GATHER] = 2.0 * C * n + 8.0 * n;
    const bool far = (parts & (HFMM_PART_FAR_FREE | HFMM_PART_FAR_REACT)) != 0;
    if (far) {
        {
            LevelInfo& lv = P->lev[L];
            const int chunk = pick_chunk32(lv.p);
            const size_t sm = (size_t)chunk * ((2 * lv.p + 1) * sizeof(cf) + (lv.p + 1) * sizeof(double));
            tm.begin(HFMM_STAGE_P2M);
            p2m32_kernel<<<(unsigned)lv.nbox, 128, sm, st>>>(P->leaf_begin, P->xy_sorted, P->q32, n, nrhs, P->x0,
                                                             P->y0, lv.h, P->k, lv.p, lv.d_log_s, chunk, lv.mult32);
            ++P->launches;
            HFMM_CUDA_TRY(cudaGetLastError());
            tm.end(HFMM_STAGE_P2M);
            P->st_flops[HFMM_STAGE_P2M] = MAC * n * lv.ncoef;
            P->st_bytes[HFMM_STAGE_P2M] = C * n + 16.0 * n + C * lv.nbox * lv.ncoef;
        }
        tm.begin(HFMM_STAGE_M2M);
        if (P->tc_on) {
            HFMM_TRY(split_mult_tc(P, L, nrhs, st));
            ++P->launches;
        }
        for (int l = L - 1; l >= P->lmin; --l) {
            LevelInfo& lv = P->lev[l];
            if (P->tc_on) {
                HFMM_TRY(launch_m2m_tc(P, l, nrhs, st));
            } else {
                m2m32_kernel<<<(unsigned)lv.nbox, 128, 0, st>>>(P->lev[l + 1].mult32, lv.t_m2m32, P->lev[l + 1].p,
                                                               lv.p, nrhs, lv.mult32);
                HFMM_CUDA_TRY(cudaGetLastError());
            }
            ++P->launches;
            P->st_flops[HFMM_STAGE_M2M] += MAC * 4.0 * lv.nbox * lv.ncoef * P->lev[l + 1].ncoef;
            P->st_bytes[HFMM_STAGE_M2M] += C * (4.0 * lv.nbox * P->lev[l + 1].ncoef + lv.nbox * lv.ncoef);
        }
        tm.end(HFMM_STAGE_M2M);
        tm.begin(HFMM_STAGE_DOWN);
        // the tensor-core pass fuses both far parts of a level; subsets run on SIMT cores
        const bool tc_down = P->tc_on && (parts & HFMM_PART_FAR_FREE) && (parts & HFMM_PART_FAR_REACT);
        for (int l = P->lmin; l <= L; ++l) {
            LevelInfo& lv = P->lev[l];
            const bool has_parent = l > P->lmin;
            const int npp = has_parent ? P->lev[l - 1].ncoef : 0;
            const int wmax = std::max(lv.ncoef, npp);
            // right-hand sides per pass: staged a~ fits 32 KB, items <= 8 per thread
            int rc = std::max(1, std::min(nrhs, (int)(32768 / (wmax * sizeof(cf)))));
            rc = std::max(1, std::min(rc, (8 * DOWN_THREADS) / lv.ncoef));
            const size_t sm = (size_t)rc * wmax * sizeof(cf);
            if (tc_down) {
                HFMM_TRY(launch_m2l_tc(P, l, nrhs, st));
            } else {
                down32_kernel<<<(unsigned)lv.nbox, DOWN_THREADS, sm, st>>>(
                    P->leaf_begin, L, l, P->lmin, nrhs, lv.p, has_parent ? P->lev[l - 1].p : 0,
                    has_parent ? P->lev[l - 1].loc32 : nullptr, has_parent ? P->lev[l - 1].t_l2l32 : nullptr,
                    lv.mult32, lv.nv ? lv.v_begin : nullptr, lv.v_src, lv.v_off, lv.t_free32,
                    lv.nr ? lv.r_begin : nullptr, lv.r_src, lv.r_tab, lv.t_react32, parts, rc, lv.loc32);
            }
            ++P->launches;
            HFMM_CUDA_TRY(cudaGetLastError());
            double pairs = 0.0;
            if (parts & HFMM_PART_FAR_FREE) pairs += (double)lv.nv;
            if (parts & HFMM_PART_FAR_REACT) pairs += (double)lv.nr;
            P->st_flops[HFMM_STAGE_DOWN] += MAC * pairs * lv.ncoef * lv.ncoef;
            if (has_parent) P->st_flops[HFMM_STAGE_DOWN] += MAC * lv.nbox * lv.ncoef * npp;
            P->st_bytes[HFMM_STAGE_DOWN] += C * lv.nbox * lv.ncoef * 2.0 +
                                            (has_parent ? C * P->lev[l - 1].nbox * npp : 0.0);
        }
        tm.end(HFMM_STAGE_DOWN);
        {
            LevelInfo& lv = P->lev[L];
            const int chunk = pick_chunk32(lv.p);
            const size_t sm = (size_t)chunk * ((2 * lv.p + 1) * sizeof(cf) + (lv.p + 1) * sizeof(double));
            tm.begin(HFMM_STAGE_L2P);
            l2p32_kernel<<<(unsigned)lv.nbox, 128, sm, st>>>(P->leaf_begin, P->xy_sorted, lv.loc32, n, nrhs, P->x0,
                                                             P->y0, lv.h, P->k, lv.p, lv.d_log_s, chunk, P->y32);
            ++P->launches;
            HFMM_CUDA_TRY(cudaGetLastError());
            tm.end(HFMM_STAGE_L2P);
            P->st_flops[HFMM_STAGE_L2P] = MAC * n * lv.ncoef;
            P->st_bytes[HFMM_STAGE_L2P] = C * lv.nbox * lv.ncoef + 16.0 * n + 2.0 * C * n;
        }
    }
    if (parts & HFMM_PART_NEAR_FREE) {
        tm.begin(HFMM_STAGE_P2P);
        p2p32b_kernel<<<(unsigned)P->lev[L].nbox, P2_THREADS, 0, st>>>(P->leaf_begin, L, P->xl32, P->q32, n, nrhs,
                                                                       (float)P->k, (float)P->lev[L].h, P->y32);
        ++P->launches;
        HFMM_CUDA_TRY(cudaGetLastError());
        tm.end(HFMM_STAGE_P2P);
        P->st_flops[HFMM_STAGE_P2P] = MAC * (double)P->p2p_point_pairs;
        P->st_bytes[HFMM_STAGE_P2P] = 3.0 * C * n + 16.0 * n;
    }
    if ((parts & HFMM_PART_NEAR_REACT) && P->nd > 0) {
        tm.begin(HFMM_STAGE_DIRECT);
        direct32_kernel<<<(unsigned)P->lev[L].nbox, 128, 0, st>>>(P->leaf_begin, P->d_begin, P->d_src, P->d_blk,
                                                                  P->d_vals32, P->q32, n, nrhs, P->y32);
        ++P->launches;
        HFMM_CUDA_TRY(cudaGetLastError());
        tm.end(HFMM_STAGE_DIRECT);
        P->st_flops[HFMM_STAGE_DIRECT] = MAC * (double)P->nd_vals;
        P->st_bytes[HFMM_STAGE_DIRECT] = 8.0 * (double)P->nd_vals;
    }
    tm.begin(HFMM_STAGE_SCATTER);
    scatter_y32<<<nb, 256, 0, st>>>(P->y32, P->perm, n, nrhs, adjoint, y);
    ++P->launches;
    HFMM_CUDA_TRY(cudaGetLastError());
    tm.end(HFMM_STAGE_SCATTER);
    P->st_bytes[HFMM_STAGE_SCATTER] = 2.0 * C * n + 8.0 * n;
    P->last_stream = st;
    return HFMM_OK;
}
