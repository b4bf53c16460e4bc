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
#include "tcgen05.cuh"

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

// Sorted FP32 strengths and fields are point-major, [n][nrhs].  Gather and
// scatter move one tile of 64 consecutive caller indices: the caller side
// ([nrhs][n]) is read / written along the points, the sorted side along the
// right-hand sides of each point (iperm: sorted position of caller index j).
constexpr int TP_PTS = 64;

constexpr int TP_THREADS = 256;
constexpr int TP_PER = TP_PTS * TP_PTS / TP_THREADS;   // elements per thread and pass

// Each pass moves a 64 x 64 tile: all loads of a thread are issued before its
// shared-memory stores (16 independent 8-byte loads in flight per thread).
// With qmax given, also the largest |Re q|, |Im q| of every right-hand side
// (float bits, an integer max: the values are non-negative; qmax zeroed before).
__global__ void __launch_bounds__(TP_THREADS) gather_q32(const cf* __restrict__ q, const int32_t* __restrict__ iperm,
                                                         int64_t n, int nrhs, bool conj_in, cf* __restrict__ qs,
                                                         unsigned* __restrict__ qmax) {
    __shared__ cf T[TP_PTS][TP_PTS + 1];
    __shared__ unsigned smax[TP_PTS];
    const int64_t j0 = (int64_t)blockIdx.x * TP_PTS;
    const int jn = (int)min((int64_t)TP_PTS, n - j0);
    for (int r0 = 0; r0 < nrhs; r0 += TP_PTS) {
        const int rn = min(TP_PTS, nrhs - r0);
        cf v[TP_PER];
#pragma unroll
        for (int u = 0; u < TP_PER; ++u) {
            const int e = threadIdx.x + u * TP_THREADS, rr = e / TP_PTS, jj = e % TP_PTS;
            v[u] = (rr < rn && jj < jn) ? q[(int64_t)(r0 + rr) * n + j0 + jj] : cfmk(0.f, 0.f);
        }
        __syncthreads();   // the previous pass has read T and smax
        if (qmax && threadIdx.x < TP_PTS) smax[threadIdx.x] = 0u;
        __syncthreads();
#pragma unroll
        for (int u = 0; u < TP_PER; ++u) {
            const int e = threadIdx.x + u * TP_THREADS, rr = e / TP_PTS, jj = e % TP_PTS;
            T[jj][rr] = conj_in ? cfmk(v[u].x, -v[u].y) : v[u];
        }
        __syncthreads();
        // every element of a thread below has right-hand side threadIdx.x % 64
        float m = 0.0f;
#pragma unroll
        for (int u = 0; u < TP_PER; ++u) {
            const int e = threadIdx.x + u * TP_THREADS, jj = e / TP_PTS, rr = e % TP_PTS;
            const cf w = T[jj][rr];
            m = fmaxf(m, fmaxf(fabsf(w.x), fabsf(w.y)));
            if (jj < jn && rr < rn) qs[(int64_t)iperm[j0 + jj] * nrhs + r0 + rr] = w;
        }
        if (qmax) {
            if (m > 0.0f) atomicMax(&smax[threadIdx.x % TP_PTS], __float_as_uint(m));
            __syncthreads();
            if (threadIdx.x < rn && smax[threadIdx.x] > 0u) atomicMax(&qmax[r0 + threadIdx.x], smax[threadIdx.x]);
        }
    }
}
__global__ void __launch_bounds__(TP_THREADS) scatter_y32(const cf* __restrict__ ys, const int32_t* __restrict__ iperm,
                                                          int64_t n, int nrhs, bool conj_out, cf* __restrict__ y) {
    __shared__ cf T[TP_PTS][TP_PTS + 1];
    const int64_t j0 = (int64_t)blockIdx.x * TP_PTS;
    const int jn = (int)min((int64_t)TP_PTS, n - j0);
    for (int r0 = 0; r0 < nrhs; r0 += TP_PTS) {
        const int rn = min(TP_PTS, nrhs - r0);
        cf v[TP_PER];
#pragma unroll
        for (int u = 0; u < TP_PER; ++u) {
            const int e = threadIdx.x + u * TP_THREADS, jj = e / TP_PTS, rr = e % TP_PTS;
            v[u] = (jj < jn && rr < rn) ? ys[(int64_t)iperm[j0 + jj] * nrhs + r0 + rr] : cfmk(0.f, 0.f);
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < TP_PER; ++u) {
            const int e = threadIdx.x + u * TP_THREADS, jj = e / TP_PTS, rr = e % TP_PTS;
            T[jj][rr] = v[u];
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < TP_PER; ++u) {
            const int e = threadIdx.x + u * TP_THREADS, rr = e / TP_PTS, jj = e % TP_PTS;
            if (rr < rn && jj < jn) {
                const cf w = T[jj][rr];
                y[(int64_t)(r0 + rr) * n + j0 + jj] = conj_out ? cfmk(w.x, -w.y) : w;
            }
        }
    }
}
__global__ void iperm_kernel(const int64_t* perm, int64_t n, int32_t* iperm) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) iperm[perm[i]] = (int32_t)i;
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

// P2P free-space part, FP32 (Algorithm 1, step 5), fused with L2P (step 4):
// one CTA of 128 threads per non-empty target leaf.  Thread (r, half) owns right-hand side r of a
// 64-wide block and NTH consecutive targets of a pass of up to 32 targets
// (NTH = 4, 8, 12 or 16 from the pass width, so little padding is computed).
// Sources are streamed per neighbour leaf in chunks of up to 32 points: their
// strengths [j][r] and the (i/4) H0 values [j][t] of the chunk are staged in
// shared memory, and the inner loop runs over the chunk's real length; the G
// reads are warp-wide broadcasts.  The leaf's local expansion enters the same
// product as extra chunks.  Results go through shared memory so the
// read-modify-write of y is coalesced along the points.
constexpr int PC_THREADS = 128;
constexpr int PC_SRC = 32;         // sources per chunk
constexpr int PC_TGT = 32;         // targets per pass
constexpr int PC_RHS = 64;         // right-hand sides per block

struct PcShared {
    cf q[PC_SRC][PC_RHS + 1];      // strengths of the chunk; reused as y staging [t][r]
    __align__(16) cf g[PC_SRC][PC_TGT];
    float2 tp[PC_TGT];
    float tj[H0_NI][H0_DEG + 1];
    float tr[H0_NI][H0_DEG + 1];
};

__device__ __forceinline__ cf green_free_f32_tab(const PcShared& S, float z) {
    const int iv = min((int)(z * H0_INV_DZ), H0_NI - 1);
    const float t = (z - ((float)iv + 0.5f) / H0_INV_DZ) * (2.0f * H0_INV_DZ);
    float jj = S.tj[iv][H0_DEG], rr = S.tr[iv][H0_DEG];
#pragma unroll
    for (int d = H0_DEG - 1; d >= 0; --d) {
        jj = fmaf(jj, t, S.tj[iv][d]);
        rr = fmaf(rr, t, S.tr[iv][d]);
    }
    const float y = fmaf(0.63661977236758134f * logf(0.5f * z), jj, rr);
    return cfmk(-0.25f * y, 0.25f * jj);
}

// acc[i] += sum_{j < sn} S.g[j][tb + i] * S.q[j][r]
template <int NTH, class SH>
__device__ __forceinline__ void pc_mac(const SH& S, int sn, int r, int tb, cf* acc) {
#pragma unroll 2
    for (int j = 0; j < sn; ++j) {
        const cf qv = S.q[j][r];
        const float4* gp = (const float4*)&S.g[j][tb];
#pragma unroll
        for (int i = 0; i < NTH; i += 2) {
            const float4 g2 = gp[i >> 1];
            cfma32(acc[i], cfmk(g2.x, g2.y), qv);
            cfma32(acc[i + 1], cfmk(g2.z, g2.w), qv);
        }
    }
}

template <int NTH>
__device__ __forceinline__ void p2p_pass(PcShared& S, const int32_t* lb, int L, int64_t b, int ix, int iy,
                                         const float2* xl, const cf* qs, int64_t n, int nrhs, int r0, int32_t t0,
                                         int w, float k, float h, bool near, const cf* loc, const cf* basis,
                                         int nc, cf* ys) {
    const int tid = threadIdx.x;
    const int r = tid & (PC_RHS - 1), half = tid >> 6;
    const int tb = half * NTH;                       // first target of this thread
    const int m = 1 << L;
    cf acc[NTH];
#pragma unroll
    for (int i = 0; i < NTH; ++i) acc[i] = cfmk(0.f, 0.f);
    __syncthreads();
    if (tid < w) S.tp[tid] = xl[t0 + tid];
    for (int dy = -1; dy <= 1 && near; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
            const int sx = ix + dx, sy = iy + dy;
            if (sx < 0 || sy < 0 || sx >= m || sy >= m) continue;
            const uint32_t s = morton((uint32_t)sx, (uint32_t)sy);
            const int32_t slo = lb[s], shi = lb[s + 1];
            const float ox = (float)(-dx) * h, oy = (float)(-dy) * h;   // c_T - c_S
            for (int32_t s0 = slo; s0 < shi; s0 += PC_SRC) {
                const int sn = min(PC_SRC, shi - s0);
                __syncthreads();
                // strengths: consecutive threads take consecutive RHS of one point
                for (int e = tid; e < sn * PC_RHS; e += PC_THREADS) {
                    const int j = e >> 6, rr = e & (PC_RHS - 1);
                    S.q[j][rr] = (r0 + rr < nrhs) ? qs[(int64_t)(s0 + j) * nrhs + r0 + rr] : cfmk(0.f, 0.f);
                }
                for (int e = tid; e < sn * w; e += PC_THREADS) {
                    const int j = e / w, t = e - j * w;
                    cf g = cfmk(0.f, 0.f);
                    if (t0 + t != s0 + j) {
                        const float2 sp = xl[s0 + j];
                        const float ddx = ox + (S.tp[t].x - sp.x);
                        const float ddy = oy + (S.tp[t].y - sp.y);
                        const float z = k * sqrtf(ddx * ddx + ddy * ddy);
                        if (z < H0_ZMAX) {
                            g = green_free_f32_tab(S, z);
                        } else {
                            const cd h0 = hankel0((double)z);
                            g = cfmk((float)(-0.25 * h0.y), (float)(0.25 * h0.x));
                        }
                    }
                    S.g[j][t] = g;
                }
                __syncthreads();
                pc_mac<NTH, PcShared>(S, sn, r, tb, acc);
            }
        }
    if (loc) {
        // L2P (Algorithm 1, step 4) as more staged chunks of the same product:
        // "strengths" beta~[r][m] of the leaf, "kernel" (i/4) conj(B[t][m])
        for (int m0 = 0; m0 < nc; m0 += PC_SRC) {
            const int mb = min(PC_SRC, nc - m0);
            __syncthreads();
            for (int e = tid; e < mb * PC_RHS; e += PC_THREADS) {
                const int rr = e / mb, j = e - rr * mb;
                S.q[j][rr] = (r0 + rr < nrhs) ? loc[((int64_t)b * nrhs + r0 + rr) * nc + m0 + j] : cfmk(0.f, 0.f);
            }
            for (int e = tid; e < mb * w; e += PC_THREADS) {
                const int t = e / mb, j = e - t * mb;
                const cf B = basis[(int64_t)(t0 + t) * nc + m0 + j];
                S.g[j][t] = cfmk(0.25f * B.y, 0.25f * B.x);
            }
            __syncthreads();
            pc_mac<NTH, PcShared>(S, mb, r, tb, acc);
        }
    }
    // stage y[t][r] in shared memory, then add it to y along the points
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NTH; ++i)
        if (tb + i < w) S.q[tb + i][r] = acc[i];
    __syncthreads();
    for (int e = tid; e < w * PC_RHS; e += PC_THREADS) {
        const int t = e >> 6, rr = e & (PC_RHS - 1);
        if (r0 + rr < nrhs) {
            cf* yy = ys + (int64_t)(t0 + t) * nrhs + r0 + rr;
            const cf a = S.q[t][rr];
            yy->x += a.x;
            yy->y += a.y;
        }
    }
}

__global__ void __launch_bounds__(PC_THREADS, 6) p2p32c_kernel(const int32_t* lb, int L, const float2* xl,
                                                            const cf* qs, int64_t n, int nrhs, float k,
                                                            float h, int near, const cf* loc,
                                                            const cf* basis, int nc, const int32_t* leaves,
                                                            cf* ys) {
    __shared__ PcShared S;
    const int64_t b = leaves ? (int64_t)leaves[blockIdx.x] : (int64_t)blockIdx.x;
    const int32_t tlo = lb[b], thi = lb[b + 1];
    if (thi <= tlo) return;
    for (int e = threadIdx.x; e < H0_NI * (H0_DEG + 1); e += blockDim.x) {
        S.tj[e / (H0_DEG + 1)][e % (H0_DEG + 1)] = c_h0j[e / (H0_DEG + 1)][e % (H0_DEG + 1)];
        S.tr[e / (H0_DEG + 1)][e % (H0_DEG + 1)] = c_h0r[e / (H0_DEG + 1)][e % (H0_DEG + 1)];
    }
    const int ix = (int)morton_x((uint32_t)b), iy = (int)morton_y((uint32_t)b);
    for (int r0 = 0; r0 < nrhs; r0 += PC_RHS)
        for (int32_t t0 = tlo; t0 < thi; t0 += PC_TGT) {
            const int w = min(PC_TGT, thi - t0);
            if (w <= 8) p2p_pass<4>(S, lb, L, b, ix, iy, xl, qs, n, nrhs, r0, t0, w, k, h, near, loc, basis, nc, ys);
            else if (w <= 16) p2p_pass<8>(S, lb, L, b, ix, iy, xl, qs, n, nrhs, r0, t0, w, k, h, near, loc, basis, nc, ys);
            else if (w <= 24) p2p_pass<12>(S, lb, L, b, ix, iy, xl, qs, n, nrhs, r0, t0, w, k, h, near, loc, basis, nc, ys);
            else p2p_pass<16>(S, lb, L, b, ix, iy, xl, qs, n, nrhs, r0, t0, w, k, h, near, loc, basis, nc, ys);
        }
}

// P2M, FP32 (Algorithm 1, step 1): one CTA of 128 threads per leaf computes
// the scaled multipoles a~[r][m] = sum over the leaf's points of
// q_r(pt) B[pt][m] with the plan-time basis B.  Same tiling as the P2P pass:
// thread (r, half) owns NTH coefficients of a pass of up to 32, points are
// streamed in chunks of 32 (strengths [j][r], basis [j][m] in shared memory).
// P2M's shared staging: the P2P tables are not needed.
struct P2mShared {
    cf q[PC_SRC][PC_RHS + 1];      // strengths of the chunk; reused as output staging [m][r]
    __align__(16) cf g[PC_SRC][PC_TGT];
};

template <int NTH>
__device__ __forceinline__ void p2m_pass(P2mShared& S, const cf* qs, const cf* basis, int64_t n, int nrhs, int r0,
                                         int32_t lo, int32_t hi, int nc, int m0, int w, cf* out, bool write_out) {
    const int tid = threadIdx.x;
    const int r = tid & (PC_RHS - 1), half = tid >> 6;
    const int tb = half * NTH;
    cf acc[NTH];
#pragma unroll
    for (int i = 0; i < NTH; ++i) acc[i] = cfmk(0.f, 0.f);
    for (int32_t s0 = lo; s0 < hi; s0 += PC_SRC) {
        const int sn = min(PC_SRC, hi - s0);
        __syncthreads();
        for (int e = tid; e < sn * PC_RHS; e += PC_THREADS) {
            const int j = e >> 6, rr = e & (PC_RHS - 1);
            S.q[j][rr] = (r0 + rr < nrhs) ? qs[(int64_t)(s0 + j) * nrhs + r0 + rr] : cfmk(0.f, 0.f);
        }
        for (int e = tid; e < sn * w; e += PC_THREADS) {
            const int j = e / w, t = e - j * w;
            S.g[j][t] = basis[(int64_t)(s0 + j) * nc + m0 + t];
        }
        __syncthreads();
        pc_mac<NTH, P2mShared>(S, sn, r, tb, acc);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NTH; ++i)
        if (tb + i < w) S.q[tb + i][r] = acc[i];
    __syncthreads();
    if (write_out)
        for (int e = tid; e < w * PC_RHS; e += PC_THREADS) {
            const int rr = e / w, t = e - rr * w;
            if (r0 + rr < nrhs) out[(int64_t)(r0 + rr) * nc + m0 + t] = S.q[t][rr];
        }
}

// Writes mult[b] and, when amma is given, its MMA-ready copy for the
// tensor-core M2M and M2L of the leaf level: f16 hi / lo, 4 KB blocks of 64
// rows x 16 K (parts interleaved per 8-row group; Re then Im, zero padding)
// per K chunk, every (row, column block
// of sblk chunks) scaled by the power of two 2^e that puts its largest entry
// in [2^14, 2^15), with 2^-e stored in asc[((b * nrc + rc) * nsb + block) * 64 + row].
// mult is written when write_mult (the SIMT passes read it) or when nc > 32
// (the MMA-ready copy is then built from it); otherwise the MMA-ready copy is
// built from the pass's shared-memory staging.
__global__ void __launch_bounds__(PC_THREADS) p2m32c_kernel(const int32_t* lb, const cf* qs, const cf* basis,
                                                            int64_t n, int nrhs, int nc, cf* mult, __half* amma,
                                                            float* asc, int kc, int nrc, int nsb, int sblk,
                                                            bool write_mult) {
    __shared__ P2mShared S;
    // [column block][row] exponents (consecutive rows in consecutive banks), in the
    // basis staging, which the MMA-ready writer no longer needs
    static_assert(sizeof(S.g) >= 16 * PC_RHS * sizeof(int), "exponents fit the basis staging");
    int (*s_e)[PC_RHS] = reinterpret_cast<int (*)[PC_RHS]>(&S.g[0][0]);
    const int64_t b = blockIdx.x;
    const int32_t lo = lb[b], hi = lb[b + 1];
    cf* out = mult + (int64_t)b * nrhs * nc;
    const bool from_smem = amma && nc <= PC_TGT;   // one pass: all coefficients staged in S.q
    const bool wo = write_mult || !from_smem;
    for (int r0 = 0; r0 < nrhs; r0 += PC_RHS) {
        for (int m0 = 0; m0 < nc; m0 += PC_TGT) {
            const int w = min(PC_TGT, nc - m0);
            if (w <= 8) p2m_pass<4>(S, qs, basis, n, nrhs, r0, lo, hi, nc, m0, w, out, wo);
            else if (w <= 16) p2m_pass<8>(S, qs, basis, n, nrhs, r0, lo, hi, nc, m0, w, out, wo);
            else if (w <= 24) p2m_pass<12>(S, qs, basis, n, nrhs, r0, lo, hi, nc, m0, w, out, wo);
            else p2m_pass<16>(S, qs, basis, n, nrhs, r0, lo, hi, nc, m0, w, out, wo);
        }
        if (amma) {
            __syncthreads();   // this block's rows of mult are written
            const int rc = r0 / PC_RHS;
            // the 16 real values of K chunk c of row r (Re a_0 .. a_{nc-1}, Im ..., zero padding)
            auto load16 = [&](int r, int c, float (&v)[16]) {
                const bool live = r0 + r < nrhs;
                const float* row = (const float*)(out + (int64_t)(r0 + r) * nc);
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const int k = c * 16 + u;
                    if (!live || k >= 2 * nc) v[u] = 0.0f;
                    else if (from_smem) v[u] = k < nc ? S.q[k][r].x : S.q[k - nc][r].y;
                    else v[u] = k < nc ? row[2 * k] : row[2 * (k - nc) + 1];
                }
            };
            // largest |entry| of every (row, column block), by integer max of the float bits
            for (int e = threadIdx.x; e < PC_RHS * 16; e += PC_THREADS) s_e[e >> 6][e & 63] = 0;
            __syncthreads();
            for (int e = threadIdx.x; e < PC_RHS * kc; e += PC_THREADS) {
                const int r = e & (PC_RHS - 1), c = e >> 6;
                float v[16];
                load16(r, c, v);
                float m = 0.0f;
#pragma unroll
                for (int u = 0; u < 16; ++u) m = fmaxf(m, fabsf(v[u]));
                if (m > 0.0f) atomicMax(&s_e[c / sblk][r], __float_as_int(m));
            }
            __syncthreads();
            for (int e = threadIdx.x; e < PC_RHS * nsb; e += PC_THREADS) {
                const int r = e & (PC_RHS - 1), blk = e >> 6;
                const int ex = tc::f16_exp(__int_as_float(s_e[blk][r]));
                s_e[blk][r] = ex;
                asc[(((int64_t)b * nrc + rc) * nsb + blk) * 64 + r] = tc::pow2f(-ex);
            }
            __syncthreads();
            // scaled hi / lo of the chunk: two 16-byte core rows per part
            for (int e = threadIdx.x; e < PC_RHS * kc; e += PC_THREADS) {
                const int r = e & (PC_RHS - 1), c = e >> 6;
                float v[16];
                load16(r, c, v);
                const float s = tc::pow2f(s_e[c / sblk][r]);
                uint16_t* d = (uint16_t*)amma + ((b * nrc + rc) * kc + c) * 2048 + (r >> 3) * 256 + (r & 7) * 8;
#pragma unroll
                for (int hf = 0; hf < 2; ++hf) {
                    uint16_t h[8], l[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) tc::split_f16(v[hf * 8 + u] * s, h[u], l[u]);
                    *(uint4*)(d + hf * 64) = tc::pack8(h);
                    *(uint4*)(d + hf * 64 + 128) = tc::pack8(l);
                }
            }
            __syncthreads();   // s_e is reused by the next RHS block
        }
    }
}

// P2M of the leaves with the MMA-ready output, one row per thread: a CTA of 64
// threads per (leaf, block of 64 right-hand sides); thread r accumulates row r
// of the leaf's scaled multipole (Eq. (multi_coeff)) in registers over the
// leaf's points, which come into shared memory 32 at a time by asynchronous
// copies (the strengths by the thread that uses them, the basis rows by all),
// then writes its own row's f16 hi / lo K chunks and 2^-e factors (layout of
// p2m32c_kernel) and, when write_mult, the FP32 row.  No CTA-wide pass follows
// the accumulation, so the short per-leaf chain overlaps across the many CTAs
// an SM holds.  The terms are added in the order of p2m32c_kernel (points in
// ascending order), so the FP32 rows are the same bits; with qmax given the
// f16 split takes the level-wide exponent instead of the row's own.  nc <= NCM,
// NCM a multiple of 8.
constexpr int PR_SRC = 32;
template <int NCM>
__global__ void __launch_bounds__(64) p2m_rows_kernel(const int32_t* lb, const cf* qs, const cf* basis, int nrhs,
                                                      int nc, cf* mult, __half* amma, float* asc, int kc, int nrc,
                                                      int nsb, int sblk, bool write_mult, const unsigned* qmax,
                                                      float gain) {
    static_assert(NCM % 8 == 0 && NCM <= 32, "row staging holds the padded K chunks");
    __shared__ union {
        cf q[PR_SRC][64];
        float row[64][2 * NCM + 1];   // odd stride: one bank per thread
    } S;
    __shared__ __align__(16) cf g[PR_SRC][NCM];
    const int r = threadIdx.x, rc = blockIdx.y, r0 = rc * 64;
    const int64_t b = blockIdx.x;
    const int32_t lo = lb[b], hi = lb[b + 1];
    const bool live = r0 + r < nrhs;
    cf acc[NCM];
#pragma unroll
    for (int m = 0; m < NCM; ++m) acc[m] = cfmk(0.f, 0.f);
    for (int32_t s0 = lo; s0 < hi; s0 += PR_SRC) {
        const int sn = min(PR_SRC, hi - s0);
        __syncthreads();   // the previous chunk's basis rows are consumed
        for (int j = 0; j < sn; ++j) {
            if (live) tc::cp_async8(&S.q[j][r], qs + (int64_t)(s0 + j) * nrhs + r0 + r);
            else S.q[j][r] = cfmk(0.f, 0.f);
        }
        const cf* gs = basis + (int64_t)s0 * nc;
        for (int e = r; e < sn * nc; e += 64) {
            const int j = e / nc;
            tc::cp_async8(&g[j][e - j * nc], gs + e);
        }
        tc::cp_async_wait_all();
        __syncthreads();   // every thread's basis copies have landed
        for (int j = 0; j < sn; ++j) {
            const cf qv = S.q[j][r];
            const float4* gp = (const float4*)&g[j][0];
#pragma unroll
            for (int m = 0; m < NCM; m += 2)
                if (m < nc) {
                    const float4 g2 = gp[m >> 1];
                    cfma32(acc[m], cfmk(g2.x, g2.y), qv);
                    if (m + 1 < nc) cfma32(acc[m + 1], cfmk(g2.z, g2.w), qv);
                }
        }
    }
    __syncthreads();   // S.q becomes the row staging
    float* row = S.row[r];
#pragma unroll
    for (int m = 0; m < NCM; ++m)
        if (m < nc) {
            row[m] = acc[m].x;
            row[nc + m] = acc[m].y;
        }
    for (int k = 2 * nc; k < kc * 16; ++k) row[k] = 0.f;
    const int64_t rb = b * nrc + rc;
    // level-wide scale (qmax given): the exponent of the bound
    // |a~_m| <= sum_j |q_j| |B[j][m]| <= sqrt(2) max(|Re q|, |Im q|) gain, with
    // a factor 2 (sqrt(2) and the FP32 rounding of the sum), the same for every leaf
    const int ex_all = qmax ? (live ? tc::f16_exp(2.0f * __uint_as_float(qmax[r0 + r]) * gain) : 0) : 0;
    for (int blk = 0; blk < nsb; ++blk) {
        const int c0 = blk * sblk, c1 = min(kc, c0 + sblk);
        float mx = 0.f;
        if (!qmax)
            for (int k = c0 * 16; k < c1 * 16; ++k) mx = fmaxf(mx, fabsf(row[k]));
        const int ex = qmax ? ex_all : tc::f16_exp(mx);
        asc[(rb * nsb + blk) * 64 + r] = tc::pow2f(-ex);
        const float s = tc::pow2f(ex);
        for (int c = c0; c < c1; ++c) {
            uint16_t* d = (uint16_t*)amma + (rb * kc + c) * 2048 + (r >> 3) * 256 + (r & 7) * 8;
#pragma unroll
            for (int hf = 0; hf < 2; ++hf) {
                uint16_t h[8], l[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) tc::split_f16(row[c * 16 + hf * 8 + u] * s, h[u], l[u]);
                *(uint4*)(d + hf * 64) = tc::pack8(h);
                *(uint4*)(d + hf * 64 + 128) = tc::pack8(l);
            }
        }
    }
    if (write_mult && live) {
        cf* out = mult + ((int64_t)b * nrhs + r0 + r) * nc;
        for (int m = 0; m < nc; ++m) out[m] = cfmk(row[m], row[nc + m]);
    }
}

// Plan-time scaled P2M basis of every sorted point (FP64, stored in FP32).
__global__ void basis32_kernel(const int32_t* lb, const double2* xs, int64_t nleaf, double x0, double y0, double h,
                               double k, int p, const double* log_s, cf* basis) {
    extern __shared__ double jt_smem[];
    const int64_t b = blockIdx.x;
    if (b >= nleaf) return;
    const int ncoef = 2 * p + 1;
    const double cx = x0 + (morton_x((uint32_t)b) + 0.5) * h;
    const double cy = y0 + (morton_y((uint32_t)b) + 0.5) * h;
    double* Jt = jt_smem + (size_t)threadIdx.x * (p + 1);
    for (int32_t i = lb[b] + threadIdx.x; i < lb[b + 1]; i += blockDim.x)
        point_basis32(xs[i].x, xs[i].y, cx, cy, k, p, -1, log_s, Jt, basis + (int64_t)i * ncoef);
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
        const int i = it / nrhs, r = it % nrhs;
        cf acc = cfmk(0.f, 0.f);
        for (int32_t e = e0; e < e1; ++e) {
            const int32_t s = d_src[e];
            const int32_t slo = lb[s], sn = lb[s + 1] - slo;
            const cf* G = vals + d_blk[e] + (int64_t)i * sn;
            const cf* qr = qs + (int64_t)slo * nrhs + r;
            for (int j = 0; j < sn; ++j) cfma32(acc, G[j], qr[(int64_t)j * nrhs]);
        }
        cf* yy = ys + (int64_t)(tlo + i) * nrhs + r;
        yy->x += acc.x;
        yy->y += acc.y;
    }
}


}  // namespace

// Host copy of the fitted FP32 H0 table (64 intervals x 6 coefficients of J0,
// then of R0), for kernels of other translation units.
const float* h0_table_host() {
    static float both[2][H0_NI][H0_DEG + 1];
    if (!h0_ready) {
        fit_h0_table();
        h0_ready = true;
    }
    std::copy(&h_h0j[0][0], &h_h0j[0][0] + H0_NI * (H0_DEG + 1), &both[0][0][0]);
    std::copy(&h_h0r[0][0], &h_h0r[0][0] + H0_NI * (H0_DEG + 1), &both[1][0][0]);
    return &both[0][0][0];
}

hfmm_status init_h0_table(cudaStream_t st) {
    if (!h0_ready) {
        fit_h0_table();
        h0_ready = true;
    }
    HFMM_CUDA_TRY(cudaMemcpyToSymbolAsync(c_h0j, h_h0j, sizeof(h_h0j), 0, cudaMemcpyHostToDevice, st));
    HFMM_CUDA_TRY(cudaMemcpyToSymbolAsync(c_h0r, h_h0r, sizeof(h_h0r), 0, cudaMemcpyHostToDevice, st));
    return HFMM_OK;
}

// Pre-split B tiles of the tensor-core near field: row n = the n-th padded
// target of the chunk's adjacent leaves, K pair j = source point j of the
// chunk, entries (Re G, -Im G) of G = (i/4) H0(k r) times 2^NT_GSCALE_EXP,
// split into f16 hi / lo in the no-swizzle core-matrix layout (half offset
// ((n / 8) * 2 + k / 8) * 64 + (n % 8) * 8 + k % 8; lo after rows * 16 halves).
// |G| stays below 2^5 for any two distinct FP32 points (|H0(z)| reaches 128
// only for z near 1e-80), so the scaled entries stay below the f16 range.
__global__ void near_tiles_kernel(const NtChunk* __restrict__ chunks, const int64_t* __restrict__ row0, int64_t nch,
                                  int64_t total, const int32_t* __restrict__ lb, int L, const float2* __restrict__ xl,
                                  float k, float h, __half* __restrict__ tiles) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total * 8;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t gr = e >> 3;
        const int j = (int)(e & 7);
        // chunk of this global row (row0: first global row of each chunk)
        int64_t lo = 0, hi = nch - 1;
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (row0[mid] <= gr) lo = mid; else hi = mid - 1;
        }
        const NtChunk ch = chunks[lo];
        const int n = (int)(gr - row0[lo]);
        // target of row n: leaves of the mask in order, each padded to a multiple of 16
        int c = 0, t = n;
        for (c = 0; c < 4; ++c) {
            if (!(ch.mask >> c & 1)) continue;
            const int64_t lf = 4 * (int64_t)ch.par + c;
            const int w = (lb[lf + 1] - lb[lf] + 15) / 16 * 16;
            if (t < w) break;
            t -= w;
        }
        const int64_t lf = 4 * (int64_t)ch.par + c;
        const int32_t tlo = lb[lf], tn = lb[lf + 1] - tlo;
        cf g = cfmk(0.f, 0.f);
        if (c < 4 && t < tn) {
            const int32_t ti = tlo + t;
            if (j < ch.cnt && ch.src + j != ti) {
                const int32_t si = ch.src + j;
                // c_T - c_S in box units: target child c of the parent, source leaf code aux
                const float ox = (float)((c & 1) - ((ch.aux & 3) - 1)) * h;
                const float oy = (float)((c >> 1) - ((ch.aux >> 2) - 1)) * h;
                const float ddx = ox + (xl[ti].x - xl[si].x);
                const float ddy = oy + (xl[ti].y - xl[si].y);
                const float z = k * sqrtf(ddx * ddx + ddy * ddy);
                if (z < H0_ZMAX) {
                    g = green_free_f32(z);
                } else {
                    const cd h0 = hankel0((double)z);
                    g = cfmk((float)(-0.25 * h0.y), (float)(0.25 * h0.x));
                }
            }
        }
        const float sc = (float)(1 << NT_GSCALE_EXP);
        uint16_t reh, rel, imh, iml;
        tc::split_f16(g.x * sc, reh, rel);
        tc::split_f16(-g.y * sc, imh, iml);
        const int k0 = 2 * j;
        const int64_t o = ((n >> 3) * 2 + (k0 >> 3)) * 64 + (n & 7) * 8 + (k0 & 7);
        uint16_t* tile = (uint16_t*)tiles + ch.boff;
        *(uint32_t*)(tile + o) = (uint32_t)reh | ((uint32_t)imh << 16);
        *(uint32_t*)(tile + (int64_t)ch.rows * 16 + o) = (uint32_t)rel | ((uint32_t)iml << 16);
    }
}

hfmm_status fill_near_tiles(hfmm_plan_s* P, int64_t nchunks, int64_t total_rows, cudaStream_t st) {
    // first global row of every chunk
    std::vector<NtChunk> h(nchunks);
    HFMM_CUDA_TRY(cudaMemcpy(h.data(), P->nt_chunks, sizeof(NtChunk) * nchunks, cudaMemcpyDeviceToHost));
    std::vector<int64_t> r0(nchunks);
    int64_t acc = 0;
    for (int64_t i = 0; i < nchunks; ++i) { r0[i] = acc; acc += h[i].rows; }
    int64_t* d_r0 = nullptr;
    HFMM_CUDA_TRY(cudaMalloc(&d_r0, sizeof(int64_t) * std::max<int64_t>(nchunks, 1)));
    cudaError_t e = cudaMemcpy(d_r0, r0.data(), sizeof(int64_t) * nchunks, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        const LevelInfo& lv = P->lev[P->L];
        near_tiles_kernel<<<8 * 152, 256, 0, st>>>(P->nt_chunks, d_r0, nchunks, total_rows, P->leaf_begin, P->L,
                                                    P->xl32, (float)P->k, (float)lv.h, P->nt_tiles);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    cudaFree(d_r0);
    if (e != cudaSuccess) {
        hfmm_set_error("near-field tiles: %s", cudaGetErrorString(e));
        return HFMM_ERR_CUDA;
    }
    return HFMM_OK;
}

hfmm_status build_local_coords(hfmm_plan_s* P, cudaStream_t st) {
    HFMM_TRY(plan_alloc(P, (void**)&P->xl32, sizeof(float2) * P->n));
    const LevelInfo& lv = P->lev[P->L];
    local_coords_kernel<<<(unsigned)lv.nbox, 128, 0, st>>>(P->leaf_begin, P->xy_sorted, lv.nbox, P->x0, P->y0, lv.h,
                                                           P->xl32);
    HFMM_CUDA_TRY(cudaGetLastError());
    HFMM_TRY(plan_alloc(P, (void**)&P->iperm32, sizeof(int32_t) * P->n));
    iperm_kernel<<<(unsigned)ceil_div(P->n, 256), 256, 0, st>>>(P->perm, P->n, P->iperm32);
    HFMM_CUDA_TRY(cudaGetLastError());
    // P2M / L2P basis of every point, once per plan
    const size_t bb = sizeof(cf) * (size_t)P->n * lv.ncoef;
    HFMM_TRY(plan_alloc(P, (void**)&P->basis32, bb));
    P->buffer_bytes += (double)bb;
    const int thr = std::max(1, std::min(128, 6000 / (lv.p + 1)));
    basis32_kernel<<<(unsigned)lv.nbox, thr, (size_t)thr * (lv.p + 1) * sizeof(double), st>>>(
        P->leaf_begin, P->xy_sorted, lv.nbox, P->x0, P->y0, lv.h, P->k, lv.p, lv.d_log_s, P->basis32);
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

// The near field on a low-priority stream concurrently with the far-field
// chain on a high-priority one (both created on first use), forked from st
// after everything already queued there.
hfmm_status fork_near_far(hfmm_plan_s* P, cudaStream_t st) {
    if (!P->far_st) {
        int least = 0, greatest = 0;
        HFMM_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        HFMM_CUDA_TRY(cudaStreamCreateWithPriority(&P->far_st, cudaStreamNonBlocking, greatest));
        HFMM_CUDA_TRY(cudaStreamCreateWithPriority(&P->near_st, cudaStreamNonBlocking, least));
        for (cudaEvent_t* e : {&P->ev_fork, &P->ev_near_done, &P->ev_far_done})
            HFMM_CUDA_TRY(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    }
    HFMM_CUDA_TRY(cudaEventRecord(P->ev_fork, st));
    HFMM_CUDA_TRY(cudaStreamWaitEvent(P->far_st, P->ev_fork, 0));
    HFMM_CUDA_TRY(cudaStreamWaitEvent(P->near_st, P->ev_fork, 0));
    return HFMM_OK;
}

hfmm_status apply_mixed(hfmm_plan_s* P, int nrhs, const cf* q, cf* y, int parts, bool adjoint,
                        cudaStream_t st) {
    const int64_t n = P->n;
    const int L = P->L;
    StageTimer tm{P, st};
    P->launches = 0;
    for (int s = 0; s < HFMM_NUM_STAGES; ++s) { P->st_flops[s] = 0.0; P->st_bytes[s] = 0.0; P->ev_used[s] = false; }
    P->ev_leaf_used = false;
    P->leaf_flops = 0.0;
    const double C = 8.0 * nrhs;
    const double MAC = 8.0 * nrhs;
    tm.begin(HFMM_STAGE_GATHER);
    const unsigned ntile = (unsigned)ceil_div(n, TP_PTS);
    if (P->qmax) HFMM_CUDA_TRY(cudaMemsetAsync(P->qmax, 0, sizeof(unsigned) * nrhs, st));
    gather_q32<<<ntile, TP_THREADS, 0, st>>>(q, P->iperm32, n, nrhs, adjoint, P->q32, P->qmax);
    ++P->launches;
    HFMM_CUDA_TRY(cudaMemsetAsync(P->y32, 0, sizeof(cf) * n * nrhs, st));
    tm.end(HFMM_STAGE_GATHER);
    P->st_bytes[HFMM_STAGE_GATHER] = 2.0 * C * n + 8.0 * n;
    const bool far = (parts & (HFMM_PART_FAR_FREE | HFMM_PART_FAR_REACT)) != 0;
    // few right-hand sides: warp-level kernels (small.cu) instead of the tensor-core tiles
    const bool small = nrhs <= P->small_rhs && !(P->flags & HFMM_FLAG_SIMT_M2L);
    auto large_path = [&]() -> hfmm_status {
        // near free-space field and, unless the downward epilogue does it, the
        // leaves' local expansions (L2P), one fused kernel
        auto near_section = [&](bool near, bool l2p, cudaStream_t ns) -> hfmm_status {
            const LevelInfo& lv = P->lev[L];
            StageTimer tn{P, ns};
            tn.begin(HFMM_STAGE_P2P);
            if (P->tc_on) {
                // P2P: tensor-core blocks of four leaves (first writer of their targets), SIMT
                // kernel for the leaves of wider blocks; a separate L2P on the SIMT kernel
                if (near) {
                    HFMM_TRY(launch_p2p_tc(P, nrhs, ns));
                    ++P->launches;
                }
                if (P->nt_nfallback > 0 && (near || l2p)) {
                    p2p32c_kernel<<<(unsigned)P->nt_nfallback, PC_THREADS, 0, ns>>>(
                        P->leaf_begin, L, P->xl32, P->q32, n, nrhs, (float)P->k, (float)lv.h, near ? 1 : 0,
                        l2p ? lv.loc32 : nullptr, P->basis32, lv.ncoef, P->nt_fallback, P->y32);
                    ++P->launches;
                    HFMM_CUDA_TRY(cudaGetLastError());
                }
                if (l2p && P->nt_nblocks > 0) {
                    p2p32c_kernel<<<(unsigned)P->nt_nleaves, PC_THREADS, 0, ns>>>(
                        P->leaf_begin, L, P->xl32, P->q32, n, nrhs, (float)P->k, (float)lv.h, 0, lv.loc32, P->basis32,
                        lv.ncoef, P->nt_leaves, P->y32);
                    ++P->launches;
                    HFMM_CUDA_TRY(cudaGetLastError());
                }
            } else {
                p2p32c_kernel<<<(unsigned)lv.nbox, PC_THREADS, 0, ns>>>(P->leaf_begin, L, P->xl32, P->q32, n, nrhs,
                                                                        (float)P->k, (float)lv.h, near ? 1 : 0,
                                                                        l2p ? lv.loc32 : nullptr, P->basis32, lv.ncoef,
                                                                        nullptr, P->y32);
                ++P->launches;
                HFMM_CUDA_TRY(cudaGetLastError());
            }
            tn.end(HFMM_STAGE_P2P);
            P->st_flops[HFMM_STAGE_P2P] = (near ? MAC * (double)P->p2p_point_pairs : 0.0) +
                                          (l2p ? MAC * n * lv.ncoef : 0.0);
            P->st_bytes[HFMM_STAGE_P2P] = 3.0 * C * n + 16.0 * n + (l2p ? C * lv.nbox * lv.ncoef + 8.0 * n * lv.ncoef : 0.0);
            return HFMM_OK;
        };
        const bool near_free = (parts & HFMM_PART_NEAR_FREE) != 0;
        // the tensor-core pass fuses both far parts of a level; subsets run on SIMT cores
        const bool tc_down = P->tc_on && (parts & HFMM_PART_FAR_FREE) && (parts & HFMM_PART_FAR_REACT);
        // L2P in the leaf-level downward epilogue: the near field is then independent
        // of the far field until the leaves' L2P adds into y32, so it runs concurrently
        // (first writer of y32) on a low-priority stream while the far-field chain runs
        // on a high-priority one: the near field fills what the chain leaves idle (the
        // coarse levels launch few CTAs); both join before the leaf-level launch
        const bool l2p_fused = far && tc_down && P->tc_l2p;
        const bool concurrent = l2p_fused && near_free;
        cudaStream_t fs = st;
        if (concurrent) {
            HFMM_TRY(fork_near_far(P, st));
            HFMM_TRY(near_section(true, false, P->near_st));
            HFMM_CUDA_TRY(cudaEventRecord(P->ev_near_done, P->near_st));
            fs = P->far_st;
        }
        if (far) {
            StageTimer tf{P, fs};
            {
                LevelInfo& lv = P->lev[L];
                tf.begin(HFMM_STAGE_P2M);
                const int nrc = (P->max_rhs + 63) / 64;
                const int nc = lv.ncoef;
                if (P->tc_on && nc <= 32) {
                    const dim3 grid((unsigned)lv.nbox, (unsigned)((nrhs + 63) / 64));
#define HFMM_P2M_ROWS(NCM)                                                                                     \
    p2m_rows_kernel<NCM><<<grid, 64, 0, fs>>>(P->leaf_begin, P->q32, P->basis32, nrhs, nc, lv.mult32, lv.tc_amma, \
                                              lv.tc_asc, lv.tc_kc, nrc, lv.tc_nb, lv.tc_nbw / 16, !tc_down,    \
                                              P->tc_leaf_runs ? P->qmax : nullptr, P->p2m_gain)
                    if (nc <= 16) HFMM_P2M_ROWS(16);
                    else if (nc <= 24) HFMM_P2M_ROWS(24);
                    else HFMM_P2M_ROWS(32);
#undef HFMM_P2M_ROWS
                } else {
                    p2m32c_kernel<<<(unsigned)lv.nbox, PC_THREADS, 0, fs>>>(
                        P->leaf_begin, P->q32, P->basis32, n, nrhs, nc, lv.mult32, P->tc_on ? lv.tc_amma : nullptr,
                        lv.tc_asc, lv.tc_kc, nrc, lv.tc_nb, lv.tc_nbw / 16, !tc_down);
                }
                ++P->launches;
                HFMM_CUDA_TRY(cudaGetLastError());
                tf.end(HFMM_STAGE_P2M);
                P->st_flops[HFMM_STAGE_P2M] = MAC * n * lv.ncoef;
                P->st_bytes[HFMM_STAGE_P2M] = C * n + 8.0 * n * lv.ncoef + C * lv.nbox * lv.ncoef;
            }
            tf.begin(HFMM_STAGE_M2M);
            for (int l = L - 1; l >= P->lmin; --l) {
                LevelInfo& lv = P->lev[l];
                if (P->tc_on) {
                    HFMM_TRY(launch_m2m_tc(P, l, nrhs, !tc_down, fs));
                } else {
                    m2m32_kernel<<<(unsigned)lv.nbox, 128, 0, fs>>>(P->lev[l + 1].mult32, lv.t_m2m32, P->lev[l + 1].p,
                                                                   lv.p, nrhs, lv.mult32);
                    HFMM_CUDA_TRY(cudaGetLastError());
                }
                ++P->launches;
                P->st_flops[HFMM_STAGE_M2M] += MAC * 4.0 * lv.nbox * lv.ncoef * P->lev[l + 1].ncoef;
                P->st_bytes[HFMM_STAGE_M2M] += C * (4.0 * lv.nbox * P->lev[l + 1].ncoef + lv.nbox * lv.ncoef);
            }
            tf.end(HFMM_STAGE_M2M);
            tf.begin(HFMM_STAGE_DOWN);
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
                    if (l == L && concurrent) HFMM_CUDA_TRY(cudaStreamWaitEvent(fs, P->ev_near_done, 0));
                    const bool leaf_ev = l == L && P->events_ready;
                    if (leaf_ev) cudaEventRecord(P->ev_leaf[0], fs);
                    HFMM_TRY(launch_m2l_tc(P, l, nrhs, l == L && !l2p_fused, l2p_fused, fs));
                    if (leaf_ev) {
                        cudaEventRecord(P->ev_leaf[1], fs);
                        P->ev_leaf_used = true;
                        P->leaf_flops = MAC * ((double)lv.nv + (double)lv.nr) * lv.ncoef * lv.ncoef +
                                        (has_parent ? MAC * lv.nbox * lv.ncoef * npp : 0.0) +
                                        (l2p_fused ? MAC * n * lv.ncoef : 0.0);
                    }
                } else {
                    down32_kernel<<<(unsigned)lv.nbox, DOWN_THREADS, sm, fs>>>(
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
            if (l2p_fused) {
                P->st_flops[HFMM_STAGE_DOWN] += MAC * n * P->lev[L].ncoef;
                P->st_bytes[HFMM_STAGE_DOWN] += 2.0 * C * n + 8.0 * n * P->lev[L].ncoef;
            }
            tf.end(HFMM_STAGE_DOWN);
        }
        if (concurrent) {
            HFMM_CUDA_TRY(cudaEventRecord(P->ev_far_done, fs));
            HFMM_CUDA_TRY(cudaStreamWaitEvent(st, P->ev_far_done, 0));
        }
        if (!l2p_fused && (near_free || far)) HFMM_TRY(near_section(near_free, far, st));
        return HFMM_OK;
    };
    if (P->ad) HFMM_TRY(apply_adaptive32(P, nrhs, parts, st));   // adaptive tree: its own FP32 passes
    else HFMM_TRY(small ? apply_small(P, nrhs, parts, st) : large_path());
    if ((parts & HFMM_PART_NEAR_REACT) && P->nd > 0 && !P->ad) {
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
    scatter_y32<<<ntile, TP_THREADS, 0, st>>>(P->y32, P->iperm32, n, nrhs, adjoint, y);
    ++P->launches;
    HFMM_CUDA_TRY(cudaGetLastError());
    tm.end(HFMM_STAGE_SCATTER);
    P->st_bytes[HFMM_STAGE_SCATTER] = 2.0 * C * n + 8.0 * n;
    P->last_stream = st;
    return HFMM_OK;
}
