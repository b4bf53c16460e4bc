// Mixed-precision apply for few right-hand sides (HFMM_MIXED, nrhs up to the
// plan's small_rhs, HFMM_SMALL_RHS_DEFAULT = 4 unless the options say
// otherwise: measured on GB300, these kernels beat the tensor-core passes up to
// 4 right-hand sides and lose from 8 on).  With one or a few right-hand sides every translation is a
// matrix-vector product, so the tensor-core tiles (M = 128 rows = two boxes x
// 64 right-hand sides) would be mostly padding.  These kernels give the work to
// warps instead: a warp owns up to 32 U output coefficients of one box (one
// lane per coefficient and U slots per lane) for R right-hand sides at once,
// streams the scaled FP32 translation matrices of tables.cu from L1 / L2 along
// its lanes and broadcasts the source coefficients from shared memory.
//
//   P2M   (Algorithm 1, step 2)  warp per leaf, lane = coefficient m
//   M2M   (step 2)               CTA per (parent box, coefficient chunk)
//   L2L + M2L (step 3)           CTA per (target box, coefficient chunk); the
//                                warps split the box's source list (parent,
//                                V list, reaction list) and their partial sums
//                                are added in a fixed order (no atomics: the
//                                result does not depend on scheduling)
//   L2P + P2P (steps 4-5)        warp per target leaf, lane = target point;
//                                H0 from the library's FP32 table
//
// Expansion layouts are those of the mixed path (scaled a~, b~ in [box][rhs][coef]).
#include <algorithm>
#include <cmath>

#include "bessel.cuh"
#include "plan.cuh"

namespace {

constexpr int SM_W = 8;                 // warps per CTA of the translation kernels
constexpr int H0N = 64, H0D = 5;        // FP32 H0 table: 64 intervals on [0, 16], degree 5
constexpr float H0_ZMAX = 16.0f, H0_INV_DZ = 4.0f;
__constant__ float c_h0[2][H0N][H0D + 1];

__device__ __forceinline__ void cfma(cf& acc, cf a, cf b) {
    acc.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x));
    acc.y = fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y));
}

// (i/4) H0(z), 0 < z < 16, from a shared-memory copy of the table
__device__ __forceinline__ cf green_tab(const float (*tj)[H0D + 1], const float (*tr)[H0D + 1], float z) {
    const int iv = min((int)(z * H0_INV_DZ), H0N - 1);
    const float t = (z - ((float)iv + 0.5f) / H0_INV_DZ) * (2.0f * H0_INV_DZ);
    float j = tj[iv][H0D], r = tr[iv][H0D];
#pragma unroll
    for (int d = H0D - 1; d >= 0; --d) {
        j = fmaf(j, t, tj[iv][d]);
        r = fmaf(r, t, tr[iv][d]);
    }
    const float y = fmaf(0.63661977236758134f * logf(0.5f * z), j, r);
    return cfmk(-0.25f * y, 0.25f * j);
}

// ---------------------------------------------------------------------------
// P2M: a~[r][m] = sum over the leaf's points j of q_r(j) B[j][m]
// ---------------------------------------------------------------------------
template <int R>
__global__ void __launch_bounds__(128) p2m_small_kernel(const int32_t* __restrict__ lb, int64_t nleaf,
                                                        const cf* __restrict__ qs, const cf* __restrict__ basis,
                                                        int nrhs, int nc, cf* __restrict__ mult) {
    const int64_t b = (int64_t)blockIdx.x * 4 + (threadIdx.x >> 5);
    if (b >= nleaf) return;
    const int lane = threadIdx.x & 31;
    const int32_t lo = lb[b], hi = lb[b + 1];
    for (int r0 = 0; r0 < nrhs; r0 += R) {
        for (int m0 = 0; m0 < nc; m0 += 32) {
            const int m = m0 + lane;
            cf acc[R];
#pragma unroll
            for (int r = 0; r < R; ++r) acc[r] = cfmk(0.f, 0.f);
            for (int32_t j = lo; j < hi; ++j) {
                const cf bv = m < nc ? basis[(int64_t)j * nc + m] : cfmk(0.f, 0.f);
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const cf qv = r0 + r < nrhs ? qs[(int64_t)j * nrhs + r0 + r] : cfmk(0.f, 0.f);
                    cfma(acc[r], bv, qv);
                }
            }
            if (m < nc)
#pragma unroll
                for (int r = 0; r < R; ++r)
                    if (r0 + r < nrhs) mult[((int64_t)b * nrhs + r0 + r) * nc + m] = acc[r];
        }
    }
}

// ---------------------------------------------------------------------------
// One source of a translation: acc[u][r] += sum_m M[m][p_u] a[r][m] for the
// lane's outputs p_u = p0 + lane + 32 u, with the source rows a staged in the
// warp's shared buffer (R rows of ncs) and M read along the lanes.
// ---------------------------------------------------------------------------
// The matrix rows are loaded SM_PF at a time before they are used, so that a
// warp keeps SM_PF x U loads in flight instead of waiting on each one.
constexpr int SM_PF = 8;

template <int R, int U>
__device__ __forceinline__ void translate_source(cf (&acc)[U][R], const cf* __restrict__ src, const cf* __restrict__ M,
                                                 int ncs, int ncout, int p0, int rows, cf* stage, int m_lo = 0,
                                                 int m_hi = 1 << 30) {
    const int lane = threadIdx.x & 31;
    m_hi = min(m_hi, ncs);
    __syncwarp();
    for (int e = lane; e < R * ncs; e += 32) stage[e] = e < rows * ncs ? src[e] : cfmk(0.f, 0.f);
    __syncwarp();
    bool pl[U];
#pragma unroll
    for (int u = 0; u < U; ++u) pl[u] = p0 + lane + 32 * u < ncout;
    const cf* Mp = M + p0 + lane;
    for (int m0 = m_lo; m0 < m_hi; m0 += SM_PF) {
        cf mv[SM_PF][U];
#pragma unroll
        for (int i = 0; i < SM_PF; ++i)
#pragma unroll
            for (int u = 0; u < U; ++u)
                mv[i][u] = (pl[u] && m0 + i < m_hi) ? __ldg(Mp + (int64_t)(m0 + i) * ncout + 32 * u) : cfmk(0.f, 0.f);
#pragma unroll
        for (int i = 0; i < SM_PF; ++i) {
            if (m0 + i >= m_hi) break;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const cf a = stage[r * ncs + m0 + i];
#pragma unroll
                for (int u = 0; u < U; ++u) cfma(acc[u][r], a, mv[i][u]);
            }
        }
    }
}

// Adds the warps' partial sums in warp order and stores them (warp 0).
template <int R, int U>
__device__ __forceinline__ void reduce_store(cf (&acc)[U][R], cf* red, cf* out, int64_t row0, int nrhs, int r0,
                                             int ncout, int p0) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
        for (int r = 0; r < R; ++r) red[((w * U + u) * R + r) * 32 + lane] = acc[u][r];
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int r = 0; r < R; ++r) {
                cf s = red[(u * R + r) * 32 + lane];
                for (int ww = 1; ww < SM_W; ++ww) {
                    const cf v = red[((ww * U + u) * R + r) * 32 + lane];
                    s.x += v.x;
                    s.y += v.y;
                }
                const int p = p0 + lane + 32 * u;
                if (p < ncout && r0 + r < nrhs) out[(row0 + r0 + r) * ncout + p] = s;
            }
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// M2M into level l: a~^P[r][j] = sum_c sum_m T~[c][m][j] a~^c[r][m]
// ---------------------------------------------------------------------------
static_assert(SM_W == 8, "M2M splits four children over two warps each");

template <int R, int U>
__global__ void __launch_bounds__(SM_W * 32) m2m_small_kernel(const int32_t* __restrict__ lb, int L, int l,
                                                              const cf* __restrict__ child, const cf* __restrict__ T,
                                                              int pc, int pp, int nrhs, int nchunk, int ncs_max,
                                                              cf* __restrict__ parent) {
    extern __shared__ float4 sm_small[];
    const int w = threadIdx.x >> 5;
    cf* stage = (cf*)sm_small + (int64_t)w * R * ncs_max;
    cf* red = (cf*)sm_small + (int64_t)SM_W * R * ncs_max;
    const int64_t b = blockIdx.x / nchunk;
    const int p0 = (blockIdx.x % nchunk) * 32 * U;
    const int ncc = 2 * pc + 1, np = 2 * pp + 1;
    for (int r0 = 0; r0 < nrhs; r0 += R) {
        cf acc[U][R];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int r = 0; r < R; ++r) acc[u][r] = cfmk(0.f, 0.f);
        // warp w: child w % 4, half w / 4 of the child's coefficients
        const int c = w & 3, half = (ncc + 1) / 2;
        int32_t lo, hi;
        box_range(lb, L, l + 1, 4 * b + c, &lo, &hi);
        if (hi > lo)
            translate_source<R, U>(acc, child + ((4 * b + c) * nrhs + r0) * (int64_t)ncc, T + (int64_t)c * ncc * np,
                                   ncc, np, p0, min(R, nrhs - r0), stage, (w >> 2) * half, (w >> 2) * half + half);
        reduce_store<R, U>(acc, red, parent, b * nrhs, nrhs, r0, np, p0);
    }
}

// ---------------------------------------------------------------------------
// Downward pass of level l: L2L from the parent plus free-space and reaction
// M2L over the box's lists (the parts mask selects the M2L terms).
// ---------------------------------------------------------------------------
template <int R, int U>
__global__ void __launch_bounds__(SM_W * 32) down_small_kernel(
    const int32_t* __restrict__ lb, int L, int l, int lmin, int nrhs, int p, int pp, const cf* __restrict__ ploc,
    const cf* __restrict__ Tl2l, const cf* __restrict__ mult, const int32_t* __restrict__ v_begin,
    const int32_t* __restrict__ v_src, const int32_t* __restrict__ v_off, const cf* __restrict__ Tfree,
    const int32_t* __restrict__ r_begin, const int32_t* __restrict__ r_src, const int32_t* __restrict__ r_tab,
    const cf* __restrict__ Treact, int parts, int nchunk, int ncs_max, cf* __restrict__ loc) {
    extern __shared__ float4 sm_small[];
    const int w = threadIdx.x >> 5;
    cf* stage = (cf*)sm_small + (int64_t)w * R * ncs_max;
    cf* red = (cf*)sm_small + (int64_t)SM_W * R * ncs_max;
    const int64_t b = blockIdx.x / nchunk;
    const int p0 = (blockIdx.x % nchunk) * 32 * U;
    int32_t lo, hi;
    box_range(lb, L, l, b, &lo, &hi);
    if (hi <= lo) return;                      // uniform over the CTA
    const int nc = 2 * p + 1, npp = 2 * pp + 1;
    const bool has_parent = (l > lmin) && ploc;
    const int64_t P = b >> 2;
    const int cchild = (int)(b & 3);
    const int nv0 = ((parts & HFMM_PART_FAR_FREE) && v_begin) ? v_begin[b] : 0;
    const int nv1 = ((parts & HFMM_PART_FAR_FREE) && v_begin) ? v_begin[b + 1] : 0;
    const int nr0 = ((parts & HFMM_PART_FAR_REACT) && r_begin) ? r_begin[b] : 0;
    const int nr1 = ((parts & HFMM_PART_FAR_REACT) && r_begin) ? r_begin[b + 1] : 0;
    const int nsrc = (has_parent ? 1 : 0) + (nv1 - nv0) + (nr1 - nr0);
    for (int r0 = 0; r0 < nrhs; r0 += R) {
        const int rows = min(R, nrhs - r0);
        cf acc[U][R];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int r = 0; r < R; ++r) acc[u][r] = cfmk(0.f, 0.f);
        for (int s = w; s < nsrc; s += SM_W) {
            if (has_parent && s == 0) {
                translate_source<R, U>(acc, ploc + (P * nrhs + r0) * (int64_t)npp, Tl2l + (int64_t)cchild * npp * nc,
                                       npp, nc, p0, rows, stage);
                continue;
            }
            int e = s - (has_parent ? 1 : 0);
            const cf* src;
            const cf* M;
            if (e < nv1 - nv0) {
                src = mult + ((int64_t)v_src[nv0 + e] * nrhs + r0) * nc;
                M = Tfree + (int64_t)v_off[nv0 + e] * nc * nc;
            } else {
                e -= nv1 - nv0;
                src = mult + ((int64_t)r_src[nr0 + e] * nrhs + r0) * nc;
                M = Treact + (int64_t)r_tab[nr0 + e] * nc * nc;
            }
            translate_source<R, U>(acc, src, M, nc, nc, p0, rows, stage);
        }
        reduce_store<R, U>(acc, red, loc, b * nrhs, nrhs, r0, nc, p0);
    }
}

// ---------------------------------------------------------------------------
// Near field and the leaves' local expansions: warp per target leaf, lane =
// target point (passes of 32), sources of the 3 x 3 neighbourhood in order.
// ---------------------------------------------------------------------------
template <int R>
__global__ void __launch_bounds__(128) near_small_kernel(const int32_t* __restrict__ lb, int L, int64_t nleaf,
                                                         const float2* __restrict__ xl, const cf* __restrict__ qs,
                                                         int nrhs, float k, float h, int near,
                                                         const cf* __restrict__ loc, const cf* __restrict__ basis,
                                                         int nc, cf* __restrict__ ys) {
    __shared__ float tj[H0N][H0D + 1], tr[H0N][H0D + 1];
    for (int e = threadIdx.x; e < H0N * (H0D + 1); e += blockDim.x) {
        tj[e / (H0D + 1)][e % (H0D + 1)] = c_h0[0][e / (H0D + 1)][e % (H0D + 1)];
        tr[e / (H0D + 1)][e % (H0D + 1)] = c_h0[1][e / (H0D + 1)][e % (H0D + 1)];
    }
    __syncthreads();
    const int64_t b = (int64_t)blockIdx.x * 4 + (threadIdx.x >> 5);
    if (b >= nleaf) return;
    const int lane = threadIdx.x & 31;
    const int32_t tlo = lb[b], thi = lb[b + 1];
    if (thi <= tlo) return;
    const int ix = (int)morton_x((uint32_t)b), iy = (int)morton_y((uint32_t)b);
    const int mside = 1 << L;
    for (int r0 = 0; r0 < nrhs; r0 += R) {
        for (int32_t t0 = tlo; t0 < thi; t0 += 32) {
            const int32_t t = t0 + lane;
            const bool live = t < thi;
            const float2 tp = live ? xl[t] : make_float2(0.f, 0.f);
            cf acc[R];
#pragma unroll
            for (int r = 0; r < R; ++r) acc[r] = cfmk(0.f, 0.f);
            for (int dy = -1; dy <= 1 && near; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const int sx = ix + dx, sy = iy + dy;
                    if (sx < 0 || sy < 0 || sx >= mside || sy >= mside) continue;
                    const uint32_t s = morton((uint32_t)sx, (uint32_t)sy);
                    const int32_t slo = lb[s], shi = lb[s + 1];
                    const float ox = (float)(-dx) * h, oy = (float)(-dy) * h;   // c_T - c_S
                    for (int32_t j0 = slo; j0 < shi; j0 += 4) {
                        // positions and strengths of up to four sources, loaded before use
                        float2 sp[4];
                        cf qv[4][R];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const bool ok = j0 + i < shi;
                            sp[i] = ok ? xl[j0 + i] : make_float2(0.f, 0.f);
#pragma unroll
                            for (int r = 0; r < R; ++r)
                                qv[i][r] = (ok && r0 + r < nrhs) ? qs[(int64_t)(j0 + i) * nrhs + r0 + r] : cfmk(0.f, 0.f);
                        }
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const int32_t j = j0 + i;
                            cf g = cfmk(0.f, 0.f);
                            if (live && j < shi && t != j) {
                                const float ddx = ox + (tp.x - sp[i].x), ddy = oy + (tp.y - sp[i].y);
                                const float z = k * sqrtf(ddx * ddx + ddy * ddy);
                                if (z < H0_ZMAX) {
                                    g = green_tab(tj, tr, z);
                                } else {
                                    const cd h0 = hankel0((double)z);
                                    g = cfmk((float)(-0.25 * h0.y), (float)(0.25 * h0.x));
                                }
                            }
#pragma unroll
                            for (int r = 0; r < R; ++r) cfma(acc[r], g, qv[i][r]);
                        }
                    }
                }
            if (loc) {
                // L2P: (i/4) sum_m b~[r][m] conj(B[t][m])
                for (int m = 0; m < nc; ++m) {
                    const cf B = live ? basis[(int64_t)t * nc + m] : cfmk(0.f, 0.f);
                    const cf g = cfmk(0.25f * B.y, 0.25f * B.x);
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const cf bt = r0 + r < nrhs ? loc[((int64_t)b * nrhs + r0 + r) * nc + m] : cfmk(0.f, 0.f);
                        cfma(acc[r], g, bt);
                    }
                }
            }
            if (live)
#pragma unroll
                for (int r = 0; r < R; ++r)
                    if (r0 + r < nrhs) {
                        cf* yy = ys + (int64_t)t * nrhs + r0 + r;
                        yy->x += acc[r].x;
                        yy->y += acc[r].y;
                    }
        }
    }
}

// right-hand sides per pass: the largest of 8, 4, 2, 1 not above nrhs whose
// staging (SM_W warps x R rows x ncs) stays within the shared-memory budget
int pick_r(int nrhs, int ncs_max, int U) {
    for (int R : {8, 4, 2, 1}) {
        if (R > 1 && R > nrhs && R / 2 >= nrhs) continue;
        const size_t smem = sizeof(cf) * ((size_t)SM_W * R * ncs_max + (size_t)SM_W * U * R * 32);
        if (smem <= 96 * 1024) return R;
    }
    return 1;
}

size_t smem_bytes(int R, int U, int ncs_max) {
    return sizeof(cf) * ((size_t)SM_W * R * ncs_max + (size_t)SM_W * U * R * 32);
}

template <int R, int U>
hfmm_status launch_down_ru(hfmm_plan_s* P, int l, int nrhs, int parts, int nchunk, int ncs_max, cudaStream_t st) {
    LevelInfo& lv = P->lev[l];
    const bool has_parent = l > P->lmin;
    const size_t sm = smem_bytes(R, U, ncs_max);
    auto kern = down_small_kernel<R, U>;
    HFMM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    kern<<<(unsigned)(lv.nbox * nchunk), SM_W * 32, sm, st>>>(
        P->leaf_begin, P->L, l, P->lmin, nrhs, lv.p, has_parent ? P->lev[l - 1].p : 0,
        has_parent ? P->lev[l - 1].loc32 : nullptr, has_parent ? P->lev[l - 1].t_l2l32 : nullptr, lv.mult32,
        lv.nv ? lv.v_begin : nullptr, lv.v_src, lv.v_off, lv.t_free32, lv.nr ? lv.r_begin : nullptr, lv.r_src,
        lv.r_tab, lv.t_react32, parts, nchunk, ncs_max, lv.loc32);
    HFMM_CUDA_TRY(cudaGetLastError());
    return HFMM_OK;
}

template <int R, int U>
hfmm_status launch_m2m_ru(hfmm_plan_s* P, int l, int nrhs, int nchunk, int ncs_max, cudaStream_t st) {
    LevelInfo& lv = P->lev[l];
    const size_t sm = smem_bytes(R, U, ncs_max);
    auto kern = m2m_small_kernel<R, U>;
    HFMM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    kern<<<(unsigned)(lv.nbox * nchunk), SM_W * 32, sm, st>>>(P->leaf_begin, P->L, l, P->lev[l + 1].mult32,
                                                              lv.t_m2m32, P->lev[l + 1].p, lv.p, nrhs, nchunk,
                                                              ncs_max, lv.mult32);
    HFMM_CUDA_TRY(cudaGetLastError());
    return HFMM_OK;
}

// outputs per lane (U) and chunks of 32 U coefficients for an output width
void pick_u(int ncout, int64_t nbox, int* U, int* nchunk) {
    // few boxes (coarse levels): narrow chunks for more CTAs; many boxes: wide
    int u = ncout <= 32 ? 1 : (nbox >= 4096 ? std::min(4, (ncout + 31) / 32) : 1);
    if (u == 3) u = 4;
    *U = u;
    *nchunk = (ncout + 32 * u - 1) / (32 * u);
}

#define HFMM_SMALL_DISPATCH(FN, ...)                                   \
    switch (R * 10 + U) {                                             \
        case 11: return FN<1, 1>(__VA_ARGS__);                        \
        case 12: return FN<1, 2>(__VA_ARGS__);                        \
        case 14: return FN<1, 4>(__VA_ARGS__);                        \
        case 21: return FN<2, 1>(__VA_ARGS__);                        \
        case 22: return FN<2, 2>(__VA_ARGS__);                        \
        case 24: return FN<2, 4>(__VA_ARGS__);                        \
        case 41: return FN<4, 1>(__VA_ARGS__);                        \
        case 42: return FN<4, 2>(__VA_ARGS__);                        \
        case 44: return FN<4, 4>(__VA_ARGS__);                        \
        case 81: return FN<8, 1>(__VA_ARGS__);                        \
        case 82: return FN<8, 2>(__VA_ARGS__);                        \
        case 84: return FN<8, 4>(__VA_ARGS__);                        \
    }

}  // namespace

hfmm_status init_small(hfmm_plan_s* P, cudaStream_t st) {
    (void)P;
    HFMM_CUDA_TRY(cudaMemcpyToSymbolAsync(c_h0, h0_table_host(), sizeof(c_h0), 0, cudaMemcpyHostToDevice, st));
    return HFMM_OK;
}

hfmm_status small_p2m(hfmm_plan_s* P, int nrhs, cudaStream_t st) {
    LevelInfo& lv = P->lev[P->L];
    const unsigned grid = (unsigned)ceil_div(lv.nbox, 4);
    if (nrhs >= 8) p2m_small_kernel<8><<<grid, 128, 0, st>>>(P->leaf_begin, lv.nbox, P->q32, P->basis32, nrhs, lv.ncoef, lv.mult32);
    else if (nrhs >= 4) p2m_small_kernel<4><<<grid, 128, 0, st>>>(P->leaf_begin, lv.nbox, P->q32, P->basis32, nrhs, lv.ncoef, lv.mult32);
    else if (nrhs >= 2) p2m_small_kernel<2><<<grid, 128, 0, st>>>(P->leaf_begin, lv.nbox, P->q32, P->basis32, nrhs, lv.ncoef, lv.mult32);
    else p2m_small_kernel<1><<<grid, 128, 0, st>>>(P->leaf_begin, lv.nbox, P->q32, P->basis32, nrhs, lv.ncoef, lv.mult32);
    HFMM_CUDA_TRY(cudaGetLastError());
    return HFMM_OK;
}

hfmm_status small_m2m(hfmm_plan_s* P, int l, int nrhs, cudaStream_t st) {
    LevelInfo& lv = P->lev[l];
    const int ncs_max = P->lev[l + 1].ncoef;
    int U, nchunk;
    pick_u(lv.ncoef, lv.nbox, &U, &nchunk);
    const int R = pick_r(nrhs, ncs_max, U);
    HFMM_SMALL_DISPATCH(launch_m2m_ru, P, l, nrhs, nchunk, ncs_max, st)
    hfmm_set_error("small m2m: no kernel for R=%d U=%d", R, U);
    return HFMM_ERR_UNSUPPORTED;
}

hfmm_status small_down(hfmm_plan_s* P, int l, int nrhs, int parts, cudaStream_t st) {
    LevelInfo& lv = P->lev[l];
    const bool has_parent = l > P->lmin;
    const int ncs_max = std::max(lv.ncoef, has_parent ? P->lev[l - 1].ncoef : 0);
    int U, nchunk;
    pick_u(lv.ncoef, lv.nbox, &U, &nchunk);
    const int R = pick_r(nrhs, ncs_max, U);
    HFMM_SMALL_DISPATCH(launch_down_ru, P, l, nrhs, parts, nchunk, ncs_max, st)
    hfmm_set_error("small downward pass: no kernel for R=%d U=%d", R, U);
    return HFMM_ERR_UNSUPPORTED;
}

hfmm_status small_near(hfmm_plan_s* P, int nrhs, bool near, bool l2p, cudaStream_t st) {
    LevelInfo& lv = P->lev[P->L];
    const unsigned grid = (unsigned)ceil_div(lv.nbox, 4);
    const cf* loc = l2p ? lv.loc32 : nullptr;
#define HFMM_NEAR(RR)                                                                                            \
    near_small_kernel<RR><<<grid, 128, 0, st>>>(P->leaf_begin, P->L, lv.nbox, P->xl32, P->q32, nrhs, (float)P->k, \
                                                (float)lv.h, near ? 1 : 0, loc, P->basis32, lv.ncoef, P->y32)
    if (nrhs >= 8) HFMM_NEAR(8);
    else if (nrhs >= 4) HFMM_NEAR(4);
    else if (nrhs >= 2) HFMM_NEAR(2);
    else HFMM_NEAR(1);
#undef HFMM_NEAR
    HFMM_CUDA_TRY(cudaGetLastError());
    return HFMM_OK;
}

hfmm_status apply_small(hfmm_plan_s* P, int nrhs, int parts, cudaStream_t st) {
    const int L = P->L;
    const int64_t n = P->n;
    StageTimer tm{P, st};
    const double MAC = 8.0 * nrhs, C = 8.0 * nrhs;
    const bool far = (parts & (HFMM_PART_FAR_FREE | HFMM_PART_FAR_REACT)) != 0;
    const bool near = (parts & HFMM_PART_NEAR_FREE) != 0;
    if (far) {
        LevelInfo& leaf = P->lev[L];
        tm.begin(HFMM_STAGE_P2M);
        HFMM_TRY(small_p2m(P, nrhs, st));
        ++P->launches;
        tm.end(HFMM_STAGE_P2M);
        P->st_flops[HFMM_STAGE_P2M] = MAC * n * leaf.ncoef;
        P->st_bytes[HFMM_STAGE_P2M] = C * n + 8.0 * n * leaf.ncoef + C * leaf.nbox * leaf.ncoef;
        tm.begin(HFMM_STAGE_M2M);
        for (int l = L - 1; l >= P->lmin; --l) {
            LevelInfo& lv = P->lev[l];
            HFMM_TRY(small_m2m(P, l, nrhs, st));
            ++P->launches;
            P->st_flops[HFMM_STAGE_M2M] += MAC * 4.0 * lv.nbox * lv.ncoef * P->lev[l + 1].ncoef;
            P->st_bytes[HFMM_STAGE_M2M] += C * (4.0 * lv.nbox * P->lev[l + 1].ncoef + lv.nbox * lv.ncoef);
        }
        tm.end(HFMM_STAGE_M2M);
        tm.begin(HFMM_STAGE_DOWN);
        for (int l = P->lmin; l <= L; ++l) {
            LevelInfo& lv = P->lev[l];
            HFMM_TRY(small_down(P, l, nrhs, parts, st));
            ++P->launches;
            double pairs = 0.0;
            if (parts & HFMM_PART_FAR_FREE) pairs += (double)lv.nv;
            if (parts & HFMM_PART_FAR_REACT) pairs += (double)lv.nr;
            P->st_flops[HFMM_STAGE_DOWN] += MAC * pairs * lv.ncoef * lv.ncoef;
            if (l > P->lmin) P->st_flops[HFMM_STAGE_DOWN] += MAC * lv.nbox * lv.ncoef * P->lev[l - 1].ncoef;
            P->st_bytes[HFMM_STAGE_DOWN] += C * lv.nbox * lv.ncoef * 2.0 +
                                            (l > P->lmin ? C * P->lev[l - 1].nbox * P->lev[l - 1].ncoef : 0.0);
        }
        tm.end(HFMM_STAGE_DOWN);
    }
    if (near || far) {
        LevelInfo& leaf = P->lev[L];
        tm.begin(HFMM_STAGE_P2P);
        HFMM_TRY(small_near(P, nrhs, near, far, st));
        ++P->launches;
        tm.end(HFMM_STAGE_P2P);
        P->st_flops[HFMM_STAGE_P2P] = (near ? MAC * (double)P->p2p_point_pairs : 0.0) +
                                      (far ? MAC * n * leaf.ncoef : 0.0);
        P->st_bytes[HFMM_STAGE_P2P] = 3.0 * C * n + 16.0 * n + (far ? C * leaf.nbox * leaf.ncoef + 8.0 * n * leaf.ncoef : 0.0);
    }
    return HFMM_OK;
}
