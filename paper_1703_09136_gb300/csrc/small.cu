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
#include <new>
#include <vector>

#include "bessel.cuh"
#include "plan.cuh"

namespace {

constexpr int SM_W = 8;                 // warps per CTA of the translation kernels
constexpr int H0N = 64, H0D = 5;        // FP32 H0 table: 64 intervals on [0, 16], degree 5
constexpr float H0_ZMAX = 16.0f, H0_INV_DZ = 4.0f;
__device__ float g_h0[2][H0N][H0D + 1];    // global memory: the CTAs copy it to shared memory with coalesced loads

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
    // L2 loads (ld.global.cg): in the persistent batch kernel the source was
    // written by another CTA of the same launch, after this SM's L1 may have
    // cached neighbouring lines
    for (int e = lane; e < R * ncs; e += 32) stage[e] = e < rows * ncs ? __ldcg(src + e) : cfmk(0.f, 0.f);
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
template <int R, int U, int NW = SM_W>
__device__ __forceinline__ void reduce_store(cf (&acc)[U][R], cf* red, cf* out, int64_t row0, int nrhs, int r0,
                                             int ncout, int p0, bool add = false) {
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
                for (int ww = 1; ww < NW; ++ww) {
                    const cf v = red[((ww * U + u) * R + r) * 32 + lane];
                    s.x += v.x;
                    s.y += v.y;
                }
                const int p = p0 + lane + 32 * u;
                if (p < ncout && r0 + r < nrhs) {
                    cf* o = out + (row0 + r0 + r) * ncout + p;
                    if (add) {
                        const cf v = *o;
                        s.x = v.x + s.x;
                        s.y = v.y + s.y;
                    }
                    *o = s;
                }
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
template <int R, int U, int NW = SM_W>
__global__ void __launch_bounds__(NW * 32) down_small_kernel(
    const int32_t* __restrict__ lb, int L, int l, int lmin, int nrhs, int p, int pp, const cf* __restrict__ ploc,
    const cf* __restrict__ Tl2l, const cf* __restrict__ mult, const int32_t* __restrict__ v_begin,
    const int32_t* __restrict__ v_src, const int32_t* __restrict__ v_off, const cf* __restrict__ Tfree,
    const int32_t* __restrict__ r_begin, const int32_t* __restrict__ r_src, const int32_t* __restrict__ r_tab,
    const cf* __restrict__ Treact, int parts, int nchunk, int ncs_max, cf* __restrict__ loc, bool react_add,
    const int32_t* __restrict__ tgt_list) {
    extern __shared__ float4 sm_small[];
    const int w = threadIdx.x >> 5;
    cf* stage = (cf*)sm_small + (int64_t)w * R * ncs_max;
    cf* red = (cf*)sm_small + (int64_t)NW * R * ncs_max;
    if (react_add) {   // L2L and V list already in loc (vblock_kernel): add the reaction list only
        ploc = nullptr;
        v_begin = nullptr;
    }
    const int64_t b = tgt_list ? (int64_t)tgt_list[blockIdx.x / nchunk] : (int64_t)(blockIdx.x / nchunk);
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
    if (react_add && nsrc == 0) return;        // uniform over the CTA
    for (int r0 = 0; r0 < nrhs; r0 += R) {
        const int rows = min(R, nrhs - r0);
        cf acc[U][R];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int r = 0; r < R; ++r) acc[u][r] = cfmk(0.f, 0.f);
        for (int s = w; s < nsrc; s += NW) {
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
        reduce_store<R, U, NW>(acc, red, loc, b * nrhs, nrhs, r0, nc, p0, react_add);
    }
}

// ---------------------------------------------------------------------------
// L2L + free-space M2L of level l for blocks of 32 target boxes (32
// consecutive Morton indices: 8 x 4 boxes, 4 x 2 parents), one right-hand
// side per CTA.  The targets of one child position c share their L2L matrix,
// and the targets of position c with a V-list source at offset o share that
// M2L matrix, so one matrix row read from L2 feeds 4 targets (a per-box pass
// reads it once per target).  The sources of the block (the 12 x 8 boxes of
// level l around it, the 8 parents' local expansions) are staged in shared
// memory once.  NWC warps (2, or 4 for CPT > 2) own the 8 targets of child
// position c, each taking every NWC-th operator of the position's list; a
// lane owns 4 targets x CPT consecutive output coefficients.  The warps' sums
// are added in a fixed order, operators and k run in increasing order: the
// result does not depend on scheduling.  The V-list entries give which
// offsets a target uses: the source of offset index o = (dx + 3) * 7 + dy + 3
// is the box (ix - dx, iy - dy) of level l, as the list builder enumerates
// it.  Reaction lists are added afterwards by down_small_kernel (react_add).
// ---------------------------------------------------------------------------
constexpr int VB_T = 32;                       // target boxes per block
constexpr int VB_WX = 12, VB_WY = 8;           // source window (boxes of level l)
constexpr int VB_SLOTS = VB_WX * VB_WY;
constexpr int VB_L2L = 49;                     // mask bit of the L2L of child position c: 49 + c
constexpr uint64_t VB_LIVE = 1ull << 63;       // mask bit: nonempty target (written)

__device__ __forceinline__ void cp_async8_vb(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;"
                 :: "r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src) : "memory");
}

// warps per child position: 2 with 2 coefficients per lane (levels of many
// blocks), 4 otherwise (levels of few blocks, the wider lanes hold more registers)
constexpr int vb_nwc(int cpt) { return cpt == 2 ? 2 : 4; }

size_t vblock_smem(int cpt, int nc, int npp) {
    const int kmax = std::max(nc, npp), ncw = nc | 1, npw = npp | 1;
    const size_t red = (size_t)4 * (vb_nwc(cpt) - 1) * 32 * 4 * cpt;   // the other warps' sums, over the window
    return sizeof(cf) * (std::max((size_t)VB_SLOTS * ncw, red) + kmax + 8 * (size_t)npw) +
           sizeof(uint64_t) * VB_T;
}

template <int CPT>
__global__ void __launch_bounds__(128 * vb_nwc(CPT), CPT == 2 ? 4 : 1)
    vblock_kernel(const int32_t* __restrict__ lb, int L, int l, int nrhs, int nc, int npp, const cf* __restrict__ ploc,
                  const cf* __restrict__ Tl2l, const cf* __restrict__ mult, const int32_t* __restrict__ v_begin,
                  const int32_t* __restrict__ v_off, const cf* __restrict__ Tfree, cf* __restrict__ loc) {
    constexpr int VB_PF = CPT == 2 ? 2 : 4;        // matrix rows per lane per fetch (two fetches in flight)
    extern __shared__ float4 sm_vb[];
    const int kmax = max(nc, npp), ncw = nc | 1, npw = npp | 1;   // odd row strides
    constexpr int NWC = vb_nwc(CPT), NT = 128 * NWC;   // warps per child position, threads
    const int wsz = max(VB_SLOTS * ncw, 4 * (NWC - 1) * 32 * 4 * CPT);
    cf* W = (cf*)sm_vb;                            // source window [slot][ncw]; then half 1's sums
    cf* Z = W + wsz;                               // kmax zeros (sources of lanes without the operator)
    cf* Pw = Z + kmax;                             // parents' local expansions [8][npw]
    uint64_t* mask = (uint64_t*)(Pw + 8 * npw);    // [32 targets]
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, c = w / NWC, h = w % NWC;
    const int r = blockIdx.y;
    const int64_t b0 = (int64_t)blockIdx.x * VB_T;
    const int bx0 = (int)morton_x((uint32_t)b0), by0 = (int)morton_y((uint32_t)b0);
    const int m = 1 << l;
    for (int e = tid; e < kmax; e += NT) Z[e] = cfmk(0.f, 0.f);
    if (tid < VB_T) {
        const int64_t b = b0 + tid;
        int32_t lo, hi;
        box_range(lb, L, l, b, &lo, &hi);
        uint64_t mk = 0;
        if (hi > lo) {
            mk = VB_LIVE;
            if (v_begin)
                for (int32_t e = v_begin[b]; e < v_begin[b + 1]; ++e) mk |= 1ull << v_off[e];
            if (ploc) mk |= 1ull << (VB_L2L + (tid & 3));
        }
        mask[tid] = mk;
    }
    // sources: slot (wx, wy) holds box (bx0 - 2 + wx, by0 - 2 + wy); boxes
    // outside the domain are never a source
    for (int s = w; s < VB_SLOTS; s += NT / 32) {
        const int sx = bx0 - 2 + s % VB_WX, sy = by0 - 2 + s / VB_WX;
        const bool in = sx >= 0 && sy >= 0 && sx < m && sy < m;
        const cf* src = in ? mult + ((int64_t)morton((uint32_t)sx, (uint32_t)sy) * nrhs + r) * nc : nullptr;
        for (int k = lane; k < nc; k += 32) {
            if (in) cp_async8_vb(W + s * ncw + k, src + k);
            else W[s * ncw + k] = cfmk(0.f, 0.f);
        }
    }
    if (ploc)
        for (int j = w; j < 8; j += NT / 32)
            for (int k = lane; k < npp; k += 32)
                cp_async8_vb(Pw + j * npw + k, ploc + ((b0 / 4 + j) * nrhs + r) * (int64_t)npp + k);
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    // this lane's targets: j = 4 tg + i of child position c (local index 4 j + c)
    const int tg = lane >> 4, cg = lane & 15;
    uint64_t tm[4], um = 0;
    int tx[4], ty[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int li = 4 * (4 * tg + i) + c;
        tm[i] = mask[li];
        tx[i] = (li & 1) | ((li >> 1) & 2) | ((li >> 2) & 4);
        ty[i] = ((li >> 1) & 1) | ((li >> 2) & 2);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) um |= mask[4 * j + c];   // operators of position c
    um &= ~VB_LIVE;
    cf acc[4][CPT];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int u = 0; u < CPT; ++u) acc[i][u] = cfmk(0.f, 0.f);
    bool live_u[CPT];
#pragma unroll
    for (int u = 0; u < CPT; ++u) live_u[u] = cg * CPT + u < nc;
    // the position's L2L first, then the V offsets in increasing order; warp h
    // takes the operators of even (h = 0) or odd (h = 1) rank
    for (int rank = 0; um; ++rank) {
        const uint64_t l2l = um & (0xFull << VB_L2L);
        const int op = __ffsll((long long)(l2l ? l2l : um)) - 1;
        um &= ~(1ull << op);
        if (rank % NWC != h) continue;
        const bool isl2l = op >= VB_L2L;
        const cf* sp[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const bool use = (tm[i] >> op) & 1;
            if (!use) sp[i] = Z;
            else if (isl2l) sp[i] = Pw + (4 * tg + i) * npw;
            else {
                const int dx = op / 7 - 3, dy = op % 7 - 3;
                sp[i] = W + ((ty[i] - dy + 2) * VB_WX + (tx[i] - dx + 2)) * ncw;
            }
        }
        const cf* M = (isl2l ? Tl2l + (int64_t)(op - VB_L2L) * npp * nc : Tfree + (int64_t)op * nc * nc) + cg * CPT;
        const int K = isl2l ? npp : nc;
        // two register sets of VB_PF matrix rows: one is used while the other is in flight
        cf ma[VB_PF][CPT], mb[VB_PF][CPT];
        auto fetch = [&](cf (&mr)[VB_PF][CPT], int k0) {
#pragma unroll
            for (int i = 0; i < VB_PF; ++i)
#pragma unroll
                for (int u = 0; u < CPT; ++u)
                    mr[i][u] = (live_u[u] && k0 + i < K) ? __ldg(M + (int64_t)(k0 + i) * nc + u) : cfmk(0.f, 0.f);
        };
        auto use = [&](const cf (&mr)[VB_PF][CPT], int k0) {
#pragma unroll
            for (int i = 0; i < VB_PF; ++i) {
                if (k0 + i >= K) break;
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const cf sv = sp[t][k0 + i];
#pragma unroll
                    for (int u = 0; u < CPT; ++u) cfma(acc[t][u], sv, mr[i][u]);
                }
            }
        };
        fetch(ma, 0);
        for (int k0 = 0; k0 < K; k0 += 2 * VB_PF) {
            if (k0 + VB_PF < K) fetch(mb, k0 + VB_PF);
            use(ma, k0);
            if (k0 + VB_PF >= K) break;
            if (k0 + 2 * VB_PF < K) fetch(ma, k0 + 2 * VB_PF);
            use(mb, k0 + VB_PF);
        }
    }
    // the sums of warps NWC c + 1 .. go to shared memory (over the window);
    // warp NWC c adds them in warp order and stores
    __syncthreads();
    cf* red = W + ((c * (NWC - 1)) * 32 + lane) * 4 * CPT;   // [c][h - 1][lane][4 CPT]
    if (h > 0) {
#pragma unroll
        for (int t = 0; t < 4; ++t)
#pragma unroll
            for (int u = 0; u < CPT; ++u) red[((h - 1) * 32) * 4 * CPT + t * CPT + u] = acc[t][u];
    }
    __syncthreads();
    if (h > 0) return;
#pragma unroll
    for (int hh = 1; hh < NWC; ++hh)
#pragma unroll
        for (int t = 0; t < 4; ++t)
#pragma unroll
            for (int u = 0; u < CPT; ++u) {
                const cf o = red[((hh - 1) * 32) * 4 * CPT + t * CPT + u];
                acc[t][u] = cfmk(acc[t][u].x + o.x, acc[t][u].y + o.y);
            }
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        if (!(tm[t] & VB_LIVE)) continue;
        const int64_t b = b0 + 4 * (4 * tg + t) + c;
#pragma unroll
        for (int u = 0; u < CPT; ++u) {
            if (!live_u[u]) continue;
            loc[(b * nrhs + r) * nc + cg * CPT + u] = acc[t][u];
        }
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
    if (near)   // an L2P-only pass needs no table
        for (int e = threadIdx.x; e < H0N * (H0D + 1); e += blockDim.x) {
            tj[e / (H0D + 1)][e % (H0D + 1)] = g_h0[0][e / (H0D + 1)][e % (H0D + 1)];
            tr[e / (H0D + 1)][e % (H0D + 1)] = g_h0[1][e / (H0D + 1)][e % (H0D + 1)];
        }
    __syncthreads();
    const int64_t b = (int64_t)blockIdx.x * 4 + (threadIdx.x >> 5);
    if (b >= nleaf) return;
    const int lane = threadIdx.x & 31;
    const int32_t tlo = lb[b], thi = lb[b + 1];
    if (thi <= tlo) return;
    const int ix = (int)morton_x((uint32_t)b), iy = (int)morton_y((uint32_t)b);
    const int mside = 1 << L;
    // leaves of at most 16 points: the two half-warps take alternate sources
    // (and alternate L2P coefficients) of the same 16 targets, then add
    const bool split = thi - tlo <= 16;
    const int half = split ? lane >> 4 : 0, nper = split ? 2 : 4, mstep = split ? 2 : 1;
    for (int r0 = 0; r0 < nrhs; r0 += R) {
        for (int32_t t0 = tlo; t0 < thi; t0 += 32) {
            const int32_t t = t0 + (split ? lane & 15 : lane);
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
                        // positions and strengths of up to four sources (two per
                        // half-warp when split), loaded before use
                        float2 sp[4];
                        cf qv[4][R];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const int32_t j = j0 + (split ? 2 * i + half : i);
                            const bool ok = i < nper && j < shi;
                            sp[i] = ok ? xl[j] : make_float2(0.f, 0.f);
#pragma unroll
                            for (int r = 0; r < R; ++r)
                                qv[i][r] = (ok && r0 + r < nrhs) ? qs[(int64_t)j * nrhs + r0 + r] : cfmk(0.f, 0.f);
                        }
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            if (i >= nper) break;
                            const int32_t j = j0 + (split ? 2 * i + half : i);
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
#pragma unroll 4
                for (int m = half; m < nc; m += mstep) {
                    const cf B = live ? basis[(int64_t)t * nc + m] : cfmk(0.f, 0.f);
                    const cf g = cfmk(0.25f * B.y, 0.25f * B.x);
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const cf bt = r0 + r < nrhs ? loc[((int64_t)b * nrhs + r0 + r) * nc + m] : cfmk(0.f, 0.f);
                        cfma(acc[r], g, bt);
                    }
                }
            }
            if (split) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    acc[r].x += __shfl_xor_sync(0xffffffffu, acc[r].x, 16);
                    acc[r].y += __shfl_xor_sync(0xffffffffu, acc[r].y, 16);
                }
            }
            if (live && lane < (split ? 16 : 32))
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


// ---------------------------------------------------------------------------
// Persistent batch kernel: every stage of every instance of a batch in one
// launch.  The work items (one CTA each) are numbered in an order in which
// every item's inputs come from items with smaller numbers: gathers and P2M
// of all instances, M2M deepest level first, then the downward passes top
// level first, each instance's near field, direct reaction and scatter right
// after its leaf level.  A CTA takes the
// next number from a counter, waits (bounded) until the segments its item
// depends on are complete, does the item and counts it done.  Because items
// are taken in order, an item only waits on items that running CTAs already
// hold, so the launch cannot deadlock whatever the number of resident CTAs.
// Data produced in the launch is read through L2 (ld.global.cg).
// ---------------------------------------------------------------------------
enum PKind { PK_GATHER = 0, PK_P2M, PK_M2M, PK_DOWN, PK_NEAR, PK_DIRECT, PK_SCATTER };

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

template <int R>
__global__ void __launch_bounds__(SM_W * 32, 3) persist_kernel(const PSeg* __restrict__ segs, int nseg, int total,
                                                            const PInst* __restrict__ insts,
                                                            const PLev* __restrict__ levs, int nrhs, int adjoint,
                                                            int ncs_max, int* __restrict__ ctr, long spin) {
    extern __shared__ float4 sm_small[];
    __shared__ float tj[H0N][H0D + 1], tr[H0N][H0D + 1];
    __shared__ int s_item, s_seg;
    for (int e = threadIdx.x; e < H0N * (H0D + 1); e += blockDim.x) {
        tj[e / (H0D + 1)][e % (H0D + 1)] = g_h0[0][e / (H0D + 1)][e % (H0D + 1)];
        tr[e / (H0D + 1)][e % (H0D + 1)] = g_h0[1][e / (H0D + 1)][e % (H0D + 1)];
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
    cf* stage = (cf*)sm_small + (int64_t)w * R * ncs_max;
    cf* red = (cf*)sm_small + (int64_t)SM_W * R * ncs_max;
    // first item of every segment, for the segment lookup of each item
    int* s_item0 = (int*)(red + (int64_t)SM_W * R * 32);
    for (int e = tid; e < nseg; e += blockDim.x) s_item0[e] = segs[e].item0;
    int* done = ctr + 2;
    int* done_item = ctr + 2 + nseg;
    for (;;) {
        __syncthreads();                       // previous item finished with s_item, s_seg
        if (tid == 0) {
            const int it = atomicAdd(ctr, 1);
            int sg = 0;
            if (it < total) {
                int lo = 0, hi = nseg - 1;     // last segment with item0 <= it
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (s_item0[mid] <= it) lo = mid; else hi = mid - 1;
                }
                sg = lo;
                const PSeg S0 = segs[sg];
                const int deps[2] = {S0.dep0, S0.dep1};
                long polls = 0;
                bool gave_up = false;
                for (int d = 0; d < 2 && !gave_up; ++d) {      // whole segments
                    if (deps[d] < 0) continue;
                    const int need = segs[deps[d]].nitems;
                    while (ld_acquire(done + deps[d]) < need) {
                        if (++polls > spin) { gave_up = true; break; }
                        __nanosleep(200);
                    }
                }
                if (S0.idep >= 0 && !gave_up) {
                    // the items of segment idep that cover this item's boxes at
                    // their level: the same boxes, the children or the parents
                    const PSeg D = segs[S0.idep];
                    const int local = it - S0.item0;
                    int64_t blo, bhi;
                    if (S0.wpb) { blo = (int64_t)local * SM_W; bhi = blo + SM_W - 1; }
                    else { blo = bhi = local / S0.nchunk; }
                    if (S0.irel == 1) { blo = 4 * blo; bhi = 4 * bhi + 3; }
                    else if (S0.irel == 2) { blo >>= 2; bhi >>= 2; }
                    const int64_t nb = (int64_t)1 << (2 * D.level);
                    bhi = min(bhi, nb - 1);
                    int ilo, ihi;
                    if (D.wpb) { ilo = (int)(blo / SM_W); ihi = (int)(bhi / SM_W); }
                    else { ilo = (int)(blo * D.nchunk); ihi = (int)((bhi + 1) * D.nchunk - 1); }
                    for (int k = ilo; k <= ihi && !gave_up; ++k)
                        while (ld_acquire(done_item + D.item0 + k) == 0) {
                            if (++polls > spin) { gave_up = true; break; }
                            __nanosleep(200);
                        }
                }
                if (gave_up) atomicExch(ctr + 1, 1);          // flag the batch and go on
                __threadfence();
            }
            s_item = it;
            s_seg = sg;
        }
        __syncthreads();
        const int it = s_item;
        if (it >= total) break;
        const PSeg S = segs[s_seg];
        const PInst I = insts[S.inst];
        const int local = it - S.item0;
        const int64_t n = I.n;
        switch (S.kind) {
            case PK_GATHER:
            case PK_SCATTER: {
                const int64_t j0 = (int64_t)local * 64;
                const int jn = (int)min((int64_t)64, n - j0);
                for (int e = tid; e < 64 * nrhs; e += blockDim.x) {
                    const int r = e >> 6, jj = e & 63;
                    if (jj >= jn) continue;
                    const int64_t j = j0 + jj;
                    const int64_t sidx = (int64_t)I.iperm[j] * nrhs + r;
                    if (S.kind == PK_GATHER) {
                        cf v = I.q[(int64_t)r * n + j];
                        if (adjoint) v.y = -v.y;
                        I.q32[sidx] = v;
                    } else {
                        cf v = __ldcg(I.y32 + sidx);
                        if (adjoint) v.y = -v.y;
                        I.y[(int64_t)r * n + j] = v;
                    }
                }
                break;
            }
            case PK_P2M: {
                const int64_t b = (int64_t)local * SM_W + w;
                const int nc = I.nc;
                if (b < ((int64_t)1 << (2 * I.L))) {
                    const int32_t lo = I.lb[b], hi = I.lb[b + 1];
                    cf* mult = levs[I.lev0 + I.L].mult;
                    for (int r0 = 0; r0 < nrhs; r0 += R)
                        for (int m0 = 0; m0 < nc; m0 += 32) {
                            const int m = m0 + lane;
                            cf acc[R];
#pragma unroll
                            for (int r = 0; r < R; ++r) acc[r] = cfmk(0.f, 0.f);
                            for (int32_t j = lo; j < hi; ++j) {
                                const cf bv = m < nc ? I.basis[(int64_t)j * nc + m] : cfmk(0.f, 0.f);
#pragma unroll
                                for (int r = 0; r < R; ++r)
                                    cfma(acc[r], bv, r0 + r < nrhs ? __ldcg(I.q32 + (int64_t)j * nrhs + r0 + r)
                                                                   : cfmk(0.f, 0.f));
                            }
                            if (m < nc)
#pragma unroll
                                for (int r = 0; r < R; ++r)
                                    if (r0 + r < nrhs) mult[(b * nrhs + r0 + r) * nc + m] = acc[r];
                        }
                }
                break;
            }
            case PK_M2M: {
                const PLev V = levs[I.lev0 + S.level];
                if (S.wpb) {                                  // one parent box per warp
                    const int64_t b = (int64_t)local * SM_W + w;
                    if (b >= ((int64_t)1 << (2 * S.level))) break;
                    const int ncc = 2 * V.pc + 1, np = 2 * V.p + 1;
                    for (int r0 = 0; r0 < nrhs; r0 += R) {
                        cf acc[1][R];
#pragma unroll
                        for (int r = 0; r < R; ++r) acc[0][r] = cfmk(0.f, 0.f);
                        for (int c = 0; c < 4; ++c) {
                            int32_t lo, hi;
                            box_range(I.lb, I.L, S.level + 1, 4 * b + c, &lo, &hi);
                            if (hi > lo)
                                translate_source<R, 1>(acc, V.cmult + ((4 * b + c) * nrhs + r0) * (int64_t)ncc,
                                                       V.Tm2m + (int64_t)c * ncc * np, ncc, np, 0, min(R, nrhs - r0),
                                                       stage);
                        }
                        if (lane < np)
#pragma unroll
                            for (int r = 0; r < R; ++r)
                                if (r0 + r < nrhs) V.mult[(b * nrhs + r0 + r) * np + lane] = acc[0][r];
                    }
                    break;
                }
                const int64_t b = local / S.nchunk;
                const int p0 = (local % S.nchunk) * 32;
                const int ncc = 2 * V.pc + 1, np = 2 * V.p + 1;
                const int c = w & 3, half = (ncc + 1) / 2;
                int32_t lo, hi;
                box_range(I.lb, I.L, S.level + 1, 4 * b + c, &lo, &hi);
                for (int r0 = 0; r0 < nrhs; r0 += R) {
                    cf acc[1][R];
#pragma unroll
                    for (int r = 0; r < R; ++r) acc[0][r] = cfmk(0.f, 0.f);
                    if (hi > lo)
                        translate_source<R, 1>(acc, V.cmult + ((4 * b + c) * nrhs + r0) * (int64_t)ncc,
                                               V.Tm2m + (int64_t)c * ncc * np, ncc, np, p0, min(R, nrhs - r0), stage,
                                               (w >> 2) * half, (w >> 2) * half + half);
                    reduce_store<R, 1>(acc, red, V.mult, b * nrhs, nrhs, r0, np, p0);
                }
                break;
            }
            case PK_DOWN: {
                const PLev V = levs[I.lev0 + S.level];
                const int l = S.level;
                const int64_t b = S.wpb ? (int64_t)local * SM_W + w : local / S.nchunk;
                const int p0 = S.wpb ? 0 : (local % S.nchunk) * 32;
                if (S.wpb && b >= ((int64_t)1 << (2 * l))) break;   // warp-uniform
                int32_t lo, hi;
                box_range(I.lb, I.L, l, b, &lo, &hi);
                if (hi <= lo) break;                     // uniform over the CTA (over the warp when wpb)
                const int nc = 2 * V.p + 1, npp = 2 * V.pp + 1;
                const bool has_parent = V.ploc != nullptr;
                const int64_t Pb = b >> 2;
                const int nv0 = V.v_begin ? V.v_begin[b] : 0, nv1 = V.v_begin ? V.v_begin[b + 1] : 0;
                const int nr0 = V.r_begin ? V.r_begin[b] : 0, nr1 = V.r_begin ? V.r_begin[b + 1] : 0;
                const int nsrc = (has_parent ? 1 : 0) + (nv1 - nv0) + (nr1 - nr0);
                for (int r0 = 0; r0 < nrhs; r0 += R) {
                    const int rows = min(R, nrhs - r0);
                    cf acc[1][R];
#pragma unroll
                    for (int r = 0; r < R; ++r) acc[0][r] = cfmk(0.f, 0.f);
                    for (int s = S.wpb ? 0 : w; s < nsrc; s += S.wpb ? 1 : SM_W) {
                        if (has_parent && s == 0) {
                            translate_source<R, 1>(acc, V.ploc + (Pb * nrhs + r0) * (int64_t)npp,
                                                   V.Tl2l + (int64_t)(b & 3) * npp * nc, npp, nc, p0, rows, stage);
                            continue;
                        }
                        int e = s - (has_parent ? 1 : 0);
                        const cf* src;
                        const cf* M;
                        if (e < nv1 - nv0) {
                            src = V.mult + ((int64_t)V.v_src[nv0 + e] * nrhs + r0) * nc;
                            M = V.Tfree + (int64_t)V.v_off[nv0 + e] * nc * nc;
                        } else {
                            e -= nv1 - nv0;
                            src = V.mult + ((int64_t)V.r_src[nr0 + e] * nrhs + r0) * nc;
                            M = V.Treact + (int64_t)V.r_tab[nr0 + e] * nc * nc;
                        }
                        translate_source<R, 1>(acc, src, M, nc, nc, p0, rows, stage);
                    }
                    if (S.wpb) {
                        if (lane < nc)
#pragma unroll
                            for (int r = 0; r < R; ++r)
                                if (r0 + r < nrhs) V.loc[(b * nrhs + r0 + r) * nc + lane] = acc[0][r];
                    } else {
                        reduce_store<R, 1>(acc, red, V.loc, b * nrhs, nrhs, r0, nc, p0);
                    }
                }
                break;
            }
            case PK_NEAR: {
                const int64_t b = (int64_t)local * SM_W + w;
                if (b >= ((int64_t)1 << (2 * I.L))) break;
                const int32_t tlo = I.lb[b], thi = I.lb[b + 1];
                const int ix = (int)morton_x((uint32_t)b), iy = (int)morton_y((uint32_t)b);
                const int mside = 1 << I.L;
                const cf* loc = levs[I.lev0 + I.L].loc;
                const int nc = I.nc;
                const float h = I.h, k = I.k;
                for (int r0 = 0; r0 < nrhs; r0 += R)
                    for (int32_t t0 = tlo; t0 < thi; t0 += 32) {
                        const int32_t t = t0 + lane;
                        const bool live = t < thi;
                        const float2 tp = live ? I.xl[t] : make_float2(0.f, 0.f);
                        cf acc[R];
#pragma unroll
                        for (int r = 0; r < R; ++r) acc[r] = cfmk(0.f, 0.f);
                        for (int dy = -1; dy <= 1; ++dy)
                            for (int dx = -1; dx <= 1; ++dx) {
                                const int sx = ix + dx, sy = iy + dy;
                                if (sx < 0 || sy < 0 || sx >= mside || sy >= mside) continue;
                                const uint32_t sb = morton((uint32_t)sx, (uint32_t)sy);
                                const int32_t slo = I.lb[sb], shi = I.lb[sb + 1];
                                const float ox = (float)(-dx) * h, oy = (float)(-dy) * h;
                                for (int32_t j = slo; j < shi; ++j) {
                                    const float2 sp = I.xl[j];
                                    cf g = cfmk(0.f, 0.f);
                                    if (live && t != j) {
                                        const float ddx = ox + (tp.x - sp.x), ddy = oy + (tp.y - sp.y);
                                        const float z = k * sqrtf(ddx * ddx + ddy * ddy);
                                        if (z < H0_ZMAX) {
                                            g = green_tab(tj, tr, z);
                                        } else {
                                            const cd h0 = hankel0((double)z);
                                            g = cfmk((float)(-0.25 * h0.y), (float)(0.25 * h0.x));
                                        }
                                    }
#pragma unroll
                                    for (int r = 0; r < R; ++r)
                                        cfma(acc[r], g, r0 + r < nrhs ? __ldcg(I.q32 + (int64_t)j * nrhs + r0 + r)
                                                                      : cfmk(0.f, 0.f));
                                }
                            }
                        for (int m = 0; m < nc; ++m) {          // L2P
                            const cf B = live ? I.basis[(int64_t)t * nc + m] : cfmk(0.f, 0.f);
                            const cf g = cfmk(0.25f * B.y, 0.25f * B.x);
#pragma unroll
                            for (int r = 0; r < R; ++r)
                                cfma(acc[r], g, r0 + r < nrhs ? __ldcg(loc + (b * nrhs + r0 + r) * nc + m)
                                                              : cfmk(0.f, 0.f));
                        }
                        if (live)
#pragma unroll
                            for (int r = 0; r < R; ++r)
                                if (r0 + r < nrhs) I.y32[(int64_t)t * nrhs + r0 + r] = acc[r];   // first writer
                    }
                break;
            }
            case PK_DIRECT: {
                const int64_t b = local;
                const int32_t e0 = I.d_begin[b], e1 = I.d_begin[b + 1];
                if (e1 <= e0) break;
                const int32_t tlo = I.lb[b], tn = I.lb[b + 1] - tlo;
                for (int itm = tid; itm < nrhs * tn; itm += blockDim.x) {
                    const int i = itm / nrhs, r = itm % nrhs;
                    cf acc = cfmk(0.f, 0.f);
                    for (int32_t e = e0; e < e1; ++e) {
                        const int32_t sb = I.d_src[e];
                        const int32_t slo = I.lb[sb], sn = I.lb[sb + 1] - slo;
                        const cf* G = I.d_vals + I.d_blk[e] + (int64_t)i * sn;
                        for (int j = 0; j < sn; ++j) cfma(acc, G[j], __ldcg(I.q32 + (int64_t)(slo + j) * nrhs + r));
                    }
                    cf* yy = I.y32 + (int64_t)(tlo + i) * nrhs + r;
                    const cf v = __ldcg(yy);
                    *yy = cfmk(v.x + acc.x, v.y + acc.y);
                }
                break;
            }
        }
        // this item's writes are visible before it is counted
        __threadfence();
        __syncthreads();
        if (tid == 0) {
            atomicExch(done_item + it, 1);
            atomicAdd(done + s_seg, 1);
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
hfmm_status launch_down_ru(hfmm_plan_s* P, int l, int nrhs, int parts, int nchunk, int ncs_max, bool react_add,
                           cudaStream_t st) {
    LevelInfo& lv = P->lev[l];
    const bool has_parent = l > P->lmin;
    const size_t sm = smem_bytes(R, U, ncs_max);
    auto kern = down_small_kernel<R, U>;
    HFMM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    kern<<<(unsigned)(lv.nbox * nchunk), SM_W * 32, sm, st>>>(
        P->leaf_begin, P->L, l, P->lmin, nrhs, lv.p, has_parent ? P->lev[l - 1].p : 0,
        has_parent ? P->lev[l - 1].loc32 : nullptr, has_parent ? P->lev[l - 1].t_l2l32 : nullptr, lv.mult32,
        lv.nv ? lv.v_begin : nullptr, lv.v_src, lv.v_off, lv.t_free32, lv.nr ? lv.r_begin : nullptr, lv.r_src,
        lv.r_tab, lv.t_react32, parts, nchunk, ncs_max, lv.loc32, react_add, nullptr);
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
    HFMM_CUDA_TRY(cudaMemcpyToSymbolAsync(g_h0, h0_table_host(), sizeof(g_h0), 0, cudaMemcpyHostToDevice, st));
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

// Reaction lists only, added onto loc, over the boxes that have one: one
// right-hand side per pass and 32 warps per target box.  The lists concentrate on the boxes of the two lowest
// rows (up to 2^(l+1) sources each at level l, the other boxes none), so
// these few CTAs carry the pass and need the width.
template <int U>
hfmm_status launch_react_u(hfmm_plan_s* P, int l, int nrhs, int parts, int nchunk, int ncs_max, cudaStream_t st) {
    constexpr int NW = 32;
    LevelInfo& lv = P->lev[l];
    const size_t sm = sizeof(cf) * ((size_t)NW * ncs_max + (size_t)NW * U * 32);
    auto kern = down_small_kernel<1, U, NW>;
    HFMM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    if (lv.n_rtgt == 0) return HFMM_OK;
    kern<<<(unsigned)(lv.n_rtgt * nchunk), NW * 32, sm, st>>>(
        P->leaf_begin, P->L, l, P->lmin, nrhs, lv.p, 0, nullptr, nullptr, lv.mult32, nullptr, lv.v_src, lv.v_off,
        lv.t_free32, lv.r_begin, lv.r_src, lv.r_tab, lv.t_react32, parts, nchunk, ncs_max, lv.loc32, true, lv.r_tgt);
    HFMM_CUDA_TRY(cudaGetLastError());
    return HFMM_OK;
}

// Levels with at least 64 blocks of 32 boxes and at most 64 coefficients run
// L2L + V lists on vblock_kernel, then the reaction lists on down_small_kernel.
int vblock_cpt(const hfmm_plan_s* P, int l) {
    const LevelInfo& lv = P->lev[l];
    const int nc = lv.ncoef, npp = l > P->lmin ? P->lev[l - 1].ncoef : 0;
    if (l < 3 || lv.nbox < 64 * VB_T || nc > 64) return 0;
    const int cpt = nc <= 32 ? 2 : nc <= 48 ? 3 : 4;
    return vblock_smem(cpt, nc, npp) <= 200 * 1024 ? cpt : 0;
}

hfmm_status small_down(hfmm_plan_s* P, int l, int nrhs, int parts, cudaStream_t st) {
    LevelInfo& lv = P->lev[l];
    const bool has_parent = l > P->lmin;
    const int ncs_max = std::max(lv.ncoef, has_parent ? P->lev[l - 1].ncoef : 0);
    int U, nchunk;
    pick_u(lv.ncoef, lv.nbox, &U, &nchunk);
    const int R = pick_r(nrhs, ncs_max, U);
    if (const int cpt = vblock_cpt(P, l)) {
        const int nc = lv.ncoef, npp = has_parent ? P->lev[l - 1].ncoef : 0;
        const size_t sm = vblock_smem(cpt, nc, npp);
        const dim3 grid((unsigned)(lv.nbox / VB_T), (unsigned)nrhs);
        const cf* ploc = has_parent ? P->lev[l - 1].loc32 : nullptr;
        const cf* tl2l = has_parent ? P->lev[l - 1].t_l2l32 : nullptr;
        const int32_t* vb = ((parts & HFMM_PART_FAR_FREE) && lv.nv) ? lv.v_begin : nullptr;
#define HFMM_VBLOCK(C)                                                                                              \
    do {                                                                                                            \
        HFMM_CUDA_TRY(cudaFuncSetAttribute(vblock_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)); \
        vblock_kernel<C><<<grid, 128 * vb_nwc(C), sm, st>>>(P->leaf_begin, P->L, l, nrhs, nc, npp, ploc, tl2l, lv.mult32, vb,    \
                                                lv.v_off, lv.t_free32, lv.loc32);                                   \
    } while (0)
        if (cpt == 2) HFMM_VBLOCK(2);
        else if (cpt == 3) HFMM_VBLOCK(3);
        else HFMM_VBLOCK(4);
#undef HFMM_VBLOCK
        HFMM_CUDA_TRY(cudaGetLastError());
        if (!((parts & HFMM_PART_FAR_REACT) && lv.nr)) return HFMM_OK;
        ++P->launches;   // the caller counts the reaction launch below
        // nc <= 64 here, so U is 1 or 2
        if (U == 1) return launch_react_u<1>(P, l, nrhs, parts, nchunk, lv.ncoef, st);
        return launch_react_u<2>(P, l, nrhs, parts, nchunk, lv.ncoef, st);
    }
    // Levels with few (box, chunk) CTAs of plans with at least 2^17 points:
    // wider CTAs (16 or 32 warps splitting the box's sources, one right-hand
    // side per pass) keep more matrix rows in flight from L2 than 8-warp CTAs
    // that leave most SMs idle.  Smaller plans keep 8 warps: they are the
    // instances of batches, whose branches fill the SMs together and where wide
    // CTAs only block co-residency (measured 2.7 -> 3.3 ms on 32 instances of
    // 4k-120k points).  The choice depends on the plan alone, so a batch gives
    // the bits of its single-plan applies.
    const int64_t ncta = lv.nbox * nchunk;
    if (U == 1 && ncta < 8 * 152 && P->n >= (1 << 17)) {
        const int nw = ncta < 2 * 152 ? 32 : 16;
        const size_t sm = sizeof(cf) * ((size_t)nw * ncs_max + (size_t)nw * 32);
        if (sm <= 200 * 1024) {
            auto kern = nw == 32 ? down_small_kernel<1, 1, 32> : down_small_kernel<1, 1, 16>;
            HFMM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
            kern<<<(unsigned)ncta, nw * 32, sm, st>>>(
                P->leaf_begin, P->L, l, P->lmin, nrhs, lv.p, has_parent ? P->lev[l - 1].p : 0,
                has_parent ? P->lev[l - 1].loc32 : nullptr, has_parent ? P->lev[l - 1].t_l2l32 : nullptr, lv.mult32,
                lv.nv ? lv.v_begin : nullptr, lv.v_src, lv.v_off, lv.t_free32, lv.nr ? lv.r_begin : nullptr,
                lv.r_src, lv.r_tab, lv.t_react32, parts, nchunk, ncs_max, lv.loc32, false, nullptr);
            HFMM_CUDA_TRY(cudaGetLastError());
            return HFMM_OK;
        }
    }
    HFMM_SMALL_DISPATCH(launch_down_ru, P, l, nrhs, parts, nchunk, ncs_max, false, st)
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
    const double MAC = 8.0 * nrhs, C = 8.0 * nrhs;
    const bool far = (parts & (HFMM_PART_FAR_FREE | HFMM_PART_FAR_REACT)) != 0;
    const bool near = (parts & HFMM_PART_NEAR_FREE) != 0;
    // Both fields: the near field (first writer of y32 after the memset) runs on
    // a low-priority stream while the far-field chain runs on a high-priority
    // one and fills the SMs that the coarse levels' few CTAs leave idle; the
    // leaves' L2P then waits for it and adds into y32.
    const bool concurrent = far && near;
    cudaStream_t fs = st;
    if (concurrent) {
        HFMM_TRY(fork_near_far(P, st));
        StageTimer tn{P, P->near_st};
        tn.begin(HFMM_STAGE_P2P);
        HFMM_TRY(small_near(P, nrhs, true, false, P->near_st));
        ++P->launches;
        tn.end(HFMM_STAGE_P2P);
        HFMM_CUDA_TRY(cudaEventRecord(P->ev_near_done, P->near_st));
        fs = P->far_st;
    }
    StageTimer tm{P, fs};
    if (far) {
        LevelInfo& leaf = P->lev[L];
        tm.begin(HFMM_STAGE_P2M);
        HFMM_TRY(small_p2m(P, nrhs, fs));
        ++P->launches;
        tm.end(HFMM_STAGE_P2M);
        P->st_flops[HFMM_STAGE_P2M] = MAC * n * leaf.ncoef;
        P->st_bytes[HFMM_STAGE_P2M] = C * n + 8.0 * n * leaf.ncoef + C * leaf.nbox * leaf.ncoef;
        tm.begin(HFMM_STAGE_M2M);
        for (int l = L - 1; l >= P->lmin; --l) {
            LevelInfo& lv = P->lev[l];
            HFMM_TRY(small_m2m(P, l, nrhs, fs));
            ++P->launches;
            P->st_flops[HFMM_STAGE_M2M] += MAC * 4.0 * lv.nbox * lv.ncoef * P->lev[l + 1].ncoef;
            P->st_bytes[HFMM_STAGE_M2M] += C * (4.0 * lv.nbox * P->lev[l + 1].ncoef + lv.nbox * lv.ncoef);
        }
        tm.end(HFMM_STAGE_M2M);
        tm.begin(HFMM_STAGE_DOWN);
        for (int l = P->lmin; l <= L; ++l) {
            LevelInfo& lv = P->lev[l];
            HFMM_TRY(small_down(P, l, nrhs, parts, fs));
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
        if (concurrent) {
            // the leaves' L2P after the near field (both add into y32)
            HFMM_CUDA_TRY(cudaStreamWaitEvent(fs, P->ev_near_done, 0));
            HFMM_TRY(small_near(P, nrhs, false, true, fs));
            ++P->launches;
            HFMM_CUDA_TRY(cudaEventRecord(P->ev_far_done, fs));
            HFMM_CUDA_TRY(cudaStreamWaitEvent(st, P->ev_far_done, 0));
        } else {
            tm.begin(HFMM_STAGE_P2P);
            HFMM_TRY(small_near(P, nrhs, near, far, st));
            ++P->launches;
            tm.end(HFMM_STAGE_P2P);
        }
        P->st_flops[HFMM_STAGE_P2P] = (near ? MAC * (double)P->p2p_point_pairs : 0.0) +
                                      (far ? MAC * n * leaf.ncoef : 0.0);
        P->st_bytes[HFMM_STAGE_P2P] = 3.0 * C * n + 16.0 * n + (far ? C * leaf.nbox * leaf.ncoef + 8.0 * n * leaf.ncoef : 0.0);
    }
    return HFMM_OK;
}

// ---------------------------------------------------------------------------
// Persistent batch: host side
// ---------------------------------------------------------------------------
struct PersistBatch {
    std::vector<PSeg> segs;
    std::vector<PInst> inst;
    std::vector<PLev> lev;
    int total = 0;
    int ncs_max = 1;
    long spin = 0;
    PSeg* d_segs = nullptr;
    PInst* d_inst = nullptr;
    PLev* d_lev = nullptr;
    int* d_ctr = nullptr;            // [0] next item, [1] error flag, [2 ..] done per segment, then per item
    int grid[4] = {0, 0, 0, 0};      // persistent CTAs for R = 1, 2, 4, 8
};

namespace {

size_t persist_smem(PersistBatch* B, int R) {
    return smem_bytes(R, 1, B->ncs_max) + sizeof(int) * B->segs.size();
}

template <int R>
hfmm_status persist_grid(PersistBatch* B, int* grid) {
    const size_t sm = persist_smem(B, R);
    auto kern = persist_kernel<R>;
    HFMM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    int per_sm = 0, dev = 0, nsm = 0;
    HFMM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, SM_W * 32, sm));
    HFMM_CUDA_TRY(cudaGetDevice(&dev));
    HFMM_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    if (per_sm < 1) {
        hfmm_set_error("persistent batch kernel does not fit an SM (%zu bytes of shared memory)", sm);
        return HFMM_ERR_UNSUPPORTED;
    }
    *grid = std::max(1, std::min(B->total, per_sm * nsm));
    return HFMM_OK;
}

template <int R>
hfmm_status persist_go(PersistBatch* B, int nrhs, bool adjoint, cudaStream_t st, int grid) {
    const size_t sm = persist_smem(B, R);
    persist_kernel<R><<<grid, SM_W * 32, sm, st>>>(B->d_segs, (int)B->segs.size(), B->total, B->d_inst, B->d_lev,
                                                  nrhs, adjoint ? 1 : 0, B->ncs_max, B->d_ctr, B->spin);
    HFMM_CUDA_TRY(cudaGetLastError());
    return HFMM_OK;
}

}  // namespace

void persist_destroy(PersistBatch* B) {
    if (!B) return;
    cudaFree(B->d_segs);
    cudaFree(B->d_inst);
    cudaFree(B->d_lev);
    cudaFree(B->d_ctr);
    delete B;
}

hfmm_status persist_create(const std::vector<hfmm_plan_s*>& plans, PersistBatch** out) {
    *out = nullptr;
    PersistBatch* B = new (std::nothrow) PersistBatch();
    if (!B) { hfmm_set_error("host allocation failed"); return HFMM_ERR_OOM; }
    const int ni = (int)plans.size();
    int Lmax = 0, dmax = 0;
    for (int i = 0; i < ni; ++i) {
        hfmm_plan_s* P = plans[i];
        PInst I{};
        I.lb = P->leaf_begin;
        I.L = P->L;
        I.lmin = P->lmin;
        I.lev0 = (int)B->lev.size();
        I.nc = P->lev[P->L].ncoef;
        I.n = P->n;
        I.k = (float)P->k;
        I.h = (float)P->lev[P->L].h;
        I.xl = P->xl32;
        I.basis = P->basis32;
        I.q32 = P->q32;
        I.y32 = P->y32;
        I.iperm = P->iperm32;
        I.d_begin = P->d_begin;
        I.d_src = P->d_src;
        I.d_blk = P->d_blk;
        I.d_vals = P->d_vals32;
        B->inst.push_back(I);
        for (int l = 0; l <= P->L; ++l) {
            const LevelInfo& lv = P->lev[l];
            PLev V{};
            if (l >= P->lmin) {
                V.p = lv.p;
                V.pp = l > P->lmin ? P->lev[l - 1].p : 0;
                V.pc = l < P->L ? P->lev[l + 1].p : 0;
                V.mult = lv.mult32;
                V.loc = lv.loc32;
                V.cmult = l < P->L ? P->lev[l + 1].mult32 : nullptr;
                V.ploc = l > P->lmin ? P->lev[l - 1].loc32 : nullptr;
                V.Tl2l = l > P->lmin ? P->lev[l - 1].t_l2l32 : nullptr;
                V.Tfree = lv.t_free32;
                V.Treact = lv.t_react32;
                V.Tm2m = lv.t_m2m32;
                V.v_begin = lv.nv ? lv.v_begin : nullptr;
                V.v_src = lv.v_src;
                V.v_off = lv.v_off;
                V.r_begin = lv.nr ? lv.r_begin : nullptr;
                V.r_src = lv.r_src;
                V.r_tab = lv.r_tab;
                B->ncs_max = std::max({B->ncs_max, lv.ncoef, l > P->lmin ? P->lev[l - 1].ncoef : 0,
                                       l < P->L ? P->lev[l + 1].ncoef : 0});
            }
            B->lev.push_back(V);
        }
        Lmax = std::max(Lmax, P->L);
        dmax = std::max(dmax, P->L - P->lmin);
        B->spin = std::max(B->spin, P->tc_spin);
    }
    // segments in dependency order; seg index of (stage, instance[, level])
    auto add = [&](int kind, int inst, int level, int nitems, int nchunk, int d0, int d1, int wpb = 0,
                   int idep = -1, int irel = 0) {
        PSeg S{kind, inst, level, nchunk, B->total, nitems, d0, d1, wpb, idep, irel, 0};
        B->total += nitems;
        B->segs.push_back(S);
        return (int)B->segs.size() - 1;
    };
    std::vector<int> s_gather(ni), s_p2m(ni), s_near(ni), s_direct(ni, -1);
    std::vector<std::vector<int>> s_up(ni), s_down(ni);
    for (int i = 0; i < ni; ++i) {
        s_up[i].assign(plans[i]->L + 1, -1);
        s_down[i].assign(plans[i]->L + 1, -1);
    }
    for (int i = 0; i < ni; ++i) s_gather[i] = add(PK_GATHER, i, 0, ceil_div(plans[i]->n, 64), 1, -1, -1);
    for (int i = 0; i < ni; ++i) {
        s_p2m[i] = add(PK_P2M, i, plans[i]->L, ceil_div(plans[i]->lev[plans[i]->L].nbox, SM_W), 1, s_gather[i], -1, 1);
        s_up[i][plans[i]->L] = s_p2m[i];
    }
    for (int d = 1; d <= dmax; ++d)
        for (int i = 0; i < ni; ++i) {
            hfmm_plan_s* P = plans[i];
            const int l = P->L - d;
            if (l < P->lmin) continue;
            const int nchunk = (P->lev[l].ncoef + 31) / 32;
            if (nchunk == 1 && P->lev[l].nbox >= 4 * SM_W)
                s_up[i][l] = add(PK_M2M, i, l, ceil_div(P->lev[l].nbox, SM_W), 1, -1, -1, 1, s_up[i][l + 1], 1);
            else
                s_up[i][l] = add(PK_M2M, i, l, (int)(P->lev[l].nbox * nchunk), nchunk, -1, -1, 0, s_up[i][l + 1], 1);
        }
    // downward passes top level first over all instances, then the near
    // fields, direct reactions and scatters
    for (int l = 0; l <= Lmax; ++l)
        for (int i = 0; i < ni; ++i) {
            hfmm_plan_s* P = plans[i];
            if (l < P->lmin || l > P->L) continue;
            const int nchunk = (P->lev[l].ncoef + 31) / 32;
            const int dprev = l > P->lmin ? s_down[i][l - 1] : -1;
            if (nchunk == 1 && P->lev[l].nbox >= 4 * SM_W)
                s_down[i][l] = add(PK_DOWN, i, l, ceil_div(P->lev[l].nbox, SM_W), 1, s_up[i][l], -1, 1, dprev, 2);
            else
                s_down[i][l] = add(PK_DOWN, i, l, (int)(P->lev[l].nbox * nchunk), nchunk, s_up[i][l], -1, 0, dprev, 2);
        }
    for (int i = 0; i < ni; ++i) {
        hfmm_plan_s* P = plans[i];
        s_near[i] = add(PK_NEAR, i, P->L, ceil_div(P->lev[P->L].nbox, SM_W), 1, s_gather[i], -1, 1, s_down[i][P->L], 0);
    }
    for (int i = 0; i < ni; ++i)
        if (plans[i]->nd > 0)
            s_direct[i] = add(PK_DIRECT, i, plans[i]->L, (int)plans[i]->lev[plans[i]->L].nbox, 1, -1, -1, 0,
                              s_near[i], 0);
    for (int i = 0; i < ni; ++i)
        add(PK_SCATTER, i, 0, ceil_div(plans[i]->n, 64), 1, s_direct[i] >= 0 ? s_direct[i] : s_near[i], -1);
    hfmm_status s = HFMM_OK;
    auto fail = [&](cudaError_t e) {
        hfmm_set_error("persistent batch setup: %s", cudaGetErrorString(e));
        persist_destroy(B);
        return e == cudaErrorMemoryAllocation ? HFMM_ERR_OOM : HFMM_ERR_CUDA;
    };
    cudaError_t e = cudaMalloc(&B->d_segs, sizeof(PSeg) * B->segs.size());
    if (e == cudaSuccess) e = cudaMalloc(&B->d_inst, sizeof(PInst) * B->inst.size());
    if (e == cudaSuccess) e = cudaMalloc(&B->d_lev, sizeof(PLev) * B->lev.size());
    if (e == cudaSuccess) e = cudaMalloc(&B->d_ctr, sizeof(int) * (2 + B->segs.size() + B->total));
    if (e == cudaSuccess)
        e = cudaMemcpy(B->d_segs, B->segs.data(), sizeof(PSeg) * B->segs.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(B->d_lev, B->lev.data(), sizeof(PLev) * B->lev.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(B->d_ctr, 0, sizeof(int) * (2 + B->segs.size() + B->total));
    if (e != cudaSuccess) return fail(e);
    if ((s = persist_grid<1>(B, &B->grid[0])) != HFMM_OK || (s = persist_grid<2>(B, &B->grid[1])) != HFMM_OK ||
        (s = persist_grid<4>(B, &B->grid[2])) != HFMM_OK || (s = persist_grid<8>(B, &B->grid[3])) != HFMM_OK) {
        persist_destroy(B);
        return s;
    }
    *out = B;
    return HFMM_OK;
}

hfmm_status persist_set_buffers(PersistBatch* B, const void* const* q, void* const* y, cudaStream_t st) {
    for (size_t i = 0; i < B->inst.size(); ++i) {
        B->inst[i].q = (const cf*)q[i];
        B->inst[i].y = (cf*)y[i];
    }
    HFMM_CUDA_TRY(cudaMemcpyAsync(B->d_inst, B->inst.data(), sizeof(PInst) * B->inst.size(), cudaMemcpyHostToDevice,
                                  st));
    HFMM_CUDA_TRY(cudaStreamSynchronize(st));
    return HFMM_OK;
}

hfmm_status persist_launch(PersistBatch* B, int nrhs, bool adjoint, cudaStream_t st) {
    HFMM_CUDA_TRY(cudaMemsetAsync(B->d_ctr, 0, sizeof(int) * (2 + B->segs.size() + B->total), st));
    if (nrhs >= 8) return persist_go<8>(B, nrhs, adjoint, st, B->grid[3]);
    if (nrhs >= 4) return persist_go<4>(B, nrhs, adjoint, st, B->grid[2]);
    if (nrhs >= 2) return persist_go<2>(B, nrhs, adjoint, st, B->grid[1]);
    return persist_go<1>(B, nrhs, adjoint, st, B->grid[0]);
}

hfmm_status persist_device_error(PersistBatch* B, int* err) {
    HFMM_CUDA_TRY(cudaDeviceSynchronize());
    HFMM_CUDA_TRY(cudaMemcpy(err, B->d_ctr + 1, sizeof(int), cudaMemcpyDeviceToHost));
    return HFMM_OK;
}
