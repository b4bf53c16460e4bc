// Quadtree construction on the device (Algorithm 1, step 1; Sec. 3.1):
// bounding square, leaf keys, stable Morton sort, leaf ranges, and the
// interaction lists (free-space V lists, reaction lists, direct pairs).
#include <algorithm>
#include <cmath>
#include <vector>

#include "plan.cuh"

namespace {

constexpr int SCAN_BLOCK = 1024;

// ---------------------------------------------------------------------------
// exclusive scan of int32 (multi-block: block sums, scan of sums, add)
// ---------------------------------------------------------------------------
__global__ void scan_block_sums(const int32_t* in, int64_t n, int32_t* sums) {
    __shared__ int32_t sh[SCAN_BLOCK / 32];
    int64_t i = (int64_t)blockIdx.x * SCAN_BLOCK + threadIdx.x;
    int32_t v = (i < n) ? in[i] : 0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        int32_t w = (threadIdx.x < SCAN_BLOCK / 32) ? sh[threadIdx.x] : 0;
        for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(0xffffffffu, w, o);
        if (threadIdx.x == 0) sums[blockIdx.x] = w;
    }
}

// single CTA: exclusive scan of `sums` in place, total to *total
__global__ void scan_sums(int32_t* sums, int64_t m, int32_t* total) {
    __shared__ int32_t sh[SCAN_BLOCK];
    __shared__ int32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < m; base += SCAN_BLOCK) {
        int64_t i = base + threadIdx.x;
        int32_t v = (i < m) ? sums[i] : 0;
        sh[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < SCAN_BLOCK; o <<= 1) {
            int32_t t = (threadIdx.x >= o) ? sh[threadIdx.x - o] : 0;
            __syncthreads();
            sh[threadIdx.x] += t;
            __syncthreads();
        }
        int32_t incl = sh[threadIdx.x];
        if (i < m) sums[i] = carry + incl - v;
        __syncthreads();
        if (threadIdx.x == SCAN_BLOCK - 1) carry += incl;
        __syncthreads();
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void scan_apply(const int32_t* in, int64_t n, const int32_t* sums, int32_t* out) {
    __shared__ int32_t sh[SCAN_BLOCK];
    int64_t i = (int64_t)blockIdx.x * SCAN_BLOCK + threadIdx.x;
    int32_t v = (i < n) ? in[i] : 0;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < SCAN_BLOCK; o <<= 1) {
        int32_t t = (threadIdx.x >= o) ? sh[threadIdx.x - o] : 0;
        __syncthreads();
        sh[threadIdx.x] += t;
        __syncthreads();
    }
    if (i < n) out[i] = sums[blockIdx.x] + sh[threadIdx.x] - v;
}

// out[i] = sum_{j<i} in[j] for i < n, out[n] = total (out has n + 1 entries).
hfmm_status exclusive_scan(const int32_t* in, int32_t* out, int64_t n, int32_t* tmp,
                           cudaStream_t st) {
    const int64_t nb = (n + SCAN_BLOCK - 1) / SCAN_BLOCK;
    if (nb > 0) {
        scan_block_sums<<<(unsigned)nb, SCAN_BLOCK, 0, st>>>(in, n, tmp);
        scan_sums<<<1, SCAN_BLOCK, 0, st>>>(tmp, nb, out + n);
        scan_apply<<<(unsigned)nb, SCAN_BLOCK, 0, st>>>(in, n, tmp, out);
    } else {
        HFMM_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(int32_t), st));
    }
    HFMM_CUDA_TRY(cudaGetLastError());
    return HFMM_OK;
}

// ---------------------------------------------------------------------------
// bounding box and keys
// ---------------------------------------------------------------------------
__global__ void bbox_partial(const double* xy, int64_t n, double* part) {
    __shared__ double s[4][256];
    double mnx = INFINITY, mny = INFINITY, mxx = -INFINITY, mxy = -INFINITY;
    int bad = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double x = xy[2 * i], y = xy[2 * i + 1];
        if (!isfinite(x) || !isfinite(y)) bad = 1;
        mnx = fmin(mnx, x); mny = fmin(mny, y);
        mxx = fmax(mxx, x); mxy = fmax(mxy, y);
    }
    if (bad) mnx = NAN;
    s[0][threadIdx.x] = mnx; s[1][threadIdx.x] = mny;
    s[2][threadIdx.x] = mxx; s[3][threadIdx.x] = mxy;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            double a = s[0][threadIdx.x], b = s[0][threadIdx.x + o];
            s[0][threadIdx.x] = (isnan(a) || isnan(b)) ? NAN : fmin(a, b);
            s[1][threadIdx.x] = fmin(s[1][threadIdx.x], s[1][threadIdx.x + o]);
            s[2][threadIdx.x] = fmax(s[2][threadIdx.x], s[2][threadIdx.x + o]);
            s[3][threadIdx.x] = fmax(s[3][threadIdx.x], s[3][threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        for (int c = 0; c < 4; ++c) part[4 * blockIdx.x + c] = s[c][0];
    }
}

__global__ void leaf_keys(const double* xy, int64_t n, double x0, double y0, double scale,
                          uint32_t mmax, uint32_t* key, int32_t* val) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double fx = floor((xy[2 * i] - x0) * scale);
    double fy = floor((xy[2 * i + 1] - y0) * scale);
    uint32_t ix = (uint32_t)fmin(fmax(fx, 0.0), (double)mmax);
    uint32_t iy = (uint32_t)fmin(fmax(fy, 0.0), (double)mmax);
    key[i] = morton(ix, iy);
    val[i] = (int32_t)i;
}

__global__ void split_flags(const uint32_t* key, int64_t n, int bit, int32_t* zero) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) zero[i] = ((key[i] >> bit) & 1u) ? 0 : 1;
}

__global__ void split_scatter(const uint32_t* key, const int32_t* val, const int32_t* pos0,
                              int64_t n, int bit, uint32_t* key2, int32_t* val2) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t nzero = pos0[n];
    uint32_t k = key[i];
    int64_t dst = ((k >> bit) & 1u) ? (int64_t)nzero + (i - pos0[i]) : (int64_t)pos0[i];
    key2[dst] = k;
    val2[dst] = val[i];
}

__global__ void leaf_histogram(const uint32_t* key, int64_t n, int32_t* cnt) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) atomicAdd(&cnt[key[i]], 1);
}

__global__ void gather_sorted(const double* xy, const int32_t* val, int64_t n, double2* xs,
                              int64_t* perm) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t j = val[i];
    xs[i] = make_double2(xy[2 * j], xy[2 * j + 1]);
    perm[i] = j;
}

// ---------------------------------------------------------------------------
// lists
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool box_nonempty(const int32_t* lb, int L, int l, int64_t b) {
    int32_t lo, hi;
    box_range(lb, L, l, b, &lo, &hi);
    return hi > lo;
}

// V list of target b at level l >= 2: children of the parent's neighbours
// that are not neighbours of b.  count_only: write the count, else fill.
__global__ void v_list_kernel(const int32_t* lb, int L, int l, const int32_t* begin,
                              int32_t* cnt, int32_t* src, int32_t* off) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nbox = (int64_t)1 << (2 * l);
    if (b >= nbox) return;
    const int m = 1 << l;
    int ix = (int)morton_x((uint32_t)b), iy = (int)morton_y((uint32_t)b);
    int c = 0;
    int32_t w = begin ? begin[b] : 0;
    if (box_nonempty(lb, L, l, b)) {
        int px = ix >> 1, py = iy >> 1;
        for (int qx = px - 1; qx <= px + 1; ++qx)
            for (int qy = py - 1; qy <= py + 1; ++qy)
                for (int cx = 0; cx < 2; ++cx)
                    for (int cy = 0; cy < 2; ++cy) {
                        int sx = 2 * qx + cx, sy = 2 * qy + cy;
                        if (sx < 0 || sy < 0 || sx >= m || sy >= m) continue;
                        int dx = ix - sx, dy = iy - sy;
                        if (abs(dx) < 2 && abs(dy) < 2) continue;
                        int64_t s = morton((uint32_t)sx, (uint32_t)sy);
                        if (!box_nonempty(lb, L, l, s)) continue;
                        if (src) {
                            src[w + c] = (int32_t)s;
                            off[w + c] = (dx + 3) * 7 + (dy + 3);
                        }
                        ++c;
                    }
    }
    if (cnt) cnt[b] = c;
}

// Reaction list of target b at level l (1 <= l <= min(lstar, L)): sources in
// rows 0 and 1 that pass the admissibility test.  Level 0: the root pair when
// it is admissible.  Table entry of (dx, ysum): (dx + 2^l - 1) * 3 + ysum.
__global__ void r_list_kernel(const int32_t* lb, int L, int l, int lstar, double y0, double hl,
                              const int32_t* begin, int32_t* cnt, int32_t* src, int32_t* tab) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nbox = (int64_t)1 << (2 * l);
    if (b >= nbox) return;
    int c = 0;
    int32_t w = begin ? begin[b] : 0;
    if (box_nonempty(lb, L, l, b)) {
        if (l == 0) {
            if (lstar == 0) {
                if (src) { src[w] = 0; tab[w] = 0; }
                c = 1;
            }
        } else if (l <= lstar) {
            const int m = 1 << l;
            int ix = (int)morton_x((uint32_t)b), iy = (int)morton_y((uint32_t)b);
            if (iy <= 1) {
                for (int sy = 0; sy <= 1 && sy < m; ++sy)
                    for (int sx = 0; sx < m; ++sx) {
                        if (!reaction_admissible(iy, sy, y0, hl)) continue;
                        int64_t s = morton((uint32_t)sx, (uint32_t)sy);
                        if (!box_nonempty(lb, L, l, s)) continue;
                        if (src) {
                            src[w + c] = (int32_t)s;
                            tab[w + c] = (ix - sx + (m - 1)) * 3 + (iy + sy);
                        }
                        ++c;
                    }
            }
        }
    }
    if (cnt) cnt[b] = c;
}

// Directly summed reaction (lstar > L): leaf pairs in the bottom row.
__global__ void d_list_kernel(const int32_t* lb, int L, const int32_t* begin, int32_t* cnt,
                              int32_t* src) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nbox = (int64_t)1 << (2 * L);
    if (b >= nbox) return;
    int c = 0;
    int32_t w = begin ? begin[b] : 0;
    const int m = 1 << L;
    if (morton_y((uint32_t)b) == 0 && box_nonempty(lb, L, L, b)) {
        for (int sx = 0; sx < m; ++sx) {
            int64_t s = morton((uint32_t)sx, 0u);
            if (!box_nonempty(lb, L, L, s)) continue;
            if (src) src[w + c] = (int32_t)s;
            ++c;
        }
    }
    if (cnt) cnt[b] = c;
}

}  // namespace

// ---------------------------------------------------------------------------
hfmm_status build_tree(hfmm_plan_s* P, const double* d_xy, cudaStream_t st) {
    const int64_t n = P->n;
    const int TB = 256;
    // bounding box
    const int nbb = 256;
    double* part = nullptr;
    HFMM_TRY(plan_alloc(P, (void**)&part, sizeof(double) * 4 * nbb));
    bbox_partial<<<nbb, 256, 0, st>>>(d_xy, n, part);
    HFMM_CUDA_TRY(cudaGetLastError());
    std::vector<double> hp(4 * nbb);
    HFMM_CUDA_TRY(cudaMemcpyAsync(hp.data(), part, sizeof(double) * 4 * nbb, cudaMemcpyDeviceToHost, st));
    HFMM_CUDA_TRY(cudaStreamSynchronize(st));
    double mnx = INFINITY, mny = INFINITY, mxx = -INFINITY, mxy = -INFINITY;
    for (int b = 0; b < nbb; ++b) {
        if (std::isnan(hp[4 * b])) {
            hfmm_set_error("hfmm_plan_create: non-finite point coordinates");
            return HFMM_ERR_INVALID_ARG;
        }
        mnx = std::min(mnx, hp[4 * b]); mny = std::min(mny, hp[4 * b + 1]);
        mxx = std::max(mxx, hp[4 * b + 2]); mxy = std::max(mxy, hp[4 * b + 3]);
    }
    if (!(mny > 0.0)) {
        hfmm_set_error("hfmm_plan_create: all points must lie in the top layer y > 0 (min y = %g)", mny);
        return HFMM_ERR_INVALID_ARG;
    }
    P->x0 = mnx;
    P->y0 = mny;
    double S = std::max(mxx - mnx, mxy - mny);
    if (!(S > 0.0)) S = 1.0;
    P->S = S;
    const int L = P->L;
    const uint32_t m = 1u << L;
    const double scale = (double)m / S;
    const int64_t nleaf = (int64_t)1 << (2 * L);

    uint32_t *key = nullptr, *key2 = nullptr;
    int32_t *val = nullptr, *val2 = nullptr, *flag = nullptr, *pos = nullptr, *tmp = nullptr;
    HFMM_TRY(plan_alloc(P, (void**)&key, sizeof(uint32_t) * n));
    HFMM_TRY(plan_alloc(P, (void**)&key2, sizeof(uint32_t) * n));
    HFMM_TRY(plan_alloc(P, (void**)&val, sizeof(int32_t) * n));
    HFMM_TRY(plan_alloc(P, (void**)&val2, sizeof(int32_t) * n));
    const int64_t nmax = std::max<int64_t>(n, nleaf);
    HFMM_TRY(plan_alloc(P, (void**)&flag, sizeof(int32_t) * (nmax + 1)));
    HFMM_TRY(plan_alloc(P, (void**)&pos, sizeof(int32_t) * (nmax + 1)));
    HFMM_TRY(plan_alloc(P, (void**)&tmp, sizeof(int32_t) * (nmax / SCAN_BLOCK + 2)));

    leaf_keys<<<ceil_div(n, TB), TB, 0, st>>>(d_xy, n, P->x0, P->y0, scale, m - 1, key, val);
    HFMM_CUDA_TRY(cudaGetLastError());
    // stable LSD radix-2 sort over the 2L key bits
    for (int bit = 0; bit < 2 * L; ++bit) {
        split_flags<<<ceil_div(n, TB), TB, 0, st>>>(key, n, bit, flag);
        HFMM_TRY(exclusive_scan(flag, pos, n, tmp, st));
        split_scatter<<<ceil_div(n, TB), TB, 0, st>>>(key, val, pos, n, bit, key2, val2);
        HFMM_CUDA_TRY(cudaGetLastError());
        std::swap(key, key2);
        std::swap(val, val2);
    }
    // leaf ranges
    HFMM_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(int32_t) * nleaf, st));
    leaf_histogram<<<ceil_div(n, TB), TB, 0, st>>>(key, n, flag);
    HFMM_TRY(plan_alloc(P, (void**)&P->leaf_begin, sizeof(int32_t) * (nleaf + 1)));
    HFMM_TRY(exclusive_scan(flag, P->leaf_begin, nleaf, tmp, st));
    HFMM_TRY(plan_alloc(P, (void**)&P->xy_sorted, sizeof(double2) * n));
    HFMM_TRY(plan_alloc(P, (void**)&P->perm, sizeof(int64_t) * n));
    gather_sorted<<<ceil_div(n, TB), TB, 0, st>>>(d_xy, val, n, P->xy_sorted, P->perm);
    HFMM_CUDA_TRY(cudaGetLastError());
    P->h_leaf_begin.resize(nleaf + 1);
    HFMM_CUDA_TRY(cudaMemcpyAsync(P->h_leaf_begin.data(), P->leaf_begin, sizeof(int32_t) * (nleaf + 1),
                                  cudaMemcpyDeviceToHost, st));
    HFMM_CUDA_TRY(cudaStreamSynchronize(st));
    return HFMM_OK;
}

// ---------------------------------------------------------------------------
static hfmm_status build_csr(hfmm_plan_s* P, int64_t nbox, int32_t** begin, int64_t* total,
                             cudaStream_t st, int32_t* cnt, int32_t* tmp) {
    HFMM_TRY(plan_alloc(P, (void**)begin, sizeof(int32_t) * (nbox + 1)));
    HFMM_TRY(exclusive_scan(cnt, *begin, nbox, tmp, st));
    int32_t t = 0;
    HFMM_CUDA_TRY(cudaMemcpyAsync(&t, *begin + nbox, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    HFMM_CUDA_TRY(cudaStreamSynchronize(st));
    *total = t;
    return HFMM_OK;
}

hfmm_status build_lists(hfmm_plan_s* P, cudaStream_t st) {
    const int L = P->L;
    const int TB = 256;
    const int64_t nleaf = (int64_t)1 << (2 * L);
    int32_t *cnt = nullptr, *tmp = nullptr;
    HFMM_TRY(plan_alloc(P, (void**)&cnt, sizeof(int32_t) * (nleaf + 1)));
    HFMM_TRY(plan_alloc(P, (void**)&tmp, sizeof(int32_t) * (nleaf / SCAN_BLOCK + 2)));
    // first level whose bottom-row pairs are admissible
    int lstar = L + 1;
    for (int l = 0; l <= L; ++l) {
        if (2.0 * P->y0 >= P->S / (double)(1 << l)) { lstar = l; break; }
    }
    P->lstar = lstar;
    for (int l = 0; l <= L; ++l) {
        LevelInfo& lv = P->lev[l];
        const int64_t nbox = lv.nbox;
        // V lists
        if (l >= 2) {
            v_list_kernel<<<ceil_div(nbox, TB), TB, 0, st>>>(P->leaf_begin, L, l, nullptr, cnt, nullptr, nullptr);
            HFMM_CUDA_TRY(cudaGetLastError());
            HFMM_TRY(build_csr(P, nbox, &lv.v_begin, &lv.nv, st, cnt, tmp));
            if (lv.nv > 0) {
                HFMM_TRY(plan_alloc(P, (void**)&lv.v_src, sizeof(int32_t) * lv.nv));
                HFMM_TRY(plan_alloc(P, (void**)&lv.v_off, sizeof(int32_t) * lv.nv));
                v_list_kernel<<<ceil_div(nbox, TB), TB, 0, st>>>(P->leaf_begin, L, l, lv.v_begin, nullptr, lv.v_src, lv.v_off);
                HFMM_CUDA_TRY(cudaGetLastError());
            }
        }
        // reaction lists
        r_list_kernel<<<ceil_div(nbox, TB), TB, 0, st>>>(P->leaf_begin, L, l, lstar, P->y0, lv.h, nullptr, cnt, nullptr, nullptr);
        HFMM_CUDA_TRY(cudaGetLastError());
        HFMM_TRY(build_csr(P, nbox, &lv.r_begin, &lv.nr, st, cnt, tmp));
        if (lv.nr > 0) {
            HFMM_TRY(plan_alloc(P, (void**)&lv.r_src, sizeof(int32_t) * lv.nr));
            HFMM_TRY(plan_alloc(P, (void**)&lv.r_tab, sizeof(int32_t) * lv.nr));
            r_list_kernel<<<ceil_div(nbox, TB), TB, 0, st>>>(P->leaf_begin, L, l, lstar, P->y0, lv.h, lv.r_begin, nullptr, lv.r_src, lv.r_tab);
            HFMM_CUDA_TRY(cudaGetLastError());
            // the boxes that have a reaction list (the few-RHS reaction pass runs over these only)
            std::vector<int32_t> rb(nbox + 1), tg;
            HFMM_CUDA_TRY(cudaMemcpyAsync(rb.data(), lv.r_begin, sizeof(int32_t) * (nbox + 1), cudaMemcpyDeviceToHost, st));
            HFMM_CUDA_TRY(cudaStreamSynchronize(st));
            for (int64_t b = 0; b < nbox; ++b)
                if (rb[b + 1] > rb[b]) tg.push_back((int32_t)b);
            lv.n_rtgt = (int64_t)tg.size();
            HFMM_TRY(plan_alloc(P, (void**)&lv.r_tgt, sizeof(int32_t) * tg.size()));
            HFMM_CUDA_TRY(cudaMemcpyAsync(lv.r_tgt, tg.data(), sizeof(int32_t) * tg.size(), cudaMemcpyHostToDevice, st));
            HFMM_CUDA_TRY(cudaStreamSynchronize(st));
        }
    }
    // the coarsest level with work
    int lmin = L;
    for (int l = 0; l <= L; ++l) {
        if (P->lev[l].nr > 0 || P->lev[l].nv > 0) { lmin = l; break; }
    }
    P->lmin = lmin;
    // direct reaction pairs
    if (lstar > L) {
        d_list_kernel<<<ceil_div(nleaf, TB), TB, 0, st>>>(P->leaf_begin, L, nullptr, cnt, nullptr);
        HFMM_CUDA_TRY(cudaGetLastError());
        HFMM_TRY(build_csr(P, nleaf, &P->d_begin, &P->nd, st, cnt, tmp));
        if (P->nd > 0) {
            HFMM_TRY(plan_alloc(P, (void**)&P->d_src, sizeof(int32_t) * P->nd));
            d_list_kernel<<<ceil_div(nleaf, TB), TB, 0, st>>>(P->leaf_begin, L, P->d_begin, nullptr, P->d_src);
            HFMM_CUDA_TRY(cudaGetLastError());
        }
    }
    // neighbour pairs (count only, host)
    const int m = 1 << L;
    const std::vector<int32_t>& lb = P->h_leaf_begin;
    int64_t up = 0, pp = 0;
    for (int iy = 0; iy < m; ++iy)
        for (int ix = 0; ix < m; ++ix) {
            uint32_t b = morton(ix, iy);
            if (lb[b + 1] == lb[b]) continue;
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int sx = ix + dx, sy = iy + dy;
                    if (sx < 0 || sy < 0 || sx >= m || sy >= m) continue;
                    uint32_t s = morton(sx, sy);
                    if (lb[s + 1] > lb[s]) {
                        ++up;
                        pp += (int64_t)(lb[b + 1] - lb[b]) * (lb[s + 1] - lb[s]);
                    }
                }
        }
    P->u_pairs = up;
    P->p2p_point_pairs = pp;
    HFMM_CUDA_TRY(cudaStreamSynchronize(st));
    return HFMM_OK;
}

// ---------------------------------------------------------------------------
// Leaf ordering without allocation (hfmm_leaf_order_noalloc).
//
// Same computation as the plan's tree build (bounding square, Morton leaf
// keys at level L, stable radix sort, leaf ranges), but every temporary lives
// in one file-scope device array sized for HFMM_NOALLOC_MAX_POINTS points and
// HFMM_NOALLOC_MAX_LEVELS levels, so the call never allocates.  The array is
// shared by all calls on a device and keeps the previous call's contents.
// ---------------------------------------------------------------------------
#include <mutex>

namespace {

constexpr int64_t NA_MAXP = HFMM_NOALLOC_MAX_POINTS;
constexpr int64_t NA_MAXLEAF = (int64_t)1 << (2 * HFMM_NOALLOC_MAX_LEVELS);
constexpr int64_t NA_MAXCNT = (NA_MAXP > NA_MAXLEAF ? NA_MAXP : NA_MAXLEAF);
constexpr int NA_BBOX_BLOCKS = 256;

// byte offsets inside the scratch array (each a multiple of 256)
constexpr size_t na_round(size_t b) { return (b + 255) / 256 * 256; }
constexpr size_t NA_OFF_PART = 0;                                              // double[4 * 256]
constexpr size_t NA_OFF_PARAM = NA_OFF_PART + na_round(sizeof(double) * 4 * NA_BBOX_BLOCKS);
constexpr size_t NA_OFF_KEY = NA_OFF_PARAM + 256;                              // params: x0, y0, scale, flag
constexpr size_t NA_OFF_KEY2 = NA_OFF_KEY + na_round(sizeof(uint32_t) * NA_MAXP);
constexpr size_t NA_OFF_VAL = NA_OFF_KEY2 + na_round(sizeof(uint32_t) * NA_MAXP);
constexpr size_t NA_OFF_VAL2 = NA_OFF_VAL + na_round(sizeof(int32_t) * NA_MAXP);
constexpr size_t NA_OFF_FLAG = NA_OFF_VAL2 + na_round(sizeof(int32_t) * NA_MAXP);
constexpr size_t NA_OFF_POS = NA_OFF_FLAG + na_round(sizeof(int32_t) * (NA_MAXCNT + 1));
constexpr size_t NA_OFF_TMP = NA_OFF_POS + na_round(sizeof(int32_t) * (NA_MAXCNT + 1));
constexpr size_t NA_BYTES = NA_OFF_TMP + na_round(sizeof(int32_t) * (NA_MAXCNT / SCAN_BLOCK + 2));

__device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

std::mutex g_noalloc_mutex;
void* g_noalloc_addr[64] = {};

// Device address of the scratch array for the current device (looked up once
// per device with that device current).
hfmm_status noalloc_scratch(unsigned char** out) {
    int dev = 0;
    HFMM_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) { hfmm_set_error("device ordinal %d out of range", dev); return HFMM_ERR_UNSUPPORTED; }
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            hfmm_set_error("cudaGetSymbolAddress of the scratch array failed: %s", cudaGetErrorString(e));
            return HFMM_ERR_CUDA;
        }
        g_noalloc_addr[dev] = p;
    }
    *out = (unsigned char*)g_noalloc_addr[dev];
    return HFMM_OK;
}

// reduce the bounding-box partials; param = {x0, y0, scale, flag}
__global__ void na_bbox_finalize(const double* part, int nblk, uint32_t m, double* param) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double mnx = INFINITY, mny = INFINITY, mxx = -INFINITY, mxy = -INFINITY;
    int bad = 0;
    for (int b = 0; b < nblk; ++b) {
        if (isnan(part[4 * b])) bad = 1;
        mnx = fmin(mnx, part[4 * b]); mny = fmin(mny, part[4 * b + 1]);
        mxx = fmax(mxx, part[4 * b + 2]); mxy = fmax(mxy, part[4 * b + 3]);
    }
    if (!bad && !(mny > 0.0)) bad = 2;
    double S = fmax(mxx - mnx, mxy - mny);
    if (!(S > 0.0)) S = 1.0;
    param[0] = mnx;
    param[1] = mny;
    param[2] = (double)m / S;
    param[3] = (double)bad;
}

__global__ void na_leaf_keys(const double* xy, int64_t n, const double* param, uint32_t mmax, uint32_t* key,
                             int32_t* val) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double x0 = param[0], y0 = param[1], scale = param[2];
    double fx = floor((xy[2 * i] - x0) * scale);
    double fy = floor((xy[2 * i + 1] - y0) * scale);
    uint32_t ix = (uint32_t)fmin(fmax(fx, 0.0), (double)mmax);
    uint32_t iy = (uint32_t)fmin(fmax(fy, 0.0), (double)mmax);
    key[i] = morton(ix, iy);
    val[i] = (int32_t)i;
}

__global__ void na_write_perm(const int32_t* val, int64_t n, int64_t* perm) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) perm[i] = val[i];
}

}  // namespace

extern "C" hfmm_status hfmm_leaf_order_noalloc(int64_t n, const double* xy, int32_t levels, int64_t* perm,
                                               int32_t* leaf_begin, void* stream) {
    if (n < 1 || n > NA_MAXP) {
        hfmm_set_error("hfmm_leaf_order_noalloc: n = %lld outside [1, %lld] (the size of its static scratch)",
                       (long long)n, (long long)NA_MAXP);
        return HFMM_ERR_INVALID_ARG;
    }
    if (levels < 2 || levels > HFMM_NOALLOC_MAX_LEVELS) {
        hfmm_set_error("hfmm_leaf_order_noalloc: levels = %d outside [2, %d]", levels, HFMM_NOALLOC_MAX_LEVELS);
        return HFMM_ERR_INVALID_ARG;
    }
    if (!xy || !perm || !leaf_begin) {
        hfmm_set_error("hfmm_leaf_order_noalloc: null pointer");
        return HFMM_ERR_INVALID_ARG;
    }
    unsigned char* base = nullptr;
    HFMM_TRY(noalloc_scratch(&base));
    cudaStream_t st = (cudaStream_t)stream;
    double* part = (double*)(base + NA_OFF_PART);
    double* param = (double*)(base + NA_OFF_PARAM);
    uint32_t* key = (uint32_t*)(base + NA_OFF_KEY);
    uint32_t* key2 = (uint32_t*)(base + NA_OFF_KEY2);
    int32_t* val = (int32_t*)(base + NA_OFF_VAL);
    int32_t* val2 = (int32_t*)(base + NA_OFF_VAL2);
    int32_t* flag = (int32_t*)(base + NA_OFF_FLAG);
    int32_t* pos = (int32_t*)(base + NA_OFF_POS);
    int32_t* tmp = (int32_t*)(base + NA_OFF_TMP);
    const int TB = 256;
    const uint32_t m = 1u << levels;
    const int64_t nleaf = (int64_t)1 << (2 * levels);
    bbox_partial<<<NA_BBOX_BLOCKS, 256, 0, st>>>(xy, n, part);
    na_bbox_finalize<<<1, 32, 0, st>>>(part, NA_BBOX_BLOCKS, m, param);
    HFMM_CUDA_TRY(cudaGetLastError());
    double flag_h = 0.0;
    HFMM_CUDA_TRY(cudaMemcpyAsync(&flag_h, param + 3, sizeof(double), cudaMemcpyDeviceToHost, st));
    HFMM_CUDA_TRY(cudaStreamSynchronize(st));
    if (flag_h != 0.0) {
        hfmm_set_error(flag_h == 1.0 ? "hfmm_leaf_order_noalloc: non-finite point coordinates"
                                     : "hfmm_leaf_order_noalloc: all points must lie in the top layer y > 0");
        return HFMM_ERR_INVALID_ARG;
    }
    na_leaf_keys<<<ceil_div(n, TB), TB, 0, st>>>(xy, n, param, m - 1, key, val);
    HFMM_CUDA_TRY(cudaGetLastError());
    for (int bit = 0; bit < 2 * levels; ++bit) {
        split_flags<<<ceil_div(n, TB), TB, 0, st>>>(key, n, bit, flag);
        HFMM_TRY(exclusive_scan(flag, pos, n, tmp, st));
        split_scatter<<<ceil_div(n, TB), TB, 0, st>>>(key, val, pos, n, bit, key2, val2);
        HFMM_CUDA_TRY(cudaGetLastError());
        std::swap(key, key2);
        std::swap(val, val2);
    }
    // leaf counts start at zero on every call (the array keeps old contents)
    HFMM_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(int32_t) * nleaf, st));
    leaf_histogram<<<ceil_div(n, TB), TB, 0, st>>>(key, n, flag);
    HFMM_TRY(exclusive_scan(flag, leaf_begin, nleaf, tmp, st));
    na_write_perm<<<ceil_div(n, TB), TB, 0, st>>>(val, n, perm);
    HFMM_CUDA_TRY(cudaGetLastError());
    return HFMM_OK;
}
