// Diagonal form of the FP64 translations at the coarse levels.
//
// Both translation operators of a level depend on the orders only through
// m - p (Sec. 3.3: the free-space C_{m-p}(D) of Graf's theorem, and the
// reaction A_{p,m} of Eq. (eq:m2loperator), which the paper remarks is a
// function of m - p alone), so each (2p+1)^2 matrix is Toeplitz and one
// translation is a correlation of the source coefficients with the 4p + 1
// entries of its table row.  Embedded in a circulant of length Q >= 4p + 1
// (a power of two), a translation becomes a pointwise product of length Q:
//
//   S_s[k]  = sum_m alpha_m e^{+2 pi i k m / Q}           (once per source box)
//   F_o[k]  = sum_n c_n     e^{-2 pi i k n / Q}           (once per table row, plan time)
//   B_t[k]  = sum_V F_o[k] S_s[k]
//           + sum_R A_e[k] S_s[(Q/2 - k) mod Q]           (the image coefficients
//             alpha^im_m = (-1)^m alpha_{-m} are a reversal and a half-length shift)
//   beta_q += (1/Q) sum_k B_t[k] e^{-2 pi i k q / Q},     q = -p .. p  (once per target box)
//
// which is the dense product exactly, up to rounding: O(Q) per pair instead
// of (2p+1)^2, plus two length-Q transforms per box.  The rounding is not the
// dense product's: a transform spreads the largest table entry over every
// output, and |H_n(k r)| grows without bound once n exceeds k r, so the form
// is only as accurate as the dense product on levels whose boxes are large
// against the wavelength.  The plan therefore tries it level by level on
// random expansions with the magnitudes of real ones (|alpha_m| = s(|m|), the
// bound of J_m over the box) and keeps it where the weighted difference to
// the dense product stays below DIAG_RTOL.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "plan.cuh"

namespace {

constexpr int DG_THREADS = 256;
constexpr int DG_MAX_LOGQ = 12;              // Q <= 4096 (64 KB of shared memory)

// In-place radix-2 transform of x[0 .. Q) in shared memory by one CTA:
//   X[k] = sum_j x[j] e^{-2 pi i j k / Q}  (plus = false)  or  e^{+2 pi i j k / Q}  (plus = true),
// with tw[j] = e^{-2 pi i j / Q}, j < Q / 2.
__device__ void cta_dft(cd* x, int logQ, const cd* __restrict__ tw, bool plus) {
    const int Q = 1 << logQ;
    for (int i = threadIdx.x; i < Q; i += blockDim.x) {
        const int j = (int)(__brev((unsigned)i) >> (32 - logQ));
        if (i < j) {
            const cd t = x[i];
            x[i] = x[j];
            x[j] = t;
        }
    }
    __syncthreads();
    for (int s = 1; s <= logQ; ++s) {
        const int half = 1 << (s - 1);
        const int stride = Q >> s;
        for (int t = threadIdx.x; t < Q / 2; t += blockDim.x) {
            const int pos = t & (half - 1);
            const int i = ((t >> (s - 1)) << s) + pos;
            cd w = tw[pos * stride];
            if (plus) w = cconj(w);
            const cd u = x[i], v = cmul(x[i + half], w);
            x[i] = cadd(u, v);
            x[i + half] = csub(u, v);
        }
        __syncthreads();
    }
}

__global__ void dg_twiddle_kernel(int Q, cd* tw) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < Q / 2; j += gridDim.x * blockDim.x) {
        double s, c;
        sincospi(-2.0 * j / Q, &s, &c);
        tw[j] = cmk(c, s);
    }
}

// Spectrum of every non-empty box's coefficients (grid: boxes x right-hand sides).
__global__ void __launch_bounds__(DG_THREADS) dg_src_kernel(const int32_t* __restrict__ lb, int L, int l, int p,
                                                            int nrhs, int logQ, const cd* __restrict__ mult,
                                                            const cd* __restrict__ tw, cd* __restrict__ spec) {
    extern __shared__ cd x[];
    const int64_t b = blockIdx.x;
    const int r = blockIdx.y;
    int32_t lo, hi;
    box_range(lb, L, l, b, &lo, &hi);
    if (hi <= lo) return;
    const int Q = 1 << logQ, nc = 2 * p + 1;
    const cd* a = mult + (b * nrhs + r) * (int64_t)nc;
    for (int j = threadIdx.x; j < Q; j += blockDim.x) x[j] = cmk(0.0, 0.0);
    __syncthreads();
    for (int m = -p + (int)threadIdx.x; m <= p; m += blockDim.x) x[m & (Q - 1)] = a[m + p];
    __syncthreads();
    cta_dft(x, logQ, tw, true);
    cd* o = spec + (b * nrhs + r) * (int64_t)Q;
    for (int j = threadIdx.x; j < Q; j += blockDim.x) o[j] = x[j];
}

// Spectrum of each table row c_n = T[i (4p + 1) + n + 2p], n = -2p .. 2p.
__global__ void __launch_bounds__(DG_THREADS) dg_op_kernel(const cd* __restrict__ T, int p, int logQ,
                                                           const cd* __restrict__ tw, cd* __restrict__ out) {
    extern __shared__ cd x[];
    const int64_t i = blockIdx.x;
    const int Q = 1 << logQ, w = 4 * p + 1;
    for (int j = threadIdx.x; j < Q; j += blockDim.x) x[j] = cmk(0.0, 0.0);
    __syncthreads();
    for (int n = -2 * p + (int)threadIdx.x; n <= 2 * p; n += blockDim.x) x[n & (Q - 1)] = T[i * w + n + 2 * p];
    __syncthreads();
    cta_dft(x, logQ, tw, false);
    for (int j = threadIdx.x; j < Q; j += blockDim.x) out[i * Q + j] = x[j];
}

// Free and reaction translations of level l into every non-empty target box,
// added to loc (grid: boxes x right-hand sides).
__global__ void __launch_bounds__(DG_THREADS) dg_m2l_kernel(
    const int32_t* __restrict__ lb, int L, int l, int p, int nrhs, int logQ, const cd* __restrict__ spec,
    const int32_t* __restrict__ v_begin, const int32_t* __restrict__ v_src, const int32_t* __restrict__ v_off,
    const cd* __restrict__ ofree, const int32_t* __restrict__ r_begin, const int32_t* __restrict__ r_src,
    const int32_t* __restrict__ r_tab, const cd* __restrict__ oreact, const cd* __restrict__ tw, int parts,
    cd* __restrict__ loc) {
    extern __shared__ cd x[];
    const int64_t b = blockIdx.x;
    const int r = blockIdx.y;
    int32_t lo, hi;
    box_range(lb, L, l, b, &lo, &hi);
    if (hi <= lo) return;
    const int Q = 1 << logQ, nc = 2 * p + 1;
    const bool vf = (parts & HFMM_PART_FAR_FREE) && v_begin;
    const bool rf = (parts & HFMM_PART_FAR_REACT) && r_begin;
    for (int k = threadIdx.x; k < Q; k += blockDim.x) {
        cd acc = cmk(0.0, 0.0);
        if (vf)
            for (int32_t e = v_begin[b]; e < v_begin[b + 1]; ++e)
                cfma(acc, ofree[(int64_t)v_off[e] * Q + k], spec[((int64_t)v_src[e] * nrhs + r) * Q + k]);
        if (rf) {
            const int km = (Q / 2 - k) & (Q - 1);
            for (int32_t e = r_begin[b]; e < r_begin[b + 1]; ++e)
                cfma(acc, oreact[(int64_t)r_tab[e] * Q + k], spec[((int64_t)r_src[e] * nrhs + r) * Q + km]);
        }
        x[k] = acc;
    }
    __syncthreads();
    cta_dft(x, logQ, tw, false);
    const double inv = 1.0 / Q;
    cd* o = loc + (b * nrhs + r) * (int64_t)nc;
    for (int q = -p + (int)threadIdx.x; q <= p; q += blockDim.x)
        o[q + p] = cadd(o[q + p], cscale(x[q & (Q - 1)], inv));
}

// Random coefficients with the magnitudes of real multipoles: alpha_m =
// w[|m|] (u + i v), u, v uniform in [-1, 1) from a counter-based hash
// (splitmix64 of the entry index).
__device__ __forceinline__ double dg_unit(uint64_t z) {
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    z ^= z >> 31;
    return (double)(z >> 11) * 0x1.0p-52 - 1.0;
}

__global__ void dg_fill_kernel(int64_t nbox, int p, const double* __restrict__ w, cd* __restrict__ mult) {
    const int nc = 2 * p + 1;
    const int64_t total = nbox * nc;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int m = (int)(i % nc) - p;
        const double a = w[m < 0 ? -m : m];
        mult[i] = cmk(a * dg_unit(2 * (uint64_t)i), a * dg_unit(2 * (uint64_t)i + 1));
    }
}

// Largest over non-empty boxes of |w (d - e)| / |w d| (w[|q|] weights, one right-hand side).
__global__ void dg_check_kernel(const int32_t* __restrict__ lb, int L, int l, int p, const cd* __restrict__ d,
                                const cd* __restrict__ e, const double* __restrict__ w,
                                unsigned long long* __restrict__ out) {
    const int64_t b = blockIdx.x;
    int32_t lo, hi;
    box_range(lb, L, l, b, &lo, &hi);
    if (hi <= lo) return;
    const int nc = 2 * p + 1;
    double num = 0.0, den = 0.0;
    for (int i = threadIdx.x; i < nc; i += blockDim.x) {
        const int q = i - p;
        const double wq = w[q < 0 ? -q : q];
        const cd a = d[b * nc + i], c = e[b * nc + i];
        num += wq * wq * cabs2(csub(a, c));
        den += wq * wq * cabs2(a);
    }
    __shared__ double sn[32], sd[32];
    for (int o = 16; o > 0; o >>= 1) {
        num += __shfl_down_sync(0xffffffffu, num, o);
        den += __shfl_down_sync(0xffffffffu, den, o);
    }
    if ((threadIdx.x & 31) == 0) { sn[threadIdx.x >> 5] = num; sd[threadIdx.x >> 5] = den; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int j = 1; j < (int)(blockDim.x >> 5); ++j) { num += sn[j]; den += sd[j]; }
        const double rel = den > 0.0 ? sqrt(num / den) : (num > 0.0 ? 1.0 : 0.0);
        atomicMax(out, (unsigned long long)__double_as_longlong(rel));
    }
}

int log2_ceil(int v) {
    int e = 0;
    while ((1 << e) < v) ++e;
    return e;
}

size_t dg_smem(int logQ) { return sizeof(cd) << logQ; }

// Shared memory beyond the default 48 KB (Q = 4096) needs the opt-in attribute.
hfmm_status dg_attributes() {
    static bool done = false;
    if (done) return HFMM_OK;
    const int bytes = (int)dg_smem(DG_MAX_LOGQ);
    HFMM_CUDA_TRY(cudaFuncSetAttribute(dg_src_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    HFMM_CUDA_TRY(cudaFuncSetAttribute(dg_op_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    HFMM_CUDA_TRY(cudaFuncSetAttribute(dg_m2l_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    done = true;
    return HFMM_OK;
}

}  // namespace

hfmm_status down64_lists(hfmm_plan_s* P, int l, int nrhs, const cd* mult, cd* loc, cudaStream_t st);

// Spectra of level l's multipoles (after they are complete).
hfmm_status diag_src(hfmm_plan_s* P, int l, int nrhs, cudaStream_t st) {
    LevelInfo& lv = P->lev[l];
    dg_src_kernel<<<dim3((unsigned)lv.nbox, (unsigned)nrhs), DG_THREADS, dg_smem(lv.diag_logq), st>>>(
        P->leaf_begin, P->L, l, lv.p, nrhs, lv.diag_logq, lv.mult, lv.diag_tw, lv.diag_spec);
    ++P->launches;
    HFMM_CUDA_TRY(cudaGetLastError());
    return HFMM_OK;
}

// Translations of level l in diagonal form, added to lv.loc.
hfmm_status diag_m2l(hfmm_plan_s* P, int l, int nrhs, int parts, cudaStream_t st) {
    LevelInfo& lv = P->lev[l];
    dg_m2l_kernel<<<dim3((unsigned)lv.nbox, (unsigned)nrhs), DG_THREADS, dg_smem(lv.diag_logq), st>>>(
        P->leaf_begin, P->L, l, lv.p, nrhs, lv.diag_logq, lv.diag_spec, lv.nv ? lv.v_begin : nullptr, lv.v_src,
        lv.v_off, lv.diag_ofree, lv.nr ? lv.r_begin : nullptr, lv.r_src, lv.r_tab, lv.diag_oreact, lv.diag_tw, parts,
        lv.loc);
    ++P->launches;
    HFMM_CUDA_TRY(cudaGetLastError());
    return HFMM_OK;
}

// Algorithmic real flops of the diagonal form at level l: the pointwise
// products of every pair plus the two transforms of every non-empty box
// (5 Q log2 Q real flops each).
double diag_flops(const hfmm_plan_s* P, int l, int nrhs, int parts) {
    const LevelInfo& lv = P->lev[l];
    const double Q = (double)(1 << lv.diag_logq);
    double pairs = 0.0;
    if (parts & HFMM_PART_FAR_FREE) pairs += (double)lv.nv;
    if (parts & HFMM_PART_FAR_REACT) pairs += (double)lv.nr;
    return 8.0 * nrhs * pairs * Q + 2.0 * 5.0 * Q * lv.diag_logq * (double)lv.nonempty * nrhs;
}

// Plan time (FP64 plans): try the diagonal form on every level with
// translations and keep it where it reproduces the dense product.
hfmm_status build_diag(hfmm_plan_s* P, cudaStream_t st) {
    P->diag_levels = 0;
    P->diag_check = 0.0;
    if (P->precision != HFMM_FP64 || (P->flags & HFMM_FLAG_DENSE_M2L) || P->ad) return HFMM_OK;
    HFMM_TRY(dg_attributes());
    for (int l = P->lmin; l <= P->L; ++l) {
        LevelInfo& lv = P->lev[l];
        lv.diag_logq = 0;
        lv.diag_err = -1.0;
        if (lv.nv + lv.nr == 0) continue;
        const int64_t span = (int64_t)1 << (2 * (P->L - l));
        lv.nonempty = 0;
        for (int64_t b = 0; b < lv.nbox; ++b)
            lv.nonempty += P->h_leaf_begin[(b + 1) * span] > P->h_leaf_begin[b * span];
        const int logQ = std::max(3, log2_ceil(4 * lv.p + 1));
        const int64_t Q = (int64_t)1 << logQ;
        if (logQ > DG_MAX_LOGQ) continue;
        // the form must save work: Q per pair against (2p + 1)^2
        if ((double)Q * 4.0 > (double)lv.ncoef * lv.ncoef) continue;
        const size_t spec_bytes = sizeof(cd) * (size_t)lv.nbox * P->max_rhs * Q;
        if (spec_bytes > DIAG_MAX_BYTES) continue;
        // weights s(n) = min(1, (k R / 2)^n / n!), R = h / sqrt(2)
        std::vector<double> w(lv.p + 1);
        const double half_kr = 0.5 * P->k * lv.h / std::sqrt(2.0);
        for (int n = 0; n <= lv.p; ++n)
            w[n] = std::min(1.0, std::exp(n * std::log(half_kr) - std::lgamma(n + 1.0)));
        cd *tw = nullptr, *ofree = nullptr, *oreact = nullptr, *spec = nullptr, *ldiag = nullptr;
        double* dw = nullptr;
        unsigned long long* derr = nullptr;
        HFMM_CUDA_TRY(cudaMallocAsync((void**)&tw, sizeof(cd) * (Q / 2), st));
        HFMM_CUDA_TRY(cudaMallocAsync((void**)&spec, sizeof(cd) * lv.nbox * Q, st));
        HFMM_CUDA_TRY(cudaMallocAsync((void**)&ldiag, sizeof(cd) * lv.nbox * lv.ncoef, st));
        HFMM_CUDA_TRY(cudaMallocAsync((void**)&dw, sizeof(double) * (lv.p + 1), st));
        HFMM_CUDA_TRY(cudaMallocAsync((void**)&derr, sizeof(unsigned long long), st));
        if (lv.nv) HFMM_CUDA_TRY(cudaMallocAsync((void**)&ofree, sizeof(cd) * 49 * Q, st));
        if (lv.nr) HFMM_CUDA_TRY(cudaMallocAsync((void**)&oreact, sizeof(cd) * lv.n_react_entries * Q, st));
        HFMM_CUDA_TRY(cudaMemcpyAsync(dw, w.data(), sizeof(double) * (lv.p + 1), cudaMemcpyHostToDevice, st));
        HFMM_CUDA_TRY(cudaMemsetAsync(derr, 0, sizeof(unsigned long long), st));
        HFMM_CUDA_TRY(cudaMemsetAsync(ldiag, 0, sizeof(cd) * lv.nbox * lv.ncoef, st));
        dg_twiddle_kernel<<<ceil_div(Q / 2, 256), 256, 0, st>>>((int)Q, tw);
        if (ofree) dg_op_kernel<<<49, DG_THREADS, dg_smem(logQ), st>>>(lv.t_free, lv.p, logQ, tw, ofree);
        if (oreact)
            dg_op_kernel<<<(unsigned)lv.n_react_entries, DG_THREADS, dg_smem(logQ), st>>>(lv.t_react, lv.p, logQ, tw,
                                                                                       oreact);
        HFMM_CUDA_TRY(cudaGetLastError());
        // the check: random multipoles (one right-hand side) through both forms
        dg_fill_kernel<<<std::min<int64_t>(ceil_div(lv.nbox * lv.ncoef, 256), 4096), 256, 0, st>>>(lv.nbox, lv.p, dw,
                                                                                                  lv.mult);
        HFMM_TRY(down64_lists(P, l, 1, lv.mult, lv.loc, st));
        lv.diag_logq = logQ;
        lv.diag_tw = tw;
        lv.diag_ofree = ofree;
        lv.diag_oreact = oreact;
        lv.diag_spec = spec;
        std::swap(lv.loc, ldiag);
        hfmm_status s = diag_src(P, l, 1, st);
        if (s == HFMM_OK) s = diag_m2l(P, l, 1, HFMM_PART_ALL, st);
        std::swap(lv.loc, ldiag);
        if (s != HFMM_OK) return s;
        dg_check_kernel<<<(unsigned)lv.nbox, 128, 0, st>>>(P->leaf_begin, P->L, l, lv.p, lv.loc, ldiag, dw, derr);
        HFMM_CUDA_TRY(cudaGetLastError());
        unsigned long long bits = 0;
        HFMM_CUDA_TRY(cudaMemcpyAsync(&bits, derr, sizeof(bits), cudaMemcpyDeviceToHost, st));
        HFMM_CUDA_TRY(cudaStreamSynchronize(st));
        double err;
        std::memcpy(&err, &bits, sizeof(err));
        lv.diag_err = err;
        HFMM_CUDA_TRY(cudaFreeAsync(spec, st));
        HFMM_CUDA_TRY(cudaFreeAsync(ldiag, st));
        HFMM_CUDA_TRY(cudaFreeAsync(dw, st));
        HFMM_CUDA_TRY(cudaFreeAsync(derr, st));
        lv.diag_spec = nullptr;
        if (!(err <= DIAG_RTOL)) {
            HFMM_CUDA_TRY(cudaFreeAsync(tw, st));
            if (ofree) HFMM_CUDA_TRY(cudaFreeAsync(ofree, st));
            if (oreact) HFMM_CUDA_TRY(cudaFreeAsync(oreact, st));
            lv.diag_logq = 0;
            lv.diag_tw = lv.diag_ofree = lv.diag_oreact = nullptr;
            continue;
        }
        // kept: the tables move into plan-owned memory, with the spectra buffer
        cd *tw2 = nullptr, *of2 = nullptr, *or2 = nullptr;
        HFMM_TRY(plan_alloc(P, (void**)&tw2, sizeof(cd) * (Q / 2)));
        HFMM_CUDA_TRY(cudaMemcpyAsync(tw2, tw, sizeof(cd) * (Q / 2), cudaMemcpyDeviceToDevice, st));
        if (ofree) {
            HFMM_TRY(plan_alloc(P, (void**)&of2, sizeof(cd) * 49 * Q));
            HFMM_CUDA_TRY(cudaMemcpyAsync(of2, ofree, sizeof(cd) * 49 * Q, cudaMemcpyDeviceToDevice, st));
        }
        if (oreact) {
            HFMM_TRY(plan_alloc(P, (void**)&or2, sizeof(cd) * lv.n_react_entries * Q));
            HFMM_CUDA_TRY(cudaMemcpyAsync(or2, oreact, sizeof(cd) * lv.n_react_entries * Q,
                                          cudaMemcpyDeviceToDevice, st));
        }
        HFMM_TRY(plan_alloc(P, (void**)&lv.diag_spec, spec_bytes));
        HFMM_CUDA_TRY(cudaFreeAsync(tw, st));
        if (ofree) HFMM_CUDA_TRY(cudaFreeAsync(ofree, st));
        if (oreact) HFMM_CUDA_TRY(cudaFreeAsync(oreact, st));
        lv.diag_tw = tw2;
        lv.diag_ofree = of2;
        lv.diag_oreact = or2;
        P->table_bytes += sizeof(cd) * (double)(Q / 2 + (ofree ? 49 * Q : 0) + (oreact ? lv.n_react_entries * Q : 0));
        P->buffer_bytes += (double)spec_bytes;
        P->diag_levels |= 1 << l;
        P->diag_check = std::max(P->diag_check, err);
    }
    HFMM_CUDA_TRY(cudaStreamSynchronize(st));
    return HFMM_OK;
}
