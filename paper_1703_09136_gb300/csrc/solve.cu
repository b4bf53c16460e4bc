// Krylov solver around the H-FMM apply: restarted GMRES for
//     (sigma I + A) x = b,   A_ij = u_{x_j}(x_i)  (Sec. 2.4),
// the dense system of a second-kind integral equation discretised on the
// plan's points.  Every operator application is one hfmm apply; the Krylov
// vectors stay on the device (dot products and updates are this file's
// kernels, accumulated in FP64); the small Hessenberg least-squares problem
// (Givens rotations) is solved on the host after each Arnoldi step.
#include <cmath>
#include <complex>
#include <vector>

#include "plan.cuh"

namespace {

using zc = std::complex<double>;

constexpr int SV_THREADS = 256;
constexpr int SV_BLOCKS = 4 * 152;

template <class T> struct Cx;
template <> struct Cx<cd> {
    static __device__ __forceinline__ double re(cd v) { return v.x; }
    static __device__ __forceinline__ double im(cd v) { return v.y; }
    static __device__ __forceinline__ cd mk(double r, double i) { return cmk(r, i); }
};
template <> struct Cx<cf> {
    static __device__ __forceinline__ double re(cf v) { return v.x; }
    static __device__ __forceinline__ double im(cf v) { return v.y; }
    static __device__ __forceinline__ cf mk(double r, double i) { return cfmk((float)r, (float)i); }
};

// partial sums of sum_i conj(a_i) b_i, one pair of doubles per block
template <class T>
__global__ void __launch_bounds__(SV_THREADS) dot_kernel(const T* __restrict__ a, const T* __restrict__ b,
                                                         int64_t n, double* __restrict__ part) {
    double sr = 0.0, si = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double ar = Cx<T>::re(a[i]), ai = Cx<T>::im(a[i]), br = Cx<T>::re(b[i]), bi = Cx<T>::im(b[i]);
        sr += ar * br + ai * bi;
        si += ar * bi - ai * br;
    }
    __shared__ double rr[SV_THREADS / 32], ri[SV_THREADS / 32];
    for (int o = 16; o > 0; o >>= 1) {
        sr += __shfl_down_sync(0xffffffffu, sr, o);
        si += __shfl_down_sync(0xffffffffu, si, o);
    }
    if ((threadIdx.x & 31) == 0) { rr[threadIdx.x >> 5] = sr; ri[threadIdx.x >> 5] = si; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tr = 0.0, ti = 0.0;
        for (int w = 0; w < SV_THREADS / 32; ++w) { tr += rr[w]; ti += ri[w]; }
        part[2 * blockIdx.x] = tr;
        part[2 * blockIdx.x + 1] = ti;
    }
}

// y = alpha x + beta y (alpha, beta complex)
template <class T>
__global__ void axpby_kernel(double ar, double ai, const T* __restrict__ x, double br, double bi, T* __restrict__ y,
                             int64_t n) {
    const bool ready = br != 0.0 || bi != 0.0;      // beta = 0: y is only written
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double xr = Cx<T>::re(x[i]), xi = Cx<T>::im(x[i]);
        const double yr = ready ? Cx<T>::re(y[i]) : 0.0, yi = ready ? Cx<T>::im(y[i]) : 0.0;
        y[i] = Cx<T>::mk(ar * xr - ai * xi + br * yr - bi * yi, ar * xi + ai * xr + br * yi + bi * yr);
    }
}

template <class T>
struct Krylov {
    hfmm_plan_s* P;
    cudaStream_t st;
    int64_t n;
    double* part;        // device partial sums
    std::vector<double> hpart;

    hfmm_status dot(const T* a, const T* b, zc* out) {
        dot_kernel<T><<<SV_BLOCKS, SV_THREADS, 0, st>>>(a, b, n, part);
        HFMM_CUDA_TRY(cudaGetLastError());
        HFMM_CUDA_TRY(cudaMemcpyAsync(hpart.data(), part, sizeof(double) * 2 * SV_BLOCKS, cudaMemcpyDeviceToHost, st));
        HFMM_CUDA_TRY(cudaStreamSynchronize(st));
        double r = 0.0, i = 0.0;
        for (int k = 0; k < SV_BLOCKS; ++k) { r += hpart[2 * k]; i += hpart[2 * k + 1]; }
        *out = zc(r, i);
        return HFMM_OK;
    }
    // y = a x + b y
    hfmm_status axpby(zc a, const T* x, zc b, T* y) {
        axpby_kernel<T><<<SV_BLOCKS, SV_THREADS, 0, st>>>(a.real(), a.imag(), x, b.real(), b.imag(), y, n);
        HFMM_CUDA_TRY(cudaGetLastError());
        return HFMM_OK;
    }
    // y = sigma v + A v
    hfmm_status op(zc sigma, const T* v, T* y) {
        if (P->precision == HFMM_MIXED)
            HFMM_TRY(apply_mixed(P, 1, (const cf*)v, (cf*)y, HFMM_PART_ALL, false, st));
        else
            HFMM_TRY(apply_fp64(P, 1, (const cd*)v, (cd*)y, HFMM_PART_ALL, false, st));
        return axpby(sigma, v, zc(1.0, 0.0), y);
    }
};

template <class T>
hfmm_status gmres(hfmm_plan_s* P, zc sigma, const T* b, T* x, double tol, int m, int maxit, int* iters,
                  double* relres, cudaStream_t st) {
    const int64_t n = P->n;
    // workspace: m + 1 Krylov vectors and one more, kept by the plan
    const size_t need = sizeof(T) * (size_t)n * (m + 2);
    if (!P->krylov || P->krylov_bytes < need) {
        HFMM_TRY(plan_alloc(P, (void**)&P->krylov, need));
        P->krylov_bytes = need;
    }
    if (!P->krylov_part) HFMM_TRY(plan_alloc(P, (void**)&P->krylov_part, sizeof(double) * 2 * SV_BLOCKS));
    Krylov<T> K{P, st, n, P->krylov_part, std::vector<double>(2 * SV_BLOCKS)};
    T* V = (T*)P->krylov;
    T* w = V + (size_t)n * (m + 1);
    auto vec = [&](int j) { return V + (size_t)n * j; };
    zc bb;
    HFMM_TRY(K.dot(b, b, &bb));
    const double bnorm = std::sqrt(bb.real());
    *iters = 0;
    *relres = 0.0;
    if (bnorm == 0.0) {
        HFMM_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(T) * n, st));
        HFMM_CUDA_TRY(cudaStreamSynchronize(st));
        return HFMM_OK;
    }
    std::vector<zc> H((size_t)(m + 1) * m), g(m + 1), cs(m), sn(m), y(m);
    while (*iters < maxit) {
        // r = b - (sigma x + A x) into V_0
        HFMM_TRY(K.op(sigma, x, vec(0)));
        HFMM_TRY(K.axpby(zc(1.0, 0.0), b, zc(-1.0, 0.0), vec(0)));
        zc rr;
        HFMM_TRY(K.dot(vec(0), vec(0), &rr));
        const double beta = std::sqrt(rr.real());
        *relres = beta / bnorm;
        if (*relres <= tol) break;
        HFMM_TRY(K.axpby(zc(1.0 / beta, 0.0), vec(0), zc(0.0, 0.0), vec(0)));
        std::fill(g.begin(), g.end(), zc(0.0, 0.0));
        g[0] = beta;
        int j = 0;
        for (; j < m && *iters < maxit; ++j) {
            ++*iters;
            HFMM_TRY(K.op(sigma, vec(j), w));
            for (int i = 0; i <= j; ++i) {          // modified Gram-Schmidt
                zc h;
                HFMM_TRY(K.dot(vec(i), w, &h));
                H[(size_t)i * m + j] = h;
                HFMM_TRY(K.axpby(-h, vec(i), zc(1.0, 0.0), w));
            }
            zc ww;
            HFMM_TRY(K.dot(w, w, &ww));
            const double hn = std::sqrt(ww.real());
            H[(size_t)(j + 1) * m + j] = hn;
            if (hn > 0.0) HFMM_TRY(K.axpby(zc(1.0 / hn, 0.0), w, zc(0.0, 0.0), vec(j + 1)));
            // Givens rotations: apply the previous ones to column j, make a new one
            for (int i = 0; i < j; ++i) {
                const zc a = H[(size_t)i * m + j], c = H[(size_t)(i + 1) * m + j];
                H[(size_t)i * m + j] = std::conj(cs[i]) * a + std::conj(sn[i]) * c;
                H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
            }
            const zc a = H[(size_t)j * m + j];
            const double den = std::sqrt(std::norm(a) + hn * hn);
            cs[j] = den > 0.0 ? a / den : zc(1.0, 0.0);
            sn[j] = den > 0.0 ? zc(hn / den, 0.0) : zc(0.0, 0.0);
            H[(size_t)j * m + j] = den;
            H[(size_t)(j + 1) * m + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = std::conj(cs[j]) * g[j];
            *relres = std::abs(g[j + 1]) / bnorm;
            if (*relres <= tol || hn == 0.0) { ++j; break; }
        }
        // y = H(0:j, 0:j)^-1 g(0:j); x += V y
        for (int i = j - 1; i >= 0; --i) {
            zc s = g[i];
            for (int k = i + 1; k < j; ++k) s -= H[(size_t)i * m + k] * y[k];
            y[i] = s / H[(size_t)i * m + i];
        }
        for (int i = 0; i < j; ++i) HFMM_TRY(K.axpby(y[i], vec(i), zc(1.0, 0.0), x));
        if (*relres <= tol) break;
    }
    // the true residual of the returned x
    HFMM_TRY(K.op(sigma, x, w));
    HFMM_TRY(K.axpby(zc(1.0, 0.0), b, zc(-1.0, 0.0), w));
    zc rr;
    HFMM_TRY(K.dot(w, w, &rr));
    *relres = std::sqrt(rr.real()) / bnorm;
    return HFMM_OK;
}

}  // namespace

extern "C" hfmm_status hfmm_solve(hfmm_plan_t P, const double* sigma, const void* b, void* x, double tol,
                                  int32_t restart, int32_t maxit, int32_t* iters, double* relres, void* stream) {
    if (!P || !sigma || !b || !x || !iters || !relres) {
        hfmm_set_error("hfmm_solve: null argument");
        return HFMM_ERR_INVALID_ARG;
    }
    if (!(tol > 0.0) || restart < 1 || restart > 1000 || maxit < 1) {
        hfmm_set_error("hfmm_solve: need tol > 0, 1 <= restart <= 1000, maxit >= 1");
        return HFMM_ERR_INVALID_ARG;
    }
    for (const void* p : {b, (const void*)x}) {
        cudaPointerAttributes a;
        const bool dev = cudaPointerGetAttributes(&a, p) == cudaSuccess && a.type == cudaMemoryTypeDevice;
        cudaGetLastError();
        if (!dev) {
            hfmm_set_error("hfmm_solve: b and x must be device buffers");
            return HFMM_ERR_INVALID_ARG;
        }
    }
    const zc s(sigma[0], sigma[1]);
    cudaStream_t st = (cudaStream_t)stream;
    int it = 0;
    double rr = 0.0;
    hfmm_status status = P->precision == HFMM_MIXED
                             ? gmres<cf>(P, s, (const cf*)b, (cf*)x, tol, restart, maxit, &it, &rr, st)
                             : gmres<cd>(P, s, (const cd*)b, (cd*)x, tol, restart, maxit, &it, &rr, st);
    *iters = it;
    *relres = rr;
    if (status != HFMM_OK) return status;
    if (rr > tol) {
        hfmm_set_error("hfmm_solve: relative residual %.3g after %d iterations (tol %.3g)", rr, it, tol);
        return HFMM_ERR_NUMERICS;
    }
    return HFMM_OK;
}
