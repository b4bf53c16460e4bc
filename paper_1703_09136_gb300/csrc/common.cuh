// Shared helpers of the H-FMM library: complex arithmetic, status handling.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>

#include "../../include/hfmm.h"

#define HD __host__ __device__ __forceinline__

// ---------------------------------------------------------------------------
// complex double as double2 (x = re, y = im)
// ---------------------------------------------------------------------------
typedef double2 cd;

HD cd cmk(double r, double i) { cd z; z.x = r; z.y = i; return z; }
HD cd cadd(cd a, cd b) { return cmk(a.x + b.x, a.y + b.y); }
HD cd csub(cd a, cd b) { return cmk(a.x - b.x, a.y - b.y); }
HD cd cmul(cd a, cd b) { return cmk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
HD cd cscale(cd a, double s) { return cmk(a.x * s, a.y * s); }
HD cd cconj(cd a) { return cmk(a.x, -a.y); }
HD cd cneg(cd a) { return cmk(-a.x, -a.y); }
HD cd cmuli(cd a) { return cmk(-a.y, a.x); }          // i * a
HD double cabs2(cd a) { return a.x * a.x + a.y * a.y; }
HD double cabsd(cd a) { return hypot(a.x, a.y); }
// acc += a * b
HD void cfma(cd& acc, cd a, cd b) {
    acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
    acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
}
HD cd cdiv(cd a, cd b) {
    // Smith's algorithm
    if (fabs(b.x) >= fabs(b.y)) {
        double r = b.y / b.x, den = b.x + b.y * r;
        return cmk((a.x + a.y * r) / den, (a.y - a.x * r) / den);
    } else {
        double r = b.x / b.y, den = b.x * r + b.y;
        return cmk((a.x * r + a.y) / den, (a.y * r - a.x) / den);
    }
}
HD cd cexpz(cd z) {
    double m = exp(z.x);
    double s, c;
    sincos(z.y, &s, &c);
    return cmk(m * c, m * s);
}
HD cd cexpi(double t) {   // e^{i t}
    double s, c;
    sincos(t, &s, &c);
    return cmk(c, s);
}
HD cd clogz(cd z) { return cmk(log(hypot(z.x, z.y)), atan2(z.y, z.x)); }
// principal square root; a purely real negative argument (imaginary part +0
// or -0) maps to +i sqrt(|x|)
HD cd csqrtz(cd z) {
    double r = hypot(z.x, z.y);
    if (r == 0.0) return cmk(0.0, 0.0);
    if (z.x >= 0.0) {
        double t = sqrt(0.5 * (r + z.x));
        return cmk(t, z.y / (2.0 * t));
    } else {
        double t = sqrt(0.5 * (r - z.x));
        double s = (z.y < 0.0) ? -1.0 : 1.0;   // a zero imaginary part counts as +0
        return cmk(fabs(z.y) / (2.0 * t), s * t);
    }
}

// complex float as float2
typedef float2 cf;
HD cf cfmk(float r, float i) { cf z; z.x = r; z.y = i; return z; }

// ---------------------------------------------------------------------------
// status / error reporting
// ---------------------------------------------------------------------------
void hfmm_set_error(const char* fmt, ...);

#define HFMM_CUDA_TRY(call)                                                        \
    do {                                                                           \
        cudaError_t _e = (call);                                                   \
        if (_e != cudaSuccess) {                                                   \
            cudaGetLastError(); /* a non-sticky error must not reach later calls */ \
            hfmm_set_error("%s:%d %s: %s", __FILE__, __LINE__, #call,               \
                           cudaGetErrorString(_e));                                \
            return _e == cudaErrorMemoryAllocation ? HFMM_ERR_OOM : HFMM_ERR_CUDA; \
        }                                                                          \
    } while (0)

#define HFMM_TRY(call)                         \
    do {                                       \
        hfmm_status _s = (call);               \
        if (_s != HFMM_OK) return _s;          \
    } while (0)

static inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }
