// C ABI of the H-FMM library (include/hfmm.h): plan lifecycle, apply entry
// points, introspection.  No exception crosses this boundary.
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "bessel.cuh"
#include "plan.cuh"
#include "tcgen05.cuh"

static thread_local std::string g_last_error;

void hfmm_set_error(const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
}

hfmm_status plan_alloc(hfmm_plan_s* P, void** ptr, size_t bytes) {
    *ptr = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e != cudaSuccess) {
        *ptr = nullptr;
        hfmm_set_error("cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? HFMM_ERR_OOM : HFMM_ERR_CUDA;
    }
    P->allocations.push_back(*ptr);
    return HFMM_OK;
}

static void plan_free(hfmm_plan_s* P) {
    if (!P) return;
    cudaDeviceSynchronize();
    if (P->events_ready) {
        for (int s = 0; s < HFMM_NUM_STAGES; ++s) { cudaEventDestroy(P->ev[s][0]); cudaEventDestroy(P->ev[s][1]); }
        cudaEventDestroy(P->ev_leaf[0]);
        cudaEventDestroy(P->ev_leaf[1]);
    }
    if (P->far_st) cudaStreamDestroy(P->far_st);
    if (P->near_st) cudaStreamDestroy(P->near_st);
    for (cudaEvent_t e : {P->ev_fork, P->ev_near_done, P->ev_far_done})
        if (e) cudaEventDestroy(e);
    for (void* p : P->allocations) cudaFree(p);
    adaptive_destroy(P->ad);
    delete P;
}

static bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device-accessible address of page-locked (registered) host memory, or
// nullptr for other pointers.  Such buffers are read and written in place by
// the gather / scatter kernels (over NVLink-C2C) instead of being staged.
static void* mapped_host_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

static int choose_levels(int64_t n, int leaf) {
    int L = 2;
    while (n > (int64_t)leaf * ((int64_t)1 << (2 * L)) && L < 15) ++L;
    return L;
}

static int p_low(double tol) {
    double d = std::max(1.0, -std::log10(tol));
    return std::max(4, (int)std::ceil(2.5 * d - 6.5));
}

// Device-pointer apply of one instance, no host synchronisation (batch graphs).
hfmm_status batch_apply_one(hfmm_plan_t P, int nrhs, const void* q, void* y, bool adjoint, cudaStream_t st) {
    if (P->precision == HFMM_MIXED) return apply_mixed(P, nrhs, (const cf*)q, (cf*)y, HFMM_PART_ALL, adjoint, st);
    return apply_fp64(P, nrhs, (const cd*)q, (cd*)y, HFMM_PART_ALL, adjoint, st);
}

extern "C" {

void hfmm_options_default(hfmm_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->tol = 1e-6;
    o->p = 0;
    o->leaf_size = 32;
    o->levels = 0;
    o->precision = HFMM_FP64;
    o->max_rhs = 1;
}

const char* hfmm_status_string(hfmm_status s) {
    switch (s) {
        case HFMM_OK: return "ok";
        case HFMM_ERR_INVALID_ARG: return "invalid argument";
        case HFMM_ERR_UNSUPPORTED: return "unsupported";
        case HFMM_ERR_OOM: return "out of memory";
        case HFMM_ERR_CUDA: return "CUDA error";
        case HFMM_ERR_NUMERICS: return "numerical tolerance not reached";
        case HFMM_ERR_TIMEOUT: return "device wait timed out";
    }
    return "unknown status";
}

const char* hfmm_last_error(void) { return g_last_error.c_str(); }

static hfmm_status validate_medium(const hfmm_medium* m) {
    if (!m) { hfmm_set_error("medium is NULL"); return HFMM_ERR_INVALID_ARG; }
    if (!(m->k[0] > 0.0) || !std::isfinite(m->k[0])) {
        hfmm_set_error("k[0] must be a positive finite wavenumber");
        return HFMM_ERR_UNSUPPORTED;
    }
    switch (m->kind) {
        case HFMM_IMPEDANCE:
            if (!std::isfinite(m->alpha) || m->alpha < 0.0) {
                hfmm_set_error("impedance alpha must be real, finite and >= 0 (got %g)", m->alpha);
                return HFMM_ERR_UNSUPPORTED;
            }
            return HFMM_OK;
        case HFMM_TWO_LAYER:
            if (!(m->k[1] > 0.0) || !std::isfinite(m->k[1])) {
                hfmm_set_error("two layers: k[1] must be positive and finite");
                return HFMM_ERR_UNSUPPORTED;
            }
            return HFMM_OK;
        case HFMM_THREE_LAYER:
            if (!(m->k[1] > 0.0) || !(m->k[2] > 0.0) || !std::isfinite(m->k[1]) || !std::isfinite(m->k[2])) {
                hfmm_set_error("three layers: k[1], k[2] must be positive and finite");
                return HFMM_ERR_UNSUPPORTED;
            }
            if (!(m->d > 0.0) || !std::isfinite(m->d)) {
                hfmm_set_error("three layers: d must be positive and finite");
                return HFMM_ERR_UNSUPPORTED;
            }
            return HFMM_OK;
    }
    hfmm_set_error("unknown medium kind %d", m->kind);
    return HFMM_ERR_INVALID_ARG;
}

static hfmm_status plan_create_one(hfmm_plan_t* out, int64_t n, const double* xy, const hfmm_medium* medium,
                                   const hfmm_options* opts, void* stream);

// Time one apply of nrhs right-hand sides (max_rhs if 0) of a plan (device
// buffers, CUDA events).
static hfmm_status time_apply(hfmm_plan_t P, cudaStream_t st, double* ms, int nrhs = 0) {
    if (nrhs <= 0) nrhs = P->max_rhs;
    const size_t esz = P->precision == HFMM_MIXED ? sizeof(cf) : sizeof(cd);
    const size_t bytes = esz * (size_t)P->n * nrhs;
    if (!P->io_q) HFMM_TRY(plan_alloc(P, (void**)&P->io_q, sizeof(cd) * (size_t)P->n * P->max_rhs));
    if (!P->io_y) HFMM_TRY(plan_alloc(P, (void**)&P->io_y, sizeof(cd) * (size_t)P->n * P->max_rhs));
    HFMM_CUDA_TRY(cudaMemsetAsync(P->io_q, 0, bytes, st));
    cudaEvent_t e0, e1;
    HFMM_CUDA_TRY(cudaEventCreate(&e0));
    HFMM_CUDA_TRY(cudaEventCreate(&e1));
    hfmm_status s = HFMM_OK;
    for (int it = 0; it < 3 && s == HFMM_OK; ++it) {
        if (it == 1) cudaEventRecord(e0, st);
        s = P->precision == HFMM_MIXED
                ? apply_mixed(P, nrhs, (const cf*)P->io_q, (cf*)P->io_y, HFMM_PART_ALL, false, st)
                : apply_fp64(P, nrhs, P->io_q, P->io_y, HFMM_PART_ALL, false, st);
    }
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float t = 0.0f;
    cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms = t / 2.0;
    return s;
}

hfmm_status hfmm_plan_create(hfmm_plan_t* out, int64_t n, const double* xy, const hfmm_medium* medium,
                             const hfmm_options* opts, void* stream) {
    if (opts && (opts->flags & HFMM_FLAG_ADAPTIVE) && (opts->flags & HFMM_FLAG_AUTOTUNE)) {
        if (out) *out = nullptr;
        hfmm_set_error("HFMM_FLAG_AUTOTUNE chooses a uniform leaf level; adaptive trees set their own depths");
        return HFMM_ERR_UNSUPPORTED;
    }
    if (!opts || !(opts->flags & HFMM_FLAG_AUTOTUNE)) return plan_create_one(out, n, xy, medium, opts, stream);
    if (!out) { hfmm_set_error("out is NULL"); return HFMM_ERR_INVALID_ARG; }
    *out = nullptr;
    hfmm_options o = *opts;
    o.flags &= ~HFMM_FLAG_AUTOTUNE;
    const int L0 = o.levels > 0 ? o.levels : choose_levels(n, o.leaf_size > 0 ? o.leaf_size : 32);
    hfmm_plan_t best = nullptr;
    double best_ms = 0.0;
    int tried[3] = {0, 0, 0};
    double times[3] = {0.0, 0.0, 0.0};
    for (int c = 0; c < 3; ++c) {
        const int L = L0 - 1 + c;
        if (L < 2 || L > 15) continue;
        o.levels = L;
        hfmm_plan_t p = nullptr;
        hfmm_status s = plan_create_one(&p, n, xy, medium, &o, stream);
        if (s != HFMM_OK) {
            if (s == HFMM_ERR_OOM) continue;            // a deeper tree may not fit: skip it
            if (best) hfmm_plan_destroy(best);
            return s;
        }
        double ms = 0.0;
        s = time_apply(p, (cudaStream_t)stream, &ms);
        if (s != HFMM_OK) {
            hfmm_plan_destroy(p);
            if (best) hfmm_plan_destroy(best);
            return s;
        }
        tried[c] = L;
        times[c] = ms;
        if (!best || ms < best_ms) {
            if (best) hfmm_plan_destroy(best);
            best = p;
            best_ms = ms;
        } else {
            hfmm_plan_destroy(p);
        }
    }
    if (!best) { hfmm_set_error("autotune: no candidate plan could be built"); return HFMM_ERR_OOM; }
    for (int c = 0; c < 3; ++c) { best->tune_levels[c] = tried[c]; best->tune_ms[c] = times[c]; }
    // mixed plans: the largest power-of-two nrhs up to which the warp-level
    // engine is faster than the tensor-core passes (unless the caller fixed it)
    if (best->precision == HFMM_MIXED && best->tc_on && opts->small_rhs == 0) {
        int cross = 0;
        for (int nr = 1; nr <= std::min(best->max_rhs, 32); nr *= 2) {
            double t_small = 0.0, t_tc = 0.0;
            best->small_rhs = nr;
            hfmm_status s = time_apply(best, (cudaStream_t)stream, &t_small, nr);
            best->small_rhs = 0;
            if (s == HFMM_OK) s = time_apply(best, (cudaStream_t)stream, &t_tc, nr);
            if (s != HFMM_OK) { hfmm_plan_destroy(best); return s; }
            if (t_small >= t_tc) break;
            cross = nr;
        }
        best->small_rhs = cross;
    }
    best->flags |= HFMM_FLAG_AUTOTUNE;
    *out = best;
    return HFMM_OK;
}

static hfmm_status plan_create_one(hfmm_plan_t* out, int64_t n, const double* xy, const hfmm_medium* medium,
                                   const hfmm_options* opts, void* stream) {
    if (!out) { hfmm_set_error("out is NULL"); return HFMM_ERR_INVALID_ARG; }
    *out = nullptr;
    if (n < 1 || n > ((int64_t)1 << 30)) { hfmm_set_error("n must be in [1, 2^30] (got %lld)", (long long)n); return HFMM_ERR_INVALID_ARG; }
    if (!xy) { hfmm_set_error("xy is NULL"); return HFMM_ERR_INVALID_ARG; }
    HFMM_TRY(validate_medium(medium));
    hfmm_options o;
    hfmm_options_default(&o);
    if (opts) o = *opts;
    if (!(o.tol > 0.0) || o.tol >= 1.0) { hfmm_set_error("tol must be in (0, 1)"); return HFMM_ERR_INVALID_ARG; }
    if (o.leaf_size < 1) o.leaf_size = 32;
    if (o.max_rhs < 1) o.max_rhs = 1;
    if (o.precision != HFMM_FP64 && o.precision != HFMM_MIXED) {
        hfmm_set_error("unknown precision %d", o.precision);
        return HFMM_ERR_INVALID_ARG;
    }
    if (o.levels < 0 || o.levels > 15) { hfmm_set_error("levels must be in [0, 15]"); return HFMM_ERR_INVALID_ARG; }
    if (o.spin_limit < 0) { hfmm_set_error("spin_limit must be >= 0"); return HFMM_ERR_INVALID_ARG; }
    if (o.small_rhs < -1) { hfmm_set_error("small_rhs must be >= -1"); return HFMM_ERR_INVALID_ARG; }
    if (!(o.quad_scale >= 0.0) || !std::isfinite(o.quad_scale) || o.quad_scale > 64.0) {
        hfmm_set_error("quad_scale must be in [0, 64] (got %g)", o.quad_scale);
        return HFMM_ERR_INVALID_ARG;
    }
    auto t0 = std::chrono::steady_clock::now();
    cudaStream_t st = (cudaStream_t)stream;
    hfmm_plan_s* P = new (std::nothrow) hfmm_plan_s();
    if (!P) { hfmm_set_error("host allocation failed"); return HFMM_ERR_OOM; }
    P->n = n;
    P->med = *medium;
    P->k = medium->k[0];
    P->tol = o.tol;
    P->precision = o.precision;
    P->max_rhs = o.max_rhs;
    P->flags = o.flags;
    P->tc_spin = o.spin_limit > 0 ? (long)o.spin_limit : tc::TC_SPIN;
    P->quad_scale = o.quad_scale > 0.0 ? o.quad_scale : 1.0;
    P->small_rhs = o.small_rhs == 0 ? HFMM_SMALL_RHS_DEFAULT : std::max(0, (int)o.small_rhs);
    P->L = o.levels > 0 ? o.levels : choose_levels(n, o.leaf_size);
    hfmm_status s = HFMM_OK;
    do {
        const double* d_xy = xy;
        if (!is_device_ptr(xy)) {
            double* tmp = nullptr;
            if ((s = plan_alloc(P, (void**)&tmp, sizeof(double) * 2 * n)) != HFMM_OK) break;
            cudaError_t e = cudaMemcpyAsync(tmp, xy, sizeof(double) * 2 * n, cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) { hfmm_set_error("copy of xy failed: %s", cudaGetErrorString(e)); s = HFMM_ERR_CUDA; break; }
            d_xy = tmp;
        }
        const bool adaptive = (o.flags & HFMM_FLAG_ADAPTIVE) != 0;
        if ((s = adaptive ? build_adaptive_tree(P, d_xy, o.leaf_size, st) : build_tree(P, d_xy, st)) != HFMM_OK) break;
        const int L = P->L;
        P->lev.resize(L + 1);
        const int base = o.p > 0 ? o.p : p_low(o.tol);
        const double dgt = std::max(1.0, -std::log10(o.tol));
        for (int l = 0; l <= L; ++l) {
            LevelInfo& lv = P->lev[l];
            lv.h = P->S / (double)(1 << l);
            lv.nbox = (int64_t)1 << (2 * l);
            const double kR = P->k * lv.h / std::sqrt(2.0);
            lv.p = base + (int)std::ceil(kR + 1.8 * std::pow(dgt, 2.0 / 3.0) *
                                                  std::pow(std::max(kR - 1.0, 0.0), 1.0 / 3.0));
            // range cap: the unscaled translation entries H_n(k r), n <= 2p, of the
            // closest translated pair (r >= min(2 h_l, 2 y0 + h_l)) stay below
            // ~e^680, |H_n(x)| ~ (n-1)! (2/x)^n / pi for x << n
            const double lx = std::log(2.0 / (P->k * std::min(2.0 * lv.h, 2.0 * P->y0 + lv.h)));
            int pcap = lv.p;
            while (pcap > 1 && std::lgamma(2.0 * pcap) + 2.0 * pcap * lx > 680.0) --pcap;
            lv.p = pcap;
            lv.ncoef = 2 * lv.p + 1;
        }
        if ((s = adaptive ? build_adaptive_lists(P, st) : build_lists(P, st)) != HFMM_OK) break;
        // expansion buffers
        const bool mixed = o.precision == HFMM_MIXED;
        const size_t esz = mixed ? sizeof(cf) : sizeof(cd);
        for (int l = P->lmin; l <= L; ++l) {
            LevelInfo& lv = P->lev[l];
            const size_t bytes = esz * (size_t)lv.nbox * o.max_rhs * lv.ncoef;
            if ((s = plan_alloc(P, mixed ? (void**)&lv.mult32 : (void**)&lv.mult, bytes)) != HFMM_OK) break;
            if ((s = plan_alloc(P, mixed ? (void**)&lv.loc32 : (void**)&lv.loc, bytes)) != HFMM_OK) break;
            P->buffer_bytes += 2.0 * bytes;
        }
        if (s != HFMM_OK) break;
        if ((s = plan_alloc(P, mixed ? (void**)&P->q32 : (void**)&P->q_sorted, esz * n * o.max_rhs)) != HFMM_OK) break;
        if ((s = plan_alloc(P, mixed ? (void**)&P->y32 : (void**)&P->y_sorted, esz * n * o.max_rhs)) != HFMM_OK) break;
        P->buffer_bytes += 2.0 * esz * n * o.max_rhs;
        if ((s = build_tables(P, st)) != HFMM_OK) break;
        if (!mixed && !adaptive && (s = build_near64(P, st)) != HFMM_OK) break;
        if (!mixed && (s = build_diag(P, st)) != HFMM_OK) break;
        if (mixed && adaptive) {
            if ((s = build_tables32(P, st)) != HFMM_OK) break;
            if ((s = build_adaptive32(P, st)) != HFMM_OK) break;
        } else if (mixed) {
            if ((s = build_tables32(P, st)) != HFMM_OK) break;
            if ((s = init_h0_table(st)) != HFMM_OK) break;
            if ((s = init_small(P, st)) != HFMM_OK) break;
            if ((s = build_local_coords(P, st)) != HFMM_OK) break;
            if (!(P->flags & HFMM_FLAG_SIMT_M2L) && (s = build_tc(P, st)) != HFMM_OK) break;
            if (P->tc_on && (s = build_p2p_tc(P, st)) != HFMM_OK) break;
        }
        if (P->flags & HFMM_FLAG_PROFILE) {
            for (int sg = 0; sg < HFMM_NUM_STAGES && s == HFMM_OK; ++sg)
                for (int k2 = 0; k2 < 2; ++k2)
                    if (cudaEventCreate(&P->ev[sg][k2]) != cudaSuccess) {
                        hfmm_set_error("cudaEventCreate failed");
                        s = HFMM_ERR_CUDA;
                    }
            for (int k2 = 0; k2 < 2 && s == HFMM_OK; ++k2)
                if (cudaEventCreate(&P->ev_leaf[k2]) != cudaSuccess) {
                    hfmm_set_error("cudaEventCreate failed");
                    s = HFMM_ERR_CUDA;
                }
            if (s != HFMM_OK) break;
            P->events_ready = true;
        }
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { hfmm_set_error("plan build failed: %s", cudaGetErrorString(e)); s = HFMM_ERR_CUDA; break; }
    } while (0);
    if (s != HFMM_OK) {
        plan_free(P);
        return s;
    }
    P->plan_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    *out = P;
    return HFMM_OK;
}

static hfmm_status apply_common(hfmm_plan_t P, int32_t nrhs, const void* q, void* y, int parts,
                                bool adjoint, void* stream) {
    if (!P) { hfmm_set_error("plan is NULL"); return HFMM_ERR_INVALID_ARG; }
    if (nrhs < 1 || nrhs > P->max_rhs) {
        hfmm_set_error("nrhs must be in [1, max_rhs=%d] (got %d)", P->max_rhs, nrhs);
        return HFMM_ERR_INVALID_ARG;
    }
    if (!q || !y) { hfmm_set_error("q or y is NULL"); return HFMM_ERR_INVALID_ARG; }
    if (q == y) { hfmm_set_error("q and y must not overlap"); return HFMM_ERR_INVALID_ARG; }
    cudaStream_t st = (cudaStream_t)stream;
    const bool mixed = P->precision == HFMM_MIXED;
    const size_t bytes = (mixed ? sizeof(cf) : sizeof(cd)) * (size_t)P->n * nrhs;
    const bool qd = is_device_ptr(q), yd = is_device_ptr(y);
    if (P->tc_err) HFMM_CUDA_TRY(cudaMemsetAsync(P->tc_err, 0, sizeof(int), st));   // this apply's flag
    // page-locked host buffers are used in place; other host buffers are staged
    void* qm = qd ? nullptr : mapped_host_ptr(q);
    void* ym = yd ? nullptr : mapped_host_ptr(y);
    const cd* dq = qd ? (const cd*)q : (const cd*)qm;
    cd* dy = yd ? (cd*)y : (cd*)ym;
    if (!dq) {
        if (!P->io_q) HFMM_TRY(plan_alloc(P, (void**)&P->io_q, sizeof(cd) * (size_t)P->n * P->max_rhs));
        HFMM_CUDA_TRY(cudaMemcpyAsync(P->io_q, q, bytes, cudaMemcpyHostToDevice, st));
        dq = P->io_q;
    }
    const bool stage_y = !dy;
    if (stage_y) {
        if (!P->io_y) HFMM_TRY(plan_alloc(P, (void**)&P->io_y, sizeof(cd) * (size_t)P->n * P->max_rhs));
        dy = P->io_y;
    }
    if (mixed) {
        HFMM_TRY(apply_mixed(P, nrhs, (const cf*)dq, (cf*)dy, parts, adjoint, st));
    } else {
        HFMM_TRY(apply_fp64(P, nrhs, dq, dy, parts, adjoint, st));
    }
    if (stage_y) {
        HFMM_CUDA_TRY(cudaMemcpyAsync(y, P->io_y, bytes, cudaMemcpyDeviceToHost, st));
    }
    if (!qd || !yd) {
        HFMM_CUDA_TRY(cudaStreamSynchronize(st));
        if (P->tc_err) {
            int e = 0;
            HFMM_CUDA_TRY(cudaMemcpy(&e, P->tc_err, sizeof(int), cudaMemcpyDeviceToHost));
            if (e) {
                hfmm_set_error("a bounded device wait gave up after %ld polls; the result is invalid", P->tc_spin);
                return HFMM_ERR_TIMEOUT;
            }
        }
    }
    return HFMM_OK;
}

hfmm_status hfmm_apply(hfmm_plan_t plan, int32_t nrhs, const void* q, void* y, void* stream) {
    return apply_common(plan, nrhs, q, y, HFMM_PART_ALL, false, stream);
}

hfmm_status hfmm_apply_parts(hfmm_plan_t plan, int32_t nrhs, const void* q, void* y, int32_t parts,
                             void* stream) {
    if (parts < 0 || parts > HFMM_PART_ALL) { hfmm_set_error("bad parts mask %d", parts); return HFMM_ERR_INVALID_ARG; }
    return apply_common(plan, nrhs, q, y, parts, false, stream);
}

hfmm_status hfmm_apply_adjoint(hfmm_plan_t plan, int32_t nrhs, const void* v, void* w, void* stream) {
    // Transposed pass: with symmetric lists, P2M^T = (4/i) L2P R, M2M^T = R L2L R,
    // M2L(D)^T = R M2L(-D) R (R: alpha_m -> (-1)^m alpha_{-m}), P2P^T = P2P, the
    // transposed tree pass is the forward pass; A^H v = conj(A^T conj v).
    return apply_common(plan, nrhs, v, w, HFMM_PART_ALL, true, stream);
}

// Widen complex64 to complex128 (gradients of mixed-precision plans run on the FP64 path).
__global__ void widen_kernel(const cf* __restrict__ in, cd* __restrict__ out, int64_t count) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = cmk((double)in[i].x, (double)in[i].y);
}

// FP64 expansion and strength buffers of a mixed-precision plan, allocated on
// its first gradient call (the FP64 tables are part of every plan).
static hfmm_status ensure_fp64_buffers(hfmm_plan_s* P) {
    for (int l = P->lmin; l <= P->L; ++l) {
        LevelInfo& lv = P->lev[l];
        const size_t bytes = sizeof(cd) * (size_t)lv.nbox * P->max_rhs * lv.ncoef;
        if (!lv.mult) HFMM_TRY(plan_alloc(P, (void**)&lv.mult, bytes));
        if (!lv.loc) HFMM_TRY(plan_alloc(P, (void**)&lv.loc, bytes));
    }
    if (!P->q_sorted) HFMM_TRY(plan_alloc(P, (void**)&P->q_sorted, sizeof(cd) * (size_t)P->n * P->max_rhs));
    if (!P->grad_q) HFMM_TRY(plan_alloc(P, (void**)&P->grad_q, sizeof(cd) * (size_t)P->n * P->max_rhs));
    if (!P->grad_g) HFMM_TRY(plan_alloc(P, (void**)&P->grad_g, sizeof(cd) * (size_t)P->n * P->max_rhs));
    return HFMM_OK;
}

hfmm_status hfmm_apply_grad(hfmm_plan_t P, int32_t nrhs, const void* q, const void* g, double* gxy,
                            void* stream) {
    if (!P) { hfmm_set_error("plan is NULL"); return HFMM_ERR_INVALID_ARG; }
    if (nrhs < 1 || nrhs > P->max_rhs) {
        hfmm_set_error("nrhs must be in [1, max_rhs=%d] (got %d)", P->max_rhs, nrhs);
        return HFMM_ERR_INVALID_ARG;
    }
    if (!q || !g || !gxy) { hfmm_set_error("q, g or gxy is NULL"); return HFMM_ERR_INVALID_ARG; }
    if (P->ad) { hfmm_set_error("position gradients are not built for adaptive trees"); return HFMM_ERR_UNSUPPORTED; }
    cudaStream_t st = (cudaStream_t)stream;
    const bool mixed = P->precision == HFMM_MIXED;
    const size_t bytes = (mixed ? sizeof(cf) : sizeof(cd)) * (size_t)P->n * nrhs;
    const bool qd = is_device_ptr(q), gd = is_device_ptr(g), od = is_device_ptr(gxy);
    const cd* dq = (const cd*)q;
    const cd* dg = (const cd*)g;
    double* dout = gxy;
    if (!qd) {
        if (!P->io_q) HFMM_TRY(plan_alloc(P, (void**)&P->io_q, sizeof(cd) * (size_t)P->n * P->max_rhs));
        HFMM_CUDA_TRY(cudaMemcpyAsync(P->io_q, q, bytes, cudaMemcpyHostToDevice, st));
        dq = P->io_q;
    }
    if (!gd) {
        if (!P->io_y) HFMM_TRY(plan_alloc(P, (void**)&P->io_y, sizeof(cd) * (size_t)P->n * P->max_rhs));
        HFMM_CUDA_TRY(cudaMemcpyAsync(P->io_y, g, bytes, cudaMemcpyHostToDevice, st));
        dg = P->io_y;
    }
    if (mixed) {
        // complex64 inputs, gradient on the FP64 path
        HFMM_TRY(ensure_fp64_buffers(P));
        const int64_t count = P->n * (int64_t)nrhs;
        const unsigned blocks = (unsigned)std::min<int64_t>((count + 255) / 256, 8 * 152);
        widen_kernel<<<blocks, 256, 0, st>>>((const cf*)dq, P->grad_q, count);
        widen_kernel<<<blocks, 256, 0, st>>>((const cf*)dg, P->grad_g, count);
        HFMM_CUDA_TRY(cudaGetLastError());
        dq = P->grad_q;
        dg = P->grad_g;
    }
    if (!od) {
        if (!P->io_gxy) HFMM_TRY(plan_alloc(P, (void**)&P->io_gxy, sizeof(double) * 2 * (size_t)P->n));
        dout = P->io_gxy;
    }
    HFMM_TRY(apply_grad_fp64(P, nrhs, dq, dg, dout, st));
    if (!od) HFMM_CUDA_TRY(cudaMemcpyAsync(gxy, dout, sizeof(double) * 2 * (size_t)P->n, cudaMemcpyDeviceToHost, st));
    if (!qd || !gd || !od) HFMM_CUDA_TRY(cudaStreamSynchronize(st));
    return HFMM_OK;
}

hfmm_status hfmm_plan_get_info(hfmm_plan_t P, hfmm_plan_info* info) {
    if (!P || !info) { hfmm_set_error("plan or info is NULL"); return HFMM_ERR_INVALID_ARG; }
    std::memset(info, 0, sizeof(*info));
    info->n = P->n;
    info->levels = P->L;
    info->lmin = P->lmin;
    for (int l = 0; l <= P->L && l < HFMM_MAX_LEVELS; ++l) info->p[l] = P->lev[l].p;
    const auto& lb = P->h_leaf_begin;
    int64_t ne = 0;
    for (size_t b = 0; b + 1 < lb.size(); ++b) ne += lb[b + 1] > lb[b];
    info->nonempty_leaves = P->ad ? adaptive_count(P, 0) : ne;
    if (P->ad) {
        info->adaptive = 1;
        info->w_pairs = adaptive_count(P, 2);
        info->x_pairs = adaptive_count(P, 3);
    }
    for (int l = 0; l <= P->L; ++l) { info->v_pairs += P->lev[l].nv; info->r_pairs += P->lev[l].nr; }
    info->direct_leaf_pairs = P->nd;
    info->u_pairs = P->u_pairs;
    info->x0 = P->x0; info->y0 = P->y0; info->size = P->S;
    info->table_bytes = P->table_bytes;
    info->buffer_bytes = P->buffer_bytes;
    info->plan_ms = P->plan_ms;
    info->precision = P->precision;
    info->max_rhs = P->max_rhs;
    info->launches_last_apply = P->launches;
    if (P->tc_err) {
        int e = 0;
        HFMM_CUDA_TRY(cudaMemcpy(&e, P->tc_err, sizeof(int), cudaMemcpyDeviceToHost));
        info->device_error = e;
    }
    for (int l = 0; l <= P->L; ++l) {
        info->tensor_levels += P->lev[l].tc_ntiles > 0 ? 1 : 0;
        info->tc_run_levels += (P->tc_on && P->lev[l].tc_runs) ? 1 : 0;
    }
    for (int s = 0; s < HFMM_NUM_STAGES; ++s) {
        info->flops_last_apply[s] = P->st_flops[s];
        info->bytes_last_apply[s] = P->st_bytes[s];
    }
    for (int c = 0; c < 3; ++c) {
        info->tune_levels[c] = P->tune_levels[c];
        info->tune_ms[c] = P->tune_ms[c];
    }
    info->near_tc_blocks = P->nt_nblocks;
    info->leaf_l2p_fused = P->tc_l2p ? 1 : 0;
    info->leaf_tc_width = P->tc_on ? P->lev[P->L].tc_nbw : 0;
    info->near_simt_leaves = P->nt_nfallback;
    info->table_check = P->table_check;
    info->small_rhs = P->precision == HFMM_MIXED && !(P->flags & HFMM_FLAG_SIMT_M2L) ? P->small_rhs : 0;
    info->diag_levels = P->diag_levels;
    info->diag_check = P->diag_check;
    return HFMM_OK;
}

hfmm_status hfmm_plan_get_stage_times(hfmm_plan_t P, double* ms) {
    if (!P || !ms) { hfmm_set_error("plan or ms is NULL"); return HFMM_ERR_INVALID_ARG; }
    if (!P->events_ready) { hfmm_set_error("plan was created without HFMM_FLAG_PROFILE"); return HFMM_ERR_INVALID_ARG; }
    HFMM_CUDA_TRY(cudaStreamSynchronize(P->last_stream));
    for (int s = 0; s < HFMM_NUM_STAGES; ++s) {
        ms[s] = 0.0;
        if (!P->ev_used[s]) continue;
        float t = 0.0f;
        HFMM_CUDA_TRY(cudaEventElapsedTime(&t, P->ev[s][0], P->ev[s][1]));
        ms[s] = t;
    }
    return HFMM_OK;
}

hfmm_status hfmm_plan_get_leaf_down(hfmm_plan_t P, double* ms, double* flops) {
    if (!P || !ms || !flops) { hfmm_set_error("plan, ms or flops is NULL"); return HFMM_ERR_INVALID_ARG; }
    if (!P->events_ready) { hfmm_set_error("plan was created without HFMM_FLAG_PROFILE"); return HFMM_ERR_INVALID_ARG; }
    *ms = 0.0;
    *flops = 0.0;
    if (!P->ev_leaf_used) return HFMM_OK;
    HFMM_CUDA_TRY(cudaStreamSynchronize(P->last_stream));
    float t = 0.0f;
    HFMM_CUDA_TRY(cudaEventElapsedTime(&t, P->ev_leaf[0], P->ev_leaf[1]));
    *ms = t;
    *flops = P->leaf_flops;
    return HFMM_OK;
}

hfmm_status hfmm_plan_get_tree(hfmm_plan_t P, int64_t* perm, int32_t* leaf_ix, int32_t* leaf_iy) {
    if (!P) { hfmm_set_error("plan is NULL"); return HFMM_ERR_INVALID_ARG; }
    if (P->ad && (leaf_ix || leaf_iy)) {
        hfmm_set_error("adaptive trees: leaves sit on many levels (hfmm_plan_get_boxes)");
        return HFMM_ERR_UNSUPPORTED;
    }
    std::vector<int64_t> hp(P->n);
    HFMM_CUDA_TRY(cudaMemcpy(hp.data(), P->perm, sizeof(int64_t) * P->n, cudaMemcpyDeviceToHost));
    if (perm) std::memcpy(perm, hp.data(), sizeof(int64_t) * P->n);
    if (leaf_ix || leaf_iy) {
        const auto& lb = P->h_leaf_begin;
        for (size_t b = 0; b + 1 < lb.size(); ++b)
            for (int32_t i = lb[b]; i < lb[b + 1]; ++i) {
                if (leaf_ix) leaf_ix[hp[i]] = (int32_t)morton_x((uint32_t)b);
                if (leaf_iy) leaf_iy[hp[i]] = (int32_t)morton_y((uint32_t)b);
            }
    }
    return HFMM_OK;
}

hfmm_status hfmm_plan_get_pairs(hfmm_plan_t P, int32_t kind, int32_t level, int32_t* out, int64_t cap,
                                int64_t* count) {
    if (P && P->ad) { hfmm_set_error("adaptive trees: use hfmm_plan_get_lists"); return HFMM_ERR_UNSUPPORTED; }
    if (!P || !count) { hfmm_set_error("plan or count is NULL"); return HFMM_ERR_INVALID_ARG; }
    if (level < 0 || level > P->L) { hfmm_set_error("level out of range"); return HFMM_ERR_INVALID_ARG; }
    std::vector<int32_t> pairs;
    auto csr = [&](const int32_t* dbeg, const int32_t* dsrc, int64_t nbox, int64_t nnz) -> hfmm_status {
        if (!dbeg || nnz == 0) return HFMM_OK;
        std::vector<int32_t> hb(nbox + 1), hs(nnz);
        HFMM_CUDA_TRY(cudaMemcpy(hb.data(), dbeg, sizeof(int32_t) * (nbox + 1), cudaMemcpyDeviceToHost));
        HFMM_CUDA_TRY(cudaMemcpy(hs.data(), dsrc, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost));
        for (int64_t b = 0; b < nbox; ++b)
            for (int32_t e = hb[b]; e < hb[b + 1]; ++e) {
                pairs.push_back((int32_t)morton_x((uint32_t)b));
                pairs.push_back((int32_t)morton_y((uint32_t)b));
                pairs.push_back((int32_t)morton_x((uint32_t)hs[e]));
                pairs.push_back((int32_t)morton_y((uint32_t)hs[e]));
            }
        return HFMM_OK;
    };
    const LevelInfo& lv = P->lev[level];
    if (kind == 0) {
        HFMM_TRY(csr(lv.v_begin, lv.v_src, lv.nbox, lv.nv));
    } else if (kind == 1) {
        HFMM_TRY(csr(lv.r_begin, lv.r_src, lv.nbox, lv.nr));
    } else if (kind == 2) {
        if (level == P->L) HFMM_TRY(csr(P->d_begin, P->d_src, lv.nbox, P->nd));
    } else if (kind == 3) {
        if (level == P->L) {
            const auto& lb = P->h_leaf_begin;
            const int m = 1 << P->L;
            for (int64_t b = 0; b < lv.nbox; ++b) {
                if (lb[b + 1] == lb[b]) continue;
                int ix = (int)morton_x((uint32_t)b), iy = (int)morton_y((uint32_t)b);
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        int sx = ix + dx, sy = iy + dy;
                        if (sx < 0 || sy < 0 || sx >= m || sy >= m) continue;
                        uint32_t s = morton(sx, sy);
                        if (lb[s + 1] == lb[s]) continue;
                        pairs.insert(pairs.end(), {ix, iy, sx, sy});
                    }
            }
        }
    } else {
        hfmm_set_error("unknown pair kind %d", kind);
        return HFMM_ERR_INVALID_ARG;
    }
    *count = (int64_t)pairs.size() / 4;
    if (*count > cap) { hfmm_set_error("capacity %lld < %lld pairs", (long long)cap, (long long)*count); return HFMM_ERR_INVALID_ARG; }
    if (out && !pairs.empty()) std::memcpy(out, pairs.data(), sizeof(int32_t) * pairs.size());
    return HFMM_OK;
}

hfmm_status hfmm_plan_get_boxes(hfmm_plan_t P, int32_t* out, int64_t cap, int64_t* count) {
    if (!P || !count) { hfmm_set_error("plan or count is NULL"); return HFMM_ERR_INVALID_ARG; }
    if (!P->ad) { hfmm_set_error("the plan has a uniform tree (hfmm_plan_get_tree)"); return HFMM_ERR_UNSUPPORTED; }
    HFMM_TRY(adaptive_boxes(P, count, nullptr));
    if (!out) return HFMM_OK;
    if (cap < *count) { hfmm_set_error("capacity %lld < %lld boxes", (long long)cap, (long long)*count); return HFMM_ERR_INVALID_ARG; }
    return adaptive_boxes(P, count, out);
}

hfmm_status hfmm_plan_get_lists(hfmm_plan_t P, int32_t kind, int32_t* out, int64_t cap, int64_t* count) {
    if (!P || !count) { hfmm_set_error("plan or count is NULL"); return HFMM_ERR_INVALID_ARG; }
    if (!P->ad) { hfmm_set_error("the plan has a uniform tree (hfmm_plan_get_pairs)"); return HFMM_ERR_UNSUPPORTED; }
    HFMM_TRY(adaptive_pairs(P, kind, count, nullptr));
    if (!out) return HFMM_OK;
    if (cap < *count) { hfmm_set_error("capacity %lld < %lld pairs", (long long)cap, (long long)*count); return HFMM_ERR_INVALID_ARG; }
    return adaptive_pairs(P, kind, count, out);
}

hfmm_status hfmm_plan_destroy(hfmm_plan_t plan) {
    plan_free(plan);
    return HFMM_OK;
}

hfmm_status hfmm_debug_wait_timeout(int64_t spin, int32_t arrive) {
    if (spin < 1) { hfmm_set_error("spin must be >= 1"); return HFMM_ERR_INVALID_ARG; }
    int timed_out = 0;
    HFMM_TRY(tc_wait_probe((long)spin, arrive ? 1 : 0, &timed_out));
    if (timed_out) {
        hfmm_set_error("bounded wait gave up after %lld polls", (long long)spin);
        return HFMM_ERR_TIMEOUT;
    }
    return HFMM_OK;
}

hfmm_status hfmm_debug_bessel(double x, int32_t nmax, double* j, double* h) {
    if (!(x > 0.0) || nmax < 0 || nmax > 100000) { hfmm_set_error("need x > 0, 0 <= nmax"); return HFMM_ERR_INVALID_ARG; }
    std::vector<double> J(nmax + 1);
    std::vector<cd> H(nmax + 1);
    bessel_j_seq(x, nmax, J.data());
    hankel_seq(x, nmax, H.data());
    if (j) std::memcpy(j, J.data(), sizeof(double) * (nmax + 1));
    if (h) for (int i = 0; i <= nmax; ++i) { h[2 * i] = H[i].x; h[2 * i + 1] = H[i].y; }
    return HFMM_OK;
}

}  // extern "C"
