// Batches of independent H-FMM problems of uneven sizes (one plan per
// instance) applied together, recorded once into one CUDA graph (on a private
// stream of the batch, so that any caller stream, the legacy default stream
// included, can launch it) and replayed on the caller's stream on every later
// call with the same buffers.
//
// Each instance's apply is a branch of the graph forked from and joined back
// to the capture stream, so branches of small and large instances run
// concurrently.  With HFMM_FLAG_PERSISTENT, mixed-precision batches with few
// right-hand sides (nrhs <= small_rhs) run instead as ONE persistent kernel
// (small.cu): a device queue of work items over every stage and level of
// every instance with bounded dependency waits; the graph then holds a
// counter reset and that launch.
#include <cstring>
#include <new>
#include <vector>

#include "plan.cuh"

struct hfmm_batch_s {
    int ninst = 0;
    std::vector<hfmm_plan_t> plans;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> joins;
    cudaEvent_t fork = nullptr;
    cudaStream_t cap = nullptr;       // capture stream
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    // what the captured graph was recorded for
    int key_nrhs = 0;
    bool key_adjoint = false;
    std::vector<const void*> key_q;
    std::vector<void*> key_y;
    PersistBatch* persist = nullptr;  // created on the first apply that takes the persistent path
    bool key_persist = false;
};

// The persistent path: asked for, every plan mixed, the warp-level engine chosen for nrhs.
static bool batch_persistent(const hfmm_batch_s* B, int nrhs) {
    for (auto p : B->plans)
        if (!(p->flags & HFMM_FLAG_PERSISTENT) || p->precision != HFMM_MIXED || nrhs > p->small_rhs ||
            (p->flags & HFMM_FLAG_SIMT_M2L) || p->ad)
            return false;
    return true;
}

hfmm_status batch_apply_one(hfmm_plan_t P, int nrhs, const void* q, void* y, bool adjoint, cudaStream_t st);

static void batch_free(hfmm_batch_s* B) {
    if (!B) return;
    cudaDeviceSynchronize();
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->graph) cudaGraphDestroy(B->graph);
    for (auto e : B->joins) cudaEventDestroy(e);
    if (B->fork) cudaEventDestroy(B->fork);
    if (B->cap) cudaStreamDestroy(B->cap);
    for (auto s : B->streams) cudaStreamDestroy(s);
    persist_destroy(B->persist);
    for (auto p : B->plans) hfmm_plan_destroy(p);
    delete B;
}

static hfmm_status batch_capture(hfmm_batch_s* B, int nrhs, const void* const* q, void* const* y, bool adjoint) {
    cudaStream_t st = B->cap;
    if (B->exec) { cudaGraphExecDestroy(B->exec); B->exec = nullptr; }
    if (B->graph) { cudaGraphDestroy(B->graph); B->graph = nullptr; }
    const bool pers = batch_persistent(B, nrhs);
    if (pers) {
        if (!B->persist) HFMM_TRY(persist_create(B->plans, &B->persist));
        HFMM_TRY(persist_set_buffers(B->persist, q, y, st));
    }
    HFMM_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    hfmm_status s = HFMM_OK;
    cudaError_t e = cudaSuccess;
    if (pers) s = persist_launch(B->persist, nrhs, adjoint, st);
    else e = cudaEventRecord(B->fork, st);
    for (int i = 0; !pers && i < B->ninst && e == cudaSuccess && s == HFMM_OK; ++i) {
        e = cudaStreamWaitEvent(B->streams[i], B->fork, 0);
        if (e != cudaSuccess) break;
        s = batch_apply_one(B->plans[i], nrhs, q[i], y[i], adjoint, B->streams[i]);
        if (s != HFMM_OK) break;
        e = cudaEventRecord(B->joins[i], B->streams[i]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, B->joins[i], 0);
    }
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(st, &g);
    if (s != HFMM_OK) { if (g) cudaGraphDestroy(g); return s; }
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        hfmm_set_error("graph capture of the batch failed: %s",
                       cudaGetErrorString(e != cudaSuccess ? e : e2));
        return HFMM_ERR_CUDA;
    }
    B->graph = g;
    HFMM_CUDA_TRY(cudaGraphInstantiate(&B->exec, g, 0));
    B->key_nrhs = nrhs;
    B->key_adjoint = adjoint;
    B->key_persist = pers;
    B->key_q.assign(q, q + B->ninst);
    B->key_y.assign(y, y + B->ninst);
    return HFMM_OK;
}

extern "C" {

hfmm_status hfmm_batch_create(hfmm_batch_t* out, int32_t ninst, const int64_t* n, const double* const* xy,
                              const hfmm_medium* medium, const hfmm_options* opts, void* stream) {
    if (!out) { hfmm_set_error("out is NULL"); return HFMM_ERR_INVALID_ARG; }
    *out = nullptr;
    if (ninst < 1 || !n || !xy) { hfmm_set_error("need ninst >= 1, n and xy"); return HFMM_ERR_INVALID_ARG; }
    hfmm_batch_s* B = new (std::nothrow) hfmm_batch_s();
    if (!B) { hfmm_set_error("host allocation failed"); return HFMM_ERR_OOM; }
    B->ninst = ninst;
    hfmm_status s = HFMM_OK;
    for (int i = 0; i < ninst && s == HFMM_OK; ++i) {
        hfmm_plan_t p = nullptr;
        s = hfmm_plan_create(&p, n[i], xy[i], medium, opts, stream);
        if (s == HFMM_OK) B->plans.push_back(p);
    }
    if (s == HFMM_OK) {
        for (int i = 0; i < ninst; ++i) {
            cudaStream_t st = nullptr;
            cudaEvent_t ev = nullptr;
            if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
                hfmm_set_error("stream / event creation failed");
                s = HFMM_ERR_CUDA;
                if (st) cudaStreamDestroy(st);
                break;
            }
            B->streams.push_back(st);
            B->joins.push_back(ev);
        }
        if (s == HFMM_OK && (cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming) != cudaSuccess ||
                             cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking) != cudaSuccess)) {
            hfmm_set_error("event / stream creation failed");
            s = HFMM_ERR_CUDA;
        }
    }
    if (s != HFMM_OK) {
        batch_free(B);
        return s;
    }
    *out = B;
    return HFMM_OK;
}

hfmm_status hfmm_batch_apply(hfmm_batch_t B, int32_t nrhs, const void* const* q, void* const* y, int32_t adjoint,
                             void* stream) {
    if (!B || !q || !y) { hfmm_set_error("batch, q or y is NULL"); return HFMM_ERR_INVALID_ARG; }
    cudaStream_t st = (cudaStream_t)stream;
    for (int i = 0; i < B->ninst; ++i) {
        cudaPointerAttributes a;
        const bool qd = cudaPointerGetAttributes(&a, q[i]) == cudaSuccess && a.type == cudaMemoryTypeDevice;
        cudaGetLastError();
        const bool yd = cudaPointerGetAttributes(&a, y[i]) == cudaSuccess && a.type == cudaMemoryTypeDevice;
        cudaGetLastError();
        if (!qd || !yd) { hfmm_set_error("hfmm_batch_apply needs device buffers (instance %d)", i); return HFMM_ERR_INVALID_ARG; }
        if (nrhs < 1 || nrhs > B->plans[i]->max_rhs) { hfmm_set_error("nrhs out of range for instance %d", i); return HFMM_ERR_INVALID_ARG; }
    }
    bool same = B->exec && B->key_nrhs == nrhs && B->key_adjoint == (adjoint != 0);
    for (int i = 0; same && i < B->ninst; ++i) same = B->key_q[i] == q[i] && B->key_y[i] == y[i];
    if (!same) {
        // one eager pass first: lazily created state (kernel attributes) is set up outside capture
        if (!B->exec) {
            for (int i = 0; i < B->ninst; ++i)
                HFMM_TRY(batch_apply_one(B->plans[i], nrhs, q[i], y[i], adjoint != 0, st));
            HFMM_CUDA_TRY(cudaStreamSynchronize(st));
        }
        HFMM_TRY(batch_capture(B, nrhs, q, y, adjoint != 0));
    }
    HFMM_CUDA_TRY(cudaGraphLaunch(B->exec, st));
    return HFMM_OK;
}

hfmm_status hfmm_apply_grad(hfmm_plan_t P, int32_t nrhs, const void* q, const void* g, double* gxy, void* stream);

hfmm_status hfmm_batch_apply_grad(hfmm_batch_t B, int32_t nrhs, const void* const* q, const void* const* g,
                                  double* const* gxy, void* stream) {
    if (!B || !q || !g || !gxy) { hfmm_set_error("batch, q, g or gxy is NULL"); return HFMM_ERR_INVALID_ARG; }
    for (int i = 0; i < B->ninst; ++i) {
        hfmm_status s = hfmm_apply_grad(B->plans[i], nrhs, q[i], g[i], gxy[i], stream);
        if (s != HFMM_OK) return s;
    }
    return HFMM_OK;
}

hfmm_status hfmm_batch_device_error(hfmm_batch_t B, int32_t* device_error) {
    if (!B || !device_error) { hfmm_set_error("batch or device_error is NULL"); return HFMM_ERR_INVALID_ARG; }
    *device_error = 0;
    if (!B->persist) return HFMM_OK;
    int e = 0;
    HFMM_TRY(persist_device_error(B->persist, &e));
    *device_error = e;
    return HFMM_OK;
}

hfmm_status hfmm_batch_get_plan(hfmm_batch_t B, int32_t i, hfmm_plan_t* plan) {
    if (!B || !plan || i < 0 || i >= B->ninst) { hfmm_set_error("bad batch index"); return HFMM_ERR_INVALID_ARG; }
    *plan = B->plans[i];
    return HFMM_OK;
}

hfmm_status hfmm_batch_destroy(hfmm_batch_t B) {
    batch_free(B);
    return HFMM_OK;
}

}  // extern "C"
