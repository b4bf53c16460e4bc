// Tensor-core downward pass (mixed path): L2L + free-space M2L + reaction M2L
// of one level as one accumulation in tensor memory (tcgen05, sm_103a).
//
// For a pair of target boxes T0, T1 with the same child position (Morton
// b and b + 4), every source step s (the parent's local expansion, each
// V-list offset, each reaction-table entry) contributes
//     beta~_T[r][p] += sum_m a~_S[r][m] M_s[m][p]
// to the scaled local coefficients of both targets (right-hand side r).
// In real arithmetic a complex product is one real GEMM,
//     D[row][n] += sum_k A[row][k] B_s[n][k],
// rows = (target, r) (2 x 64 = M 128), k = (Re a_m | Im a_m) (K = 2 nc_in,
// padded to 16), n = (Re b_p | Im b_p) (N = 2 nc, padded to 16), with
// B = [[Re M, -Im M], [Im M, Re M]] blocks.  FP32 accuracy comes from three
// TF32 products per term (hi*hi + hi*lo + lo*hi, x = hi + lo).
//
// Operands are stored MMA-ready (pre-split TF32 hi / lo, core-matrix layout):
// the multipoles of the level and the parent's local expansions are copied
// into that form after they are produced, the operators at plan time.
// Pipeline (one CTA = one target pair x 64 right-hand sides): warp 4 streams
// every K chunk with cp.async.bulk (two 64-row A halves per part plus the
// operator chunk) into a 4-stage shared-memory ring; warp 5 issues
// tcgen05.mma into one of two TMEM buffers per source step; warps 0-3 drain
// each finished step with tcgen05.ld into round-to-nearest FP32 registers
// (tensor-core accumulation truncates, so long chains in TMEM lose accuracy)
// and write the local coefficients.  Every mbarrier wait is bounded; a
// timeout sets an error flag instead of hanging.
#include <algorithm>
#include <map>
#include <vector>

#include "plan.cuh"

namespace {

constexpr int TC_STAGES = 4;
constexpr int TC_MAX_NP = 128;         // N of the real GEMM (one 128-column TMEM buffer)
constexpr long TC_SPIN = 20000000;     // bounded mbarrier polls

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    // no-swizzle K-major canonical layout: core matrices of 8 rows x 16 B;
    // K-direction core stride (LBO) 128 B, M/N-direction core stride (SBO) 512 B
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)(128 >> 4) << 16;
    d |= (uint64_t)(512 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const uint32_t a = su32(bar);
    for (long it = 0; it < TC_SPIN; ++it) {
        uint32_t ok;
        asm volatile("{\n\t.reg .pred P;\n\tmbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, P;\n\t}\n" : "=r"(ok) : "r"(a), "r"(parity) : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(su32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(su32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(su32(dst)), "l"(src), "r"(bytes), "r"(su32(bar)) : "memory");
}

__device__ __forceinline__ uint32_t tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n"
                 :: "r"(dtmem), "l"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(su32(bar)) : "memory");
}

struct TcTile { int32_t b0, b1, s0, s1; };          // boxes (-1: empty), step range
struct TcStep { int32_t kind, idx, src0, src1; };  // kind 0 free, 1 reaction, 2 L2L; src -1: none

// Pre-split B chunks: for matrix index i, chunk c, part (0 hi, 1 lo):
//   float offset ((i * kc + c) * 2 + part) * (Np * 16) + ((n / 8) * 4 + (k % 16) / 4) * 32 + (n % 8) * 4 + k % 4
// M is a column-major complex matrix [m][p] (nin x nout).
__global__ void tc_btable_kernel(const cf* M, int nmat, int nin, int nout, int Np, int kc, float* out) {
    const int64_t per = (int64_t)kc * 16 * Np;   // (n, k) entries per matrix
    const int64_t total = (int64_t)nmat * per;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / per);
        const int r = (int)(e % per);
        const int n = r / (kc * 16), k = r % (kc * 16);
        float v = 0.0f;
        if (n < 2 * nout && k < 2 * nin) {
            const int p = n % nout, m = k % nin;
            const cf z = M[(int64_t)i * nin * nout + (int64_t)m * nout + p];
            const bool re_out = n < nout, re_in = k < nin;
            v = re_out ? (re_in ? z.x : -z.y) : (re_in ? z.y : z.x);
        }
        const float hi = __uint_as_float(tf32_rna(v));
        const float lo = __uint_as_float(tf32_rna(v - hi));
        const int c = k / 16, kk = k % 16;
        const int64_t base = (((int64_t)i * kc + c) * 2) * (Np * 16);
        const int64_t core = ((n / 8) * 4 + kk / 4) * 32 + (n % 8) * 4 + kk % 4;
        out[base + core] = hi;
        out[base + Np * 16 + core] = lo;
    }
}

// MMA-ready copy of expansions: per box, per 64-row right-hand-side chunk rc,
// per K chunk c (16 real values: Re a_0..a_{nin-1} then Im), hi and lo TF32
// parts, each 64 rows x 16 floats in the no-swizzle core-matrix layout:
//   float offset (((box * nrc + rc) * kc + c) * 2 + part) * 1024
//                + ((r / 8) * 4 + kk / 4) * 32 + (r % 8) * 4 + kk % 4.
__global__ void split_rows_kernel(const cf* __restrict__ src, int64_t nbox, int nrhs, int nin, int kc, int nrc,
                                  float* __restrict__ dst) {
    const int64_t total = nbox * nrc * 64;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t box = e / (nrc * 64);
        const int rc = (int)((e / 64) % nrc);
        const int r = (int)(e % 64);
        const int rhs = rc * 64 + r;
        const cf* row = (rhs < nrhs) ? src + ((int64_t)box * nrhs + rhs) * nin : nullptr;
        for (int c = 0; c < kc; ++c) {
            float hv[16], lv[16];
#pragma unroll
            for (int kk = 0; kk < 16; ++kk) {
                const int k = 16 * c + kk;
                float v = 0.0f;
                if (row && k < 2 * nin) v = (k < nin) ? row[k].x : row[k - nin].y;
                const float h = __uint_as_float(tf32_rna(v));
                hv[kk] = h;
                lv[kk] = __uint_as_float(tf32_rna(v - h));
            }
            float* base = dst + (((box * nrc + rc) * kc + c) * 2) * 1024;
#pragma unroll
            for (int kb = 0; kb < 4; ++kb) {
                const int off = ((r >> 3) * 4 + kb) * 32 + (r & 7) * 4;
                *(float4*)(base + off) = make_float4(hv[4 * kb], hv[4 * kb + 1], hv[4 * kb + 2], hv[4 * kb + 3]);
                *(float4*)(base + 1024 + off) = make_float4(lv[4 * kb], lv[4 * kb + 1], lv[4 * kb + 2], lv[4 * kb + 3]);
            }
        }
    }
}

constexpr int TC2_THREADS = 192;   // warps 0-3 drain, warp 4 TMA, warp 5 MMA

template <int NP>
__global__ void __launch_bounds__(TC2_THREADS) m2l_tc_kernel(
    const TcTile* __restrict__ tiles, const TcStep* __restrict__ steps, const float* __restrict__ Bfree,
    const float* __restrict__ Breact, const float* __restrict__ Bl2l, const float* __restrict__ amma,
    const float* __restrict__ pmma, const float* __restrict__ zero4k, cf* __restrict__ loc, int nrhs, int nc,
    int kc, int kc2, int nrc, int* err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ volatile int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr int stage_bytes = 16384 + NP * 128;
    uint64_t* full = (uint64_t*)(smem + TC_STAGES * stage_bytes);
    uint64_t* empty = full + TC_STAGES;
    uint64_t* dfull = empty + TC_STAGES;
    uint64_t* dfree = dfull + 2;
    uint32_t* tslot = (uint32_t*)(dfree + 2);
    const TcTile tile = tiles[blockIdx.x];
    const int rc = blockIdx.y;
    const uint32_t ncols = 256;
    if (tid == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(su32(&full[s])), "r"(1));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(su32(&empty[s])), "r"(1));
        }
        for (int b = 0; b < 2; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(su32(&dfull[b])), "r"(1));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(su32(&dfree[b])), "r"(128));
        }
        asm volatile("fence.mbarrier_init.release.cluster;");
        s_abort = 0;
    }
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(su32(tslot)), "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t taddr = *tslot;
    const int nsteps = tile.s1 - tile.s0;
    if (warp < 4) {
        // ---------------- drain: FP32 round-to-nearest accumulation ----------------
        const int row = tid, tgt = row >> 6, r = rc * 64 + (row & 63);
        float acc[NP];
#pragma unroll
        for (int j = 0; j < NP; ++j) acc[j] = 0.0f;
        bool ok = true;
        for (int s = 0; s < nsteps && ok; ++s) {
            const int b = s & 1;
            bool good = !s_abort && mbar_wait(&dfull[b], (uint32_t)((s >> 1) & 1));
            good = __all_sync(0xffffffffu, good);
            if (!good) { ok = false; s_abort = 1; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t tb = taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)(b * 128);
#pragma unroll
            for (int c0 = 0; c0 < NP; c0 += 16) {
                uint32_t v[16];
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                             : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                               "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                               "=r"(v[14]), "=r"(v[15])
                             : "r"(tb + (uint32_t)c0));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int j = 0; j < 16; ++j) acc[c0 + j] += __uint_as_float(v[j]);
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(&dfree[b]);
        }
        if (!ok || s_abort) {
            if (lane == 0) atomicExch(err, 1);
        } else {
            const int box = tgt ? tile.b1 : tile.b0;
            if (box >= 0 && r < nrhs) {
                float* out = (float*)(loc + ((int64_t)box * nrhs + r) * nc);
#pragma unroll
                for (int j = 0; j < NP; ++j) {
                    if (j < nc) out[2 * j] = acc[j];
                    else if (j < 2 * nc) out[2 * (j - nc) + 1] = acc[j];
                }
            }
        }
    } else if (warp == 4 && lane == 0) {
        // ---------------- TMA: A halves (two source boxes) and the operator chunk ----------------
        int i = 0;
        for (int s = 0; s < nsteps; ++s) {
            const TcStep st = steps[tile.s0 + s];
            const bool l2l = st.kind == 2;
            const int nk = l2l ? kc2 : kc;
            const float* base = l2l ? pmma : amma;
            const float* Bm = st.kind == 0 ? Bfree + (int64_t)st.idx * nk * 32 * NP
                            : st.kind == 1 ? Breact + (int64_t)st.idx * nk * 32 * NP
                                           : Bl2l + (int64_t)st.idx * nk * 32 * NP;
            bool stop = false;
            for (int c = 0; c < nk; ++c, ++i) {
                const int stg = i % TC_STAGES;
                const uint32_t ph = (uint32_t)((i / TC_STAGES) & 1);
                if (s_abort || !mbar_wait(&empty[stg], ph ^ 1u)) { s_abort = 1; stop = true; break; }
                unsigned char* sb = smem + stg * stage_bytes;
                mbar_arrive_tx(&full[stg], (uint32_t)stage_bytes);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int src = h ? st.src1 : st.src0;
#pragma unroll
                    for (int part = 0; part < 2; ++part) {
                        const float* g = (src >= 0) ? base + ((((int64_t)src * nrc + rc) * nk + c) * 2 + part) * 1024
                                                    : zero4k;
                        bulk_g2s(sb + part * 8192 + h * 4096, g, 4096u, &full[stg]);
                    }
                }
                bulk_g2s(sb + 16384, Bm + (int64_t)c * 32 * NP, (uint32_t)(NP * 128), &full[stg]);
            }
            if (stop) break;
        }
    } else if (warp == 5 && lane == 0) {
        // ---------------- MMA issuer: one TMEM buffer per source step ----------------
        const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(NP >> 3) << 17) | ((128u >> 4) << 24);
        int i = 0;
        bool ok = true;
        for (int s = 0; s < nsteps && ok; ++s) {
            const int b = s & 1;
            if (s_abort || !mbar_wait(&dfree[b], (uint32_t)(((s >> 1) & 1) ^ 1))) { s_abort = 1; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t dt = taddr + (uint32_t)(b * 128);
            const int nk = steps[tile.s0 + s].kind == 2 ? kc2 : kc;
            uint32_t accf = 0;
            for (int c = 0; c < nk; ++c, ++i) {
                const int stg = i % TC_STAGES;
                const uint32_t ph = (uint32_t)((i / TC_STAGES) & 1);
                if (s_abort || !mbar_wait(&full[stg], ph)) { ok = false; s_abort = 1; break; }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t sb = su32(smem + stg * stage_bytes);
#pragma unroll
                for (int ks = 0; ks < 2; ++ks) {
                    const uint64_t ah = sdesc(sb + ks * 256), al = sdesc(sb + 8192 + ks * 256);
                    const uint64_t bh = sdesc(sb + 16384 + ks * 256), bl = sdesc(sb + 16384 + NP * 64 + ks * 256);
                    mma_tf32(dt, ah, bh, idesc, accf);
                    accf = 1;
                    mma_tf32(dt, ah, bl, idesc, 1);
                    mma_tf32(dt, al, bh, idesc, 1);
                }
                mma_commit(&empty[stg]);
            }
            if (ok) mma_commit(&dfull[b]);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(taddr), "r"(ncols));
}

inline int round16(int x) { return (x + 15) / 16 * 16; }

}  // namespace

// Plan-time preparation of the tensor-core downward pass for every level
// whose real GEMM width fits one TMEM buffer (2 nc <= 128); K (including the
// parent's width for L2L) is streamed in chunks of 16.
hfmm_status build_tc(hfmm_plan_s* P, cudaStream_t st) {
    const int L = P->L;
    const int grid = 4 * 152, tb = 256;
    const int nrc = (P->max_rhs + 63) / 64;
    for (int l = std::max(2, P->lmin); l <= L; ++l) {
        LevelInfo& lv = P->lev[l];
        const int Np = round16(2 * lv.ncoef);
        const bool has_parent = l > P->lmin;
        const int npp = has_parent ? P->lev[l - 1].ncoef : 0;
        if (Np > TC_MAX_NP) continue;
        if (lv.nbox < 8) continue;
        lv.tc_np = Np;
        lv.tc_kc = Np / 16;
        lv.tc_kc2 = has_parent ? round16(2 * npp) / 16 : 0;
        // MMA-ready copies: this level's multipoles and the parent's locals
        HFMM_TRY(plan_alloc(P, (void**)&lv.tc_amma, sizeof(float) * (size_t)lv.nbox * nrc * lv.tc_kc * 2048));
        P->buffer_bytes += sizeof(float) * (double)lv.nbox * nrc * lv.tc_kc * 2048;
        if (has_parent) {
            const size_t pb = sizeof(float) * (size_t)P->lev[l - 1].nbox * nrc * lv.tc_kc2 * 2048;
            HFMM_TRY(plan_alloc(P, (void**)&lv.tc_pmma, pb));
            P->buffer_bytes += (double)pb;
        }
        const size_t mat_f = (size_t)lv.tc_kc * 32 * Np;      // floats per V / reaction matrix
        HFMM_TRY(plan_alloc(P, (void**)&lv.tc_bfree, sizeof(float) * 49 * mat_f));
        tc_btable_kernel<<<grid, tb, 0, st>>>(lv.t_free32, 49, lv.ncoef, lv.ncoef, Np, lv.tc_kc, lv.tc_bfree);
        HFMM_CUDA_TRY(cudaGetLastError());
        P->table_bytes += sizeof(float) * 49.0 * mat_f;
        if (lv.t_react32 && lv.n_react_entries > 0) {
            HFMM_TRY(plan_alloc(P, (void**)&lv.tc_breact, sizeof(float) * lv.n_react_entries * mat_f));
            tc_btable_kernel<<<grid, tb, 0, st>>>(lv.t_react32, lv.n_react_entries, lv.ncoef, lv.ncoef, Np, lv.tc_kc,
                                                  lv.tc_breact);
            HFMM_CUDA_TRY(cudaGetLastError());
            P->table_bytes += sizeof(float) * (double)lv.n_react_entries * mat_f;
        }
        if (has_parent) {
            const size_t mat_l = (size_t)lv.tc_kc2 * 32 * Np;
            HFMM_TRY(plan_alloc(P, (void**)&lv.tc_bl2l, sizeof(float) * 4 * mat_l));
            tc_btable_kernel<<<grid, tb, 0, st>>>(P->lev[l - 1].t_l2l32, 4, npp, lv.ncoef, Np, lv.tc_kc2, lv.tc_bl2l);
            HFMM_CUDA_TRY(cudaGetLastError());
            P->table_bytes += sizeof(float) * 4.0 * mat_l;
        }
        // tiles (b, b + 4) with b = 8 j + c, and their source steps
        const int64_t nbox = lv.nbox;
        std::vector<int32_t> vb, vs, vo, rb, rs, rt;
        auto fetch = [&](const int32_t* db, const int32_t* ds, const int32_t* dx, int64_t nnz,
                         std::vector<int32_t>& hb, std::vector<int32_t>& hs, std::vector<int32_t>& hx) -> hfmm_status {
            hb.assign(nbox + 1, 0);
            if (!db) return HFMM_OK;
            HFMM_CUDA_TRY(cudaMemcpy(hb.data(), db, sizeof(int32_t) * (nbox + 1), cudaMemcpyDeviceToHost));
            hs.resize(nnz);
            hx.resize(nnz);
            if (nnz) {
                HFMM_CUDA_TRY(cudaMemcpy(hs.data(), ds, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost));
                HFMM_CUDA_TRY(cudaMemcpy(hx.data(), dx, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost));
            }
            return HFMM_OK;
        };
        HFMM_CUDA_TRY(cudaStreamSynchronize(st));
        HFMM_TRY(fetch(lv.nv ? lv.v_begin : nullptr, lv.v_src, lv.v_off, lv.nv, vb, vs, vo));
        HFMM_TRY(fetch(lv.nr ? lv.r_begin : nullptr, lv.r_src, lv.r_tab, lv.nr, rb, rs, rt));
        const auto& lb = P->h_leaf_begin;
        const int64_t span = (int64_t)1 << (2 * (L - l));
        auto nonempty = [&](int64_t b) { return lb[(b + 1) * span] > lb[b * span]; };
        std::vector<TcTile> tiles;
        std::vector<TcStep> steps;
        for (int64_t j = 0; j < nbox / 8; ++j)
            for (int c = 0; c < 4; ++c) {
                const int64_t b0 = 8 * j + c, b1 = 8 * j + 4 + c;
                const bool e0 = nonempty(b0), e1 = nonempty(b1);
                if (!e0 && !e1) continue;
                TcTile t;
                t.b0 = e0 ? (int32_t)b0 : -1;
                t.b1 = e1 ? (int32_t)b1 : -1;
                t.s0 = (int32_t)steps.size();
                if (has_parent) steps.push_back({2, c, e0 ? (int32_t)(b0 >> 2) : -1, e1 ? (int32_t)(b1 >> 2) : -1});
                if (!vb.empty() && lv.nv) {
                    int32_t s0[49], s1[49];
                    for (int o = 0; o < 49; ++o) s0[o] = s1[o] = -1;
                    if (e0) for (int32_t e = vb[b0]; e < vb[b0 + 1]; ++e) s0[vo[e]] = vs[e];
                    if (e1) for (int32_t e = vb[b1]; e < vb[b1 + 1]; ++e) s1[vo[e]] = vs[e];
                    for (int o = 0; o < 49; ++o)
                        if (s0[o] >= 0 || s1[o] >= 0) steps.push_back({0, o, s0[o], s1[o]});
                }
                if (lv.nr) {
                    // merge the two reaction lists by table entry (dx, ysum)
                    std::map<int32_t, std::pair<int32_t, int32_t>> mm;
                    if (e0) for (int32_t e = rb[b0]; e < rb[b0 + 1]; ++e) mm[rt[e]] = {rs[e], -1};
                    if (e1) for (int32_t e = rb[b1]; e < rb[b1 + 1]; ++e) {
                        auto it = mm.find(rt[e]);
                        if (it == mm.end()) mm[rt[e]] = {-1, rs[e]};
                        else it->second.second = rs[e];
                    }
                    for (auto& kv : mm) steps.push_back({1, kv.first, kv.second.first, kv.second.second});
                }
                t.s1 = (int32_t)steps.size();
                tiles.push_back(t);
            }
        lv.tc_ntiles = (int64_t)tiles.size();
        HFMM_TRY(plan_alloc(P, (void**)&lv.tc_tiles, sizeof(TcTile) * std::max<size_t>(tiles.size(), 1)));
        HFMM_TRY(plan_alloc(P, (void**)&lv.tc_steps, sizeof(TcStep) * std::max<size_t>(steps.size(), 1)));
        if (!tiles.empty()) {
            HFMM_CUDA_TRY(cudaMemcpy(lv.tc_tiles, tiles.data(), sizeof(TcTile) * tiles.size(), cudaMemcpyHostToDevice));
            HFMM_CUDA_TRY(cudaMemcpy(lv.tc_steps, steps.data(), sizeof(TcStep) * steps.size(), cudaMemcpyHostToDevice));
        }
    }
    HFMM_TRY(plan_alloc(P, (void**)&P->tc_err, sizeof(int)));
    HFMM_CUDA_TRY(cudaMemsetAsync(P->tc_err, 0, sizeof(int), st));
    HFMM_TRY(plan_alloc(P, (void**)&P->tc_zero, 4096));
    HFMM_CUDA_TRY(cudaMemsetAsync(P->tc_zero, 0, 4096, st));
    HFMM_CUDA_TRY(cudaStreamSynchronize(st));
    return HFMM_OK;
}

// MMA-ready copy of the multipoles of a tensor-core level (after the upward pass).
hfmm_status split_mult_tc(hfmm_plan_s* P, int l, int nrhs, cudaStream_t st) {
    LevelInfo& lv = P->lev[l];
    if (lv.tc_ntiles == 0) return HFMM_OK;
    const int nrc = (P->max_rhs + 63) / 64;
    split_rows_kernel<<<4 * 152, 128, 0, st>>>(lv.mult32, lv.nbox, nrhs, lv.ncoef, lv.tc_kc, nrc, lv.tc_amma);
    HFMM_CUDA_TRY(cudaGetLastError());
    return HFMM_OK;
}

template <int NP>
static hfmm_status launch_np(hfmm_plan_s* P, LevelInfo& lv, const float* pmma, int nrhs, cudaStream_t st) {
    const size_t smem = (size_t)TC_STAGES * (16384 + NP * 128) + 256;
    static bool attr_set = false;
    if (!attr_set) {
        HFMM_CUDA_TRY(cudaFuncSetAttribute(m2l_tc_kernel<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr_set = true;
    }
    const int nrc = (P->max_rhs + 63) / 64;
    dim3 grid((unsigned)lv.tc_ntiles, (unsigned)((nrhs + 63) / 64));
    m2l_tc_kernel<NP><<<grid, TC2_THREADS, smem, st>>>(
        (const TcTile*)lv.tc_tiles, (const TcStep*)lv.tc_steps, lv.tc_bfree, lv.tc_breact, lv.tc_bl2l, lv.tc_amma,
        pmma, P->tc_zero, lv.loc32, nrhs, lv.ncoef, lv.tc_kc, lv.tc_kc2, nrc, P->tc_err);
    HFMM_CUDA_TRY(cudaGetLastError());
    return HFMM_OK;
}

// Launch the tensor-core downward pass of level l (nrhs right-hand sides).
hfmm_status launch_m2l_tc(hfmm_plan_s* P, int l, int nrhs, cudaStream_t st) {
    LevelInfo& lv = P->lev[l];
    if (lv.tc_ntiles == 0) return HFMM_OK;
    const bool has_parent = l > P->lmin;
    const int nrc = (P->max_rhs + 63) / 64;
    if (has_parent) {
        const LevelInfo& pl = P->lev[l - 1];
        split_rows_kernel<<<4 * 152, 128, 0, st>>>(pl.loc32, pl.nbox, nrhs, pl.ncoef, lv.tc_kc2, nrc, lv.tc_pmma);
        HFMM_CUDA_TRY(cudaGetLastError());
    }
    const float* pm = has_parent ? lv.tc_pmma : nullptr;
    switch (lv.tc_np) {
        case 16: return launch_np<16>(P, lv, pm, nrhs, st);
        case 32: return launch_np<32>(P, lv, pm, nrhs, st);
        case 48: return launch_np<48>(P, lv, pm, nrhs, st);
        case 64: return launch_np<64>(P, lv, pm, nrhs, st);
        case 80: return launch_np<80>(P, lv, pm, nrhs, st);
        case 96: return launch_np<96>(P, lv, pm, nrhs, st);
        case 112: return launch_np<112>(P, lv, pm, nrhs, st);
        case 128: return launch_np<128>(P, lv, pm, nrhs, st);
    }
    hfmm_set_error("tensor-core pass: unsupported width %d", lv.tc_np);
    return HFMM_ERR_UNSUPPORTED;
}
