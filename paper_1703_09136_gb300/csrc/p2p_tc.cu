// Near field of the mixed path on tensor cores (tcgen05, sm_103a): the
// free-space P2P sum (Algorithm 1, step 5) of the four leaves of one parent
// box (a block), as one real GEMM per CTA.
//
// With rows = (right-hand side r, part) (part 0: real, 1: imaginary; M = 128
// for 64 right-hand sides), columns = the block's targets (each leaf padded to
// a multiple of 16, N <= 128) and K = (source j, re / im), the complex sum
// y_t = sum_j G_tj q_j is
//     D[(r, 0)][t] = sum_j  Re q_j Re G_tj + Im q_j (-Im G_tj)
//     D[(r, 1)][t] = sum_j  Im q_j Re G_tj + (-Re q_j)(-Im G_tj),
// so the A rows are (Re q, Im q) and (Im q, -Re q) and the B rows
// (Re G, -Im G).  The points are fixed, so the B tiles (G = (i/4) H0(k r) of
// each 8-source chunk of each source leaf of the 4 x 4 neighbourhood against
// the adjacent target leaves only) are computed once per plan, scaled by
// 2^NT_GSCALE_EXP and pre-split into f16 hi / lo in the core-matrix layout
// (fmm32.cu, near_tiles_kernel).  Per apply, warp 4 streams the tiles with
// cp.async.bulk (prefetched into L2 a few chunks ahead); warps 0-3 build the
// A rows of each chunk from the strengths, each right-hand side scaled by the
// power of two that puts its largest |Re q|, |Im q| (reduced by the gather
// kernel) in [2^14, 2^15), and split into f16 hi / lo, each thread writing
// one 16-byte core-matrix row per part (4-byte stores in this layout conflict
// on the shared-memory banks, and the build, not the tile stream or the MMAs,
// paces the pass); warp 5 issues three
// kind::f16 MMAs (hi*hi + hi*lo + lo*hi: 22 significant bits, like a TF32
// pair) per run of adjacent target leaves into one 128-column TMEM
// accumulator; warps 0-3 finally undo both scales and store y (point-major,
// [n][nrhs]; the kernel is the first writer of its targets).  The pass is
// paced by each CTA's chain of tile copy, operand build and MMA: one
// accumulator, 16 KB stages and at most 128 chunk records fit four CTAs per
// SM.  Every mbarrier wait is bounded.
#include <algorithm>
#include <vector>

#include "plan.cuh"
#include "tcgen05.cuh"

namespace {

using namespace tc;

constexpr int NT_THREADS = 192;    // warps 0-3 build A and drain, warp 4 TMA, warp 5 MMA
constexpr int NT_STAGES = 2;
constexpr int NT_MAXN = 128;       // padded targets of a block
constexpr int NT_A = 8192;         // A: 128 rows x 16 K halves, hi then lo
constexpr int NT_B = NT_MAXN * 64;  // B: up to 128 rows x 16 K halves, hi then lo
constexpr int NT_STAGE = NT_A + NT_B;
constexpr int NT_MAXCH = 128;     // chunks of a block (kept in shared memory; more: SIMT kernel)
constexpr int NT_PREF = 6;         // tiles brought into L2 ahead of their copy
constexpr size_t NT_SMEM = (size_t)NT_STAGES * NT_STAGE + 1024;

// half offset of (row, k) in a core-matrix tile (K = 16)
__device__ __forceinline__ int core_off(int row, int k) {
    return ((row >> 3) * 2 + (k >> 3)) * 64 + (row & 7) * 8 + (k & 7);
}

struct NtSmall {
    NtChunk ch[NT_MAXCH];      // the block's chunk records
    int32_t tidx[NT_MAXN];     // target of each column, -1: padding
    int32_t off[5], wid[4];
};

__global__ void __launch_bounds__(NT_THREADS, 4) p2p_tc_kernel(
    const int32_t* __restrict__ blocks, const NtChunk* __restrict__ chunks, const __half* __restrict__ tiles,
    const int32_t* __restrict__ lb, const cf* __restrict__ qs, int nrhs, const unsigned* __restrict__ qmax,
    cf* __restrict__ ys, long spin, int* err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ NtSmall S;
    __shared__ uint64_t afull[NT_STAGES], bfull[NT_STAGES], empty[NT_STAGES], done;
    __shared__ uint32_t tslot;
    __shared__ volatile int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t P = blocks[4 * blockIdx.x];
    const int cb = blocks[4 * blockIdx.x + 1];
    const int ce = blocks[4 * blockIdx.x + 2];
    const int nch = ce - cb;
    const int rc = blockIdx.y, r0 = rc * 64;
    if (tid == 0) {
        int o = 0;
        for (int c = 0; c < 4; ++c) {
            const int64_t lf = 4 * P + c;
            S.off[c] = o;
            S.wid[c] = (lb[lf + 1] - lb[lf] + 15) / 16 * 16;
            o += S.wid[c];
        }
        S.off[4] = o;
        for (int s = 0; s < NT_STAGES; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(su32(&afull[s])), "r"(4));   // a warp each
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(su32(&bfull[s])), "r"(1));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(su32(&empty[s])), "r"(1));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(su32(&done)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
        s_abort = 0;
    }
    __syncthreads();
    const int N = S.off[4];
    for (int i = tid; i < nch; i += NT_THREADS) S.ch[i] = chunks[cb + i];
    for (int n = tid; n < NT_MAXN; n += NT_THREADS) {
        int32_t ti = -1;
        if (n < N) {
            int c = 0;
            while (n >= S.off[c + 1]) ++c;
            const int64_t lf = 4 * P + c;
            const int t = n - S.off[c];
            if (t < lb[lf + 1] - lb[lf]) ti = lb[lf] + t;
        }
        S.tidx[n] = ti;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(su32(&tslot)), "r"(128));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t taddr = tslot;
    if (warp < 4) {
        // zero the accumulator (every MMA accumulates)
        const uint32_t tl = taddr + ((uint32_t)(warp * 32) << 16);
        for (int c0 = 0; c0 < 128; c0 += 16)
            asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};"
                         :: "r"(tl + (uint32_t)c0), "r"(0u) : "memory");
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp < 4) {
        // ---------------- A rows: scaled strengths of the chunk's sources ----------------
        // the power of two of each right-hand side (rows r and 64 + r share it)
        const int rr_own = tid & 63;
        const int e_own = (r0 + rr_own < nrhs) ? f16_exp(__uint_as_float(qmax[r0 + rr_own])) : 0;
        // thread tid builds row r = tid & 63 (and row 64 + r) for the chunk's
        // sources 4 g .. 4 g + 3, g = tid >> 6: one 16-byte core-matrix row per part
        const int g4 = 4 * (tid >> 6);
        auto fetch = [&](int i, cf* out) {
            const NtChunk& ch = S.ch[i];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int j = g4 + u;
                cf v = cfmk(0.f, 0.f);
                if (r0 + rr_own < nrhs && j < ch.cnt) v = qs[(int64_t)(ch.src + j) * nrhs + r0 + rr_own];
                out[u] = v;
            }
        };
        // thread (u, tid) always handles right-hand side tid & 63: one scale per thread
        const float qs_scale = pow2f(e_own);
        // strengths two chunks ahead: pa = chunk i, pb = chunk i + 1
        cf pa[4], pb[4], pn[4];
        if (nch > 0) fetch(0, pa);
        if (nch > 1) fetch(1, pb);
        for (int i = 0; i < nch; ++i) {
            const int stg = i % NT_STAGES;
            bool good = !s_abort && mbar_wait(&empty[stg], (uint32_t)(((i / NT_STAGES) & 1) ^ 1), spin);
            good = __all_sync(0xffffffffu, good);
            if (!good) { s_abort = 1; break; }
            if (i + 2 < nch) fetch(i + 2, pn);
            uint16_t* A = (uint16_t*)(smem + stg * NT_STAGE);
            {
                // rows r: (Re q, Im q); rows 64 + r: (Im q, -Re q) (the split of -x is
                // the negated split of x); K columns 2j, 2j + 1 of source j
                uint16_t h0[8], l0[8], h1[8], l1[8];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    uint16_t rh, rl, ih, il;
                    split_f16(pa[u].x * qs_scale, rh, rl);
                    split_f16(pa[u].y * qs_scale, ih, il);
                    h0[2 * u] = rh; h0[2 * u + 1] = ih;
                    l0[2 * u] = rl; l0[2 * u + 1] = il;
                    h1[2 * u] = ih; h1[2 * u + 1] = (uint16_t)(rh ^ 0x8000u);
                    l1[2 * u] = il; l1[2 * u + 1] = (uint16_t)(rl ^ 0x8000u);
                }
                const int o0 = core_off(rr_own, g4 * 2), o1 = core_off(64 + rr_own, g4 * 2);
                *(uint4*)(A + o0) = pack8(h0);
                *(uint4*)(A + 2048 + o0) = pack8(l0);
                *(uint4*)(A + o1) = pack8(h1);
                *(uint4*)(A + 2048 + o1) = pack8(l1);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&afull[stg]);
#pragma unroll
            for (int u = 0; u < 4; ++u) { pa[u] = pb[u]; pb[u] = pn[u]; }
        }
        // ---------------- drain: store y ----------------
        // always wait (bounded) for the MMA thread's final commit: no MMA may
        // still write the accumulator when TMEM is released
        bool good = mbar_wait(&done, 0u) && !s_abort;   // default bound, whatever the plan's limit
        good = __all_sync(0xffffffffu, good);
        if (!good) {
            s_abort = 1;
            if (lane == 0) atomicExch(err, 1);
        } else if (nch > 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int row = tid;
            const uint32_t tl = taddr + ((uint32_t)(warp * 32) << 16);
            const float unscale = pow2f(-(e_own + NT_GSCALE_EXP));   // row r or 64 + r: right-hand side tid & 63
            float* stg0 = (float*)smem;   // stage 0 is free now
            for (int g0 = 0; g0 < N; g0 += 16) {
                uint32_t w0[16];
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                             : "=r"(w0[0]), "=r"(w0[1]), "=r"(w0[2]), "=r"(w0[3]), "=r"(w0[4]), "=r"(w0[5]), "=r"(w0[6]),
                               "=r"(w0[7]), "=r"(w0[8]), "=r"(w0[9]), "=r"(w0[10]), "=r"(w0[11]), "=r"(w0[12]),
                               "=r"(w0[13]), "=r"(w0[14]), "=r"(w0[15])
                             : "r"(tl + (uint32_t)g0));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int u = 0; u < 16; ++u) stg0[u * 128 + row] = __uint_as_float(w0[u]) * unscale;
                asm volatile("bar.sync 1, 128;" ::: "memory");
#pragma unroll
                for (int qq = 0; qq < 8; ++qq) {
                    const int e = tid + 128 * qq, u = e >> 6, rr = e & 63;
                    const int32_t t = S.tidx[g0 + u];
                    if (t >= 0 && r0 + rr < nrhs)
                        ys[(int64_t)t * nrhs + r0 + rr] = cfmk(stg0[u * 128 + rr], stg0[u * 128 + 64 + rr]);
                }
                asm volatile("bar.sync 1, 128;" ::: "memory");
            }
        }
    } else if (warp == 4 && lane == 0) {
        // ---------------- TMA: the chunk's pre-split B tile (L2 prefetch NT_PREF chunks ahead) ----------------
        for (int i = 0; i < min(nch, NT_PREF); ++i)
            bulk_prefetch_l2(tiles + S.ch[i].boff, (uint32_t)S.ch[i].rows * 64u);
        int issued = 0;
        for (int i = 0; i < nch; ++i) {
            if (i + NT_PREF < nch)
                bulk_prefetch_l2(tiles + S.ch[i + NT_PREF].boff, (uint32_t)S.ch[i + NT_PREF].rows * 64u);
            const int stg = i % NT_STAGES;
            if (s_abort || !mbar_wait(&empty[stg], (uint32_t)(((i / NT_STAGES) & 1) ^ 1), spin)) { s_abort = 1; break; }
            const NtChunk& ch = S.ch[i];
            const uint32_t bytes = (uint32_t)ch.rows * 64u;
            mbar_arrive_tx(&bfull[stg], bytes);
            bulk_g2s(smem + stg * NT_STAGE + NT_A, tiles + ch.boff, bytes, &bfull[stg]);
            issued = i + 1;
        }
        if (s_abort) {
            // tiles still in flight land in the ring: wait for them (default bound) before the exit
            for (int k = max(0, issued - NT_STAGES); k < issued; ++k)
                mbar_wait(&bfull[k % NT_STAGES], (uint32_t)((k / NT_STAGES) & 1));
        }
    } else if (warp == 5 && lane == 0) {
        // ---------------- MMA issuer: one MMA set per run of adjacent target leaves ----------------
        for (int i = 0; i < nch; ++i) {
            const int stg = i % NT_STAGES;
            const uint32_t ph = (uint32_t)((i / NT_STAGES) & 1);
            if (s_abort || !mbar_wait(&afull[stg], ph, spin) || !mbar_wait(&bfull[stg], ph, spin)) { s_abort = 1; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const NtChunk& ch = S.ch[i];
            const uint32_t sa = su32(smem + stg * NT_STAGE), sb = sa + NT_A;
            const uint32_t lo_b = (uint32_t)ch.rows * 32u;
            for (int q = 0; q < ch.nrun; ++q) {
                const int rw = ch.run[q];
                const int nn = rw & 0xff, col = (rw >> 8) & 0xff, rowoff = rw >> 16;
                const uint32_t idesc = idesc_f16(nn);
                const uint32_t bro = (uint32_t)rowoff * 32u;
                const uint64_t ah = sdesc(sa, 256), al = sdesc(sa + 4096, 256);
                const uint64_t bh = sdesc(sb + bro, 256), bl = sdesc(sb + lo_b + bro, 256);
                const uint32_t d = taddr + (uint32_t)col;
                mma_f16(d, ah, bh, idesc, 1u);
                mma_f16(d, ah, bl, idesc, 1u);
                mma_f16(d, al, bh, idesc, 1u);
            }
            mma_commit(&empty[stg]);
        }
        mma_commit(&done);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(taddr), "r"(128));
}

}  // namespace

// Plan time: blocks (parent boxes of level L - 1) whose padded targets fit
// NT_MAXN, their source chunks and tile store ([parent, first chunk, end, 0]
// per block); the leaves of the other blocks are left to the SIMT kernel.
hfmm_status build_p2p_tc(hfmm_plan_s* P, cudaStream_t st) {
    const int L = P->L;
    if (L < 1) return HFMM_OK;
    const auto& lb = P->h_leaf_begin;
    const int m = 1 << L;
    const int64_t npar = (int64_t)1 << (2 * (L - 1));
    std::vector<int32_t> blocks, fallback, leaves;
    std::vector<NtChunk> chunks;
    int64_t boff = 0, rows = 0;
    for (int64_t par = 0; par < npar; ++par) {
        int cnt[4], wid[4], ncol = 0, ntgt = 0;
        for (int c = 0; c < 4; ++c) {
            cnt[c] = lb[4 * par + c + 1] - lb[4 * par + c];
            wid[c] = (cnt[c] + 15) / 16 * 16;
            ncol += wid[c];
            ntgt += cnt[c];
        }
        if (ntgt == 0) continue;
        if (ncol > NT_MAXN) {
            for (int c = 0; c < 4; ++c)
                if (cnt[c] > 0) fallback.push_back((int32_t)(4 * par + c));
            continue;
        }
        const int px = (int)morton_x((uint32_t)par), py = (int)morton_y((uint32_t)par);
        const int32_t c_begin = (int32_t)chunks.size();
        for (int u = 0; u < 16; ++u) {
            const int sx = 2 * px - 1 + (u & 3), sy = 2 * py - 1 + (u >> 2);
            if (sx < 0 || sy < 0 || sx >= m || sy >= m) continue;
            const uint32_t sb = morton((uint32_t)sx, (uint32_t)sy);
            const int32_t slo = lb[sb], sn = lb[sb + 1] - slo;
            if (sn == 0) continue;
            int mask = 0, r = 0;
            for (int c = 0; c < 4; ++c) {
                const int dx = (u & 3) - 1 - (c & 1), dy = (u >> 2) - 1 - (c >> 1);
                if (cnt[c] > 0 && dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1) { mask |= 1 << c; r += wid[c]; }
            }
            if (mask == 0) continue;
            int nrun = 0, run[2] = {0, 0}, rowoff = 0, col[5];
            col[0] = 0;
            for (int c = 0; c < 4; ++c) col[c + 1] = col[c] + wid[c];
            for (int c = 0; c < 4;) {
                if (!(mask >> c & 1)) { ++c; continue; }
                const int c0 = c;
                int w = 0;
                while (c < 4 && (mask >> c & 1)) w += wid[c++];
                run[nrun++] = w | (col[c0] << 8) | (rowoff << 16);
                rowoff += w;
            }
            for (int s0 = 0; s0 < sn; s0 += 8) {
                chunks.push_back({slo + s0, std::min(8, sn - s0), mask, r, boff, (int32_t)par, u, nrun, {run[0], run[1]}, 0});
                boff += (int64_t)r * 32;
                rows += r;
            }
        }
        if ((int)chunks.size() - c_begin > NT_MAXCH) {
            // too many chunks for the kernel's shared record table: SIMT kernel
            for (size_t i = c_begin; i < chunks.size(); ++i) { boff -= (int64_t)chunks[i].rows * 32; rows -= chunks[i].rows; }
            chunks.resize(c_begin);
            for (int c = 0; c < 4; ++c)
                if (cnt[c] > 0) fallback.push_back((int32_t)(4 * par + c));
            continue;
        }
        for (int c = 0; c < 4; ++c)
            if (cnt[c] > 0) leaves.push_back((int32_t)(4 * par + c));
        blocks.push_back((int32_t)par);
        blocks.push_back(c_begin);
        blocks.push_back((int32_t)chunks.size());
        blocks.push_back(0);
    }
    P->nt_nblocks = (int64_t)blocks.size() / 4;
    P->nt_nfallback = (int64_t)fallback.size();
    P->nt_nleaves = (int64_t)leaves.size();
    HFMM_TRY(plan_alloc(P, (void**)&P->nt_leaves, sizeof(int32_t) * std::max<size_t>(leaves.size(), 1)));
    if (!leaves.empty())
        HFMM_CUDA_TRY(cudaMemcpy(P->nt_leaves, leaves.data(), sizeof(int32_t) * leaves.size(), cudaMemcpyHostToDevice));
    HFMM_TRY(plan_alloc(P, (void**)&P->qmax, sizeof(unsigned) * (size_t)P->max_rhs));
    HFMM_TRY(plan_alloc(P, (void**)&P->nt_blocks, sizeof(int32_t) * std::max<size_t>(blocks.size(), 4)));
    HFMM_TRY(plan_alloc(P, (void**)&P->nt_fallback, sizeof(int32_t) * std::max<size_t>(fallback.size(), 1)));
    HFMM_TRY(plan_alloc(P, (void**)&P->nt_chunks, sizeof(NtChunk) * std::max<size_t>(chunks.size(), 1)));
    HFMM_TRY(plan_alloc(P, (void**)&P->nt_tiles, sizeof(__half) * (size_t)std::max<int64_t>(boff, 32)));
    P->table_bytes += sizeof(__half) * (double)boff + sizeof(NtChunk) * (double)chunks.size();
    if (!blocks.empty())
        HFMM_CUDA_TRY(cudaMemcpy(P->nt_blocks, blocks.data(), sizeof(int32_t) * blocks.size(), cudaMemcpyHostToDevice));
    if (!fallback.empty())
        HFMM_CUDA_TRY(cudaMemcpy(P->nt_fallback, fallback.data(), sizeof(int32_t) * fallback.size(),
                                 cudaMemcpyHostToDevice));
    if (!chunks.empty()) {
        HFMM_CUDA_TRY(cudaMemcpy(P->nt_chunks, chunks.data(), sizeof(NtChunk) * chunks.size(), cudaMemcpyHostToDevice));
        HFMM_TRY(fill_near_tiles(P, (int64_t)chunks.size(), rows, st));
    }
    return HFMM_OK;
}

// Launch the tensor-core near field over the plan's blocks; it stores (not
// adds) y of their targets, so it runs before any other writer of y32.
hfmm_status launch_p2p_tc(hfmm_plan_s* P, int nrhs, cudaStream_t st) {
    if (P->nt_nblocks == 0) return HFMM_OK;
    static bool attr_set = false;
    if (!attr_set) {
        HFMM_CUDA_TRY(cudaFuncSetAttribute(p2p_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)NT_SMEM));
        attr_set = true;
    }
    dim3 grid((unsigned)P->nt_nblocks, (unsigned)((nrhs + 63) / 64));
    p2p_tc_kernel<<<grid, NT_THREADS, NT_SMEM, st>>>(P->nt_blocks, P->nt_chunks, P->nt_tiles, P->leaf_begin, P->q32,
                                                     nrhs, P->qmax, P->y32, P->tc_spin, P->tc_err);
    HFMM_CUDA_TRY(cudaGetLastError());
    return HFMM_OK;
}
