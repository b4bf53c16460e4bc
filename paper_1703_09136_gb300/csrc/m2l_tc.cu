// Tensor-core translation passes of the mixed path (tcgen05, sm_103a): the
// downward pass of a level (L2L + free-space M2L + reaction M2L) and the M2M
// of a level, each as one accumulation in tensor memory.
//
// For a pair of target boxes T0, T1 with the same child position (Morton
// b and b + 4), every source step s contributes
//     beta~_T[r][p] += sum_m a~_S[r][m] M_s[m][p]
// to the scaled coefficients of both targets (right-hand side r).  Downward
// steps are the parent's local expansion (L2L), each V-list offset and each
// reaction-table entry; M2M steps are the four children.  In real
// arithmetic a complex product is one real GEMM,
//     D[row][n] += sum_k A[row][k] B_s[n][k],
// rows = (target, r) (2 x 64 = M 128), k = (Re a_m | Im a_m) (K = 2 nc_in,
// padded to 16), n = (Re b_p | Im b_p) (N = 2 nc padded into column blocks
// of at most 128), with B = [[Re M, -Im M], [Im M, Re M]] blocks.
//
// Operand format: f16 pairs x = hi + lo (11 + 11 significant bits, the
// precision of a TF32 pair) and three f16 products per term (hi*hi + hi*lo +
// lo*hi), at twice the TF32 tensor rate and half its operand bytes.  f16 has
// a narrow exponent range, so every operand row is scaled by a power of two
// that puts its largest entry in [2^14, 2^15): one factor per operator
// matrix (plan time) and one per (box, right-hand side, column block) of an
// expansion (written by the kernel that produces it).  A step's product is
// then exact up to the split's rounding times 2^(ea + eb), and the drain
// undoes both factors when it adds the step in FP32 (multiplying by a power
// of two is exact).  Entries far below their row's maximum keep an absolute
// error of about 2^-39 of that maximum.
//
// Operands are stored MMA-ready (pre-split, scaled, core-matrix layout): the
// leaf multipoles by P2M, every other expansion by the kernel that produces
// it, the operators at plan time.  Pipeline (one CTA = one target pair x 64
// right-hand sides x one column block): warp 4 streams every K chunk with
// cp.async.bulk (two 64-row A halves per part plus the operator block) into
// a shared-memory ring sized for the CTAs per SM; warp 5 issues tcgen05.mma
// into one of two TMEM buffers per source step (steps are cut into
// sub-steps at the column blocks of the producing level, so that one
// expansion factor covers a sub-step); warps 0-3 drain each finished step
// with tcgen05.ld into round-to-nearest FP32 registers (tensor-core
// accumulation truncates, so long chains in TMEM lose accuracy) and write the
// result.  Every mbarrier wait is bounded; a timeout sets an error flag
// instead of hanging.
#include <algorithm>
#include <cstring>
#include <map>
#include <vector>

#include "plan.cuh"
#include "tcgen05.cuh"

namespace {

using namespace tc;

// Occupancy of the tensor-core kernel.  Each CTA is one dependent chain (TMA
// -> MMA -> drain per step), so the pass is latency-bound and wants as many
// CTAs per SM as tensor memory, registers and shared memory allow.  Timing
// builds that removed one part of the chain at a time (copies, MMAs, drain)
// moved it by at most 11%, while each extra CTA per SM paid: the widths 48,
// 80 and 96 therefore keep ONE TMEM accumulation buffer (the drain of a step
// then holds back that CTA's next step, but the other CTAs fill the gap) and
// run five (48: 64 columns) or three (80, 96: 128 columns) CTAs per SM; the
// other widths keep two buffers (the drain overlaps the next step's MMAs) in a
// power-of-two allocation (128 columns for NB <= 64, 256 beyond).  The ring
// has as many stages (one 16-wide K chunk each: the two 4 KB A halves, hi and
// lo interleaved, and the B block) as fit the CTA's share of shared memory
// (at least two).
template <int NB>
struct TcCfg {
    // TMEM accumulation buffers per CTA: two (the drain of one step overlaps the
    // next step's MMAs), except at NB = 80, where one 128-column buffer lets a
    // third CTA onto the SM (the CTAs then overlap each other's drains)
    static constexpr int nbuf = (NB == 48 || NB == 80 || NB == 96) ? 1 : 2;
    // a power of two of at least 32 columns: one buffer takes the smallest that
    // holds it, two buffers at least 128
    static constexpr int tmem_cols = nbuf == 1 ? (NB <= 32 ? 32 : NB <= 64 ? 64 : 128) : (2 * NB <= 128 ? 128 : 256);
    static constexpr int buf_cols = tmem_cols / nbuf;
    static constexpr int ctas = NB == 48 ? 5 : nbuf == 1 ? 3 : 512 / tmem_cols;
    static_assert(ctas * tmem_cols <= 512, "the CTAs of an SM fit its tensor memory");
    static constexpr int stage_bytes = 8192 + NB * 64;
    // 228 KB of shared memory per SM; per CTA 1 KB reserved by the system and
    // 256 B of barriers (the kernel has no static shared memory: its 1024-byte
    // aligned dynamic block would pad any to 1 KB)
    static constexpr int budget = 233472 / ctas - 1024 - 256;
    static constexpr int stages = budget / stage_bytes < 8 ? budget / stage_bytes : 8;
    static_assert(stages >= 2, "ring needs two stages");
    static_assert((2 * stages + 4 + 3) * 8 <= 256, "barrier area fits 256 bytes");
    static constexpr size_t smem = (size_t)stages * stage_bytes + 256;
};
constexpr int TC_MAX_NP = 128;         // widest column block (one 128-column TMEM buffer)
constexpr int TC_RUN_LEVELS = 2;       // finest levels with level-wide scales (the leaves and the level above)

// Shared memory of the leaf L2P in the downward epilogue, per drain warp: its
// 32 rows of beta~ (stride NB + 1) and two buffers of the basis rows of 8
// points and its rows of y for them (the next pass's data arrive while this
// pass computes); used only where the four warps' regions fit the ring.
template <int NB>
struct TcL2p {
    static constexpr int pts = NB == 48 ? 4 : 8;
    static constexpr int buf = pts * (NB / 2) * 8 + pts * 32 * 8;
    static constexpr int warp_bytes = 32 * (NB + 1) * 4 + 2 * buf;
    static constexpr bool fits = 4 * warp_bytes <= TcCfg<NB>::stages * TcCfg<NB>::stage_bytes;
};

bool tc_l2p_fits(int nbw) {
    switch (nbw) {
        case 16: return TcL2p<16>::fits;
        case 32: return TcL2p<32>::fits;
        case 48: return TcL2p<48>::fits;
        case 64: return TcL2p<64>::fits;
        case 80: return TcL2p<80>::fits;
        case 96: return TcL2p<96>::fits;
        case 112: return TcL2p<112>::fits;
        case 128: return TcL2p<128>::fits;
    }
    return false;
}

struct TcTile { int32_t b0, b1, s0, s1; };          // boxes (-1: empty), step range
// kind 0 free M2L, 1 reaction M2L, 2 secondary source (L2L parent or M2M child);
// src -1: none; K chunks c0 .. c1 - 1 of the operator
// cont = 1: the next step of the tile accumulates onto this one in TMEM (same
// factor 2^-(ea + eb) for every row: the leaf level with level-wide scales),
// so the result is drained once after the last step of the run.
struct TcStep { int32_t kind, idx, src0, src1, c0, c1, cont; };

// Largest |Re|, |Im| of each complex matrix M[i] (nin x nout) -> 2^-e, the
// factor that undoes its f16 scaling.
__global__ void tc_bscale_kernel(const cf* M, int nin, int nout, float* sc) {
    const int i = blockIdx.x;
    const int64_t per = (int64_t)nin * nout;
    float m = 0.0f;
    for (int64_t e = threadIdx.x; e < per; e += blockDim.x) {
        const cf z = M[(int64_t)i * per + e];
        m = fmaxf(m, fmaxf(fabsf(z.x), fabsf(z.y)));
    }
    __shared__ float red[32];
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
        sc[i] = pow2f(-f16_exp(m));
    }
}

// One factor for the matrices of two tables (the larger of all their factors,
// i.e. the f16 scaling of the largest entry), written back to both.
__global__ void tc_common_scale_kernel(float* sa, int na, float* sb, int nb) {
    __shared__ float red[32];
    float m = 0.0f;
    for (int e = threadIdx.x; e < na + nb; e += blockDim.x) m = fmaxf(m, e < na ? sa[e] : sb[e - na]);
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    m = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
    for (int e = threadIdx.x; e < na + nb; e += blockDim.x) {
        if (e < na) sa[e] = m;
        else sb[e - na] = m;
    }
}

// Largest over leaves and coefficients m of sum_j |B[j][m]| (the leaf's points
// j): |a~_m| <= max_j |q_j| times this.  One warp per leaf; float bits max.
__global__ void p2m_gain_kernel(const int32_t* lb, int64_t nleaf, const cf* basis, int nc, unsigned* gmax) {
    const int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (b >= nleaf) return;
    const int32_t lo = lb[b], hi = lb[b + 1];
    float m = 0.0f;
    for (int n = lane; n < nc; n += 32) {
        float sum = 0.0f;
        for (int32_t j = lo; j < hi; ++j) {
            const cf v = basis[(int64_t)j * nc + n];
            sum += sqrtf(v.x * v.x + v.y * v.y);
        }
        m = fmaxf(m, sum);
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0 && m > 0.0f) atomicMax(gmax, __float_as_uint(m));
}

// Largest over the matrices i and output columns p of sum_m |M[i][m][p]| (M
// nin x nout complex, [m][p] layout): the factor of an infinity-norm bound.
__global__ void tc_colsum_kernel(const cf* M, int nin, int nout, unsigned* gmax) {
    const int i = blockIdx.x;
    float mx = 0.0f;
    for (int p = threadIdx.x; p < nout; p += blockDim.x) {
        float sum = 0.0f;
        for (int m = 0; m < nin; ++m) {
            const cf z = M[((int64_t)i * nin + m) * nout + p];
            sum += sqrtf(z.x * z.x + z.y * z.y);
        }
        mx = fmaxf(mx, sum);
    }
    if (mx > 0.0f) atomicMax(gmax, __float_as_uint(mx));
}

// Pre-split B chunks: for matrix index i, chunk c, part (0 hi, 1 lo):
//   half offset ((i * kc + c) * 2 + part) * (Np * 16) + ((n / 8) * 2 + (k % 16) / 8) * 64 + (n % 8) * 8 + k % 8
// of the entry scaled by 1 / sc[i].  M is a column-major complex matrix [m][p] (nin x nout).
__global__ void tc_btable_kernel(const cf* M, const float* sc, int nmat, int nin, int nout, int Np, int kc,
                                 __half* out) {
    const int64_t per = (int64_t)kc * 16 * Np;   // (n, k) entries per matrix
    const int64_t total = (int64_t)nmat * per;
    uint16_t* o = (uint16_t*)out;
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
        uint16_t hi, lo;
        split_f16(v / sc[i], hi, lo);
        const int c = k / 16, kk = k % 16;
        const int64_t base = (((int64_t)i * kc + c) * 2) * (Np * 16);
        const int64_t core = ((n / 8) * 2 + kk / 8) * 64 + (n % 8) * 8 + kk % 8;
        o[base + core] = hi;
        o[base + Np * 16 + core] = lo;
    }
}

// MMA-ready expansions: per box, per 64-row right-hand-side chunk rc, per K
// chunk c (16 real values: Re a_0..a_{nin-1} then Im, zero padded), one 4 KB
// block of 64 rows x 16 halves x (hi, lo) in the no-swizzle core-matrix
// layout with the two parts interleaved per 8-row group (row-group stride
// 512 B, part stride 256 B, K-core stride 128 B), so that one bulk copy moves
// both parts of a 64-row operand half:
//   half offset ((box * nrc + rc) * kc + c) * 2048
//               + (r / 8) * 256 + part * 128 + (kk / 8) * 64 + (r % 8) * 8 + kk % 8,
// of the coefficient times 2^e(box, rc, block, r); the factor 2^-e is stored at
//   ((box * nrc + rc) * nsb + block) * 64 + r,
// block = c / sblk, where the producing level has nsb column blocks of sblk
// K chunks.  The leaf multipoles are written in this form by P2M, all other
// expansions by the tensor-core kernel that produces them.

constexpr int TC2_THREADS = 192;   // warps 0-3 drain, warp 4 TMA, warp 5 MMA

// Store one row of a finished tile: the FP32 coefficients out[box][r][0 .. nc)
// (columns n0 .. n0 + NB - 1 of the real GEMM: Re then Im) and, when sdst is
// given, the MMA-ready copy of the row with its factor (every row of the
// 64-row block, so rows r >= nrhs stay zero).
template <int NB>
__device__ __forceinline__ void tc_store_row(const float (&acc)[NB], int box, int row, int rc, int cb, int nbz,
                                             int n0, int nrhs, int nc, int nrc, cf* __restrict__ out,
                                             __half* __restrict__ sdst, float* __restrict__ ssc, int kcd,
                                             const unsigned* __restrict__ qmax, float qgain) {
    const int rr = row & 63, r = rc * 64 + rr;
    if (out && r < nrhs) {
        float* o = (float*)(out + ((int64_t)box * nrhs + r) * nc);
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            const int g = n0 + j;
            if (g < nc) o[2 * g] = acc[j];
            else if (g < 2 * nc) o[2 * (g - nc) + 1] = acc[j];
        }
    }
    if (sdst) {
        // level-wide scale (qmax given): the exponent of the bound 2 max|q_r| qgain
        float m = 0.0f;
        if (qmax) m = r < nrhs ? 2.0f * __uint_as_float(qmax[r]) * qgain : 0.0f;
        else
#pragma unroll
            for (int j = 0; j < NB; ++j) m = fmaxf(m, fabsf(acc[j]));
        const int e = f16_exp(m);
        const float s = pow2f(e);
        ssc[(((int64_t)box * nrc + rc) * nbz + cb) * 64 + rr] = pow2f(-e);
        uint16_t* base = (uint16_t*)sdst + ((int64_t)box * nrc + rc) * kcd * 2048 + (rr >> 3) * 256 + (rr & 7) * 8;
#pragma unroll
        for (int j = 0; j < NB; j += 8) {
            const int g = n0 + j;
            if ((g >> 4) < kcd) {
                uint16_t h[8], lo[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) split_f16(acc[j + u] * s, h[u], lo[u]);
                uint16_t* d = base + (int64_t)(g >> 4) * 2048 + ((g & 15) >> 3) * 64;
                *(uint4*)d = pack8(h);
                *(uint4*)(d + 128) = pack8(lo);
            }
        }
    }
}

// One CTA = one target pair x 64 right-hand sides x one block of NB real
// output columns (columns n0 .. n0 + NB - 1 of the Np-wide GEMM) x one
// segment of the tile's steps (blockIdx.z = segment * column blocks + block).
// With one segment the result goes to the FP32 coefficients out[box][r][0 ..
// nc) and, when sdst is given, also in MMA-ready form (kcd K chunks, the
// layout above) for the next tensor-core consumer; with several segments
// (levels with too few tiles to fill the GPU) each CTA writes its partial
// sums to part and tc_reduce_kernel finishes the store.  Sources of kind 0
// and 1 are read from amma (factors asc, nsba column blocks of sba chunks),
// kind 2 from pmma (psc, nsbp, sbp); operator factors sfree, sreact, ssec.
template <int NB>
__global__ void __launch_bounds__(TC2_THREADS, TcCfg<NB>::ctas) m2l_tc_kernel(
    const TcTile* __restrict__ tiles, const TcStep* __restrict__ steps, const __half* __restrict__ Bfree,
    const __half* __restrict__ Breact, const __half* __restrict__ Bl2l, const float* __restrict__ sfree,
    const float* __restrict__ sreact, const float* __restrict__ ssec, const __half* __restrict__ amma,
    const float* __restrict__ asc, int nsba, int sba, const __half* __restrict__ pmma,
    const float* __restrict__ psc, int nsbp, int sbp, const __half* __restrict__ zero4k, cf* __restrict__ out,
    int nrhs, int nc, int kc, int kc2, int nrc, int Np, __half* __restrict__ sdst, float* __restrict__ ssc, int kcd,
    int nseg, float* __restrict__ part, const cf* __restrict__ l2p_basis, const int32_t* __restrict__ lbeg,
    cf* __restrict__ ys, long spin, int* err, const unsigned* __restrict__ qmax, float qgain) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    using CFG = TcCfg<NB>;
    constexpr int stage_bytes = CFG::stage_bytes;
    constexpr int TC_STAGES = CFG::stages;
    uint64_t* full = (uint64_t*)(smem + TC_STAGES * stage_bytes);
    uint64_t* empty = full + TC_STAGES;
    uint64_t* dfull = empty + TC_STAGES;
    uint64_t* dfree = dfull + 2;
    // barrier area after the ring: full[], empty[], dfull[2], dfree[2], then 8-byte
    // slots for the TMEM address, the MMA-completion barrier and the abort flag
    uint32_t* tslot = (uint32_t*)(dfree + 2);
    uint64_t& mdone = *(dfree + 3);
    volatile int& s_abort = *(volatile int*)(dfree + 4);
    const TcTile tile = tiles[blockIdx.x];
    const int rc = blockIdx.y;
    const int nbz = Np / NB;
    const int cb = (int)blockIdx.z % nbz, seg = (int)blockIdx.z / nbz;
    const int n0 = cb * NB;
    const uint32_t ncols = CFG::tmem_cols;
    if (tid == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(su32(&full[s])), "r"(1));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(su32(&empty[s])), "r"(1));
        }
        for (int b = 0; b < 2; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(su32(&dfull[b])), "r"(1));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(su32(&dfree[b])), "r"(128));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(su32(&mdone)), "r"(1));
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
    int sbeg = tile.s0, nsteps = tile.s1 - tile.s0;
    if (nseg > 1) {
        const int len = (nsteps + nseg - 1) / nseg;
        const int a = min(nsteps, seg * len);
        sbeg = tile.s0 + a;
        nsteps = min(nsteps, a + len) - a;
    }
    if (warp < 4) {
        // ---------------- drain: FP32 round-to-nearest accumulation ----------------
        const int row = tid, tgt = row >> 6, rr = row & 63;
        float acc[NB];
#pragma unroll
        for (int j = 0; j < NB; ++j) acc[j] = 0.0f;
        bool ok = true;
        // the factor 2^-(ea + eb) of step s for this row (0 for a missing source)
        auto factor = [&](int s) -> float {
            const TcStep st = steps[sbeg + s];
            const int src = tgt ? st.src1 : st.src0;
            if (src < 0) return 0.0f;
            const bool sec = st.kind == 2;
            const float* scs = sec ? psc : asc;
            const int nsb = sec ? nsbp : nsba, sbk = sec ? sbp : sba;
            const float fb = st.kind == 0 ? sfree[st.idx] : st.kind == 1 ? sreact[st.idx] : ssec[st.idx];
            return scs[(((int64_t)src * nrc + rc) * nsb + st.c0 / sbk) * 64 + rr] * fb;
        };
        // one drain per run of steps (a step, or the steps joined by cont); the
        // run's factor is that of any of its steps with a source for this row
        for (int s = 0, run = 0; s < nsteps && ok; ++run) {
            int e = s;
            float f = factor(s);
            while (e + 1 < nsteps && steps[sbeg + e].cont) {
                ++e;
                if (f == 0.0f) f = factor(e);
            }
            s = e + 1;
            const int b = run % CFG::nbuf;
            bool good = !s_abort && mbar_wait(&dfull[b], (uint32_t)((run / CFG::nbuf) & 1), spin);
            good = __all_sync(0xffffffffu, good);
            if (!good) { ok = false; s_abort = 1; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t tb = taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)(b * CFG::buf_cols);
#pragma unroll
            for (int c0 = 0; c0 < NB; c0 += 16) {
                uint32_t v[16];
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                             : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                               "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                               "=r"(v[14]), "=r"(v[15])
                             : "r"(tb + (uint32_t)c0));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int j = 0; j < 16; ++j) acc[c0 + j] = fmaf(__uint_as_float(v[j]), f, acc[c0 + j]);
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(&dfree[b]);
        }
        if (!ok || s_abort) {
            if (lane == 0) atomicExch(err, 1);
        } else if (part) {
            float* pp = part + ((((int64_t)seg * gridDim.x + blockIdx.x) * gridDim.y + rc) * nbz + cb) * 128 * NB +
                        (int64_t)row * NB;
#pragma unroll
            for (int j = 0; j < NB; j += 4) *(float4*)(pp + j) = make_float4(acc[j], acc[j + 1], acc[j + 2], acc[j + 3]);
        } else {
            const int box = tgt ? tile.b1 : tile.b0;   // uniform over the warp
            if (box >= 0) {
                tc_store_row<NB>(acc, box, row, rc, cb, nbz, n0, nrhs, nc, nrc, nullptr, sdst, ssc, kcd, qmax, qgain);
                if ((TcL2p<NB>::fits && l2p_basis) || out) {
                    // The warp's 32 rows of the result go to the ring once (every MMA of
                    // this CTA has completed; one region per warp); the leaf L2P and the
                    // FP32 store read them from there.
                    constexpr int WS = TcL2p<NB>::fits ? TcL2p<NB>::warp_bytes : 32 * (NB + 1) * 4;
                    static_assert(4 * WS <= TC_STAGES * stage_bytes, "staging fits the ring");
                    float* bet = (float*)(smem + warp * WS);
#pragma unroll
                    for (int j = 0; j < NB; ++j) bet[lane * (NB + 1) + j] = acc[j];
                    __syncwarp();
                    if (TcL2p<NB>::fits && l2p_basis) {
                        // L2P of the leaf (Algorithm 1, step 4), one column block:
                        // y[t][r] += sum_m beta~[r][m] (i/4) conj(B[t][m]) over the leaf's
                        // points t, eight points per pass.  The basis rows and this
                        // warp's rows of y of the next pass are copied (cp.async, second
                        // buffer) while this pass computes; the sum reads beta~ by row and
                        // the basis as broadcasts (each beta~ load feeds 32 FMAs).
                        constexpr int TCH = TcL2p<NB>::pts;
                        unsigned char* bufs = (unsigned char*)(bet + 32 * (NB + 1));
                        const float* br = bet + lane * (NB + 1);   // Re beta~_m at m, Im at nc + m
                        const int r = rc * 64 + (row & 63);
                        const bool live = r < nrhs;
                        const int32_t t0 = lbeg[box], t1 = lbeg[box + 1];
                        auto issue = [&](int32_t tc0, int k) {
                            cf* sbs = (cf*)(bufs + (k & 1) * TcL2p<NB>::buf);
                            cf* sy = sbs + TCH * (NB / 2);
                            const int tn = min(TCH, t1 - tc0);
                            for (int e = lane; e < tn * nc; e += 32)
                                cp_async8(sbs + e, l2p_basis + (int64_t)tc0 * nc + e);
                            if (live)
                                for (int t = 0; t < tn; ++t)
                                    cp_async8(sy + t * 32 + lane, ys + (int64_t)(tc0 + t) * nrhs + r);
                            asm volatile("cp.async.commit_group;" ::: "memory");
                        };
                        if (t0 < t1) issue(t0, 0);
                        int kk = 0;
                        for (int32_t tc0 = t0; tc0 < t1; tc0 += TCH, ++kk) {
                            const int tn = min(TCH, t1 - tc0);
                            if (tc0 + TCH < t1) {
                                issue(tc0 + TCH, kk + 1);
                                asm volatile("cp.async.wait_group 1;" ::: "memory");
                            } else {
                                asm volatile("cp.async.wait_group 0;" ::: "memory");
                            }
                            __syncwarp();
                            const cf* sbs = (const cf*)(bufs + (kk & 1) * TcL2p<NB>::buf);
                            const cf* sy = sbs + TCH * (NB / 2);
                            float yr[TCH], yi[TCH];
#pragma unroll
                            for (int u = 0; u < TCH; ++u) yr[u] = yi[u] = 0.0f;
                            for (int m = 0; m < nc; ++m) {
                                const float are = br[m], aim = br[nc + m];
#pragma unroll
                                for (int u = 0; u < TCH; ++u) {
                                    const cf bv = sbs[(u < tn ? u : 0) * nc + m];
                                    yr[u] = fmaf(are, bv.y, fmaf(-aim, bv.x, yr[u]));
                                    yi[u] = fmaf(are, bv.x, fmaf(aim, bv.y, yi[u]));
                                }
                            }
                            if (live) {
#pragma unroll
                                for (int u = 0; u < TCH; ++u)
                                    if (u < tn) {
                                        const cf y0 = sy[u * 32 + lane];
                                        ys[(int64_t)(tc0 + u) * nrhs + r] =
                                            cfmk(y0.x + 0.25f * yr[u], y0.y + 0.25f * yi[u]);
                                    }
                            }
                            __syncwarp();   // this buffer is the copy target two passes on
                        }
                    }
                    if (out) {
                        // FP32 coefficients: the warp's 32 rows are one contiguous range of
                        // out ([box][r][coef] complex), stored along that range
                        const int rfirst = rc * 64 + ((warp * 32) & 63);
                        const int nrows = min(32, nrhs - rfirst);
                        if (nrows > 0) {
                            float* o = (float*)(out + ((int64_t)box * nrhs + rfirst) * nc);
                            const int w2 = 2 * nc;
                            int i = lane / w2, w = lane - (lane / w2) * w2;   // f = i * w2 + w
                            for (int f = lane; f < nrows * w2; f += 32) {
                                const int g = (w & 1) * nc + (w >> 1);
                                if (g >= n0 && g < n0 + NB) o[f] = bet[i * (NB + 1) + g - n0];
                                w += 32;
                                while (w >= w2) { w -= w2; ++i; }
                            }
                        }
                    }
                }
            }
        }
    } else if (warp == 4 && lane == 0) {
        // ---------------- TMA: A halves (two source boxes) and the operator block ----------------
        // (hi and lo of a single-block operator are contiguous: one copy)
        const bool one_b = Np == NB;
        int i = 0;
        TcStep nxt = nsteps > 0 ? steps[sbeg] : TcStep{0, 0, -1, -1, 0, 0};
        for (int s = 0; s < nsteps; ++s) {
            const TcStep st = nxt;
            if (s + 1 < nsteps) nxt = steps[sbeg + s + 1];   // one step ahead
            const bool sec = st.kind == 2;
            const int nk = sec ? kc2 : kc;
            const __half* base = sec ? pmma : amma;
            const __half* Bm = st.kind == 0 ? Bfree + (int64_t)st.idx * nk * 32 * Np
                             : st.kind == 1 ? Breact + (int64_t)st.idx * nk * 32 * Np
                                            : Bl2l + (int64_t)st.idx * nk * 32 * Np;
            bool stop = false;
            for (int c = st.c0; c < st.c1; ++c, ++i) {
                const int stg = i % TC_STAGES;
                const uint32_t ph = (uint32_t)((i / TC_STAGES) & 1);
                if (s_abort || !mbar_wait(&empty[stg], ph ^ 1u, spin)) { s_abort = 1; stop = true; break; }
                unsigned char* sb = smem + stg * stage_bytes;
                mbar_arrive_tx(&full[stg], (uint32_t)stage_bytes);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int src = h ? st.src1 : st.src0;
                    const __half* g = (src >= 0) ? base + (((int64_t)src * nrc + rc) * nk + c) * 2048 : zero4k;
                    bulk_g2s(sb + h * 4096, g, 4096u, &full[stg]);
                }
                const __half* Bc = Bm + (int64_t)c * 32 * Np + (int64_t)n0 * 16;
                if (one_b) {
                    bulk_g2s(sb + 8192, Bc, (uint32_t)(NB * 64), &full[stg]);
                } else {
                    bulk_g2s(sb + 8192, Bc, (uint32_t)(NB * 32), &full[stg]);
                    bulk_g2s(sb + 8192 + NB * 32, Bc + (int64_t)Np * 16, (uint32_t)(NB * 32), &full[stg]);
                }
            }
            if (stop) break;
        }
        if (s_abort) {
            // copies still in flight land in the ring: wait for them (default bound,
            // whatever the plan's limit) before the exit
            for (int k = max(0, i - TC_STAGES); k < i; ++k)
                mbar_wait(&full[k % TC_STAGES], (uint32_t)((k / TC_STAGES) & 1));
        }
    } else if (warp == 5 && lane == 0) {
        // ---------------- MMA issuer: one TMEM buffer per run of source steps ----------------
        constexpr uint32_t idesc = idesc_f16(NB);
        int i = 0, run = 0;
        bool ok = true, cont_prev = false;
        int nk_next = nsteps > 0 ? steps[sbeg].c1 - steps[sbeg].c0 : 0;
        bool cont_next = nsteps > 0 && steps[sbeg].cont;
        for (int s = 0; s < nsteps && ok; ++s) {
            const int nk = nk_next;
            const bool cont = cont_next && s + 1 < nsteps;   // a run ends with the segment
            if (s + 1 < nsteps) {
                nk_next = steps[sbeg + s + 1].c1 - steps[sbeg + s + 1].c0;
                cont_next = steps[sbeg + s + 1].cont;
            }
            const int b = run % CFG::nbuf;
            if (!cont_prev) {
                if (s_abort || !mbar_wait(&dfree[b], (uint32_t)(((run / CFG::nbuf) & 1) ^ 1), spin)) { s_abort = 1; break; }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            }
            const uint32_t dt = taddr + (uint32_t)(b * CFG::buf_cols);
            for (int c = 0; c < nk; ++c, ++i) {
                const int stg = i % TC_STAGES;
                const uint32_t ph = (uint32_t)((i / TC_STAGES) & 1);
                if (s_abort || !mbar_wait(&full[stg], ph, spin)) { ok = false; s_abort = 1; break; }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t sb = su32(smem + stg * stage_bytes);
                const uint64_t ah = sdesc(sb, 512), al = sdesc(sb + 256, 512);
                const uint64_t bh = sdesc(sb + 8192, 256), bl = sdesc(sb + 8192 + NB * 32, 256);
                mma_f16(dt, ah, bh, idesc, (c > 0 || cont_prev) ? 1u : 0u);
                mma_f16(dt, ah, bl, idesc, 1);
                mma_f16(dt, al, bh, idesc, 1);
                mma_commit(&empty[stg]);
            }
            if (ok && !cont) {
                mma_commit(&dfull[b]);
                ++run;
            }
            cont_prev = cont;
        }
        // every MMA of this thread has completed before TMEM is released
        mma_commit(&mdone);
        mbar_wait(&mdone, 0u);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(taddr), "r"(ncols));
}

// Sum the segments' partial results of a split launch and store them like
// the single-segment epilogue; one warp per (tile, RHS block, column block,
// row), lane jq holding columns 4 jq .. 4 jq + 3 of the block.
template <int NB>
__global__ void tc_reduce_kernel(const TcTile* __restrict__ tiles, int ntiles, int nrcl, int nbz, int nseg,
                                 const float* __restrict__ part, cf* __restrict__ out, int nrhs, int nc, int nrc,
                                 __half* __restrict__ sdst, float* __restrict__ ssc, int kcd,
                                 const unsigned* __restrict__ qmax, float qgain) {
    constexpr int NQ = NB / 4;
    const int lane = threadIdx.x & 31;
    const int64_t nwarp = (int64_t)ntiles * nrcl * nbz * 128;
    const int64_t wstride = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t wi = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); wi < nwarp; wi += wstride) {
        const int row = (int)(wi % 128);
        int64_t rest = wi / 128;
        const int cb = (int)(rest % nbz);
        rest /= nbz;
        const int rc = (int)(rest % nrcl);
        const int64_t t = rest / nrcl;
        const TcTile tile = tiles[t];
        const int box = (row >> 6) ? tile.b1 : tile.b0;
        if (box < 0) continue;   // uniform over the warp
        const int jq = lane;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (jq < NQ)
            for (int sg = 0; sg < nseg; ++sg) {
                const float4 w = *(const float4*)(part + ((((int64_t)sg * ntiles + t) * nrcl + rc) * nbz + cb) * 128 * NB +
                                                  (int64_t)row * NB + 4 * jq);
                v.x += w.x; v.y += w.y; v.z += w.z; v.w += w.w;
            }
        const float a4[4] = {v.x, v.y, v.z, v.w};
        const int rr = row & 63, r = rc * 64 + rr, g0 = cb * NB + 4 * jq;
        if (out && jq < NQ && r < nrhs) {
            float* o = (float*)(out + ((int64_t)box * nrhs + r) * nc);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int g = g0 + u;
                if (g < nc) o[2 * g] = a4[u];
                else if (g < 2 * nc) o[2 * (g - nc) + 1] = a4[u];
            }
        }
        if (sdst) {
            float m = fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w)));
            for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
            if (qmax) m = r < nrhs ? 2.0f * __uint_as_float(qmax[r]) * qgain : 0.0f;   // level-wide scale
            const int e = f16_exp(m);
            if (lane == 0) ssc[(((int64_t)box * nrc + rc) * nbz + cb) * 64 + rr] = pow2f(-e);
            if (jq < NQ && (g0 >> 4) < kcd) {
                const float s = pow2f(e);
                uint16_t h[4], lo[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) split_f16(a4[u] * s, h[u], lo[u]);
                uint16_t* d = (uint16_t*)sdst + ((int64_t)box * nrc + rc) * kcd * 2048 + (rr >> 3) * 256 + (rr & 7) * 8 +
                              (int64_t)(g0 >> 4) * 2048 + ((g0 & 15) >> 3) * 64 + (g0 & 7);
                *(uint2*)d = make_uint2((uint32_t)h[0] | ((uint32_t)h[1] << 16), (uint32_t)h[2] | ((uint32_t)h[3] << 16));
                *(uint2*)(d + 128) =
                    make_uint2((uint32_t)lo[0] | ((uint32_t)lo[1] << 16), (uint32_t)lo[2] | ((uint32_t)lo[3] << 16));
            }
        }
    }
}

inline int round16(int x) { return (x + 15) / 16 * 16; }

// Width of a level's real GEMM: 2 nc columns in nb blocks of nbw <= 128
// (multiples of 16, padding spread over the blocks); K chunks of 16.
void tc_widths(int ncoef, int* nb, int* nbw, int* np, int* kc) {
    const int w = 2 * ncoef;
    *nb = (w + TC_MAX_NP - 1) / TC_MAX_NP;
    *nbw = round16((w + *nb - 1) / *nb);
    *np = *nb * *nbw;
    *kc = round16(w) / 16;
}

// Target pairs (b, b + 4) with b = 8 j + c (same child position, parents 2j
// and 2j + 1); a missing or empty box is -1.  add(b0, b1) appends the pair's
// source steps.
// Append one source step as sub-steps of sblk K chunks (the column blocks of
// the level that produced the source expansion: one factor per sub-step).
void push_step(std::vector<TcStep>& steps, int kind, int idx, int32_t s0, int32_t s1, int nk, int sblk) {
    for (int c0 = 0; c0 < nk; c0 += sblk)
        steps.push_back({kind, idx, s0, s1, c0, std::min(nk, c0 + sblk)});
}

template <class NonEmpty, class Add>
void pair_tiles(int64_t nbox, NonEmpty nonempty, Add add, std::vector<TcTile>& tiles, std::vector<TcStep>& steps) {
    const int64_t ngroups = std::max<int64_t>(1, nbox / 8);
    for (int64_t j = 0; j < ngroups; ++j)
        for (int c = 0; c < 4; ++c) {
            const int64_t b0 = 8 * j + c, b1 = 8 * j + 4 + c;
            const bool e0 = b0 < nbox && nonempty(b0), e1 = b1 < nbox && nonempty(b1);
            if (!e0 && !e1) continue;
            TcTile t;
            t.b0 = e0 ? (int32_t)b0 : -1;
            t.b1 = e1 ? (int32_t)b1 : -1;
            t.s0 = (int32_t)steps.size();
            add(t.b0, t.b1);
            t.s1 = (int32_t)steps.size();
            tiles.push_back(t);   // also without steps: the kernel then writes zeros
        }
}

hfmm_status upload_tiles(hfmm_plan_s* P, const std::vector<TcTile>& tiles, const std::vector<TcStep>& steps,
                         void** dt, void** ds, int64_t* nt, int* maxsteps) {
    *nt = (int64_t)tiles.size();
    *maxsteps = 0;
    for (const TcTile& t : tiles) *maxsteps = std::max(*maxsteps, (int)(t.s1 - t.s0));
    HFMM_TRY(plan_alloc(P, dt, sizeof(TcTile) * std::max<size_t>(tiles.size(), 1)));
    HFMM_TRY(plan_alloc(P, ds, sizeof(TcStep) * std::max<size_t>(steps.size(), 1)));
    if (!tiles.empty()) {
        HFMM_CUDA_TRY(cudaMemcpy(*dt, tiles.data(), sizeof(TcTile) * tiles.size(), cudaMemcpyHostToDevice));
        HFMM_CUDA_TRY(cudaMemcpy(*ds, steps.data(), sizeof(TcStep) * steps.size(), cudaMemcpyHostToDevice));
    }
    return HFMM_OK;
}

hfmm_status btable(hfmm_plan_s* P, const cf* M, int nmat, int nin, int nout, int Np, int kc, __half** out,
                   float** sc, cudaStream_t st) {
    const size_t halves = (size_t)nmat * kc * 32 * Np;
    HFMM_TRY(plan_alloc(P, (void**)out, sizeof(__half) * halves));
    HFMM_TRY(plan_alloc(P, (void**)sc, sizeof(float) * nmat));
    tc_bscale_kernel<<<nmat, 256, 0, st>>>(M, nin, nout, *sc);
    HFMM_CUDA_TRY(cudaGetLastError());
    tc_btable_kernel<<<4 * 152, 256, 0, st>>>(M, *sc, nmat, nin, nout, Np, kc, *out);
    HFMM_CUDA_TRY(cudaGetLastError());
    P->table_bytes += sizeof(__half) * (double)halves + sizeof(float) * (double)nmat;
    return HFMM_OK;
}

// Arguments of one launch of the tensor-core kernel: sources of kind 0 / 1
// from amma (factors asc; nsba column blocks of sba K chunks), kind 2 from
// pmma (psc, nsbp, sbp); the result to out and, when sdst is given, in
// MMA-ready form with factors ssc.
struct TcLaunch {
    const void* tiles;
    const void* steps;
    int64_t ntiles;
    const __half* Bfree;
    const __half* Breact;
    const __half* Bsec;
    const float* sfree;
    const float* sreact;
    const float* ssec;
    const __half* amma;
    const float* asc;
    int nsba, sba;
    const __half* pmma;
    const float* psc;
    int nsbp, sbp;
    cf* out;
    int nc, kc, kc2, np, nb, nbw;
    __half* sdst;
    float* ssc;
    int kcd;
    int maxsteps;
    bool l2p;        // leaf level: L2P into y32 from the epilogue
    const unsigned* qmax = nullptr;   // sdst with the level-wide scale 2 max|q_r| qgain
    float qgain = 0.0f;
};

// Segments per tile for a launch of ntiles x nb CTAs (x nrc RHS blocks): split
// the step lists when the launch would leave most SMs idle.
int tc_nseg(int64_t ntiles, int nb, int nrc, int maxsteps) {
    const int64_t ctas = ntiles * nb * nrc;
    if (ctas >= 2 * 152 || maxsteps < 4) return 1;
    const int64_t want = (4 * 152 + ctas - 1) / ctas;
    return (int)std::max<int64_t>(1, std::min<int64_t>({want, 16, maxsteps / 2}));
}

template <int NB>
hfmm_status launch_nb(hfmm_plan_s* P, const TcLaunch& a, int nrhs, cudaStream_t st) {
    const size_t smem = TcCfg<NB>::smem;
    static bool attr_set = false;
    if (!attr_set) {
        HFMM_CUDA_TRY(cudaFuncSetAttribute(m2l_tc_kernel<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr_set = true;
    }
    const int nrc = (P->max_rhs + 63) / 64;
    const int nrcl = (nrhs + 63) / 64;
    const int nseg = tc_nseg(a.ntiles, a.nb, nrc, a.maxsteps);
    float* part = nseg > 1 ? P->tc_part : nullptr;
    dim3 grid((unsigned)a.ntiles, (unsigned)nrcl, (unsigned)(a.nb * nseg));
    m2l_tc_kernel<NB><<<grid, TC2_THREADS, smem, st>>>(
        (const TcTile*)a.tiles, (const TcStep*)a.steps, a.Bfree, a.Breact, a.Bsec, a.sfree, a.sreact, a.ssec, a.amma,
        a.asc, a.nsba, a.sba, a.pmma, a.psc, a.nsbp, a.sbp, P->tc_zero, a.out, nrhs, a.nc, a.kc, a.kc2, nrc, a.np,
        a.sdst, a.ssc, a.kcd, nseg, part, a.l2p ? P->basis32 : nullptr, P->leaf_begin, P->y32, P->tc_spin, P->tc_err,
        a.qmax, a.qgain);
    HFMM_CUDA_TRY(cudaGetLastError());
    if (part) {
        const int64_t warps = a.ntiles * nrcl * a.nb * 128;
        const unsigned blocks = (unsigned)std::min<int64_t>((warps + 7) / 8, 8 * 152);
        tc_reduce_kernel<NB><<<blocks, 256, 0, st>>>((const TcTile*)a.tiles, (int)a.ntiles, nrcl, a.nb, nseg, part,
                                                      a.out, nrhs, a.nc, nrc, a.sdst, a.ssc, a.kcd, a.qmax, a.qgain);
        HFMM_CUDA_TRY(cudaGetLastError());
        ++P->launches;
    }
    return HFMM_OK;
}

hfmm_status launch_tc(hfmm_plan_s* P, const TcLaunch& a, int nrhs, cudaStream_t st) {
    if (a.ntiles == 0) return HFMM_OK;
    switch (a.nbw) {
        case 16: return launch_nb<16>(P, a, nrhs, st);
        case 32: return launch_nb<32>(P, a, nrhs, st);
        case 48: return launch_nb<48>(P, a, nrhs, st);
        case 64: return launch_nb<64>(P, a, nrhs, st);
        case 80: return launch_nb<80>(P, a, nrhs, st);
        case 96: return launch_nb<96>(P, a, nrhs, st);
        case 112: return launch_nb<112>(P, a, nrhs, st);
        case 128: return launch_nb<128>(P, a, nrhs, st);
    }
    hfmm_set_error("tensor-core pass: unsupported block width %d", a.nbw);
    return HFMM_ERR_UNSUPPORTED;
}

}  // namespace

// One bounded wait on a barrier whose phase completes only when `arrive` is
// set (the arrival happens before the wait): out = 1 if the wait gave up.
__global__ void tc_wait_probe_kernel(long spin, int arrive, int* out) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(tc::su32(&bar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
        if (arrive) tc::mbar_arrive(&bar);
        *out = tc::mbar_wait(&bar, 0u, spin) ? 0 : 1;
    }
}

hfmm_status tc_wait_probe(long spin, int arrive, int* timed_out) {
    int* d = nullptr;
    HFMM_CUDA_TRY(cudaMalloc(&d, sizeof(int)));
    tc_wait_probe_kernel<<<1, 32>>>(spin, arrive, d);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(timed_out, d, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) {
        hfmm_set_error("wait probe: %s", cudaGetErrorString(e));
        return HFMM_ERR_CUDA;
    }
    return HFMM_OK;
}

// Plan-time preparation of the tensor-core upward (M2M) and downward
// (L2L + M2L) passes of every level lmin .. L.
// Largest float of a one-word device max (float bits), read back synchronously.
hfmm_status read_fmax(hfmm_plan_s* P, unsigned* d, float* out, cudaStream_t st) {
    unsigned h = 0;
    HFMM_CUDA_TRY(cudaMemcpyAsync(&h, d, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    HFMM_CUDA_TRY(cudaStreamSynchronize(st));
    std::memcpy(out, &h, sizeof(float));
    return HFMM_OK;
}

hfmm_status build_tc(hfmm_plan_s* P, cudaStream_t st) {
    const int L = P->L;
    const int nrc = (P->max_rhs + 63) / 64;
    const auto& lb = P->h_leaf_begin;
    // Level-wide scales, so that the free and reaction steps of a tile (and the
    // four children of an M2M tile) accumulate in TMEM with one drain: the leaves,
    // when their P2M is the row kernel (bound 2 max|q_r| sum_j |B[j][m]|), and up
    // to TC_RUN_LEVELS - 1 levels above, while their rows fit one column block
    // (bound 4 max_c ||T_c|| times the bound of the level below, T_c the scaled
    // M2M shifts).
    {
        LevelInfo& lf = P->lev[L];
        if (lf.ncoef <= 32 && lf.nv + lf.nr > 0) {
            unsigned* dg = nullptr;
            HFMM_TRY(plan_alloc(P, (void**)&dg, (TC_RUN_LEVELS + 1) * sizeof(unsigned)));
            HFMM_CUDA_TRY(cudaMemsetAsync(dg, 0, (TC_RUN_LEVELS + 1) * sizeof(unsigned), st));
            p2m_gain_kernel<<<(unsigned)ceil_div(lf.nbox, 4), 128, 0, st>>>(P->leaf_begin, lf.nbox, P->basis32,
                                                                            lf.ncoef, dg);
            HFMM_CUDA_TRY(cudaGetLastError());
            HFMM_TRY(read_fmax(P, dg, &P->p2m_gain, st));
            lf.tc_runs = P->tc_leaf_runs = true;
            lf.tc_gain = P->p2m_gain;
            for (int l = L - 1, i = 1; l >= P->lmin && i < TC_RUN_LEVELS; --l, ++i) {
                LevelInfo& up = P->lev[l];
                const LevelInfo& dn = P->lev[l + 1];
                int nb, nbw, np, kc;
                tc_widths(up.ncoef, &nb, &nbw, &np, &kc);
                if (nb != 1 || up.nv + up.nr == 0 || !up.t_m2m32) break;
                tc_colsum_kernel<<<4, 128, 0, st>>>(up.t_m2m32, dn.ncoef, up.ncoef, dg + i);
                HFMM_CUDA_TRY(cudaGetLastError());
                float cs = 0.0f;
                HFMM_TRY(read_fmax(P, dg + i, &cs, st));
                up.tc_runs = true;
                up.tc_gain = 4.0f * cs * dn.tc_gain;
            }
        }
    }
    for (int l = P->lmin; l <= L; ++l) {
        LevelInfo& lv = P->lev[l];
        tc_widths(lv.ncoef, &lv.tc_nb, &lv.tc_nbw, &lv.tc_np, &lv.tc_kc);
        const bool has_parent = l > P->lmin;
        const int npp = has_parent ? P->lev[l - 1].ncoef : 0;
        lv.tc_kc2 = has_parent ? P->lev[l - 1].tc_kc : 0;
        const int Np = lv.tc_np;
        if (lv.tc_nb > 16) {
            hfmm_set_error("tensor-core pass: level %d needs %d column blocks (at most 16)", l, lv.tc_nb);
            return HFMM_ERR_UNSUPPORTED;
        }
        // MMA-ready copies (and their factors): this level's multipoles and the parent's locals
        const size_t ab = sizeof(__half) * (size_t)lv.nbox * nrc * lv.tc_kc * 2048;
        const size_t as = sizeof(float) * (size_t)lv.nbox * nrc * lv.tc_nb * 64;
        HFMM_TRY(plan_alloc(P, (void**)&lv.tc_amma, ab));
        HFMM_CUDA_TRY(cudaMemsetAsync(lv.tc_amma, 0, ab, st));
        HFMM_TRY(plan_alloc(P, (void**)&lv.tc_asc, as));
        HFMM_CUDA_TRY(cudaMemsetAsync(lv.tc_asc, 0, as, st));
        P->buffer_bytes += (double)(ab + as);
        if (has_parent) {
            const LevelInfo& pv = P->lev[l - 1];
            const size_t pb = sizeof(__half) * (size_t)pv.nbox * nrc * lv.tc_kc2 * 2048;
            const size_t ps = sizeof(float) * (size_t)pv.nbox * nrc * pv.tc_nb * 64;
            HFMM_TRY(plan_alloc(P, (void**)&lv.tc_pmma, pb));
            HFMM_CUDA_TRY(cudaMemsetAsync(lv.tc_pmma, 0, pb, st));
            HFMM_TRY(plan_alloc(P, (void**)&lv.tc_psc, ps));
            HFMM_CUDA_TRY(cudaMemsetAsync(lv.tc_psc, 0, ps, st));
            P->buffer_bytes += (double)(pb + ps);
        }
        if (lv.nv > 0)
            HFMM_TRY(btable(P, lv.t_free32, 49, lv.ncoef, lv.ncoef, Np, lv.tc_kc, &lv.tc_bfree, &lv.tc_sfree, st));
        if (lv.nr > 0 && !(lv.t_react32 && lv.n_react_entries > 0)) {
            hfmm_set_error("tensor-core pass: level %d has reaction pairs but no reaction table", l);
            return HFMM_ERR_UNSUPPORTED;
        }
        if (lv.nr > 0)
            HFMM_TRY(btable(P, lv.t_react32, lv.n_react_entries, lv.ncoef, lv.ncoef, Np, lv.tc_kc, &lv.tc_breact,
                            &lv.tc_sreact, st));
        // level-wide scales: one factor for the free and reaction tables
        const bool runs = lv.tc_runs;
        if (runs) {
            const int na = lv.nv > 0 ? 49 : 0, nr = lv.nr > 0 ? lv.n_react_entries : 0;
            tc_common_scale_kernel<<<1, 256, 0, st>>>(lv.tc_sfree, na, lv.tc_sreact, nr);
            HFMM_CUDA_TRY(cudaGetLastError());
            if (na) tc_btable_kernel<<<4 * 152, 256, 0, st>>>(lv.t_free32, lv.tc_sfree, na, lv.ncoef, lv.ncoef, Np,
                                                               lv.tc_kc, lv.tc_bfree);
            if (nr) tc_btable_kernel<<<4 * 152, 256, 0, st>>>(lv.t_react32, lv.tc_sreact, nr, lv.ncoef, lv.ncoef, Np,
                                                               lv.tc_kc, lv.tc_breact);
            HFMM_CUDA_TRY(cudaGetLastError());
        }
        if (has_parent)
            HFMM_TRY(btable(P, P->lev[l - 1].t_l2l32, 4, npp, lv.ncoef, Np, lv.tc_kc2, &lv.tc_bl2l, &lv.tc_sl2l, st));
        const int sb_own = lv.tc_nbw / 16, sb_par = has_parent ? P->lev[l - 1].tc_nbw / 16 : 1;

        // downward tiles: L2L from the parent, every V-list offset, every reaction entry
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
        const int64_t span = (int64_t)1 << (2 * (L - l));
        auto nonempty = [&](int64_t b) { return lb[(b + 1) * span] > lb[b * span]; };
        std::vector<TcTile> tiles;
        std::vector<TcStep> steps;
        pair_tiles(nbox, nonempty, [&](int32_t b0, int32_t b1) {
            const int c = (int)((b0 >= 0 ? b0 : b1) & 3);
            if (has_parent) push_step(steps, 2, c, b0 >= 0 ? b0 >> 2 : -1, b1 >= 0 ? b1 >> 2 : -1, lv.tc_kc2, sb_par);
            const size_t first = steps.size();   // the tile's free and reaction steps start here
            if (lv.nv) {
                int32_t s0[49], s1[49];
                for (int o = 0; o < 49; ++o) s0[o] = s1[o] = -1;
                if (b0 >= 0) for (int32_t e = vb[b0]; e < vb[b0 + 1]; ++e) s0[vo[e]] = vs[e];
                if (b1 >= 0) for (int32_t e = vb[b1]; e < vb[b1 + 1]; ++e) s1[vo[e]] = vs[e];
                for (int o = 0; o < 49; ++o)
                    if (s0[o] >= 0 || s1[o] >= 0) push_step(steps, 0, o, s0[o], s1[o], lv.tc_kc, sb_own);
            }
            if (lv.nr) {
                // merge the two reaction lists by table entry (dx, ysum)
                std::map<int32_t, std::pair<int32_t, int32_t>> mm;
                if (b0 >= 0) for (int32_t e = rb[b0]; e < rb[b0 + 1]; ++e) mm[rt[e]] = {rs[e], -1};
                if (b1 >= 0) for (int32_t e = rb[b1]; e < rb[b1 + 1]; ++e) {
                    auto it = mm.find(rt[e]);
                    if (it == mm.end()) mm[rt[e]] = {-1, rs[e]};
                    else it->second.second = rs[e];
                }
                for (auto& kv : mm)
                    push_step(steps, 1, kv.first, kv.second.first, kv.second.second, lv.tc_kc, sb_own);
            }
            // one run per K block: consecutive free / reaction steps over the same chunks
            if (runs)
                for (size_t j = first; j + 1 < steps.size(); ++j)
                    steps[j].cont = steps[j].c0 == steps[j + 1].c0 ? 1 : 0;
        }, tiles, steps);
        HFMM_TRY(upload_tiles(P, tiles, steps, &lv.tc_tiles, &lv.tc_steps, &lv.tc_ntiles, &lv.tc_maxsteps));
    }
    // M2M into level l from its children (level l + 1)
    for (int l = P->lmin; l < L; ++l) {
        LevelInfo& lv = P->lev[l];
        const LevelInfo& ch = P->lev[l + 1];
        HFMM_TRY(btable(P, lv.t_m2m32, 4, ch.ncoef, lv.ncoef, lv.tc_np, ch.tc_kc, &lv.tc_bm2m, &lv.tc_sm2m, st));
        // M2M from a level with level-wide scales: one factor for the four shift
        // matrices, so a tile's four children accumulate in TMEM
        const bool mruns = ch.tc_runs;
        if (mruns) {
            tc_common_scale_kernel<<<1, 256, 0, st>>>(lv.tc_sm2m, 4, nullptr, 0);
            tc_btable_kernel<<<4 * 152, 256, 0, st>>>(lv.t_m2m32, lv.tc_sm2m, 4, ch.ncoef, lv.ncoef, lv.tc_np,
                                                      ch.tc_kc, lv.tc_bm2m);
            HFMM_CUDA_TRY(cudaGetLastError());
        }
        const int64_t span = (int64_t)1 << (2 * (L - l)), cspan = span >> 2;
        auto nonempty = [&](int64_t b) { return lb[(b + 1) * span] > lb[b * span]; };
        auto cnonempty = [&](int64_t b) { return lb[(b + 1) * cspan] > lb[b * cspan]; };
        std::vector<TcTile> tiles;
        std::vector<TcStep> steps;
        pair_tiles(lv.nbox, nonempty, [&](int32_t b0, int32_t b1) {
            const size_t first = steps.size();
            for (int c = 0; c < 4; ++c) {
                const int32_t s0 = (b0 >= 0 && cnonempty(4 * (int64_t)b0 + c)) ? 4 * b0 + c : -1;
                const int32_t s1 = (b1 >= 0 && cnonempty(4 * (int64_t)b1 + c)) ? 4 * b1 + c : -1;
                if (s0 >= 0 || s1 >= 0) push_step(steps, 2, c, s0, s1, ch.tc_kc, ch.tc_nbw / 16);
            }
            if (mruns)
                for (size_t j = first; j + 1 < steps.size(); ++j)
                    steps[j].cont = steps[j].c0 == steps[j + 1].c0 ? 1 : 0;
        }, tiles, steps);
        HFMM_TRY(upload_tiles(P, tiles, steps, &lv.tc_mtiles, &lv.tc_msteps, &lv.tc_nmtiles, &lv.tc_mmaxsteps));
    }
    // partial-sum buffer of split launches (largest need over the levels)
    size_t need = 0;
    for (int l = P->lmin; l <= L; ++l) {
        const LevelInfo& lv = P->lev[l];
        const int sd = tc_nseg(lv.tc_ntiles, lv.tc_nb, nrc, lv.tc_maxsteps);
        if (sd > 1) need = std::max(need, (size_t)sd * lv.tc_ntiles * nrc * lv.tc_nb * 128 * lv.tc_nbw);
        const int sm = tc_nseg(lv.tc_nmtiles, lv.tc_nb, nrc, lv.tc_mmaxsteps);
        if (sm > 1) need = std::max(need, (size_t)sm * lv.tc_nmtiles * nrc * lv.tc_nb * 128 * lv.tc_nbw);
    }
    if (need) {
        HFMM_TRY(plan_alloc(P, (void**)&P->tc_part, sizeof(float) * need));
        P->tc_part_floats = need;
        P->buffer_bytes += sizeof(float) * (double)need;
    }
    // the leaves' L2P runs in the downward epilogue when one CTA holds a whole
    // leaf row (one column block, no step split) and its staging fits the ring
    {
        const LevelInfo& lf = P->lev[L];
        P->tc_l2p = lf.tc_nb == 1 && tc_nseg(lf.tc_ntiles, 1, nrc, lf.tc_maxsteps) == 1 && tc_l2p_fits(lf.tc_nbw);
    }
    HFMM_TRY(plan_alloc(P, (void**)&P->tc_err, sizeof(int)));
    HFMM_CUDA_TRY(cudaMemsetAsync(P->tc_err, 0, sizeof(int), st));
    HFMM_TRY(plan_alloc(P, (void**)&P->tc_zero, 4096));
    HFMM_CUDA_TRY(cudaMemsetAsync(P->tc_zero, 0, 4096, st));
    HFMM_CUDA_TRY(cudaStreamSynchronize(st));
    P->tc_on = true;
    return HFMM_OK;
}


// Tensor-core M2M into level l (children at l + 1 already MMA-ready); writes
// the MMA-ready multipoles and, when fp32_out, the FP32 ones (read only by
// the SIMT downward pass).
hfmm_status launch_m2m_tc(hfmm_plan_s* P, int l, int nrhs, bool fp32_out, cudaStream_t st) {
    LevelInfo& lv = P->lev[l];
    const LevelInfo& ch = P->lev[l + 1];
    TcLaunch a{lv.tc_mtiles, lv.tc_msteps, lv.tc_nmtiles, nullptr, nullptr, lv.tc_bm2m, nullptr, nullptr,
               lv.tc_sm2m, nullptr, nullptr, 1, 1, ch.tc_amma, ch.tc_asc, ch.tc_nb, ch.tc_nbw / 16,
               fp32_out ? lv.mult32 : nullptr, lv.ncoef, 0, ch.tc_kc, lv.tc_np, lv.tc_nb, lv.tc_nbw, lv.tc_amma, lv.tc_asc, lv.tc_kc,
               lv.tc_mmaxsteps, false};
    if (lv.tc_runs && l < P->L) {   // this level's multipoles with the level-wide scale
        a.qmax = P->qmax;
        a.qgain = lv.tc_gain;
    }
    return launch_tc(P, a, nrhs, st);
}

// Tensor-core downward pass of level l; writes the FP32 local expansions when
// fp32_out (the leaves, for a separate L2P), below the leaves their MMA-ready
// copy for the children's L2L, and at the leaves, when l2p (P->tc_l2p), adds
// the L2P of every leaf to y32 from the epilogue.
hfmm_status launch_m2l_tc(hfmm_plan_s* P, int l, int nrhs, bool fp32_out, bool l2p, cudaStream_t st) {
    LevelInfo& lv = P->lev[l];
    const bool below = l < P->L;
    const bool has_parent = l > P->lmin;
    const LevelInfo* pv = has_parent ? &P->lev[l - 1] : nullptr;
    TcLaunch a{lv.tc_tiles, lv.tc_steps, lv.tc_ntiles, lv.tc_bfree, lv.tc_breact, lv.tc_bl2l, lv.tc_sfree,
               lv.tc_sreact, lv.tc_sl2l, lv.tc_amma, lv.tc_asc, lv.tc_nb, lv.tc_nbw / 16, lv.tc_pmma, lv.tc_psc,
               pv ? pv->tc_nb : 1, pv ? pv->tc_nbw / 16 : 1, fp32_out ? lv.loc32 : nullptr, lv.ncoef, lv.tc_kc, lv.tc_kc2, lv.tc_np,
               lv.tc_nb, lv.tc_nbw, below ? P->lev[l + 1].tc_pmma : nullptr, below ? P->lev[l + 1].tc_psc : nullptr,
               below ? P->lev[l + 1].tc_kc2 : 0, lv.tc_maxsteps, l2p && l == P->L};
    return launch_tc(P, a, nrhs, st);
}
