// k_tc.cu -- tensor-core distance tiles (tcgen05 + TMA + TMEM, sm_103a).
//
// Gram tiles G = A B^T of BF16 row matrices with FP32 accumulation; the
// norm expansion |a|^2 + |b|^2 - 2<a,b> turns them into squared L2 keys
// (cosine: 1 - <a,b>/(|a||b|)).  Used for the exact join / brute-force scan
// (Sec. 3.2 NLJ): a pair becomes a candidate when its low-precision key is
// below eps_key plus a per-pair rounding bound, and every candidate is
// re-decided from the FP32 vectors (FP64 near eps) by the existing recheck
// kernel, so the result is exact.
//
// Kernel organisation (one CTA per SM, persistent over 128 x 256 output tiles):
//   warp 0      TMA producer: A (128 x 64) and B (256 x 64) BF16 boxes with
//               128-byte swizzle into a 4-stage shared-memory ring;
//   warp 1      allocates 512 TMEM columns (two 256-column FP32 accumulators)
//               and issues tcgen05.mma (M=128, N=256, K=16) from one lane;
//               tcgen05.commit releases ring stages and hands finished
//               accumulators to the epilogue;
//   warps 2-9   epilogue: tcgen05.ld 32 columns at a time from their TMEM lane
//               quarter, key + bound test, candidate append.
// Every mbarrier wait is bounded; on timeout the CTA records an error, stops,
// waits (bounded) for its own copies and MMAs, frees TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <float.h>
#include <stdint.h>

#include <algorithm>
#include <climits>
#include <functional>

#include "vj_device.cuh"
#include "vj_internal.cuh"
#include "vj_tc.cuh"

namespace {

using namespace vjtc;

constexpr int TC_BM = 128, TC_BN = 256, TC_BK = 64, TC_STAGES = 4;
constexpr int TC_EPI_WARPS = 16;
constexpr int TC_CG = TC_EPI_WARPS / 4;    // column groups: warps sharing a TMEM lane quarter
constexpr int TC_CW = TC_BN / TC_CG;       // columns per epilogue warp
constexpr int TC_THREADS = (2 + TC_EPI_WARPS) * 32;
constexpr uint32_t TC_A_BYTES = TC_BM * TC_BK * 2;  // 16 KB
constexpr uint32_t TC_B_BYTES = TC_BN * TC_BK * 2;  // 32 KB
constexpr uint32_t TC_TMEM_COLS = 512;

struct __align__(1024) TcSmem {
    uint8_t A[TC_STAGES][TC_A_BYTES];
    uint8_t B[TC_STAGES][TC_B_BYTES];
    uint64_t full[TC_STAGES];
    uint64_t empty[TC_STAGES];
    uint64_t tfull[2];
    uint64_t tempty[2];
    uint64_t drain;
    uint32_t tmem_base;
    int abort;
    float cn[2][TC_BN];   // column squared norms (L2) / inverse norms (cosine)
    float cnr[2][TC_BN];  // column norms
    __align__(16) float g[2][TC_BN];  // per-column filter thresholds
    uint8_t cvalid[2][TC_BN];
};

// kind::f16 instruction descriptor: FP32 accumulate, BF16 A and B, both
// K-major, M = 128, N = 256
constexpr uint32_t TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TC_BN >> 3) << 17) |
                              ((uint32_t)(TC_BM >> 4) << 24);

struct TcScanParams {
    int64_t nrows, ncols;  // A rows (queries), B rows (data)
    int nkb;               // K blocks of 64
    int nrt, nct;          // row / column tiles
    int metric;
    const float* a_n;      // per A row: squared norm (L2) or inverse norm (cosine)
    const float* b_n;      // per B row: same
    const int32_t* a_ids;  // query index of each A row
    float eps_key;
    float cb, c3;          // candidate bound: key - cb*|a||b| - c3*(|a|^2+|b|^2) < eps_key
    float cbmax;           // cb * (largest row norm): row-independent form of the bound
    int32_t* cq;
    int32_t* cx;
    unsigned long long* ncand;
    int64_t cap;
    int* err;
    long long spin_limit;
};

// MODE 0: exact L2 keys, 1: L2 keys with the BF16 rounding bound, 2: cosine
template <int MODE>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_tc_scan(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tB, TcScanParams P) {
    extern __shared__ uint8_t tc_raw[];
    TcSmem& S = *reinterpret_cast<TcSmem*>((reinterpret_cast<uintptr_t>(tc_raw) + 1023) & ~uintptr_t(1023));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    volatile int* abort = &S.abort;
    const int ntiles = P.nrt * P.nct;

    if (threadIdx.x == 0) {
        for (int s = 0; s < TC_STAGES; s++) {
            mbar_init(&S.full[s], 1);
            mbar_init(&S.empty[s], 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(&S.tfull[b], 1);
            mbar_init(&S.tempty[b], TC_EPI_WARPS);
        }
        mbar_init(&S.drain, 1);
        S.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&S.tmem_base)),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.tmem_base;

    if (warp == 0) {
        // ---------------- TMA producer
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0;
            uint32_t issued = 0, last_ph = 0;  // stages ever filled, parity of their last fill
            bool ok = true;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                const int rt = t % P.nrt, ct = t / P.nrt;
                for (int kb = 0; kb < P.nkb; kb++) {
                    if (!mbar_wait(&S.empty[s], ph ^ 1u, abort, P.spin_limit)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_tx(&S.full[s], TC_A_BYTES + TC_B_BYTES);
                    tma_load_2d(S.A[s], &tA, &S.full[s], kb * TC_BK, rt * TC_BM);
                    tma_load_2d(S.B[s], &tB, &S.full[s], kb * TC_BK, ct * TC_BN);
                    issued |= 1u << s;
                    last_ph = (last_ph & ~(1u << s)) | (ph << s);
                    if (++s == TC_STAGES) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
            }
            if (!ok) {
                *abort = 1;
                atomicExch(P.err, 1);
                // let this CTA's copies land before shared memory goes away
                for (int st = 0; st < TC_STAGES; st++)
                    if ((issued >> st) & 1u) {
                        for (long long i = 0; i < P.spin_limit && !mbar_test(&S.full[st], (last_ph >> st) & 1u);
                             i++) {
                        }
                    }
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0;
            int i = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, i++) {
                const int acc = i & 1;
                if (!mbar_wait(&S.tempty[acc], ((i >> 1) & 1) ^ 1u, abort, P.spin_limit)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(acc * TC_BN);
                for (int kb = 0; kb < P.nkb; kb++) {
                    if (!mbar_wait(&S.full[s], ph, abort, P.spin_limit)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t ad = sdesc_sw128(su32(S.A[s]));
                    const uint64_t bd = sdesc_sw128(su32(S.B[s]));
#pragma unroll
                    for (int kk = 0; kk < TC_BK / 16; kk++) {
                        // advance 16 BF16 (32 bytes) along K inside the swizzled rows
                        tc_mma(d, ad + (uint64_t)(kk * 2), bd + (uint64_t)(kk * 2), TC_IDESC, (kb | kk) != 0);
                    }
                    tc_commit(&S.empty[s]);
                    if (++s == TC_STAGES) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
                if (!ok) break;
                tc_commit(&S.tfull[acc]);
            }
            if (!ok) {
                *abort = 1;
                atomicExch(P.err, 1);
            }
            // all issued MMAs complete before TMEM is released
            tc_commit(&S.drain);
            for (long long k = 0; k < P.spin_limit && !mbar_test(&S.drain, 0); k++) {
            }
        }
    } else {
        // ---------------- epilogue
        const int e = warp - 2;              // 0..TC_EPI_WARPS-1
        const int quarter = warp & 3;        // TMEM lane quarter this warp may access
        const int cg = e >> 2;               // column group
        const int etid = e * 32 + lane;      // threads < TC_BN stage one column each
        // the next tile's column norm and row info are loaded one tile ahead,
        // so their latency overlaps the current tile
        // (cosine rows are unit-normalised: their norms are 1)
        auto col_norm = [&](int tt) -> float {
            const int64_t c = (int64_t)(tt / P.nrt) * TC_BN + etid;
            return (etid < TC_BN && tt < ntiles && c < P.ncols) ? (MODE == 2 ? 1.f : P.b_n[c]) : -1.f;
        };
        auto row_norm = [&](int tt) -> float {
            const int64_t r = (int64_t)(tt % P.nrt) * TC_BM + quarter * 32 + lane;
            return (tt < ntiles && r < P.nrows) ? (MODE == 2 ? 1.f : P.a_n[r]) : -1.f;
        };
        auto row_id = [&](int tt) -> int {
            const int64_t r = (int64_t)(tt % P.nrt) * TC_BM + quarter * 32 + lane;
            return (tt < ntiles && r < P.nrows) ? P.a_ids[r] : -1;
        };
        float nc_next = col_norm(blockIdx.x), rn_next = row_norm(blockIdx.x);
        int qid_next = row_id(blockIdx.x);
        int i = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, i++) {
            const int acc = i & 1;
            const int ct = t / P.nrt;
            // ---- per-tile staging (overlaps the MMA of this tile)
            // filter: a pair can only be a candidate when v - g[c] > h[r]
            //   L2:     v > ((1-c3)(|r|^2 + |c|^2) - eps^2 - cbmax |c|)/2, with
            //           cbmax >= cb |r| for every row (a conservative bound)
            //   cosine: v * cinv > (1 - cb - eps) |r|
            if (etid < TC_BN) {
                const float n = nc_next;
                const bool cvld = n >= 0.f;
                float g;
                if (MODE == 2) g = cvld ? n : 0.f;
                else g = cvld ? 0.5f * ((1.f - P.c3) * n - P.eps_key - P.cbmax * sqrtf(n)) : INFINITY;
                S.g[acc][etid] = g;
                S.cn[acc][etid] = cvld ? n : FLT_MAX;
                S.cnr[acc][etid] = cvld ? (MODE == 2 ? 1.f : sqrtf(n)) : 0.f;
                S.cvalid[acc][etid] = cvld;
            }
            const bool rv = rn_next >= 0.f;
            const float rn = rv ? rn_next : 0.f;
            const int qid = qid_next;
            if (t + (int)gridDim.x < ntiles) {
                nc_next = col_norm(t + gridDim.x);
                rn_next = row_norm(t + gridDim.x);
                qid_next = row_id(t + gridDim.x);
            }
            asm volatile("bar.sync 1, %0;" ::"r"(TC_EPI_WARPS * 32) : "memory");
            const float cbr = MODE == 1 ? P.cb * sqrtf(rn) : 0.f;
            float hr, marg;
            if (MODE == 2) {
                hr = (1.f - P.cb - P.eps_key) * (rn > 0.f ? 1.f / rn : 0.f);
                marg = 1e-5f * (fabsf(hr) + 1.f);
            } else {
                hr = 0.5f * (1.f - P.c3) * rn;
                marg = 1e-5f * (rn + P.eps_key) + 1e-30f;
            }
            const float thr = hr - marg;
            bool ok = mbar_wait(&S.tfull[acc], (i >> 1) & 1, abort, P.spin_limit);
            if (!__all_sync(VJ_FULL, ok)) {
                if (lane == 0) {
                    *abort = 1;
                    atomicExch(P.err, 1);
                }
                break;
            }
            tc_fence_after();
            const float eps_k = P.eps_key;
            const uint32_t tbase = tmem + (uint32_t)(acc * TC_BN + cg * TC_CW) + ((uint32_t)(quarter * 32) << 16);
#pragma unroll 1
            for (int ch = 0; ch < TC_CW / 32; ch++) {
                const int col0 = cg * TC_CW + ch * 32;
                uint32_t va[32];
                tmem_ld32_issue(tbase + (uint32_t)(ch * 32), va);
                tmem_wait_ld(va);
                // fast filter: two instructions per pair, four independent chains
                float m0 = -INFINITY, m1 = -INFINITY, m2 = -INFINITY, m3 = -INFINITY;
                const float4* g4 = reinterpret_cast<const float4*>(&S.g[acc][col0]);
#pragma unroll
                for (int j4 = 0; j4 < 8; j4++) {
                    const float4 g = g4[j4];
                    if (MODE == 2) {
                        m0 = fmaxf(m0, __uint_as_float(va[4 * j4 + 0]) * g.x);
                        m1 = fmaxf(m1, __uint_as_float(va[4 * j4 + 1]) * g.y);
                        m2 = fmaxf(m2, __uint_as_float(va[4 * j4 + 2]) * g.z);
                        m3 = fmaxf(m3, __uint_as_float(va[4 * j4 + 3]) * g.w);
                    } else {
                        m0 = fmaxf(m0, __uint_as_float(va[4 * j4 + 0]) - g.x);
                        m1 = fmaxf(m1, __uint_as_float(va[4 * j4 + 1]) - g.y);
                        m2 = fmaxf(m2, __uint_as_float(va[4 * j4 + 2]) - g.z);
                        m3 = fmaxf(m3, __uint_as_float(va[4 * j4 + 3]) - g.w);
                    }
                }
                const bool maybe = rv && fmaxf(fmaxf(m0, m1), fmaxf(m2, m3)) > thr;
                if (!__any_sync(VJ_FULL, maybe)) continue;
                uint32_t hit = 0;
                if (maybe) {
                    // exact candidate test for this row's 32 columns (unrolled:
                    // the TMEM registers must stay registers)
#pragma unroll
                    for (int j = 0; j < 32; j++) {
                        const float v = __uint_as_float(va[j]);
                        const float cn = S.cn[acc][col0 + j];
                        bool h;
                        if (MODE == 0) {
                            h = fmaf(-2.f, v, rn + cn) < eps_k;
                        } else if (MODE == 1) {
                            const float t = rn + cn;
                            h = fmaf(-2.f, v, t) - fmaf(cbr, S.cnr[acc][col0 + j], P.c3 * t) < eps_k;
                        } else {
                            h = 1.f - v * rn * cn - P.cb < eps_k;
                        }
                        if (h && S.cvalid[acc][col0 + j]) hit |= 1u << j;
                    }
                }
                // warp-aggregated append: one atomic per warp and chunk
                const int mine = __popc(hit);
                int incl = mine;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    int t2 = __shfl_up_sync(VJ_FULL, incl, o);
                    if (lane >= o) incl += t2;
                }
                const int total = __shfl_sync(VJ_FULL, incl, 31);
                if (total > 0) {
                    unsigned long long base = 0;
                    if (lane == 31) base = atomicAdd(P.ncand, (unsigned long long)total);
                    base = __shfl_sync(VJ_FULL, base, 31);
                    unsigned long long gq = base + (unsigned long long)(incl - mine);
                    while (hit) {
                        const int j = __ffs(hit) - 1;
                        hit &= hit - 1;
                        if ((int64_t)gq < P.cap) {
                            P.cq[gq] = qid;
                            P.cx[gq] = (int)((int64_t)ct * TC_BN + col0 + j);
                        }
                        gq++;
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&S.tempty[acc]);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS)
                     : "memory");
    }
}

// ---------------------------------------------------------------- resident-A scan
// For kp <= 128 a CTA keeps 256 query rows (two 128-row MMA operands, every
// k-block) in shared memory for a run of 128-row data tiles, so only the data
// side crosses L2 per tile (K = 128: 36 KB per 8.4 MFLOP instead of 96 KB).
// The per-column part of the candidate test rides in the GEMM: after the data
// k-blocks comes one K=16 bias step whose A side holds (1, 1, 1, 0, ...) and
// whose data side holds a three-term BF16 split of the column bias (16-column
// boxes with 32-byte swizzle), so the accumulator is 2<a,b> + bias_c and the
// epilogue is a row-wise max against one threshold per query row (one FMNMX
// per pair).  A ring stage holds one whole data tile.
constexpr int RS_BN = 128;                     // data rows per tile (MMA N)
constexpr int RS_EPI = 16;                     // epilogue warps
constexpr int RS_THREADS = (2 + RS_EPI) * 32;
constexpr uint32_t RS_BOX = 128 * 64 * 2;      // one 128-row x 64-column BF16 box
constexpr uint32_t RS_BBOX = 128 * 16 * 2;     // one 128-row x 16-column BF16 bias box
constexpr int RS_MAX_KB = 2;                   // data k-blocks (kp <= 128)
constexpr int RS_MAX_STAGES = 8;
// Candidates are appended through per-warp chunks of the output: one global
// atomic reserves RS_CHUNK slots (more if one append needs more), and the
// slots a warp leaves unused are holes (query index -1).  A counter shared by
// every warp of the grid made same-address atomics the bottleneck once the
// scanned rows had about a hundred pairs each.
constexpr int RS_CHUNK = 128;
// room for holes when a list is sized from a previous launch's count: a
// part-filled chunk per epilogue warp at the end (RS_EPI warps per CTA, one CTA
// per SM, up to 256 SMs); the chunk switches add a quarter of the count on top
constexpr int64_t RS_HOLE_SLACK = (int64_t)RS_CHUNK * 16 * 256;
constexpr uint32_t RS_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(RS_BN >> 3) << 17) |
                              ((uint32_t)(128 >> 4) << 24);

struct RsBars {
    uint64_t full[RS_MAX_STAGES];
    uint64_t empty[RS_MAX_STAGES];
    uint64_t tfull[2];
    uint64_t tempty[2];
    uint64_t afull;   // the unit's query rows have landed
    uint64_t aempty;  // the unit's MMAs are done (query rows may be replaced)
    uint64_t abar;    // the A-side bias block has landed
    uint64_t drain;
    uint32_t tmem_base;
    int abort;
};
static_assert(sizeof(RsBars) <= 1024, "barrier block");

struct RsParams {
    int64_t nrows, ncols;
    int nkb;     // data k-blocks (kp / 64)
    int bias;    // 1: a bias k-block follows the data k-blocks (L2)
    int nrp;     // 256-row query blocks
    int nct;     // data tiles
    int tpu;     // data tiles per work unit
    int nunits;  // nrp * ceil(nct / tpu), query block fastest
    int stages;
    const float* a_thr;    // per query row: candidate iff accumulator > a_thr
    const int32_t* a_ids;  // query index of each row
    const float* a_rn;     // per query row |a|^2, when keys are written
    float* ck;             // exact-key inputs: the candidate's key |a|^2 - accumulator (nullptr: none)
    int32_t* cq;
    int32_t* cx;
    unsigned long long* ncand;
    int64_t cap;
    int* err;
    long long spin_limit;
    int tstride;          // data tile t of a unit is tile t * tstride (1: every tile)
    // sample epilogue: the rows' node ids equal their row index
    float* top16;         // [nrows] 16th largest accumulator over the sampled tiles (other nodes)
};

constexpr int KN_EPI = 8;  // sample epilogue warps: one per (query block, lane quarter)

// Resident-query tensor-core kernel with two epilogues:
//   EPI_SCAN    16 warps; a pair is a candidate when its accumulator exceeds
//               the row's threshold (the brute-force route, the exact join and
//               the kNN build's candidate sweep);
//   EPI_SAMPLE   8 warps; each thread owns one row and keeps, in registers, the
//               16 largest accumulators over a sample of the data tiles (the
//               kNN build's per-row threshold).
enum { EPI_SCAN = 0, EPI_SAMPLE = 1 };

template <int EPI>
__global__ void __launch_bounds__((2 + (EPI == EPI_SAMPLE ? KN_EPI : RS_EPI)) * 32, 1)
    k_tc_res(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tAb,
             const __grid_constant__ CUtensorMap tB, const __grid_constant__ CUtensorMap tBb, RsParams P) {
    constexpr int NEPI = EPI == EPI_SAMPLE ? KN_EPI : RS_EPI;
    extern __shared__ uint8_t rs_raw[];
    uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(rs_raw) + 1023) & ~uintptr_t(1023));
    RsBars& Bb = *reinterpret_cast<RsBars*>(base);
    // bias boxes first: a misread descriptor could only reach later tiles
    uint8_t* sAb = base + 1024;                          // query-side bias box
    uint8_t* sBb = sAb + RS_BBOX;                        // [stages] data bias boxes
    uint8_t* sA = sBb + P.stages * RS_BBOX;              // [2][nkb] query boxes
    uint8_t* sB = sA + 2 * P.nkb * RS_BOX;               // [stages][nkb] data boxes
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    volatile int* abort = &Bb.abort;
    const uint32_t stage_tx = (uint32_t)P.nkb * RS_BOX + (P.bias ? RS_BBOX : 0u);

    if (threadIdx.x == 0) {
        for (int s = 0; s < P.stages; s++) {
            mbar_init(&Bb.full[s], 1);
            mbar_init(&Bb.empty[s], 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(&Bb.tfull[b], 1);
            mbar_init(&Bb.tempty[b], NEPI);
        }
        mbar_init(&Bb.afull, 1);
        mbar_init(&Bb.aempty, 1);
        mbar_init(&Bb.abar, 1);
        mbar_init(&Bb.drain, 1);
        Bb.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&Bb.tmem_base)),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = Bb.tmem_base;

    if (warp == 0) {
        // ---------------- TMA producer
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0;
            uint32_t issued = 0, last_ph = 0;  // ring stages ever filled, parity of their last fill
            int a_units = 0;                   // query blocks loaded so far
            bool ok = true;
            if (P.bias) {
                mbar_arrive_tx(&Bb.abar, RS_BBOX);
                tma_load_2d(sAb, &tAb, &Bb.abar, 0, 0);
            }
            for (int u = blockIdx.x; u < P.nunits && ok; u += gridDim.x) {
                const int rp = u % P.nrp, cc = u / P.nrp;
                const int t0 = cc * P.tpu, t1 = min(P.nct, t0 + P.tpu);
                if (a_units > 0 && !mbar_wait(&Bb.aempty, (uint32_t)((a_units - 1) & 1), abort, P.spin_limit)) {
                    ok = false;
                    break;
                }
                mbar_arrive_tx(&Bb.afull, 2u * (uint32_t)P.nkb * RS_BOX);
                for (int blk = 0; blk < 2; blk++)
                    for (int kb = 0; kb < P.nkb; kb++)
                        tma_load_2d(sA + (blk * P.nkb + kb) * RS_BOX, &tA, &Bb.afull, kb * 64, rp * 256 + blk * 128);
                a_units++;
                for (int ct = t0; ct < t1; ct++) {
                    if (!mbar_wait(&Bb.empty[s], ph ^ 1u, abort, P.spin_limit)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_tx(&Bb.full[s], stage_tx);
                    for (int kb = 0; kb < P.nkb; kb++)
                        tma_load_2d(sB + (s * P.nkb + kb) * RS_BOX, &tB, &Bb.full[s], kb * 64,
                                    ct * P.tstride * RS_BN);
                    if (P.bias) tma_load_2d(sBb + s * RS_BBOX, &tBb, &Bb.full[s], 0, ct * P.tstride * RS_BN);
                    issued |= 1u << s;
                    last_ph = (last_ph & ~(1u << s)) | (ph << s);
                    if (++s == P.stages) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
            }
            if (!ok) {
                *abort = 1;
                atomicExch(P.err, 1);
                // let this CTA's copies land before shared memory goes away
                for (int st = 0; st < P.stages; st++)
                    if ((issued >> st) & 1u)
                        for (long long i = 0; i < P.spin_limit && !mbar_test(&Bb.full[st], (last_ph >> st) & 1u); i++) {
                        }
                if (a_units > 0)
                    for (long long i = 0; i < P.spin_limit && !mbar_test(&Bb.afull, (uint32_t)((a_units - 1) & 1));
                         i++) {
                    }
                if (P.bias)
                    for (long long i = 0; i < P.spin_limit && !mbar_test(&Bb.abar, 0); i++) {
                    }
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer: D0 += A0 B^T, D1 += A1 B^T per k-step
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0;
            int i = 0, j = 0;
            bool ok = !P.bias || mbar_wait(&Bb.abar, 0, abort, P.spin_limit);
            const uint64_t abd = sdesc_sw32(su32(sAb));
            for (int u = blockIdx.x; u < P.nunits && ok; u += gridDim.x, j++) {
                const int cc = u / P.nrp;
                const int t0 = cc * P.tpu, t1 = min(P.nct, t0 + P.tpu);
                if (!mbar_wait(&Bb.afull, (uint32_t)(j & 1), abort, P.spin_limit)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                for (int ct = t0; ct < t1 && ok; ct++, i++) {
                    const int acc = i & 1;
                    if (!mbar_wait(&Bb.tempty[acc], (uint32_t)(((i >> 1) & 1) ^ 1), abort, P.spin_limit)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d0 = tmem + (uint32_t)(acc * 256), d1 = d0 + 128u;
                    if (!mbar_wait(&Bb.full[s], ph, abort, P.spin_limit)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    for (int kb = 0; kb < P.nkb; kb++) {
                        const uint64_t bd = sdesc_sw128(su32(sB + (s * P.nkb + kb) * RS_BOX));
                        const uint64_t a0 = sdesc_sw128(su32(sA + kb * RS_BOX));
                        const uint64_t a1 = sdesc_sw128(su32(sA + (P.nkb + kb) * RS_BOX));
#pragma unroll
                        for (int kk = 0; kk < 4; kk++) {
                            // advance 16 BF16 (32 bytes) along K inside the swizzled rows
                            const uint32_t accf = (kb | kk) != 0;
                            tc_mma(d0, a0 + (uint64_t)(kk * 2), bd + (uint64_t)(kk * 2), RS_IDESC, accf);
                            tc_mma(d1, a1 + (uint64_t)(kk * 2), bd + (uint64_t)(kk * 2), RS_IDESC, accf);
                        }
                    }
                    if (P.bias) {
                        // the bias step: K = 16 columns holding the three bias terms
                        const uint64_t bbd = sdesc_sw32(su32(sBb + s * RS_BBOX));
                        tc_mma(d0, abd, bbd, RS_IDESC, 1u);
                        tc_mma(d1, abd, bbd, RS_IDESC, 1u);
                    }
                    tc_commit(&Bb.empty[s]);
                    if (++s == P.stages) {
                        s = 0;
                        ph ^= 1u;
                    }
                    tc_commit(&Bb.tfull[acc]);
                }
                if (!ok) break;
                tc_commit(&Bb.aempty);  // the query rows may be replaced once these MMAs finish
            }
            if (!ok) {
                *abort = 1;
                atomicExch(P.err, 1);
            }
            tc_commit(&Bb.drain);
            for (long long k = 0; k < P.spin_limit && !mbar_test(&Bb.drain, 0); k++) {
            }
        }
    } else if constexpr (EPI == EPI_SAMPLE) {
        // ---------------- sample epilogue: warp e owns TMEM lane quarter (warp & 3)
        // of query block e >> 2, all 128 columns; lane = one row.  t[] holds
        // the row's 16 largest accumulators so far, descending (static
        // indices only: the array stays in registers).
        const int e = warp - 2;
        const int quarter = warp & 3;
        const int blk = e >> 2;
        const uint32_t lanes = (uint32_t)(quarter * 32) << 16;
        int i = 0;
        bool ok = true;
        for (int u = blockIdx.x; u < P.nunits && ok; u += gridDim.x) {
            const int rp = u % P.nrp, cc = u / P.nrp;
            const int t0 = cc * P.tpu, t1 = min(P.nct, t0 + P.tpu);
            const int64_t r = (int64_t)rp * 256 + blk * 128 + quarter * 32 + lane;
            const bool rv = r < P.nrows;
            float t[16];
#pragma unroll
            for (int k = 0; k < 16; k++) t[k] = -INFINITY;
            for (int ct = t0; ct < t1; ct++, i++) {
                const int acc = i & 1;
                const bool got = mbar_wait(&Bb.tfull[acc], (uint32_t)((i >> 1) & 1), abort, P.spin_limit);
                if (!__all_sync(VJ_FULL, got)) {
                    if (lane == 0) {
                        *abort = 1;
                        atomicExch(P.err, 1);
                    }
                    ok = false;
                    break;
                }
                tc_fence_after();
#pragma unroll 1
                for (int h = 0; h < 2; h++) {
                    uint32_t va[64];
                    tmem_ld64_issue(tmem + lanes + (uint32_t)(acc * 256 + blk * 128 + h * 64), va);
                    tmem_wait_ld64(va);
                    if (h == 1) {
                        // both halves are in registers: hand the TMEM buffer back
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&Bb.tempty[acc]);
                    }
                    if (!rv) continue;
                    const int64_t c0 = (int64_t)ct * P.tstride * RS_BN + h * 64;
                    float m0 = -INFINITY, m1 = -INFINITY, m2 = -INFINITY, m3 = -INFINITY;
#pragma unroll
                    for (int j = 0; j < 64; j += 4) {
                        m0 = fmaxf(m0, __uint_as_float(va[j + 0]));
                        m1 = fmaxf(m1, __uint_as_float(va[j + 1]));
                        m2 = fmaxf(m2, __uint_as_float(va[j + 2]));
                        m3 = fmaxf(m3, __uint_as_float(va[j + 3]));
                    }
                    if (fmaxf(fmaxf(m0, m1), fmaxf(m2, m3)) <= t[15]) continue;
                    const bool edge = c0 + 64 > P.ncols || (r >= c0 && r < c0 + 64);
#pragma unroll
                    for (int j = 0; j < 64; j++) {
                        float x = __uint_as_float(va[j]);
                        if (x <= t[15]) continue;
                        if (edge && (c0 + j >= P.ncols || c0 + j == r)) continue;
                        // insert: x sinks to its place, the 16th value drops out
#pragma unroll
                        for (int k = 0; k < 16; k++) {
                            const float hi = fmaxf(t[k], x);
                            x = fminf(t[k], x);
                            t[k] = hi;
                        }
                    }
                }
            }
            if (ok && rv) P.top16[r] = t[15];
        }
    } else {
        // ---------------- epilogue: warp e reads TMEM lane quarter (warp & 3),
        // 64 of the 256 accumulator columns: query block cg >> 1, half cg & 1
        const int e = warp - 2;
        const int quarter = warp & 3;
        const int cg = e >> 2;
        const int blk = cg >> 1, csub = cg & 1;
        int i = 0;
        bool ok = true;
        unsigned long long cbase = 0;  // this warp's output chunk: next slot, slots left
        int cleft = 0;
        for (int u = blockIdx.x; u < P.nunits && ok; u += gridDim.x) {
            const int rp = u % P.nrp, cc = u / P.nrp;
            const int t0 = cc * P.tpu, t1 = min(P.nct, t0 + P.tpu);
            const int64_t r = (int64_t)rp * 256 + blk * 128 + quarter * 32 + lane;
            const float thr = r < P.nrows ? P.a_thr[r] : INFINITY;
            const int qid = r < P.nrows ? P.a_ids[r] : -1;
            const float rnk = (P.ck && r < P.nrows) ? P.a_rn[r] : 0.f;
            for (int ct = t0; ct < t1; ct++, i++) {
                const int acc = i & 1;
                const bool got = mbar_wait(&Bb.tfull[acc], (uint32_t)((i >> 1) & 1), abort, P.spin_limit);
                if (!__all_sync(VJ_FULL, got)) {
                    if (lane == 0) {
                        *abort = 1;
                        atomicExch(P.err, 1);
                    }
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t taddr = tmem + (uint32_t)(acc * 256 + blk * 128 + csub * 64) +
                                       ((uint32_t)(quarter * 32) << 16);
                uint32_t va[64];
                tmem_ld64_issue(taddr, va);
                tmem_wait_ld64(va);
                // the accumulator is in registers: hand the TMEM buffer back now
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&Bb.tempty[acc]);
                float m0 = -INFINITY, m1 = -INFINITY, m2 = -INFINITY, m3 = -INFINITY;
#pragma unroll
                for (int j = 0; j < 64; j += 4) {
                    m0 = fmaxf(m0, __uint_as_float(va[j + 0]));
                    m1 = fmaxf(m1, __uint_as_float(va[j + 1]));
                    m2 = fmaxf(m2, __uint_as_float(va[j + 2]));
                    m3 = fmaxf(m3, __uint_as_float(va[j + 3]));
                }
                const bool maybe = fmaxf(fmaxf(m0, m1), fmaxf(m2, m3)) > thr;
                if (__any_sync(VJ_FULL, maybe)) {
                    const int64_t c0 = (int64_t)ct * P.tstride * RS_BN + csub * 64;
                    // columns past the last data row (last tile only), as masks of each half
                    const int64_t room = P.ncols - c0;
                    const uint32_t cm0 = room >= 32 ? ~0u : (room <= 0 ? 0u : ((1u << room) - 1u));
                    const uint32_t cm1 = room >= 64 ? ~0u : (room <= 32 ? 0u : ((1u << (room - 32)) - 1u));
                    uint32_t hit0 = 0, hit1 = 0;
                    if (maybe) {
#pragma unroll
                        for (int j = 0; j < 32; j++) {
                            hit0 |= (uint32_t)(__uint_as_float(va[j]) > thr) << j;
                            hit1 |= (uint32_t)(__uint_as_float(va[32 + j]) > thr) << j;
                        }
                        hit0 &= cm0;
                        hit1 &= cm1;
                    }
                    // warp-aggregated append of both halves
                    const int mine = __popc(hit0) + __popc(hit1);
                    int incl = mine;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int t2 = __shfl_up_sync(VJ_FULL, incl, o);
                        if (lane >= o) incl += t2;
                    }
                    const int total = __shfl_sync(VJ_FULL, incl, 31);
                    if (total > 0) {
                        if (total > cleft) {
                            // close the chunk (its unused slots become holes) and
                            // reserve the next one
                            for (int k = lane; k < cleft; k += 32)
                                if ((int64_t)(cbase + k) < P.cap) P.cq[cbase + k] = -1;
                            const int want = max(total, RS_CHUNK);
                            unsigned long long gb = 0;
                            if (lane == 31) gb = atomicAdd(P.ncand, (unsigned long long)want);
                            cbase = __shfl_sync(VJ_FULL, gb, 31);
                            cleft = want;
                        }
                        unsigned long long gq = cbase + (unsigned long long)(incl - mine);
                        cbase += (unsigned long long)total;
                        cleft -= total;
#pragma unroll
                        for (int h = 0; h < 2; h++) {
                            uint32_t hit = h ? hit1 : hit0;
                            while (hit) {
                                const int j = __ffs(hit) - 1;
                                hit &= hit - 1;
                                if ((int64_t)gq < P.cap) {
                                    P.cq[gq] = qid;
                                    P.cx[gq] = (int)(c0 + h * 32 + j);
                                    // integer inputs: the accumulator 2<a,b> - |b|^2 is exact.
                                    // (select by unrolled compares: a runtime index into va
                                    // would move the whole array to local memory)
                                    if (P.ck) {
                                        float o = 0.f;
#pragma unroll
                                        for (int jj = 0; jj < 32; jj++)
                                            if (jj == j) o = __uint_as_float(va[h * 32 + jj]);
                                        P.ck[gq] = rnk - o;
                                    }
                                }
                                gq++;
                            }
                        }
                    }
                }
            }
        }
        for (int k = lane; k < cleft; k += 32)
            if ((int64_t)(cbase + k) < P.cap) P.cq[cbase + k] = -1;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS)
                     : "memory");
    }
}

// FP32 rows (optionally gathered) -> BF16 rows of kp columns, zero padded,
// each row scaled by `scale` (times rscale[src] when given)
__global__ void k_to_bf16(const float* __restrict__ vec, int dp, int d, const int32_t* __restrict__ rows,
                          int64_t row0, int64_t nrows, int kp, float scale, const float* __restrict__ rscale,
                          __nv_bfloat16* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nrows * kp) return;
    const int64_t r = i / kp;
    const int k = (int)(i % kp);
    const int64_t src = rows ? (int64_t)rows[r] : row0 + r;
    const float sc = rscale ? scale * rscale[src] : scale;
    out[i] = __float2bfloat16_rn(k < d ? vec[src * dp + k] * sc : 0.f);
}

// L2 scan bias of data row c, bias_c = -(1 - c3) |c|^2 + cbmax |c| (FP64),
// stored as hi + mid + lo BF16 terms in columns 0..2 of a 16-column row
__global__ void k_bias_split(const float* __restrict__ sqn, int64_t nx, double c3, double cbmax,
                             __nv_bfloat16* __restrict__ out) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nx) return;
    const double n = (double)sqn[c];
    double b = -(1.0 - c3) * n + cbmax * sqrt(n);
    __nv_bfloat16 t[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        t[k] = __double2bfloat16(b);
        b -= (double)__bfloat162float(t[k]);
    }
    __nv_bfloat16* o = out + c * 16;
#pragma unroll
    for (int k = 0; k < 16; k++) o[k] = k < 3 ? t[k] : __float2bfloat16_rn(0.f);
}

__global__ void k_fill_abias(__nv_bfloat16* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 128 * 16) out[i] = __float2bfloat16_rn((i & 15) < 3 ? 1.f : 0.f);
}

// per scanned query row: the accumulator threshold of the resident-A scan.
//   L2:     2<a',b'> + bias_c > (1 - c3)|a|^2 - eps^2 - margin
//   cosine: <a',b'> > 1 - eps - cb - margin   (unit rows)
// margin covers the FP32 accumulation of the kp + 3 products and the BF16
// split of the bias, (kp + 16) 2^-23 times the sum of their magnitudes
__global__ void k_row_thr(const float* __restrict__ sqn, const int32_t* __restrict__ node, int64_t n, int metric,
                          int kp, float eps_key, float cb, float c3, float cbmax, double maxnorm,
                          float* __restrict__ thr) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double g = (double)(kp + 16) * 1.1920928955078125e-7;
    if (metric == 0) {
        const double rn = (double)sqn[node[i]];
        const double mag = 2.1 * sqrt(rn) * maxnorm + 1.1 * maxnorm * maxnorm + (double)cbmax * maxnorm;
        thr[i] = (float)((1.0 - (double)c3) * rn - (double)eps_key - g * mag - 1e-30);
    } else {
        thr[i] = (float)(1.0 - (double)eps_key - (double)cb - 3.0 * g);
    }
}

__global__ void k_gather_f(const float* __restrict__ src, const int32_t* __restrict__ rows, int64_t n,
                           float* __restrict__ dst) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[rows[i]];
}

// flag[0] |= any non-integer coordinate; flag[1] = max |coordinate| (integer part)
__global__ void k_int_check(const float* __restrict__ v, int64_t n, unsigned int* __restrict__ flag) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float x = v[i];
    const bool nonint = !(x == rintf(x)) || fabsf(x) > 1e9f;
    if (__any_sync(__activemask(), nonint) && nonint) atomicOr(flag, 1u);
    const unsigned int m = (unsigned int)fminf(fabsf(x), 4e9f);
    atomicMax(flag + 1, m);
}

// query index and merged node id of each scanned row
__global__ void k_query_rows(const int32_t* __restrict__ qrows, int64_t n, int32_t nx, int32_t* __restrict__ qid,
                             int32_t* __restrict__ node) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t q = qrows ? qrows[i] : (int32_t)i;
    qid[i] = q;
    node[i] = nx + q;
}

}  // namespace

// BF16 copy of the data rows and the scan's bound constants (built once per
// index, kept for later scans).  Cosine rows are stored unit-normalised.
static void ensure_data_bf16(vj_index* ix) {
    const int kp = (ix->d + TC_BK - 1) / TC_BK * TC_BK;
    if (ix->xbf.n >= (size_t)ix->n * kp) return;
    cudaStream_t s = ix->stream;
    // every node (data rows first): scans read the data rows, the kNN build all
    ix->xbf.ensure((size_t)ix->n * kp, s);
    const bool cosine = ix->metric != VJ_L2;
    k_to_bf16<<<vj_div_up(ix->n * kp, 256), 256, 0, s>>>(ix->vec.p, ix->dp, ix->d, nullptr, 0, ix->n, kp, 1.f,
                                                          cosine ? ix->invn.p : nullptr, ix->xbf.p);
    VJ_LAUNCH_CHECK();
    // Exact-key test: when every coordinate is an integer of magnitude <= 256
    // it is exact in BF16, every product is an integer below 2^16 and, with
    // d * max^2 <= 2^23, every partial sum, both norms, their sum (<= 2^24)
    // and the norm expansion stay integers exactly representable in FP32, so
    // the FP32-accumulated key is exact and needs no bound.
    DBuf<unsigned int> flag;
    flag.alloc(2, s);
    VJ_CUDA(cudaMemsetAsync(flag.p, 0, 2 * sizeof(unsigned int), s));
    k_int_check<<<vj_div_up(ix->n * ix->dp, 256), 256, 0, s>>>(ix->vec.p, ix->n * ix->dp, flag.p);
    VJ_LAUNCH_CHECK();
    unsigned int h[2] = {0, 0};
    VJ_CUDA(cudaMemcpyAsync(h, flag.p, sizeof(h), cudaMemcpyDeviceToHost, s));
    VJ_CUDA(cudaStreamSynchronize(s));
    flag.free_(s);
    const double mx = (double)h[1];
    ix->bf16_exact = !cosine && h[0] == 0 && mx <= 256.0 && (double)ix->d * mx * mx <= 8388608.0;
    // |key_bf16 - key| <= cb |a||b| + c3 (|a|^2 + |b|^2) with
    //   L2:     cb = 4ub + 2ub^2 + 2 kp 2^-23 + 4u, c3 = 3u
    //   cosine: cb = 2ub + ub^2 + 2 kp 2^-23 + 8u (unit rows), c3 = 0
    // (ub = 2^-8 BF16, u = 2^-24 FP32), each with a 1.25 margin
    const double ub = 1.0 / 256.0, u = VJ_F32_U;
    if (!cosine) {
        ix->tc_cb = (float)(1.25 * (4 * ub + 2 * ub * ub + 2.0 * kp * 2 * u + 4 * u));
        ix->tc_c3 = (float)(1.25 * 3 * u);
        if (ix->bf16_exact) {
            ix->tc_cb = 0.f;  // exact integer keys (see above)
            ix->tc_c3 = 0.f;
        }
        // row-independent form: cbmax >= cb |a| for every row
        ix->tc_cbmax = (float)(ix->tc_cb * ix->maxnorm * 1.0001);
        ix->xbias.ensure((size_t)ix->n * 16, s);
        k_bias_split<<<vj_div_up(ix->n, 256), 256, 0, s>>>(ix->sqn.p, ix->n, (double)ix->tc_c3,
                                                             (double)ix->tc_cbmax, ix->xbias.p);
        VJ_LAUNCH_CHECK();
        ix->abias.ensure(128 * 16, s);
        k_fill_abias<<<vj_div_up(128 * 16, 256), 256, 0, s>>>(ix->abias.p);
        VJ_LAUNCH_CHECK();
    } else {
        ix->tc_cb = (float)(1.25 * (2 * ub + ub * ub + 2.0 * kp * 2 * u + 8 * u));
        ix->tc_c3 = 0.f;
        ix->tc_cbmax = 0.f;
    }
}

// Candidate pairs (query index, data id) of the BF16 tensor-core scan of the
// queries `qrows` (query indices; nullptr = all) against every data row.
// Returns the candidate count (the arrays are grown and the scan re-run when
// they are too small).
int64_t vj_tc_scan_candidates(vj_index* ix, const int32_t* qrows, int64_t nr, float eps, DBuf<int32_t>& cq,
                              DBuf<int32_t>& cx, double* ms_out, DBuf<float>* ck) {
    cudaStream_t s = ix->stream;
    const int kp = (ix->d + TC_BK - 1) / TC_BK * TC_BK;
    ensure_data_bf16(ix);
    const bool cosine = ix->metric != VJ_L2;
    // kp <= 128: resident query rows and the bias step; wider rows stream
    // both operands through the ring
    const bool resident = kp <= RS_MAX_KB * TC_BK;
    DBuf<__nv_bfloat16> abf;
    DBuf<int32_t> aid, anode;
    DBuf<float> an;
    abf.alloc((size_t)nr * kp, s);
    aid.alloc(nr, s);
    anode.alloc(nr, s);
    an.alloc(nr, s);
    k_query_rows<<<vj_div_up(nr, 256), 256, 0, s>>>(qrows, nr, (int32_t)ix->nx, aid.p, anode.p);
    VJ_LAUNCH_CHECK();
    const int32_t* arow = anode.p;
    // query rows: L2 scaled by 2 for the resident form (2<a,b> + bias), cosine unit rows
    const float ascale = (!cosine && resident) ? 2.f : 1.f;
    k_to_bf16<<<vj_div_up(nr * kp, 256), 256, 0, s>>>(ix->vec.p, ix->dp, ix->d, arow, 0, nr, kp, ascale,
                                                      cosine ? ix->invn.p : nullptr, abf.p);
    VJ_LAUNCH_CHECK();
    const float eps_key = cosine ? eps : eps * eps;
    if (resident) {
        k_row_thr<<<vj_div_up(nr, 256), 256, 0, s>>>(ix->sqn.p, arow, nr, ix->metric, kp, eps_key, ix->tc_cb,
                                                      ix->tc_c3, ix->tc_cbmax, ix->maxnorm, an.p);
    } else {
        k_gather_f<<<vj_div_up(nr, 256), 256, 0, s>>>(ix->sqn.p, arow, nr, an.p);
    }
    VJ_LAUNCH_CHECK();

    DBuf<unsigned long long> ctr;
    DBuf<int> err;
    DBuf<float> rn_rows;
    ctr.alloc(1, s);
    err.alloc(1, s);
    const long long spin_limit = 1ll << 22;  // try_wait polls; seconds at most, then an error
    std::function<void()> launch;
    CUtensorMap ta, tb, tab, tbb;
    RsParams R{};
    TcScanParams P{};
    if (resident) {
        ta = make_map(abf.p, nr, kp, 128);
        tb = make_map(ix->xbf.p, ix->nx, kp, RS_BN);
        if (!cosine) {
            tab = make_map16(ix->abias.p, 128, 128);
            tbb = make_map16(ix->xbias.p, ix->nx, RS_BN);
        } else {
            tab = ta;  // unused without the bias block
            tbb = tb;
        }
        R.nrows = nr;
        R.ncols = ix->nx;
        R.nkb = kp / TC_BK;
        R.bias = cosine ? 0 : 1;
        R.nrp = (int)vj_div_up(nr, 256);
        R.nct = (int)vj_div_up(ix->nx, RS_BN);
        // work units: a 256-row query block x a run of data tiles; units run
        // query block fastest so concurrent units share data tiles in L2.
        // The run length minimises the busiest SM's load: its units' tiles
        // plus about 3 tiles of pipeline refill per unit (query rows reload)
        {
            const int64_t g = std::max(1, ix->num_sms);
            int64_t best = INT64_MAX;
            int best_tpu = R.nct;
            for (int64_t ncc = 1; ncc <= R.nct; ncc++) {
                const int64_t tpu = (R.nct + ncc - 1) / ncc;
                if (ncc > 1 && (R.nct + tpu - 1) / tpu != ncc) continue;  // same split as a smaller ncc
                const int64_t per = ((int64_t)R.nrp * ncc + g - 1) / g;
                const int64_t load = per * (tpu + 3);
                if (load < best) {
                    best = load;
                    best_tpu = (int)tpu;
                }
            }
            R.tpu = best_tpu;
        }
        R.nunits = R.nrp * (int)vj_div_up(R.nct, R.tpu);
        // ring stages of one data tile each, within 227 KB of shared memory
        const size_t fixed = 2048 + RS_BBOX + 2 * (size_t)R.nkb * RS_BOX;
        const size_t per = (size_t)R.nkb * RS_BOX + RS_BBOX;
        R.stages = (int)std::min<size_t>(RS_MAX_STAGES, (232448 - fixed) / per);
        R.a_thr = an.p;
        R.a_ids = aid.p;
        R.tstride = 1;
        // integer inputs (exact BF16 products and FP32 sums): the scan hands out
        // each candidate's exact key, and no re-check from the vectors is needed
        if (ck && !cosine && ix->bf16_exact) {
            rn_rows.alloc(nr, s);
            k_gather_f<<<vj_div_up(nr, 256), 256, 0, s>>>(ix->sqn.p, arow, nr, rn_rows.p);
            VJ_LAUNCH_CHECK();
            R.a_rn = rn_rows.p;
        }
        R.ncand = ctr.p;
        R.err = err.p;
        R.spin_limit = spin_limit;
        const size_t smem = fixed + per * (size_t)R.stages;
        VJ_CUDA(cudaFuncSetAttribute(k_tc_res<EPI_SCAN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        const int grid = std::min(R.nunits, ix->num_sms);
        launch = [&, grid, smem]() { k_tc_res<EPI_SCAN><<<grid, RS_THREADS, smem, s>>>(ta, tab, tb, tbb, R); };
    } else {
        ta = make_map(abf.p, nr, kp, TC_BM);
        tb = make_map(ix->xbf.p, ix->nx, kp, TC_BN);
        P.nrows = nr;
        P.ncols = ix->nx;
        P.nkb = kp / TC_BK;
        P.nrt = (int)vj_div_up(nr, TC_BM);
        P.nct = (int)vj_div_up(ix->nx, TC_BN);
        P.metric = ix->metric;
        P.a_n = an.p;
        P.b_n = ix->sqn.p;  // data rows are the first nx nodes
        P.a_ids = aid.p;
        P.eps_key = eps_key;
        P.cb = ix->tc_cb;
        P.c3 = ix->tc_c3;
        P.cbmax = ix->tc_cbmax;
        P.ncand = ctr.p;
        P.err = err.p;
        P.spin_limit = spin_limit;
        const int ntiles = P.nrt * P.nct;
        const int grid = std::min(ntiles, ix->num_sms);
        const size_t smem = sizeof(TcSmem) + 1024;
        const int mode = cosine ? 2 : (ix->bf16_exact ? 0 : 1);
        auto kern = mode == 0 ? k_tc_scan<0> : (mode == 1 ? k_tc_scan<1> : k_tc_scan<2>);
        VJ_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        launch = [&, grid, smem, kern]() { kern<<<grid, TC_THREADS, smem, s>>>(ta, tb, P); };
    }
    int64_t cap = std::max<int64_t>(cq.n, std::max<int64_t>(nr * 64, 1 << 20));
    unsigned long long hn = 0;
    int herr = 0;
    cudaEvent_t e0, e1;
    VJ_CUDA(cudaEventCreate(&e0));
    VJ_CUDA(cudaEventCreate(&e1));
    float ms = 0.f;
    for (int attempt = 0; attempt < 3; attempt++) {
        cq.ensure(cap, s);
        cx.ensure(cap, s);
        P.cq = R.cq = cq.p;
        P.cx = R.cx = cx.p;
        if (R.a_rn) {
            ck->ensure(cap, s);
            R.ck = ck->p;
        }
        P.cap = R.cap = (int64_t)cq.n;
        VJ_CUDA(cudaMemsetAsync(ctr.p, 0, sizeof(unsigned long long), s));
        VJ_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
        VJ_CUDA(cudaEventRecord(e0, s));
        launch();
        VJ_LAUNCH_CHECK();
        VJ_CUDA(cudaEventRecord(e1, s));
        VJ_CUDA(cudaMemcpyAsync(&hn, ctr.p, sizeof(hn), cudaMemcpyDeviceToHost, s));
        VJ_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
        VJ_CUDA(cudaStreamSynchronize(s));
        VJ_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        VJ_REQUIRE(herr == 0, VJ_ERR_TIMEOUT, "tensor-core scan: a pipeline wait timed out");
        if ((int64_t)hn <= (int64_t)cq.n) break;
        cap = (int64_t)hn + (int64_t)hn / 4 + RS_HOLE_SLACK;  // the next launch may leave other holes
    }
    VJ_REQUIRE((int64_t)hn <= (int64_t)cq.n, VJ_ERR_STATE, "tensor-core scan: candidate list still too small");
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (ms_out) *ms_out = ms;
    ix->last_scan_exact_keys = R.a_rn != nullptr;
    abf.free_(s);
    aid.free_(s);
    an.free_(s);
    anode.free_(s);
    rn_rows.free_(s);
    ctr.free_(s);
    err.free_(s);
    return (int64_t)hn;
}

// ---------------------------------------------------------------- exact kNN build
// Candidates of the exact kNN over all n nodes, on the tensor cores, in two
// sweeps of the resident kernel:
//   1. every KNN_SAMPLE-th data tile: per row the 16th largest accumulator t
//      (so about 16 * KNN_SAMPLE nodes overall are expected above it);
//   2. every tile: the nodes whose accumulator exceeds t (a hair below it),
//      listed per row (CSR).
// Every node left out has accumulator <= t, so its true key is at least
// (1 - c3)|a|^2 - t (L2) or 1 - t - cb (cosine) less the accumulation margin;
// that bound goes to the exact re-rank, whose certificate decides whether the
// row's top K is proven.
constexpr int KNN_SAMPLE = 16;

__global__ void k_knn_thr(const float* __restrict__ top, int64_t n, float* __restrict__ thr) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float t = top[i];
    thr[i] = t > -INFINITY ? t - fabsf(t) * 3.814697265625e-6f - 1e-30f : -INFINITY;
}

__global__ void k_iota(int32_t* __restrict__ v, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = (int32_t)i;
}

__global__ void k_pair_count(const int32_t* __restrict__ cq, int64_t nc, int32_t* __restrict__ counts) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < nc && cq[e] >= 0) atomicAdd(counts + cq[e], 1);  // -1: a hole
}

__global__ void k_pair_scatter(const int32_t* __restrict__ cq, const int32_t* __restrict__ cx, int64_t nc,
                               const int64_t* __restrict__ off, int32_t* __restrict__ cursor,
                               int32_t* __restrict__ ids) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nc) return;
    const int q = cq[e];
    if (q < 0) return;  // a hole
    ids[off[q] + atomicAdd(cursor + q, 1)] = cx[e];
}

// true-key lower bound of every node a row did not list (accumulator <= thr)
__global__ void k_knn_bound(const float* __restrict__ sqn, const float* __restrict__ thr_acc, int64_t n, int metric,
                            int kp, float cb, float c3, float cbmax, double maxnorm, float* __restrict__ thr) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float ta = thr_acc[i];
    if (!(ta > -INFINITY)) {
        thr[i] = -INFINITY;  // nothing was left out for a reason: no bound
        return;
    }
    const double g = (double)(kp + 16) * 1.1920928955078125e-7;
    if (metric == 0) {
        const double rn = (double)sqn[i];
        const double mag = 2.1 * sqrt(rn) * maxnorm + 1.1 * maxnorm * maxnorm + (double)cbmax * maxnorm;
        thr[i] = (float)((1.0 - (double)c3) * rn - (double)ta - g * mag);
    } else {
        thr[i] = (float)(1.0 - (double)ta - (double)cb - 3.0 * g);
    }
}

bool vj_tc_knn_candidates(vj_index* ix, DBuf<int64_t>& off, DBuf<int32_t>& ids, DBuf<float>& row_thr) {
    const int kpad = (ix->d + TC_BK - 1) / TC_BK * TC_BK;
    if (kpad > RS_MAX_KB * TC_BK || ix->n < 4096) return false;
    cudaStream_t s = ix->stream;
    ensure_data_bf16(ix);
    const bool cosine = ix->metric != VJ_L2;
    const int64_t n = ix->n;
    DBuf<__nv_bfloat16> abf;
    DBuf<float> top, thr;
    DBuf<int32_t> iota;
    DBuf<int> err;
    DBuf<unsigned long long> ctr;
    abf.alloc((size_t)n * kpad, s);
    top.alloc(n, s);
    thr.alloc(n, s);
    iota.alloc(n, s);
    err.alloc(1, s);
    ctr.alloc(1, s);
    k_to_bf16<<<vj_div_up(n * kpad, 256), 256, 0, s>>>(ix->vec.p, ix->dp, ix->d, nullptr, 0, n, kpad,
                                                      cosine ? 1.f : 2.f, cosine ? ix->invn.p : nullptr, abf.p);
    k_iota<<<vj_div_up(n, 256), 256, 0, s>>>(iota.p, n);
    VJ_LAUNCH_CHECK();
    CUtensorMap ta = make_map(abf.p, n, kpad, 128);
    CUtensorMap tb = make_map(ix->xbf.p, n, kpad, RS_BN);
    CUtensorMap tab = cosine ? ta : make_map16(ix->abias.p, 128, 128);
    CUtensorMap tbb = cosine ? tb : make_map16(ix->xbias.p, n, RS_BN);
    RsParams R{};
    R.nrows = n;
    R.ncols = n;
    R.nkb = kpad / TC_BK;
    R.bias = cosine ? 0 : 1;
    R.nrp = (int)vj_div_up(n, 256);
    const int nct_all = (int)vj_div_up(n, RS_BN);
    const size_t fixed = 2048 + RS_BBOX + 2 * (size_t)R.nkb * RS_BOX;
    const size_t per = (size_t)R.nkb * RS_BOX + RS_BBOX;
    R.stages = (int)std::min<size_t>(RS_MAX_STAGES, (232448 - fixed) / per);
    R.err = err.p;
    R.spin_limit = 1ll << 22;
    const size_t smem = fixed + per * (size_t)R.stages;
    VJ_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));

    // 1. sample sweep: one unit per 256-row block over every KNN_SAMPLE-th tile
    R.tstride = KNN_SAMPLE;
    R.nct = (nct_all + KNN_SAMPLE - 1) / KNN_SAMPLE;
    R.tpu = R.nct;
    R.nunits = R.nrp;
    R.top16 = top.p;
    VJ_CUDA(cudaFuncSetAttribute(k_tc_res<EPI_SAMPLE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_tc_res<EPI_SAMPLE><<<std::min(R.nunits, ix->num_sms), (2 + KN_EPI) * 32, smem, s>>>(ta, tab, tb, tbb, R);
    VJ_LAUNCH_CHECK();
    k_knn_thr<<<vj_div_up(n, 256), 256, 0, s>>>(top.p, n, thr.p);
    VJ_LAUNCH_CHECK();

    // 2. candidate sweep over every tile, rows are node ids
    R.tstride = 1;
    R.nct = nct_all;
    {
        const int64_t g = std::max(1, ix->num_sms);
        int64_t best = INT64_MAX;
        int best_tpu = R.nct;
        for (int64_t ncc = 1; ncc <= R.nct; ncc++) {
            const int64_t tpu = (R.nct + ncc - 1) / ncc;
            if (ncc > 1 && (R.nct + tpu - 1) / tpu != ncc) continue;
            const int64_t load = (((int64_t)R.nrp * ncc + g - 1) / g) * (tpu + 3);
            if (load < best) {
                best = load;
                best_tpu = (int)tpu;
            }
        }
        R.tpu = best_tpu;
    }
    R.nunits = R.nrp * (int)vj_div_up(R.nct, R.tpu);
    R.a_thr = thr.p;
    R.a_ids = iota.p;
    R.ncand = ctr.p;
    VJ_CUDA(cudaFuncSetAttribute(k_tc_res<EPI_SCAN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    DBuf<int32_t>& cq = ix->scan_cq;
    DBuf<int32_t>& cx = ix->scan_cx;
    int64_t cap = std::max<int64_t>(cq.n, n * (int64_t)(20 * KNN_SAMPLE) + (1 << 20));
    unsigned long long hn = 0;
    int herr = 0;
    for (int attempt = 0; attempt < 3; attempt++) {
        cq.ensure(cap, s);
        cx.ensure(cap, s);
        R.cq = cq.p;
        R.cx = cx.p;
        R.cap = (int64_t)cq.n;
        VJ_CUDA(cudaMemsetAsync(ctr.p, 0, sizeof(unsigned long long), s));
        k_tc_res<EPI_SCAN><<<std::min(R.nunits, ix->num_sms), RS_THREADS, smem, s>>>(ta, tab, tb, tbb, R);
        VJ_LAUNCH_CHECK();
        VJ_CUDA(cudaMemcpyAsync(&hn, ctr.p, sizeof(hn), cudaMemcpyDeviceToHost, s));
        VJ_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
        VJ_CUDA(cudaStreamSynchronize(s));
        VJ_REQUIRE(herr == 0, VJ_ERR_TIMEOUT, "tensor-core kNN: a pipeline wait timed out");
        if ((int64_t)hn <= (int64_t)cq.n) break;
        cap = (int64_t)hn + (int64_t)hn / 4 + RS_HOLE_SLACK;  // the next launch may leave other holes
    }
    VJ_REQUIRE((int64_t)hn <= (int64_t)cq.n, VJ_ERR_STATE, "tensor-core kNN: candidate list still too small");
    const int64_t nc = (int64_t)hn;

    // 3. candidates grouped by row (CSR) and each row's bound
    DBuf<int32_t> counts, cursor;
    counts.alloc(n, s);
    cursor.alloc(n, s);
    VJ_CUDA(cudaMemsetAsync(counts.p, 0, n * sizeof(int32_t), s));
    VJ_CUDA(cudaMemsetAsync(cursor.p, 0, n * sizeof(int32_t), s));
    if (nc > 0) k_pair_count<<<vj_div_up(nc, 256), 256, 0, s>>>(cq.p, nc, counts.p);
    VJ_LAUNCH_CHECK();
    off.ensure(n + 1, s);
    vj_exclusive_scan_i32_to_i64(counts.p, off.p, n, ix);
    ids.ensure(std::max<int64_t>(nc, 1), s);
    if (nc > 0) k_pair_scatter<<<vj_div_up(nc, 256), 256, 0, s>>>(cq.p, cx.p, nc, off.p, cursor.p, ids.p);
    VJ_LAUNCH_CHECK();
    row_thr.ensure(n, s);
    k_knn_bound<<<vj_div_up(n, 256), 256, 0, s>>>(ix->sqn.p, thr.p, n, ix->metric, kpad, ix->tc_cb, ix->tc_c3,
                                                  ix->tc_cbmax, ix->maxnorm, row_thr.p);
    VJ_LAUNCH_CHECK();
    counts.free_(s);
    cursor.free_(s);
    abf.free_(s);
    top.free_(s);
    thr.free_(s);
    iota.free_(s);
    err.free_(s);
    ctr.free_(s);
    return true;
}
