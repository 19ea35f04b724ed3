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

#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "vj_device.cuh"
#include "vj_internal.cuh"
#include "vj_tc.cuh"

namespace {

using namespace vjtc;

constexpr int TC_BK = 64;                 // K columns per TMA box (128 bytes of BF16: one swizzle row)
constexpr uint32_t TC_TMEM_COLS = 512;    // two 256-column FP32 accumulators

// ---------------------------------------------------------------- streamed tiles (kp > 128)
// For rows wider than the resident kernel holds, both operands stream through
// a ring of K blocks: a 128-row A box and a 256-row B box of 64 BF16 columns
// per stage, tcgen05.mma M=128 N=256 into one of two TMEM accumulators while
// the epilogue drains the other.  A work unit is one 128-row tile of A against
// a run of B tiles (every tstride-th tile), so a CTA keeps its A rows hot in L2
// and the units running at the same time walk the same B tiles.
//
// The epilogue works on v = acc * cs[c] + cb[c] with per-B-row scale and bias
// (L2: cs = 2 and cb = the scan bias -(1 - c3)|b|^2 + cbmax |b|, so v is the
// value the resident kernel accumulates; cosine: cs = 1/|b| for raw rows or 1
// for unit rows, cb = 0):
//   EPI_SCAN    a pair is a candidate when v > thr[row]; candidates are
//               appended through per-warp chunks as (row id, column, acc * cs);
//   EPI_SAMPLE  each row keeps the WD_TOP largest v over the unit's tiles (its
//               own column excluded) and writes the smallest of them to
//               top16[row].
// Warp 0 issues TMA, warp 1 owns TMEM and issues the MMAs, warps 2..9 are the
// epilogue (two per TMEM lane quarter, 128 columns each).  Every wait is
// bounded; an epilogue warp that gives up keeps walking its tiles (without
// touching TMEM) so that the epilogue's named barriers always fill.
enum { EPI_SCAN = 0, EPI_SAMPLE = 1 };

constexpr int WD_BM = 128, WD_BN = 256, WD_STAGES = 4;
constexpr int WD_EPI = 8;
constexpr int WD_THREADS = (2 + WD_EPI) * 32;
constexpr uint32_t WD_A_BYTES = WD_BM * TC_BK * 2;  // 16 KB
constexpr uint32_t WD_B_BYTES = WD_BN * TC_BK * 2;  // 32 KB
constexpr int WD_CHUNK = 128;                       // candidate slots reserved per warp at a time
// EPI_SAMPLE keeps the WD_TOP largest values per row.  With every 16th tile
// sampled, the WD_TOP-th sampled value lies near the row's 16 WD_TOP-th
// largest overall; a row's K = 64 nearest all stay above it unless at least
// WD_TOP of them fall in the 1/16 sample (binomial tail: about 1e-5 per row
// for 16, 1.5e-8 for 20), which is what leaves a row uncertified.
constexpr int WD_TOP = 20;

struct __align__(1024) WdSmem {
    uint8_t A[WD_STAGES][WD_A_BYTES];
    uint8_t B[WD_STAGES][WD_B_BYTES];
    uint64_t full[WD_STAGES];
    uint64_t empty[WD_STAGES];
    uint64_t tfull[2];
    uint64_t tempty[2];
    uint64_t drain;
    uint32_t tmem_base;
    int abort;
    __align__(16) float cs[2][WD_BN];
    __align__(16) float cb[2][WD_BN];
    __align__(16) float th[2][WD_BN];  // symmetric sweep: the columns' row thresholds
    float part[WD_BM][WD_TOP + 1];  // sample: the second column half's list per row
};

// kind::f16 instruction descriptor: FP32 accumulate, BF16 A and B, both
// K-major, M = 128, N = 256
constexpr uint32_t WD_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(WD_BN >> 3) << 17) |
                              ((uint32_t)(WD_BM >> 4) << 24);
// kind::f8f6f4 instruction descriptor: FP32 accumulate, E4M3 A and B (format
// code 0), both K-major, M = 128, N = 256.  A k-block is then 128 E4M3
// columns (the same 128-byte swizzle rows), four K = 32 steps.
constexpr uint32_t WD_IDESC_F8 = (1u << 4) | ((uint32_t)(WD_BN >> 3) << 17) | ((uint32_t)(WD_BM >> 4) << 24);
// kind::tf32 instruction descriptor: FP32 accumulate, TF32 A and B (format
// code 2), both K-major, M = 128, N = 256; a k-block is 32 FP32 columns, four
// K = 8 steps
constexpr uint32_t WD_IDESC_TF32 = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(WD_BN >> 3) << 17) |
                                   ((uint32_t)(WD_BM >> 4) << 24);
// operand kinds of the streamed kernel
enum { KIND_BF16 = 0, KIND_E4M3 = 1, KIND_TF32 = 2 };

struct WdParams {
    int64_t nrows, ncols;  // A rows, B rows
    int nkb;               // K blocks of 128 bytes (64 BF16 or 128 E4M3 columns)
    int kk_last;           // K steps (of 32 bytes) in the last K block; 0: all four (its tail past the
                           // row is zero, so skipping those steps changes nothing)
    int nrt;               // A row tiles
    int nct;               // B tiles a sweep visits (tile k of the sweep is B tile k * tstride)
    int tstride;
    int tpu;               // B tiles per work unit (EPI_SAMPLE: all of them)
    int nunits;            // nrt * ceil(nct / tpu), row tile fastest
    const float* cs;       // [ncols] per B row: scale of the accumulator
    const float* cb;       // [ncols] per B row: bias added before the row test
    const float* thr;      // [nrows] EPI_SCAN: candidate iff acc * cs + cb > thr
    const int32_t* a_ids;  // [nrows] id written for the row's candidates (nullptr: the row index)
    int32_t* cq;
    int32_t* cx;
    float* cw;             // acc * cs of each candidate (nullptr: not written)
    unsigned long long* ncand;
    int64_t cap;
    float* top16;          // [nrows] EPI_SAMPLE output (rows are node ids: the row's own column is skipped)
    int* err;
    long long spin_limit;
    // symmetric sweep (A = B, EPI_SCAN, tstride 1): units[u] = (row tile, first
    // B tile, end B tile); a tile strictly above its row tile's 256-row block
    // (ct > rt / 2) also tests the transposed pairs (c, r): acc * cs[r] + cb[r]
    // > thr[c], so each unordered pair is computed once
    const int4* units;
    // node ids of A row 0 (when a_ids is nullptr) and of B row 0
    int64_t row_base, col_base;
};

// (row tile, first tile, end tile) of work unit u
__device__ __forceinline__ void wd_unit(const WdParams& P, int u, int& rt, int& t0, int& t1) {
    if (P.units) {
        const int4 v = P.units[u];
        rt = v.x;
        t0 = v.y;
        t1 = v.z;
    } else {
        rt = u % P.nrt;
        const int cc = u / P.nrt;
        t0 = cc * P.tpu;
        t1 = min(P.nct, t0 + P.tpu);
    }
}

// warp-aggregated append of the pairs marked in (h0, h1) over 64 accumulator
// columns c0 .. c0 + 63: as (row, column) pairs, or, transposed, as (column,
// row) pairs; w = acc times the B row's scale (cs[j], or rs when transposed)
__device__ __forceinline__ void wd_append(const WdParams& P, const uint32_t (&va)[64], uint32_t h0, uint32_t h1,
                                          int64_t c0, int rowid, bool transposed, const float* cs, float rs,
                                          unsigned long long& cbase, int& cleft, int lane) {
    const int mine = __popc(h0) + __popc(h1);
    int incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t2 = __shfl_up_sync(VJ_FULL, incl, o);
        if (lane >= o) incl += t2;
    }
    const int total = __shfl_sync(VJ_FULL, incl, 31);
    if (total == 0) return;
    if (total > cleft) {
        // close the chunk (its unused slots become holes) and reserve the next
        for (int k = lane; k < cleft; k += 32)
            if ((int64_t)(cbase + k) < P.cap) P.cq[cbase + k] = -1;
        const int want = max(total, WD_CHUNK);
        unsigned long long gb = 0;
        if (lane == 31) gb = atomicAdd(P.ncand, (unsigned long long)want);
        cbase = __shfl_sync(VJ_FULL, gb, 31);
        cleft = want;
    }
    unsigned long long gq = cbase + (unsigned long long)(incl - mine);
    cbase += (unsigned long long)total;
    cleft -= total;
#pragma unroll
    for (int hh = 0; hh < 2; hh++) {
        uint32_t hit = hh ? h1 : h0;
        while (hit) {
            const int j = __ffs(hit) - 1;
            hit &= hit - 1;
            if ((int64_t)gq < P.cap) {
                const int col = (int)(P.col_base + c0 + hh * 32 + j);
                P.cq[gq] = transposed ? col : rowid;
                P.cx[gq] = transposed ? rowid : col;
                if (P.cw) {
                    // select by unrolled compares: a runtime index into va
                    // would move the whole array to local memory
                    float o = 0.f;
#pragma unroll
                    for (int jj = 0; jj < 32; jj++)
                        if (jj == j) o = __uint_as_float(va[hh * 32 + jj]);
                    P.cw[gq] = o * (transposed ? rs : cs[hh * 32 + j]);
                }
            }
            gq++;
        }
    }
}

template <int EPI, int KIND = KIND_BF16>
__global__ void __launch_bounds__(WD_THREADS, 1)
    k_tc_wide(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tB, WdParams P) {
    extern __shared__ uint8_t wd_raw[];
    WdSmem& S = *reinterpret_cast<WdSmem*>((reinterpret_cast<uintptr_t>(wd_raw) + 1023) & ~uintptr_t(1023));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    volatile int* abort = &S.abort;

    if (threadIdx.x == 0) {
        for (int s = 0; s < WD_STAGES; s++) {
            mbar_init(&S.full[s], 1);
            mbar_init(&S.empty[s], 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(&S.tfull[b], 1);
            mbar_init(&S.tempty[b], WD_EPI);
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
            for (int u = blockIdx.x; u < P.nunits && ok; u += gridDim.x) {
                int rt, t0, t1;
                wd_unit(P, u, rt, t0, t1);
                for (int ct = t0; ct < t1 && ok; ct++) {
                    for (int kb = 0; kb < P.nkb; kb++) {
                        if (!mbar_wait(&S.empty[s], ph ^ 1u, abort, P.spin_limit)) {
                            ok = false;
                            break;
                        }
                        mbar_arrive_tx(&S.full[s], WD_A_BYTES + WD_B_BYTES);
                        // x in elements of the map: 64 BF16, 128 E4M3 or 32 FP32 per K block
                        const int kx = kb * (KIND == KIND_E4M3 ? 128 : KIND == KIND_TF32 ? 32 : TC_BK);
                        tma_load_2d(S.A[s], &tA, &S.full[s], kx, rt * WD_BM);
                        tma_load_2d(S.B[s], &tB, &S.full[s], kx, ct * P.tstride * WD_BN);
                        issued |= 1u << s;
                        last_ph = (last_ph & ~(1u << s)) | (ph << s);
                        if (++s == WD_STAGES) {
                            s = 0;
                            ph ^= 1u;
                        }
                    }
                }
            }
            if (!ok) {
                *abort = 1;
                atomicExch(P.err, 1);
                // let this CTA's copies land before shared memory goes away
                for (int st = 0; st < WD_STAGES; st++)
                    if ((issued >> st) & 1u)
                        for (long long i = 0; i < P.spin_limit && !mbar_test(&S.full[st], (last_ph >> st) & 1u);
                             i++) {
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
            for (int u = blockIdx.x; u < P.nunits && ok; u += gridDim.x) {
                int rt, t0, t1;
                wd_unit(P, u, rt, t0, t1);
                for (int ct = t0; ct < t1 && ok; ct++, i++) {
                    const int acc = i & 1;
                    if (!mbar_wait(&S.tempty[acc], (uint32_t)(((i >> 1) & 1) ^ 1), abort, P.spin_limit)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d = tmem + (uint32_t)(acc * WD_BN);
                    for (int kb = 0; kb < P.nkb; kb++) {
                        if (!mbar_wait(&S.full[s], ph, abort, P.spin_limit)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint64_t ad = sdesc_sw128(su32(S.A[s]));
                        const uint64_t bd = sdesc_sw128(su32(S.B[s]));
                        const int nkk = (kb == P.nkb - 1 && P.kk_last > 0) ? P.kk_last : TC_BK / 16;
#pragma unroll
                        for (int kk = 0; kk < TC_BK / 16; kk++) {
                            // advance 32 bytes along K (16 BF16, 32 E4M3 or 8 TF32) inside the swizzled rows
                            if (kk < nkk) {
                                if constexpr (KIND == KIND_E4M3)
                                    tc_mma_f8(d, ad + (uint64_t)(kk * 2), bd + (uint64_t)(kk * 2), WD_IDESC_F8,
                                              (kb | kk) != 0);
                                else if constexpr (KIND == KIND_TF32)
                                    tc_mma_tf32(d, ad + (uint64_t)(kk * 2), bd + (uint64_t)(kk * 2), WD_IDESC_TF32,
                                                (kb | kk) != 0);
                                else
                                    tc_mma(d, ad + (uint64_t)(kk * 2), bd + (uint64_t)(kk * 2), WD_IDESC,
                                           (kb | kk) != 0);
                            }
                        }
                        tc_commit(&S.empty[s]);
                        if (++s == WD_STAGES) {
                            s = 0;
                            ph ^= 1u;
                        }
                    }
                    if (!ok) break;
                    tc_commit(&S.tfull[acc]);
                }
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
        // ---------------- epilogue: warp e reads TMEM lane quarter (warp & 3),
        // columns cg * 128 .. cg * 128 + 127 of each accumulator
        const int e = warp - 2;
        const int quarter = warp & 3;
        const int cg = e >> 2;
        const int etid = e * 32 + lane;  // one B column of each tile to stage
        bool dead = false;
        int i = 0;
        unsigned long long cbase = 0;  // EPI_SCAN: this warp's output chunk (next slot, slots left)
        int cleft = 0;
        for (int u = blockIdx.x; u < P.nunits; u += gridDim.x) {
            int rt, t0, t1;
            wd_unit(P, u, rt, t0, t1);
            const int64_t r = (int64_t)rt * WD_BM + quarter * 32 + lane;
            const bool rv = r < P.nrows;
            const float thr = (EPI == EPI_SCAN && rv) ? P.thr[r] : INFINITY;
            const int qid = rv ? (P.a_ids ? P.a_ids[r] : (int)(P.row_base + r)) : -1;
            // symmetric sweep: this row as a B row (scale and bias of the transposed test)
            const float rcs = (P.units && rv) ? P.cs[r] : 0.f;
            const float rcb = (P.units && rv) ? P.cb[r] : -INFINITY;
            float t[WD_TOP];
#pragma unroll
            for (int k = 0; k < WD_TOP; k++) t[k] = -INFINITY;
            for (int ct = t0; ct < t1; ct++, i++) {
                const int acc = i & 1;
                const int64_t cbase_col = (int64_t)ct * P.tstride * WD_BN;
                // stage this tile's column scale and bias (a column past the last
                // B row gets bias -inf: it never passes a test)
                const bool sym_t = P.units != nullptr && ct > (rt >> 1);  // both directions in this tile
                {
                    const int64_t c = cbase_col + etid;
                    const bool cv = c < P.ncols;
                    S.cs[acc][etid] = cv ? P.cs[c] : 0.f;
                    S.cb[acc][etid] = cv ? P.cb[c] : -INFINITY;
                    if (EPI == EPI_SCAN && sym_t) S.th[acc][etid] = cv ? P.thr[c] : INFINITY;
                }
                asm volatile("bar.sync 1, %0;" ::"r"(WD_EPI * 32) : "memory");
                if (!dead) {
                    const bool got = mbar_wait(&S.tfull[acc], (uint32_t)((i >> 1) & 1), abort, P.spin_limit);
                    if (!__all_sync(VJ_FULL, got)) {
                        if (lane == 0) {
                            *abort = 1;
                            atomicExch(P.err, 1);
                        }
                        dead = true;
                    }
                }
                if (!dead) {
                    tc_fence_after();
#pragma unroll 1
                    for (int h = 0; h < 2; h++) {
                        const int col0 = cg * 128 + h * 64;  // column within the tile
                        uint32_t va[64];
                        __syncwarp();  // lanes that skipped the last half's work rejoin before the aligned load
                        tmem_ld64_issue(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(acc * WD_BN + col0), va);
                        tmem_wait_ld64(va);
                        if (h == 1) {
                            // both halves have been read: hand the TMEM buffer back
                            tc_fence_before();
                            __syncwarp();
                            if (lane == 0) mbar_arrive(&S.tempty[acc]);
                        }
                        const float4* cs4 = reinterpret_cast<const float4*>(&S.cs[acc][col0]);
                        const float4* cb4 = reinterpret_cast<const float4*>(&S.cb[acc][col0]);
                        float m0 = -INFINITY, m1 = -INFINITY, m2 = -INFINITY, m3 = -INFINITY;
#pragma unroll
                        for (int j4 = 0; j4 < 16; j4++) {
                            const float4 a = cs4[j4], b = cb4[j4];
                            m0 = fmaxf(m0, fmaf(__uint_as_float(va[4 * j4 + 0]), a.x, b.x));
                            m1 = fmaxf(m1, fmaf(__uint_as_float(va[4 * j4 + 1]), a.y, b.y));
                            m2 = fmaxf(m2, fmaf(__uint_as_float(va[4 * j4 + 2]), a.z, b.z));
                            m3 = fmaxf(m3, fmaf(__uint_as_float(va[4 * j4 + 3]), a.w, b.w));
                        }
                        const float mx = fmaxf(fmaxf(m0, m1), fmaxf(m2, m3));
                        if constexpr (EPI == EPI_SAMPLE) {
                            if (!rv || !(mx > t[WD_TOP - 1])) continue;
                            const int64_t c0 = P.col_base + cbase_col + col0;  // node id of the first column
                            const bool self_here = qid >= c0 && qid < c0 + 64;
#pragma unroll
                            for (int j = 0; j < 64; j++) {
                                float x = fmaf(__uint_as_float(va[j]), S.cs[acc][col0 + j], S.cb[acc][col0 + j]);
                                if (!(x > t[WD_TOP - 1])) continue;
                                if (self_here && c0 + j == qid) continue;
                                // insert: x sinks to its place, the last value drops out
#pragma unroll
                                for (int k = 0; k < WD_TOP; k++) {
                                    const float hi = fmaxf(t[k], x);
                                    x = fminf(t[k], x);
                                    t[k] = hi;
                                }
                            }
                        } else {
                            const bool maybe = rv && mx > thr;
                            // the transposed test: this row's value against each column's threshold
                            bool maybe_t = false;
                            if (sym_t) {
                                const float4* th4 = reinterpret_cast<const float4*>(&S.th[acc][col0]);
                                float n0 = -INFINITY, n1 = -INFINITY, n2 = -INFINITY, n3 = -INFINITY;
#pragma unroll
                                for (int j4 = 0; j4 < 16; j4++) {
                                    const float4 th = th4[j4];
                                    n0 = fmaxf(n0, fmaf(__uint_as_float(va[4 * j4 + 0]), rcs, rcb) - th.x);
                                    n1 = fmaxf(n1, fmaf(__uint_as_float(va[4 * j4 + 1]), rcs, rcb) - th.y);
                                    n2 = fmaxf(n2, fmaf(__uint_as_float(va[4 * j4 + 2]), rcs, rcb) - th.z);
                                    n3 = fmaxf(n3, fmaf(__uint_as_float(va[4 * j4 + 3]), rcs, rcb) - th.w);
                                }
                                maybe_t = rv && fmaxf(fmaxf(n0, n1), fmaxf(n2, n3)) > 0.f;
                            }
                            if (!__any_sync(VJ_FULL, maybe || maybe_t)) continue;
                            const int64_t c0 = cbase_col + col0;
                            uint32_t hit0 = 0, hit1 = 0;
                            if (maybe) {
#pragma unroll
                                for (int j = 0; j < 32; j++) {
                                    hit0 |= (uint32_t)(fmaf(__uint_as_float(va[j]), S.cs[acc][col0 + j],
                                                            S.cb[acc][col0 + j]) > thr) << j;
                                    hit1 |= (uint32_t)(fmaf(__uint_as_float(va[32 + j]), S.cs[acc][col0 + 32 + j],
                                                            S.cb[acc][col0 + 32 + j]) > thr) << j;
                                }
                            }
                            wd_append(P, va, hit0, hit1, c0, qid, false, &S.cs[acc][col0], 0.f, cbase, cleft, lane);
                            if (__any_sync(VJ_FULL, maybe_t)) {
                                uint32_t th0 = 0, th1 = 0;
                                if (maybe_t) {
#pragma unroll
                                    for (int j = 0; j < 32; j++) {
                                        th0 |= (uint32_t)(fmaf(__uint_as_float(va[j]), rcs, rcb) > S.th[acc][col0 + j])
                                               << j;
                                        th1 |= (uint32_t)(fmaf(__uint_as_float(va[32 + j]), rcs, rcb) >
                                                          S.th[acc][col0 + 32 + j])
                                               << j;
                                    }
                                }
                                wd_append(P, va, th0, th1, c0, qid, true, nullptr, rcs, cbase, cleft, lane);
                            }
                        }
                    }
                }
            }
            if constexpr (EPI == EPI_SAMPLE) {
                // merge the two column halves' lists of each row
                const int rl = quarter * 32 + lane;
                if (cg == 1) {
#pragma unroll
                    for (int k = 0; k < WD_TOP; k++) S.part[rl][k] = t[k];
                }
                asm volatile("bar.sync 2, %0;" ::"r"(WD_EPI * 32) : "memory");
                if (cg == 0 && rv && !dead) {
#pragma unroll 1
                    for (int k2 = 0; k2 < WD_TOP; k2++) {
                        float x = S.part[rl][k2];
                        if (!(x > t[WD_TOP - 1])) break;  // the partner's list is descending
#pragma unroll
                        for (int k = 0; k < WD_TOP; k++) {
                            const float hi = fmaxf(t[k], x);
                            x = fminf(t[k], x);
                            t[k] = hi;
                        }
                    }
                    P.top16[r] = t[WD_TOP - 1];
                }
                asm volatile("bar.sync 2, %0;" ::"r"(WD_EPI * 32) : "memory");
            }
        }
        if constexpr (EPI == EPI_SCAN) {
            for (int k = lane; k < cleft; k += 32)
                if ((int64_t)(cbase + k) < P.cap) P.cq[cbase + k] = -1;
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
    // sample epilogue: the rows' node ids are row_base + row, the columns' col_base + column
    float* top16;         // [nrows] 16th largest accumulator over the sampled tiles (other nodes)
    int64_t row_base, col_base;
};

constexpr int KN_EPI = 8;  // sample epilogue warps: one per (query block, lane quarter)

// Resident-query tensor-core kernel with two epilogues:
//   EPI_SCAN    16 warps; a pair is a candidate when its accumulator exceeds
//               the row's threshold (the brute-force route, the exact join and
//               the kNN build's candidate sweep);
//   EPI_SAMPLE   8 warps; each thread owns one row and keeps, in registers, the
//               16 largest accumulators over a sample of the data tiles (the
//               kNN build's per-row threshold).

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
                    __syncwarp();  // lanes that skipped the last half's work rejoin before the aligned load
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
                    const int64_t rg = P.row_base + r, cg = P.col_base + c0;  // node ids
                    const bool edge = c0 + 64 > P.ncols || (rg >= cg && rg < cg + 64);
#pragma unroll
                    for (int j = 0; j < 64; j++) {
                        float x = __uint_as_float(va[j]);
                        if (x <= t[15]) continue;
                        if (edge && (c0 + j >= P.ncols || cg + j == rg)) continue;
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
                                    P.cx[gq] = (int)(P.col_base + c0 + h * 32 + j);
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

// flag[0] |= any non-integer coordinate; flag[1] = max |coordinate| (integer
// part); flag[2] |= any coordinate that is not exactly a BF16 value.  Grid
// stride with one atomic per warp and flag (the vectors can be GBs).
__global__ void k_int_check(const float* __restrict__ v, int64_t n, unsigned int* __restrict__ flag) {
    unsigned int nonint = 0u, nonbf = 0u, mx = 0u;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float x = v[i];
        nonint |= (unsigned int)(!(x == rintf(x)) || fabsf(x) > 1e9f);
        nonbf |= (unsigned int)((__float_as_uint(x) & 0xFFFFu) != 0u);
        mx = max(mx, (unsigned int)fminf(fabsf(x), 4e9f));
    }
    nonint = __reduce_or_sync(VJ_FULL, nonint);
    nonbf = __reduce_or_sync(VJ_FULL, nonbf);
    mx = __reduce_max_sync(VJ_FULL, mx);
    if ((threadIdx.x & 31) == 0) {
        if (nonint) atomicOr(flag, 1u);
        if (nonbf) atomicOr(flag + 2, 1u);
        atomicMax(flag + 1, mx);
    }
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

// per node, the streamed kernel's column scale and bias (v = acc * cs + cb)
//   mode 0, L2:          cs = 2, cb = -(1 - c3)|b|^2 + cbmax |b|, so v is the
//                        resident kernel's accumulator 2<a,b> + bias_b
//   mode 1, cosine raw:  cs = 1/|b| (0 for a zero row), cb = 0
//   mode 2, cosine unit: cs = 1, cb = 0
__global__ void k_wide_cols(const float* __restrict__ sqn, const float* __restrict__ invn, int64_t n, int mode,
                            double c3, double cbmax, float* __restrict__ cs, float* __restrict__ cb) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    if (mode == 0) {
        const double nn = (double)sqn[c];
        cs[c] = 2.f;
        cb[c] = (float)(-(1.0 - c3) * nn + cbmax * sqrt(nn));
    } else {
        cs[c] = mode == 1 ? invn[c] : 1.f;
        cb[c] = 0.f;
    }
}

// cosine on raw rows: a pair is a candidate iff acc / |b| > (1 - eps - cb - margin) |a|
// (margin as in k_row_thr); a zero query row has cosine distance 1 to everything
__global__ void k_row_thr_raw(const float* __restrict__ invn, const int32_t* __restrict__ node, int64_t n, int kp,
                              float eps_key, float cb, float* __restrict__ thr) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double g = (double)(kp + 16) * 1.1920928955078125e-7;
    const double t = 1.0 - (double)eps_key - (double)cb - 3.0 * g;
    const double iv = (double)invn[node ? node[i] : i];
    thr[i] = iv > 0.0 ? (float)(t / iv) : (t < 0.0 ? -INFINITY : INFINITY);
}

// exact keys of the streamed scan's candidates (integer inputs): |a|^2 + |b|^2 - 2<a,b>
__global__ void k_key_from_w(const float* __restrict__ sqn, const int32_t* __restrict__ cq,
                             const int32_t* __restrict__ cx, const float* __restrict__ cw, int64_t nc, int64_t nx,
                             float* __restrict__ ck) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nc || cq[e] < 0) return;
    ck[e] = sqn[nx + cq[e]] + sqn[cx[e]] - cw[e];
}

// ---------------------------------------------------------------- measured rounding bound
// For tile rows that are not exact copies of the inputs, the bound on a tile
// value comes from each row's own rounding error instead of the worst case
// per coordinate.  With a^ = a + da and b^ = b + db the rows as the tiles hold
// them (scale removed),
//   |<a^, b^> - <a, b>| <= |da| |b| + |a| |db| + |da| |db|      (Cauchy-Schwarz),
// and the tensor core's sum of the exact products deviates from <a^, b^> by at
// most gamma |a^| |b^|.  The scanned rows enter through their largest |da| and
// |a|, so the whole bound is a per-column constant of the epilogue.  a is the
// input row (L2) or the exact unit vector a / |a| (cosine).
constexpr float F8_MAX = 448.f;  // largest finite E4M3 value

// largest power of two s with amax * s <= 448 (1 for a zero or vanishingly
// small row, whose 448 / amax would overflow; its rounding error is then
// measured like any other)
__device__ __forceinline__ float f8_scale(float amax) {
    if (!(amax > 1e-30f)) return 1.f;
    int e;
    frexpf(F8_MAX / amax, &e);  // 448 / amax = m 2^e, m in [0.5, 1)
    return ldexpf(1.f, e - 1);
}

__device__ __forceinline__ float f8_value(__nv_fp8_storage_t q) {
    return __half2float(__half(__nv_cvt_fp8_to_halfraw(q, __NV_E4M3)));
}

// coordinate k of the row the tiles approximate: its FP32 value as quantised
// (x, or x / |x| rounded to FP32) and its exact FP64 value
__device__ __forceinline__ void tile_coord(const float* v, int k, int cosine, double inv, float& y, double& ex) {
    const double x = (double)v[k];
    ex = cosine ? x * inv : x;
    y = (float)ex;
}

// largest |coordinate| over the rows (node ids rows[0..n)), as float bits
__global__ void k_tile_amax(const float* __restrict__ vec, const double* __restrict__ sqn64, int dp, int d,
                            int cosine, const int32_t* __restrict__ rows, int64_t n, unsigned int* __restrict__ amax) {
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= n) return;
    const int64_t src = rows ? (int64_t)rows[r] : r;
    const double nn = sqn64[src];
    const double inv = (cosine && nn > 0.0) ? 1.0 / sqrt(nn) : 1.0;
    float m = 0.f;
    for (int k = lane; k < d; k += 32) {
        float y;
        double ex;
        tile_coord(vec + src * dp, k, cosine, inv, y, ex);
        m = fmaxf(m, fabsf(y));
    }
    const unsigned int mb = __reduce_max_sync(VJ_FULL, __float_as_uint(m));
    if (lane == 0) atomicMax(amax, mb);
}

// TF32 value of x (round to nearest, ties away; the low 13 mantissa bits zero)
__device__ __forceinline__ float to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// Tile rows of the rows `rows` (node ids; nullptr = 0..n-1), kb elements each
// (zero past d), warp per row:
//   KIND_BF16: out is BF16 rows already written (k_to_bf16); only the error
//              is measured;
//   KIND_E4M3: out receives E4M3 bytes of y * s, s a power of two: the row's
//              own scale (amax == nullptr) or the shared one from *amax;
//              rs[r] = 1 / s;
//   KIND_TF32: out receives the TF32 values of y as FP32 words.
// err[r] = |row^ - row| in FP64, rounded up; emax / nmax (optional) collect the
// largest error and the largest |row| (float bits, atomicMax).
template <int KIND>
__global__ void k_tile_rows(const float* __restrict__ vec, const double* __restrict__ sqn64, int dp, int d,
                            int cosine, const int32_t* __restrict__ rows, int64_t n, int kb,
                            const unsigned int* __restrict__ amax, void* __restrict__ out, float* __restrict__ rs,
                            float* __restrict__ err, unsigned int* __restrict__ emax, unsigned int* __restrict__ nmax) {
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= n) return;
    const int64_t src = rows ? (int64_t)rows[r] : r;
    const float* v = vec + src * dp;
    const double nn = sqn64[src];
    const double inv = (cosine && nn > 0.0) ? 1.0 / sqrt(nn) : 1.0;
    float s = 1.f;
    if constexpr (KIND == KIND_E4M3) {
        float m;
        if (amax) {
            m = __uint_as_float(*amax);
        } else {
            m = 0.f;
            for (int k = lane; k < d; k += 32) {
                float y;
                double ex;
                tile_coord(v, k, cosine, inv, y, ex);
                m = fmaxf(m, fabsf(y));
            }
            m = __uint_as_float(__reduce_max_sync(VJ_FULL, __float_as_uint(m)));
        }
        s = f8_scale(m);
    }
    double e2 = 0.0;
    for (int k = lane; k < kb; k += 32) {
        float y = 0.f;
        double ex = 0.0;
        if (k < d) tile_coord(v, k, cosine, inv, y, ex);
        double got;
        if constexpr (KIND == KIND_E4M3) {
            const __nv_fp8_storage_t q = __nv_cvt_float_to_fp8(y * s, __NV_SATFINITE, __NV_E4M3);
            reinterpret_cast<uint8_t*>(out)[r * (int64_t)kb + k] = q;
            got = (double)f8_value(q) / (double)s;
        } else if constexpr (KIND == KIND_TF32) {
            const float t = to_tf32(y);
            reinterpret_cast<float*>(out)[r * (int64_t)kb + k] = t;
            got = (double)t;
        } else {
            got = (double)__bfloat162float(reinterpret_cast<const __nv_bfloat16*>(out)[r * (int64_t)kb + k]);
        }
        const double t = got - ex;
        e2 += t * t;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e2 += __shfl_xor_sync(VJ_FULL, e2, o);
    if (lane == 0) {
        const float e = __double2float_ru(sqrt(e2) * (1.0 + 1e-12));
        if (KIND == KIND_E4M3 && rs) rs[r] = 1.f / s;
        if (err) err[r] = e;
        if (emax) atomicMax(emax, __float_as_uint(e));
        if (nmax) atomicMax(nmax, __float_as_uint(__double2float_ru(cosine ? 1.0 : sqrt(nn))));
    }
}

// Per data column c, the streamed epilogue's v = acc * cs + cb under the
// measured bound (q[0] = largest |coordinate| of the scanned rows (FP8: their
// shared scale), q[1] = their largest |da|, q[2] = their largest |a|):
//   beta = Da |b| + A db + Da db + gamma (A + Da)(|b| + db)
//   L2:     cs = 2 / (sa sb), cb = -|b|^2 + 2 beta   (candidate iff v > |a|^2 - eps^2 - margin)
//   cosine: cs = 1 / (sa sb), cb = beta              (candidate iff v > 1 - eps - margin)
// (BF16 tiles: sa = sb = 1.)
__global__ void k_tile_cols(const double* __restrict__ sqn64, const float* __restrict__ xerr,
                            const float* __restrict__ xrs, int64_t nx, int cosine, int f8,
                            const unsigned int* __restrict__ q, double gamma, float* __restrict__ cs,
                            float* __restrict__ cb) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nx) return;
    const double sa = f8 ? (double)f8_scale(__uint_as_float(q[0])) : 1.0;
    const double Da = (double)__uint_as_float(q[1]);
    const double A = (double)__uint_as_float(q[2]);
    const double nb = cosine ? 1.0 : sqrt(sqn64[c]);
    const double db = (double)xerr[c];
    const double beta = Da * nb + A * db + Da * db + gamma * (A + Da) * (nb + db);
    const double rsb = f8 ? (double)xrs[c] : 1.0;  // 1 / sb
    if (cosine) {
        cs[c] = (float)(rsb / sa);
        cb[c] = __double2float_ru(beta);
    } else {
        cs[c] = (float)(2.0 * rsb / sa);
        cb[c] = __double2float_ru(-sqn64[c] + 2.0 * beta);
    }
}

// per scanned row: the threshold of the measured-bound test (see k_tile_cols);
// margin covers the FP32 rounding of the epilogue, of cb and of the threshold
__global__ void k_tile_thr(const double* __restrict__ sqn64, const int32_t* __restrict__ node, int64_t n,
                           int cosine, double eps_key, double maxnorm, float* __restrict__ thr) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (cosine) {
        thr[i] = __double2float_rd(1.0 - eps_key - 1e-5);
    } else {
        const double margin = 1e-5 * (4.0 * maxnorm * maxnorm + eps_key);
        thr[i] = __double2float_rd(sqn64[node[i]] - eps_key - margin);
    }
}

}  // namespace

// BF16 copy of every node and the bound constants of the tensor-core tiles
// (built once per index, kept for later scans).
//   kp <= 128 (resident kernel): cosine rows are stored unit-normalised.
//   kp >  128 (streamed kernel): also the per-node column scale and bias; when
//   every coordinate is exactly a BF16 value, cosine rows are stored raw (the
//   epilogue divides by |b|), so the tiles' only error is the accumulation.
static void ensure_data_bf16(vj_index* ix) {
    const int kp = (ix->d + TC_BK - 1) / TC_BK * TC_BK;
    if (ix->xbf.n >= (size_t)ix->n * kp) return;
    cudaStream_t s = ix->stream;
    const bool cosine = ix->metric != VJ_L2;
    const bool wide = kp > RS_MAX_KB * TC_BK;
    // Exact-key test: when every coordinate is an integer of magnitude <= 256
    // it is exact in BF16, every product is an integer below 2^16 and, with
    // d * max^2 <= 2^23, every partial sum, both norms, their sum (<= 2^24)
    // and the norm expansion stay integers exactly representable in FP32, so
    // the FP32-accumulated key is exact and needs no bound.
    DBuf<unsigned int> flag;
    flag.alloc(3, s);
    VJ_CUDA(cudaMemsetAsync(flag.p, 0, 3 * sizeof(unsigned int), s));
    k_int_check<<<std::max(1, std::min(vj_div_up(ix->n * ix->dp, 256), 16 * ix->num_sms)), 256, 0, s>>>(
        ix->vec.p, ix->n * ix->dp, flag.p);
    VJ_LAUNCH_CHECK();
    unsigned int h[3] = {0, 0, 0};
    VJ_CUDA(cudaMemcpyAsync(h, flag.p, sizeof(h), cudaMemcpyDeviceToHost, s));
    VJ_CUDA(cudaStreamSynchronize(s));
    flag.free_(s);
    const double mx = (double)h[1];
    ix->bf16_exact = !cosine && h[0] == 0 && mx <= 256.0 && (double)ix->d * mx * mx <= 8388608.0;
    ix->bf16_lossless = h[2] == 0;
    ix->cos_raw = cosine && wide && ix->bf16_lossless;
    // every node (data rows first): scans read the data rows, the kNN build all
    ix->xbf.ensure((size_t)ix->n * kp, s);
    k_to_bf16<<<vj_div_up(ix->n * kp, 256), 256, 0, s>>>(ix->vec.p, ix->dp, ix->d, nullptr, 0, ix->n, kp, 1.f,
                                                          (cosine && !ix->cos_raw) ? ix->invn.p : nullptr, ix->xbf.p);
    VJ_LAUNCH_CHECK();
    // |key_bf16 - key| <= cb |a||b| + c3 (|a|^2 + |b|^2) with
    //   L2:     cb = 4ub + 2ub^2 + 2 kp 2^-23 + 4u, c3 = 3u
    //   cosine: cb = 2ub + ub^2 + 2 kp 2^-23 + 8u (unit rows), c3 = 0
    // (ub = 2^-8 BF16, u = 2^-24 FP32), each with a 1.25 margin.  Inputs that
    // are exactly BF16 drop the ub terms (L2 rows, and cosine raw rows whose
    // norms are applied in FP32 after the accumulation).
    const double ub = 1.0 / 256.0, u = VJ_F32_U;
    if (!cosine) {
        const double in_round = ix->bf16_lossless ? 0.0 : 4 * ub + 2 * ub * ub;
        ix->tc_cb = (float)(1.25 * (in_round + 2.0 * kp * 2 * u + 4 * u));
        ix->tc_c3 = (float)(1.25 * 3 * u);
        if (ix->bf16_exact) {
            ix->tc_cb = 0.f;  // exact integer keys (see above)
            ix->tc_c3 = 0.f;
        }
        // row-independent form: cbmax >= cb |a| for every row
        ix->tc_cbmax = (float)(ix->tc_cb * ix->maxnorm * 1.0001);
        if (!wide) {
            ix->xbias.ensure((size_t)ix->n * 16, s);
            k_bias_split<<<vj_div_up(ix->n, 256), 256, 0, s>>>(ix->sqn.p, ix->n, (double)ix->tc_c3,
                                                                 (double)ix->tc_cbmax, ix->xbias.p);
            VJ_LAUNCH_CHECK();
            ix->abias.ensure(128 * 16, s);
            k_fill_abias<<<vj_div_up(128 * 16, 256), 256, 0, s>>>(ix->abias.p);
            VJ_LAUNCH_CHECK();
        }
    } else {
        const double in_round = ix->cos_raw ? 0.0 : 2 * ub + ub * ub;
        ix->tc_cb = (float)(1.25 * (in_round + 2.0 * kp * 2 * u + 8 * u));
        ix->tc_c3 = 0.f;
        ix->tc_cbmax = 0.f;
    }
    if (wide) {
        ix->wcs.ensure(ix->n, s);
        ix->wcb.ensure(ix->n, s);
        k_wide_cols<<<vj_div_up(ix->n, 256), 256, 0, s>>>(ix->sqn.p, ix->invn.p, ix->n,
                                                            !cosine ? 0 : (ix->cos_raw ? 1 : 2), (double)ix->tc_c3,
                                                            (double)ix->tc_cbmax, ix->wcs.p, ix->wcb.p);
        VJ_LAUNCH_CHECK();
    }
}

void vj_ensure_bf16(vj_index* ix) { ensure_data_bf16(ix); }

// E4M3 row bytes: d rounded up to 32 columns (one K step), at least one 128-byte box
static int f8_row_bytes(int d) { return d <= 128 ? 128 : (d + 31) / 32 * 32; }

// TF32 rows of every node and the kNN sweeps' measured-bound columns (rows
// wider than 128 columns whose coordinates are not BF16 values).  TF32 keeps
// 11 significant bits: the bound is then far inside the spread of a row's
// nearest keys, which the certificate of the kNN lists needs.
static void ensure_knn_tf32(vj_index* ix) {
    cudaStream_t s = ix->stream;
    const int64_t n = ix->n;
    const int kp32 = (ix->d + 31) / 32 * 32;
    const int cosine = ix->metric != VJ_L2 ? 1 : 0;
    ix->xtf.ensure((size_t)n * kp32, s);
    ix->xerr_tf.ensure(n, s);
    ix->kcs.ensure(n, s);
    ix->kcb.ensure(n, s);
    DBuf<unsigned int> q;
    q.alloc(3, s);
    VJ_CUDA(cudaMemsetAsync(q.p, 0, 3 * sizeof(unsigned int), s));
    k_tile_rows<KIND_TF32><<<vj_div_up(n * 32, 256), 256, 0, s>>>(ix->vec.p, ix->sqn64.p, ix->dp, ix->d, cosine,
                                                                  nullptr, n, kp32, nullptr, ix->xtf.p, nullptr,
                                                                  ix->xerr_tf.p, q.p + 1, q.p + 2);
    VJ_LAUNCH_CHECK();
    // TF32 products are exact in FP32 (11 x 11 significant bits); the FP32
    // sum of kp32 of them: 2 kp32 2^-24 of the sum of magnitudes
    const double gamma = (double)(kp32 + 16) * 2.0 * (double)VJ_F32_U;
    k_tile_cols<<<vj_div_up(n, 256), 256, 0, s>>>(ix->sqn64.p, ix->xerr_tf.p, nullptr, n, cosine, 0, q.p, gamma,
                                                   ix->kcs.p, ix->kcb.p);
    VJ_LAUNCH_CHECK();
    unsigned int h[3];
    VJ_CUDA(cudaMemcpyAsync(h, q.p, sizeof(h), cudaMemcpyDeviceToHost, s));
    VJ_CUDA(cudaStreamSynchronize(s));
    q.free_(s);
    float fd, fa;
    memcpy(&fd, &h[1], 4);
    memcpy(&fa, &h[2], 4);
    const double Da = fd, A = fa;
    // |tile key - key| for any pair: L2 2 (2 Da A + Da^2 + gamma (A + Da)^2); cosine (unit rows) the same with A = 1
    const double beta = 2.0 * Da * A + Da * Da + gamma * (A + Da) * (A + Da);
    ix->knn_beta = cosine ? beta : 2.0 * beta;
    ix->knn_measured = true;
}

// Data side of the measured-bound scan (built once per index): the FP8 rows
// with their scales and error norms, or the error norms of the BF16 rows.
static void ensure_scan_data(vj_index* ix, bool f8) {
    cudaStream_t s = ix->stream;
    const int cosine = ix->metric != VJ_L2 ? 1 : 0;
    const int warps_grid = vj_div_up(ix->nx * 32, 256);
    if (f8) {
        const int kb8 = f8_row_bytes(ix->d);
        if (ix->kb8 == kb8 && ix->x8.n >= (size_t)ix->nx * kb8) return;
        ix->kb8 = kb8;
        ix->x8.ensure((size_t)ix->nx * kb8, s);
        ix->x8rs.ensure(ix->nx, s);
        ix->x8err.ensure(ix->nx, s);
        k_tile_rows<KIND_E4M3><<<warps_grid, 256, 0, s>>>(ix->vec.p, ix->sqn64.p, ix->dp, ix->d, cosine, nullptr, ix->nx,
                                                  kb8, nullptr, ix->x8.p, ix->x8rs.p, ix->x8err.p, nullptr, nullptr);
        VJ_LAUNCH_CHECK();
    } else {
        if (ix->xerr_bf.n >= (size_t)ix->nx) return;
        const int kp = (ix->d + TC_BK - 1) / TC_BK * TC_BK;
        ix->xerr_bf.ensure(ix->nx, s);
        // the data rows are the first nx rows of the BF16 copy
        k_tile_rows<KIND_BF16><<<warps_grid, 256, 0, s>>>(ix->vec.p, ix->sqn64.p, ix->dp, ix->d, cosine, nullptr, ix->nx,
                                                  kp, nullptr, ix->xbf.p, nullptr, ix->xerr_bf.p, nullptr, nullptr);
        VJ_LAUNCH_CHECK();
    }
}

// Work split of a sweep of nrt row tiles over nct tiles: the tiles per unit
// that minimise the busiest SM's load (its units' tiles plus `refill` tiles of
// pipeline restart per unit)
static int best_tiles_per_unit(int64_t nrt, int64_t nct, int num_sms, int64_t refill) {
    const int64_t g = std::max(1, num_sms);
    int64_t best = INT64_MAX;
    int best_tpu = (int)nct;
    for (int64_t ncc = 1; ncc <= nct; ncc++) {
        const int64_t tpu = (nct + ncc - 1) / ncc;
        if (ncc > 1 && (nct + tpu - 1) / tpu != ncc) continue;  // same split as a smaller ncc
        const int64_t load = ((nrt * ncc + g - 1) / g) * (tpu + refill);
        if (load < best) {
            best = load;
            best_tpu = (int)tpu;
        }
    }
    return best_tpu;
}

static size_t wide_smem() { return sizeof(WdSmem) + 1024; }

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
    const bool f8 = ix->p.scan == VJ_PREC_FP8;
    // kp <= 128: resident query rows and the bias step; wider rows, and FP8
    // tiles, stream both operands through the ring
    const bool resident = !f8 && kp <= RS_MAX_KB * TC_BK;
    // FP8 tiles, and BF16 tiles of inputs that are not BF16 values, take the
    // measured rounding bound (each row's own rounding error)
    const bool measured = f8 || (!resident && !ix->bf16_lossless);
    const int kb8 = f8_row_bytes(ix->d);
    DBuf<__nv_bfloat16> abf;
    DBuf<uint8_t> a8;
    DBuf<int32_t> aid, anode;
    DBuf<float> an, mcs, mcb;
    DBuf<unsigned int> qmax;
    if (f8) a8.alloc((size_t)nr * kb8, s);
    else abf.alloc((size_t)nr * kp, s);
    aid.alloc(nr, s);
    anode.alloc(nr, s);
    an.alloc(nr, s);
    k_query_rows<<<vj_div_up(nr, 256), 256, 0, s>>>(qrows, nr, (int32_t)ix->nx, aid.p, anode.p);
    VJ_LAUNCH_CHECK();
    const int32_t* arow = anode.p;
    // query rows: L2 scaled by 2 for the resident form (2<a,b> + bias), cosine
    // unit rows (raw rows for the streamed kernel on BF16-exact inputs)
    const float ascale = (!cosine && resident) ? 2.f : 1.f;
    if (!f8) {
        k_to_bf16<<<vj_div_up(nr * kp, 256), 256, 0, s>>>(ix->vec.p, ix->dp, ix->d, arow, 0, nr, kp, ascale,
                                                          (cosine && !ix->cos_raw) ? ix->invn.p : nullptr, abf.p);
        VJ_LAUNCH_CHECK();
    }
    const float eps_key = cosine ? eps : eps * eps;
    if (measured) {
        ensure_scan_data(ix, f8);
        // qmax: largest |coordinate| (FP8: the shared scale), largest |da| and |a| of the scanned rows
        qmax.alloc(3, s);
        VJ_CUDA(cudaMemsetAsync(qmax.p, 0, 3 * sizeof(unsigned int), s));
        const int wg = vj_div_up(nr * 32, 256);
        const int ci = cosine ? 1 : 0;
        if (f8) {
            k_tile_amax<<<wg, 256, 0, s>>>(ix->vec.p, ix->sqn64.p, ix->dp, ix->d, ci, arow, nr, qmax.p);
            VJ_LAUNCH_CHECK();
            k_tile_rows<KIND_E4M3><<<wg, 256, 0, s>>>(ix->vec.p, ix->sqn64.p, ix->dp, ix->d, ci, arow, nr, kb8, qmax.p, a8.p,
                                              nullptr, nullptr, qmax.p + 1, qmax.p + 2);
        } else {
            k_tile_rows<KIND_BF16><<<wg, 256, 0, s>>>(ix->vec.p, ix->sqn64.p, ix->dp, ix->d, ci, arow, nr, kp, nullptr, abf.p,
                                              nullptr, nullptr, qmax.p + 1, qmax.p + 2);
        }
        VJ_LAUNCH_CHECK();
        // gamma: the accumulation of the exact products.  BF16: FP32 sums of
        // kp terms, 2 kp 2^-24 of the sum of magnitudes (any order).  FP8: the
        // tensor core's precision inside one K = 32 step is not documented;
        // with at least 13 bits kept per aligned addend a step loses at most
        // 32 2^-13 = 2^-8 of its largest product, plus the FP32 sum of steps
        const double gamma = f8 ? (1.0 / 256.0 + (double)(kb8 / 32 + 16) * 2.0 * (double)VJ_F32_U)
                                : (double)(kp + 16) * 2.0 * (double)VJ_F32_U;
        mcs.alloc(ix->nx, s);
        mcb.alloc(ix->nx, s);
        k_tile_cols<<<vj_div_up(ix->nx, 256), 256, 0, s>>>(ix->sqn64.p, f8 ? ix->x8err.p : ix->xerr_bf.p,
                                                            f8 ? ix->x8rs.p : nullptr, ix->nx, ci, f8 ? 1 : 0,
                                                            qmax.p, gamma, mcs.p, mcb.p);
        VJ_LAUNCH_CHECK();
        k_tile_thr<<<vj_div_up(nr, 256), 256, 0, s>>>(ix->sqn64.p, arow, nr, ci, (double)eps_key, ix->maxnorm, an.p);
    } else if (ix->cos_raw) {
        k_row_thr_raw<<<vj_div_up(nr, 256), 256, 0, s>>>(ix->invn.p, arow, nr, kp, eps_key, ix->tc_cb, an.p);
    } else {
        k_row_thr<<<vj_div_up(nr, 256), 256, 0, s>>>(ix->sqn.p, arow, nr, ix->metric, kp, eps_key, ix->tc_cb,
                                                      ix->tc_c3, ix->tc_cbmax, ix->maxnorm, an.p);
    }
    VJ_LAUNCH_CHECK();

    DBuf<unsigned long long> ctr;
    DBuf<int> err;
    DBuf<float> rn_rows, cw;
    ctr.alloc(1, s);
    err.alloc(1, s);
    const long long spin_limit = 1ll << 22;  // try_wait polls; seconds at most, then an error
    std::function<void()> launch;
    CUtensorMap ta, tb, tab, tbb;
    RsParams R{};
    WdParams W{};
    // integer inputs (exact BF16 products and FP32 sums): the scan hands out
    // each candidate's exact key, and no re-check from the vectors is needed
    const bool want_keys = ck && !cosine && ix->bf16_exact && !f8;
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
        R.tpu = best_tiles_per_unit(R.nrp, R.nct, ix->num_sms, 3);
        R.nunits = R.nrp * (int)vj_div_up(R.nct, R.tpu);
        // ring stages of one data tile each, within 227 KB of shared memory
        const size_t fixed = 2048 + RS_BBOX + 2 * (size_t)R.nkb * RS_BOX;
        const size_t per = (size_t)R.nkb * RS_BOX + RS_BBOX;
        R.stages = (int)std::min<size_t>(RS_MAX_STAGES, (232448 - fixed) / per);
        R.a_thr = an.p;
        R.a_ids = aid.p;
        R.tstride = 1;
        if (want_keys) {
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
        if (f8) {
            ta = make_map_u8(a8.p, nr, kb8, WD_BM);
            tb = make_map_u8(ix->x8.p, ix->nx, kb8, WD_BN);
            W.nkb = (kb8 + 127) / 128;
            W.kk_last = (ix->d + 31) / 32 - 4 * (W.nkb - 1);
        } else {
            ta = make_map(abf.p, nr, kp, WD_BM);
            tb = make_map(ix->xbf.p, ix->nx, kp, WD_BN);
            W.nkb = kp / TC_BK;
            W.kk_last = 0;
        }
        W.nrows = nr;
        W.ncols = ix->nx;
        W.nrt = (int)vj_div_up(nr, WD_BM);
        W.nct = (int)vj_div_up(ix->nx, WD_BN);
        W.tstride = 1;
        W.tpu = best_tiles_per_unit(W.nrt, W.nct, ix->num_sms, 1);
        W.nunits = W.nrt * (int)vj_div_up(W.nct, W.tpu);
        W.cs = measured ? mcs.p : ix->wcs.p;  // data rows are the first nx nodes
        W.cb = measured ? mcb.p : ix->wcb.p;
        W.thr = an.p;
        W.a_ids = aid.p;
        W.ncand = ctr.p;
        W.err = err.p;
        W.spin_limit = spin_limit;
        const size_t smem = wide_smem();
        const int grid = std::min(W.nunits, ix->num_sms);
        if (f8) {
            VJ_CUDA(cudaFuncSetAttribute(k_tc_wide<EPI_SCAN, KIND_E4M3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem));
            launch = [&, grid, smem]() { k_tc_wide<EPI_SCAN, KIND_E4M3><<<grid, WD_THREADS, smem, s>>>(ta, tb, W); };
        } else {
            VJ_CUDA(cudaFuncSetAttribute(k_tc_wide<EPI_SCAN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem));
            launch = [&, grid, smem]() { k_tc_wide<EPI_SCAN><<<grid, WD_THREADS, smem, s>>>(ta, tb, W); };
        }
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
        W.cq = R.cq = cq.p;
        W.cx = R.cx = cx.p;
        if (want_keys) {
            ck->ensure(cap, s);
            if (resident) R.ck = ck->p;
            else {
                cw.ensure(cap, s);
                W.cw = cw.p;
            }
        }
        W.cap = R.cap = (int64_t)cq.n;
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
    if (want_keys && !resident && hn > 0) {
        k_key_from_w<<<vj_div_up((int64_t)hn, 256), 256, 0, s>>>(ix->sqn.p, cq.p, cx.p, cw.p, (int64_t)hn, ix->nx,
                                                                ck->p);
        VJ_LAUNCH_CHECK();
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (ms_out) *ms_out = ms;
    ix->last_scan_exact_keys = want_keys;
    abf.free_(s);
    a8.free_(s);
    mcs.free_(s);
    mcb.free_(s);
    qmax.free_(s);
    aid.free_(s);
    an.free_(s);
    anode.free_(s);
    rn_rows.free_(s);
    cw.free_(s);
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

__global__ void k_iota(int32_t* __restrict__ v, int64_t n, int64_t base = 0) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = (int32_t)(base + i);
}

__global__ void k_pair_count(const int32_t* __restrict__ cq, int64_t nc, int32_t* __restrict__ counts) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < nc && cq[e] >= 0) atomicAdd(counts + cq[e], 1);  // -1: a hole
}

__global__ void k_pair_scatter(const int32_t* __restrict__ cq, const int32_t* __restrict__ cx,
                               const float* __restrict__ cw, int64_t nc, const int64_t* __restrict__ off,
                               int32_t* __restrict__ cursor, int32_t* __restrict__ ids, float* __restrict__ wv) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nc) return;
    const int q = cq[e];
    if (q < 0) return;  // a hole
    const int64_t pos = off[q] + atomicAdd(cursor + q, 1);
    ids[pos] = cx[e];
    if (wv) wv[pos] = cw[e];
}

// true-key lower bound of every node a row did not list (accumulator <= thr;
// for cosine raw rows the tile value is acc / |b|)
__global__ void k_knn_bound(const float* __restrict__ sqn, const float* __restrict__ invn,
                            const float* __restrict__ thr_acc, int64_t n, int metric, int raw, int kp, float cb,
                            float c3, float cbmax, double maxnorm, float* __restrict__ thr) {
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
    } else if (raw) {
        thr[i] = (float)(1.0 - (double)ta * (double)invn[i] - (double)cb - 3.0 * g);
    } else {
        thr[i] = (float)(1.0 - (double)ta - (double)cb - 3.0 * g);
    }
}

bool vj_tc_knn_candidates(vj_index* ix, DBuf<int64_t>& off, DBuf<int32_t>& ids, DBuf<float>& row_thr,
                          DBuf<float>* cw_out) {
    const int kpad = (ix->d + TC_BK - 1) / TC_BK * TC_BK;
    const int64_t n = ix->n, nx = ix->nx;
    // blocks of (rows, candidate columns) by the index's kNN mode; a block
    // whose rows are its columns is symmetric
    struct Blk {
        int64_t r0, nr, c0, nc;
    };
    std::vector<Blk> blks;
    if (ix->knn_mode == VJ_KNN_ALL) {
        blks.push_back(Blk{0, n, 0, n});
    } else {
        blks.push_back(Blk{0, nx, 0, nx});
        if (ix->knn_mode == VJ_KNN_DATA) blks.push_back(Blk{nx, n - nx, 0, nx});
        else blks.push_back(Blk{nx, n - nx, nx, n - nx});
    }
    for (const Blk& b : blks)
        if (b.nr > 0 && b.nc < 4096) return false;  // too few tiles to sample: the SIMT sweep
    const bool wide = kpad > RS_MAX_KB * TC_BK;
    cudaStream_t s = ix->stream;
    ensure_data_bf16(ix);
    const bool cosine = ix->metric != VJ_L2;
    DBuf<__nv_bfloat16> abf;
    DBuf<float> top, thr, cw;
    DBuf<int32_t> iota;
    std::vector<DBuf<int4>> units(blks.size());
    DBuf<int> err;
    DBuf<unsigned long long> ctr;
    top.alloc(n, s);
    thr.alloc(n, s);
    err.alloc(1, s);
    ctr.alloc(1, s);
    VJ_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
    const long long spin_limit = 1ll << 22;
    DBuf<int32_t>& cq = ix->scan_cq;
    DBuf<int32_t>& cx = ix->scan_cx;
    // expected candidates per row: the sample list length times the sampling stride
    const int64_t per_row = (int64_t)(wide ? WD_TOP : 16) * KNN_SAMPLE;
    int64_t cap = std::max<int64_t>(cq.n, n * (per_row + per_row / 4) + (1 << 20));
    unsigned long long hn = 0;
    int herr = 0;
    // the candidate sweep, re-run with larger lists when they overflow
    auto sweep = [&](const std::function<void(int32_t*, int32_t*, float*, int64_t)>& launch) {
        for (int attempt = 0; attempt < 3; attempt++) {
            cq.ensure(cap, s);
            cx.ensure(cap, s);
            if (wide && cw_out) cw.ensure(cap, s);
            VJ_CUDA(cudaMemsetAsync(ctr.p, 0, sizeof(unsigned long long), s));
            launch(cq.p, cx.p, (wide && cw_out) ? cw.p : nullptr, (int64_t)cq.n);
            VJ_LAUNCH_CHECK();
            VJ_CUDA(cudaMemcpyAsync(&hn, ctr.p, sizeof(hn), cudaMemcpyDeviceToHost, s));
            VJ_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
            VJ_CUDA(cudaStreamSynchronize(s));
            VJ_REQUIRE(herr == 0, VJ_ERR_TIMEOUT, "tensor-core kNN: a pipeline wait timed out");
            if ((int64_t)hn <= (int64_t)cq.n) break;
            cap = (int64_t)hn + (int64_t)hn / 4 + RS_HOLE_SLACK;  // the next launch may leave other holes
        }
        VJ_REQUIRE((int64_t)hn <= (int64_t)cq.n, VJ_ERR_STATE, "tensor-core kNN: candidate list still too small");
    };

    if (!wide) {
        abf.alloc((size_t)n * kpad, s);
        iota.alloc(n, s);
        k_to_bf16<<<vj_div_up(n * kpad, 256), 256, 0, s>>>(ix->vec.p, ix->dp, ix->d, nullptr, 0, n, kpad,
                                                          cosine ? 1.f : 2.f, cosine ? ix->invn.p : nullptr, abf.p);
        k_iota<<<vj_div_up(n, 256), 256, 0, s>>>(iota.p, n);
        VJ_LAUNCH_CHECK();
        const int nkb = kpad / TC_BK;
        const size_t fixed = 2048 + RS_BBOX + 2 * (size_t)nkb * RS_BOX;
        const size_t per = (size_t)nkb * RS_BOX + RS_BBOX;
        const int stages = (int)std::min<size_t>(RS_MAX_STAGES, (232448 - fixed) / per);
        const size_t smem = fixed + per * (size_t)stages;
        // the block's A rows (node ids r0 ..) against its B rows (node ids c0 ..)
        struct RsBlk {
            CUtensorMap ta, tab, tb, tbb;
            RsParams R;
            int nct_all;
        };
        std::vector<RsBlk> rb;
        for (const Blk& b : blks) {
            if (b.nr <= 0) continue;
            RsBlk x;
            x.ta = make_map(abf.p + (size_t)b.r0 * kpad, b.nr, kpad, 128);
            x.tb = make_map(ix->xbf.p + (size_t)b.c0 * kpad, b.nc, kpad, RS_BN);
            x.tab = cosine ? x.ta : make_map16(ix->abias.p, 128, 128);
            x.tbb = cosine ? x.tb : make_map16(ix->xbias.p + (size_t)b.c0 * 16, b.nc, RS_BN);
            RsParams& R = x.R;
            R = RsParams{};
            R.nrows = b.nr;
            R.ncols = b.nc;
            R.nkb = nkb;
            R.bias = cosine ? 0 : 1;
            R.nrp = (int)vj_div_up(b.nr, 256);
            R.stages = stages;
            R.err = err.p;
            R.spin_limit = spin_limit;
            R.row_base = b.r0;
            R.col_base = b.c0;
            R.a_ids = iota.p + b.r0;
            x.nct_all = (int)vj_div_up(b.nc, RS_BN);
            rb.push_back(x);
        }
        // 1. sample sweep: one unit per 256-row block over every KNN_SAMPLE-th tile
        VJ_CUDA(cudaFuncSetAttribute(k_tc_res<EPI_SAMPLE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        for (RsBlk& x : rb) {
            RsParams R = x.R;
            R.tstride = KNN_SAMPLE;
            R.nct = (x.nct_all + KNN_SAMPLE - 1) / KNN_SAMPLE;
            R.tpu = R.nct;
            R.nunits = R.nrp;
            R.top16 = top.p + R.row_base;
            k_tc_res<EPI_SAMPLE><<<std::min(R.nunits, ix->num_sms), (2 + KN_EPI) * 32, smem, s>>>(x.ta, x.tab, x.tb,
                                                                                              x.tbb, R);
            VJ_LAUNCH_CHECK();
        }
        k_knn_thr<<<vj_div_up(n, 256), 256, 0, s>>>(top.p, n, thr.p);
        VJ_LAUNCH_CHECK();

        // 2. candidate sweep over every tile, rows are node ids
        for (RsBlk& x : rb) {
            RsParams& R = x.R;
            R.tstride = 1;
            R.nct = x.nct_all;
            R.tpu = best_tiles_per_unit(R.nrp, R.nct, ix->num_sms, 3);
            R.nunits = R.nrp * (int)vj_div_up(R.nct, R.tpu);
            R.a_thr = thr.p + R.row_base;
            R.ncand = ctr.p;
        }
        VJ_CUDA(cudaFuncSetAttribute(k_tc_res<EPI_SCAN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        sweep([&](int32_t* pq, int32_t* px, float*, int64_t c) {
            for (RsBlk& x : rb) {
                RsParams R = x.R;
                R.cq = pq;
                R.cx = px;
                R.cap = c;
                k_tc_res<EPI_SCAN><<<std::min(R.nunits, ix->num_sms), RS_THREADS, smem, s>>>(x.ta, x.tab, x.tb,
                                                                                          x.tbb, R);
            }
        });
    } else {
        // streamed tiles: A and B are the BF16 copies of the block's rows and
        // columns, or their TF32 copies with the measured bound when the
        // coordinates are not BF16 values
        const bool tf32 = !ix->bf16_lossless;
        const int kp32 = (ix->d + 31) / 32 * 32;
        ix->knn_measured = false;
        if (tf32) ensure_knn_tf32(ix);
        const size_t smem = wide_smem();
        struct WdBlk {
            CUtensorMap ta, tb;
            WdParams W;
            int nct_all;
        };
        std::vector<WdBlk> wb;
        for (const Blk& b : blks) {
            if (b.nr <= 0) continue;
            WdBlk x;
            WdParams& W = x.W;
            W = WdParams{};
            if (tf32) {
                x.ta = make_map_f32(ix->xtf.p + (size_t)b.r0 * kp32, b.nr, kp32, WD_BM);
                x.tb = make_map_f32(ix->xtf.p + (size_t)b.c0 * kp32, b.nc, kp32, WD_BN);
                W.nkb = kp32 / 32;
                W.kk_last = (ix->d + 7) / 8 - 4 * (W.nkb - 1);
                W.cs = ix->kcs.p + b.c0;
                W.cb = ix->kcb.p + b.c0;
            } else {
                x.ta = make_map(ix->xbf.p + (size_t)b.r0 * kpad, b.nr, kpad, WD_BM);
                x.tb = make_map(ix->xbf.p + (size_t)b.c0 * kpad, b.nc, kpad, WD_BN);
                W.nkb = kpad / TC_BK;
                W.cs = ix->wcs.p + b.c0;
                W.cb = ix->wcb.p + b.c0;
            }
            W.nrows = b.nr;
            W.ncols = b.nc;
            W.nrt = (int)vj_div_up(b.nr, WD_BM);
            W.err = err.p;
            W.spin_limit = spin_limit;
            W.row_base = b.r0;
            W.col_base = b.c0;
            x.nct_all = (int)vj_div_up(b.nc, WD_BN);
            wb.push_back(x);
        }
        // 1. sample sweep: one unit per 128-row tile over every KNN_SAMPLE-th tile
        VJ_CUDA(cudaFuncSetAttribute(k_tc_wide<EPI_SAMPLE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        VJ_CUDA(cudaFuncSetAttribute(k_tc_wide<EPI_SAMPLE, KIND_TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
        for (WdBlk& x : wb) {
            WdParams W = x.W;
            W.tstride = KNN_SAMPLE;
            W.nct = (x.nct_all + KNN_SAMPLE - 1) / KNN_SAMPLE;
            W.tpu = W.nct;
            W.nunits = W.nrt;
            W.top16 = top.p + W.row_base;
            const int grid = std::min(W.nunits, ix->num_sms);
            if (tf32) k_tc_wide<EPI_SAMPLE, KIND_TF32><<<grid, WD_THREADS, smem, s>>>(x.ta, x.tb, W);
            else k_tc_wide<EPI_SAMPLE><<<grid, WD_THREADS, smem, s>>>(x.ta, x.tb, W);
            VJ_LAUNCH_CHECK();
        }
        k_knn_thr<<<vj_div_up(n, 256), 256, 0, s>>>(top.p, n, thr.p);
        VJ_LAUNCH_CHECK();
        // 2. candidate sweep, rows are node ids.  A symmetric block (its rows
        // are its columns) has symmetric Gram tiles: row tile rt visits the B
        // tiles from its own 256-row block on (ct >= rt / 2), and tiles past
        // that block test both directions.  Units: a row tile's run of tpu
        // tiles, ordered by first tile so the units running together walk the
        // same B tiles (and the longest runs, of the first row tiles, start
        // first).  Other blocks sweep every B tile, row tile fastest.
        for (size_t k = 0; k < wb.size(); k++) {
            WdBlk& x = wb[k];
            WdParams& W = x.W;
            const int nct_all = x.nct_all;
            W.tstride = 1;
            W.nct = nct_all;
            W.thr = thr.p + W.row_base;
            W.a_ids = nullptr;
            W.ncand = ctr.p;
            if (W.row_base == W.col_base && W.nrows == W.ncols) {
                int64_t tiles = 0;
                for (int rt = 0; rt < W.nrt; rt++) tiles += nct_all - (rt >> 1);
                const int64_t tpu =
                    std::min<int64_t>(nct_all, std::max<int64_t>(64, tiles / (8 * (int64_t)ix->num_sms)));
                std::vector<int4> hu;
                for (int rt = 0; rt < W.nrt; rt++)
                    for (int64_t t0 = rt >> 1; t0 < nct_all; t0 += tpu)
                        hu.push_back(make_int4(rt, (int)t0, (int)std::min<int64_t>(nct_all, t0 + tpu), 0));
                std::stable_sort(hu.begin(), hu.end(), [](const int4& a, const int4& b) { return a.y < b.y; });
                units[k].alloc(hu.size(), s);
                VJ_CUDA(cudaMemcpyAsync(units[k].p, hu.data(), hu.size() * sizeof(int4), cudaMemcpyHostToDevice, s));
                W.units = units[k].p;
                W.nunits = (int)hu.size();
            } else {
                W.units = nullptr;
                W.tpu = (int)std::min<int64_t>(
                    nct_all, std::max<int64_t>(64, (int64_t)W.nrt * nct_all / (8 * (int64_t)ix->num_sms)));
                W.nunits = W.nrt * (int)vj_div_up(nct_all, W.tpu);
            }
        }
        VJ_CUDA(cudaFuncSetAttribute(k_tc_wide<EPI_SCAN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        VJ_CUDA(cudaFuncSetAttribute(k_tc_wide<EPI_SCAN, KIND_TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
        sweep([&](int32_t* pq, int32_t* px, float* pw, int64_t c) {
            for (WdBlk& x : wb) {
                WdParams W = x.W;
                W.cq = pq;
                W.cx = px;
                W.cw = pw;
                W.cap = c;
                const int grid = std::min(W.nunits, ix->num_sms);
                if (tf32) k_tc_wide<EPI_SCAN, KIND_TF32><<<grid, WD_THREADS, smem, s>>>(x.ta, x.tb, W);
                else k_tc_wide<EPI_SCAN><<<grid, WD_THREADS, smem, s>>>(x.ta, x.tb, W);
            }
        });
        ix->xtf.free_(s);  // the TF32 rows serve the two sweeps only
    }
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
    const bool with_w = wide && cw_out;
    if (with_w) cw_out->ensure(std::max<int64_t>(nc, 1), s);
    if (nc > 0)
        k_pair_scatter<<<vj_div_up(nc, 256), 256, 0, s>>>(cq.p, cx.p, with_w ? cw.p : nullptr, nc, off.p, cursor.p,
                                                          ids.p, with_w ? cw_out->p : nullptr);
    VJ_LAUNCH_CHECK();
    row_thr.ensure(n, s);
    // measured bound: a node left out has v = 2<a^,b^> - |b|^2 + 2 beta_b <= thr (L2), so its
    // key is at least |a|^2 - thr (cosine: 1 - thr); the BF16 form carries its bound constants
    if (ix->knn_measured)
        k_knn_bound<<<vj_div_up(n, 256), 256, 0, s>>>(ix->sqn.p, ix->invn.p, thr.p, n, ix->metric, 0, kpad, 0.f, 0.f,
                                                      0.f, ix->maxnorm, row_thr.p);
    else
        k_knn_bound<<<vj_div_up(n, 256), 256, 0, s>>>(ix->sqn.p, ix->invn.p, thr.p, n, ix->metric,
                                                      ix->cos_raw ? 1 : 0, kpad, ix->tc_cb, ix->tc_c3, ix->tc_cbmax,
                                                      ix->maxnorm, row_thr.p);
    VJ_LAUNCH_CHECK();
    if (wide) {
        // build-sized lists (hundreds of candidates per node) are not kept for later scans
        cq.free_(s);
        cx.free_(s);
    }
    counts.free_(s);
    cursor.free_(s);
    abf.free_(s);
    top.free_(s);
    thr.free_(s);
    cw.free_(s);
    iota.free_(s);
    for (auto& u : units) u.free_(s);
    err.free_(s);
    ctr.free_(s);
    return true;
}
