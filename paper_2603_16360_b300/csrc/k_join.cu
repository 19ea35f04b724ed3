// k_join.cu -- the online merged-index join (Alg. 1 with Alg. 3-8), one warp
// per query, persistent grid fed by a device ready queue.
//
// Per query q (merged node id qn = nx + qi), following Alg. 1's order:
//   Seed (Alg. 3)      S = {entry} (+ C[parent] under soft sharing) (+ q for
//                      self/soft sharing on the merged index).
//   Greedy (Alg. 4-5)  distances to S; StopGreedy on the front: stop if it is
//                      an in-range data node, if conv_threshold <= 0, or if it
//                      is not q (merged rule); otherwise pop q and evaluate its
//                      whole neighbourhood N(q).  The merged rule then stops the
//                      walk, so the greedy phase is exactly this probe.
//   CheckHybrid (6)    adapt: OOD iff d1/d2 > 1.5 (Sec. 4.4) from the probe's
//                      distances and the stored data-edge lengths.
//   Expansion (Alg. 7) non-hybrid: the in-range data closure of the probe's
//                      in-range points; its result and its visited set do not
//                      depend on pop order, so it runs frontier-parallel
//                      (several nodes' neighbour lists per batch).  Hybrid:
//                      exact pop order (in-range points first, then the
//                      bounded out-range queue, (key, id) order).  The
//                      insert-then-trim rule is applied per neighbour list as a
//                      batch: the queue after a list equals the k smallest of
//                      (queue U list's out-range nodes), k given by the size
//                      recurrence of the per-insert rule (each trim removes the
//                      current maximum, so no removed key can be smaller than a
//                      kept one).
//   UpdateCache (8)    C[q] = closest visited data node, ties by id, FP64
//                      re-decided among FP32 near-ties.
//
// Work sharing (soft) runs in three launches over the queries:
//   pass 1  every query, hybrid ones included, runs on the seeds {entry, q}
//           without waiting for its parent (longest-first order);
//   pass 2  in parallel, each query decides what C[parent] as pass 1 left it
//           changes.  V, I and the BFS closure are sets, and V is
//           {entry, q} U N(q) U (data neighbours of every result), so:
//             - C[parent] in V: nothing changes;
//             - C[parent] new and out of range: one more visited node, the
//               cache becomes the (dist, id) minimum of the two (FP64);
//             - C[parent] new and in range, a duplicate of q that would have
//               been the greedy front, or a hybrid query (its expansion
//               depends on the order of its seeds): the query re-runs with
//               the seed from the start; the re-run is staged.
//   pass 3  in MST BFS order (parents first), each query waits (bounded
//           acquire spin) for its parent's final cache; when that is the seed
//           pass 2 decided for, pass 2's outcome is committed, otherwise the
//           query decides again.  It then publishes C[q] (release store of
//           its done flag).
// The result, visited count and cache equal those of the wait-first order.
//
// Visited set: open-addressing hash in shared memory (HCAP slots); past half
// of it a query switches to its warp's global bitmap over all nodes (cleared
// from the list of set ids when the query ends).  Results: shared-memory
// list (RCAP) spilling to global memory.
// In-range decisions whose FP32 key lies within the FP32 rounding bound of eps
// are re-decided in FP64.
#include <float.h>
#include <mutex>
#include <stdio.h>
#include <string.h>

#include "vj_device.cuh"
#include "vj_internal.cuh"

namespace {

constexpr int WPB = 8;      // warps per block
constexpr int HCAP = 2048;  // shared-memory visited slots per warp
constexpr int RCAP = 256;   // shared-memory result slots per warp
constexpr int CCAP = 128;   // candidate slots per batch
constexpr int FB = 4;       // frontier nodes per BFS batch (FB * 32 <= CCAP)
constexpr int GCAP0 = 8192; // first global visited table
constexpr int OQS = 64;     // out-range queue slots per buffer kept in shared memory
// wide rows: two blocks (16 warps) per SM, registers capped at 128 -- the
// gathers are latency-bound, so resident warps matter more than the few
// registers spilled; narrow rows fit two blocks uncapped
#define JOIN_MIN_BLOCKS(NPL, U) ((NPL) * (U) >= 12 ? 2 : 1)

struct WarpSmem {
    int nlist;  // bitmap mode: ids listed in the warp's space
    int htab[HCAP];
    int rid[RCAP];
    float rd[RCAP];
    int cand[CCAP];
    float ckey[CCAP];
    // the hybrid out-range queue (two alternating buffers) when its capacity
    // fits: every pop reads it, so it stays off global memory
    float oqk[2][OQS];
    int oqi[2][OQS];
};

enum {
    C_TICKET = 0,
    C_POOL = 1,
    C_ERR = 2,
    C_DIST = 3,
    C_EXP = 4,
    C_ADJ = 5,
    C_HYB = 6,
    C_RECHK = 7,
    C_SPILL = 8,
    C_ABORT = 9,
    C_RESTART = 10,  // pass-2 re-runs
    C_TICKET2 = 11,  // pass-3 tickets (parent-ordered commit)
    C_TICKET3 = 12,  // pass-2 tickets (parallel decisions)
    C_NUM = 13
};

struct JoinParams {
    const float* vec;
    const __nv_bfloat16* xb;  // BF16 copy of the vectors for the candidate gathers (nullptr: FP32 rows)
    int kpb;                  // its row stride in BF16 values
    int hold_q;               // test knob: this query never publishes in pass 3 (-1: none)
    const float* invn;
    const int32_t* adj;
    const float* elen;
    const int32_t* parent;
    int* done;             // per-query publish flag (soft sharing, pass 2)
    uint8_t* qflag;        // per-query pass-1 record (soft sharing): QF_* bits
    float* ckey;           // per-query FP32 key of the cache C[q] (soft sharing, pass 1)
    int32_t* cache1;       // pass 1's C[q] (soft sharing)
    int32_t* sca;          // pass 2: the seed it decided for
    uint8_t* outc;         // pass 2: its decision (0 nothing, 1 one more visit, 2 re-run)
    int32_t* cout;         // pass 2: the cache after a one-more-visit decision
    int32_t* cache2;       // pass 2: a staged re-run's cache, visited count, hybrid flag,
    int32_t* steps2;       //   result count and pool segment
    uint8_t* hyb2;
    int32_t* count2;
    int64_t* seg2;
    int mode;              // 0: no soft sharing; soft sharing: 1 pass 1, 3 pass 2, 2 pass 3;
                           // 4: separate indexes with sharing, one pass in MST order
    const uint8_t* route;  // per-query plan (nullptr: none)
    const int32_t* qbeam;
    const int* order;      // dispatch order of pass 2 (MST BFS order: parents first)
    const int* order1;     // dispatch order without dependencies (mode 0, pass 1)
    int64_t nx, nq;
    int dp4, dp, d, R, metric;
    int32_t entry;
    int ws, adapt, force, hbeam, conv;
    int seed_best;  // hybrid expansion with nothing in range starts from the closest visited data node
    float eps_key;  // L2: eps^2, cosine: eps
    float band;     // |key - eps_key| <= band * scale -> FP64 re-decision
    float tie_tol;  // keys closer than this (relative / absolute) are re-decided in FP64
    double eps64;
    int32_t* cache;
    int32_t* steps;
    uint8_t* hyb;
    int32_t* count;
    int64_t* seg;
    int32_t* pool_id;
    float* pool_d;
    int64_t pool_cap;
    int32_t* wspace;
    int64_t wstride;
    uint32_t* vbits;  // per-warp visited bitmaps (vwords words each), zero between queries
    int64_t vwords;
    int gmax;   // slots of each global visited region (power of two)
    int grcap;  // global result slots per warp
    int oqcap;  // out-range queue capacity (per buffer)
    unsigned long long* ctr;
    long long spin_limit;
    // NN-Map index: per query the witness, its FP64 distance and the OOD bit
    // (nullptr: the merged-index join)
    const int32_t* nm_w;
    const double* nm_wd;
    const uint8_t* nm_ood;
    // separate (per-set) indexes: the greedy phase is Alg. 4-5's best-first
    // search on G_Y from s_Y (plus the parent's cache or result row), its
    // queue trimmed to gbeam after each expansion
    int separate;
    int gbeam;
    // probe keys from k_probe ([nq][R + 1]: slot j of q's adjacency row, then
    // the entry), bit-identical to the traversal's own (nullptr: computed in
    // the traversal)
    const float* pkeys;
    // soft sharing, pass 3: per query, 1 when an MST ancestor ends with a
    // cache other than its pass-1 one (nullptr: every query waits)
    const uint8_t* anc;
};

enum { QF_PROBED = 1 };

// does the adjacency row (R ids) contain v?  All loads issued before any test.
__device__ __forceinline__ bool row_has(const int32_t* __restrict__ row, int R, int v) {
    bool f = false;
    if ((R & 3) == 0) {
        const int4* r4 = reinterpret_cast<const int4*>(row);
        int4 x[8];
#pragma unroll
        for (int c = 0; c < 8; c++)
            if (c < R / 4) x[c] = __ldg(r4 + c);
#pragma unroll
        for (int c = 0; c < 8; c++)
            if (c < R / 4) f |= (x[c].x == v) | (x[c].y == v) | (x[c].z == v) | (x[c].w == v);
    } else {
#pragma unroll 8
        for (int j = 0; j < R; j++) f |= __ldg(row + j) == v;
    }
    return f;
}

__device__ __forceinline__ float key_band_scale(const JoinParams& P) { return P.metric == 0 ? P.eps_key : 1.0f; }

// key -> distance
__device__ __forceinline__ float key_to_dist(const JoinParams& P, float k) {
    return P.metric == 0 ? sqrtf(fmaxf(k, 0.f)) : k;
}

struct WarpSpace {
    int* hA;            // visited list of a query in bitmap mode (gmax ids)
    int* hB;
    uint32_t* bits;     // this warp's visited bitmap over all nodes (all zero between queries)
    int* grid;
    float* grd;
    float* qk[2];
    int* qi[2];
};

struct QueryState {
    int* tab;
    unsigned mask;
    int nvis;
    int vislimit;
    int region;      // -1: shared-memory hash, 0: bitmap (list of set bits in hA)
    uint32_t* bits;  // bitmap mode: the warp's bitmap, else nullptr
    int* nlist;      // bitmap mode: entries in the list (shared-memory counter)
    int* rid;
    float* rd;
    int rcap;
    int nres;
    bool rspill;
    float bk;  // best visited data key
    int bid;
    // near-tie window of the best (lanes 0..7): tk/tid, count nt, overflow flag
    float tk;
    int tid;
    int nt;
    bool tover;
};

__device__ __forceinline__ void raise_err(const JoinParams& P, int code) {
    atomicCAS(P.ctr + C_ERR, 0ull, (unsigned long long)code);
    atomicExch(P.ctr + C_ABORT, 1ull);
}

// make room for `m` more visited entries.  Past the shared-memory hash a
// query switches to the warp's global bitmap over all nodes (one atomicOr per
// candidate, no probing); the ids it sets are listed so that the bitmap is
// cleared when the query ends.
__device__ bool vis_reserve(const JoinParams& P, QueryState& s, int m, const WarpSpace& W, int lane,
                            long long& c_spill) {
    if (s.nvis + m <= s.vislimit) return true;
    if (s.bits || s.nvis + m > P.gmax) {
        if (lane == 0) raise_err(P, VJ_DERR_VISITED_OVERFLOW);
        return false;
    }
    if (lane == 0) *s.nlist = 0;
    __syncwarp();
    for (int i = lane; i < (int)s.mask + 1; i += 32) {
        const int k = s.tab[i];
        if (k >= 0) {
            atomicOr(W.bits + (k >> 5), 1u << (k & 31));
            W.hA[atomicAdd(s.nlist, 1)] = k;
        }
    }
    __syncwarp();
    if (lane == 0) c_spill++;
    s.region = 0;
    s.bits = W.bits;
    s.vislimit = P.gmax;
    return true;
}

// insert key into the visited set: true when it was not there yet
__device__ __forceinline__ bool vis_insert(QueryState& s, const WarpSpace& W, int key) {
    if (!s.bits) return hash_insert(s.tab, s.mask, key) == 1;
    const uint32_t m = 1u << (key & 31);
    if (atomicOr(s.bits + (key >> 5), m) & m) return false;
    W.hA[atomicAdd(s.nlist, 1)] = key;
    return true;
}

__device__ __forceinline__ bool vis_contains(const QueryState& s, int key) {
    if (!s.bits) return hash_contains(s.tab, s.mask, key);
    return (((volatile const uint32_t*)s.bits)[key >> 5] >> (key & 31)) & 1u;
}

// bitmap mode: clear the bits this query set
__device__ __forceinline__ void vis_release(QueryState& s, const WarpSpace& W, int lane) {
    if (!s.bits) return;
    __syncwarp();
    const int n = *s.nlist;
    for (int i = lane; i < n; i += 32) s.bits[W.hA[i] >> 5] = 0u;
    __syncwarp();
    s.bits = nullptr;
}

__device__ bool res_reserve(const JoinParams& P, QueryState& s, int m, const WarpSpace& W, int lane) {
    if (s.nres + m <= s.rcap) return true;
    if (s.rspill) {
        if (lane == 0) raise_err(P, VJ_DERR_RESULT_OVERFLOW);
        return false;
    }
    for (int i = lane; i < s.nres; i += 32) {
        W.grid[i] = s.rid[i];
        W.grd[i] = s.rd[i];
    }
    __syncwarp();
    s.rid = W.grid;
    s.rd = W.grd;
    s.rcap = P.grcap;
    s.rspill = true;
    if (s.nres + m > s.rcap) {
        if (lane == 0) raise_err(P, VJ_DERR_RESULT_OVERFLOW);
        return false;
    }
    return true;
}

// fold a chunk of data candidates (one per lane, `valid`) into the running
// best (key, id) and its near-tie window (lanes 0..7 hold the visited data
// nodes whose key is within tie_tol of the current best)
__device__ __forceinline__ void best_update(const JoinParams& P, QueryState& s, bool valid, float k, int id,
                                            int lane) {
    float mk = valid ? k : FLT_MAX;
    int mi = valid ? id : INT32_MAX;
    warp_argmin(mk, mi);
    if (mi == INT32_MAX) return;
    if (kless(mk, mi, s.bk, s.bid)) {
        s.bk = mk;
        s.bid = mi;
    }
    const float thr = P.metric == 0 ? s.bk * (1.0f + P.tie_tol) : s.bk + P.tie_tol;
    const unsigned km = __ballot_sync(VJ_FULL, lane < s.nt && s.tk <= thr);
    const unsigned am = __ballot_sync(VJ_FULL, valid && k <= thr);
    const unsigned all_old = s.nt >= 32 ? VJ_FULL : ((1u << s.nt) - 1u);
    if (am == 0 && km == all_old) return;
    const int nk = __popc(km);
    float outk = FLT_MAX;
    int outi = -1;
    unsigned m = km;
    while (m) {
        int src = __ffs(m) - 1;
        m &= m - 1;
        float a = __shfl_sync(VJ_FULL, s.tk, src);
        int b = __shfl_sync(VJ_FULL, s.tid, src);
        if (lane == __popc(km & ((1u << src) - 1u))) {
            outk = a;
            outi = b;
        }
    }
    m = am;
    while (m) {
        int src = __ffs(m) - 1;
        m &= m - 1;
        float a = __shfl_sync(VJ_FULL, k, src);
        int b = __shfl_sync(VJ_FULL, id, src);
        int dst = nk + __popc(am & ((1u << src) - 1u));
        if (dst < 8 && lane == dst) {
            outk = a;
            outi = b;
        }
    }
    int total = nk + __popc(am);
    if (total > 8) {
        s.tover = true;
        total = 8;
    }
    s.nt = total;
    s.tk = outk;
    s.tid = outi;
}

// in-range decision with FP64 re-check near eps, for one candidate per lane
__device__ __forceinline__ bool inrange_decide(const JoinParams& P, bool valid, float k, int node, int64_t qn,
                                               int lane, long long& c_rechk) {
    float scale = key_band_scale(P);
    bool in = valid && k < P.eps_key;
    bool near = valid && fabsf(k - P.eps_key) <= P.band * scale;
    unsigned nm = __ballot_sync(VJ_FULL, near);
    while (nm) {
        int src = __ffs(nm) - 1;
        nm &= nm - 1;
        int v = __shfl_sync(VJ_FULL, node, src);
        double d64 = warp_dist64(P.vec, P.dp, P.d, P.metric, qn, v, lane);
        bool in64 = d64 < P.eps64;
        if (lane == src) in = in64;
        if (lane == 0) c_rechk++;
    }
    return in;
}

// append in-range candidates (one per lane) to the result list (keys stored)
// bring a node's adjacency row toward L2 ahead of its expansion (a hint only)
__device__ __forceinline__ void prefetch_row(const JoinParams& P, int node) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(P.adj + (int64_t)node * P.R));
}

// Every result is expanded later (closure or hybrid queue): its adjacency row
// is prefetched here, off the critical path of that expansion.
__device__ __forceinline__ bool append_results(const JoinParams& P, QueryState& s, bool in, int node, float k,
                                               const WarpSpace& W, int lane) {
    unsigned m = __ballot_sync(VJ_FULL, in);
    int cnt = __popc(m);
    if (cnt == 0) return true;
    if (!res_reserve(P, s, cnt, W, lane)) return false;
    if (in) {
        int pos = s.nres + __popc(m & ((1u << lane) - 1u));
        s.rid[pos] = node;
        s.rd[pos] = k;
        if (node >= 0 && node < P.nx) prefetch_row(P, node);
    }
    s.nres += cnt;
    __syncwarp();
    return true;
}

// warp bitonic sort of one (key, id) per lane, ascending
__device__ __forceinline__ void warp_sort_pairs(float& k, int& id, int lane) {
#pragma unroll
    for (int kk = 2; kk <= 32; kk <<= 1) {
#pragma unroll
        for (int j = kk >> 1; j > 0; j >>= 1) {
            float pk = __shfl_xor_sync(VJ_FULL, k, j);
            int pi = __shfl_xor_sync(VJ_FULL, id, j);
            bool up = (lane & kk) == 0;
            bool low = (lane & j) == 0;
            bool pless = kless(pk, pi, k, id);
            bool take = (low == up) ? pless : !pless;
            if (take) {
                k = pk;
                id = pi;
            }
        }
    }
}

// number of entries of the ascending list L[0..n) that are less than (k, id)
__device__ __forceinline__ int lower_rank(const float* Lk, const int* Li, int n, float k, int id) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (kless(Lk[mid], Li[mid], k, id)) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// The separate-index greedy queue: fold one candidate per lane (`valid`)
// into the ascending queue W.qk/qi[cur][head .. head + np), keeping the
// `cap` smallest (key, id); the result lands at the start of the other
// buffer.  Keys are distinct pairs (every node is queued once).
__device__ __forceinline__ void pq_merge(WarpSpace& W, WarpSmem* S, int& cur, int& head, int& np, bool valid, float k,
                                         int id, int cap, int lane) {
    float nk = valid ? k : FLT_MAX;
    int ni = valid ? id : INT32_MAX;
    const int m = __popc(__ballot_sync(VJ_FULL, valid));
    if (m == 0) return;
    warp_sort_pairs(nk, ni, lane);
    __syncwarp();
    if (lane < m) {
        S->ckey[lane] = nk;
        S->cand[lane] = ni;
    }
    __syncwarp();
    const float* ok_ = W.qk[cur] + head;
    const int* oi_ = W.qi[cur] + head;
    float* dk = W.qk[cur ^ 1];
    int* di = W.qi[cur ^ 1];
    const int kfin = min(np + m, cap);
    for (int i = lane; i < np; i += 32) {
        const float a = ok_[i];
        const int b = oi_[i];
        const int pos = i + lower_rank(S->ckey, S->cand, m, a, b);
        if (pos < kfin) {
            dk[pos] = a;
            di[pos] = b;
        }
    }
    if (lane < m) {
        const int pos = lane + lower_rank(ok_, oi_, np, nk, ni);
        if (pos < kfin) {
            dk[pos] = nk;
            di[pos] = ni;
        }
    }
    __syncwarp();
    cur ^= 1;
    head = 0;
    np = kfin;
}

// per-warp statistics, flushed into the instance's counters
struct JoinCounters {
    long long dist = 0, exp = 0, adj = 0, hyb = 0, rechk = 0, spill = 0;
    // this warp's chunk of the instance's result pool: next slot, slots left
    // (one pool atomic per chunk instead of one per query; unused tails are
    // holes, never read: rows are located by count and segment)
    unsigned long long pbase = 0;
    int pleft = 0;
};

constexpr int POOL_CHUNK = 256;  // result-pool slots a warp reserves at a time

__device__ __forceinline__ void flush_counters(const JoinParams& P, JoinCounters& c) {
    atomicAdd(P.ctr + C_DIST, (unsigned long long)c.dist);
    atomicAdd(P.ctr + C_EXP, (unsigned long long)c.exp);
    atomicAdd(P.ctr + C_ADJ, (unsigned long long)c.adj);
    atomicAdd(P.ctr + C_HYB, (unsigned long long)c.hyb);
    atomicAdd(P.ctr + C_RECHK, (unsigned long long)c.rechk);
    atomicAdd(P.ctr + C_SPILL, (unsigned long long)c.spill);
    c = JoinCounters();
}

// One query of one join pass (the pass is P.mode): ticket t of the pass's
// dispatch order.  Returns true when this warp must stop taking tickets (a
// device error was raised, or a parent it waits for was abandoned).
template <int G, int NPL, int U>
__device__ __forceinline__ bool join_query(const JoinParams& P, int t, WarpSmem* S, int64_t gw, int lane,
                                           JoinCounters& cnt) {
    int32_t* wbase = P.wspace + gw * P.wstride;
    WarpSpace W;
    W.hA = wbase;
    W.hB = wbase + P.gmax;
    W.bits = P.vbits + gw * P.vwords;
    W.grid = wbase + 2 * (int64_t)P.gmax;
    W.grd = reinterpret_cast<float*>(W.grid + P.grcap);
    int32_t* qbase = wbase + 2 * (int64_t)P.gmax + 2 * (int64_t)P.grcap;
    if (P.oqcap <= OQS) {
        W.qk[0] = S->oqk[0];
        W.qi[0] = S->oqi[0];
        W.qk[1] = S->oqk[1];
        W.qi[1] = S->oqi[1];
    } else {
        W.qk[0] = reinterpret_cast<float*>(qbase);
        W.qi[0] = qbase + P.oqcap;
        W.qk[1] = reinterpret_cast<float*>(qbase + 2 * P.oqcap);
        W.qi[1] = qbase + 3 * P.oqcap;
    }
    const int g = lane & (G - 1);
    const int R = P.R;
    long long &c_dist = cnt.dist, &c_exp = cnt.exp, &c_adj = cnt.adj, &c_hyb = cnt.hyb, &c_rechk = cnt.rechk,
              &c_spill = cnt.spill;
    {
        const int qi = (P.mode == 2 || P.mode == 4) ? P.order[t] : P.order1[t];
        const int64_t qn = P.nx + qi;

        // q's slots: loaded at once for a full run; the decision passes (2, 3)
        // load them only when they evaluate a seed or re-run the query
        float4 q[NPL];
        bool have_q = false;
        auto need_q = [&]() {
            if (!have_q) load_slots<G, NPL>(P.vec, qn, P.dp4, g, q);
            have_q = true;
        };
        if (P.mode != 2 && P.mode != 3) need_q();
        const float invq = P.metric ? __ldg(P.invn + qn) : 0.f;
        // everything else the query reads by its index, issued together: its
        // plan, its adjacency row and the probe kernel's keys
        const uint8_t route_q = P.route ? __ldg(P.route + qi) : (uint8_t)0;
        const int beam_q = P.qbeam ? __ldg(P.qbeam + qi) : 0;
        const int adj_l = lane < P.R ? __ldg(P.adj + qn * P.R + lane) : -1;
        const float pk_l = (P.pkeys && lane < P.R) ? __ldg(P.pkeys + (int64_t)qi * (P.R + 1) + lane) : 0.f;
        const float pk_entry = P.pkeys ? __ldg(P.pkeys + (int64_t)qi * (P.R + 1) + P.R) : 0.f;

        // ---- soft sharing, passes 2 and 3: what does C[parent] change?
        // decide(sc): 0 nothing, 1 one more visit (cache -> best), 2 re-run
        auto decide = [&](int sc, int& best) -> int {
            const int flags = P.qflag[qi];
            best = P.cache1[qi];
            if (sc < 0 || sc == P.entry) return 0;
            // a hybrid expansion depends on the order its seeds enter the
            // queue: any real seed means a re-run
            if (P.hyb[qi] == 1) return 2;
            need_q();
            if (lane == 0) S->cand[0] = sc;
            __syncwarp();
            group_keys<G, NPL, U>(P.vec, P.invn, P.dp4, P.metric, q, invq, S->cand, 1, S->ckey, lane, P.xb, P.kpb);
            __syncwarp();
            const float k = S->ckey[0];
            __syncwarp();
            // sc would have been the greedy front: no probe
            if ((flags & QF_PROBED) && k <= 0.f) return 2;
            // sc in pass 1's V?  {entry, q} U N(q) (probed) U N(results) (BFS;
            // a query without expansion, flag 3, never read N(results));
            // one result per lane, its whole adjacency row loaded at once
            bool seen = false;
            if (flags & QF_PROBED) seen = lane < R && adj_l == sc;
            const int64_t sg = P.seg[qi];
            const int cnt = P.count[qi];
            // (an overflowed pool is re-run by the host: nothing to read then)
            if (P.hyb[qi] == 0 && sg + cnt <= P.pool_cap) {
                for (int base = 0; base < cnt && !__any_sync(VJ_FULL, seen); base += 32) {
                    const int u = base + lane < cnt ? P.pool_id[sg + base + lane] : -1;
                    if (u == sc) seen = true;
                    if (u >= 0) seen |= row_has(P.adj + (int64_t)u * R, R, sc);
                }
            }
            if (__any_sync(VJ_FULL, seen)) return 0;
            const bool in = inrange_decide(P, lane == 0, k, sc, qn, lane, c_rechk);
            if (__shfl_sync(VJ_FULL, in, 0) && P.hyb[qi] != 2) return 2;  // the closure grows
            // C[q] = the (dist, id) minimum of pass 1's cache and sc: by their
            // FP32 keys when those differ by more than the rounding bound, else
            // in FP64.  kb is the window's smallest key; the cache itself lies
            // within tie_tol above it, hence the wider upper margin.
            if (best < 0) {
                best = sc;
            } else {
                const float kb = P.ckey[qi];
                const bool far = P.metric == 0
                                     ? (k > kb * (1.0f + 2.5f * P.tie_tol) || kb > k * (1.0f + P.tie_tol))
                                     : (k > kb + 2.5f * P.tie_tol || kb > k + P.tie_tol);
                if (far) {
                    if (k < kb) best = sc;
                } else {
                    const double da = warp_dist64(P.vec, P.dp, P.d, P.metric, qn, best, lane);
                    const double db = warp_dist64(P.vec, P.dp, P.d, P.metric, qn, sc, lane);
                    if (db < da || (db == da && sc < best)) best = sc;
                }
            }
            return 1;
        };
        int seedc = -1;
        if (P.mode == 3) {
            // pass 2: the decision for C[parent] as pass 1 left it, in parallel
            const int par = __ldg(P.parent + qi);
            const int sc = par >= 0 ? P.cache1[par] : -1;
            int best;
            const int o = decide(sc, best);
            if (lane == 0) {
                P.sca[qi] = sc;
                P.outc[qi] = (uint8_t)o;
                P.cout[qi] = best;
            }
            __syncwarp();
            if (o != 2) return false;
            // a re-run for this seed runs here, off the parent chain; its
            // result is staged and pass 3 commits it if the seed stays
            need_q();
            seedc = sc;
            if (lane == 0) atomicAdd(P.ctr + C_RESTART, 1ull);
        }
        if (P.mode == 2) {
            // pass 3, parent before child: the final C[parent].  What pass 2
            // decided is read before the wait, so that only the commit follows it.
            const int par = __ldg(P.parent + qi);
            const int sca_q = P.sca[qi];
            const int outc_q = P.outc[qi];
            const int cout_q = P.cout[qi];
            int sc = -1;
            // no ancestor changes its cache: the parent's final cache is its
            // pass-1 cache, the seed pass 2 decided for, and nothing to wait for
            if (par >= 0 && P.anc && !P.anc[qi]) {
                sc = sca_q;
            } else if (par >= 0 && lane == 0) {
                long long spins = 0;
                unsigned ns = 32;
                for (;;) {
                    if (ld_acquire(P.done + par)) {
                        sc = *((volatile int*)(P.cache + par));
                        break;
                    }
                    if (*((volatile unsigned long long*)(P.ctr + C_ABORT))) {
                        sc = -2;
                        break;
                    }
                    if (++spins > P.spin_limit) {
                        raise_err(P, VJ_DERR_WAIT_TIMEOUT);
                        sc = -2;
                        break;
                    }
                    __nanosleep(ns);
                    if (ns < 64) ns <<= 1;  // a short poll: the chain's latency is the pass's time
                }
            }
            sc = __shfl_sync(VJ_FULL, sc, 0);
            if (sc == -2) return true;
            int best, o;
            const bool same = sc == sca_q;  // usually: pass 2 decided for this very seed
            if (same) {
                o = outc_q;
                best = cout_q;
            } else {
                o = decide(sc, best);
            }
            if (o == 2 && same) {
                // commit the re-run pass 2 staged
                if (lane == 0) {
                    c_dist += P.steps2[qi] - P.steps[qi];
                    P.cache[qi] = P.cache2[qi];
                    P.steps[qi] = P.steps2[qi];
                    P.hyb[qi] = P.hyb2[qi];
                    P.count[qi] = P.count2[qi];
                    P.seg[qi] = P.seg2[qi];
                    if (qi != P.hold_q) st_release(P.done + qi, 1);
                }
                __syncwarp();
                return false;
            }
            if (o != 2) {
                if (lane == 0) {
                    P.cache[qi] = best;
                    if (o == 1) {
                        P.steps[qi] += 1;
                        c_dist += 1;
                    }
                    if (qi != P.hold_q) st_release(P.done + qi, 1);
                }
                __syncwarp();
                return false;
            }
            // re-run from the start with the cached seed
            need_q();
            seedc = sc;
            if (lane == 0) atomicAdd(P.ctr + C_RESTART, 1ull);
        }

        // ---- separate indexes with hard or soft sharing (mode 4): one pass in
        // MST order, each query waiting (bounded acquire spin) for its
        // parent's final cache (soft) or result row (hard) before it starts
        int hcnt = 0;
        int64_t hseg = 0;
        if (P.mode == 4) {
            const int par = __ldg(P.parent + qi);
            int ok = 1;
            if (par >= 0 && lane == 0) {
                long long spins = 0;
                unsigned ns = 32;
                for (;;) {
                    if (ld_acquire(P.done + par)) {
                        if (P.ws == VJ_WS_SOFT) {
                            seedc = *((volatile int*)(P.cache + par));
                        } else {
                            hseg = *((volatile int64_t*)(P.seg + par));
                            hcnt = *((volatile int*)(P.count + par));
                            // an overflowed pool holds no row (the host re-runs the join)
                            if (hseg + hcnt > P.pool_cap || hcnt < 0) hcnt = 0;
                        }
                        break;
                    }
                    if (*((volatile unsigned long long*)(P.ctr + C_ABORT))) {
                        ok = 0;
                        break;
                    }
                    if (++spins > P.spin_limit) {
                        raise_err(P, VJ_DERR_WAIT_TIMEOUT);
                        ok = 0;
                        break;
                    }
                    __nanosleep(ns);
                    if (ns < 256) ns <<= 1;
                }
            }
            ok = __shfl_sync(VJ_FULL, ok, 0);
            if (!ok) return true;
            seedc = __shfl_sync(VJ_FULL, seedc, 0);
            hcnt = __shfl_sync(VJ_FULL, hcnt, 0);
            hseg = __shfl_sync(VJ_FULL, hseg, 0);
        }

        QueryState s;
        s.tab = S->htab;
        s.mask = HCAP - 1;
        s.nvis = 0;
        s.vislimit = HCAP / 2;
        s.region = -1;
        s.bits = nullptr;
        s.nlist = &S->nlist;
        s.rid = S->rid;
        s.rd = S->rd;
        s.rcap = RCAP;
        s.nres = 0;
        s.rspill = false;
        s.bk = FLT_MAX;
        s.bid = INT32_MAX;
        s.tk = FLT_MAX;
        s.tid = -1;
        s.nt = 0;
        s.tover = false;
        for (int i = lane; i < HCAP; i += 32) S->htab[i] = -1;
        __syncwarp();
        bool failed = false;

        bool probe = false;
        float nkey_l = FLT_MAX;
        int nid_l = -1;
        int entry_in_nq = 0, seed_in_nq = 0;
        bool nm_empty = false;  // NN-Map: the row is certified empty
        int nm_hyb = 0;         // NN-Map: the expansion's hybrid flag
        if (P.nm_w) {
            // ---- NN-Map seeding (no greedy phase): the witness w (nearest
            // data vector) and its stored FP64 distance.  Out of range: no
            // data vector is in range, and nothing is computed.  Otherwise w
            // is the one in-range seed of the expansion, visited at no cost.
            const int w = __ldg(P.nm_w + qi);
            const double wd = __ldg(P.nm_wd + qi);
            if (!(wd < P.eps64)) {
                nm_empty = true;
            } else {
                nm_hyb = P.force ? 1 : (P.adapt ? (int)__ldg(P.nm_ood + qi) : 0);
                if (lane == 0) hash_insert(s.tab, s.mask, w);
                __syncwarp();
                const float wk = P.metric == 0 ? (float)(wd * wd) : (float)wd;
                best_update(P, s, lane == 0, wk, w, lane);
                if (!append_results(P, s, lane == 0, w, wk, W, lane)) failed = true;
            }
        } else if (P.separate) {
            // ---- Alg. 3 seeds on the per-set index G_Y: s_Y, then C[parent]
            // (soft) or the parent's result row (hard); Alg. 4 evaluates them
            // all (the visited set drops repeats) and queues them.  Only the
            // gbeam + 1 smallest queued seeds can survive the first trim (one
            // pop, then the queue keeps gbeam), so the queue keeps those.
            const int nsc = seedc >= 0 ? 1 : 0;
            const int nseed = 1 + nsc + hcnt;
            int cur = 0, head = 0, np = 0;  // the queue: W.qk/qi[cur][head .. head + np), ascending
            for (int base = 0; base < nseed && !failed; base += 32) {
                const int j = base + lane;
                int v = -1;
                if (j == 0) v = P.entry;
                else if (j == 1 && nsc) v = seedc;
                else if (j < nseed) v = __ldcg(P.pool_id + hseg + (j - 1 - nsc));
                if (v >= P.nx) v = -1;
                if (!vis_reserve(P, s, 32, W, lane, c_spill)) {
                    failed = true;
                    break;
                }
                const bool nw = v >= 0 && vis_insert(s, W, v);
                const unsigned nm = __ballot_sync(VJ_FULL, nw);
                const int nc = __popc(nm);
                if (nw) S->cand[__popc(nm & ((1u << lane) - 1u))] = v;
                __syncwarp();
                if (nc == 0) continue;
                group_keys<G, NPL, U>(P.vec, P.invn, P.dp4, P.metric, q, invq, S->cand, nc, S->ckey, lane, P.xb,
                                      P.kpb);
                __syncwarp();
                s.nvis += nc;
                const bool val = lane < nc;
                const int cv = val ? S->cand[lane] : -1;
                const float ck = val ? S->ckey[lane] : FLT_MAX;
                __syncwarp();
                const bool in = inrange_decide(P, val, ck, cv, qn, lane, c_rechk);
                best_update(P, s, val, ck, cv, lane);
                if (!append_results(P, s, in, cv, ck, W, lane)) {
                    failed = true;
                    break;
                }
                pq_merge(W, S, cur, head, np, val, ck, cv, P.gbeam + 1, lane);
            }
            // ---- Alg. 4-5: pop the front and evaluate its G_Y neighbours until
            // StopGreedy: the front is an in-range data node (on G_Y: some
            // in-range node has been found, since every in-range key is below
            // every out-range one), or the front key has not decreased for
            // conv_threshold consecutive checks
            float best_front = INFINITY;
            int noimp = 0;
            while (!failed && np > 0) {
                if (s.nres > 0) break;
                const float fk = W.qk[cur][head];
                const int u = W.qi[cur][head];
                if (fk < best_front) {
                    best_front = fk;
                    noimp = 0;
                } else {
                    noimp++;
                }
                if (noimp >= P.conv) break;
                head++;
                np--;
                c_adj++;
                if (!vis_reserve(P, s, R, W, lane, c_spill)) {
                    failed = true;
                    break;
                }
                const int v = lane < R ? __ldg(P.adj + (int64_t)u * R + lane) : -1;
                const bool nw = v >= 0 && v < P.nx && vis_insert(s, W, v);
                const unsigned nm = __ballot_sync(VJ_FULL, nw);
                const int nc = __popc(nm);
                if (nw) S->cand[__popc(nm & ((1u << lane) - 1u))] = v;
                __syncwarp();
                if (nc == 0) continue;
                group_keys<G, NPL, U>(P.vec, P.invn, P.dp4, P.metric, q, invq, S->cand, nc, S->ckey, lane, P.xb,
                                      P.kpb);
                __syncwarp();
                s.nvis += nc;
                const bool val = lane < nc;
                const int cv = val ? S->cand[lane] : -1;
                const float ck = val ? S->ckey[lane] : FLT_MAX;
                __syncwarp();
                const bool in = inrange_decide(P, val, ck, cv, qn, lane, c_rechk);
                best_update(P, s, val, ck, cv, lane);
                if (!append_results(P, s, in, cv, ck, W, lane)) {
                    failed = true;
                    break;
                }
                pq_merge(W, S, cur, head, np, val, ck, cv, P.gbeam, lane);
            }
        } else {
            // ---- Alg. 4 greedy: the seeds (lanes 0..2: entry, cached seed, q)
            int sid = -1;
            if (lane == 0) sid = P.entry;
            if (lane == 1 && seedc >= 0) sid = seedc;
            if (lane == 2 && (P.ws == VJ_WS_SELF || P.ws == VJ_WS_SOFT)) sid = (int)qn;
            bool snew = false;
    #pragma unroll 1
            for (int src = 0; src < 3; src++) {
                int v = __shfl_sync(VJ_FULL, sid, src);
                int ins = 0;
                if (lane == 0 && v >= 0) ins = hash_insert(s.tab, s.mask, v);  // seeds: always the shared hash
                ins = __shfl_sync(VJ_FULL, ins, 0);
                if (lane == src) snew = ins == 1;
                __syncwarp();
            }
            unsigned sm = __ballot_sync(VJ_FULL, snew);
            if (snew) S->cand[__popc(sm & ((1u << lane) - 1u))] = sid;
            __syncwarp();
            int ns = __popc(sm);
            if (P.pkeys && seedc < 0) {
                // the entry's key is the probe kernel's; q's own key is never read
                if (snew) {
                    const int pos = __popc(sm & ((1u << lane) - 1u));
                    S->ckey[pos] = sid == P.entry ? pk_entry : 0.f;
                }
            } else {
                group_keys<G, NPL, U>(P.vec, P.invn, P.dp4, P.metric, q, invq, S->cand, ns, S->ckey, lane, P.xb,
                                      P.kpb);
            }
            __syncwarp();
            s.nvis += ns;
            float skey = FLT_MAX;
            int snode = -1;
            if (lane < ns) {
                snode = S->cand[lane];
                skey = (snode == (int)qn) ? 0.f : S->ckey[lane];
            }
            __syncwarp();
            bool sdata = lane < ns && snode < P.nx;
            bool sin = inrange_decide(P, sdata, skey, snode, qn, lane, c_rechk);
            best_update(P, s, sdata, skey, snode, lane);
            if (!append_results(P, s, sin, snode, skey, W, lane)) failed = true;

            // StopGreedy on the front = argmin (key, id) over the seeds
            float fk = lane < ns ? skey : FLT_MAX;
            int fi = lane < ns ? snode : INT32_MAX;
            bool fin = sin;
            {
                float mk = fk;
                int mi = fi;
                warp_argmin(mk, mi);
                unsigned who = __ballot_sync(VJ_FULL, fi == mi && lane < ns);
                int src = who ? __ffs(who) - 1 : 0;
                fin = __shfl_sync(VJ_FULL, sin, src);
                fi = mi;
            }
            probe = !failed && ns > 0 && !(fi < P.nx && fin) && P.conv > 0 && fi == (int)qn;

            // ---- probe N(q); lane j keeps slot j of q's list and that neighbour's key
            if (probe) {
                c_adj++;
                int v = adj_l;
                const float pk = pk_l;  // its key from the probe kernel
                nid_l = v;
                if (v == P.entry) entry_in_nq = 1;
                if (v >= 0 && v == seedc) seed_in_nq = 1;
                unsigned vm = __ballot_sync(VJ_FULL, v >= 0);
                if (!vis_reserve(P, s, __popc(vm), W, lane, c_spill)) failed = true;
                if (!failed) {
                    bool nw = v >= 0 && vis_insert(s, W, v);
                    unsigned nm = __ballot_sync(VJ_FULL, nw);
                    int nc = __popc(nm);
                    int mypos = __popc(nm & ((1u << lane) - 1u));
                    if (nw) S->cand[mypos] = v;
                    if (P.pkeys) {
                        // slot `lane` of q's row: its key from the probe kernel
                        if (nw) S->ckey[mypos] = pk;
                    } else {
                        __syncwarp();
                        group_keys<G, NPL, U>(P.vec, P.invn, P.dp4, P.metric, q, invq, S->cand, nc, S->ckey, lane,
                                              P.xb, P.kpb);
                    }
                    __syncwarp();
                    s.nvis += nc;
                    int cv = lane < nc ? S->cand[lane] : -1;
                    float ck = lane < nc ? S->ckey[lane] : FLT_MAX;
                    float kk = S->ckey[nw ? mypos : 0];
                    __syncwarp();
                    bool dat = lane < nc && cv < P.nx;
                    bool in = inrange_decide(P, dat, ck, cv, qn, lane, c_rechk);
                    best_update(P, s, dat, ck, cv, lane);
                    if (!append_results(P, s, in, cv, ck, W, lane)) failed = true;
                    if (nw) nkey_l = kk;
                    // a neighbour that was a seed keeps the seed's key
                    for (int src = 0; src < ns; src++) {
                        int sn = __shfl_sync(VJ_FULL, snode, src);
                        float sk2 = __shfl_sync(VJ_FULL, skey, src);
                        if (!nw && v == sn) nkey_l = sk2;
                    }
                }
            }
        }
        entry_in_nq = __any_sync(VJ_FULL, entry_in_nq);
        seed_in_nq = __any_sync(VJ_FULL, seed_in_nq);

        // ---- Alg. 6 CheckHybrid (adapt on the merged index decides; force
        // otherwise), or the per-query plan when one is set: a routed query
        // stops after its greedy phase (its row comes from the brute-force
        // scan); a planned beam > 0 selects the hybrid expansion with that
        // queue size, 0 the BFS expansion, and a negative beam no expansion
        // at all (the result is the probe's in-range points; flag 3)
        const bool routed = route_q != 0;
        int hbq = P.hbeam;
        int hyb = P.force;
        if (P.nm_w) {
            hyb = nm_hyb;
        } else if (P.qbeam) {
            hbq = beam_q;
            hyb = hbq > 0 ? 1 : (hbq < 0 ? 3 : 0);
        } else if (P.adapt && !P.separate && !failed && !routed) {
            if (!probe) {
                // no probe ran (a seed was the greedy front); the rule still
                // reads q's neighbourhood, evaluated here outside V
                c_adj++;
                const int v = adj_l;
                nid_l = v;
                const bool dv = v >= 0 && v < P.nx;
                const unsigned dm0 = __ballot_sync(VJ_FULL, dv);
                const int pos = __popc(dm0 & ((1u << lane) - 1u));
                if (dv) S->cand[pos] = v;
                __syncwarp();
                group_keys<G, NPL, U>(P.vec, P.invn, P.dp4, P.metric, q, invq, S->cand, __popc(dm0), S->ckey, lane, P.xb, P.kpb);
                __syncwarp();
                nkey_l = dv ? S->ckey[pos] : FLT_MAX;
                __syncwarp();
                if (lane < R) S->cand[lane] = v;  // N(q) for the pair test below
                __syncwarp();
            }
            // w in N(q) U {q}: the visited set after the probe holds N(q) and
            // the seeds (entry and C[parent] count only if they are in N(q))
            auto in_nq = [&](int w) -> bool {
                if (!probe) {
                    bool f = false;
                    for (int t = 0; t < R; t++) f |= S->cand[t] == w;
                    return f;
                }
                bool inq = vis_contains(s, w);
                if (inq && w == P.entry && !entry_in_nq) inq = false;
                if (inq && w == seedc && !seed_in_nq) inq = false;
                return inq;
            };
            const bool isd = nid_l >= 0 && nid_l < P.nx;
            float d1s = isd ? key_to_dist(P, nkey_l) : 0.f;
            const unsigned dmask = __ballot_sync(VJ_FULL, isd);
            const int n1 = __popc(dmask);
            float d2s = 0.f;
            int n2 = 0;
            unsigned dm = dmask;
            while (dm) {
                // four data neighbours' rows per round, loads issued together
                int vr[4];
                int w4[4];
                float e4[4];
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    int src = dm ? __ffs(dm) - 1 : -1;
                    if (dm) dm &= dm - 1;
                    vr[k] = src >= 0 ? __shfl_sync(VJ_FULL, nid_l, src) : -1;
                    if (src < 0) (void)__shfl_sync(VJ_FULL, nid_l, 0);
                }
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    w4[k] = (vr[k] >= 0 && lane < R) ? __ldg(P.adj + (int64_t)vr[k] * R + lane) : -1;
                    e4[k] = (vr[k] >= 0 && lane < R) ? __ldg(P.elen + (int64_t)vr[k] * R + lane) : 0.f;
                }
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    if (vr[k] >= 0) c_adj += (lane == 0);
                    int w = w4[k];
                    bool ok = w >= 0 && w < P.nx;
                    if (ok) ok = !in_nq(w);
                    if (ok) {
                        d2s += e4[k];
                        n2++;
                    }
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                d1s += __shfl_xor_sync(VJ_FULL, d1s, o);
                d2s += __shfl_xor_sync(VJ_FULL, d2s, o);
                n2 += __shfl_xor_sync(VJ_FULL, n2, o);
            }
            int ood;
            if (n1 == 0) ood = 1;
            else if (n2 == 0) ood = 0;
            else {
                float r = (d1s / (float)n1) / (d2s / (float)n2);
                ood = r > 1.5f;
                if (fabsf(r - 1.5f) <= 1e-3f) {
                    // FP64 re-decision of the ratio
                    double a1 = 0.0, a2 = 0.0;
                    unsigned dm2 = dmask;
                    while (dm2) {
                        int src = __ffs(dm2) - 1;
                        dm2 &= dm2 - 1;
                        int v = __shfl_sync(VJ_FULL, nid_l, src);
                        a1 += warp_dist64(P.vec, P.dp, P.d, P.metric, qn, v, lane);
                        for (int j = 0; j < R; j++) {
                            int w = __ldg(P.adj + (int64_t)v * R + j);
                            if (w < 0 || w >= P.nx) continue;
                            if (in_nq(w)) continue;
                            a2 += warp_dist64(P.vec, P.dp, P.d, P.metric, v, w, lane);
                        }
                    }
                    ood = (a1 / n1) / (a2 / n2) > 1.5;
                    if (lane == 0) c_rechk++;
                }
            }
            hyb = ood;
        }
        int expansions = 0;
        if (routed) {
            s.nres = 0;  // the scan supplies the row
            hyb = 2;
        }

        // ---- Alg. 7 ExpansionPhase
        if (routed || hyb == 3 || nm_empty) {
        } else if (!failed && !hyb) {
            int fp = 0;
            while (fp < s.nres) {
                const int nb = min(FB, s.nres - fp);
                if (!vis_reserve(P, s, nb * R, W, lane, c_spill)) {
                    failed = true;
                    break;
                }
                // neighbour rows of nb frontier nodes, loads issued together
                int vv[FB];
#pragma unroll
                for (int f = 0; f < FB; f++) {
                    int u = f < nb ? s.rid[fp + f] : -1;
                    vv[f] = (u >= 0 && lane < R) ? __ldg(P.adj + (int64_t)u * R + lane) : -1;
                }
                int nc = 0;
#pragma unroll
                for (int f = 0; f < FB; f++) {
                    int v = vv[f];
                    bool nw = v >= 0 && v < P.nx && vis_insert(s, W, v);
                    unsigned nm = __ballot_sync(VJ_FULL, nw);
                    if (nw) S->cand[nc + __popc(nm & ((1u << lane) - 1u))] = v;
                    nc += __popc(nm);
                }
                __syncwarp();
                c_adj += nb;
                expansions += nb;
                fp += nb;
                if (nc == 0) continue;
                group_keys<G, NPL, U>(P.vec, P.invn, P.dp4, P.metric, q, invq, S->cand, nc, S->ckey, lane, P.xb, P.kpb);
                __syncwarp();
                s.nvis += nc;
                for (int base = 0; base < nc; base += 32) {
                    int ci = base + lane;
                    int cv = ci < nc ? S->cand[ci] : -1;
                    float ck = ci < nc ? S->ckey[ci] : FLT_MAX;
                    bool val = ci < nc;
                    bool in = inrange_decide(P, val, ck, cv, qn, lane, c_rechk);
                    best_update(P, s, val, ck, cv, lane);
                    if (!append_results(P, s, in, cv, ck, W, lane)) {
                        failed = true;
                        break;
                    }
                }
                __syncwarp();
                if (failed) break;
            }
        } else if (!failed && hyb) {
            if (lane == 0) c_hyb++;
            int npend = s.nres;  // in-range entries not yet popped (rid >= 0)
            int osz = 0, oqh = 0, cur = 0;
            if (P.seed_best && s.nres == 0 && s.bid != INT32_MAX) {
                // seed-with-the-best variant: with nothing in range after the
                // greedy phase, the queue starts from the closest visited data
                // node ((dist, id) minimum, FP64 among FP32 near-ties)
                int b = s.bid;
                float bk = s.bk;
                if (s.nt > 1) {
                    double bd = 1e300;
                    int bi = INT32_MAX;
                    float bkk = s.bk;
                    for (int src = 0; src < s.nt; src++) {
                        const int v = __shfl_sync(VJ_FULL, s.tid, src);
                        const float kv = __shfl_sync(VJ_FULL, s.tk, src);
                        const double d64 = warp_dist64(P.vec, P.dp, P.d, P.metric, qn, v, lane);
                        if (d64 < bd || (d64 == bd && v < bi)) {
                            bd = d64;
                            bi = v;
                            bkk = kv;
                        }
                    }
                    b = bi;
                    bk = bkk;
                    if (lane == 0) c_rechk++;
                }
                if (lane == 0) {
                    W.qk[cur][0] = bk;
                    W.qi[cur][0] = b;
                }
                __syncwarp();
                osz = 1;
            }
            for (;;) {
                int u;
                if (npend > 0) {
                    float mk = FLT_MAX;
                    int mi = INT32_MAX, mpos = -1;
                    for (int i = lane; i < s.nres; i += 32) {
                        int id = s.rid[i];
                        if (id >= 0 && kless(s.rd[i], id, mk, mi)) {
                            mk = s.rd[i];
                            mi = id;
                            mpos = i;
                        }
                    }
                    float k0 = mk;
                    int i0 = mi;
                    warp_argmin(k0, i0);
                    unsigned who = __ballot_sync(VJ_FULL, mi == i0 && mpos >= 0);
                    int src = __ffs(who) - 1;
                    int pos = __shfl_sync(VJ_FULL, mpos, src);
                    u = i0;
                    if (lane == 0) s.rid[pos] = ~u;
                    __syncwarp();
                    npend--;
                } else if (osz > 0) {
                    u = W.qi[cur][oqh];
                    oqh++;
                    osz--;
                } else {
                    break;
                }
                expansions++;
                c_adj++;
                if (!vis_reserve(P, s, R, W, lane, c_spill)) {
                    failed = true;
                    break;
                }
                int v = lane < R ? __ldg(P.adj + (int64_t)u * R + lane) : -1;
                bool nw = v >= 0 && v < P.nx && vis_insert(s, W, v);
                unsigned nm = __ballot_sync(VJ_FULL, nw);
                int nc = __popc(nm);
                if (nw) S->cand[__popc(nm & ((1u << lane) - 1u))] = v;
                __syncwarp();
                if (nc == 0) continue;
                group_keys<G, NPL, U>(P.vec, P.invn, P.dp4, P.metric, q, invq, S->cand, nc, S->ckey, lane, P.xb, P.kpb);
                __syncwarp();
                s.nvis += nc;
                // one candidate per lane, in adjacency order (nc <= 32)
                const bool val = lane < nc;
                const int cv = val ? S->cand[lane] : -1;
                const float ck = val ? S->ckey[lane] : FLT_MAX;
                __syncwarp();
                const bool in = inrange_decide(P, val, ck, cv, qn, lane, c_rechk);
                best_update(P, s, val, ck, cv, lane);
                const bool isout = val && !in;
                if (isout) prefetch_row(P, cv);  // it may be popped from the out-range queue
                const unsigned inm = __ballot_sync(VJ_FULL, in);
                const unsigned outm = __ballot_sync(VJ_FULL, isout);
                // queue size after the per-insert rule, in adjacency order
                int np = npend, o = osz;
                for (int c = 0; c < nc; c++) {
                    if ((inm >> c) & 1u) np++;
                    else if ((outm >> c) & 1u) {
                        if (np + o + 1 <= hbq) o++;
                    }
                }
                const int kfin = o;
                if (!append_results(P, s, in, cv, ck, W, lane)) {
                    failed = true;
                    break;
                }
                npend = np;
                const int m = __popc(outm);
                if (m > 0 || oqh > 0) {
                    // new out-range entries, sorted, staged in shared memory
                    float nk = isout ? ck : FLT_MAX;
                    int ni = isout ? cv : INT32_MAX;
                    warp_sort_pairs(nk, ni, lane);
                    if (lane < m) {
                        S->ckey[lane] = nk;
                        S->cand[lane] = ni;
                    }
                    __syncwarp();
                    const float* ok_ = W.qk[cur] + oqh;
                    const int* oi_ = W.qi[cur] + oqh;
                    float* dk = W.qk[cur ^ 1];
                    int* di = W.qi[cur ^ 1];
                    // merge: the kfin smallest of old (osz) U new (m)
                    for (int i = lane; i < osz; i += 32) {
                        float a = ok_[i];
                        int b = oi_[i];
                        int pos = i + lower_rank(S->ckey, S->cand, m, a, b);
                        if (pos < kfin) {
                            dk[pos] = a;
                            di[pos] = b;
                        }
                    }
                    if (lane < m) {
                        int pos = lane + lower_rank(ok_, oi_, osz, nk, ni);
                        if (pos < kfin) {
                            dk[pos] = nk;
                            di[pos] = ni;
                        }
                    }
                    __syncwarp();
                    cur ^= 1;
                    oqh = 0;
                }
                osz = kfin;
            }
        }
        c_exp += expansions;

        // ---- Alg. 8 UpdateCache: FP64 re-decision among near-ties
        int best = (s.bid == INT32_MAX) ? -1 : s.bid;
        if (!failed && s.nt > 1) {
            double bd = 1e300;
            int bi = INT32_MAX;
            for (int src = 0; src < s.nt; src++) {
                int v = __shfl_sync(VJ_FULL, s.tid, src);
                double d64 = warp_dist64(P.vec, P.dp, P.d, P.metric, qn, v, lane);
                if (d64 < bd || (d64 == bd && v < bi)) {
                    bd = d64;
                    bi = v;
                }
            }
            best = bi;
            if (lane == 0) c_rechk++;
        }

        if (lane == 0) {
            if (P.mode == 3) {
                // staged re-run (pass 2): committed by pass 3, counted there
                P.cache2[qi] = best;
                P.steps2[qi] = s.nvis;
                P.hyb2[qi] = (uint8_t)hyb;
            } else {
                // a pass-3 re-run replaces pass 1's count of this query
                if (P.mode == 2) c_dist -= P.steps[qi];
                P.cache[qi] = best;
                P.steps[qi] = s.nvis;
                P.hyb[qi] = (uint8_t)hyb;
                c_dist += s.nvis;
            }
            if (P.mode == 1) {
                P.qflag[qi] = (uint8_t)(probe ? QF_PROBED : 0);
                P.ckey[qi] = s.bk;
                P.cache1[qi] = best;
            }
            // publish: cache[qi] is visible to whoever sees the flag
            if (P.mode == 2 && !failed) if (qi != P.hold_q) st_release(P.done + qi, 1);
        }
        vis_release(s, W, lane);
        if (failed) {
            if (lane == 0) {
                if (P.mode == 3) P.count2[qi] = 0;
                else P.count[qi] = 0;
            }
            return true;
        }

        // ---- results into the pool (the warp's chunk; a new one when it runs out)
        if (s.nres > cnt.pleft) {
            const int want = max(s.nres, POOL_CHUNK);
            unsigned long long b = 0;
            if (lane == 0) b = atomicAdd(P.ctr + C_POOL, (unsigned long long)want);
            cnt.pbase = __shfl_sync(VJ_FULL, b, 0);
            cnt.pleft = want;
        }
        const unsigned long long off = cnt.pbase;
        cnt.pbase += (unsigned long long)s.nres;
        cnt.pleft -= s.nres;
        if (lane == 0) {
            if (P.mode == 3) {
                P.count2[qi] = s.nres;
                P.seg2[qi] = (int64_t)off;
            } else {
                P.count[qi] = s.nres;
                P.seg[qi] = (int64_t)off;
            }
        }
        if ((int64_t)off + s.nres <= P.pool_cap) {
            for (int i = lane; i < s.nres; i += 32) {
                int id = s.rid[i];
                P.pool_id[off + i] = id < 0 ? ~id : id;
                P.pool_d[off + i] = key_to_dist(P, s.rd[i]);
            }
        }
        __syncwarp();
        if (P.mode == 4) {
            // publish: the cache, count, segment and pooled row are visible
            // to whoever sees the flag
            __threadfence();
            __syncwarp();
            if (lane == 0 && qi != P.hold_q) st_release(P.done + qi, 1);
        }
    }
    return false;
}

__device__ __forceinline__ int pass_ticket_slot(int mode) {
    return (mode == 2 || mode == 4) ? C_TICKET2 : mode == 3 ? C_TICKET3 : C_TICKET;
}

// one join pass over one index: warps take queries from the pass's ticket
// ---------------------------------------------------------------- probe keys
// The greedy phase of the merged index probes N(q), the query's own
// adjacency row (Alg. 4 under the merged rule), and every query's first
// seeds are the entry and q itself.  k_probe evaluates those keys for all
// queries ahead of the traversal: a warp per query streams the rows of N(q)
// and the entry through a shared-memory ring (cp.async, PB_RING stages in
// flight), so the gathers are bandwidth-bound instead of a chain of
// dependent round trips per query.  The arithmetic is group_keys'
// (the same lane slots, FMA order and group reduction), so every key equals
// the one the traversal would compute.
constexpr int PB_WARPS = 8;
constexpr int PB_RING = 8;           // stages in flight per warp
constexpr int PB_STAGE_MAX = 12288;  // bytes of one warp's ring at most

struct PbParams {
    const float* vec;
    const float* invn;
    const __nv_bfloat16* xb;  // BF16 copy (the traversal's gathers), or nullptr: FP32 rows
    int kpb;
    int dp4;
    int metric;
    const int32_t* adj;
    int R;
    int32_t entry;
    int64_t nx, nq;
    int ring;      // stages per warp (<= PB_RING)
    int rowbytes;  // bytes copied per row (16-byte multiple)
    int rowpitch;  // bytes between rows in the ring
    float* pkeys;  // [nq][R + 1]
    int bulk;      // 1: each row is one bulk copy (cp.async.bulk, mbarrier per stage)
    unsigned long long* ctr;  // the join's counters (error word) for the bounded waits
    long long spin_limit;
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
// wait until at most n (0 .. PB_RING - 1) of this thread's groups are pending
__device__ __forceinline__ void cp_async_wait_dyn(int n) {
    switch (n) {
        case 0: cp_async_wait<0>(); break;
        case 1: cp_async_wait<1>(); break;
        case 2: cp_async_wait<2>(); break;
        case 3: cp_async_wait<3>(); break;
        case 4: cp_async_wait<4>(); break;
        case 5: cp_async_wait<5>(); break;
        case 6: cp_async_wait<6>(); break;
        default: cp_async_wait<7>(); break;
    }
}

template <int G, int NPL>
__global__ void __launch_bounds__(PB_WARPS * 32) k_probe(const __grid_constant__ PbParams P) {
    extern __shared__ __align__(16) unsigned char pb_raw[];
    constexpr int NG = 32 / G;  // rows per stage (one per lane group)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int grp = lane / G, g = lane & (G - 1);
    const int64_t qi = (int64_t)blockIdx.x * PB_WARPS + warp;
    if (qi >= P.nq) return;
    unsigned char* ring = pb_raw + (size_t)warp * P.ring * NG * P.rowpitch;
    const int64_t qn = P.nx + qi;
    const int R = P.R;
    // slot j < R: adjacency slot j of q (held by lane j); slot R: the entry
    const int vl = lane < R ? __ldg(P.adj + qn * R + lane) : -1;
    float4 q[NPL];
    load_slots<G, NPL>(P.vec, qn, P.dp4, g, q);
    const float invq = P.metric ? __ldg(P.invn + qn) : 0.f;
    const float invl = (P.metric && vl >= 0) ? __ldg(P.invn + vl) : 0.f;
    const float inve = P.metric ? __ldg(P.invn + P.entry) : 0.f;
    const int nstage = (R + 1 + NG - 1) / NG;
    const int chunks = P.rowbytes >> 4;
    auto issue = [&](int st) {
        if (st < nstage) {
            unsigned char* dst = ring + (size_t)(st % P.ring) * NG * P.rowpitch;
            for (int r = 0; r < NG; r++) {
                const int slot = st * NG + r;
                const int vs = __shfl_sync(VJ_FULL, vl, slot & 31);
                const int v = slot < R ? vs : (slot == R ? P.entry : -1);
                if (v < 0) continue;
                const unsigned char* src =
                    P.xb ? reinterpret_cast<const unsigned char*>(P.xb + (int64_t)v * P.kpb)
                         : reinterpret_cast<const unsigned char*>(P.vec + (int64_t)v * P.dp4 * 4);
                for (int c = lane; c < chunks; c += 32) cp_async16(dst + (size_t)r * P.rowpitch + c * 16, src + c * 16);
            }
        }
        cp_async_commit();  // an empty group past the last stage keeps the count
    };
    // group k of this thread carries stage k: after `ring` groups are issued
    // ahead, waiting until ring - 1 are pending completes stage st
    for (int st = 0; st < P.ring; st++) issue(st);
    for (int st = 0; st < nstage; st++) {
        cp_async_wait_dyn(P.ring - 1);
        __syncwarp();
        const int slot = st * NG + grp;
        const int vs = __shfl_sync(VJ_FULL, vl, slot & 31);
        const float ils = __shfl_sync(VJ_FULL, invl, slot & 31);
        const int v = slot < R ? vs : (slot == R ? P.entry : -1);
        const float il = slot < R ? ils : inve;
        const unsigned char* row = ring + (size_t)(st % P.ring) * NG * P.rowpitch + (size_t)grp * P.rowpitch;
        float a;
        if (P.xb) {
            uint2 xr[NPL];
#pragma unroll
            for (int k = 0; k < NPL; k++) {
                const int idx = g + k * G;
                xr[k] = idx < P.dp4 ? reinterpret_cast<const uint2*>(row)[idx] : make_uint2(0u, 0u);
            }
            a = group_sum<G>(slot_accum_bf16<NPL>(xr, q, P.metric));
        } else {
            float4 x[NPL];
#pragma unroll
            for (int k = 0; k < NPL; k++) {
                const int idx = g + k * G;
                x[k] = idx < P.dp4 ? reinterpret_cast<const float4*>(row)[idx] : f4zero();
            }
            a = group_sum<G>(slot_accum<NPL>(x, q, P.metric));
        }
        if (g == 0 && slot <= R)
            P.pkeys[qi * (R + 1) + slot] = v < 0 ? FLT_MAX : (P.metric == 0 ? a : 1.0f - a * il * invq);
        __syncwarp();  // the stage's buffer is read before the next issue overwrites it
        issue(st + P.ring);
    }
    cp_async_wait<0>();
}

// The same probe with one bulk copy per row (the copy engine moves the whole
// row; one mbarrier per ring stage counts its bytes) instead of 16-byte
// copies issued by every lane.  Every wait is bounded: on timeout the join's
// error word is set and the warp stops (after its copies in flight land).
__device__ __forceinline__ void pb_bar_init(uint64_t* b) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"((uint32_t)__cvta_generic_to_shared(b)) : "memory");
}
__device__ __forceinline__ void pb_bar_expect(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(b)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool pb_bar_test(uint64_t* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"((uint32_t)__cvta_generic_to_shared(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void pb_bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* b) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            (uint32_t)__cvta_generic_to_shared(dst)),
        "l"(src), "r"(bytes), "r"((uint32_t)__cvta_generic_to_shared(b))
        : "memory");
}

template <int G, int NPL>
__global__ void __launch_bounds__(PB_WARPS * 32) k_probe_bulk(const __grid_constant__ PbParams P) {
    extern __shared__ __align__(16) unsigned char pbb_raw[];
    constexpr int NG = 32 / G;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int grp = lane / G, g = lane & (G - 1);
    const int64_t qi = (int64_t)blockIdx.x * PB_WARPS + warp;
    if (qi >= P.nq) return;
    unsigned char* ring = pbb_raw + (size_t)warp * P.ring * NG * P.rowpitch;
    uint64_t* bars = reinterpret_cast<uint64_t*>(pbb_raw + (size_t)PB_WARPS * P.ring * NG * P.rowpitch) +
                     warp * PB_RING;
    if (lane == 0) {
        for (int st = 0; st < P.ring; st++) pb_bar_init(bars + st);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    const int64_t qn = P.nx + qi;
    const int R = P.R;
    const int vl = lane < R ? __ldg(P.adj + qn * R + lane) : -1;
    float4 q[NPL];
    load_slots<G, NPL>(P.vec, qn, P.dp4, g, q);
    const float invq = P.metric ? __ldg(P.invn + qn) : 0.f;
    const float invl = (P.metric && vl >= 0) ? __ldg(P.invn + vl) : 0.f;
    const float inve = P.metric ? __ldg(P.invn + P.entry) : 0.f;
    const int nstage = (R + 1 + NG - 1) / NG;
    // lane 0 issues stage st: its rows' bytes on the stage's barrier, then one copy per row
    auto issue = [&](int st) {
        int v[NG];
        uint32_t bytes = 0;
#pragma unroll
        for (int r = 0; r < NG; r++) {
            const int slot = st * NG + r;
            const int vs = __shfl_sync(VJ_FULL, vl, slot & 31);
            v[r] = slot < R ? vs : (slot == R ? P.entry : -1);
            if (v[r] >= 0) bytes += (uint32_t)P.rowbytes;
        }
        if (lane == 0 && st < nstage) {
            uint64_t* b = bars + (st % P.ring);
            // the stage's buffer was read (generic proxy) before the copy engine refills it
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            pb_bar_expect(b, bytes);
            unsigned char* dst = ring + (size_t)(st % P.ring) * NG * P.rowpitch;
#pragma unroll
            for (int r = 0; r < NG; r++) {
                if (v[r] < 0) continue;
                const unsigned char* src =
                    P.xb ? reinterpret_cast<const unsigned char*>(P.xb + (int64_t)v[r] * P.kpb)
                         : reinterpret_cast<const unsigned char*>(P.vec + (int64_t)v[r] * P.dp4 * 4);
                pb_bulk_copy(dst + (size_t)r * P.rowpitch, src, (uint32_t)P.rowbytes, b);
            }
        }
    };
    int issued = 0;  // stages issued so far (stage k uses slot k % ring, phase k / ring)
    for (int st = 0; st < P.ring; st++)
        if (st < nstage) {
            issue(st);
            issued = st + 1;
        }
    bool ok = true;
    for (int st = 0; st < nstage; st++) {
        uint64_t* b = bars + (st % P.ring);
        const uint32_t par = (uint32_t)((st / P.ring) & 1);
        bool got = false;
        for (long long i = 0; i < P.spin_limit; i++) {
            if (pb_bar_test(b, par)) {
                got = true;
                break;
            }
        }
        if (!__all_sync(VJ_FULL, got)) {
            ok = false;
            break;
        }
        const int slot = st * NG + grp;
        const int vs = __shfl_sync(VJ_FULL, vl, slot & 31);
        const float ils = __shfl_sync(VJ_FULL, invl, slot & 31);
        const int v = slot < R ? vs : (slot == R ? P.entry : -1);
        const float il = slot < R ? ils : inve;
        const unsigned char* row = ring + (size_t)(st % P.ring) * NG * P.rowpitch + (size_t)grp * P.rowpitch;
        float a;
        if (P.xb) {
            uint2 xr[NPL];
#pragma unroll
            for (int k = 0; k < NPL; k++) {
                const int idx = g + k * G;
                xr[k] = idx < P.dp4 ? reinterpret_cast<const uint2*>(row)[idx] : make_uint2(0u, 0u);
            }
            a = group_sum<G>(slot_accum_bf16<NPL>(xr, q, P.metric));
        } else {
            float4 x[NPL];
#pragma unroll
            for (int k = 0; k < NPL; k++) {
                const int idx = g + k * G;
                x[k] = idx < P.dp4 ? reinterpret_cast<const float4*>(row)[idx] : f4zero();
            }
            a = group_sum<G>(slot_accum<NPL>(x, q, P.metric));
        }
        if (g == 0 && slot <= R)
            P.pkeys[qi * (R + 1) + slot] = v < 0 ? FLT_MAX : (P.metric == 0 ? a : 1.0f - a * il * invq);
        __syncwarp();  // the stage's buffer is read before it is refilled
        if (st + P.ring < nstage) {
            issue(st + P.ring);
            issued = st + P.ring + 1;
        }
    }
    if (!ok && lane == 0) {
        atomicCAS(P.ctr + C_ERR, 0ull, (unsigned long long)VJ_DERR_WAIT_TIMEOUT);
        atomicExch(P.ctr + C_ABORT, 1ull);
        // the copies in flight land before the block's shared memory goes away:
        // each slot's last issued stage completes its phase (bounded waits)
        for (int k = max(0, issued - P.ring); k < issued; k++)
            for (long long i = 0; i < P.spin_limit && !pb_bar_test(bars + (k % P.ring), (uint32_t)((k / P.ring) & 1));
                 i++) {
            }
    }
}

template <int G, int NPL>
void launch_probe_t(const PbParams& P, cudaStream_t st) {
    constexpr int NG = 32 / G;
    const size_t smem = (size_t)PB_WARPS * P.ring * NG * P.rowpitch;
    if (P.bulk) {
        const size_t sm2 = smem + (size_t)PB_WARPS * PB_RING * sizeof(uint64_t);
        VJ_CUDA(cudaFuncSetAttribute(k_probe_bulk<G, NPL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2));
        k_probe_bulk<G, NPL><<<(unsigned)vj_div_up(P.nq, PB_WARPS), PB_WARPS * 32, sm2, st>>>(P);
    } else {
        VJ_CUDA(cudaFuncSetAttribute(k_probe<G, NPL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_probe<G, NPL><<<(unsigned)vj_div_up(P.nq, PB_WARPS), PB_WARPS * 32, smem, st>>>(P);
    }
    VJ_LAUNCH_CHECK();
}

template <int G, int NPL, int U>
__global__ void __launch_bounds__(WPB * 32, JOIN_MIN_BLOCKS(NPL, U)) k_join(const __grid_constant__ JoinParams P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpSmem* S = reinterpret_cast<WarpSmem*>(smem_raw) + warp;
    const int64_t gw = (int64_t)blockIdx.x * WPB + warp;
    JoinCounters cnt;
    for (;;) {
        int t = 0;
        if (lane == 0) t = (int)atomicAdd(P.ctr + pass_ticket_slot(P.mode), 1ull);
        t = __shfl_sync(VJ_FULL, t, 0);
        if (t >= P.nq) break;
        if (join_query<G, NPL, U>(P, t, S, gw, lane, cnt)) break;
    }
    if (lane == 0) flush_counters(P, cnt);
}

// One join pass over up to JB_MAX independent indexes in a single launch (a
// collection of join instances).  The tickets of all instances form one
// sequence, instance after instance, each instance's part in its own dispatch
// order, so a parent's ticket still precedes its children's (pass 3 waits on
// parents of its own instance only, and a claimed ticket is always being
// worked on by a running warp).  Each instance keeps its own counters, pool
// and outputs; all share the warps' workspace.
constexpr int JB_MAX = 64;
struct JoinBatch {
    JoinParams p[JB_MAX];
    int64_t qstart[JB_MAX + 1];  // ticket offsets: instance i owns [qstart[i], qstart[i+1])
    int n;
    unsigned long long* ticket;  // one counter for this launch
};
static_assert(sizeof(JoinBatch) <= 32000, "JoinBatch must fit the kernel parameter space");

template <int G, int NPL, int U>
__global__ void __launch_bounds__(WPB * 32, JOIN_MIN_BLOCKS(NPL, U)) k_join_multi(const __grid_constant__ JoinBatch B) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpSmem* S = reinterpret_cast<WarpSmem*>(smem_raw) + warp;
    const int64_t gw = (int64_t)blockIdx.x * WPB + warp;
    const int64_t total = B.qstart[B.n];
    JoinCounters cnt;
    int cur = -1;
    for (;;) {
        long long t = 0;
        if (lane == 0) t = (long long)atomicAdd(B.ticket, 1ull);
        t = __shfl_sync(VJ_FULL, t, 0);
        if (t >= total) break;
        int lo = 0, hi = B.n - 1;  // the instance: last i with qstart[i] <= t
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (B.qstart[mid] <= t) lo = mid;
            else hi = mid - 1;
        }
        if (lo != cur) {
            if (cur >= 0 && lane == 0) flush_counters(B.p[cur], cnt);
            cnt = JoinCounters();
            cur = lo;
        }
        if (join_query<G, NPL, U>(B.p[lo], (int)(t - B.qstart[lo]), S, gw, lane, cnt)) break;
    }
    if (cur >= 0 && lane == 0) flush_counters(B.p[cur], cnt);
}

// Dispatch order for passes without dependencies: longest expected work first
// (the previous join's visited counts, in power-of-two classes), so the long
// queries start early and the kernel's tail is short.  Counting sort over 32
// classes; the order within a class is arbitrary (results do not depend on it).
constexpr int CO_CLASSES = 32;

__device__ __forceinline__ int cost_class(int steps) {
    return CO_CLASSES - 1 - min(CO_CLASSES - 1, 31 - __clz(max(steps, 0) + 1));
}

__global__ void k_cost_hist(const int32_t* __restrict__ steps, int64_t n, int* __restrict__ hist) {
    __shared__ int h[CO_CLASSES];
    if (threadIdx.x < CO_CLASSES) h[threadIdx.x] = 0;
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&h[cost_class(steps[i])], 1);
    __syncthreads();
    if (threadIdx.x < CO_CLASSES && h[threadIdx.x]) atomicAdd(&hist[threadIdx.x], h[threadIdx.x]);
}

// exclusive prefix of the class counts into cursors (one warp)
__global__ void k_cost_prefix(int* __restrict__ hist) {
    const int lane = threadIdx.x;
    const int v = hist[lane];
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(VJ_FULL, x, o);
        if (lane >= o) x += y;
    }
    hist[lane] = x - v;
}

__global__ void k_cost_scatter(const int32_t* __restrict__ steps, int64_t n, int* __restrict__ cursor,
                               int32_t* __restrict__ order) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) order[atomicAdd(&cursor[cost_class(steps[i])], 1)] = (int32_t)i;
}

// rows of routed queries: CSR rows of the scan, placed at `base` in the pool
__global__ void k_merge_routed(const int32_t* __restrict__ routed, int64_t nr, const int64_t* __restrict__ soff,
                               int64_t base, int64_t* __restrict__ seg, int32_t* __restrict__ count) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nr) return;
    const int q = routed[i];
    seg[q] = base + soff[q];
    count[q] = (int32_t)(soff[q + 1] - soff[q]);
}

// Soft sharing, between passes 2 and 3.  A query is locally changed when,
// with its parent's pass-1 cache as the seed, pass 2 decided a cache other
// than its own pass-1 cache (one more visit that found a closer node, or a
// re-run that did).  anc[q] = 1 when some MST ancestor of q is locally
// changed.  A query with anc[q] = 0 has, by induction from the root, every
// ancestor's final cache equal to its pass-1 cache, so its parent's final
// cache is the seed pass 2 decided for: pass 3 commits it without waiting.
// Pointer jumping over the parent links: after round k, anc covers the
// ancestors up to 2^k levels up and jmp points 2^k levels up.
__global__ void k_anc_init(const int32_t* __restrict__ parent, const uint8_t* __restrict__ outc,
                           const int32_t* __restrict__ cout, const int32_t* __restrict__ cache1,
                           const int32_t* __restrict__ cache2, int64_t nq, uint8_t* __restrict__ anc,
                           int32_t* __restrict__ jmp) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    const int32_t p = parent[q];
    uint8_t a = 0;
    if (p >= 0) {
        const int o = outc[p];
        a = (uint8_t)((o == 1 && cout[p] != cache1[p]) || (o == 2 && cache2[p] != cache1[p]));
    }
    anc[q] = a;
    jmp[q] = p;
}

__global__ void k_anc_jump(const uint8_t* __restrict__ anc_in, const int32_t* __restrict__ jmp_in, int64_t nq,
                           uint8_t* __restrict__ anc_out, int32_t* __restrict__ jmp_out) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    uint8_t a = anc_in[q];
    int32_t j = jmp_in[q];
    if (j >= 0) {
        a |= anc_in[j];
        j = jmp_in[j];
    }
    anc_out[q] = a;
    jmp_out[q] = j;
}

template <int G, int NPL, int U>
void launch_join_t(const JoinParams& P, int blocks, cudaStream_t st) {
    size_t smem = sizeof(WarpSmem) * WPB;
    k_join<G, NPL, U><<<blocks, WPB * 32, smem, st>>>(P);
    VJ_LAUNCH_CHECK();
}

template <int G, int NPL, int U>
void launch_join_multi_t(const JoinBatch& B, int blocks, cudaStream_t st) {
    size_t smem = sizeof(WarpSmem) * WPB;
    k_join_multi<G, NPL, U><<<blocks, WPB * 32, smem, st>>>(B);
    VJ_LAUNCH_CHECK();
}

template <class K>
int blocks_for(K kern, int num_sms) {
    size_t smem = sizeof(WarpSmem) * WPB;
    VJ_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // the largest shared-memory carveout, so two blocks' warp state fits an SM
    VJ_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared));
    int per_sm = 0;
    VJ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, WPB * 32, smem));
    if (per_sm < 1) per_sm = 1;
    return per_sm * num_sms;
}

// dispatch on the padded dimension (dp4 = dp / 4 float4 slots per vector)
struct JoinDispatch {
    int cls;  // template class: indexes of one class can share a multi-instance launch
    int blocks;
    void (*launch)(const JoinParams&, int, cudaStream_t);
    int blocks_multi;
    void (*launch_multi)(const JoinBatch&, int, cudaStream_t);
    int G;    // lanes per candidate of the class (the probe kernel's rows per stage: 32 / G)
    int NPL;  // 16-byte slots per lane
    void (*launch_probe)(const PbParams&, cudaStream_t);
};

template <int G, int NPL, int U>
JoinDispatch dispatch_t(int cls, int num_sms) {
    return {cls, blocks_for(k_join<G, NPL, U>, num_sms), launch_join_t<G, NPL, U>,
            blocks_for(k_join_multi<G, NPL, U>, num_sms), launch_join_multi_t<G, NPL, U>, G, NPL,
            launch_probe_t<G, NPL>};
}

constexpr int JOIN_CLASSES = 9;

// the classes by row capacity (16-byte slots per row: G * NPL), with their
// template parameters; the tuner may run a row on any class that holds it
struct JoinClass {
    int cls, G, NPL, U;
};
constexpr JoinClass JOIN_CLASS_TABLE[JOIN_CLASSES] = {{0, 8, 1, 4},  {1, 8, 2, 4},  {2, 8, 4, 2},
                                                      {3, 16, 4, 2}, {4, 32, 4, 2}, {8, 32, 6, 2},
                                                      {5, 32, 8, 1}, {6, 32, 16, 1}, {7, 32, 32, 1}};

JoinDispatch dispatch_cls(int cls, int num_sms) {
    switch (cls) {
        case 0: return dispatch_t<8, 1, 4>(0, num_sms);
        case 1: return dispatch_t<8, 2, 4>(1, num_sms);
        case 2: return dispatch_t<8, 4, 2>(2, num_sms);
        case 3: return dispatch_t<16, 4, 2>(3, num_sms);
        case 4: return dispatch_t<32, 4, 2>(4, num_sms);
        case 8: return dispatch_t<32, 6, 2>(8, num_sms);
        case 5: return dispatch_t<32, 8, 1>(5, num_sms);
        case 6: return dispatch_t<32, 16, 1>(6, num_sms);
        default: return dispatch_t<32, 32, 1>(7, num_sms);
    }
}

// the smallest class that holds a row of dp4 slots.  Up to 768 floats: six
// 16-byte slots per lane and two candidates in flight per warp (eight slots
// and one candidate left the warp waiting on one row's gathers at a time)
int pick_cls_only(int dp4) {
    if (dp4 <= 8) return 0;
    if (dp4 <= 16) return 1;
    if (dp4 <= 32) return 2;
    if (dp4 <= 64) return 3;
    if (dp4 <= 128) return 4;
    if (dp4 <= 192) return 8;
    if (dp4 <= 256) return 5;
    if (dp4 <= 512) return 6;
    return 7;
}

JoinDispatch pick(int dp4, int num_sms) { return dispatch_cls(pick_cls_only(dp4), num_sms); }

// Host state of one join between its phases: setup (prologue, buffers,
// parameters), the traversal passes (alone or inside a multi-instance
// launch), and the finish (brute-force rows, CSR, statistics).
struct JoinRun {
    vj_index* ix = nullptr;
    float eps = 0.f;
    int budget = 0;
    bool learned = false, soft = false;
    bool wait_first = false;  // separate indexes with sharing: one pass, parents first (mode 4)
    bool probe = false;       // probe keys from k_probe before the first pass
    PbParams pb;
    double ms_pro = 0.0;
    JoinParams P;
    JoinDispatch jd;
    int64_t wstride = 0, vwords = 0;  // this join's workspace needs per warp
    unsigned long long hc[16];
    int64_t launches = 0;
    float t_trav = 0.f, t_sws[3] = {0.f, 0.f, 0.f};
    int gather_bytes = 4;  // bytes per coordinate the traversal gathers (4 FP32, 2 BF16)
    ~JoinRun() {
        // the plan the learned prologue set lives for this join only
        if (learned && ix) {
            ix->has_route = false;
            ix->has_beam = false;
            ix->nrouted = 0;
        }
    }
};

// anc of k_anc_init / k_anc_jump for the join's index, after its pass 2 (on
// the stream, no host wait); nullptr when every query must wait (the
// wait-test knob holds a query back)
const uint8_t* anc_compute(JoinRun& r, cudaStream_t s) {
    vj_index* ix = r.ix;
    const int64_t nq = ix->nq;
    if (ix->hold_q >= 0 || nq == 0) return nullptr;
    ix->anc.ensure(2 * (size_t)nq, s);
    ix->jmp.ensure(2 * (size_t)nq, s);
    uint8_t* a[2] = {ix->anc.p, ix->anc.p + nq};
    int32_t* j[2] = {ix->jmp.p, ix->jmp.p + nq};
    const JoinParams& P = r.P;
    const int g = vj_div_up(nq, 256);
    k_anc_init<<<g, 256, 0, s>>>(P.parent, P.outc, P.cout, P.cache1, P.cache2, nq, a[0], j[0]);
    VJ_LAUNCH_CHECK();
    r.launches++;
    int cur = 0;
    for (int64_t span = 1; span < (int64_t)ix->max_depth; span <<= 1) {
        k_anc_jump<<<g, 256, 0, s>>>(a[cur], j[cur], nq, a[cur ^ 1], j[cur ^ 1]);
        VJ_LAUNCH_CHECK();
        r.launches++;
        cur ^= 1;
    }
    return a[cur];
}

void join_setup(JoinRun& r) {
    vj_index* ix = r.ix;
    cudaStream_t s = ix->stream;
    const int64_t nq = ix->nq;
    VJ_REQUIRE(ix->d <= 4096 && ix->dp / 4 <= 1024, VJ_ERR_ARG, "d too large for the join kernel");
    VJ_REQUIRE(ix->R <= 32, VJ_ERR_ARG, "the GPU join supports degree <= 32");
    VJ_REQUIRE(ix->p.work_sharing != VJ_WS_HARD || ix->separate, VJ_ERR_ARG,
               "work_sharing=hard runs on separate indexes only (the merged index's hard sharing is not built)");
    VJ_REQUIRE(ix->p.work_sharing >= 0 && ix->p.work_sharing <= 3, VJ_ERR_ARG, "bad work_sharing");

    VJ_REQUIRE(!ix->nnmap || (ix->p.learned == 0 && !ix->has_route && !ix->has_beam), VJ_ERR_STATE,
               "an NN-Map index joins from its witnesses: no learned route or per-query plan");

    // learned prologue (features -> predictor -> per-query plan) in place of
    // the d1/d2 rule
    r.learned = ix->p.learned != 0;
    if (r.learned) {
        cudaEvent_t p0, p1;
        VJ_CUDA(cudaEventCreate(&p0));
        VJ_CUDA(cudaEventCreate(&p1));
        VJ_CUDA(cudaEventRecord(p0, s));
        vj_learned_prologue(ix, r.eps);
        VJ_CUDA(cudaEventRecord(p1, s));
        VJ_CUDA(cudaEventSynchronize(p1));
        float t = 0.f;
        VJ_CUDA(cudaEventElapsedTime(&t, p0, p1));
        r.ms_pro = t;
        cudaEventDestroy(p0);
        cudaEventDestroy(p1);
    }

    ix->cache.ensure(nq, s);
    ix->steps.ensure(nq, s);
    ix->hyb.ensure(nq, s);
    ix->count.ensure(nq, s);
    ix->seg.ensure(nq, s);
    ix->done.ensure(nq, s);
    ix->qflag.ensure(nq, s);
    ix->ckey.ensure(nq, s);
    ix->cache1.ensure(nq, s);
    ix->sca.ensure(nq, s);
    ix->outc.ensure(nq, s);
    ix->cout.ensure(nq, s);
    ix->cache2.ensure(nq, s);
    ix->steps2.ensure(nq, s);
    ix->hyb2.ensure(nq, s);
    ix->count2.ensure(nq, s);
    ix->seg2.ensure(nq, s);
    ix->ctr.ensure(16, s);

    static_assert(FB * 32 <= CCAP, "BFS batch exceeds the candidate buffer");
    r.jd = ix->tune_cls >= 0 ? dispatch_cls(ix->tune_cls, ix->num_sms) : pick(ix->dp / 4, ix->num_sms);
    if (ix->tune_blocks > 0) {
        r.jd.blocks = std::min(r.jd.blocks, ix->tune_blocks);
        r.jd.blocks_multi = std::min(r.jd.blocks_multi, ix->tune_blocks);
    }
    // global visited regions: up to 2^17 slots (64K visited nodes per query),
    // no larger than needed for the whole node set
    int gmax = 1 << 17;
    while (gmax > GCAP0 && (int64_t)gmax / 4 >= ix->n) gmax >>= 1;
    if (gmax < GCAP0) gmax = GCAP0;
    const int grcap = gmax / 2;
    const int hbeam = r.budget > 0 ? r.budget : ix->p.hybrid_beam;
    // the out-range queue; on separate indexes also the greedy queue (gbeam + 1 seeds)
    const int oqcap = std::max(std::max(hbeam, ix->has_beam ? ix->plan_max_beam : 0),
                               ix->separate ? ix->p.greedy_beam + 1 : 0) + 2;
    r.wstride = ((int64_t)2 * gmax + 2 * grcap + 4 * oqcap + 31) / 32 * 32;
    r.vwords = (ix->n + 31) / 32;
    if (ix->pool_id.n == 0) {
        int64_t cap0 = std::max<int64_t>(nq * 64, 1 << 16);
        ix->pool_id.alloc(cap0, s);
        ix->pool_d.alloc(cap0, s);
    }

    JoinParams& P = r.P;
    P.vec = ix->vec.p;
    P.invn = ix->invn.p;
    P.adj = ix->adj.p;
    P.elen = ix->elen.p;
    P.parent = ix->parent.p;
    P.done = ix->done.p;
    P.qflag = ix->qflag.p;
    P.ckey = ix->ckey.p;
    P.cache1 = ix->cache1.p;
    P.sca = ix->sca.p;
    P.outc = ix->outc.p;
    P.cout = ix->cout.p;
    P.cache2 = ix->cache2.p;
    P.steps2 = ix->steps2.p;
    P.hyb2 = ix->hyb2.p;
    P.count2 = ix->count2.p;
    P.seg2 = ix->seg2.p;
    P.order = ix->order.p;
    // longest-first order from the previous join's visited counts (MST order on the first join)
    if (ix->have_costs) {
        ix->order1.ensure(nq, s);
        ix->cost_hist.ensure(CO_CLASSES, s);
        VJ_CUDA(cudaMemsetAsync(ix->cost_hist.p, 0, CO_CLASSES * sizeof(int), s));
        k_cost_hist<<<std::min<int64_t>(vj_div_up(nq, 256), 4 * (int64_t)ix->num_sms), 256, 0, s>>>(
            ix->steps.p, nq, ix->cost_hist.p);
        k_cost_prefix<<<1, 32, 0, s>>>(ix->cost_hist.p);
        k_cost_scatter<<<vj_div_up(nq, 256), 256, 0, s>>>(ix->steps.p, nq, ix->cost_hist.p, ix->order1.p);
        VJ_LAUNCH_CHECK();
        P.order1 = ix->order1.p;
    } else {
        P.order1 = ix->order.p;
    }
    P.route = ix->has_route ? ix->plan_route.p : nullptr;
    P.qbeam = ix->has_beam ? ix->plan_beam.p : nullptr;
    P.nx = ix->nx;
    P.nq = nq;
    P.dp4 = ix->dp / 4;
    P.dp = ix->dp;
    P.d = ix->d;
    P.R = ix->R;
    P.metric = ix->metric;
    P.entry = ix->entry;
    P.ws = ix->p.work_sharing;
    P.adapt = ix->p.adapt_hybrid;
    P.force = ix->p.force_hybrid;
    P.seed_best = ix->p.hybrid_seed_best;
    P.hbeam = hbeam;
    P.conv = ix->p.conv_threshold;
    P.eps_key = ix->metric == VJ_L2 ? r.eps * r.eps : r.eps;
    // Rounding bound of the traversal's FP32 keys.  A lane sums its 4 NPL
    // products (or squared differences) in one FMA chain, then log2(G) levels
    // of a pairwise tree join the lanes: the dot product's error is at most
    // gamma_m sum|x_i q_i| with m = 4 NPL + log2 G (gamma_m = m u / (1 - m u)).
    //   L2: each difference adds one rounding, squared: relative error of the
    //       key below (m + 2) u (1 + O(u));
    //   cosine: 1 - <x,q> ix iq with ix, iq the reciprocal norms rounded once
    //       from FP64: absolute error below gamma_m (Cauchy-Schwarz bounds
    //       sum|x_i q_i| by |x||q|) + 4u (the norms and two products) + 2u
    //       (the final subtraction).
    // The band adds 25 % and a few u of slack; keys within it of eps (or of
    // another key, for the FP64 tie decisions) are re-decided in FP64.
    {
        int lg = 0;
        while ((1 << lg) < r.jd.G) lg++;
        const int m = 4 * r.jd.NPL + lg;
        P.band = (float)((double)(m + 8) * VJ_F32_U * 1.25) + 1e-9f;
    }
    P.tie_tol = P.band;
    P.eps64 = (double)r.eps;
    P.cache = ix->cache.p;
    P.steps = ix->steps.p;
    P.hyb = ix->hyb.p;
    P.count = ix->count.p;
    P.seg = ix->seg.p;
    P.gmax = gmax;
    P.grcap = grcap;
    P.oqcap = oqcap;
    P.ctr = ix->ctr.p;
    P.spin_limit = ix->wait_polls > 0 ? ix->wait_polls : (1ll << 24);  // ~seconds with back-off; then VJ_DERR_WAIT_TIMEOUT
    P.hold_q = ix->hold_q;
    // BF16 gathers when asked for and exact: every coordinate is a BF16 value
    // and the BF16 copy holds the raw rows (L2, or cosine rows kept raw)
    P.xb = nullptr;
    P.kpb = 0;
    if (ix->p.gather == VJ_PREC_BF16) {
        vj_ensure_bf16(ix);
        if (ix->bf16_lossless && (ix->metric == VJ_L2 || ix->cos_raw)) {
            P.xb = ix->xbf.p;
            P.kpb = (ix->d + 63) / 64 * 64;
        }
    }
    r.gather_bytes = P.xb ? 2 : 4;
    r.soft = ix->p.work_sharing == VJ_WS_SOFT;
    // NN-Map index: the join expands from the stored witnesses on G_X, with
    // no greedy phase and no work sharing
    P.nm_w = nullptr;
    P.nm_wd = nullptr;
    P.nm_ood = nullptr;
    P.separate = ix->separate ? 1 : 0;
    P.gbeam = ix->p.greedy_beam;
    // probe keys ahead of the traversal (merged index: every query probes N(q))
    P.pkeys = nullptr;
    P.anc = nullptr;
    r.probe = false;
    if (!ix->separate && !ix->nnmap) {
        const int ng = 32 / r.jd.G;
        const int rowbytes = P.xb ? ((ix->d * 2 + 15) / 16) * 16 : ix->dp * 4;
        const int rowpitch = (rowbytes + 127) / 128 * 128;
        int ring = std::min(PB_RING, PB_STAGE_MAX / (ng * rowpitch));
        if (ix->tune_ring >= 2) ring = std::min(ring, ix->tune_ring);
        if (ring >= 2) {
            ix->pkeys.ensure((size_t)nq * (ix->R + 1), s);
            PbParams& B = r.pb;
            B.vec = ix->vec.p;
            B.invn = ix->invn.p;
            B.xb = P.xb;
            B.kpb = P.kpb;
            B.dp4 = ix->dp / 4;
            B.metric = ix->metric;
            B.adj = ix->adj.p;
            B.R = ix->R;
            B.entry = ix->entry;
            B.nx = ix->nx;
            B.nq = nq;
            B.ring = ring;
            B.rowbytes = rowbytes;
            B.rowpitch = rowpitch;
            B.bulk = ix->tune_bulk ? 1 : 0;
            B.ctr = ix->ctr.p;
            B.spin_limit = 1ll << 24;
            B.pkeys = ix->pkeys.p;
            P.pkeys = ix->pkeys.p;
            r.probe = true;
        }
    }
    if (ix->separate) {
        r.soft = false;
        r.wait_first = ix->p.work_sharing == VJ_WS_SOFT || ix->p.work_sharing == VJ_WS_HARD;
    }
    if (ix->nnmap) {
        P.nm_w = ix->nm_w.p;
        P.nm_wd = ix->nm_wd.p;
        P.nm_ood = ix->nm_ood.p;
        r.soft = false;
    }
}

// Traversal workspaces -- the warps' spill space (visited lists, result
// spill, out-range queues) and their visited bitmaps -- are large (up to 2^17
// visited slots per warp: GBs for a persistent grid) and only a running join
// needs one.  A process-wide cache lends them out per join, so memory grows
// with the number of joins running at once, not with the number of indexes.
// The cache is emptied when the last index is freed.
struct TravSpace {
    int dev = 0;
    bool busy = false;
    DBuf<int32_t> ws;
    DBuf<uint32_t> bits;  // all zero between queries
};
std::mutex g_ts_mu;
std::vector<TravSpace*> g_ts;

// free the idle spaces of this process (all devices); the caller holds g_ts_mu
void trim_idle_locked() {
    for (auto it = g_ts.begin(); it != g_ts.end();) {
        TravSpace* t = *it;
        if (t->busy) {
            ++it;
            continue;
        }
        int cur = 0;
        cudaGetDevice(&cur);
        cudaSetDevice(t->dev);
        if (t->ws.p) cudaFree(t->ws.p);
        if (t->bits.p) cudaFree(t->bits.p);
        cudaSetDevice(cur);
        delete t;
        it = g_ts.erase(it);
    }
}

class TravLease {
  public:
    TravLease(size_t ws_need, size_t bits_need, cudaStream_t s) : s_(s) {
        int dev = 0;
        VJ_CUDA(cudaGetDevice(&dev));
        {
            std::lock_guard<std::mutex> lk(g_ts_mu);
            for (TravSpace* t : g_ts)
                if (!t->busy && t->dev == dev && (!t_ || t->ws.n + t->bits.n > t_->ws.n + t_->bits.n)) t_ = t;
            if (!t_) {
                t_ = new TravSpace();
                t_->dev = dev;
                g_ts.push_back(t_);
            }
            t_->busy = true;
        }
        try {
            grow(ws_need, bits_need);
        } catch (const VjError&) {
            // out of memory: free the other idle spaces and try once more
            cudaGetLastError();
            {
                std::lock_guard<std::mutex> lk(g_ts_mu);
                trim_idle_locked();
            }
            try {
                grow(ws_need, bits_need);
            } catch (...) {
                std::lock_guard<std::mutex> lk(g_ts_mu);
                t_->busy = false;
                throw;
            }
        }
    }
    ~TravLease() {
        // after a failed join the bitmaps may hold an abandoned query's bits;
        // the stream is done with the space before another join takes it
        if (dirty_ && t_->bits.p) cudaMemsetAsync(t_->bits.p, 0, t_->bits.n * sizeof(uint32_t), s_);
        cudaStreamSynchronize(s_);
        std::lock_guard<std::mutex> lk(g_ts_mu);
        t_->busy = false;
    }
    TravLease(const TravLease&) = delete;
    TravLease& operator=(const TravLease&) = delete;
    void bind(int64_t wstride, int64_t vwords, JoinParams& P) const {
        P.wspace = t_->ws.p;
        P.wstride = wstride;
        P.vbits = t_->bits.p;
        P.vwords = vwords;
    }
    void clean() { dirty_ = false; }

  private:
    void grow(size_t ws_need, size_t bits_need) {
        if (t_->ws.n < ws_need) {
            t_->ws.free_(s_);
            t_->ws.alloc(ws_need, s_);
        }
        if (t_->bits.n < bits_need) {
            t_->bits.free_(s_);
            t_->bits.alloc(bits_need, s_);
            VJ_CUDA(cudaMemsetAsync(t_->bits.p, 0, bits_need * sizeof(uint32_t), s_));
        }
    }
    TravSpace* t_ = nullptr;
    cudaStream_t s_;
    bool dirty_ = true;
};

void bind_pool(JoinRun& r) {
    r.P.pool_id = r.ix->pool_id.p;
    r.P.pool_d = r.ix->pool_d.p;
    r.P.pool_cap = (int64_t)r.ix->pool_id.n;
}

// counters and publish flags of one attempt
void reset_attempt(JoinRun& r, cudaStream_t s) {
    VJ_CUDA(cudaMemsetAsync(r.ix->ctr.p, 0, 16 * sizeof(unsigned long long), s));
    if (r.soft || r.wait_first) VJ_CUDA(cudaMemsetAsync(r.ix->done.p, 0, r.ix->nq * sizeof(int32_t), s));
}

// after an attempt: true when the pool overflowed (then it is grown: run
// again, the join is deterministic); throws on a device error
bool pool_overflowed(JoinRun& r) {
    const unsigned long long* hc = r.hc;
    if (hc[C_ERR] != 0) {
        const int code = (int)hc[C_ERR];
        if (code == VJ_DERR_WAIT_TIMEOUT) {
            vj_set_error("join: a wait for a work-sharing parent timed out");
            throw VjError{VJ_ERR_TIMEOUT};
        }
        vj_set_error("join: device error %d (%s)", code,
                     code == VJ_DERR_VISITED_OVERFLOW ? "visited set above per-query capacity"
                     : code == VJ_DERR_RESULT_OVERFLOW ? "result list above per-query capacity"
                                                        : "queue overflow");
        throw VjError{VJ_ERR_STATE};
    }
    if ((int64_t)hc[C_POOL] <= r.P.pool_cap) return false;
    vj_index* ix = r.ix;
    const int64_t cap = (int64_t)hc[C_POOL] + hc[C_POOL] / 4 + 1024;
    ix->pool_id.free_(ix->stream);
    ix->pool_d.free_(ix->stream);
    ix->pool_id.alloc(cap, ix->stream);
    ix->pool_d.alloc(cap, ix->stream);
    return true;
}

struct Events {
    cudaEvent_t e[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    Events() {
        for (auto& x : e) VJ_CUDA(cudaEventCreate(&x));
    }
    ~Events() {
        for (auto& x : e)
            if (x) cudaEventDestroy(x);
    }
};

// the brute-force rows of routed queries, the CSR and the statistics; the
// traversal's counters are in r.hc and its times in r.t_trav / r.t_sws
void join_finish(JoinRun& r, vj_stats* st, int64_t* nnz_out) {
    vj_index* ix = r.ix;
    cudaStream_t s = ix->stream;
    const int64_t nq = ix->nq;
    const unsigned long long* hc = r.hc;
    Events ev;
    VJ_CUDA(cudaEventRecord(ev.e[0], s));
    int64_t nnz = (int64_t)hc[C_POOL];

    // ---- brute-force route: rows of the routed queries from the tensor-core
    // scan, appended to the pool behind the traversal's pairs
    double ms_scan = 0.0, ms_route = 0.0;
    int64_t scand = 0;
    if (ix->has_route && ix->nrouted > 0) {
        DBuf<int64_t> soff;
        DBuf<int32_t> sid;
        DBuf<float> sd;
        int64_t snnz = 0;
        vj_scan_rows_csr(ix, ix->routed.p, ix->nrouted, r.eps, soff, sid, sd, &snnz, &ms_route);
        ms_scan = ix->last_scan_ms;
        scand = ix->last_scan_cand;
        r.launches += 8;
        if (nnz + snnz > (int64_t)ix->pool_id.n) {
            DBuf<int32_t> nid;
            DBuf<float> nd;
            const int64_t cap = nnz + snnz + (nnz + snnz) / 4 + 1024;
            nid.alloc(cap, s);
            nd.alloc(cap, s);
            if (nnz > 0) {
                VJ_CUDA(cudaMemcpyAsync(nid.p, ix->pool_id.p, nnz * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
                VJ_CUDA(cudaMemcpyAsync(nd.p, ix->pool_d.p, nnz * sizeof(float), cudaMemcpyDeviceToDevice, s));
            }
            ix->pool_id.free_(s);
            ix->pool_d.free_(s);
            ix->pool_id = nid;
            ix->pool_d = nd;
            nid.p = nullptr;
            nd.p = nullptr;
        }
        if (snnz > 0) {
            VJ_CUDA(cudaMemcpyAsync(ix->pool_id.p + nnz, sid.p, snnz * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
            VJ_CUDA(cudaMemcpyAsync(ix->pool_d.p + nnz, sd.p, snnz * sizeof(float), cudaMemcpyDeviceToDevice, s));
        }
        k_merge_routed<<<vj_div_up(ix->nrouted, 256), 256, 0, s>>>(ix->routed.p, ix->nrouted, soff.p, nnz, ix->seg.p,
                                                                  ix->count.p);
        VJ_LAUNCH_CHECK();
        nnz += snnz;
        soff.free_(s);
        sid.free_(s);
        sd.free_(s);
    }

    // ---- CSR: offsets by scan, then per-query sorted copy
    ix->offsets.ensure(nq + 1, s);
    ix->out_id.ensure(std::max<int64_t>(nnz, 1), s);
    ix->out_d.ensure(std::max<int64_t>(nnz, 1), s);
    vj_exclusive_scan_i32_to_i64(ix->count.p, ix->offsets.p, nq, ix);
    vj_segment_sort_copy(ix->seg.p, ix->count.p, ix->offsets.p, ix->pool_id.p, ix->pool_d.p, ix->out_id.p,
                         ix->out_d.p, nq, ix);
    VJ_CUDA(cudaEventRecord(ev.e[1], s));
    // pairs in the result (the pool also holds rows that a pass-2 re-run replaced)
    VJ_CUDA(cudaMemcpyAsync(&nnz, ix->offsets.p + nq, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    VJ_CUDA(cudaStreamSynchronize(s));
    float t_csr = 0.f;
    VJ_CUDA(cudaEventElapsedTime(&t_csr, ev.e[0], ev.e[1]));

    st->ms_sws[0] = r.t_sws[0];
    st->ms_sws[1] = r.t_sws[1];
    st->ms_sws[2] = r.t_sws[2];
    st->dist_computations = (int64_t)hc[C_DIST];
    st->expansions = (int64_t)hc[C_EXP];
    st->adj_rows_read = (int64_t)hc[C_ADJ];
    st->hybrid_queries = (int64_t)hc[C_HYB];
    st->rechecks = (int64_t)hc[C_RECHK];
    st->spill_queries = (int64_t)hc[C_SPILL];
    st->ms_traverse = r.t_trav;
    st->ms_csr = std::max(0.0, (double)t_csr - ms_route);
    st->ms_route = ms_route;
    st->ms_prologue = r.ms_pro;
    st->sws_restarts = (int64_t)hc[C_RESTART];
    st->ms_total = r.ms_pro + r.t_trav + t_csr;
    ix->have_costs = true;  // this join's visited counts order the next one
    // algorithmic bytes: one vector per distance, one adjacency row per row read
    st->bytes_algorithmic = (int64_t)hc[C_DIST] * ix->d * r.gather_bytes + (int64_t)hc[C_ADJ] * ix->R * 4;
    st->kernel_launches = r.launches + (nq > 0 ? 4 : 3);  // traversal attempts + 3-kernel scan + row sort
    st->ms_scan = ms_scan;
    st->scan_candidates = scand;
    *nnz_out = nnz;
}

}  // namespace

// ------------------------------------------------------------------ host
void vj_trav_space_trim() {
    std::lock_guard<std::mutex> lk(g_ts_mu);
    trim_idle_locked();
}

void vj_run_join(vj_index* ix, float eps, int budget, vj_stats* st, int64_t* nnz_out) {
    JoinRun r;
    r.ix = ix;
    r.eps = eps;
    r.budget = budget;
    join_setup(r);
    cudaStream_t s = ix->stream;
    JoinParams& P = r.P;
    const int64_t warps = (int64_t)r.jd.blocks * WPB;
    TravLease lease((size_t)(warps * r.wstride), (size_t)(warps * r.vwords), s);
    lease.bind(r.wstride, r.vwords, P);

    Events ev;  // e[0] start, e[1] after pass 1, e[2] after pass 2, e[3] end
    for (int attempt = 0; attempt < 3; attempt++) {
        r.launches++;
        bind_pool(r);
        reset_attempt(r, s);
        VJ_CUDA(cudaEventRecord(ev.e[0], s));
        if (r.probe && attempt == 0) {
            r.jd.launch_probe(r.pb, s);
            r.launches++;
        }
        if (r.soft) {
            // speculative pass, parallel seed decisions, parent-ordered commit
            P.mode = 1;
            r.jd.launch(P, r.jd.blocks, s);
            VJ_CUDA(cudaEventRecord(ev.e[1], s));
            P.mode = 3;
            r.jd.launch(P, r.jd.blocks, s);
            VJ_CUDA(cudaEventRecord(ev.e[2], s));
            P.anc = anc_compute(r, s);
            P.mode = 2;
            r.jd.launch(P, r.jd.blocks, s);
            P.anc = nullptr;
            r.launches += 2;
        } else {
            P.mode = r.wait_first ? 4 : 0;
            r.jd.launch(P, r.jd.blocks, s);
        }
        VJ_CUDA(cudaEventRecord(ev.e[3], s));
        VJ_CUDA(cudaMemcpyAsync(r.hc, ix->ctr.p, sizeof(r.hc), cudaMemcpyDeviceToHost, s));
        VJ_CUDA(cudaStreamSynchronize(s));
        if (!pool_overflowed(r)) break;
    }
    lease.clean();  // no device error: every query cleared its bitmap bits
    VJ_REQUIRE((int64_t)r.hc[C_POOL] <= r.P.pool_cap, VJ_ERR_STATE, "join: result pool still too small");
    VJ_CUDA(cudaEventElapsedTime(&r.t_trav, ev.e[0], ev.e[3]));
    if (r.soft) {
        VJ_CUDA(cudaEventElapsedTime(&r.t_sws[0], ev.e[0], ev.e[1]));
        VJ_CUDA(cudaEventElapsedTime(&r.t_sws[1], ev.e[1], ev.e[2]));
        VJ_CUDA(cudaEventElapsedTime(&r.t_sws[2], ev.e[2], ev.e[3]));
    }
    join_finish(r, st, nnz_out);
}

// Joins of several indexes with their traversal passes fused: every pass runs
// as one launch over all instances of one kernel class (k_join_multi), so
// that small instances fill the GPU together.  Setup and finish run per
// instance, each on its own index's stream, through `par_for`.
void vj_run_join_multi(vj_index* const* ixs, const float* eps, int n, vj_stats* st, int64_t* nnz_out,
                       const vj_par_for& par_for) {
    if (n <= 0) return;
    std::vector<JoinRun> runs(n);
    for (int i = 0; i < n; i++) {
        runs[i].ix = ixs[i];
        runs[i].eps = eps[i];
        runs[i].budget = 0;
    }
    par_for(n, [&](int i) { join_setup(runs[i]); });

    // one workspace for all, sized for the widest needs; the fused passes run
    // on the largest instance's stream
    int owner = 0;
    int64_t warps = 0, wstride = 0, vwords = 0;
    for (int i = 0; i < n; i++) {
        warps = std::max<int64_t>(warps, (int64_t)runs[i].jd.blocks_multi * WPB);
        wstride = std::max(wstride, runs[i].wstride);
        vwords = std::max(vwords, runs[i].vwords);
        if (ixs[i]->n > ixs[owner]->n) owner = i;
    }
    cudaStream_t s = ixs[owner]->stream;
    for (int i = 0; i < n; i++) VJ_CUDA(cudaStreamSynchronize(ixs[i]->stream));
    TravLease lease((size_t)(warps * wstride), (size_t)(warps * vwords), s);
    for (int i = 0; i < n; i++) lease.bind(wstride, vwords, runs[i].P);
    DBuf<unsigned long long> ticket;
    ticket.alloc(1, s);
    std::vector<unsigned long long> hc((size_t)n * 16);
    std::vector<char> pending(n, 1);
    Events ev;
    static const int soft_modes[3] = {1, 3, 2};  // speculative pass, decisions, commit
    for (int attempt = 0; attempt < 3; attempt++) {
        std::vector<int> todo;
        for (int i = 0; i < n; i++)
            if (pending[i]) todo.push_back(i);
        if (todo.empty()) break;
        VJ_CUDA(cudaEventRecord(ev.e[0], s));
        if (attempt == 0) {
            for (int i : todo) {
                if (!runs[i].probe) continue;
                runs[i].jd.launch_probe(runs[i].pb, s);
                runs[i].launches++;
            }
        }
        for (int cls = 0; cls < JOIN_CLASSES; cls++) {
            std::vector<int> members;  // largest first: their long queries start early
            for (int i : todo)
                if (runs[i].jd.cls == cls) members.push_back(i);
            std::stable_sort(members.begin(), members.end(),
                             [&](int a, int b) { return ixs[a]->nq > ixs[b]->nq; });
            for (size_t c0 = 0; c0 < members.size(); c0 += JB_MAX) {
                const int nb = (int)std::min<size_t>(JB_MAX, members.size() - c0);
                JoinBatch B;
                B.n = nb;
                B.ticket = ticket.p;
                bool soft = false;
                for (int k = 0; k < nb; k++) {
                    JoinRun& r = runs[members[c0 + k]];
                    r.launches++;
                    bind_pool(r);
                    reset_attempt(r, s);
                    B.p[k] = r.P;
                    soft |= r.soft;
                }
                // soft-sharing instances run passes 1, 2 and 3; the others run
                // their single pass in the first launch and have no tickets in
                // the later ones
                const int npass = soft ? 3 : 1;
                const JoinDispatch& jd = runs[members[c0]].jd;
                for (int ps = 0; ps < npass; ps++) {
                    B.qstart[0] = 0;
                    for (int k = 0; k < nb; k++) {
                        JoinRun& r = runs[members[c0 + k]];
                        B.p[k].mode = r.soft ? soft_modes[ps] : (r.wait_first ? 4 : 0);
                        B.p[k].anc = (r.soft && soft_modes[ps] == 2) ? anc_compute(r, s) : nullptr;
                        const int64_t qk = (r.soft || ps == 0) ? r.ix->nq : 0;
                        B.qstart[k + 1] = B.qstart[k] + qk;
                        if (ps > 0 && r.soft) r.launches++;
                    }
                    VJ_CUDA(cudaMemsetAsync(ticket.p, 0, sizeof(unsigned long long), s));
                    jd.launch_multi(B, jd.blocks_multi, s);
                }
            }
        }
        VJ_CUDA(cudaEventRecord(ev.e[3], s));
        for (int i : todo)
            VJ_CUDA(cudaMemcpyAsync(&hc[(size_t)i * 16], ixs[i]->ctr.p, 16 * sizeof(unsigned long long),
                                    cudaMemcpyDeviceToHost, s));
        VJ_CUDA(cudaStreamSynchronize(s));
        float t = 0.f;
        VJ_CUDA(cudaEventElapsedTime(&t, ev.e[0], ev.e[3]));
        for (int i : todo) {
            JoinRun& r = runs[i];
            memcpy(r.hc, &hc[(size_t)i * 16], sizeof(r.hc));
            r.t_trav += t;
            try {
                pending[i] = pool_overflowed(r) ? 1 : 0;
            } catch (const VjError&) {
                char msg[900];
                snprintf(msg, sizeof(msg), "%s", vj_last_error());
                vj_set_error("instance %d: %s", i, msg);
                ticket.free_(s);
                throw;
            }
        }
    }
    ticket.free_(s);
    lease.clean();  // no device error in any instance
    for (int i = 0; i < n; i++)
        VJ_REQUIRE(!pending[i], VJ_ERR_STATE, "instance %d: join result pool still too small", i);
    // the instances' streams continue after the fused passes
    VJ_CUDA(cudaEventRecord(ev.e[4], s));
    for (int i = 0; i < n; i++) VJ_CUDA(cudaStreamWaitEvent(ixs[i]->stream, ev.e[4], 0));
    par_for(n, [&](int i) { join_finish(runs[i], st + i, nnz_out + i); });
}

// ------------------------------------------------------------------ tuning
// The traversal settings a tuner may choose for rows of dp4 slots: the
// default class (the smallest that holds the row) and the next larger ones.
int vj_join_class_count() { return JOIN_CLASSES; }
void vj_join_class_info(int k, int* cls, int* G, int* NPL, int* U) {
    const JoinClass& c = JOIN_CLASS_TABLE[k];
    *cls = c.cls;
    *G = c.G;
    *NPL = c.NPL;
    *U = c.U;
}
int vj_join_default_class(int dp4) { return pick_cls_only(dp4); }
int vj_join_max_blocks(int cls, int num_sms) { return dispatch_cls(cls, num_sms).blocks; }
