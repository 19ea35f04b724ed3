// k_join.cu -- the online merged-index join (Alg. 1 with Alg. 3-8), one warp
// per query, persistent grid fed by a device ticket counter.
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
//                      bounded out-range queue, (key, id) order) with the
//                      trim-after-insert rule.
//   UpdateCache (8)    C[q] = closest visited data node, ties by id, FP64
//                      re-decided among FP32 near-ties; then q is published
//                      (release) so its MST children can start.
//
// Work sharing dependencies: queries are taken in a topological order of the
// MST (BFS by depth), so a query's parent was taken earlier by a running warp;
// the child spins (bounded, with back-off) on the parent's done stamp.  On
// timeout the kernel records VJ_DERR_WAIT_TIMEOUT, raises an abort flag and
// every warp returns.
//
// Visited set: open-addressing hash in shared memory (HCAP slots, spills to a
// per-warp global table above half load).  Results: shared-memory list
// (RCAP) spilling to per-warp global memory.  In-range decisions whose FP32 key
// lies within the FP32 rounding bound of eps are re-decided in FP64.
#include <float.h>

#include "vj_device.cuh"
#include "vj_internal.cuh"

namespace {

constexpr int WPB = 8;     // warps per block
constexpr int HCAP = 2048; // shared-memory visited slots per warp
constexpr int RCAP = 256;  // shared-memory result slots per warp
constexpr int CCAP = 128;  // candidate slots per batch

struct WarpSmem {
    int htab[HCAP];
    int rid[RCAP];
    float rd[RCAP];
    int cand[CCAP];
    float ckey[CCAP];
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
    C_NUM = 10
};

struct JoinParams {
    const float* vec;
    const float* invn;
    const int32_t* adj;
    const float* elen;
    const int32_t* order;
    const int32_t* parent;
    int64_t nx, nq;
    int dp4, dp, d, R, metric;
    int32_t entry;
    int ws, adapt, force, hbeam, conv;
    float eps_key;  // L2: eps^2, cosine: eps
    float band;     // |key - eps_key| <= band * scale -> FP64 re-decision
    float tie_tol;  // keys closer than this (relative / absolute) are re-decided in FP64
    double eps64;
    int32_t* cache;
    int* done;
    int gen;
    int32_t* steps;
    uint8_t* hyb;
    int32_t* count;
    int64_t* seg;
    int32_t* pool_id;
    float* pool_d;
    int64_t pool_cap;
    int32_t* wspace;
    int64_t wstride;
    int gcap;   // global visited slots per warp (power of two)
    int oqcap;  // out-range queue capacity
    unsigned long long* ctr;
    long long spin_limit;
};

__device__ __forceinline__ float key_band_scale(const JoinParams& P) { return P.metric == 0 ? P.eps_key : 1.0f; }

// key -> distance
__device__ __forceinline__ float key_to_dist(const JoinParams& P, float k) {
    return P.metric == 0 ? sqrtf(fmaxf(k, 0.f)) : k;
}

struct QueryState {
    int* tab;
    unsigned mask;
    int nvis;
    int vislimit;
    bool vspill;
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

// make room for `m` more visited entries (spills shared -> global once)
__device__ bool vis_reserve(const JoinParams& P, QueryState& s, int m, int* gtab, int lane, long long& c_spill) {
    if (s.nvis + m <= s.vislimit) return true;
    if (s.vspill) {
        if (lane == 0) raise_err(P, VJ_DERR_VISITED_OVERFLOW);
        return false;
    }
    for (int i = lane; i < P.gcap; i += 32) gtab[i] = -1;
    __syncwarp();
    unsigned gmask = (unsigned)P.gcap - 1u;
    for (int i = lane; i < HCAP; i += 32) {
        int k = s.tab[i];
        if (k >= 0) hash_insert(gtab, gmask, k);
    }
    __syncwarp();
    s.tab = gtab;
    s.mask = gmask;
    s.vislimit = P.gcap / 2;
    s.vspill = true;
    if (lane == 0) c_spill++;
    if (s.nvis + m > s.vislimit) {
        if (lane == 0) raise_err(P, VJ_DERR_VISITED_OVERFLOW);
        return false;
    }
    return true;
}

__device__ bool res_reserve(const JoinParams& P, QueryState& s, int m, int* grid, float* grd, int lane) {
    if (s.nres + m <= s.rcap) return true;
    if (s.rspill) {
        if (lane == 0) raise_err(P, VJ_DERR_RESULT_OVERFLOW);
        return false;
    }
    for (int i = lane; i < s.nres; i += 32) {
        grid[i] = s.rid[i];
        grd[i] = s.rd[i];
    }
    __syncwarp();
    s.rid = grid;
    s.rd = grd;
    s.rcap = P.gcap / 2;
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
    const unsigned lt = (1u << lane) - 1u;
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
    (void)lt;
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

// append in-range candidates (one per lane) to the result list
__device__ __forceinline__ bool append_results(const JoinParams& P, QueryState& s, bool in, int node, float k,
                                               int* grid, float* grd, int lane) {
    unsigned m = __ballot_sync(VJ_FULL, in);
    int cnt = __popc(m);
    if (cnt == 0) return true;
    if (!res_reserve(P, s, cnt, grid, grd, lane)) return false;
    if (in) {
        int pos = s.nres + __popc(m & ((1u << lane) - 1u));
        s.rid[pos] = node;
        s.rd[pos] = k;  // keys stay keys until the output copy
    }
    s.nres += cnt;
    __syncwarp();
    return true;
}

template <int G, int NPL, int U>
__global__ void __launch_bounds__(WPB * 32) k_join(JoinParams P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpSmem* S = reinterpret_cast<WarpSmem*>(smem_raw) + warp;
    const int64_t gw = (int64_t)blockIdx.x * WPB + warp;
    int32_t* wbase = P.wspace + gw * P.wstride;
    int* gtab = wbase;
    int* grid = wbase + P.gcap;
    float* grd = reinterpret_cast<float*>(wbase + P.gcap + P.gcap / 2);
    float* oqk = reinterpret_cast<float*>(wbase + 2 * P.gcap);
    int* oqi = wbase + 2 * P.gcap + P.oqcap;
    const int g = lane & (G - 1);
    const int R = P.R;
    const int FB = R <= 32 ? (CCAP / 32) / ((R + 31) / 32) : 1;  // frontier nodes per BFS batch
    long long c_dist = 0, c_exp = 0, c_adj = 0, c_hyb = 0, c_rechk = 0, c_spill = 0;

    for (;;) {
        int t = 0;
        if (lane == 0) t = (int)atomicAdd(P.ctr + C_TICKET, 1ull);
        t = __shfl_sync(VJ_FULL, t, 0);
        if (t >= P.nq) break;
        if (*((volatile unsigned long long*)(P.ctr + C_ABORT))) break;
        const int qi = P.order[t];
        const int64_t qn = P.nx + qi;

        // ---- Alg. 3 SeedPhase (dependency on the MST parent under soft sharing)
        int seedc = -1;
        if (P.ws == VJ_WS_SOFT) {
            int par = P.parent[qi];
            if (par >= 0) {
                int ok = 1;
                if (lane == 0) {
                    long long spins = 0;
                    unsigned ns = 32;
                    while (ld_acquire(P.done + par) != P.gen) {
                        if (++spins > P.spin_limit ||
                            *((volatile unsigned long long*)(P.ctr + C_ABORT))) {
                            ok = 0;
                            break;
                        }
                        __nanosleep(ns);
                        if (ns < 1024) ns <<= 1;
                    }
                    if (!ok && spins > P.spin_limit) raise_err(P, VJ_DERR_WAIT_TIMEOUT);
                }
                ok = __shfl_sync(VJ_FULL, ok, 0);
                if (!ok) break;
                if (lane == 0) seedc = *((volatile int*)(P.cache + par));
                seedc = __shfl_sync(VJ_FULL, seedc, 0);
            }
        }

        float4 q[NPL];
        load_slots<G, NPL>(P.vec, qn, P.dp4, g, q);
        const float invq = P.metric ? __ldg(P.invn + qn) : 0.f;

        QueryState s;
        s.tab = S->htab;
        s.mask = HCAP - 1;
        s.nvis = 0;
        s.vislimit = HCAP / 2;
        s.vspill = false;
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

        // ---- Alg. 4 greedy: the seeds
        // lanes 0..2 hold the seed candidates: entry, cached seed, q itself
        int sid = -1;
        if (lane == 0) sid = P.entry;
        if (lane == 1 && seedc >= 0) sid = seedc;
        if (lane == 2 && (P.ws == VJ_WS_SELF || P.ws == VJ_WS_SOFT)) sid = (int)qn;
        // dedup in seed order (lane order), insert into visited
        bool snew = false;
#pragma unroll 1
        for (int src = 0; src < 3; src++) {
            int v = __shfl_sync(VJ_FULL, sid, src);
            int ins = 0;
            if (lane == 0 && v >= 0) ins = hash_insert(s.tab, s.mask, v);
            ins = __shfl_sync(VJ_FULL, ins, 0);
            if (lane == src) snew = ins == 1;
            __syncwarp();
        }
        unsigned sm = __ballot_sync(VJ_FULL, snew);
        if (snew) S->cand[__popc(sm & ((1u << lane) - 1u))] = sid;
        __syncwarp();
        int ns = __popc(sm);
        group_keys<G, NPL, U>(P.vec, P.invn, P.dp4, P.metric, q, invq, S->cand, ns, S->ckey, lane);
        __syncwarp();
        s.nvis += ns;
        float skey = FLT_MAX;
        int snode = -1;
        if (lane < ns) {
            snode = S->cand[lane];
            skey = (snode == (int)qn) ? 0.f : S->ckey[lane];
        }
        __syncwarp();
        // keys of the two possible data seeds, kept for the OOD rule
        bool sdata = lane < ns && snode < P.nx;
        bool sin = inrange_decide(P, sdata, skey, snode, qn, lane, c_rechk);
        best_update(P, s, sdata, skey, snode, lane);
        if (!append_results(P, s, sin, snode, skey, grid, grd, lane)) failed = true;

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
            fk = mk;
            fi = mi;
        }
        bool probe = !failed && ns > 0 && !(fi < P.nx && fin) && P.conv > 0 && fi == (int)qn;

        // ---- probe N(q)
        // per-lane copy of q's adjacency slot (R <= 32 handled per lane; wider
        // rows loop) with the neighbour's key for the OOD rule
        float nkey_l = FLT_MAX;
        int nid_l = -1;
        int entry_in_nq = 0, seed_in_nq = 0;
        if (probe) {
            c_adj++;
            for (int base = 0; base < R && !failed; base += 32) {
                int j = base + lane;
                int v = j < R ? __ldg(P.adj + qn * R + j) : -1;
                if (base == 0) nid_l = v;
                if (v == P.entry) entry_in_nq = 1;
                if (v >= 0 && v == seedc) seed_in_nq = 1;
                unsigned vm = __ballot_sync(VJ_FULL, v >= 0);
                if (!vis_reserve(P, s, __popc(vm), gtab, lane, c_spill)) {
                    failed = true;
                    break;
                }
                bool nw = v >= 0 && hash_insert(s.tab, s.mask, v) == 1;
                unsigned nm = __ballot_sync(VJ_FULL, nw);
                int nc = __popc(nm);
                if (nw) S->cand[__popc(nm & ((1u << lane) - 1u))] = v;
                __syncwarp();
                group_keys<G, NPL, U>(P.vec, P.invn, P.dp4, P.metric, q, invq, S->cand, nc, S->ckey, lane);
                __syncwarp();
                s.nvis += nc;
                int cv = lane < nc ? S->cand[lane] : -1;
                float ck = lane < nc ? S->ckey[lane] : FLT_MAX;
                __syncwarp();
                bool dat = lane < nc && cv < P.nx;
                bool in = inrange_decide(P, dat, ck, cv, qn, lane, c_rechk);
                best_update(P, s, dat, ck, cv, lane);
                if (!append_results(P, s, in, cv, ck, grid, grd, lane)) {
                    failed = true;
                    break;
                }
                // neighbour keys for the OOD rule (first 32 slots): freshly
                // computed ones from the candidate list, seeds from the seed lanes
                if (base == 0) {
                    int pos = nw ? __popc(nm & ((1u << lane) - 1u)) : -1;
                    float kk = __shfl_sync(VJ_FULL, ck, pos < 0 ? 0 : pos);
                    if (nw) nkey_l = kk;
                    // a neighbour that was already a seed: take the seed key
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

        // ---- Alg. 6 CheckHybrid
        int hyb = P.force;
        if (P.adapt && !failed) {
            // d1 over data neighbours of q; d2 over their data neighbours that
            // are not neighbours of q (and not q)
            bool isd = nid_l >= 0 && nid_l < P.nx;
            float d1s = isd ? key_to_dist(P, nkey_l) : 0.f;
            int n1 = __popc(__ballot_sync(VJ_FULL, isd));
            float d2s = 0.f;
            int n2 = 0;
            unsigned dm = __ballot_sync(VJ_FULL, isd);
            while (dm) {
                int src = __ffs(dm) - 1;
                dm &= dm - 1;
                int v = __shfl_sync(VJ_FULL, nid_l, src);
                c_adj++;
                for (int base = 0; base < R; base += 32) {
                    int j = base + lane;
                    int w = j < R ? __ldg(P.adj + (int64_t)v * R + j) : -1;
                    bool ok = w >= 0 && w < P.nx;
                    if (ok) {
                        bool inq = hash_contains(s.tab, s.mask, w);
                        if (inq && w == P.entry && !entry_in_nq) inq = false;
                        if (inq && w == seedc && !seed_in_nq) inq = false;
                        ok = !inq;
                    }
                    if (ok) {
                        d2s += __ldg(P.elen + (int64_t)v * R + j);
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
                    unsigned dm2 = __ballot_sync(VJ_FULL, isd);
                    while (dm2) {
                        int src = __ffs(dm2) - 1;
                        dm2 &= dm2 - 1;
                        int v = __shfl_sync(VJ_FULL, nid_l, src);
                        a1 += warp_dist64(P.vec, P.dp, P.d, P.metric, qn, v, lane);
                        for (int j = 0; j < R; j++) {
                            int w = __ldg(P.adj + (int64_t)v * R + j);
                            if (w < 0 || w >= P.nx) continue;
                            bool inq = hash_contains(s.tab, s.mask, w);
                            if (inq && w == P.entry && !entry_in_nq) inq = false;
                            if (inq && w == seedc && !seed_in_nq) inq = false;
                            if (inq) continue;
                            a2 += warp_dist64(P.vec, P.dp, P.d, P.metric, v, w, lane);
                        }
                    }
                    ood = (a1 / n1) / (a2 / n2) > 1.5;
                    if (lane == 0) c_rechk++;
                }
            }
            hyb = ood;  // Alg. 6: on the merged index adapt_hybrid decides, force otherwise
        }
        int expansions = 0;

        // ---- Alg. 7 ExpansionPhase
        if (!failed && !hyb) {
            int fp = 0;
            while (fp < s.nres) {
                int nb = min(FB, s.nres - fp);
                // gather the neighbour lists of nb frontier nodes
                if (!vis_reserve(P, s, nb * R, gtab, lane, c_spill)) {
                    failed = true;
                    break;
                }
                int nc = 0;
                for (int f = 0; f < nb; f++) {
                    int u = s.rid[fp + f];
                    for (int base = 0; base < R; base += 32) {
                        int j = base + lane;
                        int v = j < R ? __ldg(P.adj + (int64_t)u * R + j) : -1;
                        bool nw = v >= 0 && v < P.nx && hash_insert(s.tab, s.mask, v) == 1;
                        unsigned nm = __ballot_sync(VJ_FULL, nw);
                        if (nw) S->cand[nc + __popc(nm & ((1u << lane) - 1u))] = v;
                        nc += __popc(nm);
                    }
                }
                __syncwarp();
                c_adj += nb;
                expansions += nb;
                fp += nb;
                if (nc == 0) continue;
                group_keys<G, NPL, U>(P.vec, P.invn, P.dp4, P.metric, q, invq, S->cand, nc, S->ckey, lane);
                __syncwarp();
                s.nvis += nc;
                for (int base = 0; base < nc; base += 32) {
                    int ci = base + lane;
                    int cv = ci < nc ? S->cand[ci] : -1;
                    float ck = ci < nc ? S->ckey[ci] : FLT_MAX;
                    bool val = ci < nc;
                    bool in = inrange_decide(P, val, ck, cv, qn, lane, c_rechk);
                    best_update(P, s, val, ck, cv, lane);
                    if (!append_results(P, s, in, cv, ck, grid, grd, lane)) {
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
            int osz = 0;
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
                    u = oqi[0];
                    // shift the out-range queue left by one
                    for (int base = 1; base < osz; base += 32) {
                        int i = base + lane;
                        float kk = i < osz ? oqk[i] : 0.f;
                        int ii = i < osz ? oqi[i] : 0;
                        __syncwarp();
                        if (i < osz) {
                            oqk[i - 1] = kk;
                            oqi[i - 1] = ii;
                        }
                        __syncwarp();
                    }
                    osz--;
                } else {
                    break;
                }
                expansions++;
                c_adj++;
                if (!vis_reserve(P, s, R, gtab, lane, c_spill)) {
                    failed = true;
                    break;
                }
                int nc = 0;
                for (int base = 0; base < R; base += 32) {
                    int j = base + lane;
                    int v = j < R ? __ldg(P.adj + (int64_t)u * R + j) : -1;
                    bool nw = v >= 0 && v < P.nx && hash_insert(s.tab, s.mask, v) == 1;
                    unsigned nm = __ballot_sync(VJ_FULL, nw);
                    if (nw) S->cand[nc + __popc(nm & ((1u << lane) - 1u))] = v;
                    nc += __popc(nm);
                }
                __syncwarp();
                if (nc == 0) continue;
                group_keys<G, NPL, U>(P.vec, P.invn, P.dp4, P.metric, q, invq, S->cand, nc, S->ckey, lane);
                __syncwarp();
                s.nvis += nc;
                for (int base = 0; base < nc && !failed; base += 32) {
                    int ci = base + lane;
                    bool val = ci < nc;
                    int cv = val ? S->cand[ci] : -1;
                    float ck = val ? S->ckey[ci] : FLT_MAX;
                    bool in = inrange_decide(P, val, ck, cv, qn, lane, c_rechk);
                    best_update(P, s, val, ck, cv, lane);
                    // in adjacency order: in-range -> result (pending);
                    // out-range -> sorted insert, then trim if |Q| > beam
                    unsigned inm = __ballot_sync(VJ_FULL, in && val);
                    unsigned outm = __ballot_sync(VJ_FULL, !in && val);
                    int cnt_chunk = min(32, nc - base);
                    for (int c = 0; c < cnt_chunk; c++) {
                        float kc = __shfl_sync(VJ_FULL, ck, c);
                        int vc = __shfl_sync(VJ_FULL, cv, c);
                        if ((inm >> c) & 1u) {
                            if (!res_reserve(P, s, 1, grid, grd, lane)) {
                                failed = true;
                                break;
                            }
                            if (lane == 0) {
                                s.rid[s.nres] = vc;
                                s.rd[s.nres] = kc;
                            }
                            s.nres++;
                            npend++;
                            __syncwarp();
                        } else if ((outm >> c) & 1u) {
                            // position = number of queued entries less than (kc, vc)
                            int less = 0;
                            for (int i = lane; i < osz; i += 32) less += kless(oqk[i], oqi[i], kc, vc) ? 1 : 0;
                            for (int o = 16; o > 0; o >>= 1) less += __shfl_xor_sync(VJ_FULL, less, o);
                            // shift [less, osz) right by one, from the back
                            for (int top = osz - 1; top >= less; top -= 32) {
                                int i = top - lane;
                                float kk = 0.f;
                                int ii = 0;
                                bool mv = i >= less;
                                if (mv) {
                                    kk = oqk[i];
                                    ii = oqi[i];
                                }
                                __syncwarp();
                                if (mv) {
                                    oqk[i + 1] = kk;
                                    oqi[i + 1] = ii;
                                }
                                __syncwarp();
                            }
                            if (lane == 0) {
                                oqk[less] = kc;
                                oqi[less] = vc;
                            }
                            __syncwarp();
                            osz++;
                            if (npend + osz > P.hbeam) osz--;  // drop the largest key
                        }
                    }
                }
                if (failed) break;
            }
        }
        c_exp += expansions;

        // ---- Alg. 8 UpdateCache (soft): FP64 re-decision among near-ties
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
            P.cache[qi] = best;
            __threadfence();
            st_release(P.done + qi, P.gen);
            P.steps[qi] = s.nvis;
            P.hyb[qi] = (uint8_t)hyb;
            c_dist += s.nvis;
        }
        if (failed) {
            if (lane == 0) P.count[qi] = 0;
            break;
        }

        // ---- results into the pool
        unsigned long long off = 0;
        if (lane == 0) off = atomicAdd(P.ctr + C_POOL, (unsigned long long)s.nres);
        off = __shfl_sync(VJ_FULL, off, 0);
        if (lane == 0) {
            P.count[qi] = s.nres;
            P.seg[qi] = (int64_t)off;
        }
        if ((int64_t)off + s.nres <= P.pool_cap) {
            for (int i = lane; i < s.nres; i += 32) {
                int id = s.rid[i];
                P.pool_id[off + i] = id < 0 ? ~id : id;
                P.pool_d[off + i] = key_to_dist(P, s.rd[i]);
            }
        }
        __syncwarp();
    }
    if (lane == 0) {
        atomicAdd(P.ctr + C_DIST, (unsigned long long)c_dist);
        atomicAdd(P.ctr + C_EXP, (unsigned long long)c_exp);
        atomicAdd(P.ctr + C_ADJ, (unsigned long long)c_adj);
        atomicAdd(P.ctr + C_HYB, (unsigned long long)c_hyb);
        atomicAdd(P.ctr + C_RECHK, (unsigned long long)c_rechk);
        atomicAdd(P.ctr + C_SPILL, (unsigned long long)c_spill);
    }
}

template <int G, int NPL, int U>
void launch_join_t(const JoinParams& P, int blocks, cudaStream_t st) {
    size_t smem = sizeof(WarpSmem) * WPB;
    auto kern = k_join<G, NPL, U>;
    static bool attr = false;
    if (!attr) {
        VJ_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr = true;
    }
    kern<<<blocks, WPB * 32, smem, st>>>(P);
    VJ_LAUNCH_CHECK();
}

template <int G, int NPL, int U>
int blocks_for(int num_sms) {
    size_t smem = sizeof(WarpSmem) * WPB;
    auto kern = k_join<G, NPL, U>;
    VJ_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    VJ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, WPB * 32, smem));
    if (per_sm < 1) per_sm = 1;
    return per_sm * num_sms;
}

// dispatch on the padded dimension (dp4 = dp / 4 float4 slots per vector)
struct JoinDispatch {
    int blocks;
    void (*launch)(const JoinParams&, int, cudaStream_t);
};

JoinDispatch pick(int dp4, int num_sms) {
    if (dp4 <= 8) return {blocks_for<8, 1, 4>(num_sms), launch_join_t<8, 1, 4>};
    if (dp4 <= 16) return {blocks_for<8, 2, 4>(num_sms), launch_join_t<8, 2, 4>};
    if (dp4 <= 32) return {blocks_for<8, 4, 2>(num_sms), launch_join_t<8, 4, 2>};
    if (dp4 <= 64) return {blocks_for<16, 4, 2>(num_sms), launch_join_t<16, 4, 2>};
    if (dp4 <= 128) return {blocks_for<32, 4, 2>(num_sms), launch_join_t<32, 4, 2>};
    if (dp4 <= 256) return {blocks_for<32, 8, 1>(num_sms), launch_join_t<32, 8, 1>};
    if (dp4 <= 512) return {blocks_for<32, 16, 1>(num_sms), launch_join_t<32, 16, 1>};
    return {blocks_for<32, 32, 1>(num_sms), launch_join_t<32, 32, 1>};
}

}  // namespace

// ------------------------------------------------------------------ host
void vj_run_join(vj_index* ix, float eps, int budget, vj_stats* st, int64_t* nnz_out) {
    cudaStream_t s = ix->stream;
    const int64_t nq = ix->nq;
    VJ_REQUIRE(ix->d <= 4096 && ix->dp / 4 <= 1024, VJ_ERR_ARG, "d too large for the join kernel");
    VJ_REQUIRE(ix->R <= 32, VJ_ERR_ARG, "the GPU join supports degree <= 32");
    VJ_REQUIRE(ix->p.work_sharing != VJ_WS_HARD, VJ_ERR_ARG,
               "work_sharing=hard is not implemented by the GPU join");
    VJ_REQUIRE(ix->p.work_sharing >= 0 && ix->p.work_sharing <= 3, VJ_ERR_ARG, "bad work_sharing");

    ix->done.ensure(nq, s);
    ix->cache.ensure(nq, s);
    ix->steps.ensure(nq, s);
    ix->hyb.ensure(nq, s);
    ix->count.ensure(nq, s);
    ix->seg.ensure(nq, s);
    ix->ctr.ensure(16, s);
    if (ix->gen == 0) VJ_CUDA(cudaMemsetAsync(ix->done.p, 0, nq * sizeof(int), s));
    ix->gen++;
    if (ix->gen == 0x7fffffff) {
        VJ_CUDA(cudaMemsetAsync(ix->done.p, 0, nq * sizeof(int), s));
        ix->gen = 1;
    }

    JoinDispatch jd = pick(ix->dp / 4, ix->num_sms);
    const int64_t warps = (int64_t)jd.blocks * WPB;
    int gcap = 1 << 18;
    while (gcap > 4096 && (int64_t)gcap / 4 > ix->n) gcap >>= 1;
    const int hbeam = budget > 0 ? budget : ix->p.hybrid_beam;
    const int oqcap = hbeam + 2;
    const int64_t wstride = ((int64_t)2 * gcap + 2 * oqcap + 31) / 32 * 32;
    if (ix->wspace_warps < warps || ix->wspace.n < (size_t)(warps * wstride)) {
        ix->wspace.free_(s);
        ix->wspace.alloc((size_t)(warps * wstride), s);
        ix->wspace_warps = warps;
    }
    if (ix->pool_id.n == 0) {
        int64_t cap0 = std::max<int64_t>(nq * 64, 1 << 16);
        ix->pool_id.alloc(cap0, s);
        ix->pool_d.alloc(cap0, s);
    }

    JoinParams P;
    P.vec = ix->vec.p;
    P.invn = ix->invn.p;
    P.adj = ix->adj.p;
    P.elen = ix->elen.p;
    P.order = ix->order.p;
    P.parent = ix->parent.p;
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
    P.hbeam = hbeam;
    P.conv = ix->p.conv_threshold;
    P.eps_key = ix->metric == VJ_L2 ? eps * eps : eps;
    // FP32 keys: L2 squared distance by direct differences has relative error
    // below (dp+2)u; cosine key absolute error below (dp+4)u (unit vectors)
    P.band = 2.0f * (float)(ix->dp + 4) * VJ_F32_U * (ix->metric == VJ_L2 ? 1.0f : 4.0f) + 1e-6f;
    P.tie_tol = P.band;
    P.eps64 = (double)eps;
    P.cache = ix->cache.p;
    P.done = ix->done.p;
    P.gen = ix->gen;
    P.steps = ix->steps.p;
    P.hyb = ix->hyb.p;
    P.count = ix->count.p;
    P.seg = ix->seg.p;
    P.wspace = ix->wspace.p;
    P.wstride = wstride;
    P.gcap = gcap;
    P.oqcap = oqcap;
    P.ctr = ix->ctr.p;
    P.spin_limit = 1ll << 24;  // ~seconds with back-off; then VJ_DERR_WAIT_TIMEOUT

    cudaEvent_t e0, e1, e2;
    VJ_CUDA(cudaEventCreate(&e0));
    VJ_CUDA(cudaEventCreate(&e1));
    VJ_CUDA(cudaEventCreate(&e2));
    unsigned long long hc[C_NUM];
    int64_t launches = 0;
    for (int attempt = 0; attempt < 3; attempt++) {
        launches++;
        P.pool_id = ix->pool_id.p;
        P.pool_d = ix->pool_d.p;
        P.pool_cap = (int64_t)ix->pool_id.n;
        VJ_CUDA(cudaMemsetAsync(ix->ctr.p, 0, 16 * sizeof(unsigned long long), s));
        VJ_CUDA(cudaEventRecord(e0, s));
        jd.launch(P, jd.blocks, s);
        VJ_CUDA(cudaEventRecord(e1, s));
        VJ_CUDA(cudaMemcpyAsync(hc, ix->ctr.p, sizeof(hc), cudaMemcpyDeviceToHost, s));
        VJ_CUDA(cudaStreamSynchronize(s));
        if (hc[C_ERR] != 0) break;
        if ((int64_t)hc[C_POOL] <= P.pool_cap) break;
        // pool too small: grow and run again (the join is deterministic)
        int64_t cap = (int64_t)hc[C_POOL] + hc[C_POOL] / 4 + 1024;
        ix->pool_id.free_(s);
        ix->pool_d.free_(s);
        ix->pool_id.alloc(cap, s);
        ix->pool_d.alloc(cap, s);
        ix->gen++;
        P.gen = ix->gen;
    }
    if (hc[C_ERR] != 0) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaEventDestroy(e2);
        int code = (int)hc[C_ERR];
        if (code == VJ_DERR_WAIT_TIMEOUT) {
            vj_set_error("join: a soft work-sharing wait on an MST parent timed out");
            throw VjError{VJ_ERR_TIMEOUT};
        }
        vj_set_error("join: device error %d (%s)", code,
                     code == VJ_DERR_VISITED_OVERFLOW ? "visited set above per-query capacity"
                     : code == VJ_DERR_RESULT_OVERFLOW ? "result list above per-query capacity"
                                                        : "queue overflow");
        throw VjError{VJ_ERR_STATE};
    }
    const int64_t nnz = (int64_t)hc[C_POOL];

    // ---- CSR: offsets by scan, then per-query sorted copy
    ix->offsets.ensure(nq + 1, s);
    ix->out_id.ensure(std::max<int64_t>(nnz, 1), s);
    ix->out_d.ensure(std::max<int64_t>(nnz, 1), s);
    vj_exclusive_scan_i32_to_i64(ix->count.p, ix->offsets.p, nq, ix);
    vj_segment_sort_copy(ix->seg.p, ix->count.p, ix->offsets.p, ix->pool_id.p, ix->pool_d.p, ix->out_id.p,
                         ix->out_d.p, nq, ix);
    VJ_CUDA(cudaEventRecord(e2, s));
    VJ_CUDA(cudaEventSynchronize(e2));
    float t_trav = 0.f, t_csr = 0.f;
    VJ_CUDA(cudaEventElapsedTime(&t_trav, e0, e1));
    VJ_CUDA(cudaEventElapsedTime(&t_csr, e1, e2));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(e2);

    st->dist_computations = (int64_t)hc[C_DIST];
    st->expansions = (int64_t)hc[C_EXP];
    st->adj_rows_read = (int64_t)hc[C_ADJ];
    st->hybrid_queries = (int64_t)hc[C_HYB];
    st->rechecks = (int64_t)hc[C_RECHK];
    st->spill_queries = (int64_t)hc[C_SPILL];
    st->ms_traverse = t_trav;
    st->ms_csr = t_csr;
    st->ms_total = t_trav + t_csr;
    // algorithmic bytes: one vector per distance, one adjacency row per row read
    // (plus the edge-length row for each OOD row read)
    st->bytes_algorithmic = (int64_t)hc[C_DIST] * ix->d * 4 + (int64_t)hc[C_ADJ] * ix->R * 4;
    st->kernel_launches = launches + (nq > 0 ? 4 : 3);  // traversal attempts + 3-kernel scan + row sort
    *nnz_out = nnz;
}
