// k_graph.cu -- merged-index graph from the exact kNN lists (Sec. 4.3; the
// paper uses NSG as a black box, so these steps are this library's reading):
//   1. RNG prune (App. C rule): walk each node's K candidates in ascending
//      (key, id) order, keep v unless an already kept w has dist(w,v) <
//      dist(u,v); stop at R.
//   2. Reverse edges: C(v) = pruned(v) U {u : v in pruned(u)}, ascending; if
//      |C(v)| <= R keep it, else RNG-prune C(v) to R.
//   3. Entry point: the node nearest the FP64 centroid of all nodes, ties by id.
//   4. Data-edge lengths dist(u, v) for data->data edges (OOD rule, Sec. 4.4).
//   5. MST over {entry} U queries: query-query edges of the graph plus a star
//      edge (entry, q) per query (Sec. 3.2 WS), Boruvka with the total order
//      (FP64 weight, lower id, higher id); then BFS from the entry gives the
//      parent, depth and a topological processing order (Alg. 2).
// FP32 comparisons whose operands lie within their rounding bound of each
// other are re-decided in FP64, so decisions match an FP64 evaluation.
#include <float.h>

#include <vector>

#include "vj_device.cuh"
#include "vj_internal.cuh"

namespace {

constexpr int PWPB = 8;     // warps per block in the per-node kernels
constexpr int UCAP = 1024;  // shared-memory union capacity per warp

__device__ __forceinline__ bool near_equal(float a, float b, float tol, int metric) {
    return metric == 0 ? fabsf(a - b) <= tol * fmaxf(a, b) : fabsf(a - b) <= tol;
}

// RNG prune of a sorted candidate list (ids/keys in shared memory, n entries)
// for node u; kept ids/keys written to kid/kkey (shared), returns the count.
template <int G, int NPL>
__device__ int rng_prune_warp(const float* __restrict__ vec, const float* __restrict__ invn, int dp, int d,
                              int metric, float tol, int64_t u, const int* cid, const float* ckey, int n, int R,
                              int* kid, float* kkey, float* tmpk, int lane, unsigned long long* nrechk) {
    int nk = 0;
    for (int i = 0; i < n && nk < R; i++) {
        const int v = cid[i];
        const float kuv = ckey[i];
        bool keep = true;
        if (nk > 0) {
            float4 vv[NPL];
            load_slots<G, NPL>(vec, v, dp / 4, lane & (G - 1), vv);
            const float invv = metric ? __ldg(invn + v) : 0.f;
            group_keys<G, NPL, 1>(vec, invn, dp / 4, metric, vv, invv, kid, nk, tmpk, lane);
            __syncwarp();
            float kw = lane < nk ? tmpk[lane] : FLT_MAX;
            __syncwarp();
            bool rej = lane < nk && kw < kuv;
            bool nr = lane < nk && near_equal(kw, kuv, tol, metric);
            unsigned nm = __ballot_sync(VJ_FULL, nr);
            if (nm) {
                double duv = warp_dist64(vec, dp, d, metric, u, v, lane);
                while (nm) {
                    int src = __ffs(nm) - 1;
                    nm &= nm - 1;
                    int w = kid[src];
                    double dwv = warp_dist64(vec, dp, d, metric, w, v, lane);
                    if (lane == src) rej = dwv < duv;
                    if (lane == 0) atomicAdd(nrechk, 1ull);
                }
            }
            keep = !__any_sync(VJ_FULL, rej);
        }
        if (keep) {
            if (lane == 0) {
                kid[nk] = v;
                kkey[nk] = kuv;
            }
            nk++;
            __syncwarp();
        }
    }
    return nk;
}

// sort (key, id) ascending in shared memory (n <= cap, padded with (MAX, MAX))
__device__ void smem_sort_pairs(float* k, int* id, int n, int lane) {
    int P2 = 32;
    while (P2 < n) P2 <<= 1;
    for (int i = n + lane; i < P2; i += 32) {
        k[i] = FLT_MAX;
        id[i] = INT32_MAX;
    }
    __syncwarp();
    for (int kk = 2; kk <= P2; kk <<= 1) {
        for (int j = kk >> 1; j > 0; j >>= 1) {
            for (int i = lane; i < P2; i += 32) {
                int p = i ^ j;
                if (p > i) {
                    bool up = (i & kk) == 0;
                    bool gt = kless(k[p], id[p], k[i], id[i]);
                    if (gt == up) {
                        float tk = k[i];
                        int ti = id[i];
                        k[i] = k[p];
                        id[i] = id[p];
                        k[p] = tk;
                        id[p] = ti;
                    }
                }
            }
            __syncwarp();
        }
    }
}

// FP64 re-rank of near-tie runs of a sorted list of node u's neighbours
__device__ void fix_tie_runs(const float* __restrict__ vec, int dp, int d, int metric, float tol, int64_t u,
                             float* k, int* id, int n, double* s64, int lane, unsigned long long* nrechk) {
    int i0 = 0;
    while (i0 < n) {
        int i1 = i0;
        while (i1 + 1 < n && near_equal(k[i1], k[i1 + 1], tol, metric)) i1++;
        if (i1 > i0) {
            for (int e = i0; e <= i1; e++) {
                double dd = warp_dist64(vec, dp, d, metric, u, id[e], lane);
                if (lane == 0) s64[e - i0] = dd;
            }
            __syncwarp();
            if (lane == 0) {
                atomicAdd(nrechk, 1ull);
                for (int a = i0 + 1; a <= i1; a++) {
                    double da = s64[a - i0];
                    int ia = id[a];
                    float ka = k[a];
                    int b = a - 1;
                    while (b >= i0 && (s64[b - i0] > da || (s64[b - i0] == da && id[b] > ia))) {
                        s64[b - i0 + 1] = s64[b - i0];
                        id[b + 1] = id[b];
                        k[b + 1] = k[b];
                        b--;
                    }
                    s64[b - i0 + 1] = da;
                    id[b + 1] = ia;
                    k[b + 1] = ka;
                }
            }
            __syncwarp();
        }
        i0 = i1 + 1;
    }
}

struct PruneSmem {
    int cid[128];
    float ckey[128];
    int kid[32];
    float kkey[32];
    float tmpk[32];
};

// step 1
template <int G, int NPL>
__global__ void __launch_bounds__(PWPB * 32) k_prune(const float* __restrict__ vec, const float* __restrict__ invn,
                                                      int dp, int d, int64_t n, int metric, float tol, int K, int R,
                                                      const int32_t* __restrict__ knn, const float* __restrict__ knnd,
                                                      int32_t* __restrict__ pid, float* __restrict__ pkey,
                                                      int32_t* __restrict__ pcount,
                                                      unsigned long long* __restrict__ nrechk) {
    __shared__ PruneSmem sm[PWPB];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t u = (int64_t)blockIdx.x * PWPB + warp;
    if (u >= n) return;
    PruneSmem& S = sm[warp];
    int nc = 0;
    for (int e = lane; e < K; e += 32) {
        S.cid[e] = knn[u * K + e];
        S.ckey[e] = knnd[u * K + e];
    }
    __syncwarp();
    // candidates are sorted with -1 only at the tail
    for (int e = 0; e < K; e++)
        if (S.cid[e] >= 0) nc = e + 1;
    int nk = rng_prune_warp<G, NPL>(vec, invn, dp, d, metric, tol, u, S.cid, S.ckey, nc, R, S.kid, S.kkey, S.tmpk,
                                    lane, nrechk);
    if (lane < R) {
        pid[u * R + lane] = lane < nk ? S.kid[lane] : -1;
        pkey[u * R + lane] = lane < nk ? S.kkey[lane] : FLT_MAX;
    }
    if (lane == 0) pcount[u] = nk;
}

__global__ void k_indeg(const int32_t* __restrict__ pid, int64_t n, int R, int32_t* __restrict__ indeg) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * R) return;
    int v = pid[e];
    if (v >= 0) atomicAdd(indeg + v, 1);
}

__global__ void k_fill_in(const int32_t* __restrict__ pid, const float* __restrict__ pkey, int64_t n, int R,
                          const int64_t* __restrict__ inoff, int32_t* __restrict__ cursor, int32_t* __restrict__ inl,
                          float* __restrict__ inlk) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * R) return;
    int v = pid[e];
    if (v < 0) return;
    int pos = atomicAdd(cursor + v, 1);
    inl[inoff[v] + pos] = (int32_t)(e / R);
    inlk[inoff[v] + pos] = pkey[e];
}

// ---------------------------------------------------------------- tiled RNG prune (wide rows)
// Block per node: the RNG prune of a sorted candidate list, in rounds of up to
// 32 candidates.  A round stages the vectors of the nodes kept so far (<= 32)
// and of its candidates (<= 32) in shared memory, 64 dimensions at a time and
// dimension-major (a thread reads 4 consecutive rows per load), and every
// thread accumulates a 4 x 4 block of the 64 x 64 pair keys with FP32 direct
// differences (cosine: dot products, then 1 - dot/(|a||b|)).  Warp 0 then
// takes the round's decisions in list order with the rule and the FP64
// near-tie re-decision of rng_prune_warp.  Rows of d floats are read once per
// round instead of once per (candidate, kept node) pair.
constexpr int TP_THREADS = 256;
constexpr int TP_ROWS = 64;
constexpr int TP_CH = 64;  // dimensions per staged chunk

struct TpSmem {
    __align__(16) float T[TP_CH][TP_ROWS];
    float M[TP_ROWS][TP_ROWS + 1];
    int rid[TP_ROWS];  // node id of each tile row: kept nodes, then the round's candidates
    int kid[32];
    float kkey[32];
    int krow[32];
    int cid[32];
    float ckey[32];
    int nk;
};

// lists: row u's candidates are lid/lkey[base .. base + cnt), base = loff[u]
// (u * K when loff is null), cnt = lcnt[u] (when null: the entries of the K
// before the first -1).  rows: the nodes to prune (null: all nrows).
__global__ void __launch_bounds__(TP_THREADS) k_rng_tile(
    const float* __restrict__ vec, const float* __restrict__ invn, int dp, int d, int metric, float tol, int R,
    const int32_t* __restrict__ lid, const float* __restrict__ lkey, const int64_t* __restrict__ loff,
    const int32_t* __restrict__ lcnt, int K, const int32_t* __restrict__ rows, int64_t nrows,
    int32_t* __restrict__ out_id, float* __restrict__ out_key, int32_t* __restrict__ out_cnt,
    unsigned long long* __restrict__ nrechk) {
    __shared__ TpSmem S;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int64_t ri = blockIdx.x; ri < nrows; ri += gridDim.x) {
        const int64_t u = rows ? (int64_t)rows[ri] : ri;
        const int64_t base = loff ? loff[u] : u * K;
        int cnt;
        if (lcnt) {
            cnt = lcnt[u];
        } else {
            // the K-list is sorted with -1 only at the tail
            int c = 0;
            for (int e0 = 0; e0 < K; e0 += 32)
                c += __popc(__ballot_sync(VJ_FULL, e0 + lane < K && lid[base + e0 + lane] >= 0));
            cnt = c;
        }
        int nk = 0;
        for (int r0 = 0; r0 < cnt && nk < R; r0 += 32) {
            const int m = min(32, cnt - r0);
            const int nk0 = nk;
            if (tid < m) {
                const int v = lid[base + r0 + tid];
                S.cid[tid] = v;
                S.ckey[tid] = lkey[base + r0 + tid];
                S.rid[nk0 + tid] = v;
            }
            if (tid < nk0) {
                S.rid[tid] = S.kid[tid];
                S.krow[tid] = tid;
            }
            const int nt = nk0 + m;
            const int bi = tid >> 4, bj = tid & 15;  // this thread's rows bi*4.., columns bj*4..
            float acc[4][4];
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) acc[i][j] = 0.f;
            for (int k0 = 0; k0 < dp; k0 += TP_CH) {
                __syncthreads();  // tile rows known; the previous chunk consumed
                {
                    const int r = tid & (TP_ROWS - 1);
                    for (int f = tid / TP_ROWS; f < TP_CH / 4; f += TP_THREADS / TP_ROWS) {
                        float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (r < nt && k0 + f * 4 < dp)
                            x = __ldg(reinterpret_cast<const float4*>(vec + (int64_t)S.rid[r] * dp + k0 + f * 4));
                        S.T[f * 4 + 0][r] = x.x;
                        S.T[f * 4 + 1][r] = x.y;
                        S.T[f * 4 + 2][r] = x.z;
                        S.T[f * 4 + 3][r] = x.w;
                    }
                }
                __syncthreads();
                if (bi * 4 < nt && bj * 4 < nt) {
#pragma unroll 8
                    for (int k = 0; k < TP_CH; k++) {
                        const float4 a = *reinterpret_cast<const float4*>(&S.T[k][bi * 4]);
                        const float4 b = *reinterpret_cast<const float4*>(&S.T[k][bj * 4]);
                        const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
                        for (int i = 0; i < 4; i++)
#pragma unroll
                            for (int j = 0; j < 4; j++) {
                                if (metric == 0) {
                                    const float t = av[i] - bv[j];
                                    acc[i][j] = fmaf(t, t, acc[i][j]);
                                } else {
                                    acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
                                }
                            }
                    }
                }
            }
            if (bi * 4 < nt && bj * 4 < nt) {
#pragma unroll
                for (int i = 0; i < 4; i++)
#pragma unroll
                    for (int j = 0; j < 4; j++) {
                        const int ti = bi * 4 + i, tj = bj * 4 + j;
                        if (ti < nt && tj < nt)
                            S.M[ti][tj] = metric == 0 ? acc[i][j]
                                                      : 1.f - acc[i][j] * __ldg(invn + S.rid[ti]) *
                                                                  __ldg(invn + S.rid[tj]);
                    }
            }
            __syncthreads();
            if (warp == 0) {
                for (int i = 0; i < m && nk < R; i++) {
                    const int v = S.cid[i];
                    const float kuv = S.ckey[i];
                    const int trow = nk0 + i;
                    bool keep = true;
                    if (nk > 0) {
                        const float kw = lane < nk ? S.M[trow][S.krow[lane]] : FLT_MAX;
                        bool rej = lane < nk && kw < kuv;
                        const bool nr = lane < nk && near_equal(kw, kuv, tol, metric);
                        unsigned nm = __ballot_sync(VJ_FULL, nr);
                        if (nm) {
                            const double duv = warp_dist64(vec, dp, d, metric, u, v, lane);
                            while (nm) {
                                const int src = __ffs(nm) - 1;
                                nm &= nm - 1;
                                const int w = S.kid[src];
                                const double dwv = warp_dist64(vec, dp, d, metric, w, v, lane);
                                if (lane == src) rej = dwv < duv;
                                if (lane == 0) atomicAdd(nrechk, 1ull);
                            }
                        }
                        keep = !__any_sync(VJ_FULL, rej);
                    }
                    if (keep) {
                        if (lane == 0) {
                            S.kid[nk] = v;
                            S.kkey[nk] = kuv;
                            S.krow[nk] = trow;
                        }
                        nk++;
                        __syncwarp();
                    }
                }
                if (lane == 0) S.nk = nk;
            }
            __syncthreads();
            nk = S.nk;
        }
        if (tid < R) {
            out_id[u * R + tid] = tid < nk ? S.kid[tid] : -1;
            out_key[u * R + tid] = tid < nk ? S.kkey[tid] : FLT_MAX;
        }
        if (tid == 0 && out_cnt) out_cnt[u] = nk;
        __syncthreads();  // the next row overwrites the shared lists
    }
}

struct MergeSmem {
    int uid[UCAP];
    float uk[UCAP];
    double s64[UCAP];  // a tie run spans at most the whole union
    int kid[32];
    float kkey[32];
    float tmpk[32];
};

// step 2 (warp per node): union, sort, FP64 tie runs, keep or re-prune
template <int G, int NPL>
__global__ void __launch_bounds__(4 * 32) k_merge(const float* __restrict__ vec, const float* __restrict__ invn,
                                                   int dp, int d, int64_t n, int metric, float tol, int R,
                                                   const int32_t* __restrict__ pid, const float* __restrict__ pkey,
                                                   const int64_t* __restrict__ inoff, const int32_t* __restrict__ inl,
                                                   const float* __restrict__ inlk, int32_t* __restrict__ adj,
                                                   float* __restrict__ adjk, int32_t* __restrict__ big_rows,
                                                   int* __restrict__ nbig, unsigned long long* __restrict__ nrechk,
                                                   int32_t* __restrict__ stage_rows, int* __restrict__ nstage,
                                                   int32_t* __restrict__ uid_out, float* __restrict__ uk_out,
                                                   int32_t* __restrict__ ucnt) {
    extern __shared__ __align__(16) unsigned char mraw[];
    MergeSmem* sms = reinterpret_cast<MergeSmem*>(mraw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t v = (int64_t)blockIdx.x * 4 + warp;
    if (v >= n) return;
    MergeSmem& S = sms[warp];
    const int npr = 0;
    (void)npr;
    // own pruned list
    int myid = lane < R ? pid[v * R + lane] : -1;
    float myk = lane < R ? pkey[v * R + lane] : FLT_MAX;
    unsigned pm = __ballot_sync(VJ_FULL, myid >= 0);
    int nu = __popc(pm);
    if (myid >= 0) {
        int pos = __popc(pm & ((1u << lane) - 1u));
        S.uid[pos] = myid;
        S.uk[pos] = myk;
    }
    __syncwarp();
    const int64_t i0 = inoff[v], i1 = inoff[v + 1];
    if ((int64_t)R + (i1 - i0) > UCAP) {
        if (lane == 0) {
            int slot = atomicAdd(nbig, 1);
            big_rows[slot] = (int32_t)v;
        }
        return;
    }
    for (int64_t b = i0; b < i1; b += 32) {
        int64_t e = b + lane;
        int u = e < i1 ? inl[e] : -1;
        float k = e < i1 ? inlk[e] : FLT_MAX;
        // skip offers already in the own list
        bool dup = false;
        for (int j = 0; j < 32; j++) {
            int o = __shfl_sync(VJ_FULL, myid, j);
            if (u >= 0 && o == u) dup = true;
        }
        bool add = u >= 0 && !dup;
        unsigned am = __ballot_sync(VJ_FULL, add);
        if (add) {
            int pos = nu + __popc(am & ((1u << lane) - 1u));
            S.uid[pos] = u;
            S.uk[pos] = k;
        }
        nu += __popc(am);
        __syncwarp();
    }
    smem_sort_pairs(S.uk, S.uid, nu, lane);
    int nk;
    if (nu <= R) {
        // the whole union stays; its order must follow FP64 distances
        fix_tie_runs(vec, dp, d, metric, tol, v, S.uk, S.uid, nu, S.s64, lane, nrechk);
        nk = nu;
        if (lane < nk) {
            S.kid[lane] = S.uid[lane];
            S.kkey[lane] = S.uk[lane];
        }
        __syncwarp();
    } else {
        fix_tie_runs(vec, dp, d, metric, tol, v, S.uk, S.uid, nu, S.s64, lane, nrechk);
        if (stage_rows) {
            // wide rows: the sorted union goes to the tiled prune (its slot:
            // v * R + inoff[v] holds the R own entries plus the offers)
            const int64_t ub = v * R + i0;
            for (int e = lane; e < nu; e += 32) {
                uid_out[ub + e] = S.uid[e];
                uk_out[ub + e] = S.uk[e];
            }
            if (lane == 0) {
                ucnt[v] = nu;
                stage_rows[atomicAdd(nstage, 1)] = (int32_t)v;
            }
            return;
        }
        nk = rng_prune_warp<G, NPL>(vec, invn, dp, d, metric, tol, v, S.uid, S.uk, nu, R, S.kid, S.kkey, S.tmpk,
                                    lane, nrechk);
    }
    if (lane < R) {
        adj[v * R + lane] = lane < nk ? S.kid[lane] : -1;
        adjk[v * R + lane] = lane < nk ? S.kkey[lane] : FLT_MAX;
    }
}

// ---------------------------------------------------------------- entry point
constexpr int CB = 256;

// per-block FP64 partial sums of coordinates: part[blk][dim]
__global__ void k_centroid_part(const float* __restrict__ vec, int dp, int d, int64_t n, int64_t rows_per_blk,
                                double* __restrict__ part) {
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_blk;
    const int64_t r1 = min(n, r0 + rows_per_blk);
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
        double s = 0.0;
        for (int64_t r = r0; r < r1; r++) s += (double)vec[r * dp + j];
        part[(int64_t)blockIdx.x * d + j] = s;
    }
}

__global__ void k_centroid_final(const double* __restrict__ part, int nblk, int d, int64_t n,
                                 double* __restrict__ cen) {
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nblk; b++) s += part[(int64_t)b * d + j];
        cen[j] = s / (double)n;
    }
}

// warp per node: FP64 distance to the centroid; per-block argmin (d, id)
__global__ void __launch_bounds__(CB) k_entry_part(const float* __restrict__ vec, int dp, int d, int64_t n,
                                                   int metric, const double* __restrict__ cen,
                                                   double* __restrict__ bd, int32_t* __restrict__ bi) {
    __shared__ double sd[CB / 32];
    __shared__ int si[CB / 32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double best = 1e308;
    int bid = INT32_MAX;
    for (int64_t u = (int64_t)blockIdx.x * (CB / 32) + warp; u < n; u += (int64_t)gridDim.x * (CB / 32)) {
        double s0 = 0.0, s1 = 0.0, s2 = 0.0;
        for (int j = lane; j < d; j += 32) {
            double x = vec[u * dp + j], c = cen[j];
            if (metric == 0) {
                double t = x - c;
                s0 = fma(t, t, s0);
            } else {
                s0 = fma(x, c, s0);
                s1 = fma(x, x, s1);
                s2 = fma(c, c, s2);
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            s0 += __shfl_xor_sync(VJ_FULL, s0, o);
            s1 += __shfl_xor_sync(VJ_FULL, s1, o);
            s2 += __shfl_xor_sync(VJ_FULL, s2, o);
        }
        double dd = metric == 0 ? sqrt(s0) : ((s1 == 0.0 || s2 == 0.0) ? 1.0 : 1.0 - s0 / (sqrt(s1) * sqrt(s2)));
        if (dd < best || (dd == best && u < bid)) {
            best = dd;
            bid = (int)u;
        }
    }
    if (lane == 0) {
        sd[warp] = best;
        si[warp] = bid;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < CB / 32; w++)
            if (sd[w] < best || (sd[w] == best && si[w] < bid)) {
                best = sd[w];
                bid = si[w];
            }
        bd[blockIdx.x] = best;
        bi[blockIdx.x] = bid;
    }
}

__global__ void k_entry_final(const double* __restrict__ bd, const int32_t* __restrict__ bi, int nb,
                              int32_t* __restrict__ entry) {
    double best = 1e308;
    int bid = INT32_MAX;
    for (int b = 0; b < nb; b++)
        if (bd[b] < best || (bd[b] == best && bi[b] < bid)) {
            best = bd[b];
            bid = bi[b];
        }
    *entry = bid;
}

// ---------------------------------------------------------------- edge lengths
__global__ void k_elen(const int32_t* __restrict__ adj, const float* __restrict__ adjk, int64_t n, int64_t nx, int R,
                       int metric, float* __restrict__ elen) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * R) return;
    int64_t u = e / R;
    int v = adj[e];
    float l = __int_as_float(0x7fc00000);  // NaN: not a data->data edge
    if (u < nx && v >= 0 && v < nx) l = metric == 0 ? sqrtf(fmaxf(adjk[e], 0.f)) : adjk[e];
    elen[e] = l;
}

// ---------------------------------------------------------------- MST
// vertex ids: query index qi for query nodes; nq for the entry when it is a
// data node
__device__ __forceinline__ int vert_of(int64_t node, int64_t nx, int64_t nq) {
    return node >= nx ? (int)(node - nx) : (int)nq;
}

// emit edges: per query slot j < R a query-query edge (once per unordered
// pair), plus a star edge at slot R
__global__ void k_mst_edges(const int32_t* __restrict__ adj, int64_t nx, int64_t nq, int R, int32_t entry,
                            int32_t* __restrict__ ea, int32_t* __restrict__ eb) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int W = R + 1;
    if (e >= nq * W) return;
    int64_t qi = e / W;
    int j = (int)(e % W);
    int64_t u = nx + qi;
    int a = -1, b = -1;
    if (j < R) {
        int v = adj[u * R + j];
        if (v >= nx && v != u && v != entry && u != entry) {
            // keep (u,v) from u's list when u < v, or when v's list lacks u
            bool emit = u < v;
            if (!emit) {
                emit = true;
                for (int t = 0; t < R; t++)
                    if (adj[(int64_t)v * R + t] == (int)u) emit = false;
            }
            if (emit) {
                a = (int)(u < v ? u : (int64_t)v);
                b = (int)(u < v ? (int64_t)v : u);
            }
        }
    } else if (u != entry) {
        a = (int)(u < entry ? u : (int64_t)entry);
        b = (int)(u < entry ? (int64_t)entry : u);
    }
    ea[e] = a;
    eb[e] = b;
}

// warp per 32 edges: FP64 weight bits
__global__ void k_mst_weights(const float* __restrict__ vec, int dp, int d, int metric,
                              const int32_t* __restrict__ ea, const int32_t* __restrict__ eb, int64_t ne,
                              unsigned long long* __restrict__ wbits) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32;
    for (int i = 0; i < 32; i++) {
        int64_t e = w0 + i;
        if (e >= ne) break;
        int a = ea[e], b = eb[e];
        if (a < 0) {
            if (lane == 0) wbits[e] = ~0ull;
            continue;
        }
        double dd = warp_dist64(vec, dp, d, metric, a, b, lane);
        if (lane == 0) wbits[e] = (unsigned long long)__double_as_longlong(dd);
    }
}

__global__ void k_mst_init(int32_t* comp, int nv) {
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < nv) comp[v] = v;
}

// Boruvka round part 1: minimum weight per component
__global__ void k_mst_minw(const int32_t* __restrict__ ea, const int32_t* __restrict__ eb,
                           const unsigned long long* __restrict__ wbits, int64_t ne, int64_t nx, int64_t nq,
                           const int32_t* __restrict__ comp, unsigned long long* __restrict__ bw,
                           int* __restrict__ active) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne || ea[e] < 0) return;
    int ca = comp[vert_of(ea[e], nx, nq)], cb = comp[vert_of(eb[e], nx, nq)];
    if (ca == cb) return;
    atomicMin(bw + ca, wbits[e]);
    atomicMin(bw + cb, wbits[e]);
    *active = 1;
}

// part 2: among minimum-weight edges, minimum (lo, hi)
__global__ void k_mst_mint(const int32_t* __restrict__ ea, const int32_t* __restrict__ eb,
                           const unsigned long long* __restrict__ wbits, int64_t ne, int64_t nx, int64_t nq,
                           const int32_t* __restrict__ comp, const unsigned long long* __restrict__ bw,
                           unsigned long long* __restrict__ bt) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne || ea[e] < 0) return;
    int ca = comp[vert_of(ea[e], nx, nq)], cb = comp[vert_of(eb[e], nx, nq)];
    if (ca == cb) return;
    unsigned long long t = ((unsigned long long)(unsigned)ea[e] << 32) | (unsigned)eb[e];
    if (wbits[e] == bw[ca]) atomicMin(bt + ca, t);
    if (wbits[e] == bw[cb]) atomicMin(bt + cb, t);
}

// part 3: each component hooks to the other side of its chosen edge
__global__ void k_mst_hook(const int32_t* __restrict__ ea, const int32_t* __restrict__ eb,
                           const unsigned long long* __restrict__ wbits, int64_t ne, int64_t nx, int64_t nq,
                           const int32_t* __restrict__ comp, const unsigned long long* __restrict__ bw,
                           const unsigned long long* __restrict__ bt, int32_t* __restrict__ hook,
                           uint8_t* __restrict__ inmst) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne || ea[e] < 0) return;
    int ca = comp[vert_of(ea[e], nx, nq)], cb = comp[vert_of(eb[e], nx, nq)];
    if (ca == cb) return;
    unsigned long long t = ((unsigned long long)(unsigned)ea[e] << 32) | (unsigned)eb[e];
    if (wbits[e] == bw[ca] && t == bt[ca]) {
        hook[ca] = cb;
        inmst[e] = 1;
    }
    if (wbits[e] == bw[cb] && t == bt[cb]) {
        hook[cb] = ca;
        inmst[e] = 1;
    }
}

// break mutual hooks (both picked the same edge): the smaller id stays root
__global__ void k_mst_break(int32_t* hook, int nv) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nv) return;
    int h = hook[c];
    if (h != c && hook[h] == c && c < h) hook[c] = c;
}

__global__ void k_mst_jump(int32_t* hook, int nv, int* changed) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nv) return;
    int h = hook[c], hh = hook[h];
    if (h != hh) {
        hook[c] = hh;
        *changed = 1;
    }
}

__global__ void k_mst_relabel(int32_t* comp, const int32_t* hook, int nv) {
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < nv) comp[v] = hook[comp[v]];
}

// tree adjacency (both directions) from the chosen edges
__global__ void k_tree_deg(const int32_t* ea, const int32_t* eb, const uint8_t* inmst, int64_t ne, int64_t nx,
                           int64_t nq, int32_t* deg) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne || !inmst[e]) return;
    atomicAdd(deg + vert_of(ea[e], nx, nq), 1);
    atomicAdd(deg + vert_of(eb[e], nx, nq), 1);
}

__global__ void k_tree_fill(const int32_t* ea, const int32_t* eb, const uint8_t* inmst, int64_t ne, int64_t nx,
                            int64_t nq, const int64_t* off, int32_t* cur, int32_t* nbr) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne || !inmst[e]) return;
    int a = vert_of(ea[e], nx, nq), b = vert_of(eb[e], nx, nq);
    nbr[off[a] + atomicAdd(cur + a, 1)] = b;
    nbr[off[b] + atomicAdd(cur + b, 1)] = a;
}

// one BFS level over the tree
__global__ void k_tree_level(const int32_t* __restrict__ front, int nf, const int64_t* __restrict__ off,
                             const int32_t* __restrict__ nbr, int32_t* __restrict__ vdepth,
                             int32_t* __restrict__ vparent, int32_t* __restrict__ next, int* __restrict__ nnext,
                             int level) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf) return;
    int a = front[i];
    for (int64_t j = off[a]; j < off[a + 1]; j++) {
        int b = nbr[j];
        if (vdepth[b] < 0) {
            vdepth[b] = level + 1;
            vparent[b] = a;
            next[atomicAdd(nnext, 1)] = b;
        }
    }
}

__global__ void k_union_off(const int64_t* __restrict__ inoff, int64_t n, int R, int64_t* __restrict__ uoff) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) uoff[v] = v * R + inoff[v];
}

}  // namespace


void vj_build_graph(vj_index* ix) {
    cudaStream_t s = ix->stream;
    const int64_t n = ix->n, nx = ix->nx, nq = ix->nq;
    const int R = ix->R, K = ix->K, dp = ix->dp, d = ix->d, metric = ix->metric;
    const int dp4 = dp / 4;
    const float tol = 2.0f * (float)(dp + 4) * VJ_F32_U * (metric == VJ_L2 ? 1.0f : 4.0f) + 1e-7f;
    DBuf<unsigned long long> nr;
    nr.alloc(1, s);
    VJ_CUDA(cudaMemsetAsync(nr.p, 0, sizeof(unsigned long long), s));

    // nodes with a graph row: every node, or the data nodes only (G_X of an
    // NN-Map index, whose kNN lists hold data nodes only).  Separate indexes
    // keep both sets' rows: their lists never cross sets, so neither do the
    // pruned and reverse edges
    const int64_t gr = ix->graph_rows;

    // ---- 1. prune
    DBuf<int32_t> pid, pcount;
    DBuf<float> pkey;
    pid.alloc((size_t)gr * R, s);
    pkey.alloc((size_t)gr * R, s);
    pcount.alloc(gr, s);
    // rows wider than 256 floats: the tiled prune (a warp per node would
    // gather every kept vector once per candidate)
    const bool tiled = dp4 > 64;
    const int tp_grid = (int)std::min<int64_t>(gr, (int64_t)ix->num_sms * 32);
    if (tiled) {
        k_rng_tile<<<tp_grid, TP_THREADS, 0, s>>>(ix->vec.p, ix->invn.p, dp, d, metric, tol, R, ix->knn.p,
                                                  ix->knnd.p, nullptr, nullptr, K, nullptr, gr, pid.p, pkey.p,
                                                  pcount.p, nr.p);
    } else {
        VJ_DISPATCH_GN(dp4, (k_prune<G, NPL><<<vj_div_up(gr, PWPB), PWPB * 32, 0, s>>>(
                                ix->vec.p, ix->invn.p, dp, d, gr, metric, tol, K, R, ix->knn.p, ix->knnd.p, pid.p,
                                pkey.p, pcount.p, nr.p)));
    }
    VJ_LAUNCH_CHECK();

    // ---- 2. reverse edges
    DBuf<int32_t> indeg, cursor, inl;
    DBuf<int64_t> inoff;
    DBuf<float> inlk;
    indeg.alloc(gr, s);
    cursor.alloc(gr, s);
    inoff.alloc(gr + 1, s);
    VJ_CUDA(cudaMemsetAsync(indeg.p, 0, gr * sizeof(int32_t), s));
    VJ_CUDA(cudaMemsetAsync(cursor.p, 0, gr * sizeof(int32_t), s));
    k_indeg<<<vj_div_up(gr * R, 256), 256, 0, s>>>(pid.p, gr, R, indeg.p);
    VJ_LAUNCH_CHECK();
    vj_exclusive_scan_i32_to_i64(indeg.p, inoff.p, gr, ix);
    int64_t nin = 0;
    VJ_CUDA(cudaMemcpyAsync(&nin, inoff.p + gr, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    VJ_CUDA(cudaStreamSynchronize(s));
    inl.alloc(std::max<int64_t>(nin, 1), s);
    inlk.alloc(std::max<int64_t>(nin, 1), s);
    k_fill_in<<<vj_div_up(gr * R, 256), 256, 0, s>>>(pid.p, pkey.p, gr, R, inoff.p, cursor.p, inl.p, inlk.p);
    VJ_LAUNCH_CHECK();
    ix->adj.ensure((size_t)n * R, s);
    DBuf<float> adjk;
    adjk.alloc((size_t)n * R, s);
    if (gr < n) {
        // rows without a graph row (the queries of an NN-Map index): no edges
        VJ_CUDA(cudaMemsetAsync(ix->adj.p + gr * R, 0xff, (size_t)(n - gr) * R * sizeof(int32_t), s));
        VJ_CUDA(cudaMemsetAsync(adjk.p + gr * R, 0, (size_t)(n - gr) * R * sizeof(float), s));
    }
    DBuf<int32_t> big, stage, uid, ucnt;
    DBuf<float> uk;
    DBuf<int> nbig;
    big.alloc(gr, s);
    nbig.alloc(2, s);
    VJ_CUDA(cudaMemsetAsync(nbig.p, 0, 2 * sizeof(int), s));
    if (tiled) {
        stage.alloc(gr, s);
        ucnt.alloc(gr, s);
        uid.alloc((size_t)gr * R + std::max<int64_t>(nin, 1), s);
        uk.alloc((size_t)gr * R + std::max<int64_t>(nin, 1), s);
    }
    {
        size_t smem = sizeof(MergeSmem) * 4;
        VJ_DISPATCH_GN(dp4, {
            VJ_CUDA(cudaFuncSetAttribute(k_merge<G, NPL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            k_merge<G, NPL><<<vj_div_up(gr, 4), 4 * 32, smem, s>>>(
                ix->vec.p, ix->invn.p, dp, d, gr, metric, tol, R, pid.p, pkey.p, inoff.p, inl.p, inlk.p, ix->adj.p,
                adjk.p, big.p, nbig.p, nr.p, tiled ? stage.p : nullptr, nbig.p + 1, uid.p, uk.p, ucnt.p);
        });
        VJ_LAUNCH_CHECK();
    }
    int hbig[2] = {0, 0};
    VJ_CUDA(cudaMemcpyAsync(hbig, nbig.p, sizeof(hbig), cudaMemcpyDeviceToHost, s));
    VJ_CUDA(cudaStreamSynchronize(s));
    VJ_REQUIRE(hbig[0] == 0, VJ_ERR_STATE, "graph build: %d nodes have more than %d reverse-edge offers", hbig[0],
               UCAP - R);
    if (tiled && hbig[1] > 0) {
        // over-full unions of wide rows: their RNG prune, into adj / adjk
        DBuf<int64_t> uoff;
        uoff.alloc(gr, s);
        k_union_off<<<vj_div_up(gr, 256), 256, 0, s>>>(inoff.p, gr, R, uoff.p);
        VJ_LAUNCH_CHECK();
        k_rng_tile<<<(int)std::min<int64_t>(hbig[1], (int64_t)ix->num_sms * 32), TP_THREADS, 0, s>>>(
            ix->vec.p, ix->invn.p, dp, d, metric, tol, R, uid.p, uk.p, uoff.p, ucnt.p, 0, stage.p, hbig[1],
            ix->adj.p, adjk.p, nullptr, nr.p);
        VJ_LAUNCH_CHECK();
        uoff.free_(s);
    }
    stage.free_(s);
    ucnt.free_(s);
    uid.free_(s);
    uk.free_(s);

    // ---- 3. entry point: the node nearest the centroid of nodes 0 .. entry_rows-1
    // (every node of a merged index; the data set of NN-Map and separate indexes)
    {
        const int64_t er = ix->entry_rows;
        const int nblk = (int)std::min<int64_t>(1024, std::max<int64_t>(1, er / 256));
        const int64_t rpb = (er + nblk - 1) / nblk;
        DBuf<double> part, cen, bd;
        DBuf<int32_t> bi, ent;
        part.alloc((size_t)nblk * d, s);
        cen.alloc(d, s);
        k_centroid_part<<<nblk, 128, 0, s>>>(ix->vec.p, dp, d, er, rpb, part.p);
        VJ_LAUNCH_CHECK();
        k_centroid_final<<<1, 256, 0, s>>>(part.p, nblk, d, er, cen.p);
        VJ_LAUNCH_CHECK();
        const int eb = 512;
        bd.alloc(eb, s);
        bi.alloc(eb, s);
        ent.alloc(1, s);
        k_entry_part<<<eb, CB, 0, s>>>(ix->vec.p, dp, d, er, metric, cen.p, bd.p, bi.p);
        VJ_LAUNCH_CHECK();
        k_entry_final<<<1, 1, 0, s>>>(bd.p, bi.p, eb, ent.p);
        VJ_LAUNCH_CHECK();
        VJ_CUDA(cudaMemcpyAsync(&ix->entry, ent.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        VJ_CUDA(cudaStreamSynchronize(s));
        part.free_(s);
        cen.free_(s);
        bd.free_(s);
        bi.free_(s);
        ent.free_(s);
    }

    // ---- 4. edge lengths
    ix->elen.ensure((size_t)n * R, s);
    k_elen<<<vj_div_up(n * R, 256), 256, 0, s>>>(ix->adj.p, adjk.p, n, nx, R, metric, ix->elen.p);
    VJ_LAUNCH_CHECK();

    // ---- 5. MST + BFS order (an NN-Map index has no query graph: every
    // query hangs off the data side, in id order)
    if (ix->nnmap) {
        std::vector<int32_t> ho(nq), hp(nq, -1), hd(nq, 1);
        for (int64_t qi = 0; qi < nq; qi++) ho[qi] = (int32_t)qi;
        ix->order.ensure(nq, s);
        ix->parent.ensure(nq, s);
        ix->depth.ensure(nq, s);
        VJ_CUDA(cudaMemcpyAsync(ix->order.p, ho.data(), nq * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        VJ_CUDA(cudaMemcpyAsync(ix->parent.p, hp.data(), nq * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        VJ_CUDA(cudaMemcpyAsync(ix->depth.p, hd.data(), nq * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        VJ_CUDA(cudaStreamSynchronize(s));
        ix->max_depth = 1;
    } else {
        const int64_t ne = nq * (R + 1);
        const int nv = (int)nq + 1;  // queries + (possibly unused) data-entry vertex
        const bool entry_is_query = ix->entry >= nx;
        DBuf<int32_t> ea, eb, comp, hook;
        DBuf<unsigned long long> wb, bw, bt;
        DBuf<uint8_t> inmst;
        DBuf<int> flag;
        ea.alloc(ne, s);
        eb.alloc(ne, s);
        wb.alloc(ne, s);
        inmst.alloc(ne, s);
        comp.alloc(nv, s);
        hook.alloc(nv, s);
        bw.alloc(nv, s);
        bt.alloc(nv, s);
        flag.alloc(2, s);
        VJ_CUDA(cudaMemsetAsync(inmst.p, 0, ne, s));
        k_mst_edges<<<vj_div_up(ne, 256), 256, 0, s>>>(ix->adj.p, nx, nq, R, ix->entry, ea.p, eb.p);
        VJ_LAUNCH_CHECK();
        k_mst_weights<<<vj_div_up(vj_div_up(ne, 32) * 32, 256), 256, 0, s>>>(ix->vec.p, dp, d, metric, ea.p, eb.p,
                                                                              ne, wb.p);
        VJ_LAUNCH_CHECK();
        k_mst_init<<<vj_div_up(nv, 256), 256, 0, s>>>(comp.p, nv);
        VJ_LAUNCH_CHECK();
        for (int round = 0; round < 64; round++) {
            VJ_CUDA(cudaMemsetAsync(bw.p, 0xff, nv * sizeof(unsigned long long), s));
            VJ_CUDA(cudaMemsetAsync(bt.p, 0xff, nv * sizeof(unsigned long long), s));
            VJ_CUDA(cudaMemsetAsync(flag.p, 0, 2 * sizeof(int), s));
            k_mst_minw<<<vj_div_up(ne, 256), 256, 0, s>>>(ea.p, eb.p, wb.p, ne, nx, nq, comp.p, bw.p, flag.p);
            VJ_LAUNCH_CHECK();
            int act = 0;
            VJ_CUDA(cudaMemcpyAsync(&act, flag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
            VJ_CUDA(cudaStreamSynchronize(s));
            if (!act) break;
            k_mst_mint<<<vj_div_up(ne, 256), 256, 0, s>>>(ea.p, eb.p, wb.p, ne, nx, nq, comp.p, bw.p, bt.p);
            VJ_LAUNCH_CHECK();
            k_mst_init<<<vj_div_up(nv, 256), 256, 0, s>>>(hook.p, nv);
            VJ_LAUNCH_CHECK();
            k_mst_hook<<<vj_div_up(ne, 256), 256, 0, s>>>(ea.p, eb.p, wb.p, ne, nx, nq, comp.p, bw.p, bt.p, hook.p,
                                                          inmst.p);
            VJ_LAUNCH_CHECK();
            k_mst_break<<<vj_div_up(nv, 256), 256, 0, s>>>(hook.p, nv);
            VJ_LAUNCH_CHECK();
            for (int it = 0; it < 64; it++) {
                VJ_CUDA(cudaMemsetAsync(flag.p + 1, 0, sizeof(int), s));
                k_mst_jump<<<vj_div_up(nv, 256), 256, 0, s>>>(hook.p, nv, flag.p + 1);
                VJ_LAUNCH_CHECK();
                int ch = 0;
                VJ_CUDA(cudaMemcpyAsync(&ch, flag.p + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
                VJ_CUDA(cudaStreamSynchronize(s));
                if (!ch) break;
            }
            k_mst_relabel<<<vj_div_up(nv, 256), 256, 0, s>>>(comp.p, hook.p, nv);
            VJ_LAUNCH_CHECK();
        }
        // tree CSR
        DBuf<int32_t> deg, cur, nbr, vdepth, vparent, fa, fb;
        DBuf<int64_t> off;
        deg.alloc(nv, s);
        cur.alloc(nv, s);
        off.alloc(nv + 1, s);
        VJ_CUDA(cudaMemsetAsync(deg.p, 0, nv * sizeof(int32_t), s));
        VJ_CUDA(cudaMemsetAsync(cur.p, 0, nv * sizeof(int32_t), s));
        k_tree_deg<<<vj_div_up(ne, 256), 256, 0, s>>>(ea.p, eb.p, inmst.p, ne, nx, nq, deg.p);
        VJ_LAUNCH_CHECK();
        vj_exclusive_scan_i32_to_i64(deg.p, off.p, nv, ix);
        nbr.alloc(2 * (size_t)nv, s);
        k_tree_fill<<<vj_div_up(ne, 256), 256, 0, s>>>(ea.p, eb.p, inmst.p, ne, nx, nq, off.p, cur.p, nbr.p);
        VJ_LAUNCH_CHECK();
        vdepth.alloc(nv, s);
        vparent.alloc(nv, s);
        fa.alloc(nv, s);
        fb.alloc(nv, s);
        VJ_CUDA(cudaMemsetAsync(vdepth.p, 0xff, nv * sizeof(int32_t), s));
        VJ_CUDA(cudaMemsetAsync(vparent.p, 0xff, nv * sizeof(int32_t), s));
        const int root = entry_is_query ? (int)(ix->entry - nx) : (int)nq;
        int zero = 0;
        VJ_CUDA(cudaMemcpyAsync(vdepth.p + root, &zero, sizeof(int), cudaMemcpyHostToDevice, s));
        VJ_CUDA(cudaMemcpyAsync(fa.p, &root, sizeof(int), cudaMemcpyHostToDevice, s));
        // order = BFS levels (queries only)
        ix->order.ensure(nq, s);
        ix->parent.ensure(nq, s);
        ix->depth.ensure(nq, s);
        int64_t placed = 0;
        if (entry_is_query) {
            VJ_CUDA(cudaMemcpyAsync(ix->order.p, &root, sizeof(int), cudaMemcpyHostToDevice, s));
            placed = 1;
        }
        int nf = 1, level = 0;
        while (nf > 0) {
            VJ_CUDA(cudaMemsetAsync(flag.p, 0, sizeof(int), s));
            k_tree_level<<<vj_div_up(nf, 256), 256, 0, s>>>(fa.p, nf, off.p, nbr.p, vdepth.p, vparent.p, fb.p,
                                                           flag.p, level);
            VJ_LAUNCH_CHECK();
            int nn = 0;
            VJ_CUDA(cudaMemcpyAsync(&nn, flag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
            VJ_CUDA(cudaStreamSynchronize(s));
            if (nn > 0) {
                VJ_REQUIRE(placed + nn <= nq, VJ_ERR_STATE, "MST BFS placed too many vertices");
                VJ_CUDA(cudaMemcpyAsync(ix->order.p + placed, fb.p, nn * sizeof(int32_t), cudaMemcpyDeviceToDevice,
                                        s));
                placed += nn;
            }
            std::swap(fa, fb);
            nf = nn;
            level++;
        }
        VJ_REQUIRE(placed == nq, VJ_ERR_STATE, "MST does not span the queries (%lld of %lld)", (long long)placed,
                   (long long)nq);
        ix->max_depth = level - 1;
        // parent (query index, -1 for the data entry) and depth per query
        std::vector<int32_t> hp(nv), hd(nv);
        VJ_CUDA(cudaMemcpyAsync(hp.data(), vparent.p, nv * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        VJ_CUDA(cudaMemcpyAsync(hd.data(), vdepth.p, nv * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        VJ_CUDA(cudaStreamSynchronize(s));
        for (int64_t qi = 0; qi < nq; qi++) {
            int p = hp[qi];
            hp[qi] = (p < 0 || p == (int)nq) ? -1 : p;
        }
        VJ_CUDA(cudaMemcpyAsync(ix->parent.p, hp.data(), nq * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        VJ_CUDA(cudaMemcpyAsync(ix->depth.p, hd.data(), nq * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        VJ_CUDA(cudaStreamSynchronize(s));
        for (auto* b : {&ea, &eb, &comp, &hook, &deg, &cur, &nbr, &vdepth, &vparent, &fa, &fb}) b->free_(s);
        wb.free_(s);
        bw.free_(s);
        bt.free_(s);
        inmst.free_(s);
        flag.free_(s);
        off.free_(s);
    }
    adjk.free_(s);
    pid.free_(s);
    pkey.free_(s);
    pcount.free_(s);
    indeg.free_(s);
    cursor.free_(s);
    inl.free_(s);
    inlk.free_(s);
    inoff.free_(s);
    big.free_(s);
    nbig.free_(s);
    nr.free_(s);
}
