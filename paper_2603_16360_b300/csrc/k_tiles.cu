// k_tiles.cu -- dense distance tiles: the exact kNN graph of the merged node
// set (build input of Sec. 4.3) and the exact nested-loop join (Sec. 3.2).
//
// Both evaluate keys through the norm expansion |a|^2 + |b|^2 - 2<a,b> (L2,
// squared) or 1 - <a,b>/(|a||b|) (cosine) over 128 x 128 tiles of a
// register-blocked FP32 Gram product, then
//  - kNN (FP32 build tiles; the BF16 default runs on the tensor cores in
//    k_tc.cu and is re-ranked here by k_knn_rerank_csr): each block owns 128
//    rows and sweeps every column tile, keeping per
//    row the KP smallest keys (KP = K + margin); a second pass re-ranks the KP
//    candidates with direct-difference FP32 keys (FP64 among near-ties) and
//    certifies that no excluded node can enter the top K given the Gram
//    rounding bound; uncertified rows are redone by a brute-force row scan.
//  - NLJ: pairs whose Gram key is below eps_key + bound become candidates;
//    candidates are re-decided with direct-difference FP32 keys and, within
//    the FP32 bound of eps, in FP64.
#include <float.h>

#include "vj_device.cuh"
#include "vj_internal.cuh"

namespace {

constexpr int TBM = 128, TBN = 128, TBK = 8, TT = 256;

struct GramSmem {
    float As[2][TBK][TBM + 4];
    float Bs[2][TBK][TBN + 4];
};

// acc[i][j] = <row(ra + rr(i)), row(ca + cc(j))> with rr(i) = ty*4 + (i&3) +
// 64*(i>>2), cc(j) = tx*4 + (j&3) + 64*(j>>2); rows beyond the limits read 0
__device__ __forceinline__ void gram_tile(const float* __restrict__ vec, int dp, int64_t ra, int64_t ra_end,
                                          int64_t ca, int64_t ca_end, float (&acc)[8][8], GramSmem& sm) {
    const int t = threadIdx.x;
    const int lr = t >> 1, lk = (t & 1) * 4;
    const int ty = t >> 4, tx = t & 15;
#pragma unroll
    for (int i = 0; i < 8; i++)
#pragma unroll
        for (int j = 0; j < 8; j++) acc[i][j] = 0.f;
    const int64_t rA = ra + lr, rB = ca + lr;
    const float4* pA = reinterpret_cast<const float4*>(vec + rA * dp);
    const float4* pB = reinterpret_cast<const float4*>(vec + rB * dp);
    const bool okA = rA < ra_end, okB = rB < ca_end;
    float4 a4 = (okA && lk < dp) ? __ldg(pA + (lk >> 2)) : f4zero();
    float4 b4 = (okB && lk < dp) ? __ldg(pB + (lk >> 2)) : f4zero();
    sm.As[0][lk + 0][lr] = a4.x;
    sm.As[0][lk + 1][lr] = a4.y;
    sm.As[0][lk + 2][lr] = a4.z;
    sm.As[0][lk + 3][lr] = a4.w;
    sm.Bs[0][lk + 0][lr] = b4.x;
    sm.Bs[0][lk + 1][lr] = b4.y;
    sm.Bs[0][lk + 2][lr] = b4.z;
    sm.Bs[0][lk + 3][lr] = b4.w;
    __syncthreads();
    int cur = 0;
    for (int k0 = 0; k0 < dp; k0 += TBK) {
        const int kn = k0 + TBK + lk;
        const bool more = k0 + TBK < dp;
        if (more) {
            a4 = (okA && kn < dp) ? __ldg(pA + (kn >> 2)) : f4zero();
            b4 = (okB && kn < dp) ? __ldg(pB + (kn >> 2)) : f4zero();
        }
#pragma unroll
        for (int kk = 0; kk < TBK; kk++) {
            float4 x0 = *reinterpret_cast<const float4*>(&sm.As[cur][kk][ty * 4]);
            float4 x1 = *reinterpret_cast<const float4*>(&sm.As[cur][kk][64 + ty * 4]);
            float4 y0 = *reinterpret_cast<const float4*>(&sm.Bs[cur][kk][tx * 4]);
            float4 y1 = *reinterpret_cast<const float4*>(&sm.Bs[cur][kk][64 + tx * 4]);
            float a[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
            float b[8] = {y0.x, y0.y, y0.z, y0.w, y1.x, y1.y, y1.z, y1.w};
#pragma unroll
            for (int i = 0; i < 8; i++)
#pragma unroll
                for (int j = 0; j < 8; j++) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        if (more) {
            const int nx_ = cur ^ 1;
            sm.As[nx_][lk + 0][lr] = a4.x;
            sm.As[nx_][lk + 1][lr] = a4.y;
            sm.As[nx_][lk + 2][lr] = a4.z;
            sm.As[nx_][lk + 3][lr] = a4.w;
            sm.Bs[nx_][lk + 0][lr] = b4.x;
            sm.Bs[nx_][lk + 1][lr] = b4.y;
            sm.Bs[nx_][lk + 2][lr] = b4.z;
            sm.Bs[nx_][lk + 3][lr] = b4.w;
        }
        __syncthreads();
        cur ^= 1;
    }
}

__device__ __forceinline__ int tile_row(int i) { return (threadIdx.x >> 4) * 4 + (i & 3) + 64 * (i >> 2); }
__device__ __forceinline__ int tile_col(int j) { return (threadIdx.x & 15) * 4 + (j & 3) + 64 * (j >> 2); }

// ---------------------------------------------------------------- norms
__global__ void k_norms(const float* __restrict__ vec, int dp, int d, int64_t n, float* __restrict__ sqn,
                        float* __restrict__ invn, double* __restrict__ sqn64, double* __restrict__ maxn) {
    const int lane = threadIdx.x & 31;
    int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (u >= n) return;
    double s = 0.0;
    for (int i = lane; i < d; i += 32) {
        double x = vec[u * dp + i];
        s = fma(x, x, s);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(VJ_FULL, s, o);
    if (lane == 0) {
        sqn64[u] = s;
        sqn[u] = (float)s;
        invn[u] = s > 0.0 ? (float)(1.0 / sqrt(s)) : 0.f;
        // max norm (non-negative doubles order like their bit patterns)
        atomicMax(reinterpret_cast<unsigned long long*>(maxn), (unsigned long long)__double_as_longlong(sqrt(s)));
    }
}

// ---------------------------------------------------------------- kNN sweep
// smem: gram buffers, key tile [128][129], per-row candidate lists [128][KP]
template <int KP>
struct KnnSmem {
    union {
        GramSmem g;
        float D[TBM][TBN + 1];
    } u;
    float lk[TBM][KP];
    int li[TBM][KP];
};

// insert (k, id) into the ascending list L (length KP, lanes own slots
// lane, lane+32, ...); the last entry falls off
template <int KP>
__device__ __forceinline__ void list_insert(float* Lk, int* Li, float k, int id, int lane) {
    constexpr int PER = (KP + 31) / 32;
    int less = 0;
    float ok[PER];
    int oi[PER];
#pragma unroll
    for (int e = 0; e < PER; e++) {
        int pos = lane + 32 * e;
        if (pos < KP) {
            ok[e] = Lk[pos];
            oi[e] = Li[pos];
            less += kless(ok[e], oi[e], k, id) ? 1 : 0;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) less += __shfl_xor_sync(VJ_FULL, less, o);
    if (less >= KP) return;
    // new value of slot pos: pos < less: unchanged; pos == less: (k,id); pos > less: old[pos-1]
    float nk[PER];
    int ni[PER];
#pragma unroll
    for (int e = 0; e < PER; e++) {
        int pos = lane + 32 * e;
        int sp = pos - 1;  // source slot
        // old[pos-1] lives in lane (pos-1)%32, element (pos-1)/32
        int srcl = (sp + 32) & 31;
        int srce = sp >> 5;  // -1 when pos == 0 (unused)
        float ck = 0.f;
        int ci = 0;
#pragma unroll
        for (int e2 = 0; e2 < PER; e2++) {
            float tk = __shfl_sync(VJ_FULL, ok[e2], srcl);
            int ti = __shfl_sync(VJ_FULL, oi[e2], srcl);
            if (e2 == srce) {
                ck = tk;
                ci = ti;
            }
        }
        nk[e] = pos < less ? ok[e] : (pos == less ? k : ck);
        ni[e] = pos < less ? oi[e] : (pos == less ? id : ci);
    }
#pragma unroll
    for (int e = 0; e < PER; e++) {
        int pos = lane + 32 * e;
        if (pos < KP && pos >= less) {
            Lk[pos] = nk[e];
            Li[pos] = ni[e];
        }
    }
    __syncwarp();
}

template <int KP>
__global__ void __launch_bounds__(TT) k_knn_sweep(const float* __restrict__ vec, const float* __restrict__ sqn,
                                                   const float* __restrict__ invn, int dp, int64_t r0, int64_t r1,
                                                   int64_t c0, int64_t c1, int metric, int32_t* __restrict__ cand_id,
                                                   float* __restrict__ cand_key, float* __restrict__ row_thr) {
    extern __shared__ __align__(16) unsigned char sraw[];
    KnnSmem<KP>& S = *reinterpret_cast<KnnSmem<KP>*>(sraw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // rows r0 .. r1-1 against the candidate nodes c0 .. c1-1
    const int64_t ra = r0 + (int64_t)blockIdx.x * TBM;
    const int64_t n = r1;
    for (int i = threadIdx.x; i < TBM * KP; i += TT) {
        (&S.lk[0][0])[i] = FLT_MAX;
        (&S.li[0][0])[i] = INT32_MAX;
    }
    __syncthreads();
    float rn[8];
#pragma unroll
    for (int i = 0; i < 8; i++) {
        int64_t r = ra + tile_row(i);
        rn[i] = r < n ? (metric == 0 ? sqn[r] : invn[r]) : 0.f;
    }
    for (int64_t ca = c0; ca < c1; ca += TBN) {
        float acc[8][8];
        gram_tile(vec, dp, ra, n, ca, c1, acc, S.u.g);
        // keys into the tile (the gram buffers are dead after the last sync)
#pragma unroll
        for (int j = 0; j < 8; j++) {
            int64_t c = ca + tile_col(j);
            float cn = c < c1 ? (metric == 0 ? sqn[c] : invn[c]) : 0.f;
#pragma unroll
            for (int i = 0; i < 8; i++) {
                int64_t r = ra + tile_row(i);
                float key;
                if (c >= c1 || r >= n || c == r) key = FLT_MAX;
                else if (metric == 0) key = fmaxf(rn[i] + cn - 2.f * acc[i][j], 0.f);
                else key = 1.f - acc[i][j] * rn[i] * cn;
                S.u.D[tile_row(i)][tile_col(j)] = key;
            }
        }
        __syncthreads();
        // each warp updates 16 rows
        for (int rr = warp * 16; rr < warp * 16 + 16; rr++) {
            const float thr = S.lk[rr][KP - 1];
            const int thi = S.li[rr][KP - 1];
#pragma unroll
            for (int e = 0; e < TBN / 32; e++) {
                int cc = lane + 32 * e;
                float k = S.u.D[rr][cc];
                int id = (int)(ca + cc);
                unsigned m = __ballot_sync(VJ_FULL, k != FLT_MAX && kless(k, id, thr, thi));
                while (m) {
                    int src = __ffs(m) - 1;
                    m &= m - 1;
                    float kk = __shfl_sync(VJ_FULL, k, src);
                    int ii = __shfl_sync(VJ_FULL, id, src);
                    list_insert<KP>(S.lk[rr], S.li[rr], kk, ii, lane);
                }
            }
        }
        __syncthreads();
    }
    // write candidate lists
    for (int rr = warp * 16; rr < warp * 16 + 16; rr++) {
        int64_t r = ra + rr;
        if (r >= n) continue;
        for (int e = lane; e < KP; e += 32) {
            cand_id[r * KP + e] = S.li[rr][e] == INT32_MAX ? -1 : S.li[rr][e];
            cand_key[r * KP + e] = S.lk[rr][e];
        }
        if (lane == 0) row_thr[r] = S.lk[rr][KP - 1];
    }
}

// ---------------------------------------------------------------- re-rank
// warp per row: exact keys of the KP candidates, sort, FP64 near-tie runs,
// certificate; outputs the top K (ids, keys)
template <int G, int NPL>
__global__ void __launch_bounds__(256) k_knn_rerank(const float* __restrict__ vec, const float* __restrict__ invn,
                                                     const float* __restrict__ sqn, int dp, int d, int64_t n,
                                                     int metric, int KP, int K, const int32_t* __restrict__ cand_id,
                                                     const float* __restrict__ row_thr, int thr_true, double maxnorm,
                                                     const int32_t* __restrict__ rows, int64_t nrows,
                                                     int32_t* __restrict__ out_id, float* __restrict__ out_key,
                                                     int32_t* __restrict__ bad_rows, int* __restrict__ nbad,
                                                     unsigned long long* __restrict__ nrechk) {
    __shared__ int sid[8][128];
    __shared__ float skey[8][128];
    __shared__ double s64[8][128];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t w = (int64_t)blockIdx.x * 8 + warp;
    if (w >= nrows) return;
    const int64_t r = rows ? (int64_t)rows[w] : w;
    int* ids = sid[warp];
    float* keys = skey[warp];
    for (int e = lane; e < 128; e += 32) {
        ids[e] = e < KP ? cand_id[r * KP + e] : -1;
        keys[e] = FLT_MAX;
    }
    __syncwarp();
    // compact valid candidates to the front
    int nvalid = 0;
    for (int base = 0; base < 128; base += 32) {
        int v = ids[base + lane];
        unsigned m = __ballot_sync(VJ_FULL, v >= 0);
        __syncwarp();
        if (v >= 0) ids[nvalid + __popc(m & ((1u << lane) - 1u))] = v;
        nvalid += __popc(m);
        __syncwarp();
    }
    for (int e = nvalid + lane; e < 128; e += 32) ids[e] = INT32_MAX;
    __syncwarp();
    float4 q[NPL];
    load_slots<G, NPL>(vec, r, dp / 4, lane & (G - 1), q);
    const float invq = metric ? invn[r] : 0.f;
    group_keys<G, NPL, 1>(vec, invn, dp / 4, metric, q, invq, ids, nvalid, keys, lane);
    __syncwarp();
    // bitonic sort of 128 (key, id) pairs in shared memory
    for (int k = 2; k <= 128; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = lane; i < 128; i += 32) {
                int p = i ^ j;
                if (p > i) {
                    bool up = (i & k) == 0;
                    bool gt = kless(keys[p], ids[p], keys[i], ids[i]);
                    if (gt == up) {
                        float tk = keys[i];
                        int ti = ids[i];
                        keys[i] = keys[p];
                        ids[i] = ids[p];
                        keys[p] = tk;
                        ids[p] = ti;
                    }
                }
            }
            __syncwarp();
        }
    }
    // near-tie runs among the first min(K+1, nvalid) entries: FP64 re-rank
    const float tol = 2.0f * (float)(dp + 4) * VJ_F32_U * (metric == 0 ? 1.0f : 4.0f) + 1e-7f;
    const int lim = min(K + 1, nvalid);
    int i0 = 0;
    while (i0 < lim) {
        int i1 = i0;
        while (i1 + 1 < nvalid &&
               (metric == 0 ? keys[i1 + 1] - keys[i1] <= tol * keys[i1 + 1] : keys[i1 + 1] - keys[i1] <= tol))
            i1++;
        if (i1 > i0) {
            for (int e = i0; e <= i1; e++) {
                double dd = warp_dist64(vec, dp, d, metric, r, ids[e], lane);
                if (lane == 0) s64[warp][e] = dd;
            }
            __syncwarp();
            if (lane == 0) {
                atomicAdd(nrechk, 1ull);
                // insertion sort of the run by (d64, id)
                for (int a = i0 + 1; a <= i1; a++) {
                    double da = s64[warp][a];
                    int ia = ids[a];
                    float ka = keys[a];
                    int b = a - 1;
                    while (b >= i0 && (s64[warp][b] > da || (s64[warp][b] == da && ids[b] > ia))) {
                        s64[warp][b + 1] = s64[warp][b];
                        ids[b + 1] = ids[b];
                        keys[b + 1] = keys[b];
                        b--;
                    }
                    s64[warp][b + 1] = da;
                    ids[b + 1] = ia;
                    keys[b + 1] = ka;
                }
            }
            __syncwarp();
        }
        i0 = i1 + 1;
    }
    // certificate: every node outside the candidate list has a Gram key >=
    // row_thr, hence a true key >= row_thr - beta (thr_true: row_thr already
    // bounds the true key)
    bool full = nvalid >= KP;  // a short list holds every other node
    bool ok = true;
    if (full && K <= nvalid) {
        float kth = keys[K - 1];
        double an = metric == 0 ? sqrt((double)sqn[r]) : 1.0;
        double mx = metric == 0 ? maxnorm : 1.0;
        double beta = thr_true ? 0.0 : (2.0 * dp + 10.0) * (double)VJ_F32_U * (an + mx) * (an + mx) + 1e-30;
        double kth_hi = (double)kth * (1.0 + tol);
        ok = kth_hi + beta < (double)row_thr[r];
    }
    if (!ok && lane == 0) {
        int slot = atomicAdd(nbad, 1);
        bad_rows[slot] = (int32_t)r;
    }
    for (int e = lane; e < K; e += 32) {
        out_id[r * K + e] = e < nvalid ? ids[e] : -1;
        out_key[r * K + e] = e < nvalid ? keys[e] : FLT_MAX;
    }
}

// warp per row over a CSR candidate list (at most KC_CAP, the row itself
// dropped): exact keys, sort, FP64 near-tie runs, then the certificate
// against row_thr, a lower bound on the true key of every node not listed.
// Rows that cannot be certified (or list more than KC_CAP) go to bad_rows.
//
// With the streamed kernel's tile values cw (acc * cs per candidate), an
// approximate key k~ = |a|^2 + |b|^2 - cw (L2), 1 - cw / |a| (cosine, raw
// rows) or 1 - cw (cosine, unit rows) comes first, within beta of the true
// key (beta = cb |a||b| + (c3 + 4u)(|a|^2 + |b|^2), or cb + 4u for cosine,
// bounded with the largest norm).  Only the prefix with k~ <= k~_K + 2 beta
// can hold the top K; it alone gets exact keys, and every candidate after it
// has a true key above k~_min_out - beta, which joins the certificate.
constexpr int KC_CAP = 1024;
constexpr int KC_WPB = 4;

// bitonic sort of P2 (key, id) pairs in shared memory, ascending (one warp)
__device__ void bitonic_pairs(float* key, int* id, int P2, int lane) {
    for (int k = 2; k <= P2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = lane; i < P2; i += 32) {
                const int p = i ^ j;
                if (p > i) {
                    const bool up = (i & k) == 0;
                    const bool gt = kless(key[p], id[p], key[i], id[i]);
                    if (gt == up) {
                        const float tk = key[i];
                        const int ti = id[i];
                        key[i] = key[p];
                        id[i] = id[p];
                        key[p] = tk;
                        id[p] = ti;
                    }
                }
            }
            __syncwarp();
        }
    }
}

constexpr int KC_E64 = 256;  // prefix lengths ranked directly in FP64

struct KcSmem {
    int id[KC_CAP];
    float key[KC_CAP];
    double d64[128];
    double e64[KC_E64];
};

// bitonic sort of P2 (FP64 key, id) pairs in shared memory, ascending (one warp)
__device__ void bitonic_pairs64(double* key, int* id, int P2, int lane) {
    for (int k = 2; k <= P2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = lane; i < P2; i += 32) {
                const int p = i ^ j;
                if (p > i) {
                    const bool up = (i & k) == 0;
                    const bool gt = key[p] < key[i] || (key[p] == key[i] && id[p] < id[i]);
                    if (gt == up) {
                        const double tk = key[i];
                        const int ti = id[i];
                        key[i] = key[p];
                        id[i] = id[p];
                        key[p] = tk;
                        id[p] = ti;
                    }
                }
            }
            __syncwarp();
        }
    }
}

// FP64 keys of q (FP32 slots in registers, |q|^2 = qq in FP64) to cand[0..nc):
// L2 the squared distance, cosine 1 - <x,q> / (|x||q|) with |x|^2 from sqn64;
// FP32 inputs make every product exact in FP64, so these equal the
// definition's keys up to FP64 summation order.  U candidates per lane group
// in flight, as group_keys.
template <int G, int NPL, int U>
__device__ void group_keys64(const float* __restrict__ vec, const double* __restrict__ sqn64, int dp4, int metric,
                             const float4 (&q)[NPL], double qq, const int32_t* cand, int nc, double* key, int lane) {
    constexpr int NG = 32 / G;
    const int grp = lane / G, g = lane & (G - 1);
    for (int base = 0; base < nc; base += NG * U) {
        float4 x[U][NPL];
        int node[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int ci = base + u * NG + grp;
            node[u] = ci < nc ? cand[ci] : -1;
            if (node[u] >= 0) {
                load_slots<G, NPL>(vec, node[u], dp4, g, x[u]);
            } else {
#pragma unroll
                for (int k = 0; k < NPL; k++) x[u][k] = f4zero();
            }
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            double a = 0.0;
#pragma unroll
            for (int k = 0; k < NPL; k++) {
                const double xs[4] = {x[u][k].x, x[u][k].y, x[u][k].z, x[u][k].w};
                const double qs[4] = {q[k].x, q[k].y, q[k].z, q[k].w};
#pragma unroll
                for (int c = 0; c < 4; c++) {
                    if (metric == 0) {
                        const double t = xs[c] - qs[c];
                        a = fma(t, t, a);
                    } else {
                        a = fma(xs[c], qs[c], a);
                    }
                }
            }
#pragma unroll
            for (int o = G / 2; o > 0; o >>= 1) a += __shfl_xor_sync(VJ_FULL, a, o);
            const int ci = base + u * NG + grp;
            if (g == 0 && ci < nc) {
                if (metric == 0) {
                    key[ci] = a;
                } else {
                    const double xx = sqn64[node[u]];
                    key[ci] = (xx == 0.0 || qq == 0.0) ? 1.0 : 1.0 - a / (sqrt(xx) * sqrt(qq));
                }
            }
        }
    }
}

template <int G, int NPL, int U>
__global__ void __launch_bounds__(KC_WPB * 32)
    k_knn_rerank_csr(const float* __restrict__ vec, const float* __restrict__ invn, int dp, int d, int64_t n,
                     int metric, int K, const int64_t* __restrict__ off, const int32_t* __restrict__ cand,
                     const float* __restrict__ row_thr, int32_t* __restrict__ out_id, float* __restrict__ out_key,
                     int32_t* __restrict__ bad_rows, int* __restrict__ nbad, unsigned long long* __restrict__ nrechk,
                     const float* __restrict__ cw, const float* __restrict__ sqn, int raw, float cb, float c3,
                     float maxnorm, const double* __restrict__ sqn64, double beta_abs) {
    extern __shared__ uint8_t kc_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    KcSmem& S = reinterpret_cast<KcSmem*>(kc_raw)[warp];
    const int64_t r = (int64_t)blockIdx.x * KC_WPB + warp;
    if (r >= n) return;
    const int64_t b = off[r];
    const int cnt = (int)(off[r + 1] - b);
    if (cnt > KC_CAP) {
        if (lane == 0) bad_rows[atomicAdd(nbad, 1)] = (int32_t)r;
        return;
    }
    // compact the list without the row itself (with its approximate keys)
    const float rn2 = cw && metric == 0 ? sqn[r] : 0.f;
    const float rinv = cw && metric != 0 && raw ? invn[r] : 1.f;
    int nvalid = 0;
    for (int base = 0; base < cnt; base += 32) {
        const int v = base + lane < cnt ? cand[b + base + lane] : -1;
        const bool keep = v >= 0 && v != r;
        const unsigned m = __ballot_sync(VJ_FULL, keep);
        if (keep) {
            const int pos = nvalid + __popc(m & ((1u << lane) - 1u));
            S.id[pos] = v;
            if (cw) {
                const float w = cw[b + base + lane];
                S.key[pos] = metric == 0 ? (rn2 + sqn[v]) - w : 1.f - w * rinv;
            }
        }
        nvalid += __popc(m);
    }
    int P2 = 32;
    while (P2 < nvalid) P2 <<= 1;
    for (int e = nvalid + lane; e < P2; e += 32) {
        S.id[e] = INT32_MAX;
        S.key[e] = FLT_MAX;
    }
    __syncwarp();
    // tolerance of the FP32 direct-difference keys (relative for L2)
    const float tol = 2.0f * (float)(dp + 4) * VJ_F32_U * (metric == 0 ? 1.0f : 4.0f) + 1e-7f;
    float out_lo = FLT_MAX;  // approximate-key prefilter: lower bound on every dropped candidate
    bool pref = false;       // the prefilter ran
    if (cw && nvalid > K) {
        pref = true;
        bitonic_pairs(S.key, S.id, P2, lane);
        const double mx = (double)maxnorm;
        // beta_abs: the measured bound's |tile key - key| (TF32 tiles), 0 for the BF16 form
        const double beta = beta_abs + (metric == 0 ? (double)cb * sqrt((double)rn2) * mx +
                                                          ((double)c3 + 4.0 * VJ_F32_U) * ((double)rn2 + mx * mx)
                                                    : (double)cb + 4.0 * VJ_F32_U);
        // the true K-th key is at most k~_K + beta, and the certificate below
        // needs its FP32 key with margin (at most (k~_K + beta)(1 + tol) + tol
        // before rounding slack) under every dropped candidate's lower bound
        // k~ - beta: cut at k~_K + 3 beta plus twice the margin
        const double kk = (double)S.key[K - 1] + beta;
        const double lim = metric == 0 ? kk * (1.0 + 2.0 * (double)tol) + 2.0 * beta : kk + 2.0 * beta + 2.0 * (double)tol;
        int ne = 0;
        for (int base = 0; base < nvalid; base += 32) {
            const bool in = base + lane < nvalid && (double)S.key[base + lane] <= lim;
            ne += __popc(__ballot_sync(VJ_FULL, in));
        }
        if (ne < nvalid) out_lo = (float)((double)S.key[ne] - beta);
        nvalid = ne;
        P2 = 32;
        while (P2 < nvalid) P2 <<= 1;
        for (int e = nvalid + lane; e < P2; e += 32) {
            S.id[e] = INT32_MAX;
            S.key[e] = FLT_MAX;
        }
        __syncwarp();
    }
    float4 q[NPL];
    load_slots<G, NPL>(vec, r, dp / 4, lane & (G - 1), q);
    const float invq = metric ? invn[r] : 0.f;
    if (pref && nvalid <= KC_E64) {
        // the prefix in FP64: its order is the definition's (ties by id), no
        // FP32 near-tie runs to resolve
        int Q2 = 32;
        while (Q2 < nvalid) Q2 <<= 1;
        group_keys64<G, NPL, U>(vec, sqn64, dp / 4, metric, q, sqn64[r], S.id, nvalid, S.e64, lane);
        for (int e = nvalid + lane; e < Q2; e += 32) {
            S.e64[e] = DBL_MAX;
            S.id[e] = INT32_MAX;
        }
        __syncwarp();
        bitonic_pairs64(S.e64, S.id, Q2, lane);
        bool ok = nvalid >= K;
        if (ok) {
            const double kth = S.e64[K - 1];
            const double hi = kth + 1e-12 * (1.0 + fabs(kth));
            ok = hi < (double)row_thr[r] && hi < (double)out_lo;
        }
        if (!ok) {
            if (lane == 0) bad_rows[atomicAdd(nbad, 1)] = (int32_t)r;
            return;
        }
        for (int e = lane; e < K; e += 32) {
            out_id[r * K + e] = S.id[e];
            out_key[r * K + e] = (float)S.e64[e];
        }
        return;
    }
    group_keys<G, NPL, U>(vec, invn, dp / 4, metric, q, invq, S.id, nvalid, S.key, lane);
    __syncwarp();
    bitonic_pairs(S.key, S.id, P2, lane);
    // near-tie runs among the first K + 1: FP64 re-rank (runs stay below 128)
    const int lim = min(K + 1, nvalid);
    bool ok = nvalid >= K;
    int i0 = 0;
    while (i0 < lim) {
        int i1 = i0;
        while (i1 + 1 < nvalid &&
               (metric == 0 ? S.key[i1 + 1] - S.key[i1] <= tol * S.key[i1 + 1] : S.key[i1 + 1] - S.key[i1] <= tol))
            i1++;
        if (i1 > i0) {
            if (i1 - i0 >= 128) {
                ok = false;  // a tie run this long is left to the exact row scan
                break;
            }
            for (int e = i0; e <= i1; e++) {
                const double dd = warp_dist64(vec, dp, d, metric, r, S.id[e], lane);
                if (lane == 0) S.d64[e - i0] = dd;
            }
            __syncwarp();
            if (lane == 0) {
                atomicAdd(nrechk, 1ull);
                for (int a = i0 + 1; a <= i1; a++) {
                    const double da = S.d64[a - i0];
                    const int ia = S.id[a];
                    const float ka = S.key[a];
                    int c = a - 1;
                    while (c >= i0 && (S.d64[c - i0] > da || (S.d64[c - i0] == da && S.id[c] > ia))) {
                        S.d64[c + 1 - i0] = S.d64[c - i0];
                        S.id[c + 1] = S.id[c];
                        S.key[c + 1] = S.key[c];
                        c--;
                    }
                    S.d64[c + 1 - i0] = da;
                    S.id[c + 1] = ia;
                    S.key[c + 1] = ka;
                }
            }
            __syncwarp();
        }
        i0 = i1 + 1;
    }
    // certificate: the K-th key, with its rounding margin, below the bound on
    // every node not listed
    if (ok) {
        const double kth = (double)S.key[K - 1];
        const double hi = metric == 0 ? kth * (1.0 + tol) : kth + tol;
        ok = hi < (double)row_thr[r] && hi < (double)out_lo;
    }
    if (!ok) {
        if (lane == 0) bad_rows[atomicAdd(nbad, 1)] = (int32_t)r;
        return;
    }
    for (int e = lane; e < K; e += 32) {
        out_id[r * K + e] = S.id[e];
        out_key[r * K + e] = S.key[e];
    }
}

// ---------------------------------------------------------------- fallback
// warp per uncertified row: brute-force top-K' over all candidate nodes with
// direct-difference keys, then the same re-rank (run again on its output)
template <int G, int NPL>
__global__ void __launch_bounds__(256) k_knn_rowscan(const float* __restrict__ vec, const float* __restrict__ invn,
                                                      int dp, int64_t nx, int64_t n, int knn_mode, int metric, int KP,
                                                      const int32_t* __restrict__ rows, int nrows,
                                                      int32_t* __restrict__ cand_id, float* __restrict__ row_thr) {
    __shared__ int cid[8][128];
    __shared__ float ckey[8][128];
    __shared__ float lk[8][128];
    __shared__ int li[8][128];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int w = blockIdx.x * 8 + warp;
    if (w >= nrows) return;
    const int64_t r = rows[w];
    for (int e = lane; e < 128; e += 32) {
        lk[warp][e] = FLT_MAX;
        li[warp][e] = INT32_MAX;
    }
    __syncwarp();
    float4 q[NPL];
    load_slots<G, NPL>(vec, r, dp / 4, lane & (G - 1), q);
    const float invq = metric ? invn[r] : 0.f;
    // the row's candidate nodes [lo, hi)
    const int64_t lo = (knn_mode == VJ_KNN_GROUPS && r >= nx) ? nx : 0;
    const int64_t hi = knn_mode == VJ_KNN_DATA || (knn_mode == VJ_KNN_GROUPS && r < nx) ? nx : n;
    for (int64_t c0 = lo; c0 < hi; c0 += 128) {
        int nc = (hi - c0) < 128 ? (int)(hi - c0) : 128;
        for (int e = lane; e < 128; e += 32) cid[warp][e] = (int)(c0 + e);
        __syncwarp();
        group_keys<G, NPL, 1>(vec, invn, dp / 4, metric, q, invq, cid[warp], nc, ckey[warp], lane);
        __syncwarp();
        for (int e0 = 0; e0 < nc; e0 += 32) {
            int e = e0 + lane;
            float k = e < nc ? ckey[warp][e] : FLT_MAX;
            int id = (int)(c0 + e);
            bool ok = e < nc && id != r;
            float thr = lk[warp][KP - 1];
            int thi = li[warp][KP - 1];
            unsigned m = __ballot_sync(VJ_FULL, ok && kless(k, id, thr, thi));
            while (m) {
                int src = __ffs(m) - 1;
                m &= m - 1;
                float kk = __shfl_sync(VJ_FULL, k, src);
                int ii = __shfl_sync(VJ_FULL, id, src);
                list_insert<128>(lk[warp], li[warp], kk, ii, lane);
            }
        }
    }
    for (int e = lane; e < KP; e += 32) cand_id[r * KP + e] = li[warp][e] == INT32_MAX ? -1 : li[warp][e];
    // the scan saw every node: no outside candidate exists
    if (lane == 0) row_thr[r] = FLT_MAX;
}

// ---------------------------------------------------------------- NLJ
// warp per 32 candidates: direct-difference key, FP64 near eps; survivors get
// counted per query and kept (flag)
__global__ void k_nlj_recheck(const float* __restrict__ vec, const float* __restrict__ invn, int dp, int d,
                              int64_t nx, int metric, float eps_key, float band, double eps64,
                              const int32_t* __restrict__ cq, const int32_t* __restrict__ cx, int64_t nc,
                              float* __restrict__ cd, int32_t* __restrict__ counts,
                              unsigned long long* __restrict__ nrechk) {
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t e = w * 32 + lane;
    // each lane computes its own pair's key sequentially (vectors are short-lived in L2)
    const bool inb = e < nc;
    bool valid = inb && cq[e] >= 0;  // -1: a hole in the candidate list
    float key = FLT_MAX;
    int64_t qn = 0, xn = 0;
    if (valid) {
        qn = nx + cq[e];
        xn = cx[e];
        const float4* a = reinterpret_cast<const float4*>(vec + qn * dp);
        const float4* b = reinterpret_cast<const float4*>(vec + xn * dp);
        float s = 0.f;
        for (int i = 0; i < dp / 4; i++) {
            float4 x = __ldg(a + i), y = __ldg(b + i);
            if (metric == 0) {
                float t0 = x.x - y.x, t1 = x.y - y.y, t2 = x.z - y.z, t3 = x.w - y.w;
                s = fmaf(t0, t0, s);
                s = fmaf(t1, t1, s);
                s = fmaf(t2, t2, s);
                s = fmaf(t3, t3, s);
            } else {
                s = fmaf(x.x, y.x, s);
                s = fmaf(x.y, y.y, s);
                s = fmaf(x.z, y.z, s);
                s = fmaf(x.w, y.w, s);
            }
        }
        key = metric == 0 ? s : 1.f - s * invn[qn] * invn[xn];
    }
    float scale = metric == 0 ? eps_key : 1.f;
    bool in = valid && key < eps_key;
    bool near = valid && fabsf(key - eps_key) <= band * scale;
    unsigned nm = __ballot_sync(VJ_FULL, near);
    while (nm) {
        int src = __ffs(nm) - 1;
        nm &= nm - 1;
        int64_t a = __shfl_sync(VJ_FULL, qn, src), b = __shfl_sync(VJ_FULL, xn, src);
        double dd = warp_dist64(vec, dp, d, metric, a, b, lane);
        if (lane == src) in = dd < eps64;
        if (lane == 0) atomicAdd(nrechk, 1ull);
    }
    if (valid) {
        cd[e] = in ? (metric == 0 ? sqrtf(fmaxf(key, 0.f)) : key) : -1.f;
        if (in) atomicAdd(counts + cq[e], 1);
    } else if (inb) {
        cd[e] = -1.f;
    }
}

// candidates with exact integer keys K (L2 on integer inputs): a pair is in
// the join iff sqrt(K) < eps in FP64, exactly the definition's decision
__global__ void k_exact_decide(const float* __restrict__ ck, const int32_t* __restrict__ cq, int64_t nc, double eps64,
                               float* __restrict__ cd, int32_t* __restrict__ counts) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nc) return;
    if (cq[e] < 0) {  // a hole in the candidate list
        cd[e] = -1.f;
        return;
    }
    const double dd = sqrt(fmax((double)ck[e], 0.0));
    const bool in = dd < eps64;
    cd[e] = in ? sqrtf(fmaxf(ck[e], 0.f)) : -1.f;  // the traversal's FP32 distance of the same key
    if (in) atomicAdd(counts + cq[e], 1);
}

__global__ void k_nlj_scatter(const int32_t* __restrict__ cq, const int32_t* __restrict__ cx,
                              const float* __restrict__ cd, int64_t nc, const int64_t* __restrict__ offsets,
                              int32_t* __restrict__ cursor, int32_t* __restrict__ tid, float* __restrict__ td) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nc || cd[e] < 0.f) return;
    int q = cq[e];
    int pos = atomicAdd(cursor + q, 1);
    tid[offsets[q] + pos] = cx[e];
    td[offsets[q] + pos] = cd[e];
}

}  // namespace

// template dispatch on the padded dimension for the warp-per-row kernels

void vj_compute_norms(vj_index* ix, double* maxnorm_out) {
    cudaStream_t s = ix->stream;
    DBuf<double> mx;
    mx.alloc(1, s);
    VJ_CUDA(cudaMemsetAsync(mx.p, 0, sizeof(double), s));
    ix->sqn64.ensure(ix->n, s);
    k_norms<<<vj_div_up(ix->n * 32, 256), 256, 0, s>>>(ix->vec.p, ix->dp, ix->d, ix->n, ix->sqn.p, ix->invn.p,
                                                         ix->sqn64.p, mx.p);
    VJ_LAUNCH_CHECK();
    VJ_CUDA(cudaMemcpyAsync(maxnorm_out, mx.p, sizeof(double), cudaMemcpyDeviceToHost, s));
    VJ_CUDA(cudaStreamSynchronize(s));
    mx.free_(s);
}

template <int KP>
static void run_sweep(vj_index* ix, int32_t* cid, float* ckey, float* thr) {
    size_t smem = sizeof(KnnSmem<KP>);
    VJ_CUDA(cudaFuncSetAttribute(k_knn_sweep<KP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // (row range, candidate range) blocks of the index's kNN mode
    const int64_t n = ix->n, nx = ix->nx;
    int64_t blk[2][4] = {{0, n, 0, n}, {0, 0, 0, 0}};
    if (ix->knn_mode == VJ_KNN_DATA) blk[0][3] = nx;
    if (ix->knn_mode == VJ_KNN_GROUPS) {
        blk[0][1] = nx;
        blk[0][3] = nx;
        blk[1][0] = nx;
        blk[1][1] = n;
        blk[1][2] = nx;
        blk[1][3] = n;
    }
    for (auto& b : blk) {
        if (b[1] <= b[0]) continue;
        k_knn_sweep<KP><<<vj_div_up(b[1] - b[0], TBM), TT, smem, ix->stream>>>(
            ix->vec.p, ix->sqn.p, ix->invn.p, ix->dp, b[0], b[1], b[2], b[3], ix->metric, cid, ckey, thr);
        VJ_LAUNCH_CHECK();
    }
}

void vj_build_knn(vj_index* ix) {
    cudaStream_t s = ix->stream;
    const int64_t n = ix->n;
    const int K = ix->K;
    double maxnorm = 0.0;
    vj_compute_norms(ix, &maxnorm);
    ix->maxnorm = maxnorm;
    int KP = K + std::max(16, K / 4);
    KP = std::min(KP, 128);
    KP = (KP + 31) / 32 * 32;
    if (KP > 128) KP = 128;
    VJ_REQUIRE(K < KP || K == 128, VJ_ERR_ARG, "knn_k too large");
    ix->knn.ensure((size_t)n * K, s);
    ix->knnd.ensure((size_t)n * K, s);
    DBuf<int32_t> bad;
    DBuf<int> nbad;
    DBuf<unsigned long long> nr;
    bad.alloc(n, s);
    nbad.alloc(1, s);
    nr.alloc(1, s);
    VJ_CUDA(cudaMemsetAsync(nbad.p, 0, sizeof(int), s));
    VJ_CUDA(cudaMemsetAsync(nr.p, 0, sizeof(unsigned long long), s));
    const int dp4 = ix->dp / 4;
    DBuf<int32_t> cid;
    DBuf<float> ckey, thr;
    // tensor cores (BF16 tiles; per-row candidate lists with a bound on the
    // true key of every node left out) when the rows fit the resident kernel,
    // the FP32 SIMT sweep otherwise; exact re-rank and certificate either way
    bool tc = false;
    if (ix->p.precision == VJ_PREC_BF16) {
        DBuf<int64_t> coff;
        DBuf<int32_t> cids;
        DBuf<float> cthr, cw;
        tc = vj_tc_knn_candidates(ix, coff, cids, cthr, &cw);
        if (tc) {
            const int smem = KC_WPB * (int)sizeof(KcSmem);
            const float* w = cw.n > 0 ? cw.p : nullptr;  // tile values: streamed kernel only
            // rows wider than 512 floats keep four candidates' gathers in flight per warp
            auto launch = [&](auto kern) {
                VJ_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
                kern<<<vj_div_up(n, KC_WPB), KC_WPB * 32, smem, s>>>(
                    ix->vec.p, ix->invn.p, ix->dp, ix->d, n, ix->metric, K, coff.p, cids.p, cthr.p, ix->knn.p,
                    ix->knnd.p, bad.p, nbad.p, nr.p, w, ix->sqn.p, ix->knn_measured ? 0 : (ix->cos_raw ? 1 : 0),
                    ix->knn_measured ? 0.f : ix->tc_cb, ix->knn_measured ? 0.f : ix->tc_c3,
                    (float)(ix->maxnorm * 1.0001), ix->sqn64.p, ix->knn_measured ? ix->knn_beta : 0.0);
            };
            VJ_DISPATCH_GN(dp4, {
                if (dp4 > 128) launch(k_knn_rerank_csr<G, NPL, 4>);
                else launch(k_knn_rerank_csr<G, NPL, 1>);
            });
            VJ_LAUNCH_CHECK();
        }
        coff.free_(s);
        cids.free_(s);
        cthr.free_(s);
        cw.free_(s);
    }
    ix->knn_tc = tc;
    cid.alloc((size_t)n * KP, s);
    thr.alloc(n, s);
    if (!tc) {
        ckey.alloc((size_t)n * KP, s);
        switch (KP) {
            case 32: run_sweep<32>(ix, cid.p, ckey.p, thr.p); break;
            case 64: run_sweep<64>(ix, cid.p, ckey.p, thr.p); break;
            case 96: run_sweep<96>(ix, cid.p, ckey.p, thr.p); break;
            default: run_sweep<128>(ix, cid.p, ckey.p, thr.p); break;
        }
        VJ_DISPATCH_GN(dp4, (k_knn_rerank<G, NPL><<<vj_div_up(n, 8), 256, 0, s>>>(
                                ix->vec.p, ix->invn.p, ix->sqn.p, ix->dp, ix->d, n, ix->metric, KP, K, cid.p, thr.p,
                                0, maxnorm, nullptr, n, ix->knn.p, ix->knnd.p, bad.p, nbad.p, nr.p)));
        VJ_LAUNCH_CHECK();
    }
    int hb = 0;
    VJ_CUDA(cudaMemcpyAsync(&hb, nbad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    VJ_CUDA(cudaStreamSynchronize(s));
    ix->knn_uncertified = hb;
    if (hb > 0) {
        // exact row scans for the uncertified rows, then re-rank them again
        // (their scans fill cid / thr at the rows' own positions)
        VJ_DISPATCH_GN(dp4, (k_knn_rowscan<G, NPL><<<vj_div_up(hb, 8), 256, 0, s>>>(
                                ix->vec.p, ix->invn.p, ix->dp, ix->nx, n, ix->knn_mode, ix->metric, KP, bad.p, hb,
                                cid.p, thr.p)));
        VJ_LAUNCH_CHECK();
        // the row scans saw every node, so these rows certify on re-rank
        DBuf<int32_t> bad2;
        bad2.alloc(hb, s);
        VJ_CUDA(cudaMemsetAsync(nbad.p, 0, sizeof(int), s));
        VJ_DISPATCH_GN(dp4, (k_knn_rerank<G, NPL><<<vj_div_up(hb, 8), 256, 0, s>>>(
                                ix->vec.p, ix->invn.p, ix->sqn.p, ix->dp, ix->d, n, ix->metric, KP, K, cid.p, thr.p,
                                0, maxnorm, bad.p, hb, ix->knn.p, ix->knnd.p, bad2.p, nbad.p, nr.p)));
        VJ_LAUNCH_CHECK();
        bad2.free_(s);
    }
    bad.free_(s);
    nbad.free_(s);
    nr.free_(s);
    cid.free_(s);
    ckey.free_(s);
    thr.free_(s);
}

void vj_exact_join_device(vj_index* ix, float eps, DBuf<int64_t>& offsets, DBuf<int32_t>& ids, DBuf<float>& dists,
                          int64_t* nnz_out, double* ms_out) {
    vj_scan_rows_csr(ix, nullptr, ix->nq, eps, offsets, ids, dists, nnz_out, ms_out, true);
}

// Exact join rows of the queries `qrows` (nullptr: all queries) by the
// tensor-core scan and the exact re-check; CSR over all nq queries, rows of
// queries not listed are empty.
void vj_scan_rows_csr(vj_index* ix, const int32_t* qrows, int64_t nr, float eps, DBuf<int64_t>& offsets,
                      DBuf<int32_t>& ids, DBuf<float>& dists, int64_t* nnz_out, double* ms_out, bool sort_rows) {
    cudaStream_t s = ix->stream;
    const int64_t nx = ix->nx, nq = ix->nq;
    cudaEvent_t e0, e1;
    VJ_CUDA(cudaEventCreate(&e0));
    VJ_CUDA(cudaEventCreate(&e1));
    VJ_CUDA(cudaEventRecord(e0, s));
    const float eps_key = ix->metric == VJ_L2 ? eps * eps : eps;
    // candidates from the BF16 tensor-core scan (a bounded superset of the
    // result), then the exact FP32 / FP64 re-decision below
    // candidate arrays stay with the index: later scans start at the size the
    // largest earlier one needed instead of re-running the scan to grow them
    DBuf<int32_t>& cq = ix->scan_cq;
    DBuf<int32_t>& cx = ix->scan_cx;
    DBuf<float> cd;
    DBuf<unsigned long long> ctr;
    ctr.alloc(2, s);
    VJ_CUDA(cudaMemsetAsync(ctr.p, 0, 2 * sizeof(unsigned long long), s));
    double ms_scan = 0.0;
    const int64_t nc = nr > 0 ? vj_tc_scan_candidates(ix, qrows, nr, eps, cq, cx, &ms_scan, &ix->scan_ck) : 0;
    const bool exact_keys = nr > 0 && ix->last_scan_exact_keys;
    ix->last_scan_ms = ms_scan;
    ix->last_scan_cand = nc;
    DBuf<int32_t> counts, cursor;
    counts.alloc(nq, s);
    cursor.alloc(nq, s);
    cd.alloc(std::max<int64_t>(nc, 1), s);
    VJ_CUDA(cudaMemsetAsync(counts.p, 0, nq * sizeof(int32_t), s));
    VJ_CUDA(cudaMemsetAsync(cursor.p, 0, nq * sizeof(int32_t), s));
    const float band = 2.0f * (float)(ix->dp + 4) * VJ_F32_U * (ix->metric == VJ_L2 ? 1.0f : 4.0f) + 1e-6f;
    if (nc > 0 && exact_keys) {
        // integer inputs: the scan's keys are exact; decide as the FP64 definition does
        k_exact_decide<<<vj_div_up(nc, 256), 256, 0, s>>>(ix->scan_ck.p, cq.p, nc, (double)eps, cd.p, counts.p);
        VJ_LAUNCH_CHECK();
    } else if (nc > 0) {
        k_nlj_recheck<<<vj_div_up(nc, 256), 256, 0, s>>>(ix->vec.p, ix->invn.p, ix->dp, ix->d, nx, ix->metric,
                                                         eps_key, band, (double)eps, cq.p, cx.p, nc, cd.p, counts.p,
                                                         ctr.p + 1);
        VJ_LAUNCH_CHECK();
    }
    offsets.ensure(nq + 1, s);
    vj_exclusive_scan_i32_to_i64(counts.p, offsets.p, nq, ix);
    int64_t nnz = 0;
    VJ_CUDA(cudaMemcpyAsync(&nnz, offsets.p + nq, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    VJ_CUDA(cudaStreamSynchronize(s));
    DBuf<int32_t> tid;
    DBuf<float> td;
    tid.alloc(std::max<int64_t>(nnz, 1), s);
    td.alloc(std::max<int64_t>(nnz, 1), s);
    if (nc > 0) {
        k_nlj_scatter<<<vj_div_up(nc, 256), 256, 0, s>>>(cq.p, cx.p, cd.p, nc, offsets.p, cursor.p, tid.p, td.p);
        VJ_LAUNCH_CHECK();
    }
    if (sort_rows) {
        ids.ensure(std::max<int64_t>(nnz, 1), s);
        dists.ensure(std::max<int64_t>(nnz, 1), s);
        vj_segment_sort_copy(offsets.p, counts.p, offsets.p, tid.p, td.p, ids.p, dists.p, nq, ix);
    } else {
        // rows in scatter order: the caller sorts them with the rest of its result
        ids.free_(s);
        dists.free_(s);
        ids = tid;
        dists = td;
        tid = DBuf<int32_t>();
        td = DBuf<float>();
    }
    VJ_CUDA(cudaEventRecord(e1, s));
    VJ_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    VJ_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms_out = ms;
    *nnz_out = nnz;
    tid.free_(s);
    td.free_(s);
    counts.free_(s);
    cursor.free_(s);
    cd.free_(s);
    ctr.free_(s);
}
