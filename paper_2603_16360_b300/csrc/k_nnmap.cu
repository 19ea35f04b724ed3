// k_nnmap.cu -- the NN-Map index (the paper's closing design, "NN-Map"): a
// materialised top-1 join from the queries to the data set, kept beside the
// data set's own graph G_X.  Per query q it stores
//   witness   w(q): the nearest data vector ((dist, id) minimum),
//   wdist     dist(q, w(q)) in FP64 (the join's emptiness certificate: a row
//             with wdist >= eps has no data vector in range),
//   ood       the d1/d2 > 1.5 rule (Sec. 4.4) with N1 = the R nearest data
//             vectors of q, d1 = their mean distance to q, and d2 = the mean
//             length of the G_X edges from N1 to data vectors outside N1 (no
//             such edge: not OOD).
// The index build already holds what this needs: on an NN-Map index every
// node's kNN list ranks data vectors only, in (dist, id) order with FP32
// near-ties re-ranked in FP64, so a query's list starts with w(q) followed by
// the rest of N1; G_X's edge lengths are stored.  One warp per query reads its
// list head, computes the witness distance in FP64, and takes the ratio in
// FP32 from the stored keys and edge lengths, re-deciding it in FP64 when it
// lies within the FP32 error bound of 1.5.
#include <float.h>

#include "vj_device.cuh"
#include "vj_internal.cuh"

namespace {

constexpr int NM_WPB = 8;  // warps (queries) per block

__device__ __forceinline__ float nm_key_to_dist(int metric, float k) { return metric == 0 ? sqrtf(fmaxf(k, 0.f)) : k; }

__global__ void __launch_bounds__(NM_WPB * 32)
    k_nnmap(const float* __restrict__ vec, int dp, int d, int64_t nx, int64_t nq, int metric, int K, int R,
            float key_tol, const int32_t* __restrict__ knn, const float* __restrict__ knnd,
            const int32_t* __restrict__ adj, const float* __restrict__ elen, int32_t* __restrict__ w_out,
            double* __restrict__ wd_out, uint8_t* __restrict__ ood_out, unsigned long long* __restrict__ nrechk) {
    __shared__ int n1ids[NM_WPB][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t qi = (int64_t)blockIdx.x * NM_WPB + warp;
    if (qi >= nq) return;
    const int64_t qn = nx + qi;
    // N1: the first R entries of the query's data-only kNN list
    const int id = lane < R ? __ldg(knn + qn * K + lane) : -1;
    const float key = lane < R ? __ldg(knnd + qn * K + lane) : FLT_MAX;
    const bool valid = id >= 0;
    n1ids[warp][lane] = valid ? id : -1;
    __syncwarp();
    const int w = __shfl_sync(VJ_FULL, id, 0);
    const double wd = w >= 0 ? warp_dist64(vec, dp, d, metric, qn, w, lane) : 1e300;
    const unsigned vmask = __ballot_sync(VJ_FULL, valid);
    const int n1 = __popc(vmask);

    // d1 and d2 in FP32 from the stored keys and edge lengths
    float d1s = valid ? nm_key_to_dist(metric, key) : 0.f;
    float d2s = 0.f;
    int n2 = 0;
    unsigned dm = vmask;
    while (dm) {
        // four members' G_X rows per round, their loads issued together
        int vr[4];
        int u4[4];
        float e4[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            vr[k] = -1;
            if (dm) {  // dm is warp-uniform
                const int src = __ffs(dm) - 1;
                dm &= dm - 1;
                vr[k] = __shfl_sync(VJ_FULL, id, src);
            }
        }
#pragma unroll
        for (int k = 0; k < 4; k++) {
            u4[k] = (vr[k] >= 0 && lane < R) ? __ldg(adj + (int64_t)vr[k] * R + lane) : -1;
            e4[k] = (vr[k] >= 0 && lane < R) ? __ldg(elen + (int64_t)vr[k] * R + lane) : 0.f;
        }
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const int u = u4[k];
            bool ok = u >= 0 && u < nx;
            if (ok)
                for (int j = 0; j < R; j++) ok &= n1ids[warp][j] != u;
            if (ok) {
                d2s += e4[k];
                n2++;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        d1s += __shfl_xor_sync(VJ_FULL, d1s, o);
        d2s += __shfl_xor_sync(VJ_FULL, d2s, o);
        n2 += __shfl_xor_sync(VJ_FULL, n2, o);
    }
    int ood = 0;
    if (n1 > 0 && n2 > 0) {
        const float m1 = d1s / (float)n1, m2 = d2s / (float)n2;
        const float r = m1 / m2;
        // relative error of the FP32 ratio: the keys' rounding bound (relative
        // for L2 distances, absolute for cosine keys) plus the sums' rounding
        const float rel = metric == 0 ? key_tol + 64.f * VJ_F32_U
                                      : (m1 > 0.f ? key_tol / m1 : 1.f) + (m2 > 0.f ? key_tol / m2 : 1.f);
        const float band = 1e-3f + 4.f * rel;
        if (m2 > 0.f && r == r && fabsf(r - 1.5f) > 1.5f * band) {
            ood = r > 1.5f;
        } else {
            // FP64 re-decision of the ratio over the same members and edges
            double a1 = 0.0, a2 = 0.0;
            unsigned dm2 = vmask;
            while (dm2) {
                const int src = __ffs(dm2) - 1;
                dm2 &= dm2 - 1;
                const int v = __shfl_sync(VJ_FULL, id, src);
                a1 += warp_dist64(vec, dp, d, metric, qn, v, lane);
                for (int j = 0; j < R; j++) {
                    const int u = __ldg(adj + (int64_t)v * R + j);
                    if (u < 0 || u >= nx) continue;
                    bool inn1 = false;
                    for (int t = 0; t < R; t++) inn1 |= n1ids[warp][t] == u;
                    if (inn1) continue;
                    a2 += warp_dist64(vec, dp, d, metric, v, u, lane);
                }
            }
            ood = a2 > 0.0 && (a1 / n1) / (a2 / n2) > 1.5;
            if (lane == 0) atomicAdd(nrechk, 1ull);
        }
    }
    if (lane == 0) {
        w_out[qi] = w;
        wd_out[qi] = wd;
        ood_out[qi] = (uint8_t)ood;
    }
}

}  // namespace

void vj_build_nnmap(vj_index* ix) {
    cudaStream_t s = ix->stream;
    const int64_t nq = ix->nq;
    VJ_REQUIRE(ix->R <= 32 && ix->K >= ix->R, VJ_ERR_STATE, "NN-Map: degree must be <= 32 and <= knn_k");
    ix->nm_w.ensure(nq, s);
    ix->nm_wd.ensure(nq, s);
    ix->nm_ood.ensure(nq, s);
    DBuf<unsigned long long> nr;
    nr.alloc(1, s);
    VJ_CUDA(cudaMemsetAsync(nr.p, 0, sizeof(unsigned long long), s));
    // per-key rounding bound of the FP32 kNN keys (relative for squared L2
    // distances, so half of it on the distance; absolute for cosine keys)
    const float tol = 2.0f * (float)(ix->dp + 4) * VJ_F32_U * (ix->metric == VJ_L2 ? 1.0f : 4.0f) + 1e-7f;
    k_nnmap<<<vj_div_up(nq, NM_WPB), NM_WPB * 32, 0, s>>>(ix->vec.p, ix->dp, ix->d, ix->nx, nq, ix->metric, ix->K,
                                                         ix->R, tol, ix->knn.p, ix->knnd.p, ix->adj.p, ix->elen.p,
                                                         ix->nm_w.p, ix->nm_wd.p, ix->nm_ood.p, nr.p);
    VJ_LAUNCH_CHECK();
    VJ_CUDA(cudaStreamSynchronize(s));
    nr.free_(s);
}
