// k_features.cu -- per-query features of the learned predictor and the join
// prologue that turns predictor outputs into a per-query plan.
//
// Cached once per index (eps-independent), warp per query on its merged-graph
// neighbourhood N(q):
//   d1     mean dist(q, v) over data neighbours v (Sec. 4.4)
//   d2     mean dist(v, w) over data neighbours w of those v, w not in N(q)
//          and w != q (Sec. 4.4, from the stored data-edge lengths)
//   dent   dist(q, entry)
//   dnn    min dist(q, v) over data neighbours (the App. C nearest node)
//   n1     number of data neighbours
//   dn[j]  dist(q, slot j) for data neighbours, +inf otherwise
// Features for threshold eps (NF = 7, then the d coordinates of q):
//   d1/eps, d2/eps, d1/d2, dent/eps, dnn/eps, n1/R, #{data neighbours within eps}/R
#include <float.h>

#include "vj_device.cuh"
#include "vj_internal.cuh"

#include <functional>

struct vj_mlp;
void vj_mlp_forward_device(vj_mlp* m, const float* x, int64_t n, float* y_out, cudaStream_t s);
bool vj_mlp_forward_filled(vj_mlp* m, int64_t n, float* y_out, cudaStream_t s,
                           const std::function<void(__nv_bfloat16*, int, const float*, const float*)>& fill);
int vj_mlp_din(const vj_mlp* m);

namespace {

constexpr int NSTAT = 5;

__device__ __forceinline__ float lane_dist(const float* __restrict__ vec, int dp, int d, int metric, int64_t a,
                                           int64_t b, const float* __restrict__ invn) {
    const float* x = vec + a * dp;
    const float* y = vec + b * dp;
    float s = 0.f;
    for (int i = 0; i < d; i++) {
        const float t = metric == 0 ? x[i] - y[i] : 0.f;
        s = metric == 0 ? fmaf(t, t, s) : fmaf(x[i], y[i], s);
    }
    return metric == 0 ? sqrtf(fmaxf(s, 0.f)) : 1.f - s * invn[a] * invn[b];
}

__global__ void __launch_bounds__(256) k_query_stats(const float* __restrict__ vec, const float* __restrict__ invn,
                                                     int dp, int d, int metric, int64_t nx, int64_t nq, int R,
                                                     const int32_t* __restrict__ adj, const float* __restrict__ elen,
                                                     int32_t entry, float* __restrict__ stat,
                                                     float* __restrict__ dn) {
    __shared__ int nbr[8][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t qi = (int64_t)blockIdx.x * 8 + warp;
    if (qi >= nq) return;
    const int64_t qn = nx + qi;
    const int v = lane < R ? adj[qn * R + lane] : -1;
    nbr[warp][lane] = v;
    __syncwarp();
    const bool isd = v >= 0 && v < nx;
    const float dv = isd ? lane_dist(vec, dp, d, metric, qn, v, invn) : INFINITY;
    if (lane < R) dn[qi * R + lane] = dv;
    // two-hop data pairs of this lane's neighbour
    float s2 = 0.f;
    int c2 = 0;
    if (isd) {
        for (int j = 0; j < R; j++) {
            const int w = adj[(int64_t)v * R + j];
            if (w < 0 || w >= nx) continue;
            bool inq = false;
            for (int k = 0; k < 32; k++) inq |= nbr[warp][k] == w;
            if (inq) continue;
            s2 += elen[(int64_t)v * R + j];
            c2++;
        }
    }
    float s1 = isd ? dv : 0.f, mn = dv;
    int c1 = isd ? 1 : 0;
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_xor_sync(VJ_FULL, s1, o);
        s2 += __shfl_xor_sync(VJ_FULL, s2, o);
        c1 += __shfl_xor_sync(VJ_FULL, c1, o);
        c2 += __shfl_xor_sync(VJ_FULL, c2, o);
        mn = fminf(mn, __shfl_xor_sync(VJ_FULL, mn, o));
    }
    if (lane == 0) {
        stat[qi * NSTAT + 0] = c1 ? s1 / c1 : INFINITY;
        stat[qi * NSTAT + 1] = c2 ? s2 / c2 : 0.f;
        stat[qi * NSTAT + 2] = lane_dist(vec, dp, d, metric, qn, entry, invn);
        stat[qi * NSTAT + 3] = mn;
        stat[qi * NSTAT + 4] = (float)c1;
    }
}

// the seven features of query qi (every lane of the warp gets them)
__device__ __forceinline__ void query_features(const float* __restrict__ stat, const float* __restrict__ dn,
                                               int64_t qi, int R, float eps, int lane, float (&f)[VJ_NFEAT]) {
    int nin = 0;
    for (int j = lane; j < R; j += 32) nin += dn[qi * R + j] < eps;
    nin = __reduce_add_sync(VJ_FULL, nin);
    const float d1 = stat[qi * NSTAT + 0], d2 = stat[qi * NSTAT + 1], de = stat[qi * NSTAT + 2];
    const float dnn = stat[qi * NSTAT + 3], n1 = stat[qi * NSTAT + 4];
    auto cap = [](float x) { return fminf(x, 100.f); };
    f[0] = cap(d1 / eps);
    f[1] = cap(d2 / eps);
    f[2] = d2 > 0.f ? cap(d1 / d2) : 100.f;
    f[3] = cap(de / eps);
    f[4] = cap(dnn / eps);
    f[5] = n1 / (float)R;
    f[6] = (float)nin / (float)R;
}

// warp per query: the seven features, then the query's coordinates copied by
// all lanes (coalesced rows)
__global__ void k_features(const float* __restrict__ vec, int dp, int d, int64_t nx, int64_t nq, int R,
                           const float* __restrict__ stat, const float* __restrict__ dn, float eps,
                           float* __restrict__ feat) {
    const int lane = threadIdx.x & 31;
    const int64_t qi = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (qi >= nq) return;  // whole warps
    const int din = VJ_NFEAT + d;
    float* f = feat + qi * din;
    float fv[VJ_NFEAT];
    query_features(stat, dn, qi, R, eps, lane, fv);
    if (lane == 0) {
#pragma unroll
        for (int j = 0; j < VJ_NFEAT; j++) f[j] = fv[j];
    }
    const float* q = vec + (nx + qi) * dp;
    for (int i = lane; i < d; i += 32) f[VJ_NFEAT + i] = q[i];
}

// The predictor's input rows written directly: warp per query, the features
// and coordinates standardised ((v - mu) / sd) and rounded to BF16 into rows
// of k1 columns (zero padded), two columns per lane store.  The same values
// and operations as k_features followed by the predictor's own conversion.
__global__ void k_features_bf16(const float* __restrict__ vec, int dp, int d, int64_t nx, int64_t nq, int R,
                                const float* __restrict__ stat, const float* __restrict__ dn, float eps, int k1,
                                const float* __restrict__ mu, const float* __restrict__ sd,
                                __nv_bfloat16* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t qi = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (qi >= nq) return;  // whole warps
    const int din = VJ_NFEAT + d;
    float fv[VJ_NFEAT];
    query_features(stat, dn, qi, R, eps, lane, fv);
    const float* q = vec + (nx + qi) * dp;
    auto value = [&](int j) -> float {
        float v = 0.f;
        if (j < din) {
            v = j == 0 ? fv[0] : j == 1 ? fv[1] : j == 2 ? fv[2] : j == 3 ? fv[3] : j == 4 ? fv[4] : j == 5 ? fv[5]
                : j == 6 ? fv[6] : q[j - VJ_NFEAT];
            if (mu) v = (v - mu[j]) / sd[j];
        }
        return v;
    };
    __nv_bfloat162* o2 = reinterpret_cast<__nv_bfloat162*>(out + qi * k1);
    for (int j2 = lane; j2 < k1 / 2; j2 += 32) {
        __nv_bfloat162 w;
        w.x = __float2bfloat16_rn(value(2 * j2));
        w.y = __float2bfloat16_rn(value(2 * j2 + 1));
        o2[j2] = w;
    }
}

// plan from predictor outputs: route when the route logit exceeds lthr;
// otherwise the budget b = 2^y0 - 2: below -1/2 no expansion (plan -1), below
// 4 the BFS expansion (plan 0), else the hybrid queue size b (capped)
__global__ void k_plan(const float* __restrict__ y, int64_t nq, float lthr, int beam_cap,
                       uint8_t* __restrict__ route, int32_t* __restrict__ beam, int32_t* __restrict__ routed,
                       unsigned long long* __restrict__ nrouted) {
    const int64_t qi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (qi >= nq) return;
    const bool r = y[2 * qi + 1] > lthr;
    route[qi] = r ? 1 : 0;
    float b = exp2f(fminf(fmaxf(y[2 * qi], 0.f), 20.f)) - 2.f;
    int bi = b < -0.5f ? -1 : (b < 4.f ? 0 : (int)fminf(b + 0.5f, (float)beam_cap));
    if (bi > 0 && beam_cap < 4) bi = 0;  // a cap below 4 allows no hybrid search
    beam[qi] = bi;
    if (r) routed[atomicAdd(nrouted, 1ull)] = (int32_t)qi;
}

}  // namespace

static void ensure_query_stats(vj_index* ix) {
    if (ix->qstat.n >= (size_t)ix->nq * NSTAT) return;
    cudaStream_t s = ix->stream;
    ix->qstat.ensure((size_t)ix->nq * NSTAT, s);
    ix->qdn.ensure((size_t)ix->nq * ix->R, s);
    k_query_stats<<<vj_div_up(ix->nq, 8), 256, 0, s>>>(ix->vec.p, ix->invn.p, ix->dp, ix->d, ix->metric, ix->nx,
                                                       ix->nq, ix->R, ix->adj.p, ix->elen.p, ix->entry, ix->qstat.p,
                                                       ix->qdn.p);
    VJ_LAUNCH_CHECK();
}

void vj_compute_features(vj_index* ix, float eps, float* feat_dev) {
    // the features read each query's merged-graph neighbourhood, which an
    // NN-Map index does not build
    VJ_REQUIRE(!ix->nnmap, VJ_ERR_STATE, "an NN-Map index has no query neighbourhoods for the predictor features");
    ensure_query_stats(ix);
    k_features<<<vj_div_up(ix->nq * 32, 256), 256, 0, ix->stream>>>(ix->vec.p, ix->dp, ix->d, ix->nx, ix->nq,
                                                                     ix->R, ix->qstat.p, ix->qdn.p, eps, feat_dev);
    VJ_LAUNCH_CHECK();
}

// predictor outputs of every query at threshold eps into ix->pred_y
static void predictor_forward(vj_index* ix, float eps) {
    cudaStream_t s = ix->stream;
    const int64_t nq = ix->nq;
    const int din = VJ_NFEAT + ix->d;
    VJ_REQUIRE(vj_mlp_din(ix->predictor) == din, VJ_ERR_ARG, "predictor input size %d != %d features",
               vj_mlp_din(ix->predictor), din);
    ix->pred_y.ensure((size_t)nq * 2, s);
    // the tensor-core forward reads BF16 rows the features kernel writes
    // directly; other predictor shapes take the FP32 features
    VJ_REQUIRE(!ix->nnmap, VJ_ERR_STATE, "an NN-Map index has no query neighbourhoods for the predictor features");
    ensure_query_stats(ix);
    const bool fused = vj_mlp_forward_filled(
        ix->predictor, nq, ix->pred_y.p, s,
        [&](__nv_bfloat16* xbf, int k1, const float* mu, const float* sd) {
            k_features_bf16<<<vj_div_up(nq * 32, 256), 256, 0, s>>>(ix->vec.p, ix->dp, ix->d, ix->nx, nq, ix->R,
                                                                    ix->qstat.p, ix->qdn.p, eps, k1, mu, sd, xbf);
            VJ_LAUNCH_CHECK();
        });
    if (!fused) {
        ix->feat.ensure((size_t)nq * din, s);
        vj_compute_features(ix, eps, ix->feat.p);
        vj_mlp_forward_device(ix->predictor, ix->feat.p, nq, ix->pred_y.p, s);
    }
}

// the learned prologue: features -> predictor -> device plan (route flags,
// beams, routed list); returns the number of routed queries
int64_t vj_learned_prologue(vj_index* ix, float eps) {
    cudaStream_t s = ix->stream;
    const int64_t nq = ix->nq;
    VJ_REQUIRE(ix->predictor != nullptr, VJ_ERR_STATE, "learned join requested but no predictor is attached");
    predictor_forward(ix, eps);
    ix->plan_route.ensure(nq, s);
    ix->plan_beam.ensure(nq, s);
    ix->routed.ensure(nq, s);
    ix->ctr_plan.ensure(1, s);
    VJ_CUDA(cudaMemsetAsync(ix->ctr_plan.p, 0, sizeof(unsigned long long), s));
    const float t = std::min(std::max(ix->route_threshold, 1e-6f), 1.f - 1e-6f);
    const float lthr = logf(t / (1.f - t));
    k_plan<<<vj_div_up(nq, 256), 256, 0, s>>>(ix->pred_y.p, nq, lthr, ix->beam_cap, ix->plan_route.p, ix->plan_beam.p,
                                              ix->routed.p, ix->ctr_plan.p);
    VJ_LAUNCH_CHECK();
    unsigned long long nr = 0;
    VJ_CUDA(cudaMemcpyAsync(&nr, ix->ctr_plan.p, sizeof(nr), cudaMemcpyDeviceToHost, s));
    VJ_CUDA(cudaStreamSynchronize(s));
    ix->nrouted = (int64_t)nr;
    ix->has_route = true;
    ix->has_beam = true;
    ix->plan_max_beam = ix->beam_cap;
    return (int64_t)nr;
}

extern "C" vj_status vj_features(vj_index* ix, float eps, float* out) {
    try {
        VJ_REQUIRE(ix != nullptr && out != nullptr && eps > 0.f, VJ_ERR_ARG, "bad argument");
        cudaStream_t s = ix->stream;
        const int din = VJ_NFEAT + ix->d;
        DBuf<float> f;
        f.alloc((size_t)ix->nq * din, s);
        vj_compute_features(ix, eps, f.p);
        VJ_CUDA(cudaMemcpyAsync(out, f.p, (size_t)ix->nq * din * sizeof(float), cudaMemcpyDeviceToHost, s));
        VJ_CUDA(cudaStreamSynchronize(s));
        f.free_(s);
        return VJ_OK;
    } catch (const VjError& e) {
        return e.code;
    }
}

extern "C" vj_status vj_predictor_outputs(vj_index* ix, float eps, float* out) {
    try {
        VJ_REQUIRE(ix != nullptr && out != nullptr && eps > 0.f, VJ_ERR_ARG, "bad argument");
        VJ_REQUIRE(ix->predictor != nullptr, VJ_ERR_STATE, "no predictor attached");
        cudaStream_t s = ix->stream;
        const int64_t nq = ix->nq;
        predictor_forward(ix, eps);  // the learned prologue's own forward
        VJ_CUDA(cudaMemcpyAsync(out, ix->pred_y.p, (size_t)nq * 2 * sizeof(float), cudaMemcpyDeviceToHost, s));
        VJ_CUDA(cudaStreamSynchronize(s));
        return VJ_OK;
    } catch (const VjError& e) {
        return e.code;
    }
}

extern "C" vj_status vj_attach_predictor(vj_index* ix, vj_mlp* m, float route_threshold, int beam_cap) {
    try {
        VJ_REQUIRE(ix != nullptr, VJ_ERR_ARG, "index is NULL");
        VJ_REQUIRE(beam_cap >= 0 && beam_cap <= (1 << 20), VJ_ERR_ARG, "beam_cap out of range");
        VJ_REQUIRE(route_threshold > 0.f && route_threshold < 1.f, VJ_ERR_ARG, "route_threshold in (0, 1)");
        if (m) VJ_REQUIRE(vj_mlp_din(m) == VJ_NFEAT + ix->d, VJ_ERR_ARG, "predictor input size must be %d + d",
                          VJ_NFEAT);
        ix->predictor = m;
        ix->route_threshold = route_threshold;
        ix->beam_cap = beam_cap;
        return VJ_OK;
    } catch (const VjError& e) {
        return e.code;
    }
}
