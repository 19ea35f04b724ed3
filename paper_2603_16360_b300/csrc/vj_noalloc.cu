// vj_noalloc.cu -- vj_join_exact_noalloc: the exact nested-loop join for
// callers that cannot allocate device memory.
//
// Who needs it: services that run inside a fixed device-memory budget carved
// out up front (an arena handed to them by a host runtime) and may not grow it,
// and latency-critical callers that cannot afford cudaMalloc / cudaFree, which
// take allocator locks and (cudaFree) synchronize the device.  They pass their
// own input and output buffers; the only other memory this entry point touches
// is the file-scope scratch array below.
//
// Scratch: g_na_scratch, a static __device__ array of VJ_NOALLOC_SCRATCH_BYTES
// (4 MiB + 256 B: one int32 match count per query, up to
// VJ_NOALLOC_MAX_QUERIES queries).  A GPU holds it from the moment the
// library's device code is loaded there until the process exits; with lazy
// module loading (CUDA's default) that is the first call into the library on
// that device, so callers with a fixed budget should make one call before the
// budgeted phase (or set CUDA_MODULE_LOADING=EAGER).  All calls share it and it keeps the last call's
// contents; every call overwrites each count it reads before reading it, so
// nothing needs clearing, but two calls whose work overlaps on the GPU race on
// it and produce wrong results.
//
// Host code cannot use the array's name as a device address (it names a host
// shadow), so the first call on each device, with that device current, looks
// the address up with cudaGetSymbolAddress and caches it.  That first call on a
// device should therefore come before any stream capture on it.  Every call
// reads the pair count back to the host and waits for its stream.
#include <float.h>
#include <mutex>

#include "vj_device.cuh"
#include "vj_internal.cuh"

#define VJ_NOALLOC_MAX_QUERIES (1 << 20)
#define VJ_NOALLOC_SCRATCH_BYTES ((size_t)VJ_NOALLOC_MAX_QUERIES * sizeof(int32_t) + 256)

static __device__ __align__(256) unsigned char g_na_scratch[VJ_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int NA_WARPS = 8;
constexpr int NA_MAXD_SMEM = 4096;

// FP32 direct-difference key of data row x against the query held in shared
// memory (L2: squared distance; cosine: 1 - <x,q>/(|x||q|))
__device__ __forceinline__ float na_key(const float* __restrict__ xrow, const float* qs, int d, int metric,
                                        float qn2) {
    float s = 0.f, xx = 0.f;
    for (int i = 0; i < d; i++) {
        float x = __ldg(xrow + i), q = qs[i];
        if (metric == 0) {
            float t = x - q;
            s = fmaf(t, t, s);
        } else {
            s = fmaf(x, q, s);
            xx = fmaf(x, x, xx);
        }
    }
    if (metric == 0) return s;
    if (xx == 0.f || qn2 == 0.f) return 1.f;
    return 1.f - s * rsqrtf(xx) * rsqrtf(qn2);
}

__device__ __forceinline__ double na_dist64(const float* __restrict__ xrow, const float* qs, int d, int metric) {
    double s = 0.0, xx = 0.0, qq = 0.0;
    for (int i = 0; i < d; i++) {
        double x = xrow[i], q = qs[i];
        if (metric == 0) {
            double t = x - q;
            s = fma(t, t, s);
        } else {
            s = fma(x, q, s);
            xx = fma(x, x, xx);
            qq = fma(q, q, qq);
        }
    }
    if (metric == 0) return sqrt(s);
    if (xx == 0.0 || qq == 0.0) return 1.0;
    return 1.0 - s / (sqrt(xx) * sqrt(qq));
}

// in-range test of one (x, q) pair; FP64 when the FP32 key is within its
// rounding bound of eps
__device__ __forceinline__ bool na_in(const float* xrow, const float* qs, int d, int metric, float qn2,
                                      float eps_key, float band, double eps64, float* key_out) {
    float k = na_key(xrow, qs, d, metric, qn2);
    *key_out = k;
    float scale = metric == 0 ? eps_key : 1.f;
    if (fabsf(k - eps_key) <= band * scale) return na_dist64(xrow, qs, d, metric) < eps64;
    return k < eps_key;
}

// pass 1 (write == false): per-query match counts into counts[];
// pass 2 (write == true): pairs at offsets[q] in ascending data id, up to cap
template <bool WRITE>
__global__ void __launch_bounds__(NA_WARPS * 32)
    k_na_scan(const float* __restrict__ X, int64_t nx, const float* __restrict__ Q, int64_t nq, int d, int metric,
              float eps_key, float band, double eps64, int32_t* __restrict__ counts,
              const int64_t* __restrict__ offsets, int32_t* __restrict__ ids, float* __restrict__ dists,
              int64_t cap) {
    extern __shared__ float na_q[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t q = (int64_t)blockIdx.x * NA_WARPS + warp;
    float* qs = na_q + (size_t)warp * d;
    if (q < nq)
        for (int i = lane; i < d; i += 32) qs[i] = Q[q * d + i];
    __syncwarp();
    if (q >= nq) return;
    float qn2 = 0.f;
    if (metric == 1)
        for (int i = 0; i < d; i++) qn2 = fmaf(qs[i], qs[i], qn2);
    int64_t pos = WRITE ? offsets[q] : 0;
    int32_t c = 0;
    for (int64_t x0 = 0; x0 < nx; x0 += 32) {
        const int64_t x = x0 + lane;
        float k = 0.f;
        bool in = x < nx && na_in(X + x * d, qs, d, metric, qn2, eps_key, band, eps64, &k);
        unsigned m = __ballot_sync(VJ_FULL, in);
        if (WRITE && in) {
            int64_t p = pos + c + __popc(m & ((1u << lane) - 1u));
            if (p < cap) {
                ids[p] = (int32_t)x;
                dists[p] = metric == 0 ? sqrtf(fmaxf(k, 0.f)) : k;
            }
        }
        c += __popc(m);
    }
    if (!WRITE && lane == 0) counts[q] = c;
}

// single block: offsets[0..n] = exclusive scan of counts[0..n)
__global__ void __launch_bounds__(1024) k_na_offsets(const int32_t* __restrict__ counts, int64_t n,
                                                     int64_t* __restrict__ offsets) {
    __shared__ int64_t wsum[32];
    __shared__ int64_t carry;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t b = 0; b < n; b += 1024) {
        int64_t i = b + threadIdx.x;
        int64_t v = i < n ? counts[i] : 0;
        int64_t incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            int64_t t = __shfl_up_sync(VJ_FULL, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) wsum[w] = incl;
        __syncthreads();
        if (w == 0) {
            int64_t t = wsum[lane];
            for (int o = 1; o < 32; o <<= 1) {
                int64_t u = __shfl_up_sync(VJ_FULL, t, o);
                if (lane >= o) t += u;
            }
            wsum[lane] = t;
        }
        __syncthreads();
        int64_t base = carry + (w > 0 ? wsum[w - 1] : 0);
        if (i < n) offsets[i] = base + incl - v;
        __syncthreads();
        if (threadIdx.x == 0) carry += wsum[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) offsets[n] = carry;
}

std::mutex g_na_mu;
void* g_na_ptr[64] = {};  // per-device device address of g_na_scratch

}  // namespace

extern "C" vj_status vj_join_exact_noalloc(const float* X, int64_t nx, const float* Q, int64_t nq, int d,
                                           vj_metric metric, float eps, int64_t* offsets, int32_t* ids,
                                           float* dists, int64_t cap, int64_t* nnz, void* stream) {
    try {
        VJ_REQUIRE(X && Q && offsets && nnz && (cap == 0 || (ids && dists)), VJ_ERR_ARG, "NULL argument");
        VJ_REQUIRE(nx >= 1 && nq >= 1 && nx < (int64_t)INT32_MAX, VJ_ERR_ARG, "nx, nq must be >= 1 (nx < 2^31)");
        VJ_REQUIRE(nq <= VJ_NOALLOC_MAX_QUERIES, VJ_ERR_ARG,
                   "vj_join_exact_noalloc: nq = %lld exceeds the fixed scratch limit of %d queries",
                   (long long)nq, VJ_NOALLOC_MAX_QUERIES);
        VJ_REQUIRE(d >= 1 && d <= NA_MAXD_SMEM, VJ_ERR_ARG, "d must be in [1, %d]", NA_MAXD_SMEM);
        VJ_REQUIRE(metric == VJ_L2 || metric == VJ_COSINE, VJ_ERR_ARG, "unknown metric");
        VJ_REQUIRE(eps > 0.f && eps == eps, VJ_ERR_ARG, "eps must be > 0");
        VJ_REQUIRE(cap >= 0, VJ_ERR_ARG, "cap must be >= 0");
        int dev = 0;
        VJ_CUDA(cudaGetDevice(&dev));
        VJ_REQUIRE(dev >= 0 && dev < 64, VJ_ERR_ARG, "device ordinal above 63");
        void* scratch = nullptr;
        {
            std::lock_guard<std::mutex> lk(g_na_mu);
            if (!g_na_ptr[dev]) {
                void* p = nullptr;
                VJ_CUDA(cudaGetSymbolAddress(&p, g_na_scratch));
                g_na_ptr[dev] = p;
            }
            scratch = g_na_ptr[dev];
        }
        cudaStream_t s = (cudaStream_t)stream;
        int32_t* counts = reinterpret_cast<int32_t*>(scratch);
        const float eps_key = metric == VJ_L2 ? eps * eps : eps;
        const float band = 2.0f * (float)(d + 4) * VJ_F32_U * (metric == VJ_L2 ? 1.0f : 4.0f) + 1e-6f;
        const size_t smem = (size_t)NA_WARPS * d * sizeof(float);
        if (smem > 48 * 1024) {
            VJ_CUDA(cudaFuncSetAttribute(k_na_scan<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            VJ_CUDA(cudaFuncSetAttribute(k_na_scan<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        }
        const int blocks = vj_div_up(nq, NA_WARPS);
        k_na_scan<false><<<blocks, NA_WARPS * 32, smem, s>>>(X, nx, Q, nq, d, metric, eps_key, band, (double)eps,
                                                             counts, nullptr, nullptr, nullptr, 0);
        VJ_LAUNCH_CHECK();
        k_na_offsets<<<1, 1024, 0, s>>>(counts, nq, offsets);
        VJ_LAUNCH_CHECK();
        k_na_scan<true><<<blocks, NA_WARPS * 32, smem, s>>>(X, nx, Q, nq, d, metric, eps_key, band, (double)eps,
                                                            counts, offsets, ids, dists, cap);
        VJ_LAUNCH_CHECK();
        VJ_CUDA(cudaMemcpyAsync(nnz, offsets + nq, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        VJ_CUDA(cudaStreamSynchronize(s));
        VJ_REQUIRE(*nnz <= cap, VJ_ERR_STATE,
                   "vj_join_exact_noalloc: %lld pairs exceed cap = %lld (offsets hold the full CSR; pairs "
                   "beyond cap were not written)",
                   (long long)*nnz, (long long)cap);
        return VJ_OK;
    } catch (const VjError& e) {
        return e.code;
    }
}
