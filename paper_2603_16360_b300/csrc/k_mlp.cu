// k_mlp.cu -- the learned route / budget predictor: a 3-layer MLP
// (din -> h1 -> h2 -> 2, ReLU) trained on the GPU with hand-written forward,
// backward and Adam kernels.  Output 0 regresses log2(budget + 1) (squared
// error), output 1 is the route logit (binary cross-entropy with logits).
// The paper has only the d1/d2 rule (Sec. 4.4); the predictor is this
// library's addition, and that rule stays the default (learned = 0).
//
// Parameters are one flat FP32 array:
//   W1[h1][din] b1[h1] W2[h2][h1] b2[h2] W3[2][h2] b3[2]
// Inputs are standardised per feature with the mean / std of the training
// inputs before the first layer (kept with the weights).
#include <float.h>

#include <functional>

#include <mutex>
#include <numeric>
#include <random>

#include "vj_device.cuh"
#include "vj_internal.cuh"
#include "vj_tc.cuh"

struct vj_mlp {
    int din = 0, h1 = 0, h2 = 0;
    int64_t np = 0;
    DBuf<float> w, m, v, g;  // params, Adam moments, gradient
    DBuf<float> mu, sd;      // input standardisation
    bool has_norm = false;
    int64_t step = 0;
    cudaStream_t stream = nullptr;
    // activation scratch for a batch
    DBuf<float> xb, z1, a1, z2, a2, y, dy, da2, da1;
    DBuf<float> tr, tc;
    DBuf<double> loss;
    int64_t cap = 0;
    // BF16 operands of the tensor-core inference path
    DBuf<__nv_bfloat16> xbf, w1bf, w2bf;
    DBuf<int> err;
    // Serialises inference when one predictor serves indexes joined on
    // concurrent host threads (the scratch above is per predictor).
    std::mutex fwd_mu;
};

namespace {

struct Off {
    int64_t w1, b1, w2, b2, w3, b3, total;
};
Off offsets(const vj_mlp* m) {
    Off o;
    o.w1 = 0;
    o.b1 = o.w1 + (int64_t)m->h1 * m->din;
    o.w2 = o.b1 + m->h1;
    o.b2 = o.w2 + (int64_t)m->h2 * m->h1;
    o.w3 = o.b2 + m->h2;
    o.b3 = o.w3 + 2 * (int64_t)m->h2;
    o.total = o.b3 + 2;
    return o;
}

// C[i][j] (+)= sum_p A(i,p) B(p,j) with arbitrary strides (element units);
// epilogue: + bias[j], then optional ReLU into R (pre-activation kept in C)
constexpr int GT = 64, GK = 16;
__global__ void __launch_bounds__(256) k_gemm(int M, int N, int K, const float* __restrict__ A, int64_t sai,
                                              int64_t sap, const float* __restrict__ B, int64_t sbp, int64_t sbj,
                                              float* __restrict__ Cm, int64_t sci, const float* __restrict__ bias,
                                              float* __restrict__ R, int accumulate) {
    __shared__ float As[GK][GT + 1];
    __shared__ float Bs[GK][GT + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int i0 = blockIdx.y * GT, j0 = blockIdx.x * GT;
    float acc[4][4] = {};
    for (int p0 = 0; p0 < K; p0 += GK) {
        for (int e = threadIdx.x; e < GT * GK; e += 256) {
            const int r = e / GK, p = e % GK;
            const int gi = i0 + r, gp = p0 + p;
            As[p][r] = (gi < M && gp < K) ? A[(int64_t)gi * sai + (int64_t)gp * sap] : 0.f;
            const int gj = j0 + r;
            Bs[p][r] = (gj < N && gp < K) ? B[(int64_t)gp * sbp + (int64_t)gj * sbj] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int p = 0; p < GK; p++) {
            float a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                a[u] = As[p][ty * 4 + u];
                b[u] = Bs[p][tx * 4 + u];
            }
#pragma unroll
            for (int u = 0; u < 4; u++)
#pragma unroll
                for (int v = 0; v < 4; v++) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; u++) {
        const int gi = i0 + ty * 4 + u;
        if (gi >= M) continue;
#pragma unroll
        for (int v = 0; v < 4; v++) {
            const int gj = j0 + tx * 4 + v;
            if (gj >= N) continue;
            float c = acc[u][v] + (bias ? bias[gj] : 0.f);
            if (accumulate) c += Cm[(int64_t)gi * sci + gj];
            Cm[(int64_t)gi * sci + gj] = c;
            if (R) R[(int64_t)gi * sci + gj] = fmaxf(c, 0.f);
        }
    }
}

void gemm(cudaStream_t s, int M, int N, int K, const float* A, int64_t sai, int64_t sap, const float* B, int64_t sbp,
          int64_t sbj, float* C, int64_t sci, const float* bias, float* R, bool acc = false) {
    dim3 grid(vj_div_up(N, GT), vj_div_up(M, GT));
    k_gemm<<<grid, 256, 0, s>>>(M, N, K, A, sai, sap, B, sbp, sbj, C, sci, bias, R, acc ? 1 : 0);
    VJ_LAUNCH_CHECK();
}

// standardise x (n x din) with mu / sd into xb
__global__ void k_standardise(const float* __restrict__ x, int64_t n, int din, const float* __restrict__ mu,
                              const float* __restrict__ sd, float* __restrict__ xb) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * din) return;
    const int f = (int)(i % din);
    xb[i] = mu ? (x[i] - mu[f]) / sd[f] : x[i];
}

// loss and output gradient: out 0 squared error, out 1 BCE with logits; mean over n
__global__ void k_out_grad(const float* __restrict__ y, const float* __restrict__ tr, const float* __restrict__ tc,
                           int64_t n, float* __restrict__ dy, double* __restrict__ loss) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    if (i < n) {
        const float e = y[2 * i] - tr[i];
        const float z = y[2 * i + 1], t = tc[i];
        const float sig = 1.f / (1.f + expf(-z));
        dy[2 * i] = 2.f * e / (float)n;
        dy[2 * i + 1] = (sig - t) / (float)n;
        // softplus(z) - t z, computed stably
        const float sp = fmaxf(z, 0.f) + log1pf(expf(-fabsf(z)));
        l = ((double)e * e + (double)(sp - t * z)) / (double)n;
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(VJ_FULL, l, o);
    if ((threadIdx.x & 31) == 0 && l != 0.0) atomicAdd(loss, l);
}

// dA *= (Z > 0)
__global__ void k_relu_back(float* __restrict__ da, const float* __restrict__ z, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && !(z[i] > 0.f)) da[i] = 0.f;
}

// column sums of D (n x m) into g (bias gradient)
__global__ void k_colsum(const float* __restrict__ D, int64_t n, int m, float* __restrict__ g) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    float s = 0.f;
    for (int64_t i = 0; i < n; i++) s += D[i * m + j];
    g[j] = s;
}

__global__ void k_adam(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, int64_t n, float lr, float b1, float b2, float eps, float c1,
                       float c2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

void ensure_batch(vj_mlp* m, int64_t n) {
    if (n <= m->cap) return;
    cudaStream_t s = m->stream;
    m->xb.ensure((size_t)n * m->din, s);
    m->z1.ensure((size_t)n * m->h1, s);
    m->a1.ensure((size_t)n * m->h1, s);
    m->z2.ensure((size_t)n * m->h2, s);
    m->a2.ensure((size_t)n * m->h2, s);
    m->y.ensure((size_t)n * 2, s);
    m->dy.ensure((size_t)n * 2, s);
    m->da2.ensure((size_t)n * m->h2, s);
    m->da1.ensure((size_t)n * m->h1, s);
    m->tr.ensure(n, s);
    m->tc.ensure(n, s);
    m->cap = n;
}

// forward of n rows already in device memory (x: n x din); standardise when asked
void forward(vj_mlp* m, const float* x, int64_t n, bool standardise) {
    cudaStream_t s = m->stream;
    const Off o = offsets(m);
    ensure_batch(m, n);
    k_standardise<<<vj_div_up(n * m->din, 256), 256, 0, s>>>(x, n, m->din, standardise && m->has_norm ? m->mu.p : nullptr,
                                                             m->sd.p, m->xb.p);
    VJ_LAUNCH_CHECK();
    const float* W = m->w.p;
    // Z1 = X W1^T + b1: A = xb (i: din, p: 1), B(p, j) = W1[j][p] (p: 1, j: din)
    gemm(s, (int)n, m->h1, m->din, m->xb.p, m->din, 1, W + o.w1, 1, m->din, m->z1.p, m->h1, W + o.b1, m->a1.p);
    gemm(s, (int)n, m->h2, m->h1, m->a1.p, m->h1, 1, W + o.w2, 1, m->h1, m->z2.p, m->h2, W + o.b2, m->a2.p);
    gemm(s, (int)n, 2, m->h2, m->a2.p, m->h2, 1, W + o.w3, 1, m->h2, m->y.p, 2, W + o.b3, nullptr);
}

// gradient of the mean loss over n rows into m->g; loss value added to *loss
void backward(vj_mlp* m, int64_t n) {
    cudaStream_t s = m->stream;
    const Off o = offsets(m);
    const float* W = m->w.p;
    float* G = m->g.p;
    k_out_grad<<<vj_div_up(n, 256), 256, 0, s>>>(m->y.p, m->tr.p, m->tc.p, n, m->dy.p, m->loss.p);
    VJ_LAUNCH_CHECK();
    // dW3[c][j] = sum_i dy[i][c] a2[i][j];  db3 = colsum(dy)
    gemm(s, 2, m->h2, (int)n, m->dy.p, 1, 2, m->a2.p, m->h2, 1, G + o.w3, m->h2, nullptr, nullptr);
    k_colsum<<<1, 32, 0, s>>>(m->dy.p, n, 2, G + o.b3);
    VJ_LAUNCH_CHECK();
    // dA2 = dY W3 ; dZ2 = dA2 * (Z2 > 0)
    gemm(s, (int)n, m->h2, 2, m->dy.p, 2, 1, W + o.w3, m->h2, 1, m->da2.p, m->h2, nullptr, nullptr);
    k_relu_back<<<vj_div_up(n * m->h2, 256), 256, 0, s>>>(m->da2.p, m->z2.p, n * m->h2);
    VJ_LAUNCH_CHECK();
    gemm(s, m->h2, m->h1, (int)n, m->da2.p, 1, m->h2, m->a1.p, m->h1, 1, G + o.w2, m->h1, nullptr, nullptr);
    k_colsum<<<vj_div_up(m->h2, 128), 128, 0, s>>>(m->da2.p, n, m->h2, G + o.b2);
    VJ_LAUNCH_CHECK();
    gemm(s, (int)n, m->h1, m->h2, m->da2.p, m->h2, 1, W + o.w2, m->h1, 1, m->da1.p, m->h1, nullptr, nullptr);
    k_relu_back<<<vj_div_up(n * m->h1, 256), 256, 0, s>>>(m->da1.p, m->z1.p, n * m->h1);
    VJ_LAUNCH_CHECK();
    gemm(s, m->h1, m->din, (int)n, m->da1.p, 1, m->h1, m->xb.p, m->din, 1, G + o.w1, m->din, nullptr, nullptr);
    k_colsum<<<vj_div_up(m->h1, 128), 128, 0, s>>>(m->da1.p, n, m->h1, G + o.b1);
    VJ_LAUNCH_CHECK();
}

// He-uniform initialisation from a seeded host generator
void init_params(vj_mlp* m, uint64_t seed) {
    const Off o = offsets(m);
    std::vector<float> h((size_t)o.total, 0.f);
    std::mt19937_64 rng(seed);
    auto fill = [&](int64_t off, int rows, int cols) {
        const float a = sqrtf(6.f / (float)cols);
        std::uniform_real_distribution<float> U(-a, a);
        for (int64_t i = 0; i < (int64_t)rows * cols; i++) h[off + i] = U(rng);
    };
    fill(o.w1, m->h1, m->din);
    fill(o.w2, m->h2, m->h1);
    fill(o.w3, 2, m->h2);
    VJ_CUDA(cudaMemcpyAsync(m->w.p, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice, m->stream));
    VJ_CUDA(cudaMemsetAsync(m->m.p, 0, h.size() * sizeof(float), m->stream));
    VJ_CUDA(cudaMemsetAsync(m->v.p, 0, h.size() * sizeof(float), m->stream));
    VJ_CUDA(cudaStreamSynchronize(m->stream));
}


// ---------------------------------------------------------------- tensor-core inference
// Fused forward of 128 rows per CTA on the 5th-generation tensor cores:
//   D1 = X W1^T           (TMEM columns 0..h1)     X, W1 streamed by TMA
//   A2 = relu(D1 + b1)    BF16 into shared memory (128-byte swizzled K-major)
//   D2 = A2 W2^T          (TMEM columns 256..)     W2 streamed by TMA
//   y  = W3 relu(D2 + b2) + b3                     FP32 in the epilogue
// Warp 0 issues TMA, warp 1 allocates TMEM and issues tcgen05.mma, warps 2..5
// (one per TMEM lane quarter, one row per thread) run both epilogues.  Inputs
// are the standardised features and weights rounded to BF16 (FP32 accumulate).
using namespace vjtc;

constexpr int ML_EPI = 4;
constexpr int ML_THREADS = (2 + ML_EPI) * 32;
constexpr int ML_STAGES = 3;
constexpr uint32_t ML_ABOX = 128 * 64 * 2;   // 128 rows x 64 BF16
constexpr uint32_t ML_WBOX = 256 * 64 * 2;   // up to 256 rows x 64 BF16
constexpr uint32_t ML_STAGE = ML_ABOX + ML_WBOX;

struct MlBars {
    uint64_t full[ML_STAGES];
    uint64_t empty[ML_STAGES];
    uint64_t d1full, a2full, d2full, drain;
    uint32_t tmem_base;
    int abort;
};

struct MlParams {
    int64_t n;
    int nk1;     // layer-1 k-blocks of 64
    int h1, h2;  // h1: multiple of 64 up to 256; h2: multiple of 16 up to 256
    const float* b1;
    const float* b2;
    const float* w3;
    const float* b3;
    float* y;
    int* err;
    long long spin_limit;
};

__host__ __device__ constexpr uint32_t ml_idesc(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__global__ void __launch_bounds__(ML_THREADS, 1)
    k_mlp_fwd_tc(const __grid_constant__ CUtensorMap tX, const __grid_constant__ CUtensorMap tW1,
                 const __grid_constant__ CUtensorMap tW2, MlParams P) {
    extern __shared__ uint8_t ml_raw[];
    uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(ml_raw) + 1023) & ~uintptr_t(1023));
    MlBars& B = *reinterpret_cast<MlBars*>(base);
    uint8_t* ring = base + 1024;
    uint8_t* sA2 = ring + ML_STAGES * ML_STAGE;            // [h1 / 64] boxes of 128 x 64
    float* sb1 = reinterpret_cast<float*>(sA2 + (P.h1 / 64) * ML_ABOX);
    float* sb2 = sb1 + 256;
    float* sw3 = sb2 + 256;                                // [2][256]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    volatile int* abort = &B.abort;
    const int64_t row0 = (int64_t)blockIdx.x * 128;
    const int nk2 = P.h1 / 64;

    if (threadIdx.x == 0) {
        for (int s = 0; s < ML_STAGES; s++) {
            mbar_init(&B.full[s], 1);
            mbar_init(&B.empty[s], 1);
        }
        mbar_init(&B.d1full, 1);
        mbar_init(&B.a2full, 1);
        mbar_init(&B.d2full, 1);
        mbar_init(&B.drain, 1);
        B.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&B.tmem_base)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = B.tmem_base;

    if (warp == 0) {
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0, issued = 0, last_ph = 0;
            bool ok = true;
            const uint32_t w1b = (uint32_t)P.h1 * 128u, w2b = (uint32_t)P.h2 * 128u;
            for (int kb = 0; kb < P.nk1 + nk2 && ok; kb++) {
                if (!mbar_wait(&B.empty[s], ph ^ 1u, abort, P.spin_limit)) {
                    ok = false;
                    break;
                }
                uint8_t* st = ring + s * ML_STAGE;
                if (kb < P.nk1) {
                    mbar_arrive_tx(&B.full[s], ML_ABOX + w1b);
                    tma_load_2d(st, &tX, &B.full[s], kb * 64, (int)row0);
                    tma_load_2d(st + ML_ABOX, &tW1, &B.full[s], kb * 64, 0);
                } else {
                    mbar_arrive_tx(&B.full[s], w2b);
                    tma_load_2d(st + ML_ABOX, &tW2, &B.full[s], (kb - P.nk1) * 64, 0);
                }
                issued |= 1u << s;
                last_ph = (last_ph & ~(1u << s)) | (ph << s);
                if (++s == ML_STAGES) {
                    s = 0;
                    ph ^= 1u;
                }
            }
            if (!ok) {
                *abort = 1;
                atomicExch(P.err, 1);
                for (int st = 0; st < ML_STAGES; st++)
                    if ((issued >> st) & 1u)
                        for (long long i = 0; i < P.spin_limit && !mbar_test(&B.full[st], (last_ph >> st) & 1u); i++) {
                        }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0;
            bool ok = true;
            for (int kb = 0; kb < P.nk1 + nk2 && ok; kb++) {
                if (kb == P.nk1) {
                    // layer 2 reads A2, written by the epilogue warps
                    tc_commit(&B.d1full);
                    if (!mbar_wait(&B.a2full, 0, abort, P.spin_limit)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                }
                if (!mbar_wait(&B.full[s], ph, abort, P.spin_limit)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                uint8_t* st = ring + s * ML_STAGE;
                const bool l1 = kb < P.nk1;
                const uint64_t ad = sdesc_sw128(su32(l1 ? st : sA2 + (kb - P.nk1) * ML_ABOX));
                const uint64_t bd = sdesc_sw128(su32(st + ML_ABOX));
                const uint32_t d = tmem + (l1 ? 0u : 256u);
                const uint32_t idesc = l1 ? ml_idesc(P.h1) : ml_idesc(P.h2);
                const int k0 = l1 ? kb : kb - P.nk1;
#pragma unroll
                for (int kk = 0; kk < 4; kk++)
                    tc_mma(d, ad + (uint64_t)(kk * 2), bd + (uint64_t)(kk * 2), idesc, (uint32_t)((k0 | kk) != 0));
                tc_commit(&B.empty[s]);
                if (++s == ML_STAGES) {
                    s = 0;
                    ph ^= 1u;
                }
            }
            if (ok) tc_commit(&B.d2full);
            else {
                *abort = 1;
                atomicExch(P.err, 1);
            }
            tc_commit(&B.drain);
            for (long long k = 0; k < P.spin_limit && !mbar_test(&B.drain, 0); k++) {
            }
        }
    } else {
        const int et = threadIdx.x - 64;  // 0..127
        for (int i = et; i < 256; i += 128) {
            sb1[i] = i < P.h1 ? P.b1[i] : 0.f;
            sb2[i] = i < P.h2 ? P.b2[i] : 0.f;
            sw3[i] = i < P.h2 ? P.w3[i] : 0.f;
            sw3[256 + i] = i < P.h2 ? P.w3[P.h2 + i] : 0.f;
        }
        asm volatile("bar.sync 1, %0;" ::"r"(ML_EPI * 32) : "memory");
        const int quarter = warp & 3;
        const int r = quarter * 32 + lane;  // row within the tile = TMEM lane
        const uint32_t lanes = (uint32_t)(quarter * 32) << 16;
        bool ok = mbar_wait(&B.d1full, 0, abort, P.spin_limit);
        if (__all_sync(VJ_FULL, ok)) {
            tc_fence_after();
            // ---- epilogue 1: A2 = relu(D1 + b1) as BF16, 128-byte swizzled K-major
            for (int c0 = 0; c0 < P.h1; c0 += 32) {
                uint32_t v[32];
                tmem_ld32_issue(tmem + lanes + (uint32_t)c0, v);
                tmem_wait_ld(v);
                uint32_t pk[16];
#pragma unroll
                for (int j = 0; j < 16; j++) {
                    const float a = fmaxf(__uint_as_float(v[2 * j]) + sb1[c0 + 2 * j], 0.f);
                    const float b = fmaxf(__uint_as_float(v[2 * j + 1]) + sb1[c0 + 2 * j + 1], 0.f);
                    const __nv_bfloat162 h2v = __floats2bfloat162_rn(a, b);
                    pk[j] = *reinterpret_cast<const uint32_t*>(&h2v);
                }
                uint8_t* line = sA2 + (c0 / 64) * ML_ABOX + r * 128;
                const int chunk0 = ((c0 % 64) * 2) / 16;
#pragma unroll
                for (int t = 0; t < 4; t++) {
                    const int phys = (chunk0 + t) ^ (r & 7);
                    *reinterpret_cast<uint4*>(line + phys * 16) =
                        make_uint4(pk[4 * t], pk[4 * t + 1], pk[4 * t + 2], pk[4 * t + 3]);
                }
            }
            // generic-proxy stores -> visible to the tensor core's async proxy
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            tc_fence_before();
            asm volatile("bar.sync 1, %0;" ::"r"(ML_EPI * 32) : "memory");
            if (threadIdx.x == 64) mbar_arrive(&B.a2full);
            // ---- epilogue 2: y = W3 relu(D2 + b2) + b3
            ok = mbar_wait(&B.d2full, 0, abort, P.spin_limit);
            if (__all_sync(VJ_FULL, ok)) {
                tc_fence_after();
                float y0 = P.b3[0], y1 = P.b3[1];
                for (int c0 = 0; c0 < P.h2; c0 += 16) {
                    // 16 columns per step: reads stay inside D2's h2 columns
                    uint32_t v[16];
                    tmem_ld16_issue(tmem + lanes + 256u + (uint32_t)c0, v);
                    tmem_wait_ld16(v);
#pragma unroll
                    for (int j = 0; j < 16; j++) {
                        const float a = fmaxf(__uint_as_float(v[j]) + sb2[c0 + j], 0.f);
                        y0 = fmaf(a, sw3[c0 + j], y0);
                        y1 = fmaf(a, sw3[256 + c0 + j], y1);
                    }
                }
                const int64_t gr = row0 + r;
                if (gr < P.n) {
                    P.y[2 * gr] = y0;
                    P.y[2 * gr + 1] = y1;
                }
            } else if (lane == 0) {
                *abort = 1;
                atomicExch(P.err, 1);
            }
        } else if (lane == 0) {
            *abort = 1;
            atomicExch(P.err, 1);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
    }
}

// standardised features -> BF16 rows of k1 columns (zero padded)
__global__ void k_feat_bf16(const float* __restrict__ x, int64_t n, int din, int k1, const float* __restrict__ mu,
                            const float* __restrict__ sd, __nv_bfloat16* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * k1) return;
    const int64_t r = i / k1;
    const int f = (int)(i % k1);
    float v = 0.f;
    if (f < din) {
        v = x[r * din + f];
        if (mu) v = (v - mu[f]) / sd[f];
    }
    out[i] = __float2bfloat16_rn(v);
}

// rows x cols FP32 -> rows x kp BF16 (zero padded)
__global__ void k_mat_bf16(const float* __restrict__ w, int rows, int cols, int kp, __nv_bfloat16* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)rows * kp) return;
    const int r = (int)(i / kp), c = (int)(i % kp);
    out[i] = __float2bfloat16_rn(c < cols ? w[(int64_t)r * cols + c] : 0.f);
}

bool tc_shape_ok(const vj_mlp* m) {
    return m->h1 % 64 == 0 && m->h1 >= 64 && m->h1 <= 256 && m->h2 % 16 == 0 && m->h2 >= 16 && m->h2 <= 256;
}

// tensor-core forward of the n BF16 input rows in m->xbf (standardised, k1
// columns)
void forward_tc_rows(vj_mlp* m, int64_t n, float* y, cudaStream_t s) {
    const Off o = offsets(m);
    const int k1 = (m->din + 63) / 64 * 64;
    m->w1bf.ensure((size_t)m->h1 * k1, s);
    m->w2bf.ensure((size_t)m->h2 * m->h1, s);
    m->err.ensure(1, s);
    k_mat_bf16<<<vj_div_up((int64_t)m->h1 * k1, 256), 256, 0, s>>>(m->w.p + o.w1, m->h1, m->din, k1, m->w1bf.p);
    VJ_LAUNCH_CHECK();
    k_mat_bf16<<<vj_div_up((int64_t)m->h2 * m->h1, 256), 256, 0, s>>>(m->w.p + o.w2, m->h2, m->h1, m->h1, m->w2bf.p);
    VJ_LAUNCH_CHECK();
    const CUtensorMap tX = make_map(m->xbf.p, n, k1, 128);
    const CUtensorMap tW1 = make_map(m->w1bf.p, m->h1, k1, m->h1);
    const CUtensorMap tW2 = make_map(m->w2bf.p, m->h2, m->h1, m->h2);
    MlParams P;
    P.n = n;
    P.nk1 = k1 / 64;
    P.h1 = m->h1;
    P.h2 = m->h2;
    P.b1 = m->w.p + o.b1;
    P.b2 = m->w.p + o.b2;
    P.w3 = m->w.p + o.w3;
    P.b3 = m->w.p + o.b3;
    P.y = y;
    P.err = m->err.p;
    P.spin_limit = 1ll << 22;
    const size_t smem = 2048 + (size_t)ML_STAGES * ML_STAGE + (size_t)(m->h1 / 64) * ML_ABOX + 4 * 256 * sizeof(float);
    VJ_CUDA(cudaFuncSetAttribute(k_mlp_fwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    VJ_CUDA(cudaMemsetAsync(m->err.p, 0, sizeof(int), s));
    k_mlp_fwd_tc<<<(unsigned)vj_div_up(n, 128), ML_THREADS, smem, s>>>(tX, tW1, tW2, P);
    VJ_LAUNCH_CHECK();
    int herr = 0;
    VJ_CUDA(cudaMemcpyAsync(&herr, m->err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    VJ_CUDA(cudaStreamSynchronize(s));
    VJ_REQUIRE(herr == 0, VJ_ERR_TIMEOUT, "predictor forward: a pipeline wait timed out");
}

// tensor-core forward of n standardised-on-the-fly rows (x: n x din FP32)
void forward_tc(vj_mlp* m, const float* x, int64_t n, float* y, cudaStream_t s) {
    const int k1 = (m->din + 63) / 64 * 64;
    m->xbf.ensure((size_t)std::max<int64_t>(n, 1) * k1, s);
    k_feat_bf16<<<vj_div_up(n * k1, 256), 256, 0, s>>>(x, n, m->din, k1, m->has_norm ? m->mu.p : nullptr, m->sd.p,
                                                       m->xbf.p);
    VJ_LAUNCH_CHECK();
    forward_tc_rows(m, n, y, s);
}

}  // namespace

// ------------------------------------------------------------------ internal API
// the join prologue's forward: BF16 tensor cores when the widths allow
// (h1 multiple of 64, h2 multiple of 16, both <= 256), else FP32
void vj_mlp_forward_device(vj_mlp* m, const float* x, int64_t n, float* y_out, cudaStream_t s) {
    if (n <= 0) return;
    std::lock_guard<std::mutex> lk(m->fwd_mu);
    if (tc_shape_ok(m)) {
        forward_tc(m, x, n, y_out, s);  // ends with a stream synchronize
        return;
    }
    cudaStream_t keep = m->stream;
    m->stream = s;
    forward(m, x, n, true);
    VJ_CUDA(cudaMemcpyAsync(y_out, m->y.p, (size_t)n * 2 * sizeof(float), cudaMemcpyDeviceToDevice, s));
    m->stream = keep;
    VJ_CUDA(cudaStreamSynchronize(s));  // the scratch is free for the next caller
}
int vj_mlp_din(const vj_mlp* m) { return m->din; }

// the tensor-core forward with its BF16 input rows written by `fill` (the
// predictor's buffer, k1 columns, and the standardisation to apply: mu and
// sd, or nullptr); false when the shape has no tensor-core path
bool vj_mlp_forward_filled(vj_mlp* m, int64_t n, float* y_out, cudaStream_t s,
                           const std::function<void(__nv_bfloat16*, int, const float*, const float*)>& fill) {
    if (n <= 0) return true;
    if (!tc_shape_ok(m)) return false;
    std::lock_guard<std::mutex> lk(m->fwd_mu);
    const int k1 = (m->din + 63) / 64 * 64;
    m->xbf.ensure((size_t)n * k1, s);
    fill(m->xbf.p, k1, m->has_norm ? m->mu.p : nullptr, m->sd.p);
    forward_tc_rows(m, n, y_out, s);  // ends with a stream synchronize
    return true;
}

// ------------------------------------------------------------------ C ABI
template <class F>
static vj_status mlp_guard(F&& f) {
    try {
        f();
        return VJ_OK;
    } catch (const VjError& e) {
        return e.code;
    } catch (...) {
        vj_set_error("unexpected internal error");
        return VJ_ERR_STATE;
    }
}

extern "C" vj_status vj_mlp_create(int din, int h1, int h2, uint64_t seed, vj_mlp** out) {
    if (out) *out = nullptr;
    vj_mlp* m = nullptr;
    vj_status st = mlp_guard([&] {
        VJ_REQUIRE(out && din >= 1 && h1 >= 1 && h2 >= 1 && din <= 8192 && h1 <= 8192 && h2 <= 8192, VJ_ERR_ARG,
                   "bad MLP shape");
        m = new vj_mlp();
        m->din = din;
        m->h1 = h1;
        m->h2 = h2;
        VJ_CUDA(cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking));
        m->np = offsets(m).total;
        m->w.alloc(m->np, m->stream);
        m->m.alloc(m->np, m->stream);
        m->v.alloc(m->np, m->stream);
        m->g.alloc(m->np, m->stream);
        m->loss.alloc(1, m->stream);
        m->mu.alloc(din, m->stream);
        m->sd.alloc(din, m->stream);
        init_params(m, seed);
        *out = m;
    });
    if (st != VJ_OK && m) {
        cudaStreamDestroy(m->stream);
        delete m;
    }
    return st;
}

extern "C" int64_t vj_mlp_num_params(const vj_mlp* m) { return m ? m->np : 0; }

extern "C" vj_status vj_mlp_get_params(const vj_mlp* m, float* flat, float* mu, float* sd) {
    return mlp_guard([&] {
        VJ_REQUIRE(m != nullptr, VJ_ERR_ARG, "NULL predictor");
        if (flat) VJ_CUDA(cudaMemcpyAsync(flat, m->w.p, m->np * sizeof(float), cudaMemcpyDeviceToHost, m->stream));
        if (mu) VJ_CUDA(cudaMemcpyAsync(mu, m->mu.p, m->din * sizeof(float), cudaMemcpyDeviceToHost, m->stream));
        if (sd) VJ_CUDA(cudaMemcpyAsync(sd, m->sd.p, m->din * sizeof(float), cudaMemcpyDeviceToHost, m->stream));
        VJ_CUDA(cudaStreamSynchronize(m->stream));
    });
}

extern "C" vj_status vj_mlp_set_params(vj_mlp* m, const float* flat, const float* mu, const float* sd) {
    return mlp_guard([&] {
        VJ_REQUIRE(m != nullptr && flat != nullptr, VJ_ERR_ARG, "NULL argument");
        VJ_CUDA(cudaMemcpyAsync(m->w.p, flat, m->np * sizeof(float), cudaMemcpyHostToDevice, m->stream));
        if (mu && sd) {
            VJ_CUDA(cudaMemcpyAsync(m->mu.p, mu, m->din * sizeof(float), cudaMemcpyHostToDevice, m->stream));
            VJ_CUDA(cudaMemcpyAsync(m->sd.p, sd, m->din * sizeof(float), cudaMemcpyHostToDevice, m->stream));
            m->has_norm = true;
        } else {
            m->has_norm = false;
        }
        VJ_CUDA(cudaStreamSynchronize(m->stream));
    });
}

// loss and gradient (flat, host) of the mean loss over n host rows; no
// standardisation (the rows are used as given)
extern "C" vj_status vj_mlp_loss_grad(vj_mlp* m, const float* x, const float* t_reg, const float* t_cls, int64_t n,
                                      double* loss, float* grad) {
    return mlp_guard([&] {
        VJ_REQUIRE(m && x && t_reg && t_cls && n >= 1, VJ_ERR_ARG, "bad argument");
        cudaStream_t s = m->stream;
        DBuf<float> xd;
        xd.alloc((size_t)n * m->din, s);
        ensure_batch(m, n);
        VJ_CUDA(cudaMemcpyAsync(xd.p, x, (size_t)n * m->din * sizeof(float), cudaMemcpyHostToDevice, s));
        VJ_CUDA(cudaMemcpyAsync(m->tr.p, t_reg, n * sizeof(float), cudaMemcpyHostToDevice, s));
        VJ_CUDA(cudaMemcpyAsync(m->tc.p, t_cls, n * sizeof(float), cudaMemcpyHostToDevice, s));
        VJ_CUDA(cudaMemsetAsync(m->loss.p, 0, sizeof(double), s));
        forward(m, xd.p, n, false);
        backward(m, n);
        if (loss) VJ_CUDA(cudaMemcpyAsync(loss, m->loss.p, sizeof(double), cudaMemcpyDeviceToHost, s));
        if (grad) VJ_CUDA(cudaMemcpyAsync(grad, m->g.p, m->np * sizeof(float), cudaMemcpyDeviceToHost, s));
        VJ_CUDA(cudaStreamSynchronize(s));
        xd.free_(s);
    });
}

// Adam training on n host rows (standardised with their own mean / std),
// mini-batches from a seeded shuffle; returns the last epoch's mean loss
extern "C" vj_status vj_mlp_train(vj_mlp* m, const float* x, const float* t_reg, const float* t_cls, int64_t n,
                                  int epochs, int batch, float lr, uint64_t seed, double* final_loss) {
    return mlp_guard([&] {
        VJ_REQUIRE(m && x && t_reg && t_cls && n >= 1 && epochs >= 1 && batch >= 1, VJ_ERR_ARG, "bad argument");
        cudaStream_t s = m->stream;
        const int din = m->din;
        // standardisation from the training rows (host, FP64)
        std::vector<float> mu(din), sd(din);
        for (int f = 0; f < din; f++) {
            double a = 0.0, b = 0.0;
            for (int64_t i = 0; i < n; i++) {
                const double v = x[i * din + f];
                a += v;
                b += v * v;
            }
            const double mean = a / n, var = std::max(b / n - mean * mean, 0.0);
            mu[f] = (float)mean;
            sd[f] = (float)std::max(std::sqrt(var), 1e-6);
        }
        VJ_CUDA(cudaMemcpyAsync(m->mu.p, mu.data(), din * sizeof(float), cudaMemcpyHostToDevice, s));
        VJ_CUDA(cudaMemcpyAsync(m->sd.p, sd.data(), din * sizeof(float), cudaMemcpyHostToDevice, s));
        m->has_norm = true;
        DBuf<float> xd, trd, tcd;
        xd.alloc((size_t)n * din, s);
        trd.alloc(n, s);
        tcd.alloc(n, s);
        VJ_CUDA(cudaMemcpyAsync(xd.p, x, (size_t)n * din * sizeof(float), cudaMemcpyHostToDevice, s));
        VJ_CUDA(cudaMemcpyAsync(trd.p, t_reg, n * sizeof(float), cudaMemcpyHostToDevice, s));
        VJ_CUDA(cudaMemcpyAsync(tcd.p, t_cls, n * sizeof(float), cudaMemcpyHostToDevice, s));
        // batches are gathered on the host from a shuffled order
        std::vector<int64_t> perm(n);
        std::iota(perm.begin(), perm.end(), 0);
        std::mt19937_64 rng(seed);
        std::vector<float> hx((size_t)batch * din), hr(batch), hc(batch);
        DBuf<float> bx;
        bx.alloc((size_t)batch * din, s);
        ensure_batch(m, batch);
        double ep_loss = 0.0;
        for (int ep = 0; ep < epochs; ep++) {
            std::shuffle(perm.begin(), perm.end(), rng);
            ep_loss = 0.0;
            VJ_CUDA(cudaMemsetAsync(m->loss.p, 0, sizeof(double), s));
            int64_t nb = 0;
            for (int64_t b0 = 0; b0 < n; b0 += batch) {
                const int64_t bn = std::min<int64_t>(batch, n - b0);
                for (int64_t i = 0; i < bn; i++) {
                    const int64_t r = perm[b0 + i];
                    std::copy(x + r * din, x + (r + 1) * din, hx.begin() + i * din);
                    hr[i] = t_reg[r];
                    hc[i] = t_cls[r];
                }
                VJ_CUDA(cudaMemcpyAsync(bx.p, hx.data(), (size_t)bn * din * sizeof(float), cudaMemcpyHostToDevice, s));
                VJ_CUDA(cudaMemcpyAsync(m->tr.p, hr.data(), bn * sizeof(float), cudaMemcpyHostToDevice, s));
                VJ_CUDA(cudaMemcpyAsync(m->tc.p, hc.data(), bn * sizeof(float), cudaMemcpyHostToDevice, s));
                forward(m, bx.p, bn, true);
                backward(m, bn);
                m->step++;
                const float b1 = 0.9f, b2 = 0.999f;
                const float c1 = 1.f - powf(b1, (float)m->step), c2 = 1.f - powf(b2, (float)m->step);
                k_adam<<<vj_div_up(m->np, 256), 256, 0, s>>>(m->w.p, m->m.p, m->v.p, m->g.p, m->np, lr, b1, b2, 1e-8f,
                                                            c1, c2);
                VJ_LAUNCH_CHECK();
                // host buffers are reused by the next batch: wait for the copies
                VJ_CUDA(cudaStreamSynchronize(s));
                nb++;
            }
            double l = 0.0;
            VJ_CUDA(cudaMemcpyAsync(&l, m->loss.p, sizeof(double), cudaMemcpyDeviceToHost, s));
            VJ_CUDA(cudaStreamSynchronize(s));
            ep_loss = l / (double)nb;
        }
        if (final_loss) *final_loss = ep_loss;
        xd.free_(s);
        trd.free_(s);
        tcd.free_(s);
        bx.free_(s);
        VJ_CUDA(cudaStreamSynchronize(s));
    });
}

// outputs (n x 2, host) for n host rows, standardised with the stored mean / std
extern "C" vj_status vj_mlp_predict(vj_mlp* m, const float* x, int64_t n, float* out) {
    return mlp_guard([&] {
        VJ_REQUIRE(m && x && out && n >= 1, VJ_ERR_ARG, "bad argument");
        cudaStream_t s = m->stream;
        DBuf<float> xd;
        xd.alloc((size_t)n * m->din, s);
        VJ_CUDA(cudaMemcpyAsync(xd.p, x, (size_t)n * m->din * sizeof(float), cudaMemcpyHostToDevice, s));
        forward(m, xd.p, n, true);
        VJ_CUDA(cudaMemcpyAsync(out, m->y.p, (size_t)n * 2 * sizeof(float), cudaMemcpyDeviceToHost, s));
        VJ_CUDA(cudaStreamSynchronize(s));
        xd.free_(s);
    });
}

extern "C" void vj_mlp_free(vj_mlp* m) {
    if (!m) return;
    cudaStream_t s = m->stream;
    m->xbf.free_(s);
    m->w1bf.free_(s);
    m->w2bf.free_(s);
    m->err.free_(s);
    for (auto* b : {&m->w, &m->m, &m->v, &m->g, &m->mu, &m->sd, &m->xb, &m->z1, &m->a1, &m->z2, &m->a2, &m->y, &m->dy,
                    &m->da2, &m->da1, &m->tr, &m->tc})
        b->free_(s);
    m->loss.free_(s);
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
    delete m;
}
