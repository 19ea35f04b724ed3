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

#include <numeric>
#include <random>

#include "vj_device.cuh"
#include "vj_internal.cuh"

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

}  // namespace

// ------------------------------------------------------------------ internal API
void vj_mlp_forward_device(vj_mlp* m, const float* x, int64_t n, float* y_out, cudaStream_t s) {
    cudaStream_t keep = m->stream;
    m->stream = s;
    forward(m, x, n, true);
    VJ_CUDA(cudaMemcpyAsync(y_out, m->y.p, (size_t)n * 2 * sizeof(float), cudaMemcpyDeviceToDevice, s));
    m->stream = keep;
}
int vj_mlp_din(const vj_mlp* m) { return m->din; }

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
    for (auto* b : {&m->w, &m->m, &m->v, &m->g, &m->mu, &m->sd, &m->xb, &m->z1, &m->a1, &m->z2, &m->a2, &m->y, &m->dy,
                    &m->da2, &m->da1, &m->tr, &m->tc})
        b->free_(s);
    m->loss.free_(s);
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
    delete m;
}
