// vj_device.cuh -- device building blocks shared by the libvj kernels.
//
// Vector layout: node u's vector is row u of a [n][dp] FP32 array with dp = d
// rounded up to a multiple of 4 (zero padded), so every row starts on a
// 16-byte boundary and is read as float4.
//
// Group-parallel distances: a warp is split into 32/G groups of G lanes; a
// group evaluates one candidate; lane g of a group holds float4 slots
// g, g+G, ..., g+(NPL-1)G of the query vector in registers.  U candidates per
// group are in flight at once (their loads are issued before any arithmetic),
// which keeps U*NPL 16-byte gathers outstanding per lane.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#define VJ_FULL 0xffffffffu

__device__ __forceinline__ float4 f4zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }

// read-only, L1-allocating 16-byte load of vector data
__device__ __forceinline__ float4 ldv(const float4* p) { return __ldg(p); }

template <int G, int NPL>
__device__ __forceinline__ void load_slots(const float* __restrict__ vec, int64_t node, int dp4, int g,
                                           float4 (&r)[NPL]) {
    const float4* row = reinterpret_cast<const float4*>(vec) + node * (int64_t)dp4;
#pragma unroll
    for (int k = 0; k < NPL; k++) {
        int idx = g + k * G;
        r[k] = (idx < dp4) ? ldv(row + idx) : f4zero();
    }
}

// Slots from the BF16 copy of the vectors (rows of kpb BF16 values, zero
// padded): slot idx holds BF16 values 4 idx .. 4 idx + 3, one 8-byte load,
// kept raw (two uint32) until converted exactly to FP32 at use.  When every
// coordinate is a BF16 value these equal the FP32 rows' slots, and so every
// key, at half the bytes.
template <int G, int NPL>
__device__ __forceinline__ void load_raw_bf16(const __nv_bfloat16* __restrict__ xb, int64_t node, int kpb, int dp4,
                                              int g, uint2 (&r)[NPL]) {
    const uint2* row = reinterpret_cast<const uint2*>(xb + node * (int64_t)kpb);
#pragma unroll
    for (int k = 0; k < NPL; k++) {
        int idx = g + k * G;
        r[k] = (idx < dp4) ? __ldg(row + idx) : make_uint2(0u, 0u);
    }
}

// metric 0: squared L2 distance; metric 1: dot product (raw BF16 slots, each
// converted exactly to FP32 right before its four products: the same values
// and order as slot_accum on the converted slots)
template <int NPL>
__device__ __forceinline__ float slot_accum_bf16(const uint2 (&xr)[NPL], const float4 (&q)[NPL], int metric) {
    float a = 0.f;
#pragma unroll
    for (int k = 0; k < NPL; k++) {
        const float x0 = __uint_as_float(xr[k].x << 16), x1 = __uint_as_float(xr[k].x & 0xFFFF0000u);
        const float x2 = __uint_as_float(xr[k].y << 16), x3 = __uint_as_float(xr[k].y & 0xFFFF0000u);
        if (metric == 0) {
            float t0 = x0 - q[k].x, t1 = x1 - q[k].y, t2 = x2 - q[k].z, t3 = x3 - q[k].w;
            a = fmaf(t0, t0, a);
            a = fmaf(t1, t1, a);
            a = fmaf(t2, t2, a);
            a = fmaf(t3, t3, a);
        } else {
            a = fmaf(x0, q[k].x, a);
            a = fmaf(x1, q[k].y, a);
            a = fmaf(x2, q[k].z, a);
            a = fmaf(x3, q[k].w, a);
        }
    }
    return a;
}

// metric 0: squared L2 distance; metric 1: dot product
template <int NPL>
__device__ __forceinline__ float slot_accum(const float4 (&x)[NPL], const float4 (&q)[NPL], int metric) {
    float a = 0.f;
    if (metric == 0) {
#pragma unroll
        for (int k = 0; k < NPL; k++) {
            float t0 = x[k].x - q[k].x, t1 = x[k].y - q[k].y, t2 = x[k].z - q[k].z, t3 = x[k].w - q[k].w;
            a = fmaf(t0, t0, a);
            a = fmaf(t1, t1, a);
            a = fmaf(t2, t2, a);
            a = fmaf(t3, t3, a);
        }
    } else {
#pragma unroll
        for (int k = 0; k < NPL; k++) {
            a = fmaf(x[k].x, q[k].x, a);
            a = fmaf(x[k].y, q[k].y, a);
            a = fmaf(x[k].z, q[k].z, a);
            a = fmaf(x[k].w, q[k].w, a);
        }
    }
    return a;
}

template <int G>
__device__ __forceinline__ float group_sum(float a) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) a += __shfl_xor_sync(VJ_FULL, a, o);
    return a;
}

// Distance keys of q to cand[0..nc) written to key[0..nc) (shared memory).
// L2: squared distance; cosine: 1 - <x,q> * invx * invq.  With xb, the
// candidates' vectors are read from the BF16 copy (see load_raw_bf16).
template <int G, int NPL, int U>
__device__ __forceinline__ void group_keys(const float* __restrict__ vec, const float* __restrict__ invn,
                                           int dp4, int metric, const float4 (&q)[NPL], float invq,
                                           const int32_t* cand, int nc, float* key, int lane,
                                           const __nv_bfloat16* __restrict__ xb = nullptr, int kpb = 0) {
    constexpr int NG = 32 / G;
    const int grp = lane / G, g = lane & (G - 1);
    if (xb) {
        // BF16 rows: raw 8-byte slots take half the registers of converted
        // ones, so twice the candidates' gathers are in flight
        constexpr int UB = 2 * U;
        for (int base = 0; base < nc; base += NG * UB) {
            uint2 xr[UB][NPL];
            int node[UB];
#pragma unroll
            for (int u = 0; u < UB; u++) {
                int ci = base + u * NG + grp;
                node[u] = ci < nc ? cand[ci] : -1;
                if (node[u] >= 0) {
                    load_raw_bf16<G, NPL>(xb, node[u], kpb, dp4, g, xr[u]);
                } else {
#pragma unroll
                    for (int k = 0; k < NPL; k++) xr[u][k] = make_uint2(0u, 0u);
                }
            }
#pragma unroll
            for (int u = 0; u < UB; u++) {
                float a = group_sum<G>(slot_accum_bf16<NPL>(xr[u], q, metric));
                int ci = base + u * NG + grp;
                if (g == 0 && ci < nc) key[ci] = metric == 0 ? a : 1.0f - a * __ldg(invn + node[u]) * invq;
            }
        }
        return;
    }
    for (int base = 0; base < nc; base += NG * U) {
        float4 x[U][NPL];
        int node[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            int ci = base + u * NG + grp;
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
            float a = group_sum<G>(slot_accum<NPL>(x[u], q, metric));
            int ci = base + u * NG + grp;
            if (g == 0 && ci < nc) {
                key[ci] = metric == 0 ? a : 1.0f - a * __ldg(invn + node[u]) * invq;
            }
        }
    }
}

// FP64 distance between two nodes, evaluated by the whole warp.
// Returns the metric's distance (L2: sqrt of the FP64 sum of squares).
__device__ __forceinline__ double warp_dist64(const float* __restrict__ vec, int dp, int d, int metric,
                                              int64_t a, int64_t b, int lane) {
    const float* va = vec + a * (int64_t)dp;
    const float* vb = vec + b * (int64_t)dp;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int i = lane; i < d; i += 32) {
        double x = (double)va[i], y = (double)vb[i];
        if (metric == 0) {
            double t = x - y;
            s0 = fma(t, t, s0);
        } else {
            s0 = fma(x, y, s0);
            s1 = fma(x, x, s1);
            s2 = fma(y, y, s2);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(VJ_FULL, s0, o);
        s1 += __shfl_xor_sync(VJ_FULL, s1, o);
        s2 += __shfl_xor_sync(VJ_FULL, s2, o);
    }
    if (metric == 0) return sqrt(s0);
    if (s1 == 0.0 || s2 == 0.0) return 1.0;
    return 1.0 - s0 / (sqrt(s1) * sqrt(s2));
}

// integer mixing hash (xorshift-multiply)
__device__ __forceinline__ unsigned vj_mix(unsigned x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

// Open-addressing insert of `key` (>= 0) into tab[mask+1] (empty = -1).
// Returns 1 if newly inserted, 0 if present, -1 if the table is full.
__device__ __forceinline__ int hash_insert(int* tab, unsigned mask, int key) {
    unsigned h = vj_mix((unsigned)key) & mask;
    for (unsigned probe = 0; probe <= mask; probe++) {
        int prev = atomicCAS(tab + h, -1, key);
        if (prev == -1) return 1;
        if (prev == key) return 0;
        h = (h + 1) & mask;
    }
    return -1;
}

__device__ __forceinline__ bool hash_contains(const int* tab, unsigned mask, int key) {
    unsigned h = vj_mix((unsigned)key) & mask;
    for (unsigned probe = 0; probe <= mask; probe++) {
        int v = ((volatile const int*)tab)[h];
        if (v == key) return true;
        if (v == -1) return false;
        h = (h + 1) & mask;
    }
    return false;
}

// (key, id) lexicographic order
__device__ __forceinline__ bool kless(float ka, int ia, float kb, int ib) {
    return ka < kb || (ka == kb && ia < ib);
}

// warp argmin of (key, id) pairs, one per lane; result broadcast
__device__ __forceinline__ void warp_argmin(float& k, int& id) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        float k2 = __shfl_xor_sync(VJ_FULL, k, o);
        int i2 = __shfl_xor_sync(VJ_FULL, id, o);
        if (kless(k2, i2, k, id)) {
            k = k2;
            id = i2;
        }
    }
}

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int* p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// compile-time (G, NPL) choice for warp-per-row kernels from dp4 = dp/4
#define VJ_DISPATCH_GN(dp4, ...)            \
    do {                                    \
        if ((dp4) <= 8) {                   \
            constexpr int G = 8, NPL = 1;   \
            __VA_ARGS__;                    \
        } else if ((dp4) <= 16) {           \
            constexpr int G = 8, NPL = 2;   \
            __VA_ARGS__;                    \
        } else if ((dp4) <= 32) {           \
            constexpr int G = 8, NPL = 4;   \
            __VA_ARGS__;                    \
        } else if ((dp4) <= 64) {           \
            constexpr int G = 16, NPL = 4;  \
            __VA_ARGS__;                    \
        } else if ((dp4) <= 128) {          \
            constexpr int G = 32, NPL = 4;  \
            __VA_ARGS__;                    \
        } else if ((dp4) <= 256) {          \
            constexpr int G = 32, NPL = 8;  \
            __VA_ARGS__;                    \
        } else if ((dp4) <= 512) {          \
            constexpr int G = 32, NPL = 16; \
            __VA_ARGS__;                    \
        } else {                            \
            constexpr int G = 32, NPL = 32; \
            __VA_ARGS__;                    \
        }                                   \
    } while (0)
