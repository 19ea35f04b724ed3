// k_csr.cu -- result assembly: exclusive scan of per-query counts into CSR
// offsets, and a per-query copy of each query's pairs from the unordered
// result pool into its CSR row, sorted by data id.
#include "vj_device.cuh"
#include "vj_internal.cuh"

namespace {

constexpr int SCAN_T = 1024;
constexpr int SCAN_PER = 4;
constexpr int SCAN_TILE = SCAN_T * SCAN_PER;

// block-level inclusive scan of one value per thread (int64)
__device__ int64_t block_scan_incl(int64_t v, int64_t* warp_tot) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(VJ_FULL, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) warp_tot[w] = v;
    __syncthreads();
    if (w == 0) {
        int64_t t = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t u = __shfl_up_sync(VJ_FULL, t, o);
            if (lane >= o) t += u;
        }
        warp_tot[lane] = t;
    }
    __syncthreads();
    if (w > 0) v += warp_tot[w - 1];
    __syncthreads();
    return v;
}

// per tile: local exclusive scan into out, tile total into tot[blockIdx]
__global__ void __launch_bounds__(SCAN_T) k_scan_tiles(const int32_t* __restrict__ in, int64_t* __restrict__ out,
                                                       int64_t* __restrict__ tot, int64_t n) {
    __shared__ int64_t wt[32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_PER;
    int64_t v[SCAN_PER];
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_PER; i++) {
        v[i] = (base + i < n) ? (int64_t)in[base + i] : 0;
        s += v[i];
    }
    int64_t incl = block_scan_incl(s, wt);
    int64_t run = incl - s;
#pragma unroll
    for (int i = 0; i < SCAN_PER; i++) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
    if (threadIdx.x == blockDim.x - 1) tot[blockIdx.x] = incl;
}

// single block: exclusive scan of the tile totals (loops over chunks)
__global__ void __launch_bounds__(SCAN_T) k_scan_totals(int64_t* tot, int64_t ntiles, int64_t* grand) {
    __shared__ int64_t wt[32];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t b = 0; b < ntiles; b += SCAN_T) {
        int64_t i = b + threadIdx.x;
        int64_t v = i < ntiles ? tot[i] : 0;
        int64_t incl = block_scan_incl(v, wt);
        int64_t c = carry;
        if (i < ntiles) tot[i] = c + incl - v;
        __syncthreads();
        if (threadIdx.x == SCAN_T - 1) carry = c + incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) *grand = carry;
}

__global__ void k_scan_add(int64_t* __restrict__ out, const int64_t* __restrict__ tot, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += tot[i / SCAN_TILE];
}

// ---------------------------------------------------------------- segment sort
constexpr int SS_WPB = 8;
constexpr int SS_CAP = 256;  // per-warp shared-memory sort capacity (longer rows: block sort)

struct SegSmem {
    int id[SS_CAP];
    float d[SS_CAP];
};

__global__ void __launch_bounds__(SS_WPB * 32)
    k_seg_sort_copy(const int64_t* __restrict__ start, const int32_t* __restrict__ counts,
                    const int64_t* __restrict__ offsets, const int32_t* __restrict__ sid,
                    const float* __restrict__ sd, int32_t* __restrict__ did, float* __restrict__ dd, int64_t nseg,
                    int64_t* __restrict__ large, int* __restrict__ nlarge) {
    __shared__ SegSmem sm[SS_WPB];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    SegSmem& S = sm[warp];
    for (int64_t sg = (int64_t)blockIdx.x * SS_WPB + warp; sg < nseg; sg += (int64_t)gridDim.x * SS_WPB) {
        const int n = counts[sg];
        if (n == 0) continue;
        const int64_t src = start[sg], dst = offsets[sg];
        if (n <= 32) {
            int id = lane < n ? sid[src + lane] : INT32_MAX;
            float d = lane < n ? sd[src + lane] : 0.f;
            // bitonic sort by id across the warp
#pragma unroll
            for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
                for (int j = k >> 1; j > 0; j >>= 1) {
                    int pid = __shfl_xor_sync(VJ_FULL, id, j);
                    float pd = __shfl_xor_sync(VJ_FULL, d, j);
                    bool up = (lane & k) == 0;
                    bool low = (lane & j) == 0;
                    bool take = low == up ? (pid < id) : (pid > id);
                    if (take) {
                        id = pid;
                        d = pd;
                    }
                }
            }
            if (lane < n) {
                did[dst + lane] = id;
                dd[dst + lane] = d;
            }
        } else if (n <= SS_CAP) {
            int P2 = 64;
            while (P2 < n) P2 <<= 1;
            for (int i = lane; i < P2; i += 32) {
                S.id[i] = i < n ? sid[src + i] : INT32_MAX;
                S.d[i] = i < n ? sd[src + i] : 0.f;
            }
            __syncwarp();
            for (int k = 2; k <= P2; k <<= 1) {
                for (int j = k >> 1; j > 0; j >>= 1) {
                    for (int i = lane; i < P2; i += 32) {
                        int p = i ^ j;
                        if (p > i) {
                            bool up = (i & k) == 0;
                            int a = S.id[i], b = S.id[p];
                            if ((a > b) == up) {
                                float da = S.d[i], db = S.d[p];
                                S.id[i] = b;
                                S.id[p] = a;
                                S.d[i] = db;
                                S.d[p] = da;
                            }
                        }
                    }
                    __syncwarp();
                }
            }
            for (int i = lane; i < n; i += 32) {
                did[dst + i] = S.id[i];
                dd[dst + i] = S.d[i];
            }
            __syncwarp();
        } else {
            // large rows go to the block-wide sort
            if (lane == 0) large[atomicAdd(nlarge, 1)] = sg;
        }
    }
}

// ascending compare-exchange of (id, d) pairs i < p; a partner beyond the row
// end stands for +infinity and never moves
__device__ __forceinline__ void cmpx(int32_t* id, float* d, int i, int p, int n) {
    if (p >= n) return;
    const int a = id[i], b = id[p];
    if (a > b) {
        const float da = d[i], db = d[p];
        id[i] = b;
        id[p] = a;
        d[i] = db;
        d[p] = da;
    }
}

// one row sorted by one block: bitonic network in its all-ascending form (a
// mirrored compare at the start of each merge, then half-cleaners), so a row
// of any length sorts as if padded with +infinity.  In shared memory up to
// SL_CAP entries, in place in the destination beyond that.
constexpr int SL_T = 1024;
constexpr int SL_CAP = 16384;

__device__ void block_bitonic(int32_t* id, float* d, int n) {
    int P2 = 1;
    while (P2 < n) P2 <<= 1;
    for (int k = 2; k <= P2; k <<= 1) {
        const int half = k >> 1;
        for (int t = threadIdx.x; t < P2 / 2; t += blockDim.x) {
            const int i = (t / half) * k + (t % half);
            cmpx(id, d, i, i ^ (k - 1), n);
        }
        __syncthreads();
        for (int j = k >> 2; j > 0; j >>= 1) {
            for (int t = threadIdx.x; t < P2 / 2; t += blockDim.x) {
                const int i = (t / j) * 2 * j + (t % j);
                cmpx(id, d, i, i + j, n);
            }
            __syncthreads();
        }
    }
}

__global__ void __launch_bounds__(SL_T)
    k_seg_sort_large(const int64_t* __restrict__ start, const int32_t* __restrict__ counts,
                     const int64_t* __restrict__ offsets, const int32_t* __restrict__ sid,
                     const float* __restrict__ sd, int32_t* __restrict__ did, float* __restrict__ dd,
                     const int64_t* __restrict__ large, const int* __restrict__ nlarge) {
    extern __shared__ uint8_t sl_raw[];
    int* sid_s = reinterpret_cast<int*>(sl_raw);
    float* sd_s = reinterpret_cast<float*>(sl_raw + SL_CAP * sizeof(int));
    const int nl = *nlarge;
    for (int li = blockIdx.x; li < nl; li += gridDim.x) {
        const int64_t sg = large[li];
        const int n = counts[sg];
        const int64_t src = start[sg], dst = offsets[sg];
        if (n <= SL_CAP) {
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                sid_s[i] = sid[src + i];
                sd_s[i] = sd[src + i];
            }
            __syncthreads();
            block_bitonic(sid_s, sd_s, n);
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                did[dst + i] = sid_s[i];
                dd[dst + i] = sd_s[i];
            }
        } else {
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                did[dst + i] = sid[src + i];
                dd[dst + i] = sd[src + i];
            }
            __syncthreads();
            block_bitonic(did + dst, dd + dst, n);
        }
        __syncthreads();
    }
}

// column counts of a pair list
__global__ void k_col_count(const int32_t* __restrict__ ids, int64_t nnz, int32_t* __restrict__ counts) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < nnz) atomicAdd(counts + ids[e], 1);
}

// warp per row: each pair (row r, column c) goes to c's transposed row as r
__global__ void k_transpose_scatter(const int64_t* __restrict__ off, int64_t nrows, const int32_t* __restrict__ ids,
                                    const float* __restrict__ d, const int64_t* __restrict__ toff,
                                    int32_t* __restrict__ cursor, int32_t* __restrict__ tid, float* __restrict__ td) {
    const int lane = threadIdx.x & 31;
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (r >= nrows) return;
    for (int64_t e = off[r] + lane; e < off[r + 1]; e += 32) {
        const int c = ids[e];
        const int64_t pos = toff[c] + atomicAdd(cursor + c, 1);
        tid[pos] = (int32_t)r;
        td[pos] = d[e];
    }
}

}  // namespace

void vj_csr_transpose(vj_index* ix, const int64_t* off, int64_t nrows, const int32_t* ids, const float* d,
                      int64_t nnz, int64_t ncols, DBuf<int64_t>& toff, DBuf<int32_t>& tids, DBuf<float>& tds) {
    cudaStream_t s = ix->stream;
    DBuf<int32_t> counts, cursor, uid;
    DBuf<float> ud;
    counts.alloc(std::max<int64_t>(ncols, 1), s);
    cursor.alloc(std::max<int64_t>(ncols, 1), s);
    VJ_CUDA(cudaMemsetAsync(counts.p, 0, std::max<int64_t>(ncols, 1) * sizeof(int32_t), s));
    VJ_CUDA(cudaMemsetAsync(cursor.p, 0, std::max<int64_t>(ncols, 1) * sizeof(int32_t), s));
    if (nnz > 0) {
        k_col_count<<<vj_div_up(nnz, 256), 256, 0, s>>>(ids, nnz, counts.p);
        VJ_LAUNCH_CHECK();
    }
    toff.ensure(ncols + 1, s);
    vj_exclusive_scan_i32_to_i64(counts.p, toff.p, ncols, ix);
    uid.alloc(std::max<int64_t>(nnz, 1), s);
    ud.alloc(std::max<int64_t>(nnz, 1), s);
    if (nnz > 0 && nrows > 0) {
        k_transpose_scatter<<<vj_div_up(nrows * 32, 256), 256, 0, s>>>(off, nrows, ids, d, toff.p, cursor.p, uid.p,
                                                                     ud.p);
        VJ_LAUNCH_CHECK();
    }
    // the scatter order within a row is arbitrary: sort each row by id
    tids.ensure(std::max<int64_t>(nnz, 1), s);
    tds.ensure(std::max<int64_t>(nnz, 1), s);
    vj_segment_sort_copy(toff.p, counts.p, toff.p, uid.p, ud.p, tids.p, tds.p, ncols, ix);
    counts.free_(s);
    cursor.free_(s);
    uid.free_(s);
    ud.free_(s);
}

void vj_exclusive_scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, vj_index* ix) {
    // out has n + 1 entries; out[n] = total
    cudaStream_t s = ix->stream;
    const int64_t ntiles = std::max<int64_t>(1, (n + SCAN_TILE - 1) / SCAN_TILE);
    DBuf<int64_t> tot;
    tot.alloc(ntiles, s);
    k_scan_tiles<<<(unsigned)ntiles, SCAN_T, 0, s>>>(in, out, tot.p, n);
    VJ_LAUNCH_CHECK();
    k_scan_totals<<<1, SCAN_T, 0, s>>>(tot.p, ntiles, out + n);
    VJ_LAUNCH_CHECK();
    if (n > 0) {
        k_scan_add<<<vj_div_up(n, 256), 256, 0, s>>>(out, tot.p, n);
        VJ_LAUNCH_CHECK();
    }
    tot.free_(s);
}

void vj_segment_sort_copy(const int64_t* src_start, const int32_t* counts, const int64_t* offsets,
                          const int32_t* src_id, const float* src_d, int32_t* dst_id, float* dst_d, int64_t nseg,
                          vj_index* ix) {
    if (nseg == 0) return;
    cudaStream_t s = ix->stream;
    // rows longer than a warp's shared-memory sort are listed for the block-wide sort
    ix->sort_large.ensure(nseg, s);
    ix->sort_nlarge.ensure(1, s);
    VJ_CUDA(cudaMemsetAsync(ix->sort_nlarge.p, 0, sizeof(int), s));
    int blocks = (int)std::min<int64_t>(vj_div_up(nseg, SS_WPB), (int64_t)ix->num_sms * 16);
    k_seg_sort_copy<<<blocks, SS_WPB * 32, 0, s>>>(src_start, counts, offsets, src_id, src_d, dst_id, dst_d, nseg,
                                                   ix->sort_large.p, ix->sort_nlarge.p);
    VJ_LAUNCH_CHECK();
    const int smem = SL_CAP * (int)(sizeof(int) + sizeof(float));
    VJ_CUDA(cudaFuncSetAttribute(k_seg_sort_large, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    k_seg_sort_large<<<ix->num_sms, SL_T, smem, s>>>(src_start, counts, offsets, src_id, src_d, dst_id, dst_d,
                                                     ix->sort_large.p, ix->sort_nlarge.p);
    VJ_LAUNCH_CHECK();
}
