// vj_internal.cuh -- shared declarations of the libvj translation units.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <functional>
#include <string>
#include <vector>

#include "../../include/vj.h"

// ------------------------------------------------------------------ errors
void vj_set_error(const char* fmt, ...);

struct VjError {
    vj_status code;
};

#define VJ_CUDA(call)                                                                 \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess) {                                                      \
            vj_set_error("%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_)); \
            throw VjError{VJ_ERR_CUDA};                                               \
        }                                                                             \
    } while (0)

#define VJ_LAUNCH_CHECK() VJ_CUDA(cudaGetLastError())

#define VJ_REQUIRE(cond, code, ...)      \
    do {                                 \
        if (!(cond)) {                   \
            vj_set_error(__VA_ARGS__);   \
            throw VjError{code};         \
        }                                \
    } while (0)

// ------------------------------------------------------------------ constants
constexpr int VJ_NUM_SMS_HINT = 148;
constexpr int VJ_NFEAT = 7;  // scalar features of the learned predictor (before the d coordinates)
constexpr float VJ_F32_U = 5.9604645e-8f;  // unit roundoff of binary32 (2^-24)

// device error codes (written by kernels into a device word, read by the host)
enum : int {
    VJ_DERR_NONE = 0,
    VJ_DERR_WAIT_TIMEOUT = 1,   // a work-sharing dependency wait gave up
    VJ_DERR_VISITED_OVERFLOW = 2,
    VJ_DERR_RESULT_OVERFLOW = 3,
    VJ_DERR_QUEUE_OVERFLOW = 4,
};

// ------------------------------------------------------------------ device buffers
template <class T>
struct DBuf {
    T* p = nullptr;
    size_t n = 0;
    void alloc(size_t count, cudaStream_t s);
    void free_(cudaStream_t s);
    void ensure(size_t count, cudaStream_t s) {
        if (count > n) {
            free_(s);
            alloc(count, s);
        }
    }
};

template <class T>
void DBuf<T>::alloc(size_t count, cudaStream_t s) {
    n = count;
    if (count == 0) {
        p = nullptr;
        return;
    }
    cudaError_t e = cudaMallocAsync((void**)&p, count * sizeof(T), s);
    if (e != cudaSuccess) {
        p = nullptr;
        n = 0;
        vj_set_error("device allocation of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
        throw VjError{VJ_ERR_OOM};
    }
}
template <class T>
void DBuf<T>::free_(cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
    p = nullptr;
    n = 0;
}

// ------------------------------------------------------------------ the index
// candidate columns of a node's kNN list
enum {
    VJ_KNN_ALL = 0,    // every other node (merged index)
    VJ_KNN_DATA = 1,   // data nodes only (NN-Map index)
    VJ_KNN_GROUPS = 2  // nodes of its own set (separate indexes)
};

struct vj_index {
    int dev = 0;
    int64_t nx = 0, nq = 0, n = 0;
    int d = 0, dp = 0;  // dp = d rounded up to a multiple of 4 (16-byte rows)
    int R = 0, K = 0;
    vj_metric metric = VJ_L2;
    vj_params p{};
    cudaStream_t stream = nullptr;
    cudaStream_t own_stream = nullptr;  // created by vj_build, destroyed by vj_free
    int num_sms = VJ_NUM_SMS_HINT;

    DBuf<float> vec;      // [n][dp] FP32, zero padded
    DBuf<float> sqn;      // [n] squared norm (FP32 of the FP64 value)
    DBuf<float> invn;     // [n] 1/|v| (cosine), 0 for a zero vector
    DBuf<double> sqn64;   // [n] squared norm in FP64
    DBuf<int32_t> knn;    // [n][K] exact kNN ids
    DBuf<float> knnd;     // [n][K] their distance keys (L2: squared distance; cosine: distance)
    DBuf<int32_t> adj;    // [n][R] -1 padded
    DBuf<float> elen;     // [n][R] dist(u, v) for data->data edges, NaN otherwise
    int32_t entry = 0;
    DBuf<int32_t> parent; // [nq]
    DBuf<int32_t> order;  // [nq]
    DBuf<int32_t> depth;  // [nq]
    int max_depth = 0;
    DBuf<__nv_bfloat16> xbf;   // [n][kp] BF16 copy of every node, data rows first (tensor-core tiles)
    DBuf<__nv_bfloat16> xbias; // [n][16] L2: three-term BF16 split of each node's scan bias
    DBuf<__nv_bfloat16> abias; // [128][16] (1, 1, 1, 0, ...) rows: the query side of the bias step
    float tc_cb = 0.f, tc_c3 = 0.f, tc_cbmax = 0.f;  // BF16 scan bound constants
    // per-query plan (route to the brute-force scan / hybrid budget), optional
    DBuf<uint8_t> plan_route;  // [nq]
    DBuf<int32_t> plan_beam;   // [nq]
    DBuf<int32_t> routed;      // routed query indices
    int64_t nrouted = 0;
    bool has_route = false, has_beam = false;
    int plan_max_beam = 0;
    // learned predictor (optional): cached per-query statistics and the model
    DBuf<float> qstat;         // [nq][5] d1, d2, dist to entry, nearest data neighbour, #data neighbours
    DBuf<float> qdn;           // [nq][R] distances to data neighbours (+inf otherwise)
    DBuf<float> feat;          // [nq][VJ_NFEAT + d]
    DBuf<float> pred_y;        // [nq][2]
    DBuf<unsigned long long> ctr_plan;
    struct vj_mlp* predictor = nullptr;
    float route_threshold = 0.5f;
    int beam_cap = 256;
    bool bf16_exact = false;   // BF16 Gram keys are exact for these inputs (small integers)
    bool bf16_lossless = false;  // every coordinate is exactly a BF16 value
    bool cos_raw = false;      // cosine, streamed tiles: xbf holds the raw (not unit) rows, scaled in the epilogue
    DBuf<float> wcs, wcb;      // [n] streamed tiles: per-column scale and bias of the accumulator
    // streamed scan with the measured rounding bound (FP8 tiles, or BF16 tiles
    // of inputs that are not BF16 values): per data row the FP64 norm of the
    // tile row's rounding error (rounded up); FP8 also keeps its own copy of
    // the data rows (kb8 bytes each, one power-of-two scale per row, 1/scale)
    DBuf<float> xerr_bf;       // [nx] BF16 tile rows
    DBuf<uint8_t> x8;          // [nx][kb8] E4M3
    DBuf<float> x8rs, x8err;   // [nx]
    int kb8 = 0;
    // kNN build of rows wider than 128 columns whose coordinates are not BF16
    // values: TF32 tiles ([n][kp32] FP32 words holding TF32 values, freed after
    // the sweeps) under the measured bound: per node the rounding error norm
    // and the epilogue's column scale and bias; knn_beta bounds |tile key -
    // key| for the re-rank's prefilter
    DBuf<float> xtf, xerr_tf, kcs, kcb;
    bool knn_measured = false;
    double knn_beta = 0.0;
    // NN-Map index (the paper's closing design): kNN lists over data columns
    // only, the graph G_X over data rows only, and per query its witness
    // (nearest data vector), the witness's FP64 distance and the OOD bit
    bool nnmap = false;
    // separate (per-set) indexes (Sec. 3.2): the data graph G_Y over the data
    // rows and the query graph over the query rows, in one adjacency array;
    // the entry s_Y is a data node and the MST runs over the query graph
    bool separate = false;
    int knn_mode = VJ_KNN_ALL;  // which nodes a row's kNN list ranks (VJ_KNN_*)
    int64_t graph_rows = 0;     // nodes with a graph row (n, or nx for an NN-Map index)
    int64_t entry_rows = 0;     // the entry is the node nearest the centroid of nodes 0..entry_rows-1
    DBuf<float> pkeys;         // [nq][R + 1] the probe kernel's keys (N(q), then the entry)
    DBuf<int32_t> nm_w;        // [nq] witness
    DBuf<double> nm_wd;        // [nq] its distance (FP64)
    DBuf<uint8_t> nm_ood;      // [nq] OOD bit
    // traversal setting chosen by vj_autotune / vj_set_tuning: join class
    // (-1: the smallest that holds the row), persistent blocks, probe ring
    // stages (0: the defaults) and the probe's copy (1: one bulk copy per row)
    int tune_cls = -1, tune_blocks = 0, tune_ring = 0, tune_bulk = 0;
    long long wait_polls = 0;  // dependency-wait limit of the traversal (0: the default)
    int hold_q = -1;           // test knob: a query that never publishes its cache (-1: none)
    double maxnorm = 0.0;      // largest vector norm (FP64)
    double last_scan_ms = 0.0; // device time of the last tensor-core scan
    int64_t last_scan_cand = 0;
    int64_t knn_uncertified = 0;  // rows whose tile candidates needed the exact fallback
    bool knn_tc = false;          // the kNN candidates came from the tensor cores
    double ms_build = 0.0;        // device time of vj_build
    double ms_knn = 0.0;          // ... of which the exact kNN lists

    // join scratch kept across calls
    DBuf<int> done;           // [nq] publish flags of finished queries (soft sharing)
    DBuf<uint8_t> qflag;      // [nq] soft sharing: what pass 1 recorded per query
    DBuf<float> ckey;         // [nq] soft sharing: FP32 key of each query's pass-1 cache
    DBuf<int32_t> cache1, sca, cout;  // [nq] soft sharing: pass-1 cache, pass-2 seed and cache
    DBuf<uint8_t> outc;       // [nq] soft sharing: pass-2 decision
    DBuf<int32_t> cache2, steps2, count2;  // [nq] soft sharing: staged pass-2 re-runs
    DBuf<uint8_t> hyb2;
    DBuf<int64_t> seg2;
    DBuf<uint8_t> anc;        // [2][nq] soft sharing: ancestor-changed flags (pointer jumping)
    DBuf<int32_t> jmp;        // [2][nq] ... and the jump links
    DBuf<int32_t> order1;     // [nq] longest-first dispatch order (from the last join's visits)
    DBuf<int> cost_hist;
    bool have_costs = false;
    DBuf<int32_t> scan_cq, scan_cx;  // tensor-core scan candidates (query, data id)
    DBuf<float> scan_ck;             // ... and their exact keys (integer inputs)
    bool last_scan_exact_keys = false;
    DBuf<int64_t> sort_large;  // result rows handed to the block-wide sort
    DBuf<int> sort_nlarge;
    DBuf<int32_t> cache;      // [nq]
    DBuf<int32_t> steps;      // [nq]
    DBuf<uint8_t> hyb;        // [nq]
    DBuf<int32_t> count;      // [nq]
    DBuf<int64_t> seg;        // [nq] start of each query's results in the pool
    DBuf<int32_t> pool_id;    // result pool
    DBuf<float> pool_d;
    DBuf<unsigned long long> ctr;  // counters + ticket + error word
    DBuf<int64_t> offsets;    // [nq+1]
    DBuf<int32_t> out_id;
    DBuf<float> out_d;
    DBuf<unsigned char> tmp;  // scan / sort temporary storage
};

// ------------------------------------------------------------------ launchers (host)
// tiles: kNN over all nodes of the index; fills ix->knn / ix->knnd
void vj_build_knn(vj_index* ix);
// graph: prune + reverse edges + entry + edge lengths + MST order
void vj_build_graph(vj_index* ix);
// NN-Map: witness, FP64 witness distance and OOD bit of every query
void vj_build_nnmap(vj_index* ix);
// exact join pairs into CSR (device arrays owned by the caller-provided buffers)
struct CsrOut {
    int64_t nnz;
};
void vj_exact_join_device(vj_index* ix, float eps, DBuf<int64_t>& offsets, DBuf<int32_t>& ids,
                          DBuf<float>& dists, int64_t* nnz_out, double* ms_out);
// exact rows of the queries qrows (all queries when NULL) from the tensor-core
// scan, as a CSR over all nq queries; each row sorted by data id when
// sort_rows, else in scatter order (the join sorts the routed rows later)
void vj_scan_rows_csr(vj_index* ix, const int32_t* qrows, int64_t nr, float eps, DBuf<int64_t>& offsets,
                      DBuf<int32_t>& ids, DBuf<float>& dists, int64_t* nnz_out, double* ms_out,
                      bool sort_rows = false);
// approximate join; returns stats, leaves CSR in ix->offsets/out_id/out_d and per-query arrays
void vj_run_join(vj_index* ix, float eps, int budget, vj_stats* st, int64_t* nnz_out);
// traversal classes for the tuner: the k-th of vj_join_class_count() in order
// of row capacity (G * NPL 16-byte slots), the class pick() takes for dp4
// slots, and the persistent blocks of a class
int vj_join_class_count();
void vj_join_class_info(int k, int* cls, int* G, int* NPL, int* U);
int vj_join_default_class(int dp4);
int vj_join_max_blocks(int cls, int num_sms);
// free the idle traversal workspaces of the process-wide cache
void vj_trav_space_trim();
// joins of n distinct indexes (default budget) with fused traversal launches;
// par(n, fn) runs fn(0..n-1), possibly on several host threads, and throws if
// any call threw
using vj_par_for = std::function<void(int, const std::function<void(int)>&)>;
void vj_run_join_multi(vj_index* const* ixs, const float* eps, int n, vj_stats* st, int64_t* nnz_out,
                       const vj_par_for& par);

// tensor-core (tcgen05) BF16 scan of query rows against all data rows:
// candidate (query index, data id) pairs, exact after re-check
// cw (optional): per candidate, the low-precision Gram value acc * cs of the
// streamed kernel (kp > 128; left empty otherwise), for the approximate-key
// prefilter of the re-rank
bool vj_tc_knn_candidates(vj_index* ix, DBuf<int64_t>& off, DBuf<int32_t>& ids, DBuf<float>& row_thr,
                          DBuf<float>* cw = nullptr);
// BF16 copy of every node and the tiles' bound constants (built once)
void vj_ensure_bf16(vj_index* ix);
int64_t vj_tc_scan_candidates(vj_index* ix, const int32_t* qrows, int64_t nr, float eps, DBuf<int32_t>& cq,
                              DBuf<int32_t>& cx, double* ms_out, DBuf<float>* ck = nullptr);

// predictor features of every query at eps, [nq][VJ_NFEAT + d] in device memory
void vj_compute_features(vj_index* ix, float eps, float* feat_dev);
// learned prologue: features -> predictor -> per-query plan; returns #routed
int64_t vj_learned_prologue(vj_index* ix, float eps);

// utilities
void vj_exclusive_scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, vj_index* ix);
// rows <-> columns of a device CSR pair list (nrows rows over ncols columns);
// every transposed row ascending by id
void vj_csr_transpose(vj_index* ix, const int64_t* off, int64_t nrows, const int32_t* ids, const float* d,
                      int64_t nnz, int64_t ncols, DBuf<int64_t>& toff, DBuf<int32_t>& tids, DBuf<float>& tds);
void vj_segment_sort_copy(const int64_t* src_start, const int32_t* counts, const int64_t* offsets,
                          const int32_t* src_id, const float* src_d, int32_t* dst_id, float* dst_d,
                          int64_t nseg, vj_index* ix);

inline int vj_div_up(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }
