// vj_capi.cu -- the extern "C" entry points declared in include/vj.h.
// Host orchestration only: every step of a build or a join runs in the
// kernels of k_tiles.cu, k_graph.cu, k_join.cu and k_csr.cu.
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <functional>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "vj_internal.cuh"

static thread_local char g_err[1024] = "";

void vj_set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

extern "C" const char* vj_last_error(void) { return g_err; }

extern "C" void vj_default_params(vj_params* p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->degree = 32;
    p->knn_k = 64;
    p->greedy_beam = 256;
    p->conv_threshold = 10;
    p->hybrid_beam = 256;
    p->work_sharing = VJ_WS_SOFT;
    p->adapt_hybrid = 1;
    p->force_hybrid = 0;
    p->precision = VJ_PREC_BF16;
    p->learned = 0;
    p->route_bruteforce = 0;
    p->input_on_device = 0;
    p->seed = 0;
    p->gather = VJ_PREC_FP32;
    p->scan = VJ_PREC_BF16;
}

template <class F>
static vj_status guarded(F&& f) {
    try {
        f();
        return VJ_OK;
    } catch (const VjError& e) {
        return e.code;
    } catch (const std::bad_alloc&) {
        vj_set_error("host allocation failed");
        return VJ_ERR_OOM;
    } catch (...) {
        vj_set_error("unexpected internal error");
        return VJ_ERR_STATE;
    }
}

static void check_join_params(const vj_params& p) {
    VJ_REQUIRE(p.work_sharing >= VJ_WS_NONE && p.work_sharing <= VJ_WS_SELF, VJ_ERR_ARG,
               "work_sharing must be NONE, HARD, SOFT or SELF");
    VJ_REQUIRE(p.hybrid_beam >= 0 && p.hybrid_beam <= (1 << 20), VJ_ERR_ARG, "hybrid_beam out of range");
    VJ_REQUIRE(p.greedy_beam >= 1, VJ_ERR_ARG, "greedy_beam must be >= 1");
    VJ_REQUIRE(p.learned == 0 || p.learned == 1, VJ_ERR_ARG, "learned must be 0 or 1");
    VJ_REQUIRE(p.route_bruteforce == 0, VJ_ERR_ARG, "route_bruteforce is reserved and must be 0");
    VJ_REQUIRE(p.gather == VJ_PREC_FP32 || p.gather == VJ_PREC_BF16, VJ_ERR_ARG, "gather must be FP32 or BF16");
    VJ_REQUIRE(p.hybrid_seed_best == 0 || p.hybrid_seed_best == 1, VJ_ERR_ARG, "hybrid_seed_best must be 0 or 1");
    VJ_REQUIRE(p.scan == VJ_PREC_FP32 || p.scan == VJ_PREC_BF16 || p.scan == VJ_PREC_FP8, VJ_ERR_ARG,
               "scan must be FP32, BF16 or FP8");
}

static std::atomic<int64_t> g_live_indexes{0};

static void free_index(vj_index* ix) {
    if (!ix) return;
    cudaStream_t s = ix->stream;
    ix->vec.free_(s);
    ix->sqn.free_(s);
    ix->invn.free_(s);
    ix->sqn64.free_(s);
    ix->knn.free_(s);
    ix->knnd.free_(s);
    ix->adj.free_(s);
    ix->elen.free_(s);
    ix->parent.free_(s);
    ix->order.free_(s);
    ix->depth.free_(s);
    ix->qstat.free_(s);
    ix->qdn.free_(s);
    ix->feat.free_(s);
    ix->pred_y.free_(s);
    ix->ctr_plan.free_(s);
    ix->plan_route.free_(s);
    ix->plan_beam.free_(s);
    ix->routed.free_(s);
    ix->xbf.free_(s);
    ix->wcs.free_(s);
    ix->wcb.free_(s);
    ix->xerr_bf.free_(s);
    ix->x8.free_(s);
    ix->x8rs.free_(s);
    ix->x8err.free_(s);
    ix->xtf.free_(s);
    ix->anc.free_(s);
    ix->jmp.free_(s);
    ix->xerr_tf.free_(s);
    ix->kcs.free_(s);
    ix->kcb.free_(s);
    ix->pkeys.free_(s);
    ix->nm_w.free_(s);
    ix->nm_wd.free_(s);
    ix->nm_ood.free_(s);
    ix->xbias.free_(s);
    ix->abias.free_(s);
    ix->done.free_(s);
    ix->qflag.free_(s);
    ix->ckey.free_(s);
    ix->cache1.free_(s);
    ix->sca.free_(s);
    ix->cout.free_(s);
    ix->outc.free_(s);
    ix->cache2.free_(s);
    ix->steps2.free_(s);
    ix->count2.free_(s);
    ix->hyb2.free_(s);
    ix->seg2.free_(s);
    ix->order1.free_(s);
    ix->cost_hist.free_(s);
    ix->scan_cq.free_(s);
    ix->scan_cx.free_(s);
    ix->scan_ck.free_(s);
    ix->sort_large.free_(s);
    ix->sort_nlarge.free_(s);
    ix->cache.free_(s);
    ix->steps.free_(s);
    ix->hyb.free_(s);
    ix->count.free_(s);
    ix->seg.free_(s);
    ix->pool_id.free_(s);
    ix->pool_d.free_(s);
    ix->ctr.free_(s);
    ix->offsets.free_(s);
    ix->out_id.free_(s);
    ix->out_d.free_(s);
    ix->tmp.free_(s);
    cudaStreamSynchronize(s);
    if (ix->own_stream) cudaStreamDestroy(ix->own_stream);
    delete ix;
    // the last index gone: nothing will join soon, release the join workspaces
    if (g_live_indexes.fetch_sub(1) == 1) vj_trav_space_trim();
}

extern "C" vj_status vj_build(const float* X, int64_t nx, const float* Q, int64_t nq, int d, vj_metric metric,
                              const vj_params* pin, vj_index** out) {
    if (out) *out = nullptr;
    vj_index* ix = nullptr;
    vj_status st = guarded([&] {
        VJ_REQUIRE(out != nullptr, VJ_ERR_ARG, "out is NULL");
        VJ_REQUIRE(X != nullptr && Q != nullptr, VJ_ERR_ARG, "X or Q is NULL");
        VJ_REQUIRE(nx >= 1 && nq >= 1, VJ_ERR_ARG, "nx and nq must be >= 1");
        VJ_REQUIRE(nx + nq < (int64_t)INT32_MAX, VJ_ERR_ARG, "nx + nq must be < 2^31");
        VJ_REQUIRE(d >= 1 && d <= 4096, VJ_ERR_ARG, "d must be in [1, 4096]");
        VJ_REQUIRE(metric == VJ_L2 || metric == VJ_COSINE, VJ_ERR_ARG, "unknown metric");
        vj_params p;
        vj_default_params(&p);
        if (pin) p = *pin;
        VJ_REQUIRE(p.degree >= 1 && p.degree <= 32, VJ_ERR_ARG, "degree must be in [1, 32]");
        if (p.knn_k <= 0) p.knn_k = 2 * p.degree;
        VJ_REQUIRE(p.knn_k >= p.degree && p.knn_k <= 112, VJ_ERR_ARG, "knn_k must be in [degree, 112]");
        VJ_REQUIRE(p.precision == VJ_PREC_FP32 || p.precision == VJ_PREC_BF16, VJ_ERR_ARG,
                   "build tiles: FP32 or BF16 (FP8 tiles serve the scan only: vj_params.scan)");
        VJ_REQUIRE(p.nnmap == 0 || p.nnmap == 1, VJ_ERR_ARG, "nnmap must be 0 or 1");
        VJ_REQUIRE(p.separate == 0 || p.separate == 1, VJ_ERR_ARG, "separate must be 0 or 1");
        VJ_REQUIRE(!(p.nnmap && p.separate), VJ_ERR_ARG, "nnmap and separate are exclusive");
        VJ_REQUIRE(p.work_sharing != VJ_WS_HARD || p.separate, VJ_ERR_ARG,
                   "work_sharing HARD runs on separate indexes only (vj_params.separate = 1)");
        check_join_params(p);

        ix = new vj_index();
        g_live_indexes.fetch_add(1);
        VJ_CUDA(cudaGetDevice(&ix->dev));
        int sms = 0;
        VJ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ix->dev));
        ix->num_sms = sms > 0 ? sms : VJ_NUM_SMS_HINT;
        VJ_CUDA(cudaStreamCreateWithFlags(&ix->own_stream, cudaStreamNonBlocking));
        ix->stream = ix->own_stream;
        ix->nx = nx;
        ix->nq = nq;
        ix->n = nx + nq;
        ix->d = d;
        ix->dp = (d + 3) / 4 * 4;
        ix->R = p.degree;
        // at most n - 1 other nodes exist
        ix->K = (int)std::min<int64_t>(p.knn_k, ix->n - 1 > 0 ? ix->n - 1 : 1);
        ix->R = std::min(ix->R, ix->K);
        ix->metric = metric;
        ix->p = p;
        ix->nnmap = p.nnmap != 0;
        ix->separate = p.separate != 0;
        // an NN-Map index lists data candidates only, and only data rows enter
        // the graph; separate indexes list each row's own set
        ix->knn_mode = ix->nnmap ? VJ_KNN_DATA : (ix->separate ? VJ_KNN_GROUPS : VJ_KNN_ALL);
        ix->graph_rows = ix->nnmap ? nx : ix->n;
        ix->entry_rows = (ix->nnmap || ix->separate) ? nx : ix->n;
        if (ix->nnmap) {
            VJ_REQUIRE(nx >= 2, VJ_ERR_ARG, "an NN-Map index needs nx >= 2");
            ix->K = (int)std::min<int64_t>(ix->K, nx - 1);
            ix->R = std::min(ix->R, ix->K);
        }
        if (ix->separate) {
            VJ_REQUIRE(nx >= 2 && nq >= 2, VJ_ERR_ARG, "separate indexes need nx >= 2 and nq >= 2");
            ix->K = (int)std::min<int64_t>(ix->K, std::min(nx, nq) - 1);
            ix->R = std::min(ix->R, ix->K);
        }
        cudaStream_t s = ix->stream;
        ix->vec.alloc((size_t)ix->n * ix->dp, s);
        if (ix->dp != d) VJ_CUDA(cudaMemsetAsync(ix->vec.p, 0, (size_t)ix->n * ix->dp * sizeof(float), s));
        cudaMemcpyKind kind = p.input_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        VJ_CUDA(cudaMemcpy2DAsync(ix->vec.p, ix->dp * sizeof(float), X, d * sizeof(float), d * sizeof(float), nx,
                                  kind, s));
        VJ_CUDA(cudaMemcpy2DAsync(ix->vec.p + (size_t)nx * ix->dp, ix->dp * sizeof(float), Q, d * sizeof(float),
                                  d * sizeof(float), nq, kind, s));
        ix->sqn.alloc(ix->n, s);
        ix->invn.alloc(ix->n, s);
        cudaEvent_t b0, b1, b2;
        VJ_CUDA(cudaEventCreate(&b0));
        VJ_CUDA(cudaEventCreate(&b1));
        VJ_CUDA(cudaEventCreate(&b2));
        VJ_CUDA(cudaEventRecord(b0, s));
        vj_build_knn(ix);
        VJ_CUDA(cudaEventRecord(b1, s));
        vj_build_graph(ix);
        if (ix->nnmap) vj_build_nnmap(ix);
        VJ_CUDA(cudaEventRecord(b2, s));
        VJ_CUDA(cudaStreamSynchronize(s));
        float mb = 0.f, mk = 0.f;
        VJ_CUDA(cudaEventElapsedTime(&mb, b0, b2));
        VJ_CUDA(cudaEventElapsedTime(&mk, b0, b1));
        ix->ms_build = mb;
        ix->ms_knn = mk;
        cudaEventDestroy(b0);
        cudaEventDestroy(b1);
        cudaEventDestroy(b2);
        *out = ix;
    });
    if (st != VJ_OK && ix) free_index(ix);
    return st;
}

extern "C" vj_status vj_set_stream(vj_index* ix, void* stream) {
    return guarded([&] {
        VJ_REQUIRE(ix != nullptr, VJ_ERR_ARG, "index is NULL");
        VJ_CUDA(cudaStreamSynchronize(ix->stream));
        ix->stream = (cudaStream_t)stream;
    });
}

extern "C" vj_status vj_set_join_params(vj_index* ix, const vj_params* p) {
    return guarded([&] {
        VJ_REQUIRE(ix != nullptr && p != nullptr, VJ_ERR_ARG, "NULL argument");
        check_join_params(*p);
        VJ_REQUIRE(p->work_sharing != VJ_WS_HARD || ix->separate, VJ_ERR_ARG,
                   "work_sharing HARD runs on separate indexes only (vj_params.separate = 1)");
        ix->p.greedy_beam = p->greedy_beam;
        ix->p.conv_threshold = p->conv_threshold;
        ix->p.hybrid_beam = p->hybrid_beam;
        ix->p.work_sharing = p->work_sharing;
        ix->p.adapt_hybrid = p->adapt_hybrid;
        ix->p.force_hybrid = p->force_hybrid;
        ix->p.learned = p->learned;
        ix->p.gather = p->gather;
        ix->p.hybrid_seed_best = p->hybrid_seed_best;
        ix->p.scan = p->scan;
    });
}

// class table position of `cls` (-1 if none)
static int class_pos(int cls) {
    for (int k = 0; k < vj_join_class_count(); k++) {
        int c, G, NPL, U;
        vj_join_class_info(k, &c, &G, &NPL, &U);
        if (c == cls) return k;
    }
    return -1;
}

extern "C" vj_status vj_set_tuning(vj_index* ix, int lanes, int slots, int inflight, int blocks, int probe_ring,
                                   int probe_bulk) {
    return guarded([&] {
        VJ_REQUIRE(ix != nullptr, VJ_ERR_ARG, "index is NULL");
        VJ_REQUIRE(blocks >= 0, VJ_ERR_ARG, "blocks must be >= 0");
        VJ_REQUIRE(probe_ring == 0 || (probe_ring >= 2 && probe_ring <= 8), VJ_ERR_ARG,
                   "probe_ring must be 0 or 2..8");
        VJ_REQUIRE(probe_bulk == 0 || probe_bulk == 1, VJ_ERR_ARG, "probe_bulk must be 0 or 1");
        int cls = -1;
        if (lanes != 0) {
            for (int k = 0; k < vj_join_class_count() && cls < 0; k++) {
                int c, G, NPL, U;
                vj_join_class_info(k, &c, &G, &NPL, &U);
                if (G == lanes && NPL == slots && U == inflight) {
                    VJ_REQUIRE((int64_t)G * NPL >= ix->dp / 4, VJ_ERR_ARG,
                               "the class holds %d floats per row, the index has %d", G * NPL * 4, ix->d);
                    cls = c;
                }
            }
            VJ_REQUIRE(cls >= 0, VJ_ERR_ARG, "no traversal class with lanes %d, slots %d, inflight %d", lanes,
                       slots, inflight);
        }
        ix->tune_cls = cls;
        ix->tune_blocks = blocks;
        ix->tune_ring = probe_ring;
        ix->tune_bulk = probe_bulk;
    });
}

extern "C" vj_status vj_autotune(vj_index* ix, float eps, int reps, vj_tune_report* rep) {
    if (rep) memset(rep, 0, sizeof(*rep));
    if (!ix) {
        vj_set_error("index is NULL");
        return VJ_ERR_ARG;
    }
    const int saved_cls = ix->tune_cls, saved_blocks = ix->tune_blocks, saved_ring = ix->tune_ring,
              saved_bulk = ix->tune_bulk;
    const vj_status st = guarded([&] {
        VJ_REQUIRE(rep != nullptr, VJ_ERR_ARG, "report is NULL");
        VJ_REQUIRE(eps > 0.f && eps == eps, VJ_ERR_ARG, "eps must be > 0");
        VJ_REQUIRE(reps >= 1 && reps <= 10, VJ_ERR_ARG, "reps must be 1..10");
        const int dp4 = ix->dp / 4;
        const int k0 = class_pos(vj_join_default_class(dp4));
        const bool probe = !ix->separate && !ix->nnmap;
        struct Setting {
            int cls, blocks, ring, bulk;
        };
        std::vector<Setting> set;
        for (int k = k0; k < vj_join_class_count() && k < k0 + 3; k++) {
            int c, G, NPL, U;
            vj_join_class_info(k, &c, &G, &NPL, &U);
            const int mb = vj_join_max_blocks(c, ix->num_sms);
            set.push_back({c, mb, 0, 0});
            if (mb / 2 >= ix->num_sms) set.push_back({c, mb / 2, 0, 0});
        }
        if (probe) {
            set.push_back({set[0].cls, set[0].blocks, 4, 0});
            set.push_back({set[0].cls, set[0].blocks, 2, 0});
            set.push_back({set[0].cls, set[0].blocks, 0, 1});
        }
        int64_t nnz0 = -1, dc0 = -1;
        double best = 1e300;
        for (size_t i = 0; i < set.size() && (int)i < VJ_TUNE_MAX; i++) {
            ix->tune_cls = set[i].cls;
            ix->tune_blocks = set[i].blocks;
            ix->tune_ring = set[i].ring;
            ix->tune_bulk = set[i].bulk;
            std::vector<double> ms;
            int64_t nnz = 0;
            vj_stats s{};
            for (int r = 0; r <= reps; r++) {
                s = vj_stats{};
                vj_run_join(ix, eps, 0, &s, &nnz);
                if (r > 0) ms.push_back(s.ms_total);
            }
            std::sort(ms.begin(), ms.end());
            const int n = rep->n++;
            int c, G, NPL, U;
            vj_join_class_info(class_pos(set[i].cls), &c, &G, &NPL, &U);
            rep->lanes[n] = G;
            rep->slots[n] = NPL;
            rep->inflight[n] = U;
            rep->blocks[n] = set[i].blocks;
            rep->probe_ring[n] = probe ? (set[i].ring ? set[i].ring : 8) : 0;
            rep->probe_bulk[n] = probe ? set[i].bulk : 0;
            rep->ms[n] = ms[ms.size() / 2];
            if (i == 0) {
                nnz0 = nnz;
                dc0 = s.dist_computations;
            }
            rep->valid[n] = (nnz == nnz0 && s.dist_computations == dc0) ? 1 : 0;
            if (rep->valid[n] && rep->ms[n] < best) {
                best = rep->ms[n];
                rep->chosen = n;
            }
        }
        const Setting& ch = set[rep->chosen];
        ix->tune_cls = ch.cls;
        ix->tune_blocks = ch.blocks;
        ix->tune_ring = ch.ring;
        ix->tune_bulk = ch.bulk;
    });
    if (st != VJ_OK) {
        ix->tune_cls = saved_cls;
        ix->tune_blocks = saved_blocks;
        ix->tune_ring = saved_ring;
        ix->tune_bulk = saved_bulk;
    }
    return st;
}

extern "C" vj_status vj_set_wait_test(vj_index* ix, long long max_polls, int64_t hold_q) {
    return guarded([&] {
        VJ_REQUIRE(ix != nullptr, VJ_ERR_ARG, "index is NULL");
        VJ_REQUIRE(max_polls >= 0, VJ_ERR_ARG, "max_polls must be >= 0");
        VJ_REQUIRE(hold_q >= -1 && hold_q < ix->nq, VJ_ERR_ARG, "hold_q out of range");
        ix->wait_polls = max_polls;
        ix->hold_q = (int)hold_q;
    });
}

extern "C" vj_status vj_set_plan(vj_index* ix, const uint8_t* route, const int32_t* beam) {
    return guarded([&] {
        VJ_REQUIRE(ix != nullptr, VJ_ERR_ARG, "index is NULL");
        VJ_REQUIRE(!ix->nnmap || (route == nullptr && beam == nullptr), VJ_ERR_STATE,
                   "an NN-Map index joins from its witnesses: no per-query plan");
        cudaStream_t s = ix->stream;
        const int64_t nq = ix->nq;
        ix->has_route = false;
        ix->has_beam = false;
        ix->nrouted = 0;
        ix->plan_max_beam = 0;
        if (route) {
            std::vector<int32_t> ids;
            for (int64_t q = 0; q < nq; q++)
                if (route[q]) ids.push_back((int32_t)q);
            ix->plan_route.ensure(nq, s);
            VJ_CUDA(cudaMemcpyAsync(ix->plan_route.p, route, nq, cudaMemcpyHostToDevice, s));
            ix->routed.ensure(std::max<size_t>(ids.size(), 1), s);
            if (!ids.empty())
                VJ_CUDA(cudaMemcpyAsync(ix->routed.p, ids.data(), ids.size() * sizeof(int32_t),
                                        cudaMemcpyHostToDevice, s));
            ix->nrouted = (int64_t)ids.size();
            ix->has_route = true;
        }
        if (beam) {
            int mx = 0;
            for (int64_t q = 0; q < nq; q++) {
                VJ_REQUIRE(beam[q] >= -1 && beam[q] <= (1 << 20), VJ_ERR_ARG, "beam[%lld] out of range",
                           (long long)q);
                mx = std::max(mx, (int)beam[q]);
            }
            ix->plan_beam.ensure(nq, s);
            VJ_CUDA(cudaMemcpyAsync(ix->plan_beam.p, beam, nq * sizeof(int32_t), cudaMemcpyHostToDevice, s));
            ix->plan_max_beam = mx;
            ix->has_beam = true;
        }
        VJ_CUDA(cudaStreamSynchronize(s));
    });
}

// Host results live in page-locked memory (device-to-host copies at full link
// speed) from a process-wide cache of blocks in power-of-two size classes, so
// repeated joins do not pay for cudaMallocHost.  At most 8 GiB stay cached.
namespace {
std::mutex g_pin_mu;
std::multimap<size_t, void*> g_pin_free;      // class bytes -> cached block
std::unordered_map<void*, size_t> g_pin_class;  // every live or cached block
size_t g_pin_cached = 0;
constexpr size_t PIN_CACHE_MAX = (size_t)8 << 30;

void* pin_alloc(size_t bytes) {
    size_t c = 4096;
    while (c < bytes) c <<= 1;
    std::lock_guard<std::mutex> lk(g_pin_mu);
    auto it = g_pin_free.find(c);
    if (it != g_pin_free.end()) {
        void* p = it->second;
        g_pin_free.erase(it);
        g_pin_cached -= c;
        return p;
    }
    void* p = nullptr;
    if (cudaMallocHost(&p, c) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    g_pin_class[p] = c;
    return p;
}

void pin_free(void* p) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(g_pin_mu);
    auto it = g_pin_class.find(p);
    if (it == g_pin_class.end()) return;
    const size_t c = it->second;
    if (g_pin_cached + c <= PIN_CACHE_MAX) {
        g_pin_free.emplace(c, p);
        g_pin_cached += c;
    } else {
        g_pin_class.erase(it);
        cudaFreeHost(p);
    }
}
}  // namespace

static vj_result* new_result(int64_t nq, int64_t nnz, bool on_device, cudaStream_t s) {
    vj_result* r = (vj_result*)calloc(1, sizeof(vj_result));
    if (!r) throw std::bad_alloc();
    r->nq = nq;
    r->nnz = nnz;
    r->on_device = on_device ? 1 : 0;
    size_t b_off = (nq + 1) * sizeof(int64_t), b_id = std::max<int64_t>(nnz, 1) * sizeof(int32_t),
           b_d = std::max<int64_t>(nnz, 1) * sizeof(float), b_q = nq * sizeof(int32_t), b_h = nq;
    if (on_device) {
        cudaError_t e = cudaSuccess;
        e = e ? e : cudaMallocAsync((void**)&r->offsets, b_off, s);
        e = e ? e : cudaMallocAsync((void**)&r->ids, b_id, s);
        e = e ? e : cudaMallocAsync((void**)&r->dists, b_d, s);
        e = e ? e : cudaMallocAsync((void**)&r->steps, b_q, s);
        e = e ? e : cudaMallocAsync((void**)&r->cache, b_q, s);
        e = e ? e : cudaMallocAsync((void**)&r->hybrid, b_h, s);
        if (e != cudaSuccess) {
            vj_set_error("result allocation failed: %s", cudaGetErrorString(e));
            vj_result_free(r);
            throw VjError{VJ_ERR_OOM};
        }
    } else {
        r->offsets = (int64_t*)pin_alloc(b_off);
        r->ids = (int32_t*)pin_alloc(b_id);
        r->dists = (float*)pin_alloc(b_d);
        r->steps = (int32_t*)pin_alloc(b_q);
        r->cache = (int32_t*)pin_alloc(b_q);
        r->hybrid = (uint8_t*)pin_alloc(std::max<size_t>(b_h, 1));
        if (!r->offsets || !r->ids || !r->dists || !r->steps || !r->cache || !r->hybrid) {
            vj_result_free(r);
            vj_set_error("page-locked result allocation failed");
            throw VjError{VJ_ERR_OOM};
        }
    }
    return r;
}

static vj_status join_impl(vj_index* ix, float eps, int budget, vj_result** out, bool on_device) {
    if (out) *out = nullptr;
    return guarded([&] {
        VJ_REQUIRE(ix != nullptr && out != nullptr, VJ_ERR_ARG, "NULL argument");
        VJ_REQUIRE(eps > 0.f && eps == eps, VJ_ERR_ARG, "eps must be > 0");
        cudaStream_t s = ix->stream;
        vj_stats st;
        memset(&st, 0, sizeof(st));
        int64_t nnz = 0;
        vj_run_join(ix, eps, budget, &st, &nnz);
        vj_result* r = new_result(ix->nq, nnz, on_device, s);
        cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        cudaError_t e = cudaSuccess;
        e = e ? e : cudaMemcpyAsync(r->offsets, ix->offsets.p, (ix->nq + 1) * sizeof(int64_t), k, s);
        if (nnz > 0) {
            e = e ? e : cudaMemcpyAsync(r->ids, ix->out_id.p, nnz * sizeof(int32_t), k, s);
            e = e ? e : cudaMemcpyAsync(r->dists, ix->out_d.p, nnz * sizeof(float), k, s);
        }
        e = e ? e : cudaMemcpyAsync(r->steps, ix->steps.p, ix->nq * sizeof(int32_t), k, s);
        e = e ? e : cudaMemcpyAsync(r->cache, ix->cache.p, ix->nq * sizeof(int32_t), k, s);
        e = e ? e : cudaMemcpyAsync(r->hybrid, ix->hyb.p, ix->nq, k, s);
        e = e ? e : cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            vj_result_free(r);
            vj_set_error("result copy failed: %s", cudaGetErrorString(e));
            throw VjError{VJ_ERR_CUDA};
        }
        r->stats = st;
        *out = r;
    });
}

extern "C" vj_status vj_export_nnmap(const vj_index* ix, int32_t* witness, double* wdist, uint8_t* ood) {
    return guarded([&] {
        VJ_REQUIRE(ix != nullptr, VJ_ERR_ARG, "index is NULL");
        VJ_REQUIRE(ix->nnmap, VJ_ERR_STATE, "the index was built without nnmap");
        cudaStream_t s = ix->stream;
        if (witness)
            VJ_CUDA(cudaMemcpyAsync(witness, ix->nm_w.p, ix->nq * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        if (wdist) VJ_CUDA(cudaMemcpyAsync(wdist, ix->nm_wd.p, ix->nq * sizeof(double), cudaMemcpyDeviceToHost, s));
        if (ood) VJ_CUDA(cudaMemcpyAsync(ood, ix->nm_ood.p, ix->nq, cudaMemcpyDeviceToHost, s));
        VJ_CUDA(cudaStreamSynchronize(s));
    });
}

// Query-data switching: the join on an index built with the sets' roles
// swapped, transposed back to one row per original query
extern "C" vj_status vj_join_switched(vj_index* ix, float eps, vj_result** out) {
    if (out) *out = nullptr;
    return guarded([&] {
        VJ_REQUIRE(ix != nullptr && out != nullptr, VJ_ERR_ARG, "NULL argument");
        VJ_REQUIRE(eps > 0.f && eps == eps, VJ_ERR_ARG, "eps must be > 0");
        cudaStream_t s = ix->stream;
        vj_stats st;
        memset(&st, 0, sizeof(st));
        int64_t nnz = 0;
        vj_run_join(ix, eps, 0, &st, &nnz);
        DBuf<int64_t> toff;
        DBuf<int32_t> tid;
        DBuf<float> td;
        vj_csr_transpose(ix, ix->offsets.p, ix->nq, ix->out_id.p, ix->out_d.p, nnz, ix->nx, toff, tid, td);
        vj_result* r = new_result(ix->nx, nnz, false, s);
        cudaError_t e = cudaMemcpyAsync(r->offsets, toff.p, (ix->nx + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s);
        if (nnz > 0) {
            e = e ? e : cudaMemcpyAsync(r->ids, tid.p, nnz * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
            e = e ? e : cudaMemcpyAsync(r->dists, td.p, nnz * sizeof(float), cudaMemcpyDeviceToHost, s);
        }
        e = e ? e : cudaStreamSynchronize(s);
        toff.free_(s);
        tid.free_(s);
        td.free_(s);
        if (e != cudaSuccess) {
            vj_result_free(r);
            vj_set_error("result copy failed: %s", cudaGetErrorString(e));
            throw VjError{VJ_ERR_CUDA};
        }
        // per-query outputs of the swapped join belong to the other set
        memset(r->steps, 0, ix->nx * sizeof(int32_t));
        memset(r->cache, 0xff, ix->nx * sizeof(int32_t));
        memset(r->hybrid, 0, ix->nx);
        r->stats = st;
        *out = r;
    });
}

extern "C" vj_status vj_join(vj_index* ix, float eps, int budget, vj_result** out) {
    return join_impl(ix, eps, budget, out, false);
}

extern "C" vj_status vj_join_device(vj_index* ix, float eps, int budget, vj_result** out) {
    return join_impl(ix, eps, budget, out, true);
}

// Many independent joins (a collection of instances of very different
// sizes).  One instance rarely fills 148 SMs, so the traversal passes of all
// instances run fused, one launch per pass over every instance
// (vj_run_join_multi); the per-instance setup (prologue, buffers) and finish
// (brute-force rows, CSR, result copy) run on up to BATCH_WORKERS host
// threads, each instance on its own index's stream.  Each instance's result
// is the one vj_join gives for it alone.
static constexpr int BATCH_WORKERS = 8;

// fn(0..n-1) on up to BATCH_WORKERS threads; rethrows the lowest failing
// index's error (as "instance i: ...") after all calls ended
static void batch_par_for(int n, const std::function<void(int)>& fn) {
    int dev = 0;
    VJ_CUDA(cudaGetDevice(&dev));
    std::vector<vj_status> st(n, VJ_OK);
    std::vector<std::string> msg(n);
    std::atomic<int> next{0};
    auto work = [&] {
        const bool dev_ok = cudaSetDevice(dev) == cudaSuccess;
        for (int i; (i = next.fetch_add(1)) < n;) {
            if (!dev_ok) {
                st[i] = VJ_ERR_CUDA;
                msg[i] = "cudaSetDevice failed on a worker thread";
                continue;
            }
            st[i] = guarded([&] { fn(i); });
            if (st[i] != VJ_OK) msg[i] = vj_last_error();
        }
    };
    const int nw = std::min(n, BATCH_WORKERS);
    std::vector<std::thread> pool;
    pool.reserve(std::max(nw - 1, 0));
    for (int t = 1; t < nw; t++) pool.emplace_back(work);
    work();
    for (auto& t : pool) t.join();
    for (int i = 0; i < n; i++)
        if (st[i] != VJ_OK) {
            vj_set_error("instance %d: %s", i, msg[i].c_str());
            throw VjError{st[i]};
        }
}

extern "C" vj_status vj_join_batch(vj_index** ixs, const float* eps, int n, vj_result** outs) {
    return guarded([&] {
        VJ_REQUIRE(n >= 0, VJ_ERR_ARG, "n must be >= 0");
        if (n == 0) return;
        VJ_REQUIRE(ixs != nullptr && eps != nullptr && outs != nullptr, VJ_ERR_ARG, "NULL argument");
        for (int i = 0; i < n; i++) outs[i] = nullptr;
        for (int i = 0; i < n; i++) {
            VJ_REQUIRE(ixs[i] != nullptr, VJ_ERR_ARG, "index %d is NULL", i);
            VJ_REQUIRE(eps[i] > 0.f && eps[i] == eps[i], VJ_ERR_ARG, "eps[%d] must be > 0", i);
        }
        std::vector<vj_index*> uniq(ixs, ixs + n);
        std::sort(uniq.begin(), uniq.end());
        VJ_REQUIRE(std::adjacent_find(uniq.begin(), uniq.end()) == uniq.end(), VJ_ERR_ARG,
                   "an index appears twice in the batch");
        std::vector<vj_stats> st(n);
        memset(st.data(), 0, sizeof(vj_stats) * n);
        std::vector<int64_t> nnz(n, 0);
        std::vector<vj_result*> res(n, nullptr);
        try {
            vj_run_join_multi(ixs, eps, n, st.data(), nnz.data(), batch_par_for);
            batch_par_for(n, [&](int i) {
                vj_index* ix = ixs[i];
                cudaStream_t s = ix->stream;
                vj_result* r = new_result(ix->nq, nnz[i], false, s);
                res[i] = r;
                const cudaMemcpyKind k = cudaMemcpyDeviceToHost;
                VJ_CUDA(cudaMemcpyAsync(r->offsets, ix->offsets.p, (ix->nq + 1) * sizeof(int64_t), k, s));
                if (nnz[i] > 0) {
                    VJ_CUDA(cudaMemcpyAsync(r->ids, ix->out_id.p, nnz[i] * sizeof(int32_t), k, s));
                    VJ_CUDA(cudaMemcpyAsync(r->dists, ix->out_d.p, nnz[i] * sizeof(float), k, s));
                }
                VJ_CUDA(cudaMemcpyAsync(r->steps, ix->steps.p, ix->nq * sizeof(int32_t), k, s));
                VJ_CUDA(cudaMemcpyAsync(r->cache, ix->cache.p, ix->nq * sizeof(int32_t), k, s));
                VJ_CUDA(cudaMemcpyAsync(r->hybrid, ix->hyb.p, ix->nq, k, s));
                VJ_CUDA(cudaStreamSynchronize(s));
                r->stats = st[i];
            });
        } catch (...) {
            for (auto* r : res) vj_result_free(r);
            throw;
        }
        for (int i = 0; i < n; i++) outs[i] = res[i];
    });
}

extern "C" vj_status vj_join_exact(vj_index* ix, float eps, vj_result** out) {
    if (out) *out = nullptr;
    return guarded([&] {
        VJ_REQUIRE(ix != nullptr && out != nullptr, VJ_ERR_ARG, "NULL argument");
        VJ_REQUIRE(eps > 0.f && eps == eps, VJ_ERR_ARG, "eps must be > 0");
        cudaStream_t s = ix->stream;
        DBuf<int64_t> off;
        DBuf<int32_t> ids;
        DBuf<float> dd;
        int64_t nnz = 0;
        double ms = 0.0;
        vj_exact_join_device(ix, eps, off, ids, dd, &nnz, &ms);
        vj_result* r = new_result(ix->nq, nnz, false, s);
        VJ_CUDA(cudaMemcpyAsync(r->offsets, off.p, (ix->nq + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        if (nnz > 0) {
            VJ_CUDA(cudaMemcpyAsync(r->ids, ids.p, nnz * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
            VJ_CUDA(cudaMemcpyAsync(r->dists, dd.p, nnz * sizeof(float), cudaMemcpyDeviceToHost, s));
        }
        VJ_CUDA(cudaStreamSynchronize(s));
        memset(r->steps, 0, ix->nq * sizeof(int32_t));
        memset(r->cache, 0xff, ix->nq * sizeof(int32_t));
        memset(r->hybrid, 0, ix->nq);
        r->stats.ms_total = ms;
        r->stats.ms_scan = ix->last_scan_ms;
        r->stats.scan_candidates = ix->last_scan_cand;
        r->stats.dist_computations = ix->nx * ix->nq;
        off.free_(s);
        ids.free_(s);
        dd.free_(s);
        *out = r;
    });
}

extern "C" vj_status vj_export_graph(const vj_index* ix, int32_t* adj, int32_t* entry, int32_t* parent,
                                     int32_t* order, int32_t* depth) {
    return guarded([&] {
        VJ_REQUIRE(ix != nullptr, VJ_ERR_ARG, "index is NULL");
        cudaStream_t s = ix->stream;
        if (adj)
            VJ_CUDA(cudaMemcpyAsync(adj, ix->adj.p, (size_t)ix->n * ix->R * sizeof(int32_t), cudaMemcpyDeviceToHost,
                                    s));
        if (parent) VJ_CUDA(cudaMemcpyAsync(parent, ix->parent.p, ix->nq * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        if (order) VJ_CUDA(cudaMemcpyAsync(order, ix->order.p, ix->nq * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        if (depth) VJ_CUDA(cudaMemcpyAsync(depth, ix->depth.p, ix->nq * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        VJ_CUDA(cudaStreamSynchronize(s));
        if (entry) *entry = ix->entry;
    });
}

extern "C" vj_status vj_export_knn(const vj_index* ix, int32_t* ids, float* dists) {
    return guarded([&] {
        VJ_REQUIRE(ix != nullptr, VJ_ERR_ARG, "index is NULL");
        cudaStream_t s = ix->stream;
        if (ids)
            VJ_CUDA(cudaMemcpyAsync(ids, ix->knn.p, (size_t)ix->n * ix->K * sizeof(int32_t), cudaMemcpyDeviceToHost,
                                    s));
        if (dists)
            VJ_CUDA(cudaMemcpyAsync(dists, ix->knnd.p, (size_t)ix->n * ix->K * sizeof(float),
                                    cudaMemcpyDeviceToHost, s));
        VJ_CUDA(cudaStreamSynchronize(s));
    });
}

extern "C" vj_status vj_index_info(const vj_index* ix, int64_t* nx, int64_t* nq, int* d, int* degree, int* knn_k,
                                   int* max_depth) {
    return guarded([&] {
        VJ_REQUIRE(ix != nullptr, VJ_ERR_ARG, "index is NULL");
        if (nx) *nx = ix->nx;
        if (nq) *nq = ix->nq;
        if (d) *d = ix->d;
        if (degree) *degree = ix->R;
        if (knn_k) *knn_k = ix->K;
        if (max_depth) *max_depth = ix->max_depth;
    });
}

extern "C" vj_status vj_build_info(const vj_index* ix, int* knn_tensor_cores, int64_t* knn_uncertified,
                                   double* ms_build, double* ms_knn) {
    return guarded([&] {
        VJ_REQUIRE(ix != nullptr, VJ_ERR_ARG, "index is NULL");
        if (knn_tensor_cores) *knn_tensor_cores = ix->knn_tc ? 1 : 0;
        if (knn_uncertified) *knn_uncertified = ix->knn_uncertified;
        if (ms_build) *ms_build = ix->ms_build;
        if (ms_knn) *ms_knn = ix->ms_knn;
    });
}

extern "C" void vj_result_free(vj_result* r) {
    if (!r) return;
    if (r->on_device) {
        cudaFree(r->offsets);
        cudaFree(r->ids);
        cudaFree(r->dists);
        cudaFree(r->steps);
        cudaFree(r->cache);
        cudaFree(r->hybrid);
    } else {
        pin_free(r->offsets);
        pin_free(r->ids);
        pin_free(r->dists);
        pin_free(r->steps);
        pin_free(r->cache);
        pin_free(r->hybrid);
    }
    free(r);
}

extern "C" void vj_free(vj_index* ix) { free_index(ix); }
