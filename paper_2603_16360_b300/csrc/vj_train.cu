// vj_train.cu -- labels for the learned route / budget predictor and its
// training, behind vj_predictor_labels / vj_train_predictor.
//
// The paper decides per query with the d1/d2 > 1.5 rule only (Sec. 4.4); the
// predictor and these labels are this library's own.  For a set of training
// queries of an index (rows of its query set, kept apart from the queries a
// caller evaluates on):
//   1. their exact rows at eps, from the tensor-core scan with the exact
//      re-check (the nested-loop join of Sec. 3.2);
//   2. one join per ladder budget, every query planned with that budget
//      (-1 no expansion, 0 BFS, > 0 hybrid queue size): per training query its
//      row's recall against the exact row and its cost, the distance
//      evaluations it made;
//   3. budget label: the first ladder budget whose recall reaches
//      query_recall (else the last budget that ran);
//   4. route labels: queries whose cost at their budget is at least the cost
//      of a brute-force row are routed; then, while the training queries'
//      pooled recall is below pooled_recall, the query with the most missed
//      pairs per unit of extra cost (missed / (scan_row_cost - cost), ties by
//      query index) is routed.
// Training: features of every query at eps (vj_features), the training rows
// with targets log2(budget + 2) and route, Adam (vj_mlp_train).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <numeric>
#include <vector>

#include "vj_internal.cuh"

extern "C" void vj_default_train_params(vj_train_params* tp) {
    if (!tp) return;
    memset(tp, 0, sizeof(*tp));
    tp->n_ladder = 3;
    tp->ladder[0] = -1;
    tp->ladder[1] = 0;
    tp->ladder[2] = 8;
    tp->query_recall = 0.95f;
    tp->pooled_recall = 0.955f;
    tp->scan_row_cost = 0.f;
    tp->h1 = 256;
    tp->h2 = 256;
    tp->epochs = 30;
    tp->batch = 256;
    tp->lr = 1e-3f;
    tp->seed = 7;
}

namespace {

// out[i] = the rows[i]-th row of src (rows of w floats)
__global__ void k_gather_rows(const float* __restrict__ src, const int32_t* __restrict__ rows, int64_t n, int w,
                              float* __restrict__ out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * w) return;
    const int64_t i = e / w;
    out[e] = src[(int64_t)rows[i] * w + (e - i * w)];
}

// |a n b| of two ascending id lists
int64_t sorted_overlap(const int32_t* a, int64_t na, const int32_t* b, int64_t nb) {
    int64_t i = 0, j = 0, c = 0;
    while (i < na && j < nb) {
        if (a[i] < b[j]) i++;
        else if (b[j] < a[i]) j++;
        else {
            c++;
            i++;
            j++;
        }
    }
    return c;
}

struct Labels {
    std::vector<int32_t> budget;
    std::vector<uint8_t> route;
    double scan_row_cost = 0.0;
    int ladder_run = 0;  // ladder entries whose join completed
};

// the index's plan / join settings, restored when labelling ends
struct PlanGuard {
    vj_index* ix;
    vj_params p;
    explicit PlanGuard(vj_index* i) : ix(i), p(i->p) {}
    ~PlanGuard() {
        vj_set_plan(ix, nullptr, nullptr);
        ix->p = p;
    }
};

void check_train_args(vj_index* ix, float eps, const int32_t* rows, int64_t n, const vj_train_params* tp) {
    VJ_REQUIRE(ix && rows && tp && n >= 1, VJ_ERR_ARG, "NULL argument or no training rows");
    VJ_REQUIRE(!ix->nnmap, VJ_ERR_STATE, "an NN-Map index joins from its witnesses: nothing to plan or train");
    VJ_REQUIRE(eps > 0.f && eps == eps, VJ_ERR_ARG, "eps must be > 0");
    VJ_REQUIRE(tp->n_ladder >= 1 && tp->n_ladder <= 8, VJ_ERR_ARG, "n_ladder must be 1..8");
    for (int k = 0; k < tp->n_ladder; k++)
        VJ_REQUIRE(tp->ladder[k] >= -1 && tp->ladder[k] <= (1 << 20), VJ_ERR_ARG, "ladder[%d] out of range", k);
    VJ_REQUIRE(tp->query_recall > 0.f && tp->query_recall <= 1.f, VJ_ERR_ARG, "query_recall must be in (0, 1]");
    VJ_REQUIRE(tp->pooled_recall > 0.f && tp->pooled_recall <= 1.f, VJ_ERR_ARG, "pooled_recall must be in (0, 1]");
    for (int64_t i = 0; i < n; i++)
        VJ_REQUIRE(rows[i] >= 0 && rows[i] < ix->nq, VJ_ERR_ARG, "rows[%lld] out of range", (long long)i);
}

Labels make_labels(vj_index* ix, float eps, const int32_t* rows, int64_t n, const vj_train_params* tp) {
    cudaStream_t s = ix->stream;
    const int64_t nq = ix->nq;
    Labels L;
    // 1. exact rows of the training queries
    DBuf<int32_t> drows;
    drows.alloc(n, s);
    VJ_CUDA(cudaMemcpyAsync(drows.p, rows, n * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    DBuf<int64_t> eoff;
    DBuf<int32_t> eid;
    DBuf<float> ed;
    int64_t enz = 0;
    double ms_scan = 0.0;
    vj_scan_rows_csr(ix, drows.p, n, eps, eoff, eid, ed, &enz, &ms_scan, true);
    std::vector<int64_t> xo(nq + 1);
    std::vector<int32_t> xi(std::max<int64_t>(enz, 1));
    VJ_CUDA(cudaMemcpyAsync(xo.data(), eoff.p, (nq + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    if (enz > 0) VJ_CUDA(cudaMemcpyAsync(xi.data(), eid.p, enz * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    VJ_CUDA(cudaStreamSynchronize(s));
    const double scan_ms_per_row = ms_scan / (double)n;
    drows.free_(s);
    eoff.free_(s);
    eid.free_(s);
    ed.free_(s);

    // 2. one planned join per ladder budget
    const int nl = tp->n_ladder;
    std::vector<std::vector<float>> rec(nl, std::vector<float>(n, 1.f));
    std::vector<std::vector<float>> miss(nl, std::vector<float>(n, 0.f));
    std::vector<std::vector<int32_t>> cost(nl, std::vector<int32_t>(n, 0));
    double ms_per_dist = 0.0;
    {
        PlanGuard guard(ix);
        ix->p.learned = 0;
        std::vector<int32_t> plan(nq);
        std::vector<int64_t> ro(nq + 1);
        std::vector<int32_t> ri, steps(nq);
        for (int k = 0; k < nl; k++) {
            std::fill(plan.begin(), plan.end(), tp->ladder[k]);
            VJ_REQUIRE(vj_set_plan(ix, nullptr, plan.data()) == VJ_OK, VJ_ERR_STATE, "labels: plan rejected");
            vj_stats st;
            memset(&st, 0, sizeof(st));
            int64_t nnz = 0;
            try {
                vj_run_join(ix, eps, 0, &st, &nnz);
            } catch (const VjError& e) {
                // a budget this workload cannot run (e.g. a hybrid search that
                // outgrows its visited set) ends the ladder; the entries that
                // ran so far label the queries
                VJ_REQUIRE(k > 0, e.code, "labels: the first ladder join failed: %s", vj_last_error());
                break;
            }
            ri.resize(std::max<int64_t>(nnz, 1));
            VJ_CUDA(cudaMemcpyAsync(ro.data(), ix->offsets.p, (nq + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
            if (nnz > 0)
                VJ_CUDA(cudaMemcpyAsync(ri.data(), ix->out_id.p, nnz * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
            VJ_CUDA(cudaMemcpyAsync(steps.data(), ix->steps.p, nq * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
            VJ_CUDA(cudaStreamSynchronize(s));
            for (int64_t i = 0; i < n; i++) {
                const int32_t q = rows[i];
                const int64_t tot = xo[q + 1] - xo[q];
                const int64_t hit =
                    sorted_overlap(ri.data() + ro[q], ro[q + 1] - ro[q], xi.data() + xo[q], tot);
                rec[k][i] = tot > 0 ? (float)((double)hit / (double)tot) : 1.f;
                miss[k][i] = (float)(tot - hit);
                cost[k][i] = steps[q];
            }
            if (tp->ladder[k] == 0 && st.dist_computations > 0) ms_per_dist = st.ms_traverse / st.dist_computations;
            L.ladder_run = k + 1;
        }
    }
    // 3. budget labels
    const int nr = L.ladder_run;
    std::vector<int> pick(n, nr - 1);
    L.budget.assign(n, tp->ladder[nr - 1]);
    for (int64_t i = 0; i < n; i++)
        for (int k = 0; k < nr; k++)
            if (rec[k][i] >= tp->query_recall) {
                pick[i] = k;
                L.budget[i] = tp->ladder[k];
                break;
            }
    // 4. route labels: a knapsack on missed pairs per unit of extra cost
    double c_scan = tp->scan_row_cost;
    if (!(c_scan > 0.0)) {
        // measured: one scanned row in units of the BFS join's distance evaluations
        c_scan = ms_per_dist > 0.0 ? scan_ms_per_row / ms_per_dist : (double)ix->nx;
    }
    L.scan_row_cost = c_scan;
    L.route.assign(n, 0);
    double tot_all = 0.0, missed = 0.0;
    std::vector<double> gain(n);
    for (int64_t i = 0; i < n; i++) {
        const int32_t q = rows[i];
        tot_all += (double)(xo[q + 1] - xo[q]);
        const double c = cost[pick[i]][i], m = miss[pick[i]][i];
        if (c >= c_scan) {
            L.route[i] = 1;  // a brute-force row is cheaper and exact
        } else {
            missed += m;
            gain[i] = m / std::max(c_scan - c, 1e-9);
        }
    }
    const double allowed = (1.0 - (double)tp->pooled_recall) * tot_all;
    if (missed > allowed) {
        std::vector<int64_t> ord;
        for (int64_t i = 0; i < n; i++)
            if (!L.route[i] && miss[pick[i]][i] > 0.f) ord.push_back(i);
        std::stable_sort(ord.begin(), ord.end(), [&](int64_t a, int64_t b) {
            if (gain[a] != gain[b]) return gain[a] > gain[b];
            return rows[a] < rows[b];
        });
        for (int64_t i : ord) {
            if (missed <= allowed) break;
            L.route[i] = 1;
            missed -= miss[pick[i]][i];
        }
    }
    return L;
}

void fill_report(vj_train_report* rep, const Labels& L, const vj_train_params* tp, int64_t n) {
    if (!rep) return;
    rep->n = n;
    rep->routed = std::accumulate(L.route.begin(), L.route.end(), (int64_t)0);
    for (int k = 0; k < 8; k++) rep->per_budget[k] = 0;
    for (int64_t i = 0; i < n; i++)
        for (int k = 0; k < tp->n_ladder; k++)
            if (L.budget[i] == tp->ladder[k]) {
                rep->per_budget[k]++;
                break;
            }
    rep->scan_row_cost = L.scan_row_cost;
    rep->ladder_run = L.ladder_run;
}

double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace

extern "C" vj_status vj_predictor_labels(vj_index* ix, float eps, const int32_t* rows, int64_t n,
                                         const vj_train_params* tp, int32_t* budget, uint8_t* route,
                                         vj_train_report* rep) {
    try {
        check_train_args(ix, eps, rows, n, tp);
        VJ_REQUIRE(budget && route, VJ_ERR_ARG, "NULL output");
        const double t0 = now_ms();
        Labels L = make_labels(ix, eps, rows, n, tp);
        std::copy(L.budget.begin(), L.budget.end(), budget);
        std::copy(L.route.begin(), L.route.end(), route);
        if (rep) {
            memset(rep, 0, sizeof(*rep));
            fill_report(rep, L, tp, n);
            rep->ms_labels = now_ms() - t0;
        }
        return VJ_OK;
    } catch (const VjError& e) {
        return e.code;
    } catch (const std::bad_alloc&) {
        vj_set_error("host allocation failed");
        return VJ_ERR_OOM;
    }
}

extern "C" vj_status vj_train_predictor(vj_index* ix, float eps, const int32_t* rows, int64_t n,
                                        const vj_train_params* tp, vj_mlp** out, vj_train_report* rep) {
    if (out) *out = nullptr;
    vj_mlp* m = nullptr;
    try {
        check_train_args(ix, eps, rows, n, tp);
        VJ_REQUIRE(out, VJ_ERR_ARG, "NULL output");
        VJ_REQUIRE(tp->h1 >= 1 && tp->h2 >= 1 && tp->epochs >= 1 && tp->batch >= 1 && tp->lr > 0.f, VJ_ERR_ARG,
                   "bad training parameters");
        const double t0 = now_ms();
        Labels L = make_labels(ix, eps, rows, n, tp);
        const double t1 = now_ms();
        // features of every query, the training rows gathered on the host
        cudaStream_t s = ix->stream;
        const int din = VJ_NFEAT + ix->d;
        DBuf<float> f, g;
        DBuf<int32_t> drows;
        f.alloc((size_t)ix->nq * din, s);
        g.alloc((size_t)n * din, s);
        drows.alloc(n, s);
        vj_compute_features(ix, eps, f.p);
        VJ_CUDA(cudaMemcpyAsync(drows.p, rows, n * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        k_gather_rows<<<vj_div_up((int64_t)n * din, 256), 256, 0, s>>>(f.p, drows.p, n, din, g.p);
        VJ_LAUNCH_CHECK();
        std::vector<float> x((size_t)n * din), tr(n), tc(n);
        VJ_CUDA(cudaMemcpyAsync(x.data(), g.p, (size_t)n * din * sizeof(float), cudaMemcpyDeviceToHost, s));
        VJ_CUDA(cudaStreamSynchronize(s));
        f.free_(s);
        g.free_(s);
        drows.free_(s);
        for (int64_t i = 0; i < n; i++) {
            tr[i] = (float)log2((double)L.budget[i] + 2.0);
            tc[i] = (float)L.route[i];
        }
        vj_status st = vj_mlp_create(din, tp->h1, tp->h2, tp->seed, &m);
        VJ_REQUIRE(st == VJ_OK, st, "%s", vj_last_error());
        double loss = 0.0;
        st = vj_mlp_train(m, x.data(), tr.data(), tc.data(), n, tp->epochs, tp->batch, tp->lr, tp->seed, &loss);
        VJ_REQUIRE(st == VJ_OK, st, "%s", vj_last_error());
        if (rep) {
            memset(rep, 0, sizeof(*rep));
            fill_report(rep, L, tp, n);
            rep->final_loss = loss;
            rep->ms_labels = t1 - t0;
            rep->ms_train = now_ms() - t1;
        }
        *out = m;
        return VJ_OK;
    } catch (const VjError& e) {
        if (m) vj_mlp_free(m);
        return e.code;
    } catch (const std::bad_alloc&) {
        if (m) vj_mlp_free(m);
        vj_set_error("host allocation failed");
        return VJ_ERR_OOM;
    }
}
