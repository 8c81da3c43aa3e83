// autotune.cu -- picks gp_options for one graph by timing candidates on the device.
//
// Correctness never depends on the options; only speed does.  The tuner runs
// coordinate descent over small candidate sets, timing each candidate with
// CUDA events on the caller's stream (the faster of two timings), and repeats
// the pull and the push descent once when a pass changed something (the
// coordinates interact: the best resident-block count depends on the size of
// the shared-memory accumulators, for instance):
//   pull PageRank: pull_light_max, then chunk_edges, then pull_hot_slots
//                  (a few sweeps of gp_pagerank(GP_PULL) per candidate);
//   push PageRank: push_light_max, then blocks_per_sm, then push_hot_slots;
//   AUTO:          pr_auto_mode = whichever of pull and push sweeps faster
//                  (the per-graph push/pull choice of the Generic-Switch idea, Section 5);
//   BFS:           bfs_light_max, then bfs_alpha, then bfs_beta (gp_bfs(GP_AUTO)
//                  from the given sources), then bfs_groups (one gp_bfs_multi
//                  over a batch of 64 searches, the given sources repeated).
// The best options are left set on the graph and returned.
#include <algorithm>
#include <cstring>
#include <vector>

#include "gp_internal.cuh"

using namespace gp;

namespace {

struct Timer {
    cudaEvent_t a = nullptr, b = nullptr;
    Timer() {
        cudaEventCreate(&a);
        cudaEventCreate(&b);
    }
    ~Timer() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

constexpr int TUNE_WARM = 2, TUNE_SWEEPS = 6, TUNE_REPS = 2, TUNE_PASSES = 2;

// Milliseconds per sweep of gp_pagerank(mode) under the graph's current
// options: the fastest of TUNE_REPS timed runs.
int time_pr(gp_graph *g, int mode, float *out, cudaStream_t s, float &ms_per_sweep) {
    Timer t;
    int st = gp_pagerank(g, mode, 0.85f, TUNE_WARM, 0.0, nullptr, nullptr, out, nullptr, s);
    if (st != GP_OK) return st;
    float best = 0.f;
    for (int r = 0; r < TUNE_REPS; ++r) {
        GP_CUDA(cudaEventRecord(t.a, s));
        st = gp_pagerank(g, mode, 0.85f, TUNE_SWEEPS, 0.0, nullptr, nullptr, out, nullptr, s);
        if (st != GP_OK) return st;
        GP_CUDA(cudaEventRecord(t.b, s));
        GP_CUDA(cudaEventSynchronize(t.b));
        float ms = 0.f;
        GP_CUDA(cudaEventElapsedTime(&ms, t.a, t.b));
        if (r == 0 || ms < best) best = ms;
    }
    ms_per_sweep = best / TUNE_SWEEPS;
    return GP_OK;
}

int time_bfs(gp_graph *g, const int32_t *src, int nsrc, int32_t *level, cudaStream_t s, float &ms_total) {
    Timer t;
    int st = gp_bfs(g, src[0], GP_AUTO, level, nullptr, nullptr, s);
    if (st != GP_OK) return st;
    GP_CUDA(cudaEventRecord(t.a, s));
    for (int i = 0; i < nsrc && st == GP_OK; ++i) st = gp_bfs(g, src[i], GP_AUTO, level, nullptr, nullptr, s);
    if (st != GP_OK) return st;
    GP_CUDA(cudaEventRecord(t.b, s));
    GP_CUDA(cudaEventSynchronize(t.b));
    GP_CUDA(cudaEventElapsedTime(&ms_total, t.a, t.b));
    return GP_OK;
}

// Searches per gp_bfs_multi call when the group count is timed.
constexpr int TUNE_MULTI_SEARCHES = 64;

// Milliseconds of one gp_bfs_multi(GP_AUTO) over `src` with the graph's
// bfs_groups (one level vector per search): the faster of TUNE_REPS timed calls
// after one that sizes the workspace.  The calls fill summaries, so each waits
// for its searches and reports a barrier timeout at once.
int time_bfs_multi(gp_graph *g, const std::vector<int32_t> &src, int32_t *const *levels, cudaStream_t s, float &ms) {
    Timer t;
    const int k = (int)src.size();
    std::vector<gp_bfs_summary> sum((size_t)k);
    GP_TRY(gp_bfs_multi(g, src.data(), k, GP_AUTO, levels, nullptr, 0, sum.data(), s));
    float best = 0.f;
    for (int r = 0; r < TUNE_REPS; ++r) {
        GP_CUDA(cudaEventRecord(t.a, s));
        GP_TRY(gp_bfs_multi(g, src.data(), k, GP_AUTO, levels, nullptr, 0, sum.data(), s));
        GP_CUDA(cudaEventRecord(t.b, s));
        GP_CUDA(cudaEventSynchronize(t.b));
        float x = 0.f;
        GP_CUDA(cudaEventElapsedTime(&x, t.a, t.b));
        if (r == 0 || x < best) best = x;
    }
    ms = best;
    return GP_OK;
}

// Tries value v for the field at `field` (an int32 or float member of gp_options),
// keeping the best option set in `best` and the graph.
template <class T, class F>
int try_values(gp_graph *g, gp_options &best, float &best_ms, T gp_options::*field, const std::vector<T> &values,
               cudaStream_t s, F measure, int &evaluated) {
    for (T v : values) {
        if (best.*field == v) continue;
        gp_options cand = best;
        cand.*field = v;
        GP_TRY(gp_graph_set_options(g, &cand, s));
        float ms = 0.f;
        GP_TRY(measure(ms));
        ++evaluated;
        if (ms < best_ms) {
            best_ms = ms;
            best = cand;
        }
    }
    return gp_graph_set_options(g, &best, s);
}

}  // namespace

extern "C" int gp_autotune(gp_graph *g, unsigned what, const int32_t *sources, int nsources, gp_tune_result *res,
                           void *stream) {
    clear_error();
    if (!g) return set_error(GP_ERR_INVALID, "gp_autotune: graph is NULL");
    if ((what & GP_TUNE_BFS) && (!sources || nsources < 1))
        return set_error(GP_ERR_INVALID, "gp_autotune: BFS tuning needs at least one source");
    for (int i = 0; (what & GP_TUNE_BFS) && i < nsources; ++i)
        if (sources[i] < 0 || (int64_t)sources[i] >= g->n) return set_error(GP_ERR_INVALID, "gp_autotune: bad source");
    cudaStream_t s = (cudaStream_t)stream;
    if (res) memset(res, 0, sizeof(*res));
    if (g->n == 0) return GP_OK;
    DevBuf out, lvl;
    GP_TRY(dev_alloc(out, (size_t)g->n * sizeof(float), s));
    int st = dev_alloc(lvl, (size_t)g->n * sizeof(int32_t), s);
    if (st != GP_OK) {
        dev_free(out, s);
        return st;
    }
    gp_options best = g->opt;
    int evaluated = 0;
    float pull_ms = 0.f, push_ms = 0.f, bfs_ms = 0.f;
    auto pull = [&](float &ms) { return time_pr(g, GP_PULL, (float *)out.ptr, s, ms); };
    auto push = [&](float &ms) { return time_pr(g, GP_PUSH, (float *)out.ptr, s, ms); };
    auto bfs = [&](float &ms) { return time_bfs(g, sources, nsources, (int32_t *)lvl.ptr, s, ms); };
    if (st == GP_OK && (what & GP_TUNE_PULL)) {
        st = pull(pull_ms);
        ++evaluated;
        for (int pass = 0; pass < TUNE_PASSES && st == GP_OK; ++pass) {
            const gp_options before = best;
            st = try_values<int32_t>(g, best, pull_ms, &gp_options::pull_light_max, {8, 16, 32}, s, pull, evaluated);
            if (st == GP_OK) st = try_values<int32_t>(g, best, pull_ms, &gp_options::chunk_edges, {128, 256, 512}, s, pull, evaluated);
            if (st == GP_OK)
                st = try_values<int32_t>(g, best, pull_ms, &gp_options::pull_hot_slots, {0, 8192, 16384, 20480, 24576}, s, pull,
                                         evaluated);
            if (!memcmp(&before, &best, sizeof(best))) break;
        }
    }
    if (st == GP_OK && (what & GP_TUNE_PUSH)) {
        st = push(push_ms);
        ++evaluated;
        for (int pass = 0; pass < TUNE_PASSES && st == GP_OK; ++pass) {
            const gp_options before = best;
            st = try_values<int32_t>(g, best, push_ms, &gp_options::push_light_max, {8, 16, 32, 64}, s, push, evaluated);
            if (st == GP_OK) st = try_values<int32_t>(g, best, push_ms, &gp_options::blocks_per_sm, {4, 8, 12}, s, push, evaluated);
            if (st == GP_OK)
                st = try_values<int32_t>(g, best, push_ms, &gp_options::push_hot_slots,
                                         {0, 8192, 16384, 24576, 32768, 40960, 49152}, s, push, evaluated);
            if (!memcmp(&before, &best, sizeof(best))) break;
        }
    }
    if (st == GP_OK && (what & GP_TUNE_AUTO)) {
        if (!(what & GP_TUNE_PULL)) st = pull(pull_ms);
        if (st == GP_OK && !(what & GP_TUNE_PUSH)) st = push(push_ms);
        if (st == GP_OK) {
            best.pr_auto_mode = push_ms < pull_ms ? GP_PUSH : GP_PULL;
            st = gp_graph_set_options(g, &best, s);
        }
    }
    if (st == GP_OK && (what & GP_TUNE_BFS)) {
        st = bfs(bfs_ms);
        ++evaluated;
        if (st == GP_OK)
            st = try_values<int32_t>(g, best, bfs_ms, &gp_options::bfs_light_max, {8, 16, 32, 64, 128}, s, bfs, evaluated);
        if (st == GP_OK) st = try_values<float>(g, best, bfs_ms, &gp_options::bfs_alpha, {4.f, 8.f, 14.f, 24.f, 48.f}, s, bfs, evaluated);
        if (st == GP_OK) st = try_values<float>(g, best, bfs_ms, &gp_options::bfs_beta, {8.f, 24.f, 64.f}, s, bfs, evaluated);
        if (st == GP_OK) {
            // the group count of several searches per launch, on a batch of
            // TUNE_MULTI_SEARCHES searches with a level vector each (0 stands for
            // the library's 16)
            std::vector<int32_t> batch(TUNE_MULTI_SEARCHES);
            for (int i = 0; i < TUNE_MULTI_SEARCHES; ++i) batch[(size_t)i] = sources[i % nsources];
            DevBuf lv;
            if (dev_alloc(lv, (size_t)TUNE_MULTI_SEARCHES * (size_t)g->n * sizeof(int32_t), s) == GP_OK) {
                std::vector<int32_t *> ptr(TUNE_MULTI_SEARCHES);
                for (int i = 0; i < TUNE_MULTI_SEARCHES; ++i) ptr[(size_t)i] = (int32_t *)lv.ptr + (size_t)i * (size_t)g->n;
                float multi_ms = 0.f;
                auto multi = [&](float &ms) { return time_bfs_multi(g, batch, ptr.data(), s, ms); };
                st = multi(multi_ms);
                ++evaluated;
                if (st == GP_OK)
                    st = try_values<int32_t>(g, best, multi_ms, &gp_options::bfs_groups, {0, 1, 2, 4, 8, 32}, s, multi,
                                             evaluated);
                dev_free(lv, s);
            } else {
                clear_error();  // no room for the batch's level vectors: the count is left as it is
            }
        }
    }
    cudaError_t e = cudaStreamSynchronize(s);
    dev_free(out, s);
    dev_free(lvl, s);
    if (st != GP_OK) return st;
    if (e != cudaSuccess) return set_error(GP_ERR_CUDA, "gp_autotune: %s", cudaGetErrorString(e));
    if (res) {
        res->best = best;
        res->pull_ms_per_sweep = pull_ms;
        res->push_ms_per_sweep = push_ms;
        res->bfs_ms = bfs_ms;
        res->evaluated = evaluated;
    }
    return GP_OK;
}
