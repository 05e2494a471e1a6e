// Batches of models (mgt_batch_*) and the schedule autotuner (mgt_autotune).
//
// A batch runs the per-iteration work of many models in a few launches:
// line data of every point of every model; the formal solution of every
// (model, origin, line block) item in one persistent kernel per CTA width
// (bins x line groups of one origin, in warps: a model runs at its own width,
// so narrow models keep many CTAs per SM; within a width, items are taken from
// a global counter, models ordered from the most to the least work per item
// so that the short items fill the tail); and the statistical equilibrium of
// every point with per-model level counts.  mgt_batch_iterate captures the
// launches once in a CUDA graph and replays it per iteration.
//
// Each launch reads its per-model arguments from a device table.  The tables
// are rebuilt from the models before every batch call; when a model changed
// (new rays, new options) they are uploaded again and the graph is dropped.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "mgt_common.cuh"

struct mgt_batch {
    int device = 0;
    std::vector<mgt_model *> models;       // in the caller's order
    std::vector<int32_t> order;            // table slot -> caller index (most work per item first)
    // host copies of the argument tables, in table order
    std::vector<unsigned char> fs_args, se_args, ld_args;
    std::vector<int64_t> fs_end, se_end, ld_end;   // fs_end restarts at each class
    struct FsClass {
        int threads = 0, fused = 0, lines = 0, grid = 0, first = 0, count = 0;
        size_t smem = 0;
        int64_t items = 0;
        bool operator==(const FsClass &o) const
        {
            return threads == o.threads && fused == o.fused && lines == o.lines && grid == o.grid &&
                   first == o.first && count == o.count && smem == o.smem && items == o.items;
        }
    };
    std::vector<FsClass> fs_classes;               // in launch order, widest first
    std::vector<int32_t> fs_solo;                  // table slots launched on their own (large models)
    int64_t fs_solo_items = 0;
    size_t se_smem = 0;
    // device copies
    unsigned char *d_fs_args = nullptr, *d_se_args = nullptr, *d_ld_args = nullptr;
    int64_t *d_fs_end = nullptr, *d_se_end = nullptr, *d_ld_end = nullptr;
    unsigned long long *d_next = nullptr;          // one item counter per class
    int *h_err = nullptr;                          // pinned [n_models][4]: the models' device error words
    // the captured iteration
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int graph_kernels = 0;
};

namespace mgt {

namespace {

void drop_graph(mgt_batch *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

void free_batch(mgt_batch *b)
{
    drop_graph(b);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->h_err) cudaFreeHost(b->h_err);
    for (void *p : {(void *)b->d_fs_args, (void *)b->d_se_args, (void *)b->d_ld_args, (void *)b->d_fs_end,
                    (void *)b->d_se_end, (void *)b->d_ld_end, (void *)b->d_next})
        if (p) cudaFree(p);
    delete b;
}

template <typename X> mgt_status upload(X **d, const std::vector<X> &h, size_t cap_elems, cudaStream_t s)
{
    if (!*d) MGT_CUDA(cudaMalloc(d, sizeof(X) * cap_elems));
    MGT_CUDA(cudaMemcpyAsync(*d, h.data(), sizeof(X) * h.size(), cudaMemcpyHostToDevice, s));
    return MGT_OK;
}

// Work of one formal-solution item of model m (for the ordering only).
double item_cost(const mgt_model *m)
{
    const double steps_per_origin = (double)m->total_steps / (double)m->N;
    return steps_per_origin * m->Q * std::min<int32_t>(m->M, 40);
}

// Rebuild the argument tables from the models; upload them (and drop the
// graph) when anything changed.
mgt_status refresh(mgt_batch *b, cudaStream_t s)
{
    const int n = (int)b->models.size();
    for (mgt_model *m : b->models) MGT_TRY_STATUS(ensure_rays(m, MGT_FP32_MIXED, s));
    const size_t fsz = fs_args_bytes(), ssz = se_args_bytes(), lsz = ld_args_bytes();
    // each model's formal-solution arguments, CTA width and items (caller's order)
    std::vector<unsigned char> fa_c(fsz * n);
    std::vector<int> width(n), fused(n), lines(n);
    std::vector<int64_t> items(n);
    std::vector<double> cost(n);
    for (int i = 0; i < n; ++i) {
        MGT_TRY_STATUS(
            fs_batch_args(b->models[i], fa_c.data() + i * fsz, &width[i], &items[i], &fused[i], &lines[i]));
        cost[i] = item_cost(b->models[i]);
    }
    // A model of at least kSoloWaves waves of its persistent instance runs its
    // single-model launch instead: its tail is small anyway, and the
    // single-model kernel reads its arguments as constant operands, where the
    // persistent one holds them in registers (the same values either way).
    constexpr int64_t kSoloWaves = 8;
    std::vector<char> solo(n);
    for (int i = 0; i < n; ++i) {
        const size_t sm = fs_batch_smem(fa_c.data() + i * fsz, width[i]);
        const int64_t wave = fs_batch_wave(fa_c.data() + i * fsz, width[i], sm);
        solo[i] = wave > 0 && items[i] >= kSoloWaves * wave;
    }
    // order: the pooled models, widest CTAs first, unfused before fused at one
    // width, 8 lines per thread before 4, then most work per item, ties by
    // caller index; then the models launched on their own, most work first
    std::vector<int32_t> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) {
        if (solo[x] != solo[y]) return solo[x] < solo[y];
        if (solo[x]) return items[x] * cost[x] > items[y] * cost[y];
        if (width[x] != width[y]) return width[x] > width[y];
        if (fused[x] != fused[y]) return fused[x] < fused[y];
        if (lines[x] != lines[y]) return lines[x] > lines[y];
        return cost[x] > cost[y];
    });

    std::vector<unsigned char> fa(fsz * n), sa(ssz * n), la(lsz * n);
    std::vector<int64_t> fe(n), se(n), le(n);
    std::vector<mgt_batch::FsClass> classes;
    std::vector<int32_t> solo_slots;
    int64_t solo_items = 0;
    size_t se_smem = 0;
    int64_t si = 0, li = 0, fi = 0;
    for (int k = 0; k < n; ++k) {
        const int i = order[k];
        const mgt_model *m = b->models[i];
        std::memcpy(fa.data() + k * fsz, fa_c.data() + i * fsz, fsz);
        if (solo[i]) {
            solo_slots.push_back(k);
            solo_items += items[i];
            fe[k] = 0;
        } else {
            if (classes.empty() || classes.back().threads != width[i] || classes.back().fused != fused[i] ||
                classes.back().lines != lines[i]) {
                classes.emplace_back();
                classes.back().threads = width[i];
                classes.back().fused = fused[i];
                classes.back().lines = lines[i];
                classes.back().first = k;
                fi = 0;
            }
            mgt_batch::FsClass &c = classes.back();
            ++c.count;
            c.items = (fi += items[i]);
            c.smem = std::max(c.smem, fs_batch_smem(fa.data() + k * fsz, c.threads));
            fe[k] = fi;
        }
        int64_t sblocks = 0, lblocks = 0;
        size_t ssm = 0;
        MGT_TRY_STATUS(se_batch_args(m, sa.data() + k * ssz, &sblocks, &ssm));
        MGT_TRY_STATUS(ld_batch_args(m, la.data() + k * lsz, &lblocks));
        se_smem = std::max(se_smem, ssm);
        se[k] = (si += sblocks);
        le[k] = (li += lblocks);
    }
    if (li > 0x7fffffffLL || si > 0x7fffffffLL)
        return set_error(MGT_ERR_ARG, "batch: too many points for one launch");
    // each (chunk length, fused, lines per thread) runs its own instance of the
    // kernel: the shared-memory limit is set per instance, to its largest class
    auto instance = [](const mgt_batch::FsClass &c) {
        return ((c.threads == 32 && !c.fused) ? 4 : 0) + (c.fused ? 2 : 0) + (c.lines == 8 ? 1 : 0);
    };
    size_t max_smem[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (const mgt_batch::FsClass &c : classes) max_smem[instance(c)] = std::max(max_smem[instance(c)], c.smem);
    for (const mgt_batch::FsClass &c : classes)
        if (c.smem > 227 * 1024) return set_error(MGT_ERR_ARG, "batch: formal-solution shared memory above 227 KB");
    for (mgt_batch::FsClass &c : classes)
        MGT_TRY_STATUS(fs_batch_grid(c.threads, c.fused, c.lines, c.smem, max_smem[instance(c)], &c.grid));

    const bool same = order == b->order && fa == b->fs_args && sa == b->se_args && la == b->ld_args &&
                      classes == b->fs_classes && solo_slots == b->fs_solo && se_smem == b->se_smem;
    if (same && b->d_next) return MGT_OK;
    drop_graph(b);
    if (b->d_next && classes.size() != b->fs_classes.size()) {
        MGT_CUDA(cudaStreamSynchronize(s));
        MGT_CUDA(cudaFree(b->d_next));
        b->d_next = nullptr;
    }
    b->order = order;
    b->fs_args = fa;
    b->se_args = sa;
    b->ld_args = la;
    b->fs_end = fe;
    b->se_end = se;
    b->ld_end = le;
    for (const int32_t k : solo_slots) MGT_TRY_STATUS(fs_batch_solo(b->models[order[k]], s, false));
    b->fs_classes = classes;
    b->fs_solo = solo_slots;
    b->fs_solo_items = solo_items;
    b->se_smem = se_smem;
    MGT_TRY_STATUS(se_batch_prepare(se_smem));
    MGT_TRY_STATUS(upload(&b->d_fs_args, fa, fa.size(), s));
    MGT_TRY_STATUS(upload(&b->d_se_args, sa, sa.size(), s));
    MGT_TRY_STATUS(upload(&b->d_ld_args, la, la.size(), s));
    MGT_TRY_STATUS(upload(&b->d_fs_end, fe, n, s));
    MGT_TRY_STATUS(upload(&b->d_se_end, se, n, s));
    MGT_TRY_STATUS(upload(&b->d_ld_end, le, n, s));
    if (!b->d_next) MGT_CUDA(cudaMalloc(&b->d_next, sizeof(unsigned long long) * std::max<size_t>(classes.size(), 1)));
    // the host vectors must outlive the copies
    MGT_CUDA(cudaStreamSynchronize(s));
    return MGT_OK;
}

mgt_status launch_fs(mgt_batch *b, cudaStream_t s)
{
    const int n = (int)b->models.size();
    MGT_TRY_STATUS(ld_batch_launch(b->d_ld_args, b->d_ld_end, n, b->ld_end.back(), s));
    const size_t fsz = fs_args_bytes();
    for (size_t c = 0; c < b->fs_classes.size(); ++c) {
        const mgt_batch::FsClass &k = b->fs_classes[c];
        MGT_TRY_STATUS(fs_batch_launch(b->d_fs_args + k.first * fsz, b->d_fs_end + k.first, k.count, k.items,
                                       b->d_next + c, k.threads, k.fused, k.lines, k.smem, k.grid, s));
    }
    for (const int32_t k : b->fs_solo) MGT_TRY_STATUS(fs_batch_solo(b->models[b->order[k]], s, true));
    return MGT_OK;
}

mgt_status launch_se(mgt_batch *b, cudaStream_t s)
{
    return se_batch_launch(b->d_se_args, b->d_se_end, (int)b->models.size(), b->se_end.back(), b->se_smem, s);
}

mgt_status capture(mgt_batch *b)
{
    if (b->exec) return MGT_OK;
    int64_t before = 0, after = 0;
    mgt_launch_count(&before);
    MGT_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    mgt_status st = launch_fs(b, b->cap);
    if (st == MGT_OK) st = launch_se(b, b->cap);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(b->cap, &g);
    mgt_launch_count(&after);
    note_launches(before - after);          // nothing ran yet; replays are counted
    if (st != MGT_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return cuda_status(e, "cudaStreamEndCapture");
    b->graph = g;
    b->graph_kernels = (int)(after - before);
    MGT_CUDA(cudaGraphInstantiate(&b->exec, g, 0));
    return MGT_OK;
}

// The models' device error words with one synchronisation; the first model
// with an error reports it (and clears it) as its own calls would.
mgt_status check_errors(mgt_batch *b, cudaStream_t s)
{
    const int n = (int)b->models.size();
    if (!b->h_err) MGT_CUDA(cudaMallocHost(&b->h_err, sizeof(int) * 4 * n));
    for (int i = 0; i < n; ++i)
        MGT_CUDA(cudaMemcpyAsync(b->h_err + 4 * i, b->models[i]->d_err, sizeof(int) * 4, cudaMemcpyDeviceToHost, s));
    MGT_CUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < n; ++i)
        if (b->h_err[4 * i] != 0) return check_device_error(b->models[i], s);
    return MGT_OK;
}

void mark_solved(mgt_batch *b)
{
    for (mgt_model *m : b->models) {
        m->have_J = true;
        m->line_dirty = false;
    }
}

void mark_se(mgt_batch *b)
{
    for (mgt_model *m : b->models) m->line_dirty = true;
}

}  // namespace

}  // namespace mgt

using namespace mgt;

extern "C" {

mgt_status mgt_batch_create(mgt_batch **out, mgt_model *const *models, int32_t n_models, void *stream)
{
    MGT_RANGE("mgt_batch_create");
    if (!out) return set_error(MGT_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!models || n_models < 1 || n_models > 65536) return set_error(MGT_ERR_ARG, "n_models must be 1..65536");
    std::vector<mgt_model *> ms(models, models + n_models);
    for (mgt_model *m : ms)
        if (!m) return set_error(MGT_ERR_ARG, "a model is NULL");
    {
        std::vector<mgt_model *> u(ms);
        std::sort(u.begin(), u.end());
        if (std::adjacent_find(u.begin(), u.end()) != u.end())
            return set_error(MGT_ERR_ARG, "a model appears twice in the batch");
    }
    int dev = 0;
    MGT_CUDA(cudaGetDevice(&dev));
    for (mgt_model *m : ms) {
        if (m->device != dev) return set_error(MGT_ERR_ARG, "the models of a batch must live on the current device");
        if (!m->traced) return set_error(MGT_ERR_STATE, "mgt_trace_rays must be called on every model first");
        if (m->opts.pairs_per_batch > 0 && m->opts.pairs_per_batch < m->P)
            return set_error(MGT_ERR_ARG, "a batch needs every model's rays resident (pairs_per_batch = 0)");
    }
    mgt_batch *b = new mgt_batch;
    b->device = dev;
    b->models = ms;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        free_batch(b);
        return cuda_status(e, "cudaStreamCreateWithFlags");
    }
    const mgt_status st = refresh(b, s);
    if (st != MGT_OK) {
        free_batch(b);
        return st;
    }
    *out = b;
    return MGT_OK;
}

mgt_status mgt_batch_destroy(mgt_batch *b)
{
    if (!b) return MGT_OK;
    cudaDeviceSynchronize();
    free_batch(b);
    return MGT_OK;
}

mgt_status mgt_batch_formal_solve(mgt_batch *b, void *stream)
{
    MGT_RANGE("mgt_batch_formal_solve");
    if (!b) return set_error(MGT_ERR_ARG, "batch is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    MGT_TRY_STATUS(refresh(b, s));
    MGT_TRY_STATUS(launch_fs(b, s));
    mark_solved(b);
    return MGT_OK;
}

mgt_status mgt_batch_stat_equilibrium(mgt_batch *b, void *stream)
{
    MGT_RANGE("mgt_batch_stat_equilibrium");
    if (!b) return set_error(MGT_ERR_ARG, "batch is NULL");
    for (mgt_model *m : b->models)
        if (!m->have_J) return set_error(MGT_ERR_STATE, "mgt_batch_formal_solve must be called first");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    MGT_TRY_STATUS(refresh(b, s));
    MGT_TRY_STATUS(launch_se(b, s));
    mark_se(b);
    return MGT_OK;
}

mgt_status mgt_batch_iterate(mgt_batch *b, int32_t n_iter, const mgt_ng_opts *ng, mgt_ali_stats *stats,
                             void *stream)
{
    MGT_RANGE("mgt_batch_iterate");
    if (!b) return set_error(MGT_ERR_ARG, "batch is NULL");
    if (n_iter < 0) return set_error(MGT_ERR_ARG, "n_iter must be >= 0");
    const int n = (int)b->models.size();
    const mgt_ng_opts no_ng{MGT_NG_NONE, 4, 8};
    const mgt_ng_opts &o = ng ? *ng : no_ng;
    if (o.mode < MGT_NG_NONE || o.mode > MGT_NG_ADAPTIVE) return set_error(MGT_ERR_ARG, "unknown Ng mode");
    if (o.mode == MGT_NG_CLASSICAL && (o.n_steps < 2 || o.n_steps > kMaxNgHist - 1))
        return set_error(MGT_ERR_ARG, "n_steps must be 2..15");
    if (o.mode == MGT_NG_ADAPTIVE && (o.n_max < 3 || o.n_max > kMaxNgHist))
        return set_error(MGT_ERR_ARG, "n_max must be 3..16");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (stats)
        for (int i = 0; i < n; ++i) stats[i] = {0, 0, 0.0};
    MGT_TRY_STATUS(refresh(b, s));
    MGT_TRY_STATUS(capture(b));
    for (int it = 0; it < n_iter; ++it) {
        MGT_CUDA(cudaGraphLaunch(b->exec, s));
        note_launches(b->graph_kernels);
        mark_solved(b);
        mark_se(b);
        if (o.mode == MGT_NG_NONE && !stats) continue;
        // every model's Ng step, phase by phase, one host synchronisation per
        // phase for the whole batch
        for (int i = 0; i < n; ++i) MGT_TRY_STATUS(ng_begin(b->models[i], &o, s));
        MGT_CUDA(cudaStreamSynchronize(s));
        bool predicting = false;
        for (int i = 0; i < n; ++i) {
            MGT_TRY_STATUS(ng_after_push(b->models[i], s));
            predicting = predicting || b->models[i]->ng.pend.phase == 2;
        }
        if (predicting) MGT_CUDA(cudaStreamSynchronize(s));
        for (int i = 0; i < n; ++i) {
            MGT_TRY_STATUS(ng_after_predict(b->models[i], s));
            const int acc = b->models[i]->ng.pend.accepted;
            const double mr = b->models[i]->ng.pend.maxrel;
            if (stats) {
                stats[i].iterations = it + 1;
                stats[i].ng_accepted += acc;
                stats[i].last_maxrel = mr;
            }
            if (!std::isfinite(mr)) return set_error(MGT_ERR_NOT_CONVERGED, "populations became non-finite");
        }
    }
    return check_errors(b, s);
}

mgt_status mgt_batch_get_layout(const mgt_batch *b, mgt_batch_layout *layout, int32_t *order)
{
    if (!b) return set_error(MGT_ERR_ARG, "batch is NULL");
    if (layout) {
        layout->n_models = (int32_t)b->models.size();
        layout->fs_items = 0;
        layout->fs_grid = 0;
        layout->fs_threads = 0;
        layout->fs_smem_bytes = 0;
        for (const mgt_batch::FsClass &c : b->fs_classes) {
            layout->fs_items += c.items;
            layout->fs_grid += c.grid;
            layout->fs_threads = std::max(layout->fs_threads, c.threads);
            layout->fs_smem_bytes = std::max<int64_t>(layout->fs_smem_bytes, (int64_t)c.smem);
        }
        layout->fs_items += b->fs_solo_items;
        layout->fs_launches = (int32_t)(b->fs_classes.size() + b->fs_solo.size());
        layout->fs_solo = (int32_t)b->fs_solo.size();
        layout->se_blocks = b->se_end.empty() ? 0 : b->se_end.back();
        layout->graph_kernels = b->graph_kernels;
    }
    if (order) std::copy(b->order.begin(), b->order.end(), order);
    return MGT_OK;
}

mgt_status mgt_autotune(mgt_model *m, mgt_precision p, int32_t staged_only, int32_t reps, mgt_autotune_result *res,
                        void *stream)
{
    MGT_RANGE("mgt_autotune");
    if (!m) return set_error(MGT_ERR_ARG, "model is NULL");
    if (p != MGT_FP64 && p != MGT_FP32_MIXED) return set_error(MGT_ERR_ARG, "unknown precision");
    if (reps < 1 || reps > 100) return set_error(MGT_ERR_ARG, "reps must be 1..100");
    if (m->opts.pairs_per_batch > 0 && m->opts.pairs_per_batch < m->P)
        return set_error(MGT_ERR_ARG, "autotune needs the model's rays resident (pairs_per_batch = 0)");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    MGT_TRY_STATUS(ensure_rays(m, p, s));
    if (m->line_dirty) MGT_TRY_STATUS(launch_line_data(m, s));
    struct Cand {
        int schedule, lpt;
    };
    // staged_only: the automatic staged choice (0), which batched launches run;
    // otherwise schedules 1-3, and 4 where the lines fit one group
    std::vector<Cand> cands;
    const int lpts[2] = {4, 8};
    if (staged_only) {
        for (int lpt : lpts)
            if (p == MGT_FP32_MIXED || lpt == 4) cands.push_back({0, lpt});
    } else {
        for (int sch = 1; sch <= 4; ++sch)
            for (int lpt : lpts)
                if ((p == MGT_FP32_MIXED || lpt == 4) && (sch < 4 || m->M <= lpt)) cands.push_back({sch, lpt});
    }
    const mgt_solve_opts saved = m->opts;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    MGT_CUDA(cudaEventCreate(&e0));
    MGT_CUDA(cudaEventCreate(&e1));
    mgt_autotune_result r{};
    r.n_tried = (int32_t)cands.size();
    int best = -1;
    mgt_status st = MGT_OK;
    for (size_t c = 0; c < cands.size() && st == MGT_OK; ++c) {
        m->opts.schedule = cands[c].schedule;
        m->opts.lines_per_thread = cands[c].lpt;
        r.schedules[c] = cands[c].schedule;
        r.lines[c] = cands[c].lpt;
        st = launch_formal_solve(m, p, s, false);          // warm-up
        std::vector<float> t;
        for (int k = 0; k < reps && st == MGT_OK; ++k) {
            cudaEventRecord(e0, s);
            st = launch_formal_solve(m, p, s, false);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) st = cuda_status(cudaGetLastError(), "cudaEventSynchronize");
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            t.push_back(ms);
        }
        if (st != MGT_OK) break;
        std::sort(t.begin(), t.end());
        r.ms[c] = t[t.size() / 2];
        if (best < 0 || r.ms[c] < r.ms[best]) best = (int)c;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    m->opts = saved;
    if (st != MGT_OK) return st;
    m->opts.schedule = cands[best].schedule;
    m->opts.lines_per_thread = cands[best].lpt;
    r.schedule = cands[best].schedule;
    r.lines_per_thread = cands[best].lpt;
    m->have_J = true;
    if (res) *res = r;
    return check_device_error(m, s);
}

}  // extern "C"
