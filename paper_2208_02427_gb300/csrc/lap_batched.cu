// lap_batched.cu -- lap_solve_batched: the V-cycle over many independent grids of different
// sizes, every phase one launch over all problems (work lists built here, kernels in
// batch_kernels.cu and fused32_kernels.cu).
#include "lap_host.cuh"

namespace lap {

void add_items(std::vector<BatchItem>& items, int level_index, int m, int n, int points)
{
    const int per = std::max(1, points / std::max(1, m - 2));
    for (int r = 1; r <= n - 2; r += per) items.push_back(BatchItem{level_index, r, std::min(per, n - 1 - r)});
}

// First level of a problem that the small-level tail runs (both sides <= tail_size), or
// nlev when it has none.
int tail_start(const BatchLevel<double>* lv, int nlev, int tail_size)
{
    if (tail_size <= 0) return nlev;
    for (int l = 0; l < nlev; ++l)
        if (lv[l].m <= tail_size && lv[l].n <= tail_size) return l;
    return nlev;
}

// Lists of one V-cycle over problems `who`: problem q owns levels base[q] .. base[q] +
// nlev[q] - 1 of lv. Levels above a problem's tail go through item lists, the tail is one job.
// With tiles, the fine levels also get the tile items of the fused FP32 descent/ascent.
void build_lists(LevelLists& L, std::vector<BatchItem>& items, std::vector<TailJob>& jobs,
                 const std::vector<int>& who, const std::vector<int>& base,
                 const std::vector<int>& nlev, const std::vector<BatchLevel<double>>& lv,
                 int tail_size, std::vector<TileItem>* tiles, int nu1, int nu2, int tile_variant,
                 int item_points)
{
    L.fused = tiles != nullptr;
    L.tile_variant = tile_variant;
    L.tiles.assign(0, {0, 0});
    L.levels = 0;
    for (int q : who) L.levels = std::max(L.levels, nlev[q]);
    L.fine.assign(L.levels, {0, 0});
    L.all.assign(L.levels, {0, 0});
    L.coarse.assign(L.levels, {0, 0});
    L.tail.assign(L.levels, {0, 0});
    L.tiles.assign(L.levels, {0, 0});
    std::vector<int> t(who.size());
    for (size_t k = 0; k < who.size(); ++k) t[k] = tail_start(&lv[base[who[k]]], nlev[who[k]], tail_size);
    for (int l = 0; l < L.levels; ++l) {
        const int f0 = (int)items.size();
        for (size_t k = 0; k < who.size(); ++k) {
            const int q = who[k];
            if (nlev[q] - 1 > l && l < t[k])
                add_items(items, base[q] + l, lv[base[q] + l].m, lv[base[q] + l].n, item_points);
        }
        L.fine[l] = {f0, (int)items.size() - f0};
        if (tiles) {
            const int t0 = (int)tiles->size();
            for (size_t k = 0; k < who.size(); ++k) {
                const int q = who[k];
                if (!(nlev[q] - 1 > l && l < t[k])) continue;
                const BatchLevel<double>& d = lv[base[q] + l];
                int tx, ty, ntx, nty;
                fused32_tile_variant(tile_variant, d.m, d.n, nu1, nu2, &tx, &ty, &ntx, &nty);
                for (int by = 0; by < nty; ++by)
                    for (int bx = 0; bx < ntx; ++bx)
                        tiles->push_back(TileItem{base[q] + l, 1 + bx * tx, 1 + by * ty, tx, ty});
            }
            L.tiles[l] = {t0, (int)tiles->size() - t0};
        }
        const int a0 = (int)items.size();
        for (size_t k = 0; k < who.size(); ++k) {
            const int q = who[k];
            if (nlev[q] > l && l <= t[k])
                add_items(items, base[q] + l, lv[base[q] + l].m, lv[base[q] + l].n, item_points);
        }
        L.all[l] = {a0, (int)items.size() - a0};
        const int c0 = (int)items.size();
        for (size_t k = 0; k < who.size(); ++k) {
            const int q = who[k];
            if (nlev[q] - 1 == l && t[k] == nlev[q]) {
                const BatchLevel<double>& d = lv[base[q] + l];
                items.push_back(BatchItem{base[q] + l, 1, d.n - 2});
                L.max_coarse = std::max(L.max_coarse, (d.m - 2) * (d.n - 2));
            }
        }
        L.coarse[l] = {c0, (int)items.size() - c0};
        const int j0 = (int)jobs.size();
        for (size_t k = 0; k < who.size(); ++k) {
            const int q = who[k];
            if (t[k] == l && l < nlev[q]) {
                jobs.push_back(TailJob{base[q] + l, base[q] + nlev[q] - 1});
                const BatchLevel<double>& d = lv[base[q] + nlev[q] - 1];
                L.max_coarse = std::max(L.max_coarse, (d.m - 2) * (d.n - 2));
            }
        }
        L.tail[l] = {j0, (int)jobs.size() - j0};
    }
    if (tiles) {
        const int u0 = (int)items.size();
        for (size_t k = 0; k < who.size(); ++k) {
            const int q = who[k];
            if (t[k] == 0 || nlev[q] == 1) add_items(items, base[q], lv[base[q]].m, lv[base[q]].n);
        }
        L.upd0 = {u0, (int)items.size() - u0};
    }
}

}  // namespace lap

using namespace lap;

namespace {

struct BatchPlan {
    std::vector<BatchLevel<double>> lv64;
    std::vector<BatchLevel<float>> lv32;
    std::vector<int> nlev, base;       // levels and first level index per problem
    std::vector<BatchItem> norm_items; // level-0 items of every problem, problem by problem
    std::vector<int> first_item;       // per problem: its first item in the norm list (+ end)
    int max_coarse_unknowns = 0;
    int levels = 0;
};

// The work lists of one tuner candidate (a BatchConfig), on the device in one allocation, and
// the cycle graph captured with them.
struct CandPlan {
    LevelLists L;
    BatchItem* items = nullptr;
    TailJob* jobs = nullptr;
    TileItem* tiles = nullptr;
    void* dev = nullptr;
    size_t bytes = 0;
    cudaGraphExec_t exec = nullptr;
    int64_t kernels = 0;  // kernels one replay of exec launches
    // the device-resident loop: cycle after cycle as the body of a conditional (while) node
    cudaGraphExec_t loop_exec = nullptr;
    int64_t loop_kernels = 0;  // kernels one iteration of the loop launches
};

// What a call's plan depends on: the grids (sizes, spacings, pitches), the fields' addresses
// and the parameters that shape the lists and the captured cycle.
struct BatchKey {
    std::vector<lap_grid> grids;
    std::vector<const double*> psi;
    int32_t method, norm, nu1, nu2, coarsest_min, max_levels, inner_cycles, tail_size, unfused,
        tiling, item_points, persistent;
    double smoother_w, tol;
    bool operator==(const BatchKey& o) const
    {
        if (grids.size() != o.grids.size() || psi != o.psi) return false;
        for (size_t k = 0; k < grids.size(); ++k) {
            const lap_grid &a = grids[k], &b = o.grids[k];
            if (a.m != b.m || a.n != b.n || a.dx != b.dx || a.dy != b.dy || a.pitch != b.pitch)
                return false;
        }
        return method == o.method && norm == o.norm && nu1 == o.nu1 && nu2 == o.nu2 &&
               coarsest_min == o.coarsest_min && max_levels == o.max_levels &&
               inner_cycles == o.inner_cycles && tail_size == o.tail_size && unfused == o.unfused &&
               tiling == o.tiling && item_points == o.item_points && persistent == o.persistent &&
               smoother_w == o.smoother_w && tol == o.tol;
    }
};

// A plan with its level buffers and tables in the handle's arena, and the candidates' lists
// and graphs built so far. Valid while nothing else has carved the arena (epoch).
struct BatchCache : BatchCacheBase {
    lap_handle h = nullptr;
    BatchKey key;
    BatchPlan P;
    uint64_t epoch = 0;
    size_t level_bytes = 0;
    BatchLevel<double>* lv64 = nullptr;
    BatchLevel<float>* lv32 = nullptr;
    BatchItem* norm_items = nullptr;
    int *first = nullptr, *active = nullptr, *status = nullptr, *remaining = nullptr;
    long long* iters = nullptr;
    double *r0 = nullptr, *rnow = nullptr, *partials = nullptr;
    unsigned* claim = nullptr;  // item counter of the persistent launches (two words, zero between launches)
    long long* loop = nullptr;  // device-resident loop: cycles done, cycle cap
    std::vector<CandPlan> cands;  // indexed like the tuner's candidates
    ~BatchCache() override
    {
        for (CandPlan& c : cands) {
            if (c.exec) cudaGraphExecDestroy(c.exec);
            if (c.loop_exec) cudaGraphExecDestroy(c.loop_exec);
            dev_free(h, c.dev, c.bytes);
        }
    }
};

BatchKey make_key(int count, const lap_grid* grids, double* const* psi_devs, const lap_params* p)
{
    BatchKey k;
    k.grids.assign(grids, grids + count);
    k.psi.assign(psi_devs, psi_devs + count);
    k.method = p->method;
    k.norm = p->norm;
    k.nu1 = p->nu1;
    k.nu2 = p->nu2;
    k.coarsest_min = p->coarsest_min;
    k.max_levels = p->max_levels;
    k.inner_cycles = p->inner_cycles;
    k.tail_size = p->tail_size;
    k.unfused = p->unfused;
    k.tiling = p->tiling;
    k.item_points = p->item_points;
    k.persistent = p->persistent;
    k.smoother_w = p->smoother_w;
    k.tol = p->tol;
    return k;
}

// The configurations a batched solve of these parameters tries (first = the default of each
// knob): tail sizes, FP32 tilings (mixed solver, tiles allowed: the tile variants and one
// kernel per pass), work-item sizes, one CTA per item or persistent launches.
void tuner_values(const lap_params* p, std::vector<int>* tails, std::vector<int>* tilings,
                  std::vector<int>* items, std::vector<int>* persists)
{
    const bool mixed = p->method == LAP_MG_MIXED;
    *tails = tail_candidates(true, mixed, p->tail_size);
    tilings->clear();
    if (mixed && !p->unfused && fused32_supported(p->nu1, p->nu2) && p->tiling >= 0) {
        for (int v = 1; v <= FUSED32_VARIANTS; ++v)
            if ((p->tiling == 0 || p->tiling == v) && fused32_variant_supported(v, p->nu1, p->nu2))
                tilings->push_back(v);
        if (p->tiling == 0) tilings->push_back(0);
    }
    if (tilings->empty()) tilings->push_back(0);  // one kernel per pass
    if (p->item_points > 0) *items = {p->item_points};
    else *items = {BATCH_ITEM_POINTS, 2048, 32768};
    if (p->persistent != 0) *persists = {p->persistent > 0 ? 1 : 0};
    else *persists = {0, 1};
}

// The level descriptors, the norm list, the arena carved for them (level buffers first) and
// the tables uploaded (stream-ordered on s; pageable sources are staged before each copy
// returns).
std::unique_ptr<BatchCache> build_plan(lap_handle h, int count, const lap_grid* grids,
                                       double* const* psi_devs, const lap_params* p, cudaStream_t s)
{
    auto C = std::make_unique<BatchCache>();
    C->h = h;
    BatchPlan& P = C->P;
    const bool mixed = p->method == LAP_MG_MIXED;
    P.nlev.resize(count);
    P.base.resize(count);
    for (int q = 0; q < count; ++q) {
        const lap_grid* g = &grids[q];
        const int L = mg_level_count(g->m, g->n, p->coarsest_min, p->max_levels);
        P.nlev[q] = L;
        P.base[q] = (int)P.lv64.size();
        P.levels = std::max(P.levels, L);
        const Coef c = make_coef(g->dx, g->dy);
        int m = g->m, n = g->n;
        for (int l = 0; l < L; ++l) {
            BatchLevel<double> d{};
            d.m = m;
            d.n = n;
            d.pitch = l == 0 ? g->pitch : round_up(m, 32);
            d.problem = q;
            d.unit_beta = c.unit_beta;
            d.inv_d_shift = c.inv_d_shift;
            d.b2 = c.b2;
            d.d = c.d;
            d.inv_d = c.inv_d;
            BatchLevel<float> f{};
            f.m = m;
            f.n = n;
            f.pitch = round_up(m, 32);
            f.problem = q;
            f.unit_beta = c.unit_beta;
            f.inv_d_shift = 0;
            f.b2 = c.b2;
            f.d = c.d;
            f.inv_d = c.inv_d;
            if (l == L - 1) {
                if ((int64_t)(m - 2) * (n - 2) > COARSE_MAX_UNKNOWNS)
                    fail(LAP_EUNSUPPORTED, "coarsest level with more than 1024 unknowns");
                d.ainv_t = f.ainv_t = coarse_inverse(h, m, n, c.b2, c.d);
                P.max_coarse_unknowns = std::max(P.max_coarse_unknowns, (m - 2) * (n - 2));
            }
            P.lv64.push_back(d);
            P.lv32.push_back(f);
            m = (m - 1) / 2 + 1;
            n = (n - 1) / 2 + 1;
        }
    }
    for (int q = 0; q < count; ++q) {
        P.first_item.push_back((int)P.norm_items.size());
        add_items(P.norm_items, P.base[q], grids[q].m, grids[q].n);
    }
    P.first_item.push_back((int)P.norm_items.size());
    auto carve_all = [&](auto& cv) {
        for (int q = 0; q < count; ++q)
            for (int l = 0; l < P.nlev[q]; ++l) {
                const int k = P.base[q] + l;
                BatchLevel<double>& d = P.lv64[k];
                BatchLevel<float>& f = P.lv32[k];
                const bool last = l == P.nlev[q] - 1;
                if (!mixed) {
                    if (l == 0) {
                        d.u = psi_devs[q];
                        d.q = nullptr;
                    } else {
                        d.u = cv.template take<double>((size_t)d.n * d.pitch);
                        d.q = cv.template take<double>((size_t)d.n * d.pitch);
                    }
                    d.r = last ? nullptr : cv.template take<double>((size_t)d.n * d.pitch);
                } else {
                    if (l == 0) d.u = psi_devs[q];
                    f.u = cv.template take<float>((size_t)f.n * f.pitch);
                    f.q = cv.template take<float>((size_t)f.n * f.pitch);
                    f.r = last ? nullptr : cv.template take<float>((size_t)f.n * f.pitch);
                }
            }
        C->lv64 = cv.template take<BatchLevel<double>>(P.lv64.size());
        C->lv32 = cv.template take<BatchLevel<float>>(P.lv32.size());
        C->norm_items = cv.template take<BatchItem>(P.norm_items.size());
        C->first = cv.template take<int>(P.first_item.size());
        C->active = cv.template take<int>(count);
        C->status = cv.template take<int>(count);
        C->remaining = cv.template take<int>(1);
        C->iters = cv.template take<long long>(count);
        C->r0 = cv.template take<double>(count);
        C->rnow = cv.template take<double>(count);
        C->partials = cv.template take<double>(std::max<size_t>(1, P.norm_items.size()));
        C->claim = cv.template take<unsigned>(2);
        C->loop = cv.template take<long long>(2);
    };
    Sizer sz;
    carve_all(sz);
    Carver cv(arena(h, sz.off));
    carve_all(cv);
    C->epoch = h->arena_epoch;
    C->level_bytes = (size_t)((char*)C->lv64 - (char*)h->arena);
    ck(cudaMemcpyAsync(C->lv64, P.lv64.data(), P.lv64.size() * sizeof(P.lv64[0]), cudaMemcpyHostToDevice, s), "upload levels");
    ck(cudaMemcpyAsync(C->lv32, P.lv32.data(), P.lv32.size() * sizeof(P.lv32[0]), cudaMemcpyHostToDevice, s), "upload levels");
    ck(cudaMemcpyAsync(C->norm_items, P.norm_items.data(), P.norm_items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice, s), "upload items");
    ck(cudaMemcpyAsync(C->first, P.first_item.data(), P.first_item.size() * sizeof(int), cudaMemcpyHostToDevice, s), "upload items");
    ck(cudaMemsetAsync(C->claim, 0, 2 * sizeof(unsigned), s), "zero claim counter");
    C->key = make_key(count, grids, psi_devs, p);
    return C;
}

// The lists of candidate c (configuration cfg), built and uploaded on first use; called
// outside graph capture (it allocates and copies synchronously).
CandPlan& ensure_candidate(BatchCache& C, int c, const BatchConfig& cfg, const lap_params* p,
                           int count)
{
    if ((int)C.cands.size() <= c) C.cands.resize(c + 1);
    CandPlan& K = C.cands[c];
    if (K.dev) return K;
    const BatchPlan& P = C.P;
    std::vector<int> all_problems(count);
    for (int q = 0; q < count; ++q) all_problems[q] = q;
    std::vector<BatchItem> items;
    std::vector<TailJob> jobs;
    std::vector<TileItem> tiles;
    build_lists(K.L, items, jobs, all_problems, P.base, P.nlev, P.lv64, cfg.tail,
                cfg.tiles > 0 ? &tiles : nullptr, p->nu1, p->nu2, std::max(1, cfg.tiles), cfg.item);
    K.L.claim = cfg.persist != 0 ? C.claim : nullptr;
    // one allocation: items, jobs, tiles (each 256-byte aligned)
    Sizer sz;
    sz.take<BatchItem>(std::max<size_t>(1, items.size()));
    sz.take<TailJob>(std::max<size_t>(1, jobs.size()));
    sz.take<TileItem>(std::max<size_t>(1, tiles.size()));
    K.bytes = sz.off;
    K.dev = dev_alloc(C.h, K.bytes);
    Carver cv(K.dev);
    K.items = cv.take<BatchItem>(std::max<size_t>(1, items.size()));
    K.jobs = cv.take<TailJob>(std::max<size_t>(1, jobs.size()));
    K.tiles = cv.take<TileItem>(std::max<size_t>(1, tiles.size()));
    if (!items.empty())
        ck(cudaMemcpy(K.items, items.data(), items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice), "upload items");
    if (!jobs.empty())
        ck(cudaMemcpy(K.jobs, jobs.data(), jobs.size() * sizeof(TailJob), cudaMemcpyHostToDevice), "upload jobs");
    if (!tiles.empty())
        ck(cudaMemcpy(K.tiles, tiles.data(), tiles.size() * sizeof(TileItem), cudaMemcpyHostToDevice), "upload tiles");
    return K;
}

}  // namespace

extern "C" int lap_solve_batched(lap_handle h, int count, const lap_grid* grids,
                                 double* const* psi_devs, const lap_params* p, lap_result* results,
                                 void* stream)
{
    return guarded([&] {
        if (!h) fail(LAP_EINVAL, "handle is NULL");
        if (count < 1 || !grids || !psi_devs || !results) fail(LAP_EINVAL, "empty or NULL batch");
        check_params(p);
        if (p->method != LAP_MG && p->method != LAP_MG_MIXED)
            fail(LAP_EINVAL, "batched solves take LAP_MG or LAP_MG_MIXED");
        if (p->norm == LAP_NORM_MAXDELTA) fail(LAP_EINVAL, "batched solves stop on an L2 norm");
        set_device(h);
        for (int q = 0; q < count; ++q) {
            check_grid(&grids[q]);
            check_device_ptr(h, psi_devs[q], "psi");
        }
        const bool mixed = p->method == LAP_MG_MIXED;
        cudaStream_t s = (cudaStream_t)stream;
        std::vector<int> shape;
        for (int q = 0; q < count; ++q) {
            shape.push_back(grids[q].m);
            shape.push_back(grids[q].n);
        }
        BatchTuner& tuner = h->batch_tuners[tuner_key('B', p, shape)];
        if (tuner.cand.empty()) {
            std::vector<int> tails, tilings, items, persists;
            tuner_values(p, &tails, &tilings, &items, &persists);
            tuner.init(tails, tilings, items, persists);
        }
        if (mixed && !p->unfused && fused32_supported(p->nu1, p->nu2))
            ck(prepare_fused32(), "tile kernel attributes");
        // the plan of the previous call, if it was this batch and nothing has carved the arena
        // since; else a new one
        BatchCache* C = static_cast<BatchCache*>(h->batch_cache.get());
        if (!C || C->epoch != h->arena_epoch || !(C->key == make_key(count, grids, psi_devs, p))) {
            h->batch_cache.reset();  // releases the old plan's lists and graphs
            h->batch_cache = build_plan(h, count, grids, psi_devs, p, s);
            C = static_cast<BatchCache*>(h->batch_cache.get());
        }
        try {
            const BatchPlan& P = C->P;
            // per call: every level buffer zeroed (rings of corrections stay zero), every
            // problem active, no cycles done
            if (C->level_bytes) ck(cudaMemsetAsync(h->arena, 0, C->level_bytes, s), "zero levels");
            std::vector<int> ones(count, 1);
            const int cnt = count;
            ck(cudaMemcpyAsync(C->active, ones.data(), count * sizeof(int), cudaMemcpyHostToDevice, s), "upload flags");
            ck(cudaMemcpyAsync(C->status, ones.data(), count * sizeof(int), cudaMemcpyHostToDevice, s), "upload flags");
            ck(cudaMemcpyAsync(C->remaining, &cnt, sizeof(int), cudaMemcpyHostToDevice, s), "upload count");
            ck(cudaMemsetAsync(C->iters, 0, count * sizeof(long long), s), "zero iterations");
            BatchLevel<double>* lv64 = C->lv64;
            BatchLevel<float>* lv32 = C->lv32;
            int* first = C->first;
            int* active = C->active;
            int* status = C->status;
            int* remaining = C->remaining;
            long long* iters = C->iters;
            double* r0 = C->r0;
            double* rnow = C->rnow;
            double* partials = C->partials;
            const BatchList norm_list{C->norm_items, (int)P.norm_items.size()};
            const bool rel = p->norm == LAP_NORM_L2_REL;
            // ---- one cycle (V-cycle(s) and stopping test) with candidate c's lists ----
            auto cycle = [&](const CandPlan& K, cudaStream_t st) {
                const LevelLists& L = K.L;
                auto list = [&](std::pair<int, int> r) {
                    return BatchList{K.items + r.first, r.second, L.claim};
                };
                const BatchList norms{norm_list.items, norm_list.count, L.claim};
                if (mixed) {
                    for (int k = 0; k < p->inner_cycles; ++k) {
                        if (L.fused)
                            enqueue_vcycle32_fused(list, L, lv32, active, K.jobs, K.tiles, *p, p->smoother_w,
                                                   k == 0, st, k == p->inner_cycles - 1 ? lv64 : nullptr);
                        else
                            enqueue_vcycle(list, L, lv32, active, K.jobs, *p, p->smoother_w, st);
                    }
                    // fused: the level-0 ascents did psi += e except where a tail holds level 0
                    ck(launch_b_update(L.fused ? list(L.upd0) : norms, lv64, active, lv32, st),
                       "batched update");
                    ck(launch_b_sumsq(norms, lv64, active, partials, lv32, st, r0), "batched residual");
                } else {
                    enqueue_vcycle(list, L, lv64, active, K.jobs, *p, p->smoother_w, st);
                    ck(launch_b_sumsq(norms, lv64, active, partials, nullptr, st), "batched residual");
                }
                ck(launch_b_converge(partials, first, count, active, r0, rnow, iters, status, remaining,
                                     1, rel, p->tol, st), "batched convergence");
            };
            // initial residuals (and, for the mixed solver, the first FP32 right-hand sides)
            ck(launch_b_sumsq(norm_list, lv64, active, partials, mixed ? lv32 : nullptr, s), "batched residual");
            ck(launch_b_converge(partials, first, count, active, r0, rnow, iters, status, remaining, 0,
                                 rel, p->tol, s), "batched convergence");
            // one cycle of candidate c as a graph, captured on the handle's stream when first
            // used (kept with the plan for later calls) and replayed on the caller's
            auto launch_cycle = [&](int c) {
                CandPlan& K = ensure_candidate(*C, c, tuner.cand[c], p, count);
                h->last_batch = tuner.cand[c];
                h->last_batch_tuned = tuner.done;
                if (!h->use_graphs) {
                    cycle(K, s);
                    return;
                }
                if (!K.exec) {
                    if (!h->capture)
                        ck(cudaStreamCreateWithFlags(&h->capture, cudaStreamNonBlocking), "capture stream");
                    const int64_t before = launches_now();
                    ck(cudaStreamBeginCapture(h->capture, cudaStreamCaptureModeThreadLocal), "begin capture");
                    cudaGraph_t g = nullptr;
                    try {
                        cycle(K, h->capture);
                    } catch (...) {
                        cudaStreamEndCapture(h->capture, &g);
                        if (g) cudaGraphDestroy(g);
                        cudaGetLastError();
                        throw;
                    }
                    ck(cudaStreamEndCapture(h->capture, &g), "end capture");
                    K.kernels = launches_now() - before;
                    add_launches(-K.kernels);
                    const cudaError_t e = cudaGraphInstantiate(&K.exec, g, 0);
                    cudaGraphDestroy(g);
                    ck(e, "instantiate graph");
                }
                ck(cudaGraphLaunch(K.exec, s), "launch graph");
                add_launches(K.kernels);
            };
            // once the configuration is chosen: the remaining cycles on the device, each followed
            // by the loop test, as one conditional graph replayed on the caller's stream until no
            // problem is left or max_iter cycles are done; the host waits once
            auto device_loop = [&](int c, int64_t done) {
                CandPlan& K = ensure_candidate(*C, c, tuner.cand[c], p, count);
                h->last_batch = tuner.cand[c];
                h->last_batch_tuned = true;
                if (!K.loop_exec) {
                    if (!h->capture)
                        ck(cudaStreamCreateWithFlags(&h->capture, cudaStreamNonBlocking), "capture stream");
                    cudaGraph_t g = nullptr;
                    ck(cudaGraphCreate(&g, 0), "create graph");
                    try {
                        cudaGraphConditionalHandle hnd;
                        ck(cudaGraphConditionalHandleCreate(&hnd, g, 1, cudaGraphCondAssignDefault),
                           "conditional handle");
                        alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)] = {};
                        cudaGraphNodeParams* np = reinterpret_cast<cudaGraphNodeParams*>(raw);
                        np->type = cudaGraphNodeTypeConditional;
                        np->conditional.handle = hnd;
                        np->conditional.type = cudaGraphCondTypeWhile;
                        np->conditional.size = 1;
                        cudaGraphNode_t node;
                        ck(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, np), "conditional node");
                        cudaGraph_t body = np->conditional.phGraph_out[0];
                        const int64_t before = launches_now();
                        ck(cudaStreamBeginCaptureToGraph(h->capture, body, nullptr, nullptr, 0,
                                                         cudaStreamCaptureModeThreadLocal),
                           "begin capture");
                        try {
                            cycle(K, h->capture);
                            ck(launch_batch_loop_decide(C->loop, remaining, hnd, h->capture),
                               "batched loop test");
                        } catch (...) {
                            cudaGraph_t junk = nullptr;
                            cudaStreamEndCapture(h->capture, &junk);
                            cudaGetLastError();
                            throw;
                        }
                        cudaGraph_t body_out = nullptr;
                        ck(cudaStreamEndCapture(h->capture, &body_out), "end capture");
                        K.loop_kernels = launches_now() - before;
                        add_launches(-K.loop_kernels);
                        ck(cudaGraphInstantiate(&K.loop_exec, g, 0), "instantiate graph");
                    } catch (...) {
                        cudaGraphDestroy(g);
                        throw;
                    }
                    cudaGraphDestroy(g);
                }
                long long st[2] = {(long long)done, (long long)p->max_iter};
                std::memcpy(h->pinned, st, sizeof st);
                ck(cudaMemcpyAsync(C->loop, h->pinned, sizeof st, cudaMemcpyHostToDevice, s), "upload loop state");
                ck(cudaGraphLaunch(K.loop_exec, s), "launch graph");
                ck(cudaMemcpyAsync(h->pinned, C->loop, sizeof st, cudaMemcpyDeviceToHost, s), "copy loop state");
                ck(cudaStreamSynchronize(s), "stream sync");
                std::memcpy(st, h->pinned, sizeof st);
                add_launches(K.loop_kernels * (st[0] - (long long)done));
                return (int64_t)st[0];
            };
            int64_t done = 0;
            int left = count;
            while (done < p->max_iter) {
                ck(cudaMemcpyAsync(h->pinned, remaining, sizeof(int), cudaMemcpyDeviceToHost, s), "copy count");
                ck(cudaStreamSynchronize(s), "stream sync");
                std::memcpy(&left, h->pinned, sizeof(int));
                if (left == 0) break;
                if (tuner.done && h->use_graphs) {
                    done = device_loop(tuner.best, done);
                    continue;
                }
                const int64_t steps = std::min<int64_t>(p->check_every, p->max_iter - done);
                for (int64_t k = 0; k < steps; ++k) {
                    const int c = tuner.next();
                    if (tuner.done) {
                        launch_cycle(c);
                        continue;
                    }
                    if (left < count) {
                        // problems already converged make the cycle cheaper: its time is not
                        // comparable, so the best configuration so far runs untimed
                        launch_cycle(tuner.best);
                        continue;
                    }
                    // not tuned yet: time this cycle (candidate c's graph captured before e0)
                    const bool fresh = c >= (int)C->cands.size() || !C->cands[c].dev || !C->cands[c].exec;
                    if (h->use_graphs && fresh) {
                        launch_cycle(c);  // first use builds, captures and runs it once
                        ck(cudaStreamSynchronize(s), "stream sync");
                        continue;
                    }
                    ck(cudaEventRecord(tuner_event(h, 0), s), "record event");
                    launch_cycle(c);
                    ck(cudaEventRecord(tuner_event(h, 1), s), "record event");
                    ck(cudaEventSynchronize(tuner_event(h, 1)), "event sync");
                    float ms = 0.f;
                    ck(cudaEventElapsedTime(&ms, tuner_event(h, 0), tuner_event(h, 1)), "event time");
                    tuner.record(c, ms);
                }
                done += steps;
            }
            // ---- results ----
            std::vector<long long> it(count);
            std::vector<int> st(count);
            std::vector<double> a(count), z(count);
            ck(cudaMemcpyAsync(it.data(), iters, count * sizeof(long long), cudaMemcpyDeviceToHost, s), "copy results");
            ck(cudaMemcpyAsync(st.data(), status, count * sizeof(int), cudaMemcpyDeviceToHost, s), "copy results");
            ck(cudaMemcpyAsync(a.data(), r0, count * sizeof(double), cudaMemcpyDeviceToHost, s), "copy results");
            ck(cudaMemcpyAsync(z.data(), rnow, count * sizeof(double), cudaMemcpyDeviceToHost, s), "copy results");
            ck(cudaStreamSynchronize(s), "stream sync");
            for (int q = 0; q < count; ++q) {
                results[q].status = st[q];
                results[q].iters = it[q];
                results[q].r0 = a[q];
                results[q].r_final = z[q];
                results[q].last_check = rel ? (a[q] > 0 ? z[q] / a[q] : 0.0) : z[q];
            }
        } catch (...) {
            h->batch_cache.reset();  // a failed call leaves no plan behind
            throw;
        }
    });
}

extern "C" int lap_last_batch_config(lap_handle h, int32_t* tail_size, int32_t* tiling,
                                     int32_t* item_points, int32_t* persistent, int32_t* tuned)
{
    return guarded([&] {
        if (!h) fail(LAP_EINVAL, "handle is NULL");
        if (tail_size) *tail_size = h->last_batch.tail;
        if (tiling) *tiling = h->last_batch.tiles == 0 ? -1 : h->last_batch.tiles;
        if (item_points) *item_points = h->last_batch.item;
        if (persistent) *persistent = h->last_batch.item == 0 ? 0 : (h->last_batch.persist ? 1 : -1);
        if (tuned) *tuned = h->last_batch_tuned ? 1 : 0;
    });
}
