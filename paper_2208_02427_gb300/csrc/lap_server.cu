// lap_server.cu -- the serving loop: continuous batching of solve requests under an HBM
// budget (lap_server_*), on the batched V-cycle and point kernels.
#include "lap_host.cuh"

using namespace lap;

// ---- serving: continuous batching over a stream of requests ----------------------------------

namespace {

struct SrvRequest {
    int64_t id = 0;
    lap_grid g{};
    double* psi = nullptr;
    int method = LAP_MG_MIXED;  // LAP_MG, LAP_MG_MIXED or LAP_SOR_RB
    double w = 1.0, tol = 1e-10;
    int64_t max_iter = 0;       // V-cycles, or sweeps for SOR
    int state = 0;              // 0 queued, 1 running, 2 finished
    bool fresh = true;          // admitted, initial residual not yet taken
    size_t off = 0, bytes = 0;  // block of the pool holding its hierarchy
    int nlev = 1;
    std::vector<BatchLevel<double>> lv64;
    std::vector<BatchLevel<float>> lv32;
    double r0 = 0.0, rnow = 0.0;
    long long steps = 0;        // iterations run (V-cycles, or sweep batches for SOR)
    lap_result res{};
};

}  // namespace

struct lap_server_s {
    lap_handle h = nullptr;
    size_t budget = 0;
    char* pool = nullptr;
    std::map<size_t, size_t> free_blocks;  // offset -> bytes
    std::deque<int64_t> queue;
    std::map<int64_t, SrvRequest> reqs;
    int64_t next_id = 1;
    int max_running = 1024;
    int sor_sweeps = 50;
    lap_params mg{};  // nu1, nu2, coarsest_min, max_levels, smoother_w, inner_cycles
    char* stage = nullptr;
    size_t stage_bytes = 0;
    std::deque<int64_t> completed;  // finished requests, in the order their steps ended
};

namespace {

bool pool_alloc(lap_server S, size_t bytes, size_t* off)
{
    for (auto it = S->free_blocks.begin(); it != S->free_blocks.end(); ++it)
        if (it->second >= bytes) {
            *off = it->first;
            const size_t rest = it->second - bytes;
            const size_t at = it->first + bytes;
            S->free_blocks.erase(it);
            if (rest) S->free_blocks[at] = rest;
            return true;
        }
    return false;
}

void pool_free(lap_server S, size_t off, size_t bytes)
{
    auto it = S->free_blocks.emplace(off, bytes).first;
    auto next = std::next(it);
    if (next != S->free_blocks.end() && it->first + it->second == next->first) {
        it->second += next->second;
        S->free_blocks.erase(next);
    }
    if (it != S->free_blocks.begin()) {
        auto prev = std::prev(it);
        if (prev->first + prev->second == it->first) {
            prev->second += it->second;
            S->free_blocks.erase(it);
        }
    }
}

// Level descriptors of a request's hierarchy, carved from `cv` (a Sizer or a Carver).
template <class C>
void srv_levels(lap_server S, SrvRequest& r, C& cv)
{
    const Coef c = make_coef(r.g.dx, r.g.dy);
    const bool mg = r.method != LAP_SOR_RB;
    r.nlev = mg ? mg_level_count(r.g.m, r.g.n, S->mg.coarsest_min, S->mg.max_levels) : 1;
    r.lv64.assign(r.nlev, BatchLevel<double>{});
    r.lv32.assign(r.nlev, BatchLevel<float>{});
    int m = r.g.m, n = r.g.n;
    for (int l = 0; l < r.nlev; ++l) {
        BatchLevel<double>& d = r.lv64[l];
        BatchLevel<float>& f = r.lv32[l];
        d.m = f.m = m;
        d.n = f.n = n;
        d.pitch = l == 0 ? r.g.pitch : round_up(m, 32);
        f.pitch = round_up(m, 32);
        d.unit_beta = f.unit_beta = c.unit_beta;
        d.inv_d_shift = c.inv_d_shift;
        d.b2 = f.b2 = c.b2;
        d.d = f.d = c.d;
        d.inv_d = f.inv_d = c.inv_d;
        d.w = r.w;
        d.omw = 1.0 - r.w;
        const bool last = l == r.nlev - 1;
        if (mg && last) {
            if ((int64_t)(m - 2) * (n - 2) > COARSE_MAX_UNKNOWNS)
                fail(LAP_EUNSUPPORTED, "coarsest level with more than 1024 unknowns");
            d.ainv_t = f.ainv_t = nullptr;  // set at admission (needs the device)
        }
        if (l == 0) d.u = r.psi;
        if (r.method == LAP_MG) {
            if (l > 0) {
                d.u = cv.template take<double>((size_t)n * d.pitch);
                d.q = cv.template take<double>((size_t)n * d.pitch);
            }
            if (!last) d.r = cv.template take<double>((size_t)n * d.pitch);
        } else if (r.method == LAP_MG_MIXED) {
            f.u = cv.template take<float>((size_t)n * f.pitch);
            f.q = cv.template take<float>((size_t)n * f.pitch);
            if (!last) f.r = cv.template take<float>((size_t)n * f.pitch);
        }
        m = (m - 1) / 2 + 1;
        n = (n - 1) / 2 + 1;
    }
}

// Small-level tail sizes of the server's V-cycles (one CTA per request runs its levels at
// or below the size).
constexpr int SERVER_TAIL_FP64 = 33;
constexpr int SERVER_TAIL_FP32 = 129;

struct SrvPlan {
    std::vector<BatchLevel<double>> lv64;
    std::vector<BatchLevel<float>> lv32;
    std::vector<BatchItem> items;
    std::vector<TailJob> jobs;
    std::vector<TileItem> tiles;
    LevelLists mg64, mg32;
    std::pair<int, int> sor, update, init, norm;
    std::vector<int> first_init, first_norm;
    std::vector<int> sor_upto;  // items of `sor` (a prefix) swept in the step's k-th sweep
};

}  // namespace

extern "C" int lap_server_create(lap_server* out, lap_handle h, size_t hbm_budget_bytes,
                                 const lap_params* mg, int max_running, int sor_sweeps)
{
    return guarded([&] {
        if (!out || !h) fail(LAP_EINVAL, "NULL server or handle");
        *out = nullptr;
        if (max_running < 1 || sor_sweeps < 1) fail(LAP_EINVAL, "max_running and sor_sweeps must be >= 1");
        lap_params d;
        lap_default_params(&d);
        if (mg) d = *mg;
        d.method = LAP_MG;
        check_params(&d);
        set_device(h);
        lap_server S = new lap_server_s();
        S->h = h;
        S->budget = hbm_budget_bytes;
        S->mg = d;
        S->max_running = max_running;
        S->sor_sweeps = sor_sweeps;
        if (hbm_budget_bytes) {
            try {
                S->pool = (char*)dev_alloc(h, hbm_budget_bytes);
            } catch (...) {
                delete S;
                throw;
            }
            S->free_blocks[0] = hbm_budget_bytes;
        }
        *out = S;
    });
}

extern "C" void lap_server_destroy(lap_server S)
{
    if (!S) return;
    cudaSetDevice(S->h->device);
    cudaDeviceSynchronize();
    dev_free(S->h, S->pool, S->budget);
    dev_free(S->h, S->stage, S->stage_bytes);
    delete S;
}

extern "C" int lap_server_submit(lap_server S, const lap_grid* g, double* psi_dev, int method,
                                 double w, double tol, int64_t max_iter, int64_t* id)
{
    return guarded([&] {
        if (!S || !id) fail(LAP_EINVAL, "NULL server or id");
        check_grid(g);
        set_device(S->h);
        check_device_ptr(S->h, psi_dev, "psi");
        if (method != LAP_MG && method != LAP_MG_MIXED && method != LAP_SOR_RB)
            fail(LAP_EINVAL, "served methods: LAP_MG, LAP_MG_MIXED, LAP_SOR_RB");
        if (method == LAP_SOR_RB && !(w > 0.0 && w < 2.0)) fail(LAP_EINVAL, "w must lie in (0, 2)");
        if (!(tol >= 0.0) || max_iter < 0) fail(LAP_EINVAL, "tol >= 0 and max_iter >= 0");
        SrvRequest r;
        r.id = S->next_id++;
        r.g = *g;
        r.psi = psi_dev;
        r.method = method;
        r.w = method == LAP_SOR_RB ? w : 1.0;
        r.tol = tol;
        r.max_iter = max_iter;
        Sizer sz;
        srv_levels(S, r, sz);
        r.bytes = (size_t)round_up((int64_t)sz.off, 256);  // every block starts 256-byte aligned
        if (r.bytes > S->budget && r.bytes) fail(LAP_ENOMEM, "request needs more than the whole budget");
        *id = r.id;
        S->queue.push_back(r.id);
        S->reqs.emplace(r.id, std::move(r));
    });
}

extern "C" int lap_server_poll(lap_server S, int64_t id, lap_result* out)
{
    if (!S || !out) return LAP_EINVAL;
    auto it = S->reqs.find(id);
    if (it == S->reqs.end()) return LAP_EINVAL;
    if (it->second.state != 2) return 0;
    *out = it->second.res;
    S->reqs.erase(it);
    return 1;
}

extern "C" int lap_server_drain(lap_server S, int64_t* ids, lap_result* results, int capacity,
                                int* count)
{
    return guarded([&] {
        if (!S || !count || capacity < 0 || (capacity > 0 && (!ids || !results)))
            fail(LAP_EINVAL, "NULL server, arrays or count, or negative capacity");
        int n = 0;
        while (n < capacity && !S->completed.empty()) {
            const int64_t id = S->completed.front();
            S->completed.pop_front();
            auto it = S->reqs.find(id);
            if (it == S->reqs.end()) continue;  // already taken by lap_server_poll
            ids[n] = id;
            results[n] = it->second.res;
            S->reqs.erase(it);
            ++n;
        }
        *count = n;
    });
}

extern "C" int lap_server_step(lap_server S, void* stream, int* running, int* queued)
{
    return guarded([&] {
        if (!S) fail(LAP_EINVAL, "server is NULL");
        set_device(S->h);
        cudaStream_t st = (cudaStream_t)stream;
        int nrun = 0;
        for (auto& kv : S->reqs) nrun += kv.second.state == 1;
        // ---- admission: FIFO, while a slot is free and the hierarchy fits the pool ----
        while (!S->queue.empty() && nrun < S->max_running) {
            SrvRequest& r = S->reqs.at(S->queue.front());
            size_t off = 0;
            if (r.bytes && !pool_alloc(S, r.bytes, &off)) break;
            r.off = off;
            Carver cv(S->pool + off);
            srv_levels(S, r, cv);
            if (r.method != LAP_SOR_RB) {
                BatchLevel<double>& d = r.lv64[r.nlev - 1];
                const double* ainv = coarse_inverse(S->h, d.m, d.n, d.b2, d.d);
                d.ainv_t = ainv;
                r.lv32[r.nlev - 1].ainv_t = ainv;
            }
            if (r.bytes) ck(cudaMemsetAsync(S->pool + off, 0, r.bytes, st), "zero hierarchy");
            r.state = 1;
            r.fresh = true;
            S->queue.pop_front();
            ++nrun;
        }
        std::vector<SrvRequest*> run;
        for (auto& kv : S->reqs)
            if (kv.second.state == 1) run.push_back(&kv.second);
        if (queued) *queued = (int)S->queue.size();
        if (run.empty()) {
            if (running) *running = 0;
            return;
        }
        // ---- the plan of this step ----
        const int R = (int)run.size();
        SrvPlan P;
        std::vector<int> base(R);
        for (int q = 0; q < R; ++q) {
            base[q] = (int)P.lv64.size();
            for (int l = 0; l < run[q]->nlev; ++l) {
                BatchLevel<double> d = run[q]->lv64[l];
                BatchLevel<float> f = run[q]->lv32[l];
                d.problem = f.problem = q;
                P.lv64.push_back(d);
                P.lv32.push_back(f);
            }
        }
        std::vector<int> nlev(R);
        for (int q = 0; q < R; ++q) nlev[q] = run[q]->nlev;
        auto mg_lists = [&](int method, LevelLists& L) {
            std::vector<int> who;
            for (int q = 0; q < R; ++q)
                if (run[q]->method == method) who.push_back(q);
            // no timing across steps (the running set changes): fixed tail sizes
            const int ts = S->mg.tail_size != 0 ? S->mg.tail_size
                                                : (method == LAP_MG_MIXED ? SERVER_TAIL_FP32 : SERVER_TAIL_FP64);
            const bool fused = method == LAP_MG_MIXED && !S->mg.unfused &&
                               fused32_supported(S->mg.nu1, S->mg.nu2);
            build_lists(L, P.items, P.jobs, who, base, nlev, P.lv64, ts, fused ? &P.tiles : nullptr,
                        S->mg.nu1, S->mg.nu2);
        };
        mg_lists(LAP_MG, P.mg64);
        mg_lists(LAP_MG_MIXED, P.mg32);
        auto level0 = [&](auto pred, std::vector<int>* first) {
            const int i0 = (int)P.items.size();
            for (int q = 0; q < R; ++q) {
                if (first) first->push_back((int)P.items.size() - i0);
                if (pred(*run[q])) add_items(P.items, base[q], run[q]->g.m, run[q]->g.n);
            }
            if (first) first->push_back((int)P.items.size() - i0);
            return std::make_pair(i0, (int)P.items.size() - i0);
        };
        // An SOR request sweeps min(sor_sweeps, sweeps left of its max_iter) times this step, so
        // that its last check period is cut short at max_iter as lap_solve cuts it. Its items are
        // laid out by that count, largest first: sweep k takes a prefix of the list.
        {
            auto sweeps_now = [&](int q) {
                const SrvRequest& r = *run[q];
                return (int)std::min<int64_t>(S->sor_sweeps, r.max_iter - (int64_t)r.steps * S->sor_sweeps);
            };
            std::vector<int> sor_q;
            for (int q = 0; q < R; ++q)
                if (run[q]->method == LAP_SOR_RB) sor_q.push_back(q);
            std::stable_sort(sor_q.begin(), sor_q.end(),
                             [&](int a, int c) { return sweeps_now(a) > sweeps_now(c); });
            P.sor.first = (int)P.items.size();
            P.sor_upto.assign(S->sor_sweeps, 0);
            for (int q : sor_q) {
                add_items(P.items, base[q], run[q]->g.m, run[q]->g.n);
                const int upto = (int)P.items.size() - P.sor.first;
                for (int k = 0; k < sweeps_now(q); ++k) P.sor_upto[k] = upto;
            }
            P.sor.second = (int)P.items.size() - P.sor.first;
        }
        P.update = level0([](const SrvRequest& r) { return r.method == LAP_MG_MIXED; }, nullptr);
        P.init = level0([](const SrvRequest& r) { return r.fresh; }, &P.first_init);
        P.norm = level0([](const SrvRequest&) { return true; }, &P.first_norm);
        // ---- stage: descriptors, items, per-request state ----
        std::vector<int> act(R, 1), stat(R, 1);
        std::vector<long long> it(R), cap(R);
        std::vector<double> r0(R), tolv(R);
        for (int q = 0; q < R; ++q) {
            it[q] = run[q]->steps;
            r0[q] = run[q]->r0;
            tolv[q] = run[q]->tol;
            // iterations a request may run: V-cycles, or batches of sor_sweeps sweeps
            cap[q] = run[q]->method == LAP_SOR_RB ? (run[q]->max_iter + S->sor_sweeps - 1) / S->sor_sweeps
                                                  : run[q]->max_iter;
        }
        auto carve_stage = [&](auto& cv) {
            auto* lv64 = cv.template take<BatchLevel<double>>(P.lv64.size());
            auto* lv32 = cv.template take<BatchLevel<float>>(P.lv32.size());
            auto* items = cv.template take<BatchItem>(std::max<size_t>(1, P.items.size()));
            auto* jobs = cv.template take<TailJob>(std::max<size_t>(1, P.jobs.size()));
            auto* tiles = cv.template take<TileItem>(std::max<size_t>(1, P.tiles.size()));
            auto* fi = cv.template take<int>(P.first_init.size());
            auto* fn = cv.template take<int>(P.first_norm.size());
            auto* active = cv.template take<int>(R);
            auto* status = cv.template take<int>(R);
            auto* remaining = cv.template take<int>(1);
            auto* iters = cv.template take<long long>(R);
            auto* maxit = cv.template take<long long>(R);
            auto* dr0 = cv.template take<double>(R);
            auto* rnow = cv.template take<double>(R);
            auto* dtol = cv.template take<double>(R);
            auto* pinit = cv.template take<double>(std::max(1, P.init.second));
            auto* pnorm = cv.template take<double>(std::max(1, P.norm.second));
            auto* done = cv.template take<Completion>(R);
            auto* ndone = cv.template take<int>(1);
            return std::make_tuple(lv64, lv32, items, jobs, tiles, fi, fn, active, status, remaining,
                                   iters, maxit, dr0, rnow, dtol, pinit, pnorm, done, ndone);
        };
        Sizer sz;
        carve_stage(sz);
        if (sz.off > S->stage_bytes) {
            dev_free(S->h, S->stage, S->stage_bytes);
            S->stage = nullptr;
            S->stage_bytes = 0;
            const size_t nb = (size_t)round_up((int64_t)sz.off * 2, 1 << 20);
            S->stage = (char*)dev_alloc(S->h, nb);
            S->stage_bytes = nb;
        }
        Carver cv(S->stage);
        // plain variables (lambdas below capture them; capturing structured bindings is C++20)
        BatchLevel<double>* lv64;
        BatchLevel<float>* lv32;
        BatchItem* items;
        TailJob* jobs;
        TileItem* tiles;
        int *fi, *fn, *active, *status, *remaining, *ndone;
        long long *iters, *maxit;
        double *dr0, *rnow, *dtol, *pinit, *pnorm;
        Completion* done;
        std::tie(lv64, lv32, items, jobs, tiles, fi, fn, active, status, remaining, iters, maxit, dr0,
                 rnow, dtol, pinit, pnorm, done, ndone) = carve_stage(cv);
        auto up = [&](void* dst, const void* src, size_t bytes) {
            if (bytes) ck(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st), "upload plan");
        };
        up(lv64, P.lv64.data(), P.lv64.size() * sizeof(P.lv64[0]));
        up(lv32, P.lv32.data(), P.lv32.size() * sizeof(P.lv32[0]));
        up(items, P.items.data(), P.items.size() * sizeof(BatchItem));
        up(jobs, P.jobs.data(), P.jobs.size() * sizeof(TailJob));
        up(tiles, P.tiles.data(), P.tiles.size() * sizeof(TileItem));
        if (P.mg32.fused) ck(prepare_fused32(), "tile kernel attributes");
        up(fi, P.first_init.data(), P.first_init.size() * sizeof(int));
        up(fn, P.first_norm.data(), P.first_norm.size() * sizeof(int));
        up(active, act.data(), R * sizeof(int));
        up(status, stat.data(), R * sizeof(int));
        up(remaining, &R, sizeof(int));
        up(iters, it.data(), R * sizeof(long long));
        up(maxit, cap.data(), R * sizeof(long long));
        up(dr0, r0.data(), R * sizeof(double));
        up(dtol, tolv.data(), R * sizeof(double));
        ck(cudaMemsetAsync(ndone, 0, sizeof(int), st), "zero completions");
        auto list = [&](std::pair<int, int> r) { return BatchList{items + r.first, r.second}; };
        // ---- one iteration of every running request ----
        ck(launch_b_sumsq(list(P.init), lv64, active, pinit, lv32, st), "server residual");
        ck(launch_b_converge(pinit, fi, R, active, dr0, rnow, iters, status, remaining, 0, true, 0.0,
                             st, dtol, maxit, done, ndone), "server convergence");
        enqueue_vcycle(list, P.mg64, lv64, active, jobs, S->mg, S->mg.smoother_w, st);
        for (int k = 0; k < S->mg.inner_cycles && P.mg32.levels; ++k) {
            if (P.mg32.fused)
                enqueue_vcycle32_fused(list, P.mg32, lv32, active, jobs, tiles, S->mg, S->mg.smoother_w,
                                       k == 0, st, k == S->mg.inner_cycles - 1 ? lv64 : nullptr);
            else
                enqueue_vcycle(list, P.mg32, lv32, active, jobs, S->mg, S->mg.smoother_w, st);
        }
        // fused: the level-0 ascents did psi += e except where a tail holds level 0
        ck(launch_b_update(list(P.mg32.fused ? P.mg32.upd0 : P.update), lv64, active, lv32, st),
           "server update");
        for (int k = 0; k < S->sor_sweeps && P.sor.second; ++k) {
            const std::pair<int, int> swept{P.sor.first, P.sor_upto[k]};
            for (int colour = 0; colour < 2; ++colour)
                ck(launch_b_rb(list(swept), lv64, active, colour, false, 1.0, st, true), "server sweep");
        }
        ck(launch_b_sumsq(list(P.norm), lv64, active, pnorm, lv32, st, dr0), "server residual");
        ck(launch_b_converge(pnorm, fn, R, active, dr0, rnow, iters, status, remaining, 1, true, 0.0,
                             st, dtol, maxit, done, ndone), "server convergence");
        // ---- the step's completion list (written by the convergence tests), read once ----
        std::vector<Completion> fin(R);
        int nfin = 0;
        ck(cudaMemcpyAsync(&nfin, ndone, sizeof(int), cudaMemcpyDeviceToHost, st), "download completions");
        ck(cudaMemcpyAsync(fin.data(), done, R * sizeof(Completion), cudaMemcpyDeviceToHost, st),
           "download completions");
        ck(cudaMemcpyAsync(r0.data(), dr0, R * sizeof(double), cudaMemcpyDeviceToHost, st), "download norms");
        ck(cudaStreamSynchronize(st), "stream sync");
        // ---- retire finished requests; the others ran exactly one iteration ----
        std::vector<char> finished(R, 0);
        std::sort(fin.begin(), fin.begin() + nfin,
                  [&](const Completion& a, const Completion& b) { return run[a.problem]->id < run[b.problem]->id; });
        for (int k = 0; k < nfin; ++k) {
            const Completion& c = fin[k];
            SrvRequest& r = *run[c.problem];
            finished[c.problem] = 1;
            r.steps = c.iters;
            r.r0 = c.r0;
            r.rnow = c.rnow;
            r.res.status = c.status;
            // SOR: sweeps, the last batch cut short at max_iter
            r.res.iters = r.method == LAP_SOR_RB ? std::min<int64_t>(c.iters * S->sor_sweeps, r.max_iter)
                                                 : c.iters;
            r.res.r0 = c.r0;
            r.res.r_final = c.rnow;
            r.res.last_check = c.r0 > 0 ? c.rnow / c.r0 : 0.0;
            r.state = 2;
            r.fresh = false;
            if (r.bytes) pool_free(S, r.off, r.bytes);
            S->completed.push_back(r.id);
        }
        int still = 0;
        for (int q = 0; q < R; ++q) {
            if (finished[q]) continue;
            SrvRequest& r = *run[q];
            r.fresh = false;
            r.steps += 1;
            r.r0 = r0[q];
            ++still;
        }
        if (running) *running = still;
    });
}
