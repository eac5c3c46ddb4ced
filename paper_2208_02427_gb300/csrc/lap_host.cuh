// lap_host.cuh -- host-side internals shared by the C-ABI sources of liblaplace.so
// (lap_api.cu: handles, single-grid solves and component calls; lap_batched.cu: many grids
// at once; lap_server.cu: the serving loop). Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <stdexcept>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/laplace.h"
#include "lap_internal.cuh"

namespace lap {

int64_t launches_now();
void add_launches(int64_t k);

// Chooses the small-level tail size of one shape by timing. The tail changes how a V-cycle
// is launched and nothing else (every candidate gives the same iterates bit for bit), so
// the candidates are tried on the first cycles of real solves: each cycle (or check
// period) runs with the next untried candidate, its device time per cycle is recorded,
// and once every candidate has been timed the fastest is kept for the handle's lifetime.
struct TailTuner {
    std::vector<int> cand;  // tail sizes; -1 = no tail
    std::vector<double> ms; // best time per cycle seen, +inf = not tried yet
    int best = 0;
    bool done = false;
    void init(std::vector<int> c)
    {
        cand = std::move(c);
        ms.assign(cand.size(), HUGE_VAL);
        best = 0;
        done = cand.size() <= 1;
    }
    int next() const
    {
        if (done) return best;
        for (size_t i = 0; i < cand.size(); ++i)
            if (ms[i] == HUGE_VAL) return (int)i;
        return best;
    }
    void record(int i, double v)
    {
        if (done || i < 0 || i >= (int)cand.size() || !(v > 0.0)) return;
        ms[i] = std::min(ms[i], v);
        bool all = true;
        for (size_t k = 0; k < cand.size(); ++k) {
            if (ms[k] == HUGE_VAL) all = false;
            else if (ms[k] < ms[best] || ms[best] == HUGE_VAL) best = (int)k;
        }
        done = all;
    }
};

// One launch configuration of a batched V-cycle; none of its choices changes a computed value.
struct BatchConfig {
    int tail;   // small-level tail size (-1: none; see TailTuner)
    int tiles;  // FP32 levels of the mixed solver: 0 = one kernel per pass (temporal depth 1),
                // 1..FUSED32_VARIANTS = a level's whole descent / ascent per tile load (depth nu)
                // with that tile variant (CTA size and region rows)
    int item;   // interior points per work item of the per-pass kernels
    int persist;  // 1: every phase a persistent launch (resident CTAs claim its items), 0: one CTA per item
    bool operator==(const BatchConfig& o) const
    {
        return tail == o.tail && tiles == o.tiles && item == o.item && persist == o.persist;
    }
};

// Chooses a batched solve's configuration by timing real cycles, one knob at a time (a
// coordinate search): stage 0 the small-level tail (the level-to-CTA mapping), stage 1 the
// FP32 levels' temporal blocking and tile shape (mixed solver), stage 2 the work-item size of
// the per-pass kernels (when some run), stage 3 one CTA per work item or persistent launches
// (resident CTAs claiming items from a counter). A stage's candidates are the best configuration so far
// with that one knob changed; each is timed on one cycle in which every problem still runs
// (the graph of a candidate is captured on an earlier cycle), and the fastest is kept. The
// cycles being timed are real cycles of the solve, and all candidates give the same iterates.
struct BatchTuner {
    std::vector<BatchConfig> cand;
    std::vector<double> ms;  // time per cycle, +inf = not timed yet
    int best = 0;
    int stage = 0;
    int stage_begin = 0;
    bool done = false;
    std::vector<int> tails, tilings, items, persists;  // the values each stage tries
    void init(std::vector<int> tail_values, std::vector<int> tiling_values, std::vector<int> item_values,
              std::vector<int> persist_values)
    {
        tails = std::move(tail_values);
        tilings = std::move(tiling_values);
        items = std::move(item_values);
        persists = std::move(persist_values);
        cand.clear();
        ms.clear();
        best = stage = stage_begin = 0;
        done = false;
        for (int t : tails) add(BatchConfig{t, tilings.front(), items.front(), persists.front()});
        if (cand.size() <= 1) advance();
    }
    void add(BatchConfig c)
    {
        for (const BatchConfig& k : cand)
            if (k == c) return;
        cand.push_back(c);
        ms.push_back(HUGE_VAL);
    }
    int next() const
    {
        if (done) return best;
        for (size_t i = stage_begin; i < cand.size(); ++i)
            if (ms[i] == HUGE_VAL) return (int)i;
        return best;
    }
    void record(int i, double v)
    {
        if (done || i < 0 || i >= (int)cand.size() || !(v > 0.0)) return;
        ms[i] = std::min(ms[i], v);
        if (ms[best] == HUGE_VAL || ms[i] < ms[best]) best = i;
        for (size_t k = stage_begin; k < cand.size(); ++k)
            if (ms[k] == HUGE_VAL) return;
        advance();
    }
    // The next stage with more than the current best to try, or done.
    void advance()
    {
        while (stage < 3) {
            ++stage;
            stage_begin = (int)cand.size();
            const BatchConfig b = cand[best];
            const std::vector<int>& values = stage == 1 ? tilings : stage == 2 ? items : persists;
            for (int v : values) {
                BatchConfig c = b;
                if (stage == 1) c.tiles = v;
                else if (stage == 2) c.item = v;
                else c.persist = v;
                if (c == b) continue;
                if (stage == 2 && b.tiles != 0 && c.item != b.item) {
                    // with tiles the per-pass kernels only serve the tail's neighbours: skip
                    continue;
                }
                add(c);
            }
            if ((int)cand.size() > stage_begin) return;
        }
        done = true;
    }
};

extern thread_local std::string t_last_error;

struct Error {
    int code;
    std::string msg;
};

[[noreturn]] inline void fail(int code, const std::string& msg) { throw Error{code, msg}; }

inline void ck(cudaError_t e, const char* what)
{
    if (e != cudaSuccess) fail(LAP_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

template <class F>
int guarded(F&& body)
{
    try {
        body();
        return LAP_OK;
    } catch (const Error& e) {
        t_last_error = e.msg;
        return e.code;
    } catch (const std::bad_alloc&) {
        t_last_error = "host allocation failed";
        return LAP_ENOMEM;
    } catch (...) {
        t_last_error = "unexpected internal error";
        return LAP_ECUDA;
    }
}

inline int64_t round_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

// A batched solve's plan kept in the handle for the next call on the same batch (defined in
// lap_batched.cu; destroyed with the handle or when another batch or call takes the arena).
struct BatchCacheBase {
    virtual ~BatchCacheBase() = default;
};

// Host-side copy of a line-solver table set plus its device allocation.
struct LineEntry {
    LineTables t;
    double* dev = nullptr;
    size_t bytes = 0;
};

struct CoarseEntry {
    double* dev = nullptr;
    size_t bytes = 0;
};

}  // namespace lap

struct lap_handle_s {
    int device = 0;
    size_t budget = 0;    // 0 = unlimited
    size_t held = 0;      // bytes of device memory held (arena + tables)
    double* arena = nullptr;
    size_t arena_bytes = 0;
    uint64_t arena_epoch = 0;  // counts the calls that carved the arena (arena())
    std::unique_ptr<lap::BatchCacheBase> batch_cache;  // the last batched solve's plan
    double* pinned = nullptr;  // 8 doubles of pinned host memory for results
    std::map<std::tuple<int, double, double, double, int>, lap::LineEntry> lines;
    std::map<std::tuple<int, int, double>, lap::CoarseEntry> coarse;
    // CUDA graphs of whole check periods (the iterations between two stopping tests),
    // keyed by every pointer and parameter baked into them; replayed on the caller's stream
    bool use_graphs = true;
    cudaStream_t capture = nullptr;
    std::map<std::string, std::pair<cudaGraphExec_t, int64_t>> graphs;  // exec, kernels
    // Small-level tail sizes chosen by timing, per shape (see TailTuner)
    std::map<std::string, lap::TailTuner> tail_tuners;
    std::map<std::string, lap::BatchTuner> batch_tuners;  // batched solves' configurations
    lap::BatchConfig last_batch{0, 0, 0, 0};  // the configuration the last batched cycle ran
    bool last_batch_tuned = false;         // whether its tuner had finished
    cudaEvent_t ev[2] = {nullptr, nullptr};
    // y-line scratch of line relaxation: forward-elimination values and chunk ends (grown on
    // demand)
    double* lscratch = nullptr;
    size_t lscratch_bytes = 0;
    // x-line sweeps: error word, item counter and row flags; one block of at least 1 MiB,
    // allocated on first use and grown only for more than 262,140 lines
    unsigned* lsync = nullptr;
    size_t lsync_bytes = 0;
    // device copy of the field of lap_solve_host (grown on demand)
    double* hfield = nullptr;
    size_t hfield_bytes = 0;
};

namespace lap {

void set_device(lap_handle h);
void* dev_alloc(lap_handle h, size_t bytes);
void dev_free(lap_handle h, void* p, size_t bytes);
void drop_graphs(lap_handle h);
// Scratch for one call: grows (never shrinks) the handle's arena.
double* arena(lap_handle h, size_t bytes);

// Carves aligned sub-buffers out of a byte range.
struct Carver {
    char* base;
    size_t off = 0;
    explicit Carver(void* b) : base((char*)b) {}
    template <class T>
    T* take(size_t count)
    {
        off = (size_t)round_up((int64_t)off, 256);
        T* p = (T*)(base + off);
        off += count * sizeof(T);
        return p;
    }
};
// The same carving sequence without memory, to size the arena first.
struct Sizer {
    size_t off = 0;
    template <class T>
    T* take(size_t count)
    {
        off = (size_t)round_up((int64_t)off, 256) + count * sizeof(T);
        return nullptr;
    }
};

void check_grid(const lap_grid* g);
void check_device_ptr(lap_handle h, const void* p, const char* what, bool allow_null = false);
void check_params(const lap_params* p);

// line relaxation: cached tables of a line length and coefficients; the tables, coefficients
// and scratch of a half sweep (allocating only on a shape's first use); one zebra half sweep
const LineTables& line_tables(lap_handle h, int N, double alpha, double delta, double wc,
                              int max_chunks = LINE_MAX_CHUNKS);
const LineTables& line_setup(lap_handle h, const Field& f, const Coef& c, double w, int form,
                             int direction, LineCoefs* k, double** scratch);
void line_half_sweep(lap_handle h, const Field& f, const Coef& c, double w, int form,
                     int direction, cudaStream_t s);

// the coarsest level's 5-point matrix, inverted once per shape (transposed, on the device)
constexpr int COARSE_MAX_UNKNOWNS = 1024;
const double* coarse_inverse(lap_handle h, int m, int n, double b2, double d);
int mg_level_count(int m, int n, int coarsest_min, int max_levels);

// the timing-based choice of the small-level tail
std::vector<int> tail_candidates(bool batched, bool fp32, int tail_size);
std::string tuner_key(char kind, const lap_params* p, const std::vector<int>& shape);
cudaEvent_t tuner_event(lap_handle h, int k);

// ---- V-cycles over many problems (lap_batched.cu, lap_server.cu) ----
// Interior points per work item (rows are not split). Measured on the 4096-grid batch (sides
// 33..513, V(2,2) to 1e-10): FP64 145 / 140 / 140 / 145 ms at 2048 / 8192 / 16384 / 32768
// points, the mixed solver 74 / 71 / 69 / 68 ms; 8192 for both.
constexpr int BATCH_ITEM_POINTS = 8192;
void add_items(std::vector<BatchItem>& items, int level_index, int m, int n,
               int points = BATCH_ITEM_POINTS);

// Per-level work lists of one V-cycle over a set of problems: [first, count) into the items
// (fine, all, coarse) or into the tail jobs (tail).
struct LevelLists {
    std::vector<std::pair<int, int>> fine, all, coarse, tail;
    std::vector<std::pair<int, int>> tiles;  // FP32 tile items of the fine lists (fused cycle)
    std::pair<int, int> upd0{0, 0};  // fused: level-0 items of the problems without level-0 tiles
    bool fused = false;
    int tile_variant = 1;  // the fused FP32 levels' tile variant
    unsigned* claim = nullptr;  // non-null: every launch persistent, claiming items here (BatchList)
    int levels = 0;
    int max_coarse = 0;
};

// First level of a problem that the small-level tail runs (both sides <= tail_size), or
// nlev when it has none.
int tail_start(const BatchLevel<double>* lv, int nlev, int tail_size);

// Lists of one V-cycle over problems `who`: problem q owns levels base[q] .. base[q] +
// nlev[q] - 1 of lv. Levels above a problem's tail go through item lists, the tail is one job.
// With tiles, the fine levels also get the tile items of the fused FP32 descent/ascent.
void build_lists(LevelLists& L, std::vector<BatchItem>& items, std::vector<TailJob>& jobs,
                 const std::vector<int>& who, const std::vector<int>& base,
                 const std::vector<int>& nlev, const std::vector<BatchLevel<double>>& lv,
                 int tail_size, std::vector<TileItem>* tiles = nullptr, int nu1 = 0, int nu2 = 0,
                 int tile_variant = 1, int item_points = BATCH_ITEM_POINTS);

// One V-cycle over every active problem of L: descend (coarsest solves and tails start when
// the descent reaches a problem's coarsest or tail level), then ascend; each problem sees
// its own V-cycle.
template <class ListFn, class T>
void enqueue_vcycle(ListFn list, const LevelLists& L, const BatchLevel<T>* lv, const int* active,
                    const TailJob* jobs, const lap_params& p, double smoother_w, cudaStream_t st)
{
    const bool gs = smoother_w == 1.0;
    for (int l = 0; l < L.levels; ++l) {
        ck(launch_b_coarse(list(L.coarse[l]), lv, active, L.max_coarse, st), "batched coarse");
        ck(launch_b_tail(jobs + L.tail[l].first, L.tail[l].second, lv, active, p.nu1, p.nu2, gs,
                         smoother_w, L.max_coarse, st, false, L.claim),
           "batched tail");
        if (l == L.levels - 1) break;
        for (int k = 0; k < p.nu1; ++k)
            for (int colour = 0; colour < 2; ++colour)
                ck(launch_b_rb(list(L.fine[l]), lv, active, colour, gs, smoother_w, st), "batched smoother");
        ck(launch_b_defect(list(L.fine[l]), lv, active, st), "batched defect");
        ck(launch_b_restrict(list(L.all[l + 1]), lv, active, st), "batched restrict");
    }
    for (int l = L.levels - 2; l >= 0; --l) {
        ck(launch_b_prolong(list(L.fine[l]), lv, active, st), "batched prolong");
        for (int k = 0; k < p.nu2; ++k)
            for (int colour = 0; colour < 2; ++colour)
                ck(launch_b_rb(list(L.fine[l]), lv, active, colour, gs, smoother_w, st), "batched smoother");
    }
}

// The FP32 V-cycle with each fine level's descent and ascent as one tile launch over all
// problems (first: the level-0 corrections start at zero).
// fold64 (nullable): the level-0 ascent adds its result to these FP64 fields (psi += e).
template <class ListFn>
void enqueue_vcycle32_fused(ListFn list, const LevelLists& L, const BatchLevel<float>* lv,
                            const int* active, const TailJob* jobs, const TileItem* tiles,
                            const lap_params& p, double smoother_w, bool first, cudaStream_t st,
                            const BatchLevel<double>* fold64 = nullptr)
{
    const bool gs = smoother_w == 1.0;
    for (int l = 0; l < L.levels; ++l) {
        ck(launch_b_coarse(list(L.coarse[l]), lv, active, L.max_coarse, st), "batched coarse");
        ck(launch_b_tail(jobs + L.tail[l].first, L.tail[l].second, lv, active, p.nu1, p.nu2, gs,
                         smoother_w, L.max_coarse, st, false, L.claim),
           "batched tail");
        if (l == L.levels - 1) break;
        ck(launch_b_down32(tiles + L.tiles[l].first, L.tiles[l].second, lv, active, p.nu1,
                           l > 0 || first, gs, smoother_w, st, L.tile_variant, L.claim),
           "batched descent");
    }
    for (int l = L.levels - 2; l >= 0; --l)
        ck(launch_b_up32(tiles + L.tiles[l].first, L.tiles[l].second, lv, active, p.nu2, gs,
                         smoother_w, st, l == 0 ? fold64 : nullptr, L.tile_variant, L.claim),
           "batched ascent");
}

}  // namespace lap
