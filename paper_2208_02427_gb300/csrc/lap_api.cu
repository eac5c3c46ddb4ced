// lap_api.cu -- the C ABI of liblaplace.so (declared in include/laplace.h): handles,
// argument checks, host-side precomputation (line-solver tables, coarsest-grid inverse)
// and the solver loops that drive the kernels on the caller's stream.
#include "lap_host.cuh"

namespace lap {

static std::atomic<int64_t> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
int64_t launches_now() { return g_launches.load(); }
void add_launches(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

thread_local std::string t_last_error;

static std::atomic<int> g_device_sms[ATTR_DEVICES];

int device_sms()
{
    const int d = attr_slot();
    if (d >= 0) {
        const int known = g_device_sms[d].load();
        if (known > 0) return known;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d < 0 ? 0 : d) != cudaSuccess ||
        sms <= 0) {
        cudaGetLastError();
        return 152;  // the attribute query failed: GB300's count
    }
    if (d >= 0) g_device_sms[d].store(sms);
    return sms;
}

int resident_blocks(const void* kernel, int threads, size_t smem)
{
    static std::mutex mu;
    static std::map<std::tuple<const void*, int, int, size_t>, int> known;
    const int d = attr_slot();
    const auto key = std::make_tuple(kernel, d, threads, smem);
    {
        std::lock_guard<std::mutex> g(mu);
        const auto it = known.find(key);
        if (it != known.end()) return it->second;
    }
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem) != cudaSuccess ||
        per < 1) {
        cudaGetLastError();
        per = 1;
    }
    const int v = per * device_sms();
    std::lock_guard<std::mutex> g(mu);
    known[key] = v;
    return v;
}

Coef make_coef(double dx, double dy)
{
    Coef c;
    const double beta = dx / dy;
    c.b2 = beta * beta;
    c.d = 2.0 * (1.0 + c.b2);
    c.inv_d = 1.0 / c.d;
    c.unit_beta = c.b2 == 1.0;
    int e = 0;
    const double mant = std::frexp(c.inv_d, &e);
    c.inv_d_shift = (mant == 0.5 && 1 - e >= 1 && 1 - e <= 60) ? 1 - e : 0;
    return c;
}

void set_device(lap_handle h) { ck(cudaSetDevice(h->device), "cudaSetDevice"); }

void* dev_alloc(lap_handle h, size_t bytes)
{
    if (h->budget && h->held + bytes > h->budget)
        fail(LAP_ENOMEM, "HBM budget of the handle exceeded (" + std::to_string(h->held + bytes) +
                             " > " + std::to_string(h->budget) + " bytes)");
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        fail(LAP_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
    }
    ck(e, "cudaMalloc");
    h->held += bytes;
    return p;
}

void dev_free(lap_handle h, void* p, size_t bytes)
{
    if (!p) return;
    cudaFree(p);
    h->held -= bytes;
}

void drop_graphs(lap_handle h)
{
    for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second.first);
    h->graphs.clear();
}

// Scratch for one call: grows (never shrinks) the handle's arena. Nothing of the handle
// is in flight between calls (lap_solve synchronises), so regrowing is safe.
double* arena(lap_handle h, size_t bytes)
{
    ++h->arena_epoch;  // whatever was kept in the arena is overwritten from here on
    bytes = (size_t)round_up((int64_t)std::max<size_t>(bytes, 256), 1 << 20);
    if (bytes > h->arena_bytes) {
        drop_graphs(h);
        dev_free(h, h->arena, h->arena_bytes);
        h->arena = nullptr;
        h->arena_bytes = 0;
        h->arena = (double*)dev_alloc(h, bytes);
        h->arena_bytes = bytes;
    }
    return h->arena;
}

void check_grid(const lap_grid* g)
{
    if (!g) fail(LAP_EINVAL, "grid is NULL");
    if (g->m < 3 || g->n < 3) fail(LAP_EINVAL, "grid needs m >= 3 and n >= 3");
    if (!(g->dx > 0.0) || !(g->dy > 0.0) || !std::isfinite(g->dx) || !std::isfinite(g->dy))
        fail(LAP_EINVAL, "dx and dy must be finite and > 0");
    if (g->pitch < g->m) fail(LAP_EINVAL, "pitch must be >= m");
    if (g->m > LAP_GRID_MAX_M) fail(LAP_EUNSUPPORTED, "m above LAP_GRID_MAX_M (2^28)");
    if (g->n > LAP_GRID_MAX_N) fail(LAP_EUNSUPPORTED, "n above LAP_GRID_MAX_N (131070)");
    if ((int64_t)g->n * g->pitch > ((int64_t)1 << 40)) fail(LAP_EUNSUPPORTED, "field too large");
}

void check_device_ptr(lap_handle h, const void* p, const char* what, bool allow_null)
{
    if (!p) {
        if (allow_null) return;
        fail(LAP_EINVAL, std::string(what) + " is NULL");
    }
    if (((uintptr_t)p) % 8) fail(LAP_EINVAL, std::string(what) + " is not 8-byte aligned");
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        fail(LAP_EINVAL, std::string(what) + " is not a CUDA pointer");
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
        fail(LAP_EINVAL, std::string(what) + " is not device memory");
    if (h && a.device != h->device)
        fail(LAP_EINVAL, std::string(what) + " lives on another device than the handle");
}

void check_params(const lap_params* p)
{
    if (!p) fail(LAP_EINVAL, "params is NULL");
    if (p->sum_order != LAP_SUM_PAPER && p->sum_order != LAP_SUM_DIAGONAL)
        fail(LAP_EINVAL, "sum_order must be LAP_SUM_PAPER or LAP_SUM_DIAGONAL");
    if (p->sum_order == LAP_SUM_DIAGONAL && p->method != LAP_GS_RB && p->method != LAP_SOR_RB)
        fail(LAP_EINVAL, "sum_order LAP_SUM_DIAGONAL is for LAP_GS_RB and LAP_SOR_RB");
    if (p->method < LAP_JACOBI || p->method > LAP_MG_FP32) fail(LAP_EINVAL, "unknown method");
    if (p->norm < LAP_NORM_L2_REL || p->norm > LAP_NORM_MAXDELTA) fail(LAP_EINVAL, "unknown norm");
    if (!(p->tol >= 0.0)) fail(LAP_EINVAL, "tol must be >= 0");
    if (p->max_iter < 0) fail(LAP_EINVAL, "max_iter must be >= 0");
    if (p->check_every < 1) fail(LAP_EINVAL, "check_every must be >= 1");
    if ((p->method == LAP_SOR_RB || p->method == LAP_ADI || p->method == LAP_SLOR ||
         p->method == LAP_SOR_LEX) &&
        !(p->w > 0.0 && p->w < 2.0))
        fail(LAP_EINVAL, "w must lie in (0, 2)");
    if (p->method == LAP_MG_MIXED && (p->inner_cycles < 1 || p->inner_cycles > 64))
        fail(LAP_EINVAL, "inner_cycles must lie in 1..64");
    if (p->method == LAP_MG_FP32 && p->norm == LAP_NORM_MAXDELTA)
        fail(LAP_EINVAL, "LAP_MG_FP32 stops on an L2 norm");
    if (p->method == LAP_MG || p->method == LAP_MG_MIXED || p->method == LAP_MG_FP32) {
        if (p->nu1 < 0 || p->nu2 < 0 || p->nu1 + p->nu2 > 64)
            fail(LAP_EINVAL, "nu1, nu2 must be >= 0 and nu1 + nu2 <= 64");
        if (p->coarsest_min < 3) fail(LAP_EINVAL, "coarsest_min must be >= 3");
        if (p->max_levels < 0) fail(LAP_EINVAL, "max_levels must be >= 0");
        if (!(p->smoother_w > 0.0 && p->smoother_w < 2.0))
            fail(LAP_EINVAL, "smoother_w must lie in (0, 2)");
        if (p->tail_size < -1 || p->tail_size == 1 || p->tail_size == 2)
            fail(LAP_EINVAL, "tail_size must be -1, 0 or >= 3");
        if (p->tiling < -1 || p->tiling > FUSED32_VARIANTS)
            fail(LAP_EINVAL, "tiling must be -1, 0 or a tile variant 1..3");
        if (p->item_points != 0 && p->item_points < 32)
            fail(LAP_EINVAL, "item_points must be 0 or >= 32");
        if (p->persistent < -1 || p->persistent > 1)
            fail(LAP_EINVAL, "persistent must be -1, 0 or 1");
    }
    if ((p->method == LAP_ADI || p->method == LAP_SLOR) && p->line_form != LAP_FORM_A &&
        p->line_form != LAP_FORM_B)
        fail(LAP_EINVAL, "unknown line form");
}

// ---- line-solver tables --------------------------------------------------------------

constexpr int LINE_MAX_N = 16383;
constexpr int LINE_MIN_CHUNK = 16;

// Thomas solve of tridiag(-alpha, delta, -alpha) x = rhs (size len) on the host.
std::vector<double> host_thomas(int len, double alpha, double delta, const std::vector<double>& rhs)
{
    std::vector<double> den(len), xp(len), x(len);
    for (int o = 0; o < len; ++o) {
        den[o] = o == 0 ? delta : delta - alpha * alpha / den[o - 1];
        xp[o] = ((o == 0 ? 0.0 : alpha * xp[o - 1]) + rhs[o]) / den[o];
    }
    for (int o = len - 1; o >= 0; --o) x[o] = o == len - 1 ? xp[o] : xp[o] + alpha / den[o] * x[o + 1];
    return x;
}

const LineTables& line_tables(lap_handle h, int N, double alpha, double delta, double wc,
                              int max_chunks)
{
    auto key = std::make_tuple(N, alpha, delta, wc, max_chunks);
    auto it = h->lines.find(key);
    if (it != h->lines.end()) return it->second.t;
    if (N > LINE_MAX_N) fail(LAP_EUNSUPPORTED, "line longer than 16383 unknowns");
    LineTables t{};
    t.N = N;
    t.alpha = alpha;
    t.delta = delta;
    t.wc = wc;
    t.maxp = max_chunks;
    // P <= max_chunks chunks of L unknowns, each but the last followed by one separator unknown;
    // the last chunk holds the remaining 1..L unknowns (the line never ends on a separator)
    if (N <= LINE_MIN_CHUNK) {
        t.L = t.Ll = N;
        t.P = 1;
    } else {
        t.L = std::max(LINE_MIN_CHUNK, (N - (max_chunks - 1) + max_chunks - 1) / max_chunks);
        for (;; ++t.L) {
            t.P = (N + 1 + t.L) / (t.L + 1);  // ceil((N + 1) / (L + 1))
            t.Ll = N - (t.P - 1) * (t.L + 1);
            if (t.Ll >= 1) break;
        }
    }
    if (t.Ll > t.L || t.P > max_chunks) fail(LAP_ECUDA, "internal: bad line partition");
    t.stride = (t.L + 1) | 1;
    const int L = t.L, S = t.P - 1;
    t.levels = 0;
    for (int s = 1; s < S; s <<= 1) ++t.levels;

    std::vector<double> e(L), inv_den(L), sc(L + 1), F(L, 0.0);
    double den = delta;
    for (int q = 0; q < L; ++q) {
        if (q) den = delta - alpha * alpha / den;
        inv_den[q] = 1.0 / den;
        e[q] = alpha / den;
        sc[q] = wc / den;
    }
    sc[L] = wc;
    F[0] = alpha;
    for (int q = 1; q < L; ++q) F[q] = F[q - 1] * e[q - 1];
    auto influence = [&](int len, bool left) {
        std::vector<double> rhs(len, 0.0);
        rhs[left ? 0 : len - 1] = alpha;
        std::vector<double> g = host_thomas(len, alpha, delta, rhs);
        g.resize(L, 0.0);
        return g;
    };
    std::vector<double> gL = influence(L, true), gR = influence(L, false);
    std::vector<double> gLl = influence(t.Ll, true), gRl = influence(t.Ll, false);
    std::vector<double> gln(L), glnl(L);
    for (int q = 0; q < L; ++q) {
        gln[q] = gL[q] / alpha;  // (T^-1)_{q0} = (T^-1)_{0q}: T is symmetric
        glnl[q] = gLl[q] / alpha;
    }
    // the boundary layer: from K0 on, F and the first inverse rows are below 2^-64 of their
    // first entries and their terms are left out
    auto big = [](double v, double ref) { return std::fabs(v) > std::ldexp(std::fabs(ref), -64); };
    t.K0 = 1;
    for (int q = L - 1; q >= 1; --q)
        if (big(F[q], F[0]) || big(gln[q], gln[0]) || (q < t.Ll && big(glnl[q], glnl[0]))) {
            t.K0 = q + 1;
            break;
        }

    // separator system a x_{p-1} + b x_p + c x_{p+1} = rho_p, p = 0..S-1: the chunk left of
    // separator p ends in y_last + x_{p-1} gL[L-1] + x_p gR[L-1], the chunk right of it starts in
    // y_first + x_p gL'[0] + x_{p+1} gR'[0] (the last chunk's vectors for p = S - 1)
    std::vector<double> a(S), b(S), c(S);
    for (int p = 0; p < S; ++p) {
        const bool right_last = p + 1 == t.P - 1;
        a[p] = p >= 1 ? -alpha * gL[L - 1] : 0.0;
        b[p] = delta - alpha * gR[L - 1] - alpha * (right_last ? gLl[0] : gL[0]);
        c[p] = p + 1 <= S - 1 ? -alpha * gR[0] : 0.0;
    }
    // parallel cyclic reduction, one lane per separator: tables indexed [level * maxp + lane]
    const size_t mp = (size_t)max_chunks;
    std::vector<double> k1((size_t)std::max(1, t.levels) * mp, 0.0), k2(k1.size(), 0.0), invb(mp, 0.0);
    for (int lev = 0, s = 1; lev < t.levels; ++lev, s <<= 1) {
        std::vector<double> na(S), nb(S), nc(S);
        for (int p = 0; p < S; ++p) {
            const double al = p - s >= 0 ? -a[p] / b[p - s] : 0.0;
            const double ga = p + s < S ? -c[p] / b[p + s] : 0.0;
            na[p] = p - s >= 0 ? al * a[p - s] : 0.0;
            nc[p] = p + s < S ? ga * c[p + s] : 0.0;
            nb[p] = b[p] + (p - s >= 0 ? al * c[p - s] : 0.0) + (p + s < S ? ga * a[p + s] : 0.0);
            k1[(size_t)lev * mp + p] = al;
            k2[(size_t)lev * mp + p] = ga;
        }
        a.swap(na);
        b.swap(nb);
        c.swap(nc);
    }
    for (int p = 0; p < S; ++p) invb[p] = 1.0 / b[p];

    std::vector<double> blob;
    auto put = [&](const std::vector<double>& v) {
        size_t at = blob.size();
        blob.insert(blob.end(), v.begin(), v.end());
        return at;
    };
    const size_t o_e = put(e), o_id = put(inv_den), o_sc = put(sc), o_F = put(F), o_gl = put(gln),
                 o_gll = put(glnl), o_k1 = put(k1), o_k2 = put(k2), o_ib = put(invb);
    LineEntry en;
    en.bytes = blob.size() * sizeof(double);
    en.dev = (double*)dev_alloc(h, en.bytes);
    ck(cudaMemcpy(en.dev, blob.data(), en.bytes, cudaMemcpyHostToDevice), "upload line tables");
    t.e = en.dev + o_e;
    t.inv_den = en.dev + o_id;
    t.sc = en.dev + o_sc;
    t.F = en.dev + o_F;
    t.gln = en.dev + o_gl;
    t.glnl = en.dev + o_gll;
    t.k1 = en.dev + o_k1;
    t.k2 = en.dev + o_k2;
    t.invb = en.dev + o_ib;
    en.t = t;
    return h->lines.emplace(key, en).first->second.t;
}

// Row pitch (in lines) of the y-line scratch: the lines of the larger zebra colour, rounded up.
int64_t line_scratch_pitch(const Field& f, int direction)
{
    const int nlines = direction == 0 ? f.n - 2 : f.m - 2;
    return round_up((int64_t)(nlines + 1) / 2, 32);
}

// The y-line scratch for tables t (grown on demand, outside graph capture: growing drops the
// handle's graphs, which hold the old buffer).
double* line_scratch(lap_handle h, const LineTables& t, int64_t gp)
{
    const size_t bytes = line_y_scratch_doubles(t, gp) * sizeof(double);
    if (bytes > h->lscratch_bytes) {
        drop_graphs(h);
        dev_free(h, h->lscratch, h->lscratch_bytes);
        h->lscratch = nullptr;
        h->lscratch_bytes = 0;
        h->lscratch = (double*)dev_alloc(h, bytes);
        h->lscratch_bytes = bytes;
    }
    return h->lscratch;
}

// Tables, per-call coefficients and (y-lines) scratch of one zebra half sweep; allocates only
// on the first use of a shape, so calling it before a graph capture prepares the capture.
const LineTables& line_setup(lap_handle h, const Field& f, const Coef& c, double w, int form,
                             int direction, LineCoefs* k, double** scratch)
{
    const bool x = direction == 0;
    const int N = x ? f.m - 2 : f.n - 2;
    const double off = x ? 1.0 : c.b2;    // coefficient along the line
    const double cross = x ? c.b2 : 1.0;  // coefficient of the neighbouring lines
    const double alpha = form == LAP_FORM_A ? off : w * off;
    k->wc = w * cross;
    k->bnd = off / cross;
    k->c1 = form == LAP_FORM_B ? c.d * (1.0 - w) / k->wc : 0.0;
    k->omw = 1.0 - w;
    // x-lines long enough for 64 chunks of at least 48 unknowns take the two-warp cut (at 4097^2:
    // 255 -> 242 us per half sweep); shorter chunks would spend most of their length in the
    // boundary layer (about 34 positions at beta = 1), so shorter lines keep 32 chunks
    const bool cut64 = x && N >= LINE_MAX_CHUNKS_X * 48;
    const LineTables& t = line_tables(h, N, alpha, c.d, k->wc, cut64 ? LINE_MAX_CHUNKS_X : LINE_MAX_CHUNKS);
    if (x) {
        ck(prepare_line_kernels(line_smem_bytes(t)), "line kernel attributes");
        *scratch = nullptr;
        const size_t bytes = std::max<size_t>(line_x_sync_words(f.n - 2) * sizeof(unsigned), 1 << 20);
        if (bytes > h->lsync_bytes) {
            // keep a timeout that the old block recorded
            unsigned err = 0;
            if (h->lsync) ck(cudaMemcpy(&err, h->lsync, sizeof err, cudaMemcpyDeviceToHost), "read line flags");
            drop_graphs(h);
            dev_free(h, h->lsync, h->lsync_bytes);
            h->lsync = nullptr;
            h->lsync_bytes = 0;
            h->lsync = (unsigned*)dev_alloc(h, bytes);
            h->lsync_bytes = bytes;
            ck(cudaMemset(h->lsync, 0, sizeof(unsigned)), "clear line error");
            if (err) ck(cudaMemcpy(h->lsync, &err, sizeof err, cudaMemcpyHostToDevice), "keep line error");
        }
    } else {
        *scratch = line_scratch(h, t, line_scratch_pitch(f, direction));
    }
    return t;
}

// One zebra half sweep (odd lines, then even lines) in `direction` (0: x-lines = rows,
// 1: y-lines = columns), form A or B.
void line_half_sweep(lap_handle h, const Field& f, const Coef& c, double w, int form,
                     int direction, cudaStream_t s)
{
    LineCoefs k;
    double* scratch = nullptr;
    const LineTables& t = line_setup(h, f, c, w, form, direction, &k, &scratch);
    if (direction == 0) {  // both colours in one launch
        ck(launch_line_x(f.p, f.pitch, f.n - 2, t, form, k, h->lsync, s), "x-line kernel");
        return;
    }
    const int nlines = f.m - 2;
    const int64_t gp = line_scratch_pitch(f, direction);
    for (int first = 1; first <= 2; ++first) {
        const int count = first == 1 ? (nlines + 1) / 2 : nlines / 2;
        ck(launch_line_scratch(f.p, f.pitch, 1, first, count, t, form, k, scratch, gp, s),
           "y-line kernels");
    }
}

// A wait of an x-line sweep that timed out (recorded on the device; the sweep went on, with
// results that cannot be trusted) becomes an error of the next synchronising call on the
// handle: the word is read once the stream is idle, and cleared.
void check_line_waits(lap_handle h, cudaStream_t s)
{
    if (!h->lsync) return;
    ck(cudaMemcpyAsync(h->pinned, h->lsync, sizeof(unsigned), cudaMemcpyDeviceToHost, s), "read line flags");
    ck(cudaStreamSynchronize(s), "stream sync");
    unsigned word = 0;
    std::memcpy(&word, h->pinned, sizeof word);
    if (word) {
        ck(cudaMemsetAsync(h->lsync, 0, sizeof(unsigned), s), "clear line error");
        ck(cudaStreamSynchronize(s), "stream sync");
        fail(LAP_ECUDA, "an x-line sweep gave up waiting for a neighbouring line (its results are "
                        "invalid)");
    }
}

// ---- coarsest-grid inverse ------------------------------------------------------------


const double* coarse_inverse(lap_handle h, int m, int n, double b2, double d)
{
    auto key = std::make_tuple(m, n, b2);
    auto it = h->coarse.find(key);
    if (it != h->coarse.end()) return it->second.dev;
    const int mi = m - 2, N = mi * (n - 2);
    if (N > COARSE_MAX_UNKNOWNS) fail(LAP_EUNSUPPORTED, "coarsest grid has more than 1024 unknowns");
    // A (unknowns k = (j-1) mi + (i-1)): d on the diagonal, -1 across x, -b2 across y
    std::vector<double> A((size_t)N * N, 0.0), X((size_t)N * N, 0.0);
    for (int k = 0; k < N; ++k) {
        const int i = k % mi, j = k / mi;
        A[(size_t)k * N + k] = d;
        if (i > 0) A[(size_t)k * N + k - 1] = -1.0;
        if (i < mi - 1) A[(size_t)k * N + k + 1] = -1.0;
        if (j > 0) A[(size_t)k * N + k - mi] = -b2;
        if (j < n - 3) A[(size_t)k * N + k + mi] = -b2;
        X[(size_t)k * N + k] = 1.0;
    }
    // Gauss-Jordan with partial pivoting (A is symmetric positive definite, well conditioned
    // at coarsest-grid sizes)
    for (int col = 0; col < N; ++col) {
        int piv = col;
        for (int r = col + 1; r < N; ++r)
            if (std::fabs(A[(size_t)r * N + col]) > std::fabs(A[(size_t)piv * N + col])) piv = r;
        if (piv != col)
            for (int t = 0; t < N; ++t) {
                std::swap(A[(size_t)col * N + t], A[(size_t)piv * N + t]);
                std::swap(X[(size_t)col * N + t], X[(size_t)piv * N + t]);
            }
        const double inv = 1.0 / A[(size_t)col * N + col];
        for (int t = 0; t < N; ++t) {
            A[(size_t)col * N + t] *= inv;
            X[(size_t)col * N + t] *= inv;
        }
        for (int r = 0; r < N; ++r) {
            if (r == col) continue;
            const double f = A[(size_t)r * N + col];
            if (f == 0.0) continue;
            for (int t = 0; t < N; ++t) {
                A[(size_t)r * N + t] -= f * A[(size_t)col * N + t];
                X[(size_t)r * N + t] -= f * X[(size_t)col * N + t];
            }
        }
    }
    std::vector<double> xt((size_t)N * N);
    for (int r = 0; r < N; ++r)
        for (int t = 0; t < N; ++t) xt[(size_t)t * N + r] = X[(size_t)r * N + t];
    CoarseEntry e;
    e.bytes = xt.size() * sizeof(double);
    e.dev = (double*)dev_alloc(h, e.bytes);
    ck(cudaMemcpy(e.dev, xt.data(), e.bytes, cudaMemcpyHostToDevice), "upload coarse inverse");
    return h->coarse.emplace(key, e).first->second.dev;
}

int mg_level_count(int m, int n, int coarsest_min, int max_levels)
{
    int levels = 1;
    while ((max_levels <= 0 || levels < max_levels) && (m - 1) % 2 == 0 && (n - 1) % 2 == 0 &&
           (m - 1) / 2 + 1 >= coarsest_min && (n - 1) / 2 + 1 >= coarsest_min) {
        m = (m - 1) / 2 + 1;
        n = (n - 1) / 2 + 1;
        ++levels;
    }
    return levels;
}

// Tail sizes worth timing for a batch of V-cycles (one CTA per problem runs the levels at or
// below the size) and for one grid (one CTA in all).
std::vector<int> tail_candidates(bool batched, bool fp32, int tail_size)
{
    if (tail_size != 0) return {tail_size};
    if (batched) return {-1, 33, 65, 129, 257};
    return fp32 ? std::vector<int>{-1, 33, 65, 129, 257} : std::vector<int>{-1, 17, 33, 65};
}

std::string tuner_key(char kind, const lap_params* p, const std::vector<int>& shape)
{
    uint64_t hsh = 1469598103934665603ull;  // FNV-1a over the shapes
    for (int v : shape) {
        hsh ^= (uint32_t)v;
        hsh *= 1099511628211ull;
    }
    char buf[240];
    std::snprintf(buf, sizeof buf, "%c %d %d %d %d %d %.17g %d %d %d %d %d %d %zu %llx", kind,
                  p->method, p->nu1, p->nu2, p->coarsest_min, p->max_levels, p->smoother_w,
                  p->inner_cycles, p->tail_size, p->unfused, p->tiling, p->item_points,
                  p->persistent, shape.size(), (unsigned long long)hsh);
    return buf;
}

cudaEvent_t tuner_event(lap_handle h, int k)
{
    if (!h->ev[k]) ck(cudaEventCreate(&h->ev[k]), "create event");
    return h->ev[k];
}

}  // namespace lap

using namespace lap;

namespace {

// ---- multigrid hierarchy -----------------------------------------------------------------

struct Level {
    Field u;            // level 0: the caller's field; deeper: the correction
    double* q = nullptr;  // source term (levels >= 1)
    double* r = nullptr;  // residual scratch (all but the coarsest), u's pitch
};

// ---- the per-call workspace ----------------------------------------------------------------

struct Level32 {
    Field32 u;           // inner correction (level 0: e of the fine grid)
    float* q = nullptr;  // source (level 0: the FP64 residual rounded to FP32)
    float* r = nullptr;  // residual scratch (all but the coarsest)
};

struct Work {
    double* wslot = nullptr;     // {w, 1 - w} of the point sweeps, read by the kernels
    double* partials = nullptr;  // norm partial sums
    double* nrm = nullptr;       // [sum, sqrt]
    float* nscale = nullptr;     // the mixed solver's norm scale (power of two near 1/||r0||)
    LoopState* loop = nullptr;   // device-resident solve loop state
    unsigned long long* maxd = nullptr;
    double* aux = nullptr;       // Jacobi second buffer, or previous iterate for max|delta|
    std::vector<Level> levels;
    std::vector<Level32> levels32;
    // the small-level tail: level descriptors and one job per possible first level
    BatchLevel<double>* tl64 = nullptr;
    BatchLevel<float>* tl32 = nullptr;
    TailJob* tjob = nullptr;
};

template <class C>
void carve(C& cv, Work& w, const lap_grid* g, const lap_params* p)
{
    w.wslot = cv.template take<double>(2);
    w.partials = cv.template take<double>(NORM_PARTIALS_MAX);
    w.nrm = cv.template take<double>(2);
    w.nscale = cv.template take<float>(1);
    w.loop = cv.template take<LoopState>(1);
    w.maxd = cv.template take<unsigned long long>(1);
    const size_t field = (size_t)g->n * (size_t)g->pitch;
    const bool need_aux =
        p->method == LAP_JACOBI ||
        (p->norm == LAP_NORM_MAXDELTA &&
         (p->method == LAP_ADI || p->method == LAP_SLOR || p->method == LAP_MG ||
          p->method == LAP_MG_MIXED));
    w.aux = need_aux ? cv.template take<double>(field) : nullptr;
    w.levels.clear();
    if (p->method == LAP_MG) {
        const int L = mg_level_count(g->m, g->n, p->coarsest_min, p->max_levels);
        int m = g->m, n = g->n;
        for (int l = 0; l < L; ++l) {
            Level lv;
            const int64_t pitch = l == 0 ? g->pitch : round_up(m, 32);
            lv.u = Field{nullptr, m, n, pitch};
            if (l > 0) {
                lv.u.p = cv.template take<double>((size_t)n * pitch);
                lv.q = cv.template take<double>((size_t)n * pitch);
            }
            if (l < L - 1) lv.r = cv.template take<double>((size_t)n * pitch);
            w.levels.push_back(lv);
            m = (m - 1) / 2 + 1;
            n = (n - 1) / 2 + 1;
        }
        w.tl64 = cv.template take<BatchLevel<double>>(L);
        w.tjob = cv.template take<TailJob>(L);
    }
    w.levels32.clear();
    if (p->method == LAP_MG_MIXED || p->method == LAP_MG_FP32) {
        const int L = mg_level_count(g->m, g->n, p->coarsest_min, p->max_levels);
        int m = g->m, n = g->n;
        for (int l = 0; l < L; ++l) {
            Level32 lv;
            const int64_t pitch = round_up(m, 32);
            lv.u = Field32{cv.template take<float>((size_t)n * pitch), m, n, pitch};
            lv.q = cv.template take<float>((size_t)n * pitch);
            if (l < L - 1) lv.r = cv.template take<float>((size_t)n * pitch);
            w.levels32.push_back(lv);
            m = (m - 1) / 2 + 1;
            n = (n - 1) / 2 + 1;
        }
        w.tl32 = cv.template take<BatchLevel<float>>(L);
        w.tjob = cv.template take<TailJob>(L);
    }
}

size_t work_bytes(const lap_grid* g, const lap_params* p)
{
    Sizer sz;
    Work w;
    carve(sz, w, g, p);
    return sz.off;
}

// ---- the solver loop ---------------------------------------------------------------------

struct Solver {
    lap_handle h;
    cudaStream_t s;
    Field f;
    Coef c;
    const lap_params* p;
    Work w;

    double residual(const Field& u, const double* q)
    {
        ck(launch_defect_sumsq(u, q, c, w.partials, s), "residual kernel");
        ck(launch_sum_partials(w.partials, norm_blocks(u), w.nrm, s), "sum kernel");
        ck(cudaMemcpyAsync(h->pinned, w.nrm + 1, sizeof(double), cudaMemcpyDeviceToHost, s),
           "copy norm");
        ck(cudaStreamSynchronize(s), "stream sync");
        return h->pinned[0];
    }

    // Norm from partial sums already written by the last FP64 residual pass (squares of
    // norm_sc r when scaled).
    double partial_norm(const Field& u, bool scaled = false)
    {
        ck(launch_sum_partials(w.partials, mixed_norm_blocks(u.m, u.n), w.nrm, s), "sum kernel");
        ck(cudaMemcpyAsync(h->pinned, w.nrm + 1, sizeof(double), cudaMemcpyDeviceToHost, s),
           "copy norm");
        ck(cudaStreamSynchronize(s), "stream sync");
        return scaled ? h->pinned[0] / norm_sc : h->pinned[0];
    }

    // The mixed solver sums its iterations' residual squares in FP32 once r0 is known:
    // scale = 2^-e with r0 = f 2^e (so the scaled values stay in FP32's range).
    double norm_sc = 0.0;
    void set_norm_scale(double r0)
    {
        norm_sc = 0.0;
        if (!(r0 > 0.0) || !std::isfinite(r0)) return;
        const int e = std::ilogb(r0);
        if (e < -100 || e > 100) return;
        norm_sc = std::ldexp(1.0, -e);
        const float v = (float)norm_sc;  // exact: a power of two in FP32's range
        // pageable source: staged by the copy before it returns
        ck(cudaMemcpyAsync(w.nscale, &v, sizeof v, cudaMemcpyHostToDevice, s), "upload norm scale");
    }

    double read_maxd()
    {
        ck(cudaMemcpyAsync(h->pinned, w.maxd, sizeof(double), cudaMemcpyDeviceToHost, s),
           "copy max delta");
        ck(cudaStreamSynchronize(s), "stream sync");
        uint64_t bits;
        std::memcpy(&bits, h->pinned, 8);
        double v;
        std::memcpy(&v, &bits, 8);
        return v;
    }

    void copy_field(double* dst, const double* src)
    {
        ck(cudaMemcpy2DAsync(dst, f.pitch * 8, src, f.pitch * 8, (size_t)f.m * 8, f.n,
                             cudaMemcpyDeviceToDevice, s),
           "copy field");
    }

    // ---- one iteration of each method ----
    double* jac_cur = nullptr;  // Jacobi: buffer holding the current iterate
    double* jac_other = nullptr;

    void iterate(bool want_maxd)
    {
        unsigned long long* md = want_maxd ? w.maxd : nullptr;
        const bool gs = p->method == LAP_GS_RB;
        switch (p->method) {
        case LAP_JACOBI: {
            Field in{jac_cur, f.m, f.n, f.pitch};
            ck(launch_jacobi(in, jac_other, c, md, s), "jacobi kernel");
            std::swap(jac_cur, jac_other);
            break;
        }
        case LAP_GS_RB:
        case LAP_SOR_RB:
            for (int colour = 0; colour < 2; ++colour) {
                if (p->sum_order == LAP_SUM_DIAGONAL)
                    ck(launch_rb_diag(f, nullptr, gs, gs ? 1.0 : p->w, colour, md, s, w.wslot),
                       "rb kernel (diagonal pairs)");
                else
                    ck(launch_rb_colour(f, nullptr, c, gs, gs ? 1.0 : p->w, colour, md, s, w.wslot),
                       "rb kernel");
            }
            break;
        case LAP_ADI:
            line_half_sweep(h, f, c, p->w, p->line_form, 0, s);
            line_half_sweep(h, f, c, p->w, p->line_form, 1, s);
            break;
        case LAP_SLOR:
            line_half_sweep(h, f, c, p->w, p->line_form, 0, s);
            break;
        case LAP_MG:
            vcycle(0);
            break;
        case LAP_MG_FP32:
            vcycle32(0);
            break;
        case LAP_MG_MIXED: {
            const Level32& l0 = w.levels32[0];
            // with the tile kernels the last level-0 ascent also does psi += e
            const bool fold = fused32 && tail_first != 0 && w.levels32.size() > 1;
            for (int k = 0; k < p->inner_cycles; ++k) vcycle32(0, k == 0, fold && k == p->inner_cycles - 1);
            if (!fold) ck(launch_update64(f, l0.u.p, l0.u.pitch, s), "update kernel");
            // the tiles' first level-0 descent treats e as zero: no need to clear it
            const bool keep_e = fused32 && tail_first != 0 && w.levels32.size() > 1;
            ck(launch_defect64_to32(f, c, l0.q, keep_e ? nullptr : l0.u.p, l0.u.pitch, w.partials, s,
                                    norm_sc > 0.0 ? w.nscale : nullptr),
               "mixed residual kernel");
            break;
        }
        }
    }

    // First level of the small-level tail in vcycle()/vcycle32() (-1: none), see set_tail.
    int tail_first = -1;

    // Run the levels whose sides are both <= S (S > 0) as the tail; -1 = no tail.
    void set_tail(int S)
    {
        tail_first = -1;
        if (S <= 0) return;
        const int L = p->method == LAP_MG ? (int)w.levels.size() : (int)w.levels32.size();
        int m = f.m, n = f.n;
        for (int l = 0; l < L; ++l) {
            if (m <= S && n <= S) {
                tail_first = l;
                return;
            }
            m = (m - 1) / 2 + 1;
            n = (n - 1) / 2 + 1;
        }
    }

    int coarsest_unknowns() const
    {
        const int L = p->method == LAP_MG ? (int)w.levels.size() : (int)w.levels32.size();
        int m = f.m, n = f.n;
        for (int l = 1; l < L; ++l) {
            m = (m - 1) / 2 + 1;
            n = (n - 1) / 2 + 1;
        }
        return (m - 2) * (n - 2);
    }

    // Level descriptors and tail jobs of this call (level 0 is the caller's field, or the
    // FP32 correction), uploaded before any period runs.
    void upload_tail()
    {
        const bool mixed = p->method == LAP_MG_MIXED || p->method == LAP_MG_FP32;
        const int L = mixed ? (int)w.levels32.size() : (int)w.levels.size();
        std::vector<BatchLevel<double>> d(L);
        std::vector<BatchLevel<float>> g(L);
        std::vector<TailJob> jobs(L);
        int m = f.m, n = f.n;
        for (int l = 0; l < L; ++l) {
            BatchLevel<double> a{};
            a.m = m;
            a.n = n;
            a.problem = 0;
            a.unit_beta = c.unit_beta;
            a.b2 = c.b2;
            a.d = c.d;
            a.inv_d = c.inv_d;
            a.w = p->smoother_w;
            a.omw = 1.0 - p->smoother_w;
            a.ainv_t = l == L - 1 ? coarse_inverse(h, m, n, c.b2, c.d) : nullptr;
            if (mixed) {
                BatchLevel<float> b{};
                b.u = w.levels32[l].u.p;
                b.q = w.levels32[l].q;
                b.r = w.levels32[l].r;
                b.m = m;
                b.n = n;
                b.pitch = w.levels32[l].u.pitch;
                b.unit_beta = a.unit_beta;
                b.inv_d_shift = 0;
                b.b2 = a.b2;
                b.d = a.d;
                b.inv_d = a.inv_d;
                b.w = a.w;
                b.omw = a.omw;
                b.ainv_t = a.ainv_t;
                g[l] = b;
            } else {
                a.u = w.levels[l].u.p;
                a.q = w.levels[l].q;
                a.r = w.levels[l].r;
                a.pitch = w.levels[l].u.pitch;
                a.inv_d_shift = c.inv_d_shift;
                d[l] = a;
            }
            jobs[l] = TailJob{l, L - 1};
            m = (m - 1) / 2 + 1;
            n = (n - 1) / 2 + 1;
        }
        // pageable sources: the copies are staged before the calls return
        if (mixed) hl32 = g;
        if (mixed)
            ck(cudaMemcpyAsync(w.tl32, g.data(), L * sizeof(g[0]), cudaMemcpyHostToDevice, s), "upload levels");
        else
            ck(cudaMemcpyAsync(w.tl64, d.data(), L * sizeof(d[0]), cudaMemcpyHostToDevice, s), "upload levels");
        ck(cudaMemcpyAsync(w.tjob, jobs.data(), L * sizeof(TailJob), cudaMemcpyHostToDevice, s), "upload jobs");
    }

    std::vector<BatchLevel<float>> hl32;  // FP32 level descriptors (host copy)
    bool fused32 = false;                 // descents/ascents as tile kernels

    // The FP32 image of vcycle() on the correction equation. first: the first inner cycle
    // of an outer iteration (the level-0 correction starts at zero).
    void vcycle32(int l, bool first = false, bool fold = false)
    {
        Level32& lv = w.levels32[l];
        const int L = (int)w.levels32.size();
        if (l == tail_first) {
            ck(launch_b_tail(w.tjob + l, 1, w.tl32, nullptr, p->nu1, p->nu2, p->smoother_w == 1.0,
                             p->smoother_w, coarsest_unknowns(), s),
               "tail kernel");
            return;
        }
        if (l == L - 1 && p->method == LAP_MG_FP32) {
            // level 0 carries the Dirichlet ring: the tail's coarsest solve adds ring terms
            ck(launch_b_tail(w.tjob + l, 1, w.tl32, nullptr, p->nu1, p->nu2, p->smoother_w == 1.0,
                             p->smoother_w, coarsest_unknowns(), s),
               "coarse solve kernel");
            return;
        }
        if (fused32 && l < L - 1) {
            const bool gs = p->smoother_w == 1.0;
            ck(launch_down32(hl32[l], hl32[l + 1], p->nu1, p->nu2, l > 0 || first, gs, p->smoother_w, s),
               "descent kernel");
            vcycle32(l + 1);
            ck(launch_up32(hl32[l], hl32[l + 1], p->nu1, p->nu2, gs, p->smoother_w, s,
                           fold && l == 0 ? f.p : nullptr, f.pitch),
               "ascent kernel");
            return;
        }
        if (l == L - 1) {
            const double* ainv = coarse_inverse(h, lv.u.m, lv.u.n, c.b2, c.d);
            ck(launch_coarse32(lv.u, lv.q, ainv, s), "coarse solve kernel");
            return;
        }
        const bool gs = p->smoother_w == 1.0;
        for (int k = 0; k < p->nu1; ++k)
            for (int colour = 0; colour < 2; ++colour)
                ck(launch_rb32(lv.u, lv.q, c, gs, p->smoother_w, colour, s), "smoother kernel");
        Level32& cv = w.levels32[l + 1];
        ck(launch_defect32(lv.u, lv.q, lv.r, c, s), "defect kernel");
        ck(launch_restrict32(Field32{lv.r, lv.u.m, lv.u.n, lv.u.pitch}, cv.q, cv.u.p, cv.u.pitch, s),
           "restrict kernel");
        vcycle32(l + 1);
        ck(launch_prolong32(lv.u, cv.u.p, cv.u.pitch, s), "prolong kernel");
        for (int k = 0; k < p->nu2; ++k)
            for (int colour = 0; colour < 2; ++colour)
                ck(launch_rb32(lv.u, lv.q, c, gs, p->smoother_w, colour, s), "smoother kernel");
    }

    void smooth(const Level& lv, int sweeps)
    {
        const bool gs = p->smoother_w == 1.0;
        for (int k = 0; k < sweeps; ++k)
            for (int colour = 0; colour < 2; ++colour)
                ck(launch_rb_colour(lv.u, lv.q, c, gs, p->smoother_w, colour, nullptr, s, w.wslot),
                   "smoother kernel");
    }

    void vcycle(int l)
    {
        Level& lv = w.levels[l];
        const int L = (int)w.levels.size();
        if (l == tail_first) {
            ck(launch_b_tail(w.tjob + l, 1, w.tl64, nullptr, p->nu1, p->nu2, p->smoother_w == 1.0,
                             p->smoother_w, coarsest_unknowns(), s),
               "tail kernel");
            return;
        }
        if (l == L - 1) {
            const double* ainv = coarse_inverse(h, lv.u.m, lv.u.n, c.b2, c.d);
            ck(launch_coarse_solve(lv.u, lv.q, c, ainv, s), "coarse solve kernel");
            return;
        }
        smooth(lv, p->nu1);
        Level& cv = w.levels[l + 1];
        ck(launch_defect(lv.u, lv.q, lv.r, c, s), "defect kernel");
        ck(launch_restrict(Field{lv.r, lv.u.m, lv.u.n, lv.u.pitch}, cv.q, cv.u.p, cv.u.pitch, s),
           "restrict kernel");
        vcycle(l + 1);
        ck(launch_prolong_add(lv.u, cv.u.p, cv.u.pitch, s), "prolong kernel");
        smooth(lv, p->nu2);
    }

    // The whole solve in one CTA (solve_cta_kernel): point methods with the paper's stopping
    // rule on grids whose sweeps cost less than the launches and host checks of the
    // multi-CTA path (a block-wide max is order-free, so the test is the host loop's bit for
    // bit). Red-black and Jacobi up to 4096 points: about the size where one SM sweeps as
    // fast as two launches take; lexicographic grids always run on one SM.
    bool solve_cta_ok() const
    {
        if (p->norm != LAP_NORM_MAXDELTA) return false;
        if (p->sum_order == LAP_SUM_DIAGONAL) return false;  // the one-CTA sweeps sum in paper order
        if (p->method == LAP_GS_LEX || p->method == LAP_SOR_LEX) return true;
        if (p->method == LAP_ADI || p->method == LAP_SLOR)
            return (int64_t)f.m * f.n <= 4096 && solve_lines_cta_smem(f.m, f.n) <= 200 * 1024;
        return (p->method == LAP_JACOBI || p->method == LAP_GS_RB || p->method == LAP_SOR_RB) &&
               (int64_t)f.m * f.n <= 4096;
    }

    // The iterations between two stopping tests, enqueued on stream s.
    void period(int64_t steps, bool maxdelta, bool fused_maxd)
    {
        if (p->method == LAP_GS_LEX || p->method == LAP_SOR_LEX) {
            // the whole period in one launch (the field stays in shared memory)
            if (maxdelta) ck(cudaMemsetAsync(w.maxd, 0, 8, s), "zero max delta");
            const bool gs = p->method == LAP_GS_LEX;
            for (int64_t done = 0; done < steps;) {
                const int chunk = (int)std::min<int64_t>(steps - done, 1 << 20);
                const bool last = done + chunk == steps;
                ck(launch_lex_sweeps(f, c, gs, gs ? 1.0 : p->w, chunk,
                                     last && maxdelta ? w.maxd : nullptr, s),
                   "lexicographic kernel");
                done += chunk;
            }
            return;
        }
        for (int64_t st = 0; st < steps; ++st) {
            const bool last = st == steps - 1;
            if (last && maxdelta) {
                ck(cudaMemsetAsync(w.maxd, 0, 8, s), "zero max delta");
                if (!fused_maxd) copy_field(w.aux, f.p);
            }
            iterate(last && fused_maxd);
        }
    }

    // Host-side tables a period needs, built before capture (they upload synchronously).
    void prepare()
    {
        if (p->method == LAP_ADI || p->method == LAP_SLOR) {
            for (int dir = 0; dir < (p->method == LAP_ADI ? 2 : 1); ++dir) {
                LineCoefs k;
                double* scratch = nullptr;
                line_setup(h, f, c, p->w, p->line_form, dir, &k, &scratch);
            }
        }
        if (p->method == LAP_MG) {
            const Level& lv = w.levels.back();
            coarse_inverse(h, lv.u.m, lv.u.n, c.b2, c.d);
        }
        if (p->method == LAP_MG_MIXED || p->method == LAP_MG_FP32) {
            const Level32& lv = w.levels32.back();
            coarse_inverse(h, lv.u.m, lv.u.n, c.b2, c.d);
        }
        if (p->method == LAP_GS_LEX || p->method == LAP_SOR_LEX)
            ck(prepare_lex_kernels(lex_smem_bytes(f.m, f.n)), "lexicographic kernel attributes");
    }

    std::string graph_key(int64_t steps, bool maxdelta, bool fused_maxd) const
    {
        std::string k;
        auto put = [&](const void* v, size_t n) { k.append((const char*)v, n); };
        const int64_t ints[] = {p->method, f.m, f.n, f.pitch, steps, maxdelta, fused_maxd,
                                p->nu1, p->nu2, p->coarsest_min, p->max_levels, p->line_form,
                                (int64_t)w.levels.size(), p->inner_cycles,
                                (int64_t)w.levels32.size(), tail_first, fused32, norm_sc > 0.0,
                                p->sum_order};
        const double dbl[] = {c.b2, c.d, c.inv_d, p->w, p->smoother_w};
        const void* ptrs[] = {f.p, jac_cur, jac_other, w.aux, w.maxd, h->arena, h->lscratch};
        put(ints, sizeof ints);
        put(dbl, sizeof dbl);
        put(ptrs, sizeof ptrs);
        return k;
    }

    // A period as one CUDA graph: captured once on the handle's own stream, replayed on s.
    // Returns true when this call captured the graph (its first use).
    bool run_period(int64_t steps, bool maxdelta, bool fused_maxd)
    {
        if (!h->use_graphs) {
            period(steps, maxdelta, fused_maxd);
            return false;
        }
        bool captured = false;
        const std::string key = graph_key(steps, maxdelta, fused_maxd);
        auto it = h->graphs.find(key);
        if (it == h->graphs.end()) {
            prepare();
            if (h->graphs.size() >= 64) drop_graphs(h);
            if (!h->capture)
                ck(cudaStreamCreateWithFlags(&h->capture, cudaStreamNonBlocking), "capture stream");
            cudaStream_t caller = s;
            double* cur0 = jac_cur;
            double* other0 = jac_other;
            const int64_t before = launches_now();
            ck(cudaStreamBeginCapture(h->capture, cudaStreamCaptureModeThreadLocal), "begin capture");
            s = h->capture;
            cudaGraph_t g = nullptr;
            try {
                period(steps, maxdelta, fused_maxd);
            } catch (...) {
                s = caller;
                cudaStreamEndCapture(h->capture, &g);
                if (g) cudaGraphDestroy(g);
                cudaGetLastError();
                throw;
            }
            s = caller;
            ck(cudaStreamEndCapture(h->capture, &g), "end capture");
            const int64_t kernels = launches_now() - before;
            add_launches(-kernels);  // captured, not launched
            cudaGraphExec_t exec = nullptr;
            const cudaError_t e = cudaGraphInstantiate(&exec, g, 0);
            cudaGraphDestroy(g);
            ck(e, "instantiate graph");
            it = h->graphs.emplace(key, std::make_pair(exec, kernels)).first;
            jac_cur = cur0;  // the host-side ping-pong state advances on replay below
            jac_other = other0;
            captured = true;
        }
        ck(cudaGraphLaunch(it->second.first, s), "launch graph");
        add_launches(it->second.second);
        if (p->method == LAP_JACOBI && (steps & 1)) std::swap(jac_cur, jac_other);
        return captured;
    }

    // The norm of the stopping test, enqueued on s (the kernels of the host check).
    void enqueue_norm(bool maxdelta, bool fused_maxd, const Field& cur)
    {
        if (maxdelta) {
            if (!fused_maxd) ck(launch_maxdelta(f, w.aux, w.maxd, s), "max delta kernel");
        } else if (p->method == LAP_MG_FP32) {
            ck(launch_defect32_sumsq(w.levels32[0].u, w.levels32[0].q, c, w.partials, s),
               "residual kernel");
            ck(launch_sum_partials(w.partials, mixed_norm_blocks(f.m, f.n), w.nrm, s), "sum kernel");
        } else if (p->method == LAP_MG_MIXED) {
            ck(launch_sum_partials(w.partials, mixed_norm_blocks(f.m, f.n), w.nrm, s), "sum kernel");
        } else {
            ck(launch_defect_sumsq(cur, nullptr, c, w.partials, s), "residual kernel");
            ck(launch_sum_partials(w.partials, norm_blocks(cur), w.nrm, s), "sum kernel");
        }
    }

    // Device-resident loop: whole check periods, each followed by the stopping test on the
    // device, as the body of a conditional (while) node of one CUDA graph, so that the host
    // waits once per solve instead of once per period. Used once the small-level tail is
    // chosen, for full periods (Jacobi: even periods, whose buffer roles repeat).
    bool device_loop_ok(int64_t k, int64_t steps, const TailTuner* tuner) const
    {
        if (!h->use_graphs || steps != p->check_every || k + steps > p->max_iter) return false;
        if (tuner && !tuner->done) return false;
        if (p->method == LAP_JACOBI && (steps & 1)) return false;
        return true;
    }

    // Runs periods on the device until the stopping rule holds or the next period would pass
    // max_iter; returns the loop state read back.
    LoopState device_loop(int64_t k, double r0, double last_nr, bool maxdelta, bool fused_maxd)
    {
        const int64_t steps = p->check_every;
        const bool scaled = p->method == LAP_MG_MIXED && norm_sc > 0.0;
        const std::string key = graph_key(steps, maxdelta, fused_maxd) + (scaled ? "|loop-scaled" : "|loop");
        auto it = h->graphs.find(key);
        if (it == h->graphs.end()) {
            prepare();
            if (h->graphs.size() >= 64) drop_graphs(h);
            if (!h->capture)
                ck(cudaStreamCreateWithFlags(&h->capture, cudaStreamNonBlocking), "capture stream");
            cudaGraph_t g = nullptr;
            ck(cudaGraphCreate(&g, 0), "create graph");
            cudaGraphExec_t exec = nullptr;
            int64_t kernels = 0;
            cudaStream_t caller = s;
            double* cur0 = jac_cur;
            double* other0 = jac_other;
            try {
                cudaGraphConditionalHandle hnd;
                ck(cudaGraphConditionalHandleCreate(&hnd, g, 1, cudaGraphCondAssignDefault),
                   "conditional handle");
                // zero-initialised node parameters (the struct's union has no default constructor)
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
                s = h->capture;
                try {
                    period(steps, maxdelta, fused_maxd);
                    const Field cur{p->method == LAP_JACOBI ? jac_cur : f.p, f.m, f.n, f.pitch};
                    enqueue_norm(maxdelta, fused_maxd, cur);
                    ck(launch_loop_decide(w.loop, w.nrm, w.maxd, scaled ? w.nscale : nullptr, hnd, s),
                       "loop test kernel");
                } catch (...) {
                    s = caller;
                    cudaGraph_t junk = nullptr;
                    cudaStreamEndCapture(h->capture, &junk);
                    cudaGetLastError();
                    throw;
                }
                s = caller;
                cudaGraph_t body_out = nullptr;
                ck(cudaStreamEndCapture(h->capture, &body_out), "end capture");
                kernels = launches_now() - before;
                add_launches(-kernels);
                ck(cudaGraphInstantiate(&exec, g, 0), "instantiate graph");
            } catch (...) {
                s = caller;
                jac_cur = cur0;
                jac_other = other0;
                cudaGraphDestroy(g);
                throw;
            }
            cudaGraphDestroy(g);
            jac_cur = cur0;  // even periods: the buffer roles are the same after each
            jac_other = other0;
            it = h->graphs.emplace(key, std::make_pair(exec, kernels)).first;
        }
        LoopState st{};
        st.k = k;
        st.steps = steps;
        st.max_iter = p->max_iter;
        st.mode = maxdelta ? 2 : (p->norm == LAP_NORM_L2_REL ? 0 : 1);
        st.status = LAP_MAXITER;
        st.r0 = r0;
        st.tol = p->tol;
        st.last_check = NAN;
        st.last_nr = last_nr;
        static_assert(sizeof(LoopState) <= 8 * sizeof(double), "pinned buffer holds 8 doubles");
        ck(cudaMemcpyAsync(w.loop, &st, sizeof st, cudaMemcpyHostToDevice, s), "upload loop state");
        ck(cudaGraphLaunch(it->second.first, s), "launch graph");
        ck(cudaMemcpyAsync(h->pinned, w.loop, sizeof st, cudaMemcpyDeviceToHost, s), "copy loop state");
        ck(cudaStreamSynchronize(s), "stream sync");
        std::memcpy(&st, h->pinned, sizeof st);
        add_launches(it->second.second * ((st.k - k) / steps));
        return st;
    }

    void run(lap_result* out)
    {
        out->status = LAP_MAXITER;
        out->iters = 0;
        out->last_check = NAN;
        {
            const double wv = p->method == LAP_MG ? p->smoother_w : p->w;
            const double pair[2] = {wv, 1.0 - wv};  // staged by the copy before it returns
            ck(cudaMemcpyAsync(w.wslot, pair, sizeof pair, cudaMemcpyHostToDevice, s), "upload w");
        }
        if (p->method == LAP_ADI || p->method == LAP_SLOR) prepare();  // tables, scratch: before any capture
        if (p->method == LAP_JACOBI) {
            copy_field(w.aux, f.p);  // ring + initial interior in both buffers
            jac_cur = f.p;
            jac_other = w.aux;
        }
        if (p->method == LAP_MG) {
            w.levels[0].u.p = f.p;
            for (size_t l = 1; l < w.levels.size(); ++l) {
                const Field& u = w.levels[l].u;
                ck(cudaMemsetAsync(u.p, 0, (size_t)u.n * u.pitch * 8, s), "zero coarse level");
                ck(cudaMemsetAsync(w.levels[l].q, 0, (size_t)u.n * u.pitch * 8, s), "zero source");
            }
        }
        if (p->method == LAP_MG_MIXED || p->method == LAP_MG_FP32) {
            // FP32 alone needs its level-0 source zero; the mixed solver writes every interior
            // before reading it and needs only the rings zero (after upload_tail, below)
            if (p->method == LAP_MG_FP32)
                for (const Level32& lv : w.levels32) {
                    ck(cudaMemsetAsync(lv.u.p, 0, (size_t)lv.u.n * lv.u.pitch * 4, s), "zero level");
                    ck(cudaMemsetAsync(lv.q, 0, (size_t)lv.u.n * lv.u.pitch * 4, s), "zero source");
                    if (lv.r) ck(cudaMemsetAsync(lv.r, 0, (size_t)lv.u.n * lv.u.pitch * 4, s), "zero level");
                }
            fused32 = !p->unfused && fused32_supported(p->nu1, p->nu2);
            if (fused32) ck(prepare_fused32(), "tile kernel attributes");
            const Level32& l0 = w.levels32[0];
            if (p->method == LAP_MG_MIXED) {
                ck(launch_defect64_to32(f, c, l0.q, l0.u.p, l0.u.pitch, w.partials, s),
                   "mixed residual kernel");
            } else {
                // FP32 alone: psi (ring included) rounded into level 0's two buffers, q = 0
                ck(launch_to32(f, l0.u.p, l0.r, l0.u.pitch, s), "conversion kernel");
                ck(launch_defect32_sumsq(l0.u, l0.q, c, w.partials, s), "residual kernel");
            }
        }
        TailTuner* tuner = nullptr;
        const bool fp32_norm = p->method == LAP_MG_MIXED || p->method == LAP_MG_FP32;
        if (p->method == LAP_MG || fp32_norm) {
            upload_tail();
            if (p->method == LAP_MG_MIXED)
                ck(launch_zero_rings32(w.tl32, (int)w.levels32.size(), std::max(f.m, f.n), s),
                   "ring kernel");
            const char kind = p->method == LAP_MG ? 'S' : (p->method == LAP_MG_MIXED ? 'M' : 'F');
            tuner = &h->tail_tuners[tuner_key(kind, p, {f.m, f.n})];
            if (tuner->cand.empty()) tuner->init(tail_candidates(false, kind != 'S', p->tail_size));
        }
        // the mixed iteration ends with the FP64 residual's partial sums; FP32 alone with
        // its FP32 residual's
        const double r0 = fp32_norm ? partial_norm(f) : residual(f, nullptr);
        out->r0 = r0;
        if (p->method == LAP_MG_MIXED) set_norm_scale(r0);
        if (!std::isfinite(r0)) {
            out->status = LAP_DIVERGED;
        } else if ((p->norm == LAP_NORM_L2_REL && r0 == 0.0) ||
                   (p->norm == LAP_NORM_L2_ABS && r0 <= p->tol)) {
            out->status = LAP_CONVERGED;
        }
        int64_t k = 0;
        double last_nr = r0;             // the L2 norm of the current iterate, when known
        bool last_is_current = p->method != LAP_MG_FP32;
        if (out->status == LAP_MAXITER && p->max_iter > 0 && solve_cta_ok()) {
            // small grid, the paper's stopping rule: the whole solve is one kernel
            LoopState st{};
            st.k = 0;
            st.steps = p->check_every;
            st.max_iter = p->max_iter;
            st.mode = 2;
            st.status = LAP_MAXITER;
            st.r0 = r0;
            st.tol = p->tol;
            st.last_check = NAN;
            st.last_nr = r0;
            ck(cudaMemcpyAsync(w.loop, &st, sizeof st, cudaMemcpyHostToDevice, s), "upload loop state");
            if (p->method == LAP_ADI || p->method == LAP_SLOR) {
                ck(launch_solve_lines_cta(f, c, p->method == LAP_ADI, p->line_form == LAP_FORM_B,
                                          w.wslot, w.loop, s),
                   "one-CTA line solve kernel");
            } else {
                const int kind = p->method == LAP_JACOBI ? 0 : (p->method == LAP_GS_RB || p->method == LAP_SOR_RB ? 1 : 2);
                const bool gs = p->method == LAP_GS_RB || p->method == LAP_GS_LEX;
                ck(launch_solve_cta(f, c, kind, gs, w.wslot, w.loop, s), "one-CTA solve kernel");
            }
            ck(cudaMemcpyAsync(h->pinned, w.loop, sizeof st, cudaMemcpyDeviceToHost, s), "copy loop state");
            ck(cudaStreamSynchronize(s), "stream sync");
            std::memcpy(&st, h->pinned, sizeof st);
            k = st.k;
            out->status = st.status;
            out->last_check = st.last_check;
            last_is_current = false;
        }
        while (out->status == LAP_MAXITER && k < p->max_iter) {
            const int64_t steps = std::min<int64_t>(p->check_every - (k % p->check_every), p->max_iter - k);
            const bool maxdelta = p->norm == LAP_NORM_MAXDELTA;
            const bool fused_maxd = maxdelta && (p->method == LAP_JACOBI || p->method == LAP_GS_RB ||
                                                 p->method == LAP_SOR_RB || p->method == LAP_GS_LEX ||
                                                 p->method == LAP_SOR_LEX);
            if (tuner && tuner->done) set_tail(tuner->cand[tuner->best]);
            if (device_loop_ok(k, steps, tuner)) {
                const LoopState st = device_loop(k, r0, last_nr, maxdelta, fused_maxd);
                k = st.k;
                out->last_check = st.last_check;
                out->status = st.status;
                if (maxdelta) {
                    last_is_current = false;
                } else {
                    last_nr = st.last_nr;
                    last_is_current = p->method != LAP_MG_FP32;
                }
                continue;
            }
            if (tuner) {
                // the tail size of this period: the next untried candidate while tuning; a
                // period that captures its graph is not timed
                const int cidx = tuner->next();
                set_tail(tuner->cand[cidx]);
                if (tuner->done) {
                    run_period(steps, maxdelta, fused_maxd);
                } else {
                    ck(cudaEventRecord(tuner_event(h, 0), s), "record event");
                    const bool captured = run_period(steps, maxdelta, fused_maxd);
                    ck(cudaEventRecord(tuner_event(h, 1), s), "record event");
                    ck(cudaEventSynchronize(tuner_event(h, 1)), "event sync");
                    float ms = 0.f;
                    ck(cudaEventElapsedTime(&ms, tuner_event(h, 0), tuner_event(h, 1)), "event time");
                    if (!captured) tuner->record(cidx, ms / (double)steps);
                }
            } else {
                run_period(steps, maxdelta, fused_maxd);
            }
            k += steps;
            double val;
            bool conv;
            if (maxdelta) {
                if (!fused_maxd)
                    ck(launch_maxdelta(f, w.aux, w.maxd, s), "max delta kernel");
                val = read_maxd();
                conv = val <= p->tol;
                last_is_current = false;
            } else {
                const Field cur{p->method == LAP_JACOBI ? jac_cur : f.p, f.m, f.n, f.pitch};
                if (p->method == LAP_MG_FP32)
                    ck(launch_defect32_sumsq(w.levels32[0].u, w.levels32[0].q, c, w.partials, s),
                       "residual kernel");
                const double nr = fp32_norm ? partial_norm(f, p->method == LAP_MG_MIXED && norm_sc > 0.0)
                                            : residual(cur, nullptr);
                val = p->norm == LAP_NORM_L2_REL ? nr / r0 : nr;
                conv = p->norm == LAP_NORM_L2_REL ? nr <= p->tol * r0 : nr <= p->tol;
                last_nr = nr;
                last_is_current = p->method != LAP_MG_FP32;  // FP32 alone tests its FP32 residual
            }
            out->last_check = val;
            if (!std::isfinite(val))
                out->status = LAP_DIVERGED;
            else if (conv)
                out->status = LAP_CONVERGED;
        }
        out->iters = k;
        if (p->method == LAP_JACOBI && jac_cur != f.p) copy_field(f.p, jac_cur);
        if (p->method == LAP_MG_FP32)
            ck(launch_to64(f, w.levels32[0].u.p, w.levels32[0].u.pitch, s), "conversion kernel");
        // the last stopping test already took the final iterate's norm (no second pass)
        out->r_final = last_is_current ? last_nr : residual(f, nullptr);
    }
};

}  // namespace

// ============================== C ABI =======================================================

extern "C" {

void lap_default_params(lap_params* p)
{
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->method = LAP_SOR_RB;
    p->w = 1.0;
    p->tol = 1e-10;
    p->norm = LAP_NORM_L2_REL;
    p->max_iter = 100000;
    p->check_every = 1;
    p->nu1 = 2;
    p->nu2 = 2;
    p->coarsest_min = 5;
    p->max_levels = 0;
    p->smoother_w = 1.0;
    p->line_form = LAP_FORM_A;
    p->inner_cycles = 1;
}

int lap_create(lap_handle* out, size_t hbm_budget_bytes, int device)
{
    return guarded([&] {
        if (!out) fail(LAP_EINVAL, "out is NULL");
        *out = nullptr;
        int count = 0;
        ck(cudaGetDeviceCount(&count), "cudaGetDeviceCount");
        if (device < 0 || device >= count) fail(LAP_EINVAL, "no such CUDA device");
        ck(cudaSetDevice(device), "cudaSetDevice");
        lap_handle h = new lap_handle_s();
        h->device = device;
        h->budget = hbm_budget_bytes;
        cudaError_t e = cudaMallocHost(&h->pinned, 8 * sizeof(double));
        if (e != cudaSuccess) {
            delete h;
            ck(e, "cudaMallocHost");
        }
        *out = h;
    });
}

void lap_destroy(lap_handle h)
{
    if (!h) return;
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    h->batch_cache.reset();
    for (auto& kv : h->lines) dev_free(h, kv.second.dev, kv.second.bytes);
    for (auto& kv : h->coarse) dev_free(h, kv.second.dev, kv.second.bytes);
    drop_graphs(h);
    if (h->capture) cudaStreamDestroy(h->capture);
    for (cudaEvent_t e : h->ev)
        if (e) cudaEventDestroy(e);
    dev_free(h, h->lscratch, h->lscratch_bytes);
    dev_free(h, h->hfield, h->hfield_bytes);
    dev_free(h, h->lsync, h->lsync_bytes);
    dev_free(h, h->arena, h->arena_bytes);
    if (h->pinned) cudaFreeHost(h->pinned);
    delete h;
}

namespace {

// What lap_solve cannot run on a valid grid with valid parameters (LAP_EUNSUPPORTED): the
// same answer from the size query as from the solve.
void check_supported(const lap_grid* g, const lap_params* p)
{
    if (p->sum_order == LAP_SUM_DIAGONAL) {
        if (!make_coef(g->dx, g->dy).unit_beta)
            fail(LAP_EUNSUPPORTED, "sum_order LAP_SUM_DIAGONAL needs dx == dy (beta = 1)");
        if (rb_diag_walks(g->m, g->n) > RB_DIAG_MAX_WALKS)
            fail(LAP_EUNSUPPORTED, "sum_order LAP_SUM_DIAGONAL numbers its diagonal walks with "
                                   "32-bit ints: at most about 2.5e10 points (LAP_SUM_PAPER has "
                                   "no such limit)");
    }
    if (p->method == LAP_MG || p->method == LAP_MG_MIXED || p->method == LAP_MG_FP32) {
        const int L = mg_level_count(g->m, g->n, p->coarsest_min, p->max_levels);
        int m = g->m, n = g->n;
        for (int l = 1; l < L; ++l) {
            m = (m - 1) / 2 + 1;
            n = (n - 1) / 2 + 1;
        }
        if ((int64_t)(m - 2) * (n - 2) > COARSE_MAX_UNKNOWNS)
            fail(LAP_EUNSUPPORTED, "coarsest multigrid level has more than 1024 unknowns; "
                                   "use sizes with (m-1), (n-1) divisible by more powers of two");
    }
    if ((p->method == LAP_GS_LEX || p->method == LAP_SOR_LEX) &&
        (int64_t)g->m * g->n > lex_max_points())
        fail(LAP_EUNSUPPORTED, "lexicographic methods hold the grid in one SM's shared memory: "
                               "at most 28672 points");
    if ((p->method == LAP_ADI || p->method == LAP_SLOR) &&
        (g->m - 2 > LINE_MAX_N || g->n - 2 > LINE_MAX_N))
        fail(LAP_EUNSUPPORTED, "ADI lines longer than 16383 unknowns");
}

}  // namespace

int lap_workspace_bytes(const lap_grid* g, const lap_params* p, size_t* bytes)
{
    return guarded([&] {
        check_grid(g);
        check_params(p);
        if (!bytes) fail(LAP_EINVAL, "bytes is NULL");
        check_supported(g, p);
        *bytes = work_bytes(g, p);
    });
}

namespace {

// lap_solve after the handle, result and pointer checks
void solve_device(lap_handle h, const lap_grid* g, double* psi_dev, const lap_params* p,
                  lap_result* out, cudaStream_t stream)
{
    check_supported(g, p);
    Solver sv{h, stream, Field{psi_dev, g->m, g->n, g->pitch}, make_coef(g->dx, g->dy), p, {}};
    const size_t need = work_bytes(g, p);
    Carver cv(arena(h, need));
    carve(cv, sv.w, g, p);
    sv.run(out);
    check_line_waits(h, stream);
}

}  // namespace

int lap_solve(lap_handle h, const lap_grid* g, double* psi_dev, const lap_params* p,
              lap_result* out, void* stream)
{
    return guarded([&] {
        if (!h) fail(LAP_EINVAL, "handle is NULL");
        if (!out) fail(LAP_EINVAL, "result is NULL");
        check_grid(g);
        check_params(p);
        set_device(h);
        check_device_ptr(h, psi_dev, "psi");
        solve_device(h, g, psi_dev, p, out, (cudaStream_t)stream);
    });
}

int lap_solve_host(lap_handle h, const lap_grid* g, double* psi_host, int64_t host_pitch,
                   const lap_params* p, lap_result* out, void* stream)
{
    return guarded([&] {
        if (!h) fail(LAP_EINVAL, "handle is NULL");
        if (!out) fail(LAP_EINVAL, "result is NULL");
        check_grid(g);
        check_params(p);
        check_supported(g, p);  // before the field is allocated and copied
        if (!psi_host) fail(LAP_EINVAL, "psi_host is NULL");
        if (((uintptr_t)psi_host) % 8) fail(LAP_EINVAL, "psi_host is not 8-byte aligned");
        if (host_pitch < g->m) fail(LAP_EINVAL, "host_pitch must be >= m");
        set_device(h);
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, psi_host) != cudaSuccess) {
            cudaGetLastError();
            a.type = cudaMemoryTypeUnregistered;
        }
        if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged)
            fail(LAP_EINVAL, "psi_host is device memory (use lap_solve)");
        const size_t bytes = (size_t)g->n * (size_t)g->pitch * sizeof(double);
        if (bytes > h->hfield_bytes) {
            // the handle's graphs may hold the old field's address
            drop_graphs(h);
            dev_free(h, h->hfield, h->hfield_bytes);
            h->hfield = nullptr;
            h->hfield_bytes = 0;
            h->hfield = (double*)dev_alloc(h, bytes);
            h->hfield_bytes = bytes;
        }
        cudaStream_t s = (cudaStream_t)stream;
        ck(cudaMemcpy2DAsync(h->hfield, (size_t)g->pitch * 8, psi_host, (size_t)host_pitch * 8,
                             (size_t)g->m * 8, (size_t)g->n, cudaMemcpyHostToDevice, s),
           "copy the field to the device");
        solve_device(h, g, h->hfield, p, out, s);
        ck(cudaMemcpy2DAsync(psi_host, (size_t)host_pitch * 8, h->hfield, (size_t)g->pitch * 8,
                             (size_t)g->m * 8, (size_t)g->n, cudaMemcpyDeviceToHost, s),
           "copy the field to the host");
        ck(cudaStreamSynchronize(s), "stream sync");
    });
}

int lap_residual(lap_handle h, const lap_grid* g, const double* psi_dev, const double* q_dev,
                 double* out, void* stream)
{
    return guarded([&] {
        if (!h) fail(LAP_EINVAL, "handle is NULL");
        if (!out) fail(LAP_EINVAL, "out is NULL");
        check_grid(g);
        set_device(h);
        check_device_ptr(h, psi_dev, "psi");
        check_device_ptr(h, q_dev, "q", true);
        cudaStream_t s = (cudaStream_t)stream;
        Carver cv(arena(h, NORM_PARTIALS_MAX * 8 + 1024));
        double* partials = cv.take<double>(NORM_PARTIALS_MAX);
        double* nrm = cv.take<double>(2);
        const Field f{const_cast<double*>(psi_dev), g->m, g->n, g->pitch};
        const Coef c = make_coef(g->dx, g->dy);
        ck(launch_defect_sumsq(f, q_dev, c, partials, s), "residual kernel");
        ck(launch_sum_partials(partials, norm_blocks(f), nrm, s), "sum kernel");
        ck(cudaMemcpyAsync(h->pinned, nrm + 1, 8, cudaMemcpyDeviceToHost, s), "copy norm");
        ck(cudaStreamSynchronize(s), "stream sync");
        *out = h->pinned[0];
        check_line_waits(h, s);
    });
}

int lap_smooth(const lap_grid* g, double* psi_dev, const double* q_dev, double w, int nsweeps,
               void* stream)
{
    return guarded([&] {
        check_grid(g);
        if (!(w > 0.0 && w < 2.0)) fail(LAP_EINVAL, "w must lie in (0, 2)");
        if (nsweeps < 0) fail(LAP_EINVAL, "nsweeps must be >= 0");
        check_device_ptr(nullptr, psi_dev, "psi");
        check_device_ptr(nullptr, q_dev, "q", true);
        const Field f{psi_dev, g->m, g->n, g->pitch};
        const Coef c = make_coef(g->dx, g->dy);
        for (int k = 0; k < nsweeps; ++k)
            for (int colour = 0; colour < 2; ++colour)
                ck(launch_rb_colour(f, q_dev, c, w == 1.0, w, colour, nullptr, (cudaStream_t)stream),
                   "smoother kernel");
    });
}

int lap_jacobi_sweep(const lap_grid* g, const double* in_dev, double* out_dev, void* stream)
{
    return guarded([&] {
        check_grid(g);
        check_device_ptr(nullptr, in_dev, "in");
        check_device_ptr(nullptr, out_dev, "out");
        if (in_dev == out_dev) fail(LAP_EINVAL, "Jacobi needs distinct in and out buffers");
        cudaStream_t s = (cudaStream_t)stream;
        ck(cudaMemcpy2DAsync(out_dev, g->pitch * 8, in_dev, g->pitch * 8, (size_t)g->m * 8, g->n,
                             cudaMemcpyDeviceToDevice, s),
           "copy ring");
        const Field f{const_cast<double*>(in_dev), g->m, g->n, g->pitch};
        ck(launch_jacobi(f, out_dev, make_coef(g->dx, g->dy), nullptr, s), "jacobi kernel");
    });
}

int lap_restrict(const lap_grid* fine, const double* u_dev, const double* q_dev, double* r_dev,
                 double* qc_dev, double* ec_dev, int64_t pitch_c, void* stream)
{
    return guarded([&] {
        check_grid(fine);
        if ((fine->m - 1) % 2 || (fine->n - 1) % 2 || fine->m < 5 || fine->n < 5)
            fail(LAP_EINVAL, "restriction needs odd m, n >= 5");
        if (pitch_c < (fine->m - 1) / 2 + 1) fail(LAP_EINVAL, "coarse pitch too small");
        check_device_ptr(nullptr, u_dev, "u");
        check_device_ptr(nullptr, q_dev, "q", true);
        check_device_ptr(nullptr, r_dev, "r");
        check_device_ptr(nullptr, qc_dev, "qc");
        check_device_ptr(nullptr, ec_dev, "ec", true);
        cudaStream_t s = (cudaStream_t)stream;
        const Field f{const_cast<double*>(u_dev), fine->m, fine->n, fine->pitch};
        const Coef c = make_coef(fine->dx, fine->dy);
        ck(launch_defect(f, q_dev, r_dev, c, s), "defect kernel");
        ck(launch_restrict(Field{r_dev, fine->m, fine->n, fine->pitch}, qc_dev, ec_dev, pitch_c, s),
           "restrict kernel");
    });
}

int lap_prolong_add(const lap_grid* fine, double* u_dev, const double* ec_dev, int64_t pitch_c,
                    void* stream)
{
    return guarded([&] {
        check_grid(fine);
        if ((fine->m - 1) % 2 || (fine->n - 1) % 2 || fine->m < 5 || fine->n < 5)
            fail(LAP_EINVAL, "interpolation needs odd m, n >= 5");
        if (pitch_c < (fine->m - 1) / 2 + 1) fail(LAP_EINVAL, "coarse pitch too small");
        check_device_ptr(nullptr, u_dev, "u");
        check_device_ptr(nullptr, ec_dev, "ec");
        ck(launch_prolong_add(Field{u_dev, fine->m, fine->n, fine->pitch}, ec_dev, pitch_c,
                              (cudaStream_t)stream),
           "prolong kernel");
    });
}

int lap_coarse_solve(lap_handle h, const lap_grid* g, double* u_dev, const double* q_dev,
                     void* stream)
{
    return guarded([&] {
        if (!h) fail(LAP_EINVAL, "handle is NULL");
        check_grid(g);
        set_device(h);
        check_device_ptr(h, u_dev, "u");
        check_device_ptr(h, q_dev, "q", true);
        const Coef c = make_coef(g->dx, g->dy);
        const double* ainv = coarse_inverse(h, g->m, g->n, c.b2, c.d);
        ck(launch_coarse_solve(Field{u_dev, g->m, g->n, g->pitch}, q_dev, c, ainv,
                               (cudaStream_t)stream),
           "coarse solve kernel");
    });
}

int lap_line_sweep(lap_handle h, const lap_grid* g, double* psi_dev, double w, int form,
                   int direction, void* stream)
{
    return guarded([&] {
        if (!h) fail(LAP_EINVAL, "handle is NULL");
        check_grid(g);
        if (!(w > 0.0 && w < 2.0)) fail(LAP_EINVAL, "w must lie in (0, 2)");
        if (form != LAP_FORM_A && form != LAP_FORM_B) fail(LAP_EINVAL, "unknown line form");
        if (direction != 0 && direction != 1) fail(LAP_EINVAL, "direction must be 0 or 1");
        set_device(h);
        check_device_ptr(h, psi_dev, "psi");
        line_half_sweep(h, Field{psi_dev, g->m, g->n, g->pitch}, make_coef(g->dx, g->dy), w, form,
                        direction, (cudaStream_t)stream);
    });
}

int lap_check_rounding(lap_handle h, int64_t count, uint64_t seed, int64_t* mismatches)
{
    return guarded([&] {
        if (!h || !mismatches) fail(LAP_EINVAL, "handle or result is NULL");
        if (count < 0) fail(LAP_EINVAL, "count must be >= 0");
        set_device(h);
        unsigned long long* bad = (unsigned long long*)dev_alloc(h, sizeof(unsigned long long));
        try {
            ck(cudaMemset(bad, 0, sizeof(unsigned long long)), "zero counter");
            ck(launch_check_rounding(count, seed, bad, nullptr), "rounding check kernel");
            unsigned long long v = 0;
            ck(cudaMemcpy(&v, bad, sizeof v, cudaMemcpyDeviceToHost), "copy counter");
            *mismatches = (int64_t)v;
        } catch (...) {
            dev_free(h, bad, sizeof(unsigned long long));
            throw;
        }
        dev_free(h, bad, sizeof(unsigned long long));
    });
}

int lap_fp64_rate(lap_handle h, double* fma_per_s)
{
    return guarded([&] {
        if (!h || !fma_per_s) fail(LAP_EINVAL, "handle or result is NULL");
        set_device(h);
        const int blocks = 4 * device_sms();
        double* sink = (double*)dev_alloc(h, sizeof(double) * blocks);
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        try {
            ck(cudaEventCreate(&e0), "create event");
            ck(cudaEventCreate(&e1), "create event");
            const long long iters = 1 << 13;
            if (launch_fp64_rate(blocks, iters, sink, nullptr) < 0) ck(cudaGetLastError(), "rate kernel");
            ck(cudaEventRecord(e0, nullptr), "record event");
            const int64_t fmas = launch_fp64_rate(blocks, iters, sink, nullptr);
            if (fmas < 0) ck(cudaGetLastError(), "rate kernel");
            ck(cudaEventRecord(e1, nullptr), "record event");
            ck(cudaEventSynchronize(e1), "event sync");
            float ms = 0.f;
            ck(cudaEventElapsedTime(&ms, e0, e1), "event time");
            *fma_per_s = (double)fmas / (ms * 1e-3);
        } catch (...) {
            if (e0) cudaEventDestroy(e0);
            if (e1) cudaEventDestroy(e1);
            dev_free(h, sink, sizeof(double) * blocks);
            throw;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        dev_free(h, sink, sizeof(double) * blocks);
    });
}

int lap_set_graphs(lap_handle h, int enabled)
{
    return guarded([&] {
        if (!h) fail(LAP_EINVAL, "handle is NULL");
        h->use_graphs = enabled != 0;
    });
}

const char* lap_strerror(int code)
{
    switch (code) {
    case LAP_OK: return "ok";
    case LAP_EINVAL: return "invalid argument";
    case LAP_ENOMEM: return "out of device memory or over the handle's HBM budget";
    case LAP_ECUDA: return "CUDA error";
    case LAP_EUNSUPPORTED: return "unsupported size";
    default: return "unknown error";
    }
}

const char* lap_last_error(void) { return t_last_error.c_str(); }

int64_t lap_kernel_launches(void) { return g_launches.load(); }

}  // extern "C"

// ============================== residual norm without allocation =========================
//
// lap_residual_noalloc computes the same norm as lap_residual for callers that cannot make
// a device allocation (their device memory is fully reserved by another allocator or
// budget, they cannot afford the device-wide synchronisation a cudaMalloc/cudaFree pair
// implies, or they hold no lap_handle). Its scratch -- the per-block partial sums of the
// residual kernel and the final pair [sum of squares, norm] -- lives in the file-scope
// device array below instead of a handle's arena.

namespace {

// The residual kernel writes at most norm_blocks() partial sums, 6 per multiprocessor of
// the device whatever the grid size: 912 on a 152-SM GB300. The array holds 1216 (devices
// of up to 202 multiprocessors); a call that would need more is refused.
constexpr int kNoAllocPartials = 1216;
constexpr int kNoAllocDoubles = kNoAllocPartials + 2;  // partials, then [sum, sqrt(sum)]
constexpr int kNoAllocMaxDevices = 64;

// Device scratch shared by every call on a device, ~9.5 KB, held until the process exits.
// In host code this name is only a stand-in; its device address comes from
// cudaGetSymbolAddress.
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

std::mutex g_noalloc_mutex;
double* g_noalloc_addr[kNoAllocMaxDevices] = {};

// Device address of the scratch array on `device` (the current device), looked up once
// per device on the first call that runs there.
double* noalloc_scratch(int device)
{
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[device]) {
        void* p = nullptr;
        ck(cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress");
        g_noalloc_addr[device] = static_cast<double*>(p);
    }
    return g_noalloc_addr[device];
}

void check_on_device(const void* p, int device, const char* what, bool allow_null)
{
    if (!p) {
        if (allow_null) return;
        fail(LAP_EINVAL, std::string(what) + " is NULL");
    }
    if (((uintptr_t)p) % 8) fail(LAP_EINVAL, std::string(what) + " is not 8-byte aligned");
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        fail(LAP_EINVAL, std::string(what) + " is not a CUDA pointer");
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
        fail(LAP_EINVAL, std::string(what) + " is not device memory");
    if (a.device != device) fail(LAP_EINVAL, std::string(what) + " is not on the current device");
}

}  // namespace

extern "C" int lap_residual_noalloc(const lap_grid* g, const double* psi_dev, const double* q_dev,
                                    double* out_dev, void* stream)
{
    return guarded([&] {
        check_grid(g);
        int device = 0;
        ck(cudaGetDevice(&device), "cudaGetDevice");
        if (device < 0 || device >= kNoAllocMaxDevices)
            fail(LAP_EUNSUPPORTED, "lap_residual_noalloc supports device ordinals below 64");
        check_on_device(psi_dev, device, "psi", false);
        check_on_device(q_dev, device, "q", true);
        check_on_device(out_dev, device, "out", false);
        const Field f{const_cast<double*>(psi_dev), g->m, g->n, g->pitch};
        const int blocks = norm_blocks(f);
        if (blocks > kNoAllocPartials)
            fail(LAP_EUNSUPPORTED, "lap_residual_noalloc: the residual needs " +
                                       std::to_string(blocks) + " partial sums, its scratch holds " +
                                       std::to_string(kNoAllocPartials));
        double* scratch = noalloc_scratch(device);
        cudaStream_t s = (cudaStream_t)stream;
        // every partial the sum reads is written first by this call: nothing to clear
        ck(launch_defect_sumsq(f, q_dev, make_coef(g->dx, g->dy), scratch, s), "residual kernel");
        ck(launch_sum_partials(scratch, blocks, scratch + kNoAllocPartials, s), "sum kernel");
        ck(cudaMemcpyAsync(out_dev, scratch + kNoAllocPartials + 1, sizeof(double),
                           cudaMemcpyDeviceToDevice, s),
           "copy norm");
    });
}
