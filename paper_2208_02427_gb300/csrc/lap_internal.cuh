// lap_internal.cuh -- declarations shared by the kernels and the C-ABI layer of
// liblaplace.so. Not part of the public ABI (include/laplace.h is).
#pragma once

#include <cuda_runtime.h>
#include <atomic>
#include <cstdint>

namespace lap {

// cudaFuncSetAttribute acts on the current device only, so what a prepare_* function has
// already raised is recorded per device ordinal. Ordinals past the table are never recorded
// (their attributes are set again on every call, which is harmless).
constexpr int ATTR_DEVICES = 64;
inline int attr_slot()
{
    int d = -1;
    if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= ATTR_DEVICES) return -1;
    return d;
}
// Raise the recorded value of slot d to at least v.
inline void attr_record(std::atomic<size_t>* table, int d, size_t v)
{
    if (d < 0) return;
    size_t cur = table[d].load();
    while (cur < v && !table[d].compare_exchange_weak(cur, v)) {}
}

// Coefficients of the 5-point equation (E+W) + b2 (N+S) - d psi (+ q) = 0, Eq. 5.
struct Coef {
    double b2;      // beta^2, beta = dx/dy
    double d;       // 2 (1 + beta^2)
    double inv_d;   // the double nearest 1/d
    bool unit_beta; // b2 == 1: fma(b2, x, y) == x + y, the multiply is skipped
    int inv_d_shift;// > 0 when inv_d == 2^-inv_d_shift exactly (d a power of two)
};
Coef make_coef(double dx, double dy);

// A pitched field of doubles on the device.
struct Field {
    double* p;
    int m, n;
    int64_t pitch;
};

// A pitched field of floats (the inner FP32 multigrid cycle).
struct Field32 {
    float* p;
    int m, n;
    int64_t pitch;
};

// Every kernel launch of the library goes through this counter.
void note_launch();

// ---- point kernels (point_kernels.cu) -------------------------------------------
// One colour of a red-black sweep, in place: Gauss-Seidel (Eq. 6) when gs is true,
// SOR (Eq. 7) otherwise; q may be null. maxd (nullable) accumulates max|new - old| as
// the bit pattern of a non-negative double.
// wslot (nullable): device copy of {w, 1 - w}, read instead of the w argument (faster).
cudaError_t launch_rb_colour(const Field& f, const double* q, const Coef& c, bool gs, double w,
                             int colour, unsigned long long* maxd, cudaStream_t s,
                             const double* wslot = nullptr);
// The same colour pass with the neighbour sum paired along diagonals, (W + S) + (E + N), for
// beta = 1 only (rb_diag_kernel): 4 FP64 operations per SOR update instead of 5. A thread
// walks RD_K points down a diagonal, RD_BX threads per CTA. The rows are cut into strips of
// RD_K; the widest strip of an m-wide field has rb_diag_starts(m) walks, and the launch takes
// rb_diag_walks(m, n) in all, numbered with 32-bit ints: at most RB_DIAG_MAX_WALKS (a field of
// about 2.5e10 points). The launcher returns cudaErrorInvalidValue above that.
constexpr int RD_BX = 128, RD_K = 6;
constexpr int64_t RB_DIAG_MAX_WALKS = 2147483647 - RD_BX;
inline int rb_diag_starts(int m) { return (m - 2 - (2 - RD_K)) / 2 + 1; }
inline int64_t rb_diag_walks(int m, int n)
{
    return (int64_t)rb_diag_starts(m) * ((n - 2 + RD_K - 1) / RD_K);
}
cudaError_t launch_rb_diag(const Field& f, const double* q, bool gs, double w, int colour,
                           unsigned long long* maxd, cudaStream_t s, const double* wslot = nullptr);
// One Jacobi sweep (Eq. 5) from in to out (same pitch; ring not touched).
cudaError_t launch_jacobi(const Field& in, double* out, const Coef& c, unsigned long long* maxd,
                          cudaStream_t s);
// r := scaled residual on interior nodes (Eqs. 11-12); r has f's pitch.
cudaError_t launch_defect(const Field& f, const double* q, double* r, const Coef& c,
                          cudaStream_t s);
// Multiprocessors of the current device (looked up once per device ordinal).
int device_sms();
// The most partial sums a norm kernel writes: its solve-scratch buffers hold this many.
constexpr int NORM_PARTIALS_MAX = 2046;
// sum of squares of the residual into per-block partials; partials[nblocks].
// Blocks of the norm kernels (256 threads, a grid-stride walk over the interior): one per 256
// interior points, at least 1 and at most 6 per multiprocessor of the current device, all
// resident at once (912 on a 152-SM GB300); never more than NORM_PARTIALS_MAX.
inline int norm_blocks_for(int m, int n)
{
    if (m < 3 || n < 3) return 1;
    const int64_t b = ((int64_t)(m - 2) * (int64_t)(n - 2) + 255) / 256;
    int cap = 6 * device_sms();
    if (cap > NORM_PARTIALS_MAX) cap = NORM_PARTIALS_MAX;
    return b < cap ? (int)b : cap;
}
int norm_blocks(const Field& f);
cudaError_t launch_defect_sumsq(const Field& f, const double* q, const Coef& c, double* partials,
                                cudaStream_t s);
// out[0] = sum(partials[0..count)), fixed order; out[1] = sqrt(out[0]).
cudaError_t launch_sum_partials(const double* partials, int count, double* out, cudaStream_t s);
// FP64 fma issue-rate probe: blocks x 256 threads, `iters` steps of 8 independent fma chains
// each; returns the fmas issued (-1 on a launch error). sink: blocks doubles (never written
// in practice).
int64_t launch_fp64_rate(int blocks, long long iters, double* sink, cudaStream_t s);
// *bad += mismatches of the integer-pipe FP64 -> FP32 rounding against the instruction.
cudaError_t launch_check_rounding(long long count, unsigned long long seed, unsigned long long* bad,
                                  cudaStream_t s);
// State of a device-resident solve loop (host-written before launch, read back after).
struct LoopState {
    long long k;         // iterations done
    long long steps;     // iterations per period
    long long max_iter;
    int mode;            // 0 L2_REL, 1 L2_ABS, 2 MAXDELTA
    int status;          // lap_status of the last test
    double r0, tol;
    double last_check;   // the last test's value
    double last_nr;      // the L2 norm at the last test
};
// k += steps; test nrm[1] (divided by *scale when scale is set) or *maxd (MAXDELTA);
// cudaGraphSetConditional(h, keep going).
cudaError_t launch_loop_decide(LoopState* st, const double* nrm, const unsigned long long* maxd,
                               const float* scale, cudaGraphConditionalHandle h, cudaStream_t s);
// Batched solves: st[0] += 1 (cycles done), then the loop's condition := some problem still
// running (*remaining > 0) and st[0] < st[1] (the cycle cap).
cudaError_t launch_batch_loop_decide(long long* st, const int* remaining, cudaGraphConditionalHandle h,
                                     cudaStream_t s);
// maxd := max |a - b| over interior nodes (bit pattern), a and b share f's shape/pitch.
cudaError_t launch_maxdelta(const Field& a, const double* b, unsigned long long* maxd,
                            cudaStream_t s);

// ---- multigrid transfer kernels (mg_kernels.cu) ----------------------------------
// qc (coarse interior) := 0.25 ((4 r_c + 2 edges) + corners); ec (nullable) := 0 in the interior.
cudaError_t launch_restrict(const Field& fine_r, double* qc, double* ec, int64_t pitch_c,
                            cudaStream_t s);
// u (fine interior) += bilinear interpolation of ec.
cudaError_t launch_prolong_add(const Field& fine_u, const double* ec, int64_t pitch_c,
                               cudaStream_t s);
// u interior := Ainv_t^T b with b the coarse right-hand side assembled from q and u's ring.
cudaError_t launch_coarse_solve(const Field& u, const double* q, const Coef& c,
                                const double* ainv_t, cudaStream_t s);

// ---- FP32 cycle inside FP64 defect correction (mixed_kernels.cu) -----------------
int mixed_norm_blocks(int m, int n);
cudaError_t launch_rb32(const Field32& f, const float* q, const Coef& c, bool gs, double w,
                        int colour, cudaStream_t s);
cudaError_t launch_defect32(const Field32& f, const float* q, float* r, const Coef& c,
                            cudaStream_t s);
cudaError_t launch_restrict32(const Field32& fine_r, float* qc, float* ec, int64_t pitch_c,
                              cudaStream_t s);
cudaError_t launch_prolong32(const Field32& fine_u, const float* ec, int64_t pitch_c,
                             cudaStream_t s);
cudaError_t launch_coarse32(const Field32& u, const float* q, const double* ainv_t, cudaStream_t s);
// r32 := (float) FP64 residual of psi, e32 := 0 (interiors), partials := per-block sums of r^2
// (the same blocks and order as launch_defect_sumsq, so the sums are identical).
// norm_scale (nullable device slot): sum the squares in FP32 as (scale r)^2 instead of FP64.
// e32 nullable: leave the correction alone.
cudaError_t launch_defect64_to32(const Field& psi, const Coef& c, float* r32, float* e32,
                                 int64_t pitch32, double* partials, cudaStream_t s,
                                 const float* norm_scale = nullptr);
// FP32 alone: a (and b, nullable) := psi rounded to FP32 on every node; psi interior :=
// (double) u; per-block FP64 sums of the squared FP32 residual (mixed_norm_blocks blocks).
cudaError_t launch_to32(const Field& psi, float* a, float* b, int64_t pitch32, cudaStream_t s);
cudaError_t launch_to64(const Field& psi, const float* u, int64_t pitch32, cudaStream_t s);
cudaError_t launch_defect32_sumsq(const Field32& f, const float* q, const Coef& c, double* partials,
                                  cudaStream_t s);
// psi += (double) e32 on interior nodes.
cudaError_t launch_update64(const Field& psi, const float* e32, int64_t pitch32, cudaStream_t s);

// ---- lexicographic Gauss-Seidel / SOR on one SM (lex_kernels.cu) ---------------------
// nsweeps sweeps of Eq. 6 (gs) or Eq. 7 in the paper's order as diagonal wavefronts, the
// field resident in shared memory; maxd (nullable) gets max|new - old| of the last sweep.
int64_t lex_max_points();
size_t lex_smem_bytes(int m, int n);
cudaError_t prepare_lex_kernels(size_t smem);
cudaError_t launch_lex_sweeps(const Field& f, const Coef& c, bool gs, double w, int nsweeps,
                              unsigned long long* maxd, cudaStream_t s);
// A whole solve in one CTA with the stopping rule of Eq. 16 (max |change| <= tol, tested
// after every st->steps iterations, up to st->max_iter): kind 0 Jacobi (2 m n doubles of
// shared memory), 1 red-black, 2 lexicographic (m n doubles); gs or SOR with {w, 1 - w}
// from wslot. Reads st->k, steps, max_iter, tol, last_check; writes k, status, last_check.
// Zebra SLOR (adi = false) or ADI in one CTA with the field in shared memory, periods until
// the stopping rule (MAXDELTA) holds; LoopState as for launch_solve_cta.
size_t solve_lines_cta_smem(int m, int n);
cudaError_t launch_solve_lines_cta(const Field& f, const Coef& c, bool adi, int form,
                                   const double* wslot, LoopState* st, cudaStream_t s);
cudaError_t launch_solve_cta(const Field& f, const Coef& c, int kind, bool gs, const double* wslot,
                             LoopState* st, cudaStream_t s);

// ---- V-cycle over many grids (batch_kernels.cu) -------------------------------------
// One level of one problem. Level 0 of the FP64 solve is the caller's field (q null).
template <class T>
struct BatchLevel {
    T* u;  // field or correction
    T* q;  // source term (null on the FP64 fine level); FP32 level 0: the FP64 residual
    T* r;  // residual scratch (not on the coarsest level)
    int m, n;
    int64_t pitch;
    int problem;
    int unit_beta;
    int inv_d_shift;
    double b2, d, inv_d;
    double w, omw;         // per-problem SOR factor and 1 - w (batched point sweeps)
    const double* ainv_t;  // coarsest level: transposed inverse of its 5-point matrix
};
struct BatchItem {
    int level;  // index into the level array
    int row0;   // first interior row
    int rows;   // rows in this item
};
// A work list of one launch. claim (nullable): two words of device memory, zero between
// launches; with it the launch is persistent -- as many CTAs as fit the device at once, each
// taking the next unclaimed item until none is left (ItemClaim) -- and without it one CTA per
// item. Either way every item gets the same arithmetic.
struct BatchList {
    const BatchItem* items;
    int count;
    unsigned* claim = nullptr;
};
// CTAs of `kernel` (threads per CTA, dynamic shared memory) resident on the current device at
// once: multiprocessors x CTAs per multiprocessor, looked up once per kernel and device.
int resident_blocks(const void* kernel, int threads, size_t smem);
// The grid of a launch over `count` items: count, or when persistent at most resident_blocks.
inline int batch_grid(const void* kernel, int threads, size_t smem, int count, bool persist)
{
    if (!persist) return count;
    const int r = resident_blocks(kernel, threads, smem);
    return r < count ? r : count;
}
// The small-level tail of one problem's V-cycle: levels first .. last (its coarsest) of lv.
struct TailJob {
    int first, last;
};
// The Dirichlet ring of the u, q and r buffers of FP32 levels lv[0 .. count) (device
// descriptors) set to zero; max_side >= every level's m and n.
cudaError_t launch_zero_rings32(const BatchLevel<float>* lv, int count, int max_side, cudaStream_t s);
// per_level_w: Eq. 7 with each level's own w (BatchLevel::w) instead of the argument
template <class T>
cudaError_t launch_b_rb(const BatchList& l, const BatchLevel<T>* lv, const int* active, int colour,
                        bool gs, double w, cudaStream_t s, bool per_level_w = false);
template <class T>
cudaError_t launch_b_defect(const BatchList& l, const BatchLevel<T>* lv, const int* active,
                            cudaStream_t s);
// items of the coarse level; the fine level is the preceding entry of lv
template <class T>
cudaError_t launch_b_restrict(const BatchList& l, const BatchLevel<T>* lv, const int* active,
                              cudaStream_t s);
// items of the fine level; the coarse level is the following entry of lv
template <class T>
cudaError_t launch_b_prolong(const BatchList& l, const BatchLevel<T>* lv, const int* active,
                             cudaStream_t s);
template <class T>
cudaError_t launch_b_coarse(const BatchList& l, const BatchLevel<T>* lv, const int* active,
                            int max_unknowns, cudaStream_t s);
// One CTA per job runs the V-cycle from level `first` down to the coarsest and back (nu1/nu2
// smoothing sweeps, gs or SOR with w, or each level's own w); active may be null (all run).
// max_unknowns: the largest coarsest level among the jobs.
// claim (nullable): a persistent launch over the jobs (see BatchList).
template <class T>
cudaError_t launch_b_tail(const TailJob* jobs, int count, const BatchLevel<T>* lv, const int* active,
                          int nu1, int nu2, bool gs, double w, int max_unknowns, cudaStream_t s,
                          bool per_level_w = false, unsigned* claim = nullptr);
// per-item FP64 sum of squares of the residual; with lv32 also r32 := residual, e32 := 0;
// with r0 (per problem) the mixed problems sum their squares in FP32 after an exact
// power-of-two scaling from r0 (the partials are stored descaled)
cudaError_t launch_b_sumsq(const BatchList& l, const BatchLevel<double>* lv, const int* active,
                           double* partials, const BatchLevel<float>* lv32, cudaStream_t s,
                           const double* r0 = nullptr);
cudaError_t launch_b_update(const BatchList& l, const BatchLevel<double>* lv, const int* active,
                            const BatchLevel<float>* lv32, cudaStream_t s);
// A problem that left the batch in a convergence test: its index, lap_status, cycles run and
// norms (the serving loop's completion list).
struct Completion {
    int problem;
    int status;
    long long iters;
    double r0, rnow;
};
// mode 0: record r0 (retire problems already converged); mode 1: count a cycle and test.
// Problems with no items in the list are left alone; tolv (nullable) gives one tol each;
// maxit (nullable): a problem that has run its maxit[p] cycles without converging retires
// with LAP_MAXITER (in mode 0 when maxit[p] is 0); done (nullable): every retiring problem is
// appended to done[*ndone++].
cudaError_t launch_b_converge(const double* partials, const int* first_item, int count, int* active,
                              double* r0, double* rnow, long long* iters, int* status,
                              int* remaining, int mode, bool rel, double tol, cudaStream_t s,
                              const double* tolv = nullptr, const long long* maxit = nullptr,
                              Completion* done = nullptr, int* ndone = nullptr);

// ---- the FP32 cycle's levels in two tile passes (fused32_kernels.cu) --------------
// One tile of owned points [x0, x0 + tx) x [y0, y0 + ty) of level `level` of lv.
struct TileItem {
    int level, x0, y0, tx, ty;
};
// Whether nu1, nu2 sweeps fit the tile halos; tiles of a level: ntx x nty of tx x ty.
bool fused32_supported(int nu1, int nu2);
void fused32_tile(int m, int n, int nu1, int nu2, int* tx, int* ty, int* ntx, int* nty);
// Batched tile variants (CTA size and region rows, see fused32_kernels.cu): 1..FUSED32_VARIANTS;
// every variant computes the same values. 1 is the single-grid tiles' shape.
constexpr int FUSED32_VARIANTS = 3;
bool fused32_variant_supported(int variant, int nu1, int nu2);
void fused32_tile_variant(int variant, int m, int n, int nu1, int nu2, int* tx, int* ty, int* ntx,
                          int* nty);
cudaError_t prepare_fused32();  // shared-memory limit of the tile kernels (outside capture)
// Descent of level F: nu1 sweeps on u (F.u, or zeros), smoothed u -> F.r, C.q := restricted
// residual, C.u := 0. Ascent: F.u := smoothed (F.r + P C.u) after nu2 sweeps.
cudaError_t launch_down32(const BatchLevel<float>& F, const BatchLevel<float>& C, int nu1, int nu2,
                          bool zero_u, bool gs, double w, cudaStream_t s);
// psi (nullable): add the ascent's result to this FP64 field instead of storing it (the
// mixed solver's update, folded into its last level-0 ascent).
cudaError_t launch_up32(const BatchLevel<float>& F, const BatchLevel<float>& C, int nu1, int nu2,
                        bool gs, double w, cudaStream_t s, double* psi = nullptr,
                        int64_t psi_pitch = 0);
// The same over tile items of many problems (the coarse level of item level l is l + 1).
// claim (nullable): a persistent launch over the tiles (see BatchList).
cudaError_t launch_b_down32(const TileItem* items, int count, const BatchLevel<float>* lv,
                            const int* active, int nu1, bool zero_u, bool gs, double w, cudaStream_t s,
                            int variant = 1, unsigned* claim = nullptr);
// lv64 (nullable): items' FP64 fields (same level indices) take psi += result instead.
cudaError_t launch_b_up32(const TileItem* items, int count, const BatchLevel<float>* lv,
                          const int* active, int nu2, bool gs, double w, cudaStream_t s,
                          const BatchLevel<double>* lv64 = nullptr, int variant = 1,
                          unsigned* claim = nullptr);

// ---- line relaxation (line_kernels.cu) --------------------------------------------
// Constant-coefficient tridiagonal systems -alpha x_{k-1} + delta x_k - alpha x_{k+1} = b_k,
// k = 1..N, cut into P <= 32 chunks of L unknowns (the last one Ll), each but the last followed
// by one separator unknown; solved by unnormalised forward elimination per chunk, an exact
// cyclic-reduction solve of the separators, and a scaled back substitution (line_kernels.cu).
// Everything but the right-hand side depends only on (N, alpha, delta, w cross) and is
// precomputed on the host.
constexpr int LINE_MAX_CHUNKS = 32;    // y-lines (one warp per line's separators)
constexpr int LINE_MAX_CHUNKS_X = 64;  // x-lines (two warps run a line's chunks)
struct LineTables {
    int N;       // unknowns per line
    int L;       // chunk length (full chunks)
    int P;       // chunks (<= maxp); separators S = P - 1
    int maxp;    // chunk cap of this partition (32 or 64): the row stride of k1 and k2
    int Ll;      // length of the last chunk (1..L)
    int K0;      // F, gln, glnl are below 2^-64 of their first entry from position K0 on
    int levels;  // cyclic-reduction levels over the S separators
    int stride;  // x-lines: shared-memory stride of a chunk (L + 1 rounded up to odd)
    double alpha, delta, wc;
    // device arrays (one allocation)
    const double* e;        // [L] alpha / den_q (den_q the zero-end chunk's Thomas pivots)
    const double* inv_den;  // [L] 1 / den_q
    const double* sc;       // [L + 1] wc / den_q; wc at index L (a separator's output scale)
    const double* F;        // [L] forward elimination of alpha e_0: F_0 = alpha, F_q = F_{q-1} e_{q-1}
    const double* gln;      // [L] first row of the inverse of a length-L chunk matrix
    const double* glnl;     // [L] the same for the last chunk (length Ll)
    const double* k1;       // [levels * maxp] cyclic-reduction multipliers of the lower neighbour
    const double* k2;       // [levels * maxp] ... of the upper neighbour
    const double* invb;     // [maxp] 1 / reduced diagonal
};
// Per-call scalars of a half sweep: bnd = off / cross (the Dirichlet ends' coefficient in the
// scaled right-hand side), c1 = d (1 - w) / (w cross) (form B), omw = 1 - w, wc = w cross.
struct LineCoefs {
    double bnd, c1, omw, wc;
};
size_t line_smem_bytes(const LineTables& t);
cudaError_t prepare_line_kernels(size_t smem);
// x-lines: a whole zebra half sweep of the nlines interior rows (both colours) in one launch.
// sync: line_x_sync_words(nlines) words of device memory; word 0 is an error word that the
// kernel sets if a wait for a neighbouring row timed out (never cleared by the launch), the
// others are zeroed by the launch.
size_t line_x_sync_words(int nlines);
cudaError_t launch_line_x(double* psi, int64_t pitch, int nlines, const LineTables& t, int form,
                          const LineCoefs& k, unsigned* sync, cudaStream_t s);
// Lines first_line, first_line + 2, ... (count of them) through a scratch array, one thread
// per (line, chunk): element k of line l at psi + l * sx + k * sa (y-lines: sa = pitch,
// sx = 1; x-lines: sa = 1, sx = pitch). scratch holds line_y_scratch_doubles(t, gp)
// doubles, gp >= count a multiple of 32.
size_t line_y_scratch_doubles(const LineTables& t, int64_t gp);
cudaError_t launch_line_scratch(double* psi, int64_t sa, int64_t sx, int first_line, int count,
                                const LineTables& t, int form, const LineCoefs& k, double* scratch,
                                int64_t gp, cudaStream_t s);

}  // namespace lap
