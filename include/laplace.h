/*
 * laplace.h -- C ABI of liblaplace.so, a GB300 (sm_103a) solver for the 2D Laplace
 * equation discretised with the 5-point stencil, implementing the methods compared in
 * "A Comparison of SOR, ADI and Multigrid Methods for Solving Partial Differential
 * Equations" (arXiv 2208.02427): Jacobi, Gauss-Seidel and SOR (in red-black order),
 * ADI line relaxation (zebra line order) and the multigrid V-cycle.
 *
 * Conventions shared by every entry point
 *  - A field is m x n doubles, row-major with a row pitch: psi[j*pitch + i] is the
 *    paper's psi_{i,j}; i = 0..m-1 runs along x, j = 0..n-1 along y (Problem
 *    Definition, Eq. 4). pitch >= m, in elements. The outer ring (i = 0, i = m-1,
 *    j = 0, j = n-1) holds the Dirichlet data and is never written.
 *  - beta = dx/dy and d = 2(1 + beta^2) as in Eq. 5.
 *  - Device pointers are owned by the caller; the library never frees them. They must
 *    be 8-byte aligned device memory of the current device. Scratch memory belongs to
 *    a lap_handle (see lap_create) and is bounded by its HBM budget.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream). Work is stream-ordered.
 *    Entry points that return host values (lap_solve, lap_residual, lap_coarse_solve's
 *    status) synchronise that stream before they return; the others only enqueue.
 *  - Return value: LAP_OK (0) or a negative LAP_E* code; lap_strerror names it. No
 *    exception or signal crosses the ABI. After LAP_ECUDA the device state is
 *    whatever CUDA reported; the handle stays valid for lap_destroy.
 *  - A lap_handle is not thread-safe: use one handle per host thread.
 *
 * Arithmetic: FP64 throughout. Jacobi, Gauss-Seidel, SOR, the multigrid smoother,
 * residual, restriction and interpolation evaluate exactly the expressions written in
 * each entry's comment, with every multiply-add fused where the comment says fma and
 * nowhere else, so their results do not depend on the launch configuration. lap_solve's
 * Gauss-Seidel and SOR can instead sum the neighbours as (W + S) + (E + N) (lap_params
 * sum_order, beta = 1), again one fixed expression. Line solves, the coarsest-grid solve
 * and norms are reassociated for parallelism.
 */
#ifndef LAPLACE_H
#define LAPLACE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LAP_ABI_VERSION 3

enum {
    LAP_OK = 0,
    LAP_EINVAL = -1,       /* an argument is out of range (message via lap_last_error) */
    LAP_ENOMEM = -2,       /* the handle's HBM budget or the device cannot hold the scratch */
    LAP_ECUDA = -3,        /* a CUDA call failed */
    LAP_EUNSUPPORTED = -4  /* valid but outside this build's limits (e.g. very long lines) */
};

typedef enum {
    LAP_JACOBI = 0,  /* Eq. 5, out of place (a scratch copy of psi) */
    LAP_GS_RB = 1,   /* Eq. 6, red (i+j even) then black points */
    LAP_SOR_RB = 2,  /* Eq. 7, red then black points */
    LAP_ADI = 3,     /* x-lines then y-lines per iteration (ADI subsection, Eqs. 8-10) */
    LAP_MG = 4,      /* V-cycle (Multigrid Method subsection, steps 1-11) */
    LAP_MG_MIXED = 5, /* the V-cycle's correction equation (Eqs. 13-15) solved by FP32
                        V-cycles inside FP64 defect correction: per iteration,
                        inner_cycles FP32 V(nu1,nu2) cycles on L e = -R, then psi += e
                        and R = L(psi) in FP64 */
    LAP_SLOR = 6,    /* line SOR by rows alone (SLOR subsection, Eqs. 8-10): one zebra
                        x-line sweep per iteration, form line_form (A = SLORA, B = SLORB) */
    LAP_GS_LEX = 7,  /* Eq. 6 in the paper's lexicographic order (i-1, j-1 already new), as
                        diagonal wavefronts on one SM; m*n <= 28672 (else EUNSUPPORTED) */
    LAP_SOR_LEX = 8, /* Eq. 7 in lexicographic order, same limits */
    LAP_MG_FP32 = 9  /* the V-cycle of LAP_MG entirely in FP32 (psi rounded to FP32 once,
                        widened back at the end; stopping rule on the FP32 residual): the
                        plain-FP32 comparison point of LAP_MG_MIXED, which stalls near FP32
                        rounding (relative residual ~1e-6). Norm L2_REL or L2_ABS */
} lap_method;

typedef enum {
    LAP_NORM_L2_REL = 0,  /* stop when ||r(psi^k)||_2 <= tol * ||r(psi^0)||_2 */
    LAP_NORM_L2_ABS = 1,  /* stop when ||r(psi^k)||_2 <= tol */
    LAP_NORM_MAXDELTA = 2 /* stop when max|psi^k - psi^(k-1)| <= tol (Eq. 16) */
} lap_norm;

typedef enum {
    LAP_FORM_A = 0, /* SLORA: solve the line system of Eq. 8, then relax (Eq. 9) */
    LAP_FORM_B = 1  /* SLORB: relaxation inside the line system (Eq. 10) */
} lap_line_form;

typedef enum { LAP_CONVERGED = 0, LAP_MAXITER = 1, LAP_DIVERGED = 2 } lap_status;

/* Rounding order of the 4-term neighbour sum of Eqs. 5-7. The paper writes the sum without
 * fixing an order; both are the same sum and differ only in rounding. */
typedef enum {
    LAP_SUM_PAPER = 0,   /* (E + W) + beta^2 (N + S), beta^2 fused as fma(beta^2, N + S, E + W):
                            the order of the equation as printed, every method */
    LAP_SUM_DIAGONAL = 1 /* (W + S) + (E + N), beta = 1 only, for LAP_GS_RB and LAP_SOR_RB: a
                            diagonal i - j = const holds points of one colour and the pair E + N
                            of a point is the pair W + S of the next point down the diagonal, so
                            a thread walking the diagonal adds one pair per point: 4 FP64
                            operations per SOR update instead of 5, 2 per Gauss-Seidel update
                            instead of 3 (red-black sweeps are bound by the FP64 issue rate) */
} lap_sum_order;

/* The largest grid: m <= LAP_GRID_MAX_M (row indices and ring counts stay within 32-bit
 * ints) and n <= LAP_GRID_MAX_N (the point kernels launch one CTA row per two field rows,
 * at most 65535); larger grids give LAP_EUNSUPPORTED. Methods add their own limits: the
 * coarsest multigrid level holds at most 1024 unknowns, ADI/SLOR lines at most 16383,
 * lexicographic sweeps 28672 points, and LAP_SUM_DIAGONAL about 2.5e10 points. */
#define LAP_GRID_MAX_M (1 << 28)
#define LAP_GRID_MAX_N 131070

/* The grid of Eq. 4: m points along x, n along y, spacings dx and dy (> 0). */
typedef struct {
    int32_t m, n;     /* >= 3 each; at most LAP_GRID_MAX_M, LAP_GRID_MAX_N */
    double dx, dy;
    int64_t pitch;    /* row pitch of the field, in doubles, >= m */
} lap_grid;

typedef struct {
    int32_t method;       /* lap_method */
    double w;             /* relaxation factor: SOR (Eq. 7), ADI/SLOR (Eqs. 9/10); in (0, 2) */
    double tol;           /* stopping tolerance (>= 0; 0 = run max_iter iterations) */
    int32_t norm;         /* lap_norm */
    int64_t max_iter;     /* iteration cap (V-cycles for LAP_MG), >= 0 */
    int32_t check_every;  /* test the stopping rule every this many iterations (>= 1);
                             the last iteration is always tested */
    int32_t nu1, nu2;     /* LAP_MG: pre/post smoothing sweeps (red-black) */
    int32_t coarsest_min; /* LAP_MG: coarsen while both coarse sides stay >= this (>= 3) */
    int32_t max_levels;   /* LAP_MG: 0 = as many as the sizes allow */
    double smoother_w;    /* LAP_MG: smoother relaxation; 1 = Gauss-Seidel (Eq. 6) */
    int32_t line_form;    /* LAP_ADI, LAP_SLOR: lap_line_form */
    int32_t inner_cycles; /* LAP_MG_MIXED: FP32 V-cycles per FP64 correction (>= 1) */
    int32_t tail_size;    /* LAP_MG, LAP_MG_MIXED, batched: the levels whose sides are all
                             <= tail_size run as one single-CTA kernel per V-cycle (the
                             small-level tail: a CTA barrier per phase instead of a launch;
                             the same arithmetic, so the same iterates bit for bit).
                             0 = chosen by timing the first cycles of a shape (cached in the
                             handle), -1 = never; otherwise >= 3 */
    int32_t unfused;      /* LAP_MG_MIXED: 0 = each FP32 level's descent (smoothing, residual,
                             restriction) and ascent (interpolation, smoothing) run as one
                             shared-memory tile kernel each; non-zero = one kernel per pass
                             (the same values bit for bit; the reference for the tiles) */
    int32_t tiling;       /* batched LAP_MG_MIXED with unfused == 0: how the FP32 levels run.
                             0 = chosen by timing (see lap_solve_batched), -1 = one kernel per
                             pass, 1..3 = tiles of one variant (1: 512 threads over 128 x 64
                             regions, 2: 1024 threads over 128 x 64, 3: 512 threads over
                             128 x 32). Every choice gives the same values bit for bit */
    int32_t item_points;  /* batched solves: interior points per work item of the per-pass
                             kernels (>= 32), 0 = chosen by timing. No effect on the values */
    int32_t persistent;   /* batched solves: how a phase's work items map to CTAs. -1 = one
                             CTA per item, 1 = persistent: as many CTAs as fit the device at
                             once, each claiming the next unclaimed item until none is left;
                             0 = chosen by timing. No effect on the values */
    int32_t sum_order;    /* lap_sum_order (default LAP_SUM_PAPER). LAP_SUM_DIAGONAL with any
                             other method: LAP_EINVAL; with dx != dy: LAP_EUNSUPPORTED */
} lap_params;

typedef struct {
    int32_t status;  /* lap_status */
    int64_t iters;   /* iterations (V-cycles) performed */
    double r0;       /* ||r(psi^0)||_2 of the scaled residual dx^2 L(psi), Eqs. 11-12 */
    double r_final;  /* ||r||_2 after the last iteration (LAP_MG_MIXED: the stopping test's
                        norm, whose squares are summed in FP32 after a power-of-two scaling:
                        about six significant digits) */
    double last_check; /* the stopping-rule value at the last test (ratio for L2_REL) */
} lap_result;

typedef struct lap_handle_s* lap_handle;

/* Defaults: SOR w = 1.0, tol 1e-10, L2_REL, max_iter 100000, check_every 1, MG V(2,2)
 * down to coarsest side 5 with a Gauss-Seidel smoother, ADI form A, 1 inner cycle. */
void lap_default_params(lap_params* p);

/* Create a handle on CUDA device `device` whose scratch memory may grow up to
 * hbm_budget_bytes (0 = no limit beyond the device's). Returns LAP_EINVAL for a bad
 * device, LAP_ECUDA if the device cannot be made current. */
int lap_create(lap_handle* out, size_t hbm_budget_bytes, int device);

/* Free every scratch buffer and table of the handle (synchronises its device). */
void lap_destroy(lap_handle h);

/* Scratch bytes lap_solve needs for this grid and method (admission against a budget).
 * Host arithmetic: no allocation and no launch (it reads the current device's multiprocessor
 * count, 152 when there is no device). Gives the refusals lap_solve would give for the shape
 * and parameters (LAP_EINVAL, LAP_EUNSUPPORTED: the size limits above). */
int lap_workspace_bytes(const lap_grid* g, const lap_params* p, size_t* bytes);

/* Iterate p->method on psi_dev until the stopping rule (p->norm, p->tol) holds or
 * p->max_iter iterations are done; psi_dev holds the Dirichlet ring and the initial
 * interior on entry and the last iterate on return. *out (host) receives the status,
 * iteration count and norms. A non-finite norm stops the solve with LAP_DIVERGED.
 * The stopping rule is tested after iterations check_every, 2 check_every, ... and
 * after the last. Synchronises `stream` before returning. */
int lap_solve(lap_handle h, const lap_grid* g, double* psi_dev, const lap_params* p,
              lap_result* out, void* stream);

/* lap_solve on a field in host memory, end to end: psi_host (n rows of host_pitch >= m
 * doubles, row-major, i contiguous; ring and initial interior) is copied to a device field
 * that the handle owns (row pitch g->pitch doubles; allocated against the budget on first
 * use, grown when a larger grid comes, freed by lap_destroy), solved exactly as lap_solve
 * solves it (same kernels, same iterates), and the last iterate is copied back into
 * psi_host. The copies are enqueued on `stream`; pinned host memory lets them run at the
 * link's rate, pageable memory works but stages through the driver. Synchronises `stream`
 * before returning. LAP_EINVAL if psi_host is NULL, not 8-byte aligned or device memory,
 * or host_pitch < m; on an error the content of psi_host is unspecified. */
int lap_solve_host(lap_handle h, const lap_grid* g, double* psi_host, int64_t host_pitch,
                   const lap_params* p, lap_result* out, void* stream);

/* Solve `count` independent problems (grids[k], psi_devs[k], each its own size and
 * spacing) with the V-cycle: p->method LAP_MG or LAP_MG_MIXED, norm L2_REL or L2_ABS.
 * Every phase of a cycle is one launch over all problems that take part in it; each
 * problem gets exactly the arithmetic of its own lap_solve (per problem the iterates are
 * the same), stops on its own (convergence is decided on the device) and reports in
 * results[k] (host). While the launch configuration is still being chosen (below), the
 * host polls the number of problems still running every p->check_every cycles; once it is
 * chosen (and graphs are on), the remaining cycles run on the device as one conditional CUDA
 * graph that stops itself when no problem is left or p->max_iter cycles are done, and the host
 * waits once. Synchronises `stream` before returning.
 * The launch configuration -- the small-level tail size (p->tail_size), the FP32 levels'
 * temporal blocking and tile shape (p->tiling), the per-pass kernels' work-item size
 * (p->item_points) and persistent or one-CTA-per-item launches (p->persistent) -- is chosen
 * by timing where a parameter leaves it open (0): the first
 * cycles of a batch shape each run a different candidate, one knob at a time, the fastest
 * is kept in the handle for that shape. No choice changes a value.
 * The plan of a call (level descriptors, work lists, the captured cycle graphs) stays in the
 * handle: a following call with the same grids, field addresses and multigrid parameters
 * reuses it, unless another call of the handle has used its scratch memory in between. */
int lap_solve_batched(lap_handle h, int count, const lap_grid* grids, double* const* psi_devs,
                      const lap_params* p, lap_result* results, void* stream);

/* The launch configuration of the last cycle of the last lap_solve_batched call on h (no
 * counterpart in the paper; for reports): *tail_size (-1 = no tail), *tiling (-1 = one kernel
 * per pass, 1..3 = tile variant; see lap_params), *item_points, *persistent (1 = persistent
 * launches, -1 = one CTA per item), and *tuned = 1 if the choice by timing had finished for
 * that batch shape (0 while candidates were still being timed). Any pointer may be NULL. All
 * zero before the first batched solve. */
int lap_last_batch_config(lap_handle h, int32_t* tail_size, int32_t* tiling, int32_t* item_points,
                          int32_t* persistent, int32_t* tuned);

/* ---- serving: continuous batching over a stream of solve requests ----
 * A server owns a device pool of hbm_budget_bytes for the grid hierarchies of the requests it
 * runs (the fields themselves stay the caller's). lap_server_submit queues a request;
 * every lap_server_step admits queued requests first-in first-out while a running slot is
 * free (max_running) and the request's hierarchy fits the pool, then runs ONE iteration of
 * every running request as batched launches shared by all of them -- a V-cycle (p->nu1,
 * nu2, coarsest_min, max_levels, smoother_w, inner_cycles) for LAP_MG / LAP_MG_MIXED
 * requests, sor_sweeps red-black sweeps with the request's own w for LAP_SOR_RB -- and
 * tests each request's own stopping rule (L2 residual relative to its initial one <= its
 * tol) on the device. Finished requests leave and free their memory; requests that arrive
 * meanwhile join at the next step. Per request the arithmetic is that of lap_solve (SOR
 * with check_every = sor_sweeps), so results do not depend on what else is running.
 * lap_server_step synchronises `stream`; the caller must not touch a request's field
 * until lap_server_poll has returned 1 for it. A server is not thread-safe. */
typedef struct lap_server_s* lap_server;
int lap_server_create(lap_server* out, lap_handle h, size_t hbm_budget_bytes, const lap_params* p,
                      int max_running, int sor_sweeps);
void lap_server_destroy(lap_server s);
/* method: LAP_MG, LAP_MG_MIXED or LAP_SOR_RB; max_iter counts V-cycles, or sweeps for SOR
 * (an SOR request's last step sweeps only up to max_iter, as lap_solve's last check period
 * stops there; max_iter = 0 returns the initial residual, the field untouched).
 * LAP_ENOMEM if the request's hierarchy exceeds the whole pool. *id identifies it. */
int lap_server_submit(lap_server s, const lap_grid* g, double* psi_dev, int method, double w,
                      double tol, int64_t max_iter, int64_t* id);
/* *running / *queued (nullable): requests still running after the step / still queued. */
int lap_server_step(lap_server s, void* stream, int* running, int* queued);
/* 1 and *out filled if request id has finished (the request is then forgotten), 0 if not,
 * LAP_EINVAL for an unknown id. */
int lap_server_poll(lap_server s, int64_t id, lap_result* out);
/* The requests that have finished, oldest step first (within a step by id): up to capacity of
 * them are written to ids[] and results[] (host arrays) and forgotten; *count receives how
 * many. Each step reads the device-written list of the requests its convergence tests retired
 * (one copy per step), so draining costs no per-request query. Requests already taken by
 * lap_server_poll are skipped. */
int lap_server_drain(lap_server s, int64_t* ids, lap_result* results, int capacity, int* count);

/* ||r||_2 over interior nodes of the scaled residual of Eqs. 11-12,
 * r = fma(-d, psi, fma(beta^2, N + S, E + W) [+ q]), written to *out (host).
 * q_dev may be NULL (Laplace) or a field with the same pitch (coarse-level source). */
int lap_residual(lap_handle h, const lap_grid* g, const double* psi_dev, const double* q_dev,
                 double* out, void* stream);

/* nsweeps red-black sweeps in place (Eq. 6 when w == 1, Eq. 7 otherwise) of
 * (E+W) + beta^2 (N+S) - d psi + q = 0: red points then black points each sweep,
 *   g = (fma(beta^2, N + S, E + W) [+ q]) * (1/d);  psi = w == 1 ? g : fma(w, g, (1-w) psi).
 * q_dev may be NULL. This is the multigrid smoother (V-cycle steps 1, 4, 9, 11). */
int lap_smooth(const lap_grid* g, double* psi_dev, const double* q_dev, double w, int nsweeps,
               void* stream);

/* One Jacobi sweep (Eq. 5) from in_dev to out_dev (distinct buffers, same pitch; the ring
 * is copied): out = fma(beta^2, N + S, E + W) * (1/d). */
int lap_jacobi_sweep(const lap_grid* g, const double* in_dev, double* out_dev, void* stream);

/* V-cycle steps 2-3 (and 5-6): scaled residual of the fine level, restricted by full
 * weighting to the coarse level and scaled to its equation:
 *   qc(I,J) = 0.25 * ((4 r(2I,2J) + 2 ((r_W + r_E) + (r_S + r_N))) + ((r_SW + r_SE) + (r_NW + r_NE)))
 * with r as in lap_residual. Also zeroes the coarse correction ec (initial guess of steps
 * 4 and 7) when ec_dev is non-NULL. Needs (m-1), (n-1) even; the coarse grid is
 * ((m-1)/2+1) x ((n-1)/2+1) with pitch pitch_c. r_dev is a fine-size scratch field. */
int lap_restrict(const lap_grid* fine, const double* u_dev, const double* q_dev, double* r_dev,
                 double* qc_dev, double* ec_dev, int64_t pitch_c, void* stream);

/* V-cycle steps 8 and 10: u += bilinear interpolation of the coarse correction ec
 * (copy at coincident nodes, 0.5 * (a + b) on edges, 0.25 * ((a + b) + (c + d)) at
 * centres; ec's ring is read as given, zero in a V-cycle). */
int lap_prolong_add(const lap_grid* fine, double* u_dev, const double* ec_dev, int64_t pitch_c,
                    void* stream);

/* V-cycle step 7 solved exactly: u's interior := solution of (E+W) + beta^2 (N+S) - d u + q = 0
 * with u's ring as Dirichlet data. At most 1024 interior unknowns (LAP_EUNSUPPORTED beyond). */
int lap_coarse_solve(lap_handle h, const lap_grid* g, double* u_dev, const double* q_dev,
                     void* stream);

/* One zebra half-sweep of line relaxation (Eqs. 8-10): direction 0 solves every x-line
 * (row j; odd j first, then even j), direction 1 every y-line (column i; odd i first).
 * A line system is solved exactly (chunked recurrences with a cyclic-reduction solve of
 * the chunk separators); form A relaxes afterwards, form B inside the system. Only
 * enqueues. The x-line kernel's rows of the second colour wait on flags set by the first
 * colour's rows (bounded waits); a wait that gives up, which nothing but a stalled device
 * can cause, makes the next synchronising call on the handle (lap_solve, lap_residual)
 * return LAP_ECUDA. */
int lap_line_sweep(lap_handle h, const lap_grid* g, double* psi_dev, double w, int form,
                   int direction, void* stream);

/* Residual norm that allocates nothing. The paper has no counterpart: this entry point
 * exists for callers that cannot make a device allocation -- their device memory is fully
 * reserved by another allocator or budget, they cannot afford the synchronisation that
 * cudaMalloc/cudaFree imply, or they hold no lap_handle.
 * Computes the same ||r||_2 as lap_residual (same kernels, same summation order) and
 * writes it to *out_dev, one double of device memory; nothing is returned to the host
 * and the call only enqueues work on `stream` (read *out_dev after synchronising).
 * psi_dev, q_dev (may be NULL) and out_dev must live on the current device.
 * Scratch: a fixed device array of 1218 doubles (~9.5 KB) inside the library, present on
 * every device that loads it until the process exits: 1216 partial sums and the final
 * pair. The residual kernel writes 6 partial sums per multiprocessor at most, whatever
 * the grid (912 on a 152-SM GB300); on a device that would need more than 1216 the call
 * fails with LAP_EUNSUPPORTED. The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress), so make that first call before any stream capture. Every call
 * on a device shares the array and overwrites it: calls whose work overlaps on the GPU
 * (different streams or threads without ordering) race and must be serialised. */
int lap_residual_noalloc(const lap_grid* g, const double* psi_dev, const double* q_dev,
                         double* out_dev, void* stream);

/* Measurement aid (no counterpart in the paper): the FP64 fused multiply-add issue rate of
 * the handle's device, *fma_per_s (host) = fmas per second, measured by a kernel whose
 * threads run independent fma chains on register operands, timed with CUDA events on the
 * legacy default stream (one warm-up launch, one timed launch, ~20 ms). Every FP64 kernel
 * of this library issues its adds and multiplies as fmas, so this is the peak their
 * operation counts are compared against. Synchronises the device's default stream. */
int lap_fp64_rate(lap_handle h, double* fma_per_s);

/* Enable (default) or disable CUDA-graph replay in lap_solve. With graphs, the
 * iterations between two stopping tests are captured once per handle (keyed by the field,
 * sizes and parameters) and replayed as one graph launch; the kernels and results are
 * the same either way. */
int lap_set_graphs(lap_handle h, int enabled);

/* Self-check (no counterpart in the paper): the kernels replace three FP64-pipe operations
 * by integer-pipe bit manipulation that is bit-identical by construction -- rounding the
 * FP64 residual to FP32, widening the FP32 correction to FP64, and multiplying by 1/d when
 * 1/d is 2^-k. This compares each with the instruction it replaces on `count` values drawn
 * from `seed` (random bits, FP32-range edges, exact ties, all-ones fractions, zeros and
 * subnormals, exponents at most a few above zero; k = 1..4) and returns the number of
 * differences (0 expected; two NaNs count as equal) in *mismatches. Synchronises the
 * device. */
int lap_check_rounding(lap_handle h, int64_t count, uint64_t seed, int64_t* mismatches);

/* Human-readable name of a return code, and the message of the last error on this thread. */
const char* lap_strerror(int code);
const char* lap_last_error(void);

/* Number of kernels this library has launched in this process (for launch accounting). */
int64_t lap_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* LAPLACE_H */
