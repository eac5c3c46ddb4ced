// line_kernels.cu -- zebra line relaxation (SLOR / ADI half sweeps, Eqs. 8-10).
//
// Every line of one zebra colour is an independent tridiagonal system with constant
// coefficients, -alpha x_{k-1} + delta x_k - alpha x_{k+1} = b_k (k = 1..N). The kernels solve
// it scaled: with nb_k the sum of the two neighbouring lines' values, the right-hand side is
//   form A (Eqs. 8-9):  b~_k = nb_k                       and  x = cross x~,
//   form B (Eq. 10):    b~_k = fma(c1, psi_k, nb_k)       and  x = w cross x~,
// c1 = d (1 - w) / (w cross), the Dirichlet ends adding (off / cross) psi_end to b~_1 and b~_N
// (off, cross: the along-line and across-line coefficients, 1 and beta^2 for x-lines). The line
// is cut into P <= 32 chunks of L unknowns (the last holds Ll), each but the last followed by
// one separator unknown. Per chunk, with den_q the Thomas pivots of the zero-end chunk matrix
// and e_q = alpha / den_q:
//   forward    G_q = fma(e_{q-1}, G_{q-1}, b~_q)             (G_q = den_q y'_q, unnormalised)
//   separators  the chunks' zero-end solutions end in y_last = G_{L-1} / den_{L-1} and start in
//              y_first = sum_q (T^-1)_{0q} b~_q; with them the separators satisfy a small
//              tridiagonal system, solved exactly by parallel cyclic reduction over one warp;
//   back       Z_q = fma(e_{q+1}, Z_{q+1}, G_q + xl F_q),  Z_{L-1} = G_{L-1} + xl F_{L-1} + alpha xr
//              (Z_q = den_q x~_q; xl, xr the separators around the chunk; F_q the forward
//              elimination of alpha at the chunk's left end),
//   output     form A: psi = fma(sc_q, Z_q, (1 - w) psi),  form B: psi = sc_q Z_q,
//              sc_q = w cross / den_q (w cross for a separator).
// (T^-1)_{0q} and F_q decay geometrically away from the chunk's left end; from the position K0
// on, where both are below 2^-64 of their first value, their terms are left out. Per unknown
// this is 5 FP64 operations (1 add + 0-1 fma for b~, 1 forward, 1 back, 1-2 for the output)
// plus 2 within K0 of a chunk's start. All tables depend on the line length and coefficients
// only and are computed once on the host.
//
// x-lines (rows, contiguous): a CTA works on one line at a time; b~ is built into shared memory
// with coalesced loads, one warp runs the chunk recurrences (lane = chunk) and the separator
// solve (lane = separator, register shuffles), and the CTA writes the line back coalesced. The
// CTAs stay resident and take the lines of both zebra colours in order from a counter, so a
// half sweep is one launch (line_x_kernel). On GB300 each of
// an SM's four schedulers has its own FP64 unit (0.5 fma per clock; measured), and one warp's
// dependent fma chain alone keeps it busy, so the six line CTAs that fit an SM's shared memory
// are enough recurrence warps; the CTA's other warps shorten the load and store phases.
// y-lines (columns, strided by the pitch): lane = line (32 adjacent lines of a colour, so every
// row access is a contiguous 512-byte run), one thread per (line, chunk); three launches per
// colour -- forward (G to a scratch array laid out [position][line]), separators (a warp per
// line), back -- so that no transposed copy of the field is needed. (The same kernels serve
// x-lines with the strides swapped, but their lanes then read 32 rows apart and ran 20-70%
// slower than the shared-memory kernel.)
#include "lap_device.cuh"
#include "lap_internal.cuh"

namespace lap {

namespace {

constexpr unsigned FULL = 0xffffffffu;
// x-lines: threads of the CTA that builds and writes a line (measured at 4097^2: 128, 160,
// 224, 256, 288, 320 threads gave 288, 285, 269, 266, 262, 255 us per form-A half sweep, the
// form-B ones 293, 282, 258, 265, 242, 272 us), the unrolling of its load and store loops,
// and the positions per batch of the chunk recurrences
constexpr int LX_THREADS = 256;
constexpr int LX_UNROLL = 8;
constexpr int XB = 8;
constexpr int LY_WARPS = 2;      // y-lines: chunk warps per CTA of the forward and back kernels
constexpr int LS_WARPS = 4;      // y-lines: lines (warps) per CTA of the separator kernel

// Parallel cyclic reduction of the separators of one line, lane p holding separator p < S:
// returns x~ of separator p (0 for lanes p >= S).
__device__ __forceinline__ double separator_solve(const LineTables& t, int p, int S, double rho)
{
    double r = p < S ? rho : 0.0;
    for (int lev = 0, s = 1; lev < t.levels; ++lev, s <<= 1) {
        const double up = __shfl_up_sync(FULL, r, s);
        const double dn = __shfl_down_sync(FULL, r, s);
        double v = r;
        if (p < S && p >= s) v = __fma_rn(t.k1[lev * t.maxp + p], up, v);
        if (p + s < S) v = __fma_rn(t.k2[lev * t.maxp + p], dn, v);
        r = v;
    }
    return p < S ? r * t.invb[p] : 0.0;
}

// ---- x-lines --------------------------------------------------------------------------
// x-lines are cut into up to LINE_MAX_CHUNKS_X = 64 chunks, run by the CTA's first two warps
// (thread p = chunk p): the recurrences, the serial part of a line, take half the steps of a
// 32-chunk cut on two schedulers, for about a tenth more FP64 operations (the chunks' boundary
// layers cover a larger share of the shorter chunks). Values passed between neighbouring
// chunks go through ex[] in shared memory, ordered by a 64-thread barrier.
__device__ __forceinline__ void bar_chunks() { asm volatile("bar.sync 1, 64;" ::: "memory"); }

// separator_solve across the two warps: level by level, each separator's value through ex[].
__device__ __forceinline__ double separator_solve_x(const LineTables& t, int p, int S, double rho,
                                                   double* ex)
{
    double r = p < S ? rho : 0.0;
    for (int lev = 0, s = 1; lev < t.levels; ++lev, s <<= 1) {
        ex[p] = r;
        bar_chunks();
        const double up = p >= s ? ex[p - s] : 0.0;
        const double dn = p + s < LINE_MAX_CHUNKS_X ? ex[p + s] : 0.0;
        bar_chunks();
        double v = r;
        if (p < S && p >= s) v = __fma_rn(t.k1[lev * t.maxp + p], up, v);
        if (p + s < S) v = __fma_rn(t.k2[lev * t.maxp + p], dn, v);
        r = v;
    }
    return p < S ? r * t.invb[p] : 0.0;
}

// The recurrences of one line held in shared memory in chunk layout (chunk p at sm[p * Ls],
// its separator at sm[p * Ls + L]), thread p = chunk p (p < 64): b~ in, the output values' Z
// (chunk positions) and x~ (separators) out. ex: 64 doubles of shared memory.
__device__ __forceinline__ void line_recurrences(const FmaOps& o, const LineTables& t,
                                                 double* sm, int p, double* ex)
{
    const int L = t.L, P = t.P, Ls = t.stride, K0 = t.K0;
    {
        const int S = P - 1;
        const bool act = p < P;
        const int len = p == P - 1 ? t.Ll : L;
        double* y = sm + p * Ls;
        const double* __restrict__ gl = p == P - 1 ? t.glnl : t.gln;
        const double alpha = in_reg(o, t.alpha);
        double G = 0.0, D = 0.0;
        if (act) {
            const int kb = min(len, K0);
            G = y[0];
            D = fmul(o, gl[0], G);
            int q = 1;
            for (; q < kb; ++q) {
                const double b = y[q];
                D = __fma_rn(gl[q], b, D);
                G = __fma_rn(t.e[q - 1], G, b);
                y[q] = G;
            }
            // the bulk in batches: operands of XB positions loaded before the chain uses them
            for (; q + XB <= len; q += XB) {
                double bv[XB], ev[XB];
#pragma unroll
                for (int u = 0; u < XB; ++u) {
                    bv[u] = y[q + u];
                    ev[u] = t.e[q + u - 1];
                }
#pragma unroll
                for (int u = 0; u < XB; ++u) {
                    G = __fma_rn(ev[u], G, bv[u]);
                    y[q + u] = G;
                }
            }
            for (; q < len; ++q) {
                G = __fma_rn(t.e[q - 1], G, y[q]);
                y[q] = G;
            }
        }
        const double ylast = act ? fmul(o, t.inv_den[len - 1], G) : 0.0;
        ex[p] = D;
        bar_chunks();
        const double yfirst_next = p + 1 < LINE_MAX_CHUNKS_X ? ex[p + 1] : 0.0;
        bar_chunks();
        double rho = 0.0;
        if (p < S) rho = __fma_rn(alpha, fadd(o, ylast, yfirst_next), y[L]);
        const double xs = separator_solve_x(t, p, S, rho, ex);
        ex[p] = xs;
        bar_chunks();
        const double xl_ = p > 0 ? ex[p - 1] : 0.0;
        if (act) {
            const double xl = p > 0 ? xl_ : 0.0;
            const double xr = p < S ? xs : 0.0;
            int q = len - 1;
            double Gq = y[q];
            if (q < K0) Gq = __fma_rn(xl, t.F[q], Gq);
            double Z = __fma_rn(alpha, xr, Gq);
            y[q] = Z;
            --q;
            for (; q - XB + 1 >= K0; q -= XB) {
                double gv[XB], ev[XB];
#pragma unroll
                for (int u = 0; u < XB; ++u) {
                    gv[u] = y[q - u];
                    ev[u] = t.e[q - u + 1];
                }
#pragma unroll
                for (int u = 0; u < XB; ++u) {
                    Z = __fma_rn(ev[u], Z, gv[u]);
                    y[q - u] = Z;
                }
            }
            for (; q >= K0; --q) {
                Z = __fma_rn(t.e[q + 1], Z, y[q]);
                y[q] = Z;
            }
            for (; q >= 0; --q) {
                Z = __fma_rn(t.e[q + 1], Z, __fma_rn(xl, t.F[q], y[q]));
                y[q] = Z;
            }
            if (p < S) y[L] = xs;
        }
    }
}

// Phase 1 of an x-line: b~ of the row into shared memory in chunk layout, by threads tid =
// 0..nthr-1 (coalesced); each thread also adds the Dirichlet end terms of the entries it wrote.
// Loads go to L2 (ld.global.cg): rows of the first colour are written by other CTAs of the same
// launch, and L1 is not coherent between SMs.
template <int FORM>
__device__ __forceinline__ void line_x_load(const FmaOps& o, const LineTables& t, double* sm,
                                            const double* row, int64_t pitch, double bnd, double c1,
                                            int tid, int nthr)
{
    const int N = t.N, L = t.L, Ls = t.stride;
    const double* up = row - pitch;
    const double* dn = row + pitch;
#pragma unroll LX_UNROLL
    for (int k = 1 + tid; k <= N; k += nthr) {
        const double nb = fadd(o, __ldcg(up + k), __ldcg(dn + k));
        const double b = FORM == 1 ? __fma_rn(c1, __ldcg(row + k), nb) : nb;
        const int g = k - 1, p = g / (L + 1);
        sm[p * Ls + (g - p * (L + 1))] = b;
    }
    if (tid == 0) sm[0] = __fma_rn(bnd, __ldcg(row), sm[0]);
    if (tid == (N - 1) % nthr) {
        const int g = N - 1, p = g / (L + 1);
        double* e = sm + p * Ls + (g - p * (L + 1));
        *e = __fma_rn(bnd, __ldcg(row + N + 1), *e);
    }
}

// Phase 3 of an x-line: the output values written to the row (coalesced), by the same
// thread-to-element mapping as line_x_load.
template <int FORM>
__device__ __forceinline__ void line_x_store(const FmaOps& o, const LineTables& t, const double* sm,
                                             double* row, double omw, int tid, int nthr)
{
    const int N = t.N, L = t.L, Ls = t.stride;
#pragma unroll LX_UNROLL
    for (int k = 1 + tid; k <= N; k += nthr) {
        const int g = k - 1, p = g / (L + 1), q = g - p * (L + 1);
        const double v = sm[p * Ls + q];
        if (FORM == 0)
            row[k] = __fma_rn(t.sc[q], v, fmul(o, omw, __ldcg(row + k)));
        else
            row[k] = fmul(o, t.sc[q], v);
    }
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Wait until *flag != 0, at most LX_SPIN_LIMIT polls (seconds); after that the error word is
// set and the caller goes on: the host reports the error, nothing hangs.
constexpr unsigned LX_SPIN_LIMIT = 1u << 24;
__device__ __forceinline__ void wait_flag(const unsigned* flag, unsigned* err)
{
    for (unsigned it = 0; it < LX_SPIN_LIMIT; ++it) {
        if (ld_acquire(flag) != 0u) return;
        __nanosleep(128);
    }
    atomicExch(err, 1u);
}

// A whole x-line half sweep (both zebra colours) in one launch of resident CTAs. Work item
// i < nodd is row 1 + 2i (first colour), item nodd + i is row 2 + 2i (second colour); a CTA
// claims items from a counter in that order and runs the three phases on each, separated by
// CTA barriers. A second-colour row needs its two first-colour neighbours finished: they were
// claimed a colour earlier by CTAs that are running, so the wait ends (almost always at once).
// A first-colour row is published by a release store of its flag after the CTA's barrier.
// Against one launch per colour this removes the second launch's wait for the first's last
// CTAs (2048 lines on 912 CTA slots at 4097^2 left a third of the last wave idle) and lets
// CTAs at different phases overlap. sync: [0] error word (kept until the host reads it),
// [1] item counter, [2 + r] flag of row r; [1 ..] zeroed before each launch.
template <int FORM>
__global__ void __launch_bounds__(LX_THREADS, 6)
    line_x_kernel(double* __restrict__ psi, int64_t pitch, int nlines, const LineTables t,
                  double bnd, double c1, double omw, unsigned* __restrict__ sync)
{
    const FmaOps o = load_fma_ops();
    extern __shared__ double sm[];
    __shared__ int s_item;
    __shared__ double ex[LINE_MAX_CHUNKS_X];
    const int nodd = (nlines + 1) / 2;
    c1 = in_reg(o, c1);
    omw = in_reg(o, omw);
    unsigned* const done = sync + 2;
    for (;;) {
        if (threadIdx.x == 0) {
            const int item = (int)atomicAdd(sync + 1, 1u);
            if (item >= nodd && item < nlines) {
                const int r = 2 + 2 * (item - nodd);
                wait_flag(done + r - 1, sync);
                if (r + 1 <= nlines) wait_flag(done + r + 1, sync);
            }
            s_item = item;
        }
        __syncthreads();
        const int item = s_item;
        if (item >= nlines) return;
        const int r = item < nodd ? 1 + 2 * item : 2 + 2 * (item - nodd);
        double* row = psi + (int64_t)r * pitch;
        line_x_load<FORM>(o, t, sm, row, pitch, bnd, c1, threadIdx.x, LX_THREADS);
        __syncthreads();
        if (threadIdx.x < LINE_MAX_CHUNKS_X) line_recurrences(o, t, sm, threadIdx.x, ex);
        __syncthreads();
        line_x_store<FORM>(o, t, sm, row, omw, threadIdx.x, LX_THREADS);
        __syncthreads();
        if (threadIdx.x == 0 && item < nodd) {
            __threadfence();
            st_release(done + r, 1u);
        }
    }
}

// ---- lines through a scratch array: lane = line --------------------------------------
// Thread (line l = first + 2 * (32 * blockIdx.x + lane), chunk c = LY_WARPS * blockIdx.y +
// warp); element k of line l at psi + l * sx + k * sa, its neighbouring lines at +-sx
// (y-lines: sa = pitch, sx = 1, so a warp's 32 lines read one contiguous run of a row;
// x-lines: sa = 1, sx = pitch). G[(k - 1) * gp + lane index], coalesced either way. The
// loops are software-pipelined: the loads of the next PIPE positions are issued before the
// current ones are used.
constexpr int PIPE = 8;  // 16 was slower (registers), and L2 evict-last hints on G gained nothing

template <int FORM>
__global__ void __launch_bounds__(32 * LY_WARPS)
    line_forward_kernel(const double* __restrict__ psi, int64_t sa, int64_t sx, int first_line,
                        int count, const LineTables t, double bnd, double c1, double* __restrict__ G,
                        int64_t gp, double* __restrict__ ylast, double* __restrict__ yfirst)
{
    const FmaOps o = load_fma_ops();
    const int li = blockIdx.x * 32 + (threadIdx.x & 31);
    const int c = blockIdx.y * LY_WARPS + (threadIdx.x >> 5);
    if (li >= count || c >= t.P) return;
    const int L = t.L, len = c == t.P - 1 ? t.Ll : L, K0 = t.K0;
    const int k0 = 1 + c * (L + 1);
    const double* __restrict__ line = psi + (int64_t)(first_line + 2 * li) * sx;
    double* __restrict__ g = G + li + (int64_t)(k0 - 1) * gp;
    const double* __restrict__ gl = c == t.P - 1 ? t.glnl : t.gln;
    c1 = in_reg(o, c1);

    // right-hand side of chunk position q (loads only; the adds come with the recurrence)
    double ra[PIPE], rb[PIPE], rc[PIPE];
    auto load = [&](int q0, double* a, double* b_, double* cc) {
#pragma unroll
        for (int u = 0; u < PIPE; ++u)
            if (q0 + u < len) {
                const double* at = line + (int64_t)(k0 + q0 + u) * sa;
                a[u] = at[-sx];
                b_[u] = at[sx];
                if (FORM == 1) cc[u] = at[0];
            }
    };
    // position 0 (peeled: a per-step test inside the batches would issue both sides' FP64
    // operations on every step)
    double b0;
    {
        const double* at = line + (int64_t)k0 * sa;
        b0 = fadd(o, at[-sx], at[sx]);
        if (FORM == 1) b0 = __fma_rn(c1, at[0], b0);
        if (c == 0) b0 = __fma_rn(bnd, line[0], b0);  // the near Dirichlet end
    }
    double G_ = b0;
    double D = fmul(o, gl[0], b0);
    g[0] = G_;
    // positions 1.., PIPE at a time; batches that reach into the boundary layer also carry the
    // y_first sum, the others only the recurrence
    auto step = [&](int q, double a_, double b_, double c_) {
        const double nbv = fadd(o, a_, b_);
        const double b = FORM == 1 ? __fma_rn(c1, c_, nbv) : nbv;
        G_ = __fma_rn(t.e[q - 1], G_, b);
        g[(int64_t)q * gp] = G_;
        return b;
    };
    load(1, ra, rb, rc);
    for (int q0 = 1; q0 < len; q0 += PIPE) {
        double na[PIPE], nb_[PIPE], nc[PIPE];
        if (q0 + PIPE < len) load(q0 + PIPE, na, nb_, nc);
        if (q0 < K0) {
#pragma unroll
            for (int u = 0; u < PIPE; ++u) {
                const int q = q0 + u;
                if (q < len) {
                    const double b = step(q, ra[u], rb[u], rc[u]);
                    if (q < K0) D = __fma_rn(gl[q], b, D);
                }
            }
        } else if (q0 + PIPE <= len) {
#pragma unroll
            for (int u = 0; u < PIPE; ++u) step(q0 + u, ra[u], rb[u], rc[u]);
        } else {
#pragma unroll
            for (int u = 0; u < PIPE; ++u)
                if (q0 + u < len) step(q0 + u, ra[u], rb[u], rc[u]);
        }
#pragma unroll
        for (int u = 0; u < PIPE; ++u) {
            ra[u] = na[u];
            rb[u] = nb_[u];
            if (FORM == 1) rc[u] = nc[u];
        }
    }
    if (c == t.P - 1) {  // the far Dirichlet end enters b~_N with coefficient 1
        const double extra = fmul(o, bnd, line[(int64_t)(t.N + 1) * sa]);
        G_ = fadd(o, G_, extra);
        g[(int64_t)(len - 1) * gp] = G_;
        if (len - 1 < K0) D = __fma_rn(gl[len - 1], extra, D);
    }
    ylast[(int64_t)c * gp + li] = fmul(o, t.inv_den[len - 1], G_);
    yfirst[(int64_t)c * gp + li] = D;
}

// One warp per line: lane p = separator p; writes the separators' solution xs and their
// output values.
template <int FORM>
__global__ void __launch_bounds__(32 * LS_WARPS)
    line_separator_kernel(double* __restrict__ psi, int64_t sa, int64_t sx, int first_line, int count,
                          const LineTables t, double c1, double omw, double wc,
                          const double* __restrict__ ylast, const double* __restrict__ yfirst,
                          double* __restrict__ xsep, int64_t gp)
{
    const FmaOps o = load_fma_ops();
    const int li = blockIdx.x * LS_WARPS + (threadIdx.x >> 5);
    if (li >= count) return;  // warp-uniform
    const int p = threadIdx.x & 31, S = t.P - 1;
    double* line = psi + (int64_t)(first_line + 2 * li) * sx;
    double* at = line + (int64_t)((p + 1) * (t.L + 1)) * sa;
    double rho = 0.0, old = 0.0;
    if (p < S) {
        const double nb = fadd(o, at[-sx], at[sx]);
        old = at[0];
        const double b = FORM == 1 ? __fma_rn(c1, old, nb) : nb;
        const double yl = ylast[(int64_t)p * gp + li], yf = yfirst[(int64_t)(p + 1) * gp + li];
        rho = __fma_rn(t.alpha, fadd(o, yl, yf), b);
    }
    const double xs = separator_solve(t, p, S, rho);
    if (p < S) {
        xsep[(int64_t)p * gp + li] = xs;
        at[0] = FORM == 0 ? __fma_rn(wc, xs, fmul(o, omw, old)) : fmul(o, wc, xs);
    }
}

template <int FORM>
__global__ void __launch_bounds__(32 * LY_WARPS)
    line_back_kernel(double* __restrict__ psi, int64_t sa, int64_t sx, int first_line, int count,
                     const LineTables t, double omw, const double* __restrict__ G, int64_t gp,
                     const double* __restrict__ xsep)
{
    const FmaOps o = load_fma_ops();
    const int li = blockIdx.x * 32 + (threadIdx.x & 31);
    const int c = blockIdx.y * LY_WARPS + (threadIdx.x >> 5);
    if (li >= count || c >= t.P) return;
    const int L = t.L, len = c == t.P - 1 ? t.Ll : L, K0 = t.K0, S = t.P - 1;
    const int k0 = 1 + c * (L + 1);
    double* __restrict__ line = psi + (int64_t)(first_line + 2 * li) * sx + (int64_t)k0 * sa;
    const double* __restrict__ g = G + li + (int64_t)(k0 - 1) * gp;
    const double xl = c > 0 ? xsep[(int64_t)(c - 1) * gp + li] : 0.0;
    const double xr = c < S ? xsep[(int64_t)c * gp + li] : 0.0;
    omw = in_reg(o, omw);
    const double alpha = in_reg(o, t.alpha);

    // positions run backwards: batch j holds q = top - u, u = 0..PIPE-1
    double gv[PIPE], ov[PIPE];
    auto load = [&](int top, double* gg, double* oo) {
#pragma unroll
        for (int u = 0; u < PIPE; ++u)
            if (top - u >= 0) {
                gg[u] = g[(int64_t)(top - u) * gp];
                if (FORM == 0) oo[u] = line[(int64_t)(top - u) * sa];
            }
    };
    // position len - 1 (peeled), then len - 2 .. 0, PIPE at a time; batches wholly past the
    // boundary layer skip its term
    auto out = [&](int q, double Z, double old) {
        double* at = line + (int64_t)q * sa;
        *at = FORM == 0 ? __fma_rn(t.sc[q], Z, fmul(o, omw, old)) : fmul(o, t.sc[q], Z);
    };
    double Z;
    {
        const int q = len - 1;
        double Gq = g[(int64_t)q * gp];
        if (q < K0) Gq = __fma_rn(xl, t.F[q], Gq);
        Z = __fma_rn(alpha, xr, Gq);
        out(q, Z, FORM == 0 ? line[(int64_t)q * sa] : 0.0);
    }
    load(len - 2, gv, ov);
    for (int top = len - 2; top >= 0; top -= PIPE) {
        double ng[PIPE], no[PIPE];
        if (top - PIPE >= 0) load(top - PIPE, ng, no);
        if (top - PIPE + 1 >= K0) {
#pragma unroll
            for (int u = 0; u < PIPE; ++u) {
                Z = __fma_rn(t.e[top - u + 1], Z, gv[u]);
                out(top - u, Z, ov[u]);
            }
        } else {
#pragma unroll
            for (int u = 0; u < PIPE; ++u) {
                const int q = top - u;
                if (q >= 0) {
                    double Gq = gv[u];
                    if (q < K0) Gq = __fma_rn(xl, t.F[q], Gq);
                    Z = __fma_rn(t.e[q + 1], Z, Gq);
                    out(q, Z, ov[u]);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < PIPE; ++u) {
            gv[u] = ng[u];
            if (FORM == 0) ov[u] = no[u];
        }
    }
}

// ---- a whole line-relaxation solve in one CTA (small grids, the paper's stopping rule) ----
// On grids of a few thousand points (the paper's 25 x 17 chamber) every launch costs more than
// the work it does. This kernel keeps the field in shared memory and runs whole check periods
// of zebra SLOR (x-lines) or ADI (x-lines then y-lines), forms A and B, until the largest
// change of an iteration, max |psi^{k+1} - psi^k| (Eq. 16), is <= tol; a thread solves one
// line at a time by the Thomas algorithm. The pivots of the constant-coefficient line matrix
// depend on its length and coefficients only: 1/den_i and alpha/den_i are tabulated once per
// solve, so a step of the elimination is an fma and a multiply (an FP64 division costs about
// ten dependent FP64 operations on this GPU).
constexpr int LC_THREADS = 256;

// Tables of one direction: inv[i] = 1 / den_i, cc[i] = coupling / den_i, den_0 = d,
// den_i = d - coupling^2 / den_{i-1}.
__device__ __forceinline__ void cta_line_tables(int len, double d, double coupling, double* inv,
                                                double* cc)
{
    double den = d;
    for (int i = 0; i < len; ++i) {
        if (i) den = d - coupling * (coupling / den);
        inv[i] = 1.0 / den;
        cc[i] = coupling / den;
    }
}

template <int FORM>
__device__ __forceinline__ void cta_relax_line(const FmaOps& o, double* u, int m, int dir, int line,
                                               int len, double cross, double c1, double w,
                                               double coupling, const double* inv, const double* cc,
                                               double* dp)
{
    // element k (0..len+1) of the line, and of its two neighbouring lines
    auto at = [&](int l, int k) -> double& { return dir == 0 ? u[l * m + k] : u[k * m + l]; };
    double prev = 0.0;
    for (int k = 1; k <= len; ++k) {
        const double nb = fadd(o, at(line - 1, k), at(line + 1, k));
        // form A: cross (P + Q); form B: d (1 - w) psi + w cross (P + Q), here as
        // (w cross) (c1 psi + P + Q) with c1 = d (1 - w) / (w cross); `cross` is w cross there
        double r = FORM == 0 ? fmul(o, cross, nb) : fmul(o, cross, __fma_rn(c1, at(line, k), nb));
        if (k == 1) r = __fma_rn(coupling, at(line, 0), r);
        if (k == len) r = __fma_rn(coupling, at(line, len + 1), r);
        prev = fmul(o, __fma_rn(coupling, prev, r), inv[k - 1]);
        dp[k - 1] = prev;
    }
    // back substitution, then the relaxed output (form A: psi + w (x - psi); form B: x)
    double x = 0.0;
    for (int i = len - 1; i >= 0; --i) {
        x = i == len - 1 ? dp[i] : __fma_rn(cc[i], x, dp[i]);
        double& p = at(line, i + 1);
        p = FORM == 0 ? __fma_rn(w, fadd(o, x, -p), p) : x;
    }
}

// One zebra half sweep in direction dir: odd lines, then even lines, each line by one thread.
template <int FORM>
__device__ __forceinline__ void cta_half_sweep(const FmaOps& o, double* u, int m, int n, int dir,
                                               double b2, double c1, double w, const double* inv,
                                               const double* cc, double* work, int wlen)
{
    const int lines = dir == 0 ? n - 2 : m - 2, len = dir == 0 ? m - 2 : n - 2;
    const double off = dir == 0 ? 1.0 : b2, cross = dir == 0 ? b2 : 1.0;
    const double coupling = FORM == 0 ? off : w * off;
    const double rcross = FORM == 0 ? cross : w * cross;
    for (int first = 1; first <= 2; ++first) {
        for (int l = first + 2 * (int)threadIdx.x; l <= lines; l += 2 * LC_THREADS)
            cta_relax_line<FORM>(o, u, m, dir, l, len, rcross, c1, w, coupling, inv, cc,
                                 work + (size_t)threadIdx.x * wlen);
        __syncthreads();
    }
}

template <bool ADI, int FORM>
__global__ void __launch_bounds__(LC_THREADS)
    solve_lines_cta_kernel(double* __restrict__ psi, int m, int n, int64_t pitch, double b2, double d,
                           const double* __restrict__ wslot, LoopState* __restrict__ st)
{
    extern __shared__ double lsm[];
    const FmaOps o = load_fma_ops();
    const int wlen = max(m, n);
    double* u = lsm;                  // the field, dense m x n
    double* prev = u + m * n;         // the field before the period's last iteration
    double* tabs = prev + m * n;      // x-line tables (inv, cc), then y-line tables
    double* work = tabs + 4 * wlen;   // forward values: wlen doubles per thread that has a line
    const double w = wslot[0];
    // form B's right-hand side factor d (1 - w) / (w cross), per direction
    const double c1x = FORM == 1 ? d * (1.0 - w) / (w * b2) : 0.0;
    const double c1y = FORM == 1 ? d * (1.0 - w) / w : 0.0;
    const int tid = threadIdx.x;
    for (int k = tid; k < m * n; k += LC_THREADS) u[k] = psi[(int64_t)(k / m) * pitch + k % m];
    if (tid == 0) cta_line_tables(m - 2, d, FORM == 0 ? 1.0 : w, tabs, tabs + wlen);
    if (tid == 32 && ADI) cta_line_tables(n - 2, d, FORM == 0 ? b2 : w * b2, tabs + 2 * wlen, tabs + 3 * wlen);
    __shared__ unsigned long long red[LC_THREADS / 32];
    __shared__ int go;
    long long k = st->k;
    const long long every = st->steps, max_iter = st->max_iter;
    const double tol = st->tol;
    double val = st->last_check;
    int status = 1;  // LAP_MAXITER
    __syncthreads();
    while (k < max_iter) {
        const long long left = every - k % every, rest = max_iter - k;
        const long long nst = left < rest ? left : rest;
        for (long long s = 0; s < nst; ++s) {
            if (s == nst - 1) {
                for (int q = tid; q < m * n; q += LC_THREADS) prev[q] = u[q];
                __syncthreads();
            }
            cta_half_sweep<FORM>(o, u, m, n, 0, b2, c1x, w, tabs, tabs + wlen, work, wlen);
            if (ADI)
                cta_half_sweep<FORM>(o, u, m, n, 1, b2, c1y, w, tabs + 2 * wlen, tabs + 3 * wlen,
                                     work, wlen);
        }
        k += nst;
        unsigned long long dl = 0;
        for (int q = tid; q < m * n; q += LC_THREADS) {
            const unsigned long long v = abs_bits(__dadd_rn(u[q], -prev[q]));
            dl = v > dl ? v : dl;
        }
        dl = warp_max_u64(dl);
        if ((tid & 31) == 0) red[tid >> 5] = dl;
        __syncthreads();
        if (tid < 32) {
            unsigned long long v = tid < LC_THREADS / 32 ? red[tid] : 0ull;
            v = warp_max_u64(v);
            if (tid == 0) {
                val = __longlong_as_double((long long)v);
                status = !isfinite(val) ? 2 : (val <= tol ? 0 : 1);
                go = status == 1;
            }
        }
        __syncthreads();
        if (!go) break;
    }
    const int mi = m - 2;
    for (int q = tid; q < mi * (n - 2); q += LC_THREADS) {
        const int i = 1 + q % mi, j = 1 + q / mi;
        psi[(int64_t)j * pitch + i] = u[j * m + i];
    }
    if (tid == 0) {
        st->k = k;
        st->status = status;
        st->last_check = val;
    }
}

}  // namespace

size_t line_smem_bytes(const LineTables& t) { return sizeof(double) * (size_t)t.P * t.stride; }

// Raise the dynamic shared-memory limit of the x-line kernels to `smem` on the current device
// (done outside stream capture; later launches only repeat it when a longer line comes).
static std::atomic<size_t> g_line_smem_set[ATTR_DEVICES];

cudaError_t prepare_line_kernels(size_t smem)
{
    const int dev = attr_slot();
    if (smem <= 48 * 1024 || (dev >= 0 && smem <= g_line_smem_set[dev].load()))
        return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(line_x_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(line_x_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
    if (e == cudaSuccess) attr_record(g_line_smem_set, dev, smem);
    return e;
}

size_t line_x_sync_words(int nlines) { return (size_t)nlines + 4; }

cudaError_t launch_line_x(double* psi, int64_t pitch, int nlines, const LineTables& t, int form,
                          const LineCoefs& k, unsigned* sync, cudaStream_t s)
{
    if (nlines <= 0) return cudaSuccess;
    const size_t smem = line_smem_bytes(t);
    cudaError_t e = prepare_line_kernels(smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, form == 0 ? line_x_kernel<0> : line_x_kernel<1>, LX_THREADS, smem);
    if (e != cudaSuccess) return e;
    const int grid = std::min(nlines, std::max(1, per_sm) * device_sms());
    e = cudaMemsetAsync(sync + 1, 0, (line_x_sync_words(nlines) - 1) * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    if (form == 0)
        line_x_kernel<0><<<grid, LX_THREADS, smem, s>>>(psi, pitch, nlines, t, k.bnd, k.c1, k.omw, sync);
    else
        line_x_kernel<1><<<grid, LX_THREADS, smem, s>>>(psi, pitch, nlines, t, k.bnd, k.c1, k.omw, sync);
    note_launch();
    return cudaGetLastError();
}

size_t line_y_scratch_doubles(const LineTables& t, int64_t gp)
{
    return (size_t)gp * ((size_t)t.N + 3 * (size_t)t.P);
}

cudaError_t launch_line_scratch(double* psi, int64_t sa, int64_t sx, int first_line, int count,
                                const LineTables& t, int form, const LineCoefs& k, double* scratch,
                                int64_t gp, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    double* G = scratch;
    double* yl = G + (size_t)gp * t.N;
    double* yf = yl + (size_t)gp * t.P;
    double* xs = yf + (size_t)gp * t.P;
    const dim3 grid((count + 31) / 32, (t.P + LY_WARPS - 1) / LY_WARPS);
    const dim3 sgrid((count + LS_WARPS - 1) / LS_WARPS);
#define LAP_LINES(F)                                                                                 \
    do {                                                                                             \
        line_forward_kernel<F><<<grid, 32 * LY_WARPS, 0, s>>>(psi, sa, sx, first_line, count, t,      \
                                                              k.bnd, k.c1, G, gp, yl, yf);           \
        note_launch();                                                                               \
        if (t.P > 1) {                                                                               \
            line_separator_kernel<F><<<sgrid, 32 * LS_WARPS, 0, s>>>(psi, sa, sx, first_line, count,  \
                                                                     t, k.c1, k.omw, k.wc, yl, yf,   \
                                                                     xs, gp);                        \
            note_launch();                                                                           \
        }                                                                                            \
        line_back_kernel<F><<<grid, 32 * LY_WARPS, 0, s>>>(psi, sa, sx, first_line, count, t, k.omw, \
                                                           G, gp, xs);                               \
        note_launch();                                                                               \
    } while (0)
    if (form == 0) LAP_LINES(0); else LAP_LINES(1);
#undef LAP_LINES
    return cudaGetLastError();
}

// the field, its copy, the two directions' tables, and forward values for as many lines as a
// colour has (at most one per thread)
size_t solve_lines_cta_smem(int m, int n)
{
    const int per_colour = std::min(LC_THREADS, std::max((n - 1) / 2, (m - 1) / 2));
    return sizeof(double) * ((size_t)2 * m * n + (size_t)(4 + per_colour) * std::max(m, n));
}

static std::atomic<size_t> g_lines_cta_smem_set[ATTR_DEVICES];

cudaError_t launch_solve_lines_cta(const Field& f, const Coef& c, bool adi, int form,
                                   const double* wslot, LoopState* st, cudaStream_t s)
{
    const size_t smem = solve_lines_cta_smem(f.m, f.n);
    const int dev = attr_slot();
    cudaError_t e = cudaSuccess;
    if (smem > 48 * 1024 && !(dev >= 0 && smem <= g_lines_cta_smem_set[dev].load())) {
        const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
        if (e == cudaSuccess) e = cudaFuncSetAttribute(solve_lines_cta_kernel<false, 0>, a, (int)smem);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(solve_lines_cta_kernel<false, 1>, a, (int)smem);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(solve_lines_cta_kernel<true, 0>, a, (int)smem);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(solve_lines_cta_kernel<true, 1>, a, (int)smem);
        if (e == cudaSuccess) attr_record(g_lines_cta_smem_set, dev, smem);
        if (e != cudaSuccess) return e;
    }
    auto kern = adi ? (form == 0 ? solve_lines_cta_kernel<true, 0> : solve_lines_cta_kernel<true, 1>)
                    : (form == 0 ? solve_lines_cta_kernel<false, 0> : solve_lines_cta_kernel<false, 1>);
    kern<<<1, LC_THREADS, smem, s>>>(f.p, f.m, f.n, f.pitch, c.b2, c.d, wslot, st);
    note_launch();
    return cudaGetLastError();
}

}  // namespace lap
