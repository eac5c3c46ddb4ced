// point_kernels.cu -- point relaxation sweeps, residual and norms for liblaplace.so.
//
// Jacobi (Eq. 5), red-black Gauss-Seidel (Eq. 6) and SOR (Eq. 7), and the scaled
// residual r = dx^2 L(psi) (+ q) of Eqs. 11-12. Every value is computed with the same
// sequence of correctly rounded operations as the written expression (adds and
// multiplies issued as exact fmas, see FmaOps; the file is built with --fmad=false), so
// results do not depend on the launch shape.
//
// On GB300 the FP64 pipe (about 2 operations per clock per SM) and not HBM bounds these
// sweeps; the kernels spend the minimum number of FP64 operations per point: 3 adds for
// the neighbour sum (one more fma when beta != 1), the multiply by 1/d on the integer
// pipe when 1/d is a power of two, and one multiply plus one fma for the SOR blend.
#include "lap_device.cuh"
#include "lap_internal.cuh"

namespace lap {

namespace {

constexpr int RB_BX = 64, RB_BY = 4;   // red-black: 64 same-colour points x 4 rows
constexpr int JA_BX = 128, JA_BY = 2;  // Jacobi: 128 points x 2 rows
constexpr int NORM_THREADS = 256;
// 6 blocks of 256 threads per SM (at most 42 registers a thread): the norm kernels' grid of
// at most 912 blocks (152 SMs) is resident at once.
constexpr int NORM_BLOCKS_PER_SM = 6;

__device__ __forceinline__ void flush_maxd(unsigned long long v, unsigned long long* maxd)
{
    v = warp_max_u64(v);
    if ((threadIdx.x & 31) == 0 && v) atomicMax(maxd, v);
}

// One colour of a red-black sweep. Thread (t, row j) updates the t-th point of colour
// `colour` in row j: i = 1 + ((1 + j + colour) & 1) + 2t, so that (i + j) % 2 == colour.
template <bool UNIT_BETA, bool POW2, bool HAS_Q, bool GS, bool MAXD>
__global__ void __launch_bounds__(RB_BX* RB_BY)
    rb_colour_kernel(double* __restrict__ psi, const double* __restrict__ q, int m, int n,
                     int64_t pitch, int colour, double b2, double inv_d, int shift, double w,
                     double one_minus_w, unsigned long long* __restrict__ maxd,
                     const double* __restrict__ wslot)
{
    const FmaOps o = load_fma_ops();
    if (!GS && wslot) {  // w and 1 - w from device memory: register operands for the blend
        w = wslot[0];
        one_minus_w = wslot[1];
    } else if (!GS) {
        w = in_reg(o, w);
        one_minus_w = in_reg(o, one_minus_w);
    }
    if (!UNIT_BETA) b2 = in_reg(o, b2);
    if (!POW2) inv_d = in_reg(o, inv_d);
    const int j = 1 + blockIdx.y * RB_BY + threadIdx.y;
    const int i = 1 + ((1 + j + colour) & 1) + 2 * (blockIdx.x * RB_BX + threadIdx.x);
    unsigned long long dl = 0;
    if (j <= n - 2 && i <= m - 2) {
        const int64_t at = (int64_t)j * pitch + i;
        double* c = psi + at;
        double s = neighbour_sum<UNIT_BETA>(o, c[-1], c[1], c[-pitch], c[pitch], b2);
        if (HAS_Q) s = fadd(o, s, q[at]);
        const double g = times_inv_d<POW2>(o, s, inv_d, shift);
        const double old = *c;
        const double nv = GS ? g : __fma_rn(w, g, fmul(o, one_minus_w, old));
        *c = nv;
        if (MAXD) dl = abs_bits(fadd(o, nv, -old));
    }
    if (MAXD) flush_maxd(dl, maxd);
}

// One colour of a red-black sweep with the neighbour sum paired along diagonals (beta = 1):
// s = (W + S) + (E + N). A diagonal i - j = const holds points of one colour, and the pair
// E + N of point (i, j) is the pair W + S of point (i + 1, j + 1): the same two values, and
// a + b == b + a in IEEE arithmetic. A thread walks RD_K points down one diagonal and carries
// the pair, so the neighbour sum costs two FP64 adds instead of three: 4 FP64 operations per SOR
// update, 2 per Gauss-Seidel update (the multiply by 1/4 on the integer pipe). Every point gets
// the value of the same expression whatever the launch shape (the pair is computed afresh as
// W + S at the start of a walk). The rounding differs from the paper-order sum
// (E + W) + (N + S) in the last bits.
// Strip s of rows j0 = 1 + s RD_K .. j0 + RD_K - 1: walk x of the strip starts on row j0 at
// column lo + 2x, lo the first column >= 2 - RD_K of the colour, and visits (lo + 2x + k,
// j0 + k). Thread g of the launch takes walk g % starts of strip g / starts (no CTA is left
// nearly empty at the end of a strip). Walks of RD_K = 6 points in CTAs of RD_BX = 128
// threads: measured per colour pass inside the solve's graphs at 4097^2, (walk, CTA) =
// (4, 128) 63.2 us, (6, 128) 62.9, (8, 128) 64.7, (8, 256) 68.3, (16, 128) 66.0 with the
// loads one point ahead and 73.4 for walks of 32 (a longer walk adds registers, a shorter one
// pair adds), against 71.0 us for the paper-order kernel. Within a walk, taking every pair sum
// first or every (1 - w) C product first gave 63.1 and 62.9 us against 62.7 for the order
// below (a pair, then its point).

template <bool HAS_Q, bool GS, bool MAXD>
__global__ void __launch_bounds__(RD_BX)
    rb_diag_kernel(double* __restrict__ psi, const double* __restrict__ q, int m, int n,
                   int64_t pitch, int colour, int starts, double w, double one_minus_w,
                   unsigned long long* __restrict__ maxd, const double* __restrict__ wslot)
{
    const FmaOps o = load_fma_ops();
    if (!GS && wslot) {
        w = wslot[0];
        one_minus_w = wslot[1];
    } else if (!GS) {
        w = in_reg(o, w);
        one_minus_w = in_reg(o, one_minus_w);
    }
    const int g = blockIdx.x * RD_BX + threadIdx.x;
    const int strip = g / starts;
    const int j0 = 1 + strip * RD_K;
    const int lo0 = 2 - RD_K;
    const int lo = lo0 + ((lo0 + j0 + colour) & 1);
    const int is = lo + 2 * (g - strip * starts);
    // the walk's points inside the interior: k0 .. k1
    const int k0 = max(0, 1 - is);
    const int k1 = min(RD_K - 1, min(m - 2 - is, n - 2 - j0));
    unsigned long long dl = 0;
    if (k0 == 0 && k1 == RD_K - 1) {
        // a whole walk inside the interior: every operand of its RD_K points loaded before any
        // point is written (none of them is written by this pass but the walk's own centres,
        // each read before its own store), so the loads are in flight together
        const int64_t step = pitch + 1;
        const int64_t a0 = (int64_t)j0 * pitch + is;
        double E[RD_K], N[RD_K], C[RD_K], Q[RD_K];
        const double pSW0 = fadd(o, psi[a0 - 1], psi[a0 - pitch]);
#pragma unroll
        for (int k = 0; k < RD_K; ++k) {
            const int64_t a = a0 + k * step;
            E[k] = psi[a + 1];
            N[k] = psi[a + pitch];
            C[k] = psi[a];
            Q[k] = HAS_Q ? q[a] : 0.0;
        }
        double pSW = pSW0;
#pragma unroll
        for (int k = 0; k < RD_K; ++k) {
            const double pNE = fadd(o, E[k], N[k]);
            double s = fadd(o, pSW, pNE);
            if (HAS_Q) s = fadd(o, s, Q[k]);
            const double g = times_inv_d<true>(o, s, 0.25, 2);
            const double nv = GS ? g : __fma_rn(w, g, fmul(o, one_minus_w, C[k]));
            psi[a0 + k * step] = nv;
            if (MAXD) {
                const unsigned long long v = abs_bits(fadd(o, nv, -C[k]));
                dl = v > dl ? v : dl;
            }
            pSW = pNE;
        }
    } else if (k0 <= k1) {
        const int64_t step = pitch + 1;
        int64_t at = (int64_t)(j0 + k0) * pitch + (is + k0);
        double pSW = fadd(o, psi[at - 1], psi[at - pitch]);
        double E = psi[at + 1], N = psi[at + pitch], C = psi[at], Q = HAS_Q ? q[at] : 0.0;
        for (int k = k0; k <= k1; ++k) {
            // the next point's operands first: none of them is the point this step writes
            double En = 0.0, Nn = 0.0, Cn = 0.0, Qn = 0.0;
            if (k < k1) {
                const int64_t nx = at + step;
                En = psi[nx + 1];
                Nn = psi[nx + pitch];
                Cn = psi[nx];
                if (HAS_Q) Qn = q[nx];
            }
            const double pNE = fadd(o, E, N);
            double s = fadd(o, pSW, pNE);
            if (HAS_Q) s = fadd(o, s, Q);
            const double g = times_inv_d<true>(o, s, 0.25, 2);
            const double nv = GS ? g : __fma_rn(w, g, fmul(o, one_minus_w, C));
            psi[at] = nv;
            if (MAXD) {
                const unsigned long long v = abs_bits(fadd(o, nv, -C));
                dl = v > dl ? v : dl;
            }
            pSW = pNE;
            at += step;
            E = En;
            N = Nn;
            C = Cn;
            Q = Qn;
        }
    }
    if (MAXD) flush_maxd(dl, maxd);
}

template <bool UNIT_BETA, bool POW2, bool MAXD>
__global__ void __launch_bounds__(JA_BX* JA_BY)
    jacobi_kernel(const double* __restrict__ in, double* __restrict__ out, int m, int n,
                  int64_t pitch, double b2, double inv_d, int shift,
                  unsigned long long* __restrict__ maxd)
{
    const FmaOps o = load_fma_ops();
    if (!UNIT_BETA) b2 = in_reg(o, b2);
    if (!POW2) inv_d = in_reg(o, inv_d);
    const int j = 1 + blockIdx.y * JA_BY + threadIdx.y;
    const int i = 1 + blockIdx.x * JA_BX + threadIdx.x;
    unsigned long long dl = 0;
    if (j <= n - 2 && i <= m - 2) {
        const int64_t at = (int64_t)j * pitch + i;
        const double* c = in + at;
        const double s = neighbour_sum<UNIT_BETA>(o, c[-1], c[1], c[-pitch], c[pitch], b2);
        const double nv = times_inv_d<POW2>(o, s, inv_d, shift);
        out[at] = nv;
        if (MAXD) dl = abs_bits(fadd(o, nv, -*c));
    }
    if (MAXD) flush_maxd(dl, maxd);
}

// The scaled defect of Eq. 11 from loaded stencil values (q: the source term when HAS_Q).
template <bool UNIT_BETA, bool HAS_Q>
__device__ __forceinline__ double defect5(const FmaOps& o, const Stencil5& x, double q,
                                          double b2, double d)
{
    double s = neighbour_sum<UNIT_BETA>(o, x.w, x.e, x.s, x.n, b2);
    if (HAS_Q) s = fadd(o, s, q);
    return __fma_rn(-d, x.c, s);
}

template <bool UNIT_BETA, bool HAS_Q>
__device__ __forceinline__ double defect_at(const FmaOps& o, const double* __restrict__ u,
                                            const double* __restrict__ q, int64_t at,
                                            int64_t pitch, double b2, double d)
{
    const double* c = u + at;
    double s = neighbour_sum<UNIT_BETA>(o, c[-1], c[1], c[-pitch], c[pitch], b2);
    if (HAS_Q) s = fadd(o, s, q[at]);
    return __fma_rn(-d, *c, s);
}

template <bool UNIT_BETA, bool HAS_Q>
__global__ void __launch_bounds__(JA_BX* JA_BY)
    defect_kernel(const double* __restrict__ u, const double* __restrict__ q,
                  double* __restrict__ r, int m, int n, int64_t pitch, double b2, double d)
{
    const FmaOps o = load_fma_ops();
    if (!UNIT_BETA) b2 = in_reg(o, b2);
    d = in_reg(o, d);
    const int j = 1 + blockIdx.y * JA_BY + threadIdx.y;
    const int i = 1 + blockIdx.x * JA_BX + threadIdx.x;
    if (j <= n - 2 && i <= m - 2) {
        const int64_t at = (int64_t)j * pitch + i;
        r[at] = defect_at<UNIT_BETA, HAS_Q>(o, u, q, at, pitch, b2, d);
    }
}

// Sum of r^2 over the interior (a grid-stride walk, two points per step, summed in walk order);
// the per-block partial is reduced in a fixed order, so the result depends only on (m, n).
template <bool UNIT_BETA, bool HAS_Q>
__global__ void __launch_bounds__(NORM_THREADS, NORM_BLOCKS_PER_SM)
    defect_sumsq_kernel(const double* __restrict__ u, const double* __restrict__ q, int m, int n,
                        int64_t pitch, double b2, double d, double* __restrict__ partials)
{
    const FmaOps o = load_fma_ops();
    if (!UNIT_BETA) b2 = in_reg(o, b2);
    d = in_reg(o, d);
    double acc = 0.0;
    StrideWalk<NORM_THREADS> p(m, n);
    while (p.left >= 2) {
        const int64_t a0 = (int64_t)p.j * pitch + p.i;
        p.next();
        const int64_t a1 = (int64_t)p.j * pitch + p.i;
        p.next();
        const Stencil5 x0 = load5(u + a0, pitch), x1 = load5(u + a1, pitch);
        const double q0 = HAS_Q ? q[a0] : 0.0, q1 = HAS_Q ? q[a1] : 0.0;
        const double r0 = defect5<UNIT_BETA, HAS_Q>(o, x0, q0, b2, d);
        const double r1 = defect5<UNIT_BETA, HAS_Q>(o, x1, q1, b2, d);
        acc = __fma_rn(r0, r0, acc);
        acc = __fma_rn(r1, r1, acc);
    }
    if (p.left > 0) {
        const double r =
            defect_at<UNIT_BETA, HAS_Q>(o, u, q, (int64_t)p.j * pitch + p.i, pitch, b2, d);
        acc = __fma_rn(r, r, acc);
    }
    __shared__ double red[NORM_THREADS / 32];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < NORM_THREADS / 32 ? red[threadIdx.x] : 0.0;
        v = warp_sum(v);
        if (threadIdx.x == 0) partials[blockIdx.x] = v;
    }
}

__global__ void __launch_bounds__(NORM_THREADS)
    sum_partials_kernel(const double* __restrict__ partials, int count, double* __restrict__ out)
{
    double acc = 0.0;
    for (int k = threadIdx.x; k < count; k += NORM_THREADS) acc = __dadd_rn(acc, partials[k]);
    __shared__ double red[NORM_THREADS / 32];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < NORM_THREADS / 32 ? red[threadIdx.x] : 0.0;
        v = warp_sum(v);
        if (threadIdx.x == 0) {
            out[0] = v;
            out[1] = sqrt(v);
        }
    }
}

__global__ void __launch_bounds__(JA_BX* JA_BY)
    maxdelta_kernel(const double* __restrict__ a, const double* __restrict__ b, int m, int n,
                    int64_t pitch, unsigned long long* __restrict__ maxd)
{
    const FmaOps o = load_fma_ops();
    const int j = 1 + blockIdx.y * JA_BY + threadIdx.y;
    const int i = 1 + blockIdx.x * JA_BX + threadIdx.x;
    unsigned long long dl = 0;
    if (j <= n - 2 && i <= m - 2) {
        const int64_t at = (int64_t)j * pitch + i;
        dl = abs_bits(fadd(o, a[at], -b[at]));
    }
    flush_maxd(dl, maxd);
}

dim3 rb_grid(int m, int n)
{
    const int per_row = (m - 2 + 1) / 2;  // points of one colour in a row, at most
    return dim3((per_row + RB_BX - 1) / RB_BX, (n - 2 + RB_BY - 1) / RB_BY);
}

dim3 point_grid(int m, int n)
{
    return dim3((m - 2 + JA_BX - 1) / JA_BX, (n - 2 + JA_BY - 1) / JA_BY);
}

}  // namespace

#define LAP_DISPATCH_BOOL(flag, NAME, ...) \
    do {                                   \
        if (flag) {                        \
            constexpr bool NAME = true;    \
            __VA_ARGS__;                   \
        } else {                           \
            constexpr bool NAME = false;   \
            __VA_ARGS__;                   \
        }                                  \
    } while (0)

cudaError_t launch_rb_colour(const Field& f, const double* q, const Coef& c, bool gs, double w,
                             int colour, unsigned long long* maxd, cudaStream_t s,
                             const double* wslot)
{
    const dim3 grid = rb_grid(f.m, f.n), block(RB_BX, RB_BY);
    const double omw = 1.0 - w;
    LAP_DISPATCH_BOOL(c.unit_beta, UB, LAP_DISPATCH_BOOL(c.inv_d_shift > 0, P2,
        LAP_DISPATCH_BOOL(q != nullptr, HQ, LAP_DISPATCH_BOOL(gs, GS, LAP_DISPATCH_BOOL(maxd != nullptr, MD,
            rb_colour_kernel<UB, P2, HQ, GS, MD><<<grid, block, 0, s>>>(
                f.p, q, f.m, f.n, f.pitch, colour, c.b2, c.inv_d, c.inv_d_shift, w, omw, maxd,
                wslot))))));
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_rb_diag(const Field& f, const double* q, bool gs, double w, int colour,
                           unsigned long long* maxd, cudaStream_t s, const double* wslot)
{
    const int starts = rb_diag_starts(f.m);
    const int64_t walks = rb_diag_walks(f.m, f.n);
    if (walks > RB_DIAG_MAX_WALKS) return cudaErrorInvalidValue;  // the kernel's int numbering
    const int grid = (int)((walks + RD_BX - 1) / RD_BX);
    const double omw = 1.0 - w;
    LAP_DISPATCH_BOOL(q != nullptr, HQ, LAP_DISPATCH_BOOL(gs, GS, LAP_DISPATCH_BOOL(maxd != nullptr, MD,
        rb_diag_kernel<HQ, GS, MD><<<grid, RD_BX, 0, s>>>(f.p, q, f.m, f.n, f.pitch, colour, starts,
                                                           w, omw, maxd, wslot))));
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_jacobi(const Field& in, double* out, const Coef& c, unsigned long long* maxd,
                          cudaStream_t s)
{
    const dim3 grid = point_grid(in.m, in.n), block(JA_BX, JA_BY);
    LAP_DISPATCH_BOOL(c.unit_beta, UB, LAP_DISPATCH_BOOL(c.inv_d_shift > 0, P2,
        LAP_DISPATCH_BOOL(maxd != nullptr, MD,
            jacobi_kernel<UB, P2, MD><<<grid, block, 0, s>>>(in.p, out, in.m, in.n, in.pitch, c.b2,
                                                             c.inv_d, c.inv_d_shift, maxd))));
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_defect(const Field& f, const double* q, double* r, const Coef& c,
                          cudaStream_t s)
{
    const dim3 grid = point_grid(f.m, f.n), block(JA_BX, JA_BY);
    LAP_DISPATCH_BOOL(c.unit_beta, UB, LAP_DISPATCH_BOOL(q != nullptr, HQ,
        defect_kernel<UB, HQ><<<grid, block, 0, s>>>(f.p, q, r, f.m, f.n, f.pitch, c.b2, c.d)));
    note_launch();
    return cudaGetLastError();
}

int norm_blocks(const Field& f) { return norm_blocks_for(f.m, f.n); }

cudaError_t launch_defect_sumsq(const Field& f, const double* q, const Coef& c, double* partials,
                                cudaStream_t s)
{
    const int blocks = norm_blocks(f);
    LAP_DISPATCH_BOOL(c.unit_beta, UB, LAP_DISPATCH_BOOL(q != nullptr, HQ,
        defect_sumsq_kernel<UB, HQ><<<blocks, NORM_THREADS, 0, s>>>(f.p, q, f.m, f.n, f.pitch, c.b2,
                                                                    c.d, partials)));
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_sum_partials(const double* partials, int count, double* out, cudaStream_t s)
{
    sum_partials_kernel<<<1, NORM_THREADS, 0, s>>>(partials, count, out);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_maxdelta(const Field& a, const double* b, unsigned long long* maxd,
                            cudaStream_t s)
{
    maxdelta_kernel<<<point_grid(a.m, a.n), dim3(JA_BX, JA_BY), 0, s>>>(a.p, b, a.m, a.n, a.pitch,
                                                                         maxd);
    note_launch();
    return cudaGetLastError();
}

}  // namespace lap
