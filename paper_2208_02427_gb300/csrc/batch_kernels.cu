// batch_kernels.cu -- the V-cycle over many independent grids of different sizes.
//
// Every phase of a cycle (a smoother colour pass, the residual, the restriction, the
// interpolation, the coarsest solve, the residual norm) is one launch over a work list of
// (level, block of rows) items gathered from all problems that take part in that phase:
// one CTA per item, or a persistent launch whose resident CTAs claim the items from a counter
// (ItemClaim); the tuner picks one.
// Per problem the arithmetic is exactly the single-grid kernels' (same expressions, same
// roundings), so a batched solve reproduces each problem's single-grid iterates. A
// problem that has converged is skipped by every later launch (its `active` flag); the
// norm kernels decide convergence on the device.
//
// The level data are generic in T: double for the FP64 V-cycle, float for the inner cycle
// of the mixed-precision solver (FP32 inside FP64 defect correction).
#include <type_traits>

#include "lap_device.cuh"
#include "lap_internal.cuh"

namespace lap {

namespace {

constexpr int BT = 256;  // threads per work item

// Arithmetic of one precision, matching the single-grid kernels of that precision.
template <class T> struct Arith;
template <> struct Arith<double> {
    FmaOps o;
    __device__ double add(double a, double b) const { return fadd(o, a, b); }
    __device__ double mul(double a, double b) const { return fmul(o, a, b); }
    __device__ double fma(double a, double b, double c) const { return __fma_rn(a, b, c); }
    template <bool UNIT>
    __device__ double nsum(double w, double e, double s, double n, double b2) const
    {
        return neighbour_sum<UNIT>(o, w, e, s, n, b2);
    }
    template <bool POW2>
    __device__ double inv_d(double s, const BatchLevel<double>& L) const
    {
        return times_inv_d<POW2>(o, s, L.inv_d, L.inv_d_shift);
    }
    __device__ double half(double x) const { return scale_down_pow2(o, x, 1, 0.5); }
    __device__ double quarter(double x) const { return scale_down_pow2(o, x, 2, 0.25); }
    __device__ double two() const { return in_reg(o, 2.0); }
};
template <> struct Arith<float> {
    __device__ float add(float a, float b) const { return __fadd_rn(a, b); }
    __device__ float mul(float a, float b) const { return __fmul_rn(a, b); }
    __device__ float fma(float a, float b, float c) const { return __fmaf_rn(a, b, c); }
    template <bool UNIT>
    __device__ float nsum(float w, float e, float s, float n, float b2) const
    {
        const float ew = __fadd_rn(w, e), ns = __fadd_rn(s, n);
        return UNIT ? __fadd_rn(ns, ew) : __fmaf_rn(b2, ns, ew);
    }
    template <bool POW2>
    __device__ float inv_d(float s, const BatchLevel<float>& L) const
    {
        return __fmul_rn(s, (float)L.inv_d);
    }
    __device__ float half(float x) const { return __fmul_rn(0.5f, x); }
    __device__ float quarter(float x) const { return __fmul_rn(0.25f, x); }
    __device__ float two() const { return 2.0f; }
};

template <class T>
__device__ __forceinline__ Arith<T> arith();
template <>
__device__ __forceinline__ Arith<double> arith<double>() { return Arith<double>{load_fma_ops()}; }
template <>
__device__ __forceinline__ Arith<float> arith<float>() { return Arith<float>{}; }

// The flattened index k = threadIdx.x, threadIdx.x + BT, ... of an item's rows x width points
// as (row r, column c) pairs: one division per thread, then an add with carry per step.
struct Walk {
    int r, c, dr, dc, w;
    __device__ __forceinline__ explicit Walk(int width) : w(width)
    {
        r = threadIdx.x / width;
        c = threadIdx.x - r * width;
        dr = BT / width;
        dc = BT - dr * width;
    }
    __device__ __forceinline__ void next()
    {
        c += dc;
        r += dr;
        if (c >= w) {
            c -= w;
            ++r;
        }
    }
};

// A flag that is uniform over a block (a level's beta == 1, 1/d a power of two, a source
// term, GS or SOR) becomes a template argument: the loop is compiled once per value. Left a
// run-time choice inside the per-point code, the compiler evaluates both sides of the short
// FP64 branch and selects, one FP64 operation more per point (measured: the batched FP64
// residual norm at 89% FP64-pipe occupancy for half its useful throughput).
template <class F>
__device__ __forceinline__ void on_flag(bool a, F&& f)
{
    if (a) f(std::true_type{});
    else f(std::false_type{});
}

// ---- per-point arithmetic, shared by the item kernels and the small-level tail kernel ----

// Eq. 6 (GS) or Eq. 7 at interior point (i, j) of level L, in place; UNIT: beta == 1, POW2:
// 1/d = 2^-k, HQ: L.q is set.
template <class T, bool UNIT, bool POW2, bool HQ, bool GS>
__device__ __forceinline__ void rb_point(const Arith<T>& A, const BatchLevel<T>& L, int i, int j,
                                         T w, T omw)
{
    const int64_t at = (int64_t)j * L.pitch + i;
    T* c = L.u + at;
    T s = A.template nsum<UNIT>(c[-1], c[1], c[-L.pitch], c[L.pitch], (T)L.b2);
    if (HQ) s = A.add(s, L.q[at]);
    const T g = A.template inv_d<POW2>(s, L);
    *c = GS ? g : A.fma(w, g, A.mul(omw, *c));
}

// r = (E+W) + b2 (N+S) (+ q) - d u at interior point (i, j).
template <class T, bool UNIT, bool HQ>
__device__ __forceinline__ void defect_point(const Arith<T>& A, const BatchLevel<T>& L, int i, int j)
{
    const int64_t at = (int64_t)j * L.pitch + i;
    const T* c = L.u + at;
    T s = A.template nsum<UNIT>(c[-1], c[1], c[-L.pitch], c[L.pitch], (T)L.b2);
    if (HQ) s = A.add(s, L.q[at]);
    L.r[at] = A.fma(-(T)L.d, *c, s);
}

// The smoother's flags of level L (and the launch's GS flag) as template arguments of f.
template <class T, class F>
__device__ __forceinline__ void on_rb_flags(const BatchLevel<T>& L, bool gs, F&& f)
{
    on_flag(L.unit_beta != 0, [&](auto U) {
        on_flag(L.inv_d_shift > 0, [&](auto P) {
            on_flag(L.q != nullptr, [&](auto Q) { on_flag(gs, [&](auto G) { f(U, P, Q, G); }); });
        });
    });
}

// Coarse point (I, J): qc = 0.25 ((4 c + 2 edges) + corners) of the fine residual; the
// coarse correction starts at zero.
template <class T>
__device__ __forceinline__ void restrict_point(const Arith<T>& A, const BatchLevel<T>& C,
                                               const BatchLevel<T>& F, int I, int J)
{
    const int64_t pf = F.pitch;
    const T* c = F.r + (int64_t)(2 * J) * pf + 2 * I;
    const T edges = A.add(A.add(c[-1], c[1]), A.add(c[-pf], c[pf]));
    const T corners = A.add(A.add(c[-pf - 1], c[-pf + 1]), A.add(c[pf - 1], c[pf + 1]));
    const T two = A.two();
    const T t = A.fma(two, c[0], edges);
    const int64_t at = (int64_t)J * C.pitch + I;
    C.q[at] = A.quarter(A.fma(two, t, corners));
    C.u[at] = (T)0;
}

// Fine row j, coarse column I: bilinear interpolation added to fine points 2I and 2I + 1.
template <class T>
__device__ __forceinline__ void prolong_pair(const Arith<T>& A, const BatchLevel<T>& F,
                                             const BatchLevel<T>& C, int I, int j)
{
    const int64_t pc = C.pitch;
    const T* a = C.u + (int64_t)(j >> 1) * pc + I;
    const int i0 = 2 * I, i1 = 2 * I + 1;
    T* row = F.u + (int64_t)j * F.pitch;
    if ((j & 1) == 0) {
        if (i0 >= 1) row[i0] = A.add(row[i0], a[0]);
        if (i1 <= F.m - 2) row[i1] = A.add(row[i1], A.half(A.add(a[0], a[1])));
    } else {
        if (i0 >= 1) row[i0] = A.add(row[i0], A.half(A.add(a[0], a[pc])));
        if (i1 <= F.m - 2) {
            const T s = A.add(A.add(a[0], a[1]), A.add(a[pc], a[pc + 1]));
            row[i1] = A.add(row[i1], A.quarter(s));
        }
    }
}

// One smoother colour pass (Eq. 6 when gs, Eq. 7 otherwise) over the rows of each item.
template <class T>
__global__ void __launch_bounds__(BT)
    b_rb_kernel(const BatchItem* __restrict__ items, int count, unsigned* claim, const BatchLevel<T>* __restrict__ lv,
                const int* __restrict__ active, int colour, int gs, T w_arg, T omw_arg, int per_level_w)
{
    const Arith<T> A = arith<T>();
    const ItemClaim ic{claim, count};
    for (int b = ic.take(-1); b < count; b = ic.take(b)) {
        const BatchItem it = items[b];
        const BatchLevel<T> L = lv[it.level];
        if (!active[L.problem]) continue;
        const T w = per_level_w ? (T)L.w : w_arg, omw = per_level_w ? (T)L.omw : omw_arg;
        const int half_w = (L.m - 2 + 1) / 2;
        on_rb_flags(L, gs != 0, [&](auto U, auto P, auto Q, auto G) {
            for (Walk k(half_w); k.r < it.rows; k.next()) {
                const int j = it.row0 + k.r;
                const int i = 1 + ((1 + j + colour) & 1) + 2 * k.c;
                if (i <= L.m - 2)
                    rb_point<T, decltype(U)::value, decltype(P)::value, decltype(Q)::value,
                             decltype(G)::value>(A, L, i, j, w, omw);
            }
        });
    }
    ic.finish();
}

template <class T>
__global__ void __launch_bounds__(BT)
    b_defect_kernel(const BatchItem* __restrict__ items, int count, unsigned* claim,
                    const BatchLevel<T>* __restrict__ lv, const int* __restrict__ active)
{
    const Arith<T> A = arith<T>();
    const ItemClaim ic{claim, count};
    for (int b = ic.take(-1); b < count; b = ic.take(b)) {
        const BatchItem it = items[b];
        const BatchLevel<T> L = lv[it.level];
        if (!active[L.problem]) continue;
        const int wdt = L.m - 2;
        on_flag(L.unit_beta != 0, [&](auto U) {
            on_flag(L.q != nullptr, [&](auto Q) {
                for (Walk k(wdt); k.r < it.rows; k.next())
                    defect_point<T, decltype(U)::value, decltype(Q)::value>(A, L, 1 + k.c, it.row0 + k.r);
            });
        });
    }
    ic.finish();
}

// Items of the coarse level: qc from the fine residual (the level before it in lv), and the
// coarse correction zeroed.
template <class T>
__global__ void __launch_bounds__(BT)
    b_restrict_kernel(const BatchItem* __restrict__ items, int count, unsigned* claim,
                      const BatchLevel<T>* __restrict__ lv, const int* __restrict__ active)
{
    const Arith<T> A = arith<T>();
    const ItemClaim ic{claim, count};
    for (int b = ic.take(-1); b < count; b = ic.take(b)) {
        const BatchItem it = items[b];
        const BatchLevel<T> C = lv[it.level];
        if (!active[C.problem]) continue;
        const BatchLevel<T> F = lv[it.level - 1];
        const int wdt = C.m - 2;
        for (Walk k(wdt); k.r < it.rows; k.next()) restrict_point(A, C, F, 1 + k.c, it.row0 + k.r);
    }
    ic.finish();
}

// Items of the fine level: u += bilinear interpolation of the next level's correction.
template <class T>
__global__ void __launch_bounds__(BT)
    b_prolong_kernel(const BatchItem* __restrict__ items, int count, unsigned* claim,
                     const BatchLevel<T>* __restrict__ lv, const int* __restrict__ active)
{
    const Arith<T> A = arith<T>();
    const ItemClaim ic{claim, count};
    for (int b = ic.take(-1); b < count; b = ic.take(b)) {
        const BatchItem it = items[b];
        const BatchLevel<T> F = lv[it.level];
        if (!active[F.problem]) continue;
        const BatchLevel<T> C = lv[it.level + 1];
        const int pairs = (F.m - 1) / 2;  // coarse columns 0 .. mc-2
        for (Walk k(pairs); k.r < it.rows; k.next()) prolong_pair(A, F, C, k.c, it.row0 + k.r);
    }
    ic.finish();
}

// u = A^-1 b at the coarsest level L, b = q + ring terms assembled in FP64; all threads of the
// CTA take part (b: shared memory of N doubles).
template <class T>
__device__ __forceinline__ void coarse_cta(const BatchLevel<T>& L, double* b)
{
    const int mi = L.m - 2, N = mi * (L.n - 2);
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        const int i = 1 + k % mi, j = 1 + k / mi;
        const int64_t at = (int64_t)j * L.pitch + i;
        double v = L.q ? (double)L.q[at] : 0.0;
        if (i == 1) v = __dadd_rn(v, (double)L.u[at - 1]);
        if (i == L.m - 2) v = __dadd_rn(v, (double)L.u[at + 1]);
        if (j == 1) v = __fma_rn(L.b2, (double)L.u[at - L.pitch], v);
        if (j == L.n - 2) v = __fma_rn(L.b2, (double)L.u[at + L.pitch], v);
        b[k] = v;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        double x = 0.0;
        for (int l = 0; l < N; ++l) x = __fma_rn(L.ainv_t[(int64_t)l * N + k], b[l], x);
        const int i = 1 + k % mi, j = 1 + k / mi;
        L.u[(int64_t)j * L.pitch + i] = (T)x;
    }
}

// One item per problem at its coarsest level: u = A^-1 b in FP64.
template <class T>
__global__ void __launch_bounds__(1024)
    b_coarse_kernel(const BatchItem* __restrict__ items, int count, unsigned* claim,
                    const BatchLevel<T>* __restrict__ lv, const int* __restrict__ active)
{
    extern __shared__ double b[];
    const ItemClaim ic{claim, count};
    for (int k = ic.take(-1); k < count; k = ic.take(k)) {
        const BatchItem it = items[k];
        const BatchLevel<T> L = lv[it.level];
        if (!active[L.problem]) continue;
        coarse_cta(L, b);
        __syncthreads();  // b is reused by the next item
    }
    ic.finish();
}

// ---- the small-level tail: the rest of a V-cycle in one CTA ----
// Below some size a level's launches cost more than its work. The tail kernel runs the
// whole V-cycle from level `first` of one problem down to its coarsest level and back
// (smoothing, residual, restriction, coarsest solve, interpolation, smoothing) in one
// CTA, with a CTA barrier between phases instead of a launch. Rows are spread over the
// warps and same-colour points over the lanes; the per-point arithmetic is that of the
// item kernels, so the tail changes the launch structure and nothing else.
constexpr int TAIL_THREADS = 512;

template <class T>
__device__ __forceinline__ void smooth_cta(const Arith<T>& A, const BatchLevel<T>& L, int sweeps,
                                           bool gs, T w, T omw)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int half_w = (L.m - 2 + 1) / 2;
    on_rb_flags(L, gs, [&](auto U, auto P, auto Q, auto G) {
        for (int k = 0; k < sweeps; ++k)
            for (int colour = 0; colour < 2; ++colour) {
                for (int j = 1 + wid; j <= L.n - 2; j += nw)
                    for (int t = lane; t < half_w; t += 32) {
                        const int i = 1 + ((1 + j + colour) & 1) + 2 * t;
                        if (i <= L.m - 2)
                            rb_point<T, decltype(U)::value, decltype(P)::value, decltype(Q)::value,
                                     decltype(G)::value>(A, L, i, j, w, omw);
                    }
                __syncthreads();
            }
    });
}

// The V-cycle of one tail job by the whole CTA (levels jb.first .. jb.last).
template <class T>
__device__ __forceinline__ void tail_job(const TailJob& jb, const BatchLevel<T>* __restrict__ lv,
                                         int nu1, int nu2, bool gs, T w, T omw, double* b)
{
    const Arith<T> A = arith<T>();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int l = jb.first; l < jb.last; ++l) {
        const BatchLevel<T> F = lv[l];
        smooth_cta(A, F, nu1, gs != 0, w, omw);
        on_flag(F.unit_beta != 0, [&](auto U) {
            on_flag(F.q != nullptr, [&](auto Q) {
                for (int j = 1 + wid; j <= F.n - 2; j += nw)
                    for (int i = 1 + lane; i <= F.m - 2; i += 32)
                        defect_point<T, decltype(U)::value, decltype(Q)::value>(A, F, i, j);
            });
        });
        __syncthreads();
        const BatchLevel<T> C = lv[l + 1];
        for (int J = 1 + wid; J <= C.n - 2; J += nw)
            for (int I = 1 + lane; I <= C.m - 2; I += 32) restrict_point(A, C, F, I, J);
        __syncthreads();
    }
    coarse_cta(lv[jb.last], b);
    __syncthreads();
    for (int l = jb.last - 1; l >= jb.first; --l) {
        const BatchLevel<T> F = lv[l];
        const BatchLevel<T> C = lv[l + 1];
        const int pairs = (F.m - 1) / 2;
        for (int j = 1 + wid; j <= F.n - 2; j += nw)
            for (int I = lane; I < pairs; I += 32) prolong_pair(A, F, C, I, j);
        __syncthreads();
        smooth_cta(A, F, nu2, gs != 0, w, omw);
    }
}

// The tail is latency-bound (a CTA barrier per phase, few points per thread): the FP32 tail
// is held to 32 registers so that four CTAs share an SM (measured on the 4096-grid batch: 928,
// 791, 755 us per cycle's tail launches at two, three and four CTAs per SM); the FP64 one to
// two CTAs (64 registers, no spills).
template <class T>
__global__ void __launch_bounds__(TAIL_THREADS, (sizeof(T) == 4 ? 4 : 2))
    b_tail_kernel(const TailJob* __restrict__ jobs, int count, unsigned* claim, const BatchLevel<T>* __restrict__ lv,
                  const int* __restrict__ active, int nu1, int nu2, int gs, T w_arg, T omw_arg,
                  int per_level_w)
{
    extern __shared__ double b[];
    const ItemClaim ic{claim, count};
    for (int k = ic.take(-1); k < count; k = ic.take(k)) {
        const TailJob jb = jobs[k];
        if (active && !active[lv[jb.first].problem]) continue;
        const T w = per_level_w ? (T)lv[jb.first].w : w_arg;
        const T omw = per_level_w ? (T)lv[jb.first].omw : omw_arg;
        tail_job(jb, lv, nu1, nu2, gs != 0, w, omw, b);
        __syncthreads();  // shared memory and the job's levels are reused by the next job
    }
    ic.finish();
}

// FP64 residual of each item's rows: per-item sum of squares (fixed order) and, for the
// mixed solver, the residual rounded to FP32 with the FP32 correction zeroed.
// Mixed problems whose r0 is known sum (s r)^2 in FP32, s = 2^-e with r0 = f 2^e (exact
// scaling; the stopping norm needs a few digits), and store the partial descaled. The
// descaling by 2^2e is exact, so it is done once on the block's sum (the same value as
// descaling every thread's sum first). A thread takes two walk positions per step, both
// points' stencils loaded before either is used; the sums keep the walk order.
template <bool MIXED, bool UNIT, bool SCALED>
__device__ __forceinline__ double sumsq_item(const BatchItem& it, const BatchLevel<double>& L,
                                             const BatchLevel<float>* __restrict__ lv32,
                                             float sc)
{
    const Arith<double> A = arith<double>();
    const double nd = -in_reg(A.o, L.d), b2 = L.b2;
    const int wdt = L.m - 2;
    float* r32 = nullptr;
    float* e32 = nullptr;
    int64_t p32 = 0;
    if (MIXED) {
        r32 = lv32[it.level].q;
        e32 = lv32[it.level].u;
        p32 = lv32[it.level].pitch;
    }
    double acc = 0.0;
    float acc32 = 0.0f;
    auto point = [&](const Stencil5& x, int i, int j) {
        const double r = __fma_rn(nd, x.c, A.template nsum<UNIT>(x.w, x.e, x.s, x.n, b2));
        if (MIXED) {
            const float rf = to_float_rn(r);
            if (SCALED) {
                const float rs = __fmul_rn(rf, sc);
                acc32 = __fmaf_rn(rs, rs, acc32);
            } else {
                acc = __fma_rn(r, r, acc);
            }
            const int64_t at = (int64_t)j * p32 + i;
            r32[at] = rf;
            e32[at] = 0.0f;
        } else {
            acc = __fma_rn(r, r, acc);
        }
    };
    Walk k(wdt);
    while (k.r < it.rows) {
        const int j0 = it.row0 + k.r, i0 = 1 + k.c;
        k.next();
        if (k.r >= it.rows) {
            point(load5(L.u + (int64_t)j0 * L.pitch + i0, L.pitch), i0, j0);
            break;
        }
        const int j1 = it.row0 + k.r, i1 = 1 + k.c;
        k.next();
        const Stencil5 x0 = load5(L.u + (int64_t)j0 * L.pitch + i0, L.pitch);
        const Stencil5 x1 = load5(L.u + (int64_t)j1 * L.pitch + i1, L.pitch);
        point(x0, i0, j0);
        point(x1, i1, j1);
    }
    if (MIXED && SCALED) acc = (double)acc32;
    return acc;
}

// Item ib's partial sum of squares (see b_sumsq_kernel) by the whole CTA into partials[ib].
__device__ __forceinline__ void sumsq_block(const BatchItem* __restrict__ items, int ib,
                                            const BatchLevel<double>* __restrict__ lv,
                                            const int* __restrict__ active, double* __restrict__ partials,
                                            const BatchLevel<float>* __restrict__ lv32,
                                            const double* __restrict__ r0)
{
    const BatchItem it = items[ib];
    const BatchLevel<double> L = lv[it.level];
    if (!active[L.problem]) return;
    // problems solved by the FP32 inner cycle have an FP32 level 0
    const bool mixed = lv32 && lv32[it.level].q;
    float sc = 0.0f;
    if (mixed && r0) {
        const double z = r0[L.problem];
        if (z > 0.0 && isfinite(z)) {
            const int e = ilogb(z);
            if (e >= -100 && e <= 100) sc = ldexpf(1.0f, -e);
        }
    }
    double acc = 0.0;
    // the FP32 or the FP64 sum of squares, chosen per block (as a per-point choice the
    // compiler would issue the FP64 fma for every point)
    on_flag(L.unit_beta != 0, [&](auto U) {
        if (!mixed)
            acc = sumsq_item<false, decltype(U)::value, false>(it, L, lv32, 0.0f);
        else
            on_flag(sc > 0.0f, [&](auto SC) {
                acc = sumsq_item<true, decltype(U)::value, decltype(SC)::value>(it, L, lv32, sc);
            });
    });
    __shared__ double red[BT / 32];  // a persistent CTA's next claim waits for the reads below
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < BT / 32 ? red[threadIdx.x] : 0.0;
        v = warp_sum(v);
        if (threadIdx.x == 0)
            partials[ib] = sc > 0.0f ? v / ((double)sc * (double)sc) : v;  // exact
    }
}

// CLAIM: a persistent launch (compiled apart: the one-item form keeps its registers free of
// the loop's state)
template <bool CLAIM>
__global__ void __launch_bounds__(BT, 5)
    b_sumsq_kernel(const BatchItem* __restrict__ items, int count, unsigned* claim,
                   const BatchLevel<double>* __restrict__ lv, const int* __restrict__ active,
                   double* __restrict__ partials, const BatchLevel<float>* __restrict__ lv32,
                   const double* __restrict__ r0)
{
    if (!CLAIM) {
        sumsq_block(items, blockIdx.x, lv, active, partials, lv32, r0);
        return;
    }
    const ItemClaim ic{claim, count};
    for (int b = ic.take(-1); b < count; b = ic.take(b))
        sumsq_block(items, b, lv, active, partials, lv32, r0);
    ic.finish();
}

// psi += e32 (FP64 update of the mixed solver).
__global__ void __launch_bounds__(BT)
    b_update_kernel(const BatchItem* __restrict__ items, int count, unsigned* claim,
                    const BatchLevel<double>* __restrict__ lv, const int* __restrict__ active,
                    const BatchLevel<float>* __restrict__ lv32)
{
    const FmaOps o = load_fma_ops();
    const ItemClaim ic{claim, count};
    for (int b = ic.take(-1); b < count; b = ic.take(b)) {
        const BatchItem it = items[b];
        const BatchLevel<double> L = lv[it.level];
        if (!active[L.problem]) continue;
        const BatchLevel<float> E = lv32[it.level];
        const int wdt = L.m - 2;
        for (Walk k(wdt); k.r < it.rows; k.next()) {
            const int j = it.row0 + k.r, i = 1 + k.c;
            double* c = L.u + (int64_t)j * L.pitch + i;
            *c = fadd(o, *c, to_double_exact(E.u[(int64_t)j * E.pitch + i]));
        }
    }
    ic.finish();
}

// Per problem: the norm from its items' partials (fixed order), then the stopping test.
// first_item[p] .. first_item[p+1] are problem p's items in the norm list. mode 0 records
// r0; mode 1 tests ||r|| <= tol r0 (rel) or <= tol (abs) and retires converged problems, and
// (maxit) problems that have run their cycles. Retiring problems go to the completion list.
__global__ void b_converge_kernel(const double* __restrict__ partials,
                                  const int* __restrict__ first_item, int count,
                                  int* __restrict__ active, double* __restrict__ r0,
                                  double* __restrict__ rnow, long long* __restrict__ iters,
                                  int* __restrict__ status, int* __restrict__ remaining, int mode,
                                  int rel, double tol, const double* __restrict__ tolv,
                                  const long long* __restrict__ maxit, Completion* __restrict__ done,
                                  int* __restrict__ ndone)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= count || !active[p]) return;
    if (first_item[p] == first_item[p + 1]) return;  // not in this list
    if (tolv) tol = tolv[p];
    double s = 0.0;
    for (int k = first_item[p]; k < first_item[p + 1]; ++k) s = __dadd_rn(s, partials[k]);
    const double nr = sqrt(s);
    rnow[p] = nr;
    if (mode == 0) {
        r0[p] = nr;
        iters[p] = 0;
        if (!isfinite(nr)) {
            status[p] = 2;
        } else if ((rel && nr == 0.0) || (!rel && nr <= tol)) {
            status[p] = 0;
        } else if (maxit && maxit[p] <= 0) {
            status[p] = 1;  // no iteration allowed: retire with the initial norm
        } else {
            return;
        }
    } else {
        iters[p] += 1;  // cycles done while active (replayed graphs need no host counter)
        if (!isfinite(nr)) status[p] = 2;
        else if (rel ? nr <= tol * r0[p] : nr <= tol) status[p] = 0;
        else if (maxit && iters[p] >= maxit[p]) status[p] = 1;
        else return;
    }
    active[p] = 0;
    atomicSub(remaining, 1);
    if (done) {
        const int k = atomicAdd(ndone, 1);
        done[k] = Completion{p, status[p], iters[p], r0[p], nr};
    }
}

}  // namespace

template <class T>
cudaError_t launch_b_rb(const BatchList& l, const BatchLevel<T>* lv, const int* active, int colour,
                        bool gs, double w, cudaStream_t s, bool per_level_w)
{
    if (l.count == 0) return cudaSuccess;
    const int grid = batch_grid((const void*)b_rb_kernel<T>, BT, 0, l.count, l.claim != nullptr);
    b_rb_kernel<T><<<grid, BT, 0, s>>>(l.items, l.count, l.claim, lv, active, colour, gs ? 1 : 0, (T)w,
                                       (T)(1.0 - w), per_level_w ? 1 : 0);
    note_launch();
    return cudaGetLastError();
}
template <class T>
cudaError_t launch_b_defect(const BatchList& l, const BatchLevel<T>* lv, const int* active,
                            cudaStream_t s)
{
    if (l.count == 0) return cudaSuccess;
    const int grid = batch_grid((const void*)b_defect_kernel<T>, BT, 0, l.count, l.claim != nullptr);
    b_defect_kernel<T><<<grid, BT, 0, s>>>(l.items, l.count, l.claim, lv, active);
    note_launch();
    return cudaGetLastError();
}
template <class T>
cudaError_t launch_b_restrict(const BatchList& l, const BatchLevel<T>* lv, const int* active,
                              cudaStream_t s)
{
    if (l.count == 0) return cudaSuccess;
    const int grid = batch_grid((const void*)b_restrict_kernel<T>, BT, 0, l.count, l.claim != nullptr);
    b_restrict_kernel<T><<<grid, BT, 0, s>>>(l.items, l.count, l.claim, lv, active);
    note_launch();
    return cudaGetLastError();
}
template <class T>
cudaError_t launch_b_prolong(const BatchList& l, const BatchLevel<T>* lv, const int* active,
                             cudaStream_t s)
{
    if (l.count == 0) return cudaSuccess;
    const int grid = batch_grid((const void*)b_prolong_kernel<T>, BT, 0, l.count, l.claim != nullptr);
    b_prolong_kernel<T><<<grid, BT, 0, s>>>(l.items, l.count, l.claim, lv, active);
    note_launch();
    return cudaGetLastError();
}
template <class T>
cudaError_t launch_b_coarse(const BatchList& l, const BatchLevel<T>* lv, const int* active,
                            int max_unknowns, cudaStream_t s)
{
    if (l.count == 0) return cudaSuccess;
    int threads = ((max_unknowns + 31) / 32) * 32;
    threads = threads < 32 ? 32 : (threads > 1024 ? 1024 : threads);
    const size_t smem = sizeof(double) * max_unknowns;
    const int grid = batch_grid((const void*)b_coarse_kernel<T>, threads, smem, l.count, l.claim != nullptr);
    b_coarse_kernel<T><<<grid, threads, smem, s>>>(l.items, l.count, l.claim, lv, active);
    note_launch();
    return cudaGetLastError();
}

template cudaError_t launch_b_rb<double>(const BatchList&, const BatchLevel<double>*, const int*, int, bool, double, cudaStream_t, bool);
template cudaError_t launch_b_rb<float>(const BatchList&, const BatchLevel<float>*, const int*, int, bool, double, cudaStream_t, bool);
template cudaError_t launch_b_defect<double>(const BatchList&, const BatchLevel<double>*, const int*, cudaStream_t);
template cudaError_t launch_b_defect<float>(const BatchList&, const BatchLevel<float>*, const int*, cudaStream_t);
template cudaError_t launch_b_restrict<double>(const BatchList&, const BatchLevel<double>*, const int*, cudaStream_t);
template cudaError_t launch_b_restrict<float>(const BatchList&, const BatchLevel<float>*, const int*, cudaStream_t);
template cudaError_t launch_b_prolong<double>(const BatchList&, const BatchLevel<double>*, const int*, cudaStream_t);
template cudaError_t launch_b_prolong<float>(const BatchList&, const BatchLevel<float>*, const int*, cudaStream_t);
template cudaError_t launch_b_coarse<double>(const BatchList&, const BatchLevel<double>*, const int*, int, cudaStream_t);
template cudaError_t launch_b_coarse<float>(const BatchList&, const BatchLevel<float>*, const int*, int, cudaStream_t);

template <class T>
cudaError_t launch_b_tail(const TailJob* jobs, int count, const BatchLevel<T>* lv, const int* active,
                          int nu1, int nu2, bool gs, double w, int max_unknowns, cudaStream_t s,
                          bool per_level_w, unsigned* claim)
{
    if (count == 0) return cudaSuccess;
    const size_t smem = sizeof(double) * (max_unknowns > 0 ? max_unknowns : 1);
    const int grid = batch_grid((const void*)b_tail_kernel<T>, TAIL_THREADS, smem, count, claim != nullptr);
    b_tail_kernel<T><<<grid, TAIL_THREADS, smem, s>>>(jobs, count, claim, lv, active, nu1, nu2, gs ? 1 : 0,
                                                      (T)w, (T)(1.0 - w), per_level_w ? 1 : 0);
    note_launch();
    return cudaGetLastError();
}
template cudaError_t launch_b_tail<double>(const TailJob*, int, const BatchLevel<double>*, const int*, int, int, bool, double, int, cudaStream_t, bool, unsigned*);
template cudaError_t launch_b_tail<float>(const TailJob*, int, const BatchLevel<float>*, const int*, int, int, bool, double, int, cudaStream_t, bool, unsigned*);

cudaError_t launch_b_sumsq(const BatchList& l, const BatchLevel<double>* lv, const int* active,
                           double* partials, const BatchLevel<float>* lv32, cudaStream_t s,
                           const double* r0)
{
    if (l.count == 0) return cudaSuccess;
    if (l.claim) {
        const int grid = batch_grid((const void*)b_sumsq_kernel<true>, BT, 0, l.count, true);
        b_sumsq_kernel<true><<<grid, BT, 0, s>>>(l.items, l.count, l.claim, lv, active, partials, lv32, r0);
    } else {
        b_sumsq_kernel<false><<<l.count, BT, 0, s>>>(l.items, l.count, nullptr, lv, active, partials, lv32,
                                                     r0);
    }
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_b_update(const BatchList& l, const BatchLevel<double>* lv, const int* active,
                            const BatchLevel<float>* lv32, cudaStream_t s)
{
    if (l.count == 0) return cudaSuccess;
    const int grid = batch_grid((const void*)b_update_kernel, BT, 0, l.count, l.claim != nullptr);
    b_update_kernel<<<grid, BT, 0, s>>>(l.items, l.count, l.claim, lv, active, lv32);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_b_converge(const double* partials, const int* first_item, int count, int* active,
                              double* r0, double* rnow, long long* iters, int* status,
                              int* remaining, int mode, bool rel, double tol, cudaStream_t s,
                              const double* tolv, const long long* maxit, Completion* done,
                              int* ndone)
{
    b_converge_kernel<<<(count + 127) / 128, 128, 0, s>>>(partials, first_item, count, active, r0,
                                                          rnow, iters, status, remaining, mode,
                                                          rel ? 1 : 0, tol, tolv, maxit, done, ndone);
    note_launch();
    return cudaGetLastError();
}

}  // namespace lap
