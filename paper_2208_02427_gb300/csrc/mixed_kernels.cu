// mixed_kernels.cu -- FP32 multigrid cycle inside FP64 defect correction.
//
// The correction equation of the V-cycle (Eqs. 13-15: L dpsi = -R) is solved
// approximately in FP32 while the fine-grid residual R = L(psi) and the update
// psi <- psi + dpsi stay FP64:
//   1. r = dx^2 L(psi) in FP64 (the same expression as the FP64 residual), stored as
//      FP32 for the inner cycle, its sum of squares accumulated in FP64 for the stopping
//      test; the inner correction e is zeroed in the same pass;
//   2. one or more V-cycles in FP32 on (E+W) + b2 (N+S) - d e + r = 0, e = 0 on the ring;
//   3. psi += e in FP64.
// FP32 runs 62x faster than FP64 on GB300, so the inner cycle is bound by memory, not
// by arithmetic; the FP64 work per outer iteration is two passes over the fine grid.
#include "lap_device.cuh"
#include "lap_internal.cuh"

namespace lap {

namespace {

constexpr int BX = 64, BY = 4;      // red-black and transfer kernels
constexpr int PX = 128, PY = 2;     // point kernels over all interior nodes
constexpr int NORM_THREADS = 256;
// 6 blocks of 256 threads per SM (at most 42 registers a thread): the norm kernels' grid of
// at most 6 blocks per SM (norm_blocks_for; 912 on 152 SMs) is resident at once.
constexpr int NORM_BLOCKS_PER_SM = 6;

__device__ __forceinline__ float nsum32(float w_, float e_, float s_, float n_, float b2,
                                        bool unit)
{
    const float ew = __fadd_rn(w_, e_);
    const float ns = __fadd_rn(s_, n_);
    return unit ? __fadd_rn(ns, ew) : __fmaf_rn(b2, ns, ew);
}

// One colour of the FP32 red-black smoother with source q: Gauss-Seidel (Eq. 6) or SOR
// (Eq. 7), the FP32 image of rb_colour_kernel.
template <bool UNIT, bool GS>
__global__ void __launch_bounds__(BX* BY)
    rb32_kernel(float* __restrict__ u, const float* __restrict__ q, int m, int n, int64_t pitch,
                int colour, float b2, float inv_d, float w, float omw)
{
    const int j = 1 + blockIdx.y * BY + threadIdx.y;
    const int i = 1 + ((1 + j + colour) & 1) + 2 * (blockIdx.x * BX + threadIdx.x);
    if (j > n - 2 || i > m - 2) return;
    const int64_t at = (int64_t)j * pitch + i;
    float* c = u + at;
    const float s = __fadd_rn(nsum32(c[-1], c[1], c[-pitch], c[pitch], b2, UNIT), q[at]);
    const float g = __fmul_rn(s, inv_d);
    *c = GS ? g : __fmaf_rn(w, g, __fmul_rn(omw, *c));
}

template <bool UNIT>
__global__ void __launch_bounds__(PX* PY)
    defect32_kernel(const float* __restrict__ u, const float* __restrict__ q,
                    float* __restrict__ r, int m, int n, int64_t pitch, float b2, float d)
{
    const int j = 1 + blockIdx.y * PY + threadIdx.y;
    const int i = 1 + blockIdx.x * PX + threadIdx.x;
    if (j > n - 2 || i > m - 2) return;
    const int64_t at = (int64_t)j * pitch + i;
    const float* c = u + at;
    const float s = __fadd_rn(nsum32(c[-1], c[1], c[-pitch], c[pitch], b2, UNIT), q[at]);
    r[at] = __fmaf_rn(-d, *c, s);
}

// Full weighting scaled to the coarse equation, qc = 0.25 ((4 c + 2 edges) + corners);
// also zeroes the coarse correction.
__global__ void __launch_bounds__(BX* BY)
    restrict32_kernel(const float* __restrict__ r, int mf, int nf, int64_t pf,
                      float* __restrict__ qc, float* __restrict__ ec, int64_t pc)
{
    const int mc = (mf - 1) / 2 + 1, nc = (nf - 1) / 2 + 1;
    const int I = 1 + blockIdx.x * BX + threadIdx.x;
    const int J = 1 + blockIdx.y * BY + threadIdx.y;
    if (I > mc - 2 || J > nc - 2) return;
    const float* c = r + (int64_t)(2 * J) * pf + 2 * I;
    const float edges = __fadd_rn(__fadd_rn(c[-1], c[1]), __fadd_rn(c[-pf], c[pf]));
    const float corners =
        __fadd_rn(__fadd_rn(c[-pf - 1], c[-pf + 1]), __fadd_rn(c[pf - 1], c[pf + 1]));
    const float t = __fmaf_rn(2.0f, c[0], edges);
    const int64_t at = (int64_t)J * pc + I;
    qc[at] = __fmul_rn(0.25f, __fmaf_rn(2.0f, t, corners));
    ec[at] = 0.0f;
}

__global__ void __launch_bounds__(BX* BY)
    prolong32_kernel(float* __restrict__ u, int mf, int nf, int64_t pf,
                     const float* __restrict__ ec, int64_t pc)
{
    const int I = blockIdx.x * BX + threadIdx.x;
    const int j = 1 + blockIdx.y * BY + threadIdx.y;
    const int mc = (mf - 1) / 2 + 1;
    if (I > mc - 2 || j > nf - 2) return;
    const float* a = ec + (int64_t)(j >> 1) * pc + I;
    const int i0 = 2 * I, i1 = 2 * I + 1;
    float* row = u + (int64_t)j * pf;
    if ((j & 1) == 0) {
        if (i0 >= 1) row[i0] = __fadd_rn(row[i0], a[0]);
        if (i1 <= mf - 2) row[i1] = __fadd_rn(row[i1], __fmul_rn(0.5f, __fadd_rn(a[0], a[1])));
    } else {
        if (i0 >= 1) row[i0] = __fadd_rn(row[i0], __fmul_rn(0.5f, __fadd_rn(a[0], a[pc])));
        if (i1 <= mf - 2) {
            const float s = __fadd_rn(__fadd_rn(a[0], a[1]), __fadd_rn(a[pc], a[pc + 1]));
            row[i1] = __fadd_rn(row[i1], __fmul_rn(0.25f, s));
        }
    }
}

// Coarsest level: b assembled in FP64 from the FP32 source (the correction's ring is zero),
// solved with the FP64 inverse, stored back in FP32.
__global__ void __launch_bounds__(1024)
    coarse32_kernel(float* __restrict__ u, const float* __restrict__ q, int m, int n,
                    int64_t pitch, const double* __restrict__ ainv_t)
{
    extern __shared__ double b[];
    const int mi = m - 2, N = mi * (n - 2);
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        const int i = 1 + k % mi, j = 1 + k / mi;
        b[k] = (double)q[(int64_t)j * pitch + i];
    }
    __syncthreads();
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        double x = 0.0;
        for (int l = 0; l < N; ++l) x = __fma_rn(ainv_t[(int64_t)l * N + k], b[l], x);
        const int i = 1 + k % mi, j = 1 + k / mi;
        u[(int64_t)j * pitch + i] = (float)x;
    }
}

// FP64 residual of psi, stored in FP32 for the inner cycle, sum of squares per block
// (fixed-order reduction) for the stopping test; zeroes the FP32 correction e (nullable).
// With a norm scale (sc: device slot, > 0) the squares are summed per thread in FP32 as
// (sc r)^2: the norm needs a few digits, not FP64's sixteen, and this takes one of the
// five FP64 operations per point off the FP64 pipe. sc is a power of two near 1 / ||r0||,
// so the scaled squares stay within FP32's normal range down to 1e-13 ||r0||.
template <bool UNIT, bool F32NORM>
__global__ void __launch_bounds__(NORM_THREADS, NORM_BLOCKS_PER_SM)
    defect64_to32_kernel(const double* __restrict__ psi, int m, int n, int64_t pitch, double b2,
                         double d, float* __restrict__ r32, float* __restrict__ e32,
                         int64_t pitch32, double* __restrict__ partials,
                         const float* __restrict__ sc)
{
    const FmaOps o = load_fma_ops();
    if (!UNIT) b2 = in_reg(o, b2);
    d = in_reg(o, d);
    double acc = 0.0;
    float acc32 = 0.0f;
    const float scale = F32NORM ? *sc : 0.0f;
    // one point: r from its stencil values, rounded to FP32, summed, stored (e zeroed)
    auto point = [&](const Stencil5& x, int i, int j) {
        const double r = __fma_rn(-d, x.c, neighbour_sum<UNIT>(o, x.w, x.e, x.s, x.n, b2));
        const float rf = to_float_rn(r);
        if (F32NORM) {
            const float rs = __fmul_rn(rf, scale);
            acc32 = __fmaf_rn(rs, rs, acc32);
        } else {
            acc = __fma_rn(r, r, acc);
        }
        const int64_t at = (int64_t)j * pitch32 + i;
        r32[at] = rf;
        if (e32) e32[at] = 0.0f;
    };
    // a grid-stride walk, two points per step (both points' loads first), in walk order
    StrideWalk<NORM_THREADS> p(m, n);
    while (p.left >= 2) {
        const int i0 = p.i, j0 = p.j;
        p.next();
        const int i1 = p.i, j1 = p.j;
        p.next();
        const Stencil5 x0 = load5(psi + (int64_t)j0 * pitch + i0, pitch);
        const Stencil5 x1 = load5(psi + (int64_t)j1 * pitch + i1, pitch);
        point(x0, i0, j0);
        point(x1, i1, j1);
    }
    if (p.left > 0) point(load5(psi + (int64_t)p.j * pitch + p.i, pitch), p.i, p.j);
    if (F32NORM) acc = (double)acc32;
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

__global__ void __launch_bounds__(PX* PY)
    update64_kernel(double* __restrict__ psi, int m, int n, int64_t pitch,
                    const float* __restrict__ e32, int64_t pitch32)
{
    const FmaOps o = load_fma_ops();
    const int j = 1 + blockIdx.y * PY + threadIdx.y;
    const int i = 1 + blockIdx.x * PX + threadIdx.x;
    if (j > n - 2 || i > m - 2) return;
    double* c = psi + (int64_t)j * pitch + i;
    *c = fadd(o, *c, to_double_exact(e32[(int64_t)j * pitch32 + i]));
}

// ---- FP32 alone (the comparison point of the mixed solver) ----

// u32 := psi rounded to FP32 on every node (ring included), into two buffers.
__global__ void __launch_bounds__(PX* PY)
    to32_kernel(const double* __restrict__ psi, int m, int n, int64_t pitch, float* __restrict__ a,
                float* __restrict__ b, int64_t pitch32)
{
    const int j = blockIdx.y * PY + threadIdx.y;
    const int i = blockIdx.x * PX + threadIdx.x;
    if (j > n - 1 || i > m - 1) return;
    const float v = __double2float_rn(psi[(int64_t)j * pitch + i]);
    a[(int64_t)j * pitch32 + i] = v;
    if (b) b[(int64_t)j * pitch32 + i] = v;
}

// psi := (double) u32 on interior nodes.
__global__ void __launch_bounds__(PX* PY)
    to64_kernel(double* __restrict__ psi, int m, int n, int64_t pitch, const float* __restrict__ u,
                int64_t pitch32)
{
    const int j = 1 + blockIdx.y * PY + threadIdx.y;
    const int i = 1 + blockIdx.x * PX + threadIdx.x;
    if (j > n - 2 || i > m - 2) return;
    psi[(int64_t)j * pitch + i] = (double)u[(int64_t)j * pitch32 + i];
}

// Per-block sums (FP64) of the squared FP32 residual r = (E+W) + b2 (N+S) + q - d u.
template <bool UNIT>
__global__ void __launch_bounds__(NORM_THREADS, NORM_BLOCKS_PER_SM)
    defect32_sumsq_kernel(const float* __restrict__ u, const float* __restrict__ q, int m, int n,
                          int64_t pitch, float b2, float d, double* __restrict__ partials)
{
    double acc = 0.0;
    for (StrideWalk<NORM_THREADS> p(m, n); p.left > 0; p.next()) {
        const int64_t at = (int64_t)p.j * pitch + p.i;
        const float* c = u + at;
        const float s = __fadd_rn(nsum32(c[-1], c[1], c[-pitch], c[pitch], b2, UNIT), q[at]);
        const double r = (double)__fmaf_rn(-d, *c, s);
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

// The ring of every FP32 level buffer (u, q, r) of levels 0 .. count - 1 set to zero: thread k
// of block row l takes point k of level l's ring (row 0, row n - 1, column 0, column m - 1).
__global__ void zero_rings32_kernel(const BatchLevel<float>* __restrict__ lv)
{
    const BatchLevel<float> V = lv[blockIdx.y];
    const int m = V.m, n = V.n;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < 2 * m + 2 * n; k += gridDim.x * blockDim.x) {
        int64_t at;
        if (k < m) at = k;
        else if (k < 2 * m) at = (int64_t)(n - 1) * V.pitch + (k - m);
        else if (k < 2 * m + n) at = (int64_t)(k - 2 * m) * V.pitch;
        else at = (int64_t)(k - 2 * m - n) * V.pitch + (m - 1);
        V.u[at] = 0.0f;
        if (V.q) V.q[at] = 0.0f;
        if (V.r) V.r[at] = 0.0f;
    }
}

}  // namespace

cudaError_t launch_zero_rings32(const BatchLevel<float>* lv, int count, int max_side, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    const int per = 4 * max_side;
    zero_rings32_kernel<<<dim3((per + 255) / 256, count), 256, 0, s>>>(lv);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_to32(const Field& psi, float* a, float* b, int64_t pitch32, cudaStream_t s)
{
    const dim3 grid((psi.m + PX - 1) / PX, (psi.n + PY - 1) / PY), block(PX, PY);
    to32_kernel<<<grid, block, 0, s>>>(psi.p, psi.m, psi.n, psi.pitch, a, b, pitch32);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_to64(const Field& psi, const float* u, int64_t pitch32, cudaStream_t s)
{
    const dim3 grid((psi.m - 2 + PX - 1) / PX, (psi.n - 2 + PY - 1) / PY), block(PX, PY);
    to64_kernel<<<grid, block, 0, s>>>(psi.p, psi.m, psi.n, psi.pitch, u, pitch32);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_defect32_sumsq(const Field32& f, const float* q, const Coef& c, double* partials,
                                  cudaStream_t s)
{
    const int blocks = mixed_norm_blocks(f.m, f.n);
    if (c.unit_beta)
        defect32_sumsq_kernel<true><<<blocks, NORM_THREADS, 0, s>>>(f.p, q, f.m, f.n, f.pitch, (float)c.b2, (float)c.d, partials);
    else
        defect32_sumsq_kernel<false><<<blocks, NORM_THREADS, 0, s>>>(f.p, q, f.m, f.n, f.pitch, (float)c.b2, (float)c.d, partials);
    note_launch();
    return cudaGetLastError();
}

int mixed_norm_blocks(int m, int n) { return norm_blocks_for(m, n); }

cudaError_t launch_rb32(const Field32& f, const float* q, const Coef& c, bool gs, double w,
                        int colour, cudaStream_t s)
{
    const int per_row = (f.m - 2 + 1) / 2;
    const dim3 grid((per_row + BX - 1) / BX, (f.n - 2 + BY - 1) / BY), block(BX, BY);
    const float b2 = (float)c.b2, inv_d = (float)c.inv_d, wf = (float)w, omw = (float)(1.0 - w);
    if (c.unit_beta) {
        if (gs) rb32_kernel<true, true><<<grid, block, 0, s>>>(f.p, q, f.m, f.n, f.pitch, colour, b2, inv_d, wf, omw);
        else rb32_kernel<true, false><<<grid, block, 0, s>>>(f.p, q, f.m, f.n, f.pitch, colour, b2, inv_d, wf, omw);
    } else {
        if (gs) rb32_kernel<false, true><<<grid, block, 0, s>>>(f.p, q, f.m, f.n, f.pitch, colour, b2, inv_d, wf, omw);
        else rb32_kernel<false, false><<<grid, block, 0, s>>>(f.p, q, f.m, f.n, f.pitch, colour, b2, inv_d, wf, omw);
    }
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_defect32(const Field32& f, const float* q, float* r, const Coef& c,
                            cudaStream_t s)
{
    const dim3 grid((f.m - 2 + PX - 1) / PX, (f.n - 2 + PY - 1) / PY), block(PX, PY);
    if (c.unit_beta)
        defect32_kernel<true><<<grid, block, 0, s>>>(f.p, q, r, f.m, f.n, f.pitch, (float)c.b2, (float)c.d);
    else
        defect32_kernel<false><<<grid, block, 0, s>>>(f.p, q, r, f.m, f.n, f.pitch, (float)c.b2, (float)c.d);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_restrict32(const Field32& fine_r, float* qc, float* ec, int64_t pitch_c,
                              cudaStream_t s)
{
    const int mc = (fine_r.m - 1) / 2 + 1, nc = (fine_r.n - 1) / 2 + 1;
    const dim3 grid((mc - 2 + BX - 1) / BX, (nc - 2 + BY - 1) / BY);
    restrict32_kernel<<<grid, dim3(BX, BY), 0, s>>>(fine_r.p, fine_r.m, fine_r.n, fine_r.pitch, qc,
                                                      ec, pitch_c);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_prolong32(const Field32& fine_u, const float* ec, int64_t pitch_c,
                             cudaStream_t s)
{
    const int mc = (fine_u.m - 1) / 2 + 1;
    const dim3 grid((mc - 1 + BX - 1) / BX, (fine_u.n - 2 + BY - 1) / BY);
    prolong32_kernel<<<grid, dim3(BX, BY), 0, s>>>(fine_u.p, fine_u.m, fine_u.n, fine_u.pitch, ec,
                                                     pitch_c);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_coarse32(const Field32& u, const float* q, const double* ainv_t, cudaStream_t s)
{
    const int N = (u.m - 2) * (u.n - 2);
    int threads = ((N + 31) / 32) * 32;
    if (threads > 1024) threads = 1024;
    coarse32_kernel<<<1, threads, sizeof(double) * N, s>>>(u.p, q, u.m, u.n, u.pitch, ainv_t);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_defect64_to32(const Field& psi, const Coef& c, float* r32, float* e32,
                                 int64_t pitch32, double* partials, cudaStream_t s,
                                 const float* norm_scale)
{
    const int blocks = mixed_norm_blocks(psi.m, psi.n);
#define LAP_D64(U, F)                                                                            \
    defect64_to32_kernel<U, F><<<blocks, NORM_THREADS, 0, s>>>(psi.p, psi.m, psi.n, psi.pitch, c.b2, \
                                                               c.d, r32, e32, pitch32, partials, \
                                                               norm_scale)
    if (c.unit_beta) {
        if (norm_scale) LAP_D64(true, true); else LAP_D64(true, false);
    } else {
        if (norm_scale) LAP_D64(false, true); else LAP_D64(false, false);
    }
#undef LAP_D64
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_update64(const Field& psi, const float* e32, int64_t pitch32, cudaStream_t s)
{
    const dim3 grid((psi.m - 2 + PX - 1) / PX, (psi.n - 2 + PY - 1) / PY), block(PX, PY);
    update64_kernel<<<grid, block, 0, s>>>(psi.p, psi.m, psi.n, psi.pitch, e32, pitch32);
    note_launch();
    return cudaGetLastError();
}

}  // namespace lap
