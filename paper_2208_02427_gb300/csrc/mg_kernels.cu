// mg_kernels.cu -- multigrid transfer operators and the coarsest-grid solve.
//
// V-cycle steps 3/6 (restriction of the residual), 8/10 (interpolation of the coarse
// correction, Eq. 13) and 7 (the coarsest correction equation, Eq. 15, solved exactly).
// The paper names no operators: full weighting and bilinear interpolation are used, and
// coarse levels carry (E+W) + beta^2 (N+S) - d e + q = 0 with q = 4 FW(r_fine), the
// fine residual r = dx^2 R scaled to the doubled spacing.
#include "lap_device.cuh"
#include "lap_internal.cuh"

namespace lap {

namespace {

constexpr int MG_BX = 64, MG_BY = 4;

// qc(I,J) = 0.25 ((4 c + 2 edges) + corners). Since scaling by 2 is exact,
// round(4c + 2e) = 2 round(2c + e), so t = fma(2, c, e) and u = fma(2, t, corners)
// reproduce the two rounded additions of the written expression.
__global__ void __launch_bounds__(MG_BX* MG_BY)
    restrict_kernel(const double* __restrict__ r, int mf, int nf, int64_t pf,
                    double* __restrict__ qc, double* __restrict__ ec, int64_t pc)
{
    const FmaOps o = load_fma_ops();
    const int mc = (mf - 1) / 2 + 1, nc = (nf - 1) / 2 + 1;
    const int I = 1 + blockIdx.x * MG_BX + threadIdx.x;
    const int J = 1 + blockIdx.y * MG_BY + threadIdx.y;
    if (I > mc - 2 || J > nc - 2) return;
    const double* c = r + (int64_t)(2 * J) * pf + 2 * I;
    const double edges = fadd(o, fadd(o, c[-1], c[1]), fadd(o, c[-pf], c[pf]));
    const double corners =
        fadd(o, fadd(o, c[-pf - 1], c[-pf + 1]), fadd(o, c[pf - 1], c[pf + 1]));
    const double two = in_reg(o, 2.0);
    const double t = __fma_rn(two, c[0], edges);
    const double u = __fma_rn(two, t, corners);
    const int64_t at = (int64_t)J * pc + I;
    qc[at] = scale_down_pow2(o, u, 2, 0.25);
    if (ec) ec[at] = 0.0;
}

// Thread (pair I, fine row j) adds the interpolated correction to fine points (2I, j)
// and (2I + 1, j): coincident nodes copy, edges average two coarse values, centres four
// (pairs along x first).
__global__ void __launch_bounds__(MG_BX* MG_BY)
    prolong_add_kernel(double* __restrict__ u, int mf, int nf, int64_t pf,
                       const double* __restrict__ ec, int64_t pc)
{
    const FmaOps o = load_fma_ops();
    const int I = blockIdx.x * MG_BX + threadIdx.x;  // coarse column 0 .. mc-2
    const int j = 1 + blockIdx.y * MG_BY + threadIdx.y;
    const int mc = (mf - 1) / 2 + 1;
    if (I > mc - 2 || j > nf - 2) return;
    const int J = j >> 1;
    const double* a = ec + (int64_t)J * pc + I;
    const int i0 = 2 * I, i1 = 2 * I + 1;
    double* row = u + (int64_t)j * pf;
    if ((j & 1) == 0) {
        if (i0 >= 1) row[i0] = fadd(o, row[i0], a[0]);
        if (i1 <= mf - 2) row[i1] = fadd(o, row[i1], scale_down_pow2(o, fadd(o, a[0], a[1]), 1, 0.5));
    } else {
        if (i0 >= 1)
            row[i0] = fadd(o, row[i0], scale_down_pow2(o, fadd(o, a[0], a[pc]), 1, 0.5));
        if (i1 <= mf - 2) {
            const double s = fadd(o, fadd(o, a[0], a[1]), fadd(o, a[pc], a[pc + 1]));
            row[i1] = fadd(o, row[i1], scale_down_pow2(o, s, 2, 0.25));
        }
    }
}

// One CTA: b = q + ring terms (weight 1 across x, beta^2 across y), u = A^-1 b with the
// inverse precomputed on the host, stored transposed so that step l reads a row.
__global__ void __launch_bounds__(1024)
    coarse_solve_kernel(double* __restrict__ u, const double* __restrict__ q, int m, int n,
                        int64_t pitch, double b2, const double* __restrict__ ainv_t)
{
    extern __shared__ double b[];
    const int mi = m - 2, N = mi * (n - 2);
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        const int i = 1 + k % mi, j = 1 + k / mi;
        const int64_t at = (int64_t)j * pitch + i;
        double v = q ? q[at] : 0.0;
        if (i == 1) v = __dadd_rn(v, u[at - 1]);
        if (i == m - 2) v = __dadd_rn(v, u[at + 1]);
        if (j == 1) v = __fma_rn(b2, u[at - pitch], v);
        if (j == n - 2) v = __fma_rn(b2, u[at + pitch], v);
        b[k] = v;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        double x = 0.0;
        for (int l = 0; l < N; ++l) x = __fma_rn(ainv_t[(int64_t)l * N + k], b[l], x);
        const int i = 1 + k % mi, j = 1 + k / mi;
        u[(int64_t)j * pitch + i] = x;
    }
}

}  // namespace

cudaError_t launch_restrict(const Field& fine_r, double* qc, double* ec, int64_t pitch_c,
                            cudaStream_t s)
{
    const int mc = (fine_r.m - 1) / 2 + 1, nc = (fine_r.n - 1) / 2 + 1;
    const dim3 grid((mc - 2 + MG_BX - 1) / MG_BX, (nc - 2 + MG_BY - 1) / MG_BY);
    restrict_kernel<<<grid, dim3(MG_BX, MG_BY), 0, s>>>(fine_r.p, fine_r.m, fine_r.n, fine_r.pitch,
                                                         qc, ec, pitch_c);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_prolong_add(const Field& fine_u, const double* ec, int64_t pitch_c,
                               cudaStream_t s)
{
    const int mc = (fine_u.m - 1) / 2 + 1;
    const dim3 grid((mc - 1 + MG_BX - 1) / MG_BX, (fine_u.n - 2 + MG_BY - 1) / MG_BY);
    prolong_add_kernel<<<grid, dim3(MG_BX, MG_BY), 0, s>>>(fine_u.p, fine_u.m, fine_u.n,
                                                            fine_u.pitch, ec, pitch_c);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_coarse_solve(const Field& u, const double* q, const Coef& c,
                                const double* ainv_t, cudaStream_t s)
{
    const int N = (u.m - 2) * (u.n - 2);
    int threads = ((N + 31) / 32) * 32;
    if (threads > 1024) threads = 1024;
    coarse_solve_kernel<<<1, threads, sizeof(double) * N, s>>>(u.p, q, u.m, u.n, u.pitch, c.b2,
                                                                ainv_t);
    note_launch();
    return cudaGetLastError();
}

}  // namespace lap
