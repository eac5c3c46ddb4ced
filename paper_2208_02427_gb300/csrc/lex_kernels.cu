// lex_kernels.cu -- Gauss-Seidel and SOR in the paper's lexicographic order (Eqs. 6-7).
//
// Eq. 6 updates psi_{i,j} with psi_{i-1,j} and psi_{i,j-1} already new. All points of an
// anti-diagonal i + j = k depend only on diagonal k - 1 (new) and k + 1 (old), so a sweep is
// a wavefront of (m-2) + (n-2) - 1 diagonals, each updated in parallel; this visits points in
// an order equivalent to the lexicographic one (same values, bitwise). One CTA holds the
// whole field in shared memory and runs a whole check period of sweeps; grids up to
// lex_max_points() points (the paper's chamber problem is 425).
#include "lap_device.cuh"
#include "lap_internal.cuh"

namespace lap {

namespace {

constexpr int LEX_THREADS = 512;

template <bool UNIT_BETA, bool POW2, bool GS>
__global__ void __launch_bounds__(LEX_THREADS)
    lex_sweeps_kernel(double* __restrict__ psi, int m, int n, int64_t pitch, int nsweeps,
                      double b2, double inv_d, int shift, double w, double one_minus_w,
                      unsigned long long* __restrict__ maxd)
{
    const FmaOps o = load_fma_ops();
    extern __shared__ double u[];  // dense m x n copy
    const int tid = threadIdx.x;
    for (int k = tid; k < m * n; k += blockDim.x) u[k] = psi[(int64_t)(k / m) * pitch + k % m];
    __syncthreads();
    unsigned long long dl = 0;
    const int last_diag = (m - 2) + (n - 2);
    for (int sweep = 0; sweep < nsweeps; ++sweep) {
        const bool track = maxd && sweep == nsweeps - 1;
        for (int k = 2; k <= last_diag; ++k) {
            const int i_lo = k - (n - 2) > 1 ? k - (n - 2) : 1;
            const int i_hi = k - 1 < m - 2 ? k - 1 : m - 2;
            for (int i = i_lo + tid; i <= i_hi; i += blockDim.x) {
                const int j = k - i;
                double* c = u + j * m + i;
                const double s = neighbour_sum<UNIT_BETA>(o, c[-1], c[1], c[-m], c[m], b2);
                const double g = times_inv_d<POW2>(o, s, inv_d, shift);
                const double old = *c;
                const double nv = GS ? g : __fma_rn(w, g, fmul(o, one_minus_w, old));
                *c = nv;
                if (track) {
                    const unsigned long long b = abs_bits(fadd(o, nv, -old));
                    dl = b > dl ? b : dl;
                }
            }
            __syncthreads();
        }
    }
    const int mi = m - 2;  // write back the interior only: the ring is never written
    for (int k = tid; k < mi * (n - 2); k += blockDim.x) {
        const int i = 1 + k % mi, j = 1 + k / mi;
        psi[(int64_t)j * pitch + i] = u[j * m + i];
    }
    if (maxd) {
        dl = warp_max_u64(dl);
        if ((tid & 31) == 0 && dl) atomicMax(maxd, dl);
    }
}

}  // namespace

size_t lex_smem_bytes(int m, int n) { return sizeof(double) * (size_t)m * (size_t)n; }
int64_t lex_max_points() { return 224 * 1024 / sizeof(double); }

// Raise the dynamic shared-memory limit of every instantiation once (outside any stream
// capture); later launches with at most that much shared memory skip it.
static size_t g_lex_smem_set = 48 * 1024;

cudaError_t prepare_lex_kernels(size_t smem)
{
    if (smem <= g_lex_smem_set) return cudaSuccess;
    const int v = (int)smem;
    const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaFuncSetAttribute(lex_sweeps_kernel<true, true, true>, a, v);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(lex_sweeps_kernel<true, true, false>, a, v);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(lex_sweeps_kernel<true, false, true>, a, v);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(lex_sweeps_kernel<true, false, false>, a, v);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(lex_sweeps_kernel<false, true, true>, a, v);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(lex_sweeps_kernel<false, true, false>, a, v);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(lex_sweeps_kernel<false, false, true>, a, v);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(lex_sweeps_kernel<false, false, false>, a, v);
    if (e == cudaSuccess) g_lex_smem_set = smem;
    return e;
}

cudaError_t launch_lex_sweeps(const Field& f, const Coef& c, bool gs, double w, int nsweeps,
                              unsigned long long* maxd, cudaStream_t s)
{
    const size_t smem = lex_smem_bytes(f.m, f.n);
    const double omw = 1.0 - w;
    cudaError_t err = prepare_lex_kernels(smem);
#define LAP_LEX(UB, P2, G)                                                                        \
    do {                                                                                          \
        auto kern = lex_sweeps_kernel<UB, P2, G>;                                                 \
        if (err == cudaSuccess)                                                                   \
            kern<<<1, LEX_THREADS, smem, s>>>(f.p, f.m, f.n, f.pitch, nsweeps, c.b2, c.inv_d,       \
                                              c.inv_d_shift, w, omw, maxd);    \
    } while (0)
    const bool p2 = c.inv_d_shift > 0;
    if (c.unit_beta) {
        if (p2) { if (gs) LAP_LEX(true, true, true); else LAP_LEX(true, true, false); }
        else { if (gs) LAP_LEX(true, false, true); else LAP_LEX(true, false, false); }
    } else {
        if (p2) { if (gs) LAP_LEX(false, true, true); else LAP_LEX(false, true, false); }
        else { if (gs) LAP_LEX(false, false, true); else LAP_LEX(false, false, false); }
    }
#undef LAP_LEX
    note_launch();
    if (err != cudaSuccess) return err;
    return cudaGetLastError();
}

}  // namespace lap
