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

// The point methods' sweeps on a shared-memory copy, each returning the thread's largest
// |new - old| (as ordered bits) when `track`: the same per-point expressions as the
// multi-CTA kernels (Eqs. 5-7), in lexicographic wavefronts, red-black colours or Jacobi.
template <bool UNIT_BETA, bool POW2, bool GS>
__device__ __forceinline__ unsigned long long sweep_lex(const FmaOps& o, double* u, int m, int n,
                                                        double b2, double inv_d, int shift, double w,
                                                        double one_minus_w, bool track)
{
    unsigned long long dl = 0;
    const int last_diag = (m - 2) + (n - 2);
    for (int k = 2; k <= last_diag; ++k) {
        const int i_lo = k - (n - 2) > 1 ? k - (n - 2) : 1;
        const int i_hi = k - 1 < m - 2 ? k - 1 : m - 2;
        for (int i = i_lo + (int)threadIdx.x; i <= i_hi; i += blockDim.x) {
            double* c = u + (k - i) * m + i;
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
    return dl;
}

template <bool UNIT_BETA, bool POW2, bool GS>
__device__ __forceinline__ unsigned long long sweep_rb(const FmaOps& o, double* u, int m, int n,
                                                       double b2, double inv_d, int shift, double w,
                                                       double one_minus_w, bool track)
{
    unsigned long long dl = 0;
    const int half_w = (m - 2 + 1) / 2, rows = n - 2;
    for (int colour = 0; colour < 2; ++colour) {
        for (int k = threadIdx.x; k < rows * half_w; k += blockDim.x) {
            const int j = 1 + k / half_w;
            const int i = 1 + ((1 + j + colour) & 1) + 2 * (k % half_w);
            if (i > m - 2) continue;
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
    return dl;
}

template <bool UNIT_BETA, bool POW2>
__device__ __forceinline__ unsigned long long sweep_jacobi(const FmaOps& o, const double* a, double* b,
                                                           int m, int n, double b2, double inv_d,
                                                           int shift, bool track)
{
    unsigned long long dl = 0;
    const int mi = m - 2;
    for (int k = threadIdx.x; k < mi * (n - 2); k += blockDim.x) {
        const int i = 1 + k % mi, j = 1 + k / mi;
        const double* c = a + j * m + i;
        const double s = neighbour_sum<UNIT_BETA>(o, c[-1], c[1], c[-m], c[m], b2);
        const double nv = times_inv_d<POW2>(o, s, inv_d, shift);
        b[j * m + i] = nv;
        if (track) {
            const unsigned long long bb = abs_bits(fadd(o, nv, -*c));
            dl = bb > dl ? bb : dl;
        }
    }
    __syncthreads();
    return dl;
}

// nsweeps lexicographic sweeps (one check period) in one CTA; maxd gets the last sweep's
// max |new - old|.
template <bool UNIT_BETA, bool POW2, bool GS>
__global__ void __launch_bounds__(LEX_THREADS)
    lex_sweeps_kernel(double* __restrict__ psi, int m, int n, int64_t pitch, int nsweeps,
                      double b2, double inv_d, int shift, double w, double one_minus_w,
                      unsigned long long* __restrict__ maxd)
{
    const FmaOps o = load_fma_ops();
    b2 = in_reg(o, b2);
    inv_d = in_reg(o, inv_d);
    w = in_reg(o, w);
    one_minus_w = in_reg(o, one_minus_w);
    extern __shared__ double u[];  // dense m x n copy
    const int tid = threadIdx.x;
    for (int k = tid; k < m * n; k += blockDim.x) u[k] = psi[(int64_t)(k / m) * pitch + k % m];
    __syncthreads();
    unsigned long long dl = 0;
    for (int sweep = 0; sweep < nsweeps; ++sweep)
        dl = sweep_lex<UNIT_BETA, POW2, GS>(o, u, m, n, b2, inv_d, shift, w, one_minus_w,
                                            maxd && sweep == nsweeps - 1);
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

// ---- a whole solve in one CTA (small grids, the paper's stopping rule, Eq. 16) ----
// KIND 0 Jacobi, 1 red-black, 2 lexicographic. Runs check periods (check_every iterations, the
// last shortened to max_iter) until max |psi^{k+1} - psi^k| over the period's last iteration
// is <= tol (or not finite): the host loop's rule, on a block-wide max of the same bits.
template <int KIND, bool UNIT_BETA, bool POW2, bool GS>
__global__ void __launch_bounds__(LEX_THREADS)
    solve_cta_kernel(double* __restrict__ psi, int m, int n, int64_t pitch, double b2, double inv_d,
                     int shift, const double* __restrict__ wslot, LoopState* __restrict__ st)
{
    const FmaOps o = load_fma_ops();
    const double w = GS ? 1.0 : wslot[0], one_minus_w = GS ? 0.0 : wslot[1];
    b2 = in_reg(o, b2);
    inv_d = in_reg(o, inv_d);
    extern __shared__ double u[];
    double* a = u;
    double* b = KIND == 0 ? u + m * n : u;
    const int tid = threadIdx.x;
    for (int k = tid; k < m * n; k += blockDim.x) {
        const double v = psi[(int64_t)(k / m) * pitch + k % m];
        a[k] = v;
        if (KIND == 0) b[k] = v;
    }
    __shared__ unsigned long long red[LEX_THREADS / 32];
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
        unsigned long long dl = 0;
        for (long long s = 0; s < nst; ++s) {
            const bool track = s == nst - 1;
            if (KIND == 0) {
                dl = sweep_jacobi<UNIT_BETA, POW2>(o, a, b, m, n, b2, inv_d, shift, track);
                double* t = a;
                a = b;
                b = t;
            } else if (KIND == 1) {
                dl = sweep_rb<UNIT_BETA, POW2, GS>(o, a, m, n, b2, inv_d, shift, w, one_minus_w, track);
            } else {
                dl = sweep_lex<UNIT_BETA, POW2, GS>(o, a, m, n, b2, inv_d, shift, w, one_minus_w, track);
            }
        }
        k += nst;
        dl = warp_max_u64(dl);
        if ((tid & 31) == 0) red[tid >> 5] = dl;
        __syncthreads();
        if (tid < 32) {
            unsigned long long v = tid < LEX_THREADS / 32 ? red[tid] : 0ull;
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
    for (int q = tid; q < mi * (n - 2); q += blockDim.x) {
        const int i = 1 + q % mi, j = 1 + q / mi;
        psi[(int64_t)j * pitch + i] = a[j * m + i];
    }
    if (tid == 0) {
        st->k = k;
        st->status = status;
        st->last_check = val;
    }
}

}  // namespace

size_t lex_smem_bytes(int m, int n) { return sizeof(double) * (size_t)m * (size_t)n; }
int64_t lex_max_points() { return 224 * 1024 / sizeof(double); }

// Raise the dynamic shared-memory limit of every instantiation once per device (outside any
// stream capture); later launches with at most that much shared memory skip it.
static std::atomic<size_t> g_lex_smem_set[ATTR_DEVICES];

cudaError_t prepare_lex_kernels(size_t smem)
{
    const int dev = attr_slot();
    if (smem <= 48 * 1024 || (dev >= 0 && smem <= g_lex_smem_set[dev].load()))
        return cudaSuccess;
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
#define LAP_SOLVE_ATTR(K, G)                                                                    \
    if (e == cudaSuccess) e = cudaFuncSetAttribute(solve_cta_kernel<K, true, true, G>, a, v);   \
    if (e == cudaSuccess) e = cudaFuncSetAttribute(solve_cta_kernel<K, true, false, G>, a, v);  \
    if (e == cudaSuccess) e = cudaFuncSetAttribute(solve_cta_kernel<K, false, true, G>, a, v);  \
    if (e == cudaSuccess) e = cudaFuncSetAttribute(solve_cta_kernel<K, false, false, G>, a, v);
    LAP_SOLVE_ATTR(0, true)
    LAP_SOLVE_ATTR(1, true)
    LAP_SOLVE_ATTR(1, false)
    LAP_SOLVE_ATTR(2, true)
    LAP_SOLVE_ATTR(2, false)
#undef LAP_SOLVE_ATTR
    if (e == cudaSuccess) attr_record(g_lex_smem_set, dev, smem);
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

cudaError_t launch_solve_cta(const Field& f, const Coef& c, int kind, bool gs, const double* wslot,
                             LoopState* st, cudaStream_t s)
{
    const size_t smem = (kind == 0 ? 2 : 1) * lex_smem_bytes(f.m, f.n);
    cudaError_t err = prepare_lex_kernels(smem);
    const bool p2 = c.inv_d_shift > 0;
#define LAP_SC(K, G)                                                                             \
    do {                                                                                         \
        if (err != cudaSuccess) break;                                                           \
        if (c.unit_beta) {                                                                       \
            if (p2) solve_cta_kernel<K, true, true, G><<<1, LEX_THREADS, smem, s>>>(f.p, f.m, f.n, f.pitch, c.b2, c.inv_d, c.inv_d_shift, wslot, st); \
            else solve_cta_kernel<K, true, false, G><<<1, LEX_THREADS, smem, s>>>(f.p, f.m, f.n, f.pitch, c.b2, c.inv_d, c.inv_d_shift, wslot, st); \
        } else {                                                                                 \
            if (p2) solve_cta_kernel<K, false, true, G><<<1, LEX_THREADS, smem, s>>>(f.p, f.m, f.n, f.pitch, c.b2, c.inv_d, c.inv_d_shift, wslot, st); \
            else solve_cta_kernel<K, false, false, G><<<1, LEX_THREADS, smem, s>>>(f.p, f.m, f.n, f.pitch, c.b2, c.inv_d, c.inv_d_shift, wslot, st); \
        }                                                                                        \
    } while (0)
    if (kind == 0) LAP_SC(0, true);
    else if (kind == 1) { if (gs) LAP_SC(1, true); else LAP_SC(1, false); }
    else { if (gs) LAP_SC(2, true); else LAP_SC(2, false); }
#undef LAP_SC
    note_launch();
    if (err != cudaSuccess) return err;
    return cudaGetLastError();
}

}  // namespace lap
