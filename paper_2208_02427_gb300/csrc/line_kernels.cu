// line_kernels.cu -- zebra line relaxation (SLOR / ADI half-sweeps, Eqs. 8-10).
//
// Every line of one colour is an independent tridiagonal system with constant
// coefficients, -alpha x_{k-1} + delta x_k - alpha x_{k+1} = r_k (k = 1..N, Dirichlet
// ends moved into r_1 and r_N). One CTA solves one line:
//   1. the right-hand side is built from the two neighbouring lines (coalesced along the
//      line for x-lines) into shared memory, laid out chunk by chunk;
//   2. thread p runs the Thomas algorithm over its chunk of L unknowns with zero ends:
//      y'_o = fma(alpha, y'_{o-1}, r_o) * inv_den_o, y_o = fma(cpos_o, y_{o+1}, y'_o);
//   3. the P-1 separator unknowns between chunks satisfy a tridiagonal system whose
//      coefficients come from the chunk influence vectors gL, gR; it is solved exactly by
//      parallel cyclic reduction (one thread per separator, ceil(log2(P-1)) levels);
//   4. every chunk adds x_left gL + x_right gR (the exact superposition) and the line is
//      relaxed (form A: psi + w (x - psi), Eq. 9) or stored (form B, Eq. 10) and written.
// Only the right-hand side depends on the data, so inv_den, cpos, gL, gR and the
// cyclic-reduction multipliers are computed once on the host per (N, alpha, delta).
// Per unknown this costs 3 FP64 operations in the chunk solve and 2 in the fix-up, plus
// 1-3 for the right-hand side and 0-2 for the relaxation.
#include "lap_device.cuh"
#include "lap_internal.cuh"

namespace lap {

namespace {

template <int FORM, bool UNIT_CROSS>
__global__ void __launch_bounds__(256)
    line_colour_kernel(double* __restrict__ psi, int64_t sa, int64_t sx, int first_line,
                       const LineTables t, double cross, double w, double dmw, double wcross)
{
    const FmaOps o = load_fma_ops();
    extern __shared__ double sm[];
    const int N = t.N, L = t.L, P = t.P, S = P - 1, Ls = t.stride;
    double* lane = sm;              // chunk p occupies lane[p*Ls .. p*Ls + L]; slot L = separator
    double* rho = sm + (size_t)P * Ls;  // 2*S: cyclic-reduction double buffer
    double* base = psi + (int64_t)(first_line + 2 * (int)blockIdx.x) * sx;
    const double alpha = in_reg(o, t.alpha);
    cross = in_reg(o, cross);
    w = in_reg(o, w);
    dmw = in_reg(o, dmw);
    wcross = in_reg(o, wcross);

    // 1. right-hand side; the Dirichlet ends' terms are added after the loop by the threads
    //    that wrote those entries (the same fma, applied last, as written per point: a test
    //    per point would let the compiler issue both fmas for every point)
    for (int k = 1 + threadIdx.x; k <= N; k += blockDim.x) {
        const int64_t at = (int64_t)k * sa;
        const double nb = fadd(o, base[at - sx], base[at + sx]);
        double r;
        if (FORM == 0)
            r = UNIT_CROSS ? nb : fmul(o, cross, nb);
        else
            r = __fma_rn(dmw, base[at], fmul(o, wcross, nb));
        const int g = k - 1, p = g / (L + 1);
        lane[p * Ls + (g - p * (L + 1))] = r;
    }
    if (threadIdx.x == 0) lane[0] = __fma_rn(alpha, base[0], lane[0]);  // k = 1: chunk 0, slot 0
    if (threadIdx.x == (N - 1) % blockDim.x) {  // k = N, written by this thread
        const int g = N - 1, p = g / (L + 1);
        double* e = lane + p * Ls + (g - p * (L + 1));
        *e = __fma_rn(alpha, base[(int64_t)(N + 1) * sa], *e);
    }
    __syncthreads();

    // 2. Thomas inside each chunk, zero ends
    const int p = threadIdx.x;
    if (p < P) {
        const int len = p == P - 1 ? t.Ll : L;
        double* y = lane + p * Ls;
        double prev = 0.0;
        for (int q = 0; q < len; ++q) {
            prev = fmul(o, __fma_rn(alpha, prev, y[q]), t.inv_den[q]);
            y[q] = prev;
        }
        for (int q = len - 2; q >= 0; --q) {
            prev = __fma_rn(t.cpos[q], prev, y[q]);
            y[q] = prev;
        }
    }
    __syncthreads();

    // 3. separators: rho_p = r_sep + alpha (y_last(chunk p) + y_first(chunk p+1))
    if (p < S) {
        const double* yl = lane + p * Ls;
        rho[p] = __fma_rn(alpha, fadd(o, yl[L - 1], yl[Ls]), yl[L]);
    }
    __syncthreads();
    double* cur = rho;
    double* nxt = rho + S;
    for (int lev = 0, s = 1; lev < t.levels; ++lev, s <<= 1) {
        if (p < S) {
            double v = cur[p];
            if (p >= s) v = __fma_rn(t.k1[lev * S + p], cur[p - s], v);
            if (p + s < S) v = __fma_rn(t.k2[lev * S + p], cur[p + s], v);
            nxt[p] = v;
        }
        __syncthreads();
        double* tmp = cur;
        cur = nxt;
        nxt = tmp;
    }
    if (p < S) cur[p] = fmul(o, cur[p], t.invb[p]);
    __syncthreads();

    // 4. superpose the separator values onto each chunk
    if (p < P) {
        const bool last = p == P - 1;
        const int len = last ? t.Ll : L;
        const double* gl = last ? t.gLl : t.gL;
        const double* gr = last ? t.gRl : t.gR;
        double* y = lane + p * Ls;
        if (p >= 1) {
            const double xl = cur[p - 1];
            for (int q = 0; q < len; ++q) y[q] = __fma_rn(xl, gl[q], y[q]);
        }
        if (p < S) {
            const double xr = cur[p];
            for (int q = 0; q < len; ++q) y[q] = __fma_rn(xr, gr[q], y[q]);
            y[L] = xr;
        }
    }
    __syncthreads();

    // 5. relax and write back
    for (int k = 1 + threadIdx.x; k <= N; k += blockDim.x) {
        const int g = k - 1, c = g / (L + 1);
        const double x = lane[c * Ls + (g - c * (L + 1))];
        double* dst = base + (int64_t)k * sa;
        if (FORM == 0) {
            const double old = *dst;
            *dst = __fma_rn(w, fadd(o, x, -old), old);
        } else {
            *dst = x;
        }
    }
}

}  // namespace

size_t line_smem_bytes(const LineTables& t)
{
    return sizeof(double) * ((size_t)t.P * t.stride + 2 * (size_t)(t.P > 1 ? t.P - 1 : 0));
}

int line_threads(const LineTables& t)
{
    int th = ((t.P + 31) / 32) * 32;
    return th < 64 ? 64 : th;
}

// Raise the dynamic shared-memory limit of every line-kernel instantiation to `smem`
// on the current device (done outside stream capture; launches below only repeat it when a
// larger line comes).
static std::atomic<size_t> g_line_smem_set[ATTR_DEVICES];

cudaError_t prepare_line_kernels(size_t smem)
{
    const int dev = attr_slot();
    if (smem <= 48 * 1024 || (dev >= 0 && smem <= g_line_smem_set[dev].load()))
        return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(line_colour_kernel<0, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(line_colour_kernel<0, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(line_colour_kernel<1, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) attr_record(g_line_smem_set, dev, smem);
    return e;
}

namespace {

// dst[c][r] = src[r][c] for r < rows, c < cols: 32x32 tiles through shared memory (one
// column of padding), reads and writes coalesced along rows.
constexpr int TT = 32, TR = 8;
__global__ void __launch_bounds__(TT* TR)
    transpose_kernel(const double* __restrict__ src, int64_t sp, double* __restrict__ dst,
                     int64_t dp, int rows, int cols)
{
    __shared__ double tile[TT][TT + 1];
    const int c0 = blockIdx.x * TT, r0 = blockIdx.y * TT;
    for (int k = threadIdx.y; k < TT; k += TR) {
        const int r = r0 + k, c = c0 + threadIdx.x;
        if (r < rows && c < cols) tile[k][threadIdx.x] = src[(int64_t)r * sp + c];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < TT; k += TR) {
        const int c = c0 + k, r = r0 + threadIdx.x;
        if (r < rows && c < cols) dst[(int64_t)c * dp + r] = tile[threadIdx.x][k];
    }
}

}  // namespace

cudaError_t launch_transpose(const double* src, int64_t sp, double* dst, int64_t dp, int rows,
                             int cols, cudaStream_t s)
{
    const dim3 grid((cols + TT - 1) / TT, (rows + TT - 1) / TT), block(TT, TR);
    transpose_kernel<<<grid, block, 0, s>>>(src, sp, dst, dp, rows, cols);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_line_colour(double* psi, int64_t sa, int64_t sx, int first_line, int count,
                               const LineTables& t, int form, double cross, double w,
                               cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    const size_t smem = line_smem_bytes(t);
    const int threads = line_threads(t);
    const double d = t.delta;
    const double dmw = d * (1.0 - w), wcross = w * cross;
    const bool unit = cross == 1.0;
    cudaError_t err = cudaSuccess;
#define LAP_LINE(F, U)                                                                          \
    do {                                                                                        \
        auto kern = line_colour_kernel<F, U>;                                                   \
        err = prepare_line_kernels(smem);                                                       \
        if (err == cudaSuccess)                                                                 \
            kern<<<count, threads, smem, s>>>(psi, sa, sx, first_line, t, cross, w, dmw, wcross); \
    } while (0)
    if (form == 0) {
        if (unit) LAP_LINE(0, true); else LAP_LINE(0, false);
    } else {
        LAP_LINE(1, false);
    }
#undef LAP_LINE
    note_launch();
    if (err != cudaSuccess) return err;
    return cudaGetLastError();
}

}  // namespace lap
