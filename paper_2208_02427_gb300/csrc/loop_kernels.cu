// loop_kernels.cu -- the device-side stopping test of a solve loop, and a self-check.
//
// loop_decide_kernel runs inside the body of a conditional CUDA graph node: after each check
// period it applies the host loop's stopping rule (Eq. 16 or the L2 rules) and sets the
// loop's condition. check_rounding_kernel compares the residual kernels' integer-pipe
// FP64 -> FP32 rounding with the conversion instruction. fp64_rate_kernel measures the FP64
// fused multiply-add issue rate, the peak that the FP64-bound kernels are measured against.
#include "lap_device.cuh"
#include "lap_internal.cuh"

namespace lap {

namespace {

// The stopping test of a device-resident solve loop (Eq. 16 or the L2 rules), run after each
// period inside the loop body of a conditional CUDA graph: the same arithmetic as the host's
// test; clears the loop's condition when the solve stops or the next period would pass
// max_iter.
__global__ void loop_decide_kernel(LoopState* st, const double* __restrict__ nrm,
                                   const unsigned long long* __restrict__ maxd,
                                   const float* __restrict__ scale, cudaGraphConditionalHandle h)
{
    if (threadIdx.x != 0) return;
    st->k += st->steps;
    double val, nr = st->last_nr;
    bool conv;
    if (st->mode == 2) {
        val = __longlong_as_double((long long)*maxd);
        conv = val <= st->tol;
    } else {
        nr = nrm[1];
        if (scale) nr = nr / (double)*scale;
        val = st->mode == 0 ? nr / st->r0 : nr;
        conv = st->mode == 0 ? nr <= st->tol * st->r0 : nr <= st->tol;
    }
    st->last_check = val;
    st->last_nr = nr;
    int status = 1;  // LAP_MAXITER
    if (!isfinite(val)) status = 2;  // LAP_DIVERGED
    else if (conv) status = 0;       // LAP_CONVERGED
    st->status = status;
    cudaGraphSetConditional(h, status == 1 && st->k + st->steps <= st->max_iter ? 1u : 0u);
}

// The loop test of a device-resident batched solve, run after each cycle inside the body of
// a conditional CUDA graph: st[0] counts the cycles, st[1] is the cap; the loop goes on while
// some problem is still running (the convergence kernel counts them down) and the cap is not
// reached.
__global__ void batch_loop_decide_kernel(long long* st, const int* __restrict__ remaining,
                                         cudaGraphConditionalHandle h)
{
    if (threadIdx.x != 0) return;
    const long long k = st[0] + 1;
    st[0] = k;
    cudaGraphSetConditional(h, *remaining > 0 && k < st[1] ? 1u : 0u);
}

}  // namespace

namespace {

__device__ __forceinline__ unsigned long long mix64(unsigned long long x)
{
    x += 0x9e3779b97f4a7c15ull;
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
    return x ^ (x >> 31);
}

// to_float_rn against the conversion instruction, and scale_down_pow2 against the FP64
// multiply by 2^-s (s = 1..4), on `count` doubles drawn from seed: random bit patterns,
// exponents near the FP32 range's ends, exact ties, all-ones fractions, +-0 and FP64
// subnormals, and exponents within a few of zero, in turn; and to_double_exact against the
// conversion on random FP32 bit patterns, every eighth one with a zero exponent (+-0 or
// an FP32 subnormal).
__global__ void check_rounding_kernel(long long count, unsigned long long seed,
                                      unsigned long long* bad)
{
    const FmaOps o = load_fma_ops();
    unsigned long long local = 0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < count;
         k += (long long)gridDim.x * blockDim.x) {
        const unsigned long long r = mix64(seed ^ (unsigned long long)k), r2 = mix64(r);
        const unsigned long long sign_frac = r & 0x800fffffffffffffull;
        unsigned long long b;
        switch (k % 6) {
        case 0: b = r; break;
        case 1: b = sign_frac | ((unsigned long long)(1023 - 130 + (r2 % 270)) << 52); break;
        case 2: b = (r & 0x800fffffe0000000ull) | 0x10000000ull | ((unsigned long long)(1023 + (int)(r2 % 60) - 30) << 52); break;
        case 3: b = (r & 0xfff0000000000000ull) | 0x000fffffffffffffull; break;
        case 4: b = (r2 & 3) ? (r & 0x8000000000000000ull) : sign_frac; break;  // +-0, subnormal
        default: b = sign_frac | ((r2 % 8) << 52); break;
        }
        const double x = __longlong_as_double((long long)b);
        const float want = __double2float_rn(x), got = to_float_rn(x);
        if (__float_as_uint(want) != __float_as_uint(got) && !(want != want && got != got)) ++local;
        const float f = __uint_as_float((unsigned int)(k & 7 ? r2 >> 32 : (r2 >> 32) & 0x807fffffu));
        const double fw = (double)f, fg = to_double_exact(f);
        if (__double_as_longlong(fw) != __double_as_longlong(fg) && !(fw != fw && fg != fg))
            ++local;
        const int s = 1 + (int)((r2 >> 8) & 3);
        const double p = __hiloint2double((1023 - s) << 20, 0);  // 2^-s
        const double wd = __dmul_rn(x, p), gd = scale_down_pow2(o, x, s, p);
        if (__double_as_longlong(wd) != __double_as_longlong(gd) && !(wd != wd && gd != gd))
            ++local;
    }
    if (local) atomicAdd(bad, local);
}

// FP64 issue-rate probe: every thread runs CHAINS independent recurrences x = fma(x, a, b)
// for `iters` steps, with a and b in registers (in_reg; constant-bank operands issue slower,
// see lap_device.cuh), so the FP64 pipe never waits on a dependency once a few warps per SM
// are resident. fmas issued = threads * CHAINS * iters. The result is stored only when it
// equals an impossible value, which keeps the chains live.
constexpr int RATE_CHAINS = 8;
__global__ void __launch_bounds__(256)
    fp64_rate_kernel(long long iters, double a, double b, double* __restrict__ sink)
{
    const FmaOps o = load_fma_ops();
    a = in_reg(o, a);
    b = in_reg(o, b);
    double x[RATE_CHAINS];
#pragma unroll
    for (int k = 0; k < RATE_CHAINS; ++k) x[k] = (double)(threadIdx.x + 32 * k) * 1e-3;
    for (long long t = 0; t < iters; ++t) {
#pragma unroll
        for (int k = 0; k < RATE_CHAINS; ++k) x[k] = __fma_rn(x[k], a, b);
    }
    double acc = x[0];
#pragma unroll
    for (int k = 1; k < RATE_CHAINS; ++k) acc = fmax(acc, x[k]);
    if (acc == -1.0) sink[blockIdx.x] = acc;
}

}  // namespace

int64_t launch_fp64_rate(int blocks, long long iters, double* sink, cudaStream_t s)
{
    // a < 1, b > 0: every chain tends to b / (1 - a) = 1, no overflow or subnormals
    fp64_rate_kernel<<<blocks, 256, 0, s>>>(iters, 0.999999, 1e-6, sink);
    note_launch();
    if (cudaGetLastError() != cudaSuccess) return -1;
    return (int64_t)blocks * 256 * RATE_CHAINS * iters;
}

cudaError_t launch_check_rounding(long long count, unsigned long long seed, unsigned long long* bad,
                                  cudaStream_t s)
{
    check_rounding_kernel<<<152 * 8, 256, 0, s>>>(count, seed, bad);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_batch_loop_decide(long long* st, const int* remaining, cudaGraphConditionalHandle h,
                                     cudaStream_t s)
{
    batch_loop_decide_kernel<<<1, 32, 0, s>>>(st, remaining, h);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_loop_decide(LoopState* st, const double* nrm, const unsigned long long* maxd,
                               const float* scale, cudaGraphConditionalHandle h, cudaStream_t s)
{
    loop_decide_kernel<<<1, 32, 0, s>>>(st, nrm, maxd, scale, h);
    note_launch();
    return cudaGetLastError();
}

}  // namespace lap
