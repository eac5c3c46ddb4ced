// lap_device.cuh -- device helpers shared by the kernels of liblaplace.so.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace lap {

// On GB300's FP64 pipe a fused multiply-add issues at ~0.60 T/s but an add or a multiply at
// ~0.50 T/s (measured). x + y == fma(x, 1, y) and x * y == fma(x, y, -0) bit for bit, for every
// input, so adds and multiplies are issued as fmas. The 1 and -0 are loaded from device memory
// (load_fma_ops): as literals the compiler would turn the fma back into the add or multiply.
struct FmaOps {
    double one;    // 1.0
    double nzero;  // -0.0
};
// 1 and -0 in device memory. Kernels load them on entry: loaded values live in registers,
// whereas kernel arguments are read as constant-bank operands, and an FP64 fma with a
// constant-bank operand issues no faster than the add it replaces (measured on GB300).
// The array is not const, so the compiler cannot fold the loads away.
static __device__ double g_fma_consts[2] = {1.0, -0.0};

__device__ __forceinline__ FmaOps load_fma_ops()
{
    return FmaOps{g_fma_consts[0], g_fma_consts[1]};
}

// c copied into a register on the integer pipe. Kernel arguments are constant-bank operands,
// and an FP64 fma with a constant-bank operand issues at the rate of an add; an XOR with an
// integer zero that the compiler cannot see (from the loaded -0) gives a register operand
// without spending an FP64 operation. Coefficients used on every point go through this.
__device__ __forceinline__ double in_reg(const FmaOps& o, double c)
{
    const long long zero = __double_as_longlong(o.nzero) << 1;
    return __longlong_as_double(__double_as_longlong(c) ^ zero);
}

__device__ __forceinline__ double fadd(const FmaOps& o, double a, double b)
{
    return __fma_rn(a, o.one, b);
}
__device__ __forceinline__ double fmul(const FmaOps& o, double a, double b)
{
    return __fma_rn(a, b, o.nzero);
}

// The rare inputs of the integer-pipe paths below take these out-of-line functions. Written
// inline, the compiler evaluates the fallback for every input and selects the result, which
// spends the very FP64 operation the integer path saves (measured on GB300: the SOR colour
// pass at 4097^2 ran 94 us with the fallback inline, 76 us with it out of line).
static __device__ __noinline__ double fmul_rare(double x, double y, double nzero)
{
    return __fma_rn(x, y, nzero);
}
// The rare inputs of the FP32 <-> FP64 conversions below, in integer arithmetic from the
// IEEE-754 formats (no FP64-pipe instruction: a conversion instruction on a path the
// compiler evaluates for every point would cost one FP64 issue per point; measured).
// x: |x| below FP32's normal range (including FP64 subnormals), or an FP32 overflow, or
// infinite or NaN: the nearest FP32 value, ties to even (subnormal, zero or infinite); NaN
// stays NaN (quiet).
static __device__ __noinline__ float to_float_rare(double x)
{
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
    const unsigned int sign = (unsigned int)(b >> 32) & 0x80000000u;
    const int ex = (int)((b >> 52) & 0x7ff);
    const unsigned long long frac = b & 0xfffffffffffffull;
    if (ex == 0x7ff) return __uint_as_float(sign | 0x7f800000u | (frac ? 0x00400000u | (unsigned int)(frac >> 29) : 0u));
    if (ex - 1023 + 127 >= 1) return __uint_as_float(sign | 0x7f800000u);  // overflow: infinity
    if (ex == 0) return __uint_as_float(sign);  // FP64 subnormal or zero: far below 2^-150
    // |x| = m 2^(ex - 1075) with a 53-bit m; in units of 2^-149 (the FP32 subnormal step)
    // that is m / 2^sh, sh = 926 - ex >= 54 - 28 (ex <= 896 here)
    const unsigned long long m = frac | (1ull << 52);
    const int sh = 926 - ex;
    if (sh >= 64) return __uint_as_float(sign);  // below half the smallest subnormal
    unsigned int q = (unsigned int)(m >> sh);
    const unsigned long long rem = m & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (q & 1u))) ++q;  // may carry to the smallest normal
    return __uint_as_float(sign | q);
}
// f: an FP32 subnormal, infinity or NaN: (double)f exactly (NaN stays NaN, quiet).
static __device__ __noinline__ double to_double_rare(float f)
{
    const unsigned int u = __float_as_uint(f);
    const unsigned int sign = u & 0x80000000u, e = (u >> 23) & 0xffu, frac = u & 0x7fffffu;
    if (e == 0xffu) {
        const unsigned int fr = frac ? (frac | 0x00400000u) : 0u;
        return __hiloint2double((int)(sign | 0x7ff00000u | (fr >> 3)), (int)(fr << 29));
    }
    if (frac == 0) return __hiloint2double((int)sign, 0);
    // frac 2^-149 with the leading bit at position k: 2^(k - 149) (1 + the bits below k)
    const int k = 31 - __clz(frac);
    const unsigned long long mant = ((unsigned long long)frac << (52 - k)) & 0xfffffffffffffull;
    const unsigned long long bits = ((unsigned long long)sign << 32) |
                                    ((unsigned long long)(k + 874) << 52) | mant;
    return __longlong_as_double((long long)bits);
}

// (double)f, exact, on the integer pipe when f is a normal FP32 number or +-0: the 8-bit
// exponent is rebiased (127 -> 1023) and the 23-bit fraction becomes the top of the 52-bit
// one. FP32 subnormals, infinities and NaN take to_double_rare (integer arithmetic too).
__device__ __forceinline__ double to_double_exact(float f)
{
    const unsigned int u = __float_as_uint(f);
    const unsigned int e = (u >> 23) & 0xffu;
    if (e - 1u < 254u)
        return __hiloint2double(
            (int)((u & 0x80000000u) | ((e + (1023u - 127u)) << 20) | ((u >> 3) & 0xfffffu)),
            (int)(u << 29));
    if ((u << 1) == 0) return __hiloint2double((int)(u & 0x80000000u), 0);
    return to_double_rare(f);
}

// x * 2^-k for k > 0, bit-identical to __dmul_rn(x, 2^-k). On GB300 the FP64 pipe
// issues about 2 operations per clock per SM, the integer pipe 64 times more; when x is
// normal and the result stays normal the product is just the exponent field lowered by
// k, and when x is +-0 it is x itself, both done on the integer pipe. Subnormal, tiny,
// infinite and NaN inputs take the FP64 multiply.
__device__ __forceinline__ double scale_down_pow2(const FmaOps& o, double x, int k,
                                                  double two_pow_minus_k)
{
    int hi = __double2hiint(x);
    int lo = __double2loint(x);
    int e = (hi >> 20) & 0x7ff;
    if (e > k && e < 0x7ff) return __hiloint2double(hi - (k << 20), lo);
    if (((hi & 0x7fffffff) | lo) == 0) return x;
    return fmul_rare(x, two_pow_minus_k, o.nzero);
}

// Multiply by 1/d: the integer-pipe path when 1/d is an exact power of two.
template <bool POW2>
__device__ __forceinline__ double times_inv_d(const FmaOps& o, double s, double inv_d, int shift)
{
    if (POW2) return scale_down_pow2(o, s, shift, inv_d);
    return fmul(o, s, inv_d);
}

// Neighbour sum of Eq. 5: fma(beta^2, N + S, E + W); with beta == 1 the fma is the add.
template <bool UNIT_BETA>
__device__ __forceinline__ double neighbour_sum(const FmaOps& o, double w_, double e_, double s_,
                                                double n_, double b2)
{
    double ew = fadd(o, w_, e_);
    double ns = fadd(o, s_, n_);
    return UNIT_BETA ? fadd(o, ns, ew) : __fma_rn(b2, ns, ew);
}

// x rounded to the nearest FP32 value (ties to even), bit-identical to __double2float_rn,
// on the integer pipe when the result is a normal FP32 number or overflows: the 52-bit
// fraction keeps its top 23 bits and rounds on the 29 below (a carry out of the fraction
// raises the exponent, up to infinity); +-0 maps to +-0. FP32-subnormal results, overflows
// past the exponent range, infinities and NaN take to_float_rare (integer arithmetic too).
// On GB300 the conversion instruction would compete with the FP64 arithmetic of the
// residual kernels for the FP64 pipe.
__device__ __forceinline__ float to_float_rn(double x)
{
    // on the two 32-bit halves of x (formulated on one 64-bit integer, the compiler issued an
    // FP64-pipe instruction per call; measured)
    const unsigned int hi = (unsigned int)__double2hiint(x), lo = (unsigned int)__double2loint(x);
    const int e = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;
    if (e < 1 || e > 254) {
        if (((hi << 1) | lo) == 0) return __uint_as_float(hi);  // +-0
        return to_float_rare(x);
    }
    // the top 23 of the 52 fraction bits: 20 from hi, 3 from lo; round on lo's low 29 bits
    unsigned int out = ((unsigned int)e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
    const unsigned int rem = lo & 0x1fffffffu;
    if (rem > 0x10000000u || (rem == 0x10000000u && (out & 1u))) ++out;
    out |= hi & 0x80000000u;
    return __uint_as_float(out);
}

// A grid-stride walk over the interior points of an m x n field in row-major order: thread
// g = blockIdx.x * NT + threadIdx.x visits flattened points g, g + S, g + 2S, ... with
// S = gridDim.x * NT, so every thread has the same number of points to one, and at any time
// the blocks work on one contiguous window of S points (neighbour rows shared in L2). Handing
// out whole rows instead leaves the blocks that got one row more as the tail. (i, j) are the
// current point's coordinates (1-based interior); stepping needs no division.
template <int NT>
struct StrideWalk {
    int i, j, mi, di, dj;
    int64_t left;  // points still to visit, the current one included
    __device__ __forceinline__ StrideWalk(int m, int n) : i(1), j(1), mi(m - 2), di(0), dj(0), left(0)
    {
        if (m < 3 || n < 3) return;
        const int64_t total = (int64_t)(m - 2) * (int64_t)(n - 2);
        const int64_t k = (int64_t)blockIdx.x * NT + threadIdx.x;
        if (k >= total) return;
        const int64_t step = (int64_t)gridDim.x * NT;
        left = (total - 1 - k) / step + 1;
        j = 1 + (int)(k / mi);
        i = 1 + (int)(k % mi);
        dj = (int)(step / mi);
        di = (int)(step % mi);
    }
    __device__ __forceinline__ void next()
    {
        i += di;
        j += dj;
        if (i > mi) {
            i -= mi;
            ++j;
        }
        --left;
    }
};

// The five FP64 values of a 5-point stencil at c (pitch p): loaded together for two points
// before either is used, so that each thread of a grid-stride loop has two points' loads in
// flight.
struct Stencil5 {
    double c, w, e, s, n;
};
__device__ __forceinline__ Stencil5 load5(const double* __restrict__ c, int64_t p)
{
    return Stencil5{c[0], c[-1], c[1], c[-p], c[p]};
}

// Deterministic warp reductions (fixed xor tree).
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = __dadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long u = __shfl_xor_sync(0xffffffffu, v, o);
        v = u > v ? u : v;
    }
    return v;
}

// |x| as an orderable bit pattern (NaN above +inf above every finite value).
__device__ __forceinline__ unsigned long long abs_bits(double x)
{
    return static_cast<unsigned long long>(__double_as_longlong(x)) & 0x7fffffffffffffffull;
}

// The work items a CTA of a batched launch takes. Without a claim counter: item blockIdx.x
// alone (one CTA per item). With one (a persistent launch of as many CTAs as fit the device):
// each CTA takes the next unclaimed item from claim[0] until none is left, so CTAs that drew
// cheap items (small, or of converged problems) take more. claim[1] counts the CTAs that have
// finished; the last one resets both words for the next launch on the stream, which starts
// after this one ends. No CTA waits for another.
struct ItemClaim {
    unsigned* claim;
    int count;
    __device__ __forceinline__ int take(int prev) const
    {
        if (!claim) return prev < 0 ? (int)blockIdx.x : count;
        __shared__ int s_item;
        __syncthreads();  // every thread has read the previous item
        if (threadIdx.x == 0) s_item = (int)atomicAdd(claim, 1u);
        __syncthreads();
        return s_item;
    }
    __device__ __forceinline__ void finish() const
    {
        if (!claim || threadIdx.x != 0) return;
        __threadfence();
        if (atomicAdd(claim + 1, 1u) == gridDim.x - 1) {
            claim[0] = 0u;
            claim[1] = 0u;
        }
    }
};

}  // namespace lap
