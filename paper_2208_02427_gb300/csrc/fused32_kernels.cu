// fused32_kernels.cu -- the FP32 V-cycle's work on a level in two passes over memory.
//
// The inner cycle of the mixed-precision solver (FP32 on the correction equation
// (E+W) + b2 (N+S) - d e + q = 0) is memory-bound: each red-black colour pass, the
// residual, the restriction and the interpolation would each stream the level once. Here
// one tile kernel does a level's whole descent and one its whole ascent:
//   down: nu1 pre-smoothing sweeps (2 nu1 colour passes), the residual, and the
//         full-weighting restriction to the next level (whose correction it zeroes);
//   up:   the bilinear interpolation of the coarse correction, then nu2 post-smoothing
//         sweeps.
// A CTA loads its tile plus a halo into shared memory (temporal blocking: the halo shrinks
// by one point per colour pass), works there, and writes back only the points it owns.
// Every value is the one the per-pass kernels compute (same expressions, same rounding),
// so the result is the same bit for bit; halo points are computed redundantly by the
// neighbouring tiles. Tiles read u from one buffer and write another (down: u -> r slot,
// up: r slot -> u), so no tile reads a value another tile has already overwritten.
//
// Shared-memory layout: a region row keeps its even columns in one half and its odd
// columns in the other, so the points of one colour in a row are contiguous and their
// east/west neighbours are contiguous in the other half (no bank conflicts within a
// half-row access). The half stride is the 64 points plus 4 words (16-byte aligned rows):
// a descent tile's two arrays then take 68 KB, so three descent CTAs share an SM's shared
// memory (measured: the batched mixed solve of 4096 uneven grids 46.5 -> 44.5 ms against a
// half stride of 80 with two CTAs per SM).
#include <algorithm>
#include <type_traits>

#include "lap_device.cuh"
#include "lap_internal.cuh"

namespace lap {

namespace {

constexpr int FT_W = 128;               // region columns (even): 64 column pairs
constexpr int FT_H = 64;                // region rows (single-grid tiles; batched: a variant)
constexpr int FT_HS = FT_W / 2 + 4;     // half-row stride (16-byte aligned)
constexpr int FT_RS = 2 * FT_HS;        // row stride
constexpr int FT_CS = FT_W / 2 + 4;     // row stride of the staged coarse points
// floats per shared array, and of the staged coarse points, for regions of H rows
__host__ __device__ constexpr int ft_arr(int H) { return FT_RS * H; }
__host__ __device__ constexpr int ft_carr(int H) { return FT_CS * (H / 2 + 2); }
constexpr int FT_ARR = ft_arr(FT_H);

// The region of a tile: global (gx0 + lx, gy0 + ly) for local 0 <= lx < w, 0 <= ly < h.
// gx0 is even: local column lx = 2p + half sits at half `half`, index p, of its row, and
// has the parity of its global column.
struct Region {
    int gx0, gy0, w, h;
};

struct Coef32 {
    float2 b2, inv_d, d, w, omw;
    bool unit, gs;
};

__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }

__device__ __forceinline__ Coef32 coef32(const BatchLevel<float>& L, bool gs, float w, float omw)
{
    return Coef32{f2((float)L.b2), f2((float)L.inv_d), f2((float)L.d), f2(w), f2(omw),
                  L.unit_beta != 0, gs};
}

// (E+W) + b2 (N+S) for two points at once: per component the FP32 neighbour sum of the
// per-pass kernels (packed FP32 operations round each component like the scalar ones).
template <bool UNIT>
__device__ __forceinline__ float2 nsum2(float2 w_, float2 e_, float2 s_, float2 n_, const Coef32& k)
{
    const float2 ew = __fadd2_rn(w_, e_);
    const float2 ns = __fadd2_rn(s_, n_);
    return UNIT ? __fadd2_rn(ns, ew) : __ffma2_rn(k.b2, ns, ew);
}

// beta == 1 and Gauss-Seidel (w = 1) are the same for every point of a tile: the tile's code
// is compiled for each combination and chosen once per block (as run-time choices they cost
// a test and a branch in every group of points).
template <class F>
__device__ __forceinline__ void on_flag32(bool a, F&& f)
{
    if (a) f(std::true_type{});
    else f(std::false_type{});
}

// Asynchronous 4-byte copy global -> shared; completes at cp_async_wait_all.
__device__ __forceinline__ void cp_async4(float* sdst, const float* gsrc)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Stores the components of v whose flags are set (8-byte store when both are).
__device__ __forceinline__ void sts2_masked(float* p, float2 v, bool lo, bool hi)
{
    if (lo && hi) *reinterpret_cast<float2*>(p) = v;
    else if (lo) p[0] = v.x;
    else if (hi) p[1] = v.y;
}

// The region's u and q (0 outside the array; u = 0 when zero_u): each lane moves column
// pairs (gx, gx + 1), gx even, with 8-byte loads, all 16 of a thread in flight together,
// and splits them into the two halves of the row. Level pitches are even.
template <int NT, int H>
__device__ __forceinline__ void load_region(float* su, float* sq, const float* u, const float* q,
                                            int64_t pitch, int m, int n, const Region& R,
                                            bool zero_u)
{
    constexpr int NW = NT / 32, RPW = H / NW;  // region rows per warp
    static_assert(RPW >= 1 && RPW * NW == H, "region rows must be a multiple of the warps");
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    float2 vu[2 * RPW], vq[2 * RPW];
#pragma unroll
    for (int t = 0; t < RPW; ++t)
#pragma unroll
        for (int s2 = 0; s2 < 2; ++s2) {
            const int ly = wid + NW * t, p = lane + 32 * s2;
            const int gy = R.gy0 + ly, gx = R.gx0 + 2 * p;
            float2 a = make_float2(0.f, 0.f), b = make_float2(0.f, 0.f);
            if (ly < R.h && 2 * p < R.w && gy >= 0 && gy < n && gx >= 0 && gx < m) {
                const int64_t at = (int64_t)gy * pitch + gx;
                if (!zero_u) a = *reinterpret_cast<const float2*>(u + at);
                b = *reinterpret_cast<const float2*>(q + at);
                if (gx + 1 >= m) a.y = b.y = 0.f;  // past the last column (row padding)
            }
            vu[2 * t + s2] = a;
            vq[2 * t + s2] = b;
        }
#pragma unroll
    for (int t = 0; t < RPW; ++t)
#pragma unroll
        for (int s2 = 0; s2 < 2; ++s2) {
            const int ly = wid + NW * t, p = lane + 32 * s2;
            if (ly < R.h && 2 * p < R.w) {
                const int o = ly * FT_RS + p;
                su[o] = vu[2 * t + s2].x;
                su[o + FT_HS] = vu[2 * t + s2].y;
                sq[o] = vq[2 * t + s2].x;
                sq[o + FT_HS] = vq[2 * t + s2].y;
            }
        }
}

// Indices c of the half row `half` whose columns lie in [lx_lo, lx_hi] (lx = 2c + half).
__device__ __forceinline__ void half_range(int lx_lo, int lx_hi, int half, int* c_lo, int* c_hi)
{
    *c_lo = (lx_lo - half + 1) >> 1;
    *c_hi = (lx_hi - half) >> 1;
}

__device__ __forceinline__ float4 lds4(const float* p) { return *reinterpret_cast<const float4*>(p); }

// Stores the components of v at p[0..3] whose index lies in [lo, hi] (16-byte store when all do).
__device__ __forceinline__ void sts4_masked(float* p, float4 v, int c0, int lo, int hi)
{
    if (c0 >= lo && c0 + 3 <= hi) {
        *reinterpret_cast<float4*>(p) = v;
        return;
    }
    if (c0 >= lo && c0 <= hi) p[0] = v.x;
    if (c0 + 1 >= lo && c0 + 1 <= hi) p[1] = v.y;
    if (c0 + 2 >= lo && c0 + 2 <= hi) p[2] = v.z;
    if (c0 + 3 >= lo && c0 + 3 <= hi) p[3] = v.w;
}

// s = (E+W) + b2 (N+S) + q for the four points c0 .. c0 + 3 of half HALF of region row ly,
// as two float2 (points c0, c0 + 1 and c0 + 2, c0 + 3). Their west/east neighbours are in the
// other half of the row at c - 1 + HALF and c + HALF.
template <int HALF, bool UNIT>
__device__ __forceinline__ void stencil4(const float* su, const float* sq, int ly, int c0,
                                         const Coef32& k, float2& sA, float2& sB)
{
    const float* oth = su + ly * FT_RS + (1 - HALF) * FT_HS;
    const int a = ly * FT_RS + HALF * FT_HS + c0;
    const float4 o = lds4(oth + c0);
    float2 wA, wB, eA, eB;
    if (HALF == 0) {
        const float ol = oth[c0 - 1];
        wA = make_float2(ol, o.x);
        wB = make_float2(o.y, o.z);
        eA = make_float2(o.x, o.y);
        eB = make_float2(o.z, o.w);
    } else {
        const float orr = oth[c0 + 4];
        wA = make_float2(o.x, o.y);
        wB = make_float2(o.z, o.w);
        eA = make_float2(o.y, o.z);
        eB = make_float2(o.w, orr);
    }
    const float4 S = lds4(su + a - FT_RS), N = lds4(su + a + FT_RS), Q = lds4(sq + a);
    sA = __fadd2_rn(nsum2<UNIT>(wA, eA, make_float2(S.x, S.y), make_float2(N.x, N.y), k), make_float2(Q.x, Q.y));
    sB = __fadd2_rn(nsum2<UNIT>(wB, eB, make_float2(S.z, S.w), make_float2(N.z, N.w), k), make_float2(Q.z, Q.w));
}

// Eq. 6 (gs) or Eq. 7 on the four points c0 .. c0 + 3 of half HALF of row ly, those in
// [c_lo, c_hi] stored.
template <int HALF, bool UNIT, bool GS>
__device__ __forceinline__ void relax4(float* su, const float* sq, int ly, int c0, int c_lo, int c_hi,
                                       const Coef32& k)
{
    float2 sA, sB;
    stencil4<HALF, UNIT>(su, sq, ly, c0, k, sA, sB);
    float* at = su + ly * FT_RS + HALF * FT_HS + c0;
    float2 gA = __fmul2_rn(sA, k.inv_d), gB = __fmul2_rn(sB, k.inv_d);
    if (!GS) {
        const float4 old = lds4(at);
        gA = __ffma2_rn(k.w, gA, __fmul2_rn(k.omw, make_float2(old.x, old.y)));
        gB = __ffma2_rn(k.w, gB, __fmul2_rn(k.omw, make_float2(old.z, old.w)));
    }
    sts4_masked(at, make_float4(gA.x, gA.y, gB.x, gB.y), c0, c_lo, c_hi);
}

// One colour pass of Eq. 6 (gs) or Eq. 7 over the domain-interior points of the region
// but its outer ring: points (gx + gy) % 2 == colour, i.e. half (colour + gy) & 1 of row
// gy. A warp takes two rows of the same parity (ly, ly + 2: the same half), a half warp one
// row, a lane four consecutive points of its half row.
template <int NT, bool UNIT, bool GS>
__device__ __forceinline__ void colour_pass(float* su, const float* sq, const Region& R, int m, int n,
                                            int colour, const Coef32& k)
{
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int lx_lo = max(1, 1 - R.gx0), lx_hi = min(R.w - 2, m - 2 - R.gx0);
    const int ly_lo = max(1, 1 - R.gy0), ly_hi = min(R.h - 2, n - 2 - R.gy0);
    int cl0, ch0, cl1, ch1;
    half_range(lx_lo, lx_hi, 0, &cl0, &ch0);
    half_range(lx_lo, lx_hi, 1, &cl1, &ch1);
    const int c0 = 4 * (lane & 15), sub = 2 * (lane >> 4);
    for (int g = wid;; g += NW) {
        const int r = ly_lo + 4 * (g >> 1) + (g & 1);
        if (r > ly_hi) break;
        const int ly = r + sub;
        const int half = (colour + R.gy0 + r) & 1;  // the same for r and r + 2
        if (ly > ly_hi) continue;
        if (half == 0) {
            if (c0 + 3 >= cl0 && c0 <= ch0) relax4<0, UNIT, GS>(su, sq, ly, c0, cl0, ch0, k);
        } else {
            if (c0 + 3 >= cl1 && c0 <= ch1) relax4<1, UNIT, GS>(su, sq, ly, c0, cl1, ch1, k);
        }
    }
}

template <int NT, bool UNIT, bool GS>
__device__ __forceinline__ void smooth_region(float* su, const float* sq, const Region& R, int m,
                                              int n, int sweeps, const Coef32& k)
{
    for (int s = 0; s < sweeps; ++s)
        for (int colour = 0; colour < 2; ++colour) {
            colour_pass<NT, UNIT, GS>(su, sq, R, m, n, colour, k);
            __syncthreads();
        }
}

// Owned points [x0, x1) x [y0, y1) from shared memory to dst, by column pairs (gx even).
template <int NT>
__device__ __forceinline__ void store_owned(float* dst, int64_t pitch, const float* su,
                                            const Region& R, int x0, int x1, int y0, int y1)
{
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int p_lo = (x0 - R.gx0) >> 1, p_hi = (x1 - 1 - R.gx0) >> 1;
    for (int gy = y0 + wid; gy < y1; gy += NW) {
        const int ly = gy - R.gy0;
        for (int p = p_lo + lane; p <= p_hi; p += 32) {
            const int gx = R.gx0 + 2 * p;
            const float2 v = make_float2(su[ly * FT_RS + p], su[ly * FT_RS + FT_HS + p]);
            sts2_masked(dst + (int64_t)gy * pitch + gx, v, gx >= x0, gx + 1 < x1);
        }
    }
}

// Region of the tile of owned points [x0, x0 + tx) x [y0, y0 + ty) with a halo of `halo`
// points on every side; gx0 rounded down to even, the width rounded up to even.
__device__ __forceinline__ Region region_of(int x0, int y0, int tx, int ty, int halo)
{
    Region R;
    R.gx0 = (x0 - halo) & ~1;
    R.gy0 = y0 - halo;
    const int last = x0 + tx - 1 + halo;
    R.w = (last - R.gx0 + 2) & ~1;
    R.h = ty + 2 * halo;
    return R;
}

// Descent on one tile of level F: nu1 smoothing sweeps, the smoothed u of the owned points
// to F.r (the second buffer of the level), the residual, and qc = 0.25 ((4 r + 2 edges) +
// corners) with the correction zeroed at the coarse points whose centre the tile owns.
template <int NT, int H, bool UNIT, bool GS>
__device__ __forceinline__ void down_tile(const BatchLevel<float>& F, const BatchLevel<float>& C,
                                          int x0, int y0, int tx, int ty, int nu1, bool zero_u,
                                          const Coef32& k, float* su, float* sq)
{
    constexpr int NW = NT / 32;
    const int m = F.m, n = F.n;
    const Region R = region_of(x0, y0, tx, ty, 2 + 2 * nu1);
    load_region<NT, H>(su, sq, F.u, F.q, F.pitch, m, n, R, zero_u);
    __syncthreads();
    smooth_region<NT, UNIT, GS>(su, sq, R, m, n, nu1, k);
    const int x1 = min(x0 + tx, m - 1), y1 = min(y0 + ty, n - 1);
    store_owned<NT>(F.r, F.pitch, su, R, x0, x1, y0, y1);
    // residual r = (E+W) + b2 (N+S) + q - d u on the owned points and a ring of one, written
    // over q (each point reads only its own q)
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int lx_lo = max(1, x0 - 1) - R.gx0, lx_hi = min(m - 2, x1) - R.gx0;
    const int ly_lo = max(1, y0 - 1) - R.gy0, ly_hi = min(n - 2, y1) - R.gy0;
    // a warp takes rows ly, ly + 1 of one half (half warps), a lane four points
    int cl0, ch0, cl1, ch1;
    half_range(lx_lo, lx_hi, 0, &cl0, &ch0);
    half_range(lx_lo, lx_hi, 1, &cl1, &ch1);
    const int c0 = 4 * (lane & 15), sub = lane >> 4;
    const float2 nd = make_float2(-k.d.x, -k.d.y);
    for (int g = wid;; g += NW) {
        const int half = g & 1, ly = ly_lo + 2 * (g >> 1) + sub;
        if (ly_lo + 2 * (g >> 1) > ly_hi) break;
        const int clo = half ? cl1 : cl0, chi = half ? ch1 : ch0;
        if (ly > ly_hi || c0 + 3 < clo || c0 > chi) continue;
        float2 sA, sB;
        if (half == 0) stencil4<0, UNIT>(su, sq, ly, c0, k, sA, sB);
        else stencil4<1, UNIT>(su, sq, ly, c0, k, sA, sB);
        const int a = ly * FT_RS + half * FT_HS + c0;
        const float4 u4 = lds4(su + a);
        const float2 rA = __ffma2_rn(nd, make_float2(u4.x, u4.y), sA);
        const float2 rB = __ffma2_rn(nd, make_float2(u4.z, u4.w), sB);
        sts4_masked(sq + a, make_float4(rA.x, rA.y, rB.x, rB.y), c0, clo, chi);
    }
    __syncthreads();
    // restriction to the coarse points (I, J) with (2I, 2J) owned: the centre is at half 0,
    // index c = I - gx0 / 2; west/east at half 1, c - 1 and c; rows 2J - 1, 2J, 2J + 1
    const int mc = (m - 1) / 2 + 1, nc = (n - 1) / 2 + 1;
    const int I0 = max(1, (x0 + 1) >> 1), I1 = min(mc - 2, (x1 - 1) >> 1);
    const int J0 = max(1, (y0 + 1) >> 1), J1 = min(nc - 2, (y1 - 1) >> 1);
    const float* r = sq;
    for (int J = J0 + wid; J <= J1; J += NW) {
        const int ly = 2 * J - R.gy0;
        const float* r0 = r + ly * FT_RS;
        for (int I = I0 + lane; I <= I1; I += 32) {
            const int c = I - (R.gx0 >> 1);
            const float* mid = r0 + c;
            const float* odd = r0 + FT_HS + c;
            const float edges = __fadd_rn(__fadd_rn(odd[-1], odd[0]), __fadd_rn(mid[-FT_RS], mid[FT_RS]));
            const float corners = __fadd_rn(__fadd_rn(odd[-FT_RS - 1], odd[-FT_RS]),
                                            __fadd_rn(odd[FT_RS - 1], odd[FT_RS]));
            const float tt = __fmaf_rn(2.0f, mid[0], edges);
            const int64_t at = (int64_t)J * C.pitch + I;
            C.q[at] = __fmul_rn(0.25f, __fmaf_rn(2.0f, tt, corners));
            C.u[at] = 0.0f;
        }
    }
}

// Ascent on one tile of level F: u (from F.r) plus the bilinear interpolation of C.u, nu2
// smoothing sweeps, the owned points to F.u. The coarse points under the region are staged
// in shared memory (sc): a column pair p of the region lies over coarse column gx0 / 2 + p.
// With psi (the FP64 field of the mixed solver's level 0), the last ascent adds its result
// to psi in FP64 (psi += e, the update of the defect correction) instead of storing e.
template <int NT, int H, bool UNIT, bool GS>
__device__ __forceinline__ void up_tile(const BatchLevel<float>& F, const BatchLevel<float>& C,
                                        int x0, int y0, int tx, int ty, int nu2, const Coef32& k,
                                        float* su, float* sq, float* sc, double* psi,
                                        int64_t psi_pitch)
{
    constexpr int NW = NT / 32;
    const int m = F.m, n = F.n;
    const Region R = region_of(x0, y0, tx, ty, 2 * nu2);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (psi) {
        // the owned points' FP64 lines into L2 now, so that the update after the smoothing
        // does not wait on HBM (a row of at most 128 doubles spans at most 9 lines of 128 B)
        const int px1 = min(x0 + tx, m - 1), py1 = min(y0 + ty, n - 1);
        for (int gy = y0 + wid; gy < py1; gy += NW) {
            const double* row = psi + (int64_t)gy * psi_pitch;
            const uintptr_t first = reinterpret_cast<uintptr_t>(row + x0) & ~(uintptr_t)127;
            const uintptr_t line = first + 128 * (uintptr_t)lane;
            if (line <= reinterpret_cast<uintptr_t>(row + px1 - 1))
                asm volatile("prefetch.global.L2 [%0];" ::"l"(line));
        }
    }
    const int cI0 = R.gx0 >> 1, cJ0 = R.gy0 >> 1;  // floor halves (gy0 may be negative)
    const int cw = (R.w >> 1) + 1, ch = ((R.gy0 + R.h - 1) >> 1) - cJ0 + 2;
    const int mc = (m - 1) / 2 + 1, nc = (n - 1) / 2 + 1;
    for (int cy = wid; cy < ch; cy += NW) {
        const int J = cJ0 + cy;
        const bool rowin = J >= 0 && J < nc;
        for (int cx = lane; cx < cw; cx += 32) {
            const int I = cI0 + cx;
            float* d = sc + cy * FT_CS + cx;
            if (rowin && I >= 0 && I < mc) cp_async4(d, C.u + (int64_t)J * C.pitch + I);
            else *d = 0.f;
        }
    }
    load_region<NT, H>(su, sq, F.r, F.q, F.pitch, m, n, R, false);
    cp_async_wait_all();
    __syncthreads();
    // u += P e: even rows take coarse row J = gy / 2, odd rows the mean of rows J and J + 1;
    // even columns (half 0) coarse column p, odd columns (half 1) the mean of p and p + 1
    const int lx_lo = max(0, 1 - R.gx0), lx_hi = min(R.w - 1, m - 2 - R.gx0);
    const int ly_lo = max(0, 1 - R.gy0), ly_hi = min(R.h - 1, n - 2 - R.gy0);
    for (int ly = ly_lo + wid; ly <= ly_hi; ly += NW) {
        const int gy = R.gy0 + ly;
        const float* a = sc + ((gy >> 1) - cJ0) * FT_CS;
        float* row = su + ly * FT_RS;
        for (int p = lane; 2 * p <= lx_hi; p += 32) {
            const bool ok0 = 2 * p >= lx_lo, ok1 = 2 * p + 1 >= lx_lo && 2 * p + 1 <= lx_hi;
            float e0, e1;
            if ((gy & 1) == 0) {
                e0 = a[p];
                e1 = __fmul_rn(0.5f, __fadd_rn(a[p], a[p + 1]));
            } else {
                e0 = __fmul_rn(0.5f, __fadd_rn(a[p], a[p + FT_CS]));
                e1 = __fmul_rn(0.25f, __fadd_rn(__fadd_rn(a[p], a[p + 1]),
                                                __fadd_rn(a[p + FT_CS], a[p + FT_CS + 1])));
            }
            if (ok0) row[p] = __fadd_rn(row[p], e0);
            if (ok1) row[FT_HS + p] = __fadd_rn(row[FT_HS + p], e1);
        }
    }
    __syncthreads();
    smooth_region<NT, UNIT, GS>(su, sq, R, m, n, nu2, k);
    const int x1 = min(x0 + tx, m - 1), y1 = min(y0 + ty, n - 1);
    if (!psi) {
        store_owned<NT>(F.u, F.pitch, su, R, x0, x1, y0, y1);
        return;
    }
    // column pairs (gx even: 16-byte aligned double2 when the pitch is even), two per lane,
    // so that each thread has four FP64 loads in flight per row
    const FmaOps o = load_fma_ops();
    const int p_lo = (x0 - R.gx0) >> 1, p_hi = (x1 - 1 - R.gx0) >> 1;
    const bool even_pitch = (psi_pitch & 1) == 0;
    for (int gy = y0 + wid; gy < y1; gy += NW) {
        const float* row = su + (gy - R.gy0) * FT_RS;
        double* prow = psi + (int64_t)gy * psi_pitch;
        double2 v[2];
        bool lo[2], hi[2];
#pragma unroll
        for (int s2 = 0; s2 < 2; ++s2) {
            const int p = p_lo + lane + 32 * s2;
            const int gx = R.gx0 + 2 * p;
            lo[s2] = p <= p_hi && gx >= x0;
            hi[s2] = p <= p_hi && gx + 1 < x1;
            if (lo[s2] && hi[s2] && even_pitch) {
                v[s2] = *reinterpret_cast<const double2*>(prow + gx);
            } else {
                v[s2].x = lo[s2] ? prow[gx] : 0.0;
                v[s2].y = hi[s2] ? prow[gx + 1] : 0.0;
            }
        }
#pragma unroll
        for (int s2 = 0; s2 < 2; ++s2) {
            const int p = p_lo + lane + 32 * s2;
            const int gx = R.gx0 + 2 * p;
            if (!lo[s2] && !hi[s2]) continue;
            const double a = fadd(o, v[s2].x, to_double_exact(row[p]));
            const double b = fadd(o, v[s2].y, to_double_exact(row[FT_HS + p]));
            if (lo[s2] && hi[s2] && even_pitch) {
                *reinterpret_cast<double2*>(prow + gx) = make_double2(a, b);
            } else {
                if (lo[s2]) prow[gx] = a;
                if (hi[s2]) prow[gx + 1] = b;
            }
        }
    }
}

// ---- one grid: tile (blockIdx.x, blockIdx.y) of owned points 1 + (bx tx, by ty) ----
// NT threads: 512 for levels with many tiles (three descent or two ascent CTAs per SM: the
// descent's two arrays fit three times in shared memory, at 40 registers; the ascent also
// stages the coarse points), 1024 (one CTA per SM, half the rows per warp: a shorter critical
// path) for levels with fewer tiles than SMs.
template <int NT>
__global__ void __launch_bounds__(NT, NT == 512 ? 3 : 1)
    down32_kernel(BatchLevel<float> F, BatchLevel<float> C, int tx, int ty, int nu1, int zero_u,
                  int gs, float w, float omw)
{
    extern __shared__ float4 smem4[];
    float* smem = reinterpret_cast<float*>(smem4);
    const Coef32 k = coef32(F, gs != 0, w, omw);
    on_flag32(k.unit, [&](auto U) {
        on_flag32(k.gs, [&](auto G) {
            down_tile<NT, FT_H, U.value, G.value>(F, C, 1 + blockIdx.x * tx, 1 + blockIdx.y * ty, tx,
                                                  ty, nu1, zero_u != 0, k, smem, smem + FT_ARR);
        });
    });
}

template <int NT>
__global__ void __launch_bounds__(NT, 1024 / NT)
    up32_kernel(BatchLevel<float> F, BatchLevel<float> C, int tx, int ty, int nu2, int gs, float w,
                float omw, double* psi, int64_t psi_pitch)
{
    extern __shared__ float4 smem4[];
    float* smem = reinterpret_cast<float*>(smem4);
    const Coef32 k = coef32(F, gs != 0, w, omw);
    on_flag32(k.unit, [&](auto U) {
        on_flag32(k.gs, [&](auto G) {
            up_tile<NT, FT_H, U.value, G.value>(F, C, 1 + blockIdx.x * tx, 1 + blockIdx.y * ty, tx, ty,
                                                nu2, k, smem, smem + FT_ARR, smem + 2 * FT_ARR, psi,
                                                psi_pitch);
        });
    });
}

// ---- many grids: one tile item per CTA, NT threads, regions of H rows ----
template <int NT, int H>
__global__ void __launch_bounds__(NT, NT == 512 ? 3 : 1)
    b_down32_kernel(const TileItem* __restrict__ items, int count, unsigned* claim,
                    const BatchLevel<float>* __restrict__ lv,
                    const int* __restrict__ active, int nu1, int zero_u, int gs, float w, float omw)
{
    extern __shared__ float4 smem4[];
    float* smem = reinterpret_cast<float*>(smem4);
    const ItemClaim ic{claim, count};
    for (int b = ic.take(-1); b < count; b = ic.take(b)) {
        const TileItem it = items[b];
        const BatchLevel<float> F = lv[it.level];
        if (active && !active[F.problem]) continue;
        const Coef32 k = coef32(F, gs != 0, w, omw);
        on_flag32(k.unit, [&](auto U) {
            on_flag32(k.gs, [&](auto G) {
                down_tile<NT, H, U.value, G.value>(F, lv[it.level + 1], it.x0, it.y0, it.tx, it.ty,
                                                   nu1, zero_u != 0, k, smem, smem + ft_arr(H));
            });
        });
        __syncthreads();  // the next tile reloads the shared arrays
    }
    ic.finish();
}

template <int NT, int H>
__global__ void __launch_bounds__(NT, 1024 / NT)
    b_up32_kernel(const TileItem* __restrict__ items, int count, unsigned* claim,
                  const BatchLevel<float>* __restrict__ lv,
                  const int* __restrict__ active, int nu2, int gs, float w, float omw,
                  const BatchLevel<double>* __restrict__ lv64)
{
    extern __shared__ float4 smem4[];
    float* smem = reinterpret_cast<float*>(smem4);
    const ItemClaim ic{claim, count};
    for (int b = ic.take(-1); b < count; b = ic.take(b)) {
        const TileItem it = items[b];
        const BatchLevel<float> F = lv[it.level];
        if (active && !active[F.problem]) continue;
        double* psi = lv64 ? lv64[it.level].u : nullptr;
        const int64_t pp = lv64 ? lv64[it.level].pitch : 0;
        const Coef32 k = coef32(F, gs != 0, w, omw);
        on_flag32(k.unit, [&](auto U) {
            on_flag32(k.gs, [&](auto G) {
                up_tile<NT, H, U.value, G.value>(F, lv[it.level + 1], it.x0, it.y0, it.tx, it.ty, nu2,
                                                 k, smem, smem + ft_arr(H), smem + 2 * ft_arr(H), psi,
                                                 pp);
            });
        });
        __syncthreads();  // the next tile reloads the shared arrays
    }
    ic.finish();
}

constexpr size_t ft_smem(int H) { return (2 * (size_t)ft_arr(H) + ft_carr(H)) * sizeof(float); }
constexpr size_t FT_SMEM = ft_smem(FT_H);
constexpr size_t ft_smem_down(int H) { return 2 * (size_t)ft_arr(H) * sizeof(float); }
constexpr size_t FT_SMEM_DOWN = ft_smem_down(FT_H);
constexpr int FT_FEW_TILES = 152;  // below one tile per SM: 1024-thread tiles

}  // namespace

// Halo of a descent (nu1 sweeps, then a residual ring feeding the restriction) and of an
// ascent (nu2 sweeps).
static int halo_down(int nu1) { return 2 + 2 * nu1; }
static int halo_up(int nu2) { return 2 * nu2; }

// Region rows of a batched tile variant: 1 = 512 threads over 128 x 64 regions (three descent
// or two ascent CTAs per SM), 2 = 1024 threads over 128 x 64 (one CTA per SM, half the rows per
// warp: a shorter critical path per tile), 3 = 512 threads over 128 x 32 (smaller tiles, more
// of them).
static int variant_rows(int variant) { return variant == 3 ? 32 : FT_H; }

static bool tiles_fit(int H, int nu1, int nu2)
{
    const int h = std::max(halo_down(nu1), halo_up(nu2));
    return FT_W - 2 * h - 2 >= 16 && H - 2 * h >= 8;
}

bool fused32_supported(int nu1, int nu2) { return tiles_fit(FT_H, nu1, nu2); }

bool fused32_variant_supported(int variant, int nu1, int nu2)
{
    return variant >= 1 && variant <= FUSED32_VARIANTS && tiles_fit(variant_rows(variant), nu1, nu2);
}

// Balanced tiles no larger than a region of H rows allows: the interior (m-2) x (n-2) split
// into ntx x nty tiles of tx x ty owned points.
static void tile_split(int H, int m, int n, int nu1, int nu2, int* tx, int* ty, int* ntx, int* nty)
{
    const int h = std::max(halo_down(nu1), halo_up(nu2));
    const int mx = FT_W - 2 * h - 2, my = H - 2 * h;
    const int W = std::max(1, m - 2), Hh = std::max(1, n - 2);
    *ntx = (W + mx - 1) / mx;
    *nty = (Hh + my - 1) / my;
    *tx = (W + *ntx - 1) / *ntx;
    *ty = (Hh + *nty - 1) / *nty;
}

void fused32_tile(int m, int n, int nu1, int nu2, int* tx, int* ty, int* ntx, int* nty)
{
    tile_split(FT_H, m, n, nu1, nu2, tx, ty, ntx, nty);
}

void fused32_tile_variant(int variant, int m, int n, int nu1, int nu2, int* tx, int* ty, int* ntx,
                          int* nty)
{
    tile_split(variant_rows(variant), m, n, nu1, nu2, tx, ty, ntx, nty);
}

// Nonzero once the tile kernels' shared-memory limit is raised on that device.
static std::atomic<size_t> g_fused32_ready[ATTR_DEVICES];

cudaError_t prepare_fused32()
{
    const int dev = attr_slot();
    if (dev >= 0 && g_fused32_ready[dev].load() != 0) return cudaSuccess;
    const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaFuncSetAttribute(down32_kernel<512>, a, (int)FT_SMEM_DOWN);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(up32_kernel<512>, a, (int)FT_SMEM);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(down32_kernel<1024>, a, (int)FT_SMEM_DOWN);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(up32_kernel<1024>, a, (int)FT_SMEM);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(b_down32_kernel<512, 64>, a, (int)ft_smem_down(64));
    if (e == cudaSuccess) e = cudaFuncSetAttribute(b_up32_kernel<512, 64>, a, (int)ft_smem(64));
    if (e == cudaSuccess) e = cudaFuncSetAttribute(b_down32_kernel<1024, 64>, a, (int)ft_smem_down(64));
    if (e == cudaSuccess) e = cudaFuncSetAttribute(b_up32_kernel<1024, 64>, a, (int)ft_smem(64));
    if (e == cudaSuccess) e = cudaFuncSetAttribute(b_down32_kernel<512, 32>, a, (int)ft_smem_down(32));
    if (e == cudaSuccess) e = cudaFuncSetAttribute(b_up32_kernel<512, 32>, a, (int)ft_smem(32));
    if (e == cudaSuccess) attr_record(g_fused32_ready, dev, 1);
    return e;
}

cudaError_t launch_down32(const BatchLevel<float>& F, const BatchLevel<float>& C, int nu1, int nu2,
                          bool zero_u, bool gs, double w, cudaStream_t s)
{
    int tx, ty, ntx, nty;
    fused32_tile(F.m, F.n, nu1, nu2, &tx, &ty, &ntx, &nty);
    const float wf = (float)w, omw = (float)(1.0 - w);
    if (ntx * nty < FT_FEW_TILES)
        down32_kernel<1024><<<dim3(ntx, nty), 1024, FT_SMEM_DOWN, s>>>(F, C, tx, ty, nu1, zero_u ? 1 : 0,
                                                                  gs ? 1 : 0, wf, omw);
    else
        down32_kernel<512><<<dim3(ntx, nty), 512, FT_SMEM_DOWN, s>>>(F, C, tx, ty, nu1, zero_u ? 1 : 0,
                                                                gs ? 1 : 0, wf, omw);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_up32(const BatchLevel<float>& F, const BatchLevel<float>& C, int nu1, int nu2,
                        bool gs, double w, cudaStream_t s, double* psi, int64_t psi_pitch)
{
    int tx, ty, ntx, nty;
    fused32_tile(F.m, F.n, nu1, nu2, &tx, &ty, &ntx, &nty);
    const float wf = (float)w, omw = (float)(1.0 - w);
    if (ntx * nty < FT_FEW_TILES)
        up32_kernel<1024><<<dim3(ntx, nty), 1024, FT_SMEM, s>>>(F, C, tx, ty, nu2, gs ? 1 : 0, wf, omw,
                                                                psi, psi_pitch);
    else
        up32_kernel<512><<<dim3(ntx, nty), 512, FT_SMEM, s>>>(F, C, tx, ty, nu2, gs ? 1 : 0, wf, omw,
                                                              psi, psi_pitch);
    note_launch();
    return cudaGetLastError();
}

// The launch of a batched tile kernel over `count` items (nt threads, smem bytes; see BatchList).
template <class... Params, class... Args>
static void tile_launch(void (*kernel)(const TileItem*, int, unsigned*, Params...), int nt,
                        size_t smem, const TileItem* items, int count, unsigned* claim,
                        cudaStream_t s, Args... args)
{
    const int grid = batch_grid((const void*)kernel, nt, smem, count, claim != nullptr);
    kernel<<<grid, nt, smem, s>>>(items, count, claim, args...);
}

cudaError_t launch_b_down32(const TileItem* items, int count, const BatchLevel<float>* lv,
                            const int* active, int nu1, bool zero_u, bool gs, double w, cudaStream_t s,
                            int variant, unsigned* claim)
{
    if (count == 0) return cudaSuccess;
    const int z = zero_u ? 1 : 0, g = gs ? 1 : 0;
    const float wf = (float)w, omw = (float)(1.0 - w);
    if (variant == 2)
        tile_launch(b_down32_kernel<1024, 64>, 1024, ft_smem_down(64), items, count, claim, s,
                    lv, active, nu1, z, g, wf, omw);
    else if (variant == 3)
        tile_launch(b_down32_kernel<512, 32>, 512, ft_smem_down(32), items, count, claim, s,
                    lv, active, nu1, z, g, wf, omw);
    else
        tile_launch(b_down32_kernel<512, 64>, 512, ft_smem_down(64), items, count, claim, s,
                    lv, active, nu1, z, g, wf, omw);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_b_up32(const TileItem* items, int count, const BatchLevel<float>* lv,
                          const int* active, int nu2, bool gs, double w, cudaStream_t s,
                          const BatchLevel<double>* lv64, int variant, unsigned* claim)
{
    if (count == 0) return cudaSuccess;
    const int g = gs ? 1 : 0;
    const float wf = (float)w, omw = (float)(1.0 - w);
    if (variant == 2)
        tile_launch(b_up32_kernel<1024, 64>, 1024, ft_smem(64), items, count, claim, s,
                    lv, active, nu2, g, wf, omw, lv64);
    else if (variant == 3)
        tile_launch(b_up32_kernel<512, 32>, 512, ft_smem(32), items, count, claim, s,
                    lv, active, nu2, g, wf, omw, lv64);
    else
        tile_launch(b_up32_kernel<512, 64>, 512, ft_smem(64), items, count, claim, s,
                    lv, active, nu2, g, wf, omw, lv64);
    note_launch();
    return cudaGetLastError();
}

}  // namespace lap
