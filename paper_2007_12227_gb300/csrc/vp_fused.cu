// vp_fused.cu -- one-pass step: [Lambda_p^{-1}] + push + deposit + [Lambda_x^{-1}].
//
// Sec. III update w_fin = Lambda^{-1} Delta^T w_in with Lambda = Lambda_x (x) Lambda_p
// (tent basis). In cubic B-spline Galerkin mode the library keeps, between
// steps, s = Lambda_x^{-1} r where r = Delta^T w is the deposit; one step is then
//   w  = Lambda_p^{-1} s         (per column, on the source side)
//   r' = Delta^T w               (push every node, deposit with the B3 kernel)
//   s' = Lambda_x^{-1} r'        (per row, on the destination side)
// so each step reads and writes the mesh once. With the tent deposit or the
// lumped projection there is no solve and the state is w itself.
//
// One CTA owns one destination tile [X0, X0+TX) x [P0, P0+TP). It keeps a
// shared-memory window: the tile widened by the x-solve halo D and a guard
// band G. It bounds the source nodes whose pushed B3 footprint reaches the
// widened tile and gives each thread one source column. The thread walks the
// column:
//   * Galerkin: the p solve is the Thomas algorithm for tridiag(1/6, 2/3, 1/6)
//     (exact pivots near row 0), walked downwards in chunks of kC rows: the
//     forward sweep of a chunk starts kHalo rows below it (truncation
//     |z|^kHalo, z = sqrt(3) - 2) and is kept in a shared-memory column buffer;
//     the back substitution carries on from the chunk above;
//   * every node is pushed (displacement tables, vp_internal.h) and its N x N
//     taps accumulate in an N x N register ring that follows the node's base
//     row; when the ring moves one row, the row that leaves it is added to the
//     window with N shared-memory atomics.
// Contributions outside the window belong to other tiles, except rows beyond
// the open momentum edge, which are counted as lost by the tile owning the
// column. Finally each warp takes window rows, solves Lambda_x along them
// (first-order recurrences over per-lane chunks, combined across lanes by a warp
// scan, or on windowed rows by the carries of the neighbouring chunks), and the
// tile is stored once.
#include <math.h>

#include "vp_fel.cuh"
#include "vp_internal.h"
#include "vp_sum.cuh"

namespace vp {
namespace {

// look-ahead / x-solve halo: |z|^16 = 7e-10 (FP32; also keeps stores 16-byte aligned),
// |z|^28 = 1e-16 (FP64)
template <typename T>
struct Halo {
    static constexpr int value = sizeof(T) == 4 ? 16 : 28;
};
constexpr int kC = 16;              // rows per chunk of the p solve (multiple of 4)
// rows of the per-thread column buffer: one chunk, or the look-ahead above the top row
template <typename T>
struct GRows {
    static constexpr int value = kC > Halo<T>::value ? kC : Halo<T>::value;
};
constexpr int kXBig = kFusedMaxRow / 32;   // elements per lane for rows up to kFusedMaxRow

template <typename T, int BASIS>
struct FTaps;

template <typename T>
struct FTaps<T, VP_BASIS_TENT> {
    static constexpr int N = 2;
    static constexpr int LO = 0;
    __device__ __forceinline__ static void weights(T t, T *w)
    {
        w[0] = T(1) - t;
        w[1] = t;
    }
};

// FP32: three weights on the grid 2^-23, the fourth one minus them, so that the four sum to
// exactly one (see node_taps_f32); FP64: the fourth from the other three
__device__ __forceinline__ float grid23(float x) { return __fadd_rn(__fadd_rn(x, 1.f), -1.f); }
__device__ __forceinline__ double grid23(double x) { return x; }

template <typename T>
struct FTaps<T, VP_BASIS_CUBIC_BSPLINE> {
    static constexpr int N = 4;
    static constexpr int LO = -1;
    // cubic B-spline at offsets 1+t, t, 1-t, 2-t
    __device__ __forceinline__ static void weights(T t, T *w)
    {
        const T s = T(1) - t;
        const T t2 = t * t, s2 = s * s;
        const T t3 = t2 * t, s3 = s2 * s;
        const T sixth = T(1) / T(6), two3 = T(2) / T(3);
        w[0] = grid23(s3 * sixth);
        w[3] = grid23(t3 * sixth);
        w[1] = grid23(two3 - t2 + T(0.5) * t3);
        // the weights sum to one: forming w[2] from the formula instead would carry the rounding
        // of 2/3 (FP32: a mean excess of 4e-8 per axis) into the mass of every step
        w[2] = ((T(1) - w[0]) - w[3]) - w[1];
    }
};

__device__ __forceinline__ int imod(int a, int n)
{
    int r = a % n;
    return r < 0 ? r + n : r;
}

// z^n for the pole z = sqrt(3) - 2 < 0
template <typename T>
__device__ __forceinline__ T zpow(int n);

template <>
__device__ __forceinline__ float zpow<float>(int n)
{
    // log2|z| = log2(2 - sqrt(3))
    const float m = exp2f((float)n * -1.8999686269529425f);
    return (n & 1) ? -m : m;
}

template <>
__device__ __forceinline__ double zpow<double>(int n)
{
    const double m = exp2((double)n * -1.8999686269529425);
    return (n & 1) ? -m : m;
}

// range of sin over [lo, hi] in FP32 (|lo|, |hi| < 1e3), widened by 1e-4
__device__ void sin_range32(float lo, float hi, float &smin, float &smax)
{
    const float twopi = 6.28318530717958647692f;
    if (hi - lo >= twopi - 1e-4f) {
        smin = -1.f;
        smax = 1.f;
        return;
    }
    const float k = floorf(lo / twopi);
    const float a = lo - k * twopi, b = hi - k * twopi;
    const float sa = sinf(a), sb = sinf(b);
    smin = fminf(sa, sb) - 1e-4f;
    smax = fmaxf(sa, sb) + 1e-4f;
    const float h1 = 1.57079632679f, h3 = 4.71238898038f;
    if ((a <= h1 + 1e-4f && h1 - 1e-4f <= b) || (a <= h1 + twopi + 1e-4f && h1 + twopi - 1e-4f <= b))
        smax = 1.f;
    if ((a <= h3 + 1e-4f && h3 - 1e-4f <= b) || (a <= h3 + twopi + 1e-4f && h3 + twopi - 1e-4f <= b))
        smin = -1.f;
}

// Window cells. FP32: fixed-point integers at a per-tile scale, so that the deposit uses
// native integer shared-memory atomics (a float atomicAdd on shared memory is a
// compare-and-swap loop) and the sums do not depend on the order of the additions: the
// FP32 step is bit-reproducible. FP64: doubles.
__device__ __forceinline__ void wadd(float *p, float v)
{
    atomicAdd(reinterpret_cast<int *>(p), __float2int_rn(v));
}
__device__ __forceinline__ void wadd(double *p, double v) { atomicAdd(p, v); }
// raw cell value (in the tile's scaled units)
__device__ __forceinline__ double wraw(const float *p) { return (double)*reinterpret_cast<const int *>(p); }
__device__ __forceinline__ double wraw(const double *p) { return *p; }
// cell value in weight units
__device__ __forceinline__ float wget(const float *p, float iq)
{
    return (float)*reinterpret_cast<const int *>(p) * iq;
}
__device__ __forceinline__ double wget(const double *p, double) { return *p; }
__device__ __forceinline__ void wfold(float *d, const float *s)
{
    *reinterpret_cast<int *>(d) += *reinterpret_cast<const int *>(s);
}
__device__ __forceinline__ void wfold(double *d, const double *s) { *d += *s; }

template <typename T, int N>
struct Ring {
    T acc[N][N];  // [slot][column]
    int mref;     // window column of tap a = 0
    int nb;       // window row of tap b = 0 of the last node
    bool col_ok;  // all N columns inside the window
    bool live;
};

struct WinGeom {
    int WW, WH, ws;      // window width, height, row stride (elements)
    int WX0, WP0;        // grid column (unwrapped) and row of window cell (0, 0)
    int own_c0, own_c1;  // the tile's own columns, window coordinates [c0, c1)
    int np, nx, G;
    bool full;           // the tile spans the whole period
};

// One cell outside the fast window range: wrap (whole-period tiles), add, or count
// as lost (rows beyond the open momentum edge, own columns). Returns the lost weight.
template <typename T>
__device__ __noinline__ double flush_cell_slow(T *win, const WinGeom W, T v, int c, int row)
{
    if (W.full && (c < 0 || c >= W.WW)) c = W.G + imod(c - W.G, W.nx);
    const int grow = row + W.WP0;
    const bool outside = grow < 0 || grow >= W.np;
    if (c >= 0 && c < W.WW) {
        if (row >= 0 && row < W.WH) {
            wadd(win + row * W.ws + c, v);
            return 0.0;
        }
        if (outside && (W.full || (c >= W.own_c0 && c < W.own_c1))) return (double)v;
    }
    return 0.0;
}

template <typename T>
__device__ __forceinline__ void flush_cell(T *win, const WinGeom &W, T v, int c, int row, double &lost)
{
    if (row >= 0 && row < W.WH && c >= 0 && c < W.WW) wadd(win + row * W.ws + c, v);
    else lost += flush_cell_slow<T>(win, W, v, c, row);
}

template <typename T, int N>
__device__ __forceinline__ void flush_row(T *win, const WinGeom &W, const T *acc, int mref,
                                          bool col_ok, int row, double &lost)
{
    if (row >= 0 && row < W.WH && col_ok) {
        T *p = win + row * W.ws + mref;
#pragma unroll
        for (int a = 0; a < N; ++a) wadd(p + a, acc[a]);
    } else {
#pragma unroll
        for (int a = 0; a < N; ++a) lost += flush_cell_slow<T>(win, W, acc[a], mref + a, row);
    }
}

// Add one node (weights wx, wy; base window column m, row n). acc[b] always holds
// window row nb + b. DIR = +1: base rows ascend between consecutive nodes (the
// bottom row leaves); DIR = -1: they descend (the top row leaves). The row shift
// is folded into the accumulation: acc[b] = acc[b +/- 1] + wy[b] wx.
template <typename T, int N, int DIR>
__device__ __forceinline__ void ring_add(T *win, const WinGeom &W, Ring<T, N> &rg, int m, int n,
                                         const T *wx, const T *wy, double &lost)
{
    {
        // common case: one row leaves the ring, nothing else changes. Each lane decides for
        // itself (a warp vote here measured slower: lanes that fail diverge only briefly)
        const int rl = DIR > 0 ? rg.nb : rg.nb + N - 1;
        const bool fast = rg.live && n == rg.nb + DIR && m == rg.mref && rg.col_ok &&
                          (unsigned)rl < (unsigned)W.WH;
        if (fast) {
            T *p = win + rl * W.ws + rg.mref;
            if (DIR > 0) {
#pragma unroll
                for (int a = 0; a < N; ++a) wadd(p + a, rg.acc[0][a]);
#pragma unroll
                for (int b = 0; b < N - 1; ++b)
#pragma unroll
                    for (int a = 0; a < N; ++a) rg.acc[b][a] = rg.acc[b + 1][a] + wy[b] * wx[a];
#pragma unroll
                for (int a = 0; a < N; ++a) rg.acc[N - 1][a] = wy[N - 1] * wx[a];
            } else {
#pragma unroll
                for (int a = 0; a < N; ++a) wadd(p + a, rg.acc[N - 1][a]);
#pragma unroll
                for (int b = N - 1; b > 0; --b)
#pragma unroll
                    for (int a = 0; a < N; ++a) rg.acc[b][a] = rg.acc[b - 1][a] + wy[b] * wx[a];
#pragma unroll
                for (int a = 0; a < N; ++a) rg.acc[0][a] = wy[0] * wx[a];
            }
            rg.nb = n;
            return;
        }
    }
    const bool step_ok = rg.live && n == rg.nb + DIR;
    if (step_ok && (m == rg.mref + 1 || m == rg.mref - 1)) {
        // the base column moved by one: flush the column that leaves, shift the rest
        if (m > rg.mref) {
#pragma unroll
            for (int b = 0; b < N; ++b) {
                flush_cell<T>(win, W, rg.acc[b][0], rg.mref, rg.nb + b, lost);
#pragma unroll
                for (int a = 0; a < N - 1; ++a) rg.acc[b][a] = rg.acc[b][a + 1];
                rg.acc[b][N - 1] = T(0);
            }
        } else {
#pragma unroll
            for (int b = 0; b < N; ++b) {
                flush_cell<T>(win, W, rg.acc[b][N - 1], rg.mref + N - 1, rg.nb + b, lost);
#pragma unroll
                for (int a = N - 1; a > 0; --a) rg.acc[b][a] = rg.acc[b][a - 1];
                rg.acc[b][0] = T(0);
            }
        }
        rg.mref = m;
        rg.col_ok = (unsigned)m <= (unsigned)(W.WW - N);   // overflow-safe for any m
    }
    if (step_ok && m == rg.mref) {
        if (DIR > 0) {
            flush_row<T, N>(win, W, rg.acc[0], rg.mref, rg.col_ok, rg.nb, lost);
#pragma unroll
            for (int b = 0; b < N - 1; ++b)
#pragma unroll
                for (int a = 0; a < N; ++a) rg.acc[b][a] = rg.acc[b + 1][a] + wy[b] * wx[a];
#pragma unroll
            for (int a = 0; a < N; ++a) rg.acc[N - 1][a] = wy[N - 1] * wx[a];
        } else {
            flush_row<T, N>(win, W, rg.acc[N - 1], rg.mref, rg.col_ok, rg.nb + N - 1, lost);
#pragma unroll
            for (int b = N - 1; b > 0; --b)
#pragma unroll
                for (int a = 0; a < N; ++a) rg.acc[b][a] = rg.acc[b - 1][a] + wy[b] * wx[a];
#pragma unroll
            for (int a = 0; a < N; ++a) rg.acc[0][a] = wy[0] * wx[a];
        }
        rg.nb = n;
        return;
    }
    // anything else (first node, a jump): flush the whole ring and restart
    if (rg.live) {
#pragma unroll
        for (int b = 0; b < N; ++b) flush_row<T, N>(win, W, rg.acc[b], rg.mref, rg.col_ok, rg.nb + b, lost);
    }
#pragma unroll
    for (int b = 0; b < N; ++b)
#pragma unroll
        for (int a = 0; a < N; ++a) rg.acc[b][a] = wy[b] * wx[a];
    rg.mref = m;
    rg.nb = n;
    rg.col_ok = (unsigned)m <= (unsigned)(W.WW - N);
    rg.live = true;
}

template <typename T, int N>
__device__ __forceinline__ void ring_final(T *win, const WinGeom &W, Ring<T, N> &rg, double &lost)
{
    if (!rg.live) return;
#pragma unroll
    for (int b = 0; b < N; ++b) flush_row<T, N>(win, W, rg.acc[b], rg.mref, rg.col_ok, rg.nb + b, lost);
    rg.live = false;
}

// floor of x as a value and as an int without float-to-int conversion instructions:
// adding 1.5 * 2^(mantissa bits) rounds to an integer held in the low mantissa bits
// (valid for |x| < 2^22 in FP32, 2^51 in FP64); one compare turns rounding into floor.
__device__ __forceinline__ void floor_split(float x, float &fl, int &i)
{
    const float magic = 12582912.0f;   // 1.5 * 2^23
    const float t = x + magic;
    float r = t - magic;
    int k = __float_as_int(t) - 0x4B400000;
    if (r > x) {
        r -= 1.0f;
        k -= 1;
    }
    fl = r;
    i = k;
}

__device__ __forceinline__ void floor_split(double x, double &fl, int &i)
{
    const double magic = 6755399441055744.0;   // 1.5 * 2^52
    const double t = x + magic;
    double r = t - magic;
    int k = (int)(__double_as_longlong(t) - 0x4338000000000000LL);
    if (r > x) {
        r -= 1.0;
        k -= 1;
    }
    fl = r;
    i = k;
}

template <typename T>
struct ColC {
    int ui, vi;
    T uf, vf, cu1, cu2, cv1, cv2;
};

// FP32 pairs (x half, p half) in one 64-bit register, for packed FADD2 / FMUL2 / FFMA2
typedef unsigned long long f2_t;
__device__ __forceinline__ f2_t f2_pack(float a, float b)
{
    f2_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void f2_unpack(f2_t r, float &a, float &b)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ f2_t f2_add(f2_t a, f2_t b)
{
    f2_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2_t f2_mul(f2_t a, f2_t b)
{
    f2_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2_t f2_fma(f2_t a, f2_t b, f2_t c)
{
    f2_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// FP32 node: push and tap weights of the x and p axes together in packed pairs. The base
// cell is round(x - 1/2), so the fraction t lies in [0, 1] (t = 1 at an exact node gives
// the same deposit as t = 0 one cell further: the B3 and tent kernels are continuous).
// SROW: the row entry lives in shared memory (the tile's row cache), else in global memory
template <int BASIS, bool UTERM, bool SROW>
__device__ __forceinline__ void node_taps_f32(const ColC<float> &c, const RowEntry<float> &r,
                                              int colrel, int rowrel, float w, int &m, int &n,
                                              float *wx, float *wy)
{
    const float4 *rq = reinterpret_cast<const float4 *>(&r);
    const float4 q0 = SROW ? rq[0] : __ldg(rq);       // ui, vi, uf, vf
    const float4 q1 = SROW ? rq[1] : __ldg(rq + 1);   // cy, cy, sy, sy
    f2_t F = f2_add(f2_pack(c.uf, c.vf), f2_pack(q0.z, q0.w));
    F = f2_fma(f2_pack(UTERM ? c.cu1 : 0.f, c.cv1), f2_pack(q1.x, q1.y), F);
    F = f2_fma(f2_pack(UTERM ? c.cu2 : 0.f, c.cv2), f2_pack(q1.z, q1.w), F);
    const f2_t M1 = f2_pack(-1.f, -1.f), ONE = f2_pack(1.f, 1.f);
    const f2_t MAG = f2_pack(12582912.f, 12582912.f);   // 1.5 * 2^23
    const f2_t TT = f2_add(f2_add(F, f2_pack(-0.5f, -0.5f)), MAG);
    const f2_t R = f2_add(TT, f2_pack(-12582912.f, -12582912.f));
    const f2_t T = f2_fma(R, M1, F);
    float tu_bits, tv_bits;
    f2_unpack(TT, tu_bits, tv_bits);
    const int iu = __float_as_int(tu_bits) - 0x4B400000, iv = __float_as_int(tv_bits) - 0x4B400000;
    using TP = FTaps<float, BASIS>;
    m = colrel + c.ui + __float_as_int(q0.x) + iu + TP::LO;
    n = rowrel + c.vi + __float_as_int(q0.y) + iv + TP::LO;
    const f2_t S = f2_fma(T, M1, ONE);
    if (BASIS == VP_BASIS_TENT) {
        f2_unpack(S, wx[0], wy[0]);
        f2_unpack(T, wx[1], wy[1]);
    } else {
        const f2_t T2 = f2_mul(T, T), S2 = f2_mul(S, S);
        const f2_t T3 = f2_mul(T2, T), S3 = f2_mul(S2, S);
        const float sixth = 1.f / 6.f, two3 = 2.f / 3.f;
        const f2_t SIX = f2_pack(sixth, sixth);
        // three weights rounded to multiples of 2^-23 ((x + 1) - 1), the fourth 1 minus them:
        // every step is then exact and the four sum to exactly one, so the step keeps the mass
        // up to unbiased rounding whatever the fractions (a pushed node at t = 0, as in a slow
        // or resting flow, would otherwise lose 2^-26 of its weight per axis and step)
        const f2_t MONE = f2_pack(-1.f, -1.f);
        const f2_t W0 = f2_add(f2_add(f2_mul(S3, SIX), ONE), MONE);
        const f2_t W3 = f2_add(f2_add(f2_mul(T3, SIX), ONE), MONE);
        const f2_t W1 = f2_add(f2_add(f2_fma(T3, f2_pack(0.5f, 0.5f), f2_fma(T2, M1, f2_pack(two3, two3))),
                                      ONE), MONE);
        const f2_t W2 = f2_fma(W1, M1, f2_fma(W3, M1, f2_fma(W0, M1, ONE)));
        f2_unpack(W0, wx[0], wy[0]);
        f2_unpack(W1, wx[1], wy[1]);
        f2_unpack(W2, wx[2], wy[2]);
        f2_unpack(W3, wx[3], wy[3]);
    }
#pragma unroll
    for (int b = 0; b < TP::N; ++b) wy[b] *= w;
}

template <typename T, int BASIS, bool UTERM, bool SROW>
__device__ __forceinline__ void node_taps(const ColC<T> &c, const RowEntry<T> &r, int colrel,
                                          int rowrel, T w, int &m, int &n, T *wx, T *wy)
{
    if constexpr (sizeof(T) == 4) {
        node_taps_f32<BASIS, UTERM, SROW>(c, r, colrel, rowrel, w, m, n, wx, wy);
        return;
    }
    using TP = FTaps<T, BASIS>;
    T fu = c.uf + r.uf;
    if (UTERM) fu += c.cu1 * r.cy + c.cu2 * r.sy;
    const T fv = (c.vf + r.vf) + c.cv1 * r.cy + c.cv2 * r.sy;
    T flu, flv;
    int iu, iv;
    floor_split(fu, flu, iu);
    floor_split(fv, flv, iv);
    m = colrel + c.ui + r.ui + iu + TP::LO;
    n = rowrel + c.vi + r.vi + iv + TP::LO;
    TP::weights(fu - flu, wx);
    TP::weights(fv - flv, wy);
#pragma unroll
    for (int b = 0; b < TP::N; ++b) wy[b] *= w;
}

// Lambda_x^{-1} (T x = row, T = tridiag(1/6, 2/3, 1/6)) of one row of length L held in
// shared memory, by one warp. Returns each lane's elements base .. base + per - 1 in v.
// cyclic: the row is one whole period; else the row is padded by the halo on both
// sides and the recurrences start from zero at its ends (truncation |z|^halo).
// padded staging layout of a row: element c at c + c / 8, so that lanes reading
// contiguous chunks of 8 hit distinct shared-memory banks
__device__ __forceinline__ int padc(int c) { return c + (c >> 3); }

template <typename T, int kXMax>
__device__ void solve_row_x(const T *row, int L, bool cyclic, int lane, T *v, int &per, int &base,
                            bool padded, T sh, T sl)
{
    per = (L + 31) / 32;
    base = lane * per;
    const T z = (T)-0.26794919243112270647;
#pragma unroll
    for (int k = 0; k < kXMax; ++k)
        v[k] = (k < per && base + k < L) ? row[padded ? padc(base + k) : base + k] : T(0);
    const T zper = zpow<T>(per);
    // causal y_i = x_i + z y_{i-1}: lane-local sweep, then carries by a warp scan
    T y = T(0);
#pragma unroll
    for (int k = 0; k < kXMax; ++k)
        if (k < per) {
            y = v[k] + z * y;
            v[k] = y;
        }
    T endv = y;
    T zp = zper;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const T o = __shfl_up_sync(0xffffffffu, endv, off);
        if (lane >= off) endv += zp * o;
        zp *= zp;
    }
    T carry = __shfl_up_sync(0xffffffffu, endv, 1);
    if (lane == 0) carry = T(0);
    {
        T zk = z;
#pragma unroll
        for (int k = 0; k < kXMax; ++k)
            if (k < per) {
                v[k] += zk * carry;
                zk *= z;
            }
    }
    if (cyclic) {
        // y_{-1} = y_{L-1}: with E the zero-start value at L-1, y_{-1} = E / (1 - z^L)
        const int ll = (L - 1) / per, kl = (L - 1) - ll * per;
        T mine = T(0);
#pragma unroll
        for (int k = 0; k < kXMax; ++k)
            if (k == kl) mine = v[k];
        const T E = __shfl_sync(0xffffffffu, mine, ll);
        const T yprev = E / (T(1) - zpow<T>(L));
        T zk = zpow<T>(base + 1);
#pragma unroll
        for (int k = 0; k < kXMax; ++k)
            if (k < per) {
                v[k] += zk * yprev;
                zk *= z;
            }
    }
    // anticausal u_i = y_i + z u_{i+1}
    int last = per - 1;
    if (base + last >= L) last = L - 1 - base;   // may be negative for idle lanes
    T u = T(0);
#pragma unroll
    for (int k = kXMax - 1; k >= 0; --k)
        if (k <= last) {
            u = v[k] + z * u;
            v[k] = u;
        }
    T startv = u;
    zp = zper;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const T o = __shfl_down_sync(0xffffffffu, startv, off);
        if (lane + off < 32) startv += zp * o;
        zp *= zp;
    }
    T carry2 = __shfl_down_sync(0xffffffffu, startv, 1);
    if (lane == 31) carry2 = T(0);
    {
        T zk = z;
#pragma unroll
        for (int k = kXMax - 1; k >= 0; --k)
            if (k <= last) {
                v[k] += zk * carry2;
                zk *= z;
            }
    }
    if (cyclic) {
        // u_L = u_0: with S the zero-end value at 0, u_L = S / (1 - z^L)
        const T S = __shfl_sync(0xffffffffu, v[0], 0);
        const T unext = S / (T(1) - zpow<T>(L));
        // element i gets z^{L - i} u_L
#pragma unroll
        for (int k = 0; k < kXMax; ++k)
            if (k <= last) v[k] += zpow<T>(L - (base + k)) * unext;
    }
    // the scale -6z; in FP32 the unit-DC-gain scale of the step as a float pair sh + sl
#pragma unroll
    for (int k = 0; k < kXMax; ++k) v[k] = sizeof(T) == 4 ? v[k] * sh + v[k] * sl : v[k] * sh;
}

// z^n for the pole z = sqrt(3) - 2, at compile time
constexpr double zconst(int n)
{
    double r = 1.0;
    for (int k = 0; k < n; ++k) r *= -0.26794919243112270647;
    return r;
}

// Lambda_x^{-1} of one window row of exactly 32 KX elements (the common case of the
// windowed tiles): the recurrences start from zero at both row ends and every power of z
// the lane sweeps and the carries need is a compile-time constant. row == nullptr: v
// already holds the lane's KX elements.
// A lane's carry is the recurrence value at the end of the chunks next to it. Where the
// halo spans at most three chunks it sums only those chunks' zero-start end values (two
// or three shuffles, no scan): what it leaves out is weighted by |z|^halo or less, the
// truncation the recurrences already have at the window ends.
template <typename T, int KX>
__device__ __forceinline__ void solve_row_x_exact(const T *row, int lane, T *v, bool padded, T sh,
                                                  T sl)
{
    const int base = lane * KX;
    const T z = (T)zconst(1);
    if (row)
#pragma unroll
        for (int k = 0; k < KX; ++k) v[k] = row[padded ? padc(base + k) : base + k];
    // causal y_i = x_i + z y_{i-1}: lane-local, then the carry of the lanes below
    T y = T(0);
#pragma unroll
    for (int k = 0; k < KX; ++k) {
        y = v[k] + z * y;
        v[k] = y;
    }
    T endv = y;
    T carry = T(0);
    constexpr int NCH = (Halo<T>::value + KX - 1) / KX;
    if constexpr (NCH <= 3) {
#pragma unroll
        for (int c = 1; c <= NCH; ++c) {
            const T o = __shfl_up_sync(0xffffffffu, endv, c);
            if (lane >= c) carry += (T)zconst((c - 1) * KX) * o;
        }
    } else {
#pragma unroll
        for (int s = 0; s < 5; ++s) {
            const T o = __shfl_up_sync(0xffffffffu, endv, 1 << s);
            if (lane >= (1 << s)) endv += (T)zconst(KX << s) * o;
        }
        carry = __shfl_up_sync(0xffffffffu, endv, 1);
        if (lane == 0) carry = T(0);
    }
#pragma unroll
    for (int k = 0; k < KX; ++k) v[k] += (T)zconst(k + 1) * carry;
    // anticausal u_i = y_i + z u_{i+1}
    T u = T(0);
#pragma unroll
    for (int k = KX - 1; k >= 0; --k) {
        u = v[k] + z * u;
        v[k] = u;
    }
    T startv = u;
    T carry2 = T(0);
    if constexpr (NCH <= 3) {
#pragma unroll
        for (int c = 1; c <= NCH; ++c) {
            const T o = __shfl_down_sync(0xffffffffu, startv, c);
            if (lane + c < 32) carry2 += (T)zconst((c - 1) * KX) * o;
        }
    } else {
#pragma unroll
        for (int s = 0; s < 5; ++s) {
            const T o = __shfl_down_sync(0xffffffffu, startv, 1 << s);
            if (lane + (1 << s) < 32) startv += (T)zconst(KX << s) * o;
        }
        carry2 = __shfl_down_sync(0xffffffffu, startv, 1);
        if (lane == 31) carry2 = T(0);
    }
#pragma unroll
    for (int k = 0; k < KX; ++k) v[k] += (T)zconst(KX - k) * carry2;
#pragma unroll
    for (int k = 0; k < KX; ++k) v[k] = sizeof(T) == 4 ? v[k] * sh + v[k] * sl : v[k] * sh;
}

}  // namespace

// The window's own cells in weight units into the destination rows: one warp per row, FP32 rows
// with 16-byte loads of the fixed-point cells and 16-byte stores where the destination row allows.
// MAX: track max|value| in om (the stored state's per-tile maximum) and flag non-finite values
// (FP64 cells; FP32 cells are integers times a finite scale).
template <typename T, bool MAX>
__device__ __forceinline__ void store_window_rows(const T *win, const WinGeom &W, T *dst, int nx, int P0,
                                                  int X0, int TXe, int TPe, int G, int Gp, T iq, int warp,
                                                  int nwarps, int lane, float &om, bool &bad)
{
    for (int rr = warp; rr < TPe; rr += nwarps) {
        const T *row = win + (size_t)(rr + Gp) * W.ws + G;
        T *drow = dst + (size_t)(P0 + rr) * nx + X0;
        int c0 = 0;
        if constexpr (sizeof(T) == 4) {
            if ((reinterpret_cast<uintptr_t>(drow) & 15) == 0) {
                const int n4 = TXe >> 2;
                const int4 *r4 = reinterpret_cast<const int4 *>(row);
                float4 *d4 = reinterpret_cast<float4 *>(drow);
                for (int c4 = lane; c4 < n4; c4 += 32) {
                    const int4 q = r4[c4];
                    const float4 o = make_float4((float)q.x * iq, (float)q.y * iq, (float)q.z * iq, (float)q.w * iq);
                    d4[c4] = o;
                    if (MAX) om = fmaxf(om, fmaxf(fmaxf(fabsf(o.x), fabsf(o.y)), fmaxf(fabsf(o.z), fabsf(o.w))));
                }
                c0 = n4 << 2;
            }
        }
        for (int c = c0 + lane; c < TXe; c += 32) {
            const T v = wget(row + c, iq);
            drow[c] = v;
            if (MAX) {
                om = fmaxf(om, fabsf((float)v));
                bad |= !isfinite(v);
            }
        }
    }
}

// Lambda_x solve of the tile's window rows (one warp per row) and the tile store.
template <typename T, int KX>
__device__ __forceinline__ void gal_rows(T *win, const WinGeom &W, T *dst, int L, bool full, int D,
                                         int G, int Gp, int TXe, int TPe, int P0, int X0, int nx,
                                         bool want_part, int warp, int nwarps, int lane, bool &bad,
                                         T *stage_all, int stage_len, T sh, T sl, T iq, float &om)
{
    // per-warp padded copy of the row (conflict-free reads of contiguous chunks)
    const int plen = padc(L) + 8;
    const bool use_stage = stage_all != nullptr && (size_t)nwarps * plen <= (size_t)stage_len;
    T *stage = use_stage ? stage_all + (size_t)warp * plen : nullptr;
    for (int rr = warp; rr < TPe; rr += nwarps) {
        T *row = win + (size_t)(rr + Gp) * W.ws + G;
        T *dst_row = dst + (size_t)(P0 + rr) * nx + X0 - D;
        T v[KX];
        int per, base;
        const bool exact = !full && L == 32 * KX;
        // FP32 rows of 32 KX cells starting 16-byte aligned: each lane reads its chunk of
        // fixed-point cells with vector loads, without a staging copy
        const bool direct = sizeof(T) == 4 && exact && KX % 4 == 0 &&
                            ((reinterpret_cast<uintptr_t>(row) & 15) == 0);
        if (direct) {
            const int4 *r4 = reinterpret_cast<const int4 *>(row + lane * KX);
#pragma unroll
            for (int k4 = 0; k4 < KX / 4; ++k4) {
                const int4 q = r4[k4];
                v[4 * k4 + 0] = (T)q.x * iq;
                v[4 * k4 + 1] = (T)q.y * iq;
                v[4 * k4 + 2] = (T)q.z * iq;
                v[4 * k4 + 3] = (T)q.w * iq;
            }
        } else if (use_stage) {
            // window cells to weight units: into the staging copy, else in place
            for (int c = lane; c < L; c += 32) stage[padc(c)] = wget(row + c, iq);
        } else if (sizeof(T) == 4) {
            for (int c = lane; c < L; c += 32) row[c] = wget(row + c, iq);
        }
        __syncwarp();
        if (exact) {
            solve_row_x_exact<T, KX>(direct ? nullptr : (use_stage ? stage : row), lane, v,
                                     use_stage && !direct, sh, sl);
            per = KX;
            base = lane * KX;
        } else {
            solve_row_x<T, KX>(use_stage ? stage : row, L, full, lane, v, per, base, use_stage, sh, sl);
        }
        __syncwarp();
        // v * 0 is 0 for finite values and NaN otherwise
        T chk = T(0);
        T *dp = dst_row + base;
        const bool inside = per == KX && base >= D && base + KX <= D + TXe;
        if (sizeof(T) == 4 && KX % 4 == 0 && inside && ((reinterpret_cast<uintptr_t>(dp) & 15) == 0)) {
#pragma unroll
            for (int k = 0; k < KX; k += 4) {
                float4 q;
                q.x = (float)v[k];
                q.y = (float)v[k + 1];
                q.z = (float)v[k + 2];
                q.w = (float)v[k + 3];
                *reinterpret_cast<float4 *>(dp + k) = q;
            }
#pragma unroll
            for (int k = 0; k < KX; ++k) chk = fma(v[k], T(0), chk);
            if (sizeof(T) == 4)
#pragma unroll
                for (int k = 0; k < KX; ++k) om = fmaxf(om, fabsf((float)v[k]));
            if (want_part) {
                // keep s for the column sums: 16-byte stores (lanes 8 words apart: two-way bank
                // conflicts instead of the eight-way of word stores) when the row start allows
                if ((reinterpret_cast<uintptr_t>(row) & 15) == 0) {
#pragma unroll
                    for (int k = 0; k < KX; k += 4) {
                        float4 q;
                        q.x = (float)v[k];
                        q.y = (float)v[k + 1];
                        q.z = (float)v[k + 2];
                        q.w = (float)v[k + 3];
                        *reinterpret_cast<float4 *>(row + base + k) = q;
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < KX; ++k) row[base + k] = v[k];
                }
            }
        } else if (!(exact && (base + KX <= D || base >= D + TXe))) {
            // (lanes whose chunk lies in the halo store nothing)
#pragma unroll
            for (int k = 0; k < KX; ++k) {
                const int c = base + k;
                if (k < per && c >= D && c < D + TXe) {
                    dst_row[c] = v[k];
                    chk = fma(v[k], T(0), chk);
                    om = fmaxf(om, fabsf((float)v[k]));
                    if (want_part) row[c] = v[k];   // keep s for the column sums
                }
            }
        }
        bad |= chk != T(0);
    }
}

// ---------------------------------------------------------------------------
// One destination tile of one simulation (A may live in shared or global memory).
template <typename T, int BASIS, bool GAL, bool UTERM>
__device__ __forceinline__ void fused_tile(const FusedArgs<T> &A, const int tile,
                                           unsigned char *smem_raw)
{
    using TP = FTaps<T, BASIS>;
    constexpr int N = TP::N;
    constexpr int R = (BASIS == VP_BASIS_TENT) ? 1 : 2;
    T *win = reinterpret_cast<T *>(smem_raw);
    T *gcol = win + (size_t)A.ws * (A.tp + 2 * A.Gp);   // [GRows][blockDim] column buffer (Galerkin)
    // row cache: the tile's rows ja .. jb of the push's row table (when they fit)
    RowEntry<T> *rowc = reinterpret_cast<RowEntry<T> *>(gcol + (size_t)GRows<T>::value * blockDim.x);
    __shared__ int s_ia, s_ib, s_ja, s_jb, s_smax, s_omax, s_cached;
    __shared__ double s_r4[4][kFusedMaxThreads / 32];
    // Thomas pivots of tridiag(1/6, 2/3, 1/6) in T: entry kPivots holds the limit
    __shared__ T piv_cp[kPivots + 1], piv_ib[kPivots + 1];
    __shared__ T sig_s[kFusedMaxTileP];   // column-sum weights of Lambda_p^{-1} for the tile rows

    const Geometry &g = A.g;
    const int nx = g.nx, np = g.np;
    const int tix = tile % A.ntx, tip = tile / A.ntx;
    const int X0 = tix * A.tx, P0 = tip * A.tp;
    const int TXe = min(A.tx, nx - X0), TPe = min(A.tp, np - P0);
    const bool full = A.full_row != 0;
    constexpr int kHalo = Halo<T>::value;
    // x halo of the in-tile x solve (none for whole-period tiles and for a separate x pass)
    const int D = (GAL && !full && !A.xpass) ? kHalo : 0;
    const int G = A.G, Gp = A.Gp;   // guard bands: columns, rows
    WinGeom W;
    W.WW = full ? nx + 2 * G : TXe + 2 * D + 2 * G;
    W.WH = TPe + 2 * Gp;
    W.ws = A.ws;
    W.WX0 = X0 - D - G;
    W.WP0 = P0 - Gp;
    W.own_c0 = G + D;
    W.own_c1 = G + D + TXe;
    W.np = np;
    W.nx = nx;
    W.G = G;
    W.full = full;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;

    {
        const int nvec = (int)(((size_t)W.WH * W.ws * sizeof(T)) / 16);
        uint4 *w4 = reinterpret_cast<uint4 *>(win);
        for (int k = tid; k < nvec; k += blockDim.x) w4[k] = make_uint4(0, 0, 0, 0);
        for (int k = nvec * (16 / (int)sizeof(T)) + tid; k < W.WH * W.ws; k += blockDim.x) win[k] = T(0);
    }
    for (int k = tid; k <= kPivots; k += blockDim.x) {
        piv_cp[k] = (T)A.piv[2 * k];
        piv_ib[k] = (T)A.piv[2 * k + 1];
    }
    if (GAL && A.fel_partials)
        for (int k = tid; k < TPe; k += blockDim.x) sig_s[k] = (T)A.sigma[P0 + k];
    if (tid == 0) {
        const int4 e = A.tile_src ? A.tile_src[tile] : make_int4(kTileSrcUnset, 0, 0, 0);
        s_cached = e.x != kTileSrcUnset;
        s_ia = s_cached ? e.x : 0x7fffffff;
        s_ib = s_cached ? e.y : -0x7fffffff;
        s_ja = s_cached ? e.z : 0x7fffffff;
        s_jb = s_cached ? e.w : -0x7fffffff;
        s_smax = 0;
        s_omax = 0;
    }
    double al = g.alpha0, be = g.beta0, M = g.m0, phi = g.phi0;
    if (g.kind == VP_PUSH_FEL_DKD) {
        al = -A.state[ST_K_IM];
        be = A.state[ST_K_RE];
        M = A.state[ST_M];
        phi = A.state[ST_PHI];
    }
    __syncthreads();

    // ---- bound the source nodes whose footprint can reach the widened tile (FP32 with
    //      slack: every magnitude here is below 1e5 cells, where FP32 is exact to 1e-2);
    //      a push that does not change between steps gives the same bounds every step
    const bool cached = s_cached != 0;
    if (!cached) {
        const float SL = 0.05f;
        const float Mf = (float)M, phif = (float)phi;
        const float EU = fabsf((float)g.KU) * Mf, EV = fabsf((float)g.KV) * Mf;
        const float KVM = (float)g.KV * Mf;
        const float vcmin = (float)g.vc_min, vcmax = (float)g.vc_max;
        const float ucmin = (float)g.uc_min, ucmax = (float)g.uc_max;
        const float vd_min = vcmin + (float)g.vr_min - EV, vd_max = vcmax + (float)g.vr_max + EV;
        const float x0f = (float)g.x0, hxf = (float)g.hx, padf = (float)g.a_pad;
        const bool edge_lo = P0 == 0, edge_hi = P0 + TPe == np;
        const int jlo = edge_lo ? 0 : max(0, (int)floorf((float)(P0 - R) - vd_max - SL));
        const int jhi = edge_hi ? np - 1 : min(np - 1, (int)ceilf((float)(P0 + TPe - 1 + R) - vd_min + SL));
        const float acc_lo = edge_lo ? -1e30f : (float)(P0 - R);
        const float acc_hi = edge_hi ? 1e30f : (float)(P0 + TPe - 1 + R);
        int my_ia = 0x7fffffff, my_ib = -0x7fffffff, my_ja = 0x7fffffff, my_jb = -0x7fffffff;
        for (int j = jlo + tid; j <= jhi; j += blockDim.x) {
            const float4 rb = A.rowbf[j];   // u, v, y
            int ia, ib;
            float vcl = vcmin, vch = vcmax;
            float smin = -1.f, smax = 1.f;
            if (full) {
                ia = 0;
                ib = nx - 1;
            } else {
                ia = (int)floorf((float)(X0 - D - R) - rb.x - EU - ucmax - SL);
                ib = (int)ceilf((float)(X0 + TXe + D - 1 + R) - rb.x + EU - ucmin + SL);
                const int width = ib - ia + 1;
                if (width < nx - 2 * kColBlock) {
                    vcl = 1e30f;
                    vch = -1e30f;
                    const int start = imod(ia, nx);
                    int seg_lo[2], seg_hi[2], nseg = 1;
                    if (start + width <= nx) {
                        seg_lo[0] = start;
                        seg_hi[0] = start + width - 1;
                    } else {
                        seg_lo[0] = start;
                        seg_hi[0] = nx - 1;
                        seg_lo[1] = 0;
                        seg_hi[1] = start + width - 1 - nx;
                        nseg = 2;
                    }
                    for (int sg = 0; sg < nseg; ++sg)
                        for (int bq = seg_lo[sg] / kColBlock; bq <= seg_hi[sg] / kColBlock; ++bq) {
                            const float2 vb = A.vcbf[bq];
                            vcl = fminf(vcl, vb.x);
                            vch = fmaxf(vch, vb.y);
                        }
                    if (EV > 0.f)
                        sin_range32(x0f + ia * hxf - padf + rb.z + phif, x0f + ib * hxf + padf + rb.z + phif,
                                    smin, smax);
                }
            }
            float tlo = 0.f, thi = 0.f;
            if (EV > 0.f) {
                tlo = fminf(KVM * smin, KVM * smax);
                thi = fmaxf(KVM * smin, KVM * smax);
            }
            const float vlo = (float)j + rb.y + vcl + tlo - SL;
            const float vhi = (float)j + rb.y + vch + thi + SL;
            if (vhi > acc_lo && vlo < acc_hi) {
                my_ia = min(my_ia, ia);
                my_ib = max(my_ib, ib);
                my_ja = min(my_ja, j);
                my_jb = max(my_jb, j);
            }
        }
        if (my_jb >= my_ja) {
            atomicMin(&s_ia, my_ia);
            atomicMax(&s_ib, my_ib);
            atomicMin(&s_ja, my_ja);
            atomicMax(&s_jb, my_jb);
        }
    }
    __syncthreads();
    const int ia = s_ia, ib = s_ib, ja = s_ja, jb = s_jb;
    if (!cached && A.tile_src && tid == 0) A.tile_src[tile] = make_int4(ia, ib, ja, jb);
    double lost = 0.0;   // in the window's scaled units until the end of the tile

    // ---- FP32: fixed-point scale of the window from max|s| over the rows the walk reads, taken
    //      from the per-tile maxima the previous step (or vp_set_f) recorded for the state.
    //      The truncated Thomas solve keeps |w| <= 3 max|s| (forward gain 1/(beta - 1/6) <= 2.2,
    //      back substitution 1/(1 - c') <= 1.37); a cell sums the B3 taps of the nodes pushed near
    //      it, about one for an area-preserving flow: 8 times that bound fits in int32.
    T qs = T(1), iq = T(1);
    if (sizeof(T) == 4) {
        float mx = 0.f;
        if (jb >= ja) {
            const int r0 = GAL ? max(0, ja - kHalo) : ja, r1 = GAL ? min(np - 1, jb + kHalo) : jb;
            const int wsrc = min(ib - ia + 1, nx);
            for (int cidx = tid; cidx < wsrc; cidx += blockDim.x) {
                const int tc = imod(ia + cidx, nx) / A.tx;
                for (int tr = r0 / A.tp; tr <= r1 / A.tp; ++tr) mx = fmaxf(mx, A.smax_in[tr * A.ntx + tc]);
            }
        }
        if (mx > 0.f && mx <= 3.0e38f) atomicMax(&s_smax, __float_as_int(mx));
        if (__syncthreads_or(!(mx <= 3.0e38f))) {
            qs = T(0);   // a non-finite state, reported when it was written: its deposit is dropped
            iq = T(0);
        } else {
            // the scale is a power of two, so that iq = 1 / qs is exact (a rounded iq scales the
            // tile's weights by 1 +- 6e-8, a gain that repeats over the steps while the tile's
            // maximum stays put): qs = 2^(32 - e) with m = f 2^e, f in [0.5, 1), i.e. qs m in
            // [2^31, 2^32): a cell reaches 2^31 only at 4 to 8 times the largest weight (16 to 32
            // times with the Thomas gain bound), against about one for an area-preserving flow
            const float m = fmaxf(__int_as_float(s_smax), 1e-30f) * (GAL ? 3.1f : 1.f) * 8.f;
            int e2;
            frexpf(m, &e2);
            qs = (T)ldexpf(1.f, 32 - e2);
            iq = (T)ldexpf(1.f, e2 - 32);
        }
    }

    // ---- the row table of the source rows into shared memory, when it fits: every node of a
    //      row reads that row's entry, and a shared-memory load is shorter than an L1 hit
    const bool rows_cached = jb >= ja && jb - ja + 1 <= A.rowcache;
    if (rows_cached) {
        constexpr int kVec = (int)(sizeof(RowEntry<T>) / 16);
        const float4 *from = reinterpret_cast<const float4 *>(A.row + ja);
        float4 *to = reinterpret_cast<float4 *>(rowc);
        for (int k = tid; k < kVec * (jb - ja + 1); k += blockDim.x) to[k] = __ldg(from + k);
        __syncthreads();
    }
    const RowEntry<T> *srow = rowc - ja;   // srow[j]: row j (rows_cached only)

    // ---- walk the source columns
    if (jb >= ja) {
        int wsrc = ib - ia + 1;
        if (wsrc > nx) wsrc = nx;
        const T alT = (T)al, beT = (T)be, KU = (T)g.KU, KV = (T)g.KV;
        const T sixth = T(1) / T(6);
        for (int cidx = tid; cidx < wsrc; cidx += blockDim.x) {
            const int ic = ia + cidx;
            const int im = imod(ic, nx);
            const ColEntry<T> e = A.col[im];
            ColC<T> cc;
            cc.ui = e.ui;
            cc.vi = e.vi;
            cc.uf = e.uf;
            cc.vf = e.vf;
            // sine term: al sin(a + y) + be cos(a + y) = cy (al sa + be ca) + sy (al ca - be sa)
            const T Pc = alT * e.sa + beT * e.ca, Qc = alT * e.ca - beT * e.sa;
            cc.cu1 = KU * Pc;
            cc.cu2 = KU * Qc;
            cc.cv1 = KV * Pc;
            cc.cv2 = KV * Qc;
            const int colrel = ic - W.WX0;
            const T *src = A.src + im;
            Ring<T, N> rg;
            rg.live = false;
            rg.mref = 0;
            rg.nb = 0;
            rg.col_ok = false;
#pragma unroll
            for (int q = 0; q < N; ++q)
#pragma unroll
                for (int a = 0; a < N; ++a) rg.acc[q][a] = T(0);
            T wx[N], wy[N];
            if (!GAL) {
                // the deposit alone: each chunk of kC source rows is loaded first (all of its loads
                // in flight, kept in the column buffer), then walked upwards
                T *gc = gcol + tid;
                const int nth = blockDim.x;
                for (int c_lo = ja; c_lo <= jb; c_lo += kC) {
                    const int c_hi = min(jb, c_lo + kC - 1);
                    const T *sp = src + (size_t)c_lo * nx;
                    if (c_hi - c_lo + 1 == kC) {
#pragma unroll
                        for (int k = 0; k < kC; ++k) gc[k * nth] = __ldg(sp + (size_t)k * nx);
                    } else {
                        for (int k = 0; k <= c_hi - c_lo; ++k) gc[k * nth] = __ldg(sp + (size_t)k * nx);
                    }
                    if (rows_cached) {
#pragma unroll 1
                        for (int r = c_lo; r <= c_hi; ++r) {
                            int m, n;
                            node_taps<T, BASIS, UTERM, true>(cc, srow[r], colrel, r - W.WP0,
                                                             gc[(r - c_lo) * nth] * qs, m, n, wx, wy);
                            ring_add<T, N, 1>(win, W, rg, m, n, wx, wy, lost);
                        }
                    } else {
#pragma unroll 1
                        for (int r = c_lo; r <= c_hi; ++r) {
                            int m, n;
                            node_taps<T, BASIS, UTERM, false>(cc, A.row[r], colrel, r - W.WP0,
                                                              gc[(r - c_lo) * nth] * qs, m, n, wx, wy);
                            ring_add<T, N, 1>(win, W, rg, m, n, wx, wy, lost);
                        }
                    }
                }
                ring_final<T, N>(win, W, rg, lost);
            } else {
                // Lambda_p^{-1} s by the Thomas algorithm, walked downwards in chunks of
                // kC rows: forward sweep g_j = (s_j - g_{j-1}/6) / beta_j from kHalo rows
                // below the chunk (or from row 0), kept in the column buffer gcol;
                // back substitution w_j = g_j - c'_j w_{j+1} continues from the chunk above.
                T *gc = gcol + tid;
                const int nth = blockDim.x;
                T uv = T(0);
                {
                    // look-ahead above jb (exact when it reaches the last row)
                    const int top = min(np - 1, jb + kHalo);
                    if (top > jb) {
                        int rr = max(0, jb + 1 - kHalo);
                        const T *sp = src + (size_t)rr * nx;
                        T gv = T(0);
                        for (; rr <= jb; ++rr, sp += nx) gv = (*sp - sixth * gv) * piv_ib[min(rr, kPivots)];
                        for (; rr <= top; ++rr, sp += nx) {
                            gv = (*sp - sixth * gv) * piv_ib[min(rr, kPivots)];
                            gc[(rr - jb - 1) * nth] = gv;
                        }
                        for (rr = top; rr > jb; --rr) uv = gc[(rr - jb - 1) * nth] - piv_cp[min(rr, kPivots)] * uv;
                    }
                }
                const T ib_inf = piv_ib[kPivots], cp_inf = piv_cp[kPivots];
                const T ib6_inf = sixth * ib_inf;
                for (int c_hi = jb; c_hi >= ja; c_hi -= kC) {
                    const int c_lo = max(ja, c_hi - kC + 1);
                    int rr = max(0, c_lo - kHalo);
                    const T *sp = src + (size_t)rr * nx;
                    T gv = T(0);
                    if (c_lo - kHalo > kPivots) {
                        // far from the first row the pivots have their limits
                        if (c_hi - c_lo + 1 == kC) {
                            // whole chunk: warm-up and chunk rows as one unrolled sweep, so that all
                            // of its loads are in flight before the recurrence needs them
#pragma unroll
                            for (int k = 0; k < kHalo + kC; ++k) {
                                gv = __ldg(sp + (size_t)k * nx) * ib_inf - ib6_inf * gv;
                                if (k >= kHalo) gc[(k - kHalo) * nth] = gv;
                            }
                        } else {
#pragma unroll 16
                            for (; rr < c_lo; ++rr, sp += nx) gv = *sp * ib_inf - ib6_inf * gv;
#pragma unroll 16
                            for (; rr <= c_hi; ++rr, sp += nx) {
                                gv = *sp * ib_inf - ib6_inf * gv;
                                gc[(rr - c_lo) * nth] = gv;
                            }
                        }
                    } else {
                        for (; rr < c_lo; ++rr, sp += nx) gv = (*sp - sixth * gv) * piv_ib[min(rr, kPivots)];
                        for (; rr <= c_hi; ++rr, sp += nx) {
                            gv = (*sp - sixth * gv) * piv_ib[min(rr, kPivots)];
                            gc[(rr - c_lo) * nth] = gv;
                        }
                    }
                    if (c_lo > kPivots && rows_cached) {
                        const RowEntry<T> *rp = srow + c_hi;
#pragma unroll 1
                        for (int r = c_hi; r >= c_lo; --r, --rp) {
                            uv = gc[(r - c_lo) * nth] - cp_inf * uv;
                            int m, n;
                            node_taps<T, BASIS, UTERM, true>(cc, *rp, colrel, r - W.WP0, uv * qs, m, n, wx, wy);
                            ring_add<T, N, -1>(win, W, rg, m, n, wx, wy, lost);
                        }
                    } else if (c_lo > kPivots) {
                        const RowEntry<T> *rp = A.row + c_hi;
#pragma unroll 1
                        for (int r = c_hi; r >= c_lo; --r, --rp) {
                            uv = gc[(r - c_lo) * nth] - cp_inf * uv;
                            int m, n;
                            node_taps<T, BASIS, UTERM, false>(cc, *rp, colrel, r - W.WP0, uv * qs, m, n, wx, wy);
                            ring_add<T, N, -1>(win, W, rg, m, n, wx, wy, lost);
                        }
                    } else {
                        const RowEntry<T> *rp = A.row + c_hi;
                        for (int r = c_hi; r >= c_lo; --r, --rp) {
                            uv = gc[(r - c_lo) * nth] - piv_cp[min(r, kPivots)] * uv;
                            int m, n;
                            node_taps<T, BASIS, UTERM, false>(cc, *rp, colrel, r - W.WP0, uv * qs, m, n, wx, wy);
                            ring_add<T, N, -1>(win, W, rg, m, n, wx, wy, lost);
                        }
                    }
                }
                ring_final<T, N>(win, W, rg, lost);
            }
        }
    }
    __syncthreads();

    // ---- window rows beyond the open momentum edge: lost weight of the own columns
    if (W.WP0 < 0 || W.WP0 + W.WH > np)
    for (int rr = 0; rr < W.WH; ++rr) {
        const int grow = rr + W.WP0;
        if (grow >= 0 && grow < np) continue;
        const int c0 = full ? 0 : W.own_c0, c1 = full ? W.WW : W.own_c1;
        for (int c = c0 + tid; c < c1; c += blockDim.x) lost += wraw(win + rr * W.ws + c);
    }
    if (full) {
        // fold the guard columns onto the period: [-G, 0) -> [nx - G, nx), [nx, nx + G) -> [0, G)
        __syncthreads();
        for (int k = tid; k < TPe * G; k += blockDim.x) {
            const int rr = k / G + Gp, c = k - (k / G) * G;
            T *row = win + (size_t)rr * W.ws;
            wfold(row + nx + c, row + c);
            wfold(row + G + c, row + G + nx + c);
        }
    }
    __syncthreads();

    // ---- store the tile (Galerkin: after the Lambda_x solve); FEL column sums
    const bool want_part = A.fel_partials != 0;
    bool bad = false;
    float om = 0.f;   // FP32: max|s'| of the stored outputs
    double pw = 0.0, pc = 0.0, ps = 0.0;
    if (GAL && A.xpass) {
        // separate x pass: store the deposit r = Delta^T w of the own columns in weight units; the
        // row pass solves Lambda_x, records max|s'| per tile and checks the outputs
        store_window_rows<T, false>(win, W, A.dst, nx, P0, X0, TXe, TPe, G, Gp, iq, warp, nwarps, lane, om, bad);
    } else if (GAL) {
        const int L = full ? nx : TXe + 2 * D;
        const bool f32 = sizeof(T) == 4;
        const T sh = f32 ? (T)A.piv[kPivXsFused] : T(-6) * T(-0.26794919243112270647);
        const T sl = f32 ? (T)A.piv[kPivXsFused + 1] : T(0);
        if (L <= 256)
            gal_rows<T, 8>(win, W, A.dst, L, full, D, G, Gp, TXe, TPe, P0, X0, nx, want_part, warp,
                           nwarps, lane, bad, gcol, GRows<T>::value * blockDim.x, sh, sl, iq, om);
        else
            gal_rows<T, kXBig>(win, W, A.dst, L, full, D, G, Gp, TXe, TPe, P0, X0, nx, want_part,
                               warp, nwarps, lane, bad, gcol, GRows<T>::value * blockDim.x, sh, sl, iq,
                               om);
    } else {
        // no solve: the deposit is the new state (its max|w| sets the next step's window scale)
        store_window_rows<T, true>(win, W, A.dst, nx, P0, X0, TXe, TPe, G, Gp, iq, warp, nwarps, lane, om, bad);
    }
    if (want_part) {
        // FEL: column sums of w over the tile (Galerkin: sum_j w_ij = sum_j sigma_j s_ij; with a
        // separate x pass the window keeps the deposit r, and bunch_x turns its cos/sin sums into
        // those of s')
        __syncthreads();
        const bool sums_of_s = GAL && !A.xpass;
        for (int c = tid; c < TXe; c += blockDim.x) {
            // four interleaved compensated sums (rows rr = q mod 4), added in a fixed order at the
            // end: four independent chains of shared-memory loads and error-free steps instead of one
            DSum<T> acc[4];
            const T *cell = win + (size_t)Gp * W.ws + G + D + c;
            int rr = 0;
            for (; rr + 4 <= TPe; rr += 4, cell += 4 * W.ws) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    // in-tile x solve: the epilogue left s in the own columns; else the cells hold
                    // the deposit
                    const T v = sums_of_s ? cell[q * W.ws] : wget(cell + q * W.ws, iq);
                    if (GAL) acc[q].add_prod(sig_s[rr + q], v);
                    else acc[q].add(v);
                }
            }
#pragma unroll
            for (int q = 0; q < 3; ++q)
                if (rr + q < TPe) {
                    const T v = sums_of_s ? cell[q * W.ws] : wget(cell + q * W.ws, iq);
                    if (GAL) acc[q].add_prod(sig_s[rr + q], v);
                    else acc[q].add(v);
                }
            const double sum = (acc[0].value() + acc[1].value()) + (acc[2].value() + acc[3].value());
            const double2 t = A.csx[X0 + c];
            pw += sum;
            pc += sum * t.x;
            ps += sum * t.y;
        }
        pc *= A.bunch_x;
        ps *= A.bunch_x;
    }
    if (bad) atomicOr(A.err, ERRF_NONFINITE);

    // ---- per-tile reductions in a fixed order (FP64 work only where there is weight to sum)
    // FP32: record max|s'| of the tile for the next step's window scale
    if (sizeof(T) == 4 && om > 0.f) atomicMax(&s_omax, __float_as_int(om));
    const bool reduce = __syncthreads_or(lost != 0.0 || want_part);
    if (sizeof(T) == 4 && tid == 0) A.smax_out[tile] = __int_as_float(s_omax);
    if (!reduce) return;
    // lost weight back to weight units: iq = 1 / qs exactly (a power of two; 0 for a dropped deposit)
    double vals[4] = {lost * (double)iq, pw, pc, ps};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        double v = vals[q];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) s_r4[q][warp] = v;
    }
    __syncthreads();
    if (tid == 0) {
        double t[4] = {0, 0, 0, 0};
        for (int q = 0; q < 4; ++q)
            for (int w = 0; w < nwarps; ++w) t[q] += s_r4[q][w];
        A.tile_lost[tile] += t[0];
        if (want_part) {
            A.tile_part[3 * tile + 0] = t[1];
            A.tile_part[3 * tile + 1] = t[2];
            A.tile_part[3 * tile + 2] = t[3];
        }
    }
}

// The end of a single simulation's step, in the same launch: each CTA takes a ticket once its
// tile's partial sums are visible device-wide (thread 0 wrote them, then fences); the CTA that
// draws the last ticket sees every partial and finishes the step: the FEL field update from all
// tile partials in the fixed order of fel_finalize_core (the window's shared memory, no longer
// needed, is its scratch), else the step count. It then resets the counter for the next launch.
// No CTA waits on another.
template <typename T>
__device__ __forceinline__ void finish_step(const FusedArgs<T> &A, unsigned char *smem_raw)
{
    __shared__ int s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(A.ticket, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double *state = const_cast<double *>(A.state);
    if (A.fel_partials) {
        fel_finalize_core(A.tile_part, A.ntx * A.ntp, state, A.hist, A.hist_cap, A.g.dt, 0, 0,
                          reinterpret_cast<double *>(smem_raw));
    } else if (threadIdx.x == 0) {
        const double st = state[ST_STEP] + 1.0;
        state[ST_STEP] = st;
        state[ST_TAU] = st * A.g.dt;
    }
    if (threadIdx.x == 0) *A.ticket = 0;
}

template <typename T, int BASIS, bool GAL, bool UTERM, int MINB>
__global__ void __launch_bounds__(MINB == 1 ? kFusedMaxThreads : kFusedThreads2, MINB)
    step_fused_kernel(const FusedArgs<T> A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    fused_tile<T, BASIS, GAL, UTERM>(A, blockIdx.x, smem_raw);
    if (A.ticket) finish_step<T>(A, smem_raw);
}

// Batched step: CTA b takes the (instance, tile) item b of the work list (largest tiles first;
// the hardware hands out CTAs in index order as slots free up); instance k uses
// args[2 k + parity[k]] (parity = which buffer holds its current state) and its tile is skipped
// once the instance has taken its steps (left[k] == 0). One CTA per item rather than a persistent
// loop over an atomic counter: inside a loop the compiler kept the arguments of every item live
// and spilled 400 bytes per thread; one item per CTA spills 60.
template <typename T, int BASIS, bool GAL, bool UTERM, int MINB>
__global__ void __launch_bounds__(MINB == 1 ? kFusedMaxThreads : kFusedThreads2, MINB)
    step_fused_batch_kernel(const FusedArgs<T> *__restrict__ args, const int *__restrict__ parity,
                            const int *__restrict__ left, const int2 *__restrict__ items, int nitems)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(16) FusedArgs<T> sA;
    if ((int)blockIdx.x >= nitems) return;
    const int2 e = items[blockIdx.x];
    if (left[e.x] <= 0) return;   // this simulation takes no more steps in this call
    const FusedArgs<T> *src = args + 2 * e.x + parity[e.x];
    constexpr int nwords = sizeof(FusedArgs<T>) / 4;
    for (int k = threadIdx.x; k < nwords; k += blockDim.x)
        reinterpret_cast<int *>(&sA)[k] = reinterpret_cast<const int *>(src)[k];
    __syncthreads();
    fused_tile<T, BASIS, GAL, UTERM>(sA, e.y, smem_raw);
}

template <typename T>
size_t fused_smem_bytes(int ws, int wh, int threads, int rowcache)
{
    return (size_t)ws * wh * sizeof(T) + (size_t)GRows<T>::value * threads * sizeof(T) +
           (size_t)rowcache * sizeof(RowEntry<T>);
}

int fused_rowcache_rows(int precision, size_t base_bytes, int ctas)
{
    // shared memory of an SM, reserved per CTA, and the larger static shared memory of the step
    // kernels (the batched one holds its FusedArgs there); defaults if no device answers
    int dev = 0, per_sm = 233472, reserved = 1024;
    size_t stat = 4096;
    if (cudaGetDevice(&dev) == cudaSuccess) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) == cudaSuccess) per_sm = v;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrReservedSharedMemoryPerBlock, dev) == cudaSuccess) reserved = v;
        cudaFuncAttributes fa;
        const void *k = precision == VP_FP64
                            ? reinterpret_cast<const void *>(step_fused_batch_kernel<double, VP_BASIS_CUBIC_BSPLINE, true, true, 2>)
                            : reinterpret_cast<const void *>(step_fused_batch_kernel<float, VP_BASIS_CUBIC_BSPLINE, true, true, 2>);
        if (cudaFuncGetAttributes(&fa, k) == cudaSuccess) stat = fa.sharedSizeBytes + 256;
        cudaGetLastError();
    }
    const long budget = (long)per_sm / (ctas < 1 ? 1 : ctas) - reserved - (long)stat - (long)base_bytes;
    const size_t row = precision == VP_FP64 ? sizeof(RowEntry<double>) : sizeof(RowEntry<float>);
    long rows = budget > 0 ? budget / (long)row : 0;
    if (rows > 256) rows = 256;
    return rows >= 32 ? (int)rows : 0;
}

template <typename T>
cudaError_t launch_step_fused(const FusedArgs<T> &a, int threads, cudaStream_t s)
{
    const int wh = a.tp + 2 * a.Gp;
    // the last CTA's field update uses the window memory as its scratch
    const size_t smem_tile = fused_smem_bytes<T>(a.ws, wh, threads, a.rowcache);
    const size_t smem_fin = (size_t)3 * kFinThreads * sizeof(double);
    const size_t smem = smem_tile > smem_fin ? smem_tile : smem_fin;
    const int grid = a.ntx * a.ntp;
    const bool gal = a.g.basis == VP_BASIS_CUBIC_BSPLINE && a.g.projection == VP_PROJ_GALERKIN;
    const bool uterm = a.g.kind == VP_PUSH_FEL_DKD;
#define VP_LAUNCH_FUSED(B, GL, UT)                                                            \
    do {                                                                                      \
        auto k = threads > kFusedThreads2 ? step_fused_kernel<T, B, GL, UT, 1>                 \
                                          : step_fused_kernel<T, B, GL, UT, 2>;                \
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                                             (int)smem);                                      \
        if (e != cudaSuccess) return e;                                                       \
        k<<<grid, threads, smem, s>>>(a);                                                     \
    } while (0)
    if (a.g.basis == VP_BASIS_TENT) {
        if (uterm) VP_LAUNCH_FUSED(VP_BASIS_TENT, false, true);
        else VP_LAUNCH_FUSED(VP_BASIS_TENT, false, false);
    } else if (!gal) {
        if (uterm) VP_LAUNCH_FUSED(VP_BASIS_CUBIC_BSPLINE, false, true);
        else VP_LAUNCH_FUSED(VP_BASIS_CUBIC_BSPLINE, false, false);
    } else {
        if (uterm) VP_LAUNCH_FUSED(VP_BASIS_CUBIC_BSPLINE, true, true);
        else VP_LAUNCH_FUSED(VP_BASIS_CUBIC_BSPLINE, true, false);
    }
#undef VP_LAUNCH_FUSED
    return cudaGetLastError();
}

// s = Lambda_p w along columns (tridiag(1/6, 2/3, 1/6), zero beyond the open edges). Each thread
// walks one column through a chunk of kMulRows rows, so every input row is read once (plus a halo
// row at either end of the chunk): w may be host memory the device reads in place.
constexpr int kMulRows = 64;
constexpr int kMulCols = 256;

template <typename T>
__global__ void __launch_bounds__(kMulCols)
    lambda_p_mul_kernel(const T *__restrict__ w, T *__restrict__ s, int nx, int np)
{
    const int col = blockIdx.x * kMulCols + threadIdx.x;
    if (col >= nx) return;
    const int j0 = blockIdx.y * kMulRows, j1 = min(j0 + kMulRows, np);
    T lo = j0 > 0 ? w[(size_t)(j0 - 1) * nx + col] : T(0);
    T c = w[(size_t)j0 * nx + col];
#pragma unroll 8
    for (int j = j0; j < j1; ++j) {
        const T hi = j + 1 < np ? w[(size_t)(j + 1) * nx + col] : T(0);
        s[(size_t)j * nx + col] = (lo + hi) * (T(1) / T(6)) + c * (T(2) / T(3));
        lo = c;
        c = hi;
    }
}

// max|s| per tile (one CTA per tile); a non-finite value sets the error flag
__global__ void tile_max_kernel(const float *__restrict__ s, float *__restrict__ map, int nx, int np,
                                int tx, int tp, int ntx, unsigned *err)
{
    __shared__ int s_m, s_bad;
    if (threadIdx.x == 0) {
        s_m = 0;
        s_bad = 0;
    }
    __syncthreads();
    const int X0 = (blockIdx.x % ntx) * tx, P0 = (blockIdx.x / ntx) * tp;
    const int TX = min(tx, nx - X0), TP = min(tp, np - P0);
    float m = 0.f, chk = 0.f;
    for (int k = threadIdx.x; k < TX * TP; k += blockDim.x) {
        const int r = k / TX, c = k - r * TX;
        const float v = s[(size_t)(P0 + r) * nx + X0 + c];
        m = fmaxf(m, fabsf(v));
        chk = fmaf(v, 0.f, chk);
    }
    if (m > 0.f) atomicMax(&s_m, __float_as_int(m));
    if (chk != 0.f) s_bad = 1;
    __syncthreads();
    if (threadIdx.x == 0) {
        map[blockIdx.x] = s_bad ? __int_as_float(0x7f800000) : __int_as_float(s_m);
        if (s_bad) atomicOr(err, ERRF_NONFINITE);
    }
}

cudaError_t launch_tile_max(const float *s, float *map, int nx, int np, int tx, int tp, int ntx,
                            int ntp, unsigned *err, cudaStream_t st)
{
    tile_max_kernel<<<ntx * ntp, 256, 0, st>>>(s, map, nx, np, tx, tp, ntx, err);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_lambda_p_mul(const T *w, T *s, int nx, int np, cudaStream_t st)
{
    const dim3 grid((nx + kMulCols - 1) / kMulCols, (np + kMulRows - 1) / kMulRows);
    if (grid.y > 65535u) return cudaErrorInvalidConfiguration;
    lambda_p_mul_kernel<T><<<grid, kMulCols, 0, st>>>(w, s, nx, np);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_step_fused_batch(const FusedArgs<T> *args, const int *parity, const int *left,
                                    const int2 *items, int nitems, int basis, int projection,
                                    size_t smem, int threads, int grid, cudaStream_t s)
{
    const bool gal = basis == VP_BASIS_CUBIC_BSPLINE && projection == VP_PROJ_GALERKIN;
#define VP_LAUNCH_BATCH(B, GL)                                                                \
    do {                                                                                      \
        auto k = threads > kFusedThreads2 ? step_fused_batch_kernel<T, B, GL, true, 1>         \
                                          : step_fused_batch_kernel<T, B, GL, true, 2>;        \
        if (grid <= 0) /* set-up call: shared-memory attribute only (not capturable) */       \
            return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,        \
                                        (int)smem);                                           \
        k<<<grid, threads, smem, s>>>(args, parity, left, items, nitems);                     \
    } while (0)
    if (basis == VP_BASIS_TENT) VP_LAUNCH_BATCH(VP_BASIS_TENT, false);
    else if (!gal) VP_LAUNCH_BATCH(VP_BASIS_CUBIC_BSPLINE, false);
    else VP_LAUNCH_BATCH(VP_BASIS_CUBIC_BSPLINE, true);
#undef VP_LAUNCH_BATCH
    return cudaGetLastError();
}

// CTAs of the batched step kernel that fit on one SM with this dynamic shared memory and block
// size (sets the kernel's shared-memory attribute first); 0 if the query fails
int fused_batch_blocks_per_sm(int basis, int projection, size_t smem, int threads)
{
    const bool gal = basis == VP_BASIS_CUBIC_BSPLINE && projection == VP_PROJ_GALERKIN;
    const void *k = nullptr;
    const bool one = threads > kFusedThreads2;
    if (basis == VP_BASIS_TENT)
        k = one ? (const void *)step_fused_batch_kernel<float, VP_BASIS_TENT, false, true, 1>
                : (const void *)step_fused_batch_kernel<float, VP_BASIS_TENT, false, true, 2>;
    else if (!gal)
        k = one ? (const void *)step_fused_batch_kernel<float, VP_BASIS_CUBIC_BSPLINE, false, true, 1>
                : (const void *)step_fused_batch_kernel<float, VP_BASIS_CUBIC_BSPLINE, false, true, 2>;
    else
        k = one ? (const void *)step_fused_batch_kernel<float, VP_BASIS_CUBIC_BSPLINE, true, true, 1>
                : (const void *)step_fused_batch_kernel<float, VP_BASIS_CUBIC_BSPLINE, true, true, 2>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

// ---------------------------------------------------------------------------
// Lambda_x^{-1} of whole rows, for plans with a separate x pass (Sec. III: Lambda = Lambda_x (x)
// Lambda_p, with Lambda_x the cyclic tridiag(1/6, 2/3, 1/6) of the periodic coordinate).
// Thread t of a row's CTA holds the elements t K .. t K + K - 1 in registers (K = 32 FP32, 16
// FP64; only the last chunk of a row may be shorter). The causal recurrence y_i = r_i + z y_{i-1}
// and the anticausal u_i = y_i + z u_{i+1} (z = sqrt(3) - 2) run chunk-locally from zero; a
// block-wide scan of the pairs (z^len, zero-start end value) gives each chunk its exact carry,
// and the periodic closure adds z^{i+1} y_{-1} with y_{-1} = E / (1 - z^L), E the zero-start
// value at L - 1 (anticausal: z^{L-i} u_L with u_L = S / (1 - z^L)), as the whole-period tiles
// do within a warp. Nothing is truncated. A whole chunk takes its carry and closure as one term,
// z^{k+1} (carry + z^base y_{-1}), with the powers of z as compile-time constants.
// The row sits in shared memory with element c at c + V (c / (32 V)), V the elements of 16
// bytes: the coalesced 16-byte copies and the 16-byte chunk reads of a quarter warp then hit
// distinct banks. Rows are taken from the last one down: the step kernel wrote the high rows
// last (still in L2), and the next step reads the low rows first.
template <typename T>
__device__ __forceinline__ int xrow_idx(int c)
{
    constexpr int V = 16 / (int)sizeof(T), SH = sizeof(T) == 4 ? 5 : 4;
    return c + V * (c >> SH);
}

// 16 bytes of shared memory to and from V consecutive register elements
__device__ __forceinline__ void xload16(const float *p, float *v)
{
    const float4 q = *reinterpret_cast<const float4 *>(p);
    v[0] = q.x;
    v[1] = q.y;
    v[2] = q.z;
    v[3] = q.w;
}
__device__ __forceinline__ void xload16(const double *p, double *v)
{
    const double2 q = *reinterpret_cast<const double2 *>(p);
    v[0] = q.x;
    v[1] = q.y;
}
__device__ __forceinline__ void xstore16(float *p, const float *v)
{
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void xstore16(double *p, const double *v)
{
    *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
}

template <typename T>
__device__ __forceinline__ void xscan_combine(T &A, T &b, T Ao, T bo)
{
    // (A, b) after (Ao, bo) along the recurrence: b + A bo, A Ao
    b = fma(A, bo, b);
    A *= Ao;
}

// asynchronous copies from global into shared memory (cp.async): the thread goes on while the
// copies land in the padded row layout; cp.async.wait_all waits for the thread's own copies
__device__ __forceinline__ void cp_async_16(void *dst, const void *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
template <int B>
__device__ __forceinline__ void cp_async_elem(void *dst, const void *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d), "l"(src), "n"(B) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// start copying one mesh row into a padded shared-memory row buffer (16-byte copies when every
// row starts 16-byte aligned, else one element per copy)
template <typename T>
__device__ __forceinline__ void xrow_fetch(T *buf, const T *rin, int nx, bool vec)
{
    constexpr int V = 16 / (int)sizeof(T);
    if (vec)
        for (int q = threadIdx.x; q < nx / V; q += blockDim.x)
            cp_async_16(buf + xrow_idx<T>(q * V), rin + (size_t)q * V);
    else
        for (int c = threadIdx.x; c < nx; c += blockDim.x)
            cp_async_elem<(int)sizeof(T)>(buf + xrow_idx<T>(c), rin + c);
    cp_async_commit();
}

// Block-wide exclusive scan of the chunk pairs (A, b) of one recurrence direction: returns the
// value the recurrence carries into this thread's chunk, and in total the value at the row's far
// end (zero start). DOWN: the anticausal direction (from the last chunk down). One barrier: every
// warp combines the per-warp totals itself; each direction has its own sA, sB.
template <typename T, bool DOWN>
__device__ __forceinline__ T xrow_carry(T A, T b, T *sA, T *sB, T &total)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const T Ao = DOWN ? __shfl_down_sync(0xffffffffu, A, off) : __shfl_up_sync(0xffffffffu, A, off);
        const T bo = DOWN ? __shfl_down_sync(0xffffffffu, b, off) : __shfl_up_sync(0xffffffffu, b, off);
        if (DOWN ? lane + off < 32 : lane >= off) xscan_combine(A, b, Ao, bo);
    }
    if (lane == (DOWN ? 0 : 31)) {
        sA[warp] = A;
        sB[warp] = b;
    }
    T Ae = DOWN ? __shfl_down_sync(0xffffffffu, A, 1) : __shfl_up_sync(0xffffffffu, A, 1);
    T be = DOWN ? __shfl_down_sync(0xffffffffu, b, 1) : __shfl_up_sync(0xffffffffu, b, 1);
    if (lane == (DOWN ? 31 : 0)) {
        Ae = T(1);
        be = T(0);
    }
    __syncthreads();
    T c = T(0), cw = T(0);
    for (int k = 0; k < nwarps; ++k) {
        const int w = DOWN ? nwarps - 1 - k : k;
        if (w == warp) cw = c;
        c = fma(sA[w], c, sB[w]);
    }
    total = c;
    return fma(Ae, cw, be);
}

// Lambda_x^{-1} (times -1/(6z)) of one row whose elements base .. base + len - 1 this thread
// holds in v (len == K: a whole chunk), the threads of the block holding the row in order.
// sA, sB: [2][warps], one pair of arrays per direction (a row's causal scan and the next row's
// are separated by the anticausal scan's barrier and the row's store barrier).
template <typename T, int K>
__device__ __forceinline__ void xsolve_row_regs(T *v, const int base, const int len, const int nx,
                                                T (*sA)[kXRowMaxThreads / 32], T (*sB)[kXRowMaxThreads / 32])
{
    const T z = (T)zconst(1);
    const bool whole = len == K;
    // causal sweep from zero, then the carry and the periodic closure
    T y = T(0), A = T(1);
    if (whole) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            y = fma(z, y, v[k]);
            v[k] = y;
        }
        A = (T)zconst(K);
    } else {
#pragma unroll
        for (int k = 0; k < K; ++k)
            if (k < len) {
                y = fma(z, y, v[k]);
                v[k] = y;
                A *= z;
            }
    }
    {
        T E;
        const T carry = xrow_carry<T, false>(A, y, sA[0], sB[0], E);
        const T yprev = E / (T(1) - zpow<T>(nx));   // y_{-1} = y_{L-1}
        const T cin = fma(zpow<T>(base), yprev, carry);     // element base + k: z^{k+1} cin
        if (whole) {
#pragma unroll
            for (int k = 0; k < K; ++k) v[k] = fma((T)zconst(k + 1), cin, v[k]);
        } else {
            T zk = z;
#pragma unroll
            for (int k = 0; k < K; ++k)
                if (k < len) {
                    v[k] = fma(zk, cin, v[k]);
                    zk *= z;
                }
        }
    }
    // anticausal sweep from zero at the chunk end, then the carry and the periodic closure
    T u = T(0);
    A = T(1);
    if (whole) {
#pragma unroll
        for (int k = K - 1; k >= 0; --k) {
            u = fma(z, u, v[k]);
            v[k] = u;
        }
        A = (T)zconst(K);
    } else {
#pragma unroll
        for (int k = K - 1; k >= 0; --k)
            if (k < len) {
                u = fma(z, u, v[k]);
                v[k] = u;
                A *= z;
            }
    }
    {
        T S;
        const T carry = xrow_carry<T, true>(A, u, sA[1], sB[1], S);
        const T unext = S / (T(1) - zpow<T>(nx));   // u_L = u_0
        // element base + k: z^{len - k} (carry + z^{L - base - len} u_L)
        const T cin = len > 0 ? fma(zpow<T>(nx - base - len), unext, carry) : T(0);
        if (whole) {
#pragma unroll
            for (int k = 0; k < K; ++k) v[k] = fma((T)zconst(K - k), cin, v[k]);
        } else {
            T zk = z;
#pragma unroll
            for (int k = K - 1; k >= 0; --k)
                if (k < len) {
                    v[k] = fma(zk, cin, v[k]);
                    zk *= z;
                }
        }
    }
}

// Persistent: each CTA takes rows np - 1 - blockIdx.x, then gridDim.x further down, and copies
// the next row into its second buffer while it solves the current one.
template <typename T, int K, int MAXT>
__global__ void __launch_bounds__(MAXT, MAXT == 256 ? 3 : 1)
    xsolve_rows_kernel(const T *__restrict__ r, T *__restrict__ out, int nx, int np,
                       const double *__restrict__ piv, int tx, int tp, int ntx,
                       float *__restrict__ smax_out, unsigned *__restrict__ err, int row_stride, int nbuf)
{
    extern __shared__ __align__(16) unsigned char xs_raw[];
    T *buf0 = reinterpret_cast<T *>(xs_raw);
    int *tmax = reinterpret_cast<int *>(buf0 + (size_t)nbuf * row_stride);
    __shared__ T sA[2][kXRowMaxThreads / 32], sB[2][kXRowMaxThreads / 32];
    constexpr int V = 16 / (int)sizeof(T);
    const int tid = threadIdx.x;
    const bool vec = (nx % V) == 0;   // every row starts 16-byte aligned
    const T sh = sizeof(T) == 4 ? (T)piv[kPivXsFused] : T(-6) * (T)zconst(1);
    const T sl = sizeof(T) == 4 ? (T)piv[kPivXsFused + 1] : T(0);
    const int base = tid * K;
    const int len = max(0, min(K, nx - base));
    // a chunk lies in one tile when the tile width is a multiple of the chunk
    const bool one_tile = tx % K == 0;

    // zeros past the row end in every buffer (read with the last chunks, never stored)
    for (int b = 0; b < nbuf; ++b)
        for (int c = nx + tid; c < (int)blockDim.x * K; c += blockDim.x)
            buf0[(size_t)b * row_stride + xrow_idx<T>(c)] = T(0);
    if (sizeof(T) == 4)
        for (int k = tid; k < ntx; k += blockDim.x) tmax[k] = 0;
    int i = blockIdx.x;
    if (i < np) xrow_fetch(buf0, r + (size_t)(np - 1 - i) * nx, nx, vec);
    bool bad = false;
    for (int it = 0; i < np; i += gridDim.x, ++it) {
        const int row = np - 1 - i;
        T *cur = buf0 + (size_t)(nbuf == 2 ? (it & 1) : 0) * row_stride;
        cp_async_wait_all();
        __syncthreads();   // the row is in cur; the stores of the other buffer's row have read it
        const int inext = i + gridDim.x;
        if (nbuf == 2 && inext < np)
            xrow_fetch(buf0 + (size_t)((it + 1) & 1) * row_stride, r + (size_t)(np - 1 - inext) * nx, nx, vec);

        T v[K];
#pragma unroll
        for (int j = 0; j < K / V; ++j) xload16(cur + xrow_idx<T>(base + j * V), &v[j * V]);
        xsolve_row_regs<T, K>(v, base, len, nx, sA, sB);

        // the scale -6z (FP32: the step's unit-DC-gain pair sh + sl), checks, per-tile max|s'|
        T chk = T(0);
        float m = 0.f;
        if (len == K) {
#pragma unroll
            for (int k = 0; k < K; ++k) {
                v[k] = sizeof(T) == 4 ? fma(v[k], sl, v[k] * sh) : v[k] * sh;
                chk = fma(v[k], T(0), chk);
                m = fmaxf(m, fabsf((float)v[k]));
            }
        } else {
#pragma unroll
            for (int k = 0; k < K; ++k)
                if (k < len) {
                    v[k] = sizeof(T) == 4 ? fma(v[k], sl, v[k] * sh) : v[k] * sh;
                    chk = fma(v[k], T(0), chk);
                    m = fmaxf(m, fabsf((float)v[k]));
                }
        }
        bad |= chk != T(0);
        if (sizeof(T) == 4 && len > 0) {
            if (one_tile) {
                if (m > 0.f) atomicMax(&tmax[base / tx], __float_as_int(m));
            } else {
                int tc = base / tx, nb = (tc + 1) * tx;
                m = 0.f;
#pragma unroll
                for (int k = 0; k < K; ++k)
                    if (k < len) {
                        if (base + k >= nb) {
                            if (m > 0.f) atomicMax(&tmax[tc], __float_as_int(m));
                            m = 0.f;
                            ++tc;
                            nb += tx;
                        }
                        m = fmaxf(m, fabsf((float)v[k]));
                    }
                if (m > 0.f) atomicMax(&tmax[tc], __float_as_int(m));
            }
        }
#pragma unroll
        for (int j = 0; j < K / V; ++j) xstore16(cur + xrow_idx<T>(base + j * V), &v[j * V]);
        __syncthreads();

        T *rout = out + (size_t)row * nx;
        if (vec) {
            int4 *o4 = reinterpret_cast<int4 *>(rout);
            for (int q = tid; q < nx / V; q += blockDim.x)
                o4[q] = *reinterpret_cast<const int4 *>(cur + xrow_idx<T>(q * V));
        } else {
            for (int c = tid; c < nx; c += blockDim.x) rout[c] = cur[xrow_idx<T>(c)];
        }
        if (sizeof(T) == 4) {
            int *mo = reinterpret_cast<int *>(smax_out) + (size_t)(row / tp) * ntx;
            for (int k = tid; k < ntx; k += blockDim.x) {
                const int mk = tmax[k];
                if (mk != 0) {
                    atomicMax(mo + k, mk);
                    tmax[k] = 0;
                }
            }
        }
        if (nbuf == 1 && inext < np) {
            __syncthreads();
            xrow_fetch(cur, r + (size_t)(np - 1 - inext) * nx, nx, vec);
        }
    }
    if (__syncthreads_or(bad) && tid == 0) atomicOr(err, ERRF_NONFINITE);
}

void xrow_shape(int precision, int nx, int *threads, int *per)
{
    const int K = xrow_max_per(precision);
    *threads = 0;
    *per = 0;
    if (nx < 1 || (long)nx > (long)kXRowMaxThreads * K) return;
    *threads = ((nx + K - 1) / K + 31) / 32 * 32;
    *per = K;
}

// bytes of one padded row buffer (a multiple of 16): every chunk of every thread, with the pads
static size_t xrow_row_bytes(int precision, int nx)
{
    int t = 0, p = 0;
    xrow_shape(precision, nx, &t, &p);
    if (t == 0) return 0;
    const int V = precision == VP_FP64 ? 2 : 4, line = precision == VP_FP64 ? 16 : 32;
    const size_t sz = precision == VP_FP64 ? 8 : 4;
    const size_t n = (size_t)t * p;
    return ((n + V * (n / line) + V) * sz + 15) & ~(size_t)15;
}

// two row buffers (the next row is copied in while the current one is solved) when they fit
int xrow_buffers(int precision, int nx, int ntx)
{
    const size_t tm = precision == VP_FP64 ? 0 : (size_t)ntx * sizeof(int);
    return 2 * xrow_row_bytes(precision, nx) + tm <= (size_t)200 * 1024 ? 2 : 1;
}

size_t xrow_smem_bytes(int precision, int nx, int ntx)
{
    const size_t row = xrow_row_bytes(precision, nx);
    if (row == 0) return 0;
    return (size_t)xrow_buffers(precision, nx, ntx) * row +
           (precision == VP_FP64 ? 0 : (size_t)ntx * sizeof(int));
}

// block-size bound of the instantiation: rows up to 256 chunks (FP32 8192 nodes) keep their
// chunks in registers at two CTAs per SM; the larger forms serve longer rows
template <typename T>
static auto xrow_kernel(int threads)
{
    constexpr int K = sizeof(T) == 8 ? 16 : 32;
    return threads <= 256 ? xsolve_rows_kernel<T, K, 256>
                          : (threads <= 512 ? xsolve_rows_kernel<T, K, 512> : xsolve_rows_kernel<T, K, 1024>);
}

template <typename T>
static int xrow_grid_of(int nx, int np, int ntx)
{
    const int prec = sizeof(T) == 8 ? VP_FP64 : VP_FP32;
    int threads = 0, per = 0;
    xrow_shape(prec, nx, &threads, &per);
    if (threads == 0) return 0;
    const size_t smem = xrow_smem_bytes(prec, nx, ntx);
    auto k = xrow_kernel<T>(threads);
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return np;   // one CTA per row
    }
    const long g = (long)sms * (per_sm > 0 ? per_sm : 1);
    return (int)(g < np ? g : np);
}

int xrow_grid_size(int precision, int nx, int np, int ntx)
{
    return precision == VP_FP64 ? xrow_grid_of<double>(nx, np, ntx) : xrow_grid_of<float>(nx, np, ntx);
}

template <typename T>
cudaError_t launch_xsolve_rows(const T *r, T *out, int nx, int np, const double *piv, int tx, int tp,
                               int ntx, float *smax_out, unsigned *err, int grid, cudaStream_t s)
{
    const int prec = sizeof(T) == 8 ? VP_FP64 : VP_FP32;
    int threads = 0, per = 0;
    xrow_shape(prec, nx, &threads, &per);
    if (threads == 0) return cudaErrorInvalidValue;
    const size_t smem = xrow_smem_bytes(prec, nx, ntx);
    const int nbuf = xrow_buffers(prec, nx, ntx);
    const int stride = (int)(xrow_row_bytes(prec, nx) / sizeof(T));
    auto k = xrow_kernel<T>(threads);
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    if (grid <= 0 || grid > np) grid = np;
    k<<<grid, threads, smem, s>>>(r, out, nx, np, piv, tx, tp, ntx, smax_out, err, stride, nbuf);
    return cudaGetLastError();
}

template cudaError_t launch_xsolve_rows<float>(const float *, float *, int, int, const double *, int, int,
                                               int, float *, unsigned *, int, cudaStream_t);
template cudaError_t launch_xsolve_rows<double>(const double *, double *, int, int, const double *, int,
                                                int, int, float *, unsigned *, int, cudaStream_t);

template cudaError_t launch_step_fused_batch<float>(const FusedArgs<float> *, const int *, const int *,
                                                    const int2 *, int, int, int, size_t, int, int,
                                                    cudaStream_t);
template cudaError_t launch_step_fused_batch<double>(const FusedArgs<double> *, const int *, const int *,
                                                     const int2 *, int, int, int, size_t, int, int,
                                                     cudaStream_t);
template size_t fused_smem_bytes<float>(int, int, int, int);
template size_t fused_smem_bytes<double>(int, int, int, int);
template cudaError_t launch_step_fused<float>(const FusedArgs<float> &, int, cudaStream_t);
template cudaError_t launch_step_fused<double>(const FusedArgs<double> &, int, cudaStream_t);
template cudaError_t launch_lambda_p_mul<float>(const float *, float *, int, int, cudaStream_t);
template cudaError_t launch_lambda_p_mul<double>(const double *, double *, int, int, cudaStream_t);

}  // namespace vp
