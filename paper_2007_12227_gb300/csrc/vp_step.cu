// vp_step.cu -- push + deposit (Delta^T w) kernels.
//
// Sec. III: r_j' = sum_k Delta_{k j'} w_k, with Delta the overlap of the basis
// function of node k shifted by its one-step displacement (Sec. II flow) with
// the unshifted basis function of node j'. For a tensor-product basis of a
// symmetric 1-D function L the overlap is (L*L)(offset) per axis, so r is a
// deposit of every pushed node with the kernel K = L*L:
//   top-hat basis (VP_BASIS_TENT)          K = tent,     2 x 2 taps
//   tent basis    (VP_BASIS_CUBIC_BSPLINE) K = cubic B3, 4 x 4 taps
// (the common factor hx hp of Delta and Lambda cancels and is omitted).
// Along x columns wrap (periodic); rows outside [0, np) are lost (open
// momentum boundary, Sec. IV) and added to a per-tile lost-weight counter.
//
// step_tiled_kernel: one CTA owns one destination tile [X0, X0+TX) x [P0, P0+TP)
// held in shared memory. It bounds, row by row, the source nodes whose pushed
// basis function can overlap the tile, pushes them, accumulates their taps
// into the tile with shared-memory atomics, and stores the tile once with
// coalesced writes. No destination element is written by more than one CTA.
//
// step_scatter_kernel: one thread per source node, taps added to a zeroed
// destination with global atomics (the simple reference form).
#include <math.h>

#include "vp_internal.h"
#include "vp_sum.cuh"

namespace vp {
namespace {

constexpr int kThreads = 256;
constexpr int kMaxRows = 256;   // candidate source rows examined per batch

// deposit weights of the kernel for fractional offset t in [0, 1)
template <typename T, int BASIS>
struct Taps;

template <typename T>
struct Taps<T, VP_BASIS_TENT> {
    static constexpr int N = 2;
    static constexpr int LO = 0;   // first tap at base + LO
    __device__ __forceinline__ static void weights(T t, T *w)
    {
        w[0] = T(1) - t;
        w[1] = t;
    }
};

template <typename T>
struct Taps<T, VP_BASIS_SEPTIC_BSPLINE> {
    static constexpr int N = 8;
    static constexpr int LO = -3;
    __device__ __forceinline__ static void weights(T t, T *w) { septic_weights<T>(t, w); }
};

// FP32 weights rounded to the grid 2^-23 ((x + 1) - 1); FP64 weights as they are
__device__ __forceinline__ float grid23(float x) { return __fadd_rn(__fadd_rn(x, 1.f), -1.f); }
__device__ __forceinline__ double grid23(double x) { return x; }

template <typename T>
struct Taps<T, VP_BASIS_CUBIC_BSPLINE> {
    static constexpr int N = 4;
    static constexpr int LO = -1;
    __device__ __forceinline__ static void weights(T t, T *w)
    {
        // cubic B-spline at offsets 1+t, t, 1-t, 2-t
        const T s = T(1) - t;
        const T t2 = t * t, t3 = t2 * t;
        const T sixth = T(1) / T(6);
        w[0] = grid23(s * s * s * sixth);
        w[3] = grid23(t3 * sixth);
        w[1] = grid23(T(2) / T(3) - t2 + T(0.5) * t3);
        // partition of unity: in FP32 the three weights above lie on the grid 2^-23, so this
        // difference is exact and the four sum to exactly one
        w[2] = ((T(1) - w[0]) - w[3]) - w[1];
    }
};

// displacement of node (column entry c, row entry r): integer + fraction per axis
template <typename T>
__device__ __forceinline__ void displace(const ColEntry<T> &c, const RowEntry<T> &r, T al, T be,
                                         T KU, T KV, int &di, T &fu, int &dj, T &fv)
{
    const T gs = c.sa * r.cy + c.ca * r.sy;   // sin(a_i + y_j)
    const T gc = c.ca * r.cy - c.sa * r.sy;   // cos(a_i + y_j)
    const T e = al * gs + be * gc;
    di = c.ui + r.ui;
    dj = c.vi + r.vi;
    fu = (c.uf + r.uf) + KU * e;
    fv = (c.vf + r.vf) + KV * e;
}

__device__ __forceinline__ int mod_i(long a, int n)
{
    long r = a % n;
    return (int)(r < 0 ? r + n : r);
}

// range of sin over [lo, hi]
__device__ void sin_range(double lo, double hi, double &smin, double &smax)
{
    const double twopi = 6.283185307179586476925286766559;
    if (hi - lo >= twopi) {
        smin = -1.0;
        smax = 1.0;
        return;
    }
    const double a = sin(lo), b = sin(hi);
    smin = fmin(a, b);
    smax = fmax(a, b);
    const double hpi = 1.5707963267948966192313216916398;
    const double kmax = ceil((lo - hpi) / twopi);
    if (hpi + kmax * twopi <= hi) smax = 1.0;
    const double kmin = ceil((lo + hpi) / twopi);
    if (-hpi + kmin * twopi <= hi) smin = -1.0;
}

template <typename T, int BASIS>
__global__ void __launch_bounds__(kThreads) step_tiled_kernel(const StepArgs<T> A)
{
    using TP_ = Taps<T, BASIS>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int TX = A.tx, TPh = A.tp;
    T *win = reinterpret_cast<T *>(smem_raw);
    int *rl = reinterpret_cast<int *>(win + (size_t)TX * TPh);
    __shared__ int s_nkept, s_maxw;
    __shared__ double s_red[4][kThreads / 32];

    const Geometry &g = A.g;
    const int nx = g.nx, np = g.np;
    const int tile = blockIdx.x;
    const int tix = tile % A.ntx, tip = tile / A.ntx;
    const int X0 = tix * TX, P0 = tip * TPh;
    const int TXe = min(TX, nx - X0), TPe = min(TPh, np - P0);
    const int R = (BASIS == VP_BASIS_TENT) ? 1 : 2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;

    for (int k = threadIdx.x; k < TX * TPh; k += blockDim.x) win[k] = T(0);

    double al = g.alpha0, be = g.beta0, M = g.m0, phi = g.phi0;
    if (g.kind == VP_PUSH_FEL_DKD) {
        al = -A.state[ST_K_IM];
        be = A.state[ST_K_RE];
        M = A.state[ST_M];
        phi = A.state[ST_PHI];
    }
    const double EU = fabs(g.KU) * M, EV = fabs(g.KV) * M;
    const T alT = (T)al, beT = (T)be, KUT = (T)g.KU, KVT = (T)g.KV;
    const double SL = 0.02;   // slack (cells) covering rounding of the FP32 push
    const double vd_min = g.vc_min + g.vr_min - EV, vd_max = g.vc_max + g.vr_max + EV;
    const bool edge_lo = (P0 == 0), edge_hi = (P0 + TPe == np);
    // edge tiles also visit every source row that can leave the grid on their side
    const int jlo = edge_lo ? 0 : max(0, (int)floor(P0 - R - vd_max - SL));
    const int jhi = edge_hi ? np - 1 : min(np - 1, (int)ceil(P0 + TPe - 1 + R - vd_min + SL));
    const double acc_lo = edge_lo ? -1e300 : (double)(P0 - R);
    const double acc_hi = edge_hi ? 1e300 : (double)(P0 + TPe - 1 + R);

    double lost = 0.0;
    __syncthreads();

    for (int jb = jlo; jb <= jhi; jb += kMaxRows) {
        const int jend = min(jb + kMaxRows - 1, jhi);
        if (threadIdx.x == 0) {
            s_nkept = 0;
            s_maxw = 0;
        }
        __syncthreads();
        // ---- which source rows can reach the tile, and over which columns
        for (int j = jb + threadIdx.x; j <= jend; j += blockDim.x) {
            const RowBound rb = A.rowb[j];
            long ia = (long)floor(X0 - R - rb.u - EU - g.uc_max - SL);
            long ib = (long)ceil(X0 + TXe - 1 + R - rb.u + EU - g.uc_min + SL);
            if (ib - ia + 1 > nx) ib = ia + nx - 1;   // each source node at most once
            double vcl = g.vc_min, vch = g.vc_max;
            const long width = ib - ia + 1;
            if (width < nx - 2 * kColBlock) {
                vcl = 1e300;
                vch = -1e300;
                const int start = mod_i(ia, nx);
                int seg_lo[2], seg_hi[2], nseg = 1;
                if (start + width <= nx) {
                    seg_lo[0] = start;
                    seg_hi[0] = (int)(start + width - 1);
                } else {
                    seg_lo[0] = start;
                    seg_hi[0] = nx - 1;
                    seg_lo[1] = 0;
                    seg_hi[1] = (int)(start + width - 1 - nx);
                    nseg = 2;
                }
                for (int sgi = 0; sgi < nseg; ++sgi)
                    for (int b = seg_lo[sgi] / kColBlock; b <= seg_hi[sgi] / kColBlock; ++b) {
                        vcl = fmin(vcl, A.vcb[2 * b]);
                        vch = fmax(vch, A.vcb[2 * b + 1]);
                    }
            }
            double tlo = 0.0, thi = 0.0;
            if (EV > 0.0) {
                double smin, smax;
                const double plo = g.x0 + ia * g.hx - g.a_pad + rb.y + phi;
                const double phi_ = g.x0 + ib * g.hx + g.a_pad + rb.y + phi;
                sin_range(plo, phi_, smin, smax);
                const double k = g.KV * M;
                tlo = fmin(k * smin, k * smax);
                thi = fmax(k * smin, k * smax);
            }
            const double vlo = j + rb.v + vcl + tlo - SL;
            const double vhi = j + rb.v + vch + thi + SL;
            if (vhi > acc_lo && vlo < acc_hi) {
                const int k = atomicAdd(&s_nkept, 1);
                rl[4 * k] = j;
                rl[4 * k + 1] = mod_i(ia, nx);       // wrapped first source column
                rl[4 * k + 2] = (int)width;
                rl[4 * k + 3] = (int)(ia - X0);      // unwrapped first column relative to the tile
                atomicMax(&s_maxw, (int)width);
            }
        }
        __syncthreads();
        const int nk = s_nkept;
        const int nch = (s_maxw + 31) >> 5;
        const int nitems = nk * nch;
        // ---- push + deposit
        for (int it = warp; it < nitems; it += nwarps) {
            const int k = it / nch, ch = it - k * nch;
            const int j = rl[4 * k], iam = rl[4 * k + 1], wdt = rl[4 * k + 2], rel = rl[4 * k + 3];
            const int off = ch * 32 + lane;
            if (off >= wdt) continue;
            int im = iam + off;                       // wrapped source column (off < nx)
            if (im >= nx) im -= nx;
            const T w = A.src[(size_t)j * nx + im];
            if (w == T(0)) continue;
            const ColEntry<T> c = A.col[im];
            const RowEntry<T> r = A.row[j];
            int di, dj;
            T fu, fv;
            displace(c, r, alT, beT, KUT, KVT, di, fu, dj, fv);
            const T flu = floor(fu), flv = floor(fv);
            T wx[TP_::N], wy[TP_::N];
            TP_::weights(fu - flu, wx);
            TP_::weights(fv - flv, wy);
            // first destination column relative to X0 (unwrapped) and first row
            const int mu = rel + off + di + (int)flu + TP_::LO;
            const int nv = j + dj + (int)flv + TP_::LO;
            int dc[TP_::N];
            bool okc[TP_::N];
#pragma unroll
            for (int a = 0; a < TP_::N; ++a) {
                int ci = mu + a;
                if (ci < 0) ci += nx;
                if (ci >= nx) ci -= nx;
                if (ci < 0 || ci >= nx) ci = mod_i(ci, nx);   // far wrap (tiny grids only)
                dc[a] = ci;
                okc[a] = ci < TXe;
            }
#pragma unroll
            for (int b = 0; b < TP_::N; ++b) {
                const int rr = nv + b;
                const T wb = w * wy[b];
                if (rr < 0 || rr >= np) {
                    if ((rr < 0 && edge_lo) || (rr >= np && edge_hi)) {
#pragma unroll
                        for (int a = 0; a < TP_::N; ++a)
                            if (okc[a]) lost += (double)(wb * wx[a]);
                    }
                    continue;
                }
                const int dr = rr - P0;
                if (dr < 0 || dr >= TPe) continue;
                T *rowp = win + (size_t)dr * TX;
#pragma unroll
                for (int a = 0; a < TP_::N; ++a)
                    if (okc[a]) atomicAdd(rowp + dc[a], wb * wx[a]);
            }
        }
        __syncthreads();
    }

    // ---- store the tile once; FEL partial sums; finiteness
    double pc = 0.0, ps = 0.0, pw = 0.0;
    bool bad = false;
    const size_t base = (size_t)P0 * nx + X0;
    if (A.fel_partials) {
        // column-major walk so that each thread keeps one column's cos/sin
        for (int cidx = threadIdx.x; cidx < TXe; cidx += blockDim.x) {
            DSum<T> acc;
            for (int rr = 0; rr < TPe; ++rr) acc.add(win[(size_t)rr * TX + cidx]);
            const double colsum = acc.value();
            const double2 t = A.csx[X0 + cidx];
            pw += colsum;
            pc += colsum * t.x;
            ps += colsum * t.y;
        }
    }
    for (int k = threadIdx.x; k < TXe * TPe; k += blockDim.x) {
        const int rr = k / TXe, cidx = k - rr * TXe;
        const T v = win[(size_t)rr * TX + cidx];
        bad |= !isfinite(v);
        A.dst[base + (size_t)rr * nx + cidx] = v;
    }
    if (bad) atomicOr(A.err, ERRF_NONFINITE);

    // block reductions (fixed order: warp shuffle, then warps in order)
    double vals[4] = {lost, pw, pc, ps};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        double v = vals[q];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) s_red[q][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t[4] = {0, 0, 0, 0};
        for (int q = 0; q < 4; ++q)
            for (int w = 0; w < nwarps; ++w) t[q] += s_red[q][w];
        A.tile_lost[tile] += t[0];
        if (A.fel_partials) {
            A.tile_part[3 * tile + 0] = t[1];
            A.tile_part[3 * tile + 1] = t[2];
            A.tile_part[3 * tile + 2] = t[3];
        }
    }
}

template <typename T, int BASIS>
__global__ void __launch_bounds__(kThreads) step_scatter_kernel(const StepArgs<T> A, double *lost_acc)
{
    using TP_ = Taps<T, BASIS>;
    __shared__ double s_red[kThreads / 32];
    const Geometry &g = A.g;
    const int nx = g.nx, np = g.np;
    double al = g.alpha0, be = g.beta0;
    if (g.kind == VP_PUSH_FEL_DKD) {
        al = -A.state[ST_K_IM];
        be = A.state[ST_K_RE];
    }
    const T alT = (T)al, beT = (T)be, KUT = (T)g.KU, KVT = (T)g.KV;
    double lost = 0.0;
    const size_t n = (size_t)nx * np;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(idx / nx), i = (int)(idx - (size_t)j * nx);
        const T w = A.src[idx];
        if (w == T(0)) continue;
        int di, dj;
        T fu, fv;
        displace(A.col[i], A.row[j], alT, beT, KUT, KVT, di, fu, dj, fv);
        const T flu = floor(fu), flv = floor(fv);
        T wx[TP_::N], wy[TP_::N];
        TP_::weights(fu - flu, wx);
        TP_::weights(fv - flv, wy);
        const long mu = (long)i + di + (long)flu + TP_::LO;
        const int nv = j + dj + (int)flv + TP_::LO;
#pragma unroll
        for (int b = 0; b < TP_::N; ++b) {
            const int rr = nv + b;
            const T wb = w * wy[b];
            if (rr < 0 || rr >= np) {
#pragma unroll
                for (int a = 0; a < TP_::N; ++a) lost += (double)(wb * wx[a]);
                continue;
            }
#pragma unroll
            for (int a = 0; a < TP_::N; ++a) {
                int ci = (int)(mu + a);
                if (ci < 0) ci += nx;
                if (ci >= nx) ci -= nx;
                if (ci < 0 || ci >= nx) ci = mod_i(ci, nx);
                atomicAdd(A.dst + (size_t)rr * nx + ci, wb * wx[a]);
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) lost += __shfl_down_sync(0xffffffffu, lost, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = lost;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_red[w];
        if (t != 0.0) atomicAdd(lost_acc, t);
    }
}

}  // namespace

template <typename T>
size_t tiled_smem_bytes(int tx, int tp)
{
    return (size_t)tx * tp * sizeof(T) + 4 * sizeof(int) * kMaxRows;
}

template <typename T>
cudaError_t launch_step_tiled(const StepArgs<T> &a, cudaStream_t s)
{
    const size_t smem = tiled_smem_bytes<T>(a.tx, a.tp);
    const int grid = a.ntx * a.ntp;
    if (a.g.basis == VP_BASIS_TENT) {
        auto k = step_tiled_kernel<T, VP_BASIS_TENT>;
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k<<<grid, kThreads, smem, s>>>(a);
    } else {
        auto k = step_tiled_kernel<T, VP_BASIS_CUBIC_BSPLINE>;
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k<<<grid, kThreads, smem, s>>>(a);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_step_scatter(const StepArgs<T> &a, double *lost_acc, cudaStream_t s)
{
    const size_t n = (size_t)a.g.nx * a.g.np;
    int grid = (int)((n + kThreads - 1) / kThreads);
    if (grid > 152 * 64) grid = 152 * 64;
    if (a.g.basis == VP_BASIS_TENT)
        step_scatter_kernel<T, VP_BASIS_TENT><<<grid, kThreads, 0, s>>>(a, lost_acc);
    else if (a.g.basis == VP_BASIS_SEPTIC_BSPLINE)
        step_scatter_kernel<T, VP_BASIS_SEPTIC_BSPLINE><<<grid, kThreads, 0, s>>>(a, lost_acc);
    else
        step_scatter_kernel<T, VP_BASIS_CUBIC_BSPLINE><<<grid, kThreads, 0, s>>>(a, lost_acc);
    return cudaGetLastError();
}

template size_t tiled_smem_bytes<float>(int, int);
template size_t tiled_smem_bytes<double>(int, int);
template cudaError_t launch_step_tiled<float>(const StepArgs<float> &, cudaStream_t);
template cudaError_t launch_step_tiled<double>(const StepArgs<double> &, cudaStream_t);
template cudaError_t launch_step_scatter<float>(const StepArgs<float> &, double *, cudaStream_t);
template cudaError_t launch_step_scatter<double>(const StepArgs<double> &, double *, cudaStream_t);

}  // namespace vp
