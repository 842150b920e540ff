// vp_rk4.cu -- the FEL step with the classical fourth-order Runge-Kutta integrator (Sec. IV.B:
// the paper integrates its FEL equations with RK4).
//
// Every mesh node is a particle of d theta/dz = delta + eta, d eta/dz = -(K e^{i theta} + c.c.)
// with K = A + i sigma2 <e^{-i theta}>; A moves by dA/dz = <e^{-i theta}>. The four stages
// need the bunching b_s of all particles at their stage-s phases, and those phases depend on
// the amplitudes K_1 .. K_{s-1} of the earlier stages, so one step is
//   for s = 1..4: a reduction of the stage-s bunching (rk4_stage_kernel), then
//                 A_s = A + c_s b_{s-1}, K_s = A_s + i sigma2 b_s (rk4_amp_kernel);
//   the deposit of every node at its RK4 end point (rk4_deposit_kernel, global atomics);
//   A' = A + h/6 (b_1 + 2 b_2 + 2 b_3 + b_4), kept in the state for the field update.
// The push is evaluated in FP64 as increments from the node (d theta, d eta), whatever the
// precision of the weights, so the FP32 path keeps sub-cell positions. This path is the
// paper's integrator for validation; the one-pass drift-kick-drift kernel is the fast path.
#include <math.h>

#include "vp_internal.h"

namespace vp {
namespace {

constexpr int kThreads = 256;
constexpr int kRows = 256;   // rows per block of the stage reductions

// stage phases of the particle at (theta = (c0, s0), eta = p): e[s] = e^{i theta_s} for
// s < upto, and the RK4 increments of theta and eta when upto == 4
__device__ __forceinline__ void rk4_particle(double c0, double s0, double p, const double *K, double h,
                                             double delta, int upto, double2 *e, double &dth, double &dp)
{
    double pp[4], dps[4];
    e[0] = make_double2(c0, s0);
    pp[0] = p;
    dps[0] = -2.0 * (K[0] * c0 - K[1] * s0);
    for (int s = 1; s < upto; ++s) {
        const double c = (s == 3) ? h : 0.5 * h;
        double sn, cs;
        sincos(c * (delta + pp[s - 1]), &sn, &cs);
        e[s] = make_double2(c0 * cs - s0 * sn, s0 * cs + c0 * sn);
        pp[s] = p + c * dps[s - 1];
        dps[s] = -2.0 * (K[2 * s] * e[s].x - K[2 * s + 1] * e[s].y);
    }
    if (upto == 4) {
        dth = h / 6.0 * ((delta + pp[0]) + 2.0 * (delta + pp[1]) + 2.0 * (delta + pp[2]) + (delta + pp[3]));
        dp = h / 6.0 * (dps[0] + 2.0 * dps[1] + 2.0 * dps[2] + dps[3]);
    }
}

// per block (32 columns x kRows rows): sum w, sum w cos theta_s, sum w sin theta_s (FP64)
template <typename T>
__global__ void __launch_bounds__(kThreads)
    rk4_stage_kernel(const T *__restrict__ w, Geometry g, const double2 *__restrict__ csx,
                     const double *__restrict__ state, int stage, double *part)
{
    __shared__ double s_red[3][kThreads / 32];
    const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
    const int col = blockIdx.x * 32 + lane;
    const int r0 = blockIdx.y * kRows, r1 = min(r0 + kRows, g.np);
    double K[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) K[q] = state[ST_RK_K + q];
    double a[3] = {0.0, 0.0, 0.0};
    if (col < g.nx) {
        const double2 t = csx[col];
        for (int r = r0 + wy; r < r1; r += kThreads / 32) {
            const double v = (double)w[(size_t)r * g.nx + col];
            if (v == 0.0) continue;
            double2 e[4];
            double dth, dp;
            rk4_particle(t.x, t.y, g.p0 + r * g.hp, K, g.dt, g.delta, stage + 1, e, dth, dp);
            a[0] += v;
            a[1] += v * e[stage].x;
            a[2] += v * e[stage].y;
        }
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        double v = a[q];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) s_red[q][wy] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const size_t b = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
        for (int q = 0; q < 3; ++q) {
            double t = 0.0;
            for (int k = 0; k < kThreads / 32; ++k) t += s_red[q][k];
            part[3 * b + q] = t;
        }
    }
}

// b_s from the partial sums (fixed order); A_s, K_s = A_s + i sigma2 b_s; after the last
// stage A' = A + h/6 (b_1 + 2 b_2 + 2 b_3 + b_4) into ST_AH (the field update stores it)
__global__ void rk4_amp_kernel(const double *__restrict__ part, int nparts, double *state, int stage,
                               double dt, double sigma2)
{
    __shared__ double s[3][kThreads];
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (int k = threadIdx.x; k < nparts; k += blockDim.x) {
        a0 += part[3 * k];
        a1 += part[3 * k + 1];
        a2 += part[3 * k + 2];
    }
    s[0][threadIdx.x] = a0;
    s[1][threadIdx.x] = a1;
    s[2][threadIdx.x] = a2;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int q = 0; q < 3; ++q) s[q][threadIdx.x] += s[q][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    const double br = s[1][0] / s[0][0], bi = -s[2][0] / s[0][0];
    state[ST_RK_B + 2 * stage] = br;
    state[ST_RK_B + 2 * stage + 1] = bi;
    double ar = state[ST_A_RE], ai = state[ST_A_IM];
    if (stage > 0) {
        const double c = (stage == 3) ? dt : 0.5 * dt;
        ar += c * state[ST_RK_B + 2 * (stage - 1)];
        ai += c * state[ST_RK_B + 2 * (stage - 1) + 1];
    }
    state[ST_RK_K + 2 * stage] = ar - sigma2 * bi;
    state[ST_RK_K + 2 * stage + 1] = ai + sigma2 * br;
    if (stage == 3) {
        const double *b = state + ST_RK_B;
        state[ST_AH_RE] = state[ST_A_RE] + dt / 6.0 * (b[0] + 2.0 * b[2] + 2.0 * b[4] + b[6]);
        state[ST_AH_IM] = state[ST_A_IM] + dt / 6.0 * (b[1] + 2.0 * b[3] + 2.0 * b[5] + b[7]);
    }
}

template <typename T, int BASIS>
struct RkTaps;
template <typename T>
struct RkTaps<T, VP_BASIS_TENT> {
    static constexpr int N = 2, LO = 0;
    __device__ static void weights(T t, T *w)
    {
        w[0] = T(1) - t;
        w[1] = t;
    }
};
template <typename T>
struct RkTaps<T, VP_BASIS_SEPTIC_BSPLINE> {
    static constexpr int N = 8, LO = -3;
    __device__ static void weights(T t, T *w) { septic_weights<T>(t, w); }
};
template <typename T>
struct RkTaps<T, VP_BASIS_CUBIC_BSPLINE> {
    static constexpr int N = 4, LO = -1;
    __device__ static void weights(T t, T *w)
    {
        const T s = T(1) - t, t2 = t * t, t3 = t2 * t;
        w[0] = s * s * s / T(6);
        w[3] = t3 / T(6);
        w[1] = T(2) / T(3) - t2 + T(0.5) * t3;
        w[2] = (T(1) - (w[0] + w[3])) - w[1];
    }
};

// deposit of every node at its RK4 end point (global atomics into a zeroed destination)
template <typename T, int BASIS>
__global__ void __launch_bounds__(kThreads)
    rk4_deposit_kernel(const T *__restrict__ src, T *__restrict__ dst, Geometry g,
                       const double2 *__restrict__ csx, const double *__restrict__ state, double *lost_acc)
{
    using TP = RkTaps<T, BASIS>;
    __shared__ double s_red[kThreads / 32];
    double K[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) K[q] = state[ST_RK_K + q];
    const int nx = g.nx, np = g.np;
    double lost = 0.0;
    const size_t n = (size_t)nx * np;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
         idx += (size_t)gridDim.x * blockDim.x) {
        const T w = src[idx];
        if (w == T(0)) continue;
        const int j = (int)(idx / nx), i = (int)(idx - (size_t)j * nx);
        const double2 t = csx[i];
        double2 e[4];
        double dth, dp;
        rk4_particle(t.x, t.y, g.p0 + j * g.hp, K, g.dt, g.delta, 4, e, dth, dp);
        // end point in cells, as node index + displacement
        const double du = dth / g.hx, dv = dp / g.hp;
        const double fu = floor(du), fv = floor(dv);
        T wx[TP::N], wy[TP::N];
        TP::weights((T)(du - fu), wx);
        TP::weights((T)(dv - fv), wy);
        const long mu = (long)i + (long)fu + TP::LO;
        const long nv = (long)j + (long)fv + TP::LO;
#pragma unroll
        for (int b = 0; b < TP::N; ++b) {
            const long rr = nv + b;
            const T wb = w * wy[b];
            if (rr < 0 || rr >= np) {
#pragma unroll
                for (int a = 0; a < TP::N; ++a) lost += (double)(wb * wx[a]);
                continue;
            }
#pragma unroll
            for (int a = 0; a < TP::N; ++a) {
                long ci = (mu + a) % nx;
                if (ci < 0) ci += nx;
                atomicAdd(dst + (size_t)rr * nx + ci, wb * wx[a]);
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) lost += __shfl_down_sync(0xffffffffu, lost, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = lost;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tl = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) tl += s_red[k];
        if (tl != 0.0) atomicAdd(lost_acc, tl);
    }
}

}  // namespace

int rk4_stage_blocks(int nx, int np) { return ((nx + 31) / 32) * ((np + kRows - 1) / kRows); }

template <typename T>
cudaError_t launch_rk4_stages(const T *w, const Geometry &g, const double2 *csx, double *state,
                              double *part, cudaStream_t s)
{
    const dim3 grid((g.nx + 31) / 32, (g.np + kRows - 1) / kRows);
    for (int stage = 0; stage < 4; ++stage) {
        rk4_stage_kernel<T><<<grid, kThreads, 0, s>>>(w, g, csx, state, stage, part);
        rk4_amp_kernel<<<1, kThreads, 0, s>>>(part, rk4_stage_blocks(g.nx, g.np), state, stage, g.dt,
                                              g.sigma2);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_rk4_deposit(const T *src, T *dst, const Geometry &g, const double2 *csx,
                               const double *state, double *lost_acc, cudaStream_t s)
{
    const size_t n = (size_t)g.nx * g.np;
    int grid = (int)((n + kThreads - 1) / kThreads);
    if (grid > 152 * 32) grid = 152 * 32;
    if (g.basis == VP_BASIS_TENT)
        rk4_deposit_kernel<T, VP_BASIS_TENT><<<grid, kThreads, 0, s>>>(src, dst, g, csx, state, lost_acc);
    else if (g.basis == VP_BASIS_SEPTIC_BSPLINE)
        rk4_deposit_kernel<T, VP_BASIS_SEPTIC_BSPLINE><<<grid, kThreads, 0, s>>>(src, dst, g, csx, state,
                                                                                lost_acc);
    else
        rk4_deposit_kernel<T, VP_BASIS_CUBIC_BSPLINE><<<grid, kThreads, 0, s>>>(src, dst, g, csx, state,
                                                                               lost_acc);
    return cudaGetLastError();
}

template cudaError_t launch_rk4_stages<float>(const float *, const Geometry &, const double2 *, double *,
                                              double *, cudaStream_t);
template cudaError_t launch_rk4_stages<double>(const double *, const Geometry &, const double2 *,
                                               double *, double *, cudaStream_t);
template cudaError_t launch_rk4_deposit<float>(const float *, float *, const Geometry &, const double2 *,
                                               const double *, double *, cudaStream_t);
template cudaError_t launch_rk4_deposit<double>(const double *, double *, const Geometry &,
                                                const double2 *, const double *, double *, cudaStream_t);

}  // namespace vp
