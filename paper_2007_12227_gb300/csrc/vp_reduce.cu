// vp_reduce.cu -- FP64 reductions over the weights.
//
// FEL field (Sec. IV.B, dA/dz = <exp(-i Phi)>, detuning and space charge zero),
// drift-kick-drift in time:
//   A^{n+1/2} = A^n + h/2 b^n,  push with A^{n+1/2},  b^{n+1} = <exp(-i theta)>
//   of the new weights,  A^{n+1} = A^{n+1/2} + h/2 b^{n+1}.
// The bunching comes from per-block partial sums (sum w, sum w cos theta,
// sum w sin theta), reduced here in a fixed order so that results do not
// depend on scheduling.
//
// Moments (Sec. IV diagnostics: sum of weights, entropy): FP64 accumulation per
// thread, per-block partials, fixed-order final sum.
#include <math.h>

#include "vp_internal.h"
#include "vp_fel.cuh"
#include "vp_sum.cuh"

namespace vp {
namespace {

constexpr int kRedThreads = 256;
static_assert(kRedThreads == kFinThreads, "the finalize kernels run one block of kFinThreads threads");

// one block per 32-column strip x row chunk: column sums (compensated) then x cos/sin
constexpr int kFelRows = 256;

template <typename T>
__global__ void fel_partials_kernel(const T *__restrict__ w, int nx, int np,
                                    const double2 *__restrict__ csx, double *part)
{
    __shared__ double s_red[3][kRedThreads / 32];
    const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
    const int col = blockIdx.x * 32 + lane;
    const int r0 = blockIdx.y * kFelRows;
    const int r1 = min(r0 + kFelRows, np);
    DSum<T> acc;
    if (col < nx)
        for (int r = r0 + wy; r < r1; r += kRedThreads / 32) acc.add(w[(size_t)r * nx + col]);
    double pw = acc.value(), pc = 0.0, ps = 0.0;
    if (col < nx) {
        const double2 t = csx[col];
        pc = pw * t.x;
        ps = pw * t.y;
    }
    double v[3] = {pw, pc, ps};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
        if (lane == 0) s_red[q][wy] = v[q];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const size_t b = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
        for (int q = 0; q < 3; ++q) {
            double t = 0.0;
            for (int k = 0; k < kRedThreads / 32; ++k) t += s_red[q][k];
            part[3 * b + q] = t;
        }
    }
}

// FEL space charge: per block (32 columns x kFelRows rows) the sums of the state against the
// mass weights and against the half-drift phase factors e^{-i (theta_i + phi_j)}:
// per column C = sum_j s_ij rc_j, S = sum_j s_ij rs_j, then Re += cos(th) C - sin(th) S and
// Im -= sin(th) C + cos(th) S (rc, rs already carry Lambda_p^{-1} for the state s = Lambda_p w)
template <typename T>
__global__ void fel_tilde_kernel(const T *__restrict__ st, int nx, int np, const double2 *__restrict__ csx,
                                 const double *__restrict__ rc, const double *__restrict__ rs,
                                 const double *__restrict__ sig, double *part)
{
    __shared__ double s_red[3][kRedThreads / 32];
    const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
    const int col = blockIdx.x * 32 + lane;
    const int r0 = blockIdx.y * kFelRows;
    const int r1 = min(r0 + kFelRows, np);
    double m = 0.0, c = 0.0, sn = 0.0;
    if (col < nx)
        for (int r = r0 + wy; r < r1; r += kRedThreads / 32) {
            const double v = (double)st[(size_t)r * nx + col];
            m += v * (sig ? sig[r] : 1.0);
            c += v * rc[r];
            sn += v * rs[r];
        }
    double v3[3] = {m, 0.0, 0.0};
    if (col < nx) {
        const double2 t = csx[col];
        v3[1] = t.x * c - t.y * sn;
        v3[2] = -(t.y * c + t.x * sn);
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        for (int o = 16; o > 0; o >>= 1) v3[q] += __shfl_down_sync(0xffffffffu, v3[q], o);
        if (lane == 0) s_red[q][wy] = v3[q];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const size_t b = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
        for (int q = 0; q < 3; ++q) {
            double t = 0.0;
            for (int k = 0; k < kRedThreads / 32; ++k) t += s_red[q][k];
            part[3 * b + q] = t;
        }
    }
}

// K = A^{n+1/2} + i sigma2 bt, bt = <e^{-i theta~}> from the tilde partial sums (one block)
__global__ void fel_kick_kernel(const double *__restrict__ part, int nparts, double *state, double sigma2)
{
    __shared__ double s[3][kRedThreads];
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
    const double bt_re = s[1][0] / s[0][0], bt_im = s[2][0] / s[0][0];
    const double kr = state[ST_AH_RE] - sigma2 * bt_im, ki = state[ST_AH_IM] + sigma2 * bt_re;
    state[ST_K_RE] = kr;
    state[ST_K_IM] = ki;
    state[ST_M] = hypot(kr, ki);
    state[ST_PHI] = atan2(kr, -ki);
}

// FEL field update from per-block partial sums (run by one block of kFinThreads threads)
__device__ void fel_finalize_block(const double *__restrict__ part, int nparts, double *state,
                                   double *hist, int hist_cap, double dt, int init, int rk4 = 0)
{
    __shared__ double s[3 * kFinThreads];
    fel_finalize_core(part, nparts, state, hist, hist_cap, dt, init, rk4, s);
}

__global__ void fel_finalize_kernel(const double *__restrict__ part, int nparts, double *state,
                                    double *hist, int hist_cap, double dt, int init, int rk4)
{
    fel_finalize_block(part, nparts, state, hist, hist_cap, dt, init, rk4);
}

// end of a batched step: block k finishes instance k, flips its buffer parity and counts down
// the steps it still takes in this call (instances already at zero are left alone)
__global__ void batch_finalize_kernel(const BatchFinal *__restrict__ fin, int *parity, int *left)
{
    if (left[blockIdx.x] <= 0) return;
    const BatchFinal f = fin[blockIdx.x];
    if (f.fel) {
        fel_finalize_block(f.part, f.nparts, f.state, f.hist, f.hist_cap, f.dt, 0);
    } else if (threadIdx.x == 0) {
        const double st = f.state[ST_STEP] + 1.0;
        f.state[ST_STEP] = st;
        f.state[ST_TAU] = st * f.dt;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        parity[blockIdx.x] ^= 1;
        left[blockIdx.x] -= 1;
    }
}

// plain step counter for non-FEL sims
__global__ void count_step_kernel(double *state, double dt)
{
    const double st = state[ST_STEP] + 1.0;
    state[ST_STEP] = st;
    state[ST_TAU] = st * dt;
}

// w ln w in FP64, for FP32 weights too (the entropy is an FP64 reduction)
template <typename T>
__device__ __forceinline__ double wlogw(T w)
{
    const double d = (double)w;
    return d * log(d);
}

template <typename T>
__global__ void moments_kernel(const T *__restrict__ w, Geometry g, const double2 *__restrict__ csx,
                               double *part)
{
    __shared__ double s_red[kNumMoments][kRedThreads / 32];
    double acc[kNumMoments];
#pragma unroll
    for (int q = 0; q < kNumMoments; ++q) acc[q] = 0.0;
    const size_t n = (size_t)g.nx * g.np;
    const double hsep = fabs(g.v_sign);
    const bool pend = (g.kind == VP_PUSH_LEAPFROG_KDK && g.potential == VP_POT_PENDULUM);
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
         idx += (size_t)gridDim.x * blockDim.x) {
        const T wt = w[idx];
        if (wt == T(0)) continue;
        const int j = (int)(idx / g.nx), i = (int)(idx - (size_t)j * g.nx);
        const double x = g.x0 + i * g.hx, p = g.p0 + j * g.hp;
        const double ww = (double)wt;
        const double2 cs = csx[i];
        double V = 0.0;
        if (g.potential == VP_POT_PENDULUM) V = -g.v_sign * cs.x;
        else if (g.potential == VP_POT_HARMONIC) V = 0.5 * g.omega * g.omega * x * x;
        const double H = 0.5 * p * p + V;
        acc[0] += ww;
        acc[1] += ww * x;
        acc[2] += ww * p;
        acc[3] += ww * x * x;
        acc[4] += ww * p * p;
        acc[5] += ww * x * p;
        acc[6] += ww * H;
        if (pend && H < hsep) acc[7] += ww;
        if (wt > T(0)) acc[8] -= wlogw(wt);
        else acc[9] += ww;
        acc[10] += ww * cs.x;
        acc[11] += ww * cs.y;
        acc[12] = fmax(acc[12], fabs(ww));
    }
    const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < kNumMoments; ++q) {
        double v = acc[q];
        for (int o = 16; o > 0; o >>= 1) {
            const double u = __shfl_down_sync(0xffffffffu, v, o);
            v = (q == 12) ? fmax(v, u) : v + u;
        }
        if (lane == 0) s_red[q][wy] = v;
    }
    __syncthreads();
    if (threadIdx.x < kNumMoments) {
        const int q = threadIdx.x;
        double t = 0.0;
        for (int k = 0; k < kRedThreads / 32; ++k) t = (q == 12) ? fmax(t, s_red[q][k]) : t + s_red[q][k];
        part[(size_t)blockIdx.x * kNumMoments + q] = t;
    }
}

__global__ void moments_finalize_kernel(const double *__restrict__ part, int nblocks,
                                        const double *__restrict__ lost, int nlost, double *out)
{
    const int q = threadIdx.x;
    if (q < kNumMoments) {
        double t = 0.0;
        for (int b = 0; b < nblocks; ++b) {
            const double v = part[(size_t)b * kNumMoments + q];
            t = (q == 12) ? fmax(t, v) : t + v;
        }
        out[q] = t;
    } else if (q == kNumMoments) {
        double t = 0.0;
        for (int b = 0; b < nlost; ++b) t += lost[b];
        out[q] = t;
    }
}

template <typename Tin, typename Tout>
__global__ void convert_kernel(const Tin *__restrict__ in, Tout *__restrict__ out, size_t n)
{
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (size_t)gridDim.x * blockDim.x)
        out[k] = (Tout)in[k];
}

}  // namespace

int fel_partial_blocks(int nx, int np)
{
    return ((nx + 31) / 32) * ((np + kFelRows - 1) / kFelRows);
}

template <typename T>
cudaError_t launch_fel_tilde(const T *state, int nx, int np, const double2 *csx, const double *rc,
                             const double *rs, const double *sig, double *part, cudaStream_t s)
{
    dim3 grid((nx + 31) / 32, (np + kFelRows - 1) / kFelRows);
    fel_tilde_kernel<T><<<grid, kRedThreads, 0, s>>>(state, nx, np, csx, rc, rs, sig, part);
    return cudaGetLastError();
}
template cudaError_t launch_fel_tilde<float>(const float *, int, int, const double2 *, const double *,
                                             const double *, const double *, double *, cudaStream_t);
template cudaError_t launch_fel_tilde<double>(const double *, int, int, const double2 *, const double *,
                                              const double *, const double *, double *, cudaStream_t);

cudaError_t launch_fel_kick(const double *part, int nparts, double *state, double sigma2, cudaStream_t s)
{
    fel_kick_kernel<<<1, kRedThreads, 0, s>>>(part, nparts, state, sigma2);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fel_partials(const T *w, int nx, int np, const double2 *csx, double *part,
                                cudaStream_t s)
{
    dim3 grid((nx + 31) / 32, (np + kFelRows - 1) / kFelRows);
    fel_partials_kernel<T><<<grid, kRedThreads, 0, s>>>(w, nx, np, csx, part);
    return cudaGetLastError();
}

cudaError_t launch_fel_finalize(const double *part, int nparts, double *state, double *hist,
                                int hist_cap, double dt, int init, cudaStream_t s, int rk4)
{
    fel_finalize_kernel<<<1, kRedThreads, 0, s>>>(part, nparts, state, hist, hist_cap, dt, init, rk4);
    return cudaGetLastError();
}

cudaError_t launch_batch_finalize(const BatchFinal *fin, int ninst, int *parity, int *left, cudaStream_t s)
{
    batch_finalize_kernel<<<ninst, kRedThreads, 0, s>>>(fin, parity, left);
    return cudaGetLastError();
}

cudaError_t launch_count_step(double *state, double dt, cudaStream_t s)
{
    count_step_kernel<<<1, 1, 0, s>>>(state, dt);
    return cudaGetLastError();
}

int moment_blocks(int nx, int np)
{
    const size_t n = (size_t)nx * np;
    size_t b = (n + kRedThreads - 1) / kRedThreads;
    if (b > 152 * 8) b = 152 * 8;
    return (int)b;
}

template <typename T>
cudaError_t launch_moments(const T *w, const Geometry &g, const double2 *csx, double *part,
                           int nblocks, cudaStream_t s)
{
    moments_kernel<T><<<nblocks, kRedThreads, 0, s>>>(w, g, csx, part);
    return cudaGetLastError();
}

cudaError_t launch_moments_finalize(const double *part, int nblocks, const double *lost, int nlost,
                                    double *out, cudaStream_t s)
{
    moments_finalize_kernel<<<1, 32, 0, s>>>(part, nblocks, lost, nlost, out);
    return cudaGetLastError();
}

template <typename Tin, typename Tout>
cudaError_t launch_convert(const Tin *in, Tout *out, size_t n, cudaStream_t s)
{
    size_t b = (n + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    convert_kernel<Tin, Tout><<<(int)b, 256, 0, s>>>(in, out, n);
    return cudaGetLastError();
}

template cudaError_t launch_fel_partials<float>(const float *, int, int, const double2 *, double *,
                                                cudaStream_t);
template cudaError_t launch_fel_partials<double>(const double *, int, int, const double2 *,
                                                 double *, cudaStream_t);
template cudaError_t launch_moments<float>(const float *, const Geometry &, const double2 *,
                                           double *, int, cudaStream_t);
template cudaError_t launch_moments<double>(const double *, const Geometry &, const double2 *,
                                            double *, int, cudaStream_t);
template cudaError_t launch_convert<float, double>(const float *, double *, size_t, cudaStream_t);
template cudaError_t launch_convert<double, float>(const double *, float *, size_t, cudaStream_t);

}  // namespace vp
