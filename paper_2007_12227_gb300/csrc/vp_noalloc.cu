// vp_noalloc.cu -- moments of a weight array with no device allocation at all.
//
// Some callers cannot allocate device memory at the moment they want the
// diagnostics: a host application whose framework allocator already holds all
// of the device's memory (a cudaMalloc would fail, or force that allocator to
// give its cache back), or a latency-critical loop that must not take the
// implicit device synchronisation a cudaMalloc or cudaFree can bring.
// vp_moments_static gives them the same FP64 moments as vp_moments for an FP32
// or FP64 weight array they already hold on the device: its per-block partial
// sums and the final sums live in one file-scope device array of this library,
// so the caller passes only the input, the mesh description and the output.
//
// The array is kMaxBlocks * kNumMoments partial sums plus the final sums
// (about 427 KB); every GPU that loads the library holds it until the process
// exits. Meshes above kMaxNodes nodes are rejected. All calls share the array:
// calls that overlap on the GPU (different streams, or different host threads
// on one stream without ordering) race, and each call keeps the previous
// call's contents until its own blocks overwrite them (every slot it reads is
// written first in the same call, so nothing needs clearing).
//
// The sums are plain FP64 sums, formed per thread, then by warp shuffles and
// in a fixed order over the warps and the blocks, as vp_moments forms its own
// (vp_moments uses another block count, so the two differ by rounding only).
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "vp_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kPerThread = 64;                        // nodes per thread, at most
constexpr int kMaxBlocks = 4096;
constexpr long long kMaxNodes = (long long)kMaxBlocks * kThreads * kPerThread;   // 2^26
constexpr int kOut = 16;                              // final sums (13 moments used)

static __device__ __align__(256) double g_scratch[kMaxBlocks * vp::kNumMoments + kOut];

// device address of g_scratch per device, looked up once with that device current and kept
// for the life of the process (a cudaDeviceReset of that device invalidates it: this entry
// point is not meant to be used across a device reset). g_mu orders the first calls of
// several host threads.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_addr[kMaxDevices];

template <typename T>
__global__ void moments_static_kernel(const T *__restrict__ w, vp::Geometry g, double *scratch)
{
    __shared__ double s_red[vp::kNumMoments][kThreads / 32];
    double acc[vp::kNumMoments];
#pragma unroll
    for (int q = 0; q < vp::kNumMoments; ++q) acc[q] = 0.0;
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
        const double cx = cos(x), sx = sin(x);
        double V = 0.0;
        if (g.potential == VP_POT_PENDULUM) V = -g.v_sign * cx;
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
        if (wt > T(0)) acc[8] -= ww * log(ww);   // in FP64 for FP32 weights too
        else acc[9] += ww;
        acc[10] += ww * cx;
        acc[11] += ww * sx;
        acc[12] = fmax(acc[12], fabs(ww));
    }
    const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < vp::kNumMoments; ++q) {
        double v = acc[q];
        for (int o = 16; o > 0; o >>= 1) {
            const double u = __shfl_down_sync(0xffffffffu, v, o);
            v = (q == 12) ? fmax(v, u) : v + u;
        }
        if (lane == 0) s_red[q][wy] = v;
    }
    __syncthreads();
    if (threadIdx.x < vp::kNumMoments) {
        const int q = threadIdx.x;
        double t = 0.0;
        for (int k = 0; k < kThreads / 32; ++k) t = (q == 12) ? fmax(t, s_red[q][k]) : t + s_red[q][k];
        scratch[(size_t)blockIdx.x * vp::kNumMoments + q] = t;
    }
}

__global__ void moments_static_final(double *scratch, int nblocks)
{
    const int q = threadIdx.x;
    if (q >= vp::kNumMoments) return;
    double t = 0.0;
    for (int b = 0; b < nblocks; ++b) {
        const double v = scratch[(size_t)b * vp::kNumMoments + q];
        t = (q == 12) ? fmax(t, v) : t + v;
    }
    scratch[(size_t)kMaxBlocks * vp::kNumMoments + q] = t;
}

}  // namespace

extern "C" vp_status vp_moments_static(const void *w, int32_t dtype, const vp_grid *grid,
                                       const vp_pusher *pusher, double lost_mass,
                                       const double *a_re_im, vp_moments_t *out, void *stream)
{
    if (!w || !grid || !pusher || !out || (dtype != VP_FP32 && dtype != VP_FP64)) return VP_ERR_ARG;
    if (grid->nx < 4 || grid->np < 4 || !(grid->x1 > grid->x0) || !(grid->p1 > grid->p0))
        return VP_ERR_ARG;
    const long long nodes = (long long)grid->nx * grid->np;
    if (nodes > kMaxNodes) {
        fprintf(stderr, "vp_moments_static: %lld nodes exceed the static scratch limit of %lld\n",
                nodes, kMaxNodes);
        return VP_ERR_UNSUPPORTED;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return VP_ERR_CUDA;
    double *scratch = nullptr;
    {
        // the host-side name g_scratch is not a device address: look the address up once per
        // device, with that device current, and check the lookup
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_addr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return VP_ERR_CUDA;
            g_addr[dev] = static_cast<double *>(p);
        }
        scratch = g_addr[dev];
    }
    vp::Geometry g;
    memset(&g, 0, sizeof(g));
    g.nx = grid->nx;
    g.np = grid->np;
    g.x0 = grid->x0;
    g.x1 = grid->x1;
    g.p0 = grid->p0;
    g.p1 = grid->p1;
    g.hx = (grid->x1 - grid->x0) / grid->nx;
    g.hp = (grid->p1 - grid->p0) / (grid->np - 1);
    g.kind = pusher->kind;
    g.potential = pusher->potential;
    g.v_sign = pusher->v_sign;
    g.omega = pusher->omega;
    g.dt = pusher->dt;
    long long blocks = (nodes + (long long)kThreads * kPerThread - 1) / ((long long)kThreads * kPerThread);
    if (blocks < 1) blocks = 1;
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (dtype == VP_FP64)
        moments_static_kernel<double><<<(int)blocks, kThreads, 0, s>>>(static_cast<const double *>(w), g,
                                                                       scratch);
    else
        moments_static_kernel<float><<<(int)blocks, kThreads, 0, s>>>(static_cast<const float *>(w), g,
                                                                      scratch);
    moments_static_final<<<1, 32, 0, s>>>(scratch, (int)blocks);
    double m[kOut];
    if (cudaGetLastError() != cudaSuccess) return VP_ERR_CUDA;
    if (cudaMemcpyAsync(m, scratch + (size_t)kMaxBlocks * vp::kNumMoments, sizeof(m),
                        cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return VP_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return VP_ERR_CUDA;
    const double hh = g.hx * g.hp, S = m[0];
    memset(out, 0, sizeof(*out));
    out->sum_w = S;
    out->mass = S * hh;
    out->mean_x = m[1] / S;
    out->mean_p = m[2] / S;
    out->var_x = m[3] / S - out->mean_x * out->mean_x;
    out->var_p = m[4] / S - out->mean_p * out->mean_p;
    out->cov_xp = m[5] / S - out->mean_x * out->mean_p;
    out->a_re = a_re_im ? a_re_im[0] : 0.0;
    out->a_im = a_re_im ? a_re_im[1] : 0.0;
    out->energy = (pusher->kind == VP_PUSH_FEL_DKD || pusher->kind == VP_PUSH_FEL_RK4)
                      ? out->mean_p + out->a_re * out->a_re + out->a_im * out->a_im
                      : m[6] / S;
    out->trapped = m[7] * hh;
    out->entropy = m[8] * hh;
    out->neg_mass = m[9] * hh;
    out->b_re = m[10] / S;
    out->b_im = -m[11] / S;
    out->max_abs_w = m[12];
    out->lost_mass = lost_mass;
    return VP_OK;
}
