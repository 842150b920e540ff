// vp_filter.cu -- the mass-matrix solve Lambda w_fin = r (Sec. III update equation)
// for the tent basis, Lambda = (hx Tx) (x) (hp Tp), T = tridiag(1/6, 2/3, 1/6).
// The deposit omits the common factor hx hp, so here T w = r is solved per axis.
//
// x (periodic): T is cyclic. With z = sqrt(3) - 2 the root of z^2 + 4z + 1 = 0,
//   T = -(1 / (6 z)) (1 - z S)(1 - z S^{-1})   (S the cyclic shift),
// so T^{-1} r is a causal recursion y_i = r_i + z y_{i-1}, an anticausal one
// u_i = y_i + z u_{i+1}, and the factor -6z. Each thread runs the recursions
// over one chunk of a row held in shared memory; the value entering a chunk is
// the exact cyclic sum (1/(1 - z^nx)) sum_k z^k r_{i-k}, truncated after K
// terms where z^K is below the precision's round-off.
//
// p (open): T is the np x np Toeplitz block; the Thomas algorithm solves it.
// Its pivots depend only on the distance from the first row and reach their
// limit to FP64 precision within kPivots rows, so they come from a small
// table. A chunk of rows [s, e) starts the forward sweep K rows early (or at
// row 0) and the back substitution K rows late (or at row np-1); the error of
// the truncation is |z|^K.
#include <math.h>

#include "vp_internal.h"
#include "vp_sum.cuh"

namespace vp {
namespace {

constexpr double kZ = -0.26794919243112270647255365849413;   // sqrt(3) - 2

template <typename T>
struct Trunc;
template <>
struct Trunc<float> {
    static constexpr int K = 16;   // |z|^16 = 7e-10
};
template <>
struct Trunc<double> {
    static constexpr int K = 32;   // |z|^32 = 5e-19
};

__device__ __forceinline__ int padx(int i) { return i + (i >> 5); }

template <typename T>
__global__ void filter_x_kernel(const T *__restrict__ in, T *__restrict__ out, int nx, int np,
                                const double *__restrict__ piv, unsigned *err)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *buf = reinterpret_cast<T *>(smem_raw);
    const int j = blockIdx.x;
    const T *src = in + (size_t)j * nx;
    T *dst = out + (size_t)j * nx;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) buf[padx(i)] = src[i];
    __syncthreads();

    const T z = (T)kZ;
    const int K = Trunc<T>::K;
    const int L = nx < K ? nx : K;
    const T cyc = (T)(1.0 / (1.0 - pow(kZ, (double)nx)));
    const int C = (nx + blockDim.x - 1) / blockDim.x;
    const int s = threadIdx.x * C;
    const int e = min(s + C, nx);
    const bool active = s < nx;

    // causal: value y_{s-1}
    T init = T(0);
    if (active) {
        T zk = T(1);
        int idx = s - 1;
        if (idx < 0) idx += nx;
        for (int k = 0; k < L; ++k) {
            init += zk * buf[padx(idx)];
            zk *= z;
            if (--idx < 0) idx += nx;
        }
        init *= cyc;
    }
    __syncthreads();
    if (active) {
        T y = init;
        for (int i = s; i < e; ++i) {
            y = buf[padx(i)] + z * y;
            buf[padx(i)] = y;
        }
    }
    __syncthreads();
    // anticausal: value u_e
    if (active) {
        T zk = T(1);
        int idx = e;
        if (idx >= nx) idx -= nx;
        init = T(0);
        for (int k = 0; k < L; ++k) {
            init += zk * buf[padx(idx)];
            zk *= z;
            if (++idx >= nx) idx -= nx;
        }
        init *= cyc;
    }
    __syncthreads();
    // FP64: the scale -6z; FP32: the unit-DC-gain scale of the step as a float pair
    const bool f32 = sizeof(T) == 4;
    const T sh = f32 ? (T)piv[kPivXsFilter] : (T)(-6.0 * kZ);
    const T sl = f32 ? (T)piv[kPivXsFilter + 1] : T(0);
    if (active) {
        T u = init;
        for (int i = e - 1; i >= s; --i) {
            u = buf[padx(i)] + z * u;
            buf[padx(i)] = f32 ? u * sh + u * sl : u * sh;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nx; i += blockDim.x) dst[i] = buf[padx(i)];
    (void)np;
    (void)err;
}

constexpr int kPCols = 32;    // columns per warp
constexpr int kPWarps = 4;    // warps per block (adjacent column groups)
constexpr int kPChunk = 128;  // rows per chunk

// piv[2 r] = c'_r (super-diagonal factor), piv[2 r + 1] = 1 / beta_r, r < kPivots;
// piv[2 kPivots], piv[2 kPivots + 1] = their limits.
template <typename T>
__global__ void __launch_bounds__(kPCols *kPWarps)
    filter_p_kernel(const T *__restrict__ in, T *__restrict__ out, int nx, int np,
                    const double *__restrict__ piv, const double2 *__restrict__ csx,
                    double *part, int want_part, unsigned *err)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *gbuf = reinterpret_cast<T *>(smem_raw);   // [(kPChunk + K) rows][kPCols * kPWarps]
    __shared__ double s_red[3][kPWarps];
    const int K = Trunc<T>::K;
    const int W = kPCols * kPWarps;
    const int lane = threadIdx.x, wy = threadIdx.y;
    const int tid = wy * kPCols + lane;
    const int col = blockIdx.x * W + tid;
    const bool valid = col < nx;
    const int s = blockIdx.y * kPChunk;
    const int e = min(s + kPChunk, np);
    const int fe = min(e + K, np);          // forward sweep end (exclusive)
    const int fs = max(s - K, 0);           // forward sweep start
    const T sixth = (T)(1.0 / 6.0);
    const T cp_inf = (T)piv[2 * kPivots], ib_inf = (T)piv[2 * kPivots + 1];

    T g = T(0);
    if (valid) {
        for (int r = fs; r < fe; ++r) {
            const T ib = r < kPivots ? (T)piv[2 * r + 1] : ib_inf;
            const T rv = in[(size_t)r * nx + col];
            g = (rv - sixth * g) * ib;
            if (r >= s) gbuf[(size_t)(r - s) * W + tid] = g;
        }
    }
    // back substitution from fe - 1 (exact at the last row: w_{np-1} = g_{np-1})
    DSum<T> wacc;
    bool bad = false;
    if (valid) {
        T w = T(0);
        for (int r = fe - 1; r >= s; --r) {
            const T cp = r < kPivots ? (T)piv[2 * r] : cp_inf;
            const T gv = gbuf[(size_t)(r - s) * W + tid];
            w = (r == np - 1) ? gv : gv - cp * w;
            if (r < e) {
                out[(size_t)r * nx + col] = w;
                bad |= !isfinite(w);
                if (want_part) wacc.add(w);
            }
        }
    }
    if (bad) atomicOr(err, ERRF_NONFINITE);
    if (!want_part) return;
    double pw = 0.0, pc = 0.0, ps = 0.0;
    if (valid) {
        pw = wacc.value();
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
    if (tid == 0) {
        const size_t b = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
        for (int q = 0; q < 3; ++q) {
            double t = 0.0;
            for (int w = 0; w < kPWarps; ++w) t += s_red[q][w];
            part[3 * b + q] = t;
        }
    }
}

}  // namespace

template <typename T>
cudaError_t launch_filter_x(const T *in, T *out, int nx, int np, const double *piv, unsigned *err,
                            cudaStream_t s)
{
    const size_t smem = (size_t)(nx + nx / 32 + 1) * sizeof(T);
    cudaError_t e = cudaFuncSetAttribute(filter_x_kernel<T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    filter_x_kernel<T><<<np, 256, smem, s>>>(in, out, nx, np, piv, err);
    return cudaGetLastError();
}

// ---- septic B-spline Galerkin solves (cubic B-spline basis functions) ------------------
namespace {


// Along x (periodic): P7^{-1} = gain prod_i 1 / ((1 - z_i q)(1 - z_i / q)), one causal and one
// anticausal first-order recursion per pole over the row held in shared memory. Each thread
// sweeps its chunk; its start value is the geometric sum of the preceding (following) elements
// over one period, truncated at |z|^K below the rounding of T, times 1 / (1 - z^nx).
template <typename T>
__global__ void filter_x7_kernel(const T *__restrict__ in, T *__restrict__ out, int nx, int np, T sh, T sl)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *buf = reinterpret_cast<T *>(smem_raw);
    const int j = blockIdx.x;
    const T *src = in + (size_t)j * nx;
    T *dst = out + (size_t)j * nx;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) buf[padx(i)] = src[i];
    __syncthreads();
    const int C = (nx + blockDim.x - 1) / blockDim.x;
    const int s = threadIdx.x * C;
    const int e = min(s + C, nx);
    const bool active = s < nx;
    const double eps = sizeof(T) == 4 ? 1e-9 : 1e-18;
    for (int q = 0; q < 3; ++q) {
        const double zd = septic_pole(q);
        const T z = (T)zd;
        int K = (int)ceil(log(eps) / log(fabs(zd)));
        if (K > nx) K = nx;
        const T cyc = (T)(1.0 / (1.0 - pow(zd, (double)nx)));
        T init = T(0);
        if (active) {   // causal: y_{s-1}
            T zk = T(1);
            int idx = s - 1;
            if (idx < 0) idx += nx;
            for (int k = 0; k < K; ++k) {
                init += zk * buf[padx(idx)];
                zk *= z;
                if (--idx < 0) idx += nx;
            }
            init *= cyc;
        }
        __syncthreads();
        if (active) {
            T y = init;
            for (int i = s; i < e; ++i) {
                y = buf[padx(i)] + z * y;
                buf[padx(i)] = y;
            }
        }
        __syncthreads();
        if (active) {   // anticausal: u_e
            T zk = T(1);
            int idx = e;
            if (idx >= nx) idx -= nx;
            init = T(0);
            for (int k = 0; k < K; ++k) {
                init += zk * buf[padx(idx)];
                zk *= z;
                if (++idx >= nx) idx -= nx;
            }
            init *= cyc;
        }
        __syncthreads();
        if (active) {
            T u = init;
            for (int i = e - 1; i >= s; --i) {
                u = buf[padx(i)] + z * u;
                buf[padx(i)] = u;
            }
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        const T v = buf[padx(i)];
        dst[i] = v * sh + v * sl;
    }
}

// Along p (open): the np x np principal block of P7 = L D L^T, L unit lower with three
// subdiagonals; the factor rows are exact up to kLdlRows and their limit beyond
// (ldl[4 r] = D_r, ldl[4 r + m] = L_{r+m, r}). One thread per column: forward and back
// substitution.
template <typename T>
__global__ void filter_p7_kernel(const T *__restrict__ in, T *__restrict__ out, int nx, int np,
                                 const double *__restrict__ ldl)
{
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= nx) return;
    auto row = [&](int r) { return ldl + 4 * (size_t)(r < kLdlRows ? r : kLdlRows); };
    T y1 = T(0), y2 = T(0), y3 = T(0);   // y_{j-1}, y_{j-2}, y_{j-3}
    for (int j = 0; j < np; ++j) {
        T y = in[(size_t)j * nx + col];
        if (j >= 1) y -= (T)row(j - 1)[1] * y1;
        if (j >= 2) y -= (T)row(j - 2)[2] * y2;
        if (j >= 3) y -= (T)row(j - 3)[3] * y3;
        y3 = y2;
        y2 = y1;
        y1 = y;
        out[(size_t)j * nx + col] = y / (T)row(j)[0];
    }
    T w1 = T(0), w2 = T(0), w3 = T(0);   // w_{j+1}, w_{j+2}, w_{j+3}
    for (int j = np - 1; j >= 0; --j) {
        const double *rj = row(j);
        T w = out[(size_t)j * nx + col];
        if (j + 1 < np) w -= (T)rj[1] * w1;
        if (j + 2 < np) w -= (T)rj[2] * w2;
        if (j + 3 < np) w -= (T)rj[3] * w3;
        w3 = w2;
        w2 = w1;
        w1 = w;
        out[(size_t)j * nx + col] = w;
    }
}

}  // namespace

template <typename T>
cudaError_t launch_filter_x7(const T *in, T *out, int nx, int np, double sh, double sl, cudaStream_t s)
{
    const size_t smem = (size_t)(nx + nx / 32 + 1) * sizeof(T);
    cudaError_t e = cudaFuncSetAttribute(filter_x7_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    filter_x7_kernel<T><<<np, 256, smem, s>>>(in, out, nx, np, (T)sh, (T)sl);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_filter_p7(const T *in, T *out, int nx, int np, const double *ldl, cudaStream_t s)
{
    filter_p7_kernel<T><<<(nx + 127) / 128, 128, 0, s>>>(in, out, nx, np, ldl);
    return cudaGetLastError();
}

template cudaError_t launch_filter_x7<float>(const float *, float *, int, int, double, double, cudaStream_t);
template cudaError_t launch_filter_x7<double>(const double *, double *, int, int, double, double,
                                              cudaStream_t);
template cudaError_t launch_filter_p7<float>(const float *, float *, int, int, const double *, cudaStream_t);
template cudaError_t launch_filter_p7<double>(const double *, double *, int, int, const double *,
                                              cudaStream_t);

int filter_p_blocks(int nx, int np)
{
    const int W = kPCols * kPWarps;
    return ((nx + W - 1) / W) * ((np + kPChunk - 1) / kPChunk);
}

template <typename T>
cudaError_t launch_filter_p(const T *in, T *out, int nx, int np, const double *piv,
                            const double2 *csx, double *part, int want_part, unsigned *err,
                            cudaStream_t s)
{
    const int W = kPCols * kPWarps;
    const size_t smem = (size_t)(kPChunk + Trunc<T>::K) * W * sizeof(T);
    cudaError_t e = cudaFuncSetAttribute(filter_p_kernel<T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((nx + W - 1) / W, (np + kPChunk - 1) / kPChunk);
    dim3 block(kPCols, kPWarps);
    filter_p_kernel<T><<<grid, block, smem, s>>>(in, out, nx, np, piv, csx, part, want_part, err);
    return cudaGetLastError();
}

template cudaError_t launch_filter_x<float>(const float *, float *, int, int, const double *,
                                            unsigned *, cudaStream_t);
template cudaError_t launch_filter_x<double>(const double *, double *, int, int, const double *,
                                             unsigned *, cudaStream_t);
template cudaError_t launch_filter_p<float>(const float *, float *, int, int, const double *,
                                            const double2 *, double *, int, unsigned *,
                                            cudaStream_t);
template cudaError_t launch_filter_p<double>(const double *, double *, int, int, const double *,
                                             const double2 *, double *, int, unsigned *,
                                             cudaStream_t);

}  // namespace vp
