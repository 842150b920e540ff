// vp_tables.cu -- per-column and per-row push tables, built once in FP64.
//
// Each pusher of Sec. II/IV moves mesh node (x_i, p_j) by a displacement that
// splits into a part depending only on the column i, a part depending only on
// the row j, and one term KU/KV * (alpha sin(a_i + y_j) + beta cos(a_i + y_j)).
//
//   leapfrog KDK, H = p^2/2 + V(x), F = V':
//     p_half = p - h/2 F(x),  x' = x + h p_half,  p' = p_half - h/2 F(x')
//     dx = h p - h^2/2 F(x)                      -> column -h^2/2 F, row h p
//     dp = -h/2 (F(x) + F(x'))                   -> column -h/2 F(x), and
//       pendulum F = s sin: F(x') = s sin(a + y), a = x - h^2/2 F(x), y = h p
//       harmonic F = w^2 x: F(x') = w^2 ((1 - h^2 w^2/2) x + h p)  (affine)
//   exact rotation by phase omega h (Sec. IV.A): affine in (x, p)
//   FEL drift-kick-drift (Sec. IV.B, detuning and space charge zero):
//     theta~ = theta + h/2 p,  p' = p - 2 h Re(A e^{i theta~}),
//     theta' = theta~ + h/2 p'
//     dtheta = h p - h^2 Re(A e^{i(a + y)}),  dp = -2h Re(A e^{i(a + y)}),
//     a = theta, y = h p / 2;  Re(A e^{i psi}) = -A_im sin psi + A_re cos psi.
#include <math.h>

#include "vp_internal.h"

namespace vp {
namespace {

__device__ __forceinline__ void split_int(double v, int &i, double &f)
{
    const double r = rint(v);
    i = (int)r;
    f = v - r;
}

template <typename T>
__global__ void col_kernel(Geometry g, ColEntry<T> *col, double *ucol, double *vcol, double2 *csx)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.nx) return;
    const double x = g.x0 + i * g.hx;
    const double h = g.dt;
    double U = 0.0, V = 0.0, a = x;
    if (g.kind == VP_PUSH_LEAPFROG_KDK) {
        if (g.potential == VP_POT_PENDULUM) {
            const double F = g.v_sign * sin(x);
            U = -(h * h / (2.0 * g.hx)) * F;
            V = -(h / (2.0 * g.hp)) * F;
            a = x - 0.5 * h * h * F;
        } else if (g.potential == VP_POT_HARMONIC) {
            const double w2 = g.omega * g.omega;
            U = -(h * h / (2.0 * g.hx)) * w2 * x;
            V = -(h * w2 / (2.0 * g.hp)) * x * (2.0 - 0.5 * h * h * w2);
        }
    } else if (g.kind == VP_PUSH_EXACT_ROTATION) {
        const double th = g.omega * h;
        U = x * (cos(th) - 1.0) / g.hx;
        V = -g.omega * x * sin(th) / g.hp;
    }
    ColEntry<T> e;
    double f;
    split_int(U, e.ui, f);
    e.uf = (T)f;
    split_int(V, e.vi, f);
    e.vf = (T)f;
    e.sa = (T)sin(a);
    e.ca = (T)cos(a);
    col[i] = e;
    ucol[i] = U;
    vcol[i] = V;
    csx[i] = make_double2(cos(x), sin(x));
}

template <typename T>
__global__ void row_kernel(Geometry g, RowEntry<T> *row, RowBound *rowb)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= g.np) return;
    const double p = g.p0 + j * g.hp;
    const double h = g.dt;
    double U = 0.0, V = 0.0, y = 0.0;
    if (g.kind == VP_PUSH_LEAPFROG_KDK) {
        U = (h / g.hx) * p;
        if (g.potential == VP_POT_PENDULUM) {
            y = h * p;
        } else if (g.potential == VP_POT_HARMONIC) {
            const double w2 = g.omega * g.omega;
            V = -(h * h * w2 / (2.0 * g.hp)) * p;
        }
    } else if (g.kind == VP_PUSH_EXACT_ROTATION) {
        const double th = g.omega * h;
        U = p * sin(th) / (g.omega * g.hx);
        V = p * (cos(th) - 1.0) / g.hp;
    } else {
        // FEL: d theta/dz = delta + p; the kick phase is taken after the first half drift
        U = (h / g.hx) * (p + g.delta);
        y = 0.5 * h * (p + g.delta);
    }
    RowEntry<T> e;
    double f;
    split_int(U, e.ui, f);
    e.uf = (T)f;
    split_int(V, e.vi, f);
    e.vf = (T)f;
    e.sy = (T)sin(y);
    e.cy = (T)cos(y);
    e.sy2 = e.sy;
    e.cy2 = e.cy;
    row[j] = e;
    RowBound b;
    b.u = U;
    b.v = V;
    b.y = y;
    b.pad = 0.0;
    rowb[j] = b;
}

}  // namespace

cudaError_t build_tables(const Geometry &g, int precision, void *col, void *row, RowBound *rowb,
                         double *ucol, double *vcol, double2 *csx, cudaStream_t s)
{
    const int bs = 256;
    if (precision == VP_FP32) {
        col_kernel<float><<<(g.nx + bs - 1) / bs, bs, 0, s>>>(g, (ColEntry<float> *)col, ucol,
                                                             vcol, csx);
        row_kernel<float><<<(g.np + bs - 1) / bs, bs, 0, s>>>(g, (RowEntry<float> *)row, rowb);
    } else {
        col_kernel<double><<<(g.nx + bs - 1) / bs, bs, 0, s>>>(g, (ColEntry<double> *)col, ucol,
                                                               vcol, csx);
        row_kernel<double><<<(g.np + bs - 1) / bs, bs, 0, s>>>(g, (RowEntry<double> *)row, rowb);
    }
    return cudaGetLastError();
}

}  // namespace vp
