// vp_api.cu -- host side of the C ABI declared in include/vlasov.h: argument
// checks, the planner (tile shape, workspace layout, source-window bounds), and
// the per-step launch sequence
//   push + deposit  ->  [Lambda^{-1}: x solve, p solve]  ->  [FEL field update]
// on the caller's stream. The library allocates no device memory: every device
// buffer is carved out of the caller's workspace.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "vp_internal.h"

using namespace vp;

namespace {

constexpr size_t kAlign = 256;
constexpr int kDefaultHist = 4096;
constexpr size_t kMaxSmem = 220 * 1024;
constexpr int kMoutLen = 32;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct Layout {
    size_t f0, f1, tmp, col, row, rowb, vcb, rowbf, vcbf, csx, ucol, vcol, piv, ldl, sigma, smax, tsrc, rtil,
        state, hist,
        lost, part, mpart, mout, err, ticket, total;
};

struct Plan {
    Geometry g;
    int precision, projection, kernel, tx, tp, ntx, ntp, hist_cap, nlost, npart, nmblk, nblk;
    bool galerkin, fel;
    // fused kernel: guard band, window stride, threads per CTA, whole-period tiles;
    // state_s: the stored state is s = Lambda_x^{-1} r instead of the weights w
    int G, Gp, ws, threads;
    int rowcache;   // fused kernel: row-table rows a tile may cache in shared memory
    bool full_row, state_s;
    // Galerkin one-pass plan with a separate x pass: tiles without x halo store the deposit into
    // tmp, and a row pass solves Lambda_x along whole rows into the state buffer
    bool xpass;
    int xgrid;   // CTAs of the row pass (persistent)
    bool rk4;   // FEL with the RK4 integrator: the scatter kernel and stage reductions
    bool septic_gal;   // cubic B-spline basis, Galerkin: 7-band solves after the scatter deposit
    double x7_scale;   // septic x solve: the scale that gives the recursions a unit DC gain
    Layout L;
};

vp_status fail(char *msg, vp_status st, const char *fmt, ...)
{
    if (msg) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(msg, 512, fmt, ap);
        va_end(ap);
    }
    return st;
}

bool finite(double v) { return isfinite(v) != 0; }

vp_status make_plan(const vp_grid *grid, int32_t basis, const vp_pusher *pu, const vp_opts *opts,
                    Plan *P, char *msg)
{
    if (!grid || !pu || !opts) return fail(msg, VP_ERR_ARG, "NULL grid, pusher or opts");
    if (grid->nx < 4 || grid->np < 4)
        return fail(msg, VP_ERR_ARG, "grid needs nx >= 4 and np >= 4 (got %d x %d)", grid->nx,
                    grid->np);
    if ((double)grid->nx * grid->np > 2147483647.0)
        return fail(msg, VP_ERR_UNSUPPORTED, "nx * np must stay below 2^31");
    if (!finite(grid->x0) || !finite(grid->x1) || !finite(grid->p0) || !finite(grid->p1) ||
        !(grid->x1 > grid->x0) || !(grid->p1 > grid->p0))
        return fail(msg, VP_ERR_ARG, "grid ranges must be finite with x1 > x0 and p1 > p0");
    if (basis != VP_BASIS_TENT && basis != VP_BASIS_CUBIC_BSPLINE && basis != VP_BASIS_SEPTIC_BSPLINE)
        return fail(msg, VP_ERR_ARG, "unknown basis %d", basis);
    if (pu->kind < 0 || pu->kind > 3) return fail(msg, VP_ERR_ARG, "unknown pusher kind %d", pu->kind);
    if (pu->potential < 0 || pu->potential > 2)
        return fail(msg, VP_ERR_ARG, "unknown potential %d", pu->potential);
    if (!finite(pu->dt) || !finite(pu->v_sign) || !finite(pu->omega) || !finite(pu->a0_re) ||
        !finite(pu->a0_im) || !finite(pu->delta) || !finite(pu->sigma2))
        return fail(msg, VP_ERR_ARG, "pusher parameters must be finite");
    if (opts->precision != VP_FP32 && opts->precision != VP_FP64)
        return fail(msg, VP_ERR_ARG, "unknown precision %d", opts->precision);
    if (opts->projection != VP_PROJ_GALERKIN && opts->projection != VP_PROJ_LUMPED)
        return fail(msg, VP_ERR_ARG, "unknown projection %d", opts->projection);
    if (opts->kernel < 0 || opts->kernel > 4) return fail(msg, VP_ERR_ARG, "unknown kernel %d", opts->kernel);
    if (opts->tile_x < 0 || opts->tile_p < 0 || opts->history_cap < 0)
        return fail(msg, VP_ERR_ARG, "tile sizes and history capacity must be >= 0");

    Geometry &g = P->g;
    memset(&g, 0, sizeof(g));
    g.nx = grid->nx;
    g.np = grid->np;
    g.x0 = grid->x0;
    g.x1 = grid->x1;
    g.p0 = grid->p0;
    g.p1 = grid->p1;
    g.hx = (grid->x1 - grid->x0) / grid->nx;
    g.hp = (grid->p1 - grid->p0) / (grid->np - 1);
    g.basis = basis;
    g.kind = pu->kind;
    g.potential = pu->potential;
    g.projection = opts->projection;
    g.v_sign = pu->v_sign;
    g.omega = pu->omega;
    g.dt = pu->dt;
    const bool fel_kind = pu->kind == VP_PUSH_FEL_DKD || pu->kind == VP_PUSH_FEL_RK4;
    g.delta = fel_kind ? pu->delta : 0.0;
    g.sigma2 = fel_kind ? pu->sigma2 : 0.0;
    const double h = pu->dt;
    const bool pend = pu->kind == VP_PUSH_LEAPFROG_KDK && pu->potential == VP_POT_PENDULUM;
    P->fel = fel_kind;
    P->rk4 = pu->kind == VP_PUSH_FEL_RK4;
    if (pend || P->fel) {
        const double L = grid->x1 - grid->x0, per = L / (2.0 * M_PI);
        if (fabs(per - rint(per)) > 1e-9 * per || rint(per) < 1.0)
            return fail(msg, VP_ERR_ARG,
                        "pendulum and FEL need a coordinate period that is a multiple of 2 pi");
    }
    if ((pu->kind == VP_PUSH_EXACT_ROTATION ||
         (pu->kind == VP_PUSH_LEAPFROG_KDK && pu->potential == VP_POT_HARMONIC)) &&
        !(pu->omega > 0.0))
        return fail(msg, VP_ERR_ARG, "harmonic motion needs omega > 0");
    if (pend) {
        g.KV = -(h / (2.0 * g.hp));
        g.alpha0 = pu->v_sign;
        g.a_pad = 0.5 * h * h * fabs(pu->v_sign);
    } else if (P->fel) {
        g.KU = -(h * h / g.hx);
        g.KV = -(2.0 * h / g.hp);
    }

    g.m0 = hypot(g.alpha0, g.beta0);
    g.phi0 = atan2(g.beta0, g.alpha0);

    P->precision = opts->precision;
    P->projection = opts->projection;
    P->galerkin = basis == VP_BASIS_CUBIC_BSPLINE && opts->projection == VP_PROJ_GALERKIN;
    P->septic_gal = basis == VP_BASIS_SEPTIC_BSPLINE && opts->projection == VP_PROJ_GALERKIN;
    const size_t sz = opts->precision == VP_FP64 ? 8 : 4;
    const bool wide_rotation = pu->kind == VP_PUSH_EXACT_ROTATION && fabs(pu->omega * h) >= 0.5 * M_PI;
    int kernel = opts->kernel;
    P->xpass = false;
    if (kernel == VP_KERNEL_FUSED_XPASS) {
        // the one-pass tile without its x solve, then an exact row pass (cubic B-spline Galerkin;
        // the FEL's bunching sums come from the deposit through the eigenvalue of Lambda_x)
        if (!P->galerkin || P->rk4)
            return fail(msg, VP_ERR_UNSUPPORTED,
                        "the separate x pass serves cubic B-spline Galerkin plans (not the RK4 FEL)");
        int xt = 0, xper = 0;
        xrow_shape(opts->precision, grid->nx, &xt, &xper);
        if (xt == 0)
            return fail(msg, VP_ERR_UNSUPPORTED, "the x-solve row pass takes rows of at most %d nodes",
                        kXRowMaxThreads * xrow_max_per(opts->precision));
        P->xpass = true;
        kernel = VP_KERNEL_FUSED;
    }
    if (P->rk4 || basis == VP_BASIS_SEPTIC_BSPLINE) {
        // the RK4 end point is not of the tabulated displacement form, and the 8-tap septic
        // deposit has no one-pass form here: global-atomic deposit
        if (kernel == VP_KERNEL_FUSED)
            return fail(msg, VP_ERR_UNSUPPORTED,
                        "the RK4 FEL step and the septic deposit run on the scatter kernel");
        kernel = VP_KERNEL_SCATTER;
    }
    P->G = 8;   // a multiple of 4, so that the x solve's rows start 16-byte aligned
    P->Gp = 8;
    P->full_row = false;
    P->ws = 0;
    P->threads = 0;
    P->rowcache = 0;
    int ftx = 0, ftp = 0;
    if (kernel == VP_KERNEL_AUTO || kernel == VP_KERNEL_FUSED) {
        const int halo = P->galerkin && !P->xpass ? fused_halo(opts->precision) : 0;
        const int R = basis == VP_BASIS_TENT ? 1 : 2;
        const int G = P->G, Gp = P->Gp;
        ftx = opts->tile_x ? opts->tile_x : (opts->precision == VP_FP64 ? 128 : 224);
        ftp = opts->tile_p ? opts->tile_p : 64;
        bool full = false;
        // whole-period tiles when the mesh is little wider than a windowed tile; by default only
        // while the tile's source columns fit the two-CTA thread count (a default plan of more
        // threads runs one CTA per SM, and in a batch it would set that for every item)
        const bool full_fits = (grid->nx + 2 * R + 8 + 31) / 32 * 32 <= kFusedThreads2;
        if (!P->xpass && grid->nx <= kFusedMaxRow && grid->nx < ftx + 2 * halo + 2 * G + 64 &&
            (full_fits || opts->tile_x != 0 || grid->nx <= ftx + 2 * halo + 2 * G)) {
            full = true;
            ftx = grid->nx;
        }
        if (!full && ftx + 2 * halo > kFusedMaxRow) ftx = kFusedMaxRow - 2 * halo;
        ftp = std::min(std::min(ftp, grid->np), kFusedMaxTileP);
        const int WW = full ? grid->nx + 2 * G : ftx + 2 * halo + 2 * G;
        // row stride a multiple of 32 words: the rows start 16-byte aligned, and lanes that
        // deposit into adjacent columns of two neighbouring rows hit distinct banks
        const int ws = (WW + 31) / 32 * 32;
        const int wsrc = (full ? grid->nx : ftx + 2 * halo) + 2 * R + 8;
        // two CTAs per SM (up to 320 threads) unless the tile is wide: then one CTA of up
        // to 576 threads per SM
        const bool wide = (wsrc + 31) / 32 * 32 > kFusedThreads2;
        const int threads = std::min(wide ? kFusedMaxThreads : kFusedThreads2, (wsrc + 31) / 32 * 32);
        const size_t cap = wide ? (size_t)200 * 1024 : (size_t)112 * 1024;
        auto smem_of = [&](int tp_) {
            return sz == 8 ? fused_smem_bytes<double>(ws, tp_ + 2 * Gp, threads)
                           : fused_smem_bytes<float>(ws, tp_ + 2 * Gp, threads);
        };
        while (smem_of(ftp) > cap && ftp > 8) ftp /= 2;
        const size_t smem = smem_of(ftp);
        const bool ok = !wide_rotation && smem <= kMaxSmem && (full || WW < grid->nx) && ftx >= 1;
        if (ok) {
            kernel = VP_KERNEL_FUSED;
            P->full_row = full;
            P->ws = ws;
            P->threads = threads;
            // the shared memory left beside the window keeps the tile's row table
            P->rowcache = fused_rowcache_rows(opts->precision, smem, wide ? 1 : 2);
        } else if (kernel == VP_KERNEL_FUSED) {
            return fail(msg, VP_ERR_UNSUPPORTED,
                        "the fused kernel needs a mesh wider than its window (nx = %d)", grid->nx);
        } else {
            kernel = VP_KERNEL_TILED;
        }
    }
    if (kernel == VP_KERNEL_TILED && wide_rotation) kernel = VP_KERNEL_SCATTER;
    P->kernel = kernel;
    P->state_s = kernel == VP_KERNEL_FUSED && P->galerkin;
    int tx = opts->tile_x ? opts->tile_x : (opts->precision == VP_FP64 ? 64 : 128);
    int tp = opts->tile_p ? opts->tile_p : 64;
    if (kernel == VP_KERNEL_FUSED) {
        tx = ftx;
        tp = ftp;
    }
    tx = std::min(tx, grid->nx);
    tp = std::min(tp, grid->np);
    if (tx > 4096 || tp > 4096) return fail(msg, VP_ERR_ARG, "tile sides must be <= 4096");
    if (kernel == VP_KERNEL_TILED) {
        const size_t smem = sz == 8 ? tiled_smem_bytes<double>(tx, tp) : tiled_smem_bytes<float>(tx, tp);
        if (smem > kMaxSmem)
            return fail(msg, VP_ERR_UNSUPPORTED, "tile %d x %d needs %zu bytes of shared memory", tx,
                        tp, smem);
    }
    if (P->galerkin || P->septic_gal) {
        const size_t smem = (size_t)(grid->nx + grid->nx / 32 + 1) * sz;
        if (smem > kMaxSmem)
            return fail(msg, VP_ERR_UNSUPPORTED,
                        "the cyclic x solve keeps a row in shared memory: nx = %d is too large",
                        grid->nx);
    }
    P->tx = tx;
    P->tp = tp;
    P->ntx = (grid->nx + tx - 1) / tx;
    if (P->xpass && xrow_smem_bytes(opts->precision, grid->nx, P->ntx) > kMaxSmem)
        return fail(msg, VP_ERR_UNSUPPORTED, "the x-solve row pass needs %zu bytes of shared memory",
                    xrow_smem_bytes(opts->precision, grid->nx, P->ntx));
    P->xgrid = P->xpass ? xrow_grid_size(opts->precision, grid->nx, grid->np, P->ntx) : 0;
    P->ntp = (grid->np + tp - 1) / tp;
    P->hist_cap = opts->history_cap ? opts->history_cap : kDefaultHist;
    P->nlost = (kernel == VP_KERNEL_TILED || kernel == VP_KERNEL_FUSED) ? P->ntx * P->ntp : 1;
    P->npart = std::max(std::max(filter_p_blocks(grid->nx, grid->np), P->ntx * P->ntp),
                        fel_partial_blocks(grid->nx, grid->np));
    P->nmblk = moment_blocks(grid->nx, grid->np);
    P->nblk = (grid->nx + kColBlock - 1) / kColBlock;

    const size_t N = (size_t)grid->nx * grid->np;
    const size_t colsz = sz == 8 ? sizeof(ColEntry<double>) : sizeof(ColEntry<float>);
    const size_t rowsz = sz == 8 ? sizeof(RowEntry<double>) : sizeof(RowEntry<float>);
    Layout &L = P->L;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes);
        return o;
    };
    L.f0 = take(N * sz);
    L.f1 = take(N * sz);
    // a third mesh-sized buffer only where a step needs one: the deposit between the two launches of
    // the separate-x-pass plan, the x-solve output of the separate-filter path. The one-pass plan
    // reads its weights out through the idle ping-pong buffer instead
    L.tmp = take(((P->galerkin && (kernel != VP_KERNEL_FUSED || P->xpass)) || P->septic_gal) ? N * sz : 0);
    L.col = take(grid->nx * colsz);
    L.row = take(grid->np * rowsz);
    L.rowb = take(grid->np * sizeof(RowBound));
    L.vcb = take(P->nblk * 2 * sizeof(double));
    L.rowbf = take(grid->np * sizeof(float4));
    L.vcbf = take(P->nblk * sizeof(float2));
    L.csx = take(grid->nx * sizeof(double2));
    L.ucol = take(grid->nx * sizeof(double));
    L.vcol = take(grid->nx * sizeof(double));
    L.piv = take(kPivTable * sizeof(double));
    L.ldl = take(P->septic_gal ? (size_t)(kLdlRows + 1) * 4 * sizeof(double) : 0);
    L.sigma = take(grid->np * sizeof(double));
    // FP32 one-pass plans: max|s| per tile of each state buffer (the fixed-point window scale)
    L.smax = take(kernel == VP_KERNEL_FUSED && sz == 4 ? 2 * (size_t)P->ntx * P->ntp * sizeof(float) : 0);
    // FEL space charge: half-drift row factors (cos, sin) for the stored state
    L.rtil = take(P->fel && !P->rk4 && g.sigma2 != 0.0 ? 2 * (size_t)grid->np * sizeof(double) : 0);
    // one-pass plans of a push fixed for the whole run: each tile's source rectangle
    L.tsrc = take(kernel == VP_KERNEL_FUSED && !P->fel ? (size_t)P->ntx * P->ntp * sizeof(int4) : 0);
    L.state = take(ST_NSTATE * sizeof(double));
    L.hist = take((size_t)P->hist_cap * 2 * sizeof(double));
    L.lost = take(P->nlost * sizeof(double));
    L.part = take((size_t)P->npart * 3 * sizeof(double));
    L.mpart = take((size_t)P->nmblk * kNumMoments * sizeof(double));
    L.mout = take(kMoutLen * sizeof(double));
    L.err = take(sizeof(unsigned));
    L.ticket = take(kernel == VP_KERNEL_FUSED ? sizeof(int) : 0);
    L.total = off;
    return VP_OK;
}

}  // namespace

struct vp_sim {
    Plan P;
    cudaStream_t stream;
    char *ws;
    int cur;
    bool f_set;
    double a0_re, a0_im;
    double host_state[ST_NSTATE];
    double host_mout[kMoutLen];
    unsigned host_err;
    char msg[512];

    template <typename T>
    T *ptr(size_t off) const { return reinterpret_cast<T *>(ws + off); }
    void *f(int k) const { return ws + (k == 0 ? P.L.f0 : P.L.f1); }
};

namespace {

vp_status cuda_fail(vp_sim *s, cudaError_t e, const char *what)
{
    return fail(s ? s->msg : nullptr, VP_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define VP_CUDA(sim, ...)                                              \
    do {                                                               \
        cudaError_t e_ = (__VA_ARGS__);                                \
        if (e_ != cudaSuccess) return cuda_fail(sim, e_, #__VA_ARGS__); \
    } while (0)

// FP32 scale applied after the Lambda_x recursions. In exact arithmetic the x recursions
// times -6z and the p recursions with the limit pivots each leave a constant field unchanged.
// With the FP32 pole and pivots a step of the two would scale it by about 1 - 7e-8, and such
// a bias compounds from step to step into a mass drift (about 1.4e-4 after 2000 steps), far
// above the rounding noise. So the scale is (1 - z)^2 / g_p, z the FP32 pole and g_p the DC
// gain of the p recursion with the FP32 constants as the kernel forms them (ib6: the rounded
// product (1/6) ib of the one-pass kernel, else the exact product), kept as hi + lo floats.
void unit_gain_scale(double ib, double cp, bool rounded_ib6, double *hi, double *lo)
{
    const float zf = (float)-0.26794919243112270647;
    const float ibf = (float)ib, cpf = (float)cp;
    const float sixth = 1.0f / 6.0f;
    const float ib6f = sixth * ibf;
    const double ib6 = rounded_ib6 ? (double)ib6f : (double)sixth * (double)ibf;
    const double gp = (double)ibf / ((1.0 + ib6) * (1.0 + (double)cpf));
    const double c = (1.0 - (double)zf) * (1.0 - (double)zf) / gp;
    const float h = (float)c;
    *hi = (double)h;
    *lo = (double)(float)(c - (double)h);
}

template <typename T>
StepArgs<T> step_args(vp_sim *s, const void *src, void *dst)
{
    const Plan &P = s->P;
    StepArgs<T> a;
    a.src = static_cast<const T *>(src);
    a.dst = static_cast<T *>(dst);
    a.col = s->ptr<ColEntry<T>>(P.L.col);
    a.row = s->ptr<RowEntry<T>>(P.L.row);
    a.rowb = s->ptr<RowBound>(P.L.rowb);
    a.vcb = s->ptr<double>(P.L.vcb);
    a.state = s->ptr<double>(P.L.state);
    a.csx = s->ptr<double2>(P.L.csx);
    a.tile_lost = s->ptr<double>(P.L.lost);
    a.tile_part = s->ptr<double>(P.L.part);
    a.err = s->ptr<unsigned>(P.L.err);
    a.g = P.g;
    a.tx = P.tx;
    a.tp = P.tp;
    a.ntx = P.ntx;
    a.ntp = P.ntp;
    a.fel_partials = (P.fel && !P.galerkin && P.kernel == VP_KERNEL_TILED) ? 1 : 0;
    return a;
}

template <typename T>
FusedArgs<T> fused_args(vp_sim *s, const void *src, void *dst)
{
    const Plan &P = s->P;
    FusedArgs<T> a;
    a.src = static_cast<const T *>(src);
    a.dst = static_cast<T *>(dst);
    a.col = s->ptr<ColEntry<T>>(P.L.col);
    a.row = s->ptr<RowEntry<T>>(P.L.row);
    a.rowb = s->ptr<RowBound>(P.L.rowb);
    a.vcb = s->ptr<double>(P.L.vcb);
    a.rowbf = s->ptr<float4>(P.L.rowbf);
    a.vcbf = s->ptr<float2>(P.L.vcbf);
    a.state = s->ptr<double>(P.L.state);
    a.piv = s->ptr<double>(P.L.piv);
    a.sigma = s->ptr<double>(P.L.sigma);
    {
        float *m0 = s->ptr<float>(P.L.smax), *m1 = m0 + (size_t)P.ntx * P.ntp;
        const bool from0 = src == s->f(0);
        a.smax_in = from0 ? m0 : m1;
        a.smax_out = from0 ? m1 : m0;
    }
    a.tile_src = P.fel ? nullptr : s->ptr<int4>(P.L.tsrc);
    a.csx = s->ptr<double2>(P.L.csx);
    a.tile_lost = s->ptr<double>(P.L.lost);
    a.tile_part = s->ptr<double>(P.L.part);
    a.err = s->ptr<unsigned>(P.L.err);
    a.g = P.g;
    a.tx = P.tx;
    a.tp = P.tp;
    a.ntx = P.ntx;
    a.ntp = P.ntp;
    a.G = P.G;
    a.Gp = P.Gp;
    a.ws = P.ws;
    a.full_row = P.full_row ? 1 : 0;
    a.fel_partials = P.fel ? 1 : 0;
    a.ticket = s->ptr<int>(P.L.ticket);
    a.hist = s->ptr<double>(P.L.hist);
    a.hist_cap = P.hist_cap;
    a.rowcache = P.rowcache;
    a.xpass = P.xpass ? 1 : 0;
    a.bunch_x = P.xpass && P.fel ? 1.0 / (2.0 / 3.0 + cos(P.g.hx) / 3.0) : 1.0;
    return a;
}

// the weights w of the current state: the state itself, or Lambda_p^{-1} s into out, else into the
// idle ping-pong buffer (the next step's output: it overwrites them)
template <typename T>
vp_status weights_of_state(vp_sim *s, const void **w, void *out = nullptr)
{
    const Plan &P = s->P;
    if (!P.state_s) {
        *w = s->f(s->cur);
        return VP_OK;
    }
    T *tmp = out ? static_cast<T *>(out) : static_cast<T *>(s->f(1 - s->cur));
    VP_CUDA(s, launch_filter_p<T>(static_cast<const T *>(s->f(s->cur)), tmp, P.g.nx, P.g.np,
                                  s->ptr<double>(P.L.piv), s->ptr<double2>(P.L.csx),
                                  s->ptr<double>(P.L.part), 0, s->ptr<unsigned>(P.L.err), s->stream));
    *w = tmp;
    return VP_OK;
}

template <typename T>
vp_status fel_bunching(vp_sim *s, const void *w, int init)
{
    const Plan &P = s->P;
    double *part = s->ptr<double>(P.L.part);
    VP_CUDA(s, launch_fel_partials<T>(static_cast<const T *>(w), P.g.nx, P.g.np,
                                      s->ptr<double2>(P.L.csx), part, s->stream));
    VP_CUDA(s, launch_fel_finalize(part, fel_partial_blocks(P.g.nx, P.g.np), s->ptr<double>(P.L.state),
                                   s->ptr<double>(P.L.hist), P.hist_cap, P.g.dt, init, s->stream));
    return VP_OK;
}

// FEL space charge: K = A^{n+1/2} + i sigma2 <e^{-i theta~}> over the stored state st
template <typename T>
vp_status fel_space_charge(vp_sim *s, const void *st)
{
    const Plan &P = s->P;
    const double *rt = s->ptr<double>(P.L.rtil);
    double *part = s->ptr<double>(P.L.part);
    VP_CUDA(s, launch_fel_tilde<T>(static_cast<const T *>(st), P.g.nx, P.g.np, s->ptr<double2>(P.L.csx),
                                   rt, rt + P.g.np, P.state_s ? s->ptr<double>(P.L.sigma) : nullptr, part,
                                   s->stream));
    VP_CUDA(s, launch_fel_kick(part, fel_partial_blocks(P.g.nx, P.g.np), s->ptr<double>(P.L.state),
                               P.g.sigma2, s->stream));
    return VP_OK;
}

// ev (optional): VP_NPHASES + 1 events per step, recorded at the phase boundaries
template <typename T>
vp_status do_steps(vp_sim *s, int n, cudaEvent_t *ev = nullptr)
{
    const Plan &P = s->P;
    const size_t N = (size_t)P.g.nx * P.g.np;
    double *part = s->ptr<double>(P.L.part);
    double *state = s->ptr<double>(P.L.state);
    unsigned *err = s->ptr<unsigned>(P.L.err);
    for (int k = 0; k < n; ++k) {
        cudaEvent_t *e = ev ? ev + (size_t)k * (VP_NPHASES + 1) : nullptr;
        if (e) VP_CUDA(s, cudaEventRecord(e[0], s->stream));
        void *src = s->f(s->cur), *dst = s->f(1 - s->cur);
        StepArgs<T> a = step_args<T>(s, src, dst);
        if (P.kernel == VP_KERNEL_FUSED) {
            // separate x pass: the tiles store the deposit into tmp, the row pass solves it into dst
            void *tile_dst = P.xpass ? static_cast<void *>(s->ptr<T>(P.L.tmp)) : dst;
            VP_CUDA(s, launch_step_fused<T>(fused_args<T>(s, src, tile_dst), P.threads, s->stream));
        } else if (P.kernel == VP_KERNEL_TILED) {
            VP_CUDA(s, launch_step_tiled<T>(a, s->stream));
        } else {
            VP_CUDA(s, cudaMemsetAsync(dst, 0, N * sizeof(T), s->stream));
            if (P.rk4) {
                VP_CUDA(s, launch_rk4_stages<T>(static_cast<const T *>(src), P.g, s->ptr<double2>(P.L.csx),
                                                state, part, s->stream));
                VP_CUDA(s, launch_rk4_deposit<T>(static_cast<const T *>(src), static_cast<T *>(dst), P.g,
                                                 s->ptr<double2>(P.L.csx), state, s->ptr<double>(P.L.lost),
                                                 s->stream));
            } else {
                VP_CUDA(s, launch_step_scatter<T>(a, s->ptr<double>(P.L.lost), s->stream));
            }
        }
        if (e) VP_CUDA(s, cudaEventRecord(e[1], s->stream));
        int nparts = 0;
        if (P.kernel == VP_KERNEL_FUSED) {
            nparts = P.ntx * P.ntp;
            if (P.xpass) {
                float *m0 = s->ptr<float>(P.L.smax);
                float *mout = P.precision == VP_FP32 ? (src == s->f(0) ? m0 + (size_t)P.ntx * P.ntp : m0) : nullptr;
                VP_CUDA(s, launch_xsolve_rows<T>(s->ptr<T>(P.L.tmp), static_cast<T *>(dst), P.g.nx, P.g.np,
                                                 s->ptr<double>(P.L.piv), P.tx, P.tp, P.ntx, mout, err,
                                                 P.xgrid, s->stream));
                if (e) {
                    VP_CUDA(s, cudaEventRecord(e[2], s->stream));
                    VP_CUDA(s, cudaEventRecord(e[3], s->stream));
                }
            }
        } else if (P.galerkin) {
            T *tmp = s->ptr<T>(P.L.tmp);
            VP_CUDA(s, launch_filter_x<T>(static_cast<const T *>(dst), tmp, P.g.nx, P.g.np,
                                          s->ptr<double>(P.L.piv), err, s->stream));
            if (e) VP_CUDA(s, cudaEventRecord(e[2], s->stream));
            VP_CUDA(s, launch_filter_p<T>(tmp, static_cast<T *>(dst), P.g.nx, P.g.np,
                                          s->ptr<double>(P.L.piv), s->ptr<double2>(P.L.csx), part,
                                          P.fel ? 1 : 0, err, s->stream));
            if (e) VP_CUDA(s, cudaEventRecord(e[3], s->stream));
            nparts = filter_p_blocks(P.g.nx, P.g.np);
        } else if (P.septic_gal) {
            T *tmp = s->ptr<T>(P.L.tmp);
            const double sh = P.precision == VP_FP32 ? (double)(float)P.x7_scale : P.x7_scale;
            VP_CUDA(s, launch_filter_x7<T>(static_cast<const T *>(dst), tmp, P.g.nx, P.g.np, sh,
                                           P.x7_scale - sh, s->stream));
            if (e) VP_CUDA(s, cudaEventRecord(e[2], s->stream));
            VP_CUDA(s, launch_filter_p7<T>(tmp, static_cast<T *>(dst), P.g.nx, P.g.np, s->ptr<double>(P.L.ldl),
                                           s->stream));
            if (e) VP_CUDA(s, cudaEventRecord(e[3], s->stream));
            if (P.fel) {
                VP_CUDA(s, launch_fel_partials<T>(static_cast<const T *>(dst), P.g.nx, P.g.np,
                                                  s->ptr<double2>(P.L.csx), part, s->stream));
                nparts = fel_partial_blocks(P.g.nx, P.g.np);
            }
        } else if (P.fel) {
            if (P.kernel == VP_KERNEL_TILED) {
                nparts = P.ntx * P.ntp;
            } else {
                VP_CUDA(s, launch_fel_partials<T>(static_cast<const T *>(dst), P.g.nx, P.g.np,
                                                  s->ptr<double2>(P.L.csx), part, s->stream));
                nparts = fel_partial_blocks(P.g.nx, P.g.np);
            }
        }
        if (e && ((!P.galerkin && !P.septic_gal) || (P.kernel == VP_KERNEL_FUSED && !P.xpass))) {
            VP_CUDA(s, cudaEventRecord(e[2], s->stream));
            VP_CUDA(s, cudaEventRecord(e[3], s->stream));
        }
        // the one-pass kernel finishes the step itself (its last CTA: field update or step count)
        if (P.fel) {
            if (P.kernel != VP_KERNEL_FUSED)
                VP_CUDA(s, launch_fel_finalize(part, nparts, state, s->ptr<double>(P.L.hist), P.hist_cap,
                                               P.g.dt, 0, s->stream, P.rk4 ? 1 : 0));
            if (P.g.sigma2 != 0.0 && !P.rk4) {
                const vp_status sc = fel_space_charge<T>(s, dst);
                if (sc != VP_OK) return sc;
            }
        } else if (P.kernel != VP_KERNEL_FUSED) {
            VP_CUDA(s, launch_count_step(state, P.g.dt, s->stream));
        }
        if (e) VP_CUDA(s, cudaEventRecord(e[4], s->stream));
        s->cur = 1 - s->cur;
    }
    return VP_OK;
}

// the initial state block, written by a kernel from its argument (no host buffer to keep alive, so
// nothing here waits for the stream)
struct StateBlock {
    double v[ST_NSTATE];
};
__global__ void put_state_kernel(double *dst, StateBlock b)
{
    for (int k = threadIdx.x; k < ST_NSTATE; k += blockDim.x) dst[k] = b.v[k];
}

vp_status reset_state(vp_sim *s, const void *w)
{
    const Plan &P = s->P;
    StateBlock b;
    memset(&b, 0, sizeof(b));
    b.v[ST_A_RE] = s->a0_re;
    b.v[ST_A_IM] = s->a0_im;
    put_state_kernel<<<1, 32, 0, s->stream>>>(s->ptr<double>(P.L.state), b);
    VP_CUDA(s, cudaGetLastError());
    VP_CUDA(s, cudaMemsetAsync(s->ws + P.L.lost, 0, P.nlost * sizeof(double), s->stream));
    VP_CUDA(s, cudaMemsetAsync(s->ws + P.L.err, 0, sizeof(unsigned), s->stream));
    if (P.kernel == VP_KERNEL_FUSED) VP_CUDA(s, cudaMemsetAsync(s->ws + P.L.ticket, 0, sizeof(int), s->stream));
    VP_CUDA(s, cudaMemsetAsync(s->ws + P.L.hist, 0, (size_t)P.hist_cap * 2 * sizeof(double), s->stream));
    if (P.fel) {
        vp_status st = P.precision == VP_FP64 ? fel_bunching<double>(s, w, 1)
                                              : fel_bunching<float>(s, w, 1);
        if (st != VP_OK) return st;
    }
    return VP_OK;
}

vp_status check_flags(vp_sim *s)
{
    VP_CUDA(s, cudaMemcpyAsync(&s->host_err, s->ws + s->P.L.err, sizeof(unsigned),
                               cudaMemcpyDeviceToHost, s->stream));
    VP_CUDA(s, cudaStreamSynchronize(s->stream));
    if (s->host_err & ERRF_NONFINITE)
        return fail(s->msg, VP_ERR_NONFINITE, "a step produced a non-finite weight");
    if (s->host_err & ERRF_TIMEOUT)
        return fail(s->msg, VP_ERR_TIMEOUT, "a bounded device wait gave up");
    return VP_OK;
}

}  // namespace

extern "C" {

const char *vp_status_string(vp_status st)
{
    switch (st) {
    case VP_OK: return "ok";
    case VP_ERR_ARG: return "invalid argument";
    case VP_ERR_CUDA: return "CUDA error";
    case VP_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    case VP_ERR_NONFINITE: return "non-finite weight";
    case VP_ERR_TIMEOUT: return "device wait timed out";
    case VP_ERR_STATE: return "call out of order";
    case VP_ERR_UNSUPPORTED: return "unsupported size or option";
    case VP_ERR_CANCELLED: return "cancelled";
    }
    return "unknown status";
}

vp_status vp_workspace_size(const vp_grid *grid, int32_t basis, const vp_pusher *pusher,
                            const vp_opts *opts, size_t *bytes)
{
    if (!bytes) return VP_ERR_ARG;
    Plan P;
    vp_status st = make_plan(grid, basis, pusher, opts, &P, nullptr);
    if (st != VP_OK) return st;
    *bytes = P.L.total;
    return VP_OK;
}

vp_status vp_create(const vp_grid *grid, int32_t basis, const vp_pusher *pusher,
                    const vp_opts *opts, void *workspace, size_t workspace_bytes, vp_sim **out)
{
    if (!out) return VP_ERR_ARG;
    *out = nullptr;
    vp_sim *s = new (std::nothrow) vp_sim();
    if (!s) return VP_ERR_ARG;
    vp_status st = make_plan(grid, basis, pusher, opts, &s->P, s->msg);
    if (st != VP_OK) {
        delete s;
        return st;
    }
    const Plan &P = s->P;
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) % kAlign) != 0 ||
        workspace_bytes < P.L.total) {
        delete s;
        return VP_ERR_WORKSPACE;
    }
    s->ws = static_cast<char *>(workspace);
    s->stream = static_cast<cudaStream_t>(opts->stream);
    s->cur = 0;
    s->f_set = false;
    s->a0_re = s->P.fel ? pusher->a0_re : 0.0;
    s->a0_im = s->P.fel ? pusher->a0_im : 0.0;

    Geometry &g = s->P.g;
    auto cleanup = [&](vp_status code) {
        if (code != VP_OK) delete s;
        return code;
    };
    cudaError_t e = build_tables(g, P.precision, s->ws + P.L.col, s->ws + P.L.row,
                                 s->ptr<RowBound>(P.L.rowb), s->ptr<double>(P.L.ucol),
                                 s->ptr<double>(P.L.vcol), s->ptr<double2>(P.L.csx), s->stream);
    if (e != cudaSuccess) return cleanup(cuda_fail(nullptr, e, "build_tables"));
    std::vector<double> ucol(g.nx), vcol(g.nx);
    std::vector<RowBound> rowb(g.np);
    e = cudaMemcpyAsync(ucol.data(), s->ws + P.L.ucol, g.nx * sizeof(double), cudaMemcpyDeviceToHost,
                        s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(vcol.data(), s->ws + P.L.vcol, g.nx * sizeof(double),
                            cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(rowb.data(), s->ws + P.L.rowb, g.np * sizeof(RowBound),
                            cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cleanup(cuda_fail(nullptr, e, "table readback"));

    g.uc_min = *std::min_element(ucol.begin(), ucol.end());
    g.uc_max = *std::max_element(ucol.begin(), ucol.end());
    g.vc_min = *std::min_element(vcol.begin(), vcol.end());
    g.vc_max = *std::max_element(vcol.begin(), vcol.end());
    g.vr_min = 1e300;
    g.vr_max = -1e300;
    for (const RowBound &b : rowb) {
        g.vr_min = std::min(g.vr_min, b.v);
        g.vr_max = std::max(g.vr_max, b.v);
    }
    std::vector<double> vcb(2 * P.nblk);
    for (int b = 0; b < P.nblk; ++b) {
        double lo = 1e300, hi = -1e300;
        for (int i = b * kColBlock; i < std::min(g.nx, (b + 1) * kColBlock); ++i) {
            lo = std::min(lo, vcol[i]);
            hi = std::max(hi, vcol[i]);
        }
        vcb[2 * b] = lo;
        vcb[2 * b + 1] = hi;
    }
    // Thomas pivots of tridiag(1/6, 2/3, 1/6) from the first row, and their limits
    // septic basis: LDL^T factor rows of the principal block of P7 (exact for the first kLdlRows
    // rows, then the limit), and the x scale prod (1 - z_i)^2 with the poles as the kernel holds
    // them, which makes the recursions' DC gain one
    std::vector<double> ldl;
    if (P.septic_gal) {
        const double bb[4] = {2416.0 / 5040.0, 1191.0 / 5040.0, 120.0 / 5040.0, 1.0 / 5040.0};
        ldl.assign((size_t)(kLdlRows + 1) * 4, 0.0);
        auto D = [&](int r) -> double & { return ldl[(size_t)r * 4]; };
        auto Lm = [&](int r, int m) -> double & { return ldl[(size_t)r * 4 + m]; };   // L_{r+m, r}
        for (int jr = 0; jr <= kLdlRows; ++jr) {
            double d = bb[0];
            for (int k = 1; k <= 3 && jr - k >= 0; ++k) d -= Lm(jr - k, k) * Lm(jr - k, k) * D(jr - k);
            D(jr) = d;
            for (int m = 1; m <= 3; ++m) {
                double v = bb[m];
                for (int k = 1; k + m <= 3 && jr - k >= 0; ++k) v -= Lm(jr - k, m + k) * Lm(jr - k, k) * D(jr - k);
                Lm(jr, m) = v / d;
            }
        }
        double sc = 1.0;
        for (int q = 0; q < 3; ++q) {
            const double zq = P.precision == VP_FP32 ? (double)(float)septic_pole(q) : septic_pole(q);
            sc *= (1.0 - zq) * (1.0 - zq);
        }
        s->P.x7_scale = sc;
    }
    std::vector<double> piv(kPivTable, 0.0);
    double cprev = 0.0;
    for (int r = 0; r < kPivots; ++r) {
        const double beta = 2.0 / 3.0 - (r == 0 ? 0.0 : cprev / 6.0);
        piv[2 * r] = (1.0 / 6.0) / beta;
        piv[2 * r + 1] = 1.0 / beta;
        cprev = piv[2 * r];
    }
    const double beta_inf = 1.0 / 3.0 + 1.0 / (2.0 * sqrt(3.0));
    piv[2 * kPivots] = (1.0 / 6.0) / beta_inf;
    piv[2 * kPivots + 1] = 1.0 / beta_inf;
    unit_gain_scale(piv[2 * kPivots + 1], piv[2 * kPivots], true, &piv[kPivXsFused],
                    &piv[kPivXsFused + 1]);
    unit_gain_scale(piv[2 * kPivots + 1], piv[2 * kPivots], false, &piv[kPivXsFilter],
                    &piv[kPivXsFilter + 1]);
    // sigma = column sums of Lambda_p^{-1} (np x np tridiag(1/6, 2/3, 1/6), symmetric):
    // the Thomas solve of T sigma = 1
    std::vector<double> sigma(g.np, 1.0), cpv(g.np);
    {
        double beta = 2.0 / 3.0;
        cpv[0] = (1.0 / 6.0) / beta;
        sigma[0] = sigma[0] / beta;
        for (int j = 1; j < g.np; ++j) {
            beta = 2.0 / 3.0 - (1.0 / 6.0) * cpv[j - 1];
            cpv[j] = (1.0 / 6.0) / beta;
            sigma[j] = (sigma[j] - (1.0 / 6.0) * sigma[j - 1]) / beta;
        }
        for (int j = g.np - 2; j >= 0; --j) sigma[j] -= cpv[j] * sigma[j + 1];
    }
    // FEL space charge: cos and sin of the half drift h/2 (delta + p_j), times Lambda_p^{-1}
    // (symmetric) when the stored state is s = Lambda_p w, so that sum_j w_ij f_j = sum_j s_ij rf_j
    std::vector<double> rtil;
    if (P.fel && !P.rk4 && g.sigma2 != 0.0) {
        rtil.resize(2 * (size_t)g.np);
        for (int j = 0; j < g.np; ++j) {
            const double ph = 0.5 * g.dt * (g.delta + g.p0 + j * g.hp);
            rtil[j] = cos(ph);
            rtil[g.np + j] = sin(ph);
        }
        if (P.state_s)
            for (int q = 0; q < 2; ++q) {
                double *v = rtil.data() + (size_t)q * g.np;
                double beta = 2.0 / 3.0;
                v[0] /= beta;
                for (int j = 1; j < g.np; ++j) {
                    beta = 2.0 / 3.0 - (1.0 / 6.0) * cpv[j - 1];
                    v[j] = (v[j] - (1.0 / 6.0) * v[j - 1]) / beta;
                }
                for (int j = g.np - 2; j >= 0; --j) v[j] -= cpv[j] * v[j + 1];
            }
    }
    // FP32 copies of the bound tables for the one-pass kernel's tile bounds
    std::vector<float4> rowbf(g.np);
    for (int j = 0; j < g.np; ++j)
        rowbf[j] = make_float4((float)rowb[j].u, (float)rowb[j].v, (float)rowb[j].y, 0.f);
    std::vector<float2> vcbf(P.nblk);
    for (int b = 0; b < P.nblk; ++b) vcbf[b] = make_float2((float)vcb[2 * b], (float)vcb[2 * b + 1]);
    e = cudaMemcpyAsync(s->ws + P.L.rowbf, rowbf.data(), rowbf.size() * sizeof(float4),
                        cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->ws + P.L.vcbf, vcbf.data(), vcbf.size() * sizeof(float2),
                            cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cleanup(cuda_fail(nullptr, e, "bound table upload"));
    if (!rtil.empty()) {
        e = cudaMemcpyAsync(s->ws + P.L.rtil, rtil.data(), rtil.size() * sizeof(double),
                            cudaMemcpyHostToDevice, s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) return cleanup(cuda_fail(nullptr, e, "space-charge table upload"));
    }
    if (!ldl.empty()) {
        e = cudaMemcpyAsync(s->ws + P.L.ldl, ldl.data(), ldl.size() * sizeof(double),
                            cudaMemcpyHostToDevice, s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) return cleanup(cuda_fail(nullptr, e, "septic factor upload"));
    }
    e = cudaMemcpyAsync(s->ws + P.L.sigma, sigma.data(), sigma.size() * sizeof(double),
                        cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cleanup(cuda_fail(nullptr, e, "sigma upload"));
    e = cudaMemcpyAsync(s->ws + P.L.vcb, vcb.data(), vcb.size() * sizeof(double),
                        cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->ws + P.L.piv, piv.data(), piv.size() * sizeof(double),
                            cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->ws + P.L.err, 0, sizeof(unsigned), s->stream);
    if (e == cudaSuccess && P.kernel == VP_KERNEL_FUSED)
        e = cudaMemsetAsync(s->ws + P.L.ticket, 0, sizeof(int), s->stream);
    // tile source rectangles not computed yet (each entry 0x80808080 = kTileSrcUnset)
    if (e == cudaSuccess && P.kernel == VP_KERNEL_FUSED && !P.fel)
        e = cudaMemsetAsync(s->ws + P.L.tsrc, 0x80, (size_t)P.ntx * P.ntp * sizeof(int4), s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cleanup(cuda_fail(nullptr, e, "table upload"));
    *out = s;
    return VP_OK;
}

// Device address of a host buffer that kernels can read and write in place (pinned or
// registered host memory; on Grace-Blackwell the chip-to-chip link is coherent), else nullptr.
// Transfers through it run at the link's rate like a copy, and fuse the copy with the solve
// that precedes or follows it.
static void *host_device_ptr(const void *p, size_t align)
{
    if ((uintptr_t)p % align) return nullptr;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

enum class Xfer { host, device, host_async };

static vp_status set_f_common(vp_sim *s, const void *src, int32_t dtype, size_t n, Xfer mode)
{
    const bool device = mode == Xfer::device, async = mode == Xfer::host_async;
    if (!s) return VP_ERR_ARG;
    const Plan &P = s->P;
    const size_t N = (size_t)P.g.nx * P.g.np;
    if (!src || n != N || (dtype != VP_FP32 && dtype != VP_FP64))
        return fail(s->msg, VP_ERR_ARG, "set_f: need %zu values of dtype FP32/FP64", N);
    s->cur = 0;
    // the weights go to the state buffer, or to the idle buffer f1 when the state is s = Lambda_p w
    void *dst = P.state_s ? s->f(1) : s->f(0);
    const size_t szs = P.precision == VP_FP64 ? 8 : 4;
    if (async && dtype != P.precision)
        return fail(s->msg, VP_ERR_ARG, "set_f_async: the weights must have the simulation's dtype");
    // pinned host weights and the state s = Lambda_p w: Lambda_p reads them in place (the
    // asynchronous call copies them with the copy engine instead, which overlaps other streams'
    // transfers in the opposite direction)
    void *hdev = (!device && !async && dtype == P.precision && P.state_s) ? host_device_ptr(src, szs) : nullptr;
    if (hdev) {
        dst = hdev;
    } else if (dtype == P.precision) {
        VP_CUDA(s, cudaMemcpyAsync(dst, src, N * szs,
                                   device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                   s->stream));
    } else if (device) {
        if (dtype == VP_FP64)
            VP_CUDA(s, launch_convert<double, float>(static_cast<const double *>(src),
                                                     static_cast<float *>(dst), N, s->stream));
        else
            VP_CUDA(s, launch_convert<float, double>(static_cast<const float *>(src),
                                                     static_cast<double *>(dst), N, s->stream));
    } else {
        std::vector<char> tmp(N * szs);
        if (dtype == VP_FP64) {
            const double *in = static_cast<const double *>(src);
            float *o = reinterpret_cast<float *>(tmp.data());
            for (size_t k = 0; k < N; ++k) o[k] = (float)in[k];
        } else {
            const float *in = static_cast<const float *>(src);
            double *o = reinterpret_cast<double *>(tmp.data());
            for (size_t k = 0; k < N; ++k) o[k] = (double)in[k];
        }
        VP_CUDA(s, cudaMemcpyAsync(dst, tmp.data(), N * szs, cudaMemcpyHostToDevice, s->stream));
        VP_CUDA(s, cudaStreamSynchronize(s->stream));
    }
    s->f_set = true;
    vp_status st = reset_state(s, dst);
    if (st != VP_OK) return st;
    if (P.state_s) {
        if (P.precision == VP_FP64)
            VP_CUDA(s, launch_lambda_p_mul<double>(static_cast<const double *>(dst),
                                                   static_cast<double *>(s->f(0)), P.g.nx, P.g.np,
                                                   s->stream));
        else
            VP_CUDA(s, launch_lambda_p_mul<float>(static_cast<const float *>(dst),
                                                  static_cast<float *>(s->f(0)), P.g.nx, P.g.np,
                                                  s->stream));
    }
    if (P.fel && !P.rk4 && P.g.sigma2 != 0.0) {
        const vp_status sc = P.precision == VP_FP64 ? fel_space_charge<double>(s, s->f(0))
                                                    : fel_space_charge<float>(s, s->f(0));
        if (sc != VP_OK) return sc;
    }
    if (P.kernel == VP_KERNEL_FUSED && P.precision == VP_FP32)
        VP_CUDA(s, launch_tile_max(static_cast<const float *>(s->f(0)), s->ptr<float>(P.L.smax), P.g.nx,
                                   P.g.np, P.tx, P.tp, P.ntx, P.ntp, s->ptr<unsigned>(P.L.err),
                                   s->stream));
    // the caller owns the host buffer again once vp_set_f returns; the asynchronous form leaves it
    // to the caller's vp_sync
    if (mode == Xfer::host) VP_CUDA(s, cudaStreamSynchronize(s->stream));
    return VP_OK;
}

vp_status vp_set_f(vp_sim *s, const void *host, int32_t dtype, size_t n)
{
    return set_f_common(s, host, dtype, n, Xfer::host);
}

vp_status vp_set_f_async(vp_sim *s, const void *host, int32_t dtype, size_t n)
{
    return set_f_common(s, host, dtype, n, Xfer::host_async);
}

vp_status vp_set_f_device(vp_sim *s, const void *dev, int32_t dtype, size_t n)
{
    return set_f_common(s, dev, dtype, n, Xfer::device);
}

vp_status vp_step(vp_sim *s, int32_t n)
{
    if (!s) return VP_ERR_ARG;
    if (n < 0) return fail(s->msg, VP_ERR_ARG, "negative step count");
    if (!s->f_set) return fail(s->msg, VP_ERR_STATE, "vp_step before vp_set_f");
    return s->P.precision == VP_FP64 ? do_steps<double>(s, n) : do_steps<float>(s, n);
}

vp_status vp_step_profiled(vp_sim *s, int32_t n, double *phase_ms, int32_t nphases)
{
    if (!s) return VP_ERR_ARG;
    if (n < 0 || n > 4096 || !phase_ms || nphases < 1 || nphases > VP_NPHASES)
        return fail(s->msg, VP_ERR_ARG, "vp_step_profiled: 0 <= n <= 4096, 1 <= nphases <= %d",
                    VP_NPHASES);
    if (!s->f_set) return fail(s->msg, VP_ERR_STATE, "vp_step before vp_set_f");
    const size_t ne = (size_t)n * (VP_NPHASES + 1);
    std::vector<cudaEvent_t> ev(ne, nullptr);
    vp_status st = VP_OK;
    for (size_t k = 0; k < ne && st == VP_OK; ++k) {
        cudaError_t e = cudaEventCreate(&ev[k]);
        if (e != cudaSuccess) st = cuda_fail(s, e, "cudaEventCreate");
    }
    if (st == VP_OK)
        st = s->P.precision == VP_FP64 ? do_steps<double>(s, n, ev.data()) : do_steps<float>(s, n, ev.data());
    if (st == VP_OK) {
        cudaError_t e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) st = cuda_fail(s, e, "cudaStreamSynchronize");
    }
    for (int q = 0; q < nphases; ++q) phase_ms[q] = 0.0;
    for (int k = 0; k < n && st == VP_OK; ++k)
        for (int q = 0; q < nphases; ++q) {
            float ms = 0.f;
            cudaError_t e = cudaEventElapsedTime(&ms, ev[(size_t)k * (VP_NPHASES + 1) + q],
                                                 ev[(size_t)k * (VP_NPHASES + 1) + q + 1]);
            if (e != cudaSuccess) {
                st = cuda_fail(s, e, "cudaEventElapsedTime");
                break;
            }
            phase_ms[q] += ms;
        }
    for (cudaEvent_t e : ev)
        if (e) cudaEventDestroy(e);
    return st;
}

static vp_status get_f_common(vp_sim *s, void *dstp, int32_t dtype, size_t n, Xfer mode)
{
    const bool device = mode == Xfer::device, async = mode == Xfer::host_async;
    if (!s) return VP_ERR_ARG;
    const Plan &P = s->P;
    const size_t N = (size_t)P.g.nx * P.g.np;
    if (!dstp || n != N || (dtype != VP_FP32 && dtype != VP_FP64))
        return fail(s->msg, VP_ERR_ARG, "get_f: need room for %zu values of dtype FP32/FP64", N);
    if (!s->f_set) return fail(s->msg, VP_ERR_STATE, "vp_get_f before vp_set_f");
    if (async && dtype != P.precision)
        return fail(s->msg, VP_ERR_ARG, "get_f_async: the weights must have the simulation's dtype");
    const void *src = nullptr;
    const size_t szs = P.precision == VP_FP64 ? 8 : 4;
    // a pinned host buffer and the state s = Lambda_p w: the p solve writes the weights in place
    // (the asynchronous call solves into device memory and copies with the copy engine)
    void *hdev = (!device && !async && dtype == P.precision && P.state_s) ? host_device_ptr(dstp, szs) : nullptr;
    {
        vp_status st = P.precision == VP_FP64 ? weights_of_state<double>(s, &src, hdev)
                                              : weights_of_state<float>(s, &src, hdev);
        if (st != VP_OK) return st;
    }
    if (hdev) {
        // the p solve above wrote the weights into the host buffer
    } else if (dtype == P.precision) {
        VP_CUDA(s, cudaMemcpyAsync(dstp, src, N * szs,
                                   device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                   s->stream));
    } else if (device) {
        if (P.precision == VP_FP32)
            VP_CUDA(s, launch_convert<float, double>(static_cast<const float *>(src),
                                                     static_cast<double *>(dstp), N, s->stream));
        else
            VP_CUDA(s, launch_convert<double, float>(static_cast<const double *>(src),
                                                     static_cast<float *>(dstp), N, s->stream));
    } else {
        std::vector<char> tmp(N * szs);
        VP_CUDA(s, cudaMemcpyAsync(tmp.data(), src, N * szs, cudaMemcpyDeviceToHost, s->stream));
        VP_CUDA(s, cudaStreamSynchronize(s->stream));
        if (P.precision == VP_FP32) {
            const float *in = reinterpret_cast<const float *>(tmp.data());
            double *o = static_cast<double *>(dstp);
            for (size_t k = 0; k < N; ++k) o[k] = in[k];
        } else {
            const double *in = reinterpret_cast<const double *>(tmp.data());
            float *o = static_cast<float *>(dstp);
            for (size_t k = 0; k < N; ++k) o[k] = (float)in[k];
        }
    }
    if (mode != Xfer::host) return VP_OK;
    return check_flags(s);
}

vp_status vp_get_f(vp_sim *s, void *host, int32_t dtype, size_t n)
{
    return get_f_common(s, host, dtype, n, Xfer::host);
}

vp_status vp_get_f_async(vp_sim *s, void *host, int32_t dtype, size_t n)
{
    return get_f_common(s, host, dtype, n, Xfer::host_async);
}

vp_status vp_get_f_device(vp_sim *s, void *dev, int32_t dtype, size_t n)
{
    return get_f_common(s, dev, dtype, n, Xfer::device);
}

vp_status vp_moments(vp_sim *s, vp_moments_t *out)
{
    if (!s || !out) return VP_ERR_ARG;
    if (!s->f_set) return fail(s->msg, VP_ERR_STATE, "vp_moments before vp_set_f");
    const Plan &P = s->P;
    double *mpart = s->ptr<double>(P.L.mpart);
    double *mout = s->ptr<double>(P.L.mout);
    const void *w = nullptr;
    {
        vp_status st = P.precision == VP_FP64 ? weights_of_state<double>(s, &w)
                                              : weights_of_state<float>(s, &w);
        if (st != VP_OK) return st;
    }
    if (P.precision == VP_FP64)
        VP_CUDA(s, launch_moments<double>(static_cast<const double *>(w), P.g,
                                          s->ptr<double2>(P.L.csx), mpart, P.nmblk, s->stream));
    else
        VP_CUDA(s, launch_moments<float>(static_cast<const float *>(w), P.g,
                                         s->ptr<double2>(P.L.csx), mpart, P.nmblk, s->stream));
    VP_CUDA(s, launch_moments_finalize(mpart, P.nmblk, s->ptr<double>(P.L.lost), P.nlost, mout,
                                       s->stream));
    VP_CUDA(s, cudaMemcpyAsync(s->host_mout, mout, kMoutLen * sizeof(double), cudaMemcpyDeviceToHost,
                               s->stream));
    VP_CUDA(s, cudaMemcpyAsync(s->host_state, s->ws + P.L.state, sizeof(s->host_state),
                               cudaMemcpyDeviceToHost, s->stream));
    vp_status st = check_flags(s);
    const double *m = s->host_mout;
    const double hh = P.g.hx * P.g.hp;
    const double S = m[0];
    memset(out, 0, sizeof(*out));
    out->sum_w = S;
    out->mass = S * hh;
    out->mean_x = m[1] / S;
    out->mean_p = m[2] / S;
    out->var_x = m[3] / S - out->mean_x * out->mean_x;
    out->var_p = m[4] / S - out->mean_p * out->mean_p;
    out->cov_xp = m[5] / S - out->mean_x * out->mean_p;
    out->a_re = s->host_state[ST_A_RE];
    out->a_im = s->host_state[ST_A_IM];
    out->energy = P.fel ? out->mean_p + out->a_re * out->a_re + out->a_im * out->a_im : m[6] / S;
    out->trapped = m[7] * hh;
    out->entropy = m[8] * hh;
    out->neg_mass = m[9] * hh;
    out->b_re = m[10] / S;
    out->b_im = -m[11] / S;
    out->max_abs_w = m[12];
    out->lost_mass = m[kNumMoments] * hh;
    out->tau = s->host_state[ST_TAU];
    out->step = (int64_t)s->host_state[ST_STEP];
    return st;
}

vp_status vp_field_history(vp_sim *s, double *re_im, size_t max_entries, size_t *count)
{
    if (!s || !count || (!re_im && max_entries)) return VP_ERR_ARG;
    const Plan &P = s->P;
    std::vector<double> h((size_t)P.hist_cap * 2);
    VP_CUDA(s, cudaMemcpyAsync(h.data(), s->ws + P.L.hist, h.size() * sizeof(double),
                               cudaMemcpyDeviceToHost, s->stream));
    VP_CUDA(s, cudaMemcpyAsync(s->host_state, s->ws + P.L.state, sizeof(s->host_state),
                               cudaMemcpyDeviceToHost, s->stream));
    VP_CUDA(s, cudaStreamSynchronize(s->stream));
    const long step = (long)s->host_state[ST_STEP];
    size_t c = (size_t)std::min<long>(step, P.hist_cap);
    c = std::min(c, max_entries);
    for (size_t k = 0; k < c; ++k) {
        const long st = step - (long)c + (long)k;
        const long slot = st % P.hist_cap;
        re_im[2 * k] = h[2 * slot];
        re_im[2 * k + 1] = h[2 * slot + 1];
    }
    *count = P.fel ? c : 0;
    return VP_OK;
}

vp_status vp_sync(vp_sim *s)
{
    if (!s) return VP_ERR_ARG;
    return check_flags(s);
}

vp_status vp_set_stream(vp_sim *s, void *stream)
{
    if (!s) return VP_ERR_ARG;
    s->stream = static_cast<cudaStream_t>(stream);
    return VP_OK;
}

vp_status vp_state_device(vp_sim *s, void **dev)
{
    if (!s || !dev) return VP_ERR_ARG;
    if (!s->f_set) return fail(s->msg, VP_ERR_STATE, "vp_state_device before vp_set_f");
    const void *w = nullptr;
    vp_status st = s->P.precision == VP_FP64 ? weights_of_state<double>(s, &w)
                                             : weights_of_state<float>(s, &w);
    *dev = const_cast<void *>(w);
    return st;
}

vp_status vp_plan(const vp_sim *s, vp_plan_info *out)
{
    if (!s || !out) return VP_ERR_ARG;
    const Plan &P = s->P;
    memset(out, 0, sizeof(*out));
    out->kernel = P.xpass ? VP_KERNEL_FUSED_XPASS : P.kernel;
    out->tile_x = P.kernel == VP_KERNEL_SCATTER ? P.g.nx : P.tx;
    out->tile_p = P.kernel == VP_KERNEL_SCATTER ? P.g.np : P.tp;
    out->ntiles_x = P.kernel == VP_KERNEL_SCATTER ? 1 : P.ntx;
    out->ntiles_p = P.kernel == VP_KERNEL_SCATTER ? 1 : P.ntp;
    out->threads = P.kernel == VP_KERNEL_FUSED ? P.threads : 0;
    out->full_row = P.full_row ? 1 : 0;
    out->state_is_s = P.state_s ? 1 : 0;
    // step kernel (+ filters along x and p) (+ FEL partials) + field update or step counter;
    // the one-pass kernel does the field update or the count in its last CTA
    int n = P.kernel == VP_KERNEL_FUSED ? (P.xpass ? 2 : 1) : 2;
    if (P.kernel == VP_KERNEL_FUSED && P.fel && P.g.sigma2 != 0.0) n += 2;   // space-charge kick
    if (P.kernel != VP_KERNEL_FUSED && (P.galerkin || P.septic_gal)) n += 2;
    if (P.septic_gal && P.fel) n += 1;   // FEL partial sums after the septic solves
    if (P.kernel == VP_KERNEL_SCATTER && P.fel && !P.galerkin) n += 1;
    if (P.rk4) n += 8;   // four stage reductions, each with its amplitude update
    out->launches_per_step = n;
    out->workspace_bytes = (int64_t)P.L.total;
    const bool f64 = P.precision == VP_FP64;
    if (P.kernel == VP_KERNEL_FUSED)
        out->smem_bytes = (int64_t)(f64 ? fused_smem_bytes<double>(P.ws, P.tp + 2 * P.Gp, P.threads, P.rowcache)
                                        : fused_smem_bytes<float>(P.ws, P.tp + 2 * P.Gp, P.threads, P.rowcache));
    else if (P.kernel == VP_KERNEL_TILED)
        out->smem_bytes = (int64_t)(f64 ? tiled_smem_bytes<double>(P.tx, P.tp)
                                        : tiled_smem_bytes<float>(P.tx, P.tp));
    return VP_OK;
}

void vp_destroy(vp_sim *s) { delete s; }

const char *vp_last_error(const vp_sim *s) { return s ? s->msg : "NULL simulation"; }

}  // extern "C"

// ============================================================================ batching
struct vp_batch {
    std::vector<vp_sim *> sims;
    cudaStream_t stream;
    char *ws;
    FusedArgs<float> *d_args;
    int *d_parity;
    int2 *d_items;
    int *d_left;            // per simulation: steps it still takes in the current call
    BatchFinal *d_fin;
    int nitems, ninst, threads, grid, basis, projection;
    size_t smem;
    cudaGraphExec_t graph;
    bool have_graph;
    std::vector<int> host_parity;
    std::vector<int> host_left;
    char msg[512];
};

namespace {

struct BatchLayout {
    size_t args, parity, items, left, fin, total;
};

void batch_layout_of(int count, int items, BatchLayout *L);

vp_status batch_layout(vp_sim *const *sims, int count, BatchLayout *L, int *nitems, char *msg)
{
    if (!sims || count < 1) return fail(msg, VP_ERR_ARG, "batch needs at least one simulation");
    int items = 0;
    for (int k = 0; k < count; ++k) {
        const vp_sim *s = sims[k];
        if (!s) return fail(msg, VP_ERR_ARG, "simulation %d is NULL", k);
        const Plan &P = s->P;
        const Plan &P0 = sims[0]->P;
        if (P.kernel != VP_KERNEL_FUSED || P.xpass)
            return fail(msg, VP_ERR_UNSUPPORTED, "simulation %d does not use the one-pass kernel", k);
        if (P.precision != VP_FP32)
            return fail(msg, VP_ERR_UNSUPPORTED, "batches hold FP32 simulations (simulation %d)", k);
        if (P.g.basis != P0.g.basis || P.g.projection != P0.g.projection)
            return fail(msg, VP_ERR_ARG, "simulation %d differs in basis or projection", k);
        if (P.g.sigma2 != 0.0)
            return fail(msg, VP_ERR_UNSUPPORTED, "simulation %d has FEL space charge (sigma2 != 0)", k);
        items += P.ntx * P.ntp;
    }
    batch_layout_of(count, items, L);
    *nitems = items;
    return VP_OK;
}

void batch_layout_of(int count, int items, BatchLayout *L)
{
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes);
        return o;
    };
    L->args = take(sizeof(FusedArgs<float>) * 2 * count);
    L->parity = take(sizeof(int) * count);
    L->items = take(sizeof(int2) * items);
    L->left = take(sizeof(int) * count);
    L->fin = take(sizeof(BatchFinal) * count);
    L->total = off;
}

#define VP_BCUDA(b, ...)                                                                   \
    do {                                                                                   \
        cudaError_t e_ = (__VA_ARGS__);                                                    \
        if (e_ != cudaSuccess)                                                             \
            return fail(b->msg, VP_ERR_CUDA, "%s: %s", #__VA_ARGS__, cudaGetErrorString(e_)); \
    } while (0)

vp_status batch_enqueue_step(vp_batch *b)
{
    VP_BCUDA(b, launch_step_fused_batch<float>(b->d_args, b->d_parity, b->d_left, b->d_items, b->nitems,
                                               b->basis, b->projection, b->smem, b->threads, b->grid,
                                               b->stream));
    VP_BCUDA(b, launch_batch_finalize(b->d_fin, b->ninst, b->d_parity, b->d_left, b->stream));
    return VP_OK;
}

}  // namespace

size_t vp::batch_workspace_bytes(int count, int items)
{
    BatchLayout L;
    batch_layout_of(count, items, &L);
    return L.total;
}

extern "C" {

vp_status vp_batch_workspace_size(vp_sim *const *sims, int32_t count, size_t *bytes)
{
    if (!bytes) return VP_ERR_ARG;
    BatchLayout L;
    int n;
    vp_status st = batch_layout(sims, count, &L, &n, nullptr);
    if (st == VP_OK) *bytes = L.total;
    return st;
}

vp_status vp_batch_create(vp_sim *const *sims, int32_t count, void *stream, void *workspace,
                          size_t workspace_bytes, vp_batch **out)
{
    if (!out) return VP_ERR_ARG;
    *out = nullptr;
    vp_batch *b = new (std::nothrow) vp_batch();
    if (!b) return VP_ERR_ARG;
    BatchLayout L;
    int nitems = 0;
    vp_status st = batch_layout(sims, count, &L, &nitems, b->msg);
    if (st != VP_OK) {
        delete b;
        return st;
    }
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) % kAlign) || workspace_bytes < L.total) {
        delete b;
        return VP_ERR_WORKSPACE;
    }
    b->sims.assign(sims, sims + count);
    b->stream = static_cast<cudaStream_t>(stream);
    b->ws = static_cast<char *>(workspace);
    b->d_args = reinterpret_cast<FusedArgs<float> *>(b->ws + L.args);
    b->d_parity = reinterpret_cast<int *>(b->ws + L.parity);
    b->d_items = reinterpret_cast<int2 *>(b->ws + L.items);
    b->d_left = reinterpret_cast<int *>(b->ws + L.left);
    b->d_fin = reinterpret_cast<BatchFinal *>(b->ws + L.fin);
    b->nitems = nitems;
    b->ninst = count;
    b->basis = sims[0]->P.g.basis;
    b->projection = sims[0]->P.g.projection;
    b->have_graph = false;
    // tables: arguments for both buffer parities, the work list (largest tiles first), finals
    std::vector<FusedArgs<float>> args(2 * count);
    std::vector<BatchFinal> fin(count);
    std::vector<int> order(count);
    b->threads = 32;
    b->smem = 0;
    for (int k = 0; k < count; ++k) {
        vp_sim *s = sims[k];
        const Plan &P = s->P;
        args[2 * k] = fused_args<float>(s, s->f(0), s->f(1));
        args[2 * k + 1] = fused_args<float>(s, s->f(1), s->f(0));
        // the batch finishes every simulation's step in its own finalize launch
        args[2 * k].ticket = nullptr;
        args[2 * k + 1].ticket = nullptr;
        b->threads = std::max(b->threads, P.threads);
        order[k] = k;
        fin[k].state = s->ptr<double>(P.L.state);
        fin[k].part = s->ptr<double>(P.L.part);
        fin[k].hist = s->ptr<double>(P.L.hist);
        fin[k].nparts = P.ntx * P.ntp;
        fin[k].hist_cap = P.hist_cap;
        fin[k].fel = P.fel ? 1 : 0;
        fin[k].dt = P.g.dt;
    }
    for (int k = 0; k < count; ++k) {
        const Plan &P = sims[k]->P;
        b->smem = std::max(b->smem, fused_smem_bytes<float>(P.ws, P.tp + 2 * P.Gp, b->threads));
    }
    {
        // every item runs with the batch's thread count: the row cache takes what is left of
        // the shared memory beside the largest window, if the batch keeps its CTAs per SM
        const int want = b->threads > kFusedThreads2 ? 1 : 2;
        int rows = fused_rowcache_rows(VP_FP32, b->smem, want);
        if (rows > 0 && fused_batch_blocks_per_sm(b->basis, b->projection,
                                                  b->smem + (size_t)rows * sizeof(RowEntry<float>),
                                                  b->threads) < want)
            rows = 0;
        for (int k = 0; k < count; ++k) {
            const int r = std::min(rows, sims[k]->P.rowcache);
            args[2 * k].rowcache = r;
            args[2 * k + 1].rowcache = r;
        }
        b->smem += (size_t)rows * sizeof(RowEntry<float>);
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        const Plan &A = sims[a]->P, &C = sims[c]->P;
        return (size_t)A.tx * A.tp > (size_t)C.tx * C.tp;
    });
    std::vector<int2> items;
    items.reserve(nitems);
    for (int k : order)
        for (int t = 0; t < sims[k]->P.ntx * sims[k]->P.ntp; ++t) items.push_back(make_int2(k, t));
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_args, args.data(), sizeof(FusedArgs<float>) * args.size(),
                            cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_items, items.data(), sizeof(int2) * items.size(),
                            cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_fin, fin.data(), sizeof(BatchFinal) * fin.size(),
                            cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        delete b;
        return VP_ERR_CUDA;
    }
    // one CTA per item
    b->grid = std::max(1, nitems);
    e = launch_step_fused_batch<float>(nullptr, nullptr, nullptr, nullptr, 0, b->basis, b->projection,
                                       b->smem, b->threads, 0, b->stream);
    if (e != cudaSuccess) {
        delete b;
        return VP_ERR_CUDA;
    }
    *out = b;
    return VP_OK;
}

// n steps of the batch; simulation k takes min(n, limit[k]) of them (limit NULL: all n)
static vp_status batch_steps(vp_batch *b, int32_t n, const int32_t *limit, int32_t use_graph)
{
    if (!b) return VP_ERR_ARG;
    if (n < 0) return fail(b->msg, VP_ERR_ARG, "negative step count");
    b->host_parity.resize(b->ninst);
    b->host_left.resize(b->ninst);
    for (int k = 0; k < b->ninst; ++k) {
        const int take = limit ? std::max(0, std::min(n, limit[k])) : n;
        if (take > 0 && !b->sims[k]->f_set)
            return fail(b->msg, VP_ERR_STATE, "simulation %d has no weights", k);
        b->host_parity[k] = b->sims[k]->cur;
        b->host_left[k] = take;
    }
    VP_BCUDA(b, cudaMemcpyAsync(b->d_parity, b->host_parity.data(), sizeof(int) * b->ninst,
                                cudaMemcpyHostToDevice, b->stream));
    VP_BCUDA(b, cudaMemcpyAsync(b->d_left, b->host_left.data(), sizeof(int) * b->ninst,
                                cudaMemcpyHostToDevice, b->stream));
    // the legacy default stream cannot be captured: there the steps are launched directly
    if (b->stream == nullptr) use_graph = 0;
    if (use_graph && n > 0 && !b->have_graph) {
        cudaGraph_t g;
        VP_BCUDA(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        vp_status st = batch_enqueue_step(b);
        cudaError_t e = cudaStreamEndCapture(b->stream, &g);
        if (st != VP_OK) return st;
        VP_BCUDA(b, e);
        e = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
        VP_BCUDA(b, e);
        b->have_graph = true;
    }
    for (int s = 0; s < n; ++s) {
        if (use_graph) {
            VP_BCUDA(b, cudaGraphLaunch(b->graph, b->stream));
        } else {
            vp_status st = batch_enqueue_step(b);
            if (st != VP_OK) return st;
        }
    }
    // host copies of the buffer parity follow the device ones
    for (int k = 0; k < b->ninst; ++k) b->sims[k]->cur = (b->sims[k]->cur + b->host_left[k]) & 1;
    // the uploads above read host memory: complete them before the vectors are reused
    VP_BCUDA(b, cudaStreamSynchronize(b->stream));
    return VP_OK;
}

vp_status vp_batch_step(vp_batch *b, int32_t n, int32_t use_graph)
{
    return batch_steps(b, n, nullptr, use_graph);
}

vp_status vp_batch_step_each(vp_batch *b, int32_t n, const int32_t *max_steps, int32_t use_graph)
{
    if (!b || !max_steps) return VP_ERR_ARG;
    return batch_steps(b, n, max_steps, use_graph);
}

vp_status vp_batch_sync(vp_batch *b)
{
    if (!b) return VP_ERR_ARG;
    VP_BCUDA(b, cudaStreamSynchronize(b->stream));
    return VP_OK;
}

void vp_batch_destroy(vp_batch *b)
{
    if (!b) return;
    if (b->have_graph) cudaGraphExecDestroy(b->graph);
    delete b;
}

const char *vp_batch_last_error(const vp_batch *b) { return b ? b->msg : "NULL batch"; }

}  // extern "C"
