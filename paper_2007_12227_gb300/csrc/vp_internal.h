// vp_internal.h -- device data layout and launch entry points shared by the
// translation units of libvlasov (not part of the public C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "vlasov.h"

namespace vp {

// ---------------------------------------------------------------------------
// Push in displacement form (Sec. II flow of one mesh node over the step h).
//
// Every pusher of this library moves node (i, j) by
//   du = (C.ui + R.ui) + (C.uf + R.uf) + KU * s        [cells along x]
//   dv = (C.vi + R.vi) + (C.vf + R.vf) + KV * s        [cells along p]
//   s  = alpha * sin(a_i + y_j) + beta * cos(a_i + y_j)
// with per-column entries C (index i) and per-row entries R (index j) built
// once in FP64 on the device, integer parts split off so that the FP32 path
// keeps sub-cell precision, and (alpha, beta) fixed per sim or, for the FEL,
// read from the field A^{n+1/2} every step. sin/cos of the sum come from the
// angle-addition identity of the tabulated sin/cos of a_i and y_j.
// ---------------------------------------------------------------------------
template <typename T>
struct ColEntry {
    int ui, vi;
    T uf, vf, sa, ca;
};

template <typename T>
struct __align__(16) RowEntry {   // FP32: 32 bytes, two vector loads
    int ui, vi;
    T uf, vf;
    T cy, cy2, sy, sy2;   // cy2 = cy, sy2 = sy: (cos, cos) and (sin, sin) pairs for packed math
};

// FP64 per-row values used only to bound the source window of a tile.
struct RowBound {
    double u, v, y;
    double pad;
};

// Device FEL / step state (doubles).
enum {
    ST_A_RE = 0, ST_A_IM, ST_B_RE, ST_B_IM, ST_AH_RE, ST_AH_IM, ST_TAU, ST_STEP,
    ST_M, ST_PHI,   // |K| and atan2(Re K, -Im K): amplitude and phase of the sine term
    ST_K_RE, ST_K_IM,   // FEL kick amplitude K = A^{n+1/2} + i sigma2 <exp(-i theta~)>
    ST_RK_K = 16,       // RK4: K_1..K_4 (re, im), 8 slots
    ST_RK_B = 24,       // RK4: stage bunchings b_1..b_4 (re, im), 8 slots
    ST_NSTATE = 32
};

// Device error flag bits.
enum { ERRF_NONFINITE = 1u, ERRF_TIMEOUT = 2u, ERRF_WINDOW = 4u };

constexpr int kColBlock = 32;     // column block of the V-bound table
constexpr int kNumMoments = 13;   // accumulators of the moments reduction (lost follows)

struct Geometry {
    int nx, np;
    double x0, x1, p0, p1, hx, hp;
    int basis, kind, potential, projection;
    double v_sign, omega, dt;
    double delta, sigma2;   // FEL detuning and space-charge coefficient
    double KU, KV;          // coefficients of the sine term
    double alpha0, beta0;   // sine-term weights for non-FEL pushers
    double m0, phi0;        // hypot(alpha0, beta0), atan2(beta0, alpha0)
    double a_pad;           // bound on |a_i - x_i|
    double uc_min, uc_max;  // bounds of the column part of du
    double vc_min, vc_max;  // bounds of the column part of dv
    double vr_min, vr_max;  // bounds of the row part of dv
};

template <typename T>
struct StepArgs {
    const T *src;
    T *dst;
    const ColEntry<T> *col;
    const RowEntry<T> *row;
    const RowBound *rowb;
    const double *vcb;      // per 32-column block: min, max of the column part of dv
    const double *state;    // ST_* (FEL reads A^{n+1/2})
    const double2 *csx;     // (cos x_i, sin x_i) in FP64, for the FEL partial sums
    double *tile_lost;      // per tile, cumulative lost weight
    double *tile_part;      // per tile: sum w, sum w cos x, sum w sin x (FEL)
    unsigned *err;
    Geometry g;
    int tx, tp, ntx, ntp;   // tile shape and counts
    int fel_partials;       // emit FEL partials from the step kernel
};

// One-pass step kernel (vp_fused.cu): see the description there.
constexpr int kFusedMaxThreads = 576;   // one CTA per SM (wide tiles)
constexpr int kFusedThreads2 = 320;     // two CTAs per SM

template <typename T>
struct FusedArgs {
    const T *src;
    T *dst;
    const ColEntry<T> *col;
    const RowEntry<T> *row;
    const RowBound *rowb;
    const double *vcb;
    const float4 *rowbf;    // FP32 copy of rowb: u, v, y (tile bounds)
    const float2 *vcbf;     // FP32 copy of vcb
    const double *state;
    const double *piv;      // Thomas pivots of tridiag(1/6, 2/3, 1/6)
    const double *sigma;    // column sums of Lambda_p^{-1} (FEL partial sums in Galerkin mode)
    const double2 *csx;
    double *tile_lost;
    double *tile_part;
    unsigned *err;
    Geometry g;
    int tx, tp, ntx, ntp;
    int G, Gp;              // guard bands (cells) around the widened tile: columns, rows
    int ws;                 // window row stride (elements)
    int full_row;           // tiles span the whole x period (ntx == 1)
    int fel_partials;
    // FP32: max|state| per destination tile of the state read (in) and of the state written (out),
    // [ntp][ntx]; it bounds the fixed-point window of the next step
    const float *smax_in;
    float *smax_out;
    // source rectangle (ia, ib, ja, jb) per tile when the push does not change between steps
    // (NULL for the FEL); entries equal to kTileSrcUnset are computed and stored by the tile
    int4 *tile_src;
    // end of the step in the same launch: every CTA takes a ticket after its tile's partial sums
    // are visible; the CTA that draws the last one updates the FEL field from all partials (or
    // counts the step) and resets the counter. NULL: the caller finishes the step (batches).
    int *ticket;
    double *hist;           // FEL field history ring (hist_cap steps)
    int hist_cap;
    // rows of the push's row table a tile may keep in shared memory (after the window and the
    // column buffer); a tile whose source rows fit reads them there instead of through L1
    int rowcache;
    // Galerkin plans with a separate x pass: the tile stores its deposit r = Delta^T w (own
    // columns, no x halo) and xsolve_rows_kernel applies Lambda_x^{-1} to whole rows afterwards
    int xpass;
    // FEL with a separate x pass: the tile sums the deposit r instead of s' = Lambda_x^{-1} r. The
    // circulant Lambda_x has the mode exp(-i theta) as an eigenvector (eigenvalue
    // lambda_1 = 2/3 + cos(h_theta)/3; the constant mode: 1), so the cos/sin sums of s' are those of r
    // times bunch_x = 1 / lambda_1 (1 when the tile solves x itself)
    double bunch_x;
};
constexpr int kTileSrcUnset = (int)0x80808080;   // the bytes 0x80 (cudaMemset)

// Tap weights of the septic B-spline B7 (the deposit kernel of cubic B-spline basis
// functions) for a node at fraction t in [0, 1) past cell m: w[a] = B7(t + 3 - a) for the
// cells m - 3 .. m + 4, by the Cox-de Boor recursion of the cardinal B-splines
// M_d(x) = (x M_{d-1}(x) + (d + 1 - x) M_{d-1}(x - 1)) / d, M_0 = 1 on [0, 1):
// v[k] = M_d(t + k), k = 0..d, and B7(y) = M_7(y + 4).
template <typename T>
__device__ __forceinline__ void septic_weights(T t, T *w)
{
    T v[8];
    v[0] = T(1);
#pragma unroll
    for (int d = 1; d <= 7; ++d) {
        T nv[8];
#pragma unroll
        for (int k = 0; k <= d; ++k) {
            const T a = k < d ? v[k] : T(0);
            const T b = k > 0 ? v[k - 1] : T(0);
            nv[k] = ((t + T(k)) * a + (T(d + 1) - t - T(k)) * b) / T(d);
        }
#pragma unroll
        for (int k = 0; k <= d; ++k) v[k] = nv[k];
    }
#pragma unroll
    for (int a = 0; a < 8; ++a) w[a] = v[7 - a];
}

// The septic B-spline mass matrix 1/5040 (1, 120, 1191, 2416, 1191, 120, 1) factors as
// gain * prod_i 1 / ((1 - z_i q)(1 - z_i / q)) with these poles (roots inside the unit circle
// of q^6 + 120 q^5 + 1191 q^4 + 2416 q^3 + 1191 q^2 + 120 q + 1), gain = 5040 prod (-z_i).
constexpr double septic_pole(int q)
{
    return q == 0 ? -0.53528043079643816554 : (q == 1 ? -0.12255461519232669052 : -0.0091486948096082769286);
}
// Lambda_p LDL^T factor rows kept exactly (then their limit): D_j and L_{j+m, j}, m = 1..3
constexpr int kLdlRows = 96;

// ---- launch entry points (defined in the .cu files) -----------------------
cudaError_t build_tables(const Geometry &g, int precision, void *col, void *row,
                         RowBound *rowb, double *ucol, double *vcol, double2 *csx, cudaStream_t s);

template <typename T>
cudaError_t launch_step_tiled(const StepArgs<T> &a, cudaStream_t s);
template <typename T>
cudaError_t launch_step_scatter(const StepArgs<T> &a, double *lost_acc, cudaStream_t s);
template <typename T>
size_t tiled_smem_bytes(int tx, int tp);

template <typename T>
cudaError_t launch_step_fused(const FusedArgs<T> &a, int threads, cudaStream_t s);
// dynamic shared memory of the one-pass kernel: window (ws x wh), column buffer, row cache
template <typename T>
size_t fused_smem_bytes(int ws, int wh, int threads, int rowcache = 0);
// rows of RowEntry<T> that fit in the shared memory left beside base dynamic bytes, keeping
// ctas CTAs per SM (0 when fewer than 32 rows fit); queries the current device when it can
int fused_rowcache_rows(int precision, size_t base_bytes, int ctas);
// CTAs of the FP32 batched step kernel per SM at this shared memory and block size (0: unknown)
int fused_batch_blocks_per_sm(int basis, int projection, size_t smem, int threads);
// one CTA per item (grid >= nitems; grid <= 0: set the shared-memory attribute only);
// left[k]: steps simulation k still takes in this call; its items are skipped at 0
template <typename T>
cudaError_t launch_step_fused_batch(const FusedArgs<T> *args, const int *parity, const int *left,
                                    const int2 *items, int nitems, int basis, int projection,
                                    size_t smem, int threads, int grid, cudaStream_t s);

// per-instance end-of-step work of a batch: FEL field update, or the step counter
struct BatchFinal {
    double *state;
    const double *part;
    double *hist;
    int nparts, hist_cap, fel;
    double dt;
};
// finishes the step of every simulation with left[k] > 0, flips its parity, decrements left[k]
cudaError_t launch_batch_finalize(const BatchFinal *fin, int ninst, int *parity, int *left, cudaStream_t s);
// device bytes of a batch of `count` simulations with `items` tiles in all
size_t batch_workspace_bytes(int count, int items);
constexpr int fused_halo(int precision) { return precision == VP_FP64 ? 28 : 16; }
// the x-solve row pass of plans with a separate x pass: one CTA per mesh row, each thread a
// contiguous chunk of at most kXRowMaxPer elements (FP32 32, FP64 16)
constexpr int kXRowMaxThreads = 1024;
constexpr int xrow_max_per(int precision) { return precision == VP_FP64 ? 16 : 32; }
// threads and chunk length for rows of nx (0 threads: nx too long for the pass)
void xrow_shape(int precision, int nx, int *threads, int *per);
size_t xrow_smem_bytes(int precision, int nx, int ntx);
// row buffers of the pass (2: the next row is copied in while one is solved) and its grid (a
// persistent CTA count from the occupancy of the current device, at most np)
int xrow_buffers(int precision, int nx, int ntx);
int xrow_grid_size(int precision, int nx, int np, int ntx);
// s' = Lambda_x^{-1} r along every row (cyclic, exact: block-wide carries, no truncation), then
// FP32: the per-tile max|s'| into smax_out[ntp][ntx] (atomic max over the zeros the step kernel
// stored); non-finite outputs set ERRF_NONFINITE
template <typename T>
cudaError_t launch_xsolve_rows(const T *r, T *out, int nx, int np, const double *piv, int tx, int tp,
                               int ntx, float *smax_out, unsigned *err, int grid, cudaStream_t s);
constexpr int kFusedMaxRow = 512; // longest window row one warp solves
constexpr int kFusedMaxTileP = 256; // tallest tile of the fused kernel
template <typename T>
cudaError_t launch_lambda_p_mul(const T *w, T *s, int nx, int np, cudaStream_t st);
// max|s| of an FP32 state over each tile x tile_p tile into map[ntp][ntx]; non-finite -> err
cudaError_t launch_tile_max(const float *s, float *map, int nx, int np, int tx, int tp, int ntx,
                            int ntp, unsigned *err, cudaStream_t st);

template <typename T>
cudaError_t launch_filter_x(const T *in, T *out, int nx, int np, const double *piv, unsigned *err,
                            cudaStream_t s);
// septic B-spline Galerkin solves: cyclic 3-pole recursion along x (scale: float pair
// sh + sl), LDL^T of the np x np principal block along p (ldl: (kLdlRows + 1) rows of D, L1..L3)
template <typename T>
cudaError_t launch_filter_x7(const T *in, T *out, int nx, int np, double sh, double sl,
                             cudaStream_t s);
template <typename T>
cudaError_t launch_filter_p7(const T *in, T *out, int nx, int np, const double *ldl, cudaStream_t s);
template <typename T>
cudaError_t launch_filter_p(const T *in, T *out, int nx, int np, const double *piv,
                            const double2 *csx, double *part, int want_part, unsigned *err,
                            cudaStream_t s);
constexpr int kPivots = 64;       // exact Thomas pivots kept for the first rows
// Pivot table layout (doubles): [2 r] = c'_r, [2 r + 1] = 1 / beta_r for r < kPivots, then
// their limits at [2 kPivots], [2 kPivots + 1]; then the FP32 Lambda_x scale of the one-pass
// kernel and of the separate filters, each as a float pair hi + lo (see unit_gain_scale).
constexpr int kPivXsFused = 2 * kPivots + 2;
constexpr int kPivXsFilter = 2 * kPivots + 4;
constexpr int kPivTable = 2 * kPivots + 6;
int filter_p_blocks(int nx, int np);

template <typename T>
cudaError_t launch_fel_partials(const T *w, int nx, int np, const double2 *csx, double *part,
                                cudaStream_t s);
int fel_partial_blocks(int nx, int np);
// FEL space charge: per-block sums of the state against the half-drift row factors
// (rc, rs: cos and sin of h/2 (delta + p_j), times Lambda_p^{-1} when the state is s) and
// the mass weights (sig, NULL = 1), then K = A^{n+1/2} + i sigma2 <exp(-i theta~)>
template <typename T>
cudaError_t launch_fel_tilde(const T *state, int nx, int np, const double2 *csx, const double *rc,
                             const double *rs, const double *sig, double *part, cudaStream_t s);
cudaError_t launch_fel_kick(const double *part, int nparts, double *state, double sigma2,
                            cudaStream_t s);
// FEL RK4: the four stage reductions and amplitudes (part: rk4_stage_blocks x 3 doubles), and
// the deposit at the RK4 end points into a zeroed destination
int rk4_stage_blocks(int nx, int np);
template <typename T>
cudaError_t launch_rk4_stages(const T *w, const Geometry &g, const double2 *csx, double *state,
                              double *part, cudaStream_t s);
template <typename T>
cudaError_t launch_rk4_deposit(const T *src, T *dst, const Geometry &g, const double2 *csx,
                               const double *state, double *lost_acc, cudaStream_t s);
// init: first bunching after vp_set_f; rk4: A^{n+1} is the RK4 value left in ST_AH
cudaError_t launch_fel_finalize(const double *part, int nparts, double *state, double *hist,
                                int hist_cap, double dt, int init, cudaStream_t s, int rk4 = 0);
cudaError_t launch_count_step(double *state, double dt, cudaStream_t s);

template <typename T>
cudaError_t launch_moments(const T *w, const Geometry &g, const double2 *csx, double *part,
                           int nblocks, cudaStream_t s);
int moment_blocks(int nx, int np);
cudaError_t launch_moments_finalize(const double *part, int nblocks, const double *lost,
                                    int nlost, double *out, cudaStream_t s);

template <typename Tin, typename Tout>
cudaError_t launch_convert(const Tin *in, Tout *out, size_t n, cudaStream_t s);

}  // namespace vp
