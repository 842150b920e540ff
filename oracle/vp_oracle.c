/*
 * vp_oracle.c -- plain, serial, FP64 CPU oracle of the phase-space-conserving
 * Vlasov step (Edelen & Webb, "A Vlasov Algorithm Derived from Phase Space
 * Conservation").
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the library's product path may link,
 * load or call this file; only the tests, the smoke check and the benchmark's
 * CPU-baseline leg do. It shares no code with the CUDA path.
 *
 * What one step computes (Sec. III, in the paper's order):
 *   1. every mesh node k = (x_k, p_k) is pushed one step h by a particle pusher
 *      (Sec. II; leapfrog / exact rotation / FEL drift-kick-drift);
 *   2. the right-hand side of the Galerkin equation is formed,
 *        r_j' = sum_k Delta_{k j'} w_k,
 *      where Delta_{k j'} is the overlap integral of the shifted basis function
 *      of node k with the unshifted basis function of node j' (Sec. III, the
 *      definition of Delta). For a symmetric 1-D basis that integral is the
 *      autoconvolution of the basis evaluated at the offset, times the cell
 *      size, so Delta is written out in closed form:
 *        box (top-hat) basis  ->  h * tent(offset / h)
 *        tent basis           ->  h * B3(offset / h)   (cubic B-spline)
 *   3. the mass-matrix equation  Lambda w_fin = r  is solved (Sec. III, the
 *      update equation). Lambda is the overlap matrix of the unshifted basis:
 *        box basis  ->  Lambda = hx hp I (orthogonal, Sec. III)
 *        tent basis ->  Lambda = (hx Tx) (x) (hp Tp),  T = tridiag(1/6, 2/3, 1/6)
 *      cyclic along the periodic coordinate, the plain (truncated) Toeplitz
 *      matrix along the open momentum axis (Sec. IV: periodic coordinates,
 *      open momenta). LUMPED replaces Lambda by its row sums (hx hp I).
 *   4. for the FEL model the bunching <exp(-i theta)> of the new weights drives
 *      the field amplitude A (Sec. IV.B, dA/dz = <exp(-i Phi)>).
 *
 * Deposits that land on momentum rows outside the grid are lost (open
 * boundaries, Sec. IV) and accumulated in a lost-weight counter.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared vp_oracle.c -lm
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int nx, np;
    double x0, x1, p0, p1;
} or_grid;

typedef struct {
    int kind;       /* 0 leapfrog KDK, 1 exact rotation, 2 FEL DKD, 3 FEL RK4 */
    int potential;  /* 0 free, 1 pendulum V=-s cos x, 2 harmonic V=w^2 x^2/2 */
    double v_sign;
    double omega;
    double dt;
    double delta;   /* FEL detuning: d theta/dz = delta + eta */
    double sigma2;  /* FEL space charge: kick amplitude A + i sigma2 <exp(-i theta)> */
} or_pusher;

enum { OR_KDK = 0, OR_ROT = 1, OR_FEL = 2, OR_FEL_RK4 = 3 };
enum { OR_FREE = 0, OR_PEND = 1, OR_HARM = 2 };
enum { OR_TENT = 0, OR_CUBIC = 1, OR_SEPTIC = 2 };
enum { OR_GALERKIN = 0, OR_LUMPED = 1 };

#define OR_NMOM 14

static double grid_hx(const or_grid *g) { return (g->x1 - g->x0) / g->nx; }
static double grid_hp(const or_grid *g) { return (g->p1 - g->p0) / (g->np - 1); }

/* ---------------------------------------------------------------- pushers */

/* dV/dx for the Hamiltonian H = p^2/2 + V(x) (Sec. II). */
static double dVdx(const or_pusher *pu, double x)
{
    switch (pu->potential) {
    case OR_PEND: return pu->v_sign * sin(x);
    case OR_HARM: return pu->omega * pu->omega * x;
    default: return 0.0;
    }
}

static double potential(const or_pusher *pu, double x)
{
    switch (pu->potential) {
    case OR_PEND: return -pu->v_sign * cos(x);
    case OR_HARM: return 0.5 * pu->omega * pu->omega * x * x;
    default: return 0.0;
    }
}

/*
 * One step of the flow for a single phase-space point (Sec. II: the flow is
 * approximated by a particle pusher over the step h).
 *   KDK (second-order symplectic leapfrog, Sec. IV.A):
 *       p_half = p - h/2 V'(x);  x' = x + h p_half;  p' = p_half - h/2 V'(x')
 *   exact rotation (linear oscillator advanced analytically, Sec. IV.A):
 *       phase advance omega h.
 *   FEL drift-kick-drift of the 1-D FEL equations (Sec. IV.B):
 *       d theta/dz = delta + eta,  d eta/dz = -(K e^{i theta} + c.c.),
 *   with the kick amplitude K = A + i sigma2 <exp(-i theta)> taken at the half
 *   step by the caller (a_re, a_im = K):
 *       th = theta + h/2 (delta + eta);  eta' = eta - 2 h Re(K e^{i th});
 *       theta' = th + h/2 (delta + eta').
 */
void or_push(const or_pusher *pu, double a_re, double a_im,
             double x, double p, double *xo, double *po)
{
    const double h = pu->dt;
    if (pu->kind == OR_KDK) {
        double ph = p - 0.5 * h * dVdx(pu, x);
        double xn = x + h * ph;
        *po = ph - 0.5 * h * dVdx(pu, xn);
        *xo = xn;
    } else if (pu->kind == OR_ROT) {
        double ph = pu->omega * h;
        double c = cos(ph), s = sin(ph);
        *xo = x * c + p * s / pu->omega;
        *po = -pu->omega * x * s + p * c;
    } else {
        double th = x + 0.5 * h * (pu->delta + p);
        /* K e^{i th} + c.c. = 2 Re(K e^{i th}) */
        double re = a_re * cos(th) - a_im * sin(th);
        double pn = p - h * 2.0 * re;
        *xo = th + 0.5 * h * (pu->delta + pn);
        *po = pn;
    }
}

/*
 * FEL, classical fourth-order Runge-Kutta (the integrator of Sec. IV.B) for one particle of the
 * system d theta/dz = delta + eta, d eta/dz = -(K e^{i theta} + c.c.), given the kick amplitudes
 * K_1..K_4 of the four stages (k[2 s], k[2 s + 1]: re, im of stage s), which the caller forms from
 * A and the stage bunchings. th_s, p_s (may be NULL): the stage positions, s = 0..3.
 */
void or_push_rk4(const or_pusher *pu, const double *k, double x, double p, double *xo, double *po,
                 double *th_s, double *p_s)
{
    const double h = pu->dt, d = pu->delta;
    double th[4], pp[4], dp[4];
    th[0] = x;
    pp[0] = p;
    for (int s = 0; s < 4; ++s) {
        if (s > 0) {
            const double c = (s == 3) ? h : 0.5 * h;
            th[s] = x + c * (d + pp[s - 1]);
            pp[s] = p + c * dp[s - 1];
        }
        dp[s] = -2.0 * (k[2 * s] * cos(th[s]) - k[2 * s + 1] * sin(th[s]));
    }
    *xo = x + h / 6.0 * ((d + pp[0]) + 2.0 * (d + pp[1]) + 2.0 * (d + pp[2]) + (d + pp[3]));
    *po = p + h / 6.0 * (dp[0] + 2.0 * dp[1] + 2.0 * dp[2] + dp[3]);
    for (int s = 0; s < 4; ++s) {
        if (th_s) th_s[s] = th[s];
        if (p_s) p_s[s] = pp[s];
    }
}

void or_push_many(const or_pusher *pu, double a_re, double a_im, long n,
                  const double *x, const double *p, double *xo, double *po)
{
    for (long k = 0; k < n; ++k)
        or_push(pu, a_re, a_im, x[k], p[k], &xo[k], &po[k]);
}

/* ------------------------------------------------- overlap-integral kernels */

/* autoconvolution of the unit top-hat: the tent */
static double k_tent(double d)
{
    d = fabs(d);
    return d < 1.0 ? 1.0 - d : 0.0;
}

/* autoconvolution of the unit tent: the cubic B-spline */
static double k_b3(double d)
{
    d = fabs(d);
    if (d < 1.0) return 2.0 / 3.0 - d * d + 0.5 * d * d * d;
    if (d < 2.0) {
        double e = 2.0 - d;
        return e * e * e / 6.0;
    }
    return 0.0;
}

/*
 * Autoconvolution of the unit cubic B-spline: the septic B-spline B7 (Sec. III with cubic
 * B-spline basis functions), from its truncated-power definition
 *   B7(x) = 1/7! sum_{k=0..8} (-1)^k C(8, k) (x + 4 - k)_+^7,
 * evaluated at -|x| (even function), where at most four terms are nonzero.
 */
static double k_b7(double d)
{
    const double x = -fabs(d);
    if (x <= -4.0) return 0.0;
    static const double c8[9] = {1, 8, 28, 56, 70, 56, 28, 8, 1};
    double s = 0.0;
    for (int k = 0; k <= 8; ++k) {
        const double t = x + 4.0 - k;
        if (t <= 0.0) break;
        const double t7 = t * t * t * t * t * t * t;
        s += (k & 1 ? -c8[k] : c8[k]) * t7;
    }
    return s / 5040.0;
}

static double k_basis(int basis, double d)
{
    return basis == OR_TENT ? k_tent(d) : (basis == OR_CUBIC ? k_b3(d) : k_b7(d));
}

static long mod_l(long a, long n)
{
    long r = a % n;
    return r < 0 ? r + n : r;
}

/* ------------------------------------------------------ mass-matrix solves */

/* Thomas algorithm: sub a, diag b, super c (constant a, c; diag per row). */
static void thomas(int n, double a, const double *bdiag, double c,
                   double *d, double *cp)
{
    double beta = bdiag[0];
    cp[0] = c / beta;
    d[0] = d[0] / beta;
    for (int i = 1; i < n; ++i) {
        beta = bdiag[i] - a * cp[i - 1];
        cp[i] = c / beta;
        d[i] = (d[i] - a * d[i - 1]) / beta;
    }
    for (int i = n - 2; i >= 0; --i)
        d[i] -= cp[i] * d[i + 1];
}

/*
 * Cyclic symmetric tridiagonal solve (diag b, off-diagonals and corners a),
 * by the Sherman-Morrison correction of a plain tridiagonal solve.
 * Requires n >= 3. d is overwritten with the solution. work: 4n doubles.
 */
static void cyclic_solve(int n, double a, double b, double *d, double *work)
{
    double *bd = work, *z = work + n, *cp = work + 2 * n;
    const double gamma = -b;
    for (int i = 0; i < n; ++i) bd[i] = b;
    bd[0] = b - gamma;
    bd[n - 1] = b - a * a / gamma;
    /* T y = d */
    thomas(n, a, bd, a, d, cp);
    /* T z = u,  u = (gamma, 0, ..., 0, a) */
    memset(z, 0, sizeof(double) * n);
    z[0] = gamma;
    z[n - 1] = a;
    thomas(n, a, bd, a, z, cp);
    /* v = (1, 0, ..., 0, a / gamma) */
    double vy = d[0] + (a / gamma) * d[n - 1];
    double vz = z[0] + (a / gamma) * z[n - 1];
    double fac = vy / (1.0 + vz);
    for (int i = 0; i < n; ++i) d[i] -= fac * z[i];
}

/*
 * Solve Lambda w = r in place, Lambda = (hx Tx) (x) (hp Tp), Tx cyclic
 * tridiag(1/6, 2/3, 1/6) along x (rows of the [np][nx] array), Tp the
 * np x np tridiag(1/6, 2/3, 1/6) along p (columns).
 */
void or_mass_solve(const or_grid *g, double *r)
{
    const int nx = g->nx, np = g->np;
    const double hx = grid_hx(g), hp = grid_hp(g);
    int nmax = nx > np ? nx : np;
    double *work = (double *)malloc(sizeof(double) * 5 * nmax);
    double *col = work + 4 * nmax;
    /* x: cyclic, matrix hx * tridiag(1/6, 2/3, 1/6) */
    for (int j = 0; j < np; ++j)
        cyclic_solve(nx, hx / 6.0, 2.0 * hx / 3.0, r + (long)j * nx, work);
    /* p: open, matrix hp * tridiag(1/6, 2/3, 1/6) */
    double *bd = work;
    double *cp = work + nmax;
    for (int i = 0; i < nx; ++i) {
        for (int j = 0; j < np; ++j) {
            col[j] = r[(long)j * nx + i];
            bd[j] = 2.0 * hp / 3.0;
        }
        thomas(np, hp / 6.0, bd, hp / 6.0, col, cp);
        for (int j = 0; j < np; ++j) r[(long)j * nx + i] = col[j];
    }
    free(work);
}

/*
 * Galerkin mass-matrix solve for cubic B-spline basis functions: Lambda = Lambda_x (x) Lambda_p
 * with the 7-band Toeplitz matrix h B7(j - k) per axis (B7 at 0, 1, 2, 3 = 2416, 1191, 120, 1
 * over 5040). Along x (periodic) the matrix is circulant: solved exactly by its eigenvalues
 * lambda_k = h sum_d B7(d) cos(2 pi d k / nx) with a direct DFT. Along p the basis is not
 * truncated and the matrix is the np x np principal block: banded Gaussian elimination
 * (symmetric positive definite, no pivoting).
 */
void or_mass_solve7(const or_grid *g, double *r)
{
    const int nx = g->nx, np = g->np;
    const double hx = grid_hx(g), hp = grid_hp(g);
    double b[4];
    for (int d = 0; d < 4; ++d) b[d] = k_b7((double)d);
    /* x: circulant */
    double *cs = (double *)malloc(sizeof(double) * 5 * nx);
    double *sn = cs + nx, *lam = sn + nx, *re = lam + nx, *im = re + nx;
    for (int m = 0; m < nx; ++m) {
        const double twopi = 6.283185307179586476925286766559;
        cs[m] = cos(twopi * m / nx);
        sn[m] = sin(twopi * m / nx);
    }
    for (int k = 0; k < nx; ++k) {
        double l = b[0];
        for (int d = 1; d < 4; ++d) l += 2.0 * b[d] * cs[(long)d * k % nx];
        lam[k] = hx * l;
    }
    for (int j = 0; j < np; ++j) {
        double *row = r + (long)j * nx;
        for (int k = 0; k < nx; ++k) {
            double sr = 0.0, si = 0.0;
            for (int i = 0; i < nx; ++i) {
                const long m = (long)i * k % nx;
                sr += row[i] * cs[m];
                si -= row[i] * sn[m];
            }
            re[k] = sr / lam[k];
            im[k] = si / lam[k];
        }
        for (int i = 0; i < nx; ++i) {
            double s = 0.0;
            for (int k = 0; k < nx; ++k) {
                const long m = (long)i * k % nx;
                s += re[k] * cs[m] - im[k] * sn[m];
            }
            row[i] = s / nx;
        }
    }
    free(cs);
    /* p: banded elimination of the principal block (half-bandwidth 3) */
    double *a = (double *)malloc(sizeof(double) * 7 * (size_t)np);   /* a[j*7 + 3 + o]: (j, j+o) */
    double *col = (double *)malloc(sizeof(double) * (size_t)np);
    for (int i = 0; i < nx; ++i) {
        for (int j = 0; j < np; ++j) {
            for (int o = -3; o <= 3; ++o)
                a[(size_t)j * 7 + 3 + o] = (j + o >= 0 && j + o < np) ? hp * b[o < 0 ? -o : o] : 0.0;
            col[j] = r[(long)j * nx + i];
        }
        for (int k = 0; k < np; ++k) {
            const double piv = a[(size_t)k * 7 + 3];
            for (int j = k + 1; j <= k + 3 && j < np; ++j) {
                const double f = a[(size_t)j * 7 + 3 + (k - j)] / piv;
                if (f == 0.0) continue;
                for (int o = 0; o <= 3 && k + o < np; ++o)
                    a[(size_t)j * 7 + 3 + (k + o - j)] -= f * a[(size_t)k * 7 + 3 + o];
                col[j] -= f * col[k];
            }
        }
        for (int k = np - 1; k >= 0; --k) {
            double s = col[k];
            for (int o = 1; o <= 3 && k + o < np; ++o) s -= a[(size_t)k * 7 + 3 + o] * col[k + o];
            col[k] = s / a[(size_t)k * 7 + 3];
        }
        for (int j = 0; j < np; ++j) r[(long)j * nx + i] = col[j];
    }
    free(col);
    free(a);
}

/* ------------------------------------------------------------------ step */

/*
 * One step w_in -> w_out.
 * fel (FEL only, else may be NULL): [A_re, A_im, b_re, b_im] at step n on
 * entry, at step n+1 on exit, where b = <exp(-i theta)> of the weights.
 * lost (may be NULL): accumulates the weight deposited outside the momentum
 * range, in units of sum(w).
 * Returns 0 on success, nonzero on bad arguments.
 */
int or_step(const or_grid *g, int basis, int projection, const or_pusher *pu,
            double *fel, const double *w_in, double *w_out, double *lost)
{
    const int nx = g->nx, np = g->np;
    if (nx < 3 || np < 2) return 1;
    const double hx = grid_hx(g), hp = grid_hp(g);
    const long n = (long)nx * np;
    double a_re = 0.0, a_im = 0.0;
    double k_re = 0.0, k_im = 0.0;   /* kick amplitude */
    if (pu->kind == OR_FEL) {
        if (!fel) return 2;
        /* A^{n+1/2} = A^n + h/2 b^n */
        a_re = fel[0] + 0.5 * pu->dt * fel[2];
        a_im = fel[1] + 0.5 * pu->dt * fel[3];
        k_re = a_re;
        k_im = a_im;
        if (pu->sigma2 != 0.0) {
            /* space charge at the half step: the bunching of the weights at the
             * half-drifted phases th = theta + h/2 (delta + eta); K = A^{n+1/2} + i sigma2 bt */
            double s = 0.0, sc = 0.0, ss = 0.0;
            for (int j = 0; j < np; ++j) {
                const double p = g->p0 + j * hp;
                for (int i = 0; i < nx; ++i) {
                    const double w = w_in[(long)j * nx + i];
                    const double th = g->x0 + i * hx + 0.5 * pu->dt * (pu->delta + p);
                    s += w;
                    sc += w * cos(th);
                    ss += w * sin(th);
                }
            }
            const double bt_re = sc / s, bt_im = -ss / s;
            k_re = a_re - pu->sigma2 * bt_im;
            k_im = a_im + pu->sigma2 * bt_re;
        }
    }
    /* RK4 (Sec. IV.B): stage s needs the bunching b_s of all particles at their stage-s phases,
     * which depend on the amplitudes of the earlier stages: A_1 = A, A_2 = A + h/2 b_1,
     * A_3 = A + h/2 b_2, A_4 = A + h b_3, K_s = A_s + i sigma2 b_s, and
     * A' = A + h/6 (b_1 + 2 b_2 + 2 b_3 + b_4). */
    double rk[8] = {0}, a_new_re = 0.0, a_new_im = 0.0;
    if (pu->kind == OR_FEL_RK4) {
        if (!fel) return 2;
        const double h = pu->dt;
        double b[8];
        for (int s = 0; s < 4; ++s) {
            double sw = 0.0, sc = 0.0, ss = 0.0;
            for (int j = 0; j < np; ++j) {
                const double p = g->p0 + j * hp;
                for (int i = 0; i < nx; ++i) {
                    const double w = w_in[(long)j * nx + i];
                    double th[4], xo, po;
                    or_push_rk4(pu, rk, g->x0 + i * hx, p, &xo, &po, th, NULL);
                    sw += w;
                    sc += w * cos(th[s]);
                    ss += w * sin(th[s]);
                }
            }
            b[2 * s] = sc / sw;
            b[2 * s + 1] = -ss / sw;
            const double c = (s == 0) ? 0.0 : (s == 3 ? h : 0.5 * h);
            const double ar = fel[0] + (s == 0 ? 0.0 : c * b[2 * (s - 1)]);
            const double ai = fel[1] + (s == 0 ? 0.0 : c * b[2 * (s - 1) + 1]);
            rk[2 * s] = ar - pu->sigma2 * b[2 * s + 1];
            rk[2 * s + 1] = ai + pu->sigma2 * b[2 * s];
        }
        a_new_re = fel[0] + h / 6.0 * (b[0] + 2.0 * b[2] + 2.0 * b[4] + b[6]);
        a_new_im = fel[1] + h / 6.0 * (b[1] + 2.0 * b[3] + 2.0 * b[5] + b[7]);
    }
    const double radius = (basis == OR_TENT) ? 1.0 : (basis == OR_CUBIC ? 2.0 : 4.0);
    double lost_acc = 0.0;
    memset(w_out, 0, sizeof(double) * n);

    /* r_j' = sum_k Delta_{k j'} w_k */
    for (int j = 0; j < np; ++j) {
        const double p = g->p0 + j * hp;
        for (int i = 0; i < nx; ++i) {
            const double w = w_in[(long)j * nx + i];
            if (w == 0.0) continue;
            const double x = g->x0 + i * hx;
            double xf, pf;
            if (pu->kind == OR_FEL_RK4)
                or_push_rk4(pu, rk, x, p, &xf, &pf, NULL, NULL);
            else
                or_push(pu, k_re, k_im, x, p, &xf, &pf);
            const double u = (xf - g->x0) / hx;   /* pushed position, cell units */
            const double v = (pf - g->p0) / hp;
            const long c_lo = (long)ceil(u - radius), c_hi = (long)floor(u + radius);
            const long r_lo = (long)ceil(v - radius), r_hi = (long)floor(v + radius);
            for (long rr = r_lo; rr <= r_hi; ++rr) {
                const double kp = hp * k_basis(basis, rr - v);
                if (kp == 0.0) continue;
                for (long cc = c_lo; cc <= c_hi; ++cc) {
                    const double kx = hx * k_basis(basis, cc - u);
                    const double contrib = kx * kp * w;
                    if (rr < 0 || rr >= np) {
                        lost_acc += contrib;
                        continue;
                    }
                    w_out[rr * nx + mod_l(cc, nx)] += contrib;
                }
            }
        }
    }
    /* Lambda w_fin = r */
    if (basis == OR_CUBIC && projection == OR_GALERKIN) {
        or_mass_solve(g, w_out);
    } else if (basis == OR_SEPTIC && projection == OR_GALERKIN) {
        or_mass_solve7(g, w_out);
    } else {
        const double inv = 1.0 / (hx * hp);
        for (long k = 0; k < n; ++k) w_out[k] *= inv;
    }
    if (lost) *lost += lost_acc / (hx * hp);

    if (pu->kind == OR_FEL || pu->kind == OR_FEL_RK4) {
        /* b = <exp(-i theta)> over the new weights; DKD: A^{n+1} = A^{n+1/2} + h/2 b */
        double s = 0.0, sc = 0.0, ss = 0.0;
        for (int j = 0; j < np; ++j)
            for (int i = 0; i < nx; ++i) {
                const double w = w_out[(long)j * nx + i];
                const double th = g->x0 + i * hx;
                s += w;
                sc += w * cos(th);
                ss += w * sin(th);
            }
        fel[2] = sc / s;
        fel[3] = -ss / s;
        if (pu->kind == OR_FEL_RK4) {
            fel[0] = a_new_re;
            fel[1] = a_new_im;
        } else {
            fel[0] = a_re + 0.5 * pu->dt * fel[2];
            fel[1] = a_im + 0.5 * pu->dt * fel[3];
        }
    }
    return 0;
}

/* FEL: b = <exp(-i theta)> of weights w (used to start the field recursion). */
void or_bunching(const or_grid *g, const double *w, double *b_re, double *b_im)
{
    const double hx = grid_hx(g);
    double s = 0.0, sc = 0.0, ss = 0.0;
    for (int j = 0; j < g->np; ++j)
        for (int i = 0; i < g->nx; ++i) {
            const double ww = w[(long)j * g->nx + i];
            const double th = g->x0 + i * hx;
            s += ww;
            sc += ww * cos(th);
            ss += ww * sin(th);
        }
    *b_re = sc / s;
    *b_im = -ss / s;
}

/*
 * nsteps steps, ping-ponging between w (in/out) and a scratch array.
 * hist (may be NULL): 2 doubles per step, A^{n+1} (re, im) after each step.
 */
int or_run(const or_grid *g, int basis, int projection, const or_pusher *pu,
           double *fel, double *w, long nsteps, double *lost, double *hist)
{
    const long n = (long)g->nx * g->np;
    double *tmp = (double *)malloc(sizeof(double) * n);
    if (!tmp) return 3;
    for (long s = 0; s < nsteps; ++s) {
        int rc = or_step(g, basis, projection, pu, fel, w, tmp, lost);
        if (rc) { free(tmp); return rc; }
        memcpy(w, tmp, sizeof(double) * n);
        if (hist && (pu->kind == OR_FEL || pu->kind == OR_FEL_RK4)) {
            hist[2 * s] = fel[0];
            hist[2 * s + 1] = fel[1];
        }
    }
    free(tmp);
    return 0;
}

/*
 * Diagnostics of the weights (Sec. IV: sum of weights, entropy).
 * out[0]  sum w                     out[7]  energy: <H> (Hamiltonian pushers)
 * out[1]  mass = sum w hx hp                or <p> + |A|^2 (FEL)
 * out[2]  <x>                       out[8]  trapped mass, H < max V (pendulum)
 * out[3]  <p>                       out[9]  entropy -sum_{w>0} w ln w hx hp
 * out[4]  var x                     out[10] negative mass sum_{w<0} w hx hp
 * out[5]  var p                     out[11] b_re = Re <exp(-i x)>
 * out[6]  cov(x, p)                 out[12] b_im
 *                                   out[13] max |w|
 * a (FEL, may be NULL): [A_re, A_im].
 */
void or_moments(const or_grid *g, const or_pusher *pu, const double *w,
                const double *a, double *out)
{
    const double hx = grid_hx(g), hp = grid_hp(g);
    double s = 0, sx = 0, sp = 0, sxx = 0, spp = 0, sxp = 0, sh = 0, trapped = 0;
    double ent = 0, neg = 0, sc = 0, ss = 0, wmax = 0;
    const double hsep = fabs(pu->v_sign);
    for (int j = 0; j < g->np; ++j) {
        const double p = g->p0 + j * hp;
        for (int i = 0; i < g->nx; ++i) {
            const double x = g->x0 + i * hx;
            const double ww = w[(long)j * g->nx + i];
            const double hh = 0.5 * p * p + potential(pu, x);
            s += ww;
            sx += ww * x;
            sp += ww * p;
            sxx += ww * x * x;
            spp += ww * p * p;
            sxp += ww * x * p;
            sh += ww * hh;
            if (pu->kind == OR_KDK && pu->potential == OR_PEND && hh < hsep) trapped += ww;
            if (ww > 0) ent -= ww * log(ww);
            if (ww < 0) neg += ww;
            sc += ww * cos(x);
            ss += ww * sin(x);
            if (fabs(ww) > wmax) wmax = fabs(ww);
        }
    }
    const double mx = sx / s, mp = sp / s;
    out[0] = s;
    out[1] = s * hx * hp;
    out[2] = mx;
    out[3] = mp;
    out[4] = sxx / s - mx * mx;
    out[5] = spp / s - mp * mp;
    out[6] = sxp / s - mx * mp;
    if ((pu->kind == OR_FEL || pu->kind == OR_FEL_RK4))
        out[7] = mp + (a ? a[0] * a[0] + a[1] * a[1] : 0.0);
    else
        out[7] = sh / s;
    out[8] = trapped * hx * hp;
    out[9] = ent * hx * hp;
    out[10] = neg * hx * hp;
    out[11] = sc / s;
    out[12] = -ss / s;
    out[13] = wmax;
}

int or_nmom(void) { return OR_NMOM; }

/* ------------------------------------------------------ band-parallel step
 *
 * The same step as or_step, spread over host threads for timing on many cores,
 * with bitwise the same result: every target cell receives its contributions
 * in the serial order (sources in row-major order, then the tap loops), only
 * the target rows are split into bands, one per thread. A thread walks the
 * source rows whose pushed footprint reaches its band (found by a first
 * parallel pass over the source rows) and keeps the taps on its own rows. The
 * weight deposited beyond the momentum range (rows < 0 belong to the first
 * band, rows >= np to the last) is recorded per source in order and folded
 * serially in the serial order. The mass-matrix solves run row by row, then
 * column by column, each row or column with the serial arithmetic. The FEL
 * bunching is the serial sum. Supported: tent and cubic B-spline deposits,
 * Galerkin or lumped, every pusher but RK4, no space charge.
 */
#include <pthread.h>

typedef struct {
    long k;      /* source index */
    double v;    /* its contribution beyond the momentum range */
} or_lost_item;

typedef struct {
    const or_grid *g;
    int basis, projection;
    const or_pusher *pu;
    double k_re, k_im;
    const double *w_in;
    double *w_out;
    long *rlo, *rhi;          /* per source row: lowest and highest target row of its taps */
    int lo, hi;               /* rows (or columns) of this thread */
    int first, last;          /* the band takes the rows below 0 / from np up */
    or_lost_item *lost;
    long nlost, cap;
    int fail;
} or_task;

static void push_node(const or_task *t, double x, double p, double *u, double *v)
{
    const or_grid *g = t->g;
    double xf, pf;
    or_push(t->pu, t->k_re, t->k_im, x, p, &xf, &pf);
    *u = (xf - g->x0) / grid_hx(g);
    *v = (pf - g->p0) / grid_hp(g);
}

static void *pass_rows(void *arg)
{
    or_task *t = (or_task *)arg;
    const or_grid *g = t->g;
    const double radius = (t->basis == OR_TENT) ? 1.0 : 2.0;
    const double hx = grid_hx(g), hp = grid_hp(g);
    for (int j = t->lo; j < t->hi; ++j) {
        long mn = 0x7fffffffL, mx = -0x7fffffffL;
        for (int i = 0; i < g->nx; ++i) {
            if (t->w_in[(long)j * g->nx + i] == 0.0) continue;
            double u, v;
            push_node(t, g->x0 + i * hx, g->p0 + j * hp, &u, &v);
            const long r_lo = (long)ceil(v - radius), r_hi = (long)floor(v + radius);
            if (r_lo < mn) mn = r_lo;
            if (r_hi > mx) mx = r_hi;
        }
        t->rlo[j] = mn;
        t->rhi[j] = mx;
    }
    return NULL;
}

static void *pass_deposit(void *arg)
{
    or_task *t = (or_task *)arg;
    const or_grid *g = t->g;
    const int nx = g->nx, np = g->np;
    const double radius = (t->basis == OR_TENT) ? 1.0 : 2.0;
    const double hx = grid_hx(g), hp = grid_hp(g);
    const long blo = t->first ? -0x7fffffffL : t->lo, bhi = t->last ? 0x7fffffffL : t->hi;
    for (int j = 0; j < np; ++j) {
        if (t->rhi[j] < blo || t->rlo[j] >= bhi) continue;
        const double p = g->p0 + j * hp;
        for (int i = 0; i < nx; ++i) {
            const double w = t->w_in[(long)j * nx + i];
            if (w == 0.0) continue;
            double u, v;
            push_node(t, g->x0 + i * hx, p, &u, &v);
            const long c_lo = (long)ceil(u - radius), c_hi = (long)floor(u + radius);
            const long r_lo = (long)ceil(v - radius), r_hi = (long)floor(v + radius);
            for (long rr = r_lo; rr <= r_hi; ++rr) {
                if (rr < blo || rr >= bhi) continue;
                const double kp = hp * k_basis(t->basis, rr - v);
                if (kp == 0.0) continue;
                for (long cc = c_lo; cc <= c_hi; ++cc) {
                    const double kx = hx * k_basis(t->basis, cc - u);
                    const double contrib = kx * kp * w;
                    if (rr < 0 || rr >= np) {
                        if (t->nlost == t->cap) {
                            long nc = t->cap ? 2 * t->cap : 4096;
                            or_lost_item *nl = (or_lost_item *)realloc(t->lost, sizeof(or_lost_item) * nc);
                            if (!nl) { t->fail = 1; return NULL; }
                            t->lost = nl;
                            t->cap = nc;
                        }
                        t->lost[t->nlost].k = (long)j * nx + i;
                        t->lost[t->nlost].v = contrib;
                        t->nlost++;
                        continue;
                    }
                    t->w_out[rr * nx + mod_l(cc, nx)] += contrib;
                }
            }
        }
    }
    return NULL;
}

static void *pass_solve_x(void *arg)
{
    or_task *t = (or_task *)arg;
    const or_grid *g = t->g;
    const double hx = grid_hx(g);
    double *work = (double *)malloc(sizeof(double) * 4 * (size_t)g->nx);
    if (!work) { t->fail = 1; return NULL; }
    for (int j = t->lo; j < t->hi; ++j)
        cyclic_solve(g->nx, hx / 6.0, 2.0 * hx / 3.0, t->w_out + (long)j * g->nx, work);
    free(work);
    return NULL;
}

static void *pass_solve_p(void *arg)
{
    or_task *t = (or_task *)arg;
    const or_grid *g = t->g;
    const int nx = g->nx, np = g->np;
    const double hp = grid_hp(g);
    double *work = (double *)malloc(sizeof(double) * 3 * (size_t)np);
    if (!work) { t->fail = 1; return NULL; }
    double *bd = work, *cp = work + np, *col = work + 2 * np;
    for (int i = t->lo; i < t->hi; ++i) {
        for (int j = 0; j < np; ++j) {
            col[j] = t->w_out[(long)j * nx + i];
            bd[j] = 2.0 * hp / 3.0;
        }
        thomas(np, hp / 6.0, bd, hp / 6.0, col, cp);
        for (int j = 0; j < np; ++j) t->w_out[(long)j * nx + i] = col[j];
    }
    free(work);
    return NULL;
}

static void *pass_scale(void *arg)
{
    or_task *t = (or_task *)arg;
    const double inv = 1.0 / (grid_hx(t->g) * grid_hp(t->g));
    for (long k = (long)t->lo * t->g->nx; k < (long)t->hi * t->g->nx; ++k) t->w_out[k] *= inv;
    return NULL;
}

/* run fn over [0, n) split into nthreads contiguous parts */
static int run_parts(or_task *tasks, int nthreads, int n, void *(*fn)(void *))
{
    pthread_t th[256];
    for (int t = 0; t < nthreads; ++t) {
        tasks[t].lo = (int)((long)n * t / nthreads);
        tasks[t].hi = (int)((long)n * (t + 1) / nthreads);
        tasks[t].first = t == 0;
        tasks[t].last = t == nthreads - 1;
    }
    int started = 0;
    for (int t = 1; t < nthreads; ++t) {
        if (pthread_create(&th[t], NULL, fn, &tasks[t]) != 0) break;
        started = t;
    }
    fn(&tasks[0]);
    for (int t = 1; t <= started; ++t) pthread_join(th[t], NULL);
    for (int t = started + 1; t < nthreads; ++t) fn(&tasks[t]);   /* threads that did not start */
    for (int t = 0; t < nthreads; ++t)
        if (tasks[t].fail) return 1;
    return 0;
}

int or_step_par(const or_grid *g, int basis, int projection, const or_pusher *pu,
                double *fel, const double *w_in, double *w_out, double *lost, int nthreads)
{
    const int nx = g->nx, np = g->np;
    if (nx < 3 || np < 2) return 1;
    if (basis == OR_SEPTIC || pu->kind == OR_FEL_RK4 || (pu->kind == OR_FEL && pu->sigma2 != 0.0))
        return 4;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    const double hx = grid_hx(g), hp = grid_hp(g);
    const long n = (long)nx * np;
    double a_re = 0.0, a_im = 0.0;
    if (pu->kind == OR_FEL) {
        if (!fel) return 2;
        a_re = fel[0] + 0.5 * pu->dt * fel[2];
        a_im = fel[1] + 0.5 * pu->dt * fel[3];
    }
    or_task *tasks = (or_task *)calloc((size_t)nthreads, sizeof(or_task));
    long *rlo = (long *)malloc(sizeof(long) * 2 * (size_t)np);
    if (!tasks || !rlo) { free(tasks); free(rlo); return 3; }
    for (int t = 0; t < nthreads; ++t) {
        tasks[t].g = g;
        tasks[t].basis = basis;
        tasks[t].projection = projection;
        tasks[t].pu = pu;
        tasks[t].k_re = a_re;
        tasks[t].k_im = a_im;
        tasks[t].w_in = w_in;
        tasks[t].w_out = w_out;
        tasks[t].rlo = rlo;
        tasks[t].rhi = rlo + np;
    }
    memset(w_out, 0, sizeof(double) * n);
    int rc = run_parts(tasks, nthreads, np, pass_rows);
    if (!rc) rc = run_parts(tasks, nthreads, np, pass_deposit);
    /* lost weight in the serial order: by source, the first band's rows before the last's */
    double lost_acc = 0.0;
    if (!rc) {
        const or_task *a = &tasks[0], *b = &tasks[nthreads - 1];
        long ia = 0, ib = 0;
        if (nthreads == 1) {
            for (; ia < a->nlost; ++ia) lost_acc += a->lost[ia].v;
        } else {
            while (ia < a->nlost || ib < b->nlost) {
                if (ib >= b->nlost || (ia < a->nlost && a->lost[ia].k <= b->lost[ib].k))
                    lost_acc += a->lost[ia++].v;
                else
                    lost_acc += b->lost[ib++].v;
            }
        }
    }
    for (int t = 0; t < nthreads; ++t) free(tasks[t].lost);
    if (!rc) {
        if (basis == OR_CUBIC && projection == OR_GALERKIN) {
            rc = run_parts(tasks, nthreads, np, pass_solve_x);
            if (!rc) rc = run_parts(tasks, nthreads, nx, pass_solve_p);
        } else {
            rc = run_parts(tasks, nthreads, np, pass_scale);
        }
    }
    free(tasks);
    free(rlo);
    if (rc) return 3;
    if (lost) *lost += lost_acc / (hx * hp);
    if (pu->kind == OR_FEL) {
        double s = 0.0, sc = 0.0, ss = 0.0;
        for (int j = 0; j < np; ++j)
            for (int i = 0; i < nx; ++i) {
                const double w = w_out[(long)j * nx + i];
                const double th = g->x0 + i * hx;
                s += w;
                sc += w * cos(th);
                ss += w * sin(th);
            }
        fel[2] = sc / s;
        fel[3] = -ss / s;
        fel[0] = a_re + 0.5 * pu->dt * fel[2];
        fel[1] = a_im + 0.5 * pu->dt * fel[3];
    }
    return 0;
}
