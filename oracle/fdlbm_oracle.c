/*
 * fdlbm_oracle.c -- plain, slow, FP64 CPU oracle of one time step of the
 * two-dimensional 16-velocity (Kataoka-Tsutahara) multiple-relaxation-time
 * finite-difference lattice Boltzmann model with the flux-limiter convection
 * scheme (Chen, Xu, Zhang, Wang, "Two dimensional MRT LB model for
 * compressible and incompressible flows", arXiv:1305.4736).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent checker of the GPU
 * library.  Only tests, the smoke check and the CPU-baseline leg of the
 * benchmark may load it.  It shares no code, table or constant with the CUDA
 * path: the transformation matrix is built here densely from the Appendix
 * formulas and inverted here by Gauss-Jordan elimination, the limiter is the
 * literal theta/psi form, and every transform is a dense 16x16 product.
 *
 * What each function follows (paper sections / equations):
 *   velocities, eta_i ............ Sec. II (discrete velocity model, Fig. 1),
 *                                  Appendix A (eta_i = 5/2 for i = 1..4)
 *   transformation matrix M ...... Appendix A, rows m_1 .. m_16
 *   central matrix M* ............ Appendix A, rows m*_1 .. m*_16 (v -> v - u)
 *   equilibria f^eq_hat .......... Appendix A, closed forms k = 5..16;
 *                                  k = 1..4 are rho, j_x, j_y, e
 *   b, gamma, P, e ............... Sec. II: gamma = (b+2)/b, P = rho R T,
 *                                  e = b rho R T + rho u^2 (twice the energy)
 *   collision + energy-flux fix .. Eq. (3) and the modified S_88 / S_99
 *                                  collision of Sec. II
 *   forward-Euler FD update ...... Sec. III update equation (all terms at n)
 *   A_i .......................... Sec. III, A_i = 1, 1/6, 1/sqrt2, sqrt2/3
 *   limited fluxes F ............. Sec. III, outgoing / incoming x and y fluxes
 *   limiter psi, ratio theta ..... Sec. III flux limiter and smoothness ratio
 *   Lax-Wendroff / upwind ........ Sec. III: psi = 1 and psi = 0
 *   boundary ghosts .............. Sec. IV.A (fixed equilibrium ends,
 *                                  periodic y), Sec. IV.C (non-equilibrium
 *                                  extrapolation walls), Sec. V (inflow /
 *                                  outflow)
 *   Delta, Delta* ................ Sec. V: Delta = M (f - f^eq),
 *                                  Delta* = M* (f - f^eq)
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   R = 1.  theta with zero denominator -> psi = 0.  grad u by second-order
 *   central differences (ghost-cell u at the boundary).  Residuals of the
 *   conserved moments k = 1..4 are set to zero.  The energy-flux correction
 *   factor (s8/s5 - 1) is taken as 0 when s8 == s5.  Non-equilibrium
 *   extrapolation wall: mirror cell m of ghost g (-1 <-> 0, -2 <-> 1),
 *   rho_g = rho_m, u_g = 2 u_w - u_m, T_g = 2 T_w - T_m,
 *   f_g = f^eq(rho_g, u_g, T_g) + (f_m - f^eq(rho_m, u_m, T_m)).
 *   Convection is the unsplit projection: both x and y fluxes use f^n.
 *   Velocity order inside each "cyc" shell: (+,0), (0,+), (-,0), (0,-);
 *   diagonal shells: (+,+), (-,+), (-,-), (+,-).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NQ 16

enum { OR_BC_PERIODIC = 0, OR_BC_ZERO_GRADIENT = 1, OR_BC_EQUILIBRIUM = 2, OR_BC_NEQ_WALL = 3 };
enum { OR_LIM_MC = 0, OR_LIM_LW = 1, OR_LIM_UPWIND = 2 };

typedef struct {
    int nx, ny;          /* interior cells */
    int W, H;            /* nx + 4, ny + 4 (two ghost layers on each side) */
    double dx, dy, dt, b;
    double s[NQ];
    int limiter;
    int bc_kind[4];      /* 0 = x low, 1 = x high, 2 = y low, 3 = y high */
    double bc_state[4][4]; /* rho, u_x, u_y, T per edge */
    double vx[NQ], vy[NQ], eta[NQ], A[NQ];
    double M[NQ][NQ], Minv[NQ][NQ];
    double *f, *fn;      /* [NQ][H][W] */
} or_ctx;

/* ------------------------------------------------------------------------ */
/* Discrete velocity model (Sec. II) and eta_i (Appendix A).                 */
/* ------------------------------------------------------------------------ */
static void build_velocities(double vx[NQ], double vy[NQ], double eta[NQ], double A[NQ])
{
    const double r2 = sqrt(2.0);
    /* unit directions of the two axis shells and of the two diagonal shells */
    const double ax[4] = {1, 0, -1, 0}, ay[4] = {0, 1, 0, -1};
    const double dxs[4] = {1, -1, -1, 1}, dys[4] = {1, 1, -1, -1};
    for (int k = 0; k < 4; k++) {
        vx[k] = ax[k];                 vy[k] = ay[k];                 /* cyc(+-1, 0) */
        vx[4 + k] = 6.0 * ax[k];       vy[4 + k] = 6.0 * ay[k];       /* cyc(+-6, 0) */
        vx[8 + k] = r2 * dxs[k];       vy[8 + k] = r2 * dys[k];       /* sqrt2 (+-1, +-1) */
        vx[12 + k] = 3.0 / r2 * dxs[k]; vy[12 + k] = 3.0 / r2 * dys[k]; /* 3/sqrt2 (+-1, +-1) */
    }
    for (int i = 0; i < NQ; i++) eta[i] = (i < 4) ? 2.5 : 0.0;
    /* A_i of Sec. III */
    for (int i = 0; i < NQ; i++) {
        if (i < 4) A[i] = 1.0;
        else if (i < 8) A[i] = 1.0 / 6.0;
        else if (i < 12) A[i] = 1.0 / r2;
        else A[i] = r2 / 3.0;
    }
}

/* Rows m_1 .. m_16 of Appendix A, evaluated at velocity (x, y), eta. */
static void moment_row_values(double x, double y, double et, double m[NQ])
{
    const double v2 = x * x + y * y;      /* v_x^2 + v_y^2 */
    const double w = v2 + et * et;        /* v_x^2 + v_y^2 + eta^2 */
    const double d = x * x - y * y;       /* v_x^2 - v_y^2 */
    m[0] = 1.0;
    m[1] = x;
    m[2] = y;
    m[3] = w;
    m[4] = v2;
    m[5] = d;
    m[6] = x * y;
    m[7] = x * w;
    m[8] = y * w;
    m[9] = x * v2;
    m[10] = y * v2;
    m[11] = x * d;
    m[12] = y * d;
    m[13] = v2 * w;
    m[14] = x * y * w;
    m[15] = d * w;
}

static void build_M(const double vx[NQ], const double vy[NQ], const double eta[NQ], double M[NQ][NQ])
{
    for (int i = 0; i < NQ; i++) {
        double m[NQ];
        moment_row_values(vx[i], vy[i], eta[i], m);
        for (int k = 0; k < NQ; k++) M[k][i] = m[k];
    }
}

/* Gauss-Jordan elimination with partial pivoting in long double. Returns 0 on success. */
static int invert16(const double Ain[NQ][NQ], double Aout[NQ][NQ])
{
    long double a[NQ][2 * NQ];
    for (int r = 0; r < NQ; r++)
        for (int c = 0; c < 2 * NQ; c++)
            a[r][c] = (c < NQ) ? (long double)Ain[r][c] : (long double)((c - NQ) == r);
    for (int col = 0; col < NQ; col++) {
        int piv = col;
        for (int r = col + 1; r < NQ; r++)
            if (fabsl(a[r][col]) > fabsl(a[piv][col])) piv = r;
        if (a[piv][col] == 0.0L) return -1;
        if (piv != col)
            for (int c = 0; c < 2 * NQ; c++) { long double t = a[col][c]; a[col][c] = a[piv][c]; a[piv][c] = t; }
        long double p = a[col][col];
        for (int c = 0; c < 2 * NQ; c++) a[col][c] /= p;
        for (int r = 0; r < NQ; r++) {
            if (r == col) continue;
            long double fct = a[r][col];
            if (fct == 0.0L) continue;
            for (int c = 0; c < 2 * NQ; c++) a[r][c] -= fct * a[col][c];
        }
    }
    for (int r = 0; r < NQ; r++)
        for (int c = 0; c < NQ; c++) Aout[r][c] = (double)a[r][NQ + c];
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Equilibria in moment space (Appendix A).  Inputs rho, j = rho u, e, with  */
/* P = rho R T and R = 1, T = (e/rho - |u|^2)/b (Sec. II).                   */
/* ------------------------------------------------------------------------ */
static void feq_hat_from_conserved(double rho, double jx, double jy, double e, double b, double out[NQ])
{
    const double j2 = jx * jx + jy * jy;
    const double P = (e - j2 / rho) / b;       /* e = b P + |j|^2/rho */
    const double T = P / rho;                  /* R = 1 */
    out[0] = rho;
    out[1] = jx;
    out[2] = jy;
    out[3] = e;
    out[4] = 2.0 * P + j2 / rho;
    out[5] = (jx * jx - jy * jy) / rho;
    out[6] = jx * jy / rho;
    out[7] = (e + 2.0 * P) * jx / rho;
    out[8] = (e + 2.0 * P) * jy / rho;
    out[9] = (4.0 * P + jx * jx / rho + jy * jy / rho) * jx / rho;
    out[10] = (4.0 * P + jx * jx / rho + jy * jy / rho) * jy / rho;
    out[11] = (2.0 * P + jx * jx / rho - jy * jy / rho) * jx / rho;
    out[12] = (-2.0 * P + jx * jx / rho - jy * jy / rho) * jy / rho;
    out[13] = 2.0 * (b + 2.0) * rho * T * T + (6.0 + b) * T * j2 / rho + j2 * j2 / (rho * rho * rho);
    out[14] = ((b + 4.0) * P + j2 / rho) * jx * jy / (rho * rho);
    out[15] = ((b + 4.0) * P + j2 / rho) * (jx * jx - jy * jy) / (rho * rho);
}

static void feq_hat_from_primitive(double rho, double ux, double uy, double T, double b, double out[NQ])
{
    const double jx = rho * ux, jy = rho * uy;
    const double e = b * rho * T + rho * (ux * ux + uy * uy);
    feq_hat_from_conserved(rho, jx, jy, e, b, out);
}

static void matvec(const double A[NQ][NQ], const double x[NQ], double y[NQ])
{
    for (int r = 0; r < NQ; r++) {
        double acc = 0.0;
        for (int c = 0; c < NQ; c++) acc += A[r][c] * x[c];
        y[r] = acc;
    }
}

/* Conserved moments of a population vector: rho, j_x, j_y, e (Appendix A, first three relations). */
static void conserved(const or_ctx *c, const double f[NQ], double *rho, double *jx, double *jy, double *e)
{
    double r = 0, x = 0, y = 0, en = 0;
    for (int i = 0; i < NQ; i++) {
        r += f[i];
        x += f[i] * c->vx[i];
        y += f[i] * c->vy[i];
        en += f[i] * (c->vx[i] * c->vx[i] + c->vy[i] * c->vy[i] + c->eta[i] * c->eta[i]);
    }
    *rho = r; *jx = x; *jy = y; *e = en;
}

/* ------------------------------------------------------------------------ */
/* Grid access                                                               */
/* ------------------------------------------------------------------------ */
static inline size_t gidx(const or_ctx *c, int q, int ix, int iy)
{
    /* ix in [-2, nx+1], iy in [-2, ny+1] */
    return ((size_t)q * c->H + (size_t)(iy + 2)) * c->W + (size_t)(ix + 2);
}

static void load_cell(const or_ctx *c, const double *g, int ix, int iy, double f[NQ])
{
    for (int q = 0; q < NQ; q++) f[q] = g[gidx(c, q, ix, iy)];
}

static void store_cell(const or_ctx *c, double *g, int ix, int iy, const double f[NQ])
{
    for (int q = 0; q < NQ; q++) g[gidx(c, q, ix, iy)] = f[q];
}

static void feq_populations(const or_ctx *c, double rho, double ux, double uy, double T, double f[NQ])
{
    double fh[NQ];
    feq_hat_from_primitive(rho, ux, uy, T, c->b, fh);
    matvec(c->Minv, fh, f);
}

static void primitive_of(const or_ctx *c, const double f[NQ], double *rho, double *ux, double *uy, double *T)
{
    double r, jx, jy, e;
    conserved(c, f, &r, &jx, &jy, &e);
    *rho = r;
    *ux = jx / r;
    *uy = jy / r;
    *T = (e / r - (*ux) * (*ux) - (*uy) * (*uy)) / c->b;
}

/* ------------------------------------------------------------------------ */
/* Ghost cells: two layers per edge; x edges for interior rows, y edges for  */
/* interior columns (the stencil is a cross, corners are never read).        */
/* ------------------------------------------------------------------------ */
static void ghost_one(const or_ctx *c, double *g, int edge, int gx, int gy, int ix_in, int iy_in, int mx, int my)
{
    /* (gx, gy): ghost cell.  (ix_in, iy_in): source interior cell for
       periodic / zero-gradient.  (mx, my): mirror cell for the NEQ wall. */
    double f[NQ];
    const int kind = c->bc_kind[edge];
    const double *st = c->bc_state[edge];
    if (kind == OR_BC_PERIODIC || kind == OR_BC_ZERO_GRADIENT) {
        load_cell(c, g, ix_in, iy_in, f);
    } else if (kind == OR_BC_EQUILIBRIUM) {
        feq_populations(c, st[0], st[1], st[2], st[3], f);
    } else { /* OR_BC_NEQ_WALL */
        double fm[NQ], feqm[NQ], feqg[NQ];
        double rho_m, ux_m, uy_m, T_m;
        load_cell(c, g, mx, my, fm);
        primitive_of(c, fm, &rho_m, &ux_m, &uy_m, &T_m);
        feq_populations(c, rho_m, ux_m, uy_m, T_m, feqm);
        feq_populations(c, rho_m, 2.0 * st[1] - ux_m, 2.0 * st[2] - uy_m, 2.0 * st[3] - T_m, feqg);
        for (int q = 0; q < NQ; q++) f[q] = feqg[q] + (fm[q] - feqm[q]);
    }
    store_cell(c, g, gx, gy, f);
}

static int pmod(int a, int n) { int r = a % n; return r < 0 ? r + n : r; }

static void fill_ghosts(or_ctx *c, double *g)
{
    const int nx = c->nx, ny = c->ny;
    for (int iy = 0; iy < ny; iy++) {
        for (int k = 1; k <= 2; k++) {
            /* x low: ghost -k */
            int src = (c->bc_kind[0] == OR_BC_PERIODIC) ? pmod(-k, nx) : 0;
            ghost_one(c, g, 0, -k, iy, src, iy, (k - 1 < nx ? k - 1 : nx - 1), iy);
            /* x high: ghost nx-1+k */
            src = (c->bc_kind[1] == OR_BC_PERIODIC) ? pmod(nx - 1 + k, nx) : nx - 1;
            ghost_one(c, g, 1, nx - 1 + k, iy, src, iy, (nx - k >= 0 ? nx - k : 0), iy);
        }
    }
    for (int ix = 0; ix < nx; ix++) {
        for (int k = 1; k <= 2; k++) {
            int src = (c->bc_kind[2] == OR_BC_PERIODIC) ? pmod(-k, ny) : 0;
            ghost_one(c, g, 2, ix, -k, ix, src, ix, (k - 1 < ny ? k - 1 : ny - 1));
            src = (c->bc_kind[3] == OR_BC_PERIODIC) ? pmod(ny - 1 + k, ny) : ny - 1;
            ghost_one(c, g, 3, ix, ny - 1 + k, ix, src, ix, (ny - k >= 0 ? ny - k : 0));
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Flux limiter (Sec. III)                                                   */
/* ------------------------------------------------------------------------ */
static double psi_of_theta(double theta)
{
    if (theta <= 0.0) return 0.0;
    if (theta <= 1.0 / 3.0) return 2.0 * theta;
    if (theta <= 3.0) return 0.5 * (1.0 + theta);
    return 2.0;
}

/* psi at node J for a population moving with sign sigma along the axis:
   theta = (f_J - f_{J-sigma}) / (f_{J+sigma} - f_J); psi = 0 for a zero denominator. */
static double limiter_psi(int limiter, double f_minus, double f_0, double f_plus)
{
    if (limiter == OR_LIM_LW) return 1.0;
    if (limiter == OR_LIM_UPWIND) return 0.0;
    const double den = f_plus - f_0;
    if (den == 0.0) return 0.0;
    return psi_of_theta((f_0 - f_minus) / den);
}

/* ------------------------------------------------------------------------ */
/* One time step                                                             */
/* ------------------------------------------------------------------------ */
static void velocity_at(const or_ctx *c, const double *g, int ix, int iy, double *ux, double *uy)
{
    double f[NQ], r, jx, jy, e;
    load_cell(c, g, ix, iy, f);
    conserved(c, f, &r, &jx, &jy, &e);
    *ux = jx / r;
    *uy = jy / r;
}

/* Collision term C = M^-1 S_hat (f_hat - f_hat^eq) with the energy-flux
   correction of Sec. II on rows 8 and 9 (1-based).  grad = {dux/dx, dux/dy,
   duy/dx, duy/dy}. */
static void collision_term(const or_ctx *c, const double f[NQ], const double grad[4], double C[NQ])
{
    double rho, jx, jy, e, fh[NQ], fe[NQ], r[NQ];
    conserved(c, f, &rho, &jx, &jy, &e);
    matvec(c->M, f, fh);
    feq_hat_from_conserved(rho, jx, jy, e, c->b, fe);
    for (int k = 0; k < 4; k++) r[k] = 0.0;             /* conserved moments */
    for (int k = 4; k < NQ; k++) r[k] = c->s[k] * (fh[k] - fe[k]);
    const double ux = jx / rho, uy = jy / rho;
    const double P = (e - (jx * jx + jy * jy) / rho) / c->b;  /* rho T, R = 1 */
    const double dxux = grad[0], dyux = grad[1], dxuy = grad[2], dyuy = grad[3];
    const double b = c->b;
    const double k8 = (c->s[7] == c->s[4]) ? 0.0 : c->s[7] / c->s[4] - 1.0;
    const double k9 = (c->s[8] == c->s[4]) ? 0.0 : c->s[8] / c->s[4] - 1.0;
    r[7] += k8 * P * ux * (4.0 * dxux - 4.0 / b * dxux - 4.0 / b * dyuy)
          + k8 * P * uy * (2.0 * dxuy + 2.0 * dyux);
    r[8] += k9 * P * ux * (2.0 * dxuy + 2.0 * dyux)
          + k9 * P * uy * (4.0 * dyuy - 4.0 / b * dxux - 4.0 / b * dyuy);
    matvec(c->Minv, r, C);
}

static void update_interior(or_ctx *c)
{
    const int nx = c->nx, ny = c->ny;
    /* Flow velocity of every cell the central differences read: the interior
       rows over x in [-1, nx], and rows -1 and ny over the interior columns. */
    const size_t plane = (size_t)c->W * c->H;
    double *U = (double *)malloc(2 * plane * sizeof(double));
    if (!U) abort();
    double *UX = U, *UY = U + plane;
#pragma omp parallel for collapse(2) schedule(static)
    for (int iy = -1; iy <= ny; iy++) {
        for (int ix = -1; ix <= nx; ix++) {
            const int in_x = (ix >= 0 && ix < nx), in_y = (iy >= 0 && iy < ny);
            if (!in_x && !in_y) continue;                 /* corner: never read */
            const size_t k = (size_t)(iy + 2) * c->W + (size_t)(ix + 2);
            velocity_at(c, c->f, ix, iy, &UX[k], &UY[k]);
        }
    }
#define UAT(A, X, Y) A[(size_t)((Y) + 2) * c->W + (size_t)((X) + 2)]
#pragma omp parallel for collapse(2) schedule(static)
    for (int iy = 0; iy < ny; iy++) {
        for (int ix = 0; ix < nx; ix++) {
            double f[NQ], C[NQ], grad[4];
            load_cell(c, c->f, ix, iy, f);
            grad[0] = (UAT(UX, ix + 1, iy) - UAT(UX, ix - 1, iy)) / (2.0 * c->dx);
            grad[1] = (UAT(UX, ix, iy + 1) - UAT(UX, ix, iy - 1)) / (2.0 * c->dy);
            grad[2] = (UAT(UY, ix + 1, iy) - UAT(UY, ix - 1, iy)) / (2.0 * c->dx);
            grad[3] = (UAT(UY, ix, iy + 1) - UAT(UY, ix, iy - 1)) / (2.0 * c->dy);
            collision_term(c, f, grad, C);
            for (int i = 0; i < NQ; i++) {
                double conv = 0.0;
                for (int a = 0; a < 2; a++) {
                    const double v = (a == 0) ? c->vx[i] : c->vy[i];
                    if (v == 0.0) continue;                 /* zero shift: F_out = F_in */
                    const int sg = (v > 0.0) ? 1 : -1;      /* A_i v_ia = +-1 */
                    const int ox = (a == 0) ? sg : 0, oy = (a == 1) ? sg : 0;
                    const double cr = c->dt / (c->A[i] * ((a == 0) ? c->dx : c->dy));
                    const double fJp = c->f[gidx(c, i, ix + ox, iy + oy)];
                    const double fJ = c->f[gidx(c, i, ix, iy)];
                    const double fJm = c->f[gidx(c, i, ix - ox, iy - oy)];
                    const double fJmm = c->f[gidx(c, i, ix - 2 * ox, iy - 2 * oy)];
                    const double psiJ = limiter_psi(c->limiter, fJm, fJ, fJp);
                    const double psiJm = limiter_psi(c->limiter, fJmm, fJm, fJ);
                    const double Fout = fJ + 0.5 * (1.0 - cr) * (fJp - fJ) * psiJ;
                    const double Fin = fJm + 0.5 * (1.0 - cr) * (fJ - fJm) * psiJm;
                    conv += cr * (Fout - Fin);
                }
                c->fn[gidx(c, i, ix, iy)] = f[i] - conv - c->dt * C[i];
            }
        }
    }
#undef UAT
    free(U);
}

static void step_once(or_ctx *c)
{
    fill_ghosts(c, c->f);
    update_interior(c);
    double *t = c->f; c->f = c->fn; c->fn = t;
}

/* ------------------------------------------------------------------------ */
/* Public (test-only) interface                                              */
/* ------------------------------------------------------------------------ */
void or_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int or_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Dense M and M^-1 (row-major 16x16), plus velocities and eta. */
int or_matrices(double *M, double *Minv, double *vx, double *vy, double *eta)
{
    double v1[NQ], v2[NQ], e[NQ], A[NQ], m[NQ][NQ], mi[NQ][NQ];
    build_velocities(v1, v2, e, A);
    build_M(v1, v2, e, m);
    if (invert16(m, mi)) return -1;
    for (int r = 0; r < NQ; r++)
        for (int c = 0; c < NQ; c++) { if (M) M[r * NQ + c] = m[r][c]; if (Minv) Minv[r * NQ + c] = mi[r][c]; }
    for (int i = 0; i < NQ; i++) { if (vx) vx[i] = v1[i]; if (vy) vy[i] = v2[i]; if (eta) eta[i] = e[i]; }
    return 0;
}

/* Central matrix M* at flow velocity (ux, uy) (Appendix A, v -> v - u). */
void or_central_matrix(double ux, double uy, double *Mstar)
{
    double v1[NQ], v2[NQ], e[NQ], A[NQ];
    build_velocities(v1, v2, e, A);
    for (int i = 0; i < NQ; i++) {
        double m[NQ];
        moment_row_values(v1[i] - ux, v2[i] - uy, e[i], m);
        for (int k = 0; k < NQ; k++) Mstar[k * NQ + i] = m[k];
    }
}

void or_feq_hat(double rho, double ux, double uy, double T, double b, double *out)
{
    feq_hat_from_primitive(rho, ux, uy, T, b, out);
}

/* f^eq = M^-1 f^eq_hat for one state. */
int or_feq(double rho, double ux, double uy, double T, double b, double *out)
{
    double v1[NQ], v2[NQ], e[NQ], A[NQ], m[NQ][NQ], mi[NQ][NQ], fh[NQ];
    build_velocities(v1, v2, e, A);
    build_M(v1, v2, e, m);
    if (invert16(m, mi)) return -1;
    feq_hat_from_primitive(rho, ux, uy, T, b, fh);
    matvec(mi, fh, out);
    return 0;
}

/* The psi(theta) function alone, for pins of the limiter. */
double or_psi(double theta) { return psi_of_theta(theta); }

or_ctx *or_create(int nx, int ny, double dx, double dy, double dt, double gamma, const double *s,
                  int limiter, const int *bc_kind, const double *bc_state)
{
    if (nx < 1 || ny < 1 || !(dx > 0) || !(dy > 0) || !(dt > 0) || !(gamma > 1.0)) return NULL;
    or_ctx *c = (or_ctx *)calloc(1, sizeof(or_ctx));
    if (!c) return NULL;
    c->nx = nx; c->ny = ny; c->W = nx + 4; c->H = ny + 4;
    c->dx = dx; c->dy = dy; c->dt = dt;
    c->b = 2.0 / (gamma - 1.0);          /* gamma = (b+2)/b */
    for (int k = 0; k < NQ; k++) c->s[k] = s[k];
    c->limiter = limiter;
    for (int e = 0; e < 4; e++) {
        c->bc_kind[e] = bc_kind[e];
        for (int k = 0; k < 4; k++) c->bc_state[e][k] = bc_state[4 * e + k];
    }
    build_velocities(c->vx, c->vy, c->eta, c->A);
    build_M(c->vx, c->vy, c->eta, c->M);
    if (invert16(c->M, c->Minv)) { free(c); return NULL; }
    const size_t n = (size_t)NQ * c->W * c->H;
    c->f = (double *)calloc(n, sizeof(double));
    c->fn = (double *)calloc(n, sizeof(double));
    if (!c->f || !c->fn) { free(c->f); free(c->fn); free(c); return NULL; }
    return c;
}

void or_destroy(or_ctx *c)
{
    if (!c) return;
    free(c->f); free(c->fn); free(c);
}

/* Initialise every interior cell to f = M^-1 f^eq_hat(rho, u, v, T); inputs [ny][nx]. */
void or_init(or_ctx *c, const double *rho, const double *ux, const double *uy, const double *T)
{
    for (int iy = 0; iy < c->ny; iy++)
        for (int ix = 0; ix < c->nx; ix++) {
            const size_t k = (size_t)iy * c->nx + ix;
            double f[NQ];
            feq_populations(c, rho[k], ux[k], uy[k], T[k], f);
            store_cell(c, c->f, ix, iy, f);
        }
}

void or_step(or_ctx *c, int n)
{
    for (int s = 0; s < n; s++) step_once(c);
}

/* Interior populations in [16][ny][nx] order. */
void or_get_state(const or_ctx *c, double *out)
{
    for (int q = 0; q < NQ; q++)
        for (int iy = 0; iy < c->ny; iy++)
            for (int ix = 0; ix < c->nx; ix++)
                out[((size_t)q * c->ny + iy) * c->nx + ix] = c->f[gidx(c, q, ix, iy)];
}

void or_set_state(or_ctx *c, const double *in)
{
    for (int q = 0; q < NQ; q++)
        for (int iy = 0; iy < c->ny; iy++)
            for (int ix = 0; ix < c->nx; ix++)
                c->f[gidx(c, q, ix, iy)] = in[((size_t)q * c->ny + iy) * c->nx + ix];
}

/* Macroscopic fields and Delta = M f - f^eq_hat (Sec. V).  Any output may be NULL.
   delta is [16][ny][nx]. */
void or_moments(const or_ctx *c, double *rho, double *ux, double *uy, double *T, double *delta)
{
    for (int iy = 0; iy < c->ny; iy++)
        for (int ix = 0; ix < c->nx; ix++) {
            const size_t k = (size_t)iy * c->nx + ix;
            double f[NQ], r, x, y, t;
            load_cell(c, c->f, ix, iy, f);
            primitive_of(c, f, &r, &x, &y, &t);
            if (rho) rho[k] = r;
            if (ux) ux[k] = x;
            if (uy) uy[k] = y;
            if (T) T[k] = t;
            if (delta) {
                double rr, jx, jy, e, fh[NQ], fe[NQ];
                conserved(c, f, &rr, &jx, &jy, &e);
                matvec(c->M, f, fh);
                feq_hat_from_conserved(rr, jx, jy, e, c->b, fe);
                for (int q = 0; q < NQ; q++) delta[(size_t)q * c->ny * c->nx + k] = fh[q] - fe[q];
            }
        }
}

/* Delta* = M*(f - f^eq) with M* built at the cell's own flow velocity (Sec. V, Appendix A). */
void or_moments_central(const or_ctx *c, double *delta_star)
{
    for (int iy = 0; iy < c->ny; iy++)
        for (int ix = 0; ix < c->nx; ix++) {
            const size_t k = (size_t)iy * c->nx + ix;
            double f[NQ], r, x, y, t, feq[NQ], d[NQ], Ms[NQ * NQ];
            load_cell(c, c->f, ix, iy, f);
            primitive_of(c, f, &r, &x, &y, &t);
            feq_populations(c, r, x, y, t, feq);
            for (int q = 0; q < NQ; q++) d[q] = f[q] - feq[q];
            or_central_matrix(x, y, Ms);
            for (int row = 0; row < NQ; row++) {
                double acc = 0.0;
                for (int q = 0; q < NQ; q++) acc += Ms[row * NQ + q] * d[q];
                delta_star[(size_t)row * c->ny * c->nx + k] = acc;
            }
        }
}

/* Domain totals of rho, j_x, j_y, e (each times dx dy). */
void or_totals(const or_ctx *c, double *out)
{
    double t[4] = {0, 0, 0, 0};
    for (int iy = 0; iy < c->ny; iy++)
        for (int ix = 0; ix < c->nx; ix++) {
            double f[NQ], r, jx, jy, e;
            load_cell(c, c->f, ix, iy, f);
            conserved(c, f, &r, &jx, &jy, &e);
            t[0] += r; t[1] += jx; t[2] += jy; t[3] += e;
        }
    for (int k = 0; k < 4; k++) out[k] = t[k] * c->dx * c->dy;
}

/* Collision term C = M^-1 S_hat (f_hat - f_hat^eq) (with the energy-flux
   correction) of one cell, for the conservation pins.  grad = {dux/dx,
   dux/dy, duy/dx, duy/dy}. */
void or_collision(const double *f, const double *s, double gamma, const double *grad, double *C)
{
    or_ctx c;
    memset(&c, 0, sizeof(c));
    c.b = 2.0 / (gamma - 1.0);
    for (int k = 0; k < NQ; k++) c.s[k] = s[k];
    build_velocities(c.vx, c.vy, c.eta, c.A);
    build_M(c.vx, c.vy, c.eta, c.M);
    invert16(c.M, c.Minv);
    collision_term(&c, f, grad, C);
}

/* Update of one cell from its 5 x 5 neighbourhood at time n: patch is
   [16][5][5] (row = y offset -2..2, column = x offset -2..2; the corners are
   never read).  out receives the 16 populations at time n+1.  This is the
   interior update of a 1 x 1 grid whose ghost cells are the patch. */
int or_update_patch(const double *patch, double dx, double dy, double dt, double gamma,
                    const double *s, int limiter, double *out)
{
    int kinds[4] = {0, 0, 0, 0};
    double st[16] = {0};
    or_ctx *c = or_create(1, 1, dx, dy, dt, gamma, s, limiter, kinds, st);
    if (!c) return -1;
    memcpy(c->f, patch, sizeof(double) * NQ * 25);
    update_interior(c);
    for (int q = 0; q < NQ; q++) out[q] = c->fn[gidx(c, q, 0, 0)];
    or_destroy(c);
    return 0;
}
