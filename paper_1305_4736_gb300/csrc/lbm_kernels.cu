// lbm_kernels.cu -- CUDA kernels of the D2V16 MRT flux-limiter FDLBM step (sm_103a).
//
//   k_ghost    ghost cells of every edge (Sec. IV.A, IV.C, V)
//   k_step     fused step: local rho/u on the tile + 1 ring, central-difference
//              grad u, MRT collision with the energy-flux correction (Eq. 3,
//              Sec. II), flux-limited x and y convection and the forward-Euler
//              update of Sec. III, one write per population
//   k_init     f = M^-1 f_hat^eq(rho, u, v, T) per cell (Appendix A)
//   k_moments  rho, u, v, T, Delta = M f - f_hat^eq, Delta* = M*(f - f^eq) (Sec. V)
//   k_totals_* deterministic two-pass float64 totals of rho, j, e
//   k_pack / k_unpack  interior populations to / from a dense float64 buffer
//
// Storage: population planes of (ny + 4) rows by `pitch` columns; interior cell
// (x, y) at row y + 2, column x + 4.  R = double stores f in 16 planes; R = float
// stores g = f - f^eq0 (deviation mode) in 8 planes of population pairs (pidx).
#include "lbm_internal.h"

namespace lbm {

__device__ __forceinline__ constexpr int sgn_x(int q)
{
    return q < 8 ? ((q & 3) == 0 ? 1 : ((q & 3) == 2 ? -1 : 0)) : (((q & 3) == 0 || (q & 3) == 3) ? 1 : -1);
}
__device__ __forceinline__ constexpr int sgn_y(int q)
{
    return q < 8 ? ((q & 3) == 1 ? 1 : ((q & 3) == 3 ? -1 : 0)) : (((q & 3) <= 1) ? 1 : -1);
}

// Cells whose flow velocity the central differences of an interior cell read:
// the interior plus the first ghost layer of the cross (never a corner).
__device__ __forceinline__ bool u_cell(int x, int y, int nx, int ny)
{
    return (x >= -1 && x <= nx && y >= 0 && y < ny) || (y >= -1 && y <= ny && x >= 0 && x < nx);
}

template <typename R>
__device__ __forceinline__ R pick(double d, float f);
template <> __device__ __forceinline__ double pick<double>(double d, float) { return d; }
template <> __device__ __forceinline__ float pick<float>(double, float f) { return f; }

__device__ __forceinline__ void load16(const double *__restrict__ f, long long plane, long long c, double *out)
{
#pragma unroll
    for (int q = 0; q < NQ; q++) out[q] = f[q * plane + c];
}

__device__ __forceinline__ void load16(const float *__restrict__ f, long long plane, long long c, float *out)
{
    const float2 *f2p = reinterpret_cast<const float2 *>(f);
#pragma unroll
    for (int pr = 0; pr < 8; pr++) {
        const float2 v = f2p[pr * plane + c];
        out[pair_q(pr)] = v.x;
        out[pair_q(pr) + 4] = v.y;
    }
}

template <typename R, bool Dev>
__device__ __forceinline__ void velocity_of(const Params &P, const R *f, R &ux, R &uy)
{
    const Shells<R> s = shells_of(f);
    R drho, jx, jy, de;
    conserved_of(s, drho, jx, jy, de);
    const R rho = Dev ? coef<R>(P).rho0 + drho : drho;
    const R ir = recip(rho);
    ux = jx * ir;
    uy = jy * ir;
}

// ---------------------------------------------------------------------------
// Fused step (plain form): one thread per cell of a tile of TX x TY cells (TX a power
// of two, TX * TY = threads per CTA); the flow velocity of the tile + 1 ring goes
// through shared memory, the limiter reads its stencil from global memory (L1 / L2).
// Grids narrower than 32 columns use TX = the smallest power of two >= nx, so that
// every lane of a warp has a cell (GB300's float64 unit charges each warp instruction
// for all 32 lanes).  The tile body is shared by the single-grid kernel and the
// batched kernel (which walks a tile work list).
// ---------------------------------------------------------------------------
template <typename R, bool Dev, int Lim>
__device__ __forceinline__ void step_tile(const Params &P, const R *__restrict__ fin, R *__restrict__ fout,
                                          int x0, int y0, int TX, int log_tx, int TY, R *su, R *sv)
{
    const int tid = threadIdx.x, nthreads = blockDim.x;
    const int tx = tid & (TX - 1), ty = tid >> log_tx;
    const int W = TX + 2;                              // row stride of su, sv
    const int ix = x0 + tx, iy = y0 + ty;
    const int nx = P.nx, ny = P.ny, pitch = P.pitch;
    const long long plane = P.plane;
    const bool inside = (ix < nx) && (iy < ny);
    const long long c0 = (long long)(iy + OY) * pitch + (ix + OX);

    R f[NQ];
    Shells<R> sh;
    R drho = R(0), jx = R(0), jy = R(0), de = R(0), ir = R(1);
    if (inside) {
        load16(fin, plane, c0, f);
        sh = shells_of(f);
        conserved_of(sh, drho, jx, jy, de);
        const R rho = Dev ? coef<R>(P).rho0 + drho : drho;
        ir = recip(rho);
        su[(ty + 1) * W + tx + 1] = jx * ir;
        sv[(ty + 1) * W + tx + 1] = jy * ir;
    } else if (u_cell(ix, iy, nx, ny)) {
        R g[NQ];
        load16(fin, plane, c0, g);
        R a, b;
        velocity_of<R, Dev>(P, g, a, b);
        su[(ty + 1) * W + tx + 1] = a;
        sv[(ty + 1) * W + tx + 1] = b;
    }
    // ring of the tile: bottom row, top row, left column, right column
    for (int t = tid; t < 2 * (TX + TY); t += nthreads) {
        int rx, ry, lx, ly;
        if (t < TX) { rx = x0 + t; ry = y0 - 1; lx = t + 1; ly = 0; }
        else if (t < 2 * TX) { rx = x0 + t - TX; ry = y0 + TY; lx = t - TX + 1; ly = TY + 1; }
        else if (t < 2 * TX + TY) { rx = x0 - 1; ry = y0 + t - 2 * TX; lx = 0; ly = t - 2 * TX + 1; }
        else { rx = x0 + TX; ry = y0 + t - 2 * TX - TY; lx = TX + 1; ly = t - 2 * TX - TY + 1; }
        if (u_cell(rx, ry, nx, ny)) {
            R g[NQ];
            load16(fin, plane, (long long)(ry + OY) * pitch + (rx + OX), g);
            R a, b;
            velocity_of<R, Dev>(P, g, a, b);
            su[ly * W + lx] = a;
            sv[ly * W + lx] = b;
        }
    }
    __syncthreads();
    if (inside) {
        // central differences (the 1/(2 dx) factor is folded into q8, q9)
        const int k = (ty + 1) * W + tx + 1;
        const R dxux = su[k + 1] - su[k - 1];
        const R dyux = su[k + W] - su[k - W];
        const R dxuy = sv[k + 1] - sv[k - 1];
        const R dyuy = sv[k + W] - sv[k - W];

        R acc[NQ];
        collide<R, Dev>(P, sh, drho, jx, jy, de, ir, jx * ir, jy * ir, dxux, dyux, dxuy, dyuy, acc);
#pragma unroll
        for (int q = 0; q < NQ; q++) acc[q] = f[q] - acc[q];

        // limited convection: x and y projections, both from f^n (Sec. III)
        const Coef<R> &C = coef<R>(P);
#pragma unroll
        for (int q = 0; q < NQ; q++) {
            const int sx = sgn_x(q), sy = sgn_y(q);
            const int shell = q >> 2;
            auto at = [&](long long c) { return fin[pidx<R>(q, plane, c)]; };
            // sum over the axes of c_alpha (F_out - F_in) (Courant number and h/2 per axis)
            R conv = R(0);
            if (sx != 0)
                conv = C.cr[shell] * flux_diff<R, Lim>(at(c0 - 2 * sx), at(c0 - sx), f[q], at(c0 + sx), C.hh[shell]);
            if (sy != 0) {
                const long long sp = (long long)sy * pitch;
                const R ty_ = flux_diff<R, Lim>(at(c0 - 2 * sp), at(c0 - sp), f[q], at(c0 + sp), C.hhy[shell]);
                conv = sx != 0 ? conv + C.cry[shell] * ty_ : C.cry[shell] * ty_;
            }
            fout[pidx<R>(q, plane, c0)] = acc[q] - conv;
        }
    }
}

template <typename R, bool Dev, int Lim, int NT>
__global__ void __launch_bounds__(NT)
k_step(const __grid_constant__ Params P, const R *__restrict__ fin, R *__restrict__ fout, int TX, int log_tx)
{
    extern __shared__ __align__(16) unsigned char smem_plain[];
    const int TY = NT / TX;
    R *su = reinterpret_cast<R *>(smem_plain);
    R *sv = su + (TX + 2) * (TY + 2);
    step_tile<R, Dev, Lim>(P, fin, fout, blockIdx.x * TX, blockIdx.y * TY, TX, log_tx, TY, su, sv);
}

static_assert(sizeof(Params) % sizeof(int4) == 0, "Params is copied to shared memory as int4 words");

// Batched step: persistent CTAs of NT threads walk contiguous shares of a tile list spanning
// many grids; each
// tile (int4 {grid, x0, y0, log2 TX}) names its grid, whose parameter block is copied into
// shared memory when the grid changes, and its width (TY = NT / TX).  `phase` selects which
// of the two buffers is the input.  float64 groups use NT = 64: GB300 executes float64 at
// about 1.6 lane operations per cycle per SM, so small tiles spread a small grid's work over
// more SMs; float32 groups use NT = 256.
template <typename R, bool Dev, int Lim, int NT>
__global__ void __launch_bounds__(NT)
k_step_batch(const Params *__restrict__ Pall, const BatchGrid *__restrict__ G, const int4 *__restrict__ tiles,
             int ntiles, int phase)
{
    constexpr int kSmem = 3 * (NT + 2);            // max over TX of (TX + 2)(TY + 2), at TX = 1
    __shared__ R su[kSmem];
    __shared__ R sv[kSmem];
    __shared__ __align__(16) Params Ps;
    int cur_grid = -1;
    const int tid = threadIdx.x;
    // a contiguous share of the tile list per CTA: the tiles of a grid are adjacent in the
    // list, so a CTA reloads the parameter block about once per grid it touches
    const int t0 = (int)((long long)ntiles * blockIdx.x / gridDim.x);
    const int t1 = (int)((long long)ntiles * (blockIdx.x + 1) / gridDim.x);
    for (int t = t0; t < t1; t++) {
        const int4 tl = tiles[t];
        __syncthreads();                             // the previous tile is done with su, sv, Ps
        if (tl.x != cur_grid) {
            const int4 *src = reinterpret_cast<const int4 *>(Pall + tl.x);
            int4 *dst = reinterpret_cast<int4 *>(&Ps);
            for (int k = tid; k < (int)(sizeof(Params) / sizeof(int4)); k += NT) dst[k] = src[k];
            cur_grid = tl.x;
            __syncthreads();
        }
        const BatchGrid g = G[tl.x];
        const int in = g.cur ^ phase;
        const int TX = 1 << tl.w;
        step_tile<R, Dev, Lim>(Ps, (const R *)g.buf[in], (R *)g.buf[in ^ 1], tl.y, tl.z, TX, tl.w, NT / TX, su,
                               sv);
    }
}

// ---------------------------------------------------------------------------
// Ghost cells.  One thread per ghost cell: x edges cover the interior rows,
// y edges the interior columns (the stencil is a cross; corners are unused).
// ---------------------------------------------------------------------------
template <typename R, bool Dev>
__device__ __forceinline__ void ghost_cell(const Params &P, R *__restrict__ f, int idx)
{
    const int nx = P.nx, ny = P.ny;
    const long long plane = P.plane;
    const int n_x = 4 * ny, n_all = 4 * ny + 4 * nx;
    if (idx >= n_all) return;
    int edge, gx, gy, sx, sy, mx, my, n, k, along;
    if (idx < n_x) {
        edge = idx / (2 * ny);            // 0 = x-lo, 1 = x-hi
        const int r = idx % (2 * ny);
        k = r / ny + 1;                   // ghost layer 1 or 2
        along = r % ny;
        n = nx;
        gy = sy = my = along;
        if (edge == 0) { gx = -k; mx = k - 1; } else { gx = nx - 1 + k; mx = nx - k; }
        const int kind = P.edge[edge].kind;
        if (kind <= 1 && ((nx | P.pitch | (int)(plane & 1)) & 1) == 0) {
            // periodic / zero gradient with even nx, pitch and plane: the layer-1 thread copies
            // both ghost columns of its row, 16 bytes per population (pair) plane.  Ghost columns
            // x-lo: -2, -1 <- nx-2, nx-1 (periodic) or 0, 0; x-hi: nx, nx+1 <- 0, 1 or nx-1, nx-1.
            if (k == 2) return;
            const long long row = (long long)(along + OY) * P.pitch;
            const long long cg2 = row + (edge == 0 ? OX - 2 : nx + OX);
            if (kind == 0) {
                const long long cs2 = row + (edge == 0 ? nx - 2 + OX : OX);
                if constexpr (sizeof(R) == sizeof(float)) {
                    float2 *f2p = reinterpret_cast<float2 *>(f);
#pragma unroll
                    for (int pr = 0; pr < 8; pr++)
                        *reinterpret_cast<float4 *>(f2p + pr * plane + cg2) =
                            *reinterpret_cast<const float4 *>(f2p + pr * plane + cs2);
                } else {
#pragma unroll
                    for (int q = 0; q < NQ; q++)
                        *reinterpret_cast<double2 *>(f + q * plane + cg2) =
                            *reinterpret_cast<const double2 *>(f + q * plane + cs2);
                }
            } else {
                const long long cs = row + (edge == 0 ? OX : nx - 1 + OX);
                if constexpr (sizeof(R) == sizeof(float)) {
                    float2 *f2p = reinterpret_cast<float2 *>(f);
#pragma unroll
                    for (int pr = 0; pr < 8; pr++) {
                        const float2 v = f2p[pr * plane + cs];
                        *reinterpret_cast<float4 *>(f2p + pr * plane + cg2) = make_float4(v.x, v.y, v.x, v.y);
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < NQ; q++) {
                        const double v = f[q * plane + cs];
                        *reinterpret_cast<double2 *>(f + q * plane + cg2) = make_double2(v, v);
                    }
                }
            }
            return;
        }
        sx = (kind == 0) ? ((gx % n) + n) % n : (edge == 0 ? 0 : nx - 1);
    } else {
        const int j = idx - n_x;
        edge = 2 + j / (2 * nx);          // 2 = y-lo, 3 = y-hi
        const int r = j % (2 * nx);
        k = r / nx + 1;
        along = r % nx;
        n = ny;
        gx = sx = mx = along;
        if (edge == 2) { gy = -k; my = k - 1; } else { gy = ny - 1 + k; my = ny - k; }
        const int kind = P.edge[edge].kind;
        sy = (kind == 0) ? ((gy % n) + n) % n : (edge == 2 ? 0 : ny - 1);
    }
    mx = mx < 0 ? 0 : (mx >= nx ? nx - 1 : mx);
    my = my < 0 ? 0 : (my >= ny ? ny - 1 : my);
    const EdgeDev &E = P.edge[edge];
    const Coef<R> &C = coef<R>(P);
    const long long cg = (long long)(gy + OY) * P.pitch + (gx + OX);
    if (E.kind == 0 || E.kind == 1) {                       // periodic / zero gradient
        const long long cs = (long long)(sy + OY) * P.pitch + (sx + OX);
        if constexpr (sizeof(R) == sizeof(float)) {             // pair planes: one 8-byte copy per pair
            float2 *f2p = reinterpret_cast<float2 *>(f);
#pragma unroll
            for (int pr = 0; pr < 8; pr++) f2p[pr * plane + cg] = f2p[pr * plane + cs];
        } else {
#pragma unroll
            for (int q = 0; q < NQ; q++) f[pidx<R>(q, plane, cg)] = f[pidx<R>(q, plane, cs)];
        }
    } else if (E.kind == 2) {                               // fixed equilibrium
#pragma unroll
        for (int q = 0; q < NQ; q++) f[pidx<R>(q, plane, cg)] = pick<R>(E.feq[q], E.feqf[q]);
    } else {                                                // non-equilibrium extrapolation wall
        const long long cm = (long long)(my + OY) * P.pitch + (mx + OX);
        R g[NQ];
        load16(f, plane, cm, g);
        const Shells<R> s = shells_of(g);
        R drho, jx, jy, de;
        conserved_of(s, drho, jx, jy, de);
        const R rho = Dev ? C.rho0 + drho : drho;
        const R ir = recip(rho);
        const R J2 = (jx * jx + jy * jy) * ir;
        const R dP = (de - J2) * C.inv_b;
        // ghost state: rho_g = rho_m, j_g = 2 rho_m u_w - j_m, P_g = rho_m (2 T_w - T_m)
        const R uw = pick<R>(E.uw, E.uwf), vw = pick<R>(E.vw, E.vwf), Tw = pick<R>(E.Tw, E.Twf);
        const R jgx = R(2.0) * rho * uw - jx;
        const R jgy = R(2.0) * rho * vw - jy;
        const R dPg = Dev ? pick<R>(E.two_rho0_dTw, E.two_rho0_dTwf) + R(2.0) * drho * Tw - dP
                          : R(2.0) * rho * Tw - dP;
        R qm[NQ], qg[NQ], d[NQ], fd[NQ];
        feq_hat_dev<R, Dev>(C, drho, jx, jy, dP, ir, qm);
        feq_hat_dev<R, Dev>(C, drho, jgx, jgy, dPg, ir, qg);
#pragma unroll
        for (int q = 0; q < NQ; q++) d[q] = qg[q] - qm[q];
        pop_from_moments(C, d, fd);
#pragma unroll
        for (int q = 0; q < NQ; q++) f[pidx<R>(q, plane, cg)] = g[q] + fd[q];
    }
}

// first: index of the first ghost cell handled (0: every edge; 4 ny: the y edges only)
template <typename R, bool Dev>
__global__ void k_ghost(const __grid_constant__ Params P, R *__restrict__ f, int first)
{
    ghost_cell<R, Dev>(P, f, first + blockIdx.x * blockDim.x + threadIdx.x);
}

// Batched ghost fill: blockIdx.y selects the grid of the batch.
template <typename R, bool Dev>
__global__ void k_ghost_batch(const Params *__restrict__ Pall, const BatchGrid *__restrict__ G, int phase)
{
    const int gi = blockIdx.y;
    const Params &P = Pall[gi];
    const int n_all = 4 * (P.nx + P.ny);
    const BatchGrid g = G[gi];
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n_all; idx += gridDim.x * blockDim.x)
        ghost_cell<R, Dev>(P, (R *)g.buf[g.cur ^ phase], idx);
}

// ---------------------------------------------------------------------------
// Initialisation from macroscopic fields.  rho, u, v, T: [rows][nx] for interior rows
// row0 .. row0+rows-1 (device addresses, or mapped page-locked host memory).
// float64 mode: f^eq in float64.  float32 deviation mode: the deviations drho, j and
// dP = P - P0 are formed in float64 and the deviation g = f^eq - f^eq0 is evaluated from them
// in float32 (the deviation form has no cancellation against the reference state, so the
// result carries the error of its float32 storage and a few roundings more).
// A cell with rho <= 0, T <= 0 or a non-finite value sets *bad and is not written.
// ---------------------------------------------------------------------------
template <typename R, bool Dev>
__global__ void k_init(const __grid_constant__ Params P, R *__restrict__ f, const double *__restrict__ rho_i,
                       const double *__restrict__ u_i, const double *__restrict__ v_i,
                       const double *__restrict__ T_i, int row0, int rows, int *bad)
{
    const int nx = P.nx;
    const long long n = (long long)rows * nx;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int x = (int)(i % nx), y = row0 + (int)(i / nx);
    const double rho = rho_i[i], ux = u_i[i], uy = v_i[i], T = T_i[i];
    if (!(rho > 0.0) || !(T > 0.0) || !isfinite(rho) || !isfinite(T) || !isfinite(ux) || !isfinite(uy)) {
        atomicOr(bad, 1);
        return;
    }
    const long long c = (long long)(y + OY) * P.pitch + (x + OX);
    if constexpr (sizeof(R) == sizeof(float)) {
        const Coef<float> &C = P.cf;
        const float drho = (float)(rho - P.cd.rho0);
        const float dP = (float)fma(rho, T, -P.cd.P0);
        const float jx = (float)(rho * ux), jy = (float)(rho * uy);
        float q[NQ], g[NQ];
        feq_hat_dev<float, Dev>(C, drho, jx, jy, dP, recip((float)rho), q);
        pop_from_moments(C, q, g);
        float2 *f2p = reinterpret_cast<float2 *>(f);
#pragma unroll
        for (int pr = 0; pr < 8; pr++) f2p[pr * P.plane + c] = make_float2(g[pair_q(pr)], g[pair_q(pr) + 4]);
    } else {
        const Coef<double> &C = P.cd;
        const double drho = rho - C.rho0;
        const double dP = rho * T - C.P0;
        double q[NQ], g[NQ];
        feq_hat_dev<double, Dev>(C, drho, rho * ux, rho * uy, dP, 1.0 / rho, q);
        pop_from_moments(C, q, g);
#pragma unroll
        for (int qq = 0; qq < NQ; qq++) f[pidx<R>(qq, P.plane, c)] = R(g[qq]);
    }
}

// ---------------------------------------------------------------------------
// Moments (float64): rho, u, v, T, Delta and Delta* of interior rows.
// ---------------------------------------------------------------------------
template <bool Dev>
__device__ __forceinline__ void moment_rows(const Params &P, const double *g, double &rho, double &ux,
                                            double &uy, double &T, double *D, double &ir)
{
    const Shells<double> s = shells_of(g);
    const Moments<double> M = moments_of(s);
    const Coef<double> &C = P.cd;
    const double drho = M.m[0], jx = M.m[1], jy = M.m[2], de = M.m[3];
    rho = Dev ? C.rho0 + drho : drho;
    ir = 1.0 / rho;
    ux = jx * ir;
    uy = jy * ir;
    const double J2 = jx * ux + jy * uy;
    const double dP = (de - J2) * C.inv_b;
    T = (Dev ? C.P0 + dP : dP) * ir;
    double q[NQ];
    feq_hat_dev<double, Dev>(C, drho, jx, jy, dP, ir, q);
#pragma unroll
    for (int k = 0; k < NQ; k++) D[k] = M.m[k] - q[k];
}

// velocity of population i (Sec. II)
__device__ __forceinline__ void velocity_i(int i, double &vx, double &vy)
{
    const double sp[4] = {1.0, 6.0, kD3, kD4};
    vx = sgn_x(i) * sp[i >> 2];
    vy = sgn_y(i) * sp[i >> 2];
}

// WantD = false: rho, u, v, T only (the conserved moments; delta_o and dstar_o are null).
template <typename R, bool Dev, bool WantD>
__global__ void k_moments(const __grid_constant__ Params P, const R *__restrict__ f, int row0, int rows,
                          double *rho_o, double *u_o, double *v_o, double *T_o, double *delta_o,
                          double *dstar_o, int *flag)
{
    const int nx = P.nx;
    const long long n = (long long)rows * nx;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int x = (int)(i % nx), y = row0 + (int)(i / nx);
    const long long c = (long long)(y + OY) * P.pitch + (x + OX);
    double g[NQ];
#pragma unroll
    for (int q = 0; q < NQ; q++) g[q] = (double)f[pidx<R>(q, P.plane, c)];
    double rho, ux, uy, T, D[NQ], ir;
    if constexpr (WantD) {
        moment_rows<Dev>(P, g, rho, ux, uy, T, D, ir);
    } else {
        // the same expressions as moment_rows for these four
        const Coef<double> &C = P.cd;
        double drho, jx, jy, de;
        conserved_of(shells_of(g), drho, jx, jy, de);
        rho = Dev ? C.rho0 + drho : drho;
        ir = 1.0 / rho;
        ux = jx * ir;
        uy = jy * ir;
        const double J2 = jx * ux + jy * uy;
        const double dP = (de - J2) * C.inv_b;
        T = (Dev ? C.P0 + dP : dP) * ir;
    }
    if (!(rho > 0.0) || !isfinite(rho) || !isfinite(ux) || !isfinite(uy) || !isfinite(T)) atomicOr(flag, 1);
    if (rho_o) rho_o[i] = rho;
    if (u_o) u_o[i] = ux;
    if (v_o) v_o[i] = uy;
    if (T_o) T_o[i] = T;
    if constexpr (!WantD) return;
    if (delta_o) {
#pragma unroll
        for (int k = 0; k < NQ; k++) delta_o[k * n + i] = D[k];
    }
    if (dstar_o) {
        // f - f^eq = M^-1 Delta, then the rows of M* at w = v_i - u (Appendix A)
        double fn[NQ], out[NQ];
        pop_from_moments(P.cd, D, fn);
#pragma unroll
        for (int k = 0; k < NQ; k++) out[k] = 0.0;
#pragma unroll
        for (int q = 0; q < NQ; q++) {
            double vx, vy;
            velocity_i(q, vx, vy);
            const double wx = vx - ux, wy = vy - uy;
            const double w2 = wx * wx + wy * wy;
            const double we = w2 + (q < 4 ? kEta2 : 0.0);
            const double dd = wx * wx - wy * wy;
            const double a = fn[q];
            out[0] += a;
            out[1] += a * wx;
            out[2] += a * wy;
            out[3] += a * we;
            out[4] += a * w2;
            out[5] += a * dd;
            out[6] += a * wx * wy;
            out[7] += a * wx * we;
            out[8] += a * wy * we;
            out[9] += a * wx * w2;
            out[10] += a * wy * w2;
            out[11] += a * wx * dd;
            out[12] += a * wy * dd;
            out[13] += a * w2 * we;
            out[14] += a * wx * wy * we;
            out[15] += a * dd * we;
        }
#pragma unroll
        for (int k = 0; k < NQ; k++) dstar_o[k * n + i] = out[k];
    }
}

// ---------------------------------------------------------------------------
// Totals: pass 1 (fixed grid, grid-stride, block tree) and pass 2 (one block).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Totals are linear in f: pass 1 sums every population over the cells (blocks over rows,
// threads along each row, in a fixed order; in float32 storage each thread's runs of up to
// 32 cells are summed in float32 and flushed into float64 accumulators), pass 2 adds the
// block sums in a fixed order and takes the conserved moments (rho, j, e) of the 16
// population totals.
template <typename R, bool Dev>
__global__ void __launch_bounds__(kTotalsThreads)
k_totals_partial(const __grid_constant__ Params P, const R *__restrict__ f, double *partial)
{
    __shared__ double red[kTotalsThreads / 32][NQ];
    double a[NQ];
#pragma unroll
    for (int q = 0; q < NQ; q++) a[q] = 0.0;
    for (int y = blockIdx.x; y < P.ny; y += gridDim.x) {
        const long long row = (long long)(y + OY) * P.pitch + OX;
        R run[NQ];
#pragma unroll
        for (int q = 0; q < NQ; q++) run[q] = R(0);
        int cnt = 0;
        for (int x = threadIdx.x; x < P.nx; x += blockDim.x) {
            R g[NQ];
            load16(f, P.plane, row + x, g);
#pragma unroll
            for (int q = 0; q < NQ; q++) run[q] += g[q];
            if (sizeof(R) == sizeof(double) || ++cnt == 32) {
#pragma unroll
                for (int q = 0; q < NQ; q++) { a[q] += (double)run[q]; run[q] = R(0); }
                cnt = 0;
            }
        }
#pragma unroll
        for (int q = 0; q < NQ; q++) a[q] += (double)run[q];
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NQ; q++) {
        const double v = warp_sum(a[q]);
        if (lane == 0) red[w][q] = v;
    }
    __syncthreads();
    if (threadIdx.x < NQ) {
        double v = 0.0;
        for (int j = 0; j < kTotalsThreads / 32; j++) v += red[j][threadIdx.x];
        partial[blockIdx.x * NQ + threadIdx.x] = v;
    }
}

template <bool Dev>
__global__ void k_totals_final(const __grid_constant__ Params P, const double *__restrict__ partial, int nblocks,
                               double scale, double *out)
{
    __shared__ double red[32][NQ];
    __shared__ double tot[NQ];
    double a[NQ];
#pragma unroll
    for (int q = 0; q < NQ; q++) a[q] = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
        for (int q = 0; q < NQ; q++) a[q] += partial[b * NQ + q];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NQ; q++) {
        const double v = warp_sum(a[q]);
        if (lane == 0) red[w][q] = v;
    }
    __syncthreads();
    if (threadIdx.x < NQ) {
        double v = 0.0;
        for (int j = 0; j < (int)(blockDim.x >> 5); j++) v += red[j][threadIdx.x];
        tot[threadIdx.x] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const Shells<double> s = shells_of(tot);
        double rho, jx, jy, e;
        conserved_of(s, rho, jx, jy, e);
        const double n = (double)P.nx * (double)P.ny;
        if (Dev) { rho += n * P.cd.rho0; e += n * P.cd.e0; }
        out[0] = rho * scale;
        out[1] = jx * scale;
        out[2] = jy * scale;
        out[3] = e * scale;
    }
}

// ---------------------------------------------------------------------------
// Pack / unpack interior populations (float64 f; deviation mode adds f^eq0).
// ---------------------------------------------------------------------------
template <typename R, bool Dev>
__global__ void k_pack(const __grid_constant__ Params P, const R *__restrict__ f, int row0, int rows,
                       double *out)
{
    const long long n = (long long)rows * P.nx;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int x = (int)(i % P.nx), y = row0 + (int)(i / P.nx);
    const long long c = (long long)(y + OY) * P.pitch + (x + OX);
#pragma unroll
    for (int q = 0; q < NQ; q++) out[q * n + i] = (double)f[pidx<R>(q, P.plane, c)] + (Dev ? P.feq0[q] : 0.0);
}

template <typename R, bool Dev>
__global__ void k_unpack(const __grid_constant__ Params P, R *__restrict__ f, int row0, int rows,
                         const double *__restrict__ in)
{
    const long long n = (long long)rows * P.nx;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int x = (int)(i % P.nx), y = row0 + (int)(i / P.nx);
    const long long c = (long long)(y + OY) * P.pitch + (x + OX);
#pragma unroll
    for (int q = 0; q < NQ; q++) f[pidx<R>(q, P.plane, c)] = R(in[q * n + i] - (Dev ? P.feq0[q] : 0.0));
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
static inline unsigned blocks_for(long long n, int threads) { return (unsigned)((n + threads - 1) / threads); }

cudaError_t launch_init(const Params &P, int prec, void *f, const double *rho, const double *u, const double *v,
                        const double *T, int row0, int rows, int *bad, cudaStream_t st)
{
    const long long n = (long long)rows * P.nx;
    if (n == 0) return cudaSuccess;
    if (prec == 0)
        k_init<double, false><<<blocks_for(n, 256), 256, 0, st>>>(P, (double *)f, rho, u, v, T, row0, rows, bad);
    else
        k_init<float, true><<<blocks_for(n, 256), 256, 0, st>>>(P, (float *)f, rho, u, v, T, row0, rows, bad);
    return cudaGetLastError();
}

cudaError_t launch_ghost(const Params &P, int prec, void *f, cudaStream_t st, bool y_only)
{
    const int first = y_only ? 4 * P.ny : 0;
    const int n = 4 * (P.nx + P.ny) - first;
    if (prec == 0) k_ghost<double, false><<<blocks_for(n, 128), 128, 0, st>>>(P, (double *)f, first);
    else k_ghost<float, true><<<blocks_for(n, 128), 128, 0, st>>>(P, (float *)f, first);
    return cudaGetLastError();
}

// Tile width of the plain kernels for a grid nx columns wide: 32, or the smallest power of
// two >= nx for narrower grids (log2 returned).
int plain_log_tx(int nx)
{
    int l = 0;
    while ((1 << l) < nx && l < 5) l++;
    return l;
}

template <typename R, bool Dev, int NT>
static void step_launch_nt(const Params &P, const R *a, R *b, cudaStream_t st)
{
    const int log_tx = plain_log_tx(P.nx);
    const int TX = 1 << log_tx, TY = NT / TX;
    const dim3 grid((P.nx + TX - 1) / TX, (P.ny + TY - 1) / TY);
    const size_t smem = 2 * sizeof(R) * (TX + 2) * (TY + 2);
    if (P.limiter == 0) k_step<R, Dev, 0, NT><<<grid, NT, smem, st>>>(P, a, b, TX, log_tx);
    else if (P.limiter == 1) k_step<R, Dev, 1, NT><<<grid, NT, smem, st>>>(P, a, b, TX, log_tx);
    else k_step<R, Dev, 2, NT><<<grid, NT, smem, st>>>(P, a, b, TX, log_tx);
}

cudaError_t launch_step(const Params &P, int prec, const void *fin, void *fout, cudaStream_t st, int ty)
{
    // ty: rows of a 32-column tile (2, 4, 8 or 16: 64 .. 512 threads); grids narrower than
    // 32 columns keep the thread count with TX = the smallest power of two >= nx
    if (prec == 0) {
        const double *a = (const double *)fin;
        double *b = (double *)fout;
        if (ty == 2) step_launch_nt<double, false, kTX * 2>(P, a, b, st);
        else if (ty == 4) step_launch_nt<double, false, kTX * 4>(P, a, b, st);
        else if (ty == 16) step_launch_nt<double, false, kTX * 16>(P, a, b, st);
        else step_launch_nt<double, false, kTX * 8>(P, a, b, st);
    } else {
        const float *a = (const float *)fin;
        float *b = (float *)fout;
        if (ty == 2) step_launch_nt<float, true, kTX * 2>(P, a, b, st);
        else if (ty == 4) step_launch_nt<float, true, kTX * 4>(P, a, b, st);
        else if (ty == 16) step_launch_nt<float, true, kTX * 16>(P, a, b, st);
        else step_launch_nt<float, true, kTX * 8>(P, a, b, st);
    }
    return cudaGetLastError();
}

cudaError_t launch_ghost_batch(const Params *Pall, const BatchGrid *G, int ngrids, int max_ghost, int prec,
                               int phase, cudaStream_t st)
{
    if (ngrids == 0) return cudaSuccess;
    const int bx = (max_ghost + 127) / 128;
    const dim3 grid(bx < 1 ? 1 : (bx > 64 ? 64 : bx), ngrids);
    if (prec == 0) k_ghost_batch<double, false><<<grid, 128, 0, st>>>(Pall, G, phase);
    else k_ghost_batch<float, true><<<grid, 128, 0, st>>>(Pall, G, phase);
    return cudaGetLastError();
}

cudaError_t launch_step_batch(const Params *Pall, const BatchGrid *G, const int4 *tiles, int ntiles, int prec,
                              int limiter, int nt, int ctas, int phase, cudaStream_t st)
{
    if (ntiles == 0) return cudaSuccess;
    const int grid = ntiles < ctas ? ntiles : ctas;
    constexpr int N64 = kBatchThreadsFp64, N32 = kBatchThreads;
    if (prec == 0 && nt == N64) {
        if (limiter == 0) k_step_batch<double, false, 0, N64><<<grid, N64, 0, st>>>(Pall, G, tiles, ntiles, phase);
        else if (limiter == 1) k_step_batch<double, false, 1, N64><<<grid, N64, 0, st>>>(Pall, G, tiles, ntiles, phase);
        else k_step_batch<double, false, 2, N64><<<grid, N64, 0, st>>>(Pall, G, tiles, ntiles, phase);
    } else if (prec == 0) {
        if (limiter == 0) k_step_batch<double, false, 0, N32><<<grid, N32, 0, st>>>(Pall, G, tiles, ntiles, phase);
        else if (limiter == 1) k_step_batch<double, false, 1, N32><<<grid, N32, 0, st>>>(Pall, G, tiles, ntiles, phase);
        else k_step_batch<double, false, 2, N32><<<grid, N32, 0, st>>>(Pall, G, tiles, ntiles, phase);
    } else {
        if (limiter == 0) k_step_batch<float, true, 0, N32><<<grid, N32, 0, st>>>(Pall, G, tiles, ntiles, phase);
        else if (limiter == 1) k_step_batch<float, true, 1, N32><<<grid, N32, 0, st>>>(Pall, G, tiles, ntiles, phase);
        else k_step_batch<float, true, 2, N32><<<grid, N32, 0, st>>>(Pall, G, tiles, ntiles, phase);
    }
    return cudaGetLastError();
}

cudaError_t launch_moments(const Params &P, int prec, const void *f, int row0, int rows, double *rho,
                           double *u, double *v, double *T, double *delta, double *dstar, int *flag,
                           cudaStream_t st)
{
    const long long n = (long long)rows * P.nx;
    if (n == 0) return cudaSuccess;
    const bool want_d = delta || dstar;
    const dim3 g(blocks_for(n, 128)), b(128);
    if (prec == 0 && want_d)
        k_moments<double, false, true><<<g, b, 0, st>>>(P, (const double *)f, row0, rows, rho, u, v, T, delta, dstar,
                                                        flag);
    else if (prec == 0)
        k_moments<double, false, false><<<g, b, 0, st>>>(P, (const double *)f, row0, rows, rho, u, v, T, nullptr,
                                                         nullptr, flag);
    else if (want_d)
        k_moments<float, true, true><<<g, b, 0, st>>>(P, (const float *)f, row0, rows, rho, u, v, T, delta, dstar,
                                                      flag);
    else
        k_moments<float, true, false><<<g, b, 0, st>>>(P, (const float *)f, row0, rows, rho, u, v, T, nullptr,
                                                       nullptr, flag);
    return cudaGetLastError();
}

// Blocks of the totals reduction: one wave of resident blocks (the SM count x blocks per SM at
// the kernel's register use), at most kTotalsBlocks (the partials buffer).  A second, mostly
// empty wave would double the time of the row-strided reduction.
static int totals_blocks(const void *fn)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kTotalsThreads, 0);
    long long n = (long long)(sms < 1 ? 1 : sms) * (per_sm < 1 ? 1 : per_sm);
    if (n > kTotalsBlocks) n = kTotalsBlocks;
    return (int)n;
}

cudaError_t launch_totals(const Params &P, int prec, const void *f, double *partial, double *out, double scale,
                          cudaStream_t st)
{
    if (prec == 0) {
        static const int nb = totals_blocks((const void *)k_totals_partial<double, false>);
        const int g = nb < P.ny ? nb : (P.ny < 1 ? 1 : P.ny);
        k_totals_partial<double, false><<<g, kTotalsThreads, 0, st>>>(P, (const double *)f, partial);
        k_totals_final<false><<<1, 256, 0, st>>>(P, partial, g, scale, out);
    } else {
        static const int nb = totals_blocks((const void *)k_totals_partial<float, true>);
        const int g = nb < P.ny ? nb : (P.ny < 1 ? 1 : P.ny);
        k_totals_partial<float, true><<<g, kTotalsThreads, 0, st>>>(P, (const float *)f, partial);
        k_totals_final<true><<<1, 256, 0, st>>>(P, partial, g, scale, out);
    }
    return cudaGetLastError();
}

cudaError_t launch_pack(const Params &P, int prec, const void *f, int row0, int rows, double *out,
                        cudaStream_t st)
{
    const long long n = (long long)rows * P.nx;
    if (n == 0) return cudaSuccess;
    if (prec == 0) k_pack<double, false><<<blocks_for(n, 256), 256, 0, st>>>(P, (const double *)f, row0, rows, out);
    else k_pack<float, true><<<blocks_for(n, 256), 256, 0, st>>>(P, (const float *)f, row0, rows, out);
    return cudaGetLastError();
}

cudaError_t launch_unpack(const Params &P, int prec, void *f, int row0, int rows, const double *in,
                          cudaStream_t st)
{
    const long long n = (long long)rows * P.nx;
    if (n == 0) return cudaSuccess;
    if (prec == 0) k_unpack<double, false><<<blocks_for(n, 256), 256, 0, st>>>(P, (double *)f, row0, rows, in);
    else k_unpack<float, true><<<blocks_for(n, 256), 256, 0, st>>>(P, (float *)f, row0, rows, in);
    return cudaGetLastError();
}

}  // namespace lbm
