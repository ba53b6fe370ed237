// lbm_step_dd.cu -- float64-mode fused step in double-float arithmetic (sm_103a).
//
// The populations are float64 in HBM, as in the other float64 kernels; the arithmetic of the
// step runs on the float32 pipe in double-float form (lbm_dd.cuh), which GB300 executes far
// faster than float64.  Layout and staging follow the TMA-staged tile kernel: one CTA owns a
// tile of 32 columns x TR rows and one elected thread brings all 16 float64 planes of the
// tile plus its stencil halo into shared memory with one tensor copy (bounded mbarrier wait);
// then
//   split    every staged value becomes hi + lo in place (8 bytes either way);
//   phase 1  flow velocity and 1/rho on the tile + 1 ring (for grad u);
//   phase 2  per row: the MRT collision with the energy-flux correction (Eq. 3, Sec. II) in
//            the shell basis, the limited x and y convection (Sec. III; each x face difference
//            and slope is formed once, by the lane of its column, and passed to the neighbour
//            lane by a shuffle; y slopes from a sliding window down the thread's column), the
//            forward-Euler update, and one float64 store per population (the double-float
//            result rounded to float64).
// The formulas are those of the float64 kernels, operation for operation; each rounds at
// about 2^-47 instead of 2^-53, so results agree with the float64 kernels and the oracle to a
// few parts in 1e14 per step.
#include <cuda.h>

#include "lbm_dd.cuh"
#include "lbm_internal.h"
#include "lbm_tma_util.cuh"

namespace lbm {

namespace {

// ---- constants and coefficients in double-float ----------------------------------------
// Velocity-set constants that float32 does not hold exactly (Sec. II, Appendix A), split at
// compile time.
__host__ __device__ constexpr float hi_of(double x) { return (float)x; }
__host__ __device__ constexpr float lo_of(double x) { return (float)(x - (double)(float)x); }
__device__ __forceinline__ dd kd3() { return dd{hi_of(kD3), lo_of(kD3)}; }                              // sqrt2
__device__ __forceinline__ dd kd4() { return dd{hi_of(kD4), lo_of(kD4)}; }                              // 3/sqrt2
__device__ __forceinline__ dd k4s2() { return dd{hi_of(4.0 * kSqrt2), lo_of(4.0 * kSqrt2)}; }          // 4 sqrt2
__device__ __forceinline__ dd k27s2() { return dd{hi_of(27.0 / kSqrt2), lo_of(27.0 / kSqrt2)}; }       // 27/sqrt2

// ---- Appendix A rows in the shell basis (as conserved_of / moments_of) -------------------
__device__ __forceinline__ void conserved_dd(const Shells<dd> &s, dd &rho, dd &jx, dd &jy, dd &e)
{
    rho = (s.S[0] + s.S[1]) + (s.S[2] + s.S[3]);
    jx = ((s.X[0] + s.X[1] * 6.0f) + kd3() * s.X[2]) + kd4() * s.X[3];
    jy = ((s.Y[0] + s.Y[1] * 6.0f) + kd3() * s.Y[2]) + kd4() * s.Y[3];
    e = ((s.S[0] * 7.25f + s.S[1] * 36.0f) + scale2(s.S[2], 4.0f)) + s.S[3] * 9.0f;
}

// Flow velocity of the cell whose population q is at p[q * stride].
__device__ __forceinline__ void flow_dd(const dd *p, int stride, dd &u, dd &v, dd &ir)
{
    dd g[NQ];
#pragma unroll
    for (int q = 0; q < NQ; q++) g[q] = p[q * stride];
    dd rho, jx, jy, e;
    conserved_dd(shells_of(g), rho, jx, jy, e);
    ir = recip(rho);
    u = jx * ir;
    v = jy * ir;
}

// dt M^-1 S (f_hat - f_hat^eq) with the energy-flux correction (Eq. 3, Sec. II), float64 mode
// (zero reference state): the operations of collide<double, false>.
template <bool C9>
__device__ __forceinline__ void collide_dd(const Coef<dd> &C, const Shells<dd> &s, dd jx, dd jy, dd de, dd ir,
                                           dd ux, dd uy, dd dxux, dd dyux, dd dxuy, dd dyuy, dd *out)
{
    // rows 5..16 of Appendix A
    const dd x8 = ((s.X[0] * 7.25f + s.X[1] * 216.0f) + k4s2() * s.X[2]) + k27s2() * s.X[3];
    const dd y8 = ((s.Y[0] * 7.25f + s.Y[1] * 216.0f) + k4s2() * s.Y[2]) + k27s2() * s.Y[3];
    const dd m13 = ((s.S[0] * 7.25f + s.S[1] * 1296.0f) + scale2(s.S[2], 16.0f)) + s.S[3] * 81.0f;
    const dd m9 = x8 - s.X[0] * 6.25f, m10 = y8 - s.Y[0] * 6.25f;
    const dd m11 = s.X[0] + s.X[1] * 216.0f;
    const dd m12 = -(s.Y[0] + s.Y[1] * 216.0f);
    const dd m5 = s.Q[0] + s.Q[1] * 36.0f, m15 = s.Q[0] * 7.25f + s.Q[1] * 1296.0f;
    const dd m6 = scale2(s.Q[2], 2.0f) + s.Q[3] * 4.5f, m14 = scale2(s.Q[2], 8.0f) + s.Q[3] * 40.5f;
    // equilibria (Appendix A closed forms), as feq_hat_dev<R, false>
    const dd jx2 = jx * ux, jy2 = jy * uy, J2 = jx2 + jy2;
    const dd dP = (de - J2) * C.inv_b;
    const dd e_dev = fma_dd(C.b, dP, J2);
    const dd dxy = jx2 - jy2;
    const dd q4 = scale2(dP, 2.0f) + J2;
    const dd q6 = jx * uy;
    const dd e2p = e_dev + scale2(dP, 2.0f);
    const dd g4 = scale2(dP, 4.0f) + J2;
    const dd q13 = ir * (dP * fma_dd(C.two_b2, dP, C.six_b * J2) + J2 * J2);
    const dd k = fma_dd(C.b4, dP, J2);
    dd D4 = (de - s.S[0] * 6.25f) - q4;
    dd D7 = x8 - e2p * ux, D8 = y8 - e2p * uy;
    const dd D9 = m9 - g4 * ux, D10 = m10 - g4 * uy;
    const dd D11 = m11 - (scale2(dP, 2.0f) + dxy) * ux, D12 = m12 - (dxy - scale2(dP, 2.0f)) * uy;
    const dd D13 = m13 - q13;
    const dd D5 = m5 - dxy, D6 = m6 - q6;
    const dd D14 = m14 - k * ux * uy, D15 = m15 - k * dxy * ir;
    if (C9) {
        // y differences weighted by ry = dx/dy (q8, q9 carry 1/(2 dx))
        const dd div = dxux + C.ry * dyuy, shr = dxuy + C.ry * dyux;
        D7 += C.q8 * dP * (ux * (scale2(dxux, 4.0f) - C.four_inv_b * div) + scale2(uy * shr, 2.0f));
        D8 += C.q9 * dP * (scale2(ux * shr, 2.0f) + uy * (C.g4[1] * dyuy - C.four_inv_b * div));
    }
    dd S[4], X[4], Y[4], Q[4];
#pragma unroll
    for (int r = 0; r < 4; r++) {
        S[r] = C.cA[r][0] * D4 + C.cA[r][1] * D13;
        X[r] = (C.cEx[r][0] * D7 + C.cEx[r][1] * D9) + C.cEx[r][2] * D11;
        Y[r] = (C.cEy[r][0] * D8 + C.cEy[r][1] * D10) + C.cEy[r][2] * D12;
    }
    Q[0] = C.cB1[0][0] * D5 + C.cB1[0][1] * D15;
    Q[1] = C.cB1[1][0] * D5 + C.cB1[1][1] * D15;
    Q[2] = C.cB2[0][0] * D6 + C.cB2[0][1] * D14;
    Q[3] = C.cB2[1][0] * D6 + C.cB2[1][1] * D14;
    unbutterfly_axis(S[0], X[0], Y[0], Q[0], out + 0);
    unbutterfly_axis(S[1], X[1], Y[1], Q[1], out + 4);
    unbutterfly_diag(S[2], X[2], Y[2], Q[2], out + 8);
    unbutterfly_diag(S[3], X[3], Y[3], Q[3], out + 12);
}

__device__ __forceinline__ dd shfl_dd(dd v, int src)
{
    return dd{__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src)};
}
__device__ __forceinline__ dd shfl_down_dd(dd v)
{
    return dd{__shfl_down_sync(0xffffffffu, v.hi, 1), __shfl_down_sync(0xffffffffu, v.lo, 1)};
}
__device__ __forceinline__ dd shfl_up_dd(dd v)
{
    return dd{__shfl_up_sync(0xffffffffu, v.hi, 1), __shfl_up_sync(0xffffffffu, v.lo, 1)};
}

// Face differences enter the MC slope normalised (norm_lim, once per difference: each feeds two
// slopes); the other limiters use them as they are.
template <int Lim>
__device__ __forceinline__ dd norm_lim(dd a)
{
    return Lim == 0 ? norm(a) : a;
}

template <int Lim>
__device__ __forceinline__ dd slope_dd(dd a, dd b)
{
    if (Lim == 0) return mc2n(a, b);
    if (Lim == 1) return scale2(b, 2.0f);
    return dd{0.0f, 0.0f};
}

}  // namespace

// ---------------------------------------------------------------------------
// The tile body shared by the single-grid and the batched kernel: the staged float64 tile in
// shared memory (smraw) is split, then phases 1 and 2 produce the tile's new float64 values.
// ---------------------------------------------------------------------------
// P: the context's Params, or the TileGrid block of a batched launch (nx, ny, pitch, plane).
// S: the tile shape (TmaShape<double> or DdNarrowShape).
template <int Lim, bool C9, typename S, typename PP>
__device__ __forceinline__ void dd_tile(const PP &P, const Coef<dd> &C, unsigned char *smraw,
                                        double *__restrict__ fout, int x0, int y0)
{
    double *tile64 = reinterpret_cast<double *>(smraw);
    dd *tile = reinterpret_cast<dd *>(smraw);
    dd *su = tile + NQ * S::PL;
    dd *sv = su + S::UW * S::UH;
    dd *sir = sv + S::UW * S::UH;
    const int lane = threadIdx.x, ty = threadIdx.y, tid = ty * kTmaTX + lane;
    constexpr int kThreads = kTmaTX * S::TT;
    const int nx = P.nx, ny = P.ny;
    // ---- split: float64 -> hi + lo in place
    for (int k = tid; k < NQ * S::PL; k += kThreads) tile[k] = dd_split(tile64[k]);
    __syncthreads();

    // ---- phase 1: flow velocity and 1/rho on the tile plus its ring
    {
        int i = tid % S::UW, j = tid / S::UW;
        for (int k = tid; k < S::UW * S::UH; k += kThreads) {
            dd ux, uy, ir;
            flow_dd(tile + (j + 1) * S::SW + (i + S::HX - 1), S::PL, ux, uy, ir);
            su[k] = ux;
            sv[k] = uy;
            sir[k] = ir;
            i += kThreads % S::UW;
            j += kThreads / S::UW;
            if (i >= S::UW) {
                i -= S::UW;
                j++;
            }
        }
    }
    __syncthreads();

    // ---- phase 2: rows ty*KR .. ty*KR+KR-1 of the tile, column `lane`
    const int gx = x0 + lane;
    const int r0 = ty * S::KR;
    dd yw[NQ], yd[NQ], ym[NQ];
#pragma unroll
    for (int q = 0; q < NQ; q++) {
        const int sy = tsgn_y(q);
        if (sy == 0) continue;
        const dd *pc = tile + q * S::PL + (lane + S::HX);
        if (sy > 0) {
            const dd w0 = pc[r0 * S::SW], w1 = pc[(r0 + 1) * S::SW], w2 = pc[(r0 + 2) * S::SW];
            const dd d0 = norm_lim<Lim>(w1 - w0), d1 = norm_lim<Lim>(w2 - w1);
            yw[q] = w2;
            yd[q] = d1;
            ym[q] = slope_dd<Lim>(d0, d1);
        } else {
            const dd w1 = pc[(r0 + 1) * S::SW], w2 = pc[(r0 + 2) * S::SW], w3 = pc[(r0 + 3) * S::SW];
            const dd d1 = norm_lim<Lim>(w2 - w1), d2 = norm_lim<Lim>(w3 - w2);
            yw[q] = w3;
            yd[q] = d2;
            ym[q] = slope_dd<Lim>(d2, d1);
        }
    }
#pragma unroll 1
    for (int k = 0; k < S::KR; k++) {
        const int r = r0 + k;
        const int gy = y0 + r;
        const dd *p = tile + (r + 2) * S::SW + (lane + S::HX);
        // values one column outside the warp for the x stencils: lane L < 12 serves the L-th
        // x-moving population (q = 0, 2, 4, 6, 8 .. 15): D(x0 + 32) for lane 31, and the slope
        // beyond the warp's upwind end, S(x0 - 1) = mc2(D(x0 - 1), D(x0)) for populations moving
        // right, S(x0 + 32) = mc2(D(x0 + 32), D(x0 + 33)) for those moving left
        dd edgeD, edgeS = dd{0.0f, 0.0f};
        {
            const int L = lane < 12 ? lane : 0;
            const int q = L < 4 ? 2 * L : L + 4;
            const dd *row = tile + q * S::PL + (r + 2) * S::SW;    // smem column = x - x0 + HX
            edgeD = norm_lim<Lim>(row[kTmaTX + S::HX] - row[kTmaTX + S::HX - 1]);
            if (Lim == 0) {
                const int c0 = tsgn_x(q) > 0 ? 0 : kTmaTX + S::HX - 1;
                edgeS = mc2(row[c0 + 1] - row[c0], row[c0 + 2] - row[c0 + 1]);
            }
        }
        dd f[NQ];
#pragma unroll
        for (int q = 0; q < NQ; q++) f[q] = p[q * S::PL];
        const Shells<dd> sh = shells_of(f);
        dd rho, jx, jy, de;
        conserved_dd(sh, rho, jx, jy, de);
        const int ui = (r + 1) * S::UW + (lane + 1);
        const dd ir = sir[ui];
        const dd dxux = su[ui + 1] - su[ui - 1];
        const dd dyux = su[ui + S::UW] - su[ui - S::UW];
        const dd dxuy = sv[ui + 1] - sv[ui - 1];
        const dd dyuy = sv[ui + S::UW] - sv[ui - S::UW];
        dd acc[NQ];
        collide_dd<C9>(C, sh, jx, jy, de, ir, su[ui], sv[ui], dxux, dyux, dxuy, dyuy, acc);
        const bool store = gx < nx && gy < ny;
        const long long cg = (long long)(gy + OY) * P.pitch + (gx + OX);
#pragma unroll
        for (int q = 0; q < NQ; q++) {
            const int sx = tsgn_x(q), sy = tsgn_y(q);
            const int shell = q >> 2;
            dd tx = dd{0.0f, 0.0f}, tyv = dd{0.0f, 0.0f};
            if (sx != 0) {
                // this lane's face difference D(x) = f(x) - f(x-1) and slope S(x) =
                // mc2(D(x), D(x+1)); the neighbours' values by shuffles, those one column
                // outside the warp from the duty lane of this population
                const int duty = q < 8 ? q >> 1 : q - 4;
                const dd D = norm_lim<Lim>(f[q] - p[q * S::PL - 1]);
                dd Dr = shfl_down_dd(D);
                const dd eD = shfl_dd(edgeD, duty);
                if (lane == kTmaTX - 1) Dr = eD;
                if (Lim == 2) {
                    tx = sx > 0 ? D : -Dr;
                } else if (Lim == 1) {
                    tx = sx > 0 ? D + scale2(C.hh[shell], 2.0f) * (Dr - D) : (-Dr) + scale2(C.hh[shell], 2.0f) * ((-D) - (-Dr));
                } else {
                    const dd Sx = mc2n(D, Dr);
                    const dd eS = shfl_dd(edgeS, duty);
                    if (sx > 0) {
                        // upwind slope S(x - 1): from lane - 1, at lane 0 from the duty lane
                        dd Sl = shfl_up_dd(Sx);
                        if (lane == 0) Sl = eS;
                        tx = D + C.hh[shell] * (Sx - Sl);
                    } else {
                        // moving left: d1 = -D(x+1), slopes -S(x) and -S(x+1) (mc2n is odd and
                        // symmetric, up to the choice between candidates within 2^-47 of each
                        // other)
                        dd Sr = shfl_down_dd(Sx);
                        if (lane == kTmaTX - 1) Sr = eS;
                        tx = (-Dr) + C.hh[shell] * ((-Sx) - (-Sr));
                    }
                }
            }
            if (sy != 0) {
                const dd *pc = tile + q * S::PL + (lane + S::HX);
                const dd wn = pc[(r + (sy > 0 ? 3 : 4)) * S::SW];
                const dd dn = norm_lim<Lim>(wn - yw[q]);
                if (sy > 0) {
                    const dd mn = slope_dd<Lim>(yd[q], dn);
                    tyv = Lim == 2 ? yd[q] : yd[q] + C.hhy[shell] * (mn - ym[q]);
                    ym[q] = mn;
                } else {
                    const dd mn = slope_dd<Lim>(dn, yd[q]);
                    tyv = Lim == 2 ? yd[q] : yd[q] + C.hhy[shell] * (ym[q] - mn);
                    ym[q] = mn;
                }
                yw[q] = wn;
                yd[q] = dn;
            }
            // f - C - c_x (F_out - F_in)_x - c_y (F_out - F_in)_y
            dd out = f[q] - acc[q];
            if (sy > 0) out -= C.cry[shell] * tyv;
            if (sy < 0) out += C.cry[shell] * tyv;
            if (sx != 0) out -= C.cr[shell] * tx;
            if (store) fout[q * P.plane + cg] = dd_to_double(out);
        }
    }
}

// ---------------------------------------------------------------------------
// The single-grid kernel.  Shape as the float64 TMA-staged kernel: 8 warps, 32 x 32 tiles,
// 4 rows per thread, one CTA per SM (the staged tile takes 162 KB).
// ---------------------------------------------------------------------------
template <int Lim, bool Wrap, bool C9, typename S = TmaShape<double>>
__global__ void __launch_bounds__(kTmaTX * S::TT, S::CTAS)
k_step_dd(const __grid_constant__ Params P, const __grid_constant__ Coef<dd> C, const __grid_constant__ CUtensorMap tm,
          const double *__restrict__ fin, double *__restrict__ fout, int *err)
{
    extern __shared__ __align__(128) unsigned char smraw[];
    double *tile64 = reinterpret_cast<double *>(smraw);
    __shared__ __align__(8) unsigned long long bar;

    const int tid = threadIdx.y * kTmaTX + threadIdx.x;
    constexpr int kThreads = kTmaTX * S::TT;
    const int nx = P.nx;
    const int x0 = blockIdx.x * kTmaTX, y0 = blockIdx.y * S::TR;
    const unsigned bar_a = (unsigned)__cvta_generic_to_shared(&bar);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_a) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0) {
        // box origin: interior column x0 - HX = padded column x0 + OX - HX; interior row y0 - 2 =
        // padded row y0
        const unsigned dst = (unsigned)__cvta_generic_to_shared(tile64);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_a),
                     "r"((unsigned)S::tile_bytes) : "memory");
        asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                     " [%0], [%1, {%2, %3, %4}], [%5];"
                     ::"r"(dst), "l"(reinterpret_cast<unsigned long long>(&tm)), "r"(x0 + OX - S::HX), "r"(y0),
                     "r"(0), "r"(bar_a) : "memory");
    }
    const bool ok = mbar_wait(bar_a, 0);
    if (!__syncthreads_and(ok)) {
        if (tid == 0) {
            atomicExch(err, 1);
            mbar_wait(bar_a, 0);               // let a late copy land before the CTA exits (bounded)
        }
        return;
    }
    if (Wrap && (x0 < S::HX || x0 + kTmaTX + S::HX > nx)) {
        wrap_halo<double>(P, fin, tile64, x0, y0, tid, kThreads);
        __syncthreads();
    }
    dd_tile<Lim, C9, S>(P, C, smraw, fout, x0, y0);
}

// ---------------------------------------------------------------------------
// Batched form: one CTA per tile of the launch's grids (TmaBatchArgs).  Thread 0 issues the
// tile copy with the grid's tensor map from the parameter block, then the CTA copies the grid's
// TileGrid block (geometry and double-float coefficients) into shared memory while the copy is
// in flight.  The ghost cells come from the batched ghost fill, so no x wrap.  The energy-flux
// correction runs for every grid; its factors are zero where s8 = s5, which leaves the
// residuals unchanged bit for bit.
// ---------------------------------------------------------------------------
template <int Lim, typename S = TmaShape<double>>
__global__ void __launch_bounds__(kTmaTX * S::TT, S::CTAS)
k_step_dd_batch(const __grid_constant__ TmaBatchArgs A, const TileGrid<Coef<dd>> *__restrict__ TG)
{
    using T = TileGrid<Coef<dd>>;
    static_assert(sizeof(T) % 16 == 0, "TileGrid copy");
    extern __shared__ __align__(128) unsigned char smraw[];
    __shared__ __align__(16) T Ts;
    __shared__ __align__(8) unsigned long long bar;
    const int tid = threadIdx.y * kTmaTX + threadIdx.x;
    constexpr int kThreads = kTmaTX * S::TT;
    int x0, y0;
    const int g = batch_tile(A, blockIdx.x, S::TR, x0, y0);
    const unsigned bar_a = (unsigned)__cvta_generic_to_shared(&bar);
    if (tid == 0)
        batch_issue<S::TR, S::HX>(A, g, x0, y0, (unsigned)__cvta_generic_to_shared(smraw), bar_a,
                                  (unsigned)S::tile_bytes, 0);
    // the grid's block, while the tile copy is in flight
    {
        const int4 *src = reinterpret_cast<const int4 *>(TG + g);
        int4 *dst = reinterpret_cast<int4 *>(&Ts);
        for (int k = tid; k < (int)(sizeof(T) / sizeof(int4)); k += kThreads) dst[k] = src[k];
    }
    __syncthreads();                            // the barrier is initialised
    const bool ok = mbar_wait(bar_a, 0);
    if (!__syncthreads_and(ok)) {
        if (tid == 0) {
            atomicExch(A.err[g], 1);
            mbar_wait(bar_a, 0);               // let a late copy land before the CTA exits (bounded)
        }
        return;
    }
    dd_tile<Lim, true, S>(Ts, Ts.cf, smraw, static_cast<double *>(A.out[g]), x0, y0);
}

// Coefficients in double-float from the float64 tables (host).
void coef_dd(const Params &P, Coef<dd> *out)
{
    static_assert(sizeof(Coef<dd>) == sizeof(Coef<double>), "Coef layout");
    const double *src = reinterpret_cast<const double *>(&P.cd);
    dd *dst = reinterpret_cast<dd *>(out);
    for (size_t k = 0; k < sizeof(Coef<double>) / sizeof(double); k++) dst[k] = dd_host(src[k]);
}

template <int Lim, bool Wrap, typename S>
static void launch_dd_lim(const Params &P, const Coef<dd> &C, const CUtensorMap &tm, const double *a, double *b,
                          int *err, cudaStream_t st)
{
    const dim3 block(kTmaTX, S::TT);
    const dim3 grid((P.nx + kTmaTX - 1) / kTmaTX, (P.ny + S::TR - 1) / S::TR);
    if (P.has_c9) k_step_dd<Lim, Wrap, true, S><<<grid, block, S::smem_bytes, st>>>(P, C, tm, a, b, err);
    else k_step_dd<Lim, Wrap, false, S><<<grid, block, S::smem_bytes, st>>>(P, C, tm, a, b, err);
}

bool dd_narrow_supported(const Params &P)
{
    using S = DdNarrowShape;
    return P.pitch >= S::SW && P.ny + 4 >= S::SH && P.nx >= kTmaTX;
}

cudaError_t launch_step_dd(const Params &P, const void *coef, const void *tmap, const void *fin, void *fout,
                           int *err, cudaStream_t st, bool narrow)
{
    using W = TmaShape<double>;
    using N = DdNarrowShape;
    const CUtensorMap &tm = *reinterpret_cast<const CUtensorMap *>(tmap);
    const Coef<dd> &C = *reinterpret_cast<const Coef<dd> *>(coef);
    const double *a = (const double *)fin;
    double *b = (double *)fout;
    if (narrow) {
        // the ghost fill writes every ghost cell of a context on narrow tiles: no x wrap
        if (P.limiter == 0) launch_dd_lim<0, false, N>(P, C, tm, a, b, err, st);
        else if (P.limiter == 1) launch_dd_lim<1, false, N>(P, C, tm, a, b, err, st);
        else launch_dd_lim<2, false, N>(P, C, tm, a, b, err, st);
        return cudaGetLastError();
    }
    const bool wrap = (P.wrap & 1) != 0;
    if (P.limiter == 0) {
        if (wrap) launch_dd_lim<0, true, W>(P, C, tm, a, b, err, st);
        else launch_dd_lim<0, false, W>(P, C, tm, a, b, err, st);
    } else if (P.limiter == 1) {
        if (wrap) launch_dd_lim<1, true, W>(P, C, tm, a, b, err, st);
        else launch_dd_lim<1, false, W>(P, C, tm, a, b, err, st);
    } else {
        if (wrap) launch_dd_lim<2, true, W>(P, C, tm, a, b, err, st);
        else launch_dd_lim<2, false, W>(P, C, tm, a, b, err, st);
    }
    return cudaGetLastError();
}

template <typename S>
static void launch_dd_batch_shape(const TmaBatchArgs &A, const TileGrid<Coef<dd>> *tg, int limiter, int ntiles,
                                  cudaStream_t st)
{
    const dim3 block(kTmaTX, S::TT);
    if (limiter == 0) k_step_dd_batch<0, S><<<ntiles, block, S::smem_bytes, st>>>(A, tg);
    else if (limiter == 1) k_step_dd_batch<1, S><<<ntiles, block, S::smem_bytes, st>>>(A, tg);
    else k_step_dd_batch<2, S><<<ntiles, block, S::smem_bytes, st>>>(A, tg);
}

cudaError_t launch_step_dd_batch(const TmaBatchArgs &A, const TileGrid<Coef<dd>> *tg, int limiter, bool narrow,
                                 cudaStream_t st)
{
    const int ntiles = A.first[A.n];
    if (ntiles <= 0) return cudaSuccess;
    if (narrow) launch_dd_batch_shape<DdNarrowShape>(A, tg, limiter, ntiles, st);
    else launch_dd_batch_shape<TmaShape<double>>(A, tg, limiter, ntiles, st);
    return cudaGetLastError();
}

cudaError_t dd_prepare()
{
    cudaError_t e = cudaSuccess;
    auto set = [&](const void *fn) {
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TmaShape<double>::smem_bytes);
    };
    set((const void *)k_step_dd<0, false, false>);
    set((const void *)k_step_dd<0, false, true>);
    set((const void *)k_step_dd<0, true, false>);
    set((const void *)k_step_dd<0, true, true>);
    set((const void *)k_step_dd<1, false, false>);
    set((const void *)k_step_dd<1, false, true>);
    set((const void *)k_step_dd<1, true, false>);
    set((const void *)k_step_dd<1, true, true>);
    set((const void *)k_step_dd<2, false, false>);
    set((const void *)k_step_dd<2, false, true>);
    set((const void *)k_step_dd<2, true, false>);
    set((const void *)k_step_dd<2, true, true>);
    set((const void *)k_step_dd_batch<0>);
    set((const void *)k_step_dd_batch<1>);
    set((const void *)k_step_dd_batch<2>);
    // narrow tiles: within the default 48 KB of dynamic shared memory
    static_assert(DdNarrowShape::smem_bytes <= 48 * 1024, "narrow tile within the default shared memory");
    return e;
}

}  // namespace lbm
