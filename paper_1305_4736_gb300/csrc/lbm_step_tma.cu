// lbm_step_tma.cu -- fused step kernel with TMA-staged tiles (sm_103a).
//
// One CTA owns a tile of 32 columns x TR rows.  A single elected thread issues
// one 3-D tensor copy (cp.async.bulk.tensor) that brings all 16 population
// planes of the tile plus its stencil halo (2 rows, 4 columns on each side;
// the 4-column x halo keeps the copy on a 16-byte boundary) into shared
// memory; completion is tracked by an mbarrier with a bounded wait.  Then:
//   phase 1  flow velocity and 1/rho on the tile + 1 ring (for grad u)
//   phase 2  per row: MRT collision with the energy-flux correction (Eq. 3,
//            Sec. II), then the limited x and y convection of Sec. III:
//            x stencils read the staged row (one warp = one tile row), y slopes
//            slide down the thread's own column of KR rows (each slope computed
//            once); one global write per population.
// The arithmetic per value is that of the plain kernel; results agree with it
// to round-off (the compiler may contract multiply-adds differently).
#include <cuda.h>

#include "lbm_internal.h"
#include "lbm_tma_util.cuh"

namespace lbm {


// Phase 2 of the float32 kernel on population pairs: the staged tile is 8 planes of
// pairs (pair_q(pr), pair_q(pr) + 4), read and written one pair per access.
// P: the context's Params, or the TileGrid block of a batched launch (the fields read here).
template <bool Dev, int Lim, typename S = TmaShape<float>, typename PP = Params>
__device__ __forceinline__ void phase2_packed(const PP &P, const float2 *tile, const float2 *suv,
                                              int lane, int ty, int x0, int y0, float *__restrict__ fout)
{
    const Coef<float> &C = P.cf;
    const int gx = x0 + lane;
    const int r0 = ty * S::KR;
    const float2 *col = tile + (lane + S::HX);
    // sliding y-window state per y-moving pair: last value, face difference, slope
    float2 yw[8], yd[8], ym[8];
#pragma unroll
    for (int pr = 0; pr < 8; pr++) {
        const int sy = tsgn_y(pair_q(pr));
        if (sy == 0) continue;
        const float2 *pc = col + pr * S::PL;
        if (sy > 0) {
            const float2 w0 = pc[r0 * S::SW], w1 = pc[(r0 + 1) * S::SW], w2 = pc[(r0 + 2) * S::SW];
            const float2 d0 = sub2(w1, w0), d1 = sub2(w2, w1);
            yw[pr] = w2;
            yd[pr] = d1;
            ym[pr] = slope2x2<Lim>(d0, d1);
        } else {
            // downward pairs carry their oriented slope negated (slope2x2 is odd): no negations
            const float2 w1 = pc[(r0 + 1) * S::SW], w2 = pc[(r0 + 2) * S::SW], w3 = pc[(r0 + 3) * S::SW];
            const float2 d1 = sub2(w2, w1), d2 = sub2(w3, w2);
            yw[pr] = w3;
            yd[pr] = d2;
            ym[pr] = slope2x2<Lim>(d2, d1);
        }
    }
    float2 *out2 = reinterpret_cast<float2 *>(fout);
#pragma unroll 1
    for (int k = 0; k < S::KR; k++) {
        const int r = r0 + k;
        const int gy = y0 + r;
        const float2 *p = col + (r + 2) * S::SW;
        float2 fp[8];
#pragma unroll
        for (int pr = 0; pr < 8; pr++) fp[pr] = p[pr * S::PL];
        const Shells2 sh = shells2_of(fp);
        float drho, jx, jy, de;
        conserved2_of(sh, drho, jx, jy, de);
        const int ui = (r + 1) * S::UW + (lane + 1);
        const float ir = recip(Dev ? C.rho0 + drho : drho);   // as phase 1 computed it
        const float2 gx2 = sub2(suv[ui + 1], suv[ui - 1]);           // (d_x u_x, d_x u_y) x 2 dx
        const float2 gy2 = sub2(suv[ui + S::UW], suv[ui - S::UW]);   // (d_y u_x, d_y u_y) x 2 dx
        float2 acc[8];
        collide2<Dev>(P, sh, drho, jx, jy, de, ir, gx2.x, gy2.x, gx2.y, gy2.y, acc);
        const bool store = gx < P.nx && gy < P.ny;
        const long long cg = (long long)(gy + OY) * P.pitch + (gx + OX);
#pragma unroll
        for (int pr = 0; pr < 8; pr++) {
            const int qa = pair_q(pr);
            const int sx = tsgn_x(qa), sy = tsgn_y(qa);
            const int sa = qa >> 2;
            const float2 hy = ld2(&C.hhy[sa]);
            const float2 f0 = fp[pr];
            const float2 *pp = p + pr * S::PL;
            float2 tx = f2(0.f, 0.f), tyv = f2(0.f, 0.f);
            if (sx != 0) tx = flux_diff2<Lim>(pp[-2 * sx], pp[-sx], f0, pp[sx], ld2(&C.hh[sa]));
            if (sy != 0) {
                const float2 wn = col[pr * S::PL + (r + (sy > 0 ? 3 : 4)) * S::SW];
                const float2 dn = sub2(wn, yw[pr]);
                if (sy > 0) {
                    const float2 mn = slope2x2<Lim>(yd[pr], dn);
                    tyv = Lim == 2 ? yd[pr] : fma2(hy, sub2(mn, ym[pr]), yd[pr]);
                    ym[pr] = mn;
                } else {
                    // the flux negated: D(y+1) + h (slope'_{y+1} - slope'_y) with negated slopes
                    const float2 mn = slope2x2<Lim>(dn, yd[pr]);
                    tyv = Lim == 2 ? yd[pr] : fma2(hy, sub2(ym[pr], mn), yd[pr]);
                    ym[pr] = mn;
                }
                yw[pr] = wn;
                yd[pr] = dn;
            }
            // f - C - c_x (F_out - F_in)_x - c_y (F_out - F_in)_y
            float2 out = sub2(f0, acc[pr]);
            if (sy > 0) out = fma2(ld2(&C.ncry[sa]), tyv, out);
            if (sy < 0) out = fma2(ld2(&C.cry[sa]), tyv, out);
            if (sx != 0) out = fma2(ld2(&C.ncr[sa]), tx, out);
            if (store) __stcs(out2 + pr * P.plane + cg, out);   // evict-first: not re-read before it leaves L2
        }
    }
}

// Phase 1 of the tile kernels: flow velocity and 1/rho on the tile plus its ring.  Cells of the
// ring outside the domain's cross (corners, beyond the ghost layer) get values that only lanes
// whose results are not stored read.
template <typename R, bool Dev>
__device__ __forceinline__ void flow_phase(const Coef<R> &C, const R *tile, R *su, R *sv, R *sir, int tid)
{
    using S = TmaShape<R>;
    constexpr int kStep = kTmaTX * S::TT;
    int i = tid % S::UW, j = tid / S::UW;
    for (int k = tid; k < S::UW * S::UH; k += kStep) {
        R ux, uy, ir;
        if constexpr (sizeof(R) == sizeof(float))
            flow_at<Dev>(C, reinterpret_cast<const float2 *>(tile) + (j + 1) * S::SW + (i + S::HX - 1), S::PL, ux,
                         uy, ir);
        else
            flow_at<Dev>(C, tile + (j + 1) * S::SW + (i + S::HX - 1), S::PL, ux, uy, ir);
        i += kStep % S::UW;
        j += kStep / S::UW;
        if (i >= S::UW) {
            i -= S::UW;
            j++;
        }
        if constexpr (sizeof(R) == sizeof(float)) {
            reinterpret_cast<float2 *>(su)[k] = f2(ux, uy);   // float32: (u_x, u_y) pairs
        } else {
            su[k] = ux;
            sv[k] = uy;
            sir[k] = ir;
        }
    }
}

// Wrap: the grid's x halo is wrapped in the kernel (P.wrap bit 0); a separate instantiation,
// so that the other grids run a kernel without that branch.
template <typename R, bool Dev, int Lim, bool Wrap>
__global__ void __launch_bounds__(kTmaTX * TmaShape<R>::TT, TmaShape<R>::CTAS)
k_step_tma(const __grid_constant__ Params P, const __grid_constant__ CUtensorMap tm, const R *__restrict__ fin,
           R *__restrict__ fout, int *err)
{
    using S = TmaShape<R>;
    extern __shared__ __align__(128) unsigned char smraw[];
    R *tile = reinterpret_cast<R *>(smraw);
    R *su = tile + NQ * S::PL;
    R *sv = su + S::UW * S::UH;
    R *sir = sv + S::UW * S::UH;   // float64 only
    __shared__ __align__(8) unsigned long long bar;

    const int lane = threadIdx.x, ty = threadIdx.y, tid = ty * kTmaTX + lane;
    const int nx = P.nx, ny = P.ny;
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
        const unsigned dst = (unsigned)__cvta_generic_to_shared(tile);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_a),
                     "r"((unsigned)S::tile_bytes) : "memory");
        asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                     " [%0], [%1, {%2, %3, %4}], [%5];"
                     ::"r"(dst), "l"(reinterpret_cast<unsigned long long>(&tm)), "r"(x0 + OX - S::HX), "r"(y0),
                     "r"(0), "r"(bar_a) : "memory");
        if constexpr (sizeof(R) == sizeof(float)) {
            // CTAs start in launch order: bring the tile of the CTA about half a resident wave
            // later (CTAS x SMs / 2 blocks on) into L2, so that its copy is served from L2
            unsigned nsm;
            asm("mov.u32 %0, %%nsmid;" : "=r"(nsm));
            const long long b = (long long)blockIdx.y * gridDim.x + blockIdx.x;
            const long long bn = b + (long long)S::CTAS * nsm / 2;
            if (bn < (long long)gridDim.x * gridDim.y) {
                const int xn = (int)(bn % gridDim.x) * kTmaTX + OX - S::HX, yn = (int)(bn / gridDim.x) * S::TR;
                asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];"
                             ::"l"(reinterpret_cast<unsigned long long>(&tm)), "r"(xn), "r"(yn), "r"(0) : "memory");
            }
        }
    }
    const bool ok = mbar_wait(bar_a, 0);
    if (!__syncthreads_and(ok)) {
        if (tid == 0) {
            atomicExch(err, 1);
            mbar_wait(bar_a, 0);               // let a late copy land before the CTA exits (bounded)
        }
        return;
    }
    // tiles whose staged box reaches past a periodic x edge (uniform per CTA)
    if (Wrap && (x0 < S::HX || x0 + kTmaTX + S::HX > nx)) {
        wrap_halo<R>(P, fin, tile, x0, y0, tid, kTmaTX * S::TT);
        __syncthreads();
    }
    const Coef<R> &C = coef<R>(P);
    // ---- phase 1: flow velocity and 1/rho on the tile plus its ring
    flow_phase<R, Dev>(C, tile, su, sv, sir, tid);
    __syncthreads();

    // ---- phase 2: rows ty*KR .. ty*KR+KR-1 of the tile, column `lane`
    if constexpr (sizeof(R) == sizeof(float)) {
        phase2_packed<Dev, Lim>(P, reinterpret_cast<const float2 *>(tile), reinterpret_cast<const float2 *>(su),
                                lane, ty, x0, y0, fout);
    } else {
        const int gx = x0 + lane;
        const int r0 = ty * S::KR;
        // sliding y-window state per y-moving population: last value, face difference, slope
        R yw[NQ], yd[NQ], ym[NQ];
#pragma unroll
        for (int q = 0; q < NQ; q++) {
            const int sy = tsgn_y(q);
            if (sy == 0) continue;
            const R *pc = tile + q * S::PL + (lane + S::HX);
            // window index m <-> smem row r0 + m (tile row r0 + m - 2); D[m] = w[m+1] - w[m]
            if (sy > 0) {
                // oriented slope at index c: slope2(D[c-1], D[c]); carry w[2], D[1], slope at index 1
                const R w0 = pc[r0 * S::SW], w1 = pc[(r0 + 1) * S::SW], w2 = pc[(r0 + 2) * S::SW];
                const R d0 = w1 - w0, d1 = w2 - w1;
                yw[q] = w2;
                yd[q] = d1;
                ym[q] = slope2<R, Lim>(d0, d1);
            } else {
                // oriented slope at index c: slope2(-D[c], -D[c-1]); carry w[3], D[2] and the slope
                // at index 2 negated, slope2(D[2], D[1]) (slope2 is odd; no negations in float64)
                const R w1 = pc[(r0 + 1) * S::SW], w2 = pc[(r0 + 2) * S::SW], w3 = pc[(r0 + 3) * S::SW];
                const R d1 = w2 - w1, d2 = w3 - w2;
                yw[q] = w3;
                yd[q] = d2;
                ym[q] = slope2<R, Lim>(d2, d1);
            }
        }

#pragma unroll 1
        for (int k = 0; k < S::KR; k++) {
            const int r = r0 + k;
            const int gy = y0 + r;
            const R *p = tile + (r + 2) * S::SW + (lane + S::HX);
            R f[NQ];
#pragma unroll
            for (int q = 0; q < NQ; q++) f[q] = p[q * S::PL];
            const Shells<R> sh = shells_of(f);
            R drho, jx, jy, de;
            conserved_of(sh, drho, jx, jy, de);
            const int ui = (r + 1) * S::UW + (lane + 1);
            const R ir = sir[ui];
            const R dxux = su[ui + 1] - su[ui - 1];
            const R dyux = su[ui + S::UW] - su[ui - S::UW];
            const R dxuy = sv[ui + 1] - sv[ui - 1];
            const R dyuy = sv[ui + S::UW] - sv[ui - S::UW];
            R acc[NQ];
            collide<R, Dev>(P, sh, drho, jx, jy, de, ir, jx * ir, jy * ir, dxux, dyux, dxuy, dyuy, acc);
            const bool store = gx < nx && gy < ny;
            const long long cg = (long long)(gy + OY) * P.pitch + (gx + OX);
#pragma unroll
            for (int q = 0; q < NQ; q++) {
                const int sx = tsgn_x(q), sy = tsgn_y(q);
                const int shell = q >> 2;
                const R hy = C.hhy[shell];
                R tx = R(0), tyv = R(0);
                if (sx != 0) {
                    // both slopes from the staged row (sharing the upwind slope with the
                    // neighbouring lane would cost a shuffle plus a boundary-lane fix-up)
                    const R *pr = p + q * S::PL;
                    const R fm2 = pr[-2 * sx], fm1 = pr[-sx], fp1 = pr[sx];
                    tx = flux_diff<R, Lim>(fm2, fm1, f[q], fp1, C.hh[shell]);
                }
                if (sy != 0) {
                    const R *pc = tile + q * S::PL + (lane + S::HX);
                    // next window value: smem row r0 + k + 3 (sy > 0) or r0 + k + 4 (sy < 0)
                    const R wn = pc[(r + (sy > 0 ? 3 : 4)) * S::SW];
                    const R dn = wn - yw[q];
                    if (sy > 0) {
                        // D[k+2], slope at J = index k+2; flux D[k+1] + h (slope_J - slope_{J-1})
                        const R mn = slope2<R, Lim>(yd[q], dn);
                        tyv = Lim == 2 ? yd[q] : yd[q] + hy * (mn - ym[q]);
                        ym[q] = mn;
                    } else {
                        // D[k+3], slope at J - sigma = index k+3; flux -D[k+2] + h (slope_J - slope_{J+1}),
                        // carried negated: tyv = D[k+2] + h (-slope_J + slope_{J+1})
                        const R mn = slope2<R, Lim>(dn, yd[q]);
                        tyv = Lim == 2 ? yd[q] : yd[q] + hy * (ym[q] - mn);
                        ym[q] = mn;
                    }
                    yw[q] = wn;
                    yd[q] = dn;
                }
                // f - C - c_x (F_out - F_in)_x - c_y (F_out - F_in)_y
                R out = f[q] - acc[q];
                if (sy > 0) out -= C.cry[shell] * tyv;
                if (sy < 0) out += C.cry[shell] * tyv;
                if (sx != 0) out -= C.cr[shell] * tx;
                if (store) fout[q * P.plane + cg] = out;
            }
        }

    }
}

// ---------------------------------------------------------------------------
// Batched form (float32): one CTA per tile of the launch's grids (TmaBatchArgs).  Thread 0
// issues the tile copy with the grid's tensor map from the parameter block, then the CTA
// copies the grid's TileGrid block into shared memory while the copy is in flight; the
// arithmetic is that of k_step_tma.  The ghost cells come from the batched ghost fill, so no
// x wrap.
// ---------------------------------------------------------------------------
template <int Lim>
__global__ void __launch_bounds__(kTmaTX * TmaShape<float>::TT, TmaShape<float>::CTAS)
k_step_tma_batch(const __grid_constant__ TmaBatchArgs A, const TileGrid<Coef<float>> *__restrict__ TG)
{
    using S = TmaShape<float>;
    using T = TileGrid<Coef<float>>;
    static_assert(sizeof(T) % 16 == 0, "TileGrid copy");
    extern __shared__ __align__(128) unsigned char smraw[];
    float *tile = reinterpret_cast<float *>(smraw);
    float *su = tile + NQ * S::PL;
    __shared__ __align__(16) T Ts;
    __shared__ __align__(8) unsigned long long bar;

    const int lane = threadIdx.x, ty = threadIdx.y, tid = ty * kTmaTX + lane;
    constexpr int kThreads = kTmaTX * S::TT;
    int x0, y0;
    const int g = batch_tile(A, blockIdx.x, S::TR, x0, y0);
    const unsigned bar_a = (unsigned)__cvta_generic_to_shared(&bar);
    if (tid == 0)
        batch_issue<S::TR, S::HX>(A, g, x0, y0, (unsigned)__cvta_generic_to_shared(tile), bar_a,
                                  (unsigned)S::tile_bytes, S::CTAS);
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
    flow_phase<float, true>(Ts.cf, tile, su, nullptr, nullptr, tid);
    __syncthreads();
    phase2_packed<true, Lim>(Ts, reinterpret_cast<const float2 *>(tile), reinterpret_cast<const float2 *>(su), lane,
                             ty, x0, y0, static_cast<float *>(A.out[g]));
}

cudaError_t launch_step_tma_batch(const TmaBatchArgs &A, const TileGrid<Coef<float>> *tg, int limiter,
                                  cudaStream_t st)
{
    using S = TmaShape<float>;
    const int ntiles = A.first[A.n];
    if (ntiles <= 0) return cudaSuccess;
    const dim3 block(kTmaTX, S::TT);
    if (limiter == 0) k_step_tma_batch<0><<<ntiles, block, S::smem_bytes, st>>>(A, tg);
    else if (limiter == 1) k_step_tma_batch<1><<<ntiles, block, S::smem_bytes, st>>>(A, tg);
    else k_step_tma_batch<2><<<ntiles, block, S::smem_bytes, st>>>(A, tg);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Persistent double-buffered form (float32).  CTA c takes tiles c, c + G, c + 2G, ...
// (G = grid size); tile k of a CTA is staged in buffer k & 1, whose copy was issued
// while the CTA worked on tile k - 1 (or at start), and the buffer is refilled with
// tile k + 2 as soon as every thread is done with tile k.
// ---------------------------------------------------------------------------
template <bool Dev, int Lim>
__global__ void __launch_bounds__(kTmaTX * kTmaTT, 2)
k_step_tma_pipe(const __grid_constant__ Params P, const __grid_constant__ CUtensorMap tm, float *__restrict__ fout,
                int *err)
{
    using S = TmaPipeShape;
    extern __shared__ __align__(128) unsigned char smraw[];
    float2 *buf = reinterpret_cast<float2 *>(smraw);
    float2 *suv = reinterpret_cast<float2 *>(smraw + 2 * S::buf_bytes);   // (u_x, u_y)
    __shared__ __align__(8) unsigned long long bar[2];

    const int lane = threadIdx.x, ty = threadIdx.y, tid = ty * kTmaTX + lane;
    const int nx = P.nx, ny = P.ny;
    const int ntx = (nx + kTmaTX - 1) / kTmaTX;
    const int ntiles = ntx * ((ny + S::TR - 1) / S::TR);
    const unsigned bar_a = (unsigned)__cvta_generic_to_shared(bar);
    const unsigned buf_a = (unsigned)__cvta_generic_to_shared(buf);
    // copy of tile t (box origin: interior (x0 - HX, y0 - 2) = padded (x0 + OX - HX, y0)) into buffer b
    auto issue = [&](int t, int b) {
        const int x0 = (t % ntx) * kTmaTX + OX - S::HX, y0 = (t / ntx) * S::TR;
        const unsigned bb = bar_a + 8u * (unsigned)b;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bb),
                     "r"((unsigned)S::buf_bytes) : "memory");
        asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                     " [%0], [%1, {%2, %3, %4}], [%5];"
                     ::"r"(buf_a + (unsigned)(b * S::buf_bytes)), "l"(reinterpret_cast<unsigned long long>(&tm)),
                     "r"(x0), "r"(y0), "r"(0), "r"(bb) : "memory");
    };
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_a) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_a + 8u) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0) {
        if ((int)blockIdx.x < ntiles) issue(blockIdx.x, 0);
        if ((int)(blockIdx.x + gridDim.x) < ntiles) issue(blockIdx.x + gridDim.x, 1);
    }

    const Coef<float> &C = P.cf;
    int k = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, k++) {
        const int b = k & 1;
        const bool ok = mbar_wait(bar_a + 8u * (unsigned)b, (unsigned)(k >> 1) & 1u);
        const float2 *tile = buf + b * (int)(S::buf_bytes / sizeof(float2));
        const int x0 = (t % ntx) * kTmaTX, y0 = (t / ntx) * S::TR;
        // phase 1: flow velocity and 1/rho on the tile plus its ring
        if (ok) {
            constexpr int kStep = kTmaTX * kTmaTT;
            int i = tid % S::UW, j = tid / S::UW;
            for (int kk = tid; kk < S::UW * S::UH; kk += kStep) {
                float ux, uy, ir;
                flow_at<Dev>(C, tile + (j + 1) * S::SW + (i + S::HX - 1), S::PL, ux, uy, ir);
                suv[kk] = f2(ux, uy);
                i += kStep % S::UW;
                j += kStep / S::UW;
                if (i >= S::UW) {
                    i -= S::UW;
                    j++;
                }
            }
        }
        if (!__syncthreads_and(ok)) {
            // a copy wait ran out: report, let copies in flight land (bounded), stop
            if (tid == 0) {
                atomicExch(err, 1);
                mbar_wait(bar_a + 8u * (unsigned)b, (unsigned)(k >> 1) & 1u);
                if (t + (int)gridDim.x < ntiles)
                    mbar_wait(bar_a + 8u * (unsigned)(b ^ 1), (unsigned)((k + 1) >> 1) & 1u);
            }
            return;
        }
        // phase 2: rows ty*KR .. ty*KR+KR-1 of the tile, column `lane`
        phase2_packed<Dev, Lim, S>(P, tile, suv, lane, ty, x0, y0, fout);
        __syncthreads();
        if (tid == 0 && t + 2 * (int)gridDim.x < ntiles) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(t + 2 * gridDim.x, b);
        }
    }
}

bool tma_pipe_supported(const Params &P)
{
    return P.pitch >= TmaPipeShape::SW && P.ny + 4 >= TmaPipeShape::SH && P.nx >= kTmaTX;
}

cudaError_t launch_step_tma_pipe(const Params &P, const void *tmap, void *fout, int *err, cudaStream_t st)
{
    const CUtensorMap &tm = *reinterpret_cast<const CUtensorMap *>(tmap);
    using S = TmaPipeShape;
    const void *fn = P.limiter == 0 ? (const void *)k_step_tma_pipe<true, 0>
                     : P.limiter == 1 ? (const void *)k_step_tma_pipe<true, 1>
                                      : (const void *)k_step_tma_pipe<true, 2>;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kTmaTX * kTmaTT, S::smem_bytes);
    const int ntiles = ((P.nx + kTmaTX - 1) / kTmaTX) * ((P.ny + S::TR - 1) / S::TR);
    int grid = (sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
    if (grid > ntiles) grid = ntiles;
    const dim3 block(kTmaTX, kTmaTT);
    float *b = (float *)fout;
    if (P.limiter == 0) k_step_tma_pipe<true, 0><<<grid, block, S::smem_bytes, st>>>(P, tm, b, err);
    else if (P.limiter == 1) k_step_tma_pipe<true, 1><<<grid, block, S::smem_bytes, st>>>(P, tm, b, err);
    else k_step_tma_pipe<true, 2><<<grid, block, S::smem_bytes, st>>>(P, tm, b, err);
    return cudaGetLastError();
}

cudaError_t tma_pipe_prepare()
{
    cudaError_t e = cudaSuccess;
    for (const void *fn : {(const void *)k_step_tma_pipe<true, 0>, (const void *)k_step_tma_pipe<true, 1>,
                           (const void *)k_step_tma_pipe<true, 2>})
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TmaPipeShape::smem_bytes);
    return e;
}

// ---------------------------------------------------------------------------
// Failure path of the bounded copy waits: one warp waits on an mbarrier phase that nothing
// completes (no copy is issued, no thread arrives).  mbar_wait gives up at its global-timer
// limit; the kernel records that in *flag and returns, leaving no copy in flight.
__global__ void k_wait_selftest(int *flag)
{
    __shared__ __align__(8) unsigned long long bar;
    const unsigned bar_a = (unsigned)__cvta_generic_to_shared(&bar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_a) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    const bool ok = mbar_wait(bar_a, 0);
    if (!ok && threadIdx.x == 0) atomicExch(flag, 1);
}

cudaError_t wait_selftest(int *flag, float *ms)
{
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    if (ce == cudaSuccess) ce = cudaMemset(flag, 0, sizeof(int));
    if (ce == cudaSuccess) ce = cudaEventRecord(e0);
    if (ce == cudaSuccess) {
        k_wait_selftest<<<1, 32>>>(flag);
        ce = cudaGetLastError();
    }
    if (ce == cudaSuccess) ce = cudaEventRecord(e1);
    if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return ce;
}

bool tma_supported(const Params &P, int prec)
{
    const int sh = prec == 0 ? TmaShape<double>::SH : TmaShape<float>::SH;
    return P.pitch >= TmaShape<float>::SW && P.ny + 4 >= sh && P.nx >= kTmaTX;
}

template <typename R, bool Dev, bool Wrap>
static void launch_tma_lim(const Params &P, const CUtensorMap &tm, const R *a, R *b, int *err, cudaStream_t st)
{
    using S = TmaShape<R>;
    const dim3 block(kTmaTX, S::TT);
    const dim3 grid((P.nx + kTmaTX - 1) / kTmaTX, (P.ny + S::TR - 1) / S::TR);
    if (P.limiter == 0) k_step_tma<R, Dev, 0, Wrap><<<grid, block, S::smem_bytes, st>>>(P, tm, a, b, err);
    else if (P.limiter == 1) k_step_tma<R, Dev, 1, Wrap><<<grid, block, S::smem_bytes, st>>>(P, tm, a, b, err);
    else k_step_tma<R, Dev, 2, Wrap><<<grid, block, S::smem_bytes, st>>>(P, tm, a, b, err);
}

cudaError_t launch_step_tma(const Params &P, int prec, const void *tmap, const void *fin, void *fout, int *err,
                            cudaStream_t st)
{
    const CUtensorMap &tm = *reinterpret_cast<const CUtensorMap *>(tmap);
    const bool wrap = (P.wrap & 1) != 0;
    if (prec == 0) {
        const double *a = (const double *)fin;
        double *b = (double *)fout;
        if (wrap) launch_tma_lim<double, false, true>(P, tm, a, b, err, st);
        else launch_tma_lim<double, false, false>(P, tm, a, b, err, st);
    } else {
        const float *a = (const float *)fin;
        float *b = (float *)fout;
        if (wrap) launch_tma_lim<float, true, true>(P, tm, a, b, err, st);
        else launch_tma_lim<float, true, false>(P, tm, a, b, err, st);
    }
    return cudaGetLastError();
}

cudaError_t tma_prepare()
{
    cudaError_t e = cudaSuccess;
    auto set = [&](const void *fn, size_t bytes) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    };
    set((const void *)k_step_tma<double, false, 0, false>, TmaShape<double>::smem_bytes);
    set((const void *)k_step_tma<double, false, 1, false>, TmaShape<double>::smem_bytes);
    set((const void *)k_step_tma<double, false, 2, false>, TmaShape<double>::smem_bytes);
    set((const void *)k_step_tma<double, false, 0, true>, TmaShape<double>::smem_bytes);
    set((const void *)k_step_tma<double, false, 1, true>, TmaShape<double>::smem_bytes);
    set((const void *)k_step_tma<double, false, 2, true>, TmaShape<double>::smem_bytes);
    set((const void *)k_step_tma<float, true, 0, false>, TmaShape<float>::smem_bytes);
    set((const void *)k_step_tma<float, true, 1, false>, TmaShape<float>::smem_bytes);
    set((const void *)k_step_tma<float, true, 2, false>, TmaShape<float>::smem_bytes);
    set((const void *)k_step_tma<float, true, 0, true>, TmaShape<float>::smem_bytes);
    set((const void *)k_step_tma<float, true, 1, true>, TmaShape<float>::smem_bytes);
    set((const void *)k_step_tma<float, true, 2, true>, TmaShape<float>::smem_bytes);
    set((const void *)k_step_tma_batch<0>, TmaShape<float>::smem_bytes);
    set((const void *)k_step_tma_batch<1>, TmaShape<float>::smem_bytes);
    set((const void *)k_step_tma_batch<2>, TmaShape<float>::smem_bytes);
    return e;
}

}  // namespace lbm
