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

namespace lbm {

namespace {

__device__ __forceinline__ constexpr int tsgn_x(int q)
{
    return q < 8 ? ((q & 3) == 0 ? 1 : ((q & 3) == 2 ? -1 : 0)) : (((q & 3) == 0 || (q & 3) == 3) ? 1 : -1);
}
__device__ __forceinline__ constexpr int tsgn_y(int q)
{
    return q < 8 ? ((q & 3) == 1 ? 1 : ((q & 3) == 3 ? -1 : 0)) : (((q & 3) <= 1) ? 1 : -1);
}

__device__ __forceinline__ bool tu_cell(int x, int y, int nx, int ny)
{
    return (x >= -1 && x <= nx && y >= 0 && y < ny) || (y >= -1 && y <= ny && x >= 0 && x < nx);
}

// Bounded wait on phase `phase` of an mbarrier (true when the phase completed).
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned phase)
{
    for (int i = 0; i < (1 << 22); i++) {
        unsigned done;
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done) : "r"(bar), "r"(phase) : "memory");
        if (done) return true;
    }
    return false;
}

template <typename R, int Lim>
__device__ __forceinline__ R slope2(R a, R b)
{
    return Lim == 0 ? mc2(a, b) : (Lim == 1 ? R(2.0) * b : R(0.0));
}

}  // namespace

template <typename R, bool Dev, int Lim>
__global__ void __launch_bounds__(kTmaTX * kTmaTT, sizeof(R) == 4 ? 2 : 1)
k_step_tma(const __grid_constant__ Params P, const __grid_constant__ CUtensorMap tm, R *__restrict__ fout,
           int *err)
{
    using S = TmaShape<R>;
    extern __shared__ __align__(128) unsigned char smraw[];
    R *tile = reinterpret_cast<R *>(smraw);
    R *su = tile + NQ * S::PL;
    R *sv = su + S::UW * S::UH;
    R *sir = sv + S::UW * S::UH;
    __shared__ __align__(8) unsigned long long bar;

    const int lane = threadIdx.x, ty = threadIdx.y, tid = ty * kTmaTX + lane;
    const int x0 = blockIdx.x * kTmaTX, y0 = blockIdx.y * S::TR;
    const int nx = P.nx, ny = P.ny;
    const unsigned bar_a = (unsigned)__cvta_generic_to_shared(&bar);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_a) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0) {
        // box origin: interior column x0 - 4 = padded column x0; interior row y0 - 2 = padded row y0
        const unsigned dst = (unsigned)__cvta_generic_to_shared(tile);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_a),
                     "r"((unsigned)S::tile_bytes) : "memory");
        asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                     " [%0], [%1, {%2, %3, %4}], [%5];"
                     ::"r"(dst), "l"(reinterpret_cast<unsigned long long>(&tm)), "r"(x0), "r"(y0), "r"(0),
                     "r"(bar_a) : "memory");
    }
    if (!mbar_wait(bar_a, 0)) {
        if (tid == 0) atomicExch(err, 1);
        mbar_wait(bar_a, 0);               // let a late copy land before the CTA exits (bounded)
        return;
    }

    const Coef<R> &C = coef<R>(P);
    // ---- phase 1: flow velocity and 1/rho on the tile plus its ring
    for (int k = tid; k < S::UW * S::UH; k += kTmaTX * kTmaTT) {
        const int i = k % S::UW, j = k / S::UW;
        R ux = R(0), uy = R(0), ir = R(0);
        if (tu_cell(x0 - 1 + i, y0 - 1 + j, nx, ny)) {
            const R *p = tile + (j + 1) * S::SW + (i + 3);
            R g[NQ];
#pragma unroll
            for (int q = 0; q < NQ; q++) g[q] = p[q * S::PL];
            const Shells<R> sh = shells_of(g);
            R drho, jx, jy, de;
            conserved_of(sh, drho, jx, jy, de);
            const R rho = Dev ? C.rho0 + drho : drho;
            ir = recip(rho);
            ux = jx * ir;
            uy = jy * ir;
        }
        su[k] = ux;
        sv[k] = uy;
        sir[k] = ir;
    }
    __syncthreads();

    // ---- phase 2: rows ty*KR .. ty*KR+KR-1 of the tile, column `lane`
    const int gx = x0 + lane;
    const int r0 = ty * S::KR;
    // sliding y-window state per y-moving population: last value, face difference, slope
    R yw[NQ], yd[NQ], ym[NQ];
#pragma unroll
    for (int q = 0; q < NQ; q++) {
        const int sy = tsgn_y(q);
        if (sy == 0) continue;
        const R *pc = tile + q * S::PL + (lane + 4);
        // window index m <-> smem row r0 + m (tile row r0 + m - 2); D[m] = w[m+1] - w[m]
        if (sy > 0) {
            // oriented slope at index c: slope2(D[c-1], D[c]); carry w[2], D[1], slope at index 1
            const R w0 = pc[r0 * S::SW], w1 = pc[(r0 + 1) * S::SW], w2 = pc[(r0 + 2) * S::SW];
            const R d0 = w1 - w0, d1 = w2 - w1;
            yw[q] = w2;
            yd[q] = d1;
            ym[q] = slope2<R, Lim>(d0, d1);
        } else {
            // oriented slope at index c: slope2(-D[c], -D[c-1]); carry w[3], D[2], slope at index 2
            const R w1 = pc[(r0 + 1) * S::SW], w2 = pc[(r0 + 2) * S::SW], w3 = pc[(r0 + 3) * S::SW];
            const R d1 = w2 - w1, d2 = w3 - w2;
            yw[q] = w3;
            yd[q] = d2;
            ym[q] = slope2<R, Lim>(-d2, -d1);
        }
    }

#pragma unroll 1
    for (int k = 0; k < S::KR; k++) {
        const int r = r0 + k;
        const int gy = y0 + r;
        const R *p = tile + (r + 2) * S::SW + (lane + 4);
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
        collide<R, Dev>(P, sh, drho, jx, jy, de, ir, dxux, dyux, dxuy, dyuy, acc);
        const bool store = gx < nx && gy < ny;
        const long long cg = (long long)(gy + OY) * P.pitch + (gx + OX);
#pragma unroll
        for (int q = 0; q < NQ; q++) {
            const int sx = tsgn_x(q), sy = tsgn_y(q);
            const int shell = q >> 2;
            const R hh = C.hh[shell];
            R tx = R(0), tyv = R(0);
            if (sx != 0) {
                // both slopes from the staged row (sharing the upwind slope with the
                // neighbouring lane would cost a shuffle plus a boundary-lane fix-up)
                const R *pr = p + q * S::PL;
                const R fm2 = pr[-2 * sx], fm1 = pr[-sx], fp1 = pr[sx];
                tx = flux_diff<R, Lim>(fm2, fm1, f[q], fp1, hh);
            }
            if (sy != 0) {
                const R *pc = tile + q * S::PL + (lane + 4);
                // next window value: smem row r0 + k + 3 (sy > 0) or r0 + k + 4 (sy < 0)
                const R wn = pc[(r + (sy > 0 ? 3 : 4)) * S::SW];
                const R dn = wn - yw[q];
                if (sy > 0) {
                    // D[k+2], slope at J = index k+2; flux D[k+1] + h (slope_J - slope_{J-1})
                    const R mn = slope2<R, Lim>(yd[q], dn);
                    tyv = Lim == 2 ? yd[q] : yd[q] + hh * (mn - ym[q]);
                    ym[q] = mn;
                } else {
                    // D[k+3], slope at J - sigma = index k+3; flux -D[k+2] + h (slope_J - slope_{J+1})
                    const R mn = slope2<R, Lim>(-dn, -yd[q]);
                    tyv = Lim == 2 ? -yd[q] : -yd[q] + hh * (ym[q] - mn);
                    ym[q] = mn;
                }
                yw[q] = wn;
                yd[q] = dn;
            }
            const R tot = (sx != 0 && sy != 0) ? tx + tyv : (sx != 0 ? tx : tyv);
            if (store) fout[q * P.plane + cg] = (f[q] - acc[q]) - C.cr[shell] * tot;
        }
    }
}

// ---------------------------------------------------------------------------
bool tma_supported(const Params &P)
{
    return P.pitch >= kTmaTX + 8 && P.ny + 4 >= TmaShape<float>::SH && P.nx >= kTmaTX;
}

cudaError_t launch_step_tma(const Params &P, int prec, const void *tmap, void *fout, int *err, cudaStream_t st)
{
    const CUtensorMap &tm = *reinterpret_cast<const CUtensorMap *>(tmap);
    const dim3 block(kTmaTX, kTmaTT);
    if (prec == 0) {
        using S = TmaShape<double>;
        const dim3 grid((P.nx + kTmaTX - 1) / kTmaTX, (P.ny + S::TR - 1) / S::TR);
        double *b = (double *)fout;
        if (P.limiter == 0) k_step_tma<double, false, 0><<<grid, block, S::smem_bytes, st>>>(P, tm, b, err);
        else if (P.limiter == 1) k_step_tma<double, false, 1><<<grid, block, S::smem_bytes, st>>>(P, tm, b, err);
        else k_step_tma<double, false, 2><<<grid, block, S::smem_bytes, st>>>(P, tm, b, err);
    } else {
        using S = TmaShape<float>;
        const dim3 grid((P.nx + kTmaTX - 1) / kTmaTX, (P.ny + S::TR - 1) / S::TR);
        float *b = (float *)fout;
        if (P.limiter == 0) k_step_tma<float, true, 0><<<grid, block, S::smem_bytes, st>>>(P, tm, b, err);
        else if (P.limiter == 1) k_step_tma<float, true, 1><<<grid, block, S::smem_bytes, st>>>(P, tm, b, err);
        else k_step_tma<float, true, 2><<<grid, block, S::smem_bytes, st>>>(P, tm, b, err);
    }
    return cudaGetLastError();
}

cudaError_t tma_prepare()
{
    cudaError_t e = cudaSuccess;
    auto set = [&](const void *fn, size_t bytes) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    };
    set((const void *)k_step_tma<double, false, 0>, TmaShape<double>::smem_bytes);
    set((const void *)k_step_tma<double, false, 1>, TmaShape<double>::smem_bytes);
    set((const void *)k_step_tma<double, false, 2>, TmaShape<double>::smem_bytes);
    set((const void *)k_step_tma<float, true, 0>, TmaShape<float>::smem_bytes);
    set((const void *)k_step_tma<float, true, 1>, TmaShape<float>::smem_bytes);
    set((const void *)k_step_tma<float, true, 2>, TmaShape<float>::smem_bytes);
    return e;
}

}  // namespace lbm
