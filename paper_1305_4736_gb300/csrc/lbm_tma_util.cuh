// lbm_tma_util.cuh -- device helpers shared by the shared-memory-staged step
// kernels: stencil orientation of each population, the bounded mbarrier wait,
// and the limited flux difference in scalar and packed float32-pair form.
#pragma once

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

// Waits on an mbarrier phase.  try_wait carries a suspend-time hint, so a waiting warp
// sleeps until the phase completes (or the hint runs out) instead of spinning on issue
// slots that the other warps need; the wait as a whole is bounded by the global timer.
constexpr unsigned kWaitHintNs = 20000;
constexpr unsigned long long kWaitLimitNs = 2000000000ull;   // 2 s

__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned phase)
{
    unsigned done;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(done) : "r"(bar), "r"(phase), "r"(kWaitHintNs) : "memory");
    return done != 0;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait on phase `phase` of an mbarrier (true when the phase completed).
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned phase)
{
    if (mbar_try_wait(bar, phase)) return true;
    const unsigned long long t0 = global_ns();
    while (global_ns() - t0 < kWaitLimitNs)
        if (mbar_try_wait(bar, phase)) return true;
    return false;
}

// As mbar_wait, but gives up early once another warp of the CTA has raised `abort`.
__device__ __forceinline__ bool mbar_wait_or_abort(unsigned bar, unsigned phase, const volatile int *abort)
{
    if (mbar_try_wait(bar, phase)) return true;
    const unsigned long long t0 = global_ns();
    while (global_ns() - t0 < kWaitLimitNs) {
        if (mbar_try_wait(bar, phase)) return true;
        if (*abort) return false;
    }
    return false;
}

template <typename R, int Lim>
__device__ __forceinline__ R slope2(R a, R b)
{
    return Lim == 0 ? mc2(a, b) : (Lim == 1 ? R(2.0) * b : R(0.0));
}

// x halo of a tile at a periodic x edge: the staged cells left of column 0 or right of column
// nx-1 (the ghost columns, and columns beyond them in a ragged last tile) take the values of
// the wrapped interior cells of fin, as the periodic ghost fill would have written them.  The
// ghost rows come from the ghost fill (contiguous rows, cheap to copy); cells outside along
// both axes are corners of the ring, which the cross stencil of stored cells never reads.
template <typename R>
__device__ __noinline__ void wrap_halo(const Params &P, const R *__restrict__ fin, R *tile, int x0, int y0, int tid,
                                       int nthreads)
{
    using S = TmaShape<R>;
    for (int k = tid; k < S::SW * S::SH; k += nthreads) {
        const int c = k % S::SW, r = k / S::SW;
        const int x = x0 + c - S::HX, y = y0 + r - 2;
        if (!(x < 0 || x >= P.nx) || y < 0 || y >= P.ny) continue;
        const int xs = ((x % P.nx) + P.nx) % P.nx;
        const long long src = (long long)(y + OY) * P.pitch + (xs + OX);
        if constexpr (sizeof(R) == sizeof(float)) {
            const float2 *f2 = reinterpret_cast<const float2 *>(fin);
            float2 *t2 = reinterpret_cast<float2 *>(tile);
#pragma unroll
            for (int pr = 0; pr < 8; pr++) t2[pr * S::PL + k] = f2[pr * P.plane + src];
        } else {
#pragma unroll
            for (int q = 0; q < NQ; q++) tile[q * S::PL + k] = fin[q * P.plane + src];
        }
    }
}

// ---- packed float32 pairs (Blackwell f32x2 arithmetic) -------------------
// Populations q and q + 4 (q = 0..3 axis shells 1 and 2, q = 8..11 diagonal shells 3 and 4)
// move in the same direction: their stencils have the same offsets and only the per-shell
// constants differ, so their convection runs as one float2 per pair.

// Batched launches: the grid of tile b (the largest k with first[k] <= b, a binary search on
// the parameter block, uniform across the CTA) and the tile's origin (grid k's tiles start at
// row y0[k]).
__device__ __forceinline__ int batch_tile(const TmaBatchArgs &A, int b, int tr, int &x0, int &y0)
{
    int lo = 0, hi = A.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (A.first[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    const int local = b - A.first[lo], nt = A.ntx[lo];
    const int ty = local / nt;
    x0 = (local - ty * nt) * kTmaTX;
    y0 = A.y0[lo] + ty * tr;
    return lo;
}

// Prologue of a batched tile CTA (thread 0): initialise the tile barrier, issue the copy of
// grid g's tile at (x0, y0) (tiles of TR rows; the x origin HX columns left of the tile's first
// interior column), and with ctas > 0 (resident CTAs per SM) prefetch into L2 the tile half a
// resident wave further down the launch.
template <int TR, int HX>
__device__ __forceinline__ void batch_issue(const TmaBatchArgs &A, int g, int x0, int y0, unsigned dst,
                                            unsigned bar_a, unsigned bytes, int ctas)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_a) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_a), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3, %4}], [%5];"
                 ::"r"(dst), "l"(reinterpret_cast<unsigned long long>(&A.map[g])), "r"(x0 + OX - HX), "r"(y0),
                 "r"(0), "r"(bar_a) : "memory");
    if (ctas <= 0) return;
    unsigned nsm;
    asm("mov.u32 %0, %%nsmid;" : "=r"(nsm));
    const long long bn = (long long)blockIdx.x + (long long)ctas * nsm / 2;
    if (bn < A.first[A.n]) {
        int xn, yn;
        const int gn = batch_tile(A, (int)bn, TR, xn, yn);
        asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];"
                     ::"l"(reinterpret_cast<unsigned long long>(&A.map[gn])), "r"(xn + OX - HX), "r"(yn), "r"(0)
                     : "memory");
    }
}

template <int Lim>
__device__ __forceinline__ float2 slope2x2(float2 a, float2 b)
{
    if (Lim == 2) return f2(0.f, 0.f);
    if (Lim == 1) return mul2(b, f2(2.f, 2.f));
    // as mc2(float), per lane: t = +-min(|a|, |b|), positive when a and b agree in sign;
    // the result carries the sign of a + b and the magnitude min(4 max(t, 0), |a + b|)
    const float2 s = add2(a, b);
    float tx, ty;
    asm("min.xorsign.abs.f32 %0, %1, %2;" : "=f"(tx) : "f"(a.x), "f"(b.x));
    asm("min.xorsign.abs.f32 %0, %1, %2;" : "=f"(ty) : "f"(a.y), "f"(b.y));
    const float2 t4 = mul2(f2(tx, ty), f2(4.f, 4.f));
    const float mx = fmaxf(t4.x, 0.f), my = fmaxf(t4.y, 0.f);
    float rx, ry;
    asm("min.xorsign.abs.f32 %0, %1, %2;" : "=f"(rx) : "f"(mx), "f"(s.x));
    asm("min.xorsign.abs.f32 %0, %1, %2;" : "=f"(ry) : "f"(my), "f"(s.y));
    return f2(rx, ry);
}

// (F_out - F_in) of a pair in upwind order (f_{J-2s}, f_{J-s}, f_J, f_{J+s}); hh = h/2 per member.
template <int Lim>
__device__ __forceinline__ float2 flux_diff2(float2 fmm, float2 fm, float2 f0, float2 fp, float2 hh)
{
    const float2 d1 = sub2(f0, fm);
    if (Lim == 2) return d1;
    const float2 d2 = sub2(fp, f0);
    const float2 d0 = sub2(fm, fmm);
    return __ffma2_rn(hh, sub2(slope2x2<Lim>(d1, d2), slope2x2<Lim>(d0, d1)), d1);
}


}  // namespace
}  // namespace lbm
