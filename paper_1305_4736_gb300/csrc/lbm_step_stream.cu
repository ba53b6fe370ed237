// lbm_step_stream.cu -- streaming fused step kernel (sm_103a).
//
// Each CTA (8 warps) owns a 256-column strip of the grid and marches down a
// contiguous range of its rows; the ranges of all CTAs split strips x rows
// evenly (a range that reaches the bottom of a strip continues at the top of
// the next one).  Rows of all 16 population planes (the strip plus 4 halo
// columns on each side) stream through a ring of shared-memory slots.  A slot
// is filled by two tensor copies (cp.async.bulk.tensor, 136 columns each; the
// halves overlap by 8 columns so that every warp's stencil lies inside one
// half) that complete on the slot's mbarrier, and it is refilled with the row
// SLOTS further on by the warp that releases it last.  The warps advance
// independently; warp w updates columns 32w .. 32w+31 of the strip, one row
// per step:
//   - flow velocity of the next row at its own column (u(y+1), kept in
//     registers with u(y) and u(y-1)) and of the two columns left and right of
//     the warp in row y (a 16-lane reduction; float64 reduces rows y and y+1
//     together every other row), for the gradient of u;
//   - MRT collision with the energy-flux correction (Eq. 3, Sec. II);
//   - limited x convection from the staged row; limited y convection from a
//     sliding window per thread that lives for the whole range (each slope
//     computed once, Sec. III);
//   - one global write per population.
// Per-value arithmetic is that of the plain kernel; results agree with it to
// round-off (summation order of the halo velocities, multiply-add contraction).
#include <cuda.h>

#include <type_traits>

#include "lbm_internal.h"
#include "lbm_tma_util.cuh"

namespace lbm {

namespace {

// A CTA's share [b, e) of the sequence strip-major (strip, row), and the row
// copies it implies: each maximal run of rows y0 .. y1-1 of one strip (a
// segment) needs the rows y0-2 .. y1+1, in that order.
struct Span {
    long long b, e;   // share of the strip-major (strip, row) sequence
    int K1;           // copies of the first segment
    int ny;

    __device__ void coords(int k, int &strip, int &row) const
    {
        int j, K, y0;
        if (k < K1) {
            j = 0;
            K = 0;
            y0 = (int)(b % ny);
        } else {
            const int jj = (k - K1) / (ny + 4);
            j = 1 + jj;
            K = K1 + jj * (ny + 4);
            y0 = 0;
        }
        strip = (int)(b / ny) + j;
        row = y0 + (k - K) - 2;
    }
};

// Ring position of copy index k: slot k % SLOTS and the parity (k / SLOTS) & 1 of the
// slot's mbarrier phase that the copy completes; advanced one copy at a time.
template <int SLOTS>
struct RingPos {
    int slot;
    unsigned phase;
    __device__ __forceinline__ void set(int k)
    {
        slot = k % SLOTS;
        phase = (unsigned)(k / SLOTS) & 1u;
    }
    __device__ __forceinline__ void next()
    {
        if (++slot == SLOTS) {
            slot = 0;
            phase ^= 1u;
        }
    }
};

template <typename R>
__device__ __forceinline__ void issue_row(const CUtensorMap *tm, const Span &sp, int k, unsigned ring_a,
                                          unsigned bar_a)
{
    using S = StreamShape<R>;
    int strip, row;
    sp.coords(k, strip, row);
    const int slot = k % S::SLOTS;
    const unsigned bar = bar_a + 8u * (unsigned)slot;
    const unsigned dst = ring_a + (unsigned)slot * (unsigned)(S::ROW * sizeof(R));
    const int x = strip * S::W;   // padded column of interior column strip * W - 4
    const int y = row + OY;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(2u * S::copy_bytes)
                 : "memory");
    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3, %4}], [%5];"
                 ::"r"(dst), "l"(reinterpret_cast<unsigned long long>(tm)), "r"(x), "r"(y), "r"(0), "r"(bar)
                 : "memory");
    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3, %4}], [%5];"
                 ::"r"(dst + S::copy_bytes), "l"(reinterpret_cast<unsigned long long>(tm)), "r"(x + S::W / 2),
                 "r"(y), "r"(0), "r"(bar)
                 : "memory");
}

// Flow velocity of one cell from 16 lanes (lane q holds population q at p, with
// velocity (cx, cy)); lanes 0-15 and 16-31 reduce independently.
template <typename R, bool Dev>
__device__ __forceinline__ void halo_velocity(const Coef<R> &C, const R *p, R cx, R cy, R &u, R &v)
{
    const R g = *p;
    R a = g, bx = cx * g, by = cy * g;
#pragma unroll
    for (int o = 8; o >= 1; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        bx += __shfl_xor_sync(0xffffffffu, bx, o);
        by += __shfl_xor_sync(0xffffffffu, by, o);
    }
    const R rho = Dev ? C.rho0 + a : a;
    const R ir = recip(rho);
    u = bx * ir;
    v = by * ir;
}

// float64: the flow velocities of halo_velocity for two rows at once, the cell at p (row y) and
// the cell at q (row y+1).  The first level of the 16-lane reductions serves both rows: lanes
// with bit 3 clear go on with row y, the others with row y+1, and the reciprocal and the
// divisions run once for both.  Every lane of a pair adds the same two partial sums, so the
// sums are those of halo_velocity bit for bit.  u0, v0: row y of this lane's column (lanes 0-15
// the left one, 16-31 the right one); u1, v1: row y+1.
__device__ __forceinline__ void halo_velocity2(const double *p, const double *q, double cx, double cy, int lane,
                                               double &u0, double &v0, double &u1, double &v1)
{
    constexpr unsigned kAll = 0xffffffffu;
    const double ga = *p, gb = *q;
    const double xa = cx * ga, ya = cy * ga, xb = cx * gb, yb = cy * gb;
    const bool hi = (lane & 8) != 0;
    double a = hi ? gb : ga, bx = hi ? xb : xa, by = hi ? yb : ya;            // kept
    a += __shfl_xor_sync(kAll, hi ? ga : gb, 8);                                // the partner's
    bx += __shfl_xor_sync(kAll, hi ? xa : xb, 8);
    by += __shfl_xor_sync(kAll, hi ? ya : yb, 8);
#pragma unroll
    for (int o = 4; o >= 1; o >>= 1) {
        a += __shfl_xor_sync(kAll, a, o);
        bx += __shfl_xor_sync(kAll, bx, o);
        by += __shfl_xor_sync(kAll, by, o);
    }
    const double ir = recip(a);
    const double u = bx * ir, v = by * ir;
    const int base = lane & 16;
    u0 = __shfl_sync(kAll, u, base);
    v0 = __shfl_sync(kAll, v, base);
    u1 = __shfl_sync(kAll, u, base + 8);
    v1 = __shfl_sync(kAll, v, base + 8);
}

// Sliding y-window per thread: last value, face difference and oriented slope of
// each y-moving population (float32: per population pair).
template <typename R> struct Win;
template <> struct Win<float> { float2 w[8], d[8], m[8]; };
template <> struct Win<double> { double w[NQ], d[NQ], m[NQ]; };

// float64: the shells and conserved moments of a row, computed for its flow velocity one step
// before its collision, are carried to that collision (the float64 pipe bounds that kernel).
struct Carry64 {
    Shells<double> sh;
    double drho, jx, jy, de;
};

template <bool Dev>
__device__ __forceinline__ void moments_at(const Coef<double> &C, const double *p, Carry64 &c, double &u, double &v,
                                           double &ir)
{
    constexpr int BW = StreamShape<double>::BW;
    double g[NQ];
#pragma unroll
    for (int q = 0; q < NQ; q++) g[q] = p[q * BW];
    c.sh = shells_of(g);
    conserved_of(c.sh, c.drho, c.jx, c.jy, c.de);
    const double rho = Dev ? C.rho0 + c.drho : c.drho;
    ir = recip(rho);
    u = c.jx * ir;
    v = c.jy * ir;
}

// float64 MC x convection shared between lanes.  For an x-moving population with sign s,
// D(x) = f(x) - f(x-s) and the slope Sl(x) = mc2(D(x), D(x+s)); the flux difference at x is
// D(x) + h (Sl(x) - Sl(x-s)).  Each lane forms D and Sl at its own column once and takes
// D(x+s) and Sl(x-s) from its neighbours by shuffles.  The two lanes at the warp's edges
// need values one column outside the warp: per row, lanes 0..11 form D beyond the downwind
// edge of x-stencil k = lane, and lanes 12..23 the slope before the upwind edge of
// stencil k = lane - 12, in three float64 instructions for all twelve stencils.
__host__ __device__ __forceinline__ constexpr int xstencil_q(int k) { return k < 4 ? 2 * k : k + 4; }
__host__ __device__ __forceinline__ constexpr int xstencil_of(int q) { return q < 8 ? q >> 1 : q - 4; }

struct XEdge {
    int o0, o1, o2;   // this lane's three row offsets (plane * BW + column)
    double t1, E;     // lanes 0..11: D beyond the downwind edge; lanes 12..23: D(xu), Sl(xu - s)
};

// Offsets of the edge values for this lane; wcol: column of the warp's first cell in its
// half row (the warp's columns are wcol .. wcol + 31).
__device__ __forceinline__ void xedge_setup(XEdge &e, int lane, int wcol)
{
    constexpr int BW = StreamShape<double>::BW;
    const bool down = lane < 12;
    const int k = down ? lane : (lane - 12 < 11 ? lane - 12 : 11);
    const int q = xstencil_q(k), sx = tsgn_x(q);
    const int base = q * BW + wcol;
    if (down) {
        const int xd = sx > 0 ? 31 : 0;              // downwind edge lane's column
        e.o0 = base + xd;
        e.o1 = base + xd;
        e.o2 = base + xd + sx;                       // D(xd + s) = f(xd + s) - f(xd)
    } else {
        const int xu = sx > 0 ? 0 : 31;              // upwind edge lane's column
        e.o0 = base + xu - 2 * sx;
        e.o1 = base + xu - sx;
        e.o2 = base + xu;                            // Sl(xu - s) = mc2(D(xu - s), D(xu))
    }
}

__device__ __forceinline__ void xedge_row(XEdge &e, const double *row)
{
    const double p0 = row[e.o0], p1 = row[e.o1], p2 = row[e.o2];
    e.t1 = p2 - p1;
    e.E = mc2(p1 - p0, e.t1);
}

// Window at the first row y0 of a segment from rows y0-2 (a), y0-1 (b), y0 (c), y0+1 (d).
// sy > 0: oriented slope at index c is slope2(D[c-1], D[c]) (D[m] = w[m+1] - w[m]); carry
//         w(y0), D between y0-1 and y0, slope at y0-1.
// sy < 0: oriented slope at index c is slope2(-D[c], -D[c-1]); carry w(y0+1), D between y0
//         and y0+1, slope at y0.
template <int Lim>
__device__ __forceinline__ void win_init(Win<float> &W, const float2 *a, const float2 *b, const float2 *c,
                                         const float2 *d)
{
    constexpr int BW = StreamShape<float>::BW;
#pragma unroll
    for (int pr = 0; pr < 8; pr++) {
        const int sy = tsgn_y(pair_q(pr));
        if (sy == 0) continue;
        const int o = pr * BW;
        if (sy > 0) {
            const float2 d0 = sub2(b[o], a[o]), d1 = sub2(c[o], b[o]);
            W.w[pr] = c[o];
            W.d[pr] = d1;
            W.m[pr] = slope2x2<Lim>(d0, d1);
        } else {
            const float2 d1 = sub2(c[o], b[o]), d2 = sub2(d[o], c[o]);
            W.w[pr] = d[o];
            W.d[pr] = d2;
            W.m[pr] = slope2x2<Lim>(d2, d1);   // the oriented slope, negated (slope2x2 is odd)
        }
    }
}

template <int Lim>
__device__ __forceinline__ void win_init(Win<double> &W, const double *a, const double *b, const double *c,
                                         const double *d)
{
    constexpr int BW = StreamShape<double>::BW;
#pragma unroll
    for (int q = 0; q < NQ; q++) {
        const int sy = tsgn_y(q);
        if (sy == 0) continue;
        const int o = q * BW;
        if (sy > 0) {
            const double d0 = b[o] - a[o], d1 = c[o] - b[o];
            W.w[q] = c[o];
            W.d[q] = d1;
            W.m[q] = slope2<double, Lim>(d0, d1);
        } else {
            const double d1 = c[o] - b[o], d2 = d[o] - c[o];
            W.w[q] = d[o];
            W.d[q] = d2;
            W.m[q] = slope2<double, Lim>(d2, d1);   // the oriented slope, negated (slope2 is odd)
        }
    }
}

// Convection of row y and the write of the new populations.  s0, s1, s2: rows y, y+1, y+2
// at this thread's column; f: populations of the cell; acc: collision term.
template <int Lim>
__device__ __forceinline__ void convect_store(const Coef<float> &C, Win<float> &W, const float2 *fp, const float2 *acc,
                                              const float2 *s0, const float2 *s1, const float2 *s2, bool store,
                                              float *__restrict__ fout, long long plane, long long cg)
{
    constexpr int BW = StreamShape<float>::BW;
    float2 *out2 = reinterpret_cast<float2 *>(fout);
#pragma unroll
    for (int pr = 0; pr < 8; pr++) {
        const int qa = pair_q(pr);
        const int sx = tsgn_x(qa), sy = tsgn_y(qa);
        const int sa = qa >> 2;
        const int o = pr * BW;
        const float2 hy = ld2(&C.hhy[sa]);
        const float2 f0 = fp[pr];
        float2 tx = f2(0.f, 0.f), tyv = f2(0.f, 0.f);
        if (sx != 0) tx = flux_diff2<Lim>(s0[o - 2 * sx], s0[o - sx], f0, s0[o + sx], ld2(&C.hh[sa]));
        if (sy != 0) {
            const float2 wn = (sy > 0 ? s1 : s2)[o];
            const float2 dn = sub2(wn, W.w[pr]);
            if (sy > 0) {
                // flux D(y) + h (slope_y - slope_{y-1})
                const float2 mn = slope2x2<Lim>(W.d[pr], dn);
                tyv = Lim == 2 ? W.d[pr] : fma2(hy, sub2(mn, W.m[pr]), W.d[pr]);
                W.m[pr] = mn;
            } else {
                // flux -D(y+1) + h (slope_y - slope_{y+1}), carried negated with negated slopes
                const float2 mn = slope2x2<Lim>(dn, W.d[pr]);
                tyv = Lim == 2 ? W.d[pr] : fma2(hy, sub2(W.m[pr], mn), W.d[pr]);
                W.m[pr] = mn;
            }
            W.w[pr] = wn;
            W.d[pr] = dn;
        }
        // f - C - c_x (F_out - F_in)_x - c_y (F_out - F_in)_y
        float2 out = sub2(f0, acc[pr]);
        if (sy > 0) out = fma2(ld2(&C.ncry[sa]), tyv, out);
        if (sy < 0) out = fma2(ld2(&C.cry[sa]), tyv, out);
        if (sx != 0) out = fma2(ld2(&C.ncr[sa]), tx, out);
        if (store) out2[pr * plane + cg] = out;
    }
}

template <int Lim>
__device__ __forceinline__ void convect_store(const Coef<double> &C, Win<double> &W, const double *f,
                                              const double *acc, const double *s0, const double *s1,
                                              const double *s2, bool store, double *__restrict__ fout,
                                              long long plane, long long cg, const XEdge &xe, int lane)
{
    constexpr int BW = StreamShape<double>::BW;
    constexpr unsigned kAll = 0xffffffffu;
#pragma unroll
    for (int q = 0; q < NQ; q++) {
        const int sx = tsgn_x(q), sy = tsgn_y(q);
        const int shell = q >> 2;
        const int o = q * BW;
        const double hy = C.hhy[shell];
        double tx = 0.0, tyv = 0.0;
        if (sx != 0 && Lim == 0) {
            const int k = xstencil_of(q);
            const double D = f[q] - s0[o - sx];
            double Dn = sx > 0 ? __shfl_down_sync(kAll, D, 1) : __shfl_up_sync(kAll, D, 1);
            const double De = __shfl_sync(kAll, xe.t1, k);
            if (lane == (sx > 0 ? 31 : 0)) Dn = De;
            const double Sl = mc2(D, Dn);
            double Sp = sx > 0 ? __shfl_up_sync(kAll, Sl, 1) : __shfl_down_sync(kAll, Sl, 1);
            const double Se = __shfl_sync(kAll, xe.E, 12 + k);
            if (lane == (sx > 0 ? 0 : 31)) Sp = Se;
            tx = D + C.hh[shell] * (Sl - Sp);
        } else if (sx != 0) {
            tx = flux_diff<double, Lim>(s0[o - 2 * sx], s0[o - sx], f[q], s0[o + sx], C.hh[shell]);
        }
        if (sy != 0) {
            const double wn = (sy > 0 ? s1 : s2)[o];
            const double dn = wn - W.w[q];
            if (sy > 0) {
                const double mn = slope2<double, Lim>(W.d[q], dn);
                tyv = Lim == 2 ? W.d[q] : W.d[q] + hy * (mn - W.m[q]);
                W.m[q] = mn;
            } else {
                // negated oriented slopes and flux: slope2 is odd, and float64 negations would
                // take float64 instructions
                const double mn = slope2<double, Lim>(dn, W.d[q]);
                tyv = Lim == 2 ? W.d[q] : W.d[q] + hy * (W.m[q] - mn);
                W.m[q] = mn;
            }
            W.w[q] = wn;
            W.d[q] = dn;
        }
        // f - C - c_x (F_out - F_in)_x - c_y (F_out - F_in)_y
        double out = f[q] - acc[q];
        if (sy > 0) out -= C.cry[shell] * tyv;
        if (sy < 0) out += C.cry[shell] * tyv;
        if (sx != 0) out -= C.cr[shell] * tx;
        if (store) fout[q * plane + cg] = out;
    }
}

}  // namespace

template <typename R, bool Dev, int Lim>
__global__ void __launch_bounds__(32 * StreamShape<R>::WARPS, sizeof(R) == 4 ? 2 : 1)
k_step_stream(const __grid_constant__ Params P, const __grid_constant__ CUtensorMap tm, R *__restrict__ fout,
              int *err)
{
    using S = StreamShape<R>;
    static_assert(sizeof(R) == sizeof(float) || !Dev, "float64 stores f itself (halo_velocity2 takes rho = sum f)");
    constexpr int BW = S::BW;
    extern __shared__ __align__(128) unsigned char smraw[];
    R *ring = reinterpret_cast<R *>(smraw);
    __shared__ __align__(8) unsigned long long full[S::SLOTS];
    __shared__ unsigned released[S::SLOTS];
    __shared__ int abort_flag;
    __shared__ unsigned long long issued;   // row copies issued so far

    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int nx = P.nx, ny = P.ny;
    const long long T = (long long)((nx + S::W - 1) / S::W) * ny;
    Span sp;
    sp.ny = ny;
    sp.b = T * blockIdx.x / gridDim.x;
    sp.e = T * (blockIdx.x + 1) / gridDim.x;
    const long long first_end = sp.b / ny * ny + ny;
    sp.K1 = (int)((sp.e < first_end ? sp.e : first_end) - sp.b) + 4;
    const int nseg = sp.e > sp.b ? (int)((sp.e - 1) / ny - sp.b / ny + 1) : 0;
    const int nload = (int)(sp.e - sp.b) + 4 * nseg;
    const unsigned ring_a = (unsigned)__cvta_generic_to_shared(ring);
    const unsigned bar_a = (unsigned)__cvta_generic_to_shared(full);

    if (tid == 0) {
        for (int s = 0; s < S::SLOTS; s++) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_a + 8u * s) : "memory");
            released[s] = 0;
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0) {
        const int n0 = nload < S::SLOTS ? nload : S::SLOTS;
        for (int k = 0; k < n0; k++) issue_row<R>(&tm, sp, k, ring_a, bar_a);
        issued = (unsigned long long)n0;
    }

    const Coef<R> &C = coef<R>(P);
    const int h = w >> 2, wl = w & 3;
    const int col = 32 * wl + 4 + lane;                          // column inside this warp's half copy
    const int hcol = lane < 16 ? 32 * wl + 3 : 32 * wl + 36;     // column left / right of the warp
    const int hq = lane & 15;
    const R mag = hq < 4 ? R(1.0) : (hq < 8 ? R(6.0) : (hq < 12 ? R(kD3) : R(kD4)));
    const R cxl = R(tsgn_x(hq)) * mag, cyl = R(tsgn_y(hq)) * mag;
    const R *half = ring + h * S::HALF;
    using Pos = RingPos<S::SLOTS>;
    auto row_at = [&](const Pos &p) { return half + p.slot * S::ROW; };
    // a slot row seen from this lane's column: float64 planes of R, float32 planes of pairs
    using V = std::conditional_t<sizeof(R) == sizeof(float), float2, double>;
    auto colp = [&](const R *row) { return reinterpret_cast<const V *>(row) + col; };
    const int hoff = sizeof(R) == sizeof(float) ? (pair_of(hq) * BW + hcol) * 2 + member_of(hq) : hq * BW + hcol;
    [[maybe_unused]] XEdge xe{};
    if constexpr (sizeof(R) == sizeof(double)) xedge_setup(xe, lane, 32 * wl + 4);
    auto wait = [&](const Pos &p) {
        const bool ok = mbar_wait_or_abort(bar_a + 8u * (unsigned)p.slot, p.phase, &abort_flag);
        if (!ok && lane == 0) *(volatile int *)&abort_flag = 1;
        return ok;
    };
    // copy k (at ring slot `slot`) is no longer read by this warp; the last of the
    // CTA's warps to release it refills the slot with copy k + SLOTS
    auto release = [&](int k, int slot) {
        __syncwarp();
        if (lane == 0) {
            __threadfence_block();
            const unsigned old = atomicAdd(&released[slot], 1u);
            if ((old + 1) % S::WARPS == 0 && k + S::SLOTS < nload) {
                __threadfence_block();
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                issue_row<R>(&tm, sp, k + S::SLOTS, ring_a, bar_a);
                atomicMax(&issued, (unsigned long long)(k + S::SLOTS + 1));
            }
        }
    };

    bool ok = true;
    int kb = 0;   // first copy of the current segment
    for (long long pos = sp.b; ok && pos < sp.e;) {
        const int strip = (int)(pos / ny), y0 = (int)(pos % ny);
        const int len = (int)((long long)(ny - y0) < sp.e - pos ? (long long)(ny - y0) : sp.e - pos);
        const int gx = strip * S::W + 32 * w + lane;
        Pos pa, pb, pc, pd;   // copies kb .. kb+3: rows y0-2 .. y0+1
        pa.set(kb);
        pb = pa;
        pb.next();
        pc = pb;
        pc.next();
        pd = pc;
        pd.next();
        ok = wait(pa) && wait(pb) && wait(pc) && wait(pd);
        if (!ok) break;
        R u_m, v_m, u_0, v_0, ir_0, dummy;
        flow_at<Dev>(C, colp(row_at(pb)), BW, u_m, v_m, dummy);
        [[maybe_unused]] Carry64 c0;      // float64: moments of row y, carried from phase 1
        if constexpr (sizeof(R) == sizeof(float))
            flow_at<Dev>(C, colp(row_at(pc)), BW, u_0, v_0, ir_0);
        else
            moments_at<Dev>(C, colp(row_at(pc)), c0, u_0, v_0, ir_0);
        Win<R> W;
        win_init<Lim>(W, colp(row_at(pa)), colp(row_at(pb)), colp(row_at(pc)), colp(row_at(pd)));
        release(kb, pa.slot);
        release(kb + 1, pb.slot);
        Pos p0 = pc, p1 = pd, p2 = pd;   // rows y, y+1, y+2
        p2.next();
        [[maybe_unused]] R uh_next = R(0), vh_next = R(0);   // float64: halo of row y+1, from the pair
#pragma unroll 1
        for (int i = 0; i < len; i++) {
            if (!(ok = wait(p2))) break;
            const R *r0 = row_at(p0), *r1 = row_at(p1), *r2 = row_at(p2);
            R u_p, v_p, ir_p;
            [[maybe_unused]] Carry64 c1;
            if constexpr (sizeof(R) == sizeof(float))
                flow_at<Dev>(C, colp(r1), BW, u_p, v_p, ir_p);
            else
                moments_at<Dev>(C, colp(r1), c1, u_p, v_p, ir_p);
            R uh, vh;
            if constexpr (sizeof(R) == sizeof(double)) {
                if ((i & 1) == 0) {
                    halo_velocity2(r0 + hoff, r1 + hoff, cxl, cyl, lane, uh, vh, uh_next, vh_next);
                } else {
                    uh = uh_next;
                    vh = vh_next;
                }
            } else {
                halo_velocity<R, Dev>(C, r0 + hoff, cxl, cyl, uh, vh);
            }
            R uxm = __shfl_up_sync(0xffffffffu, u_0, 1), uxp = __shfl_down_sync(0xffffffffu, u_0, 1);
            R vxm = __shfl_up_sync(0xffffffffu, v_0, 1), vxp = __shfl_down_sync(0xffffffffu, v_0, 1);
            if (lane == 0) { uxm = uh; vxm = vh; }
            if (lane == 31) { uxp = uh; vxp = vh; }
            const int y = y0 + i;
            const long long cg = (long long)(y + OY) * P.pitch + (gx + OX);
            if constexpr (sizeof(R) == sizeof(float)) {
                const float2 *s0 = colp(r0);
                float2 fp[8];
#pragma unroll
                for (int pr = 0; pr < 8; pr++) fp[pr] = s0[pr * BW];
                const Shells2 sh = shells2_of(fp);
                float drho, jx, jy, de;
                conserved2_of(sh, drho, jx, jy, de);
                float2 acc[8];
                collide2<Dev>(P, sh, drho, jx, jy, de, ir_0, uxp - uxm, u_p - u_m, vxp - vxm, v_p - v_m, acc);
                convect_store<Lim>(C, W, fp, acc, s0, colp(r1), colp(r2), gx < nx, fout, P.plane, cg);
            } else {
                const double *s0 = colp(r0);
                double f[NQ];
#pragma unroll
                for (int q = 0; q < NQ; q++) f[q] = s0[q * BW];
                double acc[NQ];
                collide<double, Dev>(P, c0.sh, c0.drho, c0.jx, c0.jy, c0.de, ir_0, u_0, v_0, uxp - uxm, u_p - u_m,
                                     vxp - vxm, v_p - v_m, acc);
                if (Lim == 0) xedge_row(xe, r0);
                convect_store<Lim>(C, W, f, acc, s0, colp(r1), colp(r2), gx < nx, fout, P.plane, cg, xe, lane);
                c0 = c1;
            }
            u_m = u_0;
            u_0 = u_p;
            v_m = v_0;
            v_0 = v_p;
            ir_0 = ir_p;
            release(kb + i + 2, p0.slot);
            p0 = p1;
            p1 = p2;
            p2.next();
        }
        if (!ok) break;
        release(kb + len + 2, p0.slot);
        release(kb + len + 3, p1.slot);
        kb += len + 4;
        pos += len;
    }
    if (!ok && lane == 0) atomicExch(err, 1);
    __syncthreads();
    if (tid == 0 && abort_flag) {
        // let copies still in flight land before the CTA's shared memory is released (bounded)
        const int n = (int)issued;
        for (int k = n > S::SLOTS ? n - S::SLOTS : 0; k < n; k++)
            mbar_wait(bar_a + 8u * (unsigned)(k % S::SLOTS), (unsigned)(k / S::SLOTS) & 1u);
    }
}

// ---------------------------------------------------------------------------
bool stream_supported(const Params &P)
{
    return P.pitch >= StreamShape<float>::BW && P.pitch % 4 == 0;
}

template <typename R>
static int stream_ctas(const Params &P, const void *fn)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 32 * StreamShape<R>::WARPS,
                                                  StreamShape<R>::smem_bytes);
    if (sms < 1) sms = 1;
    if (per_sm < 1) per_sm = 1;
    const long long T = (long long)((P.nx + StreamShape<R>::W - 1) / StreamShape<R>::W) * P.ny;
    long long n = (long long)sms * per_sm;
    const long long by_rows = (T + 31) / 32;   // at least 32 rows per CTA
    if (by_rows < n) n = by_rows;
    return n < 1 ? 1 : (int)n;
}

cudaError_t launch_step_stream(const Params &P, int prec, const void *tmap, void *fout, int *err, cudaStream_t st)
{
    const CUtensorMap &tm = *reinterpret_cast<const CUtensorMap *>(tmap);
    if (prec == 0) {
        using S = StreamShape<double>;
        double *b = (double *)fout;
        const void *fn = P.limiter == 0 ? (const void *)k_step_stream<double, false, 0>
                         : P.limiter == 1 ? (const void *)k_step_stream<double, false, 1>
                                          : (const void *)k_step_stream<double, false, 2>;
        const int grid = stream_ctas<double>(P, fn);
        if (P.limiter == 0) k_step_stream<double, false, 0><<<grid, 32 * S::WARPS, S::smem_bytes, st>>>(P, tm, b, err);
        else if (P.limiter == 1) k_step_stream<double, false, 1><<<grid, 32 * S::WARPS, S::smem_bytes, st>>>(P, tm, b, err);
        else k_step_stream<double, false, 2><<<grid, 32 * S::WARPS, S::smem_bytes, st>>>(P, tm, b, err);
    } else {
        using S = StreamShape<float>;
        float *b = (float *)fout;
        const void *fn = P.limiter == 0 ? (const void *)k_step_stream<float, true, 0>
                         : P.limiter == 1 ? (const void *)k_step_stream<float, true, 1>
                                          : (const void *)k_step_stream<float, true, 2>;
        const int grid = stream_ctas<float>(P, fn);
        if (P.limiter == 0) k_step_stream<float, true, 0><<<grid, 32 * S::WARPS, S::smem_bytes, st>>>(P, tm, b, err);
        else if (P.limiter == 1) k_step_stream<float, true, 1><<<grid, 32 * S::WARPS, S::smem_bytes, st>>>(P, tm, b, err);
        else k_step_stream<float, true, 2><<<grid, 32 * S::WARPS, S::smem_bytes, st>>>(P, tm, b, err);
    }
    return cudaGetLastError();
}

cudaError_t stream_prepare()
{
    cudaError_t e = cudaSuccess;
    auto set = [&](const void *fn, size_t bytes) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    };
    set((const void *)k_step_stream<double, false, 0>, StreamShape<double>::smem_bytes);
    set((const void *)k_step_stream<double, false, 1>, StreamShape<double>::smem_bytes);
    set((const void *)k_step_stream<double, false, 2>, StreamShape<double>::smem_bytes);
    set((const void *)k_step_stream<float, true, 0>, StreamShape<float>::smem_bytes);
    set((const void *)k_step_stream<float, true, 1>, StreamShape<float>::smem_bytes);
    set((const void *)k_step_stream<float, true, 2>, StreamShape<float>::smem_bytes);
    return e;
}

}  // namespace lbm
