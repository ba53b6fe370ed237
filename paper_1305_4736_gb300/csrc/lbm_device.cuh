// lbm_device.cuh -- device-side arithmetic of the D2V16 MRT FDLBM step.
//
// Moment transforms use the rotational symmetry of the velocity set (Sec. II,
// Fig. 1): each shell of four velocities is a 4-point butterfly
//   axis shells (1,0),(0,1),(-1,0),(0,-1) x c:
//     S = sum, X = p0 - p2, Y = p1 - p3, Q = (p0 + p2) - (p1 + p3)
//   diagonal shells (+,+),(-,+),(-,-),(+,-) x d:
//     S = sum, X = (p0 - p2) - (p1 - p3), Y = (p0 - p2) + (p1 - p3),
//     Q = (p0 + p2) - (p1 + p3)
// after which the 16 rows m_1..m_16 of Appendix A fall into five small blocks:
//   isotropic  (m1, m4, m5, m14)  <- (S1..S4)
//   x-odd      (m2, m8, m10, m12) <- (X1..X4)
//   y-odd      (m3, m9, m11, m13) <- (Y1..Y4)   (m13 row negated)
//   axis quad  (m6, m16)          <- (Q1, Q2)
//   diag quad  (m7, m15)          <- (Q3, Q4)
// The inverse blocks (with dt s_k and the butterfly normalisation folded in)
// are computed on the host at create time and passed in Params.
//
// Equilibria (Appendix A) are evaluated in deviation form about a reference
// state (rho0, u = 0, T0): every quantity is a difference from the reference,
// written without cancellation.  The FP64 mode uses the zero reference, for
// which the formulas are the plain Appendix A closed forms.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace lbm {

constexpr int NQ = 16;
constexpr int OX = 4;   // column of interior x = 0 (two ghost columns at 2, 3)
constexpr int OY = 2;   // row of interior y = 0

// Velocity-set constants (Sec. II): shell speeds 1, 6, 2, 3; component of the
// diagonal shells sqrt2 and 3/sqrt2; eta^2 = 25/4 on shell 1 (Appendix A).
constexpr double kSqrt2 = 1.41421356237309504880;
constexpr double kD3 = kSqrt2;               // component of shell 3
constexpr double kD4 = 3.0 / kSqrt2;         // component of shell 4
constexpr double kW1 = 1.0 + 6.25;           // v^2 + eta^2, shell 1
constexpr double kEta2 = 6.25;

// Coefficient tables in the arithmetic type of a kernel (float tables for the
// FP32 deviation mode, so that no float64 conversion runs per thread).
template <typename R>
struct Coef {
    R b, inv_b, four_inv_b, two_b2, six_b, b4;   // b, 1/b, 4/b, 2(b+2), 6+b, b+4
    R rho0, P0, e0, P0T0;                        // reference state (zero in FP64 mode)
    // collision: inverse blocks with dt s_k and the butterfly normalisation
    R cA[4][2];            // (Delta5, Delta14)          -> S'1..4
    R cEx[4][3];           // (Delta8, Delta10, Delta12) -> X'1..4
    R cEy[4][3];           // (Delta9, Delta11, Delta13) -> Y'1..4
    R cB1[2][2];           // (Delta6, Delta16)          -> Q'1, Q'2
    R cB2[2][2];           // (Delta7, Delta15)          -> Q'3, Q'4
    // full inverse blocks with butterfly normalisation (f = M^-1 f_hat)
    R iA[4][4], iEx[4][4], iEy[4][4], iB1[2][2], iB2[2][2];
    // energy-flux correction of the collision (Sec. II): Delta8 += q8 P [...], Delta9 += q9 P [...]
    // q = (s8/s5 - 1) / s8 / (2 dx)
    R q8, q9;
    // convection: Courant number c and h/2 = (1 - c)/4 per shell
    R cr[4], hh[4];
    // the collision blocks re-ordered for shell pairs (float32 pair arithmetic): element e of
    // pair p belongs to shell 2p + e; e.g. pEx[p][j] = (cEx[2p][j], cEx[2p+1][j])
    R pA[2][2][2], pEx[2][3][2], pEy[2][3][2], pB1[2][2], pB2[2][2];
    R ncr[4];              // -cr
    // y projection (dy may differ from dx): Courant number dt / (A_i dy), its h/2 and -cr
    R cry[4], hhy[4], ncry[4];
    // the central differences are raw (f_{+1} - f_{-1}); q8, q9 carry 1/(2 dx), so a y
    // difference is weighted by ry = dx/dy; g4 = (4, 4 ry) for the pair form
    R g4[2], ry, pad_;
};

struct EdgeDev {
    int kind;
    double uw, vw, Tw;          // wall velocity / temperature (NEQ wall)
    double two_rho0_dTw;        // 2 rho0 (Tw - T0) (reference-relative, NEQ wall)
    double feq[NQ];             // fixed equilibrium (minus f^eq0 in deviation mode)
    float uwf, vwf, Twf, two_rho0_dTwf;
    float feqf[NQ];
};

struct Params {
    int nx, ny, pitch, limiter, has_c9;
    int wrap;                   // bit 0: the tile kernel wraps the x halo of periodic edge tiles
    long long plane;            // elements per population plane
    double dt, T0;
    double feq0[NQ];            // reference populations f^eq(rho0, 0, 0, T0) (deviation mode)
    Coef<double> cd;
    Coef<float> cf;
    EdgeDev edge[4];            // x-lo, x-hi, y-lo, y-hi
};

template <typename R> __host__ __device__ __forceinline__ const Coef<R> &coef(const Params &P);
template <> __host__ __device__ __forceinline__ const Coef<double> &coef<double>(const Params &P) { return P.cd; }
template <> __host__ __device__ __forceinline__ const Coef<float> &coef<float>(const Params &P) { return P.cf; }

// ---------------------------------------------------------------------------
// Packed float32 pairs (f32x2 arithmetic of sm_100 and later).  Every operation
// rounds each lane once, as the scalar operation does.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 ld2(const float *p) { return *reinterpret_cast<const float2 *>(p); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b)
{
    unsigned long long ra, rb, rd;
    asm("mov.b64 %0, {%1, %2};" : "=l"(ra) : "f"(a.x), "f"(a.y));
    asm("mov.b64 %0, {%1, %2};" : "=l"(rb) : "f"(b.x), "f"(b.y));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
    float2 d;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(d.x), "=f"(d.y) : "l"(rd));
    return d;
}

// ---------------------------------------------------------------------------
// Storage order of the populations.  float64: 16 planes; population q of the
// cell at offset c of a plane lies at q * plane + c.  float32: 8 planes of
// population pairs; pair pr holds (pair_q(pr), pair_q(pr) + 4) side by side
// (one 8-byte element per cell), so that the f32x2 arithmetic reads and writes
// a pair with one access.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ constexpr int pair_q(int pr) { return pr < 4 ? pr : pr + 4; }   // first member
__host__ __device__ __forceinline__ constexpr int pair_of(int q) { return (q & 3) | ((q >> 3) << 2); }
__host__ __device__ __forceinline__ constexpr int member_of(int q) { return (q >> 2) & 1; }

template <typename R>
__host__ __device__ __forceinline__ long long pidx(int q, long long plane, long long c);
template <>
__host__ __device__ __forceinline__ long long pidx<double>(int q, long long plane, long long c)
{
    return q * plane + c;
}
template <>
__host__ __device__ __forceinline__ long long pidx<float>(int q, long long plane, long long c)
{
    return ((long long)pair_of(q) * plane + c) * 2 + member_of(q);
}

// ---------------------------------------------------------------------------
// Shell butterflies
// ---------------------------------------------------------------------------
template <typename R>
struct Shells { R S[4], X[4], Y[4], Q[4]; };

template <typename R>
__host__ __device__ __forceinline__ void butterfly_axis(R p0, R p1, R p2, R p3, R &S, R &X, R &Y, R &Q)
{
    const R a = p0 + p2, b = p1 + p3;
    S = a + b; Q = a - b; X = p0 - p2; Y = p1 - p3;
}

template <typename R>
__host__ __device__ __forceinline__ void butterfly_diag(R p0, R p1, R p2, R p3, R &S, R &X, R &Y, R &Q)
{
    const R a = p0 + p2, b = p1 + p3, c = p0 - p2, d = p1 - p3;
    S = a + b; Q = a - b; X = c - d; Y = c + d;
}

template <typename R>
__host__ __device__ __forceinline__ Shells<R> shells_of(const R *f)
{
    Shells<R> s;
    butterfly_axis(f[0], f[1], f[2], f[3], s.S[0], s.X[0], s.Y[0], s.Q[0]);
    butterfly_axis(f[4], f[5], f[6], f[7], s.S[1], s.X[1], s.Y[1], s.Q[1]);
    butterfly_diag(f[8], f[9], f[10], f[11], s.S[2], s.X[2], s.Y[2], s.Q[2]);
    butterfly_diag(f[12], f[13], f[14], f[15], s.S[3], s.X[3], s.Y[3], s.Q[3]);
    return s;
}

// Inverse butterflies: populations from normalised shell coefficients
// (axis: S' = S/4, X' = X/2, Y' = Y/2, Q' = Q/4; diagonal: all /4).
template <typename R>
__host__ __device__ __forceinline__ void unbutterfly_axis(R S, R X, R Y, R Q, R *p)
{
    const R a = S + Q, b = S - Q;
    p[0] = a + X; p[2] = a - X; p[1] = b + Y; p[3] = b - Y;
}

template <typename R>
__host__ __device__ __forceinline__ void unbutterfly_diag(R S, R X, R Y, R Q, R *p)
{
    const R a = S + Q, b = S - Q, c = X + Y, d = X - Y;
    p[0] = a + c; p[2] = a - c; p[1] = b - d; p[3] = b + d;
}

// ---------------------------------------------------------------------------
// Moments from shells (Appendix A rows in block form)
// ---------------------------------------------------------------------------
template <typename R>
struct Moments { R m[NQ]; };   // m[k] = row k+1 of Appendix A applied to f (or g)

template <typename R>
__host__ __device__ __forceinline__ void conserved_of(const Shells<R> &s, R &rho, R &jx, R &jy, R &e)
{
    rho = (s.S[0] + s.S[1]) + (s.S[2] + s.S[3]);
    jx = s.X[0] + R(6.0) * s.X[1] + R(kD3) * s.X[2] + R(kD4) * s.X[3];
    jy = s.Y[0] + R(6.0) * s.Y[1] + R(kD3) * s.Y[2] + R(kD4) * s.Y[3];
    e = R(kW1) * s.S[0] + R(36.0) * s.S[1] + R(4.0) * s.S[2] + R(9.0) * s.S[3];
}

template <typename R>
__host__ __device__ __forceinline__ Moments<R> moments_of(const Shells<R> &s)
{
    Moments<R> M;
    conserved_of(s, M.m[0], M.m[1], M.m[2], M.m[3]);
    M.m[4] = M.m[3] - R(kEta2) * s.S[0];
    M.m[13] = R(kW1) * s.S[0] + R(1296.0) * s.S[1] + R(16.0) * s.S[2] + R(81.0) * s.S[3];
    const R x8 = R(kW1) * s.X[0] + R(216.0) * s.X[1] + R(4.0 * kSqrt2) * s.X[2] + R(27.0 / kSqrt2) * s.X[3];
    const R y8 = R(kW1) * s.Y[0] + R(216.0) * s.Y[1] + R(4.0 * kSqrt2) * s.Y[2] + R(27.0 / kSqrt2) * s.Y[3];
    M.m[7] = x8;
    M.m[8] = y8;
    M.m[9] = x8 - R(kEta2) * s.X[0];
    M.m[10] = y8 - R(kEta2) * s.Y[0];
    M.m[11] = s.X[0] + R(216.0) * s.X[1];
    M.m[12] = -(s.Y[0] + R(216.0) * s.Y[1]);
    M.m[5] = s.Q[0] + R(36.0) * s.Q[1];
    M.m[15] = R(kW1) * s.Q[0] + R(1296.0) * s.Q[1];
    M.m[6] = R(2.0) * s.Q[2] + R(4.5) * s.Q[3];
    M.m[14] = R(8.0) * s.Q[2] + R(40.5) * s.Q[3];
    return M;
}

// ---------------------------------------------------------------------------
// Equilibria (Appendix A) in deviation form.
// Inputs: drho = rho - rho0, j, dP = P - P0 (u0 = 0).  Output: f_hat^eq - f_hat^eq0,
// all 16 rows.  With rho0 = P0 = T0 = e0 = 0 this is f_hat^eq itself.
// ---------------------------------------------------------------------------
// ux, uy: the flow velocity j / rho (jx * ir, jy * ir), passed in where the caller has it.
template <typename R, bool Dev>
__host__ __device__ __forceinline__ void feq_hat_dev(const Coef<R> &C, R drho, R jx, R jy, R ux, R uy, R dP, R ir,
                                                    R *q)
{
    const R b = C.b;
    const R jx2 = jx * ux, jy2 = jy * uy, J2 = jx2 + jy2;
    const R Pt = Dev ? C.P0 + dP : dP;                   // total pressure
    const R e_dev = b * dP + J2;                          // e - e0
    const R et = Dev ? C.e0 + e_dev : e_dev;              // total e
    const R dxy = jx2 - jy2;
    q[0] = drho;
    q[1] = jx;
    q[2] = jy;
    q[3] = e_dev;
    q[4] = R(2.0) * dP + J2;
    q[5] = dxy;
    q[6] = jx * uy;
    const R e2p = et + R(2.0) * Pt;
    q[7] = e2p * ux;
    q[8] = e2p * uy;
    const R g4 = R(4.0) * Pt + J2;
    q[9] = g4 * ux;
    q[10] = g4 * uy;
    q[11] = (R(2.0) * Pt + dxy) * ux;
    q[12] = (dxy - R(2.0) * Pt) * uy;
    // row 14: 2(b+2) P^2/rho + (6+b) P J2/rho + J2^2/rho
    if (Dev) {
        const R T = Pt * ir;
        const R iso = ir * (dP * (Pt + C.P0) - C.P0T0 * drho);   // P^2/rho - P0^2/rho0
        q[13] = C.two_b2 * iso + C.six_b * T * J2 + J2 * J2 * ir;
    } else {
        q[13] = ir * (Pt * (C.two_b2 * Pt + C.six_b * J2) + J2 * J2);
    }
    const R k = C.b4 * Pt + J2;
    q[14] = k * ux * uy;
    q[15] = k * dxy * ir;
}

template <typename R, bool Dev>
__host__ __device__ __forceinline__ void feq_hat_dev(const Coef<R> &C, R drho, R jx, R jy, R dP, R ir, R *q)
{
    feq_hat_dev<R, Dev>(C, drho, jx, jy, jx * ir, jy * ir, dP, ir, q);
}

// Populations from a full moment vector q (16 rows) with the full inverse blocks.
template <typename R>
__host__ __device__ __forceinline__ void pop_from_moments(const Coef<R> &C, const R *q, R *f)
{
    R S[4], X[4], Y[4], Q[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        S[k] = C.iA[k][0] * q[0] + C.iA[k][1] * q[3] + C.iA[k][2] * q[4] + C.iA[k][3] * q[13];
        X[k] = C.iEx[k][0] * q[1] + C.iEx[k][1] * q[7] + C.iEx[k][2] * q[9] + C.iEx[k][3] * q[11];
        Y[k] = C.iEy[k][0] * q[2] + C.iEy[k][1] * q[8] + C.iEy[k][2] * q[10] + C.iEy[k][3] * q[12];
    }
    Q[0] = C.iB1[0][0] * q[5] + C.iB1[0][1] * q[15];
    Q[1] = C.iB1[1][0] * q[5] + C.iB1[1][1] * q[15];
    Q[2] = C.iB2[0][0] * q[6] + C.iB2[0][1] * q[14];
    Q[3] = C.iB2[1][0] * q[6] + C.iB2[1][1] * q[14];
    unbutterfly_axis(S[0], X[0], Y[0], Q[0], f + 0);
    unbutterfly_axis(S[1], X[1], Y[1], Q[1], f + 4);
    unbutterfly_diag(S[2], X[2], Y[2], Q[2], f + 8);
    unbutterfly_diag(S[3], X[3], Y[3], Q[3], f + 12);
}

// ---------------------------------------------------------------------------
// Flux limiter (Sec. III).  For one population along one axis, in upwind
// order (f_{J-2s}, f_{J-s}, f_J, f_{J+s}), return
//   (F_out - F_in) = (f_J - f_{J-s}) + h [psi_J D+_J - psi_{J-s} D+_{J-s}]
// with D+_J = f_{J+s} - f_J.  psi(theta) D+ is evaluated without the
// division: for the MC limiter it equals minmod(2 D-, (D- + D+)/2, 2 D+)
// (0 when D- D+ <= 0), for Lax-Wendroff D+, for upwind 0.  The magnitude
// comparisons, the sign logic and the exact scaling by 4 (an exponent
// increment) run on the integer pipe.  The scaling is exact for every normal
// number; for a subnormal min(|D-|, |D+|) (below 2.2e-308 in float64) it is
// off by that subnormal's own size.  `hh` is h/2 = (1 - c)/4 because mc2
// returns twice the slope.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double mc2(double a, double b)
{
    // 2 * minmod(2a, (a+b)/2, 2b) = sign * min(4|a|, 4|b|, |a+b|).  The integer steps are
    // written in PTX: as C++ bit operations the compiler recognises the sign-bit masks as
    // fabs and evaluates them as float64 instructions.
    const double s = a + b;
    double r;
    asm("{\n\t"
        ".reg .b64 ia, ib, is, aa, ab, m, t, sg;\n\t"
        ".reg .pred pd, pz;\n\t"
        "mov.b64 ia, %1;\n\t"
        "mov.b64 ib, %2;\n\t"
        "mov.b64 is, %3;\n\t"
        "and.b64 aa, ia, 0x7FFFFFFFFFFFFFFF;\n\t"
        "and.b64 ab, ib, 0x7FFFFFFFFFFFFFFF;\n\t"
        "min.u64 m, aa, ab;\n\t"                      // min(|a|, |b|)
        "setp.eq.u64 pz, m, 0;\n\t"
        "add.u64 m, m, 0x0020000000000000;\n\t"       // 4 min(|a|, |b|): exponent + 2
        "and.b64 is, is, 0x7FFFFFFFFFFFFFFF;\n\t"
        "min.u64 t, m, is;\n\t"
        "xor.b64 sg, ia, ib;\n\t"
        "setp.lt.s64 pd, sg, 0;\n\t"                  // the differences disagree in sign
        "or.pred pd, pd, pz;\n\t"
        "and.b64 sg, ib, 0x8000000000000000;\n\t"
        "or.b64 t, t, sg;\n\t"
        "selp.b64 t, 0, t, pd;\n\t"
        "mov.b64 %0, t;\n\t"
        "}"
        : "=d"(r)
        : "d"(a), "d"(b), "d"(s));
    return r;
}

__device__ __forceinline__ float mc2(float a, float b)
{
    // t = min(|a|, |b|) with sign(a) xor sign(b): negative exactly when the
    // one-sided differences disagree in sign, which the max with 0 turns into 0.
    // When they agree, a + b has their sign and min.xorsign.abs(max(4t, 0), a + b)
    // is sign(a + b) min(4 min(|a|, |b|), |a + b|); when they disagree it is +-0.
    float t, r;
    asm("min.xorsign.abs.f32 %0, %1, %2;" : "=f"(t) : "f"(a), "f"(b));
    const float m = fmaxf(4.0f * t, 0.0f);
    asm("min.xorsign.abs.f32 %0, %1, %2;" : "=f"(r) : "f"(m), "f"(a + b));
    return r;
}

// 1/x.  float64: Newton-Raphson iteration for the reciprocal, y <- y + y (1 - x y), which
// squares the relative error at each step, from the approximate reciprocal of PTX
// (rcp.approx.ftz.f64, about 20 correct bits); two steps reach the rounding level (within an
// ulp or so of the correctly rounded quotient) in five float64 operations, fewer than an IEEE
// division.  x is a density, positive and normal.  float32: the hardware reciprocal
// approximation (at most 2 ulp), ample for the float32 deviation mode.
__device__ __forceinline__ double recip(double x)
{
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    double e = fma(-x, y, 1.0);
    y = fma(y, e, y);
    e = fma(-x, y, 1.0);
    return fma(y, e, y);
}
__device__ __forceinline__ float recip(float x) { return __fdividef(1.0f, x); }

template <typename R, int Lim>
__device__ __forceinline__ R flux_diff(R fmm, R fm, R f0, R fp, R hh)
{
    const R d1 = f0 - fm;
    if (Lim == 2) return d1;                     // upwind
    const R d2 = fp - f0;
    if (Lim == 1) return d1 + R(2.0) * hh * (d2 - d1);   // Lax-Wendroff: psi = 1
    const R d0 = fm - fmm;
    return d1 + hh * (mc2(d1, d2) - mc2(d0, d1));
}

// ---------------------------------------------------------------------------
// Collision (Eq. 3 with the energy-flux correction of Sec. II):
//   out = dt M^-1 S (f_hat - f_hat^eq), residuals of rows 1..4 are zero.
// ---------------------------------------------------------------------------
// ux, uy: j / rho as jx * ir, jy * ir (the caller's, bit for bit).
template <typename R, bool Dev>
__device__ __forceinline__ void collide(const Params &P, const Shells<R> &sh, R drho, R jx, R jy, R de,
                                        R ir, R ux, R uy, R dxux, R dyux, R dxuy, R dyuy, R *out)
{
    const Coef<R> &C = coef<R>(P);
    const Moments<R> M = moments_of(sh);
    const R J2 = jx * ux + jy * uy;
    const R dP = (de - J2) * C.inv_b;
    R q[NQ];
    feq_hat_dev<R, Dev>(C, drho, jx, jy, ux, uy, dP, ir, q);
    R D[NQ];
    D[4] = (de - R(kEta2) * sh.S[0]) - q[4];   // row 5 from the caller's e (equal to M.m[3])
#pragma unroll
    for (int k = 5; k < NQ; k++) D[k] = M.m[k] - q[k];
    if (P.has_c9) {
        const R Pt = Dev ? C.P0 + dP : dP;
        // y differences weighted by ry = dx/dy (q8, q9 carry 1/(2 dx))
        const R div = dxux + C.ry * dyuy, shr = dxuy + C.ry * dyux;
        D[7] += C.q8 * Pt * (ux * (R(4.0) * dxux - C.four_inv_b * div) + R(2.0) * uy * shr);
        D[8] += C.q9 * Pt * (R(2.0) * ux * shr + uy * (C.g4[1] * dyuy - C.four_inv_b * div));
    }
    R S[4], X[4], Y[4], Q[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        S[k] = C.cA[k][0] * D[4] + C.cA[k][1] * D[13];
        X[k] = C.cEx[k][0] * D[7] + C.cEx[k][1] * D[9] + C.cEx[k][2] * D[11];
        Y[k] = C.cEy[k][0] * D[8] + C.cEy[k][1] * D[10] + C.cEy[k][2] * D[12];
    }
    Q[0] = C.cB1[0][0] * D[5] + C.cB1[0][1] * D[15];
    Q[1] = C.cB1[1][0] * D[5] + C.cB1[1][1] * D[15];
    Q[2] = C.cB2[0][0] * D[6] + C.cB2[0][1] * D[14];
    Q[3] = C.cB2[1][0] * D[6] + C.cB2[1][1] * D[14];
    unbutterfly_axis(S[0], X[0], Y[0], Q[0], out + 0);
    unbutterfly_axis(S[1], X[1], Y[1], Q[1], out + 4);
    unbutterfly_diag(S[2], X[2], Y[2], Q[2], out + 8);
    unbutterfly_diag(S[3], X[3], Y[3], Q[3], out + 12);
}

// ---------------------------------------------------------------------------
// Float32 collision on population pairs.  Pair pr holds populations (q, q+4)
// with q = pr for pr < 4 (axis shells 1 and 2) and q = pr + 4 for pr >= 4
// (diagonal shells 3 and 4): the two shells of a pair have the same butterfly,
// so shells, moments, the inverse blocks and the inverse butterflies run as
// f32x2 operations.  Same formulas as shells_of / conserved_of / collide; only
// the summation order of some moment rows differs.
// ---------------------------------------------------------------------------
struct Shells2 { float2 S[2], X[2], Y[2], Q[2]; };   // [0]: shells 1, 2; [1]: shells 3, 4

__device__ __forceinline__ Shells2 shells2_of(const float2 *fp)
{
    Shells2 s;
    {
        const float2 a = add2(fp[0], fp[2]), b = add2(fp[1], fp[3]);
        s.S[0] = add2(a, b);
        s.Q[0] = sub2(a, b);
        s.X[0] = sub2(fp[0], fp[2]);
        s.Y[0] = sub2(fp[1], fp[3]);
    }
    {
        const float2 a = add2(fp[4], fp[6]), b = add2(fp[5], fp[7]);
        const float2 c = sub2(fp[4], fp[6]), d = sub2(fp[5], fp[7]);
        s.S[1] = add2(a, b);
        s.Q[1] = sub2(a, b);
        s.X[1] = sub2(c, d);
        s.Y[1] = add2(c, d);
    }
    return s;
}

__device__ __forceinline__ void conserved2_of(const Shells2 &s, float &rho, float &jx, float &jy, float &e)
{
    const float2 r = add2(s.S[0], s.S[1]);
    rho = r.x + r.y;
    jx = fmaf(float(kD4), s.X[1].y, fmaf(float(kD3), s.X[1].x, fmaf(6.0f, s.X[0].y, s.X[0].x)));
    jy = fmaf(float(kD4), s.Y[1].y, fmaf(float(kD3), s.Y[1].x, fmaf(6.0f, s.Y[0].y, s.Y[0].x)));
    const float2 w = fma2(f2(float(kW1), 36.0f), s.S[0], mul2(f2(4.0f, 9.0f), s.S[1]));
    e = w.x + w.y;
}

__device__ __forceinline__ float2 bc2(float v) { return f2(v, v); }

// Flow velocity and 1/rho of the cell whose population q is at p[q * stride] (float64
// planes) or whose pair pr is at p2[pr * stride] (float32 pair planes).
template <bool Dev>
__device__ __forceinline__ void flow_at(const Coef<double> &C, const double *p, int stride, double &u, double &v,
                                        double &ir)
{
    double g[NQ], drho, jx, jy, de;
#pragma unroll
    for (int q = 0; q < NQ; q++) g[q] = p[q * stride];
    conserved_of(shells_of(g), drho, jx, jy, de);
    const double rho = Dev ? C.rho0 + drho : drho;
    ir = recip(rho);
    u = jx * ir;
    v = jy * ir;
}

template <bool Dev>
__device__ __forceinline__ void flow_at(const Coef<float> &C, const float2 *p2, int stride, float &u, float &v,
                                        float &ir)
{
    float2 fp[8];
#pragma unroll
    for (int pr = 0; pr < 8; pr++) fp[pr] = p2[pr * stride];
    float drho, jx, jy, de;
    conserved2_of(shells2_of(fp), drho, jx, jy, de);
    const float rho = Dev ? C.rho0 + drho : drho;
    ir = recip(rho);
    u = jx * ir;
    v = jy * ir;
}

// Inverse butterflies of a shell pair: acc[k] = (p_k of the first shell, p_k of the second).
__device__ __forceinline__ void unbutterfly2_axis(float2 S, float2 X, float2 Y, float2 Q, float2 *acc)
{
    const float2 a = add2(S, Q), b = sub2(S, Q);
    acc[0] = add2(a, X);
    acc[2] = sub2(a, X);
    acc[1] = add2(b, Y);
    acc[3] = sub2(b, Y);
}

__device__ __forceinline__ void unbutterfly2_diag(float2 S, float2 X, float2 Y, float2 Q, float2 *acc)
{
    const float2 a = add2(S, Q), b = sub2(S, Q), c = add2(X, Y), d = sub2(X, Y);
    acc[0] = add2(a, c);
    acc[2] = sub2(a, c);
    acc[1] = sub2(b, d);
    acc[3] = add2(b, d);
}

// acc[pr] = collision term of pair pr (dt M^-1 S (f_hat - f_hat^eq), Eq. 3 with the
// energy-flux correction of Sec. II).
template <bool Dev, typename PP>
__device__ __forceinline__ void collide2(const PP &P, const Shells2 &sh, float drho, float jx, float jy,
                                         float de, float ir, float dxux, float dyux, float dxuy, float dyuy,
                                         float2 *acc)
{
    const Coef<float> &C = P.cf;
    const float S0 = sh.S[0].x, X0 = sh.X[0].x, X1 = sh.X[0].y, Y0 = sh.Y[0].x, Y1 = sh.Y[0].y;
    const float Q0 = sh.Q[0].x, Q1 = sh.Q[0].y, Q2 = sh.Q[1].x, Q3 = sh.Q[1].y;
    // rows 5..16 of Appendix A
    const float m4 = fmaf(-float(kEta2), S0, de);
    const float2 t13 = fma2(f2(float(kW1), 1296.0f), sh.S[0], mul2(f2(16.0f, 81.0f), sh.S[1]));
    const float m13 = t13.x + t13.y;
    const float2 c8 = f2(float(4.0 * kSqrt2), float(27.0 / kSqrt2));
    const float2 t8x = fma2(f2(float(kW1), 216.0f), sh.X[0], mul2(c8, sh.X[1]));
    const float2 t8y = fma2(f2(float(kW1), 216.0f), sh.Y[0], mul2(c8, sh.Y[1]));
    const float x8 = t8x.x + t8x.y, y8 = t8y.x + t8y.y;
    const float m9 = fmaf(-float(kEta2), X0, x8), m10 = fmaf(-float(kEta2), Y0, y8);
    const float m11 = fmaf(216.0f, X1, X0), m12 = -fmaf(216.0f, Y1, Y0);
    const float m5 = fmaf(36.0f, Q1, Q0), m15 = fmaf(1296.0f, Q1, float(kW1) * Q0);
    const float m6 = fmaf(4.5f, Q3, 2.0f * Q2), m14 = fmaf(40.5f, Q3, 8.0f * Q2);

    // rows 5..16 of f_hat^eq (deviation form, as feq_hat_dev) with the x/y rows in pairs
    const float2 u2 = mul2(f2(jx, jy), bc2(ir));                  // (u_x, u_y)
    const float ux = u2.x, uy = u2.y;
    const float2 jj = mul2(f2(jx, jy), u2);                        // (j_x u_x, j_y u_y)
    const float J2 = jj.x + jj.y, dxy = jj.x - jj.y;
    const float dP = (de - J2) * C.inv_b;
    const float Pt = Dev ? C.P0 + dP : dP;
    const float e_dev = fmaf(C.b, dP, J2);
    const float et = Dev ? C.e0 + e_dev : e_dev;
    const float q4 = fmaf(2.0f, dP, J2), q5 = dxy, q6 = jx * uy;
    const float2 q7_8 = mul2(bc2(fmaf(2.0f, Pt, et)), u2);
    const float2 q9_10 = mul2(bc2(fmaf(4.0f, Pt, J2)), u2);
    const float2 q11_12 = mul2(add2(bc2(dxy), f2(2.0f * Pt, -2.0f * Pt)), u2);
    const float T = Pt * ir;
    const float iso = Dev ? ir * (dP * (Pt + C.P0) - C.P0T0 * drho) : Pt * T;
    const float q13 = C.two_b2 * iso + C.six_b * T * J2 + J2 * J2 * ir;
    const float kk = fmaf(C.b4, Pt, J2);
    const float q14 = kk * ux * uy, q15 = kk * dxy * ir;
    const float2 D4_13 = sub2(f2(m4, m13), f2(q4, q13));
    float2 D7_8 = sub2(f2(x8, y8), q7_8);
    const float2 D9_10 = sub2(f2(m9, m10), q9_10);
    const float2 D11_12 = sub2(f2(m11, m12), q11_12);
    const float2 D5_15 = sub2(f2(m5, m15), f2(q5, q15));
    const float2 D6_14 = sub2(f2(m6, m14), f2(q6, q14));
    if (P.has_c9) {
        // (D8, D9 of the paper's 1-based rows) += (q8, q9) P [u . (4 grad u - (4/b) div u) + 2 u_perp shear]
        const float div = fmaf(C.ry, dyuy, dxux), shr = fmaf(C.ry, dyux, dxuy);   // y weighted by dx/dy
        const float2 g = fma2(ld2(C.g4), f2(dxux, dyuy), bc2(-C.four_inv_b * div));
        const float2 h = fma2(f2(ux, uy), g, mul2(bc2(2.0f * shr), f2(uy, ux)));
        D7_8 = fma2(mul2(ld2(&C.q8), bc2(Pt)), h, D7_8);
    }
    const float2 d4 = bc2(D4_13.x), d13 = bc2(D4_13.y);
    const float2 S01 = fma2(ld2(C.pA[0][1]), d13, mul2(ld2(C.pA[0][0]), d4));
    const float2 S23 = fma2(ld2(C.pA[1][1]), d13, mul2(ld2(C.pA[1][0]), d4));
    const float2 d7 = bc2(D7_8.x), d9 = bc2(D9_10.x), d11 = bc2(D11_12.x);
    const float2 d8 = bc2(D7_8.y), d10 = bc2(D9_10.y), d12 = bc2(D11_12.y);
    const float2 X01 = fma2(ld2(C.pEx[0][2]), d11, fma2(ld2(C.pEx[0][1]), d9, mul2(ld2(C.pEx[0][0]), d7)));
    const float2 X23 = fma2(ld2(C.pEx[1][2]), d11, fma2(ld2(C.pEx[1][1]), d9, mul2(ld2(C.pEx[1][0]), d7)));
    const float2 Y01 = fma2(ld2(C.pEy[0][2]), d12, fma2(ld2(C.pEy[0][1]), d10, mul2(ld2(C.pEy[0][0]), d8)));
    const float2 Y23 = fma2(ld2(C.pEy[1][2]), d12, fma2(ld2(C.pEy[1][1]), d10, mul2(ld2(C.pEy[1][0]), d8)));
    const float2 Q01 = fma2(ld2(C.pB1[1]), bc2(D5_15.y), mul2(ld2(C.pB1[0]), bc2(D5_15.x)));
    const float2 Q23 = fma2(ld2(C.pB2[1]), bc2(D6_14.y), mul2(ld2(C.pB2[0]), bc2(D6_14.x)));
    unbutterfly2_axis(S01, X01, Y01, Q01, acc);
    unbutterfly2_diag(S23, X23, Y23, Q23, acc + 4);
}

}  // namespace lbm
