// lbm_api.cu -- host side of liblbm.so: the C interface declared in include/lbm.h.
//
// Responsibilities: argument validation (isotropy and Prandtl number of
// Sec. II, Courant and relaxation stability limits of the forward-Euler
// scheme of Sec. III, boundary pairing), the constant tables of the step
// (block inverses of the symmetry-factored transformation matrix, per-shell
// Courant numbers, fixed-equilibrium ghost states), device memory, chunked
// host <-> device transfers, and error reporting.  No exception crosses the
// interface: every entry point returns a status code.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "../../include/lbm.h"
#include "lbm_internal.h"

using lbm::NQ;
using lbm::Params;

struct lbm_ctx {
    Params P;
    int prec = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    lbm_allocator alloc{};
    bool own_alloc = true;
    void *buf = nullptr;          // both population buffers
    size_t buf_bytes = 0;
    void *f[2] = {nullptr, nullptr};
    int cur = 0;
    double *stage = nullptr;      // staging for chunked transfers
    size_t stage_elems = 0;
    double *aux = nullptr;        // totals partials (kTotalsBlocks * 16) + out (4) + flags
    size_t aux_bytes = 0;
    int *flag = nullptr;          // non-finite / rho <= 0 seen by the moments kernel
    int *tma_err = nullptr;       // a copy wait ran out in a TMA-fed step kernel
    int *init_err = nullptr;      // an lbm_init field value was invalid
    double *tot_out = nullptr;
    bool use_tma = false;
    bool use_stream = false;
    bool use_pipe = false;
    bool use_dd = false;          // float64 mode in double-float arithmetic (step_kernel 8)
    bool use_ddn = false;         // the same on narrow tiles of 32 x 4 (step_kernel 9)
    lbm::Coef<lbm::dd> cdd{};     // their coefficients
    int plain_ty = lbm::kTY;      // tile height of the plain step kernel
    CUtensorMap tmap[2];          // tile-copy descriptors of the two population buffers
    CUtensorMap smap[2];          // row-copy descriptors (streaming kernel)
    CUtensorMap pmap[2];          // tile-copy descriptors of the double-buffered kernel
    CUtensorMap nmap[2];          // tile-copy descriptors of the narrow double-float tiles
    // lbm_step replays pairs of steps (ghost fill + fused step, twice) from a CUDA graph per
    // starting buffer, captured on a private stream at first use; lbm_autotune drops them
    cudaGraphExec_t pair[2] = {nullptr, nullptr};
    cudaStream_t cap = nullptr;
    bool initialized = false;
    long long steps = 0;
    double dx = 0.0, dy = 0.0;
    // profiling (lbm_profile_begin / lbm_profile_end)
    bool prof = false;
    int prof_max = 0, prof_used = 0;
    std::vector<cudaEvent_t> prof_ev;   // 4 per step: ghost start/end, step start/end
    std::string err;
};

namespace {

thread_local std::string g_err;

int fail(lbm_ctx *c, int code, const std::string &msg)
{
    if (c) c->err = msg;
    else g_err = msg;
    return code;
}

int cuda_fail(lbm_ctx *c, cudaError_t e, const char *where)
{
    return fail(c, LBM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// Gauss-Jordan inverse with partial pivoting (n <= 4).  Returns false if singular.
bool invert(int n, const double *A, double *Ai)
{
    double a[4][8];
    for (int r = 0; r < n; r++)
        for (int c = 0; c < 2 * n; c++) a[r][c] = c < n ? A[r * n + c] : (c - n == r ? 1.0 : 0.0);
    for (int col = 0; col < n; col++) {
        int p = col;
        for (int r = col + 1; r < n; r++)
            if (std::fabs(a[r][col]) > std::fabs(a[p][col])) p = r;
        if (a[p][col] == 0.0) return false;
        if (p != col)
            for (int c = 0; c < 2 * n; c++) std::swap(a[p][c], a[col][c]);
        const double d = a[col][col];
        for (int c = 0; c < 2 * n; c++) a[col][c] /= d;
        for (int r = 0; r < n; r++) {
            if (r == col) continue;
            const double m = a[r][col];
            if (m != 0.0)
                for (int c = 0; c < 2 * n; c++) a[r][c] -= m * a[col][c];
        }
    }
    for (int r = 0; r < n; r++)
        for (int c = 0; c < n; c++) Ai[r * n + c] = a[r][n + c];
    return true;
}

// The five blocks of the transformation matrix in the shell-butterfly basis
// (rows of Appendix A evaluated on the velocity set of Sec. II), inverted and
// scaled by the butterfly normalisation (axis shells: S/4, X/2, Y/2, Q/4;
// diagonal shells: all /4).
bool build_inverse_blocks(lbm::Coef<double> &P)
{
    const double r2 = lbm::kSqrt2, d3 = lbm::kD3, d4 = lbm::kD4, w1 = lbm::kW1;
    // isotropic block: rows m1, m4, m5, m14; columns S1..S4
    const double A[16] = {1.0, 1.0, 1.0, 1.0,
                          w1, 36.0, 4.0, 9.0,
                          1.0, 36.0, 4.0, 9.0,
                          w1, 1296.0, 16.0, 81.0};
    // x-odd block: rows m2, m8, m10, m12; columns X1..X4
    const double E[16] = {1.0, 6.0, d3, d4,
                          w1, 216.0, 4.0 * r2, 27.0 / r2,
                          1.0, 216.0, 4.0 * r2, 27.0 / r2,
                          1.0, 216.0, 0.0, 0.0};
    double Ey[16];
    std::memcpy(Ey, E, sizeof(E));
    for (int c = 0; c < 4; c++) Ey[12 + c] = -E[12 + c];      // m13 = -v_y^3 on axis shells
    const double B1[4] = {1.0, 36.0, w1, 1296.0};              // rows m6, m16; columns Q1, Q2
    const double B2[4] = {2.0, 4.5, 8.0, 40.5};                // rows m7, m15; columns Q3, Q4
    double Ai[16], Ei[16], Eyi[16], B1i[4], B2i[4];
    if (!invert(4, A, Ai) || !invert(4, E, Ei) || !invert(4, Ey, Eyi) || !invert(2, B1, B1i) ||
        !invert(2, B2, B2i))
        return false;
    const double nS = 0.25, nXa = 0.5, nXd = 0.25, nQ = 0.25;
    for (int k = 0; k < 4; k++) {
        const double nx = k < 2 ? nXa : nXd;
        for (int j = 0; j < 4; j++) {
            P.iA[k][j] = nS * Ai[k * 4 + j];
            P.iEx[k][j] = nx * Ei[k * 4 + j];
            P.iEy[k][j] = nx * Eyi[k * 4 + j];
        }
    }
    for (int k = 0; k < 2; k++)
        for (int j = 0; j < 2; j++) {
            P.iB1[k][j] = nQ * B1i[k * 2 + j];
            P.iB2[k][j] = nQ * B2i[k * 2 + j];
        }
    return true;
}

void fold_rates(lbm::Coef<double> &P, const double *s, double dt)
{
    // collision columns: moment row k (1-based) relaxes at s_k; dt folded in
    for (int k = 0; k < 4; k++) {
        P.cA[k][0] = dt * s[4] * P.iA[k][2];      // m5
        P.cA[k][1] = dt * s[13] * P.iA[k][3];     // m14
        P.cEx[k][0] = dt * s[7] * P.iEx[k][1];    // m8
        P.cEx[k][1] = dt * s[9] * P.iEx[k][2];    // m10
        P.cEx[k][2] = dt * s[11] * P.iEx[k][3];   // m12
        P.cEy[k][0] = dt * s[8] * P.iEy[k][1];    // m9
        P.cEy[k][1] = dt * s[10] * P.iEy[k][2];   // m11
        P.cEy[k][2] = dt * s[12] * P.iEy[k][3];   // m13
    }
    for (int k = 0; k < 2; k++) {
        P.cB1[k][0] = dt * s[5] * P.iB1[k][0];    // m6
        P.cB1[k][1] = dt * s[15] * P.iB1[k][1];   // m16
        P.cB2[k][0] = dt * s[6] * P.iB2[k][0];    // m7
        P.cB2[k][1] = dt * s[14] * P.iB2[k][1];   // m15
    }
    // the same columns ordered for shell pairs (shells 2p and 2p + 1)
    for (int p = 0; p < 2; p++)
        for (int e = 0; e < 2; e++) {
            for (int j = 0; j < 2; j++) P.pA[p][j][e] = P.cA[2 * p + e][j];
            for (int j = 0; j < 3; j++) {
                P.pEx[p][j][e] = P.cEx[2 * p + e][j];
                P.pEy[p][j][e] = P.cEy[2 * p + e][j];
            }
            P.pB1[p][e] = P.cB1[e][p];
            P.pB2[p][e] = P.cB2[e][p];
        }
}

// f^eq of a state (Dev = false) or its deviation f^eq - f^eq0 from the reference
// state (Dev = true), on the host.
template <bool Dev>
void host_feq(const Params &P, double rho, double ux, double uy, double T, double *f)
{
    const lbm::Coef<double> &C = P.cd;
    const double drho = Dev ? rho - C.rho0 : rho;
    const double dP = Dev ? rho * T - C.P0 : rho * T;
    double q[NQ];
    lbm::feq_hat_dev<double, Dev>(C, drho, rho * ux, rho * uy, dP, 1.0 / rho, q);
    lbm::pop_from_moments(C, q, f);
}

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

int validate_bc_edge(const lbm_edge_bc &e, const char *name, std::string &msg)
{
    if (e.kind < LBM_BC_PERIODIC || e.kind > LBM_BC_NEQ_WALL) {
        msg = std::string("bc ") + name + ": unknown kind";
        return LBM_ERR_ARG;
    }
    if (e.kind == LBM_BC_EQUILIBRIUM &&
        (!finite_pos(e.rho) || !finite_pos(e.T) || !std::isfinite(e.u) || !std::isfinite(e.v))) {
        msg = std::string("bc ") + name + ": equilibrium state needs rho > 0, T > 0, finite u, v";
        return LBM_ERR_ARG;
    }
    if (e.kind == LBM_BC_NEQ_WALL && (!finite_pos(e.T) || !std::isfinite(e.u) || !std::isfinite(e.v))) {
        msg = std::string("bc ") + name + ": wall needs T > 0 and finite velocity";
        return LBM_ERR_ARG;
    }
    return LBM_OK;
}

void *default_alloc(size_t bytes, void *, void *)
{
    void *p = nullptr;
    return cudaMalloc(&p, bytes) == cudaSuccess ? p : nullptr;
}

void default_free(void *p, size_t, void *, void *) { cudaFree(p); }

size_t pitch_of(int nx) { return (size_t)((nx + 8 + 31) / 32 * 32); }

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }();
    return fn;
}

// 3-D copy descriptor of one population buffer: x = padded columns, y = rows
// (ny + 4), z = the 16 planes; box = box_w x box_h x all planes (the staged tile
// of the TMA-staged kernel, or one row slot of the streaming kernel).
bool make_tensor_map(CUtensorMap *tm, void *base, const Params &P, int prec, int box_w, int box_h)
{
    auto enc = tensor_map_encoder();
    if (!enc) return false;
    // float64: 16 planes of doubles; float32: 8 planes of population pairs, copied as
    // 8-byte elements (the bits are moved unchanged)
    const size_t es = 8;
    const cuuint64_t planes = prec == LBM_FP32_DEV ? NQ / 2 : NQ;
    const cuuint64_t dims[3] = {(cuuint64_t)P.pitch, (cuuint64_t)(P.ny + 4), planes};
    const cuuint64_t strides[2] = {(cuuint64_t)P.pitch * es, (cuuint64_t)P.plane * es};
    const cuuint32_t box[3] = {(cuuint32_t)box_w, (cuuint32_t)box_h, (cuuint32_t)planes};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = enc(tm, prec == LBM_FP32_DEV ? CU_TENSOR_MAP_DATA_TYPE_INT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                           3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

bool make_tile_maps(lbm_ctx *c)
{
    const int sw = lbm::TmaShape<float>::SW;
    const int sh = c->prec == LBM_FP32_DEV ? lbm::TmaShape<float>::SH : lbm::TmaShape<double>::SH;
    return make_tensor_map(&c->tmap[0], c->f[0], c->P, c->prec, sw, sh) &&
           make_tensor_map(&c->tmap[1], c->f[1], c->P, c->prec, sw, sh);
}

bool make_narrow_maps(lbm_ctx *c)
{
    const int sw = lbm::DdNarrowShape::SW, sh = lbm::DdNarrowShape::SH;
    return make_tensor_map(&c->nmap[0], c->f[0], c->P, c->prec, sw, sh) &&
           make_tensor_map(&c->nmap[1], c->f[1], c->P, c->prec, sw, sh);
}

bool make_row_maps(lbm_ctx *c)
{
    using S = lbm::StreamShape<float>;
    return make_tensor_map(&c->smap[0], c->f[0], c->P, c->prec, S::BW, 1) &&
           make_tensor_map(&c->smap[1], c->f[1], c->P, c->prec, S::BW, 1);
}

bool pipe_ready(lbm_ctx *c)
{
    using S = lbm::TmaPipeShape;
    return c->prec == LBM_FP32_DEV && lbm::tma_pipe_supported(c->P) && lbm::tma_pipe_prepare() == cudaSuccess &&
           make_tensor_map(&c->pmap[0], c->f[0], c->P, c->prec, S::SW, S::SH) &&
           make_tensor_map(&c->pmap[1], c->f[1], c->P, c->prec, S::SW, S::SH);
}

bool stream_ready(lbm_ctx *c)
{
    return lbm::stream_supported(c->P) && lbm::stream_prepare() == cudaSuccess && make_row_maps(c);
}

bool tma_ready(lbm_ctx *c)
{
    return lbm::tma_supported(c->P, c->prec) && lbm::tma_prepare() == cudaSuccess && make_tile_maps(c);
}

// The TMA-staged tile kernel takes the x halo of tiles at a periodic x edge from the wrapped
// interior itself: on a grid periodic in x it needs only the ghost rows.
bool ghost_rows_only(const lbm_ctx *c) { return (c->use_tma || c->use_dd) && (c->P.wrap & 1); }

// The double-float float64 kernel: the float64 tile maps and the Coef<dd> of the context.
bool dd_ready(lbm_ctx *c)
{
    if (c->prec != LBM_FP64 || !lbm::tma_supported(c->P, LBM_FP64) || lbm::dd_prepare() != cudaSuccess) return false;
    lbm::coef_dd(c->P, &c->cdd);
    return make_tile_maps(c);
}

// The double-float kernel on narrow tiles (grids of 4 to 31 rows): their maps and the Coef<dd>.
bool ddn_ready(lbm_ctx *c)
{
    if (c->prec != LBM_FP64 || !lbm::dd_narrow_supported(c->P) || lbm::dd_prepare() != cudaSuccess) return false;
    lbm::coef_dd(c->P, &c->cdd);
    return make_narrow_maps(c);
}

// One fused step of context c from buffer `in` into buffer in ^ 1, on stream st.
cudaError_t launch_fused_step(lbm_ctx *c, int in, cudaStream_t st)
{
    if (c->use_dd) return lbm::launch_step_dd(c->P, &c->cdd, &c->tmap[in], c->f[in], c->f[in ^ 1], c->tma_err, st);
    if (c->use_ddn)
        return lbm::launch_step_dd(c->P, &c->cdd, &c->nmap[in], c->f[in], c->f[in ^ 1], c->tma_err, st, true);
    if (c->use_pipe) return lbm::launch_step_tma_pipe(c->P, &c->pmap[in], c->f[in ^ 1], c->tma_err, st);
    if (c->use_stream) return lbm::launch_step_stream(c->P, c->prec, &c->smap[in], c->f[in ^ 1], c->tma_err, st);
    if (c->use_tma) return lbm::launch_step_tma(c->P, c->prec, &c->tmap[in], c->f[in], c->f[in ^ 1], c->tma_err, st);
    return lbm::launch_step(c->P, c->prec, c->f[in], c->f[in ^ 1], st, c->plain_ty);
}

constexpr int kGraphSteps = 16;

// The pair graph of context c starting from buffer `in` (two ghost fills and fused steps), captured
// on the context's private stream at first use.
cudaError_t step_pair_graph(lbm_ctx *c, int in)
{
    if (c->pair[in]) return cudaSuccess;
    cudaError_t ce = c->cap ? cudaSuccess : cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking);
    cudaGraph_t graph = nullptr;
    if (ce == cudaSuccess) ce = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal);
    if (ce != cudaSuccess) return ce;
    cudaError_t le = cudaSuccess;
    for (int k = 0; k < 2 && le == cudaSuccess; k++) {
        le = lbm::launch_ghost(c->P, c->prec, c->f[in ^ k], c->cap, ghost_rows_only(c));
        if (le == cudaSuccess) le = launch_fused_step(c, in ^ k, c->cap);
    }
    ce = cudaStreamEndCapture(c->cap, &graph);
    if (ce == cudaSuccess) ce = le;
    if (ce == cudaSuccess) ce = cudaGraphInstantiate(&c->pair[in], graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (ce != cudaSuccess) c->pair[in] = nullptr;
    return ce;
}

void drop_step_graphs(lbm_ctx *c)
{
    for (cudaGraphExec_t &g : c->pair) {
        if (g) cudaGraphExecDestroy(g);
        g = nullptr;
    }
}

}  // namespace

extern "C" {

size_t lbm_footprint(int nx, int ny, int precision)
{
    if (nx < 1 || ny < 1) return 0;
    const size_t es = precision == LBM_FP32_DEV ? sizeof(float) : sizeof(double);
    return 2 * (size_t)NQ * (size_t)(ny + 4) * pitch_of(nx) * es;
}

int lbm_create_ex(int nx, int ny, double dx, double dt, double gamma, double Pr, const double s_in[16],
                  int limiter, const lbm_bc *bc, const lbm_options *opt, lbm_ctx **out)
{
    if (!out) return fail(nullptr, LBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!s_in || !bc) return fail(nullptr, LBM_ERR_ARG, "s or bc is NULL");
    if (nx < 1 || ny < 1) return fail(nullptr, LBM_ERR_ARG, "nx and ny must be >= 1");
    if ((long long)nx * ny > (1LL << 31) - 1 || nx > (1 << 28) || ny > (1 << 28))
        return fail(nullptr, LBM_ERR_ARG, "grid too large");
    if (!finite_pos(dx) || !finite_pos(dt)) return fail(nullptr, LBM_ERR_ARG, "dx and dt must be finite and > 0");
    if (!std::isfinite(gamma) || !(gamma > 1.0)) return fail(nullptr, LBM_ERR_ARG, "gamma must be > 1");
    if (!finite_pos(Pr)) return fail(nullptr, LBM_ERR_ARG, "Pr must be finite and > 0");
    if (limiter < LBM_LIMITER_MC || limiter > LBM_LIMITER_UPWIND) return fail(nullptr, LBM_ERR_ARG, "unknown limiter");
    const int prec = opt ? opt->precision : LBM_FP64;
    if (prec != LBM_FP64 && prec != LBM_FP32_DEV) return fail(nullptr, LBM_ERR_ARG, "unknown precision");
    std::string msg;
    const lbm_edge_bc *edges[4] = {&bc->xlo, &bc->xhi, &bc->ylo, &bc->yhi};
    const char *names[4] = {"xlo", "xhi", "ylo", "yhi"};
    for (int e = 0; e < 4; e++) {
        const int rc = validate_bc_edge(*edges[e], names[e], msg);
        if (rc) return fail(nullptr, rc, msg);
    }
    if ((bc->xlo.kind == LBM_BC_PERIODIC) != (bc->xhi.kind == LBM_BC_PERIODIC) ||
        (bc->ylo.kind == LBM_BC_PERIODIC) != (bc->yhi.kind == LBM_BC_PERIODIC))
        return fail(nullptr, LBM_ERR_ARG, "periodic boundaries must be set on both edges of an axis");
    double s[16];
    for (int k = 0; k < 16; k++) s[k] = s_in[k];
    for (int k = 4; k < 16; k++)
        if (!std::isfinite(s[k]) || s[k] < 0.0) {
            if (k == 7 && s[k] <= 0.0) continue;
            return fail(nullptr, LBM_ERR_ARG, "relaxation rates s_5..s_16 must be finite and >= 0");
        }
    if (s[7] <= 0.0) {
        s[7] = s[8] = Pr * s[4];
    } else {
        if (!(s[4] > 0.0) || std::fabs(s[7] / s[4] - Pr) > 1e-12 * Pr)
            return fail(nullptr, LBM_ERR_ARG, "Pr must equal s_8 / s_5 (Sec. II)");
    }
    if (s[4] != s[5] || s[4] != s[6] || s[7] != s[8])
        return fail(nullptr, LBM_ERR_ARG, "isotropy requires s_5 = s_6 = s_7 and s_8 = s_9 (Sec. II)");
    for (int k = 4; k < 16; k++)
        if (s[k] * dt >= 2.0) return fail(nullptr, LBM_ERR_STABILITY, "s_k dt >= 2 for some k >= 5");
    const double dy = (opt && opt->dy > 0.0) ? opt->dy : dx;
    if (!finite_pos(dy)) return fail(nullptr, LBM_ERR_ARG, "dy must be finite and > 0");
    // largest velocity component is 6 (shell 2): Courant number 6 dt / min(dx, dy)
    if (6.0 * dt / (dx < dy ? dx : dy) > 1.0)
        return fail(nullptr, LBM_ERR_CFL, "Courant number 6 dt/min(dx, dy) exceeds 1");

    lbm_ctx *c = new (std::nothrow) lbm_ctx;
    if (!c) return fail(nullptr, LBM_ERR_OOM, "host allocation failed");
    Params &P = c->P;
    std::memset(&P, 0, sizeof(P));
    c->prec = prec;
    c->dx = dx;
    c->dy = dy;
    P.nx = nx;
    P.ny = ny;
    P.pitch = (int)pitch_of(nx);
    P.plane = (long long)(ny + 4) * P.pitch;
    P.limiter = limiter;
    P.dt = dt;
    lbm::Coef<double> &C = P.cd;
    C.b = 2.0 / (gamma - 1.0);
    C.inv_b = 1.0 / C.b;
    C.four_inv_b = 4.0 / C.b;
    C.two_b2 = 2.0 * (C.b + 2.0);
    C.six_b = 6.0 + C.b;
    C.b4 = C.b + 4.0;
    if (prec == LBM_FP32_DEV) {
        C.rho0 = (opt && opt->rho0 > 0.0) ? opt->rho0 : 1.0;
        P.T0 = (opt && opt->T0 > 0.0) ? opt->T0 : 1.0;
        C.P0 = C.rho0 * P.T0;
        C.e0 = C.b * C.P0;
        C.P0T0 = C.P0 * P.T0;
    }
    if (!build_inverse_blocks(C)) {
        delete c;
        return fail(nullptr, LBM_ERR_ARG, "transformation blocks are singular");
    }
    fold_rates(C, s, dt);
    const double k8 = (s[7] == s[4]) ? 0.0 : s[7] / s[4] - 1.0;
    const double k9 = (s[8] == s[4]) ? 0.0 : s[8] / s[4] - 1.0;
    P.has_c9 = (k8 != 0.0 || k9 != 0.0) ? 1 : 0;

    C.q8 = (k8 != 0.0) ? k8 / s[7] / (2.0 * dx) : 0.0;
    C.q9 = (k9 != 0.0) ? k9 / s[8] / (2.0 * dx) : 0.0;
    C.ry = dx / dy;
    C.g4[0] = 4.0;
    C.g4[1] = 4.0 * C.ry;
    C.pad_ = 0.0;
    // Courant number per shell and axis: dt / (A_i d_alpha), A_i = 1, 1/6, 1/sqrt2, sqrt2/3 (Sec. III)
    const double A[4] = {1.0, 1.0 / 6.0, 1.0 / lbm::kSqrt2, lbm::kSqrt2 / 3.0};
    for (int k = 0; k < 4; k++) {
        C.cr[k] = dt / (A[k] * dx);
        C.ncr[k] = -C.cr[k];
        C.hh[k] = 0.25 * (1.0 - C.cr[k]);
        C.cry[k] = dt / (A[k] * dy);
        C.ncry[k] = -C.cry[k];
        C.hhy[k] = 0.25 * (1.0 - C.cry[k]);
    }
    // the float tables are the float64 tables rounded once
    static_assert(sizeof(lbm::Coef<double>) == 2 * sizeof(lbm::Coef<float>), "Coef layout");
    {
        const double *src = reinterpret_cast<const double *>(&P.cd);
        float *dst = reinterpret_cast<float *>(&P.cf);
        for (size_t k = 0; k < sizeof(lbm::Coef<double>) / sizeof(double); k++) dst[k] = (float)src[k];
    }
    if (prec == LBM_FP32_DEV) host_feq<false>(P, C.rho0, 0.0, 0.0, P.T0, P.feq0);
    for (int e = 0; e < 4; e++) {
        lbm::EdgeDev &E = P.edge[e];
        E.kind = edges[e]->kind;
        E.uw = edges[e]->u;
        E.vw = edges[e]->v;
        E.Tw = edges[e]->T;
        E.two_rho0_dTw = 2.0 * C.rho0 * (edges[e]->T - P.T0);
        if (E.kind == LBM_BC_EQUILIBRIUM) {
            if (prec == LBM_FP32_DEV) host_feq<true>(P, edges[e]->rho, edges[e]->u, edges[e]->v, edges[e]->T, E.feq);
            else host_feq<false>(P, edges[e]->rho, edges[e]->u, edges[e]->v, edges[e]->T, E.feq);
        }
        E.uwf = (float)E.uw;
        E.vwf = (float)E.vw;
        E.Twf = (float)E.Tw;
        E.two_rho0_dTwf = (float)E.two_rho0_dTw;
        for (int q = 0; q < NQ; q++) E.feqf[q] = (float)E.feq[q];
    }

    // device, stream, allocator
    cudaError_t ce;
    if (opt && opt->device >= 0) {
        ce = cudaSetDevice(opt->device);
        if (ce != cudaSuccess) { delete c; return cuda_fail(nullptr, ce, "cudaSetDevice"); }
    }
    ce = cudaGetDevice(&c->device);
    if (ce != cudaSuccess) { delete c; return cuda_fail(nullptr, ce, "cudaGetDevice"); }
    c->stream = opt ? (cudaStream_t)opt->stream : nullptr;
    if (opt && opt->allocator && opt->allocator->alloc && opt->allocator->free) {
        c->alloc = *opt->allocator;
        c->own_alloc = false;
    } else {
        c->alloc.alloc = default_alloc;
        c->alloc.free = default_free;
        c->alloc.user = nullptr;
    }
    c->buf_bytes = lbm_footprint(nx, ny, prec);
    const size_t cells = (size_t)nx * ny;
    c->stage_elems = std::min<size_t>(20 * cells, std::max<size_t>(20 * (size_t)nx, (size_t)8 << 20));
    c->aux_bytes = sizeof(double) * (lbm::kTotalsBlocks * NQ + 4) + 64;
    c->buf = c->alloc.alloc(c->buf_bytes, c->stream, c->alloc.user);
    c->stage = c->buf ? (double *)c->alloc.alloc(c->stage_elems * sizeof(double), c->stream, c->alloc.user) : nullptr;
    c->aux = c->stage ? (double *)c->alloc.alloc(c->aux_bytes, c->stream, c->alloc.user) : nullptr;
    if (!c->buf || !c->stage || !c->aux) {
        cudaGetLastError();
        lbm_destroy(c);
        return fail(nullptr, LBM_ERR_OOM, "device allocation failed");
    }
    c->f[0] = c->buf;
    c->f[1] = (char *)c->buf + c->buf_bytes / 2;
    c->tot_out = c->aux + lbm::kTotalsBlocks * NQ;
    c->flag = (int *)(c->tot_out + 4);
    c->tma_err = c->flag + 1;
    c->init_err = c->flag + 2;
    int want = opt ? opt->step_kernel : 0;
    if (want < 0 || want > 9) {
        lbm_destroy(c);
        return fail(nullptr, LBM_ERR_ARG, "unknown step_kernel");
    }
    if (want == 3) c->plain_ty = 4;
    if (want == 4) c->plain_ty = 16;
    if (want == 7) c->plain_ty = 2;
    // automatic, float64: the double-float kernels (on GB300 the float32 pipe runs their
    // arithmetic 2.5x faster than the float64 kernels run theirs) wherever their tiles fit; on
    // grids narrower than 32 columns or lower than 4 rows the float64 pipe (about 1.6 lane
    // operations per cycle per SM): the streaming kernel when the grid gives every SM at least
    // 32 rows of a 256-column strip; else the plain kernel, on 256-cell tiles when they still
    // give every SM four tiles (their flow-velocity ring costs less), on 64-cell tiles below
    // that, which spread a small grid's float64 work over more SMs.  The double-float kernel
    // runs on 32 x 32 tiles where the grid has at least two thirds of a wave of them (one CTA
    // per SM); on smaller grids, and on grids of 4 to 31 rows, on 32 x 4 tiles (two CTAs per
    // SM): a 32 x 32 tile takes about 44 us on its SM, so a small grid finishes sooner in more,
    // shorter tiles (128 x 96: 17 us against 44 us a step)
    if (want == 0 && prec == LBM_FP64) {
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
        if (sms < 1) sms = 152;
        const long long tiles = (long long)((nx + lbm::kTmaTX - 1) / lbm::kTmaTX) *
                                ((ny + lbm::TmaShape<double>::TR - 1) / lbm::TmaShape<double>::TR);
        if (3 * tiles >= 2LL * sms && dd_ready(c)) want = 8;
        cudaGetLastError();
        if (want == 0 && ddn_ready(c)) want = 9;
        cudaGetLastError();
    }
    if (want == 0 && prec == LBM_FP64) {
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
        if (sms < 1) sms = 152;
        const long long strips = (nx + lbm::StreamShape<double>::W - 1) / lbm::StreamShape<double>::W;
        const long long cells = (long long)nx * ny;
        if (strips * ny < 32LL * sms || cells < (4LL << 20)) {
            want = cells >= 4LL * lbm::kBatchThreads * sms ? 1 : 7;
            c->plain_ty = want == 7 ? 2 : lbm::kTY;
        }
    }
    // automatic: float64 runs the streaming kernel (fewer float64 operations per cell), float32
    // the TMA-staged tile kernel (fewer instructions per cell); each falls back to the other
    // and then to the plain kernel where the grid or driver does not allow it
    if ((want == 5 || (want == 0 && prec == LBM_FP64)) && stream_ready(c)) c->use_stream = true;
    if ((want == 2 || (want == 0 && !c->use_stream)) && tma_ready(c)) c->use_tma = true;
    // x halo of periodic edge tiles wrapped inside the TMA-staged tile kernel (P.wrap bit 0), on
    // grids of at least 32 waves of its tiles (2048 cells per SM a wave): there the kernel's
    // extra loads in edge tiles cost less than the ghost columns' copy; on smaller grids a
    // kernel lasts as long as its slowest tiles, which the extra loads lengthen
    if (want == 8 && dd_ready(c)) c->use_dd = true;
    if (want == 9 && ddn_ready(c)) c->use_ddn = true;
    if ((c->use_tma || c->use_dd) && bc->xlo.kind == LBM_BC_PERIODIC) {
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
        if (sms < 1) sms = 152;
        if ((long long)nx * ny >= 32LL * 2048 * sms) c->P.wrap = 1;
    }
    if (want == 6 && pipe_ready(c)) c->use_pipe = true;
    if ((want == 2 && !c->use_tma) || (want == 5 && !c->use_stream) || (want == 6 && !c->use_pipe) ||
        (want == 8 && !c->use_dd) || (want == 9 && !c->use_ddn)) {
        lbm_destroy(c);
        return fail(nullptr, LBM_ERR_ARG, "requested step kernel unavailable for this grid or driver");
    }
    cudaGetLastError();
    ce = cudaMemsetAsync(c->buf, 0, c->buf_bytes, c->stream);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(c->aux, 0, c->aux_bytes, c->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(c->stream);
    if (ce != cudaSuccess) {
        lbm_destroy(c);
        return cuda_fail(nullptr, ce, "device initialisation");
    }
    *out = c;
    return LBM_OK;
}

int lbm_create(int nx, int ny, double dx, double dt, double gamma, double Pr, const double s[16], int limiter,
               const lbm_bc *bc, lbm_ctx **out)
{
    return lbm_create_ex(nx, ny, dx, dt, gamma, Pr, s, limiter, bc, nullptr, out);
}

// Device address of a host array of `bytes` bytes that kernels can access directly: page-locked
// memory allocated or registered through CUDA (cudaHostAlloc, cudaHostRegister, a pinned torch
// tensor), checked at both ends of the range.  nullptr for any other memory.
static void *mapped_host(const void *p, size_t bytes)
{
    if (!p || bytes == 0) return nullptr;
    cudaPointerAttributes a{}, b{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
    const char *last = static_cast<const char *>(p) + (bytes - 1);
    if (cudaPointerGetAttributes(&b, last) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (b.type != cudaMemoryTypeHost || static_cast<char *>(b.devicePointer) != static_cast<char *>(a.devicePointer) + (bytes - 1))
        return nullptr;
    return a.devicePointer;
}

static int rows_per_chunk(const lbm_ctx *c, int planes)
{
    const size_t per_row = (size_t)planes * c->P.nx;
    size_t r = c->stage_elems / per_row;
    if (r < 1) r = 1;
    if (r > (size_t)c->P.ny) r = c->P.ny;
    return (int)r;
}

int lbm_init(lbm_ctx *c, const double *rho, const double *u, const double *v, const double *T)
{
    if (!c) return fail(nullptr, LBM_ERR_ARG, "ctx is NULL");
    if (!rho || !u || !v || !T) return fail(c, LBM_ERR_ARG, "NULL field");
    cudaError_t ce = cudaSetDevice(c->device);
    if (ce != cudaSuccess) return cuda_fail(c, ce, "cudaSetDevice");
    // the fields are checked by the init kernel (rho > 0, T > 0, finite), which flags a bad cell
    c->initialized = false;
    ce = cudaMemsetAsync(c->init_err, 0, sizeof(int), c->stream);
    if (ce != cudaSuccess) return cuda_fail(c, ce, "flag reset");
    const int nx = c->P.nx, ny = c->P.ny;
    const size_t field_bytes = (size_t)nx * ny * sizeof(double);
    const double *src[4] = {rho, u, v, T};
    const double *dev[4];
    bool direct = true;
    for (int k = 0; k < 4; k++) {
        dev[k] = static_cast<const double *>(mapped_host(src[k], field_bytes));
        direct = direct && dev[k];
    }
    if (direct) {
        // page-locked host fields: the init kernel reads them over the host link itself
        ce = lbm::launch_init(c->P, c->prec, c->f[c->cur], dev[0], dev[1], dev[2], dev[3], 0, ny, c->init_err,
                              c->stream);
        if (ce != cudaSuccess) return cuda_fail(c, ce, "init kernel");
    } else {
        const int R = rows_per_chunk(c, 4);
        // one stream: each chunk's copies follow the previous chunk's kernel, so the staging
        // buffer is reused without waiting on the host
        for (int r0 = 0; r0 < ny; r0 += R) {
            const int rows = std::min(R, ny - r0);
            const size_t m = (size_t)rows * nx;
            for (int k = 0; k < 4; k++) {
                ce = cudaMemcpyAsync(c->stage + k * m, src[k] + (size_t)r0 * nx, m * sizeof(double),
                                     cudaMemcpyHostToDevice, c->stream);
                if (ce != cudaSuccess) return cuda_fail(c, ce, "init copy");
            }
            ce = lbm::launch_init(c->P, c->prec, c->f[c->cur], c->stage, c->stage + m, c->stage + 2 * m,
                                  c->stage + 3 * m, r0, rows, c->init_err, c->stream);
            if (ce != cudaSuccess) return cuda_fail(c, ce, "init kernel");
        }
    }
    int bad = 0;
    ce = cudaMemcpyAsync(&bad, c->init_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(c->stream);
    if (ce != cudaSuccess) return cuda_fail(c, ce, "init");
    if (bad) return fail(c, LBM_ERR_ARG, "init fields need rho > 0, T > 0 and finite values");
    c->initialized = true;
    c->steps = 0;
    return LBM_OK;
}

int lbm_step(lbm_ctx *c, int n)
{
    if (!c) return fail(nullptr, LBM_ERR_ARG, "ctx is NULL");
    if (n <= 0) return fail(c, LBM_ERR_STATE, "n must be >= 1");
    if (!c->initialized) return fail(c, LBM_ERR_STATE, "lbm_step before lbm_init / lbm_set_state");
    cudaError_t ce = cudaSetDevice(c->device);
    if (ce != cudaSuccess) return cuda_fail(c, ce, "cudaSetDevice");
    // runs of at least kGraphSteps steps outside profiling: pairs of steps from a graph (one
    // launch instead of four; on small grids the launches, not the kernels, set the pace)
    if (!c->prof && n >= kGraphSteps) {
        ce = step_pair_graph(c, c->cur);
        if (ce != cudaSuccess) return cuda_fail(c, ce, "step graph");
        for (; n >= 2; n -= 2) {
            ce = cudaGraphLaunch(c->pair[c->cur], c->stream);
            if (ce != cudaSuccess) return cuda_fail(c, ce, "step graph launch");
            c->steps += 2;
        }
        if (n == 0) return LBM_OK;
    }
    for (int s = 0; s < n; s++) {
        cudaEvent_t *ev = nullptr;
        if (c->prof && c->prof_used < c->prof_max) ev = &c->prof_ev[4 * c->prof_used++];
        if (ev) cudaEventRecord(ev[0], c->stream);
        ce = lbm::launch_ghost(c->P, c->prec, c->f[c->cur], c->stream, ghost_rows_only(c));
        if (ce != cudaSuccess) return cuda_fail(c, ce, "ghost kernel");
        if (ev) { cudaEventRecord(ev[1], c->stream); cudaEventRecord(ev[2], c->stream); }
        ce = launch_fused_step(c, c->cur, c->stream);
        if (ce != cudaSuccess) return cuda_fail(c, ce, "step kernel");
        if (ev) cudaEventRecord(ev[3], c->stream);
        c->cur ^= 1;
        c->steps++;
    }
    return LBM_OK;
}

static int moments_impl(lbm_ctx *c, double *rho, double *u, double *v, double *T, double *delta, double *dstar)
{
    if (!c) return fail(nullptr, LBM_ERR_ARG, "ctx is NULL");
    if (!c->initialized) return fail(c, LBM_ERR_STATE, "moments before lbm_init / lbm_set_state");
    cudaError_t ce = cudaSetDevice(c->device);
    if (ce != cudaSuccess) return cuda_fail(c, ce, "cudaSetDevice");
    const int planes = (rho ? 1 : 0) + (u ? 1 : 0) + (v ? 1 : 0) + (T ? 1 : 0) + (delta ? 16 : 0) + (dstar ? 16 : 0);
    ce = cudaMemsetAsync(c->flag, 0, sizeof(int), c->stream);
    if (ce != cudaSuccess) return cuda_fail(c, ce, "flag reset");
    const int nx = c->P.nx, ny = c->P.ny;
    const size_t plane_bytes = (size_t)nx * ny * sizeof(double);
    struct { double *h; int planes; } req[6] = {{rho, 1}, {u, 1}, {v, 1}, {T, 1}, {delta, 16}, {dstar, 16}};
    double *dev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    bool direct = planes > 0;
    for (int k = 0; k < 6; k++) {
        if (!req[k].h) continue;
        dev[k] = static_cast<double *>(mapped_host(req[k].h, req[k].planes * plane_bytes));
        direct = direct && dev[k];
    }
    if (direct) {
        // page-locked host outputs: the moments kernel writes them over the host link itself
        ce = lbm::launch_moments(c->P, c->prec, c->f[c->cur], 0, ny, dev[0], dev[1], dev[2], dev[3], dev[4], dev[5],
                                 c->flag, c->stream);
        if (ce != cudaSuccess) return cuda_fail(c, ce, "moments kernel");
    }
    const int R = rows_per_chunk(c, planes > 0 ? planes : 1);
    for (int r0 = 0; r0 < ny && !direct; r0 += R) {
        const int rows = std::min(R, ny - r0);
        const size_t m = (size_t)rows * nx;
        double *p = c->stage;
        double *d_rho = rho ? p : nullptr; p += rho ? m : 0;
        double *d_u = u ? p : nullptr; p += u ? m : 0;
        double *d_v = v ? p : nullptr; p += v ? m : 0;
        double *d_T = T ? p : nullptr; p += T ? m : 0;
        double *d_delta = delta ? p : nullptr; p += delta ? 16 * m : 0;
        double *d_dstar = dstar ? p : nullptr;
        ce = lbm::launch_moments(c->P, c->prec, c->f[c->cur], r0, rows, d_rho, d_u, d_v, d_T, d_delta, d_dstar,
                                 c->flag, c->stream);
        if (ce != cudaSuccess) return cuda_fail(c, ce, "moments kernel");
        struct { double *h, *d; int planes; } outs[6] = {{rho, d_rho, 1}, {u, d_u, 1}, {v, d_v, 1}, {T, d_T, 1},
                                                          {delta, d_delta, 16}, {dstar, d_dstar, 16}};
        for (auto &o : outs) {
            if (!o.h) continue;
            for (int k = 0; k < o.planes; k++) {
                ce = cudaMemcpyAsync(o.h + (size_t)k * nx * ny + (size_t)r0 * nx, o.d + k * m, m * sizeof(double),
                                     cudaMemcpyDeviceToHost, c->stream);
                if (ce != cudaSuccess) return cuda_fail(c, ce, "moments copy");
            }
        }
        // the next chunk's kernel follows these copies on the stream: no host wait here
    }
    int flags[2] = {0, 0};
    ce = cudaMemcpyAsync(flags, c->flag, sizeof(flags), cudaMemcpyDeviceToHost, c->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(c->stream);
    if (ce != cudaSuccess) return cuda_fail(c, ce, "moments");
    if (flags[1]) return fail(c, LBM_ERR_TIMEOUT, "a copy wait ran out in the step kernel");
    if (flags[0]) return fail(c, LBM_ERR_NONFINITE, "a cell has a non-finite value or rho <= 0");
    return LBM_OK;
}

int lbm_moments(lbm_ctx *c, double *rho, double *u, double *v, double *T, double *delta)
{
    return moments_impl(c, rho, u, v, T, delta, nullptr);
}

int lbm_moments_central(lbm_ctx *c, double *delta_star)
{
    if (c && !delta_star) return fail(c, LBM_ERR_ARG, "delta_star is NULL");
    return moments_impl(c, nullptr, nullptr, nullptr, nullptr, nullptr, delta_star);
}

int lbm_totals(lbm_ctx *c, double out[4])
{
    if (!c) return fail(nullptr, LBM_ERR_ARG, "ctx is NULL");
    if (!out) return fail(c, LBM_ERR_ARG, "out is NULL");
    if (!c->initialized) return fail(c, LBM_ERR_STATE, "totals before lbm_init / lbm_set_state");
    cudaError_t ce = cudaSetDevice(c->device);
    if (ce != cudaSuccess) return cuda_fail(c, ce, "cudaSetDevice");
    ce = lbm::launch_totals(c->P, c->prec, c->f[c->cur], c->aux, c->tot_out, c->dx * c->dy, c->stream);
    if (ce != cudaSuccess) return cuda_fail(c, ce, "totals kernel");
    double h[4];
    ce = cudaMemcpyAsync(h, c->tot_out, sizeof(h), cudaMemcpyDeviceToHost, c->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(c->stream);
    if (ce != cudaSuccess) return cuda_fail(c, ce, "totals");
    for (int k = 0; k < 4; k++) out[k] = h[k];
    return LBM_OK;
}

int lbm_get_state(lbm_ctx *c, double *f)
{
    if (!c) return fail(nullptr, LBM_ERR_ARG, "ctx is NULL");
    if (!f) return fail(c, LBM_ERR_ARG, "f is NULL");
    if (!c->initialized) return fail(c, LBM_ERR_STATE, "get_state before lbm_init / lbm_set_state");
    cudaError_t ce = cudaSetDevice(c->device);
    if (ce != cudaSuccess) return cuda_fail(c, ce, "cudaSetDevice");
    const int nx = c->P.nx, ny = c->P.ny;
    // page-locked host array: the pack kernel writes it over the host link itself
    double *dev = static_cast<double *>(mapped_host(f, (size_t)NQ * nx * ny * sizeof(double)));
    if (dev) {
        ce = lbm::launch_pack(c->P, c->prec, c->f[c->cur], 0, ny, dev, c->stream);
        if (ce != cudaSuccess) return cuda_fail(c, ce, "pack kernel");
    }
    const int R = rows_per_chunk(c, 16);
    for (int r0 = 0; r0 < ny && !dev; r0 += R) {
        const int rows = std::min(R, ny - r0);
        const size_t m = (size_t)rows * nx;
        ce = lbm::launch_pack(c->P, c->prec, c->f[c->cur], r0, rows, c->stage, c->stream);
        if (ce != cudaSuccess) return cuda_fail(c, ce, "pack kernel");
        for (int q = 0; q < NQ; q++) {
            ce = cudaMemcpyAsync(f + (size_t)q * nx * ny + (size_t)r0 * nx, c->stage + q * m, m * sizeof(double),
                                 cudaMemcpyDeviceToHost, c->stream);
            if (ce != cudaSuccess) return cuda_fail(c, ce, "state copy");
        }
    }
    ce = cudaStreamSynchronize(c->stream);   // chunks are ordered on the stream; one wait at the end
    if (ce != cudaSuccess) return cuda_fail(c, ce, "get_state");
    return LBM_OK;
}

int lbm_get_state_rows(lbm_ctx *c, int row0, int rows, double *f)
{
    if (!c) return fail(nullptr, LBM_ERR_ARG, "ctx is NULL");
    if (!f) return fail(c, LBM_ERR_ARG, "f is NULL");
    if (row0 < 0 || rows < 1 || row0 + rows > c->P.ny) return fail(c, LBM_ERR_ARG, "row window outside [0, ny)");
    if (!c->initialized) return fail(c, LBM_ERR_STATE, "get_state before lbm_init / lbm_set_state");
    cudaError_t ce = cudaSetDevice(c->device);
    if (ce != cudaSuccess) return cuda_fail(c, ce, "cudaSetDevice");
    const int nx = c->P.nx;
    double *dev = static_cast<double *>(mapped_host(f, (size_t)NQ * nx * rows * sizeof(double)));
    if (dev) {
        ce = lbm::launch_pack(c->P, c->prec, c->f[c->cur], row0, rows, dev, c->stream);
        if (ce != cudaSuccess) return cuda_fail(c, ce, "pack kernel");
    }
    const int R = rows_per_chunk(c, 16);
    for (int r = 0; r < rows && !dev; r += R) {
        const int n = std::min(R, rows - r);
        const size_t m = (size_t)n * nx;
        ce = lbm::launch_pack(c->P, c->prec, c->f[c->cur], row0 + r, n, c->stage, c->stream);
        if (ce != cudaSuccess) return cuda_fail(c, ce, "pack kernel");
        for (int q = 0; q < NQ; q++) {
            ce = cudaMemcpyAsync(f + (size_t)q * nx * rows + (size_t)r * nx, c->stage + q * m, m * sizeof(double),
                                 cudaMemcpyDeviceToHost, c->stream);
            if (ce != cudaSuccess) return cuda_fail(c, ce, "state copy");
        }
    }
    ce = cudaStreamSynchronize(c->stream);   // chunks are ordered on the stream; one wait at the end
    if (ce != cudaSuccess) return cuda_fail(c, ce, "get_state_rows");
    return LBM_OK;
}

int lbm_set_state(lbm_ctx *c, const double *f)
{
    if (!c) return fail(nullptr, LBM_ERR_ARG, "ctx is NULL");
    if (!f) return fail(c, LBM_ERR_ARG, "f is NULL");
    cudaError_t ce = cudaSetDevice(c->device);
    if (ce != cudaSuccess) return cuda_fail(c, ce, "cudaSetDevice");
    const int nx = c->P.nx, ny = c->P.ny;
    // page-locked host array: the unpack kernel reads it over the host link itself
    const double *dev = static_cast<const double *>(mapped_host(f, (size_t)NQ * nx * ny * sizeof(double)));
    if (dev) {
        ce = lbm::launch_unpack(c->P, c->prec, c->f[c->cur], 0, ny, dev, c->stream);
        if (ce != cudaSuccess) return cuda_fail(c, ce, "unpack kernel");
    }
    const int R = rows_per_chunk(c, 16);
    for (int r0 = 0; r0 < ny && !dev; r0 += R) {
        const int rows = std::min(R, ny - r0);
        const size_t m = (size_t)rows * nx;
        for (int q = 0; q < NQ; q++) {
            ce = cudaMemcpyAsync(c->stage + q * m, f + (size_t)q * nx * ny + (size_t)r0 * nx, m * sizeof(double),
                                 cudaMemcpyHostToDevice, c->stream);
            if (ce != cudaSuccess) return cuda_fail(c, ce, "state copy");
        }
        ce = lbm::launch_unpack(c->P, c->prec, c->f[c->cur], r0, rows, c->stage, c->stream);
        if (ce != cudaSuccess) return cuda_fail(c, ce, "unpack kernel");
    }
    ce = cudaStreamSynchronize(c->stream);   // chunks are ordered on the stream; one wait at the end
    if (ce != cudaSuccess) return cuda_fail(c, ce, "set_state");
    c->initialized = true;
    c->steps = 0;
    return LBM_OK;
}

int lbm_profile_begin(lbm_ctx *c, int max_steps)
{
    if (!c) return fail(nullptr, LBM_ERR_ARG, "ctx is NULL");
    if (max_steps < 1 || max_steps > (1 << 20)) return fail(c, LBM_ERR_ARG, "max_steps out of range");
    cudaError_t ce = cudaSetDevice(c->device);
    if (ce != cudaSuccess) return cuda_fail(c, ce, "cudaSetDevice");
    for (cudaEvent_t e : c->prof_ev) cudaEventDestroy(e);
    c->prof_ev.assign(4 * (size_t)max_steps, nullptr);
    for (auto &e : c->prof_ev) {
        ce = cudaEventCreate(&e);
        if (ce != cudaSuccess) return cuda_fail(c, ce, "cudaEventCreate");
    }
    c->prof = true;
    c->prof_max = max_steps;
    c->prof_used = 0;
    return LBM_OK;
}

int lbm_profile_end(lbm_ctx *c, double out[4])
{
    if (!c) return fail(nullptr, LBM_ERR_ARG, "ctx is NULL");
    if (!c->prof) return fail(c, LBM_ERR_STATE, "lbm_profile_end without lbm_profile_begin");
    if (!out) return fail(c, LBM_ERR_ARG, "out is NULL");
    cudaError_t ce = cudaSetDevice(c->device);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(c->stream);
    if (ce != cudaSuccess) return cuda_fail(c, ce, "profile sync");
    double step_ms = 0.0, ghost_ms = 0.0;
    for (int i = 0; i < c->prof_used; i++) {
        float a = 0.f, b = 0.f;
        cudaEventElapsedTime(&a, c->prof_ev[4 * i], c->prof_ev[4 * i + 1]);
        cudaEventElapsedTime(&b, c->prof_ev[4 * i + 2], c->prof_ev[4 * i + 3]);
        ghost_ms += a;
        step_ms += b;
    }
    out[0] = step_ms;
    out[1] = c->prof_used;
    out[2] = ghost_ms;
    out[3] = c->prof_used;
    for (cudaEvent_t e : c->prof_ev) cudaEventDestroy(e);
    c->prof_ev.clear();
    c->prof = false;
    c->prof_used = c->prof_max = 0;
    return LBM_OK;
}

int lbm_peak_fp64(int device, double *flops)
{
    if (!flops) return fail(nullptr, LBM_ERR_ARG, "flops is NULL");
    cudaError_t ce = cudaSetDevice(device);
    if (ce != cudaSuccess) return cuda_fail(nullptr, ce, "cudaSetDevice");
    double v = 0.0;
    ce = lbm::measure_fp64_fma(&v);
    if (ce != cudaSuccess) return cuda_fail(nullptr, ce, "fp64 peak kernel");
    *flops = v;
    return LBM_OK;
}

int lbm_wait_selftest(int device, double *elapsed_ms)
{
    cudaError_t ce = cudaSetDevice(device);
    if (ce != cudaSuccess) return cuda_fail(nullptr, ce, "cudaSetDevice");
    int *flag = nullptr;
    ce = cudaMalloc(&flag, sizeof(int));
    if (ce != cudaSuccess) return cuda_fail(nullptr, ce, "cudaMalloc");
    float ms = 0.f;
    int timed_out = 0;
    ce = lbm::wait_selftest(flag, &ms);
    if (ce == cudaSuccess) ce = cudaMemcpy(&timed_out, flag, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(flag);
    if (ce != cudaSuccess) return cuda_fail(nullptr, ce, "wait self-test");
    if (elapsed_ms) *elapsed_ms = ms;
    if (timed_out) return fail(nullptr, LBM_ERR_TIMEOUT, "the bounded wait ran out (expected)");
    return LBM_OK;
}

int lbm_autotune(lbm_ctx *c, int reps, int *choice)
{
    if (!c) return fail(nullptr, LBM_ERR_ARG, "ctx is NULL");
    if (reps < 1 || reps > 1000) return fail(c, LBM_ERR_ARG, "reps must be in [1, 1000]");
    if (!c->initialized) return fail(c, LBM_ERR_STATE, "autotune before lbm_init / lbm_set_state");
    cudaError_t ce = cudaSetDevice(c->device);
    if (ce != cudaSuccess) return cuda_fail(c, ce, "cudaSetDevice");
    // candidates: 1 = plain 32x8, 3 = plain 32x4, 4 = plain 32x16, 7 = plain 64-cell tiles,
    // 2 = TMA-staged, 5 = streaming, 6 = double-buffered TMA-staged 32x16 (float32),
    // 8 = double-float TMA-staged (float64), 9 = the same on 32 x 4 tiles
    int cands[10] = {1, 3, 4, 7, 0, 0, 0, 0, 0, 0};
    int ncand = 4;
    const bool tma_ok = c->use_tma || tma_ready(c);
    cudaGetLastError();
    const bool stream_ok = c->use_stream || stream_ready(c);
    cudaGetLastError();
    if (tma_ok) cands[ncand++] = 2;
    if (stream_ok) cands[ncand++] = 5;
    const bool pipe_ok = c->use_pipe || pipe_ready(c);
    cudaGetLastError();
    if (pipe_ok) cands[ncand++] = 6;
    const bool dd_ok = c->use_dd || dd_ready(c);
    cudaGetLastError();
    if (dd_ok) cands[ncand++] = 8;
    const bool ddn_ok = c->use_ddn || ddn_ready(c);
    cudaGetLastError();
    if (ddn_ok) cands[ncand++] = 9;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return cuda_fail(c, cudaGetLastError(), "cudaEventCreate");
    // the candidates write the other buffer without flipping it: the state does not advance
    ce = lbm::launch_ghost(c->P, c->prec, c->f[c->cur], c->stream);
    float best = 1e30f;
    int best_c = 1;
    for (int k = 0; k < ncand && ce == cudaSuccess; k++) {
        auto run = [&]() {
            const int cd = cands[k];
            if (cd == 9)
                return lbm::launch_step_dd(c->P, &c->cdd, &c->nmap[c->cur], c->f[c->cur], c->f[c->cur ^ 1],
                                           c->tma_err, c->stream, true);
            if (cd == 8)
                return lbm::launch_step_dd(c->P, &c->cdd, &c->tmap[c->cur], c->f[c->cur], c->f[c->cur ^ 1],
                                           c->tma_err, c->stream);
            if (cd == 6)
                return lbm::launch_step_tma_pipe(c->P, &c->pmap[c->cur], c->f[c->cur ^ 1], c->tma_err, c->stream);
            if (cd == 5)
                return lbm::launch_step_stream(c->P, c->prec, &c->smap[c->cur], c->f[c->cur ^ 1], c->tma_err,
                                               c->stream);
            if (cd == 2)
                return lbm::launch_step_tma(c->P, c->prec, &c->tmap[c->cur], c->f[c->cur], c->f[c->cur ^ 1], c->tma_err,
                                            c->stream);
            return lbm::launch_step(c->P, c->prec, c->f[c->cur], c->f[c->cur ^ 1], c->stream,
                                    cd == 3 ? 4 : (cd == 4 ? 16 : (cd == 7 ? 2 : 8)));
        };
        ce = run();
        if (ce != cudaSuccess) break;
        cudaEventRecord(e0, c->stream);
        for (int r = 0; r < reps && ce == cudaSuccess; r++) ce = run();
        cudaEventRecord(e1, c->stream);
        if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
        if (ce == cudaSuccess && ms < best) { best = ms; best_c = cands[k]; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (ce != cudaSuccess) return cuda_fail(c, ce, "autotune");
    c->use_tma = best_c == 2;
    c->use_stream = best_c == 5;
    c->use_pipe = best_c == 6;
    drop_step_graphs(c);
    c->use_dd = best_c == 8;
    c->use_ddn = best_c == 9;
    c->plain_ty = best_c == 3 ? 4 : (best_c == 4 ? 16 : (best_c == 7 ? 2 : 8));
    if (choice) *choice = best_c;
    return LBM_OK;
}

long long lbm_step_count(const lbm_ctx *c) { return c ? c->steps : -1; }

int lbm_step_kernel(const lbm_ctx *c)
{
    if (!c) return -1;
    if (c->use_dd) return 8;
    if (c->use_ddn) return 9;
    if (c->use_pipe) return 6;
    if (c->use_stream) return 5;
    if (c->use_tma) return 2;
    return c->plain_ty == 4 ? 3 : (c->plain_ty == 16 ? 4 : (c->plain_ty == 2 ? 7 : 1));
}

}  // extern "C"

struct lbm_batch {
    struct Group {
        int prec = 0, limiter = 0;
        std::vector<int> members;               // indices into ctxs
        std::vector<char> own;                   // member steps on its own kernel (no tiles)
        std::vector<char> tma;                   // member's tiles go to the batched TMA-staged kernel
        std::vector<lbm::BatchGrid> hG;
        void *block = nullptr;                   // device: Params[n] | BatchGrid[n] | int4[ntiles]
        size_t bytes = 0;
        lbm::Params *dP = nullptr;
        lbm::BatchGrid *dG = nullptr;
        int4 *dT = nullptr;
        int ntiles = 0, max_ghost = 0;
        int nt = lbm::kBatchThreads;             // threads (= cells) per tile
        // batched TMA-staged kernels: the row spans they serve (member index into members, first
        // row, rows; in launch order; float64 spans on 32 x 32 tiles in tk, on narrow 32 x 4
        // tiles in tkn) and one TileGrid block per span (Coef<float> or Coef<dd> by precision),
        // tk's first.  A float64 member on 32 x 32 tiles whose last tile row would hold at most
        // 24 of its rows has those rows in a narrow span.
        struct Span {
            int k, y0, rows;
        };
        std::vector<Span> tk, tkn;
        void *tblock = nullptr;
        size_t tbytes = 0;
        int ntt = 0;                             // tiles per step
    };
    std::vector<lbm_ctx *> ctxs;
    std::vector<Group> groups;
    // contexts on the streaming or the double-buffered kernel with at least a quarter wave of
    // its work: their ghost cells come from their group's batched ghost launch, their step from
    // that kernel, launched on kForks forked streams so that the grids' kernels overlap
    static constexpr int kForks = 8;
    std::vector<int> solo;
    std::vector<int> cap_cur;                   // every context's buffer parity at graph capture
    cudaStream_t fork[kForks] = {};
    cudaEvent_t ev_fork = nullptr, ev_join[kForks] = {};
    cudaStream_t stream = nullptr, cap = nullptr;
    cudaGraphExec_t exec2 = nullptr;
    lbm_allocator alloc{};
    int device = 0, ctas = 0;
};

namespace {

cudaError_t batch_upload_cur(lbm_batch *b)
{
    for (auto &g : b->groups) {
        for (size_t i = 0; i < g.members.size(); i++) g.hG[i].cur = b->ctxs[g.members[i]]->cur;
        cudaError_t ce = cudaMemcpyAsync(g.dG, g.hG.data(), g.hG.size() * sizeof(lbm::BatchGrid),
                                         cudaMemcpyHostToDevice, b->stream);
        if (ce != cudaSuccess) return ce;
    }
    return cudaSuccess;
}

// The group's batched TMA-staged launches (kTmaBatchGrids grids each) over the members `tk`
// (float32 tile kernel, or float64 double-float kernel on 32 x 32 tiles) and, in float64, over
// the members `tkn` on narrow 32 x 4 tiles, with every member's input map, output buffer and flag
// resolved for this step's parity.  The group's TileGrid table holds tk's blocks, then tkn's.
cudaError_t batch_launch_tma_list(lbm_batch *b, const lbm_batch::Group &g, const std::vector<lbm_batch::Group::Span> &list,
                                  bool narrow, const char *tg0, int phase, cudaStream_t st)
{
    static thread_local lbm::TmaBatchArgs A;
    const bool f64 = g.prec == LBM_FP64;
    const int tr = narrow ? lbm::DdNarrowShape::TR : (f64 ? lbm::TmaShape<double>::TR : lbm::TmaShape<float>::TR);
    const size_t tgb = f64 ? sizeof(lbm::TileGrid<lbm::Coef<lbm::dd>>) : sizeof(lbm::TileGrid<lbm::Coef<float>>);
    for (size_t c0 = 0; c0 < list.size(); c0 += lbm::kTmaBatchGrids) {
        const int n = (int)std::min<size_t>(lbm::kTmaBatchGrids, list.size() - c0);
        int tiles = 0;
        for (int k = 0; k < n; k++) {
            const lbm_batch::Group::Span &sp = list[c0 + k];
            const lbm_ctx *c = b->ctxs[g.members[sp.k]];
            const int in = c->cur ^ phase;
            A.map[k] = narrow ? c->nmap[in] : c->tmap[in];
            A.out[k] = c->f[in ^ 1];
            A.err[k] = c->tma_err;
            A.first[k] = tiles;
            A.ntx[k] = (c->P.nx + lbm::kTmaTX - 1) / lbm::kTmaTX;
            A.y0[k] = sp.y0;
            tiles += A.ntx[k] * ((sp.rows + tr - 1) / tr);
        }
        A.first[n] = tiles;
        A.n = n;
        const char *tg = tg0 + c0 * tgb;
        const cudaError_t ce =
            f64 ? lbm::launch_step_dd_batch(A, (const lbm::TileGrid<lbm::Coef<lbm::dd>> *)tg, g.limiter, narrow, st)
                : lbm::launch_step_tma_batch(A, (const lbm::TileGrid<lbm::Coef<float>> *)tg, g.limiter, st);
        if (ce != cudaSuccess) return ce;
    }
    return cudaSuccess;
}

cudaError_t batch_launch_tma(lbm_batch *b, const lbm_batch::Group &g, int phase, cudaStream_t st)
{
    const char *tg = (const char *)g.tblock;
    cudaError_t ce = batch_launch_tma_list(b, g, g.tk, false, tg, phase, st);
    if (ce == cudaSuccess && !g.tkn.empty())
        ce = batch_launch_tma_list(b, g, g.tkn, true, tg + g.tk.size() * sizeof(lbm::TileGrid<lbm::Coef<lbm::dd>>),
                                   phase, st);
    return ce;
}

cudaError_t batch_launch_step(lbm_batch *b, int phase, cudaStream_t st)
{
    cudaError_t ce = cudaSuccess;
    for (auto &g : b->groups) {
        ce = lbm::launch_ghost_batch(g.dP, g.dG, (int)g.members.size(), g.max_ghost, g.prec, phase, st);
        if (ce != cudaSuccess) return ce;
    }
    const int nf = std::min<int>(lbm_batch::kForks, (int)b->solo.size());
    if (nf > 0) {
        ce = cudaEventRecord(b->ev_fork, st);
        for (int k = 0; k < nf && ce == cudaSuccess; k++) ce = cudaStreamWaitEvent(b->fork[k], b->ev_fork, 0);
        if (ce != cudaSuccess) return ce;
    }
    for (auto &g : b->groups) {
        ce = lbm::launch_step_batch(g.dP, g.dG, g.dT, g.ntiles, g.prec, g.limiter, g.nt,
                                    g.nt == lbm::kBatchThreadsFp64 ? 2 * b->ctas : b->ctas, phase, st);
        if (ce == cudaSuccess && (!g.tk.empty() || !g.tkn.empty())) ce = batch_launch_tma(b, g, phase, st);
        if (ce != cudaSuccess) return ce;
    }
    for (size_t j = 0; j < b->solo.size(); j++) {
        lbm_ctx *c = b->ctxs[b->solo[j]];
        ce = launch_fused_step(c, c->cur ^ phase, b->fork[j % lbm_batch::kForks]);
        if (ce != cudaSuccess) return ce;
    }
    for (int k = 0; k < nf && ce == cudaSuccess; k++) {
        ce = cudaEventRecord(b->ev_join[k], b->fork[k]);
        if (ce == cudaSuccess) ce = cudaStreamWaitEvent(st, b->ev_join[k], 0);
    }
    return ce;
}

// Inside a batch, a context whose kernel is the TMA-staged tile kernel (float32) or the
// double-float kernel (float64) has its tiles in the group's batched TMA-staged launch, which
// serves grids of every size; a context on the streaming or the double-buffered kernel runs its
// own kernel when it fills at least a quarter of a wave (512 cells per SM; forked streams let
// several such kernels share the SMs); the other grids share the packed plain tile kernel.
bool batch_tma(const lbm_ctx *c)
{
    return (c->prec == LBM_FP32_DEV && c->use_tma) || (c->prec == LBM_FP64 && (c->use_dd || c->use_ddn));
}

bool batch_solo(const lbm_ctx *c, int sms)
{
    return (c->use_stream || c->use_pipe) && (long long)c->P.nx * c->P.ny >= 512LL * sms;
}

}  // namespace

extern "C" {

int lbm_batch_create(lbm_ctx *const *ctxs, int n, lbm_batch **out)
{
    if (!out) return fail(nullptr, LBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!ctxs || n < 1) return fail(nullptr, LBM_ERR_ARG, "need at least one context");
    for (int i = 0; i < n; i++) {
        if (!ctxs[i]) return fail(nullptr, LBM_ERR_ARG, "NULL context in batch");
        if (ctxs[i]->device != ctxs[0]->device || ctxs[i]->stream != ctxs[0]->stream)
            return fail(nullptr, LBM_ERR_ARG, "batched contexts must share device and stream");
        for (int j = 0; j < i; j++)
            if (ctxs[j] == ctxs[i]) return fail(nullptr, LBM_ERR_ARG, "context listed twice");
    }
    lbm_batch *b = new (std::nothrow) lbm_batch;
    if (!b) return fail(nullptr, LBM_ERR_OOM, "host allocation failed");
    b->ctxs.assign(ctxs, ctxs + n);
    b->stream = ctxs[0]->stream;
    b->device = ctxs[0]->device;
    b->alloc = ctxs[0]->alloc;
    cudaError_t ce = cudaSetDevice(b->device);
    int sms = 0;
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    if (ce != cudaSuccess) { delete b; return cuda_fail(nullptr, ce, "device query"); }
    b->ctas = 4 * sms;
    // a float64 member on narrow double-float tiles whose grid takes 32 x 32 tiles steps on those
    // in the batch (the same bits: the two shapes run the same operations on every value; spread
    // over a batch, the larger tiles cost less per cell)
    std::vector<char> wide(n, 0), split(n, 0);
    for (int i = 0; i < n; i++) {
        lbm_ctx *c = ctxs[i];
        wide[i] = c->use_dd || (c->use_ddn && lbm::tma_supported(c->P, LBM_FP64) && make_tile_maps(c));
        // a last 32 x 32 tile row with at most 24 of the grid's rows: those rows on narrow tiles
        // (a narrow tile costs about 1.3x per cell, a part-filled row of 32 x 32 tiles 32 / rows)
        const int rem = c->P.ny % lbm::TmaShape<double>::TR;
        split[i] = wide[i] && rem > 0 && rem <= 24 && lbm::dd_narrow_supported(c->P) && make_narrow_maps(c);
    }
    cudaGetLastError();
    for (int i = 0; i < n; i++) {
        const lbm_ctx *c = ctxs[i];
        const bool tma = batch_tma(c);
        const bool own = !tma && batch_solo(c, sms);
        if (own) b->solo.push_back(i);
        lbm_batch::Group *g = nullptr;
        for (auto &gg : b->groups)
            if (gg.prec == c->prec && gg.limiter == c->P.limiter) g = &gg;
        if (!g) {
            b->groups.emplace_back();
            g = &b->groups.back();
            g->prec = c->prec;
            g->limiter = c->P.limiter;
        }
        g->members.push_back(i);
        g->own.push_back(own ? 1 : 0);
        g->tma.push_back(tma ? 1 : 0);
    }
    for (auto &g : b->groups) {
        // float64 groups too small to give every SM four 256-cell tiles take 64-cell tiles,
        // which spread their float64 work over more SMs
        if (g.prec == LBM_FP64) {
            long long cells = 0;
            for (size_t k = 0; k < g.members.size(); k++)
                if (!g.own[k] && !g.tma[k]) cells += (long long)b->ctxs[g.members[k]]->P.nx * b->ctxs[g.members[k]]->P.ny;
            g.nt = cells >= 4LL * lbm::kBatchThreads * sms ? lbm::kBatchThreads : lbm::kBatchThreadsFp64;
        }
        std::vector<int4> tiles;
        std::vector<lbm::Params> hp;
        std::vector<lbm::TileGrid<lbm::Coef<float>>> htf;
        std::vector<lbm::TileGrid<lbm::Coef<lbm::dd>>> htd, htdn;   // float64: 32 x 32 members, narrow ones
        const int tr = g.prec == LBM_FP64 ? lbm::TmaShape<double>::TR : lbm::TmaShape<float>::TR;
        for (size_t k = 0; k < g.members.size(); k++) {
            const lbm_ctx *c = b->ctxs[g.members[k]];
            hp.push_back(c->P);
            hp.back().wrap = 0;                      // the batched ghost fill writes every ghost cell
            g.hG.push_back(lbm::BatchGrid{{c->f[0], c->f[1]}, c->tma_err, c->cur, 0});
            g.max_ghost = std::max(g.max_ghost, 4 * (c->P.nx + c->P.ny));
            if (g.tma[k]) {
                const int i = g.members[k], ntx = (c->P.nx + lbm::kTmaTX - 1) / lbm::kTmaTX;
                if (g.prec == LBM_FP64) {
                    const lbm::TileGrid<lbm::Coef<lbm::dd>> blk{c->P.nx, c->P.ny, c->P.pitch, c->P.has_c9,
                                                                c->P.plane, 0, c->cdd};
                    const int nr = lbm::DdNarrowShape::TR;
                    const int wide_rows = !wide[i] ? 0 : (split[i] ? c->P.ny - c->P.ny % tr : c->P.ny);
                    if (wide_rows > 0) {
                        g.tk.push_back({(int)k, 0, wide_rows});
                        g.ntt += ntx * ((wide_rows + tr - 1) / tr);
                        htd.push_back(blk);
                    }
                    if (wide_rows < c->P.ny) {
                        g.tkn.push_back({(int)k, wide_rows, c->P.ny - wide_rows});
                        g.ntt += ntx * ((c->P.ny - wide_rows + nr - 1) / nr);
                        htdn.push_back(blk);
                    }
                    continue;
                }
                g.tk.push_back({(int)k, 0, c->P.ny});
                g.ntt += ntx * ((c->P.ny + tr - 1) / tr);
                htf.push_back(lbm::TileGrid<lbm::Coef<float>>{c->P.nx, c->P.ny, c->P.pitch, c->P.has_c9,
                                                              c->P.plane, 0, c->P.cf});
                continue;
            }
            if (g.own[k]) continue;                  // ghost cells only
            const int lt = lbm::plain_log_tx(c->P.nx);
            const int nt = g.nt;
            const int tw = 1 << lt, th = nt >> lt;
            for (int y = 0; y < c->P.ny; y += th)
                for (int x = 0; x < c->P.nx; x += tw) tiles.push_back(make_int4((int)k, x, y, lt));
        }
        g.ntiles = (int)tiles.size();
        // sections start on 256-byte boundaries (the tile list is read as int4)
        auto up = [](size_t v) { return (v + 255) / 256 * 256; };
        const size_t np = up(hp.size() * sizeof(lbm::Params)), ng = up(g.hG.size() * sizeof(lbm::BatchGrid));
        const size_t nt = tiles.size() * sizeof(int4);
        g.bytes = np + ng + nt;
        g.block = b->alloc.alloc(g.bytes, b->stream, b->alloc.user);
        if (!g.block) { cudaGetLastError(); lbm_batch_destroy(b); return fail(nullptr, LBM_ERR_OOM, "batch tables"); }
        g.dP = (lbm::Params *)g.block;
        g.dG = (lbm::BatchGrid *)((char *)g.block + np);
        g.dT = (int4 *)((char *)g.block + np + ng);
        ce = cudaMemcpyAsync(g.dP, hp.data(), hp.size() * sizeof(lbm::Params), cudaMemcpyHostToDevice, b->stream);
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(g.dG, g.hG.data(), g.hG.size() * sizeof(lbm::BatchGrid), cudaMemcpyHostToDevice,
                                 b->stream);
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(g.dT, tiles.data(), nt, cudaMemcpyHostToDevice, b->stream);
        htd.insert(htd.end(), htdn.begin(), htdn.end());   // table order: tk, then tkn
        if (ce == cudaSuccess && (!htd.empty() || !htf.empty())) {
            const void *src = htd.empty() ? (const void *)htf.data() : (const void *)htd.data();
            g.tbytes = htd.empty() ? htf.size() * sizeof(htf[0]) : htd.size() * sizeof(htd[0]);
            g.tblock = b->alloc.alloc(g.tbytes, b->stream, b->alloc.user);
            if (!g.tblock) { cudaGetLastError(); lbm_batch_destroy(b); return fail(nullptr, LBM_ERR_OOM, "batch tables"); }
            ce = cudaMemcpyAsync(g.tblock, src, g.tbytes, cudaMemcpyHostToDevice, b->stream);
        }
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(b->stream);
        if (ce != cudaSuccess) { lbm_batch_destroy(b); return cuda_fail(nullptr, ce, "batch tables"); }
    }
    ce = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
    for (int k = 0; k < lbm_batch::kForks && ce == cudaSuccess; k++) {
        ce = cudaStreamCreateWithFlags(&b->fork[k], cudaStreamNonBlocking);
        if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&b->ev_join[k], cudaEventDisableTiming);
    }
    if (ce != cudaSuccess) { lbm_batch_destroy(b); return cuda_fail(nullptr, ce, "capture stream"); }
    *out = b;
    return LBM_OK;
}

int lbm_batch_step(lbm_batch *b, int n)
{
    if (!b) return fail(nullptr, LBM_ERR_ARG, "batch is NULL");
    lbm_ctx *c0 = b->ctxs[0];
    if (n <= 0) return fail(c0, LBM_ERR_STATE, "n must be >= 1");
    for (lbm_ctx *c : b->ctxs)
        if (!c->initialized) return fail(c0, LBM_ERR_STATE, "a batched context was never initialised");
    cudaError_t ce = cudaSetDevice(b->device);
    if (ce == cudaSuccess) ce = batch_upload_cur(b);
    if (ce != cudaSuccess) return cuda_fail(c0, ce, "batch");
    if (b->exec2) {
        // the graph's own-kernel and batched TMA-staged launches name their buffers: recapture
        // if a context was stepped alone an odd number of times since the capture
        bool same = true;
        for (size_t k = 0; k < b->ctxs.size(); k++) same = same && b->ctxs[k]->cur == b->cap_cur[k];
        if (!same) {
            ce = cudaStreamSynchronize(b->stream);
            if (ce == cudaSuccess) ce = cudaGraphExecDestroy(b->exec2);
            b->exec2 = nullptr;
            if (ce != cudaSuccess) return cuda_fail(c0, ce, "batch graph");
        }
    }
    if (n >= 2 && !b->exec2) {
        b->cap_cur.clear();
        for (lbm_ctx *c : b->ctxs) b->cap_cur.push_back(c->cur);
        // capture two steps (both buffer parities) once; replays read the tables' current contents
        cudaGraph_t graph = nullptr;
        ce = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
        if (ce == cudaSuccess) {
            cudaError_t le = batch_launch_step(b, 0, b->cap);
            if (le == cudaSuccess) le = batch_launch_step(b, 1, b->cap);
            ce = cudaStreamEndCapture(b->cap, &graph);
            if (ce == cudaSuccess) ce = le;
        }
        if (ce == cudaSuccess) ce = cudaGraphInstantiate(&b->exec2, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (ce != cudaSuccess) { b->exec2 = nullptr; return cuda_fail(c0, ce, "batch graph"); }
    }
    for (int k = 0; k + 1 < n; k += 2) {
        ce = cudaGraphLaunch(b->exec2, b->stream);
        if (ce != cudaSuccess) return cuda_fail(c0, ce, "batch graph launch");
    }
    if (n & 1) {
        ce = batch_launch_step(b, 0, b->stream);
        if (ce != cudaSuccess) return cuda_fail(c0, ce, "batch step");
        for (lbm_ctx *c : b->ctxs) c->cur ^= 1;
    }
    for (lbm_ctx *c : b->ctxs) c->steps += n;
    return LBM_OK;
}

void lbm_batch_destroy(lbm_batch *b)
{
    if (!b) return;
    cudaSetDevice(b->device);
    cudaStreamSynchronize(b->stream);
    if (b->exec2) cudaGraphExecDestroy(b->exec2);
    if (b->cap) cudaStreamDestroy(b->cap);
    for (int k = 0; k < lbm_batch::kForks; k++) {
        if (b->fork[k]) cudaStreamDestroy(b->fork[k]);
        if (b->ev_join[k]) cudaEventDestroy(b->ev_join[k]);
    }
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    for (auto &g : b->groups) {
        if (g.block && b->alloc.free) b->alloc.free(g.block, g.bytes, b->stream, b->alloc.user);
        if (g.tblock && b->alloc.free) b->alloc.free(g.tblock, g.tbytes, b->stream, b->alloc.user);
    }
    delete b;
}

const char *lbm_last_error(const lbm_ctx *c) { return c ? c->err.c_str() : g_err.c_str(); }

void lbm_destroy(lbm_ctx *c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    drop_step_graphs(c);
    if (c->cap) cudaStreamDestroy(c->cap);
    for (cudaEvent_t e : c->prof_ev) cudaEventDestroy(e);
    if (c->alloc.free) {
        if (c->aux) c->alloc.free(c->aux, c->aux_bytes, c->stream, c->alloc.user);
        if (c->stage) c->alloc.free(c->stage, c->stage_elems * sizeof(double), c->stream, c->alloc.user);
        if (c->buf) c->alloc.free(c->buf, c->buf_bytes, c->stream, c->alloc.user);
    }
    delete c;
}

}  // extern "C"
