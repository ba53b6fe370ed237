// lbm_internal.h -- launchers shared between the host API and the kernel units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "lbm_dd.cuh"
#include "lbm_device.cuh"

namespace lbm {

// Tile of the fused step kernel: TX x TY cells, one thread per cell.
constexpr int kTX = 32;
constexpr int kTY = 8;
// Fixed grid of the first totals pass (the result is deterministic for a given size).
constexpr int kTotalsBlocks = 1024;   // partials buffer: at least one wave of totals blocks
constexpr int kTotalsThreads = 256;

// All launchers enqueue on `st` and return the launch status.
// `prec` is the storage precision (0 = float64 f, 1 = float32 deviation g).
// Initialisation of interior rows row0 .. row0+rows-1 from fields [rows][nx] (device or mapped host
// addresses of the first of those rows); a bad cell sets *bad.
cudaError_t launch_init(const Params &P, int prec, void *f, const double *rho, const double *u, const double *v,
                        const double *T, int row0, int rows, int *bad, cudaStream_t st);
// Ghost cells of every edge, or (y_only) of the y edges only: the ghost rows.
cudaError_t launch_ghost(const Params &P, int prec, void *f, cudaStream_t st, bool y_only = false);
// Plain fused step with tiles of 32 x ty cells (ty = 4, 8 or 16).
cudaError_t launch_step(const Params &P, int prec, const void *fin, void *fout, cudaStream_t st, int ty = kTY);
// log2 of the plain kernels' tile width for a grid nx columns wide (5 for nx >= 32, else the
// smallest power of two >= nx); the tile has (kTX * kTY) >> log rows.
int plain_log_tx(int nx);
// threads (= cells) per CTA and tile of the batched step kernel: float32 groups, float64 groups
constexpr int kBatchThreads = kTX * kTY;
constexpr int kBatchThreadsFp64 = 64;

// One grid of a batch: its two population buffers, which one holds the current step, and the
// flag its TMA-fed kernels raise when a copy wait runs out.
struct BatchGrid {
    void *buf[2];
    int *err;
    int cur;
    int pad;
};
// Batched ghost fill (grid index = blockIdx.y) and batched fused step over a tile list
// (int4 {grid, x0, y0, 0}); `phase` = 0 reads buf[cur], 1 reads buf[cur ^ 1].
cudaError_t launch_ghost_batch(const Params *Pall, const BatchGrid *G, int ngrids, int max_ghost, int prec,
                               int phase, cudaStream_t st);
cudaError_t launch_step_batch(const Params *Pall, const BatchGrid *G, const int4 *tiles, int ntiles, int prec,
                              int limiter, int nt, int ctas, int phase, cudaStream_t st);
cudaError_t launch_moments(const Params &P, int prec, const void *f, int row0, int rows,
                           double *rho, double *u, double *v, double *T, double *delta,
                           double *dstar, int *flag, cudaStream_t st);
cudaError_t launch_totals(const Params &P, int prec, const void *f, double *partial, double *out,
                          double scale, cudaStream_t st);
cudaError_t launch_pack(const Params &P, int prec, const void *f, int row0, int rows, double *out,
                        cudaStream_t st);
cudaError_t launch_unpack(const Params &P, int prec, void *f, int row0, int rows, const double *in,
                          cudaStream_t st);

// TMA-staged step kernel: tiles of kTmaTX columns by TmaShape<R>::TR rows,
// kTmaTX x TT threads, each thread owns KR consecutive rows of one column.
// float32: 4 warps and 32 x 16 tiles (four CTAs per SM, so four tile copies in
// flight); the staged flow velocity is (u_x, u_y) pairs and 1/rho is recomputed
// from the cell's own density.  float64: 8 warps and 32 x 32 tiles, u_x, u_y and
// 1/rho staged.
constexpr int kTmaTX = 32;
constexpr int kTmaTT = 8;
template <typename R>
struct TmaShape {
    static constexpr int TT = sizeof(R) == sizeof(float) ? 4 : 8;   // warps per CTA
    static constexpr int CTAS = sizeof(R) == sizeof(float) ? (TT == 4 ? 4 : (TT == 3 ? 5 : 7)) : 1;   // per SM
    static constexpr int KR = 4;                       // rows per thread
    static constexpr int TR = TT * KR;                 // tile rows
    static constexpr int HX = 2;                       // x halo (8-byte elements: 16-byte TMA origin)
    static constexpr int SW = kTmaTX + 2 * HX;         // staged row
    static constexpr int SH = TR + 4;                  // staged rows: y halo of 2
    static constexpr int PL = SW * SH;                 // staged plane (float32: plane of pairs, in pairs)
    static constexpr int UW = kTmaTX + 2, UH = TR + 2; // flow-velocity tile with its ring
    static constexpr size_t tile_bytes = sizeof(R) * NQ * PL;
    static constexpr size_t smem_bytes = tile_bytes + sizeof(R) * (sizeof(R) == sizeof(float) ? 2 : 3) * UW * UH;
};
bool tma_supported(const Params &P, int prec);
// Narrow tiles of the double-float float64 kernel (step_kernel 9): 4 warps, 32 x 4 tiles, one
// row per thread, two CTAs per SM, for grids of 4 to 31 rows (and 32 columns or more), where the
// 32 x 32 tiles do not fit.  The staged tile is that of TmaShape<double> with 8 rows.
struct DdNarrowShape {
    static constexpr int TT = 4;
    static constexpr int CTAS = 2;
    static constexpr int KR = 1;
    static constexpr int TR = TT * KR;
    static constexpr int HX = 2;
    static constexpr int SW = kTmaTX + 2 * HX;
    static constexpr int SH = TR + 4;
    static constexpr int PL = SW * SH;
    static constexpr int UW = kTmaTX + 2, UH = TR + 2;
    static constexpr size_t tile_bytes = sizeof(double) * NQ * PL;
    static constexpr size_t smem_bytes = tile_bytes + sizeof(double) * 3 * UW * UH;
};
bool dd_narrow_supported(const Params &P);
// Batched TMA-staged steps over the tiles of up to kTmaBatchGrids grids of a batch group, one
// CTA per tile of kTmaTX x TmaShape<R>::TR cells: grid k owns the launch's tiles first[k] ..
// first[k+1] - 1, row by row from row y0[k], ntx[k] to a row.  A CTA finds its grid and tile from blockIdx
// and this parameter block alone, so that its tile copy is issued before any load from global
// memory; the host resolves each grid's input map, output buffer and error flag for the
// launch's buffer parity.  float32 (the tile kernel) and float64 in double-float arithmetic.
constexpr int kTmaBatchGrids = 128;
struct TmaBatchArgs {
    CUtensorMap map[kTmaBatchGrids];   // grid k's input buffer (box of TmaShape<R>)
    void *out[kTmaBatchGrids];          // grid k's output buffer
    int *err[kTmaBatchGrids];           // grid k's copy-wait flag
    int first[kTmaBatchGrids + 1];      // first[n] = tiles of the launch
    int ntx[kTmaBatchGrids];            // tiles per row of grid k
    int y0[kTmaBatchGrids];             // first row of grid k's tiles in this launch
    int n;                              // grids of the launch
};
// Per-grid block of a batched launch (global memory, one per grid in launch order): the
// geometry and the coefficients that the tile kernels read (C = Coef<float> or Coef<dd>); each
// CTA copies its grid's block to shared memory while its tile copy is in flight.
template <typename C>
struct TileGrid {
    int nx, ny, pitch, has_c9;
    long long plane, pad;
    C cf;
};
cudaError_t launch_step_tma_batch(const TmaBatchArgs &A, const TileGrid<Coef<float>> *tg, int limiter,
                                  cudaStream_t st);
// narrow: tiles of DdNarrowShape (the grids' maps have its box), else of TmaShape<double>.
cudaError_t launch_step_dd_batch(const TmaBatchArgs &A, const TileGrid<Coef<dd>> *tg, int limiter, bool narrow,
                                 cudaStream_t st);
// Failure-path check of the bounded mbarrier waits (lbm_wait_selftest): *flag = 1 when the
// wait on a phase that nothing completes gave up at its limit; *ms = the kernel's duration.
cudaError_t wait_selftest(int *flag, float *ms);
cudaError_t tma_prepare();   // opt the kernels in to their dynamic shared memory (once per device)
// `tmap` points to the CUtensorMap of the input buffer fin (3-D: pitch x (ny+4) x 16).  Tiles at a
// periodic x edge take their x halo from the wrapped interior of fin, so on a grid periodic in x
// the kernel needs only the ghost rows (launch_ghost with y_only).
cudaError_t launch_step_tma(const Params &P, int prec, const void *tmap, const void *fin, void *fout, int *err,
                            cudaStream_t st);

// Persistent double-buffered TMA-staged kernel (float32): CTAs walk tiles of kTmaTX columns
// by TR rows round-robin with two tile buffers, so that the copy of the next tile overlaps
// the work on the current one; each thread owns KR rows of one column.
struct TmaPipeShape {
    static constexpr int KR = 2;
    static constexpr int TR = kTmaTT * KR;
    static constexpr int HX = 2;
    static constexpr int SW = kTmaTX + 2 * HX;
    static constexpr int SH = TR + 4;
    static constexpr int PL = SW * SH;                 // staged plane of pairs, in pairs
    static constexpr int UW = kTmaTX + 2, UH = TR + 2;
    static constexpr size_t buf_bytes = sizeof(float) * NQ * PL;
    static constexpr size_t smem_bytes = 2 * buf_bytes + sizeof(float) * 3 * UW * UH;
};
bool tma_pipe_supported(const Params &P);
cudaError_t tma_pipe_prepare();
// `tmap`: CUtensorMap of the input buffer with box SW x SH x 8 pair planes.
cudaError_t launch_step_tma_pipe(const Params &P, const void *tmap, void *fout, int *err, cudaStream_t st);

// Streaming step kernel: a CTA of WARPS warps owns a strip of W columns and walks down a
// share of its rows through a ring of SLOTS row slots; a slot holds all planes of one row
// as two copies of BW columns (half strip + 4 halo columns on each side).  Sizes in
// elements of R (float32: 8 planes of pairs = 16 floats per column).
template <typename R>
struct StreamShape {
    static constexpr int WARPS = 8;
    static constexpr int W = 32 * WARPS;               // strip width
    static constexpr int BW = W / 2 + 8;               // columns per copy
    static constexpr int HALF = NQ * BW;               // elements per copy
    static constexpr int ROW = 2 * HALF;               // elements per slot
    static constexpr int SLOTS = 6;
    static constexpr unsigned copy_bytes = HALF * sizeof(R);
    static constexpr size_t smem_bytes = sizeof(R) * (size_t)SLOTS * ROW;
};
bool stream_supported(const Params &P);
cudaError_t stream_prepare();
// `tmap` points to the CUtensorMap of the input buffer with box BW x 1 x 16.
cudaError_t launch_step_stream(const Params &P, int prec, const void *tmap, void *fout, int *err, cudaStream_t st);

// Float64-mode step in double-float arithmetic on the float32 pipe (step_kernel 8): the tiles
// and tensor maps of the float64 TMA-staged kernel; `coef` is the Coef<dd> of the context
// (coef_dd).  narrow (step_kernel 9): the tiles of DdNarrowShape, `tmap` with its box, no x
// wrap in the kernel.
void coef_dd(const Params &P, Coef<dd> *out);
cudaError_t dd_prepare();
cudaError_t launch_step_dd(const Params &P, const void *coef, const void *tmap, const void *fin, void *fout,
                           int *err, cudaStream_t st, bool narrow = false);

// Sustained float64 FMA rate of the current device in FLOP/s (FMA = 2).
cudaError_t measure_fp64_fma(double *flops);

}  // namespace lbm
