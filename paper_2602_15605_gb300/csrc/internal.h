// internal.h -- shared declarations of the coupling library (not installed).
#pragma once
#include <cuda_runtime.h>
#include <atomic>
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>
#include <map>
#include <tuple>

#include "../../include/coupling.h"

namespace cpl {

// ---------------------------------------------------------------- errors
void set_error(const std::string &msg);
cpl_status fail(cpl_status s, const std::string &msg);
#define CPL_CUDA_TRY(expr)                                                      \
    do {                                                                        \
        cudaError_t e_ = (expr);                                                \
        if (e_ != cudaSuccess)                                                  \
            return ::cpl::fail(CPL_ERR_CUDA, std::string(#expr " failed: ") +  \
                                                 cudaGetErrorString(e_));       \
    } while (0)

// Spectrum bits as in coupling.h.
constexpr unsigned kTT = 1u, kTE = 2u, kEE = 4u, kEEBB = 8u, kEB = 16u;
int spec_slot(unsigned spectra, unsigned bit);   // index of bit in the requested set, -1 if absent
int spec_count(unsigned spectra);
// D_l band-power weights: w[l] = l(l+1), w[lmax + 1 + l] = 1 / (l(l+1)) (0 at l = 0).
void bin_weights_dl(int lmax, std::vector<double> &w);

// ---------------------------------------------------------------- tables
// g(p) of Eq. gdef and h(p) = 1 / ((2p + 1) g(p)) (the 1/g and 1/(J+1) tables of
// Sec. 3.1 fused), each built by the recurrence in double-double and rounded once.
void build_tables_host(int pmax, std::vector<double> &g, std::vector<double> &h);

// ---------------------------------------------------------------- tiles
// One work item of the separable l3 contraction: a TILE_I x TILE_J block of
// (i, j) = ((d - pi)/2, (s - pi)/2) in parity class pi, d = l2 - l1, s = l1 + l2.
struct Tile {
    int16_t pi;      // parity class of d (and s)
    int16_t pad;
    int32_t i0, j0;  // first row / column of the block
    int32_t cost;    // run-time model of the block (tile_time with the full l3 range)
};
static_assert(sizeof(Tile) == 16, "Tile must be 16 bytes");

// Work item of a launch: a tile of one sweep (PlainJob) and one window.
struct WorkItem {
    int32_t job;     // index into PlainArgs::jobs
    int32_t win;
    int32_t tile;    // index into the sweep's tile list
    int32_t pad;
};

constexpr int TILE_I = 32;
constexpr int TILE_J = 32;

// All tiles of the valid region lmin <= l1 <= l2 <= lmax, ordered by cost
// (largest first).
void make_tiles(int lmax, int lmin, std::vector<Tile> &tiles);
// Run time of a tile in the plain kernels when l3 <= cap, in k steps of the
// block (its k range, the staging chunks and the epilogue).
double tile_time(const Tile &t, int cap);

// ---------------------------------------------------------------- plain FP64 kernels
// Kernel families by which GEMM products they run (see plain_fp64.cu).
enum PlainMode { MODE_TT = 0, MODE_TE = 1, MODE_POL = 2, MODE_ALL = 3 };

// One sweep: the window-role group of one request (the windows of one
// pointer and the spectra they feed).  A launch runs the items of any
// number of sweeps of the same kernel variant.
struct PlainJob {
    const double *A;        // [n_win][a_stride] weights (2 l3 + 1) W / (4 pi), zero past the band
    int a_stride;
    const int *l3cap;       // [n_win] last l3 with nonzero weight
    const Tile *tiles;      // tile list of the request
    int lmax, lmin;
    double *out;            // dense [n_win][nspec][n][n] or binned [n_win][nspec][nb][nb]
    int nspec;
    int slot[5];            // output slot of TT, TE, EE, EEBB, EB (-1 = not written)
    // binning (n_bins == 0: dense)
    int n_bins;
    const int *bin_of;      // [lmax + 1] bin index or -1
    const double *bin_inv;  // [n_bins] 1 / |b|
    const double *bin_lw;   // [2][lmax + 1] l(l+1) and its inverse (D_l band powers), NULL: flat
    // operand blocks of the tabled kernel (NULL: the kernel stages its own)
    const double *atab;     // this sweep's A blocks, NA x PT_BLK doubles each
    const long long *aoff;  // [n_win][2][nib] + 1: first A block of (window, parity, row block); counts by difference
    int nib;                // row blocks per parity
};

struct PlainArgs {
    const double *g;        // [pmax + 1]
    const double *h;        // [pmax + 1]
    const PlainJob *jobs;   // sweeps (device)
    const WorkItem *items;  // (sweep, window, tile) triples to run, heaviest first
    int n_items;
    int nge;                // even-sweep contractions of the variant (0, 1, 3 or 6)
    int odd;                // whether the odd sweep runs
    const float2 *gdf;      // [pmax + 1] g and h as FP32 pairs (double-float kernels only)
    const float2 *hdf;
    const double *lcoef;    // [l][PL_COEF_N] per-l factors of the pair coefficients (plain_coef_host)
    const double *btab;     // B blocks (btab_block order), NULL: the kernel stages its own operands
    int btab_njb;           // column blocks the B table covers
    int *err;               // device error word of the tabled kernel's bounded waits
};

cudaError_t launch_plain(const PlainArgs &a, cudaStream_t st);   // variant from a.nge / a.odd
cudaError_t launch_plain_df(const PlainArgs &a, cudaStream_t st);   // the same in double-float (plain_df.cu)
cudaError_t launch_df_tables(const double *g, const double *h, int n, float2 *gdf, float2 *hdf, cudaStream_t st);
// Which template variant launch_plain runs: even-sweep contractions (0, 1,
// 3 or 6) and whether the odd sweep runs.
void plain_variant(int mode, const int slot[5], int *nge, bool *odd);
// l3 terms of a tile per parity of L, with l3 <= cap.
void tile_terms_split(const Tile &t, int lmax, int lmin, int cap, double *even, double *odd, double *pairs);
cudaError_t launch_weights(const double *W, int w_len, int n_win, const int *l3cap,
                           double *A, int a_stride, cudaStream_t st);
// Operand blocks of the tabled plain FP64 kernel: the window-independent B
// blocks of column blocks [0, njb), and one sweep's A blocks (nae even rows,
// odd: the odd row) for n_win windows from their weights A.
cudaError_t launch_btab(const double *g, const double *h, int njb, double *B, cudaStream_t st);
// Per-l factors of the FP64 epilogue's pair coefficients for l < n (zero for
// l < 2): lambda/eta = rho(l1) sigma(l2), c0(l1), c1 = alpha(l1) beta(l2),
// c2 = alpha(l1) beta'(l2), e1(l2), C = kappa(l1) mu(l2).  Layout per l:
// rho, rho^2, c0, alpha, kappa, sigma, sigma^2, beta, beta', e1, mu.
constexpr int PL_COEF_N = 11;
void plain_coef_host(int n, std::vector<double> &out);
cudaError_t launch_atab(const double *A, int a_stride, const int *l3cap, const double *g, const long long *aoff,
                        int n_win, int nib, int max_count, int nae, int odd, double *At, cudaStream_t st);
// (j1 j2 j3; 0 -1 1) rows for device arrays j2, j3 from five square-root
// tables of g and h (tab: 5 np1 FP32 pairs) held as double-float (threej.cu)
cudaError_t launch_sqrt_tables(const double *g, const double *h, int np1, float2 *tab, cudaStream_t st);
cudaError_t launch_threej_consts(const int *j2, const int *j3, int n, float4 *cst, cudaStream_t st);
cudaError_t launch_threej_m11(const float2 *tab, int np1, const int *j2, const int *j3, int n, const float4 *cst,
                              double *out, long long stride, cudaStream_t st);

// Mode decoupling (decouple.cu): one CTA per n x n system of Eq. pseudo_cl.
// kind 0: K = M[slot1], rhs = pcl[field1], out[field1] = x;
// kind 1: K = M[slot1] + M[slot2], rhs = pcl[field1] + pcl[field2], x/2 added to out[field1] and out[field2];
// kind 2: the same with "-", x/2 added to out[field1] and -x/2 to out[field2].
struct DecoupleArgs {
    const double *M;        // [n_windows][nspec][n][n]
    const double *pcl;      // [n_windows][n_rhs][n_fields][n]
    double *out;            // layout of pcl
    int *info;              // [n_sys] or NULL
    int n, ld, n_rhs, n_fields, nspec, sys_per_window;
    long long n_sys;
    int kind[5], slot1[5], slot2[5], field1[5], field2[5];
    int refine;             // FP32 LU + FP64 iterative refinement first (FP64 LU on failure)
    int l_in_ws;            // refinement: FP32 factors in the workspace slice instead of shared memory
    int direct_in_ws;       // FP64 LU: augmented matrix in the workspace slice instead of shared memory
    int df_inc;             // refinement: residuals after the first as double-float updates (FP32 pairs of K
                            // and the updates' rounding errors after the factors)
    double *ws;             // global workspace, ws_stride doubles per CTA (NULL when unused)
    size_t ws_stride;
};

// Opts kernel fn into `bytes` of dynamic shared memory on the current
// device.  The attribute belongs to the function on one device, so it is set
// once per device (bit d of `done`; devices beyond 63 set it on every call).
template <class F>
cudaError_t opt_in_smem(F *fn, int bytes, std::atomic<unsigned long long> &done) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
    if (bit && (done.load(std::memory_order_relaxed) & bit)) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_relaxed);
    return e;
}

#ifdef __CUDACC__
#define CPL_HD __host__ __device__
#else
#define CPL_HD
#endif
// Shared-memory carve of the refinement path (byte offsets).  The FP32
// factors hold the system padded to np = 32 ceil(n / 32) rows and columns
// (identity in the padding) with row stride ir_ldf(n) floats; they come
// first when they are in shared memory.
CPL_HD inline int ir_np(int n) { return (n + 31) & ~31; }

// Operand blocks of the tabled plain FP64 kernel: PT_BLK = 16 k x 32 (i or
// j) doubles per operand row.  B blocks hold the six j-side rows of column
// block jb, parity pi and k chunk c <= 2 jb + 1, ordered by (jb, pi, c), so
// the table for a smaller l_max is a prefix of a larger one.
constexpr int PT_KC = 16;    // k per chunk
constexpr int PT_BLK = 512;
constexpr int PT_BROWS = 6;
CPL_HD inline long long btab_block(int jb, int pi, int c) {
    return 2LL * jb * (jb + 1) + (long long)pi * (2 * jb + 2) + c;
}
// Error codes of the tabled kernel (device error word)
constexpr int PT_ERR_RANGE = 0x1001;   // a tile's chunks are not covered by its tables
constexpr int PT_ERR_WAIT = 0x1002;    // a bulk copy did not complete within the bounded wait
CPL_HD inline int ir_ldf(int n) { return ir_np(n) + 4; }
struct IrLayout {
    size_t L, perm, dinv, x, r, xn, rn, y, z, e, ye, part, total;
};
CPL_HD inline size_t ir_align(size_t b) { return (b + 15) & ~(size_t)15; }
CPL_HD inline IrLayout ir_layout(int n, int R, bool l_in_smem) {
    IrLayout s;
    size_t o = 0;
    const size_t np = (size_t)ir_np(n);
    s.L = o;
    if (l_in_smem) o += ir_align(sizeof(float) * np * (size_t)ir_ldf(n));
    s.perm = o; o += ir_align(sizeof(int) * np);
    s.dinv = o; o += ir_align(sizeof(float) * np);
    s.x = o;    o += ir_align(sizeof(double) * (size_t)R * n);
    s.r = o;    o += ir_align(sizeof(double) * (size_t)R * n);
    s.xn = o;   o += ir_align(sizeof(double) * 2 * (size_t)R);
    s.rn = o;   o += ir_align(sizeof(double) * 3 * (size_t)R);        // residual maxima, 3 buffers
    s.y = o;    o += ir_align(sizeof(float) * (size_t)R * np);        // the correction in FP32
    s.z = o;    o += ir_align(14 * np);                               // zero rows of y (FP32), the update errors (BF16), x (FP64)
    s.ye = o;   o += ir_align(sizeof(int) * (size_t)R);
    // one region for two uses that never meet: the slices of a one-column
    // residual (one right-hand side), and the BF16 rounding errors [R][np] of
    // the updates x received (residual updates, from 8 right-hand sides)
    s.part = s.e = o;
    o += ir_align(2 * (size_t)R * np > sizeof(double) * 512 ? 2 * (size_t)R * np : sizeof(double) * 512);
    s.total = o;
    return s;
}
constexpr int IR_NMAX = 512;   // largest n of the refined solver (16 column chunks of 32)
int decouple_smem_limit();

// Approximate covariance (cov.cu).  One combine launch adds the terms of one
// kernel build (the same window and band limit) into the dense covariance.
constexpr int COV_TERMS_PER_LAUNCH = 16;
struct CovCombineArgs {
    const double *M;        // [nspec][n][n] dense kernels of the group's build (M = (2 l2 + 1) Xi)
    int n, lmin, n_terms;
    int slot[COV_TERMS_PER_LAUNCH];            // spectrum slot of each term in M
    const double *A[COV_TERMS_PER_LAUNCH];     // [lmax + 1], indexed by l
    const double *B[COV_TERMS_PER_LAUNCH];
    double *out;            // dense [n][n]
    int accumulate;         // add to out (else overwrite)
};
struct CovBinArgs {
    const double *cov;      // dense [n][n]
    int n, lmin, nb;
    const int *edges;       // device [nb + 1]
    double *out;            // [nb][nb]
};
cudaError_t launch_cov_combine(const CovCombineArgs &a, cudaStream_t st);
cudaError_t launch_cov_bin(const CovBinArgs &a, cudaStream_t st);
cudaError_t launch_decouple(const DecoupleArgs &a, int grid, size_t smem, cudaStream_t st);
cudaError_t decouple_blocks_per_sm(size_t smem, int *n);

}  // namespace cpl
