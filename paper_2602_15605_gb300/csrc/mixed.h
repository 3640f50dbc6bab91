// mixed.h -- the batched mixed-precision path (tcgen05 tensor cores).
//
// The separable contractions S(x, y)[i, j] = sum_k x[i,k] y[j,k] of the plain
// path (see plain_fp64.cu) are run as GEMMs on the tensor cores with operands
// split into BF16 fixed-point limbs:
//
//   x[r, k] ~= 2^(E_r - 7) sum_{t < S} X_t[r, k],   X_t = x_t 2^(-8t),  x_t in [-128, 128] integer
//
// with one power-of-two scale E_r per operand row and 256-wide block of k
// (a "scale block").  Each limb is exact in BF16, every limb product is exact
// in FP32 (|x_t y_u| <= 2^14), and the sums of the products of order
// t + u = 0, 1 and 2 over a scale block are integers in their units below
// 256 * 2^14, 2 * 256 * 2^14 and 3 * 256 * 2^14 < 2^24, so the FP32
// tensor-core accumulators hold them exactly; the orders t + u >= 3 (up to
// S - 1) go to a fourth accumulator, about 2^-24 of the total.  After each scale block the four
// accumulators are drained from TMEM, scaled by
// 2^(E_r + E_c) and added in double-float (a pair of FP32 values) per
// element; FP64 is kept for the lookup tables, the weights and the final
// values.
#pragma once
#include <cstdint>

#include "internal.h"

namespace cpl {

constexpr int MX_ROWS = 128;        // GEMM tile rows: SRC sources x BI i-values (MxLayout)
constexpr int MX_BJ = 128;          // j per column block (GEMM N)
constexpr int MX_SB = 256;          // k per scale block (drain period; the exactness bound above)
// k per tile image / pipeline stage: 32 for up to 5 limbs, 16 for 6 limbs
// (so that the stages of 2 x S images still fit in shared memory)
__host__ __device__ constexpr int mx_kb(int S) { return S >= 6 ? 16 : 32; }
__host__ __device__ constexpr int mx_img_bytes(int S) { return MX_ROWS * mx_kb(S) * 2; }
__host__ __device__ constexpr int mx_stages(int S) { return S >= 6 ? 3 : 2; }
constexpr int MX_NPROD = 9;         // separable contractions
constexpr int MX_L1_FP64 = 32;      // pairs with l1 below this are evaluated in FP64

// A-side operand variants (functions of (i, k)) and B-side variants (of (j, k)).
// Even sweep: a0, a0 v, a0 v^2 | b0, b0 u, b0 u^2.  Odd sweep: a1 v | b1 u, b1 u u', b1 u u'^2.
constexpr int MX_NA = 4;
constexpr int MX_NBV = 6;
__host__ __device__ constexpr int mx_alpha(int p) { return p < 6 ? (p == 0 || p == 1 || p == 3 ? 0 : p == 2 || p == 4 ? 1 : 2) : 3; }
__host__ __device__ constexpr int mx_beta(int p) { return p < 6 ? (p == 0 ? 0 : p <= 2 ? 1 : 2) : p - 3; }

struct MxLayout {
    int S;          // limbs per operand
    int KB;         // k per tile image (mx_kb(S))
    int IMG;        // bytes per tile image
    int fA;         // k blocks per i block (BI / KB)
    int gB;         // k blocks per 128-column j block (128 / KB)
    int lmax, lmin;
    int NB;         // row blocks (BI i) per parity
    int NC;         // column blocks (128 j) of this request
    int NKB;        // k blocks (KB k) of this request
    int NBA;        // row blocks that can hold nonzero A values (i <= l3 cap / 2)
    int NKBA;       // k blocks stored per A row (k <= l3 cap / 2)
    int NSB;        // scale blocks of this request
    int SRC;        // row sources (window x role) per row group: 1, 2 or 4
    int BI;         // i per row block: 128 / SRC
    int NRG;        // row groups of SRC sources
    long long a_rg_bytes;   // bytes of one (pi, alpha, rg) slab of A images
    // B cache geometry (independent of the request except through its size)
    int NC_B;       // column blocks the B cache holds
    int NSB_B;      // scale-block stride of the B exponent arrays
    long long b_var_bytes;  // bytes of one (pi, beta) slab of B images
};

// Offsets (bytes) of one tile image.  Row block b < NBA stores k blocks
// kb = fA b .. NKBA - 1; column block c stores kb = 0 .. gB (c + 1) - 1.
// (With band-limited windows, A rows and k beyond the largest l3 cap are
// zero and are neither stored nor read.)
__host__ __device__ inline long long mx_a_off(const MxLayout &L, int pi, int alpha, int rg, int b, int kb, int t) {
    const long long blk = (long long)b * L.NKBA - (long long)L.fA * b * (b - 1) / 2 + (kb - (long long)L.fA * b);
    return ((long long)(pi * MX_NA + alpha) * L.NRG + rg) * L.a_rg_bytes + (blk * L.S + t) * L.IMG;
}
__host__ __device__ inline long long mx_b_off(const MxLayout &L, int pi, int beta, int c, int kb, int t) {
    const long long blk = (long long)L.gB * c * (c + 1) / 2 + kb;
    return (long long)(pi * MX_NBV + beta) * L.b_var_bytes + (blk * L.S + t) * L.IMG;
}
// Byte offset of element (row r, k within the block) in a 128 x KB tile image:
// K-major core matrices of 8 rows x 16 bytes, K-adjacent cores 128 B apart
// (LBO), 8-row groups KB * 16 B apart (SBO), no swizzle.
__host__ __device__ inline int mx_img_off(int r, int kk, int KB) {
    return (r >> 3) * (KB * 16) + (kk >> 3) * 128 + (r & 7) * 16 + (kk & 7) * 2;
}

struct MxItem {
    int16_t pi, p;
    int16_t kb_lo, kb_hi;
    int32_t tile;      // index into the job's intermediate buffer
    int16_t rg, b;
    int16_t c, job;
};
static_assert(sizeof(MxItem) == 20, "MxItem layout");

// Per-request data of one GEMM launch (a launch may serve a batch of requests).
struct MxJob {
    MxLayout L;
    const uint8_t *Aimg;
    const int16_t *eA, *emaxA;     // [pi][alpha][row_global][NSB], [pi][alpha][row_global]
    float *inter;                  // [tile][9][2 planes (hi, lo)][128 cols][128 rows], column-major
};

struct MxGemmArgs {
    const MxJob *jobs;
    const uint8_t *Bimg;           // shared, window-independent B images (one cache for all jobs)
    const int16_t *eB, *emaxB;     // [pi][beta][j][NSB_B], [pi][beta][j]
    const MxItem *items;           // in ticket order (see mixed_host.cu)
    int n_items;
    int *ticket;                   // next item to take; zero before the launch
    int *err;                      // device error word (bounded waits)
};

struct MxPrepAArgs {
    const float *Ah, *Al;          // weights as double-float mantissas [nsrc][a_stride]
    const int *Ae;                 // and their exponents
    int a_stride;
    const float *gh, *gl;          // g table as double-float
    const int *l3cap;              // [nsrc] last l3 with nonzero weight
    int nsrc;
    int alpha_mask;                // which A variants the request uses (bit alpha)
    const int *src_role;           // [nsrc] role bits per source: a row group builds only the
                                   // variants its sources' contractions read
    uint8_t *Aimg;
    int16_t *eA, *emaxA;
    MxLayout L;
};

struct MxPrepBArgs {
    const float *gh, *gl, *hh, *hl;
    uint8_t *Bimg;
    int16_t *eB, *emaxB;
    int c_lo;                      // first column block to build (the cache grows)
    MxLayout L;
};

struct MxEpiArgs {
    const float *inter;
    const int32_t *tile_of;        // [pi][NRG][NB][NC] -> tile index or -1
    const int16_t *emaxA, *emaxB;
    const int *src_win, *src_role; // per source: window index and role bits (CPL_* spectra it feeds)
    const int *l3cap;              // per source: last l3 with a nonzero weight
    int nsrc;
    int lmax, lmin;
    double *out;
    int nspec;
    int slot[5];
    int n_bins;
    const int *bin_of;
    const double *bin_inv;
    const double *bin_lw;          // [2][lmax + 1] l(l+1) and its inverse (D_l band powers), NULL: flat
    const void *coef;              // [l][MX_COEF_N] per-l factors of the pair coefficients: {float h, l; int e}
    MxLayout L;
};

// Per-l factors of the pair coefficients (lambda/eta, c0, c1, c2, C, e0, e1 of
// plain_fp64.cu are products of a function of l1 and a function of l2):
// MX_COEF_A factors of l1, then MX_COEF_B factors of l2.
constexpr int MX_COEF_A = 9, MX_COEF_B = 12, MX_COEF_N = MX_COEF_A + MX_COEF_B;
// Host build of the factors for l < n into out[n * MX_COEF_N * 3] (h, l as
// float bits, e), from FP64 (53 bits; the extended double-float holds 48).
void mx_coef_host(int n, std::vector<uint32_t> &out);

struct MxBandArgs {   // double-float evaluation of the pairs with l1 < MX_L1_FP64
    const float *gh, *gl, *hh, *hl;   // g and h as FP32 pairs
    const float *Ah, *Al;          // [nsrc][a_stride] weights A = (Ah + Al) 2^Ae
    const int *Ae;
    int a_stride;
    const int *l3cap;
    const int *src_win, *src_role;
    int nsrc;
    int lmax, lmin;
    double *out;
    int nspec;
    int slot[5];
    int n_bins;
    const int *bin_of;
    const double *bin_inv;
    const double *bin_lw;          // [2][lmax + 1] l(l+1) and its inverse (D_l band powers), NULL: flat
};

cudaError_t mx_launch_tables_dd(const double *g, const double *h, int n, float *gh, float *gl, float *hh,
                                float *hl, cudaStream_t st);
cudaError_t mx_launch_weights_dd(const double *A, int n_src, int a_stride, float *Ah, float *Al, int *Ae,
                                 cudaStream_t st);
cudaError_t mx_launch_prep_a(const MxPrepAArgs &a, cudaStream_t st);
cudaError_t mx_launch_prep_b(const MxPrepBArgs &a, int c_hi, cudaStream_t st);
cudaError_t mx_launch_gemm(const MxGemmArgs &a, int S, int grid, cudaStream_t st);
cudaError_t mx_launch_epilogue(const MxEpiArgs &a, cudaStream_t st);
cudaError_t mx_launch_band(const MxBandArgs &a, cudaStream_t st);
size_t mx_gemm_smem_bytes(int S);
cudaError_t mx_gemm_prepare(int S);   // shared-memory attribute; call before launching (not under capture)

}  // namespace cpl
