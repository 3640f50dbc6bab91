// mixed_epi.cu -- epilogue of the mixed-precision path, and the FP64 band of
// small l1 pairs.
//
// k_mixed_epilogue (binned output) and k_mixed_epilogue_dense: one thread per
// pair (parity, i, j) with l1 >= MX_L1_FP64 loops over the row sources
// (window x role).  The nine separable contractions of the pair come from
// the GEMM's double-float outputs with their power-of-two frames; the pair
// coefficients (lambda/eta, c0, c1, c2, e0, e1, C of plain_fp64.cu) are
// formed once per pair in extended double-float (FP32 pairs with an integer
// exponent) as products of per-l factors, and the spectra are combined in
// that form and converted to FP64 with integer operations (the binned
// variant then applies the (2l+1) / |bin| weights in FP64).
//
// k_mixed_band: pairs with l1 < MX_L1_FP64 outside the GEMM.  For them the
// polynomial expansion of the polarisation factor cancels by up to two
// orders of magnitude, which the limb contraction's 1e-10-level error would
// amplify; their l3 sums are short (2 l1 + 1 terms) and run in double-float
// (~1e-14 per contraction), the combination in FP64.
#include <cuda_runtime.h>

#include "dd.cuh"
#include "mixed.h"

namespace cpl {
namespace {

// Whether A variant v feeds one of the first np contractions.
__device__ __forceinline__ bool mx_alpha_used(int v, int np) {
    return v == 0 || (v == 1 && np > 2) || (v == 2 && np > 4) || (v == 3 && np > 6);
}

// Pair coefficients of the spectra in the order TE[0..2], EE[0..5],
// EE->BB[0..2] (the formulas of plain_fp64.cu): each is the product of a
// factor of l1 and a factor of l2 from the per-l table (mx_coef_host).
__device__ __forceinline__ void pair_coeffs(const void *coef, int l1, int l2, xdf (&qTE)[3], xdf (&qEE)[6],
                                            xdf (&qB)[3]) {
    const xdf *T1 = reinterpret_cast<const xdf *>(coef) + (size_t)l1 * MX_COEF_N;
    const xdf *T2 = reinterpret_cast<const xdf *>(coef) + (size_t)l2 * MX_COEF_N + MX_COEF_A;
    qTE[0] = xdf_mul(T1[0], T2[0]);                 //  r c0
    qTE[1] = xdf_neg(xdf_mul(T1[1], T2[1]));        // -r c1
    qTE[2] = xdf_neg(xdf_mul(T1[1], T2[2]));        // -r c2
    qEE[0] = xdf_mul(T1[2], T2[3]);                 //  r^2 c0^2
    qEE[1] = xdf_neg(xdf_mul(T1[3], T2[4]));        // -2 r^2 c0 c1
    qEE[2] = xdf_neg(xdf_mul(T1[3], T2[5]));        // -2 r^2 c0 c2
    qEE[3] = xdf_mul(T1[4], T2[6]);                 //  r^2 c1^2
    qEE[4] = xdf_mul(T1[5], T2[7]);                 //  2 r^2 c1 c2
    qEE[5] = xdf_mul(T1[4], T2[8]);                 //  r^2 c2^2
    qB[0] = xdf_mul(T1[6], T2[9]);                  //  C e0^2
    qB[1] = xdf_neg(xdf_mul(T1[7], T2[10]));        // -2 C e0 e1
    qB[2] = xdf_mul(T1[8], T2[11]);                 //  C e1^2
}

// The same coefficients without renormalising each product: mantissa
// (T1 T2 mantissas, |h| in [1, 4)) and the summed exponents.  The dense
// epilogue's frame sums take the exponent of every term anyway.
__device__ __forceinline__ xdf xdf_mul_raw(const xdf &a, const xdf &b) {
    const dfl m = df_mul(dfl{a.h, a.l}, dfl{b.h, b.l});
    return {m.h, m.l, a.e + b.e};
}
// T1: the MX_COEF_A factors of l1, T2: the MX_COEF_B factors of l2.
__device__ __forceinline__ void pair_coeffs_raw(const xdf *T1, const xdf *T2, xdf (&c)[12]) {
    c[0] = xdf_mul_raw(T1[0], T2[0]);              //  r c0
    c[1] = xdf_neg(xdf_mul_raw(T1[1], T2[1]));     // -r c1
    c[2] = xdf_neg(xdf_mul_raw(T1[1], T2[2]));     // -r c2
    c[3] = xdf_mul_raw(T1[2], T2[3]);              //  r^2 c0^2
    c[4] = xdf_neg(xdf_mul_raw(T1[3], T2[4]));     // -2 r^2 c0 c1
    c[5] = xdf_neg(xdf_mul_raw(T1[3], T2[5]));     // -2 r^2 c0 c2
    c[6] = xdf_mul_raw(T1[4], T2[6]);              //  r^2 c1^2
    c[7] = xdf_mul_raw(T1[5], T2[7]);              //  2 r^2 c1 c2
    c[8] = xdf_mul_raw(T1[4], T2[8]);              //  r^2 c2^2
    c[9] = xdf_mul_raw(T1[6], T2[9]);              //  C e0^2
    c[10] = xdf_neg(xdf_mul_raw(T1[7], T2[10]));   // -2 C e0 e1
    c[11] = xdf_mul_raw(T1[8], T2[11]);            //  C e1^2
}

// Binned-output epilogue.  One thread per pair (parity, i, j), i fastest
// across the block (the GEMM output is column-major, so the reads coalesce);
// each pair's band-power contributions are added to the output with FP64
// atomics.  Sources whose band limit L_w < |l2 - l1| contribute nothing to
// the pair and are skipped.
__global__ void __launch_bounds__(128) k_mixed_epilogue(const MxEpiArgs a) {
    const MxLayout &L = a.L;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    const int pi = blockIdx.z;
    const int l1 = j - i, l2 = i + j + pi;
    if (l1 < max(a.lmin, MX_L1_FP64) || l2 > a.lmax || l1 > l2) return;
    const int b1 = a.bin_of[l1], b2 = a.bin_of[l2];
    if (b1 < 0 || b2 < 0) return;

    xdf qTE[3], qEE[6], qB[3];
    pair_coeffs(a.coef, l1, l2, qTE, qEE, qB);
    const int b = i / L.BI, ii = i % L.BI, c = j / MX_BJ, cc = j % MX_BJ;
    const long long nrows = (long long)L.NRG * L.NB * MX_ROWS;
    const long long ncols = (long long)L.NC_B * MX_BJ;
    const unsigned bits[5] = {kTT, kTE, kEE, kEEBB, kEB};
    double f12 = (2.0 * l2 + 1.0) * a.bin_inv[b1];
    double f21 = (2.0 * l1 + 1.0) * a.bin_inv[b2];
    if (a.bin_lw) {   // D_l band powers: l1(l1+1) / (l2(l2+1)) and its mirror
        const double *iw = a.bin_lw + a.lmax + 1;
        f12 *= a.bin_lw[l1] * iw[l2];
        f21 *= a.bin_lw[l2] * iw[l1];
    }
    for (int s = 0; s < a.nsrc; ++s) {
        const int role = a.src_role[s];
        if (role == 0 || l2 - l1 > a.l3cap[s]) continue;
        const int w = a.src_win[s];
        const int rg = s / L.SRC, slot = s % L.SRC;
        const int tile = a.tile_of[(((long long)pi * L.NRG + rg) * L.NB + b) * L.NC + c];
        if (tile < 0) continue;
        xdf S[MX_NPROD];
        const int r = slot * L.BI + ii;
        const long long rowg = ((long long)rg * L.NB + b) * MX_ROWS + r;
        const bool pol = (role & (kEE | kEEBB | kEB)) != 0;
        const bool odd = (role & (kEEBB | kEB)) != 0;
        const int np = pol ? (odd ? 9 : 6) : (role & kTE) ? 3 : 1;
#pragma unroll
        for (int p = 0; p < MX_NPROD; ++p) {
            S[p] = {0.f, 0.f, 0};
            if (p >= np) continue;
            const float *src = a.inter + ((long long)tile * MX_NPROD + p) * 2 * (MX_ROWS * MX_BJ);
            const float hi = src[cc * MX_ROWS + r], lo = src[MX_ROWS * MX_BJ + cc * MX_ROWS + r];
            const int E = (int)a.emaxA[((long long)pi * MX_NA + mx_alpha(p)) * nrows + rowg] +
                          (int)a.emaxB[((long long)pi * MX_NBV + mx_beta(p)) * ncols + j] - 14;
            S[p] = xdf_make(df_quick(hi, lo), E);
        }
        xdf X[5];
        X[0] = S[0];
        X[1] = X[2] = X[3] = X[4] = xdf{0.f, 0.f, 0};
        if (role & kTE) {
            X[1] = xdf_mul(qTE[0], S[0]);
            X[1] = xdf_add(X[1], xdf_mul(qTE[1], S[1]));
            X[1] = xdf_add(X[1], xdf_mul(qTE[2], S[2]));
        }
        if (pol) {
#pragma unroll
            for (int p = 0; p < 6; ++p) X[2] = xdf_add(X[2], xdf_mul(qEE[p], S[p]));
            if (odd) {
                X[3] = xdf_mul(qB[0], S[6]);
                X[3] = xdf_add(X[3], xdf_mul(qB[1], S[7]));
                X[3] = xdf_add(X[3], xdf_mul(qB[2], S[8]));
                X[4] = xdf_add(X[2], xdf_neg(X[3]));
            }
        }
#pragma unroll
        for (int x = 0; x < 5; ++x) {
            if (!(role & bits[x]) || a.slot[x] < 0) continue;
            const double v = xdf_to_double(X[x]);
            if (v == 0.0) continue;
            double *base = a.out + ((size_t)w * a.nspec + a.slot[x]) * (size_t)a.n_bins * (size_t)a.n_bins;
            atomicAdd(base + (size_t)b1 * a.n_bins + b2, v * f12);
            if (l1 != l2) atomicAdd(base + (size_t)b2 * a.n_bins + b1, v * f21);
        }
    }
}


// Dense-output epilogue with coalesced writes.  One block covers an 8 x 16
// block of (i, j) in both parities: 256 pairs, one per thread, i fastest (the
// GEMM output is column-major, so 8 consecutive i are one 32-byte sector),
// whose rows of M (fixed l1, l2 = l1 + d) and mirrored rows (fixed l2,
// l1 = l2 - d) are runs of 16 consecutive elements.  Each thread forms its pair's 12 combination
// coefficients once in extended double-float and keeps them in registers;
// per row source it combines the contractions in one exponent frame per
// spectrum, converts each spectrum to FP64 with integer operations, scales it
// by (2 l2 + 1) and (2 l1 + 1) in FP64, and stages the two values in shared
// memory for row-wise writes.  Blocks that hold no valid pair return at once.
constexpr int EB_I = 8, EB_J = 16, EB_P = 2 * EB_I * EB_J, EB_T = EB_P;
constexpr int EB_NL1 = EB_I + EB_J - 1, EB_NL2 = EB_I + EB_J;   // l1 and l2 values of a block

struct Term {
    dfl m;   // mantissa
    int x;   // exponent of the unit
};

// sum_t m_t 2^(x_t) in one frame: returns (dd, exponent).  The frame E is the
// largest term's exponent; terms below 2^-90 of 2^E are dropped (even after
// the expansion's cancellation, at most 2^7, they lie far below FP64's
// rounding of the result), which keeps every shift k = x_t - E inside FP32's
// normal exponent range (|m_t| < 2^34 and normal), so one multiplication by
// 2^k scales each part.
template <int N>
__device__ __forceinline__ xdf frame_sum(const Term (&t)[N]) {
    int E = -1000000;
    int lg[N];
#pragma unroll
    for (int q = 0; q < N; ++q) {
        lg[q] = ilogbf_fast(fabsf(t[q].m.h));
        if (t[q].m.h != 0.0f) E = max(E, t[q].x + lg[q]);
    }
    if (E == -1000000) return {0.f, 0.f, 0};
    dfl s = {0.f, 0.f};
#pragma unroll
    for (int q = 0; q < N; ++q) {
        if (t[q].m.h == 0.0f || t[q].x + lg[q] - E < -90) continue;
        const float f = pow2f(t[q].x - E);
        s = df_add(s, dfl{t[q].m.h * f, t[q].m.l * f});
    }
    return {s.h, s.l, E};
}

__device__ __forceinline__ Term term(xdf c, dfl m, int e) { return {df_mul(dfl{c.h, c.l}, m), c.e + e}; }

// Shared memory of one block: the staged rows of M, and the pair
// coefficients (kept out of registers so that more blocks fit an SM).
struct EpiSmem {
    double stage[5][2][EB_P];
    float cfh[12][EB_T], cfl[12][EB_T];
    int cfe[12][EB_T];
};

__global__ void __launch_bounds__(EB_T, 4) k_mixed_epilogue_dense(const MxEpiArgs a) {
    extern __shared__ __align__(16) uint8_t epi_smem[];
    EpiSmem &sm = *reinterpret_cast<EpiSmem *>(epi_smem);
    const MxLayout &L = a.L;
    const int i0 = blockIdx.y * EB_I, j0 = blockIdx.x * EB_J;
    const int q = threadIdx.x;
    const int L1min = max(a.lmin, MX_L1_FP64);
    const int pi = q / (EB_I * EB_J), jj = (q / EB_I) % EB_J, ii = q % EB_I;
    const int i = i0 + ii, j = j0 + jj;
    const int l1 = j - i, l2 = i + j + pi;
    const bool valid = !(l1 < L1min || l2 > a.lmax || l1 > l2);
    // a block without a valid pair (l1 = j - i >= L1min and l2 = i + j + pi <= lmax
    // fail for all of its i, j) has nothing to write
    if (j0 + EB_J - 1 - i0 < L1min || i0 + j0 > a.lmax) return;

    // ---- the block's per-l factors, staged in shared memory (coalesced rows of
    // the table instead of 21 gathers per thread), in the stage buffer, which
    // the source loop only uses later: l1 = j - i spans EB_NL1 values, l2 =
    // i + j + pi EB_NL2
    {
        xdf *T1s = reinterpret_cast<xdf *>(&sm.stage[0][0][0]);
        xdf *T2s = T1s + EB_NL1 * MX_COEF_A;
        const xdf *tab = reinterpret_cast<const xdf *>(a.coef);
        const int l1lo = j0 - i0 - (EB_I - 1), l2lo = i0 + j0;
        for (int e = q; e < EB_NL1 * MX_COEF_A; e += EB_T) {
            const int l = l1lo + e / MX_COEF_A;
            if (l >= 0 && l <= a.lmax) T1s[e] = tab[(size_t)l * MX_COEF_N + e % MX_COEF_A];
        }
        for (int e = q; e < EB_NL2 * MX_COEF_B; e += EB_T) {
            const int l = l2lo + e / MX_COEF_B;
            if (l <= a.lmax) T2s[e] = tab[(size_t)l * MX_COEF_N + MX_COEF_A + e % MX_COEF_B];
        }
        __syncthreads();
        // ---- coefficients of this thread's pair (TE[0..2], EE[3..8], EE->BB[9..11])
        if (valid) {
            xdf c[12];
            pair_coeffs_raw(T1s + (l1 - l1lo) * MX_COEF_A, T2s + (l2 - l2lo) * MX_COEF_B, c);
#pragma unroll
            for (int x = 0; x < 12; ++x) {
                sm.cfh[x][q] = c[x].h;
                sm.cfl[x][q] = c[x].l;
                sm.cfe[x][q] = c[x].e;
            }
        }
        __syncthreads();   // the stage buffer is free again
    }
    const double f12 = 2.0 * l2 + 1.0, f21 = 2.0 * l1 + 1.0;   // M[l1][l2] and the mirror M[l2][l1]

    const long long nrows = (long long)L.NRG * L.NB * MX_ROWS;
    const long long ncols = (long long)L.NC_B * MX_BJ;
    const int n = a.lmax - a.lmin + 1;
    const int b32 = i0 / L.BI, c128 = j0 / MX_BJ;
    const unsigned bits[5] = {kTT, kTE, kEE, kEEBB, kEB};
    // this thread's share of the row writes, the same for every source and
    // spectrum: output offset and index into the staged [2][EB_P] values
    // (rows M[l1][l2 = l1 + d] and mirrored M[l2][l1 = l2 - d], d = 2 i0 .. 2 i0 + 2 EB_I - 1)
    constexpr int NROW = EB_I + EB_J, NWR = (2 * NROW * 2 * EB_I + EB_T - 1) / EB_T;
    long long woff[NWR];
    int widx[NWR];
#pragma unroll
    for (int k = 0; k < NWR; ++k) {
        widx[k] = -1;
        woff[k] = 0;
        const int e = q + k * EB_T;
        if (e >= 2 * NROW * 2 * EB_I) continue;
        const int mirror = e / (NROW * 2 * EB_I);
        const int rr = (e / (2 * EB_I)) % NROW, dl = e % (2 * EB_I);
        const int epi = dl & 1, eii = dl >> 1, ei = i0 + eii, d = 2 * ei + epi;
        const int el1 = mirror ? i0 + j0 + rr - d : j0 - i0 - (EB_I - 1) + rr;
        const int el2 = el1 + d;
        const int ejj = el1 + ei - j0;
        if (ejj < 0 || ejj >= EB_J) continue;
        if (el1 < L1min || el2 > a.lmax || el1 > el2) continue;
        if (mirror && el1 == el2) continue;
        const int pq = (epi * EB_J + ejj) * EB_I + eii;
        widx[k] = mirror * EB_P + pq;
        woff[k] = mirror ? (long long)(el2 - a.lmin) * n + (el1 - a.lmin) : (long long)(el1 - a.lmin) * n + (el2 - a.lmin);
    }
    // column frames of the six B variants: the same for every source
    int eBv[MX_NBV];
#pragma unroll
    for (int v = 0; v < MX_NBV; ++v)
        eBv[v] = valid ? (int)a.emaxB[((long long)pi * MX_NBV + v) * ncols + j] : 0;
    for (int s = 0; s < a.nsrc; ++s) {
        const int role = a.src_role[s];
        if (role == 0) continue;
        const int w = a.src_win[s];
        const int rg = s / L.SRC, slot = s % L.SRC;
        const bool pol = (role & (kEE | kEEBB | kEB)) != 0;
        const bool odd = (role & (kEEBB | kEB)) != 0;
        const int np = pol ? (odd ? 9 : 6) : (role & kTE) ? 3 : 1;
        if (valid) {
            const int tile = a.tile_of[(((long long)pi * L.NRG + rg) * L.NB + b32) * L.NC + c128];
            const int r = slot * L.BI + (i % L.BI), cc = j % MX_BJ;
            const long long rowg = ((long long)rg * L.NB + b32) * MX_ROWS + r;
            int eAv[MX_NA];
#pragma unroll
            for (int v = 0; v < MX_NA; ++v)
                eAv[v] = (tile >= 0 && mx_alpha_used(v, np)) ? (int)a.emaxA[((long long)pi * MX_NA + v) * nrows + rowg] : 0;
            const float *src0 = a.inter + (long long)(tile < 0 ? 0 : tile) * MX_NPROD * 2 * (MX_ROWS * MX_BJ) +
                                cc * MX_ROWS + r;
            // contraction p of this pair as (mantissa, exponent); zero where the tile is empty
            auto S = [&](int p) -> Term {
                if (tile < 0) return Term{dfl{0.f, 0.f}, 0};
                const float *sp = src0 + (long long)p * 2 * (MX_ROWS * MX_BJ);
                return Term{dfl{sp[0], sp[MX_ROWS * MX_BJ]}, eAv[mx_alpha(p)] + eBv[mx_beta(p)] - 14};
            };
            auto T = [&](int c, int p) -> Term {
                const Term t = S(p);
                return term(xdf{sm.cfh[c][q], sm.cfl[c][q], sm.cfe[c][q]}, t.m, t.x);
            };
            xdf X[5];
            {
                const Term t0 = S(0);
                X[0] = xdf{t0.m.h, t0.m.l, t0.x};
            }
            X[1] = X[2] = X[3] = X[4] = xdf{0.f, 0.f, 0};
            if (role & kTE) {
                const Term t[3] = {T(0, 0), T(1, 1), T(2, 2)};
                X[1] = frame_sum(t);
            }
            if (pol) {
                const Term t[6] = {T(3, 0), T(4, 1), T(5, 2), T(6, 3), T(7, 4), T(8, 5)};
                X[2] = frame_sum(t);
                if (odd) {
                    const Term u[3] = {T(9, 6), T(10, 7), T(11, 8)};
                    X[3] = frame_sum(u);
                    const Term v[2] = {Term{dfl{X[2].h, X[2].l}, X[2].e}, Term{dfl{-X[3].h, -X[3].l}, X[3].e}};
                    X[4] = frame_sum(v);
                }
            }
#pragma unroll
            for (int x = 0; x < 5; ++x) {
                if (!(role & bits[x])) continue;
                const double v = xdf_to_double(X[x]);
                sm.stage[x][0][q] = v * f12;
                sm.stage[x][1][q] = v * f21;
            }
        }
        __syncthreads();
        for (int x = 0; x < 5; ++x) {
            if (!(role & bits[x]) || a.slot[x] < 0) continue;
            double *base = a.out + ((size_t)w * a.nspec + a.slot[x]) * (size_t)n * (size_t)n;
            const double *stg = &sm.stage[x][0][0];
#pragma unroll
            for (int k = 0; k < NWR; ++k)
                if (widx[k] >= 0) base[woff[k]] = stg[widx[k]];
        }
        __syncthreads();
    }
}

__device__ __forceinline__ void put_out_d(const MxBandArgs &a, int w, int slot, int l1, int l2, double xi) {
    if (slot < 0) return;
    const double m12 = (2.0 * l2 + 1.0) * xi, m21 = (2.0 * l1 + 1.0) * xi;
    if (a.n_bins == 0) {
        const int n = a.lmax - a.lmin + 1;
        double *base = a.out + ((size_t)w * a.nspec + slot) * (size_t)n * (size_t)n;
        base[(size_t)(l1 - a.lmin) * n + (l2 - a.lmin)] = m12;
        if (l1 != l2) base[(size_t)(l2 - a.lmin) * n + (l1 - a.lmin)] = m21;
    } else {
        const int b1 = a.bin_of[l1], b2 = a.bin_of[l2];
        if (b1 < 0 || b2 < 0) return;
        double *base = a.out + ((size_t)w * a.nspec + slot) * (size_t)a.n_bins * (size_t)a.n_bins;
        double w12 = a.bin_inv[b1], w21 = a.bin_inv[b2];
        if (a.bin_lw) {
            const double *iw = a.bin_lw + a.lmax + 1;
            w12 *= a.bin_lw[l1] * iw[l2];
            w21 *= a.bin_lw[l2] * iw[l1];
        }
        if (m12 != 0.0) atomicAdd(base + (size_t)b1 * a.n_bins + b2, m12 * w12);
        if (l1 != l2 && m21 != 0.0) atomicAdd(base + (size_t)b2 * a.n_bins + b1, m21 * w21);
    }
}

// One thread per (pair with l1 < MX_L1_FP64, source): the separable sums of
// plain_fp64.cu over the pair's few l3 terms, in double-float relative to
// 2^E0, E0 the largest weight exponent over the pair's l3 range (the weights
// of such a short range differ by a few orders of magnitude at most, so the
// scaled terms stay inside FP32's range), then to FP64 for the combination.
// Only the contractions the source's spectra use are formed.
__device__ __forceinline__ dfl pair_df(const float *h, const float *l, int q) { return {h[q], l[q]}; }

__global__ void __launch_bounds__(128) k_mixed_band(const MxBandArgs a) {
    const int l2 = blockIdx.x * blockDim.x + threadIdx.x;
    const int l1 = a.lmin + blockIdx.y;
    const int s = blockIdx.z;
    if (l1 >= MX_L1_FP64 || l2 < l1 || l2 > a.lmax) return;
    const int d = l2 - l1, sm = l1 + l2, pi = d & 1;
    const int i = (d - pi) >> 1, j = (sm - pi) >> 1;
    const float *Ah = a.Ah + (size_t)s * a.a_stride, *Al = a.Al + (size_t)s * a.a_stride;
    const int *Ae = a.Ae + (size_t)s * a.a_stride;
    const int cap = a.l3cap[s];
    const int role = a.src_role[s], w = a.src_win[s];
    const bool pol = (role & (kTE | kEE | kEEBB | kEB)) != 0;
    const bool need_ee = (role & (kEE | kEB)) != 0, odd = (role & (kEEBB | kEB)) != 0;
    int E0 = -2147483647;
    for (int l3 = d; l3 <= min(sm, cap); ++l3)
        if (Ah[l3] != 0.f) E0 = max(E0, Ae[l3]);
    dfl S[MX_NPROD];
#pragma unroll
    for (int p = 0; p < MX_NPROD; ++p) S[p] = {0.f, 0.f};
    if (E0 != -2147483647) {
        // even sweep: l3 = 2k + pi, i <= k <= j
        for (int k = i; k <= j; ++k) {
            const int l3 = 2 * k + pi;
            if (l3 > cap) break;
            const int f = Ae[l3] - E0;
            const dfl mA = {scale2(Ah[l3], f), scale2(Al[l3], f)};
            const dfl a0 = df_mul(df_mul(mA, pair_df(a.gh, a.gl, i + k + pi)), pair_df(a.gh, a.gl, k - i));
            const dfl b0 = df_mul(pair_df(a.gh, a.gl, j - k), pair_df(a.hh, a.hl, j + k + pi));
            const dfl t = df_mul(a0, b0);
            S[0] = df_add(S[0], t);
            if (pol) {
                const dfl u = df_int_prod(2 * j + 2 * k + 2 * pi + 2, 2 * j - 2 * k + 1);
                const dfl v = df_int_prod(2 * k + 2 * i + 2 * pi + 1, 2 * k - 2 * i);
                const dfl tu = df_mul(t, u);
                S[1] = df_add(S[1], tu);
                S[2] = df_add(S[2], df_mul(tu, v));
                if (need_ee) {
                    const dfl tuu = df_mul(tu, u);
                    const dfl tuuv = df_mul(tuu, v);
                    S[3] = df_add(S[3], tuu);
                    S[4] = df_add(S[4], tuuv);
                    S[5] = df_add(S[5], df_mul(tuuv, v));
                }
            }
        }
        // odd sweep: l3 = 2k + 1 - pi, i + pi <= k <= j + pi - 1
        if (odd) {
            for (int k = i + pi; k <= j + pi - 1; ++k) {
                const int l3 = 2 * k + 1 - pi;
                if (l3 > cap) break;
                const int f = Ae[l3] - E0;
                const dfl mA = {scale2(Ah[l3], f), scale2(Al[l3], f)};
                const dfl v1 = df_int_prod(2 * i + 2 * k + 2, 2 * k + 1 - 2 * i - 2 * pi);
                const dfl u1 = df_int_prod(2 * j + 2 * k + 3, 2 * j - 2 * k + 2 * pi);
                const dfl up = df_int_prod(2 * j + 2 * k + 4, 2 * j - 2 * k + 2 * pi + 1);
                const dfl a1v = df_mul(df_mul(df_mul(mA, pair_df(a.gh, a.gl, i + k + 1)),
                                              pair_df(a.gh, a.gl, k - i - pi)), v1);
                const dfl b1u = df_mul(df_mul(pair_df(a.gh, a.gl, j - k + pi), pair_df(a.hh, a.hl, j + k + 1)), u1);
                const dfl t = df_mul(a1v, b1u);
                const dfl tu = df_mul(t, up);
                S[6] = df_add(S[6], t);
                S[7] = df_add(S[7], tu);
                S[8] = df_add(S[8], df_mul(tu, up));
            }
        }
    }
    double D[MX_NPROD];
#pragma unroll
    for (int p = 0; p < MX_NPROD; ++p)
        D[p] = E0 == -2147483647 ? 0.0 : ldexp((double)S[p].h + (double)S[p].l, E0);
    if (role & kTT) put_out_d(a, w, a.slot[0], l1, l2, D[0]);
    if (role & (kTE | kEE | kEEBB | kEB)) {
        const double L1 = l1, L2 = l2;
        const double eta2 = (L1 - 1.0) * (L1 + 2.0) * (L2 - 1.0) * L2;
        const double c1 = 1.0 / (L1 * (L1 + 1.0) * (L2 + 1.0));
        const double r2 = L1 * (L1 + 1.0) * (L2 + 1.0) * (L2 + 2.0) / eta2;
        const double c0 = 1.0 + 2.0 / L1, c2 = c1 / (2.0 * (L2 + 2.0));
        if (role & kTE) put_out_d(a, w, a.slot[1], l1, l2, sqrt(r2) * (c0 * D[0] - c1 * D[1] - c2 * D[2]));
        const double ee = r2 * (c0 * c0 * D[0] - 2.0 * c0 * c1 * D[1] - 2.0 * c0 * c2 * D[2] + c1 * c1 * D[3] +
                                2.0 * c1 * c2 * D[4] + c2 * c2 * D[5]);
        if (role & kEE) put_out_d(a, w, a.slot[2], l1, l2, ee);
        const double e0 = L1 + 2.0, e1 = 1.0 / (2.0 * (L2 + 2.0));
        const double bb = (L2 + 2.0) * c1 / eta2 * (e0 * e0 * D[6] - 2.0 * e0 * e1 * D[7] + e1 * e1 * D[8]);
        if (role & kEEBB) put_out_d(a, w, a.slot[3], l1, l2, bb);
        if (role & kEB) put_out_d(a, w, a.slot[4], l1, l2, ee - bb);
    }
}

}  // namespace

cudaError_t mx_launch_epilogue(const MxEpiArgs &a, cudaStream_t st) {
    const int NI = a.L.NBA * a.L.BI;   // rows beyond hold no nonzero value (band limit)
    if (a.n_bins > 0) {
        dim3 grid((NI + 127) / 128, a.lmax + 1, 2);
        k_mixed_epilogue<<<grid, 128, 0, st>>>(a);
        return cudaGetLastError();
    }
    dim3 grid((a.lmax + 1 + EB_J - 1) / EB_J, NI / EB_I);
    static std::atomic<unsigned long long> attr{0};
    const cudaError_t e = opt_in_smem(k_mixed_epilogue_dense, (int)sizeof(EpiSmem), attr);
    if (e != cudaSuccess) return e;
    k_mixed_epilogue_dense<<<grid, EB_T, sizeof(EpiSmem), st>>>(a);
    return cudaGetLastError();
}

cudaError_t mx_launch_band(const MxBandArgs &a, cudaStream_t st) {
    const int rows = MX_L1_FP64 - a.lmin;
    if (rows <= 0 || a.nsrc == 0) return cudaSuccess;
    dim3 grid((a.lmax + 1 + 127) / 128, rows, a.nsrc);
    k_mixed_band<<<grid, 128, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace cpl
