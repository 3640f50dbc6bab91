// plain_fp64.cu -- FP64 coupling kernels (the plain path).
//
// The l3 sums of App. A are evaluated as separable contractions.  With
// d = l2 - l1 >= 0, s = l1 + l2 and the parity class pi = d mod 2, write
// d = 2i + pi, s = 2j + pi (so l1 = j - i, l2 = i + j + pi).
//
// Even sweep (L = l1 + l2 + l3 even, l3 = 2k + pi, i <= k <= j).  The
// halved triangle variables of Eq. trianglecombos are p1 = i + k + pi,
// p2 = k - i, p3 = j - k, p = j + k + pi, so Eq. 000_sq_main splits into a
// factor of (i, k) and a factor of (j, k):
//     (2 l3 + 1) W_l3 / (4 pi) X^2 = a0[i,k] b0[j,k],
//     a0 = A(l3) g(i + k + pi) g(k - i),   b0 = g(j - k) h(j + k + pi),
// with A(l) = (2l + 1) W_l / (4 pi) and h(p) = 1 / ((2p + 1) g(p)).  The
// (0,-2,2) symbol of Eq. 022_linear, once the (0,-1,1) symbols of App. B
// are reduced with Eq. joneevensimp, is X (lambda/eta) P with
//     P = c0 - c1 u - c2 u v,   c0 = 1 + 2/l1,
//     c1 = 1 / (l1 (l1+1) (l2+1)),   c2 = c1 / (2 (l2 + 2)),
//     u = (L + 2)(s - l3 + 1) = (2j + 2k + 2pi + 2)(2j - 2k + 1)   [a function of (j, k)]
//     v = (l3 + d + 1)(l3 - d) = (2k + 2i + 2pi + 1)(2k - 2i)     [a function of (i, k)]
// (lambda, eta of Sec. 3.2 with j1 = l3, j2 = l1, j3 = l2).  Hence
//     Xi_TT = S(a0, b0)
//     Xi_TE = (lambda/eta) [c0 S(a0,b0) - c1 S(a0,b0 u) - c2 S(a0 v,b0 u)]
//     Xi_EE = (lambda/eta)^2 [c0^2 S(a0,b0) - 2c0c1 S(a0,b0u) - 2c0c2 S(a0v,b0u)
//                             + c1^2 S(a0,b0u^2) + 2c1c2 S(a0v,b0u^2) + c2^2 S(a0v^2,b0u^2)]
// where S(x, y)[i, j] = sum_k x[i,k] y[j,k].
//
// Odd sweep (L odd, l3 = 2k + 1 - pi, i + pi <= k <= j + pi - 1).  Combining
// Eqs. joneodd and joneevenshifted with Eq. 022_rearranged and the identity of
// Eq. joneevensimp gives
//     (l1 l2 l3; -2 2 0)^2 = C (u v) (e0 - e1 u')^2 Z^2,
//     Z = (l3 l1 l2+1; 0 0 0),  e0 = l1 + 2,  e1 = 1 / (2 (l2 + 2)),
//     C = (l2 + 2) / (eta^2 l1 (l1 + 1) (l2 + 1)),  u' = (L + 3)(s - l3 + 2),
// and Z^2 again splits:  (2 l3 + 1) W / (4 pi) Z^2 = a1[i,k] b1[j,k],
//     a1 = A(l3) g(i + k + 1) g(k - i - pi),   b1 = g(j - k + pi) h(j + k + 1).
// So Xi_EEBB = C [e0^2 S(a1 v, b1 u) - 2 e0 e1 S(a1 v, b1 u u') + e1^2 S(a1 v, b1 u u'^2)].
//
// Each CTA owns a TILE_I x TILE_J block of (i, j) in one parity class and
// one window, stages the operand rows of an l3 chunk in shared memory
// (built from the g / h tables, Sec. 3.1), and runs the contractions as
// register-tiled FP64 FMAs: 1 FMA per l3 term for TT, 6 per even term for
// TT+TE+EE, 3 per odd term for EE->BB.  The FP64 pipe bounds this path.
#include <cuda_runtime.h>

#include <cmath>

#include "internal.h"
#include "mbar.cuh"

namespace cpl {
namespace {

constexpr int KC = 16;          // l3 chunk (in k units) staged per step
constexpr int NT = 256;         // threads per CTA (16 x 16, each 2 x 2 outputs)

template <int NGE, bool ODD>
struct Shape {
    static constexpr int NAE = NGE == 0 ? 0 : NGE == 1 ? 1 : NGE == 3 ? 2 : 3;  // a0, a0 v, a0 v^2
    static constexpr int NBE = NAE;                                          // b0, b0 u, b0 u^2
    static constexpr int NAO = ODD ? 1 : 0;                                  // a1 v
    static constexpr int NBO = ODD ? 3 : 0;                                  // b1 u, b1 u u', b1 u u'^2
    static constexpr int NA = NAE + NAO;
    static constexpr int NB = NBE + NBO;
    static constexpr int NG = NGE + (ODD ? 3 : 0);
};

// Exact product of two integer factors as a double: one 64-bit integer
// multiply and one conversion (the same value as converting both factors and
// multiplying in FP64, with two fewer FP64-pipe instructions).
__device__ __forceinline__ double int_prod(int a, int b) { return (double)((long long)a * (long long)b); }

__device__ __forceinline__ void write_out(const PlainJob &p, int win, int slot, int l1, int l2,
                                          double xi) {
    if (slot < 0) return;
    const double m12 = (2.0 * l2 + 1.0) * xi;   // M[l1][l2] = (2 l2 + 1) Xi
    const double m21 = (2.0 * l1 + 1.0) * xi;   // M[l2][l1] = (2 l1 + 1) Xi (only Xi is symmetric)
    if (p.n_bins == 0) {
        const int n = p.lmax - p.lmin + 1;
        double *base = p.out + ((size_t)win * p.nspec + slot) * (size_t)n * (size_t)n;
        base[(size_t)(l1 - p.lmin) * n + (l2 - p.lmin)] = m12;
        if (l1 != l2) base[(size_t)(l2 - p.lmin) * n + (l1 - p.lmin)] = m21;
    } else {
        const int b1 = p.bin_of[l1], b2 = p.bin_of[l2];
        if (b1 < 0 || b2 < 0) return;
        const int nb = p.n_bins;
        double *base = p.out + ((size_t)win * p.nspec + slot) * (size_t)nb * (size_t)nb;
        double w12 = p.bin_inv[b1], w21 = p.bin_inv[b2];
        if (p.bin_lw) {   // D_l band powers: l1(l1+1) / (l2(l2+1)) and its mirror
            const double *iw = p.bin_lw + p.lmax + 1;
            w12 *= p.bin_lw[l1] * iw[l2];
            w21 *= p.bin_lw[l2] * iw[l1];
        }
        atomicAdd(base + (size_t)b1 * nb + b2, m12 * w12);
        if (l1 != l2) atomicAdd(base + (size_t)b2 * nb + b1, m21 * w21);
    }
}

template <int NGE, bool ODD>
using Acc = double[Shape<NGE, ODD>::NG > 0 ? Shape<NGE, ODD>::NG : 1][2][2];

// k steps kk0 <= kk < kk1 of one staged l3 chunk of the register-tiled
// contractions: operand rows sa [NA][KC][TILE_I] and sb [NB][KC][TILE_J]
// (shared memory) into this thread's 2 x 2 outputs, rows ar and ar + RS of
// the tile, columns bc and bc + CS.
template <int NGE, bool ODD, int RS, int CS>
__device__ __forceinline__ void fma_chunk(const double *sa, const double *sb, int kk0, int kk1, int ar, int bc,
                                          Acc<NGE, ODD> &acc) {
    using S = Shape<NGE, ODD>;
#pragma unroll 2
    for (int kk = kk0; kk < kk1; ++kk) {
        double a[S::NA > 0 ? S::NA : 1][2], b[S::NB > 0 ? S::NB : 1][2];
#pragma unroll
        for (int q = 0; q < S::NA; ++q) {
            a[q][0] = sa[(q * KC + kk) * TILE_I + ar];
            a[q][1] = sa[(q * KC + kk) * TILE_I + ar + RS];
        }
#pragma unroll
        for (int q = 0; q < S::NB; ++q) {
            b[q][0] = sb[(q * KC + kk) * TILE_J + bc];
            b[q][1] = sb[(q * KC + kk) * TILE_J + bc + CS];
        }
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                if (NGE >= 1) acc[0][r][c] = fma(a[0][r], b[0][c], acc[0][r][c]);
                if (NGE >= 3) {
                    acc[1][r][c] = fma(a[0][r], b[1][c], acc[1][r][c]);
                    acc[2][r][c] = fma(a[1][r], b[1][c], acc[2][r][c]);
                }
                if (NGE >= 6) {
                    acc[3][r][c] = fma(a[0][r], b[2][c], acc[3][r][c]);
                    acc[4][r][c] = fma(a[1][r], b[2][c], acc[4][r][c]);
                    acc[5][r][c] = fma(a[2][r], b[2][c], acc[5][r][c]);
                }
                if (ODD) {
                    acc[NGE + 0][r][c] = fma(a[S::NAE][r], b[S::NBE][c], acc[NGE + 0][r][c]);
                    acc[NGE + 1][r][c] = fma(a[S::NAE][r], b[S::NBE + 1][c], acc[NGE + 1][r][c]);
                    acc[NGE + 2][r][c] = fma(a[S::NAE][r], b[S::NBE + 2][c], acc[NGE + 2][r][c]);
                }
            }
    }
}

// Per-pair combination of the contractions (the App. A kernels through the
// separable forms above) and the writes of both mirror entries; this
// thread's pairs are rows i0 + ar + RS r and columns j0 + bc + CS c.  The
// pair coefficients are products of per-l factors (lcoef, plain_coef_host):
// lambda/eta = rho(l1) sigma(l2), c1 = alpha(l1) beta(l2), c2 = alpha(l1)
// beta'(l2), C = kappa(l1) mu(l2), so no division or square root runs here.
template <int NGE, bool ODD, int RS, int CS>
__device__ __forceinline__ void epilogue(const double *__restrict__ lcoef, const PlainJob &p, int win, int pi,
                                         int i0, int j0, int ar, int bc, const Acc<NGE, ODD> &acc) {
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int i = i0 + ar + RS * r, j = j0 + bc + CS * c;
            const int l1 = j - i, l2 = i + j + pi;
            if (l1 < p.lmin || l2 > p.lmax || l1 > l2) continue;
            if (NGE >= 1) write_out(p, win, p.slot[0], l1, l2, acc[0][r][c]);
            double ee = 0.0, eebb = 0.0;
            if (NGE >= 3 || ODD) {
                const double *F1 = lcoef + (size_t)l1 * PL_COEF_N;   // rho, rho^2, c0, alpha, kappa
                const double *F2 = lcoef + (size_t)l2 * PL_COEF_N;   // sigma, sigma^2, beta, beta', e1, mu at 5..10
                if (NGE >= 3) {
                    const double c0 = F1[2], c1 = F1[3] * F2[7], c2 = F1[3] * F2[8];
                    const double s00 = acc[0][r][c], s01 = acc[1][r][c], s11 = acc[2][r][c];
                    const double xp = c0 * s00 - c1 * s01 - c2 * s11;
                    write_out(p, win, p.slot[1], l1, l2, (F1[0] * F2[5]) * xp);
                    if (NGE >= 6) {
                        const double r2 = F1[1] * F2[6];   // (lambda/eta)^2
                        const double s02 = acc[3][r][c], s12 = acc[4][r][c], s22 = acc[5][r][c];
                        const double xp2 = c0 * c0 * s00 - 2.0 * c0 * c1 * s01 - 2.0 * c0 * c2 * s11 +
                                           c1 * c1 * s02 + 2.0 * c1 * c2 * s12 + c2 * c2 * s22;
                        ee = r2 * xp2;
                        write_out(p, win, p.slot[2], l1, l2, ee);
                    }
                }
                if (ODD) {
                    const double e0 = (double)(l1 + 2), e1 = F2[9];
                    const double Cc = F1[4] * F2[10];   // (l2+2) / (eta^2 l1 (l1+1) (l2+1))
                    const double t0 = acc[NGE][r][c], t1 = acc[NGE + 1][r][c], t2 = acc[NGE + 2][r][c];
                    eebb = Cc * (e0 * e0 * t0 - 2.0 * e0 * e1 * t1 + e1 * e1 * t2);
                    write_out(p, win, p.slot[3], l1, l2, eebb);
                    if (NGE >= 6) write_out(p, win, p.slot[4], l1, l2, ee - eebb);
                }
            }
        }
}

template <int NGE, bool ODD>
__global__ void __launch_bounds__(NT) k_plain(const PlainArgs pa) {
    using S = Shape<NGE, ODD>;
    __shared__ double sa[S::NA > 0 ? S::NA : 1][KC][TILE_I];
    __shared__ double sb[S::NB > 0 ? S::NB : 1][KC][TILE_J];

    const WorkItem it = pa.items[blockIdx.x];
    const PlainJob &p = pa.jobs[it.job];
    const int win = it.win;
    const Tile t = p.tiles[it.tile];
    const int pi = t.pi, i0 = t.i0, j0 = t.j0;
    const double *__restrict__ A = p.A + (size_t)win * p.a_stride;
    const double *__restrict__ g = pa.g;
    const double *__restrict__ h = pa.h;
    const int cap = p.l3cap[win];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;

    // k ranges of the block (before the per-element triangle checks)
    const int kcap_e = (cap - pi) >> 1;              // l3 = 2k + pi <= cap
    const int kcap_o = (cap - 1 + pi) >> 1;          // l3 = 2k + 1 - pi <= cap
    const int khi_e = min(j0 + TILE_J - 1, kcap_e);
    const int khi_o = min(j0 + TILE_J - 2 + pi, kcap_o);
    int k_lo = i0, k_hi = -1;
    if (NGE > 0) k_hi = khi_e;
    if (ODD) k_hi = max(k_hi, khi_o);

    Acc<NGE, ODD> acc;
#pragma unroll
    for (int q = 0; q < S::NG; ++q)
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int c = 0; c < 2; ++c) acc[q][r][c] = 0.0;

    for (int kb = k_lo; kb <= k_hi; kb += KC) {
        __syncthreads();
        // ---- operand rows (i side)
        for (int idx = tid; idx < KC * TILE_I; idx += NT) {
            const int ii = idx % TILE_I, kk = idx / TILE_I;
            const int i = i0 + ii, k = kb + kk;
            if (NGE > 0) {
                double a0 = 0.0, v = 0.0;
                if (k >= i && k <= khi_e) {
                    a0 = A[2 * k + pi] * g[i + k + pi] * g[k - i];
                    v = int_prod(2 * k + 2 * i + 2 * pi + 1, 2 * k - 2 * i);
                }
                sa[0][kk][ii] = a0;
                if (S::NAE > 1) sa[1][kk][ii] = a0 * v;
                if (S::NAE > 2) sa[2][kk][ii] = a0 * v * v;
            }
            if (ODD) {
                double a1v = 0.0;
                if (k >= i + pi && k <= khi_o) {
                    const double v1 = int_prod(2 * i + 2 * k + 2, 2 * k + 1 - 2 * i - 2 * pi);
                    a1v = A[2 * k + 1 - pi] * g[i + k + 1] * g[k - i - pi] * v1;
                }
                sa[S::NAE][kk][ii] = a1v;
            }
        }
        // ---- operand columns (j side)
        for (int idx = tid; idx < KC * TILE_J; idx += NT) {
            const int jj = idx % TILE_J, kk = idx / TILE_J;
            const int j = j0 + jj, k = kb + kk;
            if (NGE > 0) {
                double b0 = 0.0, u = 0.0;
                if (k <= j && k <= khi_e) {
                    b0 = g[j - k] * h[j + k + pi];
                    u = int_prod(2 * j + 2 * k + 2 * pi + 2, 2 * j - 2 * k + 1);
                }
                sb[0][kk][jj] = b0;
                if (S::NBE > 1) sb[1][kk][jj] = b0 * u;
                if (S::NBE > 2) sb[2][kk][jj] = b0 * u * u;
            }
            if (ODD) {
                double b1u = 0.0, up = 0.0;
                if (k <= j + pi - 1 && k <= khi_o) {
                    const double u1 = int_prod(2 * j + 2 * k + 3, 2 * j - 2 * k + 2 * pi);
                    up = int_prod(2 * j + 2 * k + 4, 2 * j - 2 * k + 2 * pi + 1);
                    b1u = g[j - k + pi] * h[j + k + 1] * u1;
                }
                sb[S::NBE][kk][jj] = b1u;
                sb[S::NBE + 1][kk][jj] = b1u * up;
                sb[S::NBE + 2][kk][jj] = b1u * up * up;
            }
        }
        __syncthreads();
        fma_chunk<NGE, ODD, 16, 16>(&sa[0][0][0], &sb[0][0][0], 0, min(KC, k_hi - kb + 1), ty, tx, acc);
    }

    epilogue<NGE, ODD, 16, 16>(pa.lcoef, p, win, pi, i0, j0, ty, tx, acc);
}

// ---------------------------------------------------------------- tabled kernel
// k_plain recomputes the operand rows of each l3 chunk in every tile that
// covers it: a row block's i-side rows are rebuilt by each of its column
// tiles and a column block's j-side rows by each row tile, about 20 FP64-pipe
// instructions (products and integer conversions) per staged element.  The
// tabled form computes each block once -- B blocks (j side, window
// independent, cached per context) and A blocks (i side, per sweep and
// window) -- and a tile streams its chunks into shared memory with two bulk
// copies per chunk, double-buffered.  Values, zero pattern and the order of
// every operation are those of k_plain, so the two kernels agree bit for bit.
static_assert(TILE_I == 32 && TILE_J == 32 && KC == PT_KC && KC * TILE_I == PT_BLK, "operand block geometry");

// B blocks: column block jb, parity pi, chunk c <= 2 jb + 1 (k <= j0 + 31):
// rows b0, b0 u, b0 u^2 (even sweep) and b1 u, b1 u u', b1 u u'^2 (odd sweep)
// as [6][KC][TILE_J], zero where k lies outside the pair's range.  (A band
// limit needs no zeros here: the A side is zero past it.)
__global__ void k_btab(const double *__restrict__ g, const double *__restrict__ h, int njb, double *__restrict__ B) {
    const int c = blockIdx.x, jb = blockIdx.y, pi = blockIdx.z;
    if (jb >= njb || c > 2 * jb + 1) return;
    double *blk = B + (size_t)btab_block(jb, pi, c) * PT_BROWS * PT_BLK;
    for (int e = threadIdx.x; e < PT_BLK; e += blockDim.x) {
        const int kk = e / TILE_J, jj = e % TILE_J;
        const int j = jb * TILE_J + jj, k = c * KC + kk;
        double b0 = 0.0, u = 0.0;
        if (k <= j) {
            b0 = g[j - k] * h[j + k + pi];
            u = int_prod(2 * j + 2 * k + 2 * pi + 2, 2 * j - 2 * k + 1);
        }
        blk[e] = b0;
        blk[PT_BLK + e] = b0 * u;
        blk[2 * PT_BLK + e] = b0 * u * u;
        double b1u = 0.0, up = 0.0;
        if (k <= j + pi - 1) {
            const double u1 = int_prod(2 * j + 2 * k + 3, 2 * j - 2 * k + 2 * pi);
            up = int_prod(2 * j + 2 * k + 4, 2 * j - 2 * k + 2 * pi + 1);
            b1u = g[j - k + pi] * h[j + k + 1] * u1;
        }
        blk[3 * PT_BLK + e] = b1u;
        blk[4 * PT_BLK + e] = b1u * up;
        blk[5 * PT_BLK + e] = b1u * up * up;
    }
}

// A blocks of one sweep: window w, parity pi, row block ib, chunk
// c = 2 ib + m: the even rows a0, a0 v, a0 v^2 (the first nae) and, if odd,
// a1 v, as [nae + odd][KC][TILE_I]; zero outside the pair range and past the
// window's band (l3 > cap).
__global__ void k_atab(const double *__restrict__ A, int a_stride, const int *__restrict__ l3cap,
                       const double *__restrict__ g, const long long *__restrict__ aoff, int nib, int nae, int odd,
                       double *__restrict__ At) {
    const int m = blockIdx.x, ib = blockIdx.y, w = blockIdx.z >> 1, pi = blockIdx.z & 1;
    const size_t idx = ((size_t)w * 2 + pi) * nib + ib;
    const long long first = aoff[idx];
    if (m >= aoff[idx + 1] - first) return;
    const int na = nae + odd;
    double *blk = At + (size_t)(first + m) * na * PT_BLK;
    const double *__restrict__ Aw = A + (size_t)w * a_stride;
    const int cap = l3cap[w];
    const int c = 2 * ib + m;
    for (int e = threadIdx.x; e < PT_BLK; e += blockDim.x) {
        const int kk = e / TILE_I, ii = e % TILE_I;
        const int i = ib * TILE_I + ii, k = c * KC + kk;
        if (nae > 0) {
            double a0 = 0.0, v = 0.0;
            if (k >= i && 2 * k + pi <= cap) {
                a0 = Aw[2 * k + pi] * g[i + k + pi] * g[k - i];
                v = int_prod(2 * k + 2 * i + 2 * pi + 1, 2 * k - 2 * i);
            }
            blk[e] = a0;
            if (nae > 1) blk[PT_BLK + e] = a0 * v;
            if (nae > 2) blk[2 * PT_BLK + e] = a0 * v * v;
        }
        if (odd) {
            double a1v = 0.0;
            if (k >= i + pi && 2 * k + 1 - pi <= cap) {
                const double v1 = int_prod(2 * i + 2 * k + 2, 2 * k + 1 - 2 * i - 2 * pi);
                a1v = Aw[2 * k + 1 - pi] * g[i + k + 1] * g[k - i - pi] * v1;
            }
            blk[nae * PT_BLK + e] = a1v;
        }
    }
}

template <int NGE, bool ODD>
__global__ void __launch_bounds__(NT, 2) k_plain_tab(const PlainArgs pa) {
    using S = Shape<NGE, ODD>;
    constexpr int NA = S::NA, NB = S::NB;
    constexpr int BQ0 = NGE > 0 ? 0 : 3;             // first B row the variant reads
    constexpr int STAGE = (NA + NB) * PT_BLK;        // doubles per pipeline stage
    static_assert(NGE == 0 || !ODD || S::NBE == 3, "B rows of the variant must be contiguous");
    extern __shared__ __align__(128) double stage[];   // [2][NA + NB][KC][32]
    __shared__ __align__(8) uint64_t full[2];

    const WorkItem it = pa.items[blockIdx.x];
    const PlainJob &p = pa.jobs[it.job];
    const int win = it.win;
    const Tile t = p.tiles[it.tile];
    const int pi = t.pi, i0 = t.i0, j0 = t.j0;
    const int cap = p.l3cap[win];
    const int tid = threadIdx.x;
    // Each warp owns a 16 x 8 block of the tile (rows 16 h .., columns 8 q ..),
    // each thread rows ar, ar + 8 and columns bc, bc + 4 of it.  A warp skips
    // the k steps before its first row's range and after its last column's
    // (its products there are exact zeros) and all of them when its block has
    // no valid pair.  The two warps of each SM sub-partition (w and w + 4) take
    // opposite halves and column quarters q, 3 - q, so that every
    // sub-partition skips equally.
    const int warp = tid >> 5, lane = tid & 31;
    const int wh = warp >> 2, wq = wh ? 3 - (warp & 3) : (warp & 3);
    const int ar = 16 * wh + (lane >> 2), bc = 8 * wq + (lane & 3);

    // the k range k_plain runs (same bounds)
    const int kcap_e = (cap - pi) >> 1, kcap_o = (cap - 1 + pi) >> 1;
    const int k_lo = i0;
    int k_hi = -1;
    if (NGE > 0) k_hi = min(j0 + TILE_J - 1, kcap_e);
    if (ODD) k_hi = max(k_hi, min(j0 + TILE_J - 2 + pi, kcap_o));
    const int nch = k_hi >= k_lo ? (k_hi - k_lo) / KC + 1 : 0;
    // this warp's k range (same bounds as the tile's, for its rows and columns)
    const int wi0 = i0 + 16 * wh, wj1 = j0 + 8 * wq + 7;
    const int wk_lo = wi0;
    int wk_hi = -1;
    if (NGE > 0) wk_hi = min(wj1, kcap_e);
    if (ODD) wk_hi = max(wk_hi, min(wj1 - 1 + pi, kcap_o));
    // a valid pair (j - i >= lmin, i + j <= lmax - pi) in the block exists iff one does on its first row
    if (max(j0 + 8 * wq, wi0 + p.lmin) > min(wj1, p.lmax - pi - wi0)) wk_hi = -1;
    const int ib = i0 / TILE_I, jb = j0 / TILE_J;
    const size_t aidx = ((size_t)win * 2 + pi) * p.nib + ib;
    const long long afirst = p.aoff[aidx];
    if (nch > p.aoff[aidx + 1] - afirst || (nch > 0 && (jb >= pa.btab_njb || k_lo / KC + nch - 1 > 2 * jb + 1))) {
        if (tid == 0) atomicCAS(pa.err, 0, PT_ERR_RANGE);
        return;
    }
    const double *asrc = p.atab + (size_t)afirst * NA * PT_BLK;
    const double *bsrc = pa.btab + ((size_t)btab_block(jb, pi, k_lo / KC) * PT_BROWS + BQ0) * PT_BLK;

    const uint32_t bar0 = mbar::smem_u32(&full[0]), bar1 = mbar::smem_u32(&full[1]);
    if (tid == 0) {
        mbar::init(bar0, 1);
        mbar::init(bar1, 1);
        mbar::fence_init();
    }
    __syncthreads();
    auto issue = [&](int m) {   // chunk m into stage m & 1 (one thread)
        const uint32_t bar = (m & 1) ? bar1 : bar0;
        const uint32_t dst = mbar::smem_u32(stage + (m & 1) * STAGE);
        mbar::expect_tx(bar, STAGE * 8);
        mbar::copy_g2s(dst, asrc + (size_t)m * NA * PT_BLK, NA * PT_BLK * 8, bar);
        mbar::copy_g2s(dst + NA * PT_BLK * 8, bsrc + (size_t)m * PT_BROWS * PT_BLK, NB * PT_BLK * 8, bar);
    };
    if (tid == 0) {
        if (nch > 0) issue(0);
        if (nch > 1) issue(1);
    }

    Acc<NGE, ODD> acc;
#pragma unroll
    for (int q = 0; q < S::NG; ++q)
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int c = 0; c < 2; ++c) acc[q][r][c] = 0.0;

    for (int m = 0; m < nch; ++m) {
        const bool got = mbar::wait((m & 1) ? bar1 : bar0, (m >> 1) & 1);
        if (!__syncthreads_and(got)) {
            // record, let the copies this CTA issued finish (bounded), leave
            if (tid == 0) {
                atomicCAS(pa.err, 0, PT_ERR_WAIT);
                if (m + 1 < nch) mbar::wait(((m + 1) & 1) ? bar1 : bar0, ((m + 1) >> 1) & 1);
                mbar::wait((m & 1) ? bar1 : bar0, (m >> 1) & 1);
            }
            return;
        }
        const double *st = stage + (m & 1) * STAGE;
        const int kb = k_lo + m * KC;
        const int kk0 = max(0, wk_lo - kb), kk1 = min(KC, wk_hi - kb + 1);
        if (kk0 < kk1) fma_chunk<NGE, ODD, 8, 4>(st, st + NA * PT_BLK, kk0, kk1, ar, bc, acc);
        __syncthreads();   // stage m & 1 is free again
        if (tid == 0 && m + 2 < nch) issue(m + 2);
    }

    epilogue<NGE, ODD, 8, 4>(pa.lcoef, p, win, pi, i0, j0, ar, bc, acc);
}

__global__ void k_weights(const double *__restrict__ W, int w_len, const int *__restrict__ l3cap,
                          double *__restrict__ A, int a_stride) {
    const int win = blockIdx.y;
    const int cap = l3cap[win];
    const double inv4pi = 0.07957747154594767;   // 1 / (4 pi)
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < a_stride; l += gridDim.x * blockDim.x) {
        double v = 0.0;
        if (l <= cap && l < w_len) v = (2.0 * l + 1.0) * W[(size_t)win * w_len + l] * inv4pi;
        A[(size_t)win * a_stride + l] = v;
    }
}

}  // namespace

cudaError_t launch_weights(const double *W, int w_len, int n_win, const int *l3cap, double *A,
                           int a_stride, cudaStream_t st) {
    dim3 grid((a_stride + 255) / 256, n_win);
    k_weights<<<grid, 256, 0, st>>>(W, w_len, l3cap, A, a_stride);
    return cudaGetLastError();
}

void plain_variant(int mode, const int slot[5], int *nge, bool *odd) {
    *odd = slot[3] >= 0 || slot[4] >= 0;
    if (mode == MODE_TT) {
        *nge = 1;
        *odd = false;
    } else if (mode == MODE_TE) {
        *nge = 3;
        *odd = false;
    } else {
        const bool even = slot[0] >= 0 || slot[1] >= 0 || slot[2] >= 0 || slot[4] >= 0;
        *nge = even ? 6 : 0;
    }
}

void plain_coef_host(int n, std::vector<double> &out) {
    out.assign((size_t)n * PL_COEF_N, 0.0);
    for (int l = 2; l < n; ++l) {
        const double L = l;
        double *f = out.data() + (size_t)l * PL_COEF_N;
        const double rho2 = L * (L + 1.0) / ((L - 1.0) * (L + 2.0));
        const double al = 1.0 / (L * (L + 1.0));
        const double s2 = (L + 1.0) * (L + 2.0) / ((L - 1.0) * L);
        f[0] = std::sqrt(rho2);                             // rho
        f[1] = rho2;
        f[2] = 1.0 + 2.0 / L;                               // c0
        f[3] = al;                                          // alpha
        f[4] = al / ((L - 1.0) * (L + 2.0));                // kappa
        f[5] = std::sqrt(s2);                               // sigma
        f[6] = s2;
        f[7] = 1.0 / (L + 1.0);                             // beta
        f[8] = 1.0 / (2.0 * (L + 1.0) * (L + 2.0));         // beta'
        f[9] = 1.0 / (2.0 * (L + 2.0));                     // e1
        f[10] = (L + 2.0) / ((L + 1.0) * (L - 1.0) * L);    // mu
    }
}

cudaError_t launch_btab(const double *g, const double *h, int njb, double *B, cudaStream_t st) {
    if (njb <= 0) return cudaSuccess;
    k_btab<<<dim3(2 * njb, njb, 2), 256, 0, st>>>(g, h, njb, B);
    return cudaGetLastError();
}

cudaError_t launch_atab(const double *A, int a_stride, const int *l3cap, const double *g, const long long *aoff,
                        int n_win, int nib, int max_count, int nae, int odd, double *At, cudaStream_t st) {
    if (max_count <= 0 || nib <= 0 || n_win <= 0) return cudaSuccess;
    k_atab<<<dim3(max_count, nib, 2 * n_win), 256, 0, st>>>(A, a_stride, l3cap, g, aoff, nib, nae, odd, At);
    return cudaGetLastError();
}

template <int NGE, bool ODD>
static cudaError_t launch_tab(const PlainArgs &a, cudaStream_t st) {
    using S = Shape<NGE, ODD>;
    const int smem = 2 * (S::NA + S::NB) * PT_BLK * (int)sizeof(double);
    static std::atomic<unsigned long long> attr{0};   // per variant
    const cudaError_t e = opt_in_smem(k_plain_tab<NGE, ODD>, smem, attr);
    if (e != cudaSuccess) return e;
    k_plain_tab<NGE, ODD><<<a.n_items, NT, smem, st>>>(a);
    return cudaGetLastError();
}

// One CTA per work item; the variant (even contractions, odd sweep) is the
// same for every sweep of the launch (plain_variant of each sweep).  With
// operand tables (a.btab) the tabled kernel runs.
cudaError_t launch_plain(const PlainArgs &a, cudaStream_t st) {
    if (a.n_items == 0) return cudaSuccess;
    dim3 grid(a.n_items);
    const int nge = a.nge;
    const bool odd = a.odd != 0;
    if (a.btab) {
        if (nge == 1 && !odd) return launch_tab<1, false>(a, st);
        if (nge == 3 && !odd) return launch_tab<3, false>(a, st);
        if (nge == 6 && odd) return launch_tab<6, true>(a, st);
        if (nge == 6) return launch_tab<6, false>(a, st);
        if (nge == 0 && odd) return launch_tab<0, true>(a, st);
        return cudaErrorInvalidValue;
    }
    if (nge == 1) k_plain<1, false><<<grid, NT, 0, st>>>(a);
    else if (nge == 3) k_plain<3, false><<<grid, NT, 0, st>>>(a);
    else if (nge == 6 && odd) k_plain<6, true><<<grid, NT, 0, st>>>(a);
    else if (nge == 6) k_plain<6, false><<<grid, NT, 0, st>>>(a);
    else if (odd) k_plain<0, true><<<grid, NT, 0, st>>>(a);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace cpl
