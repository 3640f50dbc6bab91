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

#include "internal.h"

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

    double acc[S::NG > 0 ? S::NG : 1][2][2];
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
        const int kn = min(KC, k_hi - kb + 1);
#pragma unroll 2
        for (int kk = 0; kk < kn; ++kk) {
            double a[S::NA > 0 ? S::NA : 1][2], b[S::NB > 0 ? S::NB : 1][2];
#pragma unroll
            for (int q = 0; q < S::NA; ++q) {
                a[q][0] = sa[q][kk][ty];
                a[q][1] = sa[q][kk][ty + 16];
            }
#pragma unroll
            for (int q = 0; q < S::NB; ++q) {
                b[q][0] = sb[q][kk][tx];
                b[q][1] = sb[q][kk][tx + 16];
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

    // ---- epilogue: combine the contractions per pair and write both mirror entries
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int i = i0 + ty + 16 * r, j = j0 + tx + 16 * c;
            const int l1 = j - i, l2 = i + j + pi;
            if (l1 < p.lmin || l2 > p.lmax || l1 > l2) continue;
            if (NGE >= 1) write_out(p, win, p.slot[0], l1, l2, acc[0][r][c]);
            double ee = 0.0, eebb = 0.0;
            if (NGE >= 3 || ODD) {
                const double L1 = l1, L2 = l2;
                const double eta2 = (L1 - 1.0) * (L1 + 2.0) * (L2 - 1.0) * L2;
                const double c1 = 1.0 / (L1 * (L1 + 1.0) * (L2 + 1.0));
                if (NGE >= 3) {
                    const double r2 = L1 * (L1 + 1.0) * (L2 + 1.0) * (L2 + 2.0) / eta2;  // (lambda/eta)^2
                    const double c0 = 1.0 + 2.0 / L1;
                    const double c2 = c1 / (2.0 * (L2 + 2.0));
                    const double s00 = acc[0][r][c], s01 = acc[1][r][c], s11 = acc[2][r][c];
                    const double xp = c0 * s00 - c1 * s01 - c2 * s11;
                    write_out(p, win, p.slot[1], l1, l2, sqrt(r2) * xp);
                    if (NGE >= 6) {
                        const double s02 = acc[3][r][c], s12 = acc[4][r][c], s22 = acc[5][r][c];
                        const double xp2 = c0 * c0 * s00 - 2.0 * c0 * c1 * s01 - 2.0 * c0 * c2 * s11 +
                                           c1 * c1 * s02 + 2.0 * c1 * c2 * s12 + c2 * c2 * s22;
                        ee = r2 * xp2;
                        write_out(p, win, p.slot[2], l1, l2, ee);
                    }
                }
                if (ODD) {
                    const double e0 = L1 + 2.0, e1 = 1.0 / (2.0 * (L2 + 2.0));
                    const double Cc = (L2 + 2.0) * c1 / eta2;   // (l2+2) / (eta^2 l1 (l1+1) (l2+1))
                    const double t0 = acc[NGE][r][c], t1 = acc[NGE + 1][r][c], t2 = acc[NGE + 2][r][c];
                    eebb = Cc * (e0 * e0 * t0 - 2.0 * e0 * e1 * t1 + e1 * e1 * t2);
                    write_out(p, win, p.slot[3], l1, l2, eebb);
                    if (NGE >= 6) write_out(p, win, p.slot[4], l1, l2, ee - eebb);
                }
            }
        }
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

// One CTA per work item; the variant (even contractions, odd sweep) is the
// same for every sweep of the launch (plain_variant of each sweep).
cudaError_t launch_plain(const PlainArgs &a, cudaStream_t st) {
    if (a.n_items == 0) return cudaSuccess;
    dim3 grid(a.n_items);
    const int nge = a.nge;
    const bool odd = a.odd != 0;
    if (nge == 1) k_plain<1, false><<<grid, NT, 0, st>>>(a);
    else if (nge == 3) k_plain<3, false><<<grid, NT, 0, st>>>(a);
    else if (nge == 6 && odd) k_plain<6, true><<<grid, NT, 0, st>>>(a);
    else if (nge == 6) k_plain<6, false><<<grid, NT, 0, st>>>(a);
    else if (odd) k_plain<0, true><<<grid, NT, 0, st>>>(a);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace cpl
