// plain_df.cu -- the plain path in double-float arithmetic (CPL_DF32).
//
// Same separable contractions, tiles and epilogue as plain_fp64.cu (see the
// derivation there), but every operand and every product is an unevaluated
// pair of FP32 numbers (hi + lo, ~48-bit significand) and the l3 sums run on
// the FP32 pipe, which GB300 issues at 64x its FP64 rate:
//
// * operands: the g and h tables as FP32 pairs (built once per table size),
//   the integer factors u, v as exact two-products, the window weight of
//   each staged l3 scaled by 2^-E (E from the largest |A| over the tile's l3
//   range, found with integer compares on the FP64 bit patterns) so the
//   pairs stay inside FP32's exponent range; terms 2^126 below the tile's
//   largest weight are lost, far below the error metric;
// * products: p = a_h b_h exactly as (p, fma(a_h, b_h, -p)) plus the two
//   cross terms; sums: compensated summation (a two-sum per term, the
//   errors gathered in a low word) over chunks of 16 l3 values, each chunk
//   then added to the running total with an accurate pair addition.  Two output columns share each
//   instruction (packed f32x2 add, mul, fma);
// * epilogue: hi + lo in FP64 times 2^E, then the FP64 combination of the
//   contractions and the writes of plain_fp64.cu.
// FP64 work per tile: the weights of each staged l3 chunk and the epilogue.
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

// ---- FP32-pair arithmetic (explicitly rounded operations: no contraction)
__device__ __forceinline__ float2 two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return make_float2(p, fmaf(a, b, -p));
}
__device__ __forceinline__ float2 fast_two_sum(float a, float b) {   // |a| >= |b|
    const float s = __fadd_rn(a, b);
    return make_float2(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
    const float p = __fmul_rn(a.x, b.x);
    float e = fmaf(a.x, b.x, -p);
    e = fmaf(a.x, b.y, e);
    e = fmaf(a.y, b.x, e);
    return fast_two_sum(p, e);
}
// Exact product of two integers below 2^24 as an FP32 pair.
__device__ __forceinline__ float2 int_prod(int a, int b) { return two_prod((float)a, (float)b); }

// Packed pairs: .x / .y are two independent values (two output columns).
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    float2 r;
    asm("sub.rn.f32x2 %0, %1, %2;"
        : "=l"(*reinterpret_cast<unsigned long long *>(&r))
        : "l"(*reinterpret_cast<unsigned long long *>(&a)), "l"(*reinterpret_cast<unsigned long long *>(&b)));
    return r;
}
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

// acc (hi2, lo2) += a * b for a scalar pair a and packed pairs b (bh2, bl2):
// the product's rounding error from fma, the sum's from a two-sum, both
// collected in lo (compensated summation: lo is not renormalised into hi
// until the chunk is added to the total, so a chunk of n terms is as
// accurate as if summed in twice the working precision plus O(n^2 u^2)).
__device__ __forceinline__ void df_fma2(float2 &hi, float2 &lo, float2 ah2, float2 al2, float2 bh, float2 bl) {
    const float2 p = __fmul2_rn(ah2, bh);
    float2 e = __ffma2_rn(ah2, bh, neg2(p));
    e = __ffma2_rn(ah2, bl, e);
    e = __ffma2_rn(al2, bh, e);
    const float2 s = __fadd2_rn(hi, p);
    const float2 z = sub2(s, hi);
    const float2 t = __fadd2_rn(sub2(hi, sub2(s, z)), sub2(p, z));
    lo = __fadd2_rn(lo, __fadd2_rn(t, e));
    hi = s;
}

// (Th, Tl) += (Ch, Cl), packed, with an accurate pair addition.
__device__ __forceinline__ void df_add2(float2 &Th, float2 &Tl, float2 Ch, float2 Cl) {
    const float2 s = __fadd2_rn(Th, Ch);
    const float2 z = sub2(s, Th);
    float2 e = __fadd2_rn(sub2(Th, sub2(s, z)), sub2(Ch, z));
    const float2 t = __fadd2_rn(Tl, Cl);
    const float2 z2 = sub2(t, Tl);
    const float2 f = __fadd2_rn(sub2(Tl, sub2(t, z2)), sub2(Cl, z2));
    e = __fadd2_rn(e, t);
    float2 h = __fadd2_rn(s, e);
    e = sub2(e, sub2(h, s));
    e = __fadd2_rn(e, f);
    Th = __fadd2_rn(h, e);
    Tl = sub2(e, sub2(Th, h));
}

__device__ __forceinline__ float2 split_double(double x) {
    const float h = __double2float_rn(x);
    return make_float2(h, __double2float_rn(x - (double)h));
}

__device__ __forceinline__ void write_out(const PlainJob &p, int win, int slot, int l1, int l2, double xi) {
    if (slot < 0) return;
    const double m12 = (2.0 * l2 + 1.0) * xi;   // M[l1][l2] = (2 l2 + 1) Xi
    const double m21 = (2.0 * l1 + 1.0) * xi;   // M[l2][l1] = (2 l1 + 1) Xi
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
__global__ void __launch_bounds__(NT, 1) k_plain_df(const PlainArgs pa) {
    using S = Shape<NGE, ODD>;
    constexpr int NG = S::NG > 0 ? S::NG : 1;
    __shared__ float2 sa[S::NA > 0 ? S::NA : 1][KC][TILE_I];
    __shared__ float2 sb[S::NB > 0 ? S::NB : 1][KC][TILE_J];
    __shared__ float2 sw[2][KC];                       // scaled weights: even l3 = 2k + pi, odd l3 = 2k + 1 - pi
    __shared__ unsigned long long smax[NT / 32];

    const WorkItem it = pa.items[blockIdx.x];
    const PlainJob &p = pa.jobs[it.job];
    const int win = it.win;
    const Tile t = p.tiles[it.tile];
    const int pi = t.pi, i0 = t.i0, j0 = t.j0;
    const double *__restrict__ A = p.A + (size_t)win * p.a_stride;
    const float2 *__restrict__ gdf = pa.gdf;
    const float2 *__restrict__ hdf = pa.hdf;
    const int cap = p.l3cap[win];
    const int tid = threadIdx.x, lane = tid & 31;
    // warp blocks of 16 x 8 pairs (rows ar, ar + 8, columns bc, bc + 4 per
    // thread) with their own k ranges, as in the tabled FP64 kernel: the two
    // warps of a sub-partition take opposite row halves and column quarters
    const int warp = tid >> 5;
    const int wh = warp >> 2, wq = wh ? 3 - (warp & 3) : (warp & 3);
    const int ar = 16 * wh + (lane >> 2), bc = 8 * wq + (lane & 3);

    const int kcap_e = (cap - pi) >> 1;
    const int kcap_o = (cap - 1 + pi) >> 1;
    const int khi_e = min(j0 + TILE_J - 1, kcap_e);
    const int khi_o = min(j0 + TILE_J - 2 + pi, kcap_o);
    int k_lo = i0, k_hi = -1;
    if (NGE > 0) k_hi = khi_e;
    if (ODD) k_hi = max(k_hi, khi_o);
    // this warp's k range; none when its block holds no valid pair (the
    // steps outside it multiply exact zeros)
    const int wi0 = i0 + 16 * wh, wj1 = j0 + 8 * wq + 7;
    int wk_hi = -1;
    if (NGE > 0) wk_hi = min(wj1, kcap_e);
    if (ODD) wk_hi = max(wk_hi, min(wj1 - 1 + pi, kcap_o));
    if (max(j0 + 8 * wq, wi0 + p.lmin) > min(wj1, p.lmax - pi - wi0)) wk_hi = -1;

    // tile scale 2^-E: E from the largest |A| over the tile's l3 range
    {
        const int l3_lo = 2 * k_lo + pi;
        const int l3_hi = max(NGE > 0 ? 2 * khi_e + pi : -1, ODD ? 2 * khi_o + 1 - pi : -1);
        unsigned long long mb = 0ull;
        for (int l = l3_lo + tid; l <= l3_hi; l += NT) {
            const unsigned long long b = (unsigned long long)__double_as_longlong(A[l]) & 0x7fffffffffffffffull;
            mb = b > mb ? b : mb;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long w = __shfl_xor_sync(0xffffffffu, mb, o);
            mb = w > mb ? w : mb;
        }
        if (lane == 0) smax[tid >> 5] = mb;
        __syncthreads();
    }
    unsigned long long mb = 0ull;
#pragma unroll
    for (int q = 0; q < NT / 32; ++q) mb = smax[q] > mb ? smax[q] : mb;
    const int E = mb ? max((int)((mb >> 52) & 0x7ff), 1) - 1023 : 0;   // |A| < 2^(E+1)
    const double scale = ldexp(1.0, -E);
    if (!mb) k_hi = -1;                                               // every weight is zero

    float2 th[NG][2], tl[NG][2];
#pragma unroll
    for (int q = 0; q < NG; ++q)
#pragma unroll
        for (int r = 0; r < 2; ++r) th[q][r] = tl[q][r] = make_float2(0.f, 0.f);

    for (int kb = k_lo; kb <= k_hi; kb += KC) {
        __syncthreads();
        if (tid < 2 * KC) {
            const int kk = tid % KC, od = tid / KC, k = kb + kk;
            const bool ok = od ? (ODD && k <= khi_o) : (NGE > 0 && k <= khi_e);
            sw[od][kk] = ok ? split_double(A[od ? 2 * k + 1 - pi : 2 * k + pi] * scale) : make_float2(0.f, 0.f);
        }
        __syncthreads();
        // ---- operand rows (i side)
        for (int idx = tid; idx < KC * TILE_I; idx += NT) {
            const int ii = idx % TILE_I, kk = idx / TILE_I;
            const int i = i0 + ii, k = kb + kk;
            if (NGE > 0) {
                float2 a0 = make_float2(0.f, 0.f), v = a0;
                if (k >= i && k <= khi_e) {
                    a0 = df_mul(df_mul(sw[0][kk], gdf[i + k + pi]), gdf[k - i]);
                    v = int_prod(2 * k + 2 * i + 2 * pi + 1, 2 * k - 2 * i);
                }
                sa[0][kk][ii] = a0;
                if (S::NAE > 1) {
                    const float2 a0v = df_mul(a0, v);
                    sa[1][kk][ii] = a0v;
                    if (S::NAE > 2) sa[2][kk][ii] = df_mul(a0v, v);
                }
            }
            if (ODD) {
                float2 a1v = make_float2(0.f, 0.f);
                if (k >= i + pi && k <= khi_o) {
                    const float2 v1 = int_prod(2 * i + 2 * k + 2, 2 * k + 1 - 2 * i - 2 * pi);
                    a1v = df_mul(df_mul(df_mul(sw[1][kk], gdf[i + k + 1]), gdf[k - i - pi]), v1);
                }
                sa[S::NAE][kk][ii] = a1v;
            }
        }
        // ---- operand columns (j side)
        for (int idx = tid; idx < KC * TILE_J; idx += NT) {
            const int jj = idx % TILE_J, kk = idx / TILE_J;
            const int j = j0 + jj, k = kb + kk;
            if (NGE > 0) {
                float2 b0 = make_float2(0.f, 0.f), u = b0;
                if (k <= j && k <= khi_e) {
                    b0 = df_mul(gdf[j - k], hdf[j + k + pi]);
                    u = int_prod(2 * j + 2 * k + 2 * pi + 2, 2 * j - 2 * k + 1);
                }
                sb[0][kk][jj] = b0;
                if (S::NBE > 1) {
                    const float2 b0u = df_mul(b0, u);
                    sb[1][kk][jj] = b0u;
                    if (S::NBE > 2) sb[2][kk][jj] = df_mul(b0u, u);
                }
            }
            if (ODD) {
                float2 b1u = make_float2(0.f, 0.f), up = b1u;
                if (k <= j + pi - 1 && k <= khi_o) {
                    const float2 u1 = int_prod(2 * j + 2 * k + 3, 2 * j - 2 * k + 2 * pi);
                    up = int_prod(2 * j + 2 * k + 4, 2 * j - 2 * k + 2 * pi + 1);
                    b1u = df_mul(df_mul(gdf[j - k + pi], hdf[j + k + 1]), u1);
                }
                const float2 b1uu = df_mul(b1u, up);
                sb[S::NBE][kk][jj] = b1u;
                sb[S::NBE + 1][kk][jj] = b1uu;
                sb[S::NBE + 2][kk][jj] = df_mul(b1uu, up);
            }
        }
        __syncthreads();
        const int kk0 = max(0, wi0 - kb), kk1 = min(min(KC, k_hi - kb + 1), wk_hi - kb + 1);
        float2 ch[NG][2], cl[NG][2];
#pragma unroll
        for (int q = 0; q < NG; ++q)
#pragma unroll
            for (int r = 0; r < 2; ++r) ch[q][r] = cl[q][r] = make_float2(0.f, 0.f);
        for (int kk = kk0; kk < kk1; ++kk) {
            float2 ah[S::NA > 0 ? S::NA : 1][2], al[S::NA > 0 ? S::NA : 1][2];
            float2 bh[S::NB > 0 ? S::NB : 1], bl[S::NB > 0 ? S::NB : 1];
#pragma unroll
            for (int q = 0; q < S::NA; ++q)
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const float2 x = sa[q][kk][ar + 8 * r];
                    ah[q][r] = make_float2(x.x, x.x);
                    al[q][r] = make_float2(x.y, x.y);
                }
#pragma unroll
            for (int q = 0; q < S::NB; ++q) {
                const float2 x0 = sb[q][kk][bc], x1 = sb[q][kk][bc + 4];
                bh[q] = make_float2(x0.x, x1.x);
                bl[q] = make_float2(x0.y, x1.y);
            }
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                if (NGE >= 1) df_fma2(ch[0][r], cl[0][r], ah[0][r], al[0][r], bh[0], bl[0]);
                if (NGE >= 3) {
                    df_fma2(ch[1][r], cl[1][r], ah[0][r], al[0][r], bh[1], bl[1]);
                    df_fma2(ch[2][r], cl[2][r], ah[1][r], al[1][r], bh[1], bl[1]);
                }
                if (NGE >= 6) {
                    df_fma2(ch[3][r], cl[3][r], ah[0][r], al[0][r], bh[2], bl[2]);
                    df_fma2(ch[4][r], cl[4][r], ah[1][r], al[1][r], bh[2], bl[2]);
                    df_fma2(ch[5][r], cl[5][r], ah[2][r], al[2][r], bh[2], bl[2]);
                }
                if (ODD) {
                    df_fma2(ch[NGE + 0][r], cl[NGE + 0][r], ah[S::NAE][r], al[S::NAE][r], bh[S::NBE], bl[S::NBE]);
                    df_fma2(ch[NGE + 1][r], cl[NGE + 1][r], ah[S::NAE][r], al[S::NAE][r], bh[S::NBE + 1],
                            bl[S::NBE + 1]);
                    df_fma2(ch[NGE + 2][r], cl[NGE + 2][r], ah[S::NAE][r], al[S::NAE][r], bh[S::NBE + 2],
                            bl[S::NBE + 2]);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < S::NG; ++q)
#pragma unroll
            for (int r = 0; r < 2; ++r) df_add2(th[q][r], tl[q][r], ch[q][r], cl[q][r]);
    }

    // ---- epilogue (FP64): unscale the pair totals and combine as plain_fp64.cu
    const double unscale = ldexp(1.0, E);
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int i = i0 + ar + 8 * r, j = j0 + bc + 4 * c;
            const int l1 = j - i, l2 = i + j + pi;
            if (l1 < p.lmin || l2 > p.lmax || l1 > l2) continue;
            double acc[NG];
#pragma unroll
            for (int q = 0; q < S::NG; ++q)
                acc[q] = ((double)(c ? th[q][r].y : th[q][r].x) + (double)(c ? tl[q][r].y : tl[q][r].x)) * unscale;
            if (NGE >= 1) write_out(p, win, p.slot[0], l1, l2, acc[0]);
            double ee = 0.0, eebb = 0.0;
            if (NGE >= 3 || ODD) {
                const double L1 = l1, L2 = l2;
                const double eta2 = (L1 - 1.0) * (L1 + 2.0) * (L2 - 1.0) * L2;
                const double c1 = 1.0 / (L1 * (L1 + 1.0) * (L2 + 1.0));
                if (NGE >= 3) {
                    const double r2 = L1 * (L1 + 1.0) * (L2 + 1.0) * (L2 + 2.0) / eta2;   // (lambda/eta)^2
                    const double c0 = 1.0 + 2.0 / L1;
                    const double c2 = c1 / (2.0 * (L2 + 2.0));
                    const double s00 = acc[0], s01 = acc[1], s11 = acc[2];
                    const double xp = c0 * s00 - c1 * s01 - c2 * s11;
                    write_out(p, win, p.slot[1], l1, l2, sqrt(r2) * xp);
                    if (NGE >= 6) {
                        const double s02 = acc[3], s12 = acc[4], s22 = acc[5];
                        const double xp2 = c0 * c0 * s00 - 2.0 * c0 * c1 * s01 - 2.0 * c0 * c2 * s11 +
                                           c1 * c1 * s02 + 2.0 * c1 * c2 * s12 + c2 * c2 * s22;
                        ee = r2 * xp2;
                        write_out(p, win, p.slot[2], l1, l2, ee);
                    }
                }
                if (ODD) {
                    const double e0 = L1 + 2.0, e1 = 1.0 / (2.0 * (L2 + 2.0));
                    const double Cc = (L2 + 2.0) * c1 / eta2;
                    const double t0 = acc[NGE], t1 = acc[NGE + 1], t2 = acc[NGE + 2];
                    eebb = Cc * (e0 * e0 * t0 - 2.0 * e0 * e1 * t1 + e1 * e1 * t2);
                    write_out(p, win, p.slot[3], l1, l2, eebb);
                    if (NGE >= 6) write_out(p, win, p.slot[4], l1, l2, ee - eebb);
                }
            }
        }
}

__global__ void k_df_tables(const double *__restrict__ g, const double *__restrict__ h, int n, float2 *gdf,
                            float2 *hdf) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        gdf[q] = split_double(g[q]);
        hdf[q] = split_double(h[q]);
    }
}

}  // namespace

cudaError_t launch_df_tables(const double *g, const double *h, int n, float2 *gdf, float2 *hdf, cudaStream_t st) {
    k_df_tables<<<(n + 255) / 256, 256, 0, st>>>(g, h, n, gdf, hdf);
    return cudaGetLastError();
}

cudaError_t launch_plain_df(const PlainArgs &a, cudaStream_t st) {
    if (a.n_items == 0) return cudaSuccess;
    dim3 grid(a.n_items);
    const int nge = a.nge;
    const bool odd = a.odd != 0;
    if (nge == 1) k_plain_df<1, false><<<grid, NT, 0, st>>>(a);
    else if (nge == 3) k_plain_df<3, false><<<grid, NT, 0, st>>>(a);
    else if (nge == 6 && odd) k_plain_df<6, true><<<grid, NT, 0, st>>>(a);
    else if (nge == 6) k_plain_df<6, false><<<grid, NT, 0, st>>>(a);
    else if (odd) k_plain_df<0, true><<<grid, NT, 0, st>>>(a);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace cpl
