// threej.cu -- (j1 j2 j3; 0 -1 1) columns from the g table (App. B).
//
// With J = j1 + j2 + j3, J_{-++} = -j1 + j2 + j3, J_{+-+} = j1 - j2 + j3,
// J_{++-} = j1 + j2 - j3 and X(j1, j2, j3) = (j1 j2 j3; 0 0 0):
//   even J (Eq. joneevensimp):
//     (j1 j2 j3; 0 -1 1) = sqrt((j2+1)(j3+1) / (j2 j3))
//                          (1 - (J+2)(J_{-++}+1) / (2 (j2+1)(j3+1))) X(j1, j2, j3)
//   odd J (Eq. joneodd):
//     (j1 j2 j3; 0 -1 1) = -1/2 sqrt((J+2)(J_{-++}+1)(J_{+-+}+1) J_{++-} / (j2 (j2+1) j3 (j3+1)))
//                          X(j1, j2, j3 + 1)
// and X of an even triple (j1, j2, j3), L = 2p (Eq. 000_sq_main with the
// h table):  X = (-1)^p sqrt(g(p - j1) g(p - j2) g(p - j3) h(p)),
// h(p) = 1 / ((2p + 1) g(p)).  The square roots are taken once per table
// entry (k_sqrt_tables, held as FP32 pairs), and an element is four or five
// double-float products on the FP32 pipe, converted to FP64 by widening both
// parts from their bits and one FP64 addition: GB300's FP64 pipe would
// otherwise bound the kernel.  (With
// separate roots of the integer factors and the bracket of the even case
// formed as 1 - (J+2)(J_{-++}+1) / (2 (j2+1)(j3+1)) in double-float, an
// element took seven or eight products and a sum: 0.113 ms instead of
// ~0.09 for 4096 rows at j2, j3 in [1000, 3000].)
#include <cuda_runtime.h>

#include "dd.cuh"
#include "internal.h"

namespace cpl {
namespace {

// Square-root tables as double-float (FP32 pairs, ~48 bits), for p < np1,
// each root taken once in FP64: sg = sqrt g(p), sh = sqrt h(p) for the (0 0 0)
// symbol of an even triple, and for the odd-J formula, whose square root
// (J+2)(J_{-++}+1)(J_{+-+}+1) J_{++-} g(p'-j1) g(p'-j2) g(p'-j3-1) h(p')
// (2p' = J + 1) regroups factor by factor: J + 2 = 2p' + 1 cancels the
// (2p' + 1) of h, and J_{-++}+1 = 2(p'-j1), J_{+-+}+1 = 2(p'-j2),
// J_{++-} = 2(p'-j3-1) + 1 pair with the g beside them:
//   sa = sqrt(2p g(p)), sb = sqrt((2p+1) g(p)), sc = 1 / sqrt(g(p)).
__global__ void k_sqrt_tables(const double *__restrict__ g, const double *__restrict__ h, int np1, float2 *sg,
                              float2 *sh, float2 *sa, float2 *sb, float2 *sc) {
    auto split = [](double x) {
        const float hi = (float)x;
        return make_float2(hi, (float)(x - (double)hi));
    };
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < np1; q += gridDim.x * blockDim.x) {
        const double gq = g[q];
        sg[q] = split(sqrt(gq));
        sh[q] = split(sqrt(h[q]));
        sa[q] = split(sqrt(2.0 * q * gq));
        sb[q] = split(sqrt((2.0 * q + 1.0) * gq));
        sc[q] = split(1.0 / sqrt(gq));
    }
}

__device__ __forceinline__ dfl ld(const float2 *__restrict__ t, int i) {
    const float2 v = t[i];
    return {v.x, v.y};
}
__device__ __forceinline__ dfl dfl_of(double x) {
    const float hi = (float)x;
    return {hi, (float)(x - (double)hi)};
}

struct SqrtTabs {
    const float2 *sg, *sh, *sa, *sb, *sc;
};

// (j1 j2 j3; 0 -1 1) for j1 in [|j2 - j3|, j2 + j3] (J = j1 + j2 + j3):
//   even J: ce N X(j1, j2, j3), N = 2(j2+1)(j3+1) - (J+2)(J_{-++}+1) exact
//           (a difference of two exact products of integers below 2^24) and
//           ce = sqrt((j2+1)(j3+1) / (j2 j3)) / (2 (j2+1)(j3+1));
//   odd J:  so (-1)^p' sa(p'-j1) sa(p'-j2) sb(p'-j3-1) sc(p'),
//           so = -1/2 / sqrt(j2 (j2+1) j3 (j3+1))
// (J_{++-} >= 1 for odd J, so (j1, j2, j3 + 1) is a triangle).
__device__ __forceinline__ double m11(const SqrtTabs &T, int j1, int j2, int j3, dfl ce, dfl so) {
    const int J = j1 + j2 + j3;
    dfl v;
    if ((J & 1) == 0) {
        const int p = J >> 1;
        const dfl x = df_mul(df_mul(ld(T.sg, p - j1), ld(T.sg, p - j2)), df_mul(ld(T.sg, p - j3), ld(T.sh, p)));
        const dfl nn = df_add(df_int_prod(2 * (j2 + 1), j3 + 1), df_neg(df_int_prod(J + 2, j2 + j3 - j1 + 1)));
        v = df_mul(df_mul(ce, nn), x);
        if (p & 1) v = df_neg(v);
    } else {
        const int p = (J + 1) >> 1;
        const dfl x = df_mul(df_mul(ld(T.sa, p - j1), ld(T.sa, p - j2)), df_mul(ld(T.sb, p - j3 - 1), ld(T.sc, p)));
        v = df_mul(so, x);
        if (p & 1) v = df_neg(v);
    }
    // FP64 from the pair: its parts widened from their bits, one FP64 addition
    return df_to_double(v);
}

// Per-row constants of m11 in FP64, one thread per row (apart from the row
// kernel, whose blocks would otherwise wait on one thread's FP64 square
// roots and divisions): cst[q] = (ce.h, ce.l, so.h, so.l).
__global__ void k_threej_consts(const int *__restrict__ j2s, const int *__restrict__ j3s, int n, float4 *cst) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const double d2 = j2s[q], d3 = j3s[q];
    const dfl ce = dfl_of(sqrt((d2 + 1.0) * (d3 + 1.0) / (d2 * d3)) / (2.0 * (d2 + 1.0) * (d3 + 1.0)));
    const dfl so = dfl_of(-0.5 / sqrt(d2 * (d2 + 1.0) * d3 * (d3 + 1.0)));
    cst[q] = make_float4(ce.h, ce.l, so.h, so.l);
}

// One row (j2, j3) per block.  Each thread takes two neighbours j1, j1 + 1
// (at every step all lanes of a warp have the same parity of J, so the two
// formulas do not diverge) and stores them as one 16-byte pair; a row that
// starts off a 16-byte boundary takes its first element alone.
__global__ void __launch_bounds__(256) k_threej_m11(SqrtTabs T, const int *__restrict__ j2s,
                                                    const int *__restrict__ j3s, const float4 *__restrict__ cst,
                                                    double *out, long long stride) {
    const int q = blockIdx.x;
    const int j2 = j2s[q], j3 = j3s[q];
    const int jmin = abs(j2 - j3), jmax = j2 + j3;
    double *row = out + (long long)q * stride;
    const float4 c4 = cst[q];
    const dfl ce = {c4.x, c4.y}, so = {c4.z, c4.w};
    auto value = [&](long long idx) {
        const int j1 = jmin + (int)idx;
        return j1 > jmax ? 0.0 : m11(T, j1, j2, j3, ce, so);
    };
    const int off = (reinterpret_cast<unsigned long long>(row) & 15) ? 1 : 0;
    if (off && threadIdx.x == 0) row[0] = value(0);
    for (long long pair = threadIdx.x; off + 2 * pair < stride; pair += blockDim.x) {
        const long long idx = off + 2 * pair;
        const double v0 = value(idx);
        if (idx + 1 < stride) {
            const double v1 = value(idx + 1);
            *reinterpret_cast<double2 *>(row + idx) = make_double2(v0, v1);
        } else {
            row[idx] = v0;
        }
    }
}

}  // namespace

cudaError_t launch_sqrt_tables(const double *g, const double *h, int np1, float2 *tab, cudaStream_t st) {
    k_sqrt_tables<<<(np1 + 255) / 256, 256, 0, st>>>(g, h, np1, tab, tab + np1, tab + 2 * np1, tab + 3 * np1,
                                                      tab + 4 * np1);
    return cudaGetLastError();
}

cudaError_t launch_threej_consts(const int *j2, const int *j3, int n, float4 *cst, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_threej_consts<<<(n + 255) / 256, 256, 0, st>>>(j2, j3, n, cst);
    return cudaGetLastError();
}

cudaError_t launch_threej_m11(const float2 *tab, int np1, const int *j2, const int *j3, int n, const float4 *cst,
                              double *out, long long stride, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const SqrtTabs T{tab, tab + np1, tab + 2 * np1, tab + 3 * np1, tab + 4 * np1};
    k_threej_m11<<<n, 256, 0, st>>>(T, j2, j3, cst, out, stride);
    return cudaGetLastError();
}

}  // namespace cpl
