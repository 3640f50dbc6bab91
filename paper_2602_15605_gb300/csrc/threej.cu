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
// entry (sqrt g, sqrt h, sqrt n, held as FP32 pairs), and an element is a
// few double-float products on the FP32 pipe, converted to FP64 with integer
// operations: GB300's FP64 pipe would otherwise bound the kernel.
#include <cuda_runtime.h>

#include "dd.cuh"
#include "internal.h"

namespace cpl {
namespace {

// Square-root tables as double-float (FP32 pairs, ~48 bits): sg = sqrt g,
// sh = sqrt h for p < np1, sn = sqrt n for n < nn; each root taken once in FP64.
__global__ void k_sqrt_tables(const double *__restrict__ g, const double *__restrict__ h, int np1, int nn,
                              float2 *sg, float2 *sh, float2 *sn) {
    auto split = [](double x) {
        const float hi = (float)x;
        return make_float2(hi, (float)(x - (double)hi));
    };
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < np1 || q < nn; q += gridDim.x * blockDim.x) {
        if (q < np1) {
            sg[q] = split(sqrt(g[q]));
            sh[q] = split(sqrt(h[q]));
        }
        if (q < nn) sn[q] = split(sqrt((double)q));
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

// (0 0 0) symbol of a triple with even sum 2p (the caller guarantees the
// triangle), as a product of square-rooted table entries
__device__ __forceinline__ dfl x000(const float2 *__restrict__ sg, const float2 *__restrict__ sh, int a, int b, int c) {
    const int p = (a + b + c) >> 1;
    const dfl x = df_mul(df_mul(ld(sg, p - a), ld(sg, p - b)), df_mul(ld(sg, p - c), ld(sh, p)));
    return (p & 1) ? df_neg(x) : x;
}

__global__ void __launch_bounds__(256) k_threej_m11(const float2 *__restrict__ sg, const float2 *__restrict__ sh,
                                                    const float2 *__restrict__ sn, const int *__restrict__ j2s,
                                                    const int *__restrict__ j3s, double *out, long long stride) {
    __shared__ dfl cst[3];
    const int q = blockIdx.x;
    const int j2 = j2s[q], j3 = j3s[q];
    const int jmin = abs(j2 - j3), jmax = j2 + j3;
    double *row = out + (long long)q * stride;
    if (threadIdx.x == 0) {
        // per-row constants, in FP64 once: the even-J prefactor, 1 / (2 (j2+1)(j3+1))
        // and the odd-J normalisation
        const double d2 = j2, d3 = j3;
        cst[0] = dfl_of(sqrt((d2 + 1.0) * (d3 + 1.0) / (d2 * d3)));
        cst[1] = dfl_of(1.0 / (2.0 * (d2 + 1.0) * (d3 + 1.0)));
        cst[2] = dfl_of(-0.5 / sqrt(d2 * (d2 + 1.0) * d3 * (d3 + 1.0)));
    }
    __syncthreads();
    const dfl ev = cst[0], inv2 = cst[1], sod = cst[2];
    // each thread takes two neighbours j1, j1 + 1: at every step all lanes of a
    // warp have the same parity of J, so the two formulas do not diverge
    for (long long pair = threadIdx.x; 2 * pair < stride; pair += blockDim.x) {
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const long long idx = 2 * pair + t;
            if (idx >= stride) break;
            const int j1 = jmin + (int)idx;
            if (j1 > jmax) {
                row[idx] = 0.0;
                continue;
            }
            const int J = j1 + j2 + j3;
            const int Jmpp = j2 + j3 - j1, Jpmp = j1 - j2 + j3, Jppm = j1 + j2 - j3;
            dfl v;
            if ((J & 1) == 0) {
                // 1 - (J+2)(J_{-++}+1) / (2 (j2+1)(j3+1)); J + 2 and J_{-++} + 1 are exact in FP32 (< 2^24)
                const dfl tt = df_mul(df_mul(inv2, dfl{(float)(J + 2), 0.0f}), dfl{(float)(Jmpp + 1), 0.0f});
                const dfl f = df_add(dfl{1.0f, 0.0f}, df_neg(tt));
                v = df_mul(df_mul(ev, f), x000(sg, sh, j1, j2, j3));
            } else {
                // J_{++-} >= 1 here (odd, and j1 >= |j2 - j3|), so (j1, j2, j3 + 1) is a triangle
                const dfl r = df_mul(df_mul(ld(sn, J + 2), ld(sn, Jmpp + 1)), df_mul(ld(sn, Jpmp + 1), ld(sn, Jppm)));
                v = df_mul(df_mul(sod, r), x000(sg, sh, j1, j2, j3 + 1));
            }
            // FP64 from the pair with integer operations (the FP64 pipe stays idle)
            row[idx] = xdf_to_double(xdf{v.h, v.l, 0});
        }
    }
}

}  // namespace

cudaError_t launch_sqrt_tables(const double *g, const double *h, int np1, int nn, float2 *sg, float2 *sh, float2 *sn,
                               cudaStream_t st) {
    const int n = np1 > nn ? np1 : nn;
    k_sqrt_tables<<<(n + 255) / 256, 256, 0, st>>>(g, h, np1, nn, sg, sh, sn);
    return cudaGetLastError();
}

cudaError_t launch_threej_m11(const float2 *sg, const float2 *sh, const float2 *sn, const int *j2, const int *j3,
                              int n, double *out, long long stride, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_threej_m11<<<n, 256, 0, st>>>(sg, sh, sn, j2, j3, out, stride);
    return cudaGetLastError();
}

}  // namespace cpl
