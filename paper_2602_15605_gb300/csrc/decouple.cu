// decouple.cu -- mode decoupling: the underlying spectra from measured
// pseudo-spectra by solving Eq. pseudo_cl, one CTA per linear system.
//
// Systems per window (App. A kernels, library slot order):
//   TT:  K^TT x = pcl^TT          TE: K^TE x = pcl^TE       EB: K^EB x = pcl^EB
//   EE/BB: [[K^EE, K^EEBB], [K^EEBB, K^EE]] [x^EE; x^BB] = [pcl^EE; pcl^BB]
// The block system is symmetric under exchanging its halves, so the
// orthogonal change of basis (EE + BB, EE - BB) splits it exactly into
//   (K^EE + K^EEBB) s = pcl^EE + pcl^BB,   (K^EE - K^EEBB) t = pcl^EE - pcl^BB,
// x^EE = (s + t) / 2, x^BB = (s - t) / 2: two n x n solves instead of one
// 2n x 2n solve (a quarter of the flops), each on its own CTA.  The two CTAs
// add s/2 and +-t/2 into zeroed outputs with atomics; two addends onto zero
// give the same rounded sum in either order, so the result is deterministic.
//
// Each CTA holds the augmented matrix [K | pcl^T] (n rows, ld = n + n_rhs
// padded to odd for conflict-free column reads) in shared memory when it
// fits, else in a global workspace slice (L2-resident at these sizes), and
// runs Gaussian elimination with partial pivoting (the largest |a_ik|, the
// lowest row on ties) followed by back substitution, all in FP64.  A zero or
// non-finite pivot marks the system singular: info = k + 1 and NaN outputs.
#include <cmath>

#include "internal.h"

namespace cpl {
namespace {

constexpr int DC_THREADS = 512;
constexpr int DC_WARPS = DC_THREADS / 32;

__device__ __forceinline__ void argmax_combine(double &v, int &i, double v2, int i2) {
    if (v2 > v || (v2 == v && i2 < i)) {
        v = v2;
        i = i2;
    }
}

__global__ void __launch_bounds__(DC_THREADS) k_decouple(DecoupleArgs a) {
    extern __shared__ __align__(16) double dsm[];
    __shared__ double red_v[DC_WARPS];
    __shared__ int red_i[DC_WARPS];
    __shared__ int piv_s, bad_s;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n = a.n, ld = a.ld, R = a.n_rhs, nf = a.n_fields;
    double *A = a.ws ? a.ws + (size_t)blockIdx.x * a.ws_stride : dsm;

    for (long long sys = blockIdx.x; sys < a.n_sys; sys += gridDim.x) {
        const int w = (int)(sys / a.sys_per_window), q = (int)(sys % a.sys_per_window);
        const int kind = a.kind[q];
        const double *K1 = a.M + ((size_t)w * a.nspec + a.slot1[q]) * (size_t)n * n;
        const double *K2 = a.M + ((size_t)w * a.nspec + a.slot2[q]) * (size_t)n * n;
        const double *P = a.pcl + (size_t)w * R * nf * n;
        const int f1 = a.field1[q], f2 = a.field2[q];

        // ---- load [K | pcl^T]
        for (int idx = tid; idx < n * n; idx += DC_THREADS) {
            const int i = idx / n, j = idx - i * n;
            double v = K1[idx];
            if (kind == 1) v = v + K2[idx];
            else if (kind == 2) v = v - K2[idx];
            A[(size_t)i * ld + j] = v;
        }
        for (int idx = tid; idx < R * n; idx += DC_THREADS) {
            const int r = idx / n, i = idx - r * n;
            double b = P[((size_t)r * nf + f1) * n + i];
            if (kind == 1) b = b + P[((size_t)r * nf + f2) * n + i];
            else if (kind == 2) b = b - P[((size_t)r * nf + f2) * n + i];
            A[(size_t)i * ld + n + r] = b;
        }
        __syncthreads();

        // ---- elimination with partial pivoting
        int bad = 0;
        for (int k = 0; k < n; ++k) {
            double best = -1.0;
            int bi = n;
            for (int i = k + tid; i < n; i += DC_THREADS) {
                const double v = fabs(A[(size_t)i * ld + k]);
                if (v > best) {   // NaN never wins; rows visited in increasing order
                    best = v;
                    bi = i;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double v2 = __shfl_xor_sync(0xffffffffu, best, o);
                const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
                argmax_combine(best, bi, v2, i2);
            }
            if (lane == 0) {
                red_v[warp] = best;
                red_i[warp] = bi;
            }
            __syncthreads();
            if (warp == 0) {
                double v = lane < DC_WARPS ? red_v[lane] : -1.0;
                int i = lane < DC_WARPS ? red_i[lane] : n;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const double v2 = __shfl_xor_sync(0xffffffffu, v, o);
                    const int i2 = __shfl_xor_sync(0xffffffffu, i, o);
                    argmax_combine(v, i, v2, i2);
                }
                if (lane == 0) {
                    piv_s = i;
                    bad_s = (v > 0.0 && v <= 1.7976931348623157e308) ? 0 : k + 1;
                }
            }
            __syncthreads();
            if (bad_s) {
                bad = bad_s;
                break;
            }
            const int p = piv_s;
            if (p != k) {
                for (int j = k + tid; j < ld; j += DC_THREADS) {
                    const double t = A[(size_t)k * ld + j];
                    A[(size_t)k * ld + j] = A[(size_t)p * ld + j];
                    A[(size_t)p * ld + j] = t;
                }
                __syncthreads();
            }
            const double rinv = 1.0 / A[(size_t)k * ld + k];
            const double *rowk = A + (size_t)k * ld;
            for (int i = k + 1 + warp; i < n; i += DC_WARPS) {
                double *rowi = A + (size_t)i * ld;
                const double l = rowi[k] * rinv;
                for (int j = k + 1 + lane; j < ld; j += 32) rowi[j] = fma(-l, rowk[j], rowi[j]);
            }
            __syncthreads();
        }

        // ---- back substitution on the n_rhs columns
        if (!bad) {
            for (int k = n - 1; k >= 0; --k) {
                const double ukk = A[(size_t)k * ld + k];
                for (int r = tid; r < R; r += DC_THREADS) A[(size_t)k * ld + n + r] /= ukk;
                __syncthreads();
                for (int idx = tid; idx < k * R; idx += DC_THREADS) {
                    const int i = idx / R, r = idx - i * R;
                    double *bi = A + (size_t)i * ld + n + r;
                    *bi = fma(-A[(size_t)i * ld + k], A[(size_t)k * ld + n + r], *bi);
                }
                __syncthreads();
            }
        }

        // ---- outputs
        double *O = a.out + (size_t)w * R * nf * n;
        for (int idx = tid; idx < R * n; idx += DC_THREADS) {
            const int r = idx / n, i = idx - r * n;
            const double x = bad ? __longlong_as_double(0x7ff8000000000000LL) : A[(size_t)i * ld + n + r];
            double *o1 = O + ((size_t)r * nf + f1) * n + i;
            if (kind == 0) {
                *o1 = x;
            } else {
                double *o2 = O + ((size_t)r * nf + f2) * n + i;
                atomicAdd(o1, 0.5 * x);
                atomicAdd(o2, (kind == 1 ? 0.5 : -0.5) * x);
            }
        }
        if (tid == 0 && a.info) a.info[sys] = bad;
        __syncthreads();   // A is reused by the CTA's next system
    }
}

}  // namespace

int decouple_smem_limit() { return 226 * 1024; }   // dynamic part; the static reduction scratch fits in the rest

cudaError_t launch_decouple(const DecoupleArgs &a, int grid, size_t smem, cudaStream_t st) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_decouple, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             decouple_smem_limit());
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_decouple<<<grid, DC_THREADS, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t decouple_blocks_per_sm(size_t smem, int *n) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, k_decouple, DC_THREADS, smem);
}

}  // namespace cpl
