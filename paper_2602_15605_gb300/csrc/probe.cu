// probe.cu -- FP64 pipe throughput probe (the denominator of the plain path's
// roofline).
//
// The plain path's kernels are bound by the FP64 pipe; the peak they are
// measured against is the pipe's sustained rate of fused multiply-adds on
// this GPU, which this kernel measures.  Every thread runs the inner loop of
// a register-tiled product fed from shared memory, as the contraction
// kernels do: per k, 4 + 4 operands loaded from a 32-deep panel and a 4 x 4
// tile of accumulators acc[r][c] = fma(a[r], b[c], acc[r][c]).  (Measured on
// GB300: streams of FP64 fused multiply-adds whose operands all stay in
// registers -- the same tile with loop-invariant operands, or independent
// chains a = a m + c -- issue at only 0.84 of the rate this form reaches,
// 0.997 of 2 FMA per clock per SM.)  Nothing is read from global memory; the
// only store is conditional on a value the sums never reach, which keeps
// the compiler from removing them.
#include <cuda_runtime.h>

#include <string>

#include "internal.h"

namespace cpl {
namespace {

constexpr int PROBE_NT = 256;     // threads per block: a 16 x 16 grid of 4 x 4 tiles
constexpr int PROBE_T = 4;        // register tile: PROBE_T x PROBE_T accumulators per thread
constexpr int PROBE_KP = 32;      // depth of the shared-memory panel
constexpr int PROBE_PASSES = 2;   // panel passes per iteration: 2 x 32 k x 16 FMAs = 1024 per thread

__global__ void __launch_bounds__(PROBE_NT) k_fp64_probe(int iters, double m, double c, double *sink) {
    __shared__ double sa[PROBE_KP][16 * PROBE_T], sb[PROBE_KP][16 * PROBE_T];
    for (int e = threadIdx.x; e < PROBE_KP * 16 * PROBE_T; e += PROBE_NT) {
        (&sa[0][0])[e] = m + 1e-9 * e;
        (&sb[0][0])[e] = c * (1 + (e & 7));
    }
    __syncthreads();
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[PROBE_T][PROBE_T];
#pragma unroll
    for (int r = 0; r < PROBE_T; ++r)
#pragma unroll
        for (int q = 0; q < PROBE_T; ++q) acc[r][q] = 0.0;
    for (int it = 0; it < iters * PROBE_PASSES; ++it) {
#pragma unroll 4
        for (int k = 0; k < PROBE_KP; ++k) {
            double a[PROBE_T], b[PROBE_T];
#pragma unroll
            for (int r = 0; r < PROBE_T; ++r) a[r] = sa[k][ty + 16 * r];
#pragma unroll
            for (int q = 0; q < PROBE_T; ++q) b[q] = sb[k][tx + 16 * q];
#pragma unroll
            for (int r = 0; r < PROBE_T; ++r)
#pragma unroll
                for (int q = 0; q < PROBE_T; ++q) acc[r][q] = fma(a[r], b[q], acc[r][q]);
        }
    }
    double s = 0.0;
#pragma unroll
    for (int r = 0; r < PROBE_T; ++r)
#pragma unroll
        for (int q = 0; q < PROBE_T; ++q) s += acc[r][q];
    if (s == -1.0) sink[0] = s;   // never true: every term is positive
}

}  // namespace
}  // namespace cpl

using namespace cpl;

extern "C" cpl_status cpl_probe_fp64(int n_blocks, int iters, double *sink, double *flop, void *stream) {
    if (n_blocks < 1 || iters < 1 || !sink || !flop)
        return fail(CPL_ERR_ARG, "cpl_probe_fp64 needs n_blocks >= 1, iters >= 1 and non-NULL sink and flop");
    if (n_blocks > (1 << 20) || iters > (1 << 20)) return fail(CPL_ERR_RANGE, "cpl_probe_fp64: too much work");
    k_fp64_probe<<<n_blocks, PROBE_NT, 0, (cudaStream_t)stream>>>(iters, 0.999999, 1e-6, sink);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(CPL_ERR_CUDA, std::string("probe launch failed: ") + cudaGetErrorString(e));
    *flop = 2.0 * PROBE_T * PROBE_T * PROBE_KP * PROBE_PASSES * (double)iters * PROBE_NT * (double)n_blocks;
    return CPL_OK;
}
