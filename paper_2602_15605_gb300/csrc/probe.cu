// probe.cu -- FP64 pipe throughput probe (the denominator of the plain path's
// roofline).
//
// The plain path's kernels are bound by the FP64 pipe; the peak they are
// measured against is the pipe's sustained rate of fused multiply-adds on
// this GPU, which this kernel measures.  Every thread runs the inner loop of
// a register-tiled product, acc[r][c] = fma(x[r], y[c], acc[r][c]) over a
// 4 x 4 tile, with all three operands in registers as in the contraction
// kernels (an earlier form with chains a = a * m + c, m and c kernel
// parameters, reached only 0.84 of the contraction kernel's own rate).  16
// independent accumulators per thread and several warps per scheduler cover
// the pipe's latency.  Nothing is read from memory; the only store is
// conditional on a value the sums never reach, which keeps the compiler from
// removing them.
#include <cuda_runtime.h>

#include <string>

#include "internal.h"

namespace cpl {
namespace {

constexpr int PROBE_NT = 256;     // threads per block
constexpr int PROBE_T = 4;        // register tile: PROBE_T x PROBE_T accumulators per thread
constexpr int PROBE_UNROLL = 4;   // tile updates per loop iteration

__global__ void __launch_bounds__(PROBE_NT) k_fp64_probe(int iters, double m, double c, double *sink) {
    double x[PROBE_T], y[PROBE_T], acc[PROBE_T][PROBE_T];
#pragma unroll
    for (int q = 0; q < PROBE_T; ++q) {
        x[q] = m + 1e-9 * (threadIdx.x + q);
        y[q] = c * (q + 1);
    }
#pragma unroll
    for (int r = 0; r < PROBE_T; ++r)
#pragma unroll
        for (int q = 0; q < PROBE_T; ++q) acc[r][q] = 0.0;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < PROBE_UNROLL; ++u)
#pragma unroll
            for (int r = 0; r < PROBE_T; ++r)
#pragma unroll
                for (int q = 0; q < PROBE_T; ++q) acc[r][q] = fma(x[r], y[q], acc[r][q]);
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
    if (n_blocks > (1 << 20) || iters > (1 << 24)) return fail(CPL_ERR_RANGE, "cpl_probe_fp64: too much work");
    k_fp64_probe<<<n_blocks, PROBE_NT, 0, (cudaStream_t)stream>>>(iters, 0.999999, 1e-6, sink);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(CPL_ERR_CUDA, std::string("probe launch failed: ") + cudaGetErrorString(e));
    *flop = 2.0 * PROBE_T * PROBE_T * PROBE_UNROLL * (double)iters * PROBE_NT * (double)n_blocks;
    return CPL_OK;
}
