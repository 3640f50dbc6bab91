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
// Two solvers, both Gaussian elimination with partial pivoting (the largest
// |a_ik|, the lowest row on ties):
//
// * Refined (few right-hand sides): GB300's FP64 pipe issues 2 FMA/clk/SM
//   against 128 for FP32, so the O(n^3) factorisation runs in FP32 on
//   K 2^-e (a power-of-two scale, exact) and the answer is brought to FP64
//   accuracy by iterative refinement: x += K^-1 r with the FP32 factors,
//   r = b - K x in FP64 from the FP64 matrix (from 8 right-hand sides only
//   the first, and that one on the FP64 and FP32 pipes at once, some
//   right-hand sides as FP64 chains and the others as error-free
//   triple-float products; each later residual is the previous one minus K
//   times the update x received, in double-float on the FP32 pipe), until
//   max|r| <= max|x| |K|_inf eps sqrt(n) for every right-hand side (the
//   stopping rule of LAPACK's mixed-precision dsgesv, at most 30 steps).
//   Each right-hand side is scaled by a power of two before it is rounded to
//   FP32.  A zero FP32 pivot, a non-finite value or no convergence sends
//   the system to the FP64 solver.
// * FP64: elimination on the augmented matrix [K | pcl^T] (ld = n + n_rhs,
//   padded to odd for conflict-free column reads) and back substitution.
//   A zero or non-finite pivot marks the system singular: info = k + 1 and
//   NaN outputs.
//
// Matrices live in shared memory when they fit, else in a per-CTA slice of a
// global workspace (L2-resident at these sizes).  Every reduction has a fixed
// order, so results are deterministic.
#include <cuda_bf16.h>

#include <cmath>

#include <algorithm>

#include "ctx.h"
#include "internal.h"

namespace cpl {
namespace {

constexpr int DC_THREADS = 512;
constexpr int DC_WARPS = DC_THREADS / 32;
constexpr int IR_ITMAX = 30;
constexpr int IR_RB = 8;          // right-hand sides per pass of a residual thread
constexpr int IR_INC_MIN = 8;     // right-hand sides from which the residuals after the first are double-float updates
static_assert(IR_INC_MIN > 1, "the update errors share shared memory with the one-column residual's slices");
constexpr double EPS64 = 1.1102230246251565e-16;   // 2^-53

// One system: K = K1 (+ or -) K2 and b = P[f1] (+ or -) P[f2] by kind.
struct SysView {
    const double *K1, *K2, *P;
    int kind, f1, f2, nf, n;
    __device__ __forceinline__ double k(size_t idx) const {
        double v = K1[idx];
        if (kind == 1) v = v + K2[idx];
        else if (kind == 2) v = v - K2[idx];
        return v;
    }
    __device__ __forceinline__ double b(int r, int i) const {
        double v = P[((size_t)r * nf + f1) * n + i];
        if (kind == 1) v = v + P[((size_t)r * nf + f2) * n + i];
        else if (kind == 2) v = v - P[((size_t)r * nf + f2) * n + i];
        return v;
    }
};

struct Scratch {           // static shared scalars of the block reductions
    double red_v[DC_WARPS];
    int red_i[DC_WARPS];
    double pv;
    int piv;
    double wnorm[2][DC_WARPS];            // per-warp |K|_inf and max |K_ij| candidates
    unsigned long long pkey[2][DC_WARPS]; // per-warp pivot keys of the refined solver's panel (2 buffers)
    float prow[32], krow[32];             // the panel's pivot row and the row it replaces
};

// a[m] and a[m] = v for a run-time m, without indexing the register array
// (which would place it in local memory)
template <int N>
__device__ __forceinline__ float pick(const float (&a)[N], int m) {
    float v = 0.f;
#pragma unroll
    for (int q = 0; q < N; ++q) v = q == m ? a[q] : v;
    return v;
}
template <int N>
__device__ __forceinline__ void put(float (&a)[N], int m, float v) {
#pragma unroll
    for (int q = 0; q < N; ++q) a[q] = q == m ? v : a[q];
}

__device__ __forceinline__ void argmax_combine(double &v, int &i, double v2, int i2) {
    if (v2 > v || (v2 == v && i2 < i)) {
        v = v2;
        i = i2;
    }
}

__device__ __forceinline__ void warp_argmax(double &v, int &i) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double v2 = __shfl_xor_sync(0xffffffffu, v, o);
        const int i2 = __shfl_xor_sync(0xffffffffu, i, o);
        argmax_combine(v, i, v2, i2);
    }
}

// Block-wide argmax of per-thread (v, i); all threads find the winner in
// sc.piv / sc.pv on return.
__device__ __forceinline__ void block_argmax(double v, int i, int nfill, Scratch &sc) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    warp_argmax(v, i);
    if (lane == 0) {
        sc.red_v[warp] = v;
        sc.red_i[warp] = i;
    }
    __syncthreads();
    if (warp == 0) {
        v = lane < DC_WARPS ? sc.red_v[lane] : -1.0;
        i = lane < DC_WARPS ? sc.red_i[lane] : nfill;
        warp_argmax(v, i);
        if (lane == 0) {
            sc.piv = i;
            sc.pv = v;
        }
    }
    __syncthreads();
}

__device__ __forceinline__ bool finite_pos(double v) { return v > 0.0 && v <= 1.7976931348623157e308; }


__device__ __forceinline__ unsigned long long pivot_key(float v, int i) {
    return ((unsigned long long)__float_as_uint(fabsf(v)) << 32) | (unsigned long long)(0xFFFFFFFFu - (unsigned)i);
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    return v;
}

// The refined solver's factorisation: LAPACK's right-looking blocked LU
// with 32-column panels of fl32(K) in L (row-major, ld = np + 4), on the
// system padded to np = 32 NC with identity rows and columns
// (the padding never pivots and leaves the n x n factors unchanged):
//   panel: 32 elimination steps on its columns with the panel in registers
//          (warp w holds rows w + 16 m, lane = column).  Each pivot is found
//          while the previous step updates that column: the lane that owns
//          it offers (|a|, ~row) as one 64-bit key over its warp's rows, and
//          every thread takes the largest of the 16 keys after the barrier
//          (largest |a|, lowest row on ties, independent of timing).  The
//          pivot row and the row it replaces pass through shared memory, the
//          rest of the two rows is swapped in place, and each row's
//          multiplier reaches its warp's lanes by a shuffle: two barriers a
//          step and no shared-memory traffic per element (with the panel in
//          shared memory every element's load, update and store sat on the
//          step's critical path, ~2.8k clocks a step at n = 160, against
//          ~1.7k).  Measured slower: 8 warps with twice the rows each, and one
//          barrier a step with every warp posting its candidate row (the
//          extra selects and stores cost more than the barrier saved);
//   U12 = L11^-1 A12: one thread per column, the 32 unknowns in registers;
//   A22 -= L21 U12: register tiles of 4 x 4, 32-deep, float4 shared loads.
// perm[i] is the original row now at position i, dinv[k] = 1 / U_kk.  Its
// own function (not inlined) so that the panel's registers are allocated
// apart from the refinement's arrays.  Returns false on a zero or non-finite
// pivot.
template <int NC>
__device__ __noinline__ bool lu_fp32(float *L, int *perm, float *dinv, Scratch &sc) {
    constexpr int NP = 32 * NC;
    constexpr int LDF = NP + 4;
    constexpr int RPW = NP / DC_WARPS;   // panel rows per warp
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
#pragma unroll 1
    for (int c = 0; c < NC; ++c) {
        const int k0 = 32 * c;
        // the panel in registers: warp w holds rows w + DC_WARPS m, lane =
        // column k0 + lane
        float a[RPW];
#pragma unroll
        for (int m = 0; m < RPW; ++m) a[m] = L[(size_t)(warp + DC_WARPS * m) * LDF + k0 + lane];
        if (lane == 0) {   // pivot key of column k0 over this warp's rows >= k0
            unsigned long long best = 0ull;
#pragma unroll
            for (int m = 0; m < RPW; ++m) {
                const int i = warp + DC_WARPS * m;
                const unsigned long long q = pivot_key(a[m], i);
                if (i >= k0) best = q > best ? q : best;
            }
            sc.pkey[0][warp] = best;
        }
        __syncthreads();
        for (int t = 0; t < 32; ++t) {
            const int k = k0 + t;
            const unsigned long long kk = warp_max_u64(lane < DC_WARPS ? sc.pkey[t & 1][lane] : 0ull);
            const int p = (int)(0xFFFFFFFFu - (unsigned)(kk & 0xFFFFFFFFull));
            const float pv = __uint_as_float((unsigned)(kk >> 32));
            if (!(pv > 0.f && pv <= 3.4028234663852886e38f)) return false;   // the same decision in every thread
            const int wk = k % DC_WARPS, mk = k / DC_WARPS, wp = p % DC_WARPS, mp = p / DC_WARPS;
            // rows p and k of the panel through shared memory
            if (warp == wp) sc.prow[lane] = pick(a, mp);
            if (warp == wk && p != k) sc.krow[lane] = pick(a, mk);
            __syncthreads();
            const float pr = sc.prow[lane];   // the pivot row's entry in this lane's column
            if (p != k) {
                if (warp == wk) put(a, mk, pr);
                if (warp == wp) put(a, mp, sc.krow[lane]);
                // the rest of rows k and p (the factors left of the panel, the
                // trailing columns right of it) in place
                for (int j = tid; j < NP - 32; j += DC_THREADS) {
                    const int col = j < k0 ? j : j + 32;
                    const float tmp = L[(size_t)k * LDF + col];
                    L[(size_t)k * LDF + col] = L[(size_t)p * LDF + col];
                    L[(size_t)p * LDF + col] = tmp;
                }
                if (tid == 0) {
                    const int tmp = perm[k];
                    perm[k] = perm[p];
                    perm[p] = tmp;
                }
            }
            const float rinv = 1.0f / sc.prow[t];
            if (tid == 0) dinv[k] = rinv;
            // rows below k: the multiplier l = a_ik / a_kk replaces a_ik (lane
            // t), the columns right of it take a_ij - l a_kj; lane t + 1 keeps
            // the pivot key of column k + 1 over this warp's rows
            unsigned long long kbest = 0ull;
#pragma unroll
            for (int m = 0; m < RPW; ++m) {
                const int i = warp + DC_WARPS * m;
                if (i > k) {   // the same in every lane: rows at or above k are skipped whole
                    const float l = __shfl_sync(0xffffffffu, a[m], t) * rinv;
                    const float u = fmaf(-l, pr, a[m]);
                    if (lane > t) a[m] = u;
                    else if (lane == t) a[m] = l;
                    const unsigned long long q = pivot_key(u, i);
                    if (lane == t + 1) kbest = q > kbest ? q : kbest;
                }
            }
            if (t < 31 && lane == t + 1) sc.pkey[(t + 1) & 1][warp] = kbest;
            __syncthreads();
        }
#pragma unroll
        for (int m = 0; m < RPW; ++m) {
            const int i = warp + DC_WARPS * m;
            if (i >= k0) L[(size_t)i * LDF + k0 + lane] = a[m];
        }
        __syncthreads();
        if (c + 1 == NC) break;
        // U12 = L11^-1 A12, one thread per column of A12
        const int j1 = k0 + 32, ncol = NP - j1;
        for (int q = tid; q < ncol; q += DC_THREADS) {
            const int j = j1 + q;
            float u[32];
#pragma unroll
            for (int t = 0; t < 32; ++t) {
                float v = L[(size_t)(k0 + t) * LDF + j];
#pragma unroll
                for (int s2 = 0; s2 < t; ++s2) v = fmaf(-L[(size_t)(k0 + t) * LDF + k0 + s2], u[s2], v);
                u[t] = v;
            }
#pragma unroll
            for (int t = 1; t < 32; ++t) L[(size_t)(k0 + t) * LDF + j] = u[t];
        }
        __syncthreads();
        // A22 -= L21 U12 in 4 x 4 register tiles
        const int nb = ncol / 4;
        for (int q = tid; q < nb * nb; q += DC_THREADS) {
            const int rb = q / nb, cb = q - rb * nb;
            const int i0 = j1 + 4 * rb, c0 = j1 + 4 * cb;
            float acc[4][4];
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) acc[x][y] = 0.f;
#pragma unroll 8
            for (int s2 = 0; s2 < 32; ++s2) {
                const float4 u4 = *reinterpret_cast<const float4 *>(L + (size_t)(k0 + s2) * LDF + c0);
#pragma unroll
                for (int x = 0; x < 4; ++x) {
                    const float lv = L[(size_t)(i0 + x) * LDF + k0 + s2];
                    acc[x][0] = fmaf(lv, u4.x, acc[x][0]);
                    acc[x][1] = fmaf(lv, u4.y, acc[x][1]);
                    acc[x][2] = fmaf(lv, u4.z, acc[x][2]);
                    acc[x][3] = fmaf(lv, u4.w, acc[x][3]);
                }
            }
#pragma unroll
            for (int x = 0; x < 4; ++x) {
                float4 *d = reinterpret_cast<float4 *>(L + (size_t)(i0 + x) * LDF + c0);
                float4 v = *d;
                v.x -= acc[x][0];
                v.y -= acc[x][1];
                v.z -= acc[x][2];
                v.w -= acc[x][3];
                *d = v;
            }
        }
        __syncthreads();
    }
    return true;
}

// The exponent frexp would give for finite m > 0, read from the bits for a
// normal m.
__device__ __forceinline__ int frexp_exp(double m) {
    const int ex = (int)((__double_as_longlong(m) >> 52) & 0x7ff);
    if (ex != 0) return ex - 1022;
    int e;
    frexp(m, &e);
    return e;
}
// (double) f * 2^k with integer operations when f and the result are
// normal, else by conversion and ldexp.
__device__ __forceinline__ double widen_scaled(float f, int k) {
    const unsigned u = __float_as_uint(f);
    const int ef = (int)((u >> 23) & 0xff);
    const int ed = ef - 127 + 1023 + k;
    if (ef != 0 && ef != 255 && ed >= 1 && ed <= 2046) {
        const unsigned long long b = ((unsigned long long)(u >> 31) << 63) | ((unsigned long long)ed << 52) |
                                     ((unsigned long long)(u & 0x7fffffu) << 29);
        return __longlong_as_double((long long)b);
    }
    return ldexp((double)f, k);
}
// fl32(v 2^k) with integer operations (round to nearest even at the 29th
// fraction bit; a carry into the exponent field is the correct result) when
// v and the result are normal, else by ldexp and conversion.
__device__ __forceinline__ float narrow_scaled(double v, int k) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int ex = (int)((b >> 52) & 0x7ff);
    const int ef = ex - 1023 + 127 + k;
    if (ex != 0 && ex != 0x7ff && ef >= 1 && ef <= 253) {
        const unsigned long long m = b & 0x000fffffffffffffull;
        const unsigned long long rnd = m + 0x0fffffffull + ((m >> 29) & 1ull);
        const unsigned f = ((unsigned)ef << 23) + (unsigned)(rnd >> 29);
        return __uint_as_float(f | ((unsigned)(b >> 32) & 0x80000000u));
    }
    return (float)ldexp(v, k);
}

// The diagonal block's 32 dependent steps of the forward substitution for
// one or two right-hand sides (v1, v2: this lane's row), with the row's
// factors lk[t] in registers: step t takes y_t by a shuffle from lane t and
// the rows below it (lanes > t, rows < n) subtract l_it y_t.
template <bool TWO>
__device__ __forceinline__ void fwd_chain(float &v1, float &v2, const float (&lk)[32], int lane, bool row_ok, int tn) {
#pragma unroll
    for (int t = 0; t < 32; ++t) {
        if (t < tn) {
            const bool act = lane > t && row_ok;
            const float y1 = __shfl_sync(0xffffffffu, v1, t);
            const float y2 = TWO ? __shfl_sync(0xffffffffu, v2, t) : 0.f;
            if (act) {
                v1 = fmaf(-lk[t], y1, v1);
                if (TWO) v2 = fmaf(-lk[t], y2, v2);
            }
        }
    }
}
// The backward counterpart: step t (from the last) scales y_t by 1 / U_tt
// (dk[t]) on lane t and the rows above it (lanes < t) subtract u_it y_t.
template <bool TWO>
__device__ __forceinline__ void bwd_chain(float &v1, float &v2, const float (&uk)[32], const float (&dk)[32], int lane,
                                          int tn) {
#pragma unroll
    for (int t = 31; t >= 0; --t) {
        if (t < tn) {
            const float y1 = __shfl_sync(0xffffffffu, v1, t) * dk[t];
            const float y2 = TWO ? __shfl_sync(0xffffffffu, v2, t) * dk[t] : 0.f;
            if (lane == t) {
                v1 = y1;
                if (TWO) v2 = y2;
            } else if (lane < t) {
                v1 = fmaf(-uk[t], y1, v1);
                if (TWO) v2 = fmaf(-uk[t], y2, v2);
            }
        }
    }
}

// x += K^-1 r through the FP32 factors of lu_fp32, for every right-hand
// side: r is scaled by 2^-e (e the exponent of max |r|, whose bits are
// rmax[r], so the FP32 values neither overflow nor lose range), permuted
// into Y ([R][np] in shared memory), and the two substitutions run blocked
// by 32 rows.  In each block
// one warp per right-hand side (two at a time, interleaved) runs the block's
// 32 dependent steps on values held in registers, taking each step's y_k by
// a shuffle; then every thread applies the block to the rows below it (above
// it on the way back), one (right-hand side, row) pair at a time.  Every y_i
// receives the same FMAs in the same order as in an unblocked column sweep.
// A right-hand side whose residual is 0 or not finite is left unchanged;
// xnb[r] (zero on entry) gets the bits of max |x| (NaN bits for a NaN
// residual, which never converges).  With E (incremental residuals), the
// rounding error of each FP64 update x + 2^e y is kept: the update actually
// applied is 2^e (y - E), which the next residual subtracts.  From
// IR_BLK_MIN right-hand sides the block updates run in blk_update_fwd and
// blk_update_bwd.  The caller's barrier follows.
constexpr int YE_SKIP = -0x7fffffff - 1;   // ye[r]: residual 0 or infinite, no correction
constexpr int YE_NAN = YE_SKIP + 1;        // ye[r]: NaN residual
constexpr int IR_OB = 4;                    // right-hand sides per thread in the blocked updates
constexpr int IR_BLK_MIN = 16;              // right-hand sides from which the block updates are blocked

// Rows r0 .. r0 + cnt - 1 of every right-hand side take the forward block's
// 32 columns b0 .. b0 + 31.  A thread takes one row and up to IR_OB
// right-hand sides, the row's 32 factors loaded once (consecutive threads:
// consecutive rows of the same right-hand sides, whose y are broadcast).
// Each y_i receives its FMAs in column order, as in the one-pair-a-thread
// loop that serves fewer right-hand sides.  A function of its own, so that
// its registers do not crowd the dependent chains beside it.
__device__ __noinline__ void blk_update_fwd(int R, int NP, int LDF, int b0, int r0, int cnt, const float *L, float *Y,
                                            const int *ye) {
    const int tid = threadIdx.x;
    const int ngr = (R + IR_OB - 1) / IR_OB;
    for (int q = tid; q < ngr * cnt; q += DC_THREADS) {
        const int rg = q / cnt, ii = r0 + (q - rg * cnt);
        float lr[32];
        const float4 *Li = reinterpret_cast<const float4 *>(L + (size_t)ii * LDF + b0);
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const float4 l4 = Li[t];
            lr[4 * t] = l4.x;
            lr[4 * t + 1] = l4.y;
            lr[4 * t + 2] = l4.z;
            lr[4 * t + 3] = l4.w;
        }
#pragma unroll
        for (int u = 0; u < IR_OB; ++u) {
            const int r = rg * IR_OB + u;
            if (r >= R || ye[r] <= YE_NAN) continue;
            const float4 *yb = reinterpret_cast<const float4 *>(Y + (size_t)r * NP + b0);
            float y = Y[(size_t)r * NP + ii];
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const float4 y4 = yb[t];
                y = fmaf(-lr[4 * t], y4.x, y);
                y = fmaf(-lr[4 * t + 1], y4.y, y);
                y = fmaf(-lr[4 * t + 2], y4.z, y);
                y = fmaf(-lr[4 * t + 3], y4.w, y);
            }
            Y[(size_t)r * NP + ii] = y;
        }
    }
}

// Rows 0 .. b0 - 1 of every right-hand side take the backward block's
// columns b0 .. b0 + tn - 1, the last first; blocked over right-hand sides
// as in blk_update_fwd.
__device__ __noinline__ void blk_update_bwd(int R, int NP, int LDF, int b0, int tn, const float *L, float *Y,
                                            const int *ye) {
    const int tid = threadIdx.x;
    const int ngr = (R + IR_OB - 1) / IR_OB;
    for (int q = tid; q < ngr * b0; q += DC_THREADS) {
        const int rg = q / b0, ii = q - rg * b0;
        const float *Li = L + (size_t)ii * LDF + b0;
        if (tn == 32) {
            float lr[32];
            const float4 *L4 = reinterpret_cast<const float4 *>(Li);
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const float4 l4 = L4[t];
                lr[4 * t] = l4.x;
                lr[4 * t + 1] = l4.y;
                lr[4 * t + 2] = l4.z;
                lr[4 * t + 3] = l4.w;
            }
#pragma unroll
            for (int u = 0; u < IR_OB; ++u) {
                const int r = rg * IR_OB + u;
                if (r >= R || ye[r] <= YE_NAN) continue;
                const float4 *y4p = reinterpret_cast<const float4 *>(Y + (size_t)r * NP + b0);
                float y = Y[(size_t)r * NP + ii];
#pragma unroll
                for (int t = 7; t >= 0; --t) {
                    const float4 y4 = y4p[t];
                    y = fmaf(-lr[4 * t + 3], y4.w, y);
                    y = fmaf(-lr[4 * t + 2], y4.z, y);
                    y = fmaf(-lr[4 * t + 1], y4.y, y);
                    y = fmaf(-lr[4 * t], y4.x, y);
                }
                Y[(size_t)r * NP + ii] = y;
            }
        } else {
            for (int u = 0; u < IR_OB; ++u) {
                const int r = rg * IR_OB + u;
                if (r >= R || ye[r] <= YE_NAN) continue;
                const float *yb = Y + (size_t)r * NP + b0;
                float y = Y[(size_t)r * NP + ii];
                for (int t = tn - 1; t >= 0; --t) y = fmaf(-Li[t], yb[t], y);
                Y[(size_t)r * NP + ii] = y;
            }
        }
    }
}

template <int NC>
__device__ __noinline__ void ir_correct(int n, int R, const float *L, const int *perm, const float *dinv, double *xs,
                                        const double *rs, const unsigned long long *rmax, float *Y, int *ye,
                                        unsigned long long *xnb, __nv_bfloat16 *E) {
    constexpr int NP = 32 * NC;
    constexpr int LDF = NP + 4;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // element by element (the FP64 scaling and conversions spread over all warps)
    for (int q = tid; q < R * NP; q += DC_THREADS) {
        const int r = q / NP, i = q - r * NP;
        // max |r| from its bits: positive and finite, or 0 / inf (no
        // correction), or a NaN pattern (above the infinity's)
        const unsigned long long mb = rmax[r];
        const bool solve = mb != 0ull && mb < 0x7ff0000000000000ull;
        int e = 0;
        if (solve) e = frexp_exp(__longlong_as_double((long long)mb));
        float yv = 0.f;
        if (solve && i < n) {
            const double rv = rs[(size_t)r * n + perm[i]];
            yv = narrow_scaled(rv, -e);
        }
        Y[q] = yv;
        if (i == 0) ye[r] = solve ? e : (mb > 0x7ff0000000000000ull ? YE_NAN : YE_SKIP);
    }
    __syncthreads();
    const int nb = (n + 31) / 32;
    // forward: L y = 2^-e P r (unit lower factor)
    for (int c = 0; c < nb; ++c) {
        const int b0 = 32 * c, i = b0 + lane, tn = min(32, n - b0);
        if (warp < R) {   // this row's 32 factors of the block, loaded once
            float lk[32];
            const float4 *l4 = reinterpret_cast<const float4 *>(L + (size_t)i * LDF + b0);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const float4 v = l4[q];
                lk[4 * q] = v.x;
                lk[4 * q + 1] = v.y;
                lk[4 * q + 2] = v.z;
                lk[4 * q + 3] = v.w;
            }
            for (int r = warp; r < R; r += 2 * DC_WARPS) {
                const int r2 = r + DC_WARPS;
                const bool s1 = ye[r] > YE_NAN, s2 = r2 < R && ye[r2] > YE_NAN;
                float v1 = s1 ? Y[(size_t)r * NP + i] : 0.f, v2 = s2 ? Y[(size_t)r2 * NP + i] : 0.f;
                if (s2) fwd_chain<true>(v1, v2, lk, lane, i < n, tn);
                else fwd_chain<false>(v1, v2, lk, lane, i < n, tn);
                if (s1) Y[(size_t)r * NP + i] = v1;
                if (s2) Y[(size_t)r2 * NP + i] = v2;
            }
        }
        __syncthreads();
        const int r0 = b0 + 32, cnt = n - r0;
        if (cnt > 0) {   // rows r0 .. n-1 take the block's 32 columns
            if (R >= IR_BLK_MIN) {
                blk_update_fwd(R, NP, LDF, b0, r0, cnt, L, Y, ye);
            } else {   // few right-hand sides: one (right-hand side, row) a thread
                for (int q = tid; q < R * cnt; q += DC_THREADS) {
                    const int r = q / cnt, ii = r0 + (q - r * cnt);
                    if (ye[r] <= YE_NAN) continue;
                    const float4 *Li = reinterpret_cast<const float4 *>(L + (size_t)ii * LDF + b0);
                    const float4 *yb = reinterpret_cast<const float4 *>(Y + (size_t)r * NP + b0);
                    float y = Y[(size_t)r * NP + ii];
#pragma unroll
                    for (int t = 0; t < 8; ++t) {
                        const float4 l4 = Li[t], y4 = yb[t];
                        y = fmaf(-l4.x, y4.x, y);
                        y = fmaf(-l4.y, y4.y, y);
                        y = fmaf(-l4.z, y4.z, y);
                        y = fmaf(-l4.w, y4.w, y);
                    }
                    Y[(size_t)r * NP + ii] = y;
                }
            }
            __syncthreads();
        }
    }
    // backward: U y = y (U_kk = 1 / dinv[k])
    for (int c = nb - 1; c >= 0; --c) {
        const int b0 = 32 * c, i = b0 + lane, tn = min(32, n - b0);
        if (warp < R) {   // this row's 32 factors of the block and the block's 1 / U_kk
            float uk[32], dk[32];
            const float4 *u4 = reinterpret_cast<const float4 *>(L + (size_t)i * LDF + b0);
            const float4 *d4 = reinterpret_cast<const float4 *>(dinv + b0);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const float4 v = u4[q], d = d4[q];
                uk[4 * q] = v.x;
                uk[4 * q + 1] = v.y;
                uk[4 * q + 2] = v.z;
                uk[4 * q + 3] = v.w;
                dk[4 * q] = d.x;
                dk[4 * q + 1] = d.y;
                dk[4 * q + 2] = d.z;
                dk[4 * q + 3] = d.w;
            }
            for (int r = warp; r < R; r += 2 * DC_WARPS) {
                const int r2 = r + DC_WARPS;
                const bool s1 = ye[r] > YE_NAN, s2 = r2 < R && ye[r2] > YE_NAN;
                float v1 = s1 ? Y[(size_t)r * NP + i] : 0.f, v2 = s2 ? Y[(size_t)r2 * NP + i] : 0.f;
                if (s2) bwd_chain<true>(v1, v2, uk, dk, lane, tn);
                else bwd_chain<false>(v1, v2, uk, dk, lane, tn);
                if (s1) Y[(size_t)r * NP + i] = v1;
                if (s2) Y[(size_t)r2 * NP + i] = v2;
            }
        }
        __syncthreads();
        if (b0 > 0) {   // rows 0 .. b0-1 take the block's columns, the last first
            if (R >= IR_BLK_MIN) {
                blk_update_bwd(R, NP, LDF, b0, tn, L, Y, ye);
            } else {
                for (int q = tid; q < R * b0; q += DC_THREADS) {
                    const int r = q / b0, ii = q - r * b0;
                    if (ye[r] <= YE_NAN) continue;
                    const float *Li = L + (size_t)ii * LDF + b0;
                    const float *yb = Y + (size_t)r * NP + b0;
                    float y = Y[(size_t)r * NP + ii];
                    if (tn == 32) {
                        const float4 *L4 = reinterpret_cast<const float4 *>(Li);
                        const float4 *y4p = reinterpret_cast<const float4 *>(yb);
#pragma unroll
                        for (int t = 7; t >= 0; --t) {
                            const float4 l4 = L4[t], y4 = y4p[t];
                            y = fmaf(-l4.w, y4.w, y);
                            y = fmaf(-l4.z, y4.z, y);
                            y = fmaf(-l4.y, y4.y, y);
                            y = fmaf(-l4.x, y4.x, y);
                        }
                    } else {
                        for (int t = tn - 1; t >= 0; --t) y = fmaf(-Li[t], yb[t], y);
                    }
                    Y[(size_t)r * NP + ii] = y;
                }
            }
            __syncthreads();
        }
    }
    // x += 2^e y, element by element; max |x| per right-hand side into xnb
    // (zero before the call) by atomicMax, a warp at a time where its lanes
    // share the right-hand side
    for (int q0 = warp * 32; q0 < R * n; q0 += DC_THREADS) {
        const int q = q0 + lane;
        const bool ok = q < R * n;
        const int r = ok ? q / n : R - 1, i = q - r * n;
        unsigned long long xb = 0ull;
        if (ok) {
            const int e = ye[r];
            double xv = xs[q];
            if (e > YE_NAN) {
                const double d = widen_scaled(Y[(size_t)r * NP + i], e);
                const double s = xv + d;
                if (E) {
                    // the exact rounding error of s = x + d (a fast two-sum
                    // with the larger magnitude first, compared on the bits),
                    // in units of 2^e, to BF16: it is at most 2^-53 |x|, and
                    // 8 bits of it leave the tracked update within 2^-61 |x|
                    const long long bx = __double_as_longlong(xv) & 0x7fffffffffffffffll;
                    const long long bd = __double_as_longlong(d) & 0x7fffffffffffffffll;
                    const double big = bx >= bd ? xv : d, small = bx >= bd ? d : xv;
                    const double err = small - (s - big);
                    const bool zero = (__double_as_longlong(err) & 0x7fffffffffffffffll) == 0;
                    E[(size_t)r * NP + i] = __float2bfloat16_rn(zero ? 0.f : narrow_scaled(err, -e));
                }
                xv = s;
                xs[q] = xv;
            } else if (E) {
                E[(size_t)r * NP + i] = __float2bfloat16_rn(0.f);
            }
            xb = e == YE_NAN ? 0x7ff8000000000000ull   // a NaN residual never converges
                             : (unsigned long long)__double_as_longlong(fabs(xv));
        }
        const int ra = __shfl_sync(0xffffffffu, r, 0), rb = __shfl_sync(0xffffffffu, r, 31);
        if (ra == rb) {
            xb = warp_max_u64(xb);
            if (lane == 0) atomicMax(xnb + r, xb);
        } else if (ok) {
            atomicMax(xnb + r, xb);
        }
    }
}

// Layouts of K's copies for the residuals, in groups of consecutive columns:
// the FP64 copy Kt as [j / 4][i][j % 4], the FP32 pairs Kf as [j / 8][i][j % 8].
// A warp's lanes (consecutive rows i) read 4 or 8 columns each as one
// contiguous run, and the fill's warps (consecutive columns j of one row)
// write 4 or 8 neighbours into one run.
__device__ __forceinline__ size_t kt_idx(int n, int i, int j) { return ((size_t)(j >> 2) * n + i) * 4 + (j & 3); }
__device__ __forceinline__ size_t kf_idx(int n, int i, int j) { return ((size_t)(j >> 3) * n + i) * 8 + (j & 7); }

// The refinement's residual r = b - K x in FP64, K_ij at Kt[kt_idx(n, i, j)]:
// thread (g, i) takes row i of right-hand sides g, g + G, g + 2G, ...
// (G = DC_THREADS / n groups), IR_RB of them a pass, so a row of K is read
// ceil(R / (G IR_RB)) times instead of R.  Every sum runs over j in order
// (one FMA chain per element, the rounding of a plain dot product); max |r|
// per right-hand side goes into rnb as bits, by atomicMax.  A single
// right-hand side is summed in G slices instead (G chains of n / G FMAs, so
// that all G n threads work).  Its own function for its registers.
__device__ __noinline__ void ir_residual(int n, int R, int kind, const double *Kt, const double *xs, double *rs,
                                         const double *P1, const double *P2, size_t pstride, unsigned long long *rnb,
                                         double *part) {
    const int tid = threadIdx.x, lane = tid & 31;
    const int G = DC_THREADS / n;
    const int g = tid / n, i = tid - g * n;
    if (R == 1 && G > 1) {
        // one right-hand side: the G groups each sum a slice of j (whole
        // multiples of 4) into part[g n + i], and thread (0, i) adds the
        // slices in order -- the rounding of a sum in G pieces
        const int seg = ((n + G - 1) / G + 3) & ~3;
        if (g < G) {
            const int j0 = min(n, g * seg), j1 = min(n, j0 + seg);
            double acc = 0.0;
            int j = j0;
            for (; j + 4 <= j1; j += 4) {
                const double2 *kp = reinterpret_cast<const double2 *>(Kt + kt_idx(n, i, j));
                const double2 ka = kp[0], kb = kp[1];
                const double k0 = ka.x, k1 = ka.y, k2 = kb.x, k3 = kb.y;
                acc = fma(k0, xs[j], acc);
                acc = fma(k1, xs[j + 1], acc);
                acc = fma(k2, xs[j + 2], acc);
                acc = fma(k3, xs[j + 3], acc);
            }
            for (; j < j1; ++j) acc = fma(Kt[kt_idx(n, i, j)], xs[j], acc);
            part[g * n + i] = acc;
        }
        __syncthreads();
        if (g == 0) {
            double acc = part[i];
            for (int q = 1; q < G; ++q) acc += part[q * n + i];
            const double u = P1[i], w = P2[i];
            const double rv = (kind == 0 ? u : (kind == 1 ? u + w : u - w)) - acc;
            rs[i] = rv;
            atomicMax(rnb, (unsigned long long)__double_as_longlong(fabs(rv)));
        }
        return;
    }
    const int g0 = __shfl_sync(0xffffffffu, g, 0), g31 = __shfl_sync(0xffffffffu, g, 31);
    const bool whole = g0 == g31 && g31 < G;   // the warp's lanes share their right-hand sides
    const int mine = g < G && g < R ? (R - g + G - 1) / G : 0;
    for (int q0 = 0; q0 < mine; q0 += IR_RB) {
        const int nb = min(IR_RB, mine - q0);
        const double *xb = xs + (size_t)(g + G * q0) * n;
        const size_t xstride = (size_t)G * n;
        double acc[IR_RB];
#pragma unroll
        for (int b = 0; b < IR_RB; ++b) acc[b] = 0.0;
        int j = 0;
        for (; j + 4 <= n; j += 4) {
            const double2 *kp = reinterpret_cast<const double2 *>(Kt + kt_idx(n, i, j));
            const double2 ka = kp[0], kb = kp[1];
            const double k0 = ka.x, k1 = ka.y, k2 = kb.x, k3 = kb.y;
#pragma unroll
            for (int b = 0; b < IR_RB; ++b) {
                if (b < nb) {
                    const double *x = xb + b * xstride + j;
                    acc[b] = fma(k0, x[0], acc[b]);
                    acc[b] = fma(k1, x[1], acc[b]);
                    acc[b] = fma(k2, x[2], acc[b]);
                    acc[b] = fma(k3, x[3], acc[b]);
                }
            }
        }
        for (; j < n; ++j) {
            const double kv = Kt[kt_idx(n, i, j)];
#pragma unroll
            for (int b = 0; b < IR_RB; ++b)
                if (b < nb) acc[b] = fma(kv, xb[b * xstride + j], acc[b]);
        }
#pragma unroll
        for (int b = 0; b < IR_RB; ++b) {
            if (b < nb) {
                const int r = g + G * (q0 + b);
                const double u = P1[r * pstride + i], w = P2[r * pstride + i];
                const double rv = (kind == 0 ? u : (kind == 1 ? u + w : u - w)) - acc[b];
                rs[(size_t)r * n + i] = rv;
                // bits of |r|: NaN patterns exceed every number's
                unsigned long long q = (unsigned long long)__double_as_longlong(fabs(rv));
                if (whole) {
                    q = warp_max_u64(q);
                    if (lane == 0) atomicMax(rnb + r, q);
                } else {
                    atomicMax(rnb + r, q);
                }
            }
        }
    }
}


// Kl = fl32(v - f) and the rest Kll = v - f - Kl for f = fl32(v), with
// integer operations: v - f is exact in FP64 (at most half an FP32 ulp of v,
// so below 2^28 units of v's last place), the difference d of the mantissas
// rounds to FP32 as Kl, and d minus that rounding (at most 5 bits) is Kll,
// so v = f + Kl + Kll exactly.  Both are 0 where v, f or a result is not a
// normal number: the parts are then coarser, by at most FP32's smallest
// normal number (2^-126) times |x| per entry; the solver uses them only when
// |K|_inf >= 2^-40, where that stays far below |K|_inf 2^-53 |x|.
__device__ __forceinline__ float scaled_int_float(float x, int k, bool neg) {
    const unsigned b = __float_as_uint(x);
    const int e = (int)((b >> 23) & 0xff) + k;
    if (x == 0.f || e < 1 || e > 254) return 0.f;
    const unsigned r = (b & 0x807fffffu) | ((unsigned)e << 23);
    return __uint_as_float(neg ? r ^ 0x80000000u : r);
}
__device__ __forceinline__ void low_parts(double v, float f, float &l, float &ll) {
    l = ll = 0.f;
    const long long bv = __double_as_longlong(v);
    const int ev = (int)((bv >> 52) & 0x7ff);
    const unsigned bf = __float_as_uint(f);
    const int ef = (int)((bf >> 23) & 0xff);
    const int sh = ef - ev + 925;
    if (ev == 0 || ev == 0x7ff || ef == 0 || ef == 0xff || (sh != 29 && sh != 30)) return;
    const long long mv = (bv & ((1ll << 52) - 1)) | (1ll << 52);
    const long long mf = (long long)((bf & 0x7fffffu) | 0x800000u) << sh;
    const int d = (int)(mv - mf);   // |d| <= 2^28
    const float dh = __int2float_rn(d);
    const int dl = d - __float2int_rn(dh);
    l = scaled_int_float(dh, ev - 1075, bv < 0);
    ll = scaled_int_float(__int2float_rn(dl), ev - 1075, bv < 0);
}

// The first residual r = b - K x0 of many right-hand sides on both of the
// SM's pipes at once.  x0 = 2^e Y (the first correction, exact in FP32).  In
// one pass over j a thread forms NF of its right-hand sides as FP64 FMA
// chains from K's FP64 copy Kt (as ir_residual does) and NT of them as
// error-free triple-float products on the FP32 pipe: K = Kh + Kl + Kll
// exactly (Kf and Kll), each Kh y and Kl y with its fma error, and the sum
// cascaded over three levels -- two-sums on the first two, the third level
// holding terms below 2^-48 of the first -- so that its error stays near
// 2^-70 of sum |K_ij y_j|, below what an FP64 FMA chain leaves.  The three
// levels reach FP64 as r = ((b - S1) - S2) - S3.  Slots beyond a thread's
// right-hand sides read zero rows (ZD for x, Z for Y).  FP64 issues 2 FMAs
// per clock per SM and FP32 64 times that, so with NF : NT near 5 : 6 the
// two pipes finish together, in about half the time of an all-FP64 residual.
template <int NF, int NT>
__device__ __noinline__ void ir_residual_first(int n, int R, int NP, int kind, const double *Kt, const float2 *Kf,
                                               const float *Kll, const double *xs, const float *Y, const int *ye,
                                               const double *ZD, const float *Z, double *rs, const double *P1,
                                               const double *P2, size_t pstride, unsigned long long *rnb, int q0) {
    const int tid = threadIdx.x, lane = tid & 31;
    const int G = DC_THREADS / n;
    const int g = tid / n, i = tid - g * n;
    const int g0 = __shfl_sync(0xffffffffu, g, 0), g31 = __shfl_sync(0xffffffffu, g, 31);
    const bool whole = g0 == g31 && g31 < G;
    const int mine = g < G && g < R ? (R - g + G - 1) / G : 0;
    if (q0 >= mine) return;
    const int nb = min(NF + NT, mine - q0);
    // row of slot b: x (FP64) for b < NF, Y (FP32) after; zero rows past nb
    const double *xb = xs + (size_t)(g + G * q0) * n;
    const float *yb = Y + (size_t)(g + G * (q0 + NF)) * NP;
    const size_t xstride = (size_t)G * n, ystride = (size_t)G * NP;
#define XROW(b) ((b) < nb ? xb + (b) * xstride : ZD)
#define YROW(b) (NF + (b) < nb ? yb + (b) * ystride : Z)
    double acc[NF > 0 ? NF : 1];
    float s1[NT > 0 ? NT : 1], s2[NT > 0 ? NT : 1], s3[NT > 0 ? NT : 1];
#pragma unroll
    for (int b = 0; b < NF; ++b) acc[b] = 0.0;
#pragma unroll
    for (int b = 0; b < NT; ++b) s1[b] = s2[b] = s3[b] = 0.f;
    auto two_sum = [](float a, float b, float &s, float &e) {
        s = a + b;
        const float bb = s - a;
        e = (a - (s - bb)) + (b - bb);
    };
    auto term3 = [&](float kh, float kl, float kll, float y, int b) {
        const float p1 = kh * y, q1 = fmaf(kh, y, -p1);
        const float p2 = kl * y, q2 = fmaf(kl, y, -p2);
        float t1, t2, t3, t4;
        two_sum(s1[b], p1, s1[b], t1);
        two_sum(s2[b], t1, s2[b], t2);
        two_sum(s2[b], q1, s2[b], t3);
        two_sum(s2[b], p2, s2[b], t4);
        s3[b] += ((t2 + t3) + (t4 + q2)) + kll * y;
    };
    // four columns a step (one group of Kt, half a group of Kf and Kll)
    const int n4 = n & ~3;
    int j = 0;
    for (; j < n4; j += 4) {
        double kd[4];
        float2 kf[4];
        float kq[4];
        if (NF > 0) {
            const double2 *p = reinterpret_cast<const double2 *>(Kt + kt_idx(n, i, j));
            const double2 v0 = p[0], v1 = p[1];
            kd[0] = v0.x;
            kd[1] = v0.y;
            kd[2] = v1.x;
            kd[3] = v1.y;
        }
        if (NT > 0) {
            const float4 *p = reinterpret_cast<const float4 *>(Kf + kf_idx(n, i, j));
            const float4 v0 = p[0], v1 = p[1];
            kf[0] = make_float2(v0.x, v0.y);
            kf[1] = make_float2(v0.z, v0.w);
            kf[2] = make_float2(v1.x, v1.y);
            kf[3] = make_float2(v1.z, v1.w);
            const float4 q = *reinterpret_cast<const float4 *>(Kll + kf_idx(n, i, j));
            kq[0] = q.x;
            kq[1] = q.y;
            kq[2] = q.z;
            kq[3] = q.w;
        }
#pragma unroll
        for (int b = 0; b < NF; ++b) {   // x rows start at r n doubles: 8-byte loads
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[b] = fma(kd[u], XROW(b)[j + u], acc[b]);
        }
#pragma unroll
        for (int b = 0; b < NT; ++b) {
            const float4 y4 = *reinterpret_cast<const float4 *>(YROW(b) + j);
            term3(kf[0].x, kf[0].y, kq[0], y4.x, b);
            term3(kf[1].x, kf[1].y, kq[1], y4.y, b);
            term3(kf[2].x, kf[2].y, kq[2], y4.z, b);
            term3(kf[3].x, kf[3].y, kq[3], y4.w, b);
        }
    }
    for (; j < n; ++j) {
        const double kv = Kt[kt_idx(n, i, j)];
        const float2 kfv = Kf[kf_idx(n, i, j)];
        const float kqv = Kll[kf_idx(n, i, j)];
#pragma unroll
        for (int b = 0; b < NF; ++b) acc[b] = fma(kv, XROW(b)[j], acc[b]);
#pragma unroll
        for (int b = 0; b < NT; ++b) term3(kfv.x, kfv.y, kqv, YROW(b)[j], b);
    }
#undef XROW
#undef YROW
#pragma unroll
    for (int b = 0; b < NF + NT; ++b) {
        if (b < nb) {
            const int r = g + G * (q0 + b);
            const double u = P1[r * pstride + i], w = P2[r * pstride + i];
            const double bv = kind == 0 ? u : (kind == 1 ? u + w : u - w);
            double rv;
            if (b < NF) {
                rv = bv - acc[b < NF ? b : 0];
            } else {
                const int bt = b >= NF ? b - NF : 0, e = ye[r];
                rv = e > YE_NAN ? ((bv - widen_scaled(s1[bt], e)) - widen_scaled(s2[bt], e)) - widen_scaled(s3[bt], e)
                                : bv;
            }
            rs[(size_t)r * n + i] = rv;
            unsigned long long q = (unsigned long long)__double_as_longlong(fabs(rv));
            if (whole) {
                q = warp_max_u64(q);
                if (lane == 0) atomicMax(rnb + r, q);
            } else {
                atomicMax(rnb + r, q);
            }
        }
    }
}

// A residual update on the FP32 pipe in double-float: r <- r - K 2^e (Y - E)
// for the update 2^e (Y - E) that the last correction applied to x (Y its
// FP32 values, E the rounding errors of the FP64 additions in BF16, both in
// units of 2^e), with K held as FP32 pairs Kf[kf_idx(n, i, j)] = (fl32(K_ij),
// fl32(K_ij - fl32(K_ij))): each product K_ij Y_j as hi * y (exact with its
// fma error) plus lo * y, summed over j in order with a two-sum on the high
// part, minus hi * E_j in the low part; the sum is brought to FP64 once per
// element.  Its error, ~n 2^-48 |K| |2^e Y|, is far below FP64's rounding of
// |K| |x| once the first correction has been applied (|2^e Y| ~ cond(K)
// 2^-24 |x| and less after every step), so r stays the residual of the FP64
// x as closely as an FP64 residual would.  The threads are grouped as in
// ir_residual; one call is the pass over a thread's right-hand sides
// q0 .. q0 + W - 1 (W = 8, or 4 for a short last pass); the slots of a pass
// beyond its right-hand sides read the zero rows Z (Y) and ZE (E), whose
// terms leave the sums unchanged, so the pass runs without branches.
template <int W>
__device__ __noinline__ void ir_residual_inc(int n, int R, int NP, const float2 *Kf, const float *Y,
                                             const __nv_bfloat16 *E, const float *Z, const __nv_bfloat16 *ZE,
                                             const int *ye, double *rs, unsigned long long *rnb, int q0) {
    const int tid = threadIdx.x, lane = tid & 31;
    const int G = DC_THREADS / n;
    const int g = tid / n, i = tid - g * n;
    const int g0 = __shfl_sync(0xffffffffu, g, 0), g31 = __shfl_sync(0xffffffffu, g, 31);
    const bool whole = g0 == g31 && g31 < G;
    const int mine = g < G && g < R ? (R - g + G - 1) / G : 0;
    const int n8 = n & ~7;
    if (q0 < mine) {
        const int nb = min(W, mine - q0);
        const float *yb = Y + (size_t)(g + G * q0) * NP;
        const __nv_bfloat16 *eb = E + (size_t)(g + G * q0) * NP;
        const size_t ystride = (size_t)G * NP;
        float sh[W], sl[W];
#pragma unroll
        for (int b = 0; b < W; ++b) sh[b] = sl[b] = 0.f;
        auto term = [&](float2 k, float y, float ev, int b) {
            const float p = k.x * y;
            const float pe = fmaf(k.x, y, -p);
            const float t = sh[b] + p;
            const float bb = t - sh[b];
            const float err = (sh[b] - (t - bb)) + (p - bb);
            sh[b] = t;
            sl[b] = fmaf(-k.x, ev, sl[b] + (err + fmaf(k.y, y, pe)));
        };
        // eight columns of K a step, the next eight loading while these are used
        float2 k[8];
        if (n8 > 0) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float4 v = reinterpret_cast<const float4 *>(Kf + kf_idx(n, i, 0))[u];
                k[2 * u] = make_float2(v.x, v.y);
                k[2 * u + 1] = make_float2(v.z, v.w);
            }
        }
        int j = 0;
        for (; j < n8; j += 8) {
            float2 kc[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) kc[u] = k[u];
            if (j + 8 < n8) {
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const float4 v = reinterpret_cast<const float4 *>(Kf + kf_idx(n, i, j + 8))[u];
                    k[2 * u] = make_float2(v.x, v.y);
                    k[2 * u + 1] = make_float2(v.z, v.w);
                }
            }
#pragma unroll
            for (int b = 0; b < W; ++b) {
                // Y and E rows start 16-byte aligned (NP a multiple of 32, j of 8)
                const float *yr = (b < nb ? yb + b * ystride : Z) + j;
                const __nv_bfloat16 *er = (b < nb ? eb + b * ystride : ZE) + j;
                const float4 y0 = *reinterpret_cast<const float4 *>(yr);
                const float4 y1 = *reinterpret_cast<const float4 *>(yr + 4);
                const uint4 e8 = *reinterpret_cast<const uint4 *>(er);
                // BF16 to FP32: the 16 bits are the top of the FP32 pattern
                term(kc[0], y0.x, __uint_as_float(e8.x << 16), b);
                term(kc[1], y0.y, __uint_as_float(e8.x & 0xffff0000u), b);
                term(kc[2], y0.z, __uint_as_float(e8.y << 16), b);
                term(kc[3], y0.w, __uint_as_float(e8.y & 0xffff0000u), b);
                term(kc[4], y1.x, __uint_as_float(e8.z << 16), b);
                term(kc[5], y1.y, __uint_as_float(e8.z & 0xffff0000u), b);
                term(kc[6], y1.z, __uint_as_float(e8.w << 16), b);
                term(kc[7], y1.w, __uint_as_float(e8.w & 0xffff0000u), b);
            }
        }
        for (; j < n; ++j) {
            const float2 kv = Kf[kf_idx(n, i, j)];
#pragma unroll
            for (int b = 0; b < W; ++b) {
                const float *yr = b < nb ? yb + b * ystride : Z;
                const __nv_bfloat16 *er = b < nb ? eb + b * ystride : ZE;
                term(kv, yr[j], __bfloat162float(er[j]), b);
            }
        }
#pragma unroll
        for (int b = 0; b < W; ++b) {
            if (b < nb) {
                const int r = g + G * (q0 + b);
                const int e = ye[r];
                const double kx = e > YE_NAN ? widen_scaled(sh[b], e) + widen_scaled(sl[b], e) : 0.0;
                const double rv = rs[(size_t)r * n + i] - kx;
                rs[(size_t)r * n + i] = rv;
                unsigned long long q = (unsigned long long)__double_as_longlong(fabs(rv));
                if (whole) {
                    q = warp_max_u64(q);
                    if (lane == 0) atomicMax(rnb + r, q);
                } else {
                    atomicMax(rnb + r, q);
                }
            }
        }
    }
}

// FP32 LU + FP64 iterative refinement for n <= 32 NC.  Returns true with the
// solution in xs[r * n + i] when every right-hand side met the stopping
// rule; false sends the system to the FP64 solver.
//
// GB300 runs FP64 arithmetic, comparisons and conversions at 1/64 of the
// FP32 rate, so besides the residual's n^2 FMAs per right-hand side the
// solver spends no FP64 instruction per matrix element: K is rounded to FP32
// unscaled (an entry outside FP32's range becomes inf or 0 and the
// factorisation falls back), |K|_inf comes from FP32 row sums, maxima are
// taken on the bit patterns of non-negative doubles, and each residual
// element is one thread's sum, so no FP64 reduction is needed.  The FP64
// matrix (K1 +- K2 for kind 1 and 2) is copied once into Kc (global
// scratch) in groups of 4 columns (kt_idx), so that the residual's loads
// coalesce.
// The factorisation is lu_fp32's.
template <int NC>
__device__ __noinline__ bool solve_refined(const SysView &S, int n, int R, float *L, double *Kc, float2 *Kf,
                                           unsigned char *base, const IrLayout &lay, Scratch &sc) {
    constexpr int NP = 32 * NC;
    constexpr int LDF = NP + 4;
    constexpr int G2 = NC <= 4 ? 4 : (NC <= 8 ? 2 : 1);   // rows per group in the fill
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int kind = S.kind;
    const double *K1 = S.K1, *K2 = S.K2;
    const double *P1 = S.P + (size_t)S.f1 * n, *P2 = S.P + (size_t)S.f2 * n;
    const size_t pstride = (size_t)S.nf * n;
    double *Kt = Kc;   // K_ij of the residuals (K1 +- K2 for kind 1 and 2) at kt_idx(n, i, j)
    int *perm = reinterpret_cast<int *>(base + lay.perm);
    float *dinv = reinterpret_cast<float *>(base + lay.dinv);
    double *xs = reinterpret_cast<double *>(base + lay.x);
    double *rs = reinterpret_cast<double *>(base + lay.r);
    unsigned long long *xn = reinterpret_cast<unsigned long long *>(base + lay.xn);   // [2][R] bits of max |x|
    unsigned long long *rn = reinterpret_cast<unsigned long long *>(base + lay.rn);   // [3][R] bits of max |r|
    float *Y = reinterpret_cast<float *>(base + lay.y);     // [R][np] the correction's FP32 values
    int *ye = reinterpret_cast<int *>(base + lay.ye);       // [R] their power-of-two scale
    __nv_bfloat16 *E = reinterpret_cast<__nv_bfloat16 *>(base + lay.e);   // [R][np] rounding errors of the updates
    float *Z = reinterpret_cast<float *>(base + lay.z);     // [np] zeros, [np] BF16 zeros, [np] FP64 zeros
    __nv_bfloat16 *ZE = reinterpret_cast<__nv_bfloat16 *>(Z + ir_np(n));
    const double *ZD = reinterpret_cast<const double *>(Z + ir_np(n) + ir_np(n) / 2);
    // the exact third FP32 part of K for the first residual, after the pairs
    float *Kll = Kf ? reinterpret_cast<float *>(Kf + (size_t)((n + 7) / 8) * 8 * n) : nullptr;
    double *part = reinterpret_cast<double *>(base + lay.part);   // [DC_THREADS] slices of a residual

    // L = fl32(K) padded with identity (Kt = the FP64 K in column groups, on the way), FP32 row sums of |L|
    float wrow = 0.f;
    for (int i0 = warp; i0 < NP; i0 += G2 * DC_WARPS) {
        double v[G2][NC];
#pragma unroll
        for (int g = 0; g < G2; ++g) {
            const int i = i0 + g * DC_WARPS;
#pragma unroll
            for (int m = 0; m < NC; ++m) {
                const int j = lane + 32 * m;
                v[g][m] = (i < n && j < n) ? __ldg(K1 + (size_t)i * n + j) : (i == j ? 1.0 : 0.0);
            }
        }
#pragma unroll
        for (int g = 0; g < G2; ++g) {
            const int i = i0 + g * DC_WARPS;
#pragma unroll
            for (int m = 0; m < NC; ++m) {
                const int j = lane + 32 * m;
                if (i < n && j < n) {
                    if (kind) {
                        const double w = __ldg(K2 + (size_t)i * n + j);
                        v[g][m] = kind == 1 ? v[g][m] + w : v[g][m] - w;
                    }
                    Kt[kt_idx(n, i, j)] = v[g][m];
                }
            }
        }
#pragma unroll
        for (int g = 0; g < G2; ++g) {
            const int i = i0 + g * DC_WARPS;
            float rsum = 0.f;
#pragma unroll
            for (int m = 0; m < NC; ++m) {
                const int j = lane + 32 * m;
                const float f = (float)v[g][m];
                if (i < NP) L[(size_t)i * LDF + j] = f;
                if (i < n) rsum += fabsf(f);
                // K as FP32 pairs for the double-float residual updates, in groups of 8 columns
                if (Kf && i < n && j < n) {
                    float kl, kll;
                    low_parts(v[g][m], f, kl, kll);
                    Kf[kf_idx(n, i, j)] = make_float2(f, kl);
                    Kll[kf_idx(n, i, j)] = kll;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) rsum += __shfl_xor_sync(0xffffffffu, rsum, o);
            wrow = fmaxf(wrow, rsum);
        }
    }
    if (lane == 0) sc.wnorm[0][warp] = (double)wrow;
    for (int i = tid; i < NP; i += DC_THREADS) perm[i] = i;
    if (Kf)
        for (int i = tid; i < 3 * NP + NP / 2; i += DC_THREADS) Z[i] = 0.f;   // the zero rows of Y, E and x
    for (int r = tid; r < R; r += DC_THREADS) rn[r] = rn[2 * (size_t)R + r] = 0ull;
    for (int idx = tid; idx < R * n; idx += DC_THREADS) {
        const int r = idx / n, i = idx - r * n;
        const double u = P1[r * pstride + i], w = P2[r * pstride + i];
        xs[idx] = 0.0;
        rs[idx] = kind == 0 ? u : (kind == 1 ? u + w : u - w);
    }
    __syncthreads();
    float amax = 0.f;
#pragma unroll
    for (int q = 0; q < DC_WARPS; ++q) amax = fmaxf(amax, (float)sc.wnorm[0][q]);
    if (!(amax > 0.f && amax <= 3.4028234663852886e38f)) return false;
    const double anrm = (double)amax;
    // the FP32-pipe residuals (first residual and updates) need K's FP32
    // parts to carry it exactly; below this norm they would not
    const bool many = Kf && amax >= 0x1p-40f;

    // blocked FP32 factorisation: L U = rows perm[0..np-1] of the padded fl32(K)
    if (!lu_fp32<NC>(L, perm, dinv, sc)) return false;

    // refinement: it = 0 is the first solve from x = 0, scaled by max |b|
    // (its bits into rn's third buffer, which the first correction reads)
    for (int q0 = warp * 32; q0 < R * n; q0 += DC_THREADS) {
        const int q = q0 + lane;
        const bool ok = q < R * n;
        const int r = ok ? q / n : R - 1;
        unsigned long long b = ok ? (unsigned long long)__double_as_longlong(fabs(rs[q])) : 0ull;
        if (__shfl_sync(0xffffffffu, r, 0) == __shfl_sync(0xffffffffu, r, 31)) {
            b = warp_max_u64(b);
            if (lane == 0) atomicMax(rn + 2 * (size_t)R + r, b);
        } else if (ok) {
            atomicMax(rn + 2 * (size_t)R + r, b);
        }
    }
    __syncthreads();
    const double cte = anrm * EPS64 * sqrt((double)n);
    for (int it = 0; it <= IR_ITMAX; ++it) {
        unsigned long long *xnb = xn + (it & 1) * R;
        // bits of max |r| per right-hand side, three buffers: this
        // iteration's was zeroed before the last barrier of the previous
        // one, the next one's (last read two iterations ago) is zeroed now
        unsigned long long *rnb = rn + (size_t)(it % 3) * R;
        for (int r = tid; r < R; r += DC_THREADS) {
            rn[(size_t)((it + 1) % 3) * R + r] = 0ull;
            xnb[r] = 0ull;   // last read two iterations ago
        }
        // with many right-hand sides, only the first residual b - K x runs
        // in FP64; each later one is the previous minus K times the update
        // the correction applied, in double-float on the FP32 pipe
        const bool inc = many && it > 0;
        // x += K^-1 r through the FP32 factors (from x = 0 at it = 0, exact)
        ir_correct<NC>(n, R, L, perm, dinv, xs, rs, rn + (size_t)((it + 2) % 3) * R, Y, ye, xnb, inc ? E : nullptr);
        __syncthreads();
        if (many && !inc) {
            // the first residual of many right-hand sides on the FP64 and FP32 pipes at once
            const int per = (R + DC_THREADS / n - 1) / (DC_THREADS / n);   // right-hand sides per thread
            if (per <= 5) {
                ir_residual(n, R, kind, Kt, xs, rs, P1, P2, pstride, rnb, part);
            } else {
                for (int q0 = 0; q0 < per;) {
                    const int rem = per - q0;
                    if (rem >= 10) {
                        ir_residual_first<5, 6>(n, R, NP, kind, Kt, Kf, Kll, xs, Y, ye, ZD, Z, rs, P1, P2, pstride, rnb, q0);
                        q0 += 11;
                    } else if (rem >= 6) {
                        ir_residual_first<4, 5>(n, R, NP, kind, Kt, Kf, Kll, xs, Y, ye, ZD, Z, rs, P1, P2, pstride, rnb, q0);
                        q0 += 9;
                    } else {
                        ir_residual_first<4, 0>(n, R, NP, kind, Kt, Kf, Kll, xs, Y, ye, ZD, Z, rs, P1, P2, pstride, rnb, q0);
                        q0 += 4;
                    }
                }
            }
        } else if (inc) {
            const int per = (R + DC_THREADS / n - 1) / (DC_THREADS / n);   // right-hand sides per thread
            for (int q0 = 0; q0 < per; q0 += 8) {
                if (per - q0 > 4) ir_residual_inc<8>(n, R, NP, Kf, Y, E, Z, ZE, ye, rs, rnb, q0);
                else ir_residual_inc<4>(n, R, NP, Kf, Y, E, Z, ZE, ye, rs, rnb, q0);
            }
        }
        else ir_residual(n, R, kind, Kt, xs, rs, P1, P2, pstride, rnb, part);
        __syncthreads();
        bool conv = true;
        for (int r = 0; r < R && conv; ++r) {
            const double rmax = __longlong_as_double((long long)rnb[r]);
            const double xmax = __longlong_as_double((long long)xnb[r]);
            if (!(rmax <= xmax * cte)) conv = false;
        }
        if (conv) return true;
    }
    return false;
}

__device__ bool solve_refined_n(const SysView &S, int n, int R, float *L, double *Kc, float2 *Kf, unsigned char *base,
                                const IrLayout &lay, Scratch &sc) {
    switch ((n + 31) / 32) {
        case 1: return solve_refined<1>(S, n, R, L, Kc, Kf, base, lay, sc);
        case 2: return solve_refined<2>(S, n, R, L, Kc, Kf, base, lay, sc);
        case 3: return solve_refined<3>(S, n, R, L, Kc, Kf, base, lay, sc);
        case 4: return solve_refined<4>(S, n, R, L, Kc, Kf, base, lay, sc);
        case 5: return solve_refined<5>(S, n, R, L, Kc, Kf, base, lay, sc);
        case 6: return solve_refined<6>(S, n, R, L, Kc, Kf, base, lay, sc);
        case 7: return solve_refined<7>(S, n, R, L, Kc, Kf, base, lay, sc);
        case 8: return solve_refined<8>(S, n, R, L, Kc, Kf, base, lay, sc);
        case 9: case 10: return solve_refined<10>(S, n, R, L, Kc, Kf, base, lay, sc);
        case 11: case 12: return solve_refined<12>(S, n, R, L, Kc, Kf, base, lay, sc);
        case 13: case 14: return solve_refined<14>(S, n, R, L, Kc, Kf, base, lay, sc);
        case 15: case 16: return solve_refined<16>(S, n, R, L, Kc, Kf, base, lay, sc);
        default: return false;
    }
}

// FP64 elimination on [K | b] and back substitution.  Returns 0, or k + 1
// when the k-th pivot was zero or not finite; x[r] of row i is then at
// A[i * ld + n + r].
__device__ int solve_fp64(const SysView &S, int n, int ld, int R, double *A, Scratch &sc) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int idx = tid; idx < n * n; idx += DC_THREADS) {
        const int i = idx / n, j = idx - i * n;
        A[(size_t)i * ld + j] = S.k(idx);
    }
    for (int idx = tid; idx < R * n; idx += DC_THREADS) {
        const int r = idx / n, i = idx - r * n;
        A[(size_t)i * ld + n + r] = S.b(r, i);
    }
    __syncthreads();
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
        block_argmax(best, bi, n, sc);
        if (!finite_pos(sc.pv)) return k + 1;
        const int p = sc.piv;
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
    return 0;
}

__global__ void __launch_bounds__(DC_THREADS, 1) k_decouple(DecoupleArgs a) {
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ Scratch sc;

    const int tid = threadIdx.x;
    const int n = a.n, ld = a.ld, R = a.n_rhs, nf = a.n_fields;
    // workspace slice: the refined solver's FP64 K1 +- K2 (n^2, rounded up to
    // 16 bytes), then its FP32 factors when they are not in shared memory,
    // then K as FP32 pairs for the residual updates; the FP64 solver's
    // augmented matrix from the start when it is not in shared memory
    double *slice = a.ws ? a.ws + (size_t)blockIdx.x * a.ws_stride : nullptr;
    const IrLayout lay = ir_layout(n, R, !a.l_in_ws);
    double *Kc = slice;
    const size_t kc_d = (size_t)((n + 3) / 4) * 4 * n;                           // doubles of Kc (whole column groups)
    const size_t f32_d = a.l_in_ws ? ((size_t)ir_np(n) * ir_ldf(n) + 1) / 2 : 0;   // doubles of the FP32 factors
    float2 *Kf = a.df_inc ? reinterpret_cast<float2 *>(slice + kc_d + f32_d) : nullptr;
    float *L = a.l_in_ws ? reinterpret_cast<float *>(slice + kc_d)
                         : reinterpret_cast<float *>(dsm + lay.L);
    double *A = a.direct_in_ws ? slice : reinterpret_cast<double *>(dsm);
    const double *xs = reinterpret_cast<const double *>(dsm + lay.x);

    for (long long sys = blockIdx.x; sys < a.n_sys; sys += gridDim.x) {
        const int w = (int)(sys / a.sys_per_window), q = (int)(sys % a.sys_per_window);
        SysView S;
        S.kind = a.kind[q];
        S.K1 = a.M + ((size_t)w * a.nspec + a.slot1[q]) * (size_t)n * n;
        S.K2 = a.M + ((size_t)w * a.nspec + a.slot2[q]) * (size_t)n * n;
        S.P = a.pcl + (size_t)w * R * nf * n;
        S.f1 = a.field1[q];
        S.f2 = a.field2[q];
        S.nf = nf;
        S.n = n;

        const bool refined = a.refine && solve_refined_n(S, n, R, L, Kc, Kf, dsm, lay, sc);
        __syncthreads();   // the FP64 solver reuses the refinement's shared memory
        const int bad = refined ? 0 : solve_fp64(S, n, ld, R, A, sc);

        double *O = a.out + (size_t)w * R * nf * n;
        for (int idx = tid; idx < R * n; idx += DC_THREADS) {
            const int r = idx / n, i = idx - r * n;
            const double x = bad ? __longlong_as_double(0x7ff8000000000000LL)
                                 : (refined ? xs[(size_t)r * n + i] : A[(size_t)i * ld + n + r]);
            double *o1 = O + ((size_t)r * nf + S.f1) * n + i;
            if (S.kind == 0) {
                *o1 = x;
            } else {
                double *o2 = O + ((size_t)r * nf + S.f2) * n + i;
                atomicAdd(o1, 0.5 * x);
                atomicAdd(o2, (S.kind == 1 ? 0.5 : -0.5) * x);
            }
        }
        if (tid == 0 && a.info) a.info[sys] = bad;
        __syncthreads();   // shared memory is reused by the CTA's next system
    }
}

}  // namespace

int decouple_smem_limit() { return 226 * 1024; }   // dynamic part; the static Scratch fits in the rest

cudaError_t launch_decouple(const DecoupleArgs &a, int grid, size_t smem, cudaStream_t st) {
    static std::atomic<unsigned long long> attr{0};
    const cudaError_t e = opt_in_smem(k_decouple, decouple_smem_limit(), attr);
    if (e != cudaSuccess) return e;
    k_decouple<<<grid, DC_THREADS, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t decouple_blocks_per_sm(size_t smem, int *n) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, k_decouple, DC_THREADS, smem);
}

}  // namespace cpl

// ---------------------------------------------------------------- entry point
using namespace cpl;

extern "C" {

cpl_status cpl_decouple(cpl_ctx *c, int n, int n_windows, unsigned spectra, const double *M, const double *pcl,
                        int n_rhs, double *out, int *info, void *stream) {
    if (!c) return fail(CPL_ERR_ARG, "ctx is NULL");
    if (!M || !pcl || !out) return fail(CPL_ERR_ARG, "M, pcl and out must be non-NULL");
    if (n < 1 || n > CPL_DECOUPLE_NMAX) return fail(CPL_ERR_RANGE, "n must be in 1 .. CPL_DECOUPLE_NMAX");
    if (n_windows < 1) return fail(CPL_ERR_ARG, "n_windows must be >= 1");
    if (n_rhs < 1 || n_rhs > CPL_DECOUPLE_RHS_MAX) return fail(CPL_ERR_RANGE, "n_rhs must be in 1 .. CPL_DECOUPLE_RHS_MAX");
    if (spectra == 0 || (spectra & ~31u)) return fail(CPL_ERR_ARG, "spectra must be a non-empty set of CPL_* bits");
    if (!(spectra & kEE) != !(spectra & kEEBB))
        return fail(CPL_ERR_ARG, "CPL_EE and CPL_EEBB must be decoupled together (the EE/BB system)");
    DecoupleArgs a{};
    a.M = M;
    a.pcl = pcl;
    a.out = out;
    a.info = info;
    a.n = n;
    a.n_rhs = n_rhs;
    a.ld = (n + n_rhs) | 1;
    a.nspec = spec_count(spectra);
    // fields TT, TE, EE, BB, EB of the requested set, systems TT, TE, EE+EEBB, EE-EEBB, EB
    int nf = 0, fTT = -1, fTE = -1, fEE = -1, fBB = -1, fEB = -1;
    if (spectra & kTT) fTT = nf++;
    if (spectra & kTE) fTE = nf++;
    if (spectra & kEE) { fEE = nf++; fBB = nf++; }
    if (spectra & kEB) fEB = nf++;
    a.n_fields = nf;
    int q = 0;
    auto add = [&](int kind, int s1, int s2, int f1, int f2) {
        a.kind[q] = kind; a.slot1[q] = s1; a.slot2[q] = s2; a.field1[q] = f1; a.field2[q] = f2; ++q;
    };
    if (fTT >= 0) add(0, spec_slot(spectra, kTT), spec_slot(spectra, kTT), fTT, fTT);
    if (fTE >= 0) add(0, spec_slot(spectra, kTE), spec_slot(spectra, kTE), fTE, fTE);
    if (fEE >= 0) {
        add(1, spec_slot(spectra, kEE), spec_slot(spectra, kEEBB), fEE, fBB);
        add(2, spec_slot(spectra, kEE), spec_slot(spectra, kEEBB), fEE, fBB);
    }
    if (fEB >= 0) add(0, spec_slot(spectra, kEB), spec_slot(spectra, kEB), fEB, fEB);
    a.sys_per_window = q;
    a.n_sys = (long long)q * n_windows;

    cpl_status s;
    if ((s = select_device(c)) != CPL_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    int nsm = 0;
    CPL_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device));
    // FP64 solver: augmented matrix in shared memory when it fits.  Refined
    // solver (FP32 factors + FP64 residuals) when it needs fewer FP64
    // operations: its residuals cost about 3 n^2 n_rhs per system against
    // n^3 / 3 + 1.5 n^2 n_rhs for the FP64 solve, i.e. n_rhs <= 2n/9.
    const size_t limit = (size_t)decouple_smem_limit();
    const size_t direct_bytes = sizeof(double) * (size_t)n * a.ld;
    a.direct_in_ws = direct_bytes > limit;
    a.refine = 9 * n_rhs <= 2 * n && n <= IR_NMAX;
    size_t ir_bytes = 0;
    if (a.refine) {
        ir_bytes = ir_layout(n, n_rhs, true).total;
        a.l_in_ws = ir_bytes > limit;
        if (a.l_in_ws) ir_bytes = ir_layout(n, n_rhs, false).total;
        if (ir_bytes > limit) {
            a.refine = 0;
            a.l_in_ws = 0;
            ir_bytes = 0;
        }
    }
    const size_t smem = std::max(ir_bytes, a.direct_in_ws ? (size_t)0 : direct_bytes);
    int bps = 0;
    CPL_CUDA_TRY(decouple_blocks_per_sm(smem, &bps));
    const int grid = (int)std::min<long long>(a.n_sys, (long long)nsm * std::max(bps, 1));
    if (a.direct_in_ws || a.refine) {
        // one slice per CTA: the refined solver's FP64 K1 +- K2 (n^2 doubles,
        // whole 16-byte units), when not in shared memory its padded FP32
        // factors, and from IR_INC_MIN right-hand sides K as FP32 pairs; or the
        // FP64 solver's augmented matrix -- the larger, even
        const size_t kc = (size_t)((n + 3) / 4) * 4 * n;   // whole groups of 4 columns
        const size_t f32 = a.l_in_ws ? ((size_t)ir_np(n) * ir_ldf(n) + 1) / 2 : 0;
        a.df_inc = a.refine && n_rhs >= IR_INC_MIN;
        // FP32 pairs of K and its exact third parts, whole groups of 8 columns (8 n doubles, then 4 n)
        const size_t kf = a.df_inc ? (size_t)((n + 7) / 8) * 12 * n : 0;
        const size_t fp64 = a.direct_in_ws ? (size_t)n * a.ld : 0;
        a.ws_stride = (std::max(a.refine ? kc + f32 + kf : 0, fp64) + 1) & ~(size_t)1;
        CPL_CUDA_TRY(cudaStreamWaitEvent(st, c->done, 0));
        if ((s = c->dec_ws.ensure(sizeof(double) * a.ws_stride * grid, "decoupling workspace")) != CPL_OK) return s;
        a.ws = c->dec_ws.as<double>();
    }
    if (fEE >= 0)
        CPL_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(double) * (size_t)n_windows * n_rhs * nf * n, st));
    {
        LaunchScope ls(c, "decouple", st);
        CPL_CUDA_TRY(launch_decouple(a, grid, smem, st));
        const double nn = n, R = n_rhs;
        const double flop = (double)a.n_sys * ((nn - 1) * nn * (2 * nn - 1) / 3.0 + 2.0 * R * nn * (nn - 1));
        ls.done(flop, 8.0 * (double)a.n_sys * (nn * nn + 2.0 * R * nn));
    }
    if (a.ws) CPL_CUDA_TRY(cudaEventRecord(c->done, st));
    return CPL_OK;
}

}  // extern "C"
