// mixed_prep.cu -- operand preparation of the mixed-precision path.
//
// Writes the BF16 limb images of the separable operands (see plain_fp64.cu
// for their definitions; the formulas are repeated next to each variant) in
// the exact shared-memory layout the tensor-core GEMM consumes (mixed.h:
// mx_img_off), together with the per-(row, MX_SB-k scale block) power-of-two
// exponents.  Values are formed in double-float from double-float copies of
// the FP64 g / h tables and weights; the weights carry a separate integer
// exponent because window spectra reach below the FP32 range.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "dd.cuh"
#include "mixed.h"

namespace cpl {
namespace {

constexpr int16_t EXP_ZERO = -32000;   // exponent of an all-zero block
constexpr int MPL = MX_SB / 32;          // k values per lane in one scale block

__global__ void k_tables_dd(const double *__restrict__ g, const double *__restrict__ h, int n,
                            float *gh, float *gl, float *hh, float *hl) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const double a = g[p], b = h[p];
        const float ah = (float)a, bh = (float)b;
        gh[p] = ah;
        gl[p] = (float)(a - (double)ah);
        hh[p] = bh;
        hl[p] = (float)(b - (double)bh);
    }
}

// A(l) = m 2^e with m in [1, 2) held as double-float; A = 0 -> m = 0.
__global__ void k_weights_dd(const double *__restrict__ A, int total, float *Ah, float *Al, int *Ae) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) {
        const double a = A[q];
        if (a == 0.0) {
            Ah[q] = 0.f;
            Al[q] = 0.f;
            Ae[q] = 0;
            continue;
        }
        int e;
        const double m = frexp(a, &e);          // a = m 2^e, |m| in [0.5, 1)
        const float mh = (float)m;
        Ah[q] = mh;
        Al[q] = (float)(m - (double)mh);
        Ae[q] = e;
    }
}

// exponent E with |x| < 2^E for x = m 2^e (m != 0)
__device__ __forceinline__ int value_exp(dfl m, int e) { return e + ilogbf_fast(fabsf(m.h)) + 1; }

template <int S>
__device__ __forceinline__ void put_limbs(uint8_t *img_t0, int off, dfl y, int img_bytes) {
    // y in (-128.x, 128.x); limb t is stored pre-scaled by 2^(-8t)
#pragma unroll
    for (int t = 0; t < S; ++t) {
        const float l = rintf(y.h);
        const dfl z = df_two_sum(y.h - l, y.l);
        y.h = z.h * 256.0f;
        y.l = z.l * 256.0f;
        const __nv_bfloat16 v = __float2bfloat16_rn(l * pow2f(-8 * t));
        *reinterpret_cast<__nv_bfloat16 *>(img_t0 + (size_t)t * img_bytes + off) = v;
    }
}

__device__ __forceinline__ int warp_max(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// The four A-side values x_q(i, k) of one (source, i, k), as double-float
// mantissas with an exponent (the weight keeps its own exponent because
// window spectra reach below the FP32 range): x = val 2^(e - ilogb(val) - 1)
// relative to value_exp.  vex[q] = EXP_ZERO for a zero value.
__device__ __forceinline__ void a_values(const MxPrepAArgs &a, int vmask, const float *Ah, const float *Al,
                                         const int *Ae, int cap, int i, int k, int pi, dfl (&val)[MX_NA],
                                         int (&vex)[MX_NA]) {
#pragma unroll
    for (int q = 0; q < MX_NA; ++q) {
        val[q] = {0.f, 0.f};
        vex[q] = EXP_ZERO;
    }
    // even sweep: l3 = 2k + pi, a0 = A(l3) g(i+k+pi) g(k-i), v = (2k+2i+2pi+1)(2k-2i)
    const int l3e = 2 * k + pi;
    if ((vmask & 7) && k >= i && l3e <= cap && Ah[l3e] != 0.f) {
        const dfl A = {Ah[l3e], Al[l3e]};
        const dfl g1 = {a.gh[i + k + pi], a.gl[i + k + pi]};
        const dfl g2 = {a.gh[k - i], a.gl[k - i]};
        const dfl a0 = df_mul(df_mul(A, g1), g2);
        const int e = Ae[l3e];
        val[0] = a0;
        vex[0] = a0.h != 0.f ? value_exp(a0, e) : EXP_ZERO;
        if (k > i && (vmask & 6)) {
            const dfl v = df_int_prod(2 * k + 2 * i + 2 * pi + 1, 2 * k - 2 * i);
            const dfl a0v = df_mul(a0, v);
            const dfl a0v2 = df_mul(a0v, v);
            val[1] = a0v;
            vex[1] = a0v.h != 0.f ? value_exp(a0v, e) : EXP_ZERO;
            val[2] = a0v2;
            vex[2] = a0v2.h != 0.f ? value_exp(a0v2, e) : EXP_ZERO;
        }
    }
    // odd sweep: l3 = 2k + 1 - pi, a1 v = A(l3) g(i+k+1) g(k-i-pi) (2i+2k+2)(2k+1-2i-2pi)
    const int l3o = 2 * k + 1 - pi;
    if ((vmask & 8) && k >= i + pi && l3o <= cap && Ah[l3o] != 0.f) {
        const dfl A = {Ah[l3o], Al[l3o]};
        const dfl g1 = {a.gh[i + k + 1], a.gl[i + k + 1]};
        const dfl g2 = {a.gh[k - i - pi], a.gl[k - i - pi]};
        const dfl v1 = df_int_prod(2 * i + 2 * k + 2, 2 * k + 1 - 2 * i - 2 * pi);
        const dfl x = df_mul(df_mul(df_mul(A, g1), g2), v1);
        if (x.h != 0.f) {
            val[3] = x;
            vex[3] = value_exp(x, Ae[l3o]);
        }
    }
}

// Variants of the A operand that the contractions of a source with these role
// bits read (mx_alpha of its products): a0 always, a0 v from TE on, a0 v^2
// with EE, a1 v with the odd sweep.
__device__ __forceinline__ int variants_of_role(int role) {
    if (role & (kEE | kEEBB | kEB)) return (role & (kEEBB | kEB)) ? 15 : 7;
    if (role & kTE) return 3;
    if (role & kTT) return 1;
    return 0;
}

// Packed FP32 pairs (sm_100+ f32x2 instructions): two values per instruction.
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;"
        : "=l"(r)
        : "l"(*reinterpret_cast<unsigned long long *>(&a)), "l"(*reinterpret_cast<unsigned long long *>(&b)));
    return *reinterpret_cast<float2 *>(&r);
}

// One block per (parity, row group, row block, octet of 8 tile rows): the 8
// rows belong to one source (BI >= 8) and are 8 consecutive values of i.
// Thread (warp w, lane) owns tile row 8 o + (lane & 7) and the 8 consecutive
// k = sb MX_SB + 32 w + 8 (lane >> 3) + 0..7 of each scale block sb, so that
// for every limb it writes one 16-byte core-matrix row and each warp writes
// whole 128-byte core matrices.  Pass 1 computes the values, keeps them in
// shared memory (each thread its own 8 x 4 slots) and finds the row maxima
// of the exponents (shuffles over the 4 lanes of a row, then shared memory
// over the 8 warps); pass 2 writes the limbs of the kept values (a value's
// shift against the row maximum needs only its weight's exponent), two values
// per packed instruction.  A block builds only the variants that the
// contractions of its row group's sources read.
template <int S>
__global__ void __launch_bounds__(256) k_prep_a(const MxPrepAArgs a) {
    constexpr int NW = 256 / 32;
    static_assert(MX_SB == 32 * NW, "one scale block per pass of the block");
    __shared__ int wmax[2][NW][8][MX_NA];
    extern __shared__ float2 kept[];                        // [8 m][MX_NA][256]: values of pass 1
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int q8 = lane & 7, kg = lane >> 3;
    const MxLayout &L = a.L;
    int blk = blockIdx.x;
    const int o = blk % (MX_ROWS / 8);
    blk /= MX_ROWS / 8;
    const int b = blk % L.NBA;
    blk /= L.NBA;
    const int rg = blk % L.NRG;
    const int pi = blk / L.NRG;
    const int r = 8 * o + q8;                            // row in the 128-row tile
    const int slot = r / L.BI, ii = r % L.BI;
    const int s = rg * L.SRC + slot;
    const int i = b * L.BI + ii;
    const long long row_global = ((long long)rg * L.NB + b) * MX_ROWS + r;
    const long long nrows = (long long)L.NRG * L.NB * MX_ROWS;
    const bool live = s < a.nsrc;
    const int cap = live ? a.l3cap[s] : -1;
    int vmask = 0;   // the same for the whole block (its rows lie in one row group)
    for (int x = 0; x < L.SRC; ++x)
        if (rg * L.SRC + x < a.nsrc) vmask |= variants_of_role(a.src_role[rg * L.SRC + x]);
    vmask &= a.alpha_mask;
    const float *Ah = a.Ah + (size_t)(live ? s : 0) * a.a_stride;
    const float *Al = a.Al + (size_t)(live ? s : 0) * a.a_stride;
    const int *Ae = a.Ae + (size_t)(live ? s : 0) * a.a_stride;

    int emax[MX_NA];
#pragma unroll
    for (int q = 0; q < MX_NA; ++q) emax[q] = EXP_ZERO;
    const int sb0 = (b * L.BI) / MX_SB;
    const int sb_end = (L.NKBA * L.KB + MX_SB - 1) / MX_SB;
    for (int sb = sb0; sb < sb_end; ++sb) {
        const int k0 = sb * MX_SB + 32 * w + 8 * kg;
        // ---- pass 1: maxima of the value exponents over the row's scale block
        int bmax[MX_NA];
#pragma unroll
        for (int q = 0; q < MX_NA; ++q) bmax[q] = EXP_ZERO;
#pragma unroll 1
        for (int m = 0; m < 8; ++m) {
            dfl val[MX_NA];
            int vex[MX_NA];
            a_values(a, vmask, Ah, Al, Ae, cap, i, k0 + m, pi, val, vex);
#pragma unroll
            for (int q = 0; q < MX_NA; ++q) {
                if (!((vmask >> q) & 1)) continue;
                bmax[q] = max(bmax[q], vex[q]);
                kept[(m * MX_NA + q) * 256 + tid] = make_float2(val[q].h, val[q].l);
            }
        }
        const int buf = sb & 1;
#pragma unroll
        for (int q = 0; q < MX_NA; ++q) {
            int v = max(bmax[q], __shfl_xor_sync(0xffffffffu, bmax[q], 8));
            v = max(v, __shfl_xor_sync(0xffffffffu, v, 16));
            if (kg == 0) wmax[buf][w][q8][q] = v;
        }
        __syncthreads();
        int E[MX_NA];
#pragma unroll
        for (int q = 0; q < MX_NA; ++q) {
            E[q] = EXP_ZERO;
#pragma unroll
            for (int x = 0; x < NW; ++x) E[q] = max(E[q], wmax[buf][x][q8][q]);
            emax[q] = max(emax[q], E[q]);
            if (w == 0 && kg == 0 && ((vmask >> q) & 1))
                a.eA[(((long long)pi * MX_NA + q) * nrows + row_global) * L.NSB + sb] = (int16_t)E[q];
        }
        // ---- pass 2: limbs of the 8 values, one 16-byte store per limb and variant
        const int kb = k0 / L.KB;
        if (kb < L.fA * b || kb >= L.NKBA) continue;
#pragma unroll
        for (int q = 0; q < MX_NA; ++q) {
            if (!((vmask >> q) & 1)) continue;
            uint32_t pk[S][4];
#pragma unroll
            for (int mp = 0; mp < 4; ++mp) {
                // values m = 2 mp (x lane, low half of each word) and 2 mp + 1 (y lane)
                float yv[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
#pragma unroll
                for (int x = 0; x < 2; ++x) {
                    const int m = 2 * mp + x;
                    const float2 kv = kept[(m * MX_NA + q) * 256 + tid];
                    if (kv.x != 0.f && E[q] != EXP_ZERO) {
                        // y = x 2^(7 - E), x = val 2^(vex - ilogb(val) - 1) = val 2^(weight exponent)
                        const int l3 = q < 3 ? 2 * (k0 + m) + pi : 2 * (k0 + m) + 1 - pi;
                        const int sh = Ae[l3] + 7 - E[q];
                        yv[x][0] = scale2(kv.x, sh);
                        yv[x][1] = scale2(kv.y, sh);
                    }
                }
                float2 yh = make_float2(yv[0][0], yv[1][0]), yl = make_float2(yv[0][1], yv[1][1]);
#pragma unroll
                for (int t = 0; t < S; ++t) {
                    // digit l = rint(yh); the rest (yh - l) + yl by a fast two-sum, which is
                    // exact here: yh - l is exact, and when it is nonzero it is at least
                    // ulp(yh) >= 2 |yl|
                    const float2 l = make_float2(rintf(yh.x), rintf(yh.y));
                    const float2 d = f2sub(yh, l);
                    const float2 sm = __fadd2_rn(d, yl);
                    const float2 er = f2sub(yl, f2sub(sm, d));
                    yh = __fmul2_rn(sm, make_float2(256.0f, 256.0f));
                    yl = __fmul2_rn(er, make_float2(256.0f, 256.0f));
                    const float sc = pow2f(-8 * t);
                    const float2 lv = __fmul2_rn(l, make_float2(sc, sc));
                    const __nv_bfloat162 b2 = __floats2bfloat162_rn(lv.x, lv.y);   // .x in the low half
                    pk[t][mp] = *reinterpret_cast<const uint32_t *>(&b2);
                }
            }
            uint8_t *img = a.Aimg + mx_a_off(L, pi, q, rg, b, kb, 0) + mx_img_off(r, k0 % L.KB, L.KB);
#pragma unroll
            for (int t = 0; t < S; ++t)
                *reinterpret_cast<uint4 *>(img + (size_t)t * L.IMG) = make_uint4(pk[t][0], pk[t][1], pk[t][2], pk[t][3]);
        }
    }
    if (w == 0 && kg == 0) {
#pragma unroll
        for (int q = 0; q < MX_NA; ++q)
            if ((vmask >> q) & 1) a.emaxA[((long long)pi * MX_NA + q) * nrows + row_global] = (int16_t)emax[q];
    }
}

// One warp per (parity, j) for the column blocks [c_lo, c_hi): all six variants.
template <int S>
__global__ void __launch_bounds__(256) k_prep_b(const MxPrepBArgs a, int c_hi) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const MxLayout &L = a.L;
    const int nj = (c_hi - a.c_lo) * MX_BJ;
    if (warp >= 2 * nj) return;
    const int j = a.c_lo * MX_BJ + warp % nj;
    const int pi = warp / nj;
    const int c = j / MX_BJ, jj = j % MX_BJ;
    const long long ncols = (long long)L.NC_B * MX_BJ;
    int emax[MX_NBV];
#pragma unroll
    for (int q = 0; q < MX_NBV; ++q) emax[q] = EXP_ZERO;
    const int nkb_c = L.gB * (c + 1);   // k blocks stored for this column block
    const int sb_hi = (nkb_c * L.KB - 1) / MX_SB;
    for (int sb = 0; sb <= sb_hi; ++sb) {
        dfl val[MX_NBV][MPL];
        int bexp[MX_NBV];
#pragma unroll
        for (int q = 0; q < MX_NBV; ++q) bexp[q] = EXP_ZERO;
#pragma unroll
        for (int m = 0; m < MPL; ++m) {
            const int k = sb * MX_SB + lane + 32 * m;
#pragma unroll
            for (int q = 0; q < MX_NBV; ++q) val[q][m] = {0.f, 0.f};
            // even: b0 = g(j-k) h(j+k+pi), u = (2j+2k+2pi+2)(2j-2k+1)
            if (k <= j) {
                const dfl b0 = df_mul(dfl{a.gh[j - k], a.gl[j - k]}, dfl{a.hh[j + k + pi], a.hl[j + k + pi]});
                const dfl u = df_int_prod(2 * j + 2 * k + 2 * pi + 2, 2 * j - 2 * k + 1);
                val[0][m] = b0;
                val[1][m] = df_mul(b0, u);
                val[2][m] = df_mul(val[1][m], u);
            }
            // odd: b1 = g(j-k+pi) h(j+k+1), u1 = (2j+2k+3)(2j-2k+2pi), u' = (2j+2k+4)(2j-2k+2pi+1)
            if (k <= j + pi - 1) {
                const dfl b1 = df_mul(dfl{a.gh[j - k + pi], a.gl[j - k + pi]}, dfl{a.hh[j + k + 1], a.hl[j + k + 1]});
                const dfl u1 = df_int_prod(2 * j + 2 * k + 3, 2 * j - 2 * k + 2 * pi);
                const dfl up = df_int_prod(2 * j + 2 * k + 4, 2 * j - 2 * k + 2 * pi + 1);
                val[3][m] = df_mul(b1, u1);
                val[4][m] = df_mul(val[3][m], up);
                val[5][m] = df_mul(val[4][m], up);
            }
#pragma unroll
            for (int q = 0; q < MX_NBV; ++q)
                if (val[q][m].h != 0.f) bexp[q] = max(bexp[q], value_exp(val[q][m], 0));
        }
#pragma unroll
        for (int q = 0; q < MX_NBV; ++q) {
            const int E = warp_max(bexp[q]);
            if (lane == 0) a.eB[(((long long)pi * MX_NBV + q) * ncols + j) * L.NSB_B + sb] = (int16_t)E;
            emax[q] = max(emax[q], E);
#pragma unroll
            for (int m = 0; m < MPL; ++m) {
                const int k = sb * MX_SB + lane + 32 * m;
                const int kb = k / L.KB;
                if (kb >= nkb_c) continue;
                dfl y = {0.f, 0.f};
                if (val[q][m].h != 0.f && E != EXP_ZERO) {
                    const int sh = 7 - E;
                    y.h = scale2(val[q][m].h, sh);
                    y.l = scale2(val[q][m].l, sh);
                }
                uint8_t *img = a.Bimg + mx_b_off(L, pi, q, c, kb, 0);
                put_limbs<S>(img, mx_img_off(jj, k % L.KB, L.KB), y, L.IMG);
            }
        }
    }
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < MX_NBV; ++q) a.emaxB[((long long)pi * MX_NBV + q) * ncols + j] = (int16_t)emax[q];
    }
}

}  // namespace

cudaError_t mx_launch_tables_dd(const double *g, const double *h, int n, float *gh, float *gl, float *hh,
                                float *hl, cudaStream_t st) {
    k_tables_dd<<<(n + 255) / 256, 256, 0, st>>>(g, h, n, gh, gl, hh, hl);
    return cudaGetLastError();
}

cudaError_t mx_launch_weights_dd(const double *A, int n_src, int a_stride, float *Ah, float *Al, int *Ae,
                                 cudaStream_t st) {
    const int total = n_src * a_stride;
    k_weights_dd<<<(total + 255) / 256, 256, 0, st>>>(A, total, Ah, Al, Ae);
    return cudaGetLastError();
}

cudaError_t mx_launch_prep_a(const MxPrepAArgs &a, cudaStream_t st) {
    const long long octets = 2LL * a.L.NRG * a.L.NBA * (MX_ROWS / 8);
    if (octets == 0) return cudaSuccess;
    if (a.L.BI < 8 || a.L.KB % 8 != 0) return cudaErrorInvalidValue;
    const int blocks = (int)octets;
    const int smem = 8 * MX_NA * 256 * (int)sizeof(float2);   // the kept values
    static std::atomic<unsigned long long> attr[3];
    cudaError_t e;
    switch (a.L.S) {
        case 4:
            if ((e = opt_in_smem(k_prep_a<4>, smem, attr[0])) != cudaSuccess) return e;
            k_prep_a<4><<<blocks, 256, smem, st>>>(a);
            break;
        case 5:
            if ((e = opt_in_smem(k_prep_a<5>, smem, attr[1])) != cudaSuccess) return e;
            k_prep_a<5><<<blocks, 256, smem, st>>>(a);
            break;
        case 6:
            if ((e = opt_in_smem(k_prep_a<6>, smem, attr[2])) != cudaSuccess) return e;
            k_prep_a<6><<<blocks, 256, smem, st>>>(a);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t mx_launch_prep_b(const MxPrepBArgs &a, int c_hi, cudaStream_t st) {
    if (c_hi <= a.c_lo) return cudaSuccess;
    const long long warps = 2LL * (c_hi - a.c_lo) * MX_BJ;
    const int blocks = (int)((warps * 32 + 255) / 256);
    switch (a.L.S) {
        case 4: k_prep_b<4><<<blocks, 256, 0, st>>>(a, c_hi); break;
        case 5: k_prep_b<5><<<blocks, 256, 0, st>>>(a, c_hi); break;
        case 6: k_prep_b<6><<<blocks, 256, 0, st>>>(a, c_hi); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace cpl
