// mixed_gemm.cu -- the tcgen05 limb GEMM of the mixed-precision path.
//
// A work item is one (job, parity, contraction p, row group, i-block, j-block):
//   C[r, c] = sum_k x[r, k] y[c, k]   (128 x 128 output, k over the item's range)
// with x, y given as S BF16 fixed-point limbs per element (mixed.h).  The
// kernel is persistent: each CTA takes the next item of a list with an
// atomic ticket (the producer lane draws it and passes it to the MMA and
// drain roles through a 4-slot ring in shared memory), keeps one TMEM
// allocation and carries its pipeline counters across items, so one launch
// serves a whole batch of requests (MxJob) and the write-out of an item
// overlaps the MMAs of the next.
//
// Warp roles (18 warps):
//   warp 0      producer: one elected lane streams the KB-k tile images of
//               all limbs of x and y into a shared-memory ring (2 stages of
//               32 k for S <= 5 limbs, 3 stages of 16 k for S = 6) with
//               cp.async.bulk, signalling an mbarrier with the byte count.
//   warp 1      allocates 512 TMEM columns; one elected lane issues, for each
//               16-k step, the limb products x_t y_u with t + u < S as
//               tcgen05.mma (M=128, N=128, K=16, BF16 in, FP32 accumulate)
//               into four TMEM accumulators by order t + u = 0, 1, 2, >= 3,
//               and commits each stage back to the producer.
//   warps 2-17  drain: after every 256-k scale block, read the four
//               accumulators with tcgen05.ld, combine them, scale by
//               2^(E_row + E_col) relative to the row / column maxima, and add
//               into a double-float running sum per element (high part in
//               registers, low part in shared memory, renormalised once at
//               the end).
// The four accumulators fill TMEM, so they cannot be double-buffered; instead
// they are released in two steps.  The drain loads the order >= 3
// accumulator first and releases it at once; the MMA lane then issues the
// order >= 3 products (15 of the 21 for S = 6) of the next block's first
// stages while the drain still reads and combines orders 0-2, and issues
// their order 0-2 products once those three accumulators are released too.
// The accumulators of orders 0, 1 and 2 are integers below 2^24 in their
// units over a 256-k block (|limb| <= 128, at most 3 products per k), so the
// tensor core holds them exactly whatever its internal rounding; only the
// order >= 3 accumulator, 2^-24 of the total, is inexact.  (Measured: with
// orders >= 2 in one inexact accumulator the error reached 5e-9, consistent
// with truncating accumulation.)
// Every wait on an mbarrier is bounded (2 s of globaltimer); on expiry the
// CTA records an error code, stops issuing, waits (bounded) for the work it
// already issued, frees its TMEM and exits.
#include <cuda_runtime.h>

#include "dd.cuh"
#include "mbar.cuh"
#include "mixed.h"

namespace cpl {
namespace {

constexpr int NTH = 576;                   // 2 control warps + 16 drain warps (96 registers each)
constexpr int LPAD = MX_ROWS + 1;          // padded stride of the [col][row] planes
__device__ __forceinline__ void umma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}
// K-major, no-swizzle shared-memory matrix descriptor: core matrices of
// 8 rows x 16 bytes; LBO = offset between K-adjacent cores (128 B), SBO =
// offset between 8-row groups (KB * 16 B); bits 46-47 = descriptor version 1.
template <int KB>
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)(128 >> 4) << 16;
    d |= (uint64_t)((KB * 16) >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}
__device__ __forceinline__ void umma(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{ .reg .pred p; setp.ne.u32 p, %4, 0; tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(
            tmem_d),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
        : "memory");
}

#define TMEM_LD8(addr, r)                                                                    \
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"        \
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), \
                   "=r"(r[7])                                                                      \
                 : "r"(addr))

#define TMEM_LD4(addr, r)                                                                    \
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"                   \
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])                                  \
                 : "r"(addr))

constexpr int TQ = 4;                      // ticket ring slots

// Packed FP32 pairs (sm_100+ f32x2 instructions): the drain handles two
// adjacent columns of a row per instruction.
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;"
        : "=l"(r)
        : "l"(*reinterpret_cast<unsigned long long *>(&a)), "l"(*reinterpret_cast<unsigned long long *>(&b)));
    return *reinterpret_cast<float2 *>(&r);
}
struct dfl2 {
    float2 h, l;
};
// error-free sum of two packed pairs (Knuth two-sum, lane-wise)
__device__ __forceinline__ dfl2 two_sum2(float2 a, float2 b) {
    const float2 s = __fadd2_rn(a, b);
    const float2 bb = f2sub(s, a);
    const float2 e = __fadd2_rn(f2sub(a, f2sub(s, bb)), f2sub(b, bb));
    return {s, e};
}
__device__ __forceinline__ float2 u2f2(uint32_t a, uint32_t b) { return make_float2(__uint_as_float(a), __uint_as_float(b)); }
// 2^e as a float for the scale factors of a block: 0 below 2^-126 (such a
// block is below 2^-126 of the element's largest block)
__device__ __forceinline__ float pow2_or_zero(int e) { return e < -126 ? 0.0f : pow2f(min(e, 0)); }

// Stages at the start of a scale block whose order >= 3 products are issued
// before the accumulators of orders 0-2 are free again (see the MMA issuer).
template <int S>
__host__ __device__ constexpr int mx_npre() { return S >= 6 ? 3 : 1; }

struct Shared {
    uint64_t full[3], empty[3], acc_full, acc_empty3, acc_empty012, done;
    uint64_t tfull[TQ], tempty[TQ];
    int tick[TQ];
    uint32_t tmem;
    int abort;          // set by any role on a timed-out wait
    int dabort;         // drain-local copy, written only before the drain barrier
    float2 fcol[MX_BJ / 2];   // per column pair: 2^(E_col(block) - E_col(max)), or 0
};

template <int S>
__global__ void __launch_bounds__(NTH, 1) k_mixed_gemm(const MxGemmArgs a) {
    extern __shared__ __align__(128) uint8_t dsm[];
    __shared__ Shared sh;
    constexpr int KB = mx_kb(S);                 // k per stage
    constexpr int IMG = mx_img_bytes(S);
    constexpr int NST = mx_stages(S);
    constexpr int KPS = MX_SB / KB;              // k blocks per scale block
    constexpr uint32_t STAGE = 2u * S * IMG;
    float2 *Ls = reinterpret_cast<float2 *>(dsm + NST * STAGE);   // [64 column pairs][LPAD]

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t s_full0 = mbar::smem_u32(&sh.full[0]), s_empty0 = mbar::smem_u32(&sh.empty[0]);
    const uint32_t s_accf = mbar::smem_u32(&sh.acc_full), s_done = mbar::smem_u32(&sh.done);
    const uint32_t s_acce3 = mbar::smem_u32(&sh.acc_empty3), s_acce012 = mbar::smem_u32(&sh.acc_empty012);

    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(mbar::smem_u32(&sh.tmem)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int q = 0; q < NST; ++q) {
            mbar::init(s_full0 + 8 * q, 1);
            mbar::init(s_empty0 + 8 * q, 1);
        }
        mbar::init(s_accf, 1);
        mbar::init(s_acce3, 16);
        mbar::init(s_acce012, 16);
        mbar::init(s_done, 1);
        for (int q = 0; q < TQ; ++q) {
            mbar::init(mbar::smem_u32(&sh.tfull[q]), 1);
            mbar::init(mbar::smem_u32(&sh.tempty[q]), 2);   // MMA lane + drain
        }
        sh.abort = 0;
        sh.dabort = 0;
        mbar::fence_init();
        asm volatile("fence.proxy.async.shared::cta;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = sh.tmem;
    const uint32_t stage_base = mbar::smem_u32(dsm);

    // Every role takes the items in ticket order and keeps its pipeline
    // counters running across items, so the mbarrier phases stay in step.
    if (warp == 0) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            int n = 0;
            for (int nt = 0; !*(volatile int *)&sh.abort; ++nt) {
                // draw a ticket and publish it
                const int ts = nt % TQ;
                if (nt >= TQ && !mbar::wait(mbar::smem_u32(&sh.tempty[ts]), ((nt / TQ) - 1) & 1)) {
                    atomicExch(a.err, 17);
                    sh.abort = 1;
                    break;
                }
                int w = atomicAdd(a.ticket, 1);
                if (w >= a.n_items) w = -1;
                sh.tick[ts] = w;
                mbar::arrive(mbar::smem_u32(&sh.tfull[ts]));
                if (w < 0) break;
                const MxItem it = a.items[w];
                const MxJob &J = a.jobs[it.job];
                const MxLayout &L = J.L;
                const int alpha = mx_alpha(it.p), beta = mx_beta(it.p);
                const uint8_t *Ab = J.Aimg + mx_a_off(L, it.pi, alpha, it.rg, it.b, L.fA * it.b, 0);
                for (int kb = it.kb_lo; kb <= it.kb_hi; ++kb, ++n) {
                    if (*(volatile int *)&sh.abort) break;
                    const int s = n % NST, u = n / NST;
                    if (u > 0 && !mbar::wait(s_empty0 + 8 * s, (u - 1) & 1)) {
                        atomicExch(a.err, 11);
                        sh.abort = 1;
                        break;
                    }
                    const uint32_t fb = s_full0 + 8 * s;
                    mbar::expect_tx(fb, STAGE);
                    const uint8_t *asrc = Ab + (long long)(kb - L.fA * it.b) * S * IMG;
                    const uint8_t *bsrc = a.Bimg + mx_b_off(L, it.pi, beta, it.c, kb, 0);
                    const uint32_t dst = stage_base + s * STAGE;
                    mbar::copy_g2s(dst, asrc, S * IMG, fb);
                    mbar::copy_g2s(dst + S * IMG, bsrc, S * IMG, fb);
                }
            }
            // wait (bounded) for the copies still in flight before the CTA may exit
            for (int q = n - NST; q < n; ++q) {
                if (q < 0) continue;
                if (!mbar::wait(s_full0 + 8 * (q % NST), (q / NST) & 1)) atomicExch(a.err, 12);
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(MX_BJ >> 3) << 17) |
                                   ((uint32_t)(MX_ROWS >> 4) << 24);
            // Issues the limb products of one stage whose order t + u lies in
            // [olo, ohi] (orders >= 3 share accumulator 3); a product is the
            // first of its accumulator in the scale block when flagged so.
            auto issue = [&](int s, int olo, int ohi, bool first3, bool first012) {
                const uint32_t abase = stage_base + s * STAGE;
                const uint32_t bbase = abase + S * IMG;
#pragma unroll
                for (int k16 = 0; k16 < KB / 16; ++k16) {
#pragma unroll
                    for (int t = 0; t < S; ++t) {
#pragma unroll
                        for (int u = 0; u + t < S; ++u) {
                            if (t + u < olo || t + u > ohi) continue;
                            const int acc = (t + u) < 3 ? (t + u) : 3;
                            // the first product of each accumulator (lowest t for that order,
                            // k16 = 0) overwrites it; the rest accumulate
                            const bool first = k16 == 0 && (acc == 3 ? (first3 && t == 0 && u == 3)
                                                                     : (first012 && t == 0));
                            const uint64_t ad = umma_desc<KB>(abase + t * IMG + k16 * 256);
                            const uint64_t bd = umma_desc<KB>(bbase + u * IMG + k16 * 256);
                            umma(tmem + acc * MX_BJ, ad, bd, idesc, first ? 0u : 1u);
                        }
                    }
                }
            };
            constexpr int NPRE = mx_npre<S>();
            int n = 0, m = 0;
            bool bad = false;
            for (int nt = 0; !bad && !*(volatile int *)&sh.abort; ++nt) {
                const int ts = nt % TQ;
                if (!mbar::wait(mbar::smem_u32(&sh.tfull[ts]), (nt / TQ) & 1)) {
                    atomicExch(a.err, 18);
                    sh.abort = 1;
                    break;
                }
                const int w = *(volatile int *)&sh.tick[ts];
                mbar::arrive(mbar::smem_u32(&sh.tempty[ts]));
                if (w < 0) break;
                const MxItem it = a.items[w];
                // one scale block (the item's k blocks inside one 256-k block) per pass
                for (int kb = it.kb_lo; kb <= it.kb_hi;) {
                    if (*(volatile int *)&sh.abort) { bad = true; break; }
                    const int kend = min((int)it.kb_hi, (kb / KPS) * KPS + KPS - 1);
                    const int nkb = kend - kb + 1;
                    const int pre = min(NPRE, nkb);
                    // (1) accumulator 3 is free once the drain has loaded it: the
                    // order >= 3 products of the block's first `pre` stages run
                    // while the drain still combines orders 0-2 of the last block
                    if (m > 0 && !mbar::wait(s_acce3, (m - 1) & 1)) {
                        atomicExch(a.err, 13);
                        bad = true;
                        break;
                    }
                    for (int q = 0; q < pre && !bad; ++q) {
                        const int s = (n + q) % NST;
                        if (!mbar::wait(s_full0 + 8 * s, ((n + q) / NST) & 1)) {
                            atomicExch(a.err, 14);
                            bad = true;
                            break;
                        }
                        asm volatile("tcgen05.fence::after_thread_sync;");
                        issue(s, 3, S - 1, q == 0, false);
                    }
                    if (bad) break;
                    // (2) then orders 0-2 of those stages, once their accumulators are free
                    if (m > 0 && !mbar::wait(s_acce012, (m - 1) & 1)) {
                        atomicExch(a.err, 13);
                        bad = true;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    for (int q = 0; q < pre; ++q) {
                        const int s = (n + q) % NST;
                        issue(s, 0, 2, false, q == 0);
                        umma_commit(s_empty0 + 8 * s);
                    }
                    // (3) the block's remaining stages, all orders
                    for (int q = pre; q < nkb; ++q) {
                        const int s = (n + q) % NST;
                        if (!mbar::wait(s_full0 + 8 * s, ((n + q) / NST) & 1)) {
                            atomicExch(a.err, 14);
                            bad = true;
                            break;
                        }
                        asm volatile("tcgen05.fence::after_thread_sync;");
                        issue(s, 0, S - 1, false, false);
                        umma_commit(s_empty0 + 8 * s);
                    }
                    if (bad) break;
                    umma_commit(s_accf);
                    ++m;
                    n += nkb;
                    kb = kend + 1;
                }
            }
            if (bad) sh.abort = 1;
            // all issued MMAs complete before TMEM is released
            umma_commit(s_done);
            if (!mbar::wait(s_done, 0)) atomicExch(a.err, 15);
        }
    } else {
        // ------------------------------------------------------------ drain
        // 16 warps: warp (2 + dw) reads TMEM lane quarter (warp & 3) and
        // columns [32 (dw >> 2), +32); one thread per (row, 32 columns).
        const int dw = warp - 2;
        const int q = warp & 3, quarter = dw >> 2;
        const int row = 32 * q + lane, c0 = 32 * quarter;
        const int dtid = tid - 64;               // 0..511
        const uint32_t lane_addr = tmem + ((uint32_t)(32 * q) << 16);
        int m = 0;
        for (int nt = 0;; ++nt) {
            const int ts = nt % TQ;
            const bool tok = !*(volatile int *)&sh.abort && mbar::wait(mbar::smem_u32(&sh.tfull[ts]), (nt / TQ) & 1);
            if (!tok) sh.dabort = 1;
            const int w = *(volatile int *)&sh.tick[ts];
            // (T): every drain thread has read the ticket; the abort decision is uniform
            asm volatile("bar.sync 1, 512;" ::: "memory");
            if (*(volatile int *)&sh.dabort) {
                if (dtid == 0) {
                    atomicExch(a.err, 19);
                    sh.abort = 1;
                }
                break;
            }
            if (w < 0) break;
            if (dtid == 0) mbar::arrive(mbar::smem_u32(&sh.tempty[ts]));
            bool stop = false;
            const MxItem it = a.items[w];
            const MxJob &J = a.jobs[it.job];
            const MxLayout &L = J.L;
            const int alpha = mx_alpha(it.p), beta = mx_beta(it.p);
            const long long nrows = (long long)L.NRG * L.NB * MX_ROWS;
            const long long ncols = (long long)L.NC_B * MX_BJ;
            const long long rowg = ((long long)it.rg * L.NB + it.b) * MX_ROWS + row;
            const int16_t *eArow = J.eA + (((long long)it.pi * MX_NA + alpha) * nrows + rowg) * L.NSB;
            const int emA = J.emaxA[((long long)it.pi * MX_NA + alpha) * nrows + rowg];
            const int j0 = it.c * MX_BJ;
            const int16_t *eBcol = a.eB + ((long long)it.pi * MX_NBV + beta) * ncols * L.NSB_B;
            const int16_t *emB = a.emaxB + ((long long)it.pi * MX_NBV + beta) * ncols;
            // running sum per element: high part in registers, low part (left
            // unnormalised until the end) in shared memory; each thread owns
            // its 32 cells of Ls, so no barrier is needed around the reset
            float2 H[16];
#pragma unroll
            for (int x = 0; x < 16; ++x) H[x] = make_float2(0.f, 0.f);
            for (int x = 0; x < 16; ++x) Ls[(c0 / 2 + x) * LPAD + row] = make_float2(0.f, 0.f);
            for (int kb = it.kb_lo; kb <= it.kb_hi; ++kb) {
                const bool slast = (kb == it.kb_hi) || (kb % KPS == KPS - 1);
                if (!slast) continue;
                const int sb = kb / KPS;
                if (dtid < MX_BJ) {
                    const int j = j0 + dtid;
                    reinterpret_cast<float *>(sh.fcol)[dtid] =
                        pow2_or_zero((int)eBcol[(long long)j * L.NSB_B + sb] - (int)emB[j]);
                }
                const float fa = pow2_or_zero((int)eArow[sb] - emA);
                const float2 fa2 = make_float2(fa, fa);
                const bool ok = !*(volatile int *)&sh.abort && mbar::wait(s_accf, m & 1);
                if (!ok) sh.dabort = 1;
                // (A): column exponents visible; the abort decision is the same for all drain threads
                asm volatile("bar.sync 1, 512;" ::: "memory");
                if (*(volatile int *)&sh.dabort) {
                    if (dtid == 0) {
                        atomicExch(a.err, 16);
                        sh.abort = 1;
                    }
                    stop = true;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                // order >= 3 first: once it is in registers its accumulator is
                // released, and the MMAs of the next block start on it; its
                // values join the low parts below (one update of the shared
                // low part per element and block)
                uint32_t r3[32];
#pragma unroll
                for (int g = 0; g < 4; ++g) TMEM_LD8(lane_addr + 3 * MX_BJ + (uint32_t)(c0 + 8 * g), (r3 + 8 * g));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;");
                __syncwarp();
                if (lane == 0) mbar::arrive(s_acce3);
#pragma unroll
                for (int g = 0; g < 8; ++g) {
                    uint32_t r0[4], r1[4], r2[4];
                    const uint32_t col = (uint32_t)(c0 + 4 * g);
                    TMEM_LD4(lane_addr + col, r0);
                    TMEM_LD4(lane_addr + MX_BJ + col, r1);
                    TMEM_LD4(lane_addr + 2 * MX_BJ + col, r2);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    if (g == 7) {
                        // orders 0-2 are in registers: release their accumulators
                        asm volatile("tcgen05.fence::before_thread_sync;");
                        __syncwarp();
                        if (lane == 0) mbar::arrive(s_acce012);
                    }
#pragma unroll
                    for (int x = 0; x < 4; x += 2) {
                        const int cp = (c0 + 4 * g + x) / 2;   // column pair
                        // scale of this block relative to the element's frame (0 if negligible)
                        const float2 F = __fmul2_rn(fa2, sh.fcol[cp]);
                        // block value: orders 0, 1 and 2 summed exactly (two two-sums:
                        // with decaying operands order 2 can reach 2^-8 of order 0, so
                        // it must not be folded into the residue of the first sum);
                        // the residues and order >= 3 are then added in FP32
                        const dfl2 v01 = two_sum2(u2f2(r0[x], r0[x + 1]), u2f2(r1[x], r1[x + 1]));
                        const dfl2 v = two_sum2(v01.h, u2f2(r2[x], r2[x + 1]));
                        const float2 vlo = __fadd2_rn(__fadd2_rn(v01.l, v.l), u2f2(r3[4 * g + x], r3[4 * g + x + 1]));
                        const dfl2 z = two_sum2(H[2 * g + x / 2], __fmul2_rn(v.h, F));
                        H[2 * g + x / 2] = z.h;
                        float2 &ls = Ls[cp * LPAD + row];
                        ls = __fadd2_rn(ls, __fadd2_rn(z.l, __fmul2_rn(vlo, F)));
                    }
                }
                // (B): every drain thread is done with the column exponents
                asm volatile("bar.sync 1, 512;" ::: "memory");
                ++m;
            }
            if (stop) break;
            // ---- write the element sums, column-major: [plane][col][row]; per
            // column the 32 lanes of a warp store 32 consecutive rows.  The
            // accumulators are already released, so the MMA of the next item
            // runs meanwhile.
            float *dst = J.inter + ((long long)it.tile * MX_NPROD + it.p) * 2 * (MX_ROWS * MX_BJ);
#pragma unroll
            for (int x = 0; x < 16; ++x) {
                const float2 lo = Ls[(c0 / 2 + x) * LPAD + row];
                const dfl v0 = df_quick(H[x].x, lo.x), v1 = df_quick(H[x].y, lo.y);
                dst[(c0 + 2 * x) * MX_ROWS + row] = v0.h;
                dst[(c0 + 2 * x + 1) * MX_ROWS + row] = v1.h;
                dst[MX_ROWS * MX_BJ + (c0 + 2 * x) * MX_ROWS + row] = v0.l;
                dst[MX_ROWS * MX_BJ + (c0 + 2 * x + 1) * MX_ROWS + row] = v1.l;
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
    }
}

}  // namespace

size_t mx_gemm_smem_bytes(int S) {
    return (size_t)mx_stages(S) * 2 * S * mx_img_bytes(S) + (size_t)(MX_BJ / 2) * LPAD * sizeof(float2);
}

cudaError_t mx_gemm_prepare(int S) {
    const int smem = (int)mx_gemm_smem_bytes(S);
    switch (S) {
        case 4: return cudaFuncSetAttribute(k_mixed_gemm<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        case 5: return cudaFuncSetAttribute(k_mixed_gemm<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        case 6: return cudaFuncSetAttribute(k_mixed_gemm<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t mx_launch_gemm(const MxGemmArgs &a, int S, int grid, cudaStream_t st) {
    if (a.n_items == 0) return cudaSuccess;
    if (grid <= 0 || grid > a.n_items) grid = a.n_items;
    const size_t smem = mx_gemm_smem_bytes(S);
    switch (S) {
        case 4: k_mixed_gemm<4><<<grid, NTH, smem, st>>>(a); break;
        case 5: k_mixed_gemm<5><<<grid, NTH, smem, st>>>(a); break;
        case 6: k_mixed_gemm<6><<<grid, NTH, smem, st>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace cpl
