// noalloc.cu -- cpl_build_noalloc: the plain FP64 build without device allocation.
//
// Some callers cannot call cudaMalloc: an application whose own allocator
// owns the whole device memory budget from start-up, a real-time pipeline
// that must never hit the implicit device synchronisation cudaMalloc /
// cudaFree can cause, or code running where allocation calls are not
// allowed.  For them this entry point runs the same separable FP64
// contraction as cpl_build (a variant of its kernel that takes its tile from
// the launch grid instead of a work list), but keeps its scratch -- the g / h
// lookup tables and the per-window l3 weights -- in one file-scope device
// array of fixed size, so nothing is allocated on the device at any call.
// The caller passes the windows and the output, both on the current device;
// the per-window l3 caps travel by value in the kernel arguments.
//
// The array lives in every GPU that loads this library until the process
// exits; host code cannot use its name as a device address, so its address
// is looked up once per device with cudaGetSymbolAddress, by the first call
// made on that device, which also writes the g / h tables into the array
// once, for the largest supported l_max (a table prefix does not depend on
// its length), with a synchronous host-to-device copy.  Make that first call
// before any stream capture.  Later calls only launch kernels: they read no
// host memory.  All calls share the array and it keeps the last call's
// contents: the tables never change after the set-up, and every call
// rewrites the weights it reads before using them; two calls whose work
// overlaps on the GPU (different streams without ordering, or different host
// threads) race on the weights.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"

namespace cpl {
namespace {

constexpr int NA_MAX_LMAX = 4096;
constexpr int NA_MAX_WINDOWS = 4;
constexpr size_t NA_SCRATCH_BYTES = size_t(1) << 20;   // 1 MiB
constexpr int NA_MAX_DEVICES = 64;
constexpr int NT = 256;
constexpr int KC = 16;

}  // namespace
}  // namespace cpl

// The scratch of cpl_build_noalloc (see the header comment above).
static __device__ __align__(256) unsigned char g_noalloc_scratch[cpl::NA_SCRATCH_BYTES];

namespace cpl {
namespace {

struct NaCaps {
    int v[NA_MAX_WINDOWS];   // last l3 with a nonzero weight, per window
};

struct NaArgs {
    const double *g, *h, *A;
    int a_stride;
    NaCaps l3cap;
    int lmax, lmin;
    double *out;
    int nspec;
    int slot[5];
};

// The same contraction as k_plain (plain_fp64.cu), dense output only; the
// epilogue forms the pair coefficients directly (the context path reads
// per-l factor tables, for which the fixed scratch array has no room), so the
// two agree to rounding.  The (parity, i-block) pair is blockIdx.y, the
// j-block blockIdx.x and the window blockIdx.z.  Blocks without a valid pair
// return at once.
// Exact product of two integer factors as a double (one 64-bit multiply and
// one conversion instead of two conversions and an FP64 multiply).
__device__ __forceinline__ double int_prod(int a, int b) { return (double)((long long)a * (long long)b); }

template <int NGE, bool ODD>
__global__ void __launch_bounds__(NT) k_plain_noalloc(const NaArgs p) {
    constexpr int NAE = NGE == 0 ? 0 : NGE == 1 ? 1 : NGE == 3 ? 2 : 3;
    constexpr int NBE = NAE;
    constexpr int NA = NAE + (ODD ? 1 : 0);
    constexpr int NB = NBE + (ODD ? 3 : 0);
    constexpr int NG = NGE + (ODD ? 3 : 0);
    __shared__ double sa[NA > 0 ? NA : 1][KC][TILE_I];
    __shared__ double sb[NB > 0 ? NB : 1][KC][TILE_J];

    const int pi = blockIdx.y & 1;
    const int i0 = (blockIdx.y >> 1) * TILE_I, j0 = blockIdx.x * TILE_J;
    const int win = blockIdx.z;
    // a valid pair exists iff one exists in the block's first row
    if (2 * i0 + pi > p.lmax - p.lmin) return;
    if (max(j0, i0 + p.lmin) > min(j0 + TILE_J - 1, p.lmax - pi - i0)) return;

    const double *__restrict__ A = p.A + (size_t)win * p.a_stride;
    const double *__restrict__ g = p.g;
    const double *__restrict__ h = p.h;
    const int cap = p.l3cap.v[win];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int kcap_e = (cap - pi) >> 1;
    const int kcap_o = (cap - 1 + pi) >> 1;
    const int khi_e = min(j0 + TILE_J - 1, kcap_e);
    const int khi_o = min(j0 + TILE_J - 2 + pi, kcap_o);
    int k_hi = -1;
    if (NGE > 0) k_hi = khi_e;
    if (ODD) k_hi = max(k_hi, khi_o);

    double acc[NG > 0 ? NG : 1][2][2];
#pragma unroll
    for (int q = 0; q < NG; ++q)
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int c = 0; c < 2; ++c) acc[q][r][c] = 0.0;

    for (int kb = i0; kb <= k_hi; kb += KC) {
        __syncthreads();
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
                if (NAE > 1) sa[1][kk][ii] = a0 * v;
                if (NAE > 2) sa[2][kk][ii] = a0 * v * v;
            }
            if (ODD) {
                double a1v = 0.0;
                if (k >= i + pi && k <= khi_o) {
                    const double v1 = int_prod(2 * i + 2 * k + 2, 2 * k + 1 - 2 * i - 2 * pi);
                    a1v = A[2 * k + 1 - pi] * g[i + k + 1] * g[k - i - pi] * v1;
                }
                sa[NAE][kk][ii] = a1v;
            }
        }
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
                if (NBE > 1) sb[1][kk][jj] = b0 * u;
                if (NBE > 2) sb[2][kk][jj] = b0 * u * u;
            }
            if (ODD) {
                double b1u = 0.0, up = 0.0;
                if (k <= j + pi - 1 && k <= khi_o) {
                    const double u1 = int_prod(2 * j + 2 * k + 3, 2 * j - 2 * k + 2 * pi);
                    up = int_prod(2 * j + 2 * k + 4, 2 * j - 2 * k + 2 * pi + 1);
                    b1u = g[j - k + pi] * h[j + k + 1] * u1;
                }
                sb[NBE][kk][jj] = b1u;
                sb[NBE + 1][kk][jj] = b1u * up;
                sb[NBE + 2][kk][jj] = b1u * up * up;
            }
        }
        __syncthreads();
        const int kn = min(KC, k_hi - kb + 1);
#pragma unroll 2
        for (int kk = 0; kk < kn; ++kk) {
            double a[NA > 0 ? NA : 1][2], b[NB > 0 ? NB : 1][2];
#pragma unroll
            for (int q = 0; q < NA; ++q) {
                a[q][0] = sa[q][kk][ty];
                a[q][1] = sa[q][kk][ty + 16];
            }
#pragma unroll
            for (int q = 0; q < NB; ++q) {
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
                        acc[NGE + 0][r][c] = fma(a[NAE][r], b[NBE][c], acc[NGE + 0][r][c]);
                        acc[NGE + 1][r][c] = fma(a[NAE][r], b[NBE + 1][c], acc[NGE + 1][r][c]);
                        acc[NGE + 2][r][c] = fma(a[NAE][r], b[NBE + 2][c], acc[NGE + 2][r][c]);
                    }
                }
        }
    }

    const int n = p.lmax - p.lmin + 1;
    auto put = [&](int slot, int l1, int l2, double xi) {
        if (slot < 0) return;
        double *base = p.out + ((size_t)win * p.nspec + slot) * (size_t)n * (size_t)n;
        base[(size_t)(l1 - p.lmin) * n + (l2 - p.lmin)] = (2.0 * l2 + 1.0) * xi;
        if (l1 != l2) base[(size_t)(l2 - p.lmin) * n + (l1 - p.lmin)] = (2.0 * l1 + 1.0) * xi;
    };
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int i = i0 + ty + 16 * r, j = j0 + tx + 16 * c;
            const int l1 = j - i, l2 = i + j + pi;
            if (l1 < p.lmin || l2 > p.lmax || l1 > l2) continue;
            if (NGE >= 1) put(p.slot[0], l1, l2, acc[0][r][c]);
            double ee = 0.0;
            if (NGE >= 3 || ODD) {
                const double L1 = l1, L2 = l2;
                const double eta2 = (L1 - 1.0) * (L1 + 2.0) * (L2 - 1.0) * L2;
                const double c1 = 1.0 / (L1 * (L1 + 1.0) * (L2 + 1.0));
                if (NGE >= 3) {
                    const double r2 = L1 * (L1 + 1.0) * (L2 + 1.0) * (L2 + 2.0) / eta2;
                    const double c0 = 1.0 + 2.0 / L1;
                    const double c2 = c1 / (2.0 * (L2 + 2.0));
                    const double s00 = acc[0][r][c], s01 = acc[1][r][c], s11 = acc[2][r][c];
                    put(p.slot[1], l1, l2, sqrt(r2) * (c0 * s00 - c1 * s01 - c2 * s11));
                    if (NGE >= 6) {
                        const double s02 = acc[3][r][c], s12 = acc[4][r][c], s22 = acc[5][r][c];
                        ee = r2 * (c0 * c0 * s00 - 2.0 * c0 * c1 * s01 - 2.0 * c0 * c2 * s11 +
                                   c1 * c1 * s02 + 2.0 * c1 * c2 * s12 + c2 * c2 * s22);
                        put(p.slot[2], l1, l2, ee);
                    }
                }
                if (ODD) {
                    const double e0 = L1 + 2.0, e1 = 1.0 / (2.0 * (L2 + 2.0));
                    const double Cc = (L2 + 2.0) * c1 / eta2;
                    const double t0 = acc[NGE][r][c], t1 = acc[NGE + 1][r][c], t2 = acc[NGE + 2][r][c];
                    const double eebb = Cc * (e0 * e0 * t0 - 2.0 * e0 * e1 * t1 + e1 * e1 * t2);
                    put(p.slot[3], l1, l2, eebb);
                    if (NGE >= 6) put(p.slot[4], l1, l2, ee - eebb);
                }
            }
        }
}

// Weights A(l3) = (2 l3 + 1) W(l3) / (4 pi), zero above the window's cap and
// up to a_stride: the formula and rounding of the context path's weight
// kernel, with the caps taken by value.
__global__ void k_weights_noalloc(const double *__restrict__ W, int w_len, const NaCaps caps,
                                  double *__restrict__ A, int a_stride) {
    const int win = blockIdx.y;
    const int cap = caps.v[win];
    const double inv4pi = 0.07957747154594767;   // 1 / (4 pi)
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < a_stride; l += gridDim.x * blockDim.x) {
        double v = 0.0;
        if (l <= cap && l < w_len) v = (2.0 * l + 1.0) * W[(size_t)win * w_len + l] * inv4pi;
        A[(size_t)win * a_stride + l] = v;
    }
}

// Scratch layout: g | h (both for p <= NA_PMAX, written once per device) |
// A[role][window][a_stride] (rewritten by every call).
constexpr int NA_PMAX = 2 * NA_MAX_LMAX + 2 * (TILE_I + TILE_J) + 16;
constexpr size_t NA_OFF_G = 0;
constexpr size_t NA_OFF_H = (NA_OFF_G + sizeof(double) * (NA_PMAX + 1) + 255) & ~size_t(255);
constexpr size_t NA_OFF_A = (NA_OFF_H + sizeof(double) * (NA_PMAX + 1) + 255) & ~size_t(255);
static_assert(NA_OFF_A + sizeof(double) * (2 * NA_MAX_LMAX + 2) * NA_MAX_WINDOWS * 3 <= NA_SCRATCH_BYTES,
              "the largest request must fit the no-allocation scratch");

std::mutex g_na_mutex;
unsigned char *g_na_ptr[NA_MAX_DEVICES] = {};

// Set-up on `dev` (the current device), once: the device address of
// g_noalloc_scratch, and the g / h tables written into it.
cpl_status na_scratch(int dev, unsigned char **ptr) {
    if (dev < 0 || dev >= NA_MAX_DEVICES) return fail(CPL_ERR_RANGE, "device index too large");
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(CPL_ERR_CUDA, std::string("cudaGetSymbolAddress of the no-allocation scratch failed: ") +
                                          cudaGetErrorString(e));
        unsigned char *base = static_cast<unsigned char *>(p);
        std::vector<double> g, h;
        build_tables_host(NA_PMAX, g, h);
        e = cudaMemcpy(base + NA_OFF_G, g.data(), sizeof(double) * (NA_PMAX + 1), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(base + NA_OFF_H, h.data(), sizeof(double) * (NA_PMAX + 1), cudaMemcpyHostToDevice);
        if (e != cudaSuccess)
            return fail(CPL_ERR_CUDA, std::string("writing the lookup tables into the no-allocation scratch failed: ") +
                                          cudaGetErrorString(e));
        g_na_ptr[dev] = base;
    }
    *ptr = g_na_ptr[dev];
    return CPL_OK;
}

// A pointer the kernels may dereference on `dev`: device memory of that
// device, or managed memory.
cpl_status na_check_ptr(const void *p, int dev, const char *what) {
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(CPL_ERR_ARG, std::string(what) + " is not a CUDA pointer: " + cudaGetErrorString(e));
    }
    if (at.type == cudaMemoryTypeManaged) return CPL_OK;
    if (at.type != cudaMemoryTypeDevice)
        return fail(CPL_ERR_ARG, std::string(what) + " must be device memory (got a host pointer)");
    if (at.device != dev)
        return fail(CPL_ERR_ARG, std::string(what) + " lies on another device than the current one");
    return CPL_OK;
}

cpl_status na_launch(int nge, bool odd, const NaArgs &a, dim3 grid, cudaStream_t st) {
    if (nge == 1) k_plain_noalloc<1, false><<<grid, NT, 0, st>>>(a);
    else if (nge == 3) k_plain_noalloc<3, false><<<grid, NT, 0, st>>>(a);
    else if (nge == 6 && odd) k_plain_noalloc<6, true><<<grid, NT, 0, st>>>(a);
    else if (nge == 6) k_plain_noalloc<6, false><<<grid, NT, 0, st>>>(a);
    else if (odd) k_plain_noalloc<0, true><<<grid, NT, 0, st>>>(a);
    else return fail(CPL_ERR_ARG, "nothing to compute");
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(CPL_ERR_CUDA, std::string("kernel launch failed: ") + cudaGetErrorString(e));
    return CPL_OK;
}

}  // namespace
}  // namespace cpl

using namespace cpl;

extern "C" cpl_status cpl_build_noalloc(const cpl_request *r, double *out, void *stream) {
    if (!r) return fail(CPL_ERR_ARG, "request is NULL");
    if (!out) return fail(CPL_ERR_ARG, "out is NULL");
    // limits of the fixed scratch
    if (r->lmax > NA_MAX_LMAX)
        return fail(CPL_ERR_RANGE, "cpl_build_noalloc supports lmax <= 4096 (its scratch array is 1 MiB)");
    if (r->n_windows > NA_MAX_WINDOWS)
        return fail(CPL_ERR_RANGE, "cpl_build_noalloc supports at most 4 windows (its scratch array is 1 MiB)");
    if (r->precision != CPL_FP64) return fail(CPL_ERR_UNSUPPORTED, "cpl_build_noalloc runs the plain FP64 path only");
    if (r->bin_edges || r->n_bins) return fail(CPL_ERR_UNSUPPORTED, "cpl_build_noalloc writes dense output only");
    // the same argument rules as cpl_build
    if (r->lmax < 2) return fail(CPL_ERR_ARG, "lmax must be >= 2");
    if (r->lmin < 0 || r->lmin > r->lmax) return fail(CPL_ERR_ARG, "lmin must lie in [0, lmax]");
    if (r->spectra == 0 || (r->spectra & ~31u)) return fail(CPL_ERR_ARG, "spectra must be a non-empty OR of CPL_* bits");
    if ((r->spectra & (kTE | kEE | kEEBB | kEB)) && r->lmin < 2)
        return fail(CPL_ERR_ARG, "polarisation spectra need lmin >= 2");
    if (r->n_windows < 1) return fail(CPL_ERR_ARG, "n_windows must be >= 1");
    if ((r->spectra & kTT) && !r->W_tt) return fail(CPL_ERR_ARG, "W_tt is NULL but CPL_TT is requested");
    if ((r->spectra & kTE) && !r->W_tp) return fail(CPL_ERR_ARG, "W_tp is NULL but CPL_TE is requested");
    if ((r->spectra & (kEE | kEEBB | kEB)) && !r->W_pp)
        return fail(CPL_ERR_ARG, "W_pp is NULL but a polarisation spectrum is requested");
    if (r->w_len < 1) return fail(CPL_ERR_ARG, "w_len must be >= 1");
    NaCaps caps;
    for (int w = 0; w < NA_MAX_WINDOWS; ++w) caps.v[w] = -1;
    for (int w = 0; w < r->n_windows; ++w) {
        int top = 2 * r->lmax;
        if (r->band_limit) {
            if (r->band_limit[w] < 0) return fail(CPL_ERR_ARG, "band_limit entries must be >= 0");
            top = std::min(top, r->band_limit[w]);
        }
        if (r->w_len < top + 1)
            return fail(CPL_ERR_ARG, "w_len too short: the l3 sum needs W up to min(2 lmax, band_limit)");
        caps.v[w] = top;
    }

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(CPL_ERR_CUDA, std::string("cudaGetDevice failed: ") + cudaGetErrorString(e));

    // window roles that share a pointer share one sweep (as in cpl_build)
    struct Role {
        const double *W;
        unsigned spectra;
    } roles[3];
    int nroles = 0;
    auto add = [&](const double *W, unsigned bits) {
        if (!(r->spectra & bits)) return;
        for (int q = 0; q < nroles; ++q)
            if (roles[q].W == W) {
                roles[q].spectra |= (r->spectra & bits);
                return;
            }
        roles[nroles++] = {W, r->spectra & bits};
    };
    add(r->W_tt, kTT);
    add(r->W_tp, kTE);
    add(r->W_pp, kEE | kEEBB | kEB);

    // the kernels dereference these: device memory of the current device
    cpl_status s;
    const char *role_name[3] = {"W_tt", "W_tp", "W_pp"};
    for (int q = 0; q < nroles; ++q) {
        const char *nm = roles[q].W == r->W_tt ? role_name[0] : roles[q].W == r->W_tp ? role_name[1] : role_name[2];
        if ((s = na_check_ptr(roles[q].W, dev, nm)) != CPL_OK) return s;
    }
    if ((s = na_check_ptr(out, dev, "out")) != CPL_OK) return s;

    unsigned char *base = nullptr;
    if ((s = na_scratch(dev, &base)) != CPL_OK) return s;

    const int a_stride = 2 * r->lmax + 2;
    const size_t end = NA_OFF_A + sizeof(double) * (size_t)a_stride * r->n_windows * nroles;
    if (end > NA_SCRATCH_BYTES) return fail(CPL_ERR_RANGE, "request does not fit the 1 MiB no-allocation scratch");

    cudaStream_t st = (cudaStream_t)stream;
    const int nib = (r->lmax - r->lmin) / 2 / TILE_I + 1;
    const int njb = r->lmax / TILE_J + 1;
    const dim3 grid(njb, 2 * nib, r->n_windows);
    for (int q = 0; q < nroles; ++q) {
        double *A = reinterpret_cast<double *>(base + NA_OFF_A) + (size_t)q * a_stride * r->n_windows;
        k_weights_noalloc<<<dim3((a_stride + 255) / 256, r->n_windows), 256, 0, st>>>(roles[q].W, r->w_len, caps, A,
                                                                                      a_stride);
        e = cudaGetLastError();
        if (e != cudaSuccess) return fail(CPL_ERR_CUDA, std::string("kernel launch failed: ") + cudaGetErrorString(e));
        NaArgs a;
        std::memset(&a, 0, sizeof(a));
        a.g = reinterpret_cast<const double *>(base + NA_OFF_G);
        a.h = reinterpret_cast<const double *>(base + NA_OFF_H);
        a.A = A;
        a.a_stride = a_stride;
        a.l3cap = caps;
        a.lmax = r->lmax;
        a.lmin = r->lmin;
        a.out = out;
        a.nspec = spec_count(r->spectra);
        const unsigned bits[5] = {kTT, kTE, kEE, kEEBB, kEB};
        for (int b = 0; b < 5; ++b) a.slot[b] = (roles[q].spectra & bits[b]) ? spec_slot(r->spectra, bits[b]) : -1;
        int mode = (roles[q].spectra & (kEE | kEEBB | kEB)) ? MODE_POL : (roles[q].spectra & kTE) ? MODE_TE : MODE_TT;
        int nge;
        bool odd;
        plain_variant(mode, a.slot, &nge, &odd);
        if ((s = na_launch(nge, odd, a, grid, st)) != CPL_OK) return s;
    }
    return CPL_OK;
}
