// cov.cu -- approximate Gaussian covariance of pseudo-spectra from
// coupling-type kernels (Sec. 2; Sec. 4.3, band-limited covariance):
//
//   Cov_{l1 l2} = sum_t Xi_{X_t}(l1, l2; W~_t) (A^t_l1 B^t_l2 + A^t_l2 B^t_l1) / 2,
//   Xi_X(l1, l2; W~) = M_X[l1][l2] / (2 l2 + 1)    (App. A kernels on W~)
//
// The kernels come from the coupling build; here two memory-bound passes:
//
// k_cov_combine: 32 x 32 tiles of the upper triangle (tile row <= tile
//   column).  Each element with l1 <= l2 reads M_t[l1][l2] of every term of
//   the group (coalesced along l2), forms the sum, adds it to (or writes it
//   into) Cov[l1][l2] and, through a shared-memory transpose, Cov[l2][l1]:
//   the result is symmetric bit for bit and the lower triangle of M is never
//   read.
// k_cov_bin: Cov_bb' = (1/|b||b'|) sum over the bin rectangle, one warp per
//   bin pair b <= b' in a fixed summation order (lane-strided columns, rows
//   in order, then a fixed shuffle tree), mirrored to (b', b).
#include <algorithm>
#include <vector>

#include "ctx.h"
#include "internal.h"

namespace cpl {
namespace {

constexpr int CT = 32;   // tile edge

__global__ void __launch_bounds__(CT * 8) k_cov_combine(CovCombineArgs a) {
    __shared__ double tile[CT][CT + 1];
    // tile pair (I, J), I <= J, from the linear block index over the upper triangle
    const int nt = (a.n + CT - 1) / CT;
    int q = blockIdx.x, I = 0;
    while (q >= nt - I) {
        q -= nt - I;
        ++I;
    }
    const int J = I + q;
    const int tx = threadIdx.x & (CT - 1), ty = threadIdx.x / CT;   // 32 x 8 threads, 4 rows each
    const int j = J * CT + tx;
    double v[CT / 8];
#pragma unroll
    for (int rr = 0; rr < CT / 8; ++rr) v[rr] = 0.0;
    if (j < a.n) {
        const int l2 = a.lmin + j;
        const double inv = 0.5 / (2.0 * l2 + 1.0);
        // Xi s = M (A_l1 b'_l2 + a'_l2 B_l1), a' = A / (2 (2 l2 + 1)), b' likewise:
        // three FP64 operations per element and term (GB300's FP64 rate is 1/64 of FP32)
        for (int t = 0; t < a.n_terms; ++t) {
            const double a2 = a.A[t][l2] * inv, b2 = a.B[t][l2] * inv;
            const double *Mt = a.M + (size_t)a.slot[t] * a.n * a.n;
#pragma unroll
            for (int rr = 0; rr < CT / 8; ++rr) {
                const int i = I * CT + ty + 8 * rr;
                if (i < a.n && i <= j) {
                    const int l1 = a.lmin + i;
                    v[rr] = fma(Mt[(size_t)i * a.n + j], fma(a2, a.B[t][l1], a.A[t][l1] * b2), v[rr]);
                }
            }
        }
    }
#pragma unroll
    for (int rr = 0; rr < CT / 8; ++rr) {
        const int r = ty + 8 * rr, i = I * CT + r;
        if (i < a.n && j < a.n && i <= j) {
            double *o = a.out + (size_t)i * a.n + j;
            if (a.accumulate) v[rr] += *o;
            *o = v[rr];
        }
        tile[r][tx] = v[rr];
    }
    if (I == J) {
        __syncthreads();
        // diagonal tile: mirror the strict upper part inside the tile
        for (int r = ty; r < CT; r += 8) {
            const int i = I * CT + r, jj = I * CT + tx;
            if (r > tx && i < a.n) a.out[(size_t)i * a.n + jj] = tile[tx][r];   // (i, jj) mirrors (jj, i)
        }
        return;
    }
    __syncthreads();
    // off-diagonal tile: Cov[J-tile row][I-tile column] = transpose
    for (int r = ty; r < CT; r += 8) {
        const int i = J * CT + r, jj = I * CT + tx;
        if (i < a.n && jj < a.n) a.out[(size_t)i * a.n + jj] = tile[tx][r];
    }
}

__global__ void __launch_bounds__(256) k_cov_bin(CovBinArgs a) {
    const int lane = threadIdx.x & 31;
    const long long w = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
    const long long npairs = (long long)a.nb * (a.nb + 1) / 2;
    if (w >= npairs) return;
    int b = 0;
    long long q = w;
    while (q >= a.nb - b) {
        q -= a.nb - b;
        ++b;
    }
    const int c = b + (int)q;
    const int r0 = a.edges[b] - a.lmin, r1 = a.edges[b + 1] - a.lmin;
    const int c0 = a.edges[c] - a.lmin, c1 = a.edges[c + 1] - a.lmin;
    double s = 0.0;
    for (int i = r0; i < r1; ++i)
        for (int j = c0 + lane; j < c1; j += 32) s += a.cov[(size_t)i * a.n + j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
        const double v = s / ((double)(r1 - r0) * (double)(c1 - c0));
        a.out[(size_t)b * a.nb + c] = v;
        a.out[(size_t)c * a.nb + b] = v;
    }
}

}  // namespace

cudaError_t launch_cov_combine(const CovCombineArgs &a, cudaStream_t st) {
    const long long nt = (a.n + CT - 1) / CT;
    const long long blocks = nt * (nt + 1) / 2;
    k_cov_combine<<<(unsigned)blocks, CT * 8, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_cov_bin(const CovBinArgs &a, cudaStream_t st) {
    const long long npairs = (long long)a.nb * (a.nb + 1) / 2;
    k_cov_bin<<<(unsigned)((npairs + 7) / 8), 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace cpl

// ---------------------------------------------------------------- entry point
using namespace cpl;

extern "C" {

cpl_status cpl_cov_gaussian(cpl_ctx *c, int lmax, int lmin, const cpl_cov_term *terms, int n_terms, int w_len,
                            int precision, const int *bin_edges, int n_bins, double *out, void *stream) {
    if (!c) return fail(CPL_ERR_ARG, "ctx is NULL");
    if (!terms || n_terms < 1 || !out) return fail(CPL_ERR_ARG, "terms (n_terms >= 1) and out must be given");
    if (lmax < 2 || lmin < 0 || lmin > lmax) return fail(CPL_ERR_RANGE, "need lmax >= 2 and 0 <= lmin <= lmax");
    // group the terms by (window, band limit): one kernel build per group
    struct Group {
        const double *W;
        int band;
        unsigned spectra;
        std::vector<int> idx;
    };
    std::vector<Group> groups;
    for (int t = 0; t < n_terms; ++t) {
        const cpl_cov_term &T = terms[t];
        const unsigned b = T.spectrum;
        if (b == 0 || (b & (b - 1)) || b > kEB) return fail(CPL_ERR_ARG, "each term needs exactly one CPL_* spectrum bit");
        if (!T.W || !T.A || !T.B) return fail(CPL_ERR_ARG, "each term needs W, A and B");
        if (T.band_limit < -1) return fail(CPL_ERR_ARG, "band_limit must be >= -1");
        Group *g = nullptr;
        for (auto &x : groups)
            if (x.W == T.W && x.band == T.band_limit) g = &x;
        if (!g) {
            groups.push_back(Group{T.W, T.band_limit, 0u, {}});
            g = &groups.back();
        }
        g->spectra |= b;
        g->idx.push_back(t);
    }
    // validate every build (and the binning) before any device work
    const int n = lmax - lmin + 1;
    std::vector<cpl_request> reqs(groups.size());
    for (size_t q = 0; q < groups.size(); ++q) {
        cpl_request &r = reqs[q];
        r = cpl_request{};
        r.lmax = lmax;
        r.lmin = lmin;
        r.n_windows = 1;
        r.W_tt = r.W_tp = r.W_pp = groups[q].W;
        r.w_len = w_len;
        r.band_limit = groups[q].band >= 0 ? &groups[q].band : nullptr;
        r.spectra = groups[q].spectra;
        r.precision = precision;
        size_t nd = 0;
        cpl_status s = cpl_output_size(&r, &nd);
        if (s != CPL_OK) return s;
    }
    if (bin_edges || n_bins) {
        cpl_request rb = reqs[0];
        rb.bin_edges = bin_edges;
        rb.n_bins = n_bins;
        size_t nd = 0;
        cpl_status s = cpl_output_size(&rb, &nd);
        if (s != CPL_OK) return s;
    }
    cpl_status s;
    if ((s = select_device(c)) != CPL_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    int max_spec = 1;
    for (auto &g : groups) max_spec = std::max(max_spec, spec_count(g.spectra));
    const size_t nn = (size_t)n * n;
    CPL_CUDA_TRY(cudaStreamWaitEvent(st, c->done, 0));
    if ((s = c->cov_M.ensure(sizeof(double) * nn * max_spec, "covariance kernels")) != CPL_OK) return s;
    // the sum is formed in context scratch and written to `out` only at the
    // end (binning or one copy), so a failure part-way leaves `out` untouched
    const bool binned = bin_edges != nullptr;
    if ((s = c->cov_dense.ensure(sizeof(double) * nn, "dense covariance")) != CPL_OK) return s;
    if (binned) {
        if ((s = c->cov_edges.ensure(sizeof(int) * (n_bins + 1), "covariance bin edges")) != CPL_OK) return s;
        CPL_CUDA_TRY(cudaMemcpyAsync(c->cov_edges.ptr, bin_edges, sizeof(int) * (n_bins + 1), cudaMemcpyHostToDevice, st));
    }
    double *dense = c->cov_dense.as<double>();
    bool first = true;
    for (size_t q = 0; q < groups.size(); ++q) {
        if ((s = cpl_build(c, &reqs[q], c->cov_M.as<double>(), stream)) != CPL_OK) return s;
        const auto &idx = groups[q].idx;
        for (size_t t0 = 0; t0 < idx.size(); t0 += COV_TERMS_PER_LAUNCH) {
            CovCombineArgs a{};
            a.M = c->cov_M.as<double>();
            a.n = n;
            a.lmin = lmin;
            a.n_terms = (int)std::min<size_t>(COV_TERMS_PER_LAUNCH, idx.size() - t0);
            for (int k = 0; k < a.n_terms; ++k) {
                const cpl_cov_term &T = terms[idx[t0 + k]];
                a.slot[k] = spec_slot(groups[q].spectra, T.spectrum);
                a.A[k] = T.A;
                a.B[k] = T.B;
            }
            a.out = dense;
            a.accumulate = first ? 0 : 1;
            first = false;
            LaunchScope ls(c, "cov_combine", st);
            CPL_CUDA_TRY(launch_cov_combine(a, st));
            ls.done(3.0 * 2.0 * a.n_terms * 0.5 * (double)nn,
                    8.0 * (double)nn * (0.5 * a.n_terms + (a.accumulate ? 2.0 : 1.0)));
        }
    }
    if (binned) {
        CovBinArgs b{};
        b.cov = dense;
        b.n = n;
        b.lmin = lmin;
        b.nb = n_bins;
        b.edges = c->cov_edges.as<int>();
        b.out = out;
        LaunchScope ls(c, "cov_bin", st);
        CPL_CUDA_TRY(launch_cov_bin(b, st));
        ls.done((double)nn, 8.0 * (double)nn);
    } else {
        CPL_CUDA_TRY(cudaMemcpyAsync(out, dense, sizeof(double) * nn, cudaMemcpyDeviceToDevice, st));
    }
    CPL_CUDA_TRY(cudaEventRecord(c->done, st));
    return CPL_OK;
}

}  // extern "C"
