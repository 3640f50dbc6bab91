/*
 * coupling.h -- C ABI of the GB300 (sm_103a) mode-coupling-matrix library.
 *
 * The library assembles the pseudo-C_ell mode-coupling matrices of
 * Kiddier & Gratton, "Fast computation of temperature and polarization
 * coupling matrices" (arXiv 2602.15605):
 *
 *   M^X_{l1 l2} = (2 l2 + 1) Xi_X(l1, l2, W)                       (App. A)
 *   Xi_X = 1/(4 pi) sum_{l3} (2 l3 + 1) W_{l3} S_X(l1, l2, l3)     (Eqs. K_TT, K_EE)
 *
 * for the spectrum kernels
 *   CPL_TT    S = (l1 l2 l3; 0 0 0)^2                              (Eq. K_TT)
 *   CPL_TE    S = [L even] (l1 l2 l3; 0 0 0)(l1 l2 l3; -2 2 0)     (Eq. Sig_TE; TB is identical)
 *   CPL_EE    S = [L even] (l1 l2 l3; -2 2 0)^2                    (Eq. K_EE "+" sign; BB is identical)
 *   CPL_EEBB  S = [L odd]  (l1 l2 l3; -2 2 0)^2                    (Eq. K_EE "-" sign: the paper's
 *                                                                  odd-parity "EB" kernel, i.e. the
 *                                                                  EE <-> BB leakage block)
 *   CPL_EB    S = S_EE - S_EEBB                                    (the EB -> EB block of the MASTER
 *                                                                  polarisation system; a
 *                                                                  convention the paper leaves open)
 * with L = l1 + l2 + l3 and l3 over the triangle |l1 - l2| .. l1 + l2.
 * The 3j values are never produced by a per-(l1, l2) recursion: they come
 * from the lookup table g(p) of Eqs. gdef / g_rec through the closed form of
 * Eq. 000_sq_main and the (0,-2,2) reduction of Eq. 022_linear (Sec. 3).
 *
 * Conventions for every call:
 *   - Every call returns a cpl_status.  On any status other than CPL_OK the
 *     output buffers are left untouched and cpl_last_error() returns a
 *     one-line message (thread-local, valid until the next call on the same
 *     thread).
 *   - Device pointers are plain CUDA device addresses on the context's
 *     device.  The caller owns every input and output buffer; the context
 *     owns its lookup tables, tile lists and scratch.
 *   - Calls that take a stream are asynchronous on that stream (a
 *     cudaStream_t passed as void*; NULL is the legacy default stream).
 *     Argument errors are reported synchronously.  A device-side fault or
 *     an exceeded device wait surfaces at the next call on the context or
 *     at cpl_ctx_sync().
 *   - A context may be used from one host thread at a time.
 */
#ifndef COUPLING_H
#define COUPLING_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CPL_OK = 0,
    CPL_ERR_ARG = 1,         /* invalid argument (NULL pointer, bad size, bad combination) */
    CPL_ERR_RANGE = 2,       /* a size is outside what the library supports */
    CPL_ERR_OOM = 3,         /* a device or host allocation failed */
    CPL_ERR_CUDA = 4,        /* a CUDA runtime call or kernel launch failed */
    CPL_ERR_TIMEOUT = 5,     /* a bounded device-side wait ran out */
    CPL_ERR_UNSUPPORTED = 6  /* the request is valid but this library build or device cannot run it */
} cpl_status;

/* Spectrum bits; OR them into cpl_request.spectra.  Outputs are stored in
 * increasing bit order of the requested set. */
enum {
    CPL_TT = 1,
    CPL_TE = 2,    /* = TB */
    CPL_EE = 4,    /* = BB */
    CPL_EEBB = 8,  /* odd-parity kernel */
    CPL_EB = 16    /* EE - EEBB */
};

typedef enum {
    CPL_FP64 = 0,        /* plain FP64 arithmetic throughout (target <= 1e-11 relative) */
    CPL_MIXED_BF16 = 1,  /* l3 contraction on tcgen05 tensor cores with BF16 fixed-point
                            limbs and exact FP32 partial sums; FP64 tables, scales and
                            final values (bound 1e-9 relative, see mixed_slices) */
    CPL_DF32 = 2         /* the plain path's contractions in double-float (pairs of FP32,
                            ~48-bit significands) on the FP32 pipe; weights scaled per tile,
                            FP64 epilogue; lmax <= CPL_DF32_LMAX (target <= 1e-11 relative
                            like CPL_FP64; measured <= 4e-13) */
} cpl_precision;
#define CPL_DF32_LMAX 10000

typedef struct cpl_ctx cpl_ctx;

/*
 * One coupling-matrix request.
 *
 *   lmax, lmin   rows and columns run over l = lmin .. lmax.  lmax >= 2 and
 *                0 <= lmin <= lmax; lmin >= 2 when any polarisation spectrum
 *                is requested (the (-2 2 0) symbol needs l1, l2 >= 2).
 *   n_windows    number of windows W stacked in each W_* array (>= 1).
 *   W_tt/tp/pp   window power spectra, [n_windows][w_len] row-major FP64:
 *                W_tt feeds CPL_TT, W_tp feeds CPL_TE, W_pp feeds CPL_EE,
 *                CPL_EEBB and CPL_EB (App. A: the spectrum of the mask pair
 *                applied to the two maps).  Device pointers for cpl_build /
 *                cpl_build_batch, host pointers for cpl_build_host.  A
 *                window that no requested spectrum uses may be NULL.  Passing
 *                the same pointer for several roles lets the library share
 *                one l3 sweep between them.
 *   w_len        entries per window.  The l3 sum needs W_L for L <= 2 lmax
 *                (Sec. 4); entries beyond w_len - 1 are taken as zero, which
 *                is exact only for band-limited windows, so w_len < 2 lmax + 1
 *                requires band_limit.
 *   band_limit   host array [n_windows] of L_w (last l3 kept), or NULL for
 *                none.  Terms with l3 > L_w are skipped, which is exact when
 *                W is zero above L_w (Sec. 4.3).
 *   spectra      OR of CPL_* bits (non-empty).
 *   precision    cpl_precision.
 *   mixed_slices number of BF16 limbs per operand for CPL_MIXED_BF16 (4..6);
 *                0 selects the default, 6 (measured error <= 2.2e-10 against
 *                the stated 1e-9 bound; 5 limbs ~6e-10, 4 limbs ~1e-7).
 *   bin_edges    host array [n_bins + 1] of increasing multipoles inside
 *                [lmin, lmax + 1], or NULL for dense output.  Bin b holds
 *                l in [bin_edges[b], bin_edges[b+1]); the binned matrix is
 *                M_bb' = (1/|b|) sum_{l1 in b} sum_{l2 in b'} M_{l1 l2}.
 *   n_bins       number of bins (0 when bin_edges is NULL).
 *   bin_weight   0: flat band powers as above.  1: band powers of
 *                D_l = l(l+1) C_l / 2pi, i.e. P_bl = l(l+1) / (2pi |b|) and
 *                Q_lb = 2pi / (l(l+1)):  M_bb' = (1/|b|) sum_{l1 in b}
 *                sum_{l2 in b'} [l1(l1+1) / (l2(l2+1))] M_{l1 l2}; needs
 *                bin_edges[0] >= 1.  Ignored (must be 0) without bin_edges.
 */
typedef struct {
    int lmax;
    int lmin;
    int n_windows;
    const double *W_tt;
    const double *W_tp;
    const double *W_pp;
    int w_len;
    const int *band_limit;
    unsigned spectra;
    int precision;
    int mixed_slices;
    const int *bin_edges;
    int n_bins;
    int bin_weight;
} cpl_request;

/* Library version string (static storage). */
const char *cpl_version(void);

/* Message of the last failed call on this thread ("" if none). */
const char *cpl_last_error(void);

/*
 * Create a context on CUDA device `device` (which must be an sm_103 GPU for
 * any compute call).  *ctx receives an opaque handle the caller releases
 * with cpl_ctx_destroy.  Allocates nothing on the device until first use.
 */
cpl_status cpl_ctx_create(cpl_ctx **ctx, int device);

/* Synchronise the context's device work and release everything it owns.
 * NULL is accepted. */
cpl_status cpl_ctx_destroy(cpl_ctx *ctx);

/* Wait for all work the context queued and report any device-side error
 * (CPL_ERR_TIMEOUT for an exceeded bounded wait, CPL_ERR_CUDA otherwise,
 * including an internal inconsistency a kernel detected). */
cpl_status cpl_ctx_sync(cpl_ctx *ctx);

/*
 * Number of doubles the output of `r` occupies:
 *   dense   n_windows * nspec * n * n,   n = lmax - lmin + 1
 *   binned  n_windows * nspec * n_bins * n_bins
 * with nspec the number of bits set in r->spectra.  Validates r.
 */
cpl_status cpl_output_size(const cpl_request *r, size_t *n_doubles);

/*
 * Build the coupling matrices of `r` into `out` (device, caller-owned,
 * cpl_output_size doubles), asynchronously on `stream`.
 *
 * Dense layout: out[w][spec][l1 - lmin][l2 - lmin], spec in increasing bit
 * order of r->spectra.  Binned layout: out[w][spec][b][b'].  Elements that
 * the parity selection or the band limit make exactly zero are written as
 * exactly 0.0.  The W_* pointers are device pointers.
 *
 * Memory: CPL_FP64 builds read precomputed operand blocks of the separable
 * l3 contractions (Sec. 3.1 tables times the integer polarisation factors):
 * a window-independent part cached in the context (about 48 lmax^2 bytes,
 * kept for the largest lmax seen: 0.43 GB at lmax 3000, 4.7 GB at 10000)
 * and a per-call part (about 28 lmax^2 bytes per window with all spectra,
 * less with a band limit).  When both together would exceed half of the
 * device's free memory, or the environment variable CPL_PLAIN_TABLES is
 * "0", the kernels build the operands themselves instead (same results,
 * bit for bit; about 10% slower).
 */
cpl_status cpl_build(cpl_ctx *ctx, const cpl_request *r, double *out, void *stream);

/*
 * Host-only dry run of a plain-path build (CPL_FP64 or CPL_DF32) of `r`: no
 * context, no device work; the W_* pointers are not read.  Validation as
 * cpl_output_size; CPL_ERR_UNSUPPORTED for CPL_MIXED_BF16.
 *   n_tiles        32 x 32 blocks of (i, j) = ((d - pi)/2, (s - pi)/2),
 *                  d = l2 - l1, s = l1 + l2, pi = d mod 2, covering the
 *                  pairs lmin <= l1 <= l2 <= lmax
 *   n_items        (window, tile) work items over all contraction launches;
 *                  a tile whose smallest l3 exceeds a window's band limit is
 *                  dropped for that window
 *   n_launches     contraction launches (one per kernel variant; window roles
 *                  that share a pointer share one sweep)
 *   terms_even     l3 terms of the sums of App. A over the pairs l1 <= l2 with
 *   terms_odd      l1 + l2 + l3 even / odd, within each window's band, summed
 *                  over windows
 *   flop           algorithmic FLOP of the contractions: 2 per term and
 *                  separable contraction (1, 3 or 6 per even term by the
 *                  spectra a sweep serves, 3 per odd term) -- the count behind
 *                  the plain path's roofline
 *   table_bytes_b  CPL_FP64 operand blocks shared by all windows (a context
 *                  keeps them for the largest lmax it has built); 0 for DF32
 *   table_bytes_a  CPL_FP64 per-call operand blocks; 0 for CPL_DF32
 */
typedef struct {
    long long n_tiles, n_items;
    int n_launches;
    double terms_even, terms_odd, flop;
    unsigned long long table_bytes_b, table_bytes_a;
} cpl_plan_info;
cpl_status cpl_plan_info_fp64(const cpl_request *r, cpl_plan_info *info);

/*
 * The same request with HOST buffers: W_* are host pointers and `out_host`
 * is a host buffer of cpl_output_size doubles.  The library copies the
 * windows to the device, builds, copies the result back and returns when
 * `out_host` is filled (synchronous).  Staging memory is owned by the
 * context and reused across calls.  When `out_host` is page-locked the
 * device-to-host copies overlap the build: for CPL_FP64 and CPL_DF32 each
 * kernel variant's output blocks travel while the later variants run; for a
 * dense CPL_MIXED_BF16 request whose windows form several role groups (for
 * instance separate W^TT, W^TP, W^PP) each group is built as a request of
 * its own, most contractions first, and its planes travel while the later
 * groups compute.  The result is the same as cpl_build's (bit for bit in the
 * dense cases).
 */
cpl_status cpl_build_host(cpl_ctx *ctx, const cpl_request *r, double *out_host);

/*
 * A batch of independent requests (ragged lmax, band limits, window
 * counts, bins): jobs[q] writes outs[q] (device pointers, each of
 * cpl_output_size(jobs + q) doubles).  All jobs must use the same precision
 * (and, for CPL_MIXED_BF16, the same mixed_slices).  The work items of all
 * jobs are merged:
 *   CPL_MIXED_BF16  one persistent tensor-core GEMM launch takes the items of
 *                   every job by an atomic ticket (jobs that do not fit the
 *                   scratch budget together run as several such chunks); the
 *                   batch is planned once per signature (every field of every
 *                   request, pointers included, and the contents of the
 *                   band-limit and bin-edge arrays), its launch sequence is
 *                   captured into a CUDA graph on the first call and replayed
 *                   on later calls with the same signature;
 *   CPL_FP64        one launch per kernel variant over the items of every
 *                   job, heaviest first.
 * Results equal those of cpl_build on each job (bit for bit for dense
 * output; binned sums are accumulated in no fixed order).
 */
cpl_status cpl_build_batch(cpl_ctx *ctx, const cpl_request *jobs, int n_jobs,
                           double *const *outs, void *stream);

/*
 * cpl_build_noalloc -- the plain FP64 build of `r` without any device
 * allocation.  The paper has no counterpart: this entry point exists for
 * callers that cannot call cudaMalloc (an application whose own allocator
 * owns the device memory budget, a pipeline that must not take the device
 * synchronisation an allocation can cause, or code where allocation calls
 * are not allowed).
 *
 * It computes the same matrices as cpl_build with CPL_FP64 and dense output
 * (equal to rounding: it forms the pair coefficients directly rather than
 * from the context's per-l factor table) into `out` (device, caller-owned,
 * cpl_output_size doubles) on the CURRENT CUDA device, asynchronously on
 * `stream`.  W_* and `out` must be device memory of the current device (or
 * managed memory): anything else -- a host pointer, another GPU's memory --
 * fails with CPL_ERR_ARG before any work is queued.  It needs no context:
 * its scratch (the g / h lookup tables and the window weights) is one fixed
 * 1 MiB device array inside the library, which every GPU that loads the
 * library holds until the process exits.  Limits of that array:
 * lmax <= 4096 and n_windows <= 4; larger requests fail with CPL_ERR_RANGE,
 * binned output and CPL_MIXED_BF16 with CPL_ERR_UNSUPPORTED.
 *   - The first call on a device sets the array up: it looks up the array's
 *     device address (cudaGetSymbolAddress) and writes the lookup tables
 *     into it with a synchronous host-to-device copy.  Make that first call
 *     before any stream capture.  Later calls only launch kernels (the
 *     per-window l3 caps travel in the kernel arguments) and read no host
 *     memory.
 *   - All calls share the array and it keeps the last call's contents: the
 *     tables never change after the set-up, and each call rewrites the
 *     weights it reads.  Calls whose GPU work overlaps -- different streams
 *     without ordering between them, or different host threads -- race on
 *     the weights and must be serialised by the caller.
 */
cpl_status cpl_build_noalloc(const cpl_request *r, double *out, void *stream);

/*
 * Per-kernel accounting (diagnostics).  Every context counts the kernel
 * launches it issues, per kernel family.  With profiling enabled
 * (cpl_ctx_profile(ctx, 1)) it also brackets each launch with CUDA events
 * on the launching stream and records the algorithmic work of the launch:
 *   flop   floating-point operations the method needs (an FMA counts 2;
 *          for the mixed path, 2 per window-term per contraction, not the
 *          limb products actually issued),
 *   bytes  DRAM bytes the launch must move at minimum (inputs read once,
 *          outputs written once).
 * cpl_ctx_stats waits for the recorded events, writes up to `max` entries
 * to `out` (host), sets *n to the number of kernel families and, when
 * `reset` is non-zero, clears the counters.
 */
typedef struct {
    char name[40];        /* kernel family */
    long long launches;   /* launches since the last reset */
    double ms;            /* summed event-timed duration of those launches (profiling only) */
    double flop;          /* algorithmic FLOP of the timed launches */
    double bytes;         /* algorithmic DRAM bytes of the timed launches */
    double issued_flop;   /* floating-point operations the timed launches issue: the
                             tensor-core limb products for the mixed path, equal to
                             flop for the FP64 kernels */
} cpl_kernel_stat;

cpl_status cpl_ctx_profile(cpl_ctx *ctx, int enable);
cpl_status cpl_ctx_stats(cpl_ctx *ctx, cpl_kernel_stat *out, int max, int *n, int reset);

/*
 * Tile-shape autotuner of the mixed-precision path (the persistent batched
 * scheduler's tile choice).  The tuned parameters are the row shape of a
 * tensor-core tile (1, 2 or 4 row sources x 128, 64 or 32 values of i) and
 * the order in which the persistent kernel takes a job's work items
 * (grouped by contraction or by tile).  They change the speed only: every
 * candidate computes bit-identical matrices.
 *
 *   mode CPL_TUNE_OFF      built-in choice (row sources = window count
 *                          rounded up to 1, 2 or 4; order by contraction);
 *   mode CPL_TUNE_MEASURE  on the first request of a shape (l_max, l_min,
 *                          window count, window-role grouping, spectra,
 *                          l3 caps, binning, mixed_slices) every candidate
 *                          runs the request's full launch sequence on its
 *                          own buffers, timed with CUDA events, and the
 *                          fastest is kept for that shape.  The first call
 *                          of a shape therefore blocks until the candidates
 *                          have run (about 2 x 6 builds).
 *
 * With a non-NULL `cache_path` the choices are also read from and appended
 * to that file (one JSON object per line: {"key": [...], "src": n,
 * "order": n, "ms": t}); unreadable lines are ignored.  Returns
 * CPL_ERR_ARG for an unknown mode.
 */
typedef enum { CPL_TUNE_OFF = 0, CPL_TUNE_MEASURE = 1 } cpl_tune_mode;
cpl_status cpl_ctx_tune(cpl_ctx *ctx, int mode, const char *cache_path);

/*
 * Test hook (host-side fault injection; the paper has no counterpart): the
 * n-th device allocation that the context makes from now on fails with
 * CPL_ERR_OOM, exactly as if cudaMalloc had failed (n = 0 disables).  The
 * failing call returns the status with the output untouched, and the
 * context stays usable: caches whose buffers the failure freed are rebuilt
 * by the next call.  CPL_ERR_ARG for n < 0.
 */
cpl_status cpl_ctx_inject_alloc_failure(cpl_ctx *ctx, int n);

/*
 * cpl_ctx_validate -- optional input validation (off by default).  When
 * enabled, cpl_build, cpl_build_batch and cpl_build_host (and the builds of
 * cpl_cov_gaussian) first check every window entry the request reads
 * (n_windows x w_len values of each distinct W pointer) on the device and
 * return CPL_ERR_ARG, naming the window and l, if one is NaN or Inf; nothing
 * is written.  The check waits for its result, so validated calls are
 * synchronous on their stream.
 */
cpl_status cpl_ctx_validate(cpl_ctx *ctx, int enable);

/*
 * cpl_threej_m11 -- the Wigner symbols (j1 j2 j3; 0 -1 1) for every j1 of
 * each given (j2, j3): the (0,-1,1) configuration that appears in the
 * lensing quadratic-estimator and aberration weights (Sec. 1; App. B,
 * "Obtaining J(-1,1) symbols").  They come from the g table like the
 * coupling matrices: for even J = j1 + j2 + j3 from the (0 0 0) symbol of
 * the same triple (Eq. joneevensimp), for odd J from the (0 0 0) symbol of
 * (j1, j2, j3 + 1) (Eq. joneodd); no recursion.
 *
 *   j2, j3      host arrays [n] with 1 <= j2, j3 and j2 + j3 <= CPL_THREEJ_JMAX
 *               (m = -1, 1 needs j >= 1);
 *   out         device array [n][out_stride] FP64 (caller-owned): row q holds
 *               j1 = |j2 - j3| .. j2 + j3 at out[q * out_stride + j1 - |j2 - j3|]
 *               and zeros in the rest of the row;
 *   out_stride  >= 2 min(j2, j3) + 1 for every q.
 * Asynchronous on `stream`.
 * CPL_ERR_ARG / CPL_ERR_RANGE for invalid arguments (output untouched).
 */
#define CPL_THREEJ_JMAX 200000
cpl_status cpl_threej_m11(cpl_ctx *ctx, const int *j2, const int *j3, int n, double *out, long long out_stride,
                          void *stream);

/*
 * cpl_decouple -- mode decoupling: the underlying spectra C from measured
 * pseudo-spectra by solving the linear systems of Eq. pseudo_cl (Sec. 2;
 * kernels of App. A) for every window and right-hand side:
 *
 *   TT:     K^TT C^TT = pcl^TT            TE: K^TE C^TE = pcl^TE (TB alike)
 *   EE/BB:  K^EE C^EE + K^EEBB C^BB = pcl^EE,  K^EEBB C^EE + K^EE C^BB = pcl^BB
 *   EB:     K^EB C^EB = pcl^EB,  K^EB = K^EE - K^EEBB (the CPL_EB block)
 *
 * K[l1][l2] is a cpl_build output block (row l1 = pseudo-spectrum
 * multipole).  For binned output the same equations hold for the band powers
 * pcl_b = (1/|b|) sum_{l in b} pcl_l, exactly when C is constant inside
 * each bin.
 *
 *   n          block size: lmax - lmin + 1 (dense) or n_bins (binned),
 *              1 <= n <= CPL_DECOUPLE_NMAX.
 *   n_windows  windows stacked in M (>= 1).
 *   spectra    the spectrum set M was built with.  CPL_EE and CPL_EEBB must
 *              come together (the EE/BB system couples through EE->BB).
 *   M          device, [n_windows][nspec][n][n] FP64, the cpl_build layout
 *              (spectra in increasing bit order); read only.
 *   pcl        device, [n_windows][n_rhs][n_fields][n] FP64: the fields TT,
 *              TE, EE, BB, EB of the requested set in that order (EE and BB
 *              both present with CPL_EE); read only.
 *   n_rhs      pseudo-spectra per window (e.g. simulations),
 *              1 <= n_rhs <= CPL_DECOUPLE_RHS_MAX.
 *   out        device, layout of pcl (caller-owned, must not overlap M or
 *              pcl): the decoupled spectra.
 *   info       device int [n_windows][n_systems] or NULL; systems per window
 *              in the order TT, TE, EE+EEBB, EE-EEBB, EB (present ones
 *              only).  0 on success; k + 1 when the k-th pivot of that system
 *              was zero or not finite, in which case its outputs are NaN.
 *   stream     cudaStream_t or NULL.
 *
 * Each system is solved by Gaussian elimination with partial pivoting; the
 * EE/BB system is split exactly into (K^EE +- K^EEBB) systems.  With few
 * right-hand sides (n_rhs <= 2n/9, n <= 512) the factorisation runs in FP32
 * and iterative refinement with residuals of FP64 accuracy brings every
 * solution to max|pcl - K C| <= max|C| |K|_inf 2^-53 sqrt(n) (the stopping
 * rule of LAPACK's dsgesv).  From 8 right-hand sides (and |K|_inf >= 2^-40)
 * the first residual runs partly as exact triple-FP32 products (where a
 * thread of the solver holds more than 5 right-hand sides) and each
 * later one is the previous residual minus K times the update the solution
 * received, in FP32 pairs; with fewer every residual is an FP64 product.
 * A system whose FP32 factors fail (a zero pivot, entries
 * outside FP32's range, no convergence in 30 steps) and every system with
 * more right-hand sides is solved in FP64.  Results are deterministic.
 * Asynchronous on `stream`; CPL_ERR_ARG / CPL_ERR_RANGE for invalid
 * arguments (output untouched).
 */
#define CPL_DECOUPLE_NMAX 1024
#define CPL_DECOUPLE_RHS_MAX 4096
cpl_status cpl_decouple(cpl_ctx *ctx, int n, int n_windows, unsigned spectra, const double *M, const double *pcl,
                        int n_rhs, double *out, int *info, void *stream);

/*
 * cpl_cov_gaussian -- approximate Gaussian covariance of pseudo-spectra from
 * coupling-type kernels (Sec. 2 and Sec. 4.3, band-limited covariance
 * matrices): when the spectra vary little across the masks' band limit the
 * covariance reduces to kernels of the squared masks,
 *
 *   Cov_{l1 l2} = sum_t Xi_{X_t}(l1, l2; W~_t) (A^t_l1 B^t_l2 + A^t_l2 B^t_l1) / 2,
 *   Xi_X(l1, l2; W~) = (1/4pi) sum_l3 (2 l3 + 1) W~_l3 S_X(l1, l2, l3)
 *
 * (S_X of App. A; Xi is the coupling matrix without its (2 l2 + 1)), with W~
 * the power spectrum of the product of the squared masks and the l3 sum cut
 * at the band limit.  One term per Wick pairing of the four fields, e.g. the
 * TT auto-spectrum: one term X = CPL_TT, A = C^TT, B = 2 C^TT (full sky:
 * 2 C_l^2 / (2l + 1) on the diagonal).
 *
 *   lmax, lmin   as in cpl_request (lmin >= 2 with a polarisation kernel).
 *   terms[t]     spectrum: one CPL_* bit (the kernel X_t); W: device [w_len]
 *                FP64; band_limit: last l3 kept, or -1 for none (then w_len
 *                must reach 2 lmax + 1); A, B: device [lmax + 1] FP64
 *                indexed by l.  Terms with the same W pointer and band limit
 *                share one kernel build.
 *   n_terms      >= 1.
 *   w_len        entries of each W.
 *   precision    cpl_precision of the kernel builds.
 *   bin_edges    host [n_bins + 1] as in cpl_request, or NULL: binned output
 *                Cov_bb' = (1/|b||b'|) sum_{l1 in b} sum_{l2 in b'} Cov_{l1 l2}.
 *   out          device, caller-owned: [n][n] (n = lmax - lmin + 1) or
 *                [n_bins][n_bins] FP64, exactly symmetric.
 *   stream       cudaStream_t or NULL.
 * Asynchronous on `stream`; deterministic.  The sum is formed in context
 * scratch and `out` is written last, so on any error status `out` is
 * untouched.
 */
typedef struct {
    unsigned spectrum;
    const double *W;
    int band_limit;
    const double *A;
    const double *B;
} cpl_cov_term;
cpl_status cpl_cov_gaussian(cpl_ctx *ctx, int lmax, int lmin, const cpl_cov_term *terms, int n_terms, int w_len,
                            int precision, const int *bin_edges, int n_bins, double *out, void *stream);

/*
 * FP64 pipe throughput probe: the measured denominator of the plain path's
 * roofline (the paper's GPU comparison is an FP64 measurement, Sec. 4.2).
 * Launches n_blocks blocks of 256 threads on `stream`; every thread runs
 * 1024 x iters fused multiply-adds: a 4 x 4 tile of accumulators
 * acc[r][c] = fma(a[r], b[c], acc[r][c]) whose operands it loads from a
 * 32-deep shared-memory panel, as the contraction kernels do (no global
 * memory traffic).  *flop (host) receives the floating-point operations the
 * launch performs (an FMA counts 2): 2 * 1024 * iters * 256 * n_blocks.  The caller times the launch with events
 * on `stream`.  `sink` is a device double the kernel could write (it never
 * does; the condition keeps the sums from being optimised away).
 * Errors: CPL_ERR_ARG for n_blocks < 1, iters < 1 or a NULL pointer,
 * CPL_ERR_RANGE for n_blocks > 2^20 or iters > 2^20, CPL_ERR_CUDA if the
 * launch fails.
 */
cpl_status cpl_probe_fp64(int n_blocks, int iters, double *sink, double *flop, void *stream);

/*
 * Lookup table of Eqs. gdef / g_rec, as the library builds it: out[p] =
 * g(p) = (2p)! / (2^{2p} (p!)^2) for p = 0 .. pmax, each value the
 * double-double recurrence g(p) = (p - 1/2)/p g(p-1), g(0) = 1, rounded once
 * to FP64.  Host-only (no device work); out_host holds pmax + 1 doubles.
 */
cpl_status cpl_g_table(int pmax, double *out_host);

/*
 * The second lookup table, as the library builds it: out[p] = h(p) =
 * 1 / ((2p + 1) g(p)) for p = 0 .. pmax.  It fuses the (J + 1)^{-1} and 1/g
 * factors of Eq. 000_sq_main (with J = 2p, the J-dependent part
 * 1 / ((J + 1) g(J/2)) is one load).  Formed from the same double-double
 * recurrence as g, then a double-double reciprocal, rounded once to FP64.
 * Host-only (no device work); out_host holds pmax + 1 doubles.  Errors:
 * CPL_ERR_ARG for pmax < 0 or a NULL out_host, CPL_ERR_RANGE for
 * pmax > 2^24.
 */
cpl_status cpl_h_table(int pmax, double *out_host);

#ifdef __cplusplus
}
#endif

#endif /* COUPLING_H */
