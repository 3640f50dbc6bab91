// ctx.h -- the context object behind cpl_ctx (internal).
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <memory>
#include <string>
#include <utility>
#include <vector>

#include "internal.h"

namespace cpl {

// Allocation-failure hook of the calling thread's current context
// (cpl_ctx_inject_alloc_failure): when it counts down to zero, the
// allocation fails as if cudaMalloc had.
extern thread_local int *t_alloc_fault;

// A device buffer that only grows.
struct DevBuf {
    void *ptr = nullptr;
    size_t cap = 0;
    cpl_status ensure(size_t bytes, const char *what) {
        if (bytes <= cap) return CPL_OK;
        if (ptr) cudaFree(ptr);
        ptr = nullptr;
        cap = 0;
        if (t_alloc_fault && *t_alloc_fault > 0 && --*t_alloc_fault == 0)
            return fail(CPL_ERR_OOM, std::string("device allocation failed for ") + what + " (injected)");
        size_t want = std::max(bytes, (size_t)256);
        if (cudaMalloc(&ptr, want) != cudaSuccess) {
            cudaGetLastError();
            return fail(CPL_ERR_OOM, std::string("device allocation failed for ") + what);
        }
        cap = want;
        return CPL_OK;
    }
    void release() {
        if (ptr) cudaFree(ptr);
        ptr = nullptr;
        cap = 0;
    }
    template <class T>
    T *as() const { return static_cast<T *>(ptr); }
};

struct TileSet {
    std::vector<Tile> host;
    DevBuf dev;
    // per-tile l3 term counts (even, odd, pairs) for windows without a band
    // limit (cap >= 2 lmax), filled on first use by the launch accounting
    std::vector<double> terms;
    // the same under band limits (cap -> counts), bounded in number of caps
    std::map<int, std::vector<double>> band_terms;
};


struct MxPlan;                    // a planned batch (mixed_host.cu)
struct MxPlanDeleter {
    void operator()(MxPlan *p) const;
};

// One autotuner decision: the key describes a request shape (mixed_host.cu
// tune_key), src / order the chosen row shape and item order.
struct TuneEntry {
    std::vector<long long> key;
    int src = 0, order = 0;
    double ms = 0.0;
};

// Scratch and caches of the mixed-precision path.
struct MixedState {
    int S = 0;                   // limbs the B cache was built with
    int NC_B = 0;                // column blocks in the B cache
    DevBuf Bimg, eB, emaxB;      // window-independent operand images (cache)
    int pmax_dd = -1;
    DevBuf gdd;                  // g, h as double-float: gh | gl | hh | hl
    DevBuf arena;                // per-job scratch of the running chunk (A images, weights, GEMM output)
    DevBuf ticket;               // work-item ticket of the persistent GEMM
    DevBuf err;                  // device error word of the bounded waits
    DevBuf coef;                 // per-l factors of the pair coefficients (MX_COEF_N per l, extended double-float)
    int coef_n = 0;              // l < coef_n covered
    std::vector<std::unique_ptr<MxPlan, MxPlanDeleter>> plans;   // cached plans (LRU)
    unsigned long long clock = 0;
    int nsm = 0;
    cudaStream_t cap_stream = nullptr;   // stream used only for graph capture
    int tune_mode = 0;                   // cpl_tune_mode
    std::string tune_path;               // persisted choices ("" = none)
    std::vector<TuneEntry> tuned;
};

}  // namespace cpl

using cpl::DevBuf;
using cpl::TileSet;

struct cpl_ctx {
    cpl::MixedState mx;
    int device = 0;
    int pmax = -1;
    DevBuf g, h;                 // lookup tables (Sec. 3.1)
    std::vector<std::unique_ptr<TileSet>> tile_sets;
    std::vector<std::pair<long long, TileSet *>> tile_index;   // key (lmax, lmin)
    DevBuf weights;              // FP64 path: A(l3) per sweep and window
    DevBuf items;                // FP64 path: sweep table, caps, bins and work items of the last build
    DevBuf stage_w, stage_out;   // cpl_build_host staging
    DevBuf threej_idx;           // cpl_threej_m11: (j2, j3) of the last call
    DevBuf sqrt_tab;             // cpl_threej_m11: five square-root tables of g and h (pmax + 1 each), FP32 pairs
    int sq_pmax = -1;
    DevBuf df_tab;               // CPL_DF32: g | h as FP32 pairs (pmax + 1 each)
    int df_pmax = -1;
    DevBuf ptab_b;               // tabled FP64 kernel: B operand blocks (window independent)
    int ptab_njb = 0;            // column blocks ptab_b covers (0: none)
    DevBuf ptab_a;               // tabled FP64 kernel: A operand blocks of the last build
    DevBuf pl_coef;              // FP64 epilogue: per-l factors of the pair coefficients
    int pl_coef_n = 0;           // l < pl_coef_n covered
    DevBuf dec_ws;               // cpl_decouple: augmented systems too large for shared memory
    DevBuf cov_M, cov_dense, cov_edges;   // cpl_cov_gaussian: kernels of one build, dense covariance, bin edges
    cudaStream_t own_stream = nullptr;
    cudaStream_t copy_stream = nullptr;      // cpl_build_host: device-to-host copies overlapped with later kernels
    std::vector<cudaEvent_t> copy_ev;        // its ordering events (one per kernel variant)
    cudaEvent_t done = nullptr;  // orders scratch reuse across caller streams
    // per-kernel accounting (cpl_ctx_stats)
    struct KStat {
        std::string name;
        long long launches = 0;
        double ms = 0.0, flop = 0.0, bytes = 0.0, issued = 0.0;
    };
    struct Pending {
        int idx;
        cudaEvent_t a, b;
        double flop, bytes, issued;
    };
    int alloc_fault = 0;         // cpl_ctx_inject_alloc_failure countdown (0 = off)
    bool profiling = false;
    bool validate_w = false;     // cpl_ctx_validate: check windows for NaN / Inf before building
    DevBuf check;                // its device result word
    std::vector<KStat> kstats;
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> ev_pool;
};

namespace cpl {
cpl_status ensure_tables(cpl_ctx *c, int lmax);
cpl_status get_tiles(cpl_ctx *c, int lmax, int lmin, TileSet **out);
cpl_status build_mixed(cpl_ctx *c, const cpl_request *r, double *out, cudaStream_t st);
cpl_status build_mixed_batch(cpl_ctx *c, const cpl_request *reqs, double *const *outs, int n, cudaStream_t st,
                             bool use_graph);
cpl_status set_tuning(cpl_ctx *c, int mode, const char *path);
int stat_index(cpl_ctx *c, const char *name);
void record_launch(cpl_ctx *c, int idx, cudaEvent_t a, cudaStream_t st, double flop, double bytes,
                   double issued = -1.0);
cudaEvent_t begin_launch(cpl_ctx *c, cudaStream_t st);
cudaEvent_t take_event(cpl_ctx *c);
// Makes the context's device current and points the allocation-failure hook
// at the context (every public entry point calls it before device work).
cpl_status select_device(cpl_ctx *c);
// The device error word of the bounded waits (mx.err), allocated and zeroed
// on first use.
cpl_status ensure_err_word(cpl_ctx *c, cudaStream_t st);

// Brackets one kernel launch: counts it and, when profiling, times it with
// events on the launching stream.
struct LaunchScope {
    cpl_ctx *c;
    int idx;
    cudaStream_t st;
    cudaEvent_t a = nullptr;
    LaunchScope(cpl_ctx *c_, const char *name, cudaStream_t st_) : c(c_), idx(stat_index(c_, name)), st(st_) {
        if (c->profiling) {
            a = take_event(c);
            if (a) cudaEventRecord(a, st);
        }
    }
    void done(double flop, double bytes) {
        c->kstats[idx].launches++;
        if (c->profiling && a) {
            cudaEvent_t b = take_event(c);
            if (b) {
                cudaEventRecord(b, st);
                c->pending.push_back({idx, a, b, flop, bytes, flop});
                return;
            }
            c->ev_pool.push_back(a);
        }
    }
};
}  // namespace cpl
