// api.cu -- the C ABI of coupling.h: validation, context, orchestration.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "ctx.h"

#define CPL_VERSION_STRING "paper_2602_15605_gb300 coupling 0.1 (sm_103a)"

namespace cpl {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

thread_local int *t_alloc_fault = nullptr;

cpl_status fail(cpl_status s, const std::string &msg) {
    set_error(msg);
    return s;
}

int spec_count(unsigned s) {
    int c = 0;
    for (int b = 0; b < 5; ++b) c += (s >> b) & 1u;
    return c;
}

void bin_weights_dl(int lmax, std::vector<double> &w) {
    w.assign(2 * (size_t)(lmax + 1), 0.0);
    for (int l = 1; l <= lmax; ++l) {
        const double x = (double)l * (double)(l + 1);
        w[l] = x;
        w[lmax + 1 + l] = 1.0 / x;
    }
}

int spec_slot(unsigned s, unsigned bit) {
    if (!(s & bit)) return -1;
    int c = 0;
    for (unsigned b = 1; b < bit; b <<= 1) c += (s & b) ? 1 : 0;
    return c;
}

}  // namespace cpl

using namespace cpl;


namespace cpl {

int stat_index(cpl_ctx *c, const char *name) {
    for (size_t q = 0; q < c->kstats.size(); ++q)
        if (c->kstats[q].name == name) return (int)q;
    c->kstats.push_back(cpl_ctx::KStat());
    c->kstats.back().name = name;
    return (int)c->kstats.size() - 1;
}

cudaEvent_t take_event(cpl_ctx *c) {
    if (!c->ev_pool.empty()) {
        cudaEvent_t e = c->ev_pool.back();
        c->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

cudaEvent_t begin_launch(cpl_ctx *c, cudaStream_t st) {
    if (!c->profiling) return nullptr;
    cudaEvent_t a = take_event(c);
    if (a) cudaEventRecord(a, st);
    return a;
}

void record_launch(cpl_ctx *c, int idx, cudaEvent_t a, cudaStream_t st, double flop, double bytes, double issued) {
    if (issued < 0.0) issued = flop;
    c->kstats[idx].launches++;
    if (c->profiling && a) {
        cudaEvent_t b = take_event(c);
        if (b) {
            cudaEventRecord(b, st);
            c->pending.push_back({idx, a, b, flop, bytes, issued});
            return;
        }
        c->ev_pool.push_back(a);
    }
}

cpl_status select_device(cpl_ctx *c) {
    t_alloc_fault = &c->alloc_fault;   // allocations of this call count against the context's hook
    CPL_CUDA_TRY(cudaSetDevice(c->device));
    return CPL_OK;
}

bool wants_pol(unsigned s) { return (s & (kTE | kEE | kEEBB | kEB)) != 0; }

cpl_status validate(const cpl_request *r, bool device_ptrs) {
    (void)device_ptrs;
    if (!r) return fail(CPL_ERR_ARG, "request is NULL");
    if (r->lmax < 2) return fail(CPL_ERR_ARG, "lmax must be >= 2");
    if (r->lmax > 32000) return fail(CPL_ERR_RANGE, "lmax above 32000 is not supported");
    if (r->lmin < 0 || r->lmin > r->lmax) return fail(CPL_ERR_ARG, "lmin must lie in [0, lmax]");
    if (r->spectra == 0 || (r->spectra & ~31u)) return fail(CPL_ERR_ARG, "spectra must be a non-empty OR of CPL_* bits");
    if (wants_pol(r->spectra) && r->lmin < 2)
        return fail(CPL_ERR_ARG, "polarisation spectra need lmin >= 2");
    if (r->n_windows < 1) return fail(CPL_ERR_ARG, "n_windows must be >= 1");
    if (r->n_windows > 65535) return fail(CPL_ERR_RANGE, "n_windows above 65535 is not supported");
    if ((r->spectra & kTT) && !r->W_tt) return fail(CPL_ERR_ARG, "W_tt is NULL but CPL_TT is requested");
    if ((r->spectra & kTE) && !r->W_tp) return fail(CPL_ERR_ARG, "W_tp is NULL but CPL_TE is requested");
    if ((r->spectra & (kEE | kEEBB | kEB)) && !r->W_pp)
        return fail(CPL_ERR_ARG, "W_pp is NULL but a polarisation spectrum is requested");
    if (r->w_len < 1) return fail(CPL_ERR_ARG, "w_len must be >= 1");
    const int need = 2 * r->lmax;
    for (int w = 0; w < r->n_windows; ++w) {
        int top = need;
        if (r->band_limit) {
            if (r->band_limit[w] < 0) return fail(CPL_ERR_ARG, "band_limit entries must be >= 0");
            top = std::min(top, r->band_limit[w]);
        }
        if (r->w_len < top + 1)
            return fail(CPL_ERR_ARG, "w_len too short: the l3 sum needs W up to min(2 lmax, band_limit)");
    }
    if (r->precision != CPL_FP64 && r->precision != CPL_MIXED_BF16 && r->precision != CPL_DF32)
        return fail(CPL_ERR_ARG, "unknown precision");
    if (r->precision == CPL_DF32 && r->lmax > CPL_DF32_LMAX)
        return fail(CPL_ERR_RANGE, "CPL_DF32 needs lmax <= CPL_DF32_LMAX (FP32 exponent range of the contractions)");
    if (r->precision == CPL_MIXED_BF16 && r->mixed_slices != 0 &&
        (r->mixed_slices < 4 || r->mixed_slices > 6))
        return fail(CPL_ERR_ARG, "mixed_slices must be 0 or in 4..6");
    if (r->bin_edges) {
        if (r->n_bins < 1) return fail(CPL_ERR_ARG, "n_bins must be >= 1 with bin_edges");
        if (r->bin_edges[0] < r->lmin || r->bin_edges[r->n_bins] > r->lmax + 1)
            return fail(CPL_ERR_ARG, "bin_edges must lie inside [lmin, lmax + 1]");
        for (int b = 0; b < r->n_bins; ++b)
            if (r->bin_edges[b + 1] <= r->bin_edges[b]) return fail(CPL_ERR_ARG, "bin_edges must increase");
    } else if (r->n_bins != 0) {
        return fail(CPL_ERR_ARG, "n_bins must be 0 without bin_edges");
    }
    if (r->bin_weight != 0 && r->bin_weight != 1) return fail(CPL_ERR_ARG, "bin_weight must be 0 or 1");
    if (r->bin_weight && (!r->bin_edges || r->bin_edges[0] < 1))
        return fail(CPL_ERR_ARG, "bin_weight = 1 needs bin_edges starting at l >= 1");
    return CPL_OK;
}

}  // namespace cpl

namespace {

size_t out_doubles(const cpl_request *r) {
    const size_t ns = (size_t)spec_count(r->spectra);
    if (r->bin_edges) return (size_t)r->n_windows * ns * (size_t)r->n_bins * (size_t)r->n_bins;
    const size_t n = (size_t)(r->lmax - r->lmin + 1);
    return (size_t)r->n_windows * ns * n * n;
}

}  // namespace

namespace cpl {

cpl_status ensure_tables(cpl_ctx *c, int lmax) {
    const int need = 2 * lmax + 2 * (TILE_I + TILE_J) + 16;
    if (need <= c->pmax) return CPL_OK;
    const int pmax = std::max(need, 2 * c->pmax);
    std::vector<double> g, h;
    build_tables_host(pmax, g, h);
    cpl_status s;
    c->pmax = -1;   // invalid until both tables are rebuilt (a failed reallocation frees them)
    if ((s = c->g.ensure(sizeof(double) * (pmax + 1), "g table")) != CPL_OK) return s;
    if ((s = c->h.ensure(sizeof(double) * (pmax + 1), "h table")) != CPL_OK) return s;
    CPL_CUDA_TRY(cudaMemcpy(c->g.ptr, g.data(), sizeof(double) * (pmax + 1), cudaMemcpyHostToDevice));
    CPL_CUDA_TRY(cudaMemcpy(c->h.ptr, h.data(), sizeof(double) * (pmax + 1), cudaMemcpyHostToDevice));
    c->pmax = pmax;
    return CPL_OK;
}

cpl_status ensure_err_word(cpl_ctx *c, cudaStream_t st) {
    if (c->mx.err.ptr) return CPL_OK;
    cpl_status s;
    if ((s = c->mx.err.ensure(sizeof(int), "device error word")) != CPL_OK) return s;
    CPL_CUDA_TRY(cudaMemsetAsync(c->mx.err.ptr, 0, sizeof(int), st));
    return CPL_OK;
}

cpl_status get_tiles(cpl_ctx *c, int lmax, int lmin, TileSet **out) {
    const long long key = (long long)lmax * 65536LL + lmin;
    for (auto &kv : c->tile_index)
        if (kv.first == key) {
            *out = kv.second;
            return CPL_OK;
        }
    auto ts = std::make_unique<TileSet>();
    make_tiles(lmax, lmin, ts->host);
    cpl_status s = ts->dev.ensure(sizeof(Tile) * std::max<size_t>(ts->host.size(), 1), "tile list");
    if (s != CPL_OK) return s;
    if (!ts->host.empty())
        CPL_CUDA_TRY(cudaMemcpy(ts->dev.ptr, ts->host.data(), sizeof(Tile) * ts->host.size(),
                                cudaMemcpyHostToDevice));
    *out = ts.get();
    c->tile_index.emplace_back(key, ts.get());
    c->tile_sets.push_back(std::move(ts));
    return CPL_OK;
}

}  // namespace cpl

namespace {

// Work items (window, tile) of one request with their run-time costs
// (tile_time; a band-limited window shortens a tile's k range).  A tile whose
// smallest |d| exceeds a window's last l3 contributes nothing for that window
// and is dropped (the output is pre-zeroed in that case).
void make_items(const TileSet &ts, const std::vector<int> &caps, bool banded,
                std::vector<std::pair<double, WorkItem>> &items) {
    const std::vector<Tile> &tiles = ts.host;
    items.clear();
    const int nw = (int)caps.size();
    for (int ti = 0; ti < (int)tiles.size(); ++ti) {
        const Tile &t = tiles[ti];
        for (int w = 0; w < nw; ++w) {
            if (banded && 2 * t.i0 + t.pi > caps[w]) continue;
            const double cost = banded ? tile_time(t, caps[w]) : (double)t.cost;
            items.emplace_back(cost, WorkItem{0, w, ti, 0});
        }
    }
}

struct Group {
    const double *W;
    unsigned spectra;   // spectra this window pointer serves
};

// The window-role groups of a request: roles that share a pointer share one
// sweep (PlainJob) and one kernel variant.
std::vector<Group> window_groups(const cpl_request *r) {
    std::vector<Group> groups;
    auto add = [&](const double *W, unsigned b) {
        if (!(r->spectra & b)) return;
        for (auto &g : groups)
            if (g.W == W) {
                g.spectra |= (r->spectra & b);
                return;
            }
        groups.push_back({W, r->spectra & b});
    };
    add(r->W_tt, kTT);
    add(r->W_tp, kTE);
    add(r->W_pp, kEE | kEEBB | kEB);
    return groups;
}

// A blocks of the tabled kernel for row block ib and parity pi of a window
// whose l3 ends at cap: the chunks 2 ib .. of the block's k range, which
// ends at min(lmax - pi - i0 + 31, cap / 2) (the last column of the block's
// last tile, or the band).
int a_block_count(int lmax, int lmin, int pi, int ib, int cap) {
    const int imax = (lmax - lmin - pi) / 2;   // rows of this parity's tiles
    if (lmax - lmin - pi < 0 || TILE_I * ib > imax) return 0;
    const int cend = std::min((lmax - pi - TILE_I * ib + TILE_J - 1) / PT_KC, (cap / 2) / PT_KC) + 1;
    return std::max(0, cend - 2 * ib);
}

// l3 cap of each window of a request (its band limit, else 2 lmax or the
// end of W), and whether any window is band-limited.
bool window_caps(const cpl_request *r, std::vector<int> &caps) {
    bool banded = false;
    caps.resize(r->n_windows);
    for (int w = 0; w < r->n_windows; ++w) {
        int cap = std::min(2 * r->lmax, r->w_len - 1);
        if (r->band_limit) cap = std::min(cap, r->band_limit[w]);
        if (cap < 2 * r->lmax) banded = true;
        caps[w] = cap;
    }
    return banded;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// The plain FP64 build of a batch of requests on `st` (device pointers).
// Every request's window-role groups become sweeps (PlainJob); the work
// items of all sweeps that run the same kernel variant are merged into one
// list, heaviest first, and run by one launch; the launches run longest
// first.  With host_outs, the output blocks a launch completes are copied
// to host_outs on c->copy_stream while the later launches run (the caller
// synchronises that stream).
cpl_status build_fp64_batch(cpl_ctx *c, const cpl_request *reqs, double *const *outs, int n, cudaStream_t st,
                            double *const *host_outs = nullptr) {
    cpl_status s;
    int lmax_all = 2;
    for (int q = 0; q < n; ++q) lmax_all = std::max(lmax_all, reqs[q].lmax);
    if ((s = ensure_tables(c, lmax_all)) != CPL_OK) return s;
    const bool df = reqs[0].precision == CPL_DF32;
    if (df && c->df_pmax != c->pmax) {
        // g and h as FP32 pairs for the double-float kernels
        const int np1 = c->pmax + 1;
        c->df_pmax = -1;
        CPL_CUDA_TRY(cudaStreamWaitEvent(st, c->done, 0));
        if ((s = c->df_tab.ensure(sizeof(float2) * 2 * (size_t)np1, "double-float tables")) != CPL_OK) return s;
        float2 *t2 = c->df_tab.as<float2>();
        LaunchScope ls(c, "df_tables", st);
        CPL_CUDA_TRY(launch_df_tables(c->g.as<double>(), c->h.as<double>(), np1, t2, t2 + np1, st));
        ls.done(0.0, 32.0 * np1);
        c->df_pmax = c->pmax;
    }

    struct JobInfo {
        TileSet *ts = nullptr;
        std::vector<int> caps;
        bool banded = false;
        int nb = 0;
        std::vector<int> bin_of;
        std::vector<double> bin_inv;
        std::vector<double> bin_lw;   // D_l weighting: l(l+1) | 1 / (l(l+1)), or empty
        std::vector<std::pair<double, WorkItem>> items;
        size_t o_cap = 0, o_binof = 0, o_bininv = 0, o_binlw = 0;
    };
    struct Sweep {
        int job;
        Group G;
        int slot[5];
        int nge;
        bool odd;
        size_t a_off;   // doubles into the weights buffer
        // tabled kernel: A-block offsets [n_win][2][nib] + 1 and the sweep's place in the A table
        int nib = 0, nae = 0, max_count = 0;
        std::vector<long long> aoff;
        size_t atab_off = 0;   // doubles into the A table
        size_t o_aoff = 0;     // bytes into the metadata buffer
    };
    std::vector<JobInfo> jobs(n);
    std::vector<Sweep> sweeps;
    const unsigned bits[5] = {kTT, kTE, kEE, kEEBB, kEB};
    size_t a_total = 0;
    for (int q = 0; q < n; ++q) {
        const cpl_request *r = reqs + q;
        JobInfo &J = jobs[q];
        if ((s = get_tiles(c, r->lmax, r->lmin, &J.ts)) != CPL_OK) return s;
        const int nw = r->n_windows;
        J.banded = window_caps(r, J.caps);
        J.nb = r->bin_edges ? r->n_bins : 0;
        if (J.nb) {
            J.bin_of.assign(r->lmax + 1, -1);
            J.bin_inv.assign(J.nb, 0.0);
            for (int b = 0; b < J.nb; ++b) {
                for (int l = r->bin_edges[b]; l < r->bin_edges[b + 1]; ++l) J.bin_of[l] = b;
                J.bin_inv[b] = 1.0 / (double)(r->bin_edges[b + 1] - r->bin_edges[b]);
            }
            if (r->bin_weight) bin_weights_dl(r->lmax, J.bin_lw);
        }
        make_items(*J.ts, J.caps, J.banded, J.items);
        // window roles sharing one pointer share one sweep
        const std::vector<Group> groups = window_groups(r);
        const int a_stride = 2 * r->lmax + 2;
        for (const Group &G : groups) {
            Sweep sw;
            sw.job = q;
            sw.G = G;
            for (int x = 0; x < 5; ++x) sw.slot[x] = (G.spectra & bits[x]) ? spec_slot(r->spectra, bits[x]) : -1;
            const int mode = (G.spectra & (kEE | kEEBB | kEB)) ? MODE_POL : (G.spectra & kTE) ? MODE_TE : MODE_TT;
            plain_variant(mode, sw.slot, &sw.nge, &sw.odd);
            sw.a_off = a_total;
            a_total += (size_t)a_stride * nw;
            sweeps.push_back(sw);
        }
    }

    // ---- operand tables of the tabled FP64 kernel (sizes; built after the weights)
    bool tab = !df;
    if (const char *e = std::getenv("CPL_PLAIN_TABLES")) tab = tab && std::strcmp(e, "0") != 0;
    int njb_need = 0;
    size_t atab_total = 0;   // doubles
    if (tab) {
        for (Sweep &sw : sweeps) {
            const cpl_request *r = reqs + sw.job;
            const JobInfo &J = jobs[sw.job];
            const int nw = r->n_windows;
            sw.nae = sw.nge == 0 ? 0 : sw.nge == 1 ? 1 : sw.nge == 3 ? 2 : 3;
            const int na = sw.nae + (sw.odd ? 1 : 0);
            sw.nib = (r->lmax - r->lmin) / 2 / TILE_I + 1;
            sw.aoff.assign((size_t)nw * 2 * sw.nib + 1, 0);
            long long blocks = 0;
            for (int w = 0; w < nw; ++w)
                for (int pi = 0; pi < 2; ++pi) {
                    for (int ib = 0; ib < sw.nib; ++ib) {
                        const int count = a_block_count(r->lmax, r->lmin, pi, ib, J.caps[w]);
                        sw.aoff[((size_t)w * 2 + pi) * sw.nib + ib] = blocks;
                        blocks += count;
                        sw.max_count = std::max(sw.max_count, count);
                    }
                }
            sw.aoff.back() = blocks;
            sw.atab_off = atab_total;
            atab_total += (size_t)blocks * na * PT_BLK;
            njb_need = std::max(njb_need, r->lmax / TILE_J + 1);
        }
        // budget: the tables may take at most half of the free device memory
        size_t need = 0;
        if (njb_need > c->ptab_njb) need += sizeof(double) * (size_t)btab_block(njb_need, 0, 0) * PT_BROWS * PT_BLK;
        if (sizeof(double) * atab_total > c->ptab_a.cap) need += sizeof(double) * atab_total;
        size_t free_b = 0, total_b = 0;
        if (need > 0 && (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess || need > free_b / 2)) {
            cudaGetLastError();
            tab = false;
        }
    }

    // ---- items per kernel variant, heaviest first
    auto vkey = [](int nge, bool odd) { return nge * 2 + (odd ? 1 : 0); };
    std::vector<int> keys;
    for (const Sweep &sw : sweeps)
        if (std::find(keys.begin(), keys.end(), vkey(sw.nge, sw.odd)) == keys.end()) keys.push_back(vkey(sw.nge, sw.odd));
    std::vector<std::vector<WorkItem>> vitems(keys.size());
    for (size_t k = 0; k < keys.size(); ++k) {
        std::vector<std::pair<double, WorkItem>> tmp;
        for (size_t x = 0; x < sweeps.size(); ++x) {
            if (vkey(sweeps[x].nge, sweeps[x].odd) != keys[k]) continue;
            for (auto it : jobs[sweeps[x].job].items) {
                it.second.job = (int32_t)x;
                tmp.push_back(it);
            }
        }
        std::stable_sort(tmp.begin(), tmp.end(), [](const std::pair<double, WorkItem> &a,
                                                    const std::pair<double, WorkItem> &b) { return a.first > b.first; });
        vitems[k].reserve(tmp.size());
        for (auto &p : tmp) vitems[k].push_back(p.second);
    }
    // launch order: the longest variant first (its output blocks can then be
    // copied out while the shorter ones run)
    std::vector<size_t> korder(keys.size());
    {
        std::vector<double> kcost(keys.size(), 0.0);
        for (size_t x = 0; x < sweeps.size(); ++x) {
            const size_t k = std::find(keys.begin(), keys.end(), vkey(sweeps[x].nge, sweeps[x].odd)) - keys.begin();
            const double per = (double)(sweeps[x].nge + (sweeps[x].odd ? 3 : 0));
            for (const auto &it : jobs[sweeps[x].job].items) kcost[k] += per * it.first;
        }
        for (size_t k = 0; k < keys.size(); ++k) korder[k] = k;
        std::stable_sort(korder.begin(), korder.end(), [&](size_t a, size_t b) { return kcost[a] > kcost[b]; });
    }

    // ---- one metadata buffer: sweep table, caps, bins, items
    size_t o = 0;
    const size_t o_jobs = o;
    o = align256(o + sizeof(PlainJob) * sweeps.size());
    for (JobInfo &J : jobs) {
        J.o_cap = o;
        o = align256(o + sizeof(int) * J.caps.size());
        J.o_binof = o;
        o = align256(o + sizeof(int) * J.bin_of.size());
        J.o_bininv = o;
        o = align256(o + sizeof(double) * J.bin_inv.size());
        J.o_binlw = o;
        o = align256(o + sizeof(double) * J.bin_lw.size());
    }
    std::vector<size_t> o_items(keys.size());
    for (size_t k = 0; k < keys.size(); ++k) {
        o_items[k] = o;
        o = align256(o + sizeof(WorkItem) * vitems[k].size());
    }
    if (tab)
        for (Sweep &sw : sweeps) {
            sw.o_aoff = o;
            o = align256(o + sizeof(long long) * sw.aoff.size());
        }
    if ((s = c->items.ensure(std::max<size_t>(o, 256), "work items")) != CPL_OK) return s;
    if ((s = c->weights.ensure(sizeof(double) * std::max<size_t>(a_total, 1), "weights")) != CPL_OK) return s;
    if (tab) {
        if (njb_need > c->ptab_njb) {
            c->ptab_njb = 0;   // invalid until rebuilt
            if ((s = c->ptab_b.ensure(sizeof(double) * (size_t)btab_block(njb_need, 0, 0) * PT_BROWS * PT_BLK,
                                      "operand B table")) != CPL_OK)
                return s;
        }
        if ((s = c->ptab_a.ensure(sizeof(double) * std::max<size_t>(atab_total, 1), "operand A table")) != CPL_OK)
            return s;
        if ((s = ensure_err_word(c, st)) != CPL_OK) return s;
    }
    if (!df && c->pl_coef_n < lmax_all + 1) {
        // per-l factors of the epilogue's pair coefficients (the same values for every call)
        c->pl_coef_n = 0;
        if ((s = c->pl_coef.ensure(sizeof(double) * PL_COEF_N * (size_t)(lmax_all + 1), "pair coefficient factors")) !=
            CPL_OK)
            return s;
        std::vector<double> hc;
        plain_coef_host(lmax_all + 1, hc);
        CPL_CUDA_TRY(cudaMemcpyAsync(c->pl_coef.ptr, hc.data(), sizeof(double) * hc.size(), cudaMemcpyHostToDevice, st));
        c->pl_coef_n = lmax_all + 1;
    }
    uint8_t *dmeta = c->items.as<uint8_t>();
    double *dA = c->weights.as<double>();
    std::vector<uint8_t> host(o, 0);
    for (size_t x = 0; x < sweeps.size(); ++x) {
        const Sweep &sw = sweeps[x];
        const cpl_request *r = reqs + sw.job;
        const JobInfo &J = jobs[sw.job];
        PlainJob pj;
        std::memset(&pj, 0, sizeof(pj));
        pj.A = dA + sw.a_off;
        pj.a_stride = 2 * r->lmax + 2;
        pj.l3cap = reinterpret_cast<const int *>(dmeta + J.o_cap);
        pj.tiles = J.ts->dev.as<Tile>();
        pj.lmax = r->lmax;
        pj.lmin = r->lmin;
        pj.out = outs[sw.job];
        pj.nspec = spec_count(r->spectra);
        for (int q = 0; q < 5; ++q) pj.slot[q] = sw.slot[q];
        pj.n_bins = J.nb;
        pj.bin_of = J.nb ? reinterpret_cast<const int *>(dmeta + J.o_binof) : nullptr;
        pj.bin_inv = J.nb ? reinterpret_cast<const double *>(dmeta + J.o_bininv) : nullptr;
        pj.bin_lw = J.bin_lw.empty() ? nullptr : reinterpret_cast<const double *>(dmeta + J.o_binlw);
        if (tab) {
            pj.atab = c->ptab_a.as<double>() + sw.atab_off;
            pj.aoff = reinterpret_cast<const long long *>(dmeta + sw.o_aoff);
            pj.nib = sw.nib;
        }
        std::memcpy(host.data() + o_jobs + x * sizeof(PlainJob), &pj, sizeof(pj));
    }
    for (const JobInfo &J : jobs) {
        std::memcpy(host.data() + J.o_cap, J.caps.data(), sizeof(int) * J.caps.size());
        if (J.nb) {
            std::memcpy(host.data() + J.o_binof, J.bin_of.data(), sizeof(int) * J.bin_of.size());
            std::memcpy(host.data() + J.o_bininv, J.bin_inv.data(), sizeof(double) * J.bin_inv.size());
            if (!J.bin_lw.empty())
                std::memcpy(host.data() + J.o_binlw, J.bin_lw.data(), sizeof(double) * J.bin_lw.size());
        }
    }
    for (size_t k = 0; k < keys.size(); ++k)
        if (!vitems[k].empty())
            std::memcpy(host.data() + o_items[k], vitems[k].data(), sizeof(WorkItem) * vitems[k].size());
    if (tab)
        for (const Sweep &sw : sweeps)
            std::memcpy(host.data() + sw.o_aoff, sw.aoff.data(), sizeof(long long) * sw.aoff.size());

    CPL_CUDA_TRY(cudaStreamWaitEvent(st, c->done, 0));
    CPL_CUDA_TRY(cudaMemcpyAsync(dmeta, host.data(), o, cudaMemcpyHostToDevice, st));
    for (int q = 0; q < n; ++q)
        if (jobs[q].nb || jobs[q].banded) CPL_CUDA_TRY(cudaMemsetAsync(outs[q], 0, sizeof(double) * out_doubles(reqs + q), st));
    for (const Sweep &sw : sweeps) {
        const cpl_request *r = reqs + sw.job;
        const int a_stride = 2 * r->lmax + 2;
        LaunchScope ls(c, "window_weights", st);
        CPL_CUDA_TRY(launch_weights(sw.G.W, r->w_len, r->n_windows,
                                    reinterpret_cast<const int *>(dmeta + jobs[sw.job].o_cap), dA + sw.a_off, a_stride,
                                    st));
        ls.done(0.0, 16.0 * (double)a_stride * r->n_windows);
    }
    if (tab) {
        if (njb_need > c->ptab_njb) {
            LaunchScope ls(c, "plain_tables_b", st);
            CPL_CUDA_TRY(launch_btab(c->g.as<double>(), c->h.as<double>(), njb_need, c->ptab_b.as<double>(), st));
            ls.done(0.0, 8.0 * (double)btab_block(njb_need, 0, 0) * PT_BROWS * PT_BLK);
            c->ptab_njb = njb_need;
        }
        for (const Sweep &sw : sweeps) {
            const cpl_request *r = reqs + sw.job;
            LaunchScope ls(c, "plain_tables_a", st);
            CPL_CUDA_TRY(launch_atab(dA + sw.a_off, 2 * r->lmax + 2, reinterpret_cast<const int *>(dmeta + jobs[sw.job].o_cap),
                                     c->g.as<double>(), reinterpret_cast<const long long *>(dmeta + sw.o_aoff),
                                     r->n_windows, sw.nib, sw.max_count, sw.nae, sw.odd ? 1 : 0,
                                     c->ptab_a.as<double>() + sw.atab_off, st));
            ls.done(0.0, 8.0 * (double)sw.aoff.back() * (sw.nae + (sw.odd ? 1 : 0)) * PT_BLK);
        }
    }
    if (host_outs) {
        if (!c->copy_stream) CPL_CUDA_TRY(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
        while (c->copy_ev.size() < keys.size()) {
            cudaEvent_t e;
            CPL_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            c->copy_ev.push_back(e);
        }
    }
    for (size_t ko = 0; ko < korder.size(); ++ko) {
        const size_t k = korder[ko];
        PlainArgs a;
        std::memset(&a, 0, sizeof(a));
        a.g = c->g.as<double>();
        a.h = c->h.as<double>();
        a.jobs = reinterpret_cast<const PlainJob *>(dmeta + o_jobs);
        a.items = reinterpret_cast<const WorkItem *>(dmeta + o_items[k]);
        a.n_items = (int)vitems[k].size();
        a.nge = keys[k] / 2;
        a.odd = keys[k] & 1;
        const bool odd = a.odd != 0;
        const char *kname = df ? (a.nge == 1 ? "plain_df_tt" : a.nge == 3 ? "plain_df_te"
                                  : (a.nge == 6 && odd) ? "plain_df_pol" : a.nge == 6 ? "plain_df_even" : "plain_df_odd")
                               : (a.nge == 1 ? "plain_fp64_tt" : a.nge == 3 ? "plain_fp64_te"
                                  : (a.nge == 6 && odd) ? "plain_fp64_pol" : a.nge == 6 ? "plain_fp64_even" : "plain_fp64_odd");
        if (df) {
            a.gdf = c->df_tab.as<float2>();
            a.hdf = a.gdf + (c->pmax + 1);
        }
        if (!df) a.lcoef = c->pl_coef.as<double>();
        if (tab) {
            a.btab = c->ptab_b.as<double>();
            a.btab_njb = c->ptab_njb;
            a.err = c->mx.err.as<int>();
        }
        double flop = 0.0, bytes = 0.0;
        if (c->profiling) {
            // 2 FLOP per FMA: nge FMAs per even-L term, 3 per odd-L term;
            // bytes: each written spectrum stores both mirror entries once.
            for (const WorkItem &it : vitems[k]) {
                const Sweep &sw = sweeps[it.job];
                const cpl_request *r = reqs + sw.job;
                const JobInfo &J = jobs[sw.job];
                int nslots = 0;
                for (int q = 0; q < 5; ++q) nslots += sw.slot[q] >= 0;
                double e, od, np;
                if (J.caps[it.win] >= 2 * r->lmax) {
                    std::vector<double> &T = J.ts->terms;
                    if (T.size() != 3 * J.ts->host.size()) {
                        T.resize(3 * J.ts->host.size());
                        for (size_t q = 0; q < J.ts->host.size(); ++q)
                            tile_terms_split(J.ts->host[q], r->lmax, r->lmin, 2 * r->lmax, &T[3 * q], &T[3 * q + 1],
                                             &T[3 * q + 2]);
                    }
                    e = T[3 * it.tile];
                    od = T[3 * it.tile + 1];
                    np = T[3 * it.tile + 2];
                } else {
                    if (J.ts->band_terms.size() > 64 && !J.ts->band_terms.count(J.caps[it.win])) J.ts->band_terms.clear();
                    std::vector<double> &T = J.ts->band_terms[J.caps[it.win]];
                    if (T.size() != 3 * J.ts->host.size()) {
                        T.resize(3 * J.ts->host.size());
                        for (size_t q = 0; q < J.ts->host.size(); ++q) {
                            const Tile &tq = J.ts->host[q];
                            if (2 * tq.i0 + tq.pi > J.caps[it.win]) {   // dropped for this cap: no work
                                T[3 * q] = T[3 * q + 1] = T[3 * q + 2] = 0.0;
                                continue;
                            }
                            tile_terms_split(tq, r->lmax, r->lmin, J.caps[it.win], &T[3 * q], &T[3 * q + 1], &T[3 * q + 2]);
                        }
                    }
                    e = T[3 * it.tile];
                    od = T[3 * it.tile + 1];
                    np = T[3 * it.tile + 2];
                }
                flop += 2.0 * (a.nge * e + (odd ? 3.0 : 0.0) * od);
                bytes += (J.nb ? 0.0 : 16.0) * nslots * np;
            }
        }
        LaunchScope ls(c, kname, st);
        CPL_CUDA_TRY(df ? launch_plain_df(a, st) : launch_plain(a, st));
        ls.done(flop, bytes);
        if (host_outs) {
            // the blocks (window, slot) this launch wrote, to the host behind it
            CPL_CUDA_TRY(cudaEventRecord(c->copy_ev[ko], st));
            CPL_CUDA_TRY(cudaStreamWaitEvent(c->copy_stream, c->copy_ev[ko], 0));
            for (const Sweep &sw : sweeps) {
                if (vkey(sw.nge, sw.odd) != keys[k]) continue;
                const cpl_request *r = reqs + sw.job;
                const int nspec = spec_count(r->spectra);
                const size_t blk = out_doubles(r) / ((size_t)r->n_windows * nspec);
                for (int w = 0; w < r->n_windows; ++w)
                    for (int q = 0; q < 5; ++q) {
                        if (sw.slot[q] < 0) continue;
                        const size_t off = ((size_t)w * nspec + sw.slot[q]) * blk;
                        CPL_CUDA_TRY(cudaMemcpyAsync(host_outs[sw.job] + off, outs[sw.job] + off, sizeof(double) * blk,
                                                     cudaMemcpyDeviceToHost, c->copy_stream));
                    }
            }
        }
    }
    CPL_CUDA_TRY(cudaEventRecord(c->done, st));
    return CPL_OK;
}

cpl_status build_fp64(cpl_ctx *c, const cpl_request *r, double *out, cudaStream_t st) {
    double *outs[1] = {out};
    return build_fp64_batch(c, r, outs, 1, st);
}

// Lowest index of a non-finite value among n doubles (atomicMin; ~0 if none).
__global__ void k_first_nonfinite(const double *__restrict__ W, long long n, unsigned long long *first) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(W[q]);
        if (((b >> 52) & 0x7ff) == 0x7ff) atomicMin(first, (unsigned long long)q);
    }
}

// cpl_ctx_validate: the windows a request reads must be finite.  Runs before
// any output is written and waits for its answer on `st`.
cpl_status check_windows(cpl_ctx *c, const cpl_request *r, cudaStream_t st) {
    if (!c->validate_w) return CPL_OK;
    cpl_status s;
    if ((s = c->check.ensure(sizeof(unsigned long long), "window check")) != CPL_OK) return s;
    const double *W[3] = {r->W_tt, r->W_tp, r->W_pp};
    const char *names[3] = {"W_tt", "W_tp", "W_pp"};
    const long long n = (long long)r->n_windows * r->w_len;
    for (int q = 0; q < 3; ++q) {
        if (!W[q]) continue;
        bool seen = false;
        for (int p = 0; p < q; ++p) seen |= W[p] == W[q];
        if (seen) continue;
        unsigned long long first = ~0ull;
        CPL_CUDA_TRY(cudaMemcpyAsync(c->check.ptr, &first, sizeof(first), cudaMemcpyHostToDevice, st));
        const int blocks = (int)std::min<long long>((n + 255) / 256, 4096);
        k_first_nonfinite<<<blocks, 256, 0, st>>>(W[q], n, c->check.as<unsigned long long>());
        CPL_CUDA_TRY(cudaGetLastError());
        CPL_CUDA_TRY(cudaMemcpyAsync(&first, c->check.ptr, sizeof(first), cudaMemcpyDeviceToHost, st));
        CPL_CUDA_TRY(cudaStreamSynchronize(st));
        if (first != ~0ull)
            return fail(CPL_ERR_ARG, std::string(names[q]) + " of window " + std::to_string(first / r->w_len) +
                                         " is NaN or Inf at l = " + std::to_string(first % r->w_len));
    }
    return CPL_OK;
}

cpl_status build_one(cpl_ctx *c, const cpl_request *r, double *out, cudaStream_t st) {
    if (r->precision == CPL_MIXED_BF16) return build_mixed(c, r, out, st);
    return build_fp64(c, r, out, st);
}

// Contractions a window-role group's GEMM runs (the separable products of its spectra).
int group_products(unsigned spectra) {
    if (spectra & (kEE | kEEBB | kEB)) return (spectra & (kEEBB | kEB)) ? 9 : 6;
    if (spectra & kTE) return 3;
    return 1;
}

// cpl_build_host for a mixed-precision dense request whose windows form
// several role groups, into page-locked out_host: one build per group
// (a request of the group's spectra and window), most contractions first,
// each into its own region of the output staging buffer; once a group's
// build is done on the GPU its spectrum planes are copied to their places in
// out_host on the copy stream (one strided copy per plane over the windows)
// while the later groups compute.  The caller synchronises st; the copy
// stream is synchronised here.
cpl_status build_mixed_host_split(cpl_ctx *c, const cpl_request *rd, double *out_host, cudaStream_t st) {
    std::vector<Group> groups = window_groups(rd);
    std::stable_sort(groups.begin(), groups.end(), [](const Group &a, const Group &b) {
        return group_products(a.spectra) > group_products(b.spectra);
    });
    if (!c->copy_stream) CPL_CUDA_TRY(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
    while (c->copy_ev.size() < groups.size()) {
        cudaEvent_t e;
        CPL_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        c->copy_ev.push_back(e);
    }
    const size_t plane = (size_t)(rd->lmax - rd->lmin + 1) * (size_t)(rd->lmax - rd->lmin + 1);
    const int nspec = spec_count(rd->spectra);
    const unsigned bits[5] = {kTT, kTE, kEE, kEEBB, kEB};
    double *stage = c->stage_out.as<double>();
    cpl_status s;
    // every group's build is queued (and can fail, e.g. on an allocation)
    // before any copy is: on an error the host buffer stays untouched
    std::vector<size_t> first(groups.size());   // each group's offset in the staging buffer (doubles)
    size_t used = 0;
    for (size_t gi = 0; gi < groups.size(); ++gi) {
        const Group &G = groups[gi];
        cpl_request sub = *rd;
        sub.spectra = G.spectra;
        sub.W_tt = (G.spectra & kTT) ? G.W : nullptr;
        sub.W_tp = (G.spectra & kTE) ? G.W : nullptr;
        sub.W_pp = (G.spectra & (kEE | kEEBB | kEB)) ? G.W : nullptr;
        first[gi] = used;
        if ((s = build_one(c, &sub, stage + used, st)) != CPL_OK) return s;
        CPL_CUDA_TRY(cudaEventRecord(c->copy_ev[gi], st));
        used += (size_t)rd->n_windows * spec_count(G.spectra) * plane;
    }
    // the copies of a group wait for its build only, so they run while the
    // later groups compute
    for (size_t gi = 0; gi < groups.size(); ++gi) {
        const Group &G = groups[gi];
        const int nsub = spec_count(G.spectra);
        const double *dst = stage + first[gi];
        CPL_CUDA_TRY(cudaStreamWaitEvent(c->copy_stream, c->copy_ev[gi], 0));
        for (int b = 0; b < 5; ++b) {
            if (!(G.spectra & bits[b])) continue;
            const int ss = spec_slot(G.spectra, bits[b]), fs = spec_slot(rd->spectra, bits[b]);
            // plane ss of every window of the group's output to plane fs of out_host
            CPL_CUDA_TRY(cudaMemcpy2DAsync(out_host + (size_t)fs * plane, sizeof(double) * plane * nspec,
                                           dst + (size_t)ss * plane, sizeof(double) * plane * nsub,
                                           sizeof(double) * plane, rd->n_windows, cudaMemcpyDeviceToHost,
                                           c->copy_stream));
        }
    }
    const cudaError_t e = cudaStreamSynchronize(c->copy_stream);
    if (e != cudaSuccess) return fail(CPL_ERR_CUDA, std::string("device error: ") + cudaGetErrorString(e));
    return CPL_OK;
}

}  // namespace

extern "C" {

const char *cpl_version(void) { return CPL_VERSION_STRING; }

const char *cpl_last_error(void) { return g_last_error.c_str(); }

cpl_status cpl_ctx_create(cpl_ctx **ctx, int device) {
    if (!ctx) return fail(CPL_ERR_ARG, "ctx is NULL");
    *ctx = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess) {
        cudaGetLastError();
        n = 0;
    }
    if (device < 0 || device >= n) return fail(CPL_ERR_ARG, "no such CUDA device");
    cudaDeviceProp prop;
    CPL_CUDA_TRY(cudaGetDeviceProperties(&prop, device));
    if (prop.major != 10 || prop.minor != 3)
        return fail(CPL_ERR_UNSUPPORTED, std::string("this library is built for sm_103 (GB300); device is ") +
                                             prop.name);
    auto c = new (std::nothrow) cpl_ctx();
    if (!c) return fail(CPL_ERR_OOM, "host allocation failed");
    c->device = device;
    cudaSetDevice(device);
    if (cudaEventCreateWithFlags(&c->done, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return fail(CPL_ERR_CUDA, "could not create the context's stream / event");
    }
    *ctx = c;
    return CPL_OK;
}

cpl_status cpl_ctx_destroy(cpl_ctx *c) {
    if (!c) return CPL_OK;
    if (t_alloc_fault == &c->alloc_fault) t_alloc_fault = nullptr;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    c->g.release();
    c->h.release();
    for (auto &t : c->tile_sets) t->dev.release();
    c->weights.release();
    c->items.release();
    c->ptab_a.release();
    c->ptab_b.release();
    c->pl_coef.release();
    c->stage_w.release();
    c->stage_out.release();
    c->threej_idx.release();
    c->sqrt_tab.release();
    c->mx.plans.clear();
    for (DevBuf *b : {&c->mx.Bimg, &c->mx.eB, &c->mx.emaxB, &c->mx.gdd, &c->mx.arena, &c->mx.ticket, &c->mx.err})
        b->release();
    if (c->mx.cap_stream) cudaStreamDestroy(c->mx.cap_stream);
    for (auto &p : c->pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (auto e : c->ev_pool) cudaEventDestroy(e);
    if (c->done) cudaEventDestroy(c->done);
    if (c->own_stream) cudaStreamDestroy(c->own_stream);
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    for (auto e : c->copy_ev) cudaEventDestroy(e);
    delete c;
    return CPL_OK;
}

cpl_status cpl_ctx_sync(cpl_ctx *c) {
    if (!c) return fail(CPL_ERR_ARG, "ctx is NULL");
    cpl_status s;
    if ((s = select_device(c)) != CPL_OK) return s;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return fail(CPL_ERR_CUDA, std::string("device error: ") + cudaGetErrorString(e));
    if (c->mx.err.ptr) {
        int code = 0;
        e = cudaMemcpy(&code, c->mx.err.ptr, sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return fail(CPL_ERR_CUDA, std::string("device error: ") + cudaGetErrorString(e));
        if (code != 0) {
            cudaMemset(c->mx.err.ptr, 0, sizeof(int));
            if (code == PT_ERR_RANGE)
                return fail(CPL_ERR_CUDA, "internal error: the tabled FP64 kernel found a tile outside its operand "
                                          "tables (code " + std::to_string(code) + ")");
            return fail(CPL_ERR_TIMEOUT, std::string(code == PT_ERR_WAIT ? "a bounded wait of the tabled FP64 kernel ran out"
                                                                         : "a bounded device wait of the tensor-core kernel ran out") +
                                             " (code " + std::to_string(code) + ")");
        }
    }
    return CPL_OK;
}

cpl_status cpl_output_size(const cpl_request *r, size_t *n_doubles) {
    if (!n_doubles) return fail(CPL_ERR_ARG, "n_doubles is NULL");
    cpl_status s = validate(r, true);
    if (s != CPL_OK) return s;
    *n_doubles = out_doubles(r);
    return CPL_OK;
}

cpl_status cpl_plan_info_fp64(const cpl_request *r, cpl_plan_info *info) {
    if (!info) return fail(CPL_ERR_ARG, "info is NULL");
    cpl_status s = validate(r, true);
    if (s != CPL_OK) return s;
    if (r->precision == CPL_MIXED_BF16)
        return fail(CPL_ERR_UNSUPPORTED, "cpl_plan_info_fp64 plans the plain path (CPL_FP64, CPL_DF32)");
    cpl_plan_info pi_;
    std::memset(&pi_, 0, sizeof(pi_));
    std::vector<Tile> tiles;
    make_tiles(r->lmax, r->lmin, tiles);
    pi_.n_tiles = (long long)tiles.size();
    std::vector<int> caps;
    const bool banded = window_caps(r, caps);
    // per window: kept tiles and their even / odd l3 terms (the launch accounting's counts)
    const int nw = r->n_windows;
    std::vector<double> E(nw, 0.0), O(nw, 0.0);
    std::vector<long long> kept(nw, 0);
    for (int w = 0; w < nw; ++w)
        for (const Tile &t : tiles) {
            if (banded && 2 * t.i0 + t.pi > caps[w]) continue;
            double e, od, np;
            tile_terms_split(t, r->lmax, r->lmin, caps[w], &e, &od, &np);
            E[w] += e;
            O[w] += od;
            ++kept[w];
        }
    for (int w = 0; w < nw; ++w) {
        pi_.terms_even += E[w];
        pi_.terms_odd += O[w];
    }
    const unsigned bits[5] = {kTT, kTE, kEE, kEEBB, kEB};
    std::vector<int> variants;
    const int nib = (r->lmax - r->lmin) / 2 / TILE_I + 1;
    for (const Group &G : window_groups(r)) {
        int slot[5];
        for (int x = 0; x < 5; ++x) slot[x] = (G.spectra & bits[x]) ? spec_slot(r->spectra, bits[x]) : -1;
        const int mode = (G.spectra & (kEE | kEEBB | kEB)) ? MODE_POL : (G.spectra & kTE) ? MODE_TE : MODE_TT;
        int nge;
        bool odd;
        plain_variant(mode, slot, &nge, &odd);
        const int key = nge * 2 + (odd ? 1 : 0);
        if (std::find(variants.begin(), variants.end(), key) == variants.end()) variants.push_back(key);
        const int na = (nge == 0 ? 0 : nge == 1 ? 1 : nge == 3 ? 2 : 3) + (odd ? 1 : 0);
        for (int w = 0; w < nw; ++w) {
            pi_.n_items += kept[w];
            pi_.flop += 2.0 * (nge * E[w] + (odd ? 3.0 : 0.0) * O[w]);
            if (r->precision == CPL_FP64)
                for (int p = 0; p < 2; ++p)
                    for (int ib = 0; ib < nib; ++ib)
                        pi_.table_bytes_a += (unsigned long long)a_block_count(r->lmax, r->lmin, p, ib, caps[w]) * na *
                                             PT_BLK * sizeof(double);
        }
    }
    pi_.n_launches = (int)variants.size();
    if (r->precision == CPL_FP64)
        pi_.table_bytes_b =
            (unsigned long long)btab_block(r->lmax / TILE_J + 1, 0, 0) * PT_BROWS * PT_BLK * sizeof(double);
    *info = pi_;
    return CPL_OK;
}

cpl_status cpl_build(cpl_ctx *c, const cpl_request *r, double *out, void *stream) {
    if (!c) return fail(CPL_ERR_ARG, "ctx is NULL");
    if (!out) return fail(CPL_ERR_ARG, "out is NULL");
    cpl_status s = validate(r, true);
    if (s != CPL_OK) return s;
    if ((s = select_device(c)) != CPL_OK) return s;
    if ((s = check_windows(c, r, (cudaStream_t)stream)) != CPL_OK) return s;
    return build_one(c, r, out, (cudaStream_t)stream);
}

cpl_status cpl_build_host(cpl_ctx *c, const cpl_request *r, double *out_host) {
    if (!c) return fail(CPL_ERR_ARG, "ctx is NULL");
    if (!out_host) return fail(CPL_ERR_ARG, "out_host is NULL");
    cpl_status s = validate(r, false);
    if (s != CPL_OK) return s;
    if ((s = select_device(c)) != CPL_OK) return s;
    cudaStream_t st = c->own_stream;
    // stage the distinct windows
    const double *srcs[3] = {r->W_tt, r->W_tp, r->W_pp};
    const double *dsts[3] = {nullptr, nullptr, nullptr};
    const size_t wbytes = sizeof(double) * (size_t)r->n_windows * (size_t)r->w_len;
    if ((s = c->stage_w.ensure(3 * wbytes, "window staging")) != CPL_OK) return s;
    int used = 0;
    for (int q = 0; q < 3; ++q) {
        if (!srcs[q]) continue;
        for (int p = 0; p < q; ++p)
            if (srcs[p] == srcs[q]) dsts[q] = dsts[p];
        if (dsts[q]) continue;
        double *d = reinterpret_cast<double *>(static_cast<char *>(c->stage_w.ptr) + used * wbytes);
        CPL_CUDA_TRY(cudaMemcpyAsync(d, srcs[q], wbytes, cudaMemcpyHostToDevice, st));
        dsts[q] = d;
        ++used;
    }
    const size_t ob = sizeof(double) * out_doubles(r);
    if ((s = c->stage_out.ensure(ob, "output staging")) != CPL_OK) return s;
    cpl_request rd = *r;
    rd.W_tt = dsts[0];
    rd.W_tp = dsts[1];
    rd.W_pp = dsts[2];
    if ((s = check_windows(c, &rd, st)) != CPL_OK) return s;
    cudaError_t e;
    // overlapped copies need page-locked memory (a copy to pageable memory
    // would hold the host until it ends, delaying the later launches)
    cudaPointerAttributes pa;
    bool pinned = cudaPointerGetAttributes(&pa, out_host) == cudaSuccess && pa.type == cudaMemoryTypeHost;
    cudaGetLastError();
    if (rd.precision == CPL_MIXED_BF16 && pinned && !rd.bin_edges && window_groups(&rd).size() > 1) {
        // one build per window-role group, the group with the most contractions
        // first; each group's matrices travel to the host on the copy stream
        // while the later groups compute
        if ((s = build_mixed_host_split(c, &rd, out_host, st)) != CPL_OK) return s;
    } else if (rd.precision == CPL_MIXED_BF16 || !pinned) {
        if ((s = build_one(c, &rd, c->stage_out.as<double>(), st)) != CPL_OK) return s;
        CPL_CUDA_TRY(cudaMemcpyAsync(out_host, c->stage_out.ptr, ob, cudaMemcpyDeviceToHost, st));
    } else {
        // each launch's output blocks travel while the later launches run
        double *douts[1] = {c->stage_out.as<double>()};
        double *houts[1] = {out_host};
        s = build_fp64_batch(c, &rd, douts, 1, st, houts);
        if (c->copy_stream) {
            e = cudaStreamSynchronize(c->copy_stream);
            if (e != cudaSuccess && s == CPL_OK) return fail(CPL_ERR_CUDA, std::string("device error: ") + cudaGetErrorString(e));
        }
        if (s != CPL_OK) return s;
    }
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(CPL_ERR_CUDA, std::string("device error: ") + cudaGetErrorString(e));
    return CPL_OK;
}

cpl_status cpl_build_batch(cpl_ctx *c, const cpl_request *jobs, int n_jobs, double *const *outs,
                           void *stream) {
    if (!c) return fail(CPL_ERR_ARG, "ctx is NULL");
    if (!jobs || !outs || n_jobs < 1) return fail(CPL_ERR_ARG, "jobs / outs must be non-empty");
    cpl_status s;
    for (int q = 0; q < n_jobs; ++q) {
        if ((s = validate(jobs + q, true)) != CPL_OK) return s;
        if (!outs[q]) return fail(CPL_ERR_ARG, "an output pointer is NULL");
        if (jobs[q].precision != jobs[0].precision) return fail(CPL_ERR_ARG, "all jobs must use one precision");
    }
    if ((s = select_device(c)) != CPL_OK) return s;
    for (int q = 0; q < n_jobs; ++q)
        if ((s = check_windows(c, jobs + q, (cudaStream_t)stream)) != CPL_OK) return s;
    if (jobs[0].precision == CPL_MIXED_BF16)
        return cpl::build_mixed_batch(c, jobs, outs, n_jobs, (cudaStream_t)stream, true);
    return build_fp64_batch(c, jobs, outs, n_jobs, (cudaStream_t)stream);
}

cpl_status cpl_threej_m11(cpl_ctx *c, const int *j2, const int *j3, int n, double *out, long long out_stride,
                          void *stream) {
    if (!c) return fail(CPL_ERR_ARG, "ctx is NULL");
    if (n < 0 || (n > 0 && (!j2 || !j3 || !out))) return fail(CPL_ERR_ARG, "j2, j3 and out must be non-NULL");
    if (n == 0) return CPL_OK;
    int smax = 0;
    for (int q = 0; q < n; ++q) {
        if (j2[q] < 1 || j3[q] < 1) return fail(CPL_ERR_ARG, "j2 and j3 must be >= 1 for m = -1, 1");
        if ((long long)j2[q] + j3[q] > CPL_THREEJ_JMAX) return fail(CPL_ERR_RANGE, "j2 + j3 exceeds CPL_THREEJ_JMAX");
        if (out_stride < 2LL * std::min(j2[q], j3[q]) + 1) return fail(CPL_ERR_ARG, "out_stride too small");
        smax = std::max(smax, j2[q] + j3[q]);
    }
    cpl_status s;
    if ((s = select_device(c)) != CPL_OK) return s;
    if ((s = ensure_tables(c, smax + 1)) != CPL_OK) return s;
    // (j2, j3) of the rows, then their constants (16 bytes each)
    if ((s = c->threej_idx.ensure(sizeof(int) * 2 * (size_t)n + 16 * (size_t)n + 16, "3j indices")) != CPL_OK)
        return s;
    cudaStream_t st = (cudaStream_t)stream;
    int *d = c->threej_idx.as<int>();
    CPL_CUDA_TRY(cudaStreamWaitEvent(st, c->done, 0));
    // square roots of the g and h tables (five per entry), once per table size
    const int np1 = c->pmax + 1;
    if (c->sq_pmax != c->pmax) {
        c->sq_pmax = -1;
        if ((s = c->sqrt_tab.ensure(sizeof(float2) * 5 * (size_t)np1, "square-root tables")) != CPL_OK) return s;
        CPL_CUDA_TRY(launch_sqrt_tables(c->g.as<double>(), c->h.as<double>(), np1, c->sqrt_tab.as<float2>(), st));
        c->sq_pmax = c->pmax;
    }
    CPL_CUDA_TRY(cudaMemcpyAsync(d, j2, sizeof(int) * n, cudaMemcpyHostToDevice, st));
    CPL_CUDA_TRY(cudaMemcpyAsync(d + n, j3, sizeof(int) * n, cudaMemcpyHostToDevice, st));
    float4 *cst = reinterpret_cast<float4 *>(c->threej_idx.as<unsigned char>() + ((8 * (size_t)n + 15) & ~(size_t)15));
    {
        LaunchScope ls(c, "threej_consts", st);
        CPL_CUDA_TRY(launch_threej_consts(d, d + n, n, cst, st));
        ls.done(0.0, 24.0 * (double)n);
    }
    {
        LaunchScope ls(c, "threej_m11", st);
        CPL_CUDA_TRY(launch_threej_m11(c->sqrt_tab.as<float2>(), np1, d, d + n, n, cst, out, out_stride, st));
        ls.done(0.0, 8.0 * (double)n * (double)out_stride);
    }
    CPL_CUDA_TRY(cudaEventRecord(c->done, st));
    return CPL_OK;
}

cpl_status cpl_ctx_inject_alloc_failure(cpl_ctx *c, int n) {
    if (!c) return fail(CPL_ERR_ARG, "ctx is NULL");
    if (n < 0) return fail(CPL_ERR_ARG, "n must be >= 0");
    c->alloc_fault = n;
    return CPL_OK;
}

cpl_status cpl_ctx_tune(cpl_ctx *c, int mode, const char *cache_path) {
    if (!c) return fail(CPL_ERR_ARG, "ctx is NULL");
    if (mode != CPL_TUNE_OFF && mode != CPL_TUNE_MEASURE) return fail(CPL_ERR_ARG, "unknown tuning mode");
    return cpl::set_tuning(c, mode, cache_path);
}

cpl_status cpl_ctx_validate(cpl_ctx *c, int enable) {
    if (!c) return fail(CPL_ERR_ARG, "ctx is NULL");
    c->validate_w = enable != 0;
    return CPL_OK;
}

cpl_status cpl_ctx_profile(cpl_ctx *c, int enable) {
    if (!c) return fail(CPL_ERR_ARG, "ctx is NULL");
    c->profiling = enable != 0;
    return CPL_OK;
}

cpl_status cpl_ctx_stats(cpl_ctx *c, cpl_kernel_stat *out, int max, int *n, int reset) {
    if (!c) return fail(CPL_ERR_ARG, "ctx is NULL");
    if (max > 0 && !out) return fail(CPL_ERR_ARG, "out is NULL");
    cpl_status s;
    if ((s = select_device(c)) != CPL_OK) return s;
    for (auto &p : c->pending) {
        cudaError_t e = cudaEventSynchronize(p.b);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, p.a, p.b);
        if (e != cudaSuccess) return fail(CPL_ERR_CUDA, std::string("event timing failed: ") + cudaGetErrorString(e));
        c->kstats[p.idx].ms += ms;
        c->kstats[p.idx].flop += p.flop;
        c->kstats[p.idx].bytes += p.bytes;
        c->kstats[p.idx].issued += p.issued;
        c->ev_pool.push_back(p.a);
        c->ev_pool.push_back(p.b);
    }
    c->pending.clear();
    const int nk = (int)c->kstats.size();
    for (int q = 0; q < nk && q < max; ++q) {
        std::memset(&out[q], 0, sizeof(cpl_kernel_stat));
        std::strncpy(out[q].name, c->kstats[q].name.c_str(), sizeof(out[q].name) - 1);
        out[q].launches = c->kstats[q].launches;
        out[q].ms = c->kstats[q].ms;
        out[q].flop = c->kstats[q].flop;
        out[q].bytes = c->kstats[q].bytes;
        out[q].issued_flop = c->kstats[q].issued;
    }
    if (n) *n = nk;
    if (reset)
        for (auto &k : c->kstats) k.launches = 0, k.ms = k.flop = k.bytes = k.issued = 0.0;
    return CPL_OK;
}

cpl_status cpl_g_table(int pmax, double *out_host) {
    if (pmax < 0 || !out_host) return fail(CPL_ERR_ARG, "pmax must be >= 0 and out_host non-NULL");
    if (pmax > 1 << 24) return fail(CPL_ERR_RANGE, "pmax too large");
    std::vector<double> g, h;
    build_tables_host(pmax, g, h);
    std::memcpy(out_host, g.data(), sizeof(double) * (size_t)(pmax + 1));
    return CPL_OK;
}

cpl_status cpl_h_table(int pmax, double *out_host) {
    if (pmax < 0 || !out_host) return fail(CPL_ERR_ARG, "pmax must be >= 0 and out_host non-NULL");
    if (pmax > 1 << 24) return fail(CPL_ERR_RANGE, "pmax too large");
    std::vector<double> g, h;
    build_tables_host(pmax, g, h);
    std::memcpy(out_host, h.data(), sizeof(double) * (size_t)(pmax + 1));
    return CPL_OK;
}

}  // extern "C"
