// mixed_host.cu -- orchestration of the mixed-precision build (CPL_MIXED_BF16),
// for one request or a batch of them.
//
// A batch is planned once on the host and cached in the context under its
// signature (every field of every request, including pointers and the
// contents of the band-limit and bin-edge arrays).  The plan holds the work
// item list, the per-job tables and the job descriptors in device memory, so
// executing it only launches kernels and clears buffers -- the sequence that
// cpl_build_batch captures once into a CUDA graph and replays.
//
// Execution, per chunk of jobs (jobs are grouped so that their per-job
// scratch fits the scratch budget; a chunk is usually the whole batch):
//   1. per job: FP64 weights per row source (window x role), their
//      double-float copies, and the A-side limb images;
//   2. ONE persistent tcgen05 GEMM over the work items of every job of the
//      chunk, taken with an atomic ticket (mixed_gemm.cu);
//   3. per job: the epilogue (l1 >= MX_L1_FP64) and the FP64 band
//      (l1 < MX_L1_FP64).
// The window-independent B-side images and the double-float lookup tables
// are cached in the context for the largest l_max seen.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cmath>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "ctx.h"
#include "mixed.h"

namespace cpl {

namespace {

struct Source {
    const double *W;
    int win;
    unsigned role;
};

struct Group {
    const double *W;
    unsigned spectra;
};

struct TileRec {
    int pi, rg, b, c, kb_lo, kb_hi;
};

int products_for(unsigned role) {
    if (role & (kEE | kEEBB | kEB)) return (role & (kEEBB | kEB)) ? 9 : 6;
    if (role & kTE) return 3;
    if (role & kTT) return 1;
    return 0;
}

// sum over j in [ja, jb] of max(0, min(j + off, capv))
double sum_clip_min(long long ja, long long jb, long long off, long long capv) {
    if (capv <= 0 || jb < ja) return 0.0;
    double tot = 0.0;
    const long long a0 = std::max(ja, -off + 1), a1 = std::min(jb, capv - off);
    if (a1 >= a0) tot += (double)(a1 - a0 + 1) * (double)((a0 + off) + (a1 + off)) / 2.0;
    const long long b0 = std::max(ja, capv - off + 1);
    if (jb >= b0) tot += (double)(jb - b0 + 1) * (double)capv;
    return tot;
}

// l3 terms (even L, odd L) of the pairs (i, j), j in [ja, jb], of one row i
// with l3 <= cap: even count min(j, kce) - i + 1, odd count min(j - i, kco - i - pi + 1).
void row_terms(int i, int ja, int jb, int pi, int cap, double *even, double *odd) {
    const long long kce = (cap - pi) >> 1, kco = (cap - 1 + pi) >> 1;
    *even += sum_clip_min(ja, jb, -i + 1, kce - i + 1);
    *odd += sum_clip_min(ja, jb, -i, kco - i - pi + 1);
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

// Tunable shape of one job: row sources per tile (0 = built-in choice) and
// the order of its work items (0: by contraction, 1: by tile).
struct MxParams {
    int src = 0;
    int order = 0;
};

// The host-side plan of one request.
struct MxJobPlan {
    cpl_request r;                     // copy; its host arrays are not read after planning
    double *out = nullptr;
    std::vector<Group> groups;
    std::vector<int> group_start;
    std::vector<Source> src;
    int nsrc = 0;
    std::vector<int> src_cap, src_win, src_role;
    MxLayout L;
    int a_stride = 0;
    int alpha_mask = 1;
    std::vector<TileRec> tiles;
    std::vector<int32_t> tile_of;
    std::vector<MxItem> items;         // job-local order (plan_job)
    double kblocks = 0.0;              // sum of item k blocks (cost)
    int nb = 0;
    std::vector<int> bin_of;
    std::vector<double> bin_inv;
    std::vector<double> bin_lw;        // D_l weighting: l(l+1) | 1 / (l(l+1)), or empty
    double gemm_flop = -1.0, gemm_issued = 0.0;   // profiling (flop computed on first use)
    // scratch: offsets relative to the job's base in the arena
    size_t o_A64 = 0, o_Add = 0, o_Aimg = 0, o_eA = 0, o_emaxA = 0, o_inter = 0, scratch_bytes = 0;
    size_t base = 0;                   // the job's base in the arena
    // metadata: offsets into the plan's meta buffer
    size_t m_cap = 0, m_src = 0, m_tile_of = 0, m_bin_of = 0, m_bin_inv = 0, m_bin_lw = 0;
};

struct MxChunk {
    std::vector<int> jobs;             // indices into MxPlan::jobs
    size_t m_items = 0, m_jobs = 0;    // meta offsets of the item list and the MxJob table
    int n_items = 0;
    size_t scratch = 0;
};

// A planned batch.  The device pointers it bakes into its kernel arguments
// (arena, caches, tables) are remembered so that a CUDA graph captured from
// it is re-captured when one of them has moved.
struct MxPlan {
    std::vector<long long> sig;
    int S = 0;
    std::vector<MxJobPlan> jobs;
    std::vector<MxChunk> chunks;
    size_t scratch = 0;                // arena bytes needed (largest chunk)
    DevBuf meta;
    std::vector<const void *> baked;
    cudaGraphExec_t exec = nullptr;
    std::vector<long long> graph_launches;   // kernel launches per replay, by stat index
    unsigned long long last_use = 0;
    ~MxPlan() {
        if (exec) cudaGraphExecDestroy(exec);
        meta.release();
    }
};

namespace {

// Row sources, caps, geometry, tiles and items of one request.
void plan_job(const cpl_request *r, double *out, int S, MxParams prm, MxJobPlan &J) {
    J.r = *r;
    J.out = out;
    const int lmax = r->lmax, lmin = r->lmin, nw = r->n_windows;
    auto add = [&](const double *W, unsigned bits) {
        if (!(r->spectra & bits)) return;
        for (auto &g : J.groups)
            if (g.W == W) {
                g.spectra |= (r->spectra & bits);
                return;
            }
        J.groups.push_back({W, r->spectra & bits});
    };
    add(r->W_tt, kTT);
    add(r->W_tp, kTE);
    add(r->W_pp, kEE | kEEBB | kEB);
    // rows of a GEMM tile: SRC sources x BI i-values, SRC the smallest power
    // of two >= the windows per role (at most 4), so few windows waste no rows
    const int SRC = prm.src ? prm.src : nw >= 3 ? 4 : nw == 2 ? 2 : 1;
    const int BI = MX_ROWS / SRC;
    for (auto &g : J.groups) {
        J.group_start.push_back((int)J.src.size());
        for (int w = 0; w < nw; ++w) J.src.push_back({g.W, w, g.spectra});
        while (J.src.size() % SRC) J.src.push_back({nullptr, -1, 0u});   // pad the row group
    }
    J.nsrc = (int)J.src.size();
    std::vector<int> caps_w(nw);
    for (int w = 0; w < nw; ++w) {
        int cap = std::min(2 * lmax, r->w_len - 1);
        if (r->band_limit) cap = std::min(cap, r->band_limit[w]);
        caps_w[w] = cap;
    }
    J.src_cap.resize(J.nsrc);
    J.src_win.resize(J.nsrc);
    J.src_role.resize(J.nsrc);
    for (int s = 0; s < J.nsrc; ++s) {
        J.src_cap[s] = J.src[s].win >= 0 ? caps_w[J.src[s].win] : -1;
        J.src_win[s] = J.src[s].win;
        J.src_role[s] = (int)J.src[s].role;
    }

    MxLayout &L = J.L;
    std::memset(&L, 0, sizeof(L));
    L.S = S;
    L.SRC = SRC;
    L.BI = BI;
    L.KB = mx_kb(S);
    L.IMG = mx_img_bytes(S);
    L.fA = L.BI / L.KB;
    L.gB = MX_BJ / L.KB;
    L.lmax = lmax;
    L.lmin = lmin;
    L.NB = (lmax - lmin) / 2 / L.BI + 1;
    L.NC = (lmax + 1 + MX_BJ - 1) / MX_BJ;
    L.NKB = lmax / L.KB + 1;
    L.NSB = (L.NKB * L.KB + MX_SB - 1) / MX_SB;
    L.NRG = J.nsrc / L.SRC;
    // A values a(i, k) vanish unless k >= i and l3 = 2k + pi or 2k + 1 - pi <= cap
    int cap_max = 0;
    for (int q = 0; q < J.nsrc; ++q) cap_max = std::max(cap_max, J.src_cap[q]);
    const int kA = cap_max >> 1;
    L.NKBA = std::min(L.NKB, kA / L.KB + 1);
    L.NBA = std::min(L.NB, kA / L.BI + 1);
    L.a_rg_bytes = ((long long)L.NBA * L.NKBA - (long long)L.fA * L.NBA * (L.NBA - 1) / 2) * S * L.IMG;
    J.a_stride = 2 * lmax + 2;

    unsigned role_union = 0;
    for (auto &g : J.groups) role_union |= g.spectra;
    J.alpha_mask = 1;
    if (role_union & (kTE | kEE | kEEBB | kEB)) J.alpha_mask |= 2;
    if (role_union & (kEE | kEEBB | kEB)) J.alpha_mask |= 4;
    if (role_union & (kEEBB | kEB)) J.alpha_mask |= 8;

    // ---- tiles and work items
    const int L1min = std::max(lmin, MX_L1_FP64);
    J.tile_of.assign((size_t)2 * L.NRG * L.NB * L.NC, -1);
    for (int pi = 0; pi < 2; ++pi)
        for (int b = 0; b < L.NB; ++b)
            for (int cb = 0; cb < L.NC; ++cb) {
                const int i0 = b * L.BI;
                const int ja = std::max(cb * MX_BJ, i0 + L1min), jb = std::min(cb * MX_BJ + MX_BJ - 1, lmax - pi - i0);
                if (ja > jb) continue;
                for (int rg = 0; rg < L.NRG; ++rg) {
                    int kcap = -1;
                    for (int q = 0; q < L.SRC; ++q) {
                        const int cap = J.src_cap[rg * L.SRC + q];
                        if (cap < 0) continue;
                        kcap = std::max(kcap, std::max((cap - pi) >> 1, (cap - 1 + pi) >> 1));
                    }
                    const int kb_lo = L.fA * b, kb_hi = std::min(std::min(L.gB * (cb + 1) - 1, L.NKB - 1), kcap / L.KB);
                    if (kcap < i0 || kb_hi < kb_lo) continue;   // the whole tile is zero (band limit)
                    J.tile_of[(((size_t)pi * L.NRG + rg) * L.NB + b) * L.NC + cb] = (int32_t)J.tiles.size();
                    J.tiles.push_back({pi, rg, b, cb, kb_lo, kb_hi});
                }
            }
    // order 0: parity, contraction, row block, column block, row group -- a
    // run of consecutive items shares its A images (same row block) and its
    // B images (same column block) through L2, and the cost of the items of
    // one (parity, contraction) segment falls with the row block, so each
    // segment ends with its lightest items.  order 1: parity, tile, then the
    // contractions of the tile (the same A and B tiles in all their variants).
    auto push = [&](int pi, int p, size_t t) {
        const TileRec &T = J.tiles[t];
        int need = 0;
        for (int q = 0; q < L.SRC; ++q) need = std::max(need, products_for(J.src[T.rg * L.SRC + q].role));
        if (p >= need) return;
        MxItem it;
        it.pi = (int16_t)pi;
        it.p = (int16_t)p;
        it.kb_lo = (int16_t)T.kb_lo;
        it.kb_hi = (int16_t)T.kb_hi;
        it.tile = (int32_t)t;
        it.rg = (int16_t)T.rg;
        it.b = (int16_t)T.b;
        it.c = (int16_t)T.c;
        it.job = 0;
        J.items.push_back(it);
        J.kblocks += (double)(T.kb_hi - T.kb_lo + 1);
    };
    for (int pi = 0; pi < 2; ++pi) {
        if (prm.order == 0) {
            for (int p = 0; p < MX_NPROD; ++p)
                for (size_t t = 0; t < J.tiles.size(); ++t)
                    if (J.tiles[t].pi == pi) push(pi, p, t);
        } else {
            for (size_t t = 0; t < J.tiles.size(); ++t)
                if (J.tiles[t].pi == pi)
                    for (int p = 0; p < MX_NPROD; ++p) push(pi, p, t);
        }
    }
    const double nlp = (double)S * (S + 1) / 2;
    J.gemm_issued = 2.0 * MX_ROWS * MX_BJ * J.kblocks * L.KB * nlp;

    J.nb = r->bin_edges ? r->n_bins : 0;
    if (J.nb) {
        J.bin_of.assign(lmax + 1, -1);
        J.bin_inv.assign(J.nb, 0.0);
        for (int bq = 0; bq < J.nb; ++bq) {
            for (int l = r->bin_edges[bq]; l < r->bin_edges[bq + 1]; ++l) J.bin_of[l] = bq;
            J.bin_inv[bq] = 1.0 / (double)(r->bin_edges[bq + 1] - r->bin_edges[bq]);
        }
        if (r->bin_weight) bin_weights_dl(lmax, J.bin_lw);
    }
    J.r.band_limit = nullptr;          // host arrays are consumed here
    J.r.bin_edges = nullptr;

    // ---- per-job scratch (offsets relative to the job's base in the arena)
    const long long nrows = (long long)L.NRG * L.NB * MX_ROWS;
    size_t o = 0;
    J.o_A64 = o;
    o = align256(o + sizeof(double) * (size_t)J.nsrc * J.a_stride);
    J.o_Add = o;
    o = align256(o + (sizeof(float) * 2 + sizeof(int)) * (size_t)J.nsrc * J.a_stride);
    J.o_Aimg = o;
    o = align256(o + (size_t)2 * MX_NA * L.NRG * L.a_rg_bytes);
    J.o_eA = o;
    o = align256(o + sizeof(int16_t) * 2 * MX_NA * nrows * L.NSB);
    J.o_emaxA = o;
    o = align256(o + sizeof(int16_t) * 2 * MX_NA * nrows);
    J.o_inter = o;
    o = align256(o + sizeof(float) * (size_t)std::max<size_t>(J.tiles.size(), 1) * MX_NPROD * 2 * MX_ROWS * MX_BJ);
    J.scratch_bytes = o;
}

// Algorithmic FLOP of the GEMM items of one job: 2 per (source, l3 term,
// contraction) over the pairs the GEMM serves.
double job_gemm_flop(const MxJobPlan &J) {
    const MxLayout &L = J.L;
    const int L1min = std::max(L.lmin, MX_L1_FP64);
    double flop = 0.0;
    for (const TileRec &t : J.tiles)
        for (int q = 0; q < L.SRC; ++q) {
            const Source &sr = J.src[t.rg * L.SRC + q];
            if (sr.win < 0) continue;
            const int np = products_for(sr.role);
            const int n_even = std::min(np, 6), n_odd = np > 6 ? 3 : 0;
            double e = 0, o = 0;
            for (int di = 0; di < L.BI; ++di) {
                const int i = t.b * L.BI + di;
                const int ja = std::max(t.c * MX_BJ, i + L1min), jb = std::min(t.c * MX_BJ + MX_BJ - 1, L.lmax - t.pi - i);
                if (ja <= jb) row_terms(i, ja, jb, t.pi, J.src_cap[t.rg * L.SRC + q], &e, &o);
            }
            flop += 2.0 * (n_even * e + n_odd * o);
        }
    return flop;
}

void push_sig(std::vector<long long> &sig, const cpl_request *r, const double *out) {
    sig.push_back(r->lmax);
    sig.push_back(r->lmin);
    sig.push_back(r->n_windows);
    sig.push_back((long long)(uintptr_t)r->W_tt);
    sig.push_back((long long)(uintptr_t)r->W_tp);
    sig.push_back((long long)(uintptr_t)r->W_pp);
    sig.push_back(r->w_len);
    sig.push_back((long long)r->spectra);
    sig.push_back((long long)r->precision);
    sig.push_back(r->mixed_slices);
    sig.push_back((long long)(uintptr_t)out);
    sig.push_back(r->band_limit ? 1 : 0);
    if (r->band_limit)
        for (int w = 0; w < r->n_windows; ++w) sig.push_back(r->band_limit[w]);
    const int nb = r->bin_edges ? r->n_bins : 0;
    sig.push_back(nb);
    for (int q = 0; nb && q <= nb; ++q) sig.push_back(r->bin_edges[q]);
    sig.push_back(r->bin_weight);
}

// Scratch budget for one chunk: CPL_MIXED_SCRATCH_GB if set, else 70% of
// what is free plus what the arena already holds.
size_t scratch_budget(const DevBuf &arena) {
    if (const char *e = std::getenv("CPL_MIXED_SCRATCH_GB")) {
        const double gb = std::atof(e);
        if (gb > 0) return (size_t)(gb * 1e9);
    }
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        cudaGetLastError();
        return (size_t)64e9;
    }
    return (size_t)(0.7 * (double)(fr + arena.cap));
}

// Group the jobs (largest first) into chunks whose scratch fits the budget.
void make_chunks(MxPlan &P, size_t budget) {
    std::vector<int> order(P.jobs.size());
    for (size_t q = 0; q < order.size(); ++q) order[q] = (int)q;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return P.jobs[a].kblocks > P.jobs[b].kblocks; });
    P.chunks.clear();
    P.scratch = 0;
    for (int q : order) {
        const size_t need = P.jobs[q].scratch_bytes;
        if (P.chunks.empty() || (P.chunks.back().scratch + need > budget && !P.chunks.back().jobs.empty()))
            P.chunks.push_back(MxChunk{});
        MxChunk &C = P.chunks.back();
        P.jobs[q].base = C.scratch;
        C.jobs.push_back(q);
        C.scratch += need;
        P.scratch = std::max(P.scratch, C.scratch);
    }
}

// Device pointers that the plan's kernel arguments and job tables contain.
std::vector<const void *> baked_ptrs(cpl_ctx *c) {
    const MixedState &M = c->mx;
    return {c->g.ptr, c->h.ptr, M.gdd.ptr, M.Bimg.ptr, M.eB.ptr, M.emaxB.ptr, M.arena.ptr, M.err.ptr, M.ticket.ptr,
            M.coef.ptr};
}

// Write the plan's metadata (per-job tables, item lists, job descriptors
// with the current arena address) to its device buffer.
cpl_status materialize(cpl_ctx *c, MxPlan &P, cudaStream_t st) {
    MixedState &M = c->mx;
    std::vector<uint8_t> host;
    auto put = [&](const void *p, size_t n) {
        const size_t o = host.size();
        host.resize(align256(o + n));
        if (n) std::memcpy(host.data() + o, p, n);
        return o;
    };
    for (MxJobPlan &J : P.jobs) {
        J.m_cap = put(J.src_cap.data(), sizeof(int) * J.nsrc);
        std::vector<int> wr(2 * (size_t)J.nsrc);
        for (int q = 0; q < J.nsrc; ++q) {
            wr[q] = J.src_win[q];
            wr[J.nsrc + q] = J.src_role[q];
        }
        J.m_src = put(wr.data(), sizeof(int) * wr.size());
        J.m_tile_of = put(J.tile_of.data(), sizeof(int32_t) * J.tile_of.size());
        J.m_bin_of = put(J.bin_of.data(), sizeof(int) * J.bin_of.size());
        J.m_bin_inv = put(J.bin_inv.data(), sizeof(double) * J.bin_inv.size());
        J.m_bin_lw = put(J.bin_lw.data(), sizeof(double) * J.bin_lw.size());
    }
    uint8_t *arena = M.arena.as<uint8_t>();
    for (MxChunk &C : P.chunks) {
        std::vector<MxItem> items;
        std::vector<MxJob> jt;
        for (size_t q = 0; q < C.jobs.size(); ++q) {
            const MxJobPlan &J = P.jobs[C.jobs[q]];
            MxJob d;
            d.L = J.L;
            uint8_t *base = arena + J.base;
            d.Aimg = base + J.o_Aimg;
            d.eA = reinterpret_cast<const int16_t *>(base + J.o_eA);
            d.emaxA = reinterpret_cast<const int16_t *>(base + J.o_emaxA);
            d.inter = reinterpret_cast<float *>(base + J.o_inter);
            jt.push_back(d);
            for (MxItem it : J.items) {
                it.job = (int16_t)q;
                items.push_back(it);
            }
        }
        C.n_items = (int)items.size();
        C.m_items = put(items.data(), sizeof(MxItem) * items.size());
        C.m_jobs = put(jt.data(), sizeof(MxJob) * jt.size());
    }
    cpl_status s;
    if ((s = P.meta.ensure(std::max<size_t>(host.size(), 256), "mixed plan metadata")) != CPL_OK) return s;
    CPL_CUDA_TRY(cudaMemcpyAsync(P.meta.ptr, host.data(), host.size(), cudaMemcpyHostToDevice, st));
    if (P.exec) {
        cudaGraphExecDestroy(P.exec);
        P.exec = nullptr;
    }
    return CPL_OK;
}

// The launch sequence of a plan (kernels and memsets only, so that it can be
// captured into a CUDA graph).
cpl_status run_plan(cpl_ctx *c, MxPlan &P, cudaStream_t st) {
    MixedState &M = c->mx;
    const int np1 = c->pmax + 1;
    const float *gh = M.gdd.as<float>(), *gl = gh + np1;
    uint8_t *meta = P.meta.as<uint8_t>();
    uint8_t *arena = M.arena.as<uint8_t>();
    const unsigned bits[5] = {kTT, kTE, kEE, kEEBB, kEB};
    const int S = P.S;
    for (const MxChunk &C : P.chunks) {
        // ---- 1. weights and A-side images, per job
        for (int q : C.jobs) {
            const MxJobPlan &J = P.jobs[q];
            const MxLayout &L = J.L;
            uint8_t *base = arena + J.base;
            double *A64 = reinterpret_cast<double *>(base + J.o_A64);
            const int *cap = reinterpret_cast<const int *>(meta + J.m_cap);
            CPL_CUDA_TRY(cudaMemsetAsync(A64, 0, sizeof(double) * (size_t)J.nsrc * J.a_stride, st));
            for (size_t gi = 0; gi < J.groups.size(); ++gi) {
                const int s0 = J.group_start[gi];
                const int idx = stat_index(c, "mixed_weights");
                cudaEvent_t ev = begin_launch(c, st);
                CPL_CUDA_TRY(launch_weights(J.groups[gi].W, J.r.w_len, J.r.n_windows, cap + s0,
                                            A64 + (size_t)s0 * J.a_stride, J.a_stride, st));
                record_launch(c, idx, ev, st, 0.0, 16.0 * (double)J.a_stride * J.r.n_windows);
            }
            float *Ah = reinterpret_cast<float *>(base + J.o_Add), *Al = Ah + (size_t)J.nsrc * J.a_stride;
            int *Ae = reinterpret_cast<int *>(Al + (size_t)J.nsrc * J.a_stride);
            {
                const int idx = stat_index(c, "mixed_weights_dd");
                cudaEvent_t ev = begin_launch(c, st);
                CPL_CUDA_TRY(mx_launch_weights_dd(A64, J.nsrc, J.a_stride, Ah, Al, Ae, st));
                record_launch(c, idx, ev, st, 0.0, 20.0 * (double)J.nsrc * J.a_stride);
            }
            MxPrepAArgs pa;
            std::memset(&pa, 0, sizeof(pa));
            pa.Ah = Ah;
            pa.Al = Al;
            pa.Ae = Ae;
            pa.a_stride = J.a_stride;
            pa.gh = gh;
            pa.gl = gl;
            pa.l3cap = cap;
            pa.src_role = reinterpret_cast<const int *>(meta + J.m_src) + J.nsrc;
            pa.nsrc = J.nsrc;
            pa.alpha_mask = J.alpha_mask;
            pa.Aimg = base + J.o_Aimg;
            pa.eA = reinterpret_cast<int16_t *>(base + J.o_eA);
            pa.emaxA = reinterpret_cast<int16_t *>(base + J.o_emaxA);
            pa.L = L;
            const int idx = stat_index(c, "mixed_prep_a");
            cudaEvent_t ev = begin_launch(c, st);
            CPL_CUDA_TRY(mx_launch_prep_a(pa, st));
            record_launch(c, idx, ev, st, 0.0, (double)2 * 4 * L.NRG * L.a_rg_bytes);
        }
        // ---- 2. one persistent GEMM over every item of the chunk
        if (C.n_items > 0) {
            MxGemmArgs ga;
            std::memset(&ga, 0, sizeof(ga));
            ga.jobs = reinterpret_cast<const MxJob *>(meta + C.m_jobs);
            ga.Bimg = M.Bimg.as<uint8_t>();
            ga.eB = M.eB.as<int16_t>();
            ga.emaxB = M.emaxB.as<int16_t>();
            ga.items = reinterpret_cast<const MxItem *>(meta + C.m_items);
            ga.n_items = C.n_items;
            ga.ticket = M.ticket.as<int>();
            ga.err = M.err.as<int>();
            double flop = 0.0, issued = 0.0;
            if (c->profiling)
                for (int q : C.jobs) {
                    MxJobPlan &J = P.jobs[q];
                    if (J.gemm_flop < 0) J.gemm_flop = job_gemm_flop(J);
                    flop += J.gemm_flop;
                    issued += J.gemm_issued;
                }
            CPL_CUDA_TRY(cudaMemsetAsync(M.ticket.ptr, 0, sizeof(int), st));
            const int idx = stat_index(c, S == 6 ? "mixed_gemm_s6" : S == 5 ? "mixed_gemm_s5" : "mixed_gemm_s4");
            cudaEvent_t ev = begin_launch(c, st);
            CPL_CUDA_TRY(mx_launch_gemm(ga, S, std::min(C.n_items, M.nsm), st));
            record_launch(c, idx, ev, st, flop, 0.0, issued);
        }
        // ---- 3. epilogue and FP64 band, per job
        for (int q : C.jobs) {
            const MxJobPlan &J = P.jobs[q];
            uint8_t *base = arena + J.base;
            const int nspec = spec_count(J.r.spectra);
            const int *srcp = reinterpret_cast<const int *>(meta + J.m_src);
            if (J.nb) {
                const size_t n_out = (size_t)J.r.n_windows * nspec * J.nb * J.nb;
                CPL_CUDA_TRY(cudaMemsetAsync(J.out, 0, sizeof(double) * n_out, st));
            } else if (J.L.NBA < J.L.NB) {
                // band-limited dense output: pairs beyond the band are zero and the
                // epilogue covers only the row blocks that hold nonzero values
                const size_t n = (size_t)(J.r.lmax - J.r.lmin + 1);
                CPL_CUDA_TRY(cudaMemsetAsync(J.out, 0, sizeof(double) * J.r.n_windows * nspec * n * n, st));
            }
            MxEpiArgs ea;
            std::memset(&ea, 0, sizeof(ea));
            ea.inter = reinterpret_cast<const float *>(base + J.o_inter);
            ea.tile_of = reinterpret_cast<const int32_t *>(meta + J.m_tile_of);
            ea.emaxA = reinterpret_cast<const int16_t *>(base + J.o_emaxA);
            ea.emaxB = M.emaxB.as<int16_t>();
            ea.src_win = srcp;
            ea.src_role = srcp + J.nsrc;
            ea.l3cap = reinterpret_cast<const int *>(meta + J.m_cap);
            ea.nsrc = J.nsrc;
            ea.lmax = J.r.lmax;
            ea.lmin = J.r.lmin;
            ea.out = J.out;
            ea.nspec = nspec;
            for (int x = 0; x < 5; ++x) ea.slot[x] = spec_slot(J.r.spectra, bits[x]);
            ea.n_bins = J.nb;
            ea.bin_of = J.nb ? reinterpret_cast<const int *>(meta + J.m_bin_of) : nullptr;
            ea.bin_inv = J.nb ? reinterpret_cast<const double *>(meta + J.m_bin_inv) : nullptr;
            ea.bin_lw = J.bin_lw.empty() ? nullptr : reinterpret_cast<const double *>(meta + J.m_bin_lw);
            ea.coef = M.coef.ptr;
            ea.L = J.L;
            {
                const int idx = stat_index(c, "mixed_epilogue");
                cudaEvent_t ev = begin_launch(c, st);
                CPL_CUDA_TRY(mx_launch_epilogue(ea, st));
                record_launch(c, idx, ev, st, 0.0, 0.0);
            }
            MxBandArgs ba;
            std::memset(&ba, 0, sizeof(ba));
            {
                const int np1 = c->pmax + 1;
                const float *gd = M.gdd.as<float>();
                ba.gh = gd;
                ba.gl = gd + np1;
                ba.hh = gd + 2 * np1;
                ba.hl = gd + 3 * np1;
                ba.Ah = reinterpret_cast<const float *>(base + J.o_Add);
                ba.Al = ba.Ah + (size_t)J.nsrc * J.a_stride;
                ba.Ae = reinterpret_cast<const int *>(ba.Al + (size_t)J.nsrc * J.a_stride);
            }
            ba.a_stride = J.a_stride;
            ba.l3cap = reinterpret_cast<const int *>(meta + J.m_cap);
            ba.src_win = srcp;
            ba.src_role = srcp + J.nsrc;
            ba.nsrc = J.nsrc;
            ba.lmax = J.r.lmax;
            ba.lmin = J.r.lmin;
            ba.out = J.out;
            ba.nspec = nspec;
            for (int x = 0; x < 5; ++x) ba.slot[x] = spec_slot(J.r.spectra, bits[x]);
            ba.n_bins = J.nb;
            ba.bin_of = ea.bin_of;
            ba.bin_inv = ea.bin_inv;
            ba.bin_lw = ea.bin_lw;
            if (J.r.lmin < MX_L1_FP64) {
                const int idx = stat_index(c, "mixed_band");
                cudaEvent_t ev = begin_launch(c, st);
                CPL_CUDA_TRY(mx_launch_band(ba, st));
                record_launch(c, idx, ev, st, 0.0, 0.0);
            }
        }
    }
    return CPL_OK;
}

}  // namespace

void MxPlanDeleter::operator()(MxPlan *p) const { delete p; }

void mx_coef_host(int n, std::vector<uint32_t> &out) {
    out.assign((size_t)n * MX_COEF_N * 3, 0u);
    auto put = [&](size_t at, double x) {   // x = m 2^e with 1 <= |m| < 2, m as an FP32 pair
        if (x == 0.0) return;
        int k;
        const double f = std::frexp(x, &k);   // x = f 2^k, 0.5 <= |f| < 1
        const double m = 2.0 * f;
        const float h = (float)m, l = (float)(m - (double)h);
        std::memcpy(&out[3 * at], &h, 4);
        std::memcpy(&out[3 * at + 1], &l, 4);
        const int e = k - 1;
        std::memcpy(&out[3 * at + 2], &e, 4);
    };
    for (int l = 2; l < n; ++l) {
        const double L = l;
        // l1 factors: rho = sqrt(l(l+1) / ((l-1)(l+2))) (lambda/eta = rho(l1) sigma(l2)),
        // c0 = (l+2)/l, alpha = 1/(l(l+1)) (c1 = alpha beta), kappa = alpha / ((l-1)(l+2))
        const double rho2 = L * (L + 1.0) / ((L - 1.0) * (L + 2.0)), rho = std::sqrt(rho2);
        const double c0 = (L + 2.0) / L, al = 1.0 / (L * (L + 1.0)), ka = al / ((L - 1.0) * (L + 2.0));
        const double A[MX_COEF_A] = {rho * c0, rho * al, rho2 * c0 * c0, 2.0 * rho2 * c0 * al, rho2 * al * al,
                                     2.0 * rho2 * al * al, ka * (L + 2.0) * (L + 2.0), ka * (L + 2.0), ka};
        // l2 factors: sigma = sqrt((l+1)(l+2) / ((l-1) l)), beta = 1/(l+1),
        // beta' = 1/(2(l+1)(l+2)) (c2 = alpha beta'), mu = (l+2)/((l+1)(l-1) l) (C = kappa mu)
        const double s2 = (L + 1.0) * (L + 2.0) / ((L - 1.0) * L), s = std::sqrt(s2);
        const double be = 1.0 / (L + 1.0), bp = 1.0 / (2.0 * (L + 1.0) * (L + 2.0));
        const double mu = (L + 2.0) / ((L + 1.0) * (L - 1.0) * L);
        const double B[MX_COEF_B] = {s, s * be, s * bp, s2, s2 * be, s2 * bp, s2 * be * be, s2 * be * bp, s2 * bp * bp,
                                     mu, mu / (L + 2.0), mu / (4.0 * (L + 2.0) * (L + 2.0))};
        for (int q = 0; q < MX_COEF_A; ++q) put((size_t)l * MX_COEF_N + q, A[q]);
        for (int q = 0; q < MX_COEF_B; ++q) put((size_t)l * MX_COEF_N + MX_COEF_A + q, B[q]);
    }
}

// Shared state every plan relies on: lookup tables, their double-float
// copies, the B-side image cache, the arena, the ticket and the error word.
static cpl_status ensure_common(cpl_ctx *c, int S, int nc_max, size_t scratch, cudaStream_t st) {
    MixedState &M = c->mx;
    cpl_status s;
    if (M.nsm == 0) {
        int nsm = 0;
        CPL_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device));
        M.nsm = std::max(1, nsm);
    }
    if (M.S != S || M.NC_B < nc_max) {
        M.NC_B = M.S == S ? std::max(M.NC_B, nc_max) : nc_max;
        M.S = S;
        M.Bimg.release();   // rebuilt below
    }
    // tables must cover j + k + 1 for j, k < NC_B * 128 (the B cache)
    if ((s = ensure_tables(c, M.NC_B * MX_BJ + 64)) != CPL_OK) return s;
    const int np1 = c->pmax + 1;
    if (M.pmax_dd != c->pmax) {
        if ((s = M.gdd.ensure(sizeof(float) * 4 * (size_t)np1, "double-float tables")) != CPL_OK) return s;
        float *gd = M.gdd.as<float>();
        const int idx = stat_index(c, "mixed_tables_dd");
        cudaEvent_t ev = begin_launch(c, st);
        CPL_CUDA_TRY(mx_launch_tables_dd(c->g.as<double>(), c->h.as<double>(), np1, gd, gd + np1, gd + 2 * np1,
                                         gd + 3 * np1, st));
        record_launch(c, idx, ev, st, 0.0, 48.0 * np1);
        M.pmax_dd = c->pmax;
        M.Bimg.release();   // the B cache is rebuilt with the new tables
    }
    // pair-coefficient factors for every l the B cache can reach
    if (M.coef_n < M.NC_B * MX_BJ + 2) {
        const int n = M.NC_B * MX_BJ + 2;
        M.coef_n = 0;
        if ((s = M.coef.ensure(sizeof(uint32_t) * 3 * (size_t)n * MX_COEF_N, "pair coefficient factors")) != CPL_OK)
            return s;
        std::vector<uint32_t> host;
        mx_coef_host(n, host);
        CPL_CUDA_TRY(cudaMemcpyAsync(M.coef.ptr, host.data(), sizeof(uint32_t) * host.size(), cudaMemcpyHostToDevice, st));
        M.coef_n = n;
    }
    if (!M.Bimg.ptr) {
        MxLayout L;
        std::memset(&L, 0, sizeof(L));
        L.S = S;
        L.KB = mx_kb(S);
        L.IMG = mx_img_bytes(S);
        L.gB = MX_BJ / L.KB;
        L.NC_B = M.NC_B;
        L.NSB_B = M.NC_B;
        L.b_var_bytes = (long long)L.gB * L.NC_B * (L.NC_B + 1) / 2 * S * L.IMG;
        const long long ncols_B = (long long)L.NC_B * MX_BJ;
        // the cache counts as built only when all three buffers exist (Bimg set)
        if ((s = M.eB.ensure(sizeof(int16_t) * 2 * MX_NBV * ncols_B * L.NSB_B, "mixed B exponents")) != CPL_OK)
            return s;
        if ((s = M.emaxB.ensure(sizeof(int16_t) * 2 * MX_NBV * ncols_B, "mixed B maxima")) != CPL_OK) return s;
        if ((s = M.Bimg.ensure((size_t)2 * MX_NBV * L.b_var_bytes, "mixed B images")) != CPL_OK) return s;
        const float *gh = M.gdd.as<float>();
        MxPrepBArgs pb;
        std::memset(&pb, 0, sizeof(pb));
        pb.gh = gh;
        pb.gl = gh + np1;
        pb.hh = gh + 2 * np1;
        pb.hl = gh + 3 * np1;
        pb.Bimg = M.Bimg.as<uint8_t>();
        pb.eB = M.eB.as<int16_t>();
        pb.emaxB = M.emaxB.as<int16_t>();
        pb.c_lo = 0;
        pb.L = L;
        const int idx = stat_index(c, "mixed_prep_b");
        cudaEvent_t ev = begin_launch(c, st);
        const cudaError_t le = mx_launch_prep_b(pb, L.NC_B, st);
        if (le != cudaSuccess) {
            M.Bimg.release();
            return fail(CPL_ERR_CUDA, std::string("mx_launch_prep_b failed: ") + cudaGetErrorString(le));
        }
        record_launch(c, idx, ev, st, 0.0, (double)2 * MX_NBV * L.b_var_bytes);
    }
    if ((s = M.arena.ensure(std::max<size_t>(scratch, 256), "mixed scratch arena")) != CPL_OK) return s;
    if ((s = ensure_err_word(c, st)) != CPL_OK) return s;
    if ((s = M.ticket.ensure(sizeof(int), "mixed ticket")) != CPL_OK) return s;
    CPL_CUDA_TRY(mx_gemm_prepare(S));
    return CPL_OK;
}

// Make the shared state fit the plan and (re)write its metadata if a device
// pointer or the B-cache geometry it depends on has changed.
static cpl_status prepare_plan(cpl_ctx *c, MxPlan &P, cudaStream_t st) {
    MixedState &M = c->mx;
    cpl_status s;
    int nc_max = 0;
    for (const MxJobPlan &J : P.jobs) nc_max = std::max(nc_max, J.L.NC);
    if ((s = ensure_common(c, P.S, nc_max, P.scratch, st)) != CPL_OK) return s;
    std::vector<const void *> baked = baked_ptrs(c);
    baked.push_back(reinterpret_cast<const void *>((uintptr_t)M.NC_B));
    baked.push_back(reinterpret_cast<const void *>((uintptr_t)c->pmax));
    if (baked != P.baked) {
        for (MxJobPlan &J : P.jobs) {   // the B geometry of every job follows the (possibly grown) cache
            J.L.NC_B = M.NC_B;
            J.L.NSB_B = M.NC_B;
            J.L.b_var_bytes = (long long)J.L.gB * M.NC_B * (M.NC_B + 1) / 2 * P.S * J.L.IMG;
        }
        if ((s = materialize(c, P, st)) != CPL_OK) return s;
        P.baked = baked;
    }
    return CPL_OK;
}

namespace {

// Shape of a request as the tuner sees it: everything that changes the
// work items or their costs, but no pointer values.
std::vector<long long> tune_key(const cpl_request *r, int S) {
    std::vector<long long> k = {S, r->lmax, r->lmin, r->n_windows, (long long)r->spectra,
                                r->bin_edges ? r->n_bins : 0};
    const double *W[3] = {r->W_tt, r->W_tp, r->W_pp};
    const unsigned bits[3] = {kTT, kTE, kEE | kEEBB | kEB};
    int shared = 0;   // which requested roles share one window pointer
    for (int a = 0; a < 3; ++a)
        for (int b = a + 1; b < 3; ++b)
            shared = 2 * shared + ((r->spectra & bits[a]) && (r->spectra & bits[b]) && W[a] == W[b] ? 1 : 0);
    k.push_back(shared);
    for (int w = 0; w < r->n_windows; ++w) {
        int cap = std::min(2 * r->lmax, r->w_len - 1);
        if (r->band_limit) cap = std::min(cap, r->band_limit[w]);
        k.push_back(cap);
    }
    return k;
}

void append_tune_file(const std::string &path, const TuneEntry &e) {
    if (path.empty()) return;
    FILE *f = std::fopen(path.c_str(), "a");
    if (!f) return;
    std::fprintf(f, "{\"key\": [");
    for (size_t q = 0; q < e.key.size(); ++q) std::fprintf(f, "%s%lld", q ? ", " : "", e.key[q]);
    std::fprintf(f, "], \"src\": %d, \"order\": %d, \"ms\": %.4f}\n", e.src, e.order, e.ms);
    std::fclose(f);
}

bool parse_tune_line(const std::string &ln, TuneEntry &e) {
    const size_t k0 = ln.find("\"key\""), b0 = ln.find('[', k0 == std::string::npos ? 0 : k0);
    const size_t b1 = ln.find(']', b0 == std::string::npos ? 0 : b0);
    const size_t s0 = ln.find("\"src\""), o0 = ln.find("\"order\""), m0 = ln.find("\"ms\"");
    if (k0 == std::string::npos || b0 == std::string::npos || b1 == std::string::npos || s0 == std::string::npos ||
        o0 == std::string::npos)
        return false;
    e.key.clear();
    const char *p = ln.c_str() + b0 + 1, *end = ln.c_str() + b1;
    while (p < end) {
        char *q = nullptr;
        const long long v = std::strtoll(p, &q, 10);
        if (q == p) {
            ++p;
            continue;
        }
        e.key.push_back(v);
        p = q;
    }
    e.src = std::atoi(ln.c_str() + ln.find(':', s0) + 1);
    e.order = std::atoi(ln.c_str() + ln.find(':', o0) + 1);
    e.ms = m0 == std::string::npos ? 0.0 : std::atof(ln.c_str() + ln.find(':', m0) + 1);
    return !e.key.empty() && (e.src == 1 || e.src == 2 || e.src == 4) && (e.order == 0 || e.order == 1);
}

// The tuned parameters of one request: from the cache, or measured now by
// running every candidate's full launch sequence on the request's own
// buffers (all candidates compute identical results).
cpl_status tune_job(cpl_ctx *c, const cpl_request *r, double *out, int S, cudaStream_t st, MxParams *best) {
    MixedState &M = c->mx;
    *best = MxParams{};
    if (M.tune_mode != CPL_TUNE_MEASURE) return CPL_OK;
    const std::vector<long long> key = tune_key(r, S);
    for (const TuneEntry &e : M.tuned)
        if (e.key == key) {
            best->src = e.src;
            best->order = e.order;
            return CPL_OK;
        }
    std::vector<MxParams> cand;
    for (int src : {1, 2, 4})
        if (src < 2 * std::max(1, r->n_windows))
            for (int order : {0, 1}) cand.push_back(MxParams{src, order});
    // tuning runs are not part of the caller's accounting
    const bool prof = c->profiling;
    c->profiling = false;
    std::vector<long long> launches(c->kstats.size());
    for (size_t q = 0; q < launches.size(); ++q) launches[q] = c->kstats[q].launches;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cpl_status s = CPL_OK;
    double best_ms = 1e300;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        s = fail(CPL_ERR_CUDA, "event creation failed");
    }
    for (size_t q = 0; q < cand.size() && s == CPL_OK; ++q) {
        MxPlan P;
        P.S = S;
        P.jobs.resize(1);
        plan_job(r, out, S, cand[q], P.jobs[0]);
        make_chunks(P, scratch_budget(M.arena));
        if ((s = prepare_plan(c, P, st)) != CPL_OK) break;
        float ms = 0.f;
        for (int rep = 0; rep < 2 && s == CPL_OK; ++rep) {
            if (cudaEventRecord(e0, st) != cudaSuccess) s = fail(CPL_ERR_CUDA, "event record failed");
            if (s == CPL_OK) s = run_plan(c, P, st);
            if (s == CPL_OK && (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
                s = fail(CPL_ERR_CUDA, std::string("tuning run failed: ") + cudaGetErrorString(cudaGetLastError()));
        }
        if (s == CPL_OK && ms < best_ms) {
            best_ms = ms;
            *best = cand[q];
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    c->profiling = prof;
    for (size_t q = 0; q < c->kstats.size(); ++q) c->kstats[q].launches = q < launches.size() ? launches[q] : 0;
    if (s != CPL_OK) return s;
    TuneEntry e;
    e.key = key;
    e.src = best->src;
    e.order = best->order;
    e.ms = best_ms;
    M.tuned.push_back(e);
    append_tune_file(M.tune_path, e);
    return CPL_OK;
}

}  // namespace

cpl_status set_tuning(cpl_ctx *c, int mode, const char *path) {
    MixedState &M = c->mx;
    M.tune_mode = mode;
    M.tune_path = path ? path : "";
    if (!M.tune_path.empty()) {
        FILE *f = std::fopen(M.tune_path.c_str(), "r");
        if (f) {
            char buf[1 << 16];
            while (std::fgets(buf, sizeof(buf), f)) {
                TuneEntry e;
                if (!parse_tune_line(buf, e)) continue;
                bool dup = false;
                for (TuneEntry &o : M.tuned)
                    if (o.key == e.key) {
                        o = e;
                        dup = true;
                    }
                if (!dup) M.tuned.push_back(e);
            }
            std::fclose(f);
        }
    }
    return CPL_OK;
}

// Build a batch of mixed-precision requests on `st`.  With use_graph (and
// profiling off) the launch sequence is captured once per plan into a CUDA
// graph and replayed.
cpl_status build_mixed_batch(cpl_ctx *c, const cpl_request *reqs, double *const *outs, int n, cudaStream_t st,
                             bool use_graph) {
    MixedState &M = c->mx;
    const int S = reqs[0].mixed_slices ? reqs[0].mixed_slices : 6;
    if (S < 4 || S > 6) return fail(CPL_ERR_UNSUPPORTED, "the mixed path supports mixed_slices 4..6 (0 = 6)");
    for (int q = 1; q < n; ++q)
        if ((reqs[q].mixed_slices ? reqs[q].mixed_slices : 6) != S)
            return fail(CPL_ERR_ARG, "all jobs of a mixed batch must use the same mixed_slices");

    std::vector<long long> sig;
    sig.push_back(n);
    for (int q = 0; q < n; ++q) push_sig(sig, reqs + q, outs[q]);
    MxPlan *P = nullptr;
    for (auto &p : M.plans)
        if (p->sig == sig) P = p.get();
    if (!P) {
        if (M.plans.size() >= 8) {   // evict the least recently used plan
            auto it = std::min_element(M.plans.begin(), M.plans.end(),
                                       [](const auto &a, const auto &b) { return a->last_use < b->last_use; });
            CPL_CUDA_TRY(cudaEventSynchronize(c->done));
            M.plans.erase(it);
        }
        std::unique_ptr<MxPlan, MxPlanDeleter> np(new MxPlan);
        np->sig = sig;
        np->S = S;
        np->jobs.resize(n);
        cpl_status ts;
        for (int q = 0; q < n; ++q) {
            MxParams prm;
            CPL_CUDA_TRY(cudaStreamWaitEvent(st, c->done, 0));
            if ((ts = tune_job(c, reqs + q, outs[q], S, st, &prm)) != CPL_OK) return ts;
            plan_job(reqs + q, outs[q], S, prm, np->jobs[q]);
        }
        make_chunks(*np, scratch_budget(M.arena));
        P = np.get();
        M.plans.push_back(std::move(np));
    }
    P->last_use = ++M.clock;

    cpl_status s;
    CPL_CUDA_TRY(cudaStreamWaitEvent(st, c->done, 0));
    if ((s = prepare_plan(c, *P, st)) != CPL_OK) return s;

    if (use_graph && !c->profiling) {
        if (!P->exec) {
            if (!M.cap_stream) CPL_CUDA_TRY(cudaStreamCreateWithFlags(&M.cap_stream, cudaStreamNonBlocking));
            std::vector<long long> before(c->kstats.size());
            for (size_t q = 0; q < before.size(); ++q) before[q] = c->kstats[q].launches;
            CPL_CUDA_TRY(cudaStreamBeginCapture(M.cap_stream, cudaStreamCaptureModeThreadLocal));
            const cpl_status rs = run_plan(c, *P, M.cap_stream);
            cudaGraph_t g = nullptr;
            const cudaError_t ce = cudaStreamEndCapture(M.cap_stream, &g);
            // the capture ran nothing: take its launch counts back, keep them per replay
            P->graph_launches.assign(c->kstats.size(), 0);
            for (size_t q = 0; q < c->kstats.size(); ++q) {
                const long long b0 = q < before.size() ? before[q] : 0;
                P->graph_launches[q] = c->kstats[q].launches - b0;
                c->kstats[q].launches = b0;
            }
            if (rs != CPL_OK) {
                if (g) cudaGraphDestroy(g);
                return rs;
            }
            if (ce != cudaSuccess) {
                cudaGetLastError();
                return fail(CPL_ERR_CUDA, std::string("graph capture failed: ") + cudaGetErrorString(ce));
            }
            const cudaError_t ie = cudaGraphInstantiate(&P->exec, g, 0);
            cudaGraphDestroy(g);
            if (ie != cudaSuccess) {
                P->exec = nullptr;
                cudaGetLastError();
                return fail(CPL_ERR_CUDA, std::string("graph instantiation failed: ") + cudaGetErrorString(ie));
            }
        }
        CPL_CUDA_TRY(cudaGraphLaunch(P->exec, st));
        for (size_t q = 0; q < P->graph_launches.size() && q < c->kstats.size(); ++q)
            c->kstats[q].launches += P->graph_launches[q];
    } else {
        if ((s = run_plan(c, *P, st)) != CPL_OK) return s;
    }
    CPL_CUDA_TRY(cudaEventRecord(c->done, st));
    return CPL_OK;
}

cpl_status build_mixed(cpl_ctx *c, const cpl_request *r, double *out, cudaStream_t st) {
    double *outs[1] = {out};
    return build_mixed_batch(c, r, outs, 1, st, false);
}

}  // namespace cpl
