// mixed_host.cu -- orchestration of the mixed-precision build (CPL_MIXED_BF16).
//
// Sequence on the caller's stream:
//   1. FP64 weights per row source (window x role), then their double-float
//      copies; the lookup tables as double-float (cached).
//   2. B-side limb images (window-independent, cached in the context and
//      grown with l_max), A-side limb images of this request.
//   3. The tcgen05 limb GEMM over all work items (parity, contraction,
//      row group, i-block, j-block), ordered so that concurrently running
//      CTAs share their A and B images through L2.
//   4. The epilogue (l1 >= MX_L1_FP64) and the FP64 band (l1 < MX_L1_FP64).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
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

}  // namespace

cpl_status build_mixed(cpl_ctx *c, const cpl_request *r, double *out, cudaStream_t st) {
    MixedState &M = c->mx;
    const int S = r->mixed_slices ? r->mixed_slices : 6;
    if (S < 4 || S > 6) return fail(CPL_ERR_UNSUPPORTED, "the mixed path supports mixed_slices 4..6 (0 = 6)");
    const int lmax = r->lmax, lmin = r->lmin, nw = r->n_windows;
    CPL_CUDA_TRY(cudaStreamWaitEvent(st, c->done, 0));

    // ---- row sources: window roles sharing a pointer share one sweep
    struct Group {
        const double *W;
        unsigned spectra;
    };
    std::vector<Group> groups;
    auto add = [&](const double *W, unsigned bits) {
        if (!(r->spectra & bits)) return;
        for (auto &g : groups)
            if (g.W == W) {
                g.spectra |= (r->spectra & bits);
                return;
            }
        groups.push_back({W, r->spectra & bits});
    };
    add(r->W_tt, kTT);
    add(r->W_tp, kTE);
    add(r->W_pp, kEE | kEEBB | kEB);
    // rows of a GEMM tile: SRC sources x BI i-values, SRC the smallest power
    // of two >= the windows per role (at most 4), so few windows waste no rows
    const int SRC = nw >= 3 ? 4 : nw == 2 ? 2 : 1;
    const int BI = MX_ROWS / SRC;
    std::vector<Source> src;
    std::vector<int> group_start;
    for (auto &g : groups) {
        group_start.push_back((int)src.size());
        for (int w = 0; w < nw; ++w) src.push_back({g.W, w, g.spectra});
        while (src.size() % SRC) src.push_back({nullptr, -1, 0u});   // pad the row group
    }
    const int nsrc = (int)src.size();

    std::vector<int> caps_w(nw);
    for (int w = 0; w < nw; ++w) {
        int cap = std::min(2 * lmax, r->w_len - 1);
        if (r->band_limit) cap = std::min(cap, r->band_limit[w]);
        caps_w[w] = cap;
    }
    std::vector<int> src_cap(nsrc), src_win(nsrc), src_role(nsrc);
    for (int s = 0; s < nsrc; ++s) {
        src_cap[s] = src[s].win >= 0 ? caps_w[src[s].win] : -1;
        src_win[s] = src[s].win;
        src_role[s] = (int)src[s].role;
    }

    // ---- geometry
    MxLayout L;
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
    L.NSB = (L.NKB + 3) / 4;
    L.NRG = nsrc / L.SRC;
    L.a_rg_bytes = ((long long)L.NB * L.NKB - (long long)L.fA * L.NB * (L.NB - 1) / 2) * S * L.IMG;
    if (M.S != S || M.NC_B < L.NC) {
        M.S = S;
        M.NC_B = std::max(L.NC, M.NC_B);
        M.NC_B = std::max(M.NC_B, L.NC);
        M.Bimg.release();   // rebuilt below
    }
    L.NC_B = M.NC_B;
    L.NSB_B = M.NC_B;
    L.b_var_bytes = (long long)L.gB * L.NC_B * (L.NC_B + 1) / 2 * S * L.IMG;

    cpl_status s;
    // tables must cover j + k + 1 for j, k < NC_B * 128 (the B cache)
    if ((s = ensure_tables(c, L.NC_B * MX_BJ + 64)) != CPL_OK) return s;
    const int np1 = c->pmax + 1;
    if (M.pmax_dd != c->pmax) {
        if ((s = M.gdd.ensure(sizeof(float) * 4 * (size_t)np1, "double-float tables")) != CPL_OK) return s;
        float *gd = M.gdd.as<float>();
        CPL_CUDA_TRY(mx_launch_tables_dd(c->g.as<double>(), c->h.as<double>(), np1, gd, gd + np1, gd + 2 * np1,
                                         gd + 3 * np1, st));
        M.pmax_dd = c->pmax;
        M.Bimg.release();   // the B cache is rebuilt with the new tables
    }
    const float *gh = M.gdd.as<float>(), *gl = gh + np1, *hh = gh + 2 * np1, *hl = gh + 3 * np1;

    const long long ncols_B = (long long)L.NC_B * MX_BJ;
    if (!M.Bimg.ptr) {
        if ((s = M.Bimg.ensure((size_t)2 * MX_NBV * L.b_var_bytes, "mixed B images")) != CPL_OK) return s;
        if ((s = M.eB.ensure(sizeof(int16_t) * 2 * MX_NBV * ncols_B * L.NSB_B, "mixed B exponents")) != CPL_OK)
            return s;
        if ((s = M.emaxB.ensure(sizeof(int16_t) * 2 * MX_NBV * ncols_B, "mixed B maxima")) != CPL_OK) return s;
        MxPrepBArgs pb;
        std::memset(&pb, 0, sizeof(pb));
        pb.gh = gh;
        pb.gl = gl;
        pb.hh = hh;
        pb.hl = hl;
        pb.Bimg = M.Bimg.as<uint8_t>();
        pb.eB = M.eB.as<int16_t>();
        pb.emaxB = M.emaxB.as<int16_t>();
        pb.c_lo = 0;
        pb.L = L;
        const int idx = stat_index(c, "mixed_prep_b");
        cudaEvent_t ev = begin_launch(c, st);
        CPL_CUDA_TRY(mx_launch_prep_b(pb, L.NC_B, st));
        record_launch(c, idx, ev, st, 0.0, (double)2 * MX_NBV * L.b_var_bytes);
    }

    // ---- per-source weights: FP64 (band kernel) and double-float mantissa / exponent
    const int a_stride = 2 * lmax + 2;
    if ((s = M.A64.ensure(sizeof(double) * (size_t)nsrc * a_stride, "mixed weights")) != CPL_OK) return s;
    if ((s = M.Add.ensure((sizeof(float) * 2 + sizeof(int)) * (size_t)nsrc * a_stride, "mixed weights dd")) != CPL_OK)
        return s;
    if ((s = M.l3cap.ensure(sizeof(int) * (size_t)nsrc, "mixed caps")) != CPL_OK) return s;
    if ((s = M.src.ensure(sizeof(int) * 2 * (size_t)nsrc, "mixed sources")) != CPL_OK) return s;
    if ((s = M.err.ensure(sizeof(int), "mixed error word")) != CPL_OK) return s;
    CPL_CUDA_TRY(cudaMemcpyAsync(M.l3cap.ptr, src_cap.data(), sizeof(int) * nsrc, cudaMemcpyHostToDevice, st));
    std::vector<int> wr(2 * (size_t)nsrc);
    for (int q = 0; q < nsrc; ++q) {
        wr[q] = src_win[q];
        wr[nsrc + q] = src_role[q];
    }
    CPL_CUDA_TRY(cudaMemcpyAsync(M.src.ptr, wr.data(), sizeof(int) * 2 * nsrc, cudaMemcpyHostToDevice, st));
    CPL_CUDA_TRY(cudaMemsetAsync(M.A64.ptr, 0, sizeof(double) * (size_t)nsrc * a_stride, st));
    CPL_CUDA_TRY(cudaMemsetAsync(M.err.ptr, 0, sizeof(int), st));
    double *A64 = M.A64.as<double>();
    for (size_t gi = 0; gi < groups.size(); ++gi) {
        const int s0 = group_start[gi];
        CPL_CUDA_TRY(launch_weights(groups[gi].W, r->w_len, nw, M.l3cap.as<int>() + s0, A64 + (size_t)s0 * a_stride,
                                    a_stride, st));
    }
    float *Ah = M.Add.as<float>(), *Al = Ah + (size_t)nsrc * a_stride;
    int *Ae = reinterpret_cast<int *>(Al + (size_t)nsrc * a_stride);
    CPL_CUDA_TRY(mx_launch_weights_dd(A64, nsrc, a_stride, Ah, Al, Ae, st));

    // ---- A-side images
    unsigned role_union = 0;
    for (auto &g : groups) role_union |= g.spectra;
    int alpha_mask = 1;
    if (role_union & (kTE | kEE | kEEBB | kEB)) alpha_mask |= 2;
    if (role_union & (kEE | kEEBB | kEB)) alpha_mask |= 4;
    if (role_union & (kEEBB | kEB)) alpha_mask |= 8;
    const long long nrows = (long long)L.NRG * L.NB * MX_ROWS;
    if ((s = M.Aimg.ensure((size_t)2 * MX_NA * L.NRG * L.a_rg_bytes, "mixed A images")) != CPL_OK) return s;
    if ((s = M.eA.ensure(sizeof(int16_t) * 2 * MX_NA * nrows * L.NSB, "mixed A exponents")) != CPL_OK) return s;
    if ((s = M.emaxA.ensure(sizeof(int16_t) * 2 * MX_NA * nrows, "mixed A maxima")) != CPL_OK) return s;
    {
        MxPrepAArgs pa;
        std::memset(&pa, 0, sizeof(pa));
        pa.Ah = Ah;
        pa.Al = Al;
        pa.Ae = Ae;
        pa.a_stride = a_stride;
        pa.gh = gh;
        pa.gl = gl;
        pa.l3cap = M.l3cap.as<int>();
        pa.nsrc = nsrc;
        pa.alpha_mask = alpha_mask;
        pa.Aimg = M.Aimg.as<uint8_t>();
        pa.eA = M.eA.as<int16_t>();
        pa.emaxA = M.emaxA.as<int16_t>();
        pa.L = L;
        const int idx = stat_index(c, "mixed_prep_a");
        cudaEvent_t ev = begin_launch(c, st);
        CPL_CUDA_TRY(mx_launch_prep_a(pa, st));
        record_launch(c, idx, ev, st, 0.0, (double)2 * 4 * L.NRG * L.a_rg_bytes);
    }

    // ---- tiles and work items
    const int L1min = std::max(lmin, MX_L1_FP64);
    std::vector<int32_t> tile_of((size_t)2 * L.NRG * L.NB * L.NC, -1);
    struct TileRec {
        int pi, rg, b, c, kb_lo, kb_hi;
    };
    std::vector<TileRec> tiles;
    for (int pi = 0; pi < 2; ++pi)
        for (int b = 0; b < L.NB; ++b)
            for (int cb = 0; cb < L.NC; ++cb) {
                const int i0 = b * L.BI;
                const int ja = std::max(cb * MX_BJ, i0 + L1min), jb = std::min(cb * MX_BJ + MX_BJ - 1, lmax - pi - i0);
                if (ja > jb) continue;
                for (int rg = 0; rg < L.NRG; ++rg) {
                    int kcap = -1;
                    for (int q = 0; q < L.SRC; ++q) {
                        const int cap = src_cap[rg * L.SRC + q];
                        if (cap < 0) continue;
                        kcap = std::max(kcap, std::max((cap - pi) >> 1, (cap - 1 + pi) >> 1));
                    }
                    const int kb_lo = L.fA * b, kb_hi = std::min(std::min(L.gB * (cb + 1) - 1, L.NKB - 1), kcap / L.KB);
                    if (kcap < i0 || kb_hi < kb_lo) continue;   // the whole tile is zero (band limit)
                    tile_of[(((size_t)pi * L.NRG + rg) * L.NB + b) * L.NC + cb] = (int32_t)tiles.size();
                    tiles.push_back({pi, rg, b, cb, kb_lo, kb_hi});
                }
            }
    std::vector<MxItem> items;
    // order: parity, contraction, row block, column block, row group
    for (int pi = 0; pi < 2; ++pi)
        for (int p = 0; p < MX_NPROD; ++p)
            for (const TileRec &t : tiles) {
                if (t.pi != pi) continue;
                int need = 0;
                for (int q = 0; q < L.SRC; ++q) need = std::max(need, products_for(src[t.rg * L.SRC + q].role));
                if (p >= need) continue;
                MxItem it;
                it.pi = (int16_t)pi;
                it.p = (int16_t)p;
                it.kb_lo = (int16_t)t.kb_lo;
                it.kb_hi = (int16_t)t.kb_hi;
                it.tile = (int32_t)(&t - tiles.data());
                it.rg = (int16_t)t.rg;
                it.b = (int16_t)t.b;
                it.c = (int16_t)t.c;
                it.pad = 0;
                items.push_back(it);
            }
    // stable order within a parity/contraction: b, then c, then rg (tiles are generated in that order)
    const size_t inter_floats = (size_t)std::max<size_t>(tiles.size(), 1) * MX_NPROD * 2 * MX_ROWS * MX_BJ;
    if ((s = M.inter.ensure(sizeof(float) * inter_floats, "mixed intermediate")) != CPL_OK) return s;
    if ((s = M.items.ensure(sizeof(MxItem) * std::max<size_t>(items.size(), 1), "mixed items")) != CPL_OK) return s;
    if ((s = M.tile_of.ensure(sizeof(int32_t) * tile_of.size(), "mixed tile map")) != CPL_OK) return s;
    if (!items.empty())
        CPL_CUDA_TRY(cudaMemcpyAsync(M.items.ptr, items.data(), sizeof(MxItem) * items.size(), cudaMemcpyHostToDevice, st));
    CPL_CUDA_TRY(cudaMemcpyAsync(M.tile_of.ptr, tile_of.data(), sizeof(int32_t) * tile_of.size(),
                                 cudaMemcpyHostToDevice, st));

    // ---- GEMM
    {
        MxGemmArgs ga;
        std::memset(&ga, 0, sizeof(ga));
        ga.Aimg = M.Aimg.as<uint8_t>();
        ga.Bimg = M.Bimg.as<uint8_t>();
        ga.eA = M.eA.as<int16_t>();
        ga.emaxA = M.emaxA.as<int16_t>();
        ga.eB = M.eB.as<int16_t>();
        ga.emaxB = M.emaxB.as<int16_t>();
        ga.items = M.items.as<MxItem>();
        ga.n_items = (int)items.size();
        ga.inter = M.inter.as<float>();
        ga.err = M.err.as<int>();
        ga.L = L;
        double flop = 0.0, issued = 0.0;
        if (c->profiling) {
            // issued: 2 x 128 x 128 x k x (limb products) per item
            const double nlp = (double)S * (S + 1) / 2;
            for (const MxItem &it : items)
                issued += 2.0 * MX_ROWS * MX_BJ * (double)(it.kb_hi - it.kb_lo + 1) * L.KB * nlp;
            // algorithmic work: 2 FLOP per (source, l3 term, contraction) over the pairs the GEMM serves
            for (const TileRec &t : tiles)
                for (int q = 0; q < L.SRC; ++q) {
                    const Source &sr = src[t.rg * L.SRC + q];
                    if (sr.win < 0) continue;
                    const int np = products_for(sr.role);
                    const int n_even = std::min(np, 6), n_odd = np > 6 ? 3 : 0;
                    double e = 0, o = 0;
                    for (int di = 0; di < L.BI; ++di) {
                        const int i = t.b * L.BI + di;
                        const int ja = std::max(t.c * MX_BJ, i + L1min), jb = std::min(t.c * MX_BJ + MX_BJ - 1, lmax - t.pi - i);
                        if (ja <= jb) row_terms(i, ja, jb, t.pi, src_cap[t.rg * L.SRC + q], &e, &o);
                    }
                    flop += 2.0 * (n_even * e + n_odd * o);
                }
        }
        const int idx = stat_index(c, S == 6 ? "mixed_gemm_s6" : S == 5 ? "mixed_gemm_s5" : "mixed_gemm_s4");
        cudaEvent_t ev = begin_launch(c, st);
        CPL_CUDA_TRY(mx_launch_gemm(ga, st));
        record_launch(c, idx, ev, st, flop, 0.0, issued);
    }

    // ---- epilogue and FP64 band
    const int nb = r->bin_edges ? r->n_bins : 0;
    std::vector<int> bin_of;
    std::vector<double> bin_inv;
    if (nb) {
        bin_of.assign(lmax + 1, -1);
        bin_inv.assign(nb, 0.0);
        for (int bq = 0; bq < nb; ++bq) {
            for (int l = r->bin_edges[bq]; l < r->bin_edges[bq + 1]; ++l) bin_of[l] = bq;
            bin_inv[bq] = 1.0 / (double)(r->bin_edges[bq + 1] - r->bin_edges[bq]);
        }
        if ((s = c->bins_of.ensure(sizeof(int) * bin_of.size(), "bin map")) != CPL_OK) return s;
        if ((s = c->bins_inv.ensure(sizeof(double) * nb, "bin sizes")) != CPL_OK) return s;
        CPL_CUDA_TRY(cudaMemcpyAsync(c->bins_of.ptr, bin_of.data(), sizeof(int) * bin_of.size(), cudaMemcpyHostToDevice, st));
        CPL_CUDA_TRY(cudaMemcpyAsync(c->bins_inv.ptr, bin_inv.data(), sizeof(double) * nb, cudaMemcpyHostToDevice, st));
        size_t n_out = (size_t)nw * spec_count(r->spectra) * nb * nb;
        CPL_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(double) * n_out, st));
    }
    const unsigned bits[5] = {kTT, kTE, kEE, kEEBB, kEB};
    {
        MxEpiArgs ea;
        std::memset(&ea, 0, sizeof(ea));
        ea.inter = M.inter.as<float>();
        ea.tile_of = M.tile_of.as<int32_t>();
        ea.emaxA = M.emaxA.as<int16_t>();
        ea.emaxB = M.emaxB.as<int16_t>();
        ea.src_win = M.src.as<int>();
        ea.src_role = M.src.as<int>() + nsrc;
        ea.nsrc = nsrc;
        ea.lmax = lmax;
        ea.lmin = lmin;
        ea.out = out;
        ea.nspec = spec_count(r->spectra);
        for (int q = 0; q < 5; ++q) ea.slot[q] = spec_slot(r->spectra, bits[q]);
        ea.n_bins = nb;
        ea.bin_of = nb ? c->bins_of.as<int>() : nullptr;
        ea.bin_inv = nb ? c->bins_inv.as<double>() : nullptr;
        ea.L = L;
        const int idx = stat_index(c, "mixed_epilogue");
        cudaEvent_t ev = begin_launch(c, st);
        CPL_CUDA_TRY(mx_launch_epilogue(ea, st));
        record_launch(c, idx, ev, st, 0.0, 0.0);
    }
    {
        MxBandArgs ba;
        std::memset(&ba, 0, sizeof(ba));
        ba.g = c->g.as<double>();
        ba.h = c->h.as<double>();
        ba.A = A64;
        ba.a_stride = a_stride;
        ba.l3cap = M.l3cap.as<int>();
        ba.src_win = M.src.as<int>();
        ba.src_role = M.src.as<int>() + nsrc;
        ba.nsrc = nsrc;
        ba.lmax = lmax;
        ba.lmin = lmin;
        ba.out = out;
        ba.nspec = spec_count(r->spectra);
        for (int q = 0; q < 5; ++q) ba.slot[q] = spec_slot(r->spectra, bits[q]);
        ba.n_bins = nb;
        ba.bin_of = nb ? c->bins_of.as<int>() : nullptr;
        ba.bin_inv = nb ? c->bins_inv.as<double>() : nullptr;
        const int idx = stat_index(c, "mixed_band_fp64");
        cudaEvent_t ev = begin_launch(c, st);
        CPL_CUDA_TRY(mx_launch_band(ba, st));
        record_launch(c, idx, ev, st, 0.0, 0.0);
    }
    CPL_CUDA_TRY(cudaEventRecord(c->done, st));
    return CPL_OK;
}

}  // namespace cpl
