"""Mixed-precision (tcgen05, BF16 fixed-point limbs) path vs the CPU oracle (GPU).

Bar: per-element relative error (against the oracle's S_abs) <= 1e-9 for
every spectrum, the bound this path states; elements that are zero by parity
or band exactly 0.0.  Cases span several 128 x 128 GEMM tiles, ragged tails,
row groups with padding (window counts not a multiple of 4), separate and
shared window roles, band limits and binning.
"""
import numpy as np
import pytest

import oracle
from paper_2602_15605_gb300 import coupling, windows
from parity_util import per_spectrum, sample_pairs

pytestmark = pytest.mark.gpu
TOL = 1e-9
ALLN = ["TT", "TE", "EE", "EEBB", "EB"]


@pytest.fixture(scope="module")
def ctx():
    from paper_2602_15605_gb300 import build_ext
    build_ext.build()
    c = coupling.Context(0)
    yield c
    c.close()


def dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def names(spectra):
    return [n for b, n in zip(coupling.SPEC_BITS, ALLN) if spectra & b]


def mixed(ctx, lmax, Wt, Wc, Wp, spectra, **kw):
    M = ctx.build(lmax, Wt, Wc, Wp, spectra, precision=coupling.MIXED_BF16, **kw)
    ctx.sync()
    return M.cpu().numpy()


def test_shared_window_dense(ctx):
    lmax = 300
    W = windows.mask_like(lmax, seed=31)
    d = dev(W)
    got = mixed(ctx, lmax, d, d, d, coupling.ALL)
    ref, sab = oracle.coupling_dense(lmax, W, W, W, coupling.ALL)
    errs = per_spectrum(got, ref, sab, ALLN)
    print("mixed shared 300:", errs)
    assert max(errs.values()) <= TOL, errs


def test_separate_windows_dense(ctx):
    lmax = 257
    Wt, Wc, Wp = (windows.gaussian_taper(lmax, s) for s in (2, 3, 4))
    got = mixed(ctx, lmax, dev(Wt), dev(Wc), dev(Wp), coupling.ALL)
    ref, sab = oracle.coupling_dense(lmax, Wt, Wc, Wp, coupling.ALL)
    errs = per_spectrum(got, ref, sab, ALLN)
    print("mixed separate 257:", errs)
    assert max(errs.values()) <= TOL, errs


def test_many_windows_padding(ctx):
    lmax = 200
    W = np.stack([windows.mask_like(lmax, seed=40 + q) for q in range(6)])
    d = dev(W)
    got = mixed(ctx, lmax, d, d, d, coupling.TT | coupling.EE | coupling.EEBB)
    ref, sab = oracle.coupling_dense(lmax, W, W, W, coupling.TT | coupling.EE | coupling.EEBB)
    errs = per_spectrum(got, ref, sab, ["TT", "EE", "EEBB"])
    assert max(errs.values()) <= TOL, errs


@pytest.mark.parametrize("spectra", [coupling.TT, coupling.TE, coupling.EE | coupling.EB])
def test_subsets(ctx, spectra):
    lmax = 150
    Wt, Wc, Wp = (windows.gaussian_taper(lmax, s) for s in (5, 6, 7))
    got = mixed(ctx, lmax, dev(Wt), dev(Wc), dev(Wp), spectra)
    ref, sab = oracle.coupling_dense(lmax, Wt, Wc, Wp, spectra)
    errs = per_spectrum(got, ref, sab, names(spectra))
    assert max(errs.values()) <= TOL, errs


def test_band_limited_binned(ctx):
    lmax = 400
    W = np.stack([windows.random_positive(lmax, seed=s, band=b) for s, b in ((1, 64), (2, 128), (3, 33))])
    bl = [64, 128, 33]
    edges = oracle.bin_edges(2, lmax, 50)
    d = dev(W)
    got = ctx.build(lmax, d, d, d, coupling.ALL, band_limit=bl, bin_edges=edges, precision=coupling.MIXED_BF16)
    ctx.sync()
    ref, sab = oracle.coupling_dense(lmax, W, W, W, coupling.ALL, band_limit=bl)
    errs = per_spectrum(got.cpu().numpy(), oracle.bin_matrix(ref, 2, edges), oracle.bin_matrix(sab, 2, edges), ALLN)
    assert max(errs.values()) <= TOL, errs
    dense = mixed(ctx, lmax, d, d, d, coupling.ALL, band_limit=bl)
    errs = per_spectrum(dense, ref, sab, ALLN)
    assert max(errs.values()) <= TOL, errs


def test_full_spin_1500_sampled(ctx):
    lmax = 1500
    W = windows.mask_like(lmax, seed=77)
    d = dev(W)
    M = ctx.build(lmax, d, d, d, coupling.ALL, precision=coupling.MIXED_BF16)
    ctx.sync()
    l1, l2 = sample_pairs(lmax, n_random=4000)
    got = M[:, :, l1 - 2, l2 - 2].cpu().numpy()
    ref, sab = oracle.coupling_pairs(l1, l2, W, W, W, coupling.ALL)
    errs = per_spectrum(got, ref, sab, ALLN)
    print("mixed 1500 sampled:", errs)
    assert max(errs.values()) <= TOL, errs


def test_mixed_matches_plain_fp64_many_windows(ctx):
    # 12 windows (3 row groups) at l_max = 500 against the parity-tested FP64 path
    lmax = 500
    W = np.stack([windows.mask_like(lmax, seed=100 + q) for q in range(12)])
    d = dev(W)
    Mm = mixed(ctx, lmax, d, d, d, coupling.TT | coupling.EE | coupling.EEBB)
    Mp = ctx.build(lmax, d, d, d, coupling.TT | coupling.EE | coupling.EEBB).cpu().numpy()
    # TT, EE and EE->BB have non-negative terms, so |M| is the S_abs scale
    m = np.abs(Mp) > 1e-280
    rel = np.max(np.abs(Mm[m] - Mp[m]) / np.abs(Mp[m]))
    print("mixed vs fp64 (12 windows, 500):", rel)
    assert rel <= TOL
    assert np.all(Mm[~m] == 0.0)


def test_five_limbs_faster_variant(ctx):
    # mixed_slices = 5: about 5x fewer limb products than the default 6 at a
    # bound of 5e-9 (the EE->BB expansion amplifies its ~2e-10 contraction error)
    lmax = 300
    W = windows.mask_like(lmax, seed=31)
    d = dev(W)
    M = ctx.build(lmax, d, d, d, coupling.ALL, precision=coupling.MIXED_BF16, slices=5)
    ctx.sync()
    ref, sab = oracle.coupling_dense(lmax, W, W, W, coupling.ALL)
    errs = per_spectrum(M.cpu().numpy(), ref, sab, ALLN)
    print("mixed s=5 300:", errs)
    assert max(errs.values()) <= 5e-9, errs


def test_four_and_five_limbs_across_scale_blocks(ctx):
    # mixed_slices = 4 and 5 run the 32-k stage variant of the GEMM (two stages,
    # the order >= 3 products of one stage issued ahead of orders 0-2); l_max
    # 700 gives items of up to three 256-k scale blocks.  Bounds: 4 limbs keep
    # ~32 bits (measured ~1e-7), 5 limbs ~40 (the 5e-9 above)
    lmax = 700
    W = np.stack([windows.mask_like(lmax, seed=70 + q) for q in range(2)])
    d = dev(W)
    l1, l2 = sample_pairs(lmax, n_random=4000, band=3)
    ref, sab = oracle.coupling_pairs(l1, l2, W, W, W, coupling.ALL)
    import torch
    a = torch.as_tensor(l1 - 2, device="cuda", dtype=torch.long)
    b = torch.as_tensor(l2 - 2, device="cuda", dtype=torch.long)
    for S, bound in ((4, 1e-6), (5, 5e-9)):
        M = ctx.build(lmax, d, d, d, coupling.ALL, precision=coupling.MIXED_BF16, slices=S)
        ctx.sync()
        errs = per_spectrum(M[:, :, a, b].cpu().numpy(), ref, sab, ALLN)
        print("mixed s=%d 700 x 2:" % S, errs)
        assert max(errs.values()) <= bound, (S, errs)


@pytest.mark.parametrize("shared_tt_pp", [False, True])
def test_build_host_pinned_split_matches_device(ctx, shared_tt_pp):
    # page-locked output of a mixed build with several window-role groups: one
    # build per group, each group's planes copied to their places while the
    # later groups compute (two windows; with W^TT = W^PP the groups are
    # {TT, EE, EE->BB, EB} and {TE}, whose planes interleave in the output)
    import torch
    lmax = 257
    Wt, Wc, Wp = (np.stack([windows.mask_like(lmax, seed=s + q) for q in range(2)]) for s in (90, 91, 92))
    if shared_tt_pp:
        Wp = Wt
    dWt, dWc = dev(Wt), dev(Wc)
    dWp = dWt if shared_tt_pp else dev(Wp)
    Md = ctx.build(lmax, dWt, dWc, dWp, coupling.ALL, precision=coupling.MIXED_BF16).cpu().numpy()
    pinned = torch.full(Md.shape, -1.0, dtype=torch.float64, pin_memory=True).numpy()
    Mh = ctx.build_host(lmax, Wt, Wc, Wt if shared_tt_pp else Wp, coupling.ALL, precision=coupling.MIXED_BF16,
                        out=pinned)
    # the per-source limb contractions do not depend on which sources share a
    # GEMM, so the split build is bit-identical to the single one
    assert np.array_equal(Md, Mh)
    pageable = ctx.build_host(lmax, Wt, Wc, Wt if shared_tt_pp else Wp, coupling.ALL, precision=coupling.MIXED_BF16)
    assert np.array_equal(pageable, Mh)


def test_two_windows_row_shape(ctx):
    # two windows per role: GEMM tiles of 2 sources x 64 i-values
    lmax = 333
    W = np.stack([windows.mask_like(lmax, seed=60 + q) for q in range(2)])
    d = dev(W)
    got = mixed(ctx, lmax, d, d, d, coupling.ALL)
    ref, sab = oracle.coupling_dense(lmax, W, W, W, coupling.ALL)
    errs = per_spectrum(got, ref, sab, ALLN)
    assert max(errs.values()) <= TOL, errs


def _ragged_jobs():
    """Three requests of different shape: l_max, window count (row shape 1, 2
    and 4 sources per tile), band limits, binning, separate window roles."""
    jobs, host = [], []
    W1 = windows.mask_like(97, seed=201)
    jobs.append(dict(lmax=97, W_tt=dev(W1), W_tp=dev(W1), W_pp=dev(W1), spectra=coupling.ALL))
    host.append(dict(lmax=97, W=(W1, W1, W1), band_limit=None, bin_edges=None))
    W2 = np.stack([windows.random_positive(260, seed=202 + q, band=b) for q, b in enumerate((70, 150, 41))])
    d2 = dev(W2)
    jobs.append(dict(lmax=260, W_tt=d2, W_tp=d2, W_pp=d2, spectra=coupling.ALL, band_limit=[70, 150, 41]))
    host.append(dict(lmax=260, W=(W2, W2, W2), band_limit=[70, 150, 41], bin_edges=None))
    Wt, Wc, Wp = (np.stack([windows.gaussian_taper(333, 210 + 3 * q + s) for q in range(2)]) for s in range(3))
    edges = oracle.bin_edges(2, 333, 50)
    jobs.append(dict(lmax=333, W_tt=dev(Wt), W_tp=dev(Wc), W_pp=dev(Wp), spectra=coupling.TT | coupling.TE |
                     coupling.EB, bin_edges=edges))
    host.append(dict(lmax=333, W=(Wt, Wc, Wp), band_limit=None, bin_edges=edges))
    for j in jobs:
        j["precision"] = coupling.MIXED_BF16
    return jobs, host


def _check_job(got, job, h):
    spectra = job["spectra"]
    ref, sab = oracle.coupling_dense(h["lmax"], *h["W"], spectra, band_limit=h["band_limit"])
    if h["bin_edges"] is not None:
        ref = oracle.bin_matrix(ref, 2, h["bin_edges"])
        sab = oracle.bin_matrix(sab, 2, h["bin_edges"])
    errs = per_spectrum(got, ref, sab, names(spectra))
    assert max(errs.values()) <= TOL, (h["lmax"], errs)
    return errs


def _same(a, b, binned):
    if binned:
        assert np.allclose(a, b, rtol=1e-13, atol=0.0)
    else:
        assert np.array_equal(a, b)


def test_batch_ragged_matches_oracle_and_single(ctx):
    # one persistent GEMM over the items of all three jobs, captured into a graph
    jobs, host = _ragged_jobs()
    outs = ctx.build_batch(jobs)
    ctx.sync()
    for o, j, h in zip(outs, jobs, host):
        got = o.cpu().numpy()
        print("batch job", h["lmax"], _check_job(got, j, h))
        single = ctx.build(**j)
        ctx.sync()
        # every item runs the same arithmetic in the batch and alone (binned
        # sums are accumulated with atomics, in no fixed order)
        _same(got, single.cpu().numpy(), h["bin_edges"] is not None)


def test_batch_graph_replay_sees_new_window_values(ctx):
    import torch
    jobs, host = _ragged_jobs()
    outs = ctx.build_batch(jobs)
    ctx.sync()
    first = [o.cpu().numpy().copy() for o in outs]
    before = ctx.stats()
    # same pointers and shapes: the second call replays the captured graph
    # and must read the windows' current contents
    scale = 0.5
    seen = set()
    for j in jobs:
        for key in ("W_tt", "W_tp", "W_pp"):
            W = j[key]
            if W.data_ptr() not in seen:
                seen.add(W.data_ptr())
                W.mul_(scale)
    torch.cuda.synchronize()
    outs2 = ctx.build_batch(jobs, outs=outs)
    ctx.sync()
    after = ctx.stats()
    for o, f, h in zip(outs2, first, host):
        # M is linear in W and the limb split is exact under scaling by 2^-1
        _same(o.cpu().numpy(), f * scale, h["bin_edges"] is not None)
    g0 = before.get("mixed_gemm_s6", {}).get("launches", 0)
    g1 = after.get("mixed_gemm_s6", {}).get("launches", 0)
    assert g1 == g0 + 1   # one persistent GEMM launch for the whole batch


def test_autotuner_is_exact_and_cached(tmp_path):
    # every tuner candidate computes the same matrices: the tuned build equals
    # the built-in one bit for bit, the choice is cached per shape and
    # persisted, and a new context reads it back instead of measuring again
    import json
    path = tmp_path / "tune.jsonl"
    lmax = 333
    W = np.stack([windows.mask_like(lmax, seed=70 + q) for q in range(3)])
    plain = coupling.Context(0)
    d = dev(W)
    ref = plain.build(lmax, d, d, d, coupling.ALL, precision=coupling.MIXED_BF16).cpu().numpy()
    plain.close()
    t = coupling.Context(0)
    t.tune(True, path)
    got = t.build(lmax, d, d, d, coupling.ALL, precision=coupling.MIXED_BF16).cpu().numpy()
    t.sync()
    assert np.array_equal(got, ref)
    lines = [json.loads(x) for x in path.read_text().splitlines()]
    assert len(lines) == 1 and lines[0]["src"] in (1, 2, 4) and lines[0]["order"] in (0, 1)
    assert lines[0]["key"][1] == lmax and lines[0]["ms"] > 0
    t.build(lmax, d, d, d, coupling.ALL, precision=coupling.MIXED_BF16)   # cached: no new measurement
    t.sync()
    assert len(path.read_text().splitlines()) == 1
    t.close()
    u = coupling.Context(0)
    u.tune(True, path)
    again = u.build(lmax, d, d, d, coupling.ALL, precision=coupling.MIXED_BF16).cpu().numpy()
    u.sync()
    assert np.array_equal(again, ref)
    assert len(path.read_text().splitlines()) == 1   # read from the file
    with pytest.raises(coupling.CouplingError):
        u.tune(7)
    u.close()


def test_autotuned_batch_matches_untuned(ctx):
    jobs, host = _ragged_jobs()
    ref = [o.cpu().numpy() for o in ctx.build_batch(jobs)]
    t = coupling.Context(0)
    t.tune(True)
    outs = t.build_batch(jobs)
    t.sync()
    for o, r, h in zip(outs, ref, host):
        _same(o.cpu().numpy(), r, h["bin_edges"] is not None)
    t.close()


def test_batch_split_into_chunks_matches(ctx, monkeypatch):
    # a scratch budget smaller than any job puts every job in its own chunk
    # (one persistent GEMM launch each); the results must not change
    jobs, host = _ragged_jobs()
    ref = [o.cpu().numpy() for o in ctx.build_batch(jobs)]
    monkeypatch.setenv("CPL_MIXED_SCRATCH_GB", "0.000001")
    c = coupling.Context(0)
    c.profile(True)
    c.stats(reset=True)
    outs = c.build_batch(jobs)    # profiling on: eager launches, counted
    c.sync()
    st = c.stats()
    assert st["mixed_gemm_s6"]["launches"] == len(jobs)
    for o, r, h in zip(outs, ref, host):
        _same(o.cpu().numpy(), r, h["bin_edges"] is not None)
    c.close()


def test_tt_lmin_zero_two_windows(ctx):
    # l1 from 0 (TT only): the FP64 band covers l1 < 32, the GEMM the rest
    lmax = 111
    W = np.stack([windows.mask_like(lmax, seed=80), windows.mask_like(lmax, seed=81)])
    d = dev(W)
    got = mixed(ctx, lmax, d, None, None, coupling.TT, lmin=0)
    ref, sab = oracle.coupling_dense(lmax, W, spectra=coupling.TT, lmin=0)
    errs = per_spectrum(got, ref, sab, ["TT"])
    assert max(errs.values()) <= TOL, errs
