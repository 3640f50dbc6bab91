"""Plain FP64 path vs the CPU oracle, element by element (GPU).

Bar: per-element relative error (against S_abs) <= 1e-11 for every
spectrum; elements that are zero by parity or band exactly 0.0.  Sizes span
several 32 x 32 tiles with ragged tails; the full-size l_max = 3000 case and
an l_max = 10000 build are checked on sampled pairs, and identities that hold at any size (full sky,
constant window) are checked on whole matrices.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2602_15605_gb300 import coupling, windows
from parity_util import per_spectrum, rel_err, sample_pairs

pytestmark = pytest.mark.gpu
TOL = 1e-11
ALLN = ["TT", "TE", "EE", "EEBB", "EB"]


@pytest.fixture(scope="module")
def ctx():
    import torch
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


def check_dense(ctx, lmax, Wt, Wc, Wp, spectra, lmin=2, band_limit=None, tol=TOL, shared=False):
    if shared:
        W = dev(Wt)
        M = ctx.build(lmax, W, W, W, spectra, lmin=lmin, band_limit=band_limit)
    else:
        M = ctx.build(lmax, dev(Wt) if Wt is not None else None, dev(Wc) if Wc is not None else None,
                      dev(Wp) if Wp is not None else None, spectra, lmin=lmin, band_limit=band_limit)
    got = M.cpu().numpy()
    ref, sab = oracle.coupling_dense(lmax, Wt, Wc, Wp, spectra, lmin=lmin, band_limit=band_limit)
    errs = per_spectrum(got, ref, sab, names(spectra))
    assert max(errs.values()) <= tol, errs
    return errs


def test_tt_512_full_matrix(ctx):
    # one mask-like window, l_max = 512, l <= 1024, output 511 x 511
    W = windows.tt_512()
    errs = check_dense(ctx, 512, W, None, None, coupling.TT)
    print("TT 512:", errs)


def test_full_spin_separate_windows_dense(ctx):
    lmax = 157   # several tiles and ragged tails in both parities
    Wt, Wc, Wp = (windows.gaussian_taper(lmax, s) for s in (2, 3, 4))
    print(check_dense(ctx, lmax, Wt, Wc, Wp, coupling.ALL))


def test_full_spin_shared_window_dense(ctx):
    lmax = 130
    W = windows.mask_like(lmax, seed=21)
    print(check_dense(ctx, lmax, W, W, W, coupling.ALL, shared=True))


@pytest.mark.parametrize("spectra", [coupling.TT, coupling.TE, coupling.EE, coupling.EEBB, coupling.EB,
                                     coupling.EE | coupling.EEBB, coupling.TT | coupling.EB,
                                     coupling.TE | coupling.EEBB])
def test_spectrum_subsets(ctx, spectra):
    lmax = 75
    Wt, Wc, Wp = (windows.gaussian_taper(lmax, s) for s in (5, 6, 7))
    check_dense(ctx, lmax, Wt, Wc, Wp, spectra)


def test_tt_lmin_zero_and_multi_window(ctx):
    lmax = 97
    W = np.stack([windows.random_positive(lmax, seed=s) for s in range(3)])
    check_dense(ctx, lmax, W, None, None, coupling.TT, lmin=0)


def test_small_edge_sizes(ctx):
    for lmax, lmin in [(2, 2), (3, 2), (5, 5), (33, 2), (34, 3), (64, 2), (65, 2)]:
        W = windows.random_positive(lmax, seed=lmax)
        check_dense(ctx, lmax, W, W, W, coupling.ALL, lmin=lmin)


def test_band_limited_dense(ctx):
    lmax = 120
    W = np.stack([windows.random_positive(lmax, seed=s, band=b) for s, b in ((1, 10), (2, 33), (3, 64))])
    bl = [10, 33, 64]
    check_dense(ctx, lmax, W, W, W, coupling.ALL, band_limit=bl)
    # band-limited equals full sweep on the same (zero above L_w) windows
    Mb = ctx.build(lmax, dev(W), dev(W), dev(W), coupling.ALL, band_limit=bl).cpu().numpy()
    Mf = ctx.build(lmax, dev(W), dev(W), dev(W), coupling.ALL).cpu().numpy()
    assert np.array_equal(Mb, Mf)


def test_binned(ctx):
    lmax = 140
    W = np.stack([windows.random_positive(lmax, seed=s, band=b) for s, b in ((4, 20), (5, 40))])
    edges = oracle.bin_edges(2, lmax, 25)
    got = ctx.build(lmax, dev(W), dev(W), dev(W), coupling.ALL, band_limit=[20, 40], bin_edges=edges)
    ref, sab = oracle.coupling_dense(lmax, W, W, W, coupling.ALL)
    Rb = oracle.bin_matrix(ref, 2, edges)
    Sb = oracle.bin_matrix(sab, 2, edges)
    errs = per_spectrum(got.cpu().numpy(), Rb, Sb, ALLN)
    assert max(errs.values()) <= TOL, errs


def test_full_spin_3000_sampled(ctx):
    # separate W^TT, W^TP, W^PP, l_max = 3000, l <= 6000: sampled pairs
    lmax = 3000
    Wt, Wc, Wp = windows.full_spin_3000(lmax)
    M = ctx.build(lmax, dev(Wt), dev(Wc), dev(Wp), coupling.ALL)
    l1, l2 = sample_pairs(lmax, n_random=6000)
    got = M[:, :, l1 - 2, l2 - 2].cpu().numpy()
    ref, sab = oracle.coupling_pairs(l1, l2, Wt, Wc, Wp, coupling.ALL)
    errs = per_spectrum(got, ref, sab, ALLN)
    print("full spin 3000 sampled:", errs)
    assert max(errs.values()) <= TOL, errs


def test_full_sky_identity_large(ctx):
    lmax = 700
    W = windows.full_sky(lmax)
    M = ctx.build(lmax, dev(W), dev(W), dev(W), coupling.ALL).cpu().numpy()
    I = np.eye(lmax - 1)
    for s, want in enumerate((I, I, I, 0 * I, I)):
        assert np.max(np.abs(M[0, s] - want)) < 1e-12, ALLN[s]


def test_constant_window_large(ctx):
    lmax = 600
    W = windows.constant(lmax)
    M = ctx.build(lmax, dev(W), None, dev(W), coupling.TT | coupling.EE | coupling.EEBB).cpu().numpy()
    col = (2 * np.arange(2, lmax + 1) + 1)[None, :]
    assert np.max(np.abs(M[0, 0] / col - 1)) < 1e-11
    assert np.max(np.abs((M[0, 1] + M[0, 2]) / col - 1)) < 1e-11


def test_build_host_matches_device(ctx):
    lmax = 90
    Wt, Wc, Wp = (windows.gaussian_taper(lmax, s) for s in (8, 9, 10))
    Md = ctx.build(lmax, dev(Wt), dev(Wc), dev(Wp), coupling.ALL).cpu().numpy()
    Mh = ctx.build_host(lmax, Wt, Wc, Wp, coupling.ALL)
    assert np.array_equal(Md, Mh)


@pytest.mark.parametrize("binned", [False, True])
def test_build_host_pinned_overlapped_copies(ctx, binned):
    # page-locked output: each launch's blocks are copied out while the later
    # launches run (three launches: separate windows; two windows per role)
    import torch
    lmax = 130
    Wt, Wc, Wp = (np.stack([windows.mask_like(lmax, seed=s + q) for q in range(2)]) for s in (60, 70, 80))
    edges = list(range(2, lmax + 2, 16)) + ([lmax + 1] if (lmax - 1) % 16 else []) if binned else None
    Md = ctx.build(lmax, dev(Wt), dev(Wc), dev(Wp), coupling.ALL, bin_edges=edges).cpu().numpy()
    pinned = torch.full(Md.shape, -1.0, dtype=torch.float64, pin_memory=True).numpy()
    Mh = ctx.build_host(lmax, Wt, Wc, Wp, coupling.ALL, bin_edges=edges, out=pinned)
    if binned:   # FP64 atomics: order not fixed
        assert np.max(np.abs(Mh - Md)) <= 1e-14 * np.max(np.abs(Md))
    else:
        assert np.array_equal(Md, Mh)
    pageable = ctx.build_host(lmax, Wt, Wc, Wp, coupling.ALL, bin_edges=edges)
    assert np.max(np.abs(pageable - Mh)) <= 1e-14 * np.max(np.abs(Md))


def test_batch_matches_single(ctx):
    jobs = []
    for lm, s in ((40, 1), (77, 2), (130, 3)):
        W = dev(windows.mask_like(lm, seed=s))
        jobs.append(dict(lmax=lm, W_tt=W, W_tp=W, W_pp=W, spectra=coupling.ALL))
    outs = ctx.build_batch(jobs)
    for j, o in zip(jobs, outs):
        single = ctx.build(**j)
        assert np.array_equal(o.cpu().numpy(), single.cpu().numpy())


def test_argument_errors_leave_output_untouched(ctx):
    import torch
    lmax = 20
    W = dev(windows.random_positive(lmax, seed=1))
    out = torch.full((1, 1, lmax - 1, lmax - 1), 7.0, dtype=torch.float64, device="cuda")
    with pytest.raises(coupling.CouplingError) as e:
        ctx.build(lmax, W, None, None, coupling.EE, out=out)   # W_pp missing
    assert e.value.status == 1
    with pytest.raises(coupling.CouplingError):
        ctx.build(lmax, W, None, None, coupling.TT, lmin=-1)
    torch.cuda.synchronize()
    assert torch.all(out == 7.0)


def test_batch_mixed_variants_band_and_bins(ctx):
    # one launch per kernel variant over the items of all jobs: a TT-only
    # job, a full spin set with separate windows, a band-limited binned job
    jobs = []
    W1 = dev(windows.mask_like(88, seed=11))
    jobs.append(dict(lmax=88, W_tt=W1, spectra=coupling.TT))
    Wt, Wc, Wp = (dev(windows.gaussian_taper(121, s)) for s in (12, 13, 14))
    jobs.append(dict(lmax=121, W_tt=Wt, W_tp=Wc, W_pp=Wp, spectra=coupling.ALL))
    Wb = np.stack([windows.random_positive(150, seed=15 + q, band=b) for q, b in enumerate((40, 90))])
    jobs.append(dict(lmax=150, W_tt=dev(Wb), W_tp=dev(Wb), W_pp=dev(Wb), spectra=coupling.TE | coupling.EEBB,
                     band_limit=[40, 90], bin_edges=oracle.bin_edges(2, 150, 20)))
    outs = ctx.build_batch(jobs)
    ctx.sync()
    for q, (j, o) in enumerate(zip(jobs, outs)):
        single = ctx.build(**j).cpu().numpy()
        if "bin_edges" in j:
            assert np.allclose(o.cpu().numpy(), single, rtol=1e-14, atol=0.0)
        else:
            assert np.array_equal(o.cpu().numpy(), single)
    # and the band-limited binned job against the oracle
    ref, sab = oracle.coupling_dense(150, Wb, Wb, Wb, coupling.TE | coupling.EEBB, band_limit=[40, 90])
    e = oracle.bin_edges(2, 150, 20)
    errs = per_spectrum(outs[2].cpu().numpy(), oracle.bin_matrix(ref, 2, e), oracle.bin_matrix(sab, 2, e), ["TE", "EEBB"])
    assert max(errs.values()) <= 1e-11, errs


def test_lmax_10000_separate_windows_sampled(ctx):
    """The tabled kernel at l_max = 10000 (operand tables of ~7 GB, 64-bit
    block offsets) with three separate windows, so that all three kernel
    variants run: sampled pairs against the oracle, every spectrum, including
    the last row and near-diagonal pairs."""
    import torch
    lmax = 10000
    W = windows.ragged_jobs(lmaxes=(lmax,), n_win=3, seed0=900)[0][1]
    M = ctx.build(lmax, dev(W[0]), dev(W[1]), dev(W[2]), coupling.ALL)
    rng = np.random.default_rng(11000)
    d = rng.integers(2, lmax - 2, size=120)
    P = np.concatenate([rng.integers(2, lmax + 1, size=(900, 2)),
                        np.stack([np.full(120, lmax), rng.integers(2, lmax + 1, size=120)], axis=1),
                        np.stack([d, d + rng.integers(0, 3, size=120)], axis=1)]).astype(np.int32)
    l1, l2 = P[:, 0], P[:, 1]
    got = M[:, :, torch.as_tensor(l1 - 2, device="cuda"), torch.as_tensor(l2 - 2, device="cuda")].cpu().numpy()
    del M
    torch.cuda.empty_cache()
    assert np.all(np.isfinite(got))
    ref, sab = oracle.coupling_pairs(l1, l2, W[0], W[1], W[2], coupling.ALL)
    errs = per_spectrum(got, ref, sab, ALLN)
    print("fp64 10000 sampled vs oracle:", errs)
    assert max(errs.values()) <= TOL


def _sampled_large(ctx, lmax, spectra, seed, n_random=400, n_edge=60):
    import torch
    W = windows.mask_like(lmax, seed=seed)
    M = ctx.build(lmax, dev(W), dev(W), dev(W), spectra)
    rng = np.random.default_rng(seed)
    d = rng.integers(2, lmax - 2, size=n_edge)
    P = np.concatenate([rng.integers(2, lmax + 1, size=(n_random, 2)),
                        np.stack([np.full(n_edge, lmax), rng.integers(2, lmax + 1, size=n_edge)], axis=1),
                        np.stack([d, d], axis=1),
                        np.stack([d, d + rng.integers(1, 3, size=n_edge)], axis=1)]).astype(np.int32)
    l1, l2 = P[:, 0], P[:, 1]
    got = M[:, :, torch.as_tensor(l1 - 2, device="cuda"), torch.as_tensor(l2 - 2, device="cuda")].cpu().numpy()
    del M
    torch.cuda.empty_cache()
    assert np.all(np.isfinite(got))
    ref, sab = oracle.coupling_pairs(l1, l2, W, W, W, spectra)
    return per_spectrum(got, ref, sab, names(spectra))


def test_lmax_20000_polarisation_sampled(ctx):
    # EE and EE->BB (the spectrum whose odd sweep cancels the most) at
    # l_max = 20000: sampled pairs incl. the diagonal and the last row
    errs = _sampled_large(ctx, 20000, coupling.EE | coupling.EEBB, seed=20000)
    print("fp64 20000 sampled vs oracle:", errs)
    assert max(errs.values()) <= TOL


def test_lmax_32000_tt_sampled(ctx):
    # the largest l_max the library accepts (operand tables ~50 GB)
    errs = _sampled_large(ctx, 32000, coupling.TT, seed=32000)
    print("fp64 32000 sampled vs oracle:", errs)
    assert max(errs.values()) <= TOL
