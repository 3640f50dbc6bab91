"""Double-float plain path (CPL_DF32) vs the CPU oracle and the FP64 path (GPU).

Bar: per-element relative error against S_abs (reading 10) <= 1e-11 for
every spectrum, the plain path's target; elements zero by parity or band
exactly 0.0.  Cases: whole matrices against the oracle (TT at l_max = 512, the full spin set with
separate windows, lmin = 0, a band limit, binning), the full-size l_max =
3000 workload on sampled pairs against the oracle and on every element of
the non-negative spectra (TT, EE, EE->BB, where S_abs equals the value)
against the parity-tested FP64 path, the band-limited l_max = 8000 binned
workload against the FP64 path, and a zero window.
"""
import numpy as np
import pytest

import oracle
from paper_2602_15605_gb300 import coupling, windows
from parity_util import per_spectrum, rel_err, sample_pairs

pytestmark = pytest.mark.gpu
TOL = 1e-11
ALLN = ["TT", "TE", "EE", "EEBB", "EB"]
DF = coupling.DF32


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


def dense_vs_oracle(ctx, lmax, Wt, Wc, Wp, spectra, lmin=2, band_limit=None):
    M = ctx.build(lmax, dev(Wt) if Wt is not None else None, dev(Wc) if Wc is not None else None,
                  dev(Wp) if Wp is not None else None, spectra, lmin=lmin, band_limit=band_limit, precision=DF)
    got = M.cpu().numpy()
    ref, sab = oracle.coupling_dense(lmax, Wt, Wc, Wp, spectra, lmin=lmin, band_limit=band_limit)
    errs = per_spectrum(got, ref, sab, names(spectra))
    assert max(errs.values()) <= TOL, errs
    return errs


def test_tt_512(ctx):
    print("df TT 512:", dense_vs_oracle(ctx, 512, windows.tt_512(), None, None, coupling.TT))


def test_full_spin_separate_windows(ctx):
    lmax = 250
    Wt, Wc, Wp = (windows.gaussian_taper(lmax, s) for s in (11, 12, 13))
    print("df full spin 250:", dense_vs_oracle(ctx, lmax, Wt, Wc, Wp, coupling.ALL))


def test_tt_lmin0_and_band_limit(ctx):
    lmax = 140
    W = windows.random_positive(lmax, seed=5, band=40)
    print("df lmin 0:", dense_vs_oracle(ctx, lmax, W, None, None, coupling.TT, lmin=0))
    print("df band 40:", dense_vs_oracle(ctx, lmax, W, W, W, coupling.ALL, band_limit=[40]))


def test_binned_vs_oracle(ctx):
    lmax = 160
    W = windows.mask_like(lmax, seed=3)
    edges = oracle.bin_edges(2, lmax, 7)
    d = dev(W)
    got = ctx.build(lmax, d, d, d, coupling.ALL, bin_edges=edges, precision=DF).cpu().numpy()
    ref, sab = oracle.coupling_dense(lmax, W, W, W, coupling.ALL)
    errs = per_spectrum(got, oracle.bin_matrix(ref, 2, edges), oracle.bin_matrix(sab, 2, edges), ALLN)
    print("df binned:", errs)
    assert max(errs.values()) <= TOL


def test_zero_window(ctx):
    lmax = 70
    W = dev(np.zeros(2 * lmax + 1))
    M = ctx.build(lmax, W, W, W, coupling.ALL, precision=DF).cpu().numpy()
    assert np.all(M == 0.0)


def test_full_spin_3000(ctx):
    lmax = 3000
    Wt, Wc, Wp = windows.full_spin_3000()
    dW = [dev(W) for W in (Wt, Wc, Wp)]
    Md = ctx.build(lmax, *dW, coupling.ALL, precision=DF).cpu().numpy()
    Mf = ctx.build(lmax, *dW, coupling.ALL).cpu().numpy()
    # sampled pairs against the oracle, every spectrum
    l1, l2 = sample_pairs(lmax, n_random=3000)
    ref, sab = oracle.coupling_pairs(l1, l2, Wt, Wc, Wp, coupling.ALL)
    got = Md[:, :, l1 - 2, l2 - 2]
    errs = per_spectrum(got, ref, sab, ALLN)
    print("df 3000 sampled vs oracle:", errs)
    assert max(errs.values()) <= TOL
    # every element of the non-negative spectra against the FP64 path
    for s, nm in ((0, "TT"), (2, "EE"), (3, "EEBB")):
        a, b = Md[0, s], Mf[0, s]
        m = np.abs(b) > 1e-280
        assert np.all(a[~m] == 0.0) or np.max(np.abs(a[~m])) < 1e-280, nm
        e = float(np.max(np.abs(a[m] - b[m]) / np.abs(b[m])))
        print("df 3000 %s vs fp64 (all elements): %.3g" % (nm, e))
        assert e <= TOL, (nm, e)


def test_band_limited_8000_binned(ctx):
    lmax = 8000
    W, Lw = windows.band_limited(lmax)
    edges = oracle.bin_edges(2, lmax, 50)
    d = dev(W)
    Md = ctx.build(lmax, d, d, d, coupling.ALL, band_limit=Lw, bin_edges=edges, precision=DF).cpu().numpy()
    Mf = ctx.build(lmax, d, d, d, coupling.ALL, band_limit=Lw, bin_edges=edges).cpu().numpy()
    for s, nm in enumerate(ALLN):
        a, b = Md[:, s], Mf[:, s]
        if nm in ("TT", "EE", "EEBB"):
            m = np.abs(b) > 1e-280
            assert np.all(a[~m] == 0.0), nm
            e = float(np.max(np.abs(a[m] - b[m]) / np.abs(b[m])))
        else:
            e = float(np.max(np.abs(a - b)) / np.max(np.abs(b)))
        print("df 8000 binned %s vs fp64: %.3g" % (nm, e))
        assert e <= TOL, (nm, e)


def test_lmax_limit_10000_sampled(ctx):
    """At CPL_DF32_LMAX (where the polarisation contractions come closest to
    FP32's exponent range): sampled pairs against the oracle, every spectrum,
    including the last rows and near-diagonal pairs."""
    lmax = 10000
    W = windows.ragged_jobs(lmaxes=(lmax,), n_win=1)[0][1]
    d = dev(W)
    M = ctx.build(lmax, d, d, d, coupling.ALL, precision=DF)
    rng = np.random.default_rng(10000)
    P = [rng.integers(2, lmax + 1, size=(1200, 2)),
         np.stack([np.full(150, lmax), rng.integers(2, lmax + 1, size=150)], axis=1),
         np.stack([d := rng.integers(2, lmax - 2, size=150), d + rng.integers(0, 3, size=150)], axis=1)]
    P = np.concatenate(P).astype(np.int32)
    l1, l2 = P[:, 0], P[:, 1]
    import torch
    got = M[:, :, torch.as_tensor(l1 - 2, device="cuda"), torch.as_tensor(l2 - 2, device="cuda")].cpu().numpy()
    assert np.all(np.isfinite(got))
    ref, sab = oracle.coupling_pairs(l1, l2, W, W, W, coupling.ALL)
    errs = per_spectrum(got, ref, sab, ALLN)
    print("df 10000 sampled vs oracle:", errs)
    assert max(errs.values()) <= TOL

