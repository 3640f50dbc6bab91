"""Parity of cpl_cov_gaussian (GPU) with the covariance oracle.

Bar: |Cov - Cov_oracle| <= tol * Cov_abs element by element, Cov_abs = the
same sum with every l3 term and every spectrum product in absolute value
(the error metric of the coupling matrices, reading 10), tol = 1e-11 with FP64
kernels and 1e-9 with mixed-precision kernels; the result must be exactly
symmetric.  Cases: several terms over two windows (one band-limited),
polarisation kernels, binned output, the full-sky cosmic variance, and
sampled bins of a binned covariance at l_max = 8000 with band-limited
squared-mask spectra.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import cov as oc
from paper_2602_15605_gb300 import coupling, windows

pytestmark = pytest.mark.gpu


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


def abs_scale(lmax, terms, lmin=2):
    """Cov_abs: sum_t Xi_abs |A_l1 B_l2 + A_l2 B_l1| / 2 over the upper triangle, mirrored."""
    l = np.arange(lmin, lmax + 1)
    out = np.zeros((l.size, l.size))
    for sp, W, band, A, B in terms:
        _, S = oracle.coupling_dense(lmax, W, W, W, sp, lmin=lmin, band_limit=None if band is None else [band])
        X = np.triu(S[0, 0] / (2.0 * l + 1.0)[None, :])
        X = X + np.triu(X, 1).T
        a, b = np.asarray(A)[l], np.asarray(B)[l]
        out += X * 0.5 * np.abs(np.outer(a, b) + np.outer(b, a))
    return out


def run(ctx, lmax, terms, **kw):
    t = [(sp, dev(W), band, dev(A), dev(B)) for sp, W, band, A, B in terms]
    out = ctx.cov_gaussian(lmax, t, **kw)
    ctx.sync()
    return out.cpu().numpy()


def spectra(lmax, seed):
    rng = np.random.default_rng(seed)
    l = np.arange(lmax + 1, dtype=np.float64)
    return [1e3 / (l + 10.0) ** 2 * (1 + 0.1 * rng.uniform(-1, 1, lmax + 1)) for _ in range(3)]


def terms_small(lmax):
    W1 = windows.mask_like(lmax, seed=70)
    W2 = windows.random_positive(lmax, seed=71, band=12)
    C1, C2, C3 = spectra(lmax, 3)
    return [(coupling.TT, W1, None, C1, 2 * C1), (coupling.EE, W1, None, C2, 2 * C2),
            (coupling.TE, W2, 12, C1, C3), (coupling.EEBB, W2, 12, C3, C2)]


@pytest.mark.parametrize("precision,tol", [(coupling.FP64, 1e-11), (coupling.MIXED_BF16, 1e-9)])
def test_dense_terms(ctx, precision, tol):
    lmax = 64
    T = terms_small(lmax)
    got = run(ctx, lmax, T, precision=precision)
    ref = oc.gaussian(lmax, T)
    sab = abs_scale(lmax, T)
    m = sab > 1e-280
    e = np.max(np.abs(got[m] - ref[m]) / sab[m])
    print("dense cov, precision %d: %.3g" % (precision, e))
    assert e <= tol
    assert np.all(got[~m] == 0.0)
    assert np.array_equal(got, got.T)


def test_binned(ctx):
    lmax, delta = 121, 10
    T = terms_small(lmax)[:3]
    edges = oracle.bin_edges(2, lmax, delta)
    got = run(ctx, lmax, T, bin_edges=edges)
    ref = oc.gaussian(lmax, T, bin_edges=edges)
    sab = oc.bin_cov(abs_scale(lmax, T), 2, edges)
    e = np.max(np.abs(got - ref) / sab)
    print("binned cov: %.3g" % e)
    assert e <= 1e-11
    assert np.array_equal(got, got.T)


def test_full_sky_cosmic_variance(ctx):
    lmax = 200
    W = windows.full_sky(lmax)
    C = spectra(lmax, 9)[0]
    got = run(ctx, lmax, [(coupling.TT, W, None, C, 2 * C)])
    l = np.arange(2, lmax + 1)
    want = 2 * C[2:] ** 2 / (2 * l + 1)
    assert np.max(np.abs(np.diag(got) / want - 1)) < 1e-13
    assert np.max(np.abs(got - np.diag(np.diag(got)))) == 0.0


def test_argument_errors(ctx):
    lmax = 20
    W = dev(windows.full_sky(lmax))
    C = dev(np.ones(lmax + 1))
    with pytest.raises(coupling.CouplingError):
        ctx.cov_gaussian(lmax, [(coupling.TT | coupling.EE, W, None, C, C)])
    with pytest.raises(coupling.CouplingError):
        ctx.cov_gaussian(lmax, [(coupling.EE, W, None, C, C)], lmin=0)


def test_full_size_band_limited_binned(ctx):
    """l_max = 8000, squared-mask spectra band-limited at L_cut = 64 and 512,
    TT and EE terms, Delta l = 50 bins: sampled bins against the oracle."""
    lmax = 8000
    Wa = windows.random_positive(lmax, seed=81, band=64)
    Wb = windows.random_positive(lmax, seed=82, band=512)
    C1, C2, _ = spectra(lmax, 5)
    T = [(coupling.TT, Wa, 64, C1, 2 * C1), (coupling.EE, Wb, 512, C2, 2 * C2), (coupling.EEBB, Wb, 512, C2, C2)]
    edges = oracle.bin_edges(2, lmax, 50)
    got = run(ctx, lmax, T, bin_edges=edges)
    assert np.array_equal(got, got.T)
    for (b1, b2) in ((0, 0), (3, 4), (40, 40), (100, 105), (159, 158), (20, 30)):
        r1 = np.arange(edges[b1], edges[b1 + 1])
        r2 = np.arange(edges[b2], edges[b2 + 1])
        L1, L2 = np.meshgrid(r1, r2, indexing="ij")
        lo, hi = np.minimum(L1, L2).ravel(), np.maximum(L1, L2).ravel()
        val = np.zeros(lo.size)
        sab = np.zeros(lo.size)
        for sp, W, band, A, B in T:
            M, S = oracle.coupling_pairs(lo, hi, W, W, W, sp, band_limit=[band])
            s = 0.5 * (A[lo] * B[hi] + A[hi] * B[lo])
            val += M[0, 0] / (2 * hi + 1) * s
            sab += S[0, 0] / (2 * hi + 1) * np.abs(s)
        want = val.sum() / lo.size
        scale = sab.sum() / lo.size
        if scale == 0:
            assert got[b1, b2] == 0.0
            continue
        e = abs(got[b1, b2] - want) / scale
        print("bin (%d, %d): %.3g" % (b1, b2, e))
        assert e <= 1e-11
