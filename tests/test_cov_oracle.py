"""Pins of the approximate-covariance oracle (oracle/cov.py), all on CPU.

- Full sky (squared-mask spectrum W~ = 4 pi delta_l0): Xi = delta / (2l + 1),
  so the TT auto term gives the textbook cosmic variance 2 C_l^2 / (2l + 1)
  on the diagonal and zero elsewhere; the same for EE, and EE->BB vanishes.
- Binned full sky: Var(C_b) = (1/|b|^2) sum_{l in b} 2 C_l^2 / (2l + 1).
- Partial sky, white spectra: sum_l2 (2 l2 + 1) Cov_{l1 l2} = 2 C^2 w4 on rows
  with complete l3 ranges, w4 = (1/4pi) sum_l (2l + 1) W~_l the sky mean of the
  squared-mask product (3j orthogonality over l2).  Returning M instead of
  Xi, or Xi transposed, fails it.
- Cov is exactly symmetric and linear in its terms.
"""
import math

import numpy as np

from oracle import cov as oc
from paper_2602_15605_gb300 import windows

TT, TE, EE, EEBB, EB = 1, 2, 4, 8, 16


def test_full_sky_cosmic_variance():
    lmax = 40
    W = windows.full_sky(lmax)
    l = np.arange(lmax + 1, dtype=np.float64)
    C = 1.0 / (l + 1.0) ** 2
    for sp in (TT, EE):
        cov = oc.gaussian(lmax, [(sp, W, None, C, 2 * C)])
        ll = l[2:]
        want = np.diag(2.0 * C[2:] ** 2 / (2 * ll + 1))
        assert np.max(np.abs(cov - want)) <= 1e-15 * np.max(want), sp
    assert np.max(np.abs(oc.kernel(lmax, W, EEBB))) < 1e-17


def test_binned_full_sky_variance():
    lmax, delta = 41, 5
    W = windows.full_sky(lmax)
    l = np.arange(lmax + 1, dtype=np.float64)
    C = 1.0 + 0.1 * np.sin(l)
    edges = list(range(2, lmax + 1, delta)) + [lmax + 1]
    covb = oc.gaussian(lmax, [(TT, W, None, C, 2 * C)], bin_edges=edges)
    for b in range(len(edges) - 1):
        ls = np.arange(edges[b], edges[b + 1])
        want = np.sum(2 * C[ls] ** 2 / (2 * ls + 1)) / len(ls) ** 2
        assert abs(covb[b, b] - want) <= 1e-14 * want
    assert np.max(np.abs(covb - np.diag(np.diag(covb)))) < 1e-18


def test_white_spectrum_row_sums_give_w4():
    lmax, Lw = 70, 10
    W = windows.random_positive(lmax, seed=12, band=Lw)
    w4 = np.sum((2 * np.arange(W.size) + 1) * W) / (4 * math.pi)
    N = 1.7
    C = np.full(lmax + 1, N)
    for sp in (TT,):
        cov = oc.gaussian(lmax, [(sp, W, Lw, C, 2 * C)])
        l2 = np.arange(2, lmax + 1)
        rows = (cov * (2 * l2 + 1)[None, :]).sum(axis=1)
        inner = slice(Lw, lmax - Lw - 1)
        assert np.max(np.abs(rows[inner] / (2 * N * N * w4) - 1.0)) < 1e-12
    # EE + EE->BB kernels together satisfy the same identity
    e = oc.kernel(lmax, W, EE, band_limit=Lw) + oc.kernel(lmax, W, EEBB, band_limit=Lw)
    rows = (e * (2 * np.arange(2, lmax + 1) + 1)[None, :]).sum(axis=1)
    assert np.max(np.abs(rows[Lw:lmax - Lw - 1] / w4 - 1.0)) < 1e-12


def test_symmetry_and_linearity():
    lmax = 30
    W1 = windows.random_positive(lmax, seed=2)
    W2 = windows.random_positive(lmax, seed=3, band=8)
    rng = np.random.default_rng(0)
    A, B, D = (rng.uniform(0.5, 1.5, size=lmax + 1) for _ in range(3))
    c1 = oc.gaussian(lmax, [(TT, W1, None, A, B)])
    c2 = oc.gaussian(lmax, [(TE, W2, 8, B, D)])
    c12 = oc.gaussian(lmax, [(TT, W1, None, A, B), (TE, W2, 8, B, D)])
    assert np.array_equal(c12, c12.T) and np.array_equal(c1, c1.T)
    assert np.max(np.abs(c12 - (c1 + c2))) <= 1e-15 * np.max(np.abs(c12))
