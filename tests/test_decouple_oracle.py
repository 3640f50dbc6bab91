"""Pins of the mode-decoupling oracle (oracle/decouple.py), all on CPU.

What fixes the decoupled spectra independently of the solver:
- full sky (W = 4 pi delta_l0): K = I and K^EEBB = 0, so decoupling is the
  identity (Sec. 2 with the full-sky limit of the kernels);
- white noise: with C = N in every field, the forward model of Eq. pseudo_cl
  gives N times the mean of the squared mask, (1/4pi) sum_l (2l+1) W_l, in
  TT, EE and BB on rows whose l3 range is complete (orthogonality of the 3j
  symbols over l2).  A transposed K, a missing EE->BB leakage term or a
  swapped block fails it;
- decoupling inverts the forward model for random spectra;
- binned: when C is constant inside each bin, decoupling the binned
  pseudo-spectra with the binned matrices returns the bin values exactly;
- the (EE + BB, EE - BB) split used by the GPU solver equals the 2n x 2n
  block solve.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import decouple as dc
from paper_2602_15605_gb300 import windows

ALL = dc.TT | dc.TE | dc.EE | dc.EEBB | dc.EB


def _dense(lmax, W, spectra, lmin=2, **kw):
    M, _ = oracle.coupling_dense(lmax, W, W, W, spectra, lmin=lmin, **kw)
    return M


def test_fields_and_validation():
    assert dc.fields(ALL) == ["TT", "TE", "EE", "BB", "EB"]
    assert dc.fields(dc.TT | dc.EB) == ["TT", "EB"]
    with pytest.raises(ValueError):
        dc.fields(dc.EE)
    with pytest.raises(ValueError):
        dc.fields(dc.TT | dc.EEBB)


def test_full_sky_decoupling_is_identity():
    lmax = 30
    M = _dense(lmax, windows.full_sky(lmax), ALL)
    rng = np.random.default_rng(1)
    pcl = rng.uniform(0.5, 2.0, size=(1, 3, 5, lmax - 1))
    assert np.max(np.abs(dc.decouple(M, pcl, ALL) - pcl)) < 1e-13


def test_white_noise_pseudo_spectrum_is_mean_squared_mask():
    lmax, Lw = 64, 12
    W = windows.random_positive(lmax, seed=21, band=Lw)
    w2 = np.sum((2 * np.arange(W.size) + 1) * W) / (4 * math.pi)
    sp = dc.TT | dc.EE | dc.EEBB
    M = _dense(lmax, W, sp)
    N = 3.5
    C = np.full((1, 1, 3, lmax - 1), N)              # TT, EE, BB
    pc = dc.forward(M, C, sp)[0, 0]
    rows = slice(Lw, lmax - Lw - 1)                  # l1 = Lw + 2 .. lmax - Lw: complete l2 ranges
    for f in range(3):
        assert np.max(np.abs(pc[f, rows] / (N * w2) - 1.0)) < 1e-12, f
    # E-only input: the leakage into BB is what completes the EE row sum
    C[0, 0, 2] = 0.0
    pc = dc.forward(M, C, sp)[0, 0]
    assert np.max(np.abs((pc[1, rows] + pc[2, rows]) / (N * w2) - 1.0)) < 1e-12
    assert np.min(pc[2, rows]) > 0.0


def _mask_windows(lmax, n):
    return np.stack([windows.mask_like(lmax, seed=40 + q) for q in range(n)])


def test_decouple_inverts_forward():
    lmax = 40
    W = _mask_windows(lmax, 2)
    M = np.concatenate([_dense(lmax, W[q], ALL) for q in range(2)])
    rng = np.random.default_rng(5)
    C = rng.uniform(0.1, 1.0, size=(2, 3, 5, lmax - 1))
    pc = dc.forward(M, C, ALL)
    got = dc.decouple(M, pc, ALL)
    assert np.max(np.abs(got - C) / np.abs(C)) < 1e-10


def test_binned_piecewise_constant_is_exact():
    lmax, delta = 62, 6
    W = windows.mask_like(lmax, seed=77)
    M = _dense(lmax, W, ALL)
    edges = oracle.bin_edges(2, lmax, delta)
    nb = len(edges) - 1
    rng = np.random.default_rng(9)
    Cb = rng.uniform(0.2, 1.0, size=(1, 2, 5, nb))
    sizes = np.diff(edges)
    C = np.repeat(Cb, sizes, axis=-1)                 # constant inside each bin
    pc = dc.forward(M, C, ALL)
    pcb = dc.bin_vector(pc, 2, edges)
    Mb = oracle.bin_matrix(M, 2, edges)
    got = dc.decouple(Mb, pcb, ALL)
    assert np.max(np.abs(got - Cb) / Cb) < 1e-11
    # a planted mistake: the transposed binned matrix does not recover the bins
    bad = dc.decouple(np.swapaxes(Mb, -1, -2), pcb, ALL)
    assert np.max(np.abs(bad - Cb) / Cb) > 1e-3


def test_sum_difference_split_equals_block_solve():
    lmax = 36
    W = windows.mask_like(lmax, seed=3)
    sp = dc.EE | dc.EEBB
    M = _dense(lmax, W, sp)
    rng = np.random.default_rng(2)
    pcl = rng.uniform(0.1, 1.0, size=(1, 4, 2, lmax - 1))
    ref = dc.decouple(M, pcl, sp)
    A, B = M[0, 0], M[0, 1]
    s = np.linalg.solve(A + B, (pcl[0, :, 0] + pcl[0, :, 1]).T).T
    t = np.linalg.solve(A - B, (pcl[0, :, 0] - pcl[0, :, 1]).T).T
    assert np.max(np.abs(0.5 * (s + t) - ref[0, :, 0]) / np.abs(ref[0, :, 0])) < 1e-11
    assert np.max(np.abs(0.5 * (s - t) - ref[0, :, 1]) / np.abs(ref[0, :, 1])) < 1e-11


def test_dl_binning_single_l_bins_and_piecewise_constant_recovery():
    # weight=1 with one multipole per bin is M l1(l1+1) / (l2(l2+1)); with
    # wider bins, spectra whose D_l = l(l+1) C_l / 2pi is constant in each bin
    # are recovered exactly as D_b from the D_l-weighted binned system
    lmax, delta = 62, 6
    W = windows.mask_like(lmax, seed=78)
    M = _dense(lmax, W, ALL)
    l = np.arange(2, lmax + 1, dtype=np.float64)
    one = oracle.bin_matrix(M, 2, oracle.bin_edges(2, lmax, 1), weight=1)
    assert np.max(np.abs(one - M * (l * (l + 1))[:, None] / (l * (l + 1))[None, :])) < 1e-15 * np.max(np.abs(M))
    edges = oracle.bin_edges(2, lmax, delta)
    rng = np.random.default_rng(19)
    Db = rng.uniform(0.2, 1.0, size=(1, 1, 5, len(edges) - 1))
    C = np.repeat(Db, np.diff(edges), axis=-1) * (2 * np.pi / (l * (l + 1)))
    pcb = dc.bin_vector(dc.forward(M, C, ALL), 2, edges, weight=1)
    got = dc.decouple(oracle.bin_matrix(M, 2, edges, weight=1), pcb, ALL)
    assert np.max(np.abs(got - Db) / Db) < 1e-11
    # the flat binning does not recover D_b from the same input
    bad = dc.decouple(oracle.bin_matrix(M, 2, edges), dc.bin_vector(dc.forward(M, C, ALL), 2, edges), ALL)
    assert np.max(np.abs(bad - Db) / Db) > 1e-3

