"""cpl_build_noalloc: the build for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc at all: their own allocator owns the
device memory budget, or they must not take the device synchronisation an
allocation can cause.  The entry point therefore keeps its scratch (the g / h
lookup tables and the window weights) in a fixed device array inside the
library instead of buffers a context allocates.  These tests call it through
the C ABI and check:

- two calls in a row against cpl_build on the same inputs, at the plain
  path's tolerance (1e-11): element by element for TT, EE and EE->BB, whose
  l3 terms are all non-negative, and normwise for the signed TE and EB, whose
  elements can cancel to near zero (the two paths form the pair coefficients
  differently, so they agree to rounding, not bit for bit);
- a whole matrix, and sampled pairs of the largest layout the array holds
  (l_max 4096, 4 windows, separate W^TT, W^TP, W^PP: ~0.92 MiB of the 1 MiB),
  against the CPU oracle in its S_abs metric at 1e-11;
- the polarisation-only kernel (EE->BB alone) with an odd lmin, and a TE-only
  request with lmin = 5, against cpl_build;
- that a call after the first leaves the device's free memory unchanged;
- that sizes beyond the array's limits and pointers the kernels cannot
  dereference (host memory) are refused before any work is queued.

This file is collected last on purpose, so a failure here comes after every
other test has run.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2602_15605_gb300 import coupling, windows
from parity_util import per_spectrum, sample_pairs

pytestmark = pytest.mark.gpu
TOL = 1e-11
ALLN = ["TT", "TE", "EE", "EEBB", "EB"]


def dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


SIGNED = (1, 4)   # TE and EB slots of the full spectrum set


def close(a, b, signed=SIGNED):
    a = a.cpu().numpy()
    b = b.cpu().numpy()
    assert a.shape == b.shape
    assert np.all(np.isfinite(a))
    zero = b == 0
    assert np.all(a[zero] == 0.0)
    for w in range(b.shape[0]):
        for s in range(b.shape[1]):
            scale = np.max(np.abs(b[w, s])) or 1.0
            if s in signed:
                rel = np.max(np.abs(a[w, s] - b[w, s])) / scale
            else:
                rel = np.max(np.abs(a[w, s] - b[w, s]) / np.maximum(np.abs(b[w, s]), 1e-300 * scale))
            assert rel <= TOL, (w, s, rel)


@pytest.fixture(scope="module")
def ctx():
    from paper_2602_15605_gb300 import build_ext
    build_ext.build()
    c = coupling.Context(0)
    yield c
    c.close()


def test_two_calls_match_cpl_build(ctx):
    import torch
    # call 1: full spin set from three separate windows
    lmax = 300
    Wt, Wc, Wp = (dev(windows.gaussian_taper(lmax, s)) for s in (2, 3, 4))
    got1 = coupling.build_noalloc(lmax, Wt, Wc, Wp, coupling.ALL)
    want1 = ctx.build(lmax, Wt, Wc, Wp, coupling.ALL)
    # call 2, right after: a different size, two shared windows, band limits
    lmax2 = 517
    W2 = dev(np.stack([windows.random_positive(lmax2, seed=5, band=90),
                       windows.random_positive(lmax2, seed=6, band=400)]))
    got2 = coupling.build_noalloc(lmax2, W2, W2, W2, coupling.ALL, band_limit=[90, 400])
    want2 = ctx.build(lmax2, W2, W2, W2, coupling.ALL, band_limit=[90, 400])
    torch.cuda.synchronize()
    close(got1, want1)
    close(got2, want2)


def test_whole_matrix_against_the_oracle():
    import torch
    lmax = 160
    Wt = np.stack([windows.gaussian_taper(lmax, s) for s in (11, 12)])
    Wc = np.stack([windows.gaussian_taper(lmax, s) for s in (13, 14)])
    Wp = np.stack([windows.gaussian_taper(lmax, s) for s in (15, 16)])
    got = coupling.build_noalloc(lmax, dev(Wt), dev(Wc), dev(Wp), coupling.ALL)
    torch.cuda.synchronize()
    ref, sab = oracle.coupling_dense(lmax, Wt, Wc, Wp, coupling.ALL)
    err = per_spectrum(got.cpu().numpy(), ref, sab, ALLN)
    assert max(err.values()) <= TOL, err


def test_largest_layout_sampled_against_the_oracle():
    # l_max 4096 x 4 windows x 3 separate roles: the weights fill ~0.79 MiB
    # of the array after the ~0.13 MiB of tables
    import torch
    lmax = 4096
    Wt = np.stack([windows.gaussian_taper(lmax, 20 + q) for q in range(4)])
    Wc = np.stack([windows.gaussian_taper(lmax, 30 + q) for q in range(4)])
    Wp = np.stack([windows.gaussian_taper(lmax, 40 + q) for q in range(4)])
    got = coupling.build_noalloc(lmax, dev(Wt), dev(Wc), dev(Wp), coupling.ALL)
    torch.cuda.synchronize()
    l1, l2 = sample_pairs(lmax, n_random=3000, band=2)
    a = torch.as_tensor(l1 - 2, device="cuda", dtype=torch.long)
    b = torch.as_tensor(l2 - 2, device="cuda", dtype=torch.long)
    g = got[:, :, a, b].cpu().numpy()
    del got
    ref, sab = oracle.coupling_pairs(l1, l2, Wt, Wc, Wp, coupling.ALL)
    err = per_spectrum(g, ref, sab, ALLN)
    assert max(err.values()) <= TOL, err


def test_polarisation_only_and_odd_lmin(ctx):
    import torch
    lmax = 400
    Wp = dev(np.stack([windows.gaussian_taper(lmax, s) for s in (7, 8, 9)]))
    got = coupling.build_noalloc(lmax, None, None, Wp, coupling.EEBB, lmin=3)
    want = ctx.build(lmax, None, None, Wp, coupling.EEBB, lmin=3)
    Wc = dev(windows.gaussian_taper(lmax, 10))
    got_te = coupling.build_noalloc(lmax, None, Wc, None, coupling.TE, lmin=5)
    want_te = ctx.build(lmax, None, Wc, None, coupling.TE, lmin=5)
    torch.cuda.synchronize()
    close(got, want, signed=())
    close(got_te, want_te, signed=(0,))


def test_no_device_memory_taken():
    import torch
    lmax = 1000
    W = dev(np.stack([windows.mask_like(lmax, seed=s) for s in (1, 2)]))
    out = torch.empty((2, 5, lmax - 1, lmax - 1), dtype=torch.float64, device="cuda")
    coupling.build_noalloc(lmax, W, W, W, coupling.ALL, out=out)   # loads the kernels
    first = out.clone()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    coupling.build_noalloc(lmax, W, W, W, coupling.ALL, out=out)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0, (free0, free1)
    assert torch.equal(out, first)   # deterministic


def _raw_call(lmax, W_ptr, out_ptr, n_windows, w_len):
    """cpl_build_noalloc through the C ABI with raw addresses (TT only)."""
    L = coupling.load()
    L.cpl_build_noalloc.argtypes = [ctypes.POINTER(coupling.Request), ctypes.c_void_p, ctypes.c_void_p]
    r = coupling.Request()
    r.lmax, r.lmin, r.n_windows, r.w_len = lmax, 2, n_windows, w_len
    r.W_tt = W_ptr
    r.spectra, r.precision = coupling.TT, coupling.FP64
    return L.cpl_build_noalloc(ctypes.byref(r), ctypes.c_void_p(out_ptr), ctypes.c_void_p(0))


def test_pointers_outside_device_memory_are_refused():
    import torch
    lmax = 50
    Wh = np.ascontiguousarray(windows.mask_like(lmax, seed=3))          # host (pageable) memory
    Wd = dev(Wh)
    out = torch.full((lmax - 1, lmax - 1), 7.0, dtype=torch.float64, device="cuda")
    out_host = np.zeros((lmax - 1, lmax - 1))
    assert _raw_call(lmax, Wh.ctypes.data, out.data_ptr(), 1, Wh.size) == 1        # CPL_ERR_ARG
    assert _raw_call(lmax, Wd.data_ptr(), out_host.ctypes.data, 1, Wh.size) == 1   # CPL_ERR_ARG
    pinned = torch.empty(Wh.size, dtype=torch.float64, pin_memory=True)
    assert _raw_call(lmax, pinned.data_ptr(), out.data_ptr(), 1, Wh.size) == 1     # page-locked host memory
    torch.cuda.synchronize()
    assert bool((out == 7.0).all())       # nothing was queued
    assert not np.any(out_host)
    assert _raw_call(lmax, Wd.data_ptr(), out.data_ptr(), 1, Wh.size) == 0
    torch.cuda.synchronize()
    assert not bool((out == 7.0).all())


def test_limits_are_refused():
    import torch
    W = dev(windows.random_positive(4097, seed=1))
    with pytest.raises(coupling.CouplingError) as e:
        coupling.build_noalloc(4097, W, None, None, coupling.TT, out=torch.empty(1, device="cuda"))
    assert e.value.status == 2
    W5 = dev(np.stack([windows.random_positive(20, seed=s) for s in range(5)]))
    with pytest.raises(coupling.CouplingError) as e:
        coupling.build_noalloc(20, W5, None, None, coupling.TT, out=torch.empty(1, device="cuda"))
    assert e.value.status == 2
