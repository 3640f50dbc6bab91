"""cpl_build_noalloc: the build for callers that cannot allocate device memory.

The entry point keeps its scratch in a fixed device array inside the library
instead of buffers a context allocates.  These tests call it through the C ABI
twice in a row and compare each result with cpl_build's on the same inputs,
at the plain path's tolerance (1e-11): element by element for TT, EE and
EE->BB, whose l3 terms are all non-negative, and normwise for the signed TE
and EB, whose elements can cancel to near zero (the two paths form the pair
coefficients differently, so they agree to rounding, not bit for bit); they
also check that sizes beyond the array's limits are refused.  This file is collected last on
purpose, so a failure here comes after every other test has run.
"""
import numpy as np
import pytest

from paper_2602_15605_gb300 import coupling, windows

pytestmark = pytest.mark.gpu
TOL = 1e-11


def dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


SIGNED = (1, 4)   # TE and EB slots of the full spectrum set


def close(a, b):
    a = a.cpu().numpy()
    b = b.cpu().numpy()
    assert a.shape == b.shape
    assert np.all(np.isfinite(a))
    zero = b == 0
    assert np.all(a[zero] == 0.0)
    for w in range(b.shape[0]):
        for s in range(b.shape[1]):
            scale = np.max(np.abs(b[w, s])) or 1.0
            if s in SIGNED:
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
