"""The tabled plain FP64 kernel (precomputed operand blocks streamed by bulk
copies) against the kernel that stages its own operands (GPU).

Both evaluate the same products in the same order, so dense outputs must
agree bit for bit; binned outputs (FP64 atomics, order not fixed) to a few
ulps.  CPL_PLAIN_TABLES=0 selects the self-staging kernel.  Cases cover
separate and shared windows, lmin = 0, band limits that cut tiles in the
middle of a chunk, a batch with two l_max (one B table for both), the B
table growing between calls, and the kernel accounting showing which kernel
ran.  Parity of the tabled kernel against the oracle is the plain path's
parity suite, which runs it by default.
"""
import os

import numpy as np
import pytest

from paper_2602_15605_gb300 import coupling, windows

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2602_15605_gb300 import build_ext
    build_ext.build()
    c = coupling.Context(0)
    c.profile(True)
    yield c
    c.close()


def dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def both(ctx, fn):
    """fn() with the tabled kernel and with the self-staging one."""
    old = os.environ.get("CPL_PLAIN_TABLES")
    try:
        os.environ.pop("CPL_PLAIN_TABLES", None)
        ctx.stats(reset=True)
        tab = fn()
        ctx.sync()
        st_tab = ctx.stats(reset=True)
        os.environ["CPL_PLAIN_TABLES"] = "0"
        ref = fn()
        ctx.sync()
        st_ref = ctx.stats(reset=True)
    finally:
        if old is None:
            os.environ.pop("CPL_PLAIN_TABLES", None)
        else:
            os.environ["CPL_PLAIN_TABLES"] = old
    launches = lambda st: st.get("plain_tables_a", {}).get("launches", 0)
    assert launches(st_tab) > 0 and launches(st_ref) == 0
    return tab, ref


def equal_bits(a, b):
    import torch
    if isinstance(a, (list, tuple)):
        return all(equal_bits(x, y) for x, y in zip(a, b))
    return torch.equal(a.view(torch.int64), b.view(torch.int64))


def test_full_spin_separate_windows_two_per_role(ctx):
    lmax = 300
    Wt = np.stack([windows.mask_like(lmax, seed=s) for s in (1, 2)])
    Wc = np.stack([windows.mask_like(lmax, seed=s) for s in (3, 4)])
    Wp = np.stack([windows.mask_like(lmax, seed=s) for s in (5, 6)])
    d = [dev(x) for x in (Wt, Wc, Wp)]
    tab, ref = both(ctx, lambda: ctx.build(lmax, *d, coupling.ALL))
    assert equal_bits(tab, ref)
    assert float(tab.abs().max()) > 0.0


def test_shared_window_tt_lmin0_ragged(ctx):
    lmax = 333   # ragged tails in i and j
    W = dev(windows.mask_like(lmax, seed=11))
    tab, ref = both(ctx, lambda: ctx.build(lmax, W, None, None, coupling.TT, lmin=0))
    assert equal_bits(tab, ref)


@pytest.mark.parametrize("spectra", [coupling.TE, coupling.EEBB, coupling.EE | coupling.EB])
def test_single_variants(ctx, spectra):
    # TE alone (3 even contractions), EE->BB alone (odd sweep only), EE + EB (6 even + odd)
    lmax = 200
    W = dev(windows.mask_like(lmax, seed=21))
    tab, ref = both(ctx, lambda: ctx.build(lmax, W, W, W, spectra))
    assert equal_bits(tab, ref)


def test_band_limits_inside_chunks(ctx):
    # caps that end in the middle of a 16-k chunk and of a tile, one window unbanded
    lmax = 400
    W = np.stack([windows.mask_like(lmax, seed=30 + q) for q in range(3)])
    band = [45, 2 * lmax, 301]
    d = dev(W)
    tab, ref = both(ctx, lambda: ctx.build(lmax, d, d, d, coupling.ALL, band_limit=band))
    assert equal_bits(tab, ref)


def test_binned_within_ulps(ctx):
    lmax = 350
    W = dev(windows.mask_like(lmax, seed=40))
    edges = list(range(2, lmax + 2, 25))
    if edges[-1] != lmax + 1:
        edges.append(lmax + 1)
    tab, ref = both(ctx, lambda: ctx.build(lmax, W, W, W, coupling.ALL, bin_edges=edges))
    t, r = tab.cpu().numpy(), ref.cpu().numpy()
    scale = np.max(np.abs(r))
    assert np.max(np.abs(t - r)) <= 1e-14 * scale


def test_batch_two_lmax_and_growing_b_table(ctx):
    W1 = dev(windows.mask_like(150, seed=50))
    W2 = dev(windows.mask_like(420, seed=51))
    jobs = [dict(lmax=150, W_tt=W1, W_tp=W1, W_pp=W1, spectra=coupling.ALL),
            dict(lmax=420, W_tt=W2, W_tp=W2, W_pp=W2, spectra=coupling.ALL)]
    tab, ref = both(ctx, lambda: ctx.build_batch(jobs))
    assert equal_bits(tab, ref)
    # a fresh context: small l_max first, then a larger one (the B table grows), then small again
    c = coupling.Context(0)
    try:
        c.profile(True)
        outs = [both(c, lambda lm=lm, W=W: c.build(lm, W, W, W, coupling.ALL))
                for lm, W in ((150, W1), (420, W2), (150, W1))]
    finally:
        c.close()
    for tab, ref in outs:
        assert equal_bits(tab, ref)
    assert equal_bits(outs[0][0], outs[2][0])


def test_launch_accounting_equals_host_plan(ctx):
    # the FLOP the profiled launches report (the roofline's numerator) equal
    # the host dry run's count, which the CPU tests pin to brute force
    lmax = 333
    W = [dev(windows.mask_like(lmax, seed=70 + q)) for q in range(3)]
    band = [40, 2 * lmax]
    Wb = [dev(np.stack([windows.mask_like(lmax, seed=80 + q), windows.mask_like(lmax, seed=90 + q)])) for q in range(3)]
    for args, kw, plan_kw in [((lmax, *W, coupling.ALL), {}, dict(n_windows=1)),
                              ((lmax, Wb[0], Wb[0], Wb[0], coupling.ALL), dict(band_limit=band),
                               dict(n_windows=2, band_limit=band, shared=True))]:
        ctx.stats(reset=True)
        ctx.build(*args, **kw)
        ctx.sync()
        st = ctx.stats(reset=True)
        flop = sum(v["flop"] for k, v in st.items() if k.startswith("plain_fp64_"))
        plan = coupling.plan_info(lmax, spectra=coupling.ALL, **plan_kw)
        assert flop == plan["flop"], (flop, plan["flop"])
        launches = sum(v["launches"] for k, v in st.items() if k.startswith("plain_fp64_"))
        assert launches == plan["n_launches"]
