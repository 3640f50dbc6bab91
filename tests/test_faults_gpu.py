"""Host-side fault injection (GPU): allocation failures injected through the
context hook surface as CPL_ERR_OOM with the output untouched, and the same
context then builds correctly (caches freed by the failure are rebuilt).
No test here faults, traps or stalls the GPU."""
import numpy as np
import pytest

from paper_2602_15605_gb300 import coupling, windows

pytestmark = pytest.mark.gpu


def dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _sweep(build_fn, ref, max_n):
    """Fail the n-th allocation of a fresh context for n = 1, 2, ...; until the
    build needs fewer than n allocations, each must fail cleanly and leave the
    context usable."""
    import torch
    failures = 0
    for n in range(1, max_n + 1):
        c = coupling.Context(0)
        try:
            c.inject_alloc_failure(n)
            out = torch.full(ref.shape, 7.0, dtype=torch.float64, device="cuda")
            try:
                build_fn(c, out)
                c.sync()
                ok = True
            except coupling.CouplingError as e:
                ok = False
                assert e.status == 3, e          # CPL_ERR_OOM
                assert "injected" in str(e)
                torch.cuda.synchronize()
                assert torch.all(out == 7.0)     # untouched
                failures += 1
            c.inject_alloc_failure(0)
            build_fn(c, out)                     # the same context recovers
            c.sync()
            assert np.array_equal(out.cpu().numpy(), ref), n
        finally:
            c.close()
        if ok:
            break
    return failures


def test_fp64_allocation_failures():
    lmax = 90
    Wt, Wc, Wp = (dev(windows.gaussian_taper(lmax, s)) for s in (3, 4, 5))
    c = coupling.Context(0)
    ref = c.build(lmax, Wt, Wc, Wp, coupling.ALL).cpu().numpy()
    c.close()
    n = _sweep(lambda c, out: c.build(lmax, Wt, Wc, Wp, coupling.ALL, out=out), ref, 12)
    assert n >= 3   # tables, tile list, weights, metadata: several allocations fail in turn


def test_mixed_allocation_failures():
    lmax = 140
    W = dev(np.stack([windows.mask_like(lmax, seed=90 + q) for q in range(3)]))
    c = coupling.Context(0)
    ref = c.build(lmax, W, W, W, coupling.ALL, precision=coupling.MIXED_BF16).cpu().numpy()
    c.close()
    n = _sweep(lambda c, out: c.build(lmax, W, W, W, coupling.ALL, precision=coupling.MIXED_BF16, out=out),
               ref, 20)
    assert n >= 6   # tables, double-float tables, B cache (3), arena, error word, ticket, plan metadata


def test_mixed_host_split_allocation_failures():
    # cpl_build_host into page-locked memory with three window-role groups:
    # one build per group, copies overlapped with the later groups.  A failure
    # in any group's build must leave the host buffer untouched (every build is
    # queued before any copy), and the context must recover.
    import torch
    lmax = 120
    Wt, Wc, Wp = (windows.mask_like(lmax, seed=s) for s in (11, 12, 13))
    c = coupling.Context(0)
    ref = c.build(lmax, dev(Wt), dev(Wc), dev(Wp), coupling.ALL, precision=coupling.MIXED_BF16).cpu().numpy()
    c.close()
    failures = 0
    for n in range(1, 40):
        c = coupling.Context(0)
        try:
            c.inject_alloc_failure(n)
            host = torch.full(ref.shape, 7.0, dtype=torch.float64, pin_memory=True).numpy()
            try:
                c.build_host(lmax, Wt, Wc, Wp, coupling.ALL, precision=coupling.MIXED_BF16, out=host)
                ok = True
            except coupling.CouplingError as e:
                ok = False
                assert e.status == 3, e          # CPL_ERR_OOM
                assert np.all(host == 7.0)       # untouched
                failures += 1
            c.inject_alloc_failure(0)
            c.build_host(lmax, Wt, Wc, Wp, coupling.ALL, precision=coupling.MIXED_BF16, out=host)
            assert np.array_equal(host, ref), n
        finally:
            c.close()
        if ok:
            break
    assert failures >= 5   # staging, tables, B cache, arena, plan metadata of the group builds


def test_df32_allocation_failures():
    lmax = 90
    Wt, Wc, Wp = (dev(windows.gaussian_taper(lmax, s)) for s in (6, 7, 8))
    c = coupling.Context(0)
    ref = c.build(lmax, Wt, Wc, Wp, coupling.ALL, precision=coupling.DF32).cpu().numpy()
    c.close()
    n = _sweep(lambda c, out: c.build(lmax, Wt, Wc, Wp, coupling.ALL, precision=coupling.DF32, out=out), ref, 12)
    assert n >= 4   # tables, double-float tables, tile list, weights, metadata


def test_decouple_allocation_failures():
    # n = 300 with 3 right-hand sides: the refined solver's workspace is allocated
    import torch
    rng = np.random.default_rng(2)
    n = 300
    M = dev(rng.normal(size=(2, 3, n, n)) + 3 * n ** 0.5 * np.eye(n))
    pcl = dev(rng.normal(size=(2, 3, 3, n)))
    sp = coupling.TT | coupling.EE | coupling.EEBB
    c = coupling.Context(0)
    ref = c.decouple(M, pcl, sp).cpu().numpy()
    c.close()
    n_fail = _sweep(lambda c, out: c.decouple(M, pcl, sp, out=out), ref, 4)
    assert n_fail >= 1


def test_cov_allocation_failures():
    lmax = 80
    W1 = dev(windows.mask_like(lmax, seed=4))
    W2 = dev(windows.random_positive(lmax, seed=5, band=10))
    C = dev(1.0 / (np.arange(lmax + 1) + 5.0) ** 2)
    terms = [(coupling.TT, W1, None, C, 2 * C), (coupling.EE, W2, 10, C, C)]
    c = coupling.Context(0)
    ref = c.cov_gaussian(lmax, terms).cpu().numpy()
    c.close()
    n = _sweep(lambda c, out: c.cov_gaussian(lmax, terms, out=out), ref, 16)
    assert n >= 4   # scratch, tables, tiles, weights and metadata of two builds


def test_injection_arguments():
    c = coupling.Context(0)
    with pytest.raises(coupling.CouplingError):
        c.inject_alloc_failure(-1)
    c.close()
