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


def test_injection_arguments():
    c = coupling.Context(0)
    with pytest.raises(coupling.CouplingError):
        c.inject_alloc_failure(-1)
    c.close()
