"""Optional window validation (cpl_ctx_validate) on the GPU: a NaN or Inf in
any window a request reads is reported as CPL_ERR_ARG naming the window and
l, before any output is written; valid inputs give bit-identical results with
and without the check."""
import numpy as np
import pytest

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


@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf])
@pytest.mark.parametrize("role", [0, 1, 2])
def test_nonfinite_window_rejected(ctx, bad, role):
    import torch
    lmax = 40
    W = [np.stack([windows.mask_like(lmax, seed=s + q) for q in range(3)]) for s in (1, 10, 20)]
    W[role][1, 17] = bad
    Wd = [dev(w) for w in W]
    out = torch.full((3, 5, lmax - 1, lmax - 1), 7.0, dtype=torch.float64, device="cuda")
    ctx.validate(True)
    try:
        with pytest.raises(coupling.CouplingError) as e:
            ctx.build(lmax, *Wd, coupling.ALL, out=out)
        assert e.value.status == 1 and "window 1" in str(e.value) and "l = 17" in str(e.value)
        assert torch.all(out == 7.0)
        host = np.full((3, 5, lmax - 1, lmax - 1), 7.0)
        with pytest.raises(coupling.CouplingError):
            ctx.build_host(lmax, *W, coupling.ALL, out=host)
        assert np.all(host == 7.0)
        with pytest.raises(coupling.CouplingError):
            ctx.build_batch([dict(lmax=lmax, W_tt=Wd[0], W_tp=Wd[1], W_pp=Wd[2], spectra=coupling.ALL)],
                            outs=[out])
        assert torch.all(out == 7.0)
    finally:
        ctx.validate(False)


def test_valid_windows_identical_with_and_without_check(ctx):
    lmax = 60
    W = dev(np.stack([windows.mask_like(lmax, seed=5), windows.mask_like(lmax, seed=6)]))
    a = ctx.build(lmax, W, W, W, coupling.ALL).cpu().numpy()
    ctx.validate(True)
    try:
        b = ctx.build(lmax, W, W, W, coupling.ALL).cpu().numpy()
        m = ctx.build(lmax, W, W, W, coupling.ALL, precision=coupling.MIXED_BF16).cpu().numpy()
    finally:
        ctx.validate(False)
    m0 = ctx.build(lmax, W, W, W, coupling.ALL, precision=coupling.MIXED_BF16).cpu().numpy()
    assert np.array_equal(a, b) and np.array_equal(m, m0)


def test_covariance_window_checked(ctx):
    lmax = 30
    Wt = windows.mask_like(lmax, seed=2)
    Wt[5] = np.nan
    C = dev(np.ones(lmax + 1))
    ctx.validate(True)
    try:
        with pytest.raises(coupling.CouplingError):
            ctx.cov_gaussian(lmax, [(coupling.TT, dev(Wt), None, C, C)])
    finally:
        ctx.validate(False)
