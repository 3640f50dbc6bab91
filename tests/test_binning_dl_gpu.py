"""D_l band powers (bin_weight = 1) on the GPU, every precision, against the
oracle's weighted binning M_bb' = (1/|b|) sum sum l1(l1+1)/(l2(l2+1)) M.

Bars as for flat binning: 1e-11 (FP64, double-float) and 1e-9 (mixed) in the
binned S_abs metric; cases with and without a band limit (the mixed path's
l1 < 32 pairs take the band kernel's binned writes)."""
import numpy as np
import pytest

import oracle
from paper_2602_15605_gb300 import coupling, windows
from parity_util import per_spectrum

pytestmark = pytest.mark.gpu
ALLN = ["TT", "TE", "EE", "EEBB", "EB"]


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


@pytest.mark.parametrize("precision,tol", [(coupling.FP64, 1e-11), (coupling.DF32, 1e-11),
                                           (coupling.MIXED_BF16, 1e-9)])
@pytest.mark.parametrize("band", [None, 45])
def test_dl_binning(ctx, precision, tol, band):
    lmax = 180
    W = np.stack([windows.mask_like(lmax, seed=31 + q) if band is None
                  else windows.random_positive(lmax, seed=31 + q, band=band) for q in range(2)])
    edges = oracle.bin_edges(2, lmax, 11)
    d = dev(W)
    bl = None if band is None else [band, band]
    got = ctx.build(lmax, d, d, d, coupling.ALL, band_limit=bl, bin_edges=edges, bin_weight=1,
                    precision=precision).cpu().numpy()
    ref, sab = oracle.coupling_dense(lmax, W, W, W, coupling.ALL, band_limit=bl)
    errs = per_spectrum(got, oracle.bin_matrix(ref, 2, edges, weight=1),
                        oracle.bin_matrix(sab, 2, edges, weight=1), ALLN)
    print("D_l binning, precision %d, band %s:" % (precision, band), errs)
    assert max(errs.values()) <= tol, errs
    # and it differs from the flat binning
    flat = ctx.build(lmax, d, d, d, coupling.ALL, band_limit=bl, bin_edges=edges,
                     precision=precision).cpu().numpy()
    assert np.max(np.abs(flat - got)) > 1e-3 * np.max(np.abs(got))
