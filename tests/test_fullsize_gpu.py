"""Full-size parity of the mixed-precision path (GPU): the large workloads,
launched as bench.py launches them, checked against the CPU oracle on
sampled outputs it can compute one by one.

- 36 cross-window spectra at l_max = 4000, all spin blocks (one request);
- the ragged batch of 8 jobs, l_max 1000 .. 10000, 4 windows each, run as one
  cpl_build_batch (persistent GEMM, CUDA graph);
- 16 band-limited windows at l_max = 8000 with Delta l = 50 band powers:
  selected bins against the binned oracle, every bin against the FP64 path.

Bar: 1e-9 in the oracle's S_abs metric for the mixed path; bins that the
band limits make zero are exactly 0.
"""
import numpy as np
import pytest

import oracle
from paper_2602_15605_gb300 import coupling, windows
from parity_util import per_spectrum

pytestmark = pytest.mark.gpu
TOL = 1e-9
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


def pairs_for(lmax, seed, n_random=300):
    """Random pairs, near-diagonal pairs, pairs across the l1 = 32 boundary
    of the FP64 band, and pairs on the last row and column."""
    rng = np.random.default_rng(seed)
    p = [rng.integers(2, lmax + 1, size=(n_random, 2))]
    l1 = rng.integers(2, lmax - 2, size=60)
    p.append(np.stack([l1, l1 + rng.integers(0, 3, size=60)], axis=1))
    l1 = rng.integers(29, 36, size=40)
    p.append(np.stack([l1, rng.integers(29, lmax + 1, size=40)], axis=1))
    l2 = rng.integers(2, lmax + 1, size=40)
    p.append(np.stack([np.full(40, lmax), l2], axis=1))
    P = np.concatenate(p).astype(np.int32)
    return P[:, 0], P[:, 1]


def gather(M, l1, l2, lmin=2):
    import torch
    a = torch.as_tensor(l1 - lmin, device=M.device, dtype=torch.long)
    b = torch.as_tensor(l2 - lmin, device=M.device, dtype=torch.long)
    return M[:, :, a, b].cpu().numpy()


def test_36_windows_4000_sampled(ctx):
    lmax = 4000
    W = windows.mask_pairs(lmax)
    d = dev(W)
    M = ctx.build(lmax, d, d, d, coupling.ALL, precision=coupling.MIXED_BF16)
    ctx.sync()
    l1, l2 = pairs_for(lmax, seed=41, n_random=200)
    got = gather(M, l1, l2)
    ref, sab = oracle.coupling_pairs(l1, l2, W, W, W, coupling.ALL)
    errs = per_spectrum(got, ref, sab, ALLN)
    print("36 windows, 4000:", errs)
    assert max(errs.values()) <= TOL, errs


def test_ragged_batch_full_size_sampled(ctx):
    jobs_w = windows.ragged_jobs()
    jobs = []
    for lm, W in jobs_w:
        d = dev(W)
        jobs.append(dict(lmax=lm, W_tt=d, W_tp=d, W_pp=d, spectra=coupling.ALL, precision=coupling.MIXED_BF16))
    outs = ctx.build_batch(jobs)
    outs = ctx.build_batch(jobs, outs=outs)   # the graph replay
    ctx.sync()
    for q, ((lm, W), M) in enumerate(zip(jobs_w, outs)):
        l1, l2 = pairs_for(lm, seed=500 + q, n_random=150)
        got = gather(M, l1, l2)
        ref, sab = oracle.coupling_pairs(l1, l2, W, W, W, coupling.ALL)
        errs = per_spectrum(got, ref, sab, ALLN)
        print("batch job l_max=%d:" % lm, errs)
        assert max(errs.values()) <= TOL, (lm, errs)


def test_band_limited_8000_binned(ctx):
    lmax = 8000
    W, Lw = windows.band_limited(lmax)
    edges = oracle.bin_edges(2, lmax, 50)
    nb = len(edges) - 1
    d = dev(W)
    Mm = ctx.build(lmax, d, d, d, coupling.ALL, band_limit=Lw, bin_edges=edges,
                   precision=coupling.MIXED_BF16).cpu().numpy()
    Mp = ctx.build(lmax, d, d, d, coupling.ALL, band_limit=Lw, bin_edges=edges).cpu().numpy()
    ctx.sync()
    # every bin against the FP64 path: TT, EE, EE->BB have non-negative terms
    for s, nm in enumerate(ALLN):
        a, b = Mm[:, s], Mp[:, s]
        if nm in ("TT", "EE", "EEBB"):
            m = np.abs(b) > 1e-280
            assert np.all(a[~m] == 0.0), nm
            e = np.max(np.abs(a[m] - b[m]) / np.abs(b[m]))
        else:
            e = np.max(np.abs(a - b)) / np.max(np.abs(b))
        assert e <= TOL, (nm, e)
    # selected bins against the oracle: on the diagonal, next to it, and one
    # beyond every band limit (exactly zero)
    for (b1, b2) in ((3, 3), (40, 41), (120, 119), (60, 75)):
        r1 = np.arange(edges[b1], edges[b1 + 1])
        r2 = np.arange(edges[b2], edges[b2 + 1])
        L1, L2 = np.meshgrid(r1, r2, indexing="ij")
        ref, sab = oracle.coupling_pairs(L1.ravel(), L2.ravel(), W, W, W, coupling.ALL, band_limit=Lw)
        rb = ref.sum(axis=-1) / len(r1)
        sb = sab.sum(axis=-1) / len(r1)
        got = Mm[:, :, b1, b2]
        if np.all(sb == 0):
            assert np.all(got == 0.0), (b1, b2)
            continue
        m = sb > 1e-280
        e = np.max(np.abs(got[m] - rb[m]) / sb[m])
        print("bin (%d, %d): %.3g" % (b1, b2, e))
        assert e <= TOL, (b1, b2, e)
    assert nb == 160
