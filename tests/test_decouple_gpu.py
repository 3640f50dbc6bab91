"""Parity of cpl_decouple (GPU) with the decoupling oracle.

Bar, per system K x = b of Eq. pseudo_cl (the EE/BB one as its 2n x 2n
block matrix):
  forward error  max|x - x_oracle| / max|x_oracle| <= 8 n eps cond_inf(K)
  backward error max|K x - b| / (|K|_inf max|x| + max|b|) <= 8 n eps
(both are the textbook bounds of LU with partial pivoting, with a small
growth factor; eps = 2^-53).  Cases: dense and binned coupling matrices from
the oracle, shared-memory and global-workspace sizes on both sides of the
switch, several right-hand sides, n = 1 and n = CPL_DECOUPLE_NMAX, singular
systems, and the full-size binned workload (16 band-limited windows,
l_max = 8000, Delta l = 50) checked through the backward error.
"""
import numpy as np
import pytest

import oracle
from oracle import decouple as dc
from paper_2602_15605_gb300 import coupling, windows

pytestmark = pytest.mark.gpu
EPS = 2.0 ** -53
ALL = coupling.ALL


@pytest.fixture(scope="module")
def ctx():
    from paper_2602_15605_gb300 import build_ext
    build_ext.build()
    c = coupling.Context(0)
    yield c
    c.close()


def dev(a, dtype=None):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype or torch.float64, device="cuda")


def systems(M, pcl, x, spectra):
    """(K, b, x) of every system of Eq. pseudo_cl, the EE/BB one as a block matrix."""
    f = dc.fields(spectra)
    slots = [b for b in (1, 2, 4, 8, 16) if spectra & b]
    out = []
    for w in range(M.shape[0]):
        for bit, name in ((1, "TT"), (2, "TE"), (16, "EB")):
            if spectra & bit:
                K = M[w, slots.index(bit)]
                out.append((K, pcl[w, :, f.index(name)].T, x[w, :, f.index(name)].T))
        if spectra & 4:
            A, B = M[w, slots.index(4)], M[w, slots.index(8)]
            K = np.block([[A, B], [B, A]])
            ie, ib = f.index("EE"), f.index("BB")
            out.append((K, np.concatenate([pcl[w, :, ie], pcl[w, :, ib]], axis=1).T,
                        np.concatenate([x[w, :, ie], x[w, :, ib]], axis=1).T))
    return out


def check(M, pcl, got, spectra, ref=None):
    worst_f = worst_b = 0.0
    for q, (K, b, x) in enumerate(systems(M, pcl, got, spectra)):
        n = K.shape[0]
        bw = np.max(np.abs(K @ x - b)) / (np.max(np.abs(K).sum(axis=1)) * np.max(np.abs(x)) + np.max(np.abs(b)))
        assert bw <= 8 * n * EPS, (q, bw)
        worst_b = max(worst_b, bw / (n * EPS))
        if ref is not None:
            xr = systems(M, pcl, ref, spectra)[q][2]
            fe = np.max(np.abs(x - xr)) / np.max(np.abs(xr))
            kappa = np.linalg.cond(K, np.inf)
            assert fe <= 8 * n * EPS * kappa, (q, fe, kappa)
            worst_f = max(worst_f, fe / (n * EPS * kappa))
    return worst_f, worst_b


def run(ctx, M, pcl, spectra):
    import torch
    info = torch.full((M.shape[0], coupling.decouple_systems(spectra)), -7, dtype=torch.int32, device="cuda")
    out = ctx.decouple(dev(M), dev(pcl), spectra, info=info)
    ctx.sync()
    return out.cpu().numpy(), info.cpu().numpy()


def test_dense_small_all_spectra(ctx):
    lmax = 40
    W = np.stack([windows.mask_like(lmax, seed=60 + q) for q in range(3)])
    M = np.concatenate([oracle.coupling_dense(lmax, W[q], W[q], W[q], ALL)[0] for q in range(3)])
    rng = np.random.default_rng(11)
    pcl = rng.uniform(0.1, 1.0, size=(3, 4, 5, lmax - 1))
    got, info = run(ctx, M, pcl, ALL)
    assert np.all(info == 0)
    print("dense 39:", check(M, pcl, got, ALL, dc.decouple(M, pcl, ALL)))


@pytest.mark.parametrize("lmax,delta,n_rhs", [(300, 5, 1), (300, 1, 3), (161, 1, 1), (161, 1, 20)])
def test_binned_and_dense_sizes(ctx, lmax, delta, n_rhs):
    # n = 60 (shared memory), 299 (global), 160 with one right-hand side
    # (shared memory, 206 KB) and with 20 (global)
    W = windows.mask_like(lmax, seed=90)
    sp = coupling.TT | coupling.EE | coupling.EEBB | coupling.EB
    Md = oracle.coupling_dense(lmax, W, W, W, sp)[0]
    edges = oracle.bin_edges(2, lmax, delta)
    M = oracle.bin_matrix(Md, 2, edges) if delta > 1 else Md
    n = M.shape[-1]
    rng = np.random.default_rng(n + n_rhs)
    pcl = rng.uniform(0.1, 1.0, size=(1, n_rhs, 4, n))
    got, info = run(ctx, M, pcl, sp)
    assert np.all(info == 0)
    print("n=%d rhs=%d:" % (n, n_rhs), check(M, pcl, got, sp, dc.decouple(M, pcl, sp)))


def test_piecewise_constant_recovery(ctx):
    lmax, delta = 200, 10
    W = windows.mask_like(lmax, seed=5)
    M = oracle.coupling_dense(lmax, W, W, W, ALL)[0]
    edges = oracle.bin_edges(2, lmax, delta)
    nb = len(edges) - 1
    rng = np.random.default_rng(3)
    Cb = rng.uniform(0.2, 1.0, size=(1, 2, 5, nb))
    pcb = dc.bin_vector(dc.forward(M, np.repeat(Cb, np.diff(edges), axis=-1), ALL), 2, edges)
    got, info = run(ctx, oracle.bin_matrix(M, 2, edges), pcb, ALL)
    assert np.all(info == 0)
    assert np.max(np.abs(got - Cb) / Cb) < 1e-11


@pytest.mark.parametrize("n", [1, 2, 1024])
def test_generic_matrices_edge_sizes(ctx, n):
    # G + 3 sqrt(n) I (condition number <= 5 for Gaussian G), rows permuted so
    # that partial pivoting has to find every pivot away from the diagonal
    rng = np.random.default_rng(n)
    sp = coupling.TT | coupling.TE
    M = rng.normal(size=(2, 2, n, n)) + np.eye(n) * (3.0 * n ** 0.5)
    for w in range(2):
        for s_ in range(2):
            M[w, s_] = M[w, s_][rng.permutation(n)]
    pcl = rng.normal(size=(2, 2, 2, n))
    got, info = run(ctx, M, pcl, sp)
    assert np.all(info == 0)
    print("n=%d:" % n, check(M, pcl, got, sp, dc.decouple(M, pcl, sp)))


def test_ill_conditioned_system_falls_back_to_fp64(ctx):
    # Hilbert matrix, cond ~ 5e11: the FP32 factors carry no digit, so the
    # refinement cannot converge and the FP64 solver answers (backward error bar)
    n = 9
    H = 1.0 / (np.arange(n)[:, None] + np.arange(n)[None, :] + 1.0)
    rng = np.random.default_rng(4)
    pcl = rng.normal(size=(1, 1, 1, n))
    got, info = run(ctx, H[None, None], pcl, coupling.TT)
    assert np.all(info == 0)
    print("hilbert 9:", check(H[None, None], pcl, got, coupling.TT))


@pytest.mark.parametrize("scale", [1e200, 1e-200])
def test_matrices_outside_fp32_range(ctx, scale):
    # entries beyond FP32's range: the refined solver's FP32 factors fail and
    # the FP64 solver answers; the result scales exactly with 1 / scale
    lmax = 60
    W = windows.mask_like(lmax, seed=17)
    M = oracle.coupling_dense(lmax, W, W, W, coupling.TT)[0]
    rng = np.random.default_rng(5)
    pcl = rng.uniform(0.1, 1.0, size=(1, 1, 1, lmax - 1))
    got, info = run(ctx, M * scale, pcl, coupling.TT)
    assert np.all(info == 0)
    print("scale %g:" % scale, check(M * scale, pcl, got, coupling.TT, dc.decouple(M * scale, pcl, coupling.TT)))


def test_refined_and_fp64_solvers_agree(ctx):
    # n_rhs <= 2n/9 takes the refined solver, more right-hand sides the FP64
    # one: the first right-hand side must agree to the forward-error bar
    lmax = 161
    W = windows.mask_like(lmax, seed=31)
    sp = coupling.TT | coupling.EE | coupling.EEBB
    M = oracle.coupling_dense(lmax, W, W, W, sp)[0]
    rng = np.random.default_rng(7)
    pcl = rng.uniform(0.1, 1.0, size=(1, 100, 3, 160))
    many, _ = run(ctx, M, pcl, sp)
    one, _ = run(ctx, M, np.ascontiguousarray(pcl[:, :1]), sp)
    ref = dc.decouple(M, pcl[:, :1], sp)
    print("refined:", check(M, pcl[:, :1], one, sp, ref), "fp64:", check(M, pcl[:, :1], many[:, :1], sp, ref))


@pytest.mark.parametrize("n,cond", [(96, 1e5), (96, 1e6), (160, 1e5)])
def test_many_rhs_residual_updates(ctx, n, cond):
    # From 8 right-hand sides the first residual runs on the FP64 and FP32
    # pipes at once (FP64 chains for some right-hand sides, error-free
    # triple-float products for the others: 4 + 5 of them a thread at
    # n = 96, 5 + 6 at n = 160), and the later ones are updates r - K d in
    # double-float.  Matrices with a set condition number (U diag(s) V^T, s
    # log-spaced) make the refinement take several update steps (cond 2^-24
    # per step); one right-hand side is zero (no correction), one tiny.  The
    # answer must meet the forward and backward bars, and agree with the
    # single-right-hand-side solves (FP64 residuals throughout) to the
    # forward bar.
    R = 32
    rng = np.random.default_rng(int(np.log10(cond)) + n)
    M = np.empty((1, 1, n, n))
    U, _ = np.linalg.qr(rng.normal(size=(n, n)))
    V, _ = np.linalg.qr(rng.normal(size=(n, n)))
    M[0, 0] = (U * np.logspace(0, -np.log10(cond), n)) @ V.T
    pcl = rng.normal(size=(1, R, 1, n))
    pcl[0, 3] = 0.0
    pcl[0, 7] *= 1e-250
    got, info = run(ctx, M, pcl, coupling.TT)
    assert np.all(info == 0)
    assert np.all(got[0, 3] == 0.0)
    ref = dc.decouple(M, pcl, coupling.TT)
    print("cond %.0e:" % cond, check(M, pcl, got, coupling.TT, ref))
    kappa = np.linalg.cond(M[0, 0], np.inf)
    for r in (0, 7, 31):
        one, _ = run(ctx, M, np.ascontiguousarray(pcl[:, r:r + 1]), coupling.TT)
        fe = np.max(np.abs(one[0, 0] - got[0, r])) / np.max(np.abs(one[0, 0]))
        assert fe <= 8 * n * EPS * kappa, (r, fe)


def test_many_rhs_tiny_norm_uses_fp64_residuals(ctx):
    # Below |K|_inf = 2^-40 the FP32 parts of K no longer carry it exactly,
    # so the solver keeps every residual in FP64 there: a coupling matrix
    # scaled by 1e-20 with 32 right-hand sides meets the bars, and its
    # solution scales exactly with 1 / scale against the unscaled solve.
    lmax = 161
    W = windows.mask_like(lmax, seed=41)
    M = oracle.coupling_dense(lmax, W, W, W, coupling.TT)[0]
    rng = np.random.default_rng(9)
    pcl = rng.uniform(0.1, 1.0, size=(1, 32, 1, lmax - 1))
    scale = 1e-20
    got, info = run(ctx, M * scale, pcl, coupling.TT)
    assert np.all(info == 0)
    ref = dc.decouple(M * scale, pcl, coupling.TT)
    print("tiny norm:", check(M * scale, pcl, got, coupling.TT, ref))
    one, _ = run(ctx, M, pcl, coupling.TT)
    n = lmax - 1
    kappa = np.linalg.cond(M[0, 0], np.inf)
    fe = np.max(np.abs(got * scale - one)) / np.max(np.abs(one))
    assert fe <= 8 * n * EPS * kappa, fe


def test_singular_systems_report_info(ctx):
    n = 12
    sp = coupling.TT | coupling.EE | coupling.EEBB
    rng = np.random.default_rng(8)
    M = rng.normal(size=(2, 3, n, n)) + 4 * np.eye(n)
    M[0, 0] = 0.0                       # TT of window 0: first pivot is zero
    M[1, 2] = M[1, 1]                   # window 1: EE - EEBB = 0 (EE + EEBB = 2 EE stays regular)
    pcl = rng.normal(size=(2, 1, 3, n))
    got, info = run(ctx, M, pcl, sp)
    assert info[0, 0] == 1 and np.all(np.isnan(got[0, :, 0]))
    assert info[0, 1] == 0 and info[0, 2] == 0
    assert info[1, 0] == 0 and info[1, 2] == 1
    assert np.all(np.isnan(got[1, :, 1:3]))      # EE and BB share the failed difference system
    assert np.all(np.isfinite(got[0, :, 1:3])) and np.all(np.isfinite(got[1, :, 0]))


def test_argument_errors(ctx):
    import torch
    M = torch.zeros((1, 1, 4, 4), dtype=torch.float64, device="cuda")
    p = torch.zeros((1, 1, 2, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(coupling.CouplingError):
        ctx.decouple(M, p, coupling.EE)                      # EE without EE->BB (rejected by the library)
    big = torch.zeros((1, 1, 1025, 1025), dtype=torch.float64, device="cuda")
    with pytest.raises(coupling.CouplingError):
        ctx.decouple(big, torch.zeros((1, 1, 1, 1025), dtype=torch.float64, device="cuda"), coupling.TT)


def test_full_size_binned_band_limited(ctx):
    """The binned coupling matrices of 16 band-limited windows at l_max = 8000
    (Delta l = 50, 160 bins, all spectra), decoupled for 8 right-hand sides:
    backward error of every system at the full size."""
    import torch
    lmax = 8000
    W, Lw = windows.band_limited(lmax)
    edges = oracle.bin_edges(2, lmax, 50)
    d = dev(W)
    M = ctx.build(lmax, d, d, d, ALL, band_limit=Lw, bin_edges=edges, precision=coupling.MIXED_BF16)
    rng = np.random.default_rng(12)
    pcl = rng.uniform(0.1, 1.0, size=(16, 8, 5, len(edges) - 1))
    info = torch.full((16, 5), -7, dtype=torch.int32, device="cuda")
    out = ctx.decouple(M, dev(pcl), ALL, info=info)
    ctx.sync()
    assert np.all(info.cpu().numpy() == 0)
    print("full size:", check(M.cpu().numpy(), pcl, out.cpu().numpy(), ALL))
