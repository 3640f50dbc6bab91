"""One representative launch of a library kernel on synthetic inputs, small
enough to profile (a few hundred MB on the device at most).

    python profile_cases.py decouple   # k_decouple: 80 systems of 160 x 160, 1 rhs
    python profile_cases.py decouple32 # k_decouple: the same systems, 32 rhs
    python profile_cases.py threej     # k_threej_m11: 4096 rows, j2, j3 in [1000, 3000]
    python profile_cases.py cov        # k_cov_combine: TT + EE terms, l_max 3000, L_cut 64
    python profile_cases.py plain_df   # k_plain_df: full spin set, l_max 3000, CPL_DF32
    python profile_cases.py mixed      # the mixed path's kernels: full spin set, l_max 3000

Each case runs its call three times (the first includes one-off set-up) and
prints the last call's event time.
"""
import sys

import numpy as np


def _event_ms(fn):
    import torch
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b)


def case_decouple(ctx, n_rhs=1):
    """The decoupling workload's shape: 16 windows x 5 systems (TT, TE, EE+EEBB,
    EE-EEBB, EB) of 160 x 160 coupling-like matrices (diagonally dominant
    with Gaussian off-diagonal entries), n_rhs right-hand sides."""
    import torch
    from paper_2602_15605_gb300 import coupling
    rng = np.random.default_rng(1)
    n = 160
    M = rng.normal(scale=0.02, size=(16, 5, n, n)) + np.eye(n)
    M[:, 3] *= 0.3                       # EE->BB smaller than EE
    pcl = rng.uniform(0.1, 1.0, size=(16, n_rhs, 5, n))
    Md = torch.as_tensor(M, device="cuda")
    pd = torch.as_tensor(pcl, device="cuda")
    out = torch.empty_like(pd)
    ms = 0.0
    for _ in range(3):
        ms = _event_ms(lambda: ctx.decouple(Md, pd, coupling.ALL, out=out))
    return ms


def case_decouple32(ctx):
    """case_decouple with 32 right-hand sides per window."""
    return case_decouple(ctx, n_rhs=32)


def case_threej(ctx):
    """(j1 j2 j3; 0 -1 1) rows for 4096 pairs (j2, j3) uniform in [1000, 3000]
    (the bench's workload), rows padded to 2 min(j2, j3) + 1."""
    import torch
    rng = np.random.default_rng(31)
    j2 = rng.integers(1000, 3001, size=4096)
    j3 = rng.integers(1000, 3001, size=4096)
    stride = int(2 * np.minimum(j2, j3).max() + 1)
    out = torch.empty((4096, stride), dtype=torch.float64, device="cuda")
    ms = 0.0
    for _ in range(3):
        ms = _event_ms(lambda: ctx.threej_m11(j2, j3, out=out, stride=stride))
    return ms


def case_cov(ctx):
    """Covariance from two Wick terms (TT and EE kernels) at l_max = 3000 with
    a squared-mask spectrum band-limited at L_cut = 64, dense output."""
    import torch
    from paper_2602_15605_gb300 import coupling, windows
    lmax, lcut = 3000, 64
    l = np.arange(lmax + 1, dtype=np.float64)
    Ct = torch.as_tensor(1e3 / (l + 10.0) ** 2, device="cuda")
    Ce = torch.as_tensor(20.0 / (l + 10.0) ** 2, device="cuda")
    W = torch.as_tensor(windows.random_positive(lmax, seed=90 + lcut, band=lcut), device="cuda")
    terms = [(coupling.TT, W, lcut, Ct, 2 * Ct), (coupling.EE, W, lcut, Ce, 2 * Ce)]
    out = torch.empty((lmax - 1, lmax - 1), dtype=torch.float64, device="cuda")
    ms = 0.0
    for _ in range(3):
        ms = _event_ms(lambda: ctx.cov_gaussian(lmax, terms, out=out))
    return ms


def case_plain_df(ctx):
    """The full spin set at l_max = 3000 from three separate windows (the
    bench's workload) in CPL_DF32: one launch per kernel variant."""
    import torch
    from paper_2602_15605_gb300 import coupling, windows
    d = [torch.as_tensor(W, device="cuda") for W in windows.full_spin_3000()]
    out = torch.empty((1, 5, 2999, 2999), dtype=torch.float64, device="cuda")
    ms = 0.0
    for _ in range(3):
        ms = _event_ms(lambda: ctx.build(3000, *d, coupling.ALL, precision=coupling.DF32, out=out))
    return ms


def case_mixed(ctx):
    """The full spin set at l_max = 3000 from three separate windows (the
    bench's workload) in CPL_MIXED_BF16."""
    import torch
    from paper_2602_15605_gb300 import coupling, windows
    d = [torch.as_tensor(W, device="cuda") for W in windows.full_spin_3000()]
    out = torch.empty((1, 5, 2999, 2999), dtype=torch.float64, device="cuda")
    ms = 0.0
    for _ in range(3):
        ms = _event_ms(lambda: ctx.build(3000, *d, coupling.ALL, precision=coupling.MIXED_BF16, out=out))
    return ms


CASES = {"decouple": case_decouple, "decouple32": case_decouple32, "threej": case_threej, "cov": case_cov, "plain_df": case_plain_df, "mixed": case_mixed}


def main(argv):
    if len(argv) != 1 or argv[0] not in CASES:
        print("usage: python profile_cases.py {%s}" % "|".join(CASES))
        return 2
    from paper_2602_15605_gb300 import build_ext, coupling
    build_ext.build()
    ctx = coupling.Context(0)
    try:
        ms = CASES[argv[0]](ctx)
        ctx.sync()
    finally:
        ctx.close()
    print("%s: %.4f ms" % (argv[0], ms))
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
