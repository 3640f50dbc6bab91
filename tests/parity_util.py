"""Shared helpers of the GPU parity tests: the per-element error metric.

e = max over elements with S_abs > tiny of |M_gpu - M_oracle| / S_abs,
where S_abs = (2 l2 + 1)/(4 pi) sum |(2 l3 + 1) W S_X| is returned by the
oracle (for TT, EE and EE->BB every term is >= 0, so this is the plain
relative error; for TE and EB it avoids dividing by cancellations).
Elements the parity or band selection makes exactly zero (S_abs == 0) must
be exactly 0 on the GPU.
"""
import numpy as np

TINY = 1e-280


def rel_err(gpu, ref, sabs):
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    sabs = np.asarray(sabs, dtype=np.float64)
    assert gpu.shape == ref.shape == sabs.shape, (gpu.shape, ref.shape, sabs.shape)
    assert np.all(np.isfinite(gpu)), "non-finite GPU output"
    zero = sabs == 0
    if np.any(zero):
        assert np.all(gpu[zero] == 0.0), "elements zero by selection are not exactly 0"
    m = sabs > TINY
    if not np.any(m):
        return 0.0
    return float(np.max(np.abs(gpu[m] - ref[m]) / sabs[m]))


def per_spectrum(gpu, ref, sabs, names):
    """{name: error} over axis 1 (spectrum) of [n_win, nspec, ...] arrays."""
    return {nm: rel_err(gpu[:, s], ref[:, s], sabs[:, s]) for s, nm in enumerate(names)}


def sample_pairs(lmax, lmin=2, n_random=20000, seed=12345, band=8):
    """Sampled (l1, l2) pairs for full-size checks: every pair with
    |l1 - l2| <= band, the rows l1 in {lmin, lmin+1, lmax/2, lmax} and
    n_random uniform pairs."""
    rng = np.random.default_rng(seed)
    ls = np.arange(lmin, lmax + 1)
    pairs = set()
    for l1 in ls:
        for d in range(-band, band + 1):
            l2 = l1 + d
            if lmin <= l2 <= lmax:
                pairs.add((int(l1), int(l2)))
    for l1 in (lmin, lmin + 1, (lmin + lmax) // 2, lmax):
        for l2 in ls:
            pairs.add((int(l1), int(l2)))
    r = rng.integers(lmin, lmax + 1, size=(n_random, 2))
    for a, b in r:
        pairs.add((int(a), int(b)))
    p = np.array(sorted(pairs), dtype=np.int32)
    return p[:, 0], p[:, 1]
