"""Seeded synthetic window power spectra W_l (inputs only).

The paper measures on the ACT DR6 survey mask (Sec. 4), whose spectrum is not
available here; these generators stand in for it with spectra shaped like
survey masks: a monopole W_0 = 4 pi f_sky^2, a steep power law and a high-l
taper.  This module holds random numbers and shapes only -- none of the
coupling arithmetic -- so the CUDA library, the CPU oracle and the benchmark
can all draw the same inputs from it.

Every generator returns float64 numpy arrays of length 2*lmax + 1 (or wider
when asked), indexed by l.
"""
import math

import numpy as np

FOUR_PI = 4.0 * math.pi


def mask_like(lmax, seed, w_len=None, amp=0.02, slope=2.5, taper=300.0, sigma=0.1,
              fsky2=0.36):
    """W_0 = 4 pi fsky2, W_l = amp (l+1)^-slope exp(-(l/taper)^2) exp(N(0, sigma^2)).

    With the defaults (fsky2 = 0.6^2) this is the single TT window of the
    l_max = 512 workload."""
    n = 2 * lmax + 1 if w_len is None else int(w_len)
    rng = np.random.default_rng(seed)
    ell = np.arange(n, dtype=np.float64)
    noise = np.exp(rng.normal(0.0, sigma, size=n))
    W = amp * (ell + 1.0) ** (-slope) * np.exp(-(ell / taper) ** 2) * noise
    W[0] = FOUR_PI * fsky2
    return W


def gaussian_taper(lmax, seed, w_len=None, amp=0.02):
    """Power law (l+1)^-a, a ~ U(2,3), times exp(-l^2 / (2 sigma_l^2)),
    sigma_l ~ U(200, 800), with W_0 = 4 pi fsky^2, fsky ~ U(0.3, 0.8)."""
    n = 2 * lmax + 1 if w_len is None else int(w_len)
    rng = np.random.default_rng(seed)
    a = rng.uniform(2.0, 3.0)
    sig = rng.uniform(200.0, 800.0)
    fsky = rng.uniform(0.3, 0.8)
    ell = np.arange(n, dtype=np.float64)
    W = amp * (ell + 1.0) ** (-a) * np.exp(-ell ** 2 / (2.0 * sig ** 2))
    W[0] = FOUR_PI * fsky ** 2
    return W


def tt_512():
    """TT only, l_max = 512: one window, seed 1, W for l = 0..1024."""
    return mask_like(512, seed=1)


def full_spin_3000(lmax=3000):
    """Separate temperature / cross / polarisation windows W^TT, W^TP, W^PP
    for the full spin-0 / spin-2 set (seeds 2, 3, 4)."""
    return tuple(gaussian_taper(lmax, s) for s in (2, 3, 4))


def mask_pairs(lmax=4000, n_masks=8, seed0=100):
    """All unordered pairs i <= j of n_masks synthetic masks (28 crosses + 8
    autos for 8 masks), each pair's spectrum drawn with seed seed0 + pair
    index.  Returns [n_pairs, 2*lmax+1]."""
    out = []
    q = 0
    for i in range(n_masks):
        for j in range(i, n_masks):
            out.append(mask_like(lmax, seed=seed0 + q))
            q += 1
    return np.stack(out)


def band_limited(lmax=8000, n_win=16, seed0=200, choice_seed=7, cuts=(64, 128, 256, 512)):
    """n_win windows with W = 0 above a per-window L_w drawn from `cuts`.
    Returns (W [n_win, 2*lmax+1], L_w [n_win])."""
    rng = np.random.default_rng(choice_seed)
    Lw = rng.choice(np.asarray(cuts), size=n_win)
    W = np.stack([mask_like(lmax, seed=seed0 + i) for i in range(n_win)])
    for i in range(n_win):
        W[i, Lw[i] + 1:] = 0.0
    return W, Lw.astype(np.int32)


RAGGED_LMAX = (1000, 2000, 3000, 4000, 6000, 8000, 9000, 10000)


def ragged_jobs(lmaxes=RAGGED_LMAX, n_win=4, seed0=300):
    """One list entry per job: (lmax, W [n_win, 2*lmax+1])."""
    jobs = []
    s = seed0
    for lm in lmaxes:
        jobs.append((lm, np.stack([mask_like(lm, seed=s + q) for q in range(n_win)])))
        s += n_win
    return jobs


def full_sky(lmax, w_len=None):
    """W_l = 4 pi delta_{l0}: an unmasked sky (coupling matrix = identity)."""
    n = 2 * lmax + 1 if w_len is None else int(w_len)
    W = np.zeros(n)
    W[0] = FOUR_PI
    return W


def constant(lmax, w_len=None, value=FOUR_PI):
    """W_l = value for every l."""
    n = 2 * lmax + 1 if w_len is None else int(w_len)
    return np.full(n, float(value))


def random_positive(lmax, seed, w_len=None, band=None):
    """Generic positive test window, optionally zero above `band`."""
    n = 2 * lmax + 1 if w_len is None else int(w_len)
    rng = np.random.default_rng(seed)
    W = rng.uniform(0.1, 1.0, size=n) * (np.arange(n) + 1.0) ** -1.5
    W[0] = rng.uniform(1.0, 10.0)
    if band is not None:
        W[band + 1:] = 0.0
    return W
