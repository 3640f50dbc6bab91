"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these compare the oracle with itself: the references are the exact
Racah sum (rational arithmetic), the paper's closed form for the squared
(0 0 0) symbol (Eq. 000_sq_main with g of Eq. gdef), the paper's Appendix B
reductions of the (0,-2,2) symbol evaluated independently at 40 digits, and
identities of the assembled matrices (full sky, constant window, column sums,
linearity, band-limit exactness).  The last test plants mistakes in the
oracle and checks that each one trips at least one pin.
"""
import math
import os
import random
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import racah
from paper_2602_15605_gb300 import windows

mp = pytest.importorskip("mpmath")

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "threej_sq_exact.txt")


# ---------------------------------------------------------------- Racah itself
def test_racah_special_values():
    # (l l 0; m -m 0) = (-1)^(l-m) / sqrt(2l+1)
    for l in range(0, 12):
        for m in range(-l, l + 1):
            s, sq = racah.threej_exact(l, l, 0, m, -m, 0)
            assert sq == Fraction(1, 2 * l + 1)
            assert s == (-1) ** ((l - m) % 2)


def test_racah_symmetries():
    rnd = random.Random(5)
    for _ in range(60):
        j1, j2 = rnd.randint(0, 12), rnd.randint(0, 12)
        j3 = rnd.randint(abs(j1 - j2), j1 + j2)
        m1 = rnd.randint(-j1, j1)
        m2 = rnd.randint(max(-j2, -j3 - m1), min(j2, j3 - m1))
        m3 = -m1 - m2
        J = j1 + j2 + j3
        s0, q0 = racah.threej_exact(j1, j2, j3, m1, m2, m3)
        # cyclic permutation: unchanged (Eq. permutation)
        assert racah.threej_exact(j2, j3, j1, m2, m3, m1) == (s0, q0)
        # odd permutation and m-flip: factor (-1)^J (Eq. mflip)
        s1, q1 = racah.threej_exact(j2, j1, j3, m2, m1, m3)
        assert q1 == q0 and s1 == s0 * (-1) ** (J % 2)
        s2, q2 = racah.threej_exact(j1, j2, j3, -m1, -m2, -m3)
        assert q2 == q0 and s2 == s0 * (-1) ** (J % 2)


def test_racah_orthogonality_exact():
    # sum_j3 (2 j3 + 1) (j1 j2 j3; m1 m2 m3)^2 = 1 for fixed m1, m2
    for (j1, j2, m1, m2) in [(3, 5, 0, 0), (4, 4, -2, 2), (7, 2, 1, -1), (9, 11, -2, 2), (6, 6, 0, 0)]:
        tot = Fraction(0)
        for j3 in range(abs(j1 - j2), j1 + j2 + 1):
            tot += (2 * j3 + 1) * racah.threej_exact(j1, j2, j3, m1, m2, -m1 - m2)[1]
        assert tot == 1
    # sum over m1, m2 at fixed j3, m3: (2 j3 + 1) sum (..)^2 = 1
    for (j1, j2, j3, m3) in [(3, 4, 5, 0), (5, 5, 2, 1)]:
        tot = Fraction(0)
        for m1 in range(-j1, j1 + 1):
            m2 = -m1 - m3
            if abs(m2) <= j2:
                tot += racah.threej_exact(j1, j2, j3, m1, m2, m3)[1]
        assert (2 * j3 + 1) * tot == 1


def test_000_closed_form_equals_racah():
    # Eq. 000_sq_main with Eq. gdef, exactly, against the Racah sum
    for j1 in range(0, 16):
        for j2 in range(0, 16):
            for j3 in range(abs(j1 - j2), j1 + j2 + 1):
                assert racah.threej000_sq_closed(j1, j2, j3) == racah.threej_exact(j1, j2, j3, 0, 0, 0)[1]


def test_g_definition_and_recurrence():
    # Eq. gdef, Eq. g_rec and the Stirling asymptote g ~ (pi p)^(-1/2)
    assert racah.g_exact(0) == 1
    assert racah.g_exact(1) == Fraction(1, 2)
    assert racah.g_exact(2) == Fraction(3, 8)
    for p in range(1, 300):
        assert racah.g_exact(p) == (Fraction(2 * p - 1, 2 * p)) * racah.g_exact(p - 1)
    for p in (100, 1000, 10000):
        rel = float(racah.g_exact(p)) * math.sqrt(math.pi * p) - 1.0
        assert abs(rel + 1.0 / (8 * p)) < 1.0 / (8 * p) * 0.01 + 1e-12


def test_golden_file_matches_racah():
    n = 0
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        a, b, c, m1, m2, m3, s, sq = line.split()
        got = racah.threej_exact(int(a), int(b), int(c), int(m1), int(m2), int(m3))
        assert got == (int(s), Fraction(sq))
        n += 1
    assert n >= 40


# ---------------------------------------------------------------- S-G oracle
def test_oracle_column_vs_golden():
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        l1, l2, l3, m1, m2, m3, s, sq = line.split()
        l1, l2, l3, m1, m2 = int(l1), int(l2), int(l3), int(m1), int(m2)
        want = int(s) * math.sqrt(float(Fraction(sq)))
        # (l1 l2 l3; m1 m2 0) = (l3 l1 l2; 0 m1 m2) (cyclic)
        jmin, col = oracle.threej_column(l1, l2, 0, m1, m2)
        got = col[l3 - jmin] if jmin <= l3 <= l1 + l2 else 0.0
        assert abs(got - want) < 2e-15


def test_oracle_vs_racah_all_small():
    worst = 0.0
    for l1 in range(0, 25):
        for l2 in range(0, 25):
            for (m1, m2) in ((0, 0), (-2, 2)):
                if abs(m1) > l1 or abs(m2) > l2:
                    continue
                jmin, col = oracle.threej_column(l1, l2, 0, m1, m2)
                for k, l3 in enumerate(range(jmin, l1 + l2 + 1)):
                    ex = racah.threej_float(l3, l1, l2, 0, m1, m2)
                    worst = max(worst, abs(col[k] - ex))
    assert worst < 1e-14


def test_oracle_vs_racah_random_to_40():
    rnd = random.Random(11)
    for _ in range(80):
        l1, l2 = rnd.randint(2, 40), rnd.randint(2, 40)
        jmin, col = oracle.threej_column(l1, l2, 0, -2, 2)
        jmin0, col0 = oracle.threej_column(l1, l2, 0, 0, 0)
        for l3 in rnd.sample(range(jmin, l1 + l2 + 1), min(5, l1 + l2 + 1 - jmin)):
            assert abs(col[l3 - jmin] - racah.threej_float(l1, l2, l3, -2, 2, 0)) < 1e-14
            assert abs(col0[l3 - jmin0] - racah.threej_float(l1, l2, l3, 0, 0, 0)) < 1e-14


def test_oracle_000_large_l_vs_closed_form():
    # Eq. 000_sq_main evaluated exactly at l up to 6000
    rnd = random.Random(3)
    for _ in range(12):
        l1, l2 = rnd.randint(1000, 6000), rnd.randint(2, 6000)
        jmin, col = oracle.threej_column(l1, l2, 0, 0, 0)
        for l3 in rnd.sample(range(jmin, l1 + l2 + 1), 4):
            ex = racah.threej000_sq_closed(l1, l2, l3)
            got = col[l3 - jmin] ** 2
            if ex == 0:
                assert got < 1e-300
            else:
                assert abs(got / float(ex) - 1.0) < 1e-12


def _mp000(j1, j2, j3):
    """(j1 j2 j3; 0 0 0) at 40 digits: sign (-1)^(J/2) times the root of the
    exact square of Eq. 000_sq_main."""
    sq = racah.threej000_sq_closed(j1, j2, j3)
    if sq == 0:
        return mp.mpf(0)
    J = j1 + j2 + j3
    return (-1) ** ((J // 2) % 2) * mp.sqrt(mp.mpf(sq.numerator) / mp.mpf(sq.denominator))


def _mp000_lg(j1, j2, j3):
    """The same as _mp000 from log-gamma values of Eq. 000_sq_main's
    factorials (fast at large j; 40 digits)."""
    J = j1 + j2 + j3
    if J % 2 or j3 < abs(j1 - j2) or j3 > j1 + j2:
        return mp.mpf(0)
    g = J // 2
    lf = lambda n: mp.loggamma(n + 1)
    sq = mp.exp(lf(J - 2 * j1) + lf(J - 2 * j2) + lf(J - 2 * j3) - lf(J + 1)
                + 2 * (lf(g) - lf(g - j1) - lf(g - j2) - lf(g - j3)))
    return (-1) ** (g % 2) * mp.sqrt(sq)


def _paper_022(j1, j2, j3, f000=None):
    """(j1 j2 j3; 0 -2 2) from the paper's Appendix B at 40 digits.

    Even J: Eq. 022_linear_closedform with alpha, beta of App. B.3.
    Odd J: Eq. 022_rearranged with the (0,-1,1) symbols of Eq. joneodd
    (at j3) and Eq. joneevenshifted (at j3 + 1); the (0 0 0) term vanishes.
    f000 evaluates (0 0 0) symbols (default: the exact closed form).
    """
    _mp000 = f000 or globals()["_mp000"]
    J = j1 + j2 + j3
    Jm, Jp, Jq = -j1 + j2 + j3, j1 - j2 + j3, j1 + j2 - j3
    lam = mp.sqrt(mp.mpf(j2 * (j2 + 1) * (j3 + 1) * (j3 + 2)))
    eta = mp.sqrt(mp.mpf((j2 - 1) * (j2 + 2) * (j3 - 1) * j3))
    if J % 2 == 0:
        alpha = lam + 2 * lam / j2 * (1 - mp.mpf((J + 2) * (Jm + 1)) / (2 * (j2 + 1) * (j3 + 1)))
        prod = (J + 2) * (Jm + 1) * (Jp + 1) * Jq * (J + 3) * (Jm + 2) * (Jp + 2) * (Jq - 1)
        beta = mp.sqrt(mp.mpf(max(prod, 0))) / (2 * lam)
        return (alpha * _mp000(j1, j2, j3) + beta * _mp000(j1, j2, j3 + 2)) / eta
    big = mp.mpf((J + 2) * (Jm + 1) * (Jp + 1) * Jq)
    j11_here = -mp.sqrt(big / (j2 * (j2 + 1) * j3 * (j3 + 1))) / 2 * _mp000(j1, j2, j3 + 1)
    j11_next = (mp.sqrt(mp.mpf((j2 + 1) * (j3 + 2)) / (j2 * (j3 + 1))) * _mp000(j1, j2, j3 + 1)
                + mp.sqrt(mp.mpf((J + 3) * (J + 4) * (Jm + 2) * (Jm + 3)) /
                          (j2 * (j2 + 1) * (j3 + 1) * (j3 + 2))) / 2 * _mp000(j1, j2 + 1, j3 + 2))
    return (2 * mp.sqrt(mp.mpf(j3 * (j3 + 2))) * j11_here - mp.sqrt(big) * j11_next) / eta


def test_paper_appendix_b_helper_matches_racah():
    # the 40-digit evaluation of the paper's formulas is itself right
    mp.mp.dps = 40
    for (l1, l2, l3) in [(2, 2, 0), (2, 2, 3), (3, 5, 4), (5, 3, 7), (7, 9, 3), (10, 12, 15), (4, 4, 8), (6, 11, 6)]:
        ex = racah.threej_float(l3, l1, l2, 0, -2, 2)
        assert abs(float(_paper_022(l3, l1, l2)) - ex) < 1e-15


def test_oracle_pol_large_l_vs_paper_appendix_b():
    mp.mp.dps = 40
    rnd = random.Random(17)
    worst = 0.0
    for _ in range(8):
        l1, l2 = rnd.randint(500, 3000), rnd.randint(500, 3000)
        jmin, col = oracle.threej_column(l1, l2, 0, -2, 2)
        for l3 in rnd.sample(range(jmin, l1 + l2 + 1), 4):
            ref = _paper_022(l3, l1, l2)
            scale = float(mp.sqrt(1 / mp.mpf(2 * max(l1, l2) + 1)))
            worst = max(worst, abs(col[l3 - jmin] - float(ref)) / scale)
    assert worst < 1e-12


def test_oracle_pol_diagonal_small_odd_j_large_l():
    # On the diagonal (j2 = j3) the recursion's lower end is j = 0, where the
    # odd-j symbols are smallest; relative accuracy there, against App. B at
    # 40 digits and the closed forms of (0 l l; 0 m -m) and (1 l l; 0 m -m)
    mp.mp.dps = 40
    for l in (5000, 12000, 20000, 30000):
        jmin, col = oracle.threej_column(l, l, 0, -2, 2)
        assert jmin == 0
        sgn = -1.0 if l % 2 else 1.0                      # (-1)^(l - m), m = -2
        assert abs(col[0] / (sgn / math.sqrt(2 * l + 1)) - 1.0) < 1e-12
        assert abs(col[1] / (sgn * -2.0 / math.sqrt(l * (l + 1.0) * (2 * l + 1))) - 1.0) < 1e-12
        for j in (3, 5):
            ref = float(_paper_022(j, l, l))
            assert abs(col[j] / ref - 1.0) < 1e-12, (l, j, col[j], ref)


def test_oracle_m11_diagonal_small_odd_j_large_l():
    # the same lower end for (j l l; 0 -1 1): closed forms at j = 0, 1 and
    # App. B's Eq. joneodd at 40 digits for odd j
    mp.mp.dps = 40
    for l in (8000, 25000):
        jmin, col = oracle.threej_column(l, l, 0, -1, 1)
        assert jmin == 0
        sgn = 1.0 if (l + 1) % 2 == 0 else -1.0           # (-1)^(l - m), m = -1
        assert abs(col[0] / (sgn / math.sqrt(2 * l + 1)) - 1.0) < 1e-12
        assert abs(col[1] / (sgn * -1.0 / math.sqrt(l * (l + 1.0) * (2 * l + 1))) - 1.0) < 1e-12
        for j in (3, 7):
            ref = float(_paper_011(j, l, l))
            assert abs(col[j] / ref - 1.0) < 1e-12, (l, j, col[j], ref)


def test_oracle_eebb_diagonal_element_vs_40_digits():
    # A whole l3 sum where the odd-j symbols carry the weight: M^EEBB(l, l)
    # with a mask-like window (weight concentrated at small l3), against the
    # App. A sum evaluated with App. B's symbols at 40 digits
    mp.mp.dps = 40
    lmax, l = 10000, 9000
    W = windows.mask_like(lmax, seed=lmax)
    ref, _ = oracle.coupling_pairs(np.array([l], np.int32), np.array([l], np.int32), W, W, W, oracle.EEBB)
    tot = mp.mpf(0)
    for l3 in range(1, 2 * l + 1, 2):   # odd L = 2 l + l3
        if W[l3] == 0.0:
            continue
        tot += (2 * l3 + 1) * mp.mpf(W[l3]) * _paper_022(l3, l, l, f000=_mp000_lg) ** 2
    want = (2 * l + 1) * tot / (4 * mp.pi)
    assert abs(float(ref[0, 0, 0] / want) - 1.0) < 1e-12


def _paper_011(j1, j2, j3):
    """(j1 j2 j3; 0 -1 1) from the paper's Appendix B at 40 digits: Eq. joneeven
    (two (0 0 0) symbols) for even J, Eq. joneodd for odd J."""
    J = j1 + j2 + j3
    Jm, Jp, Jq = -j1 + j2 + j3, j1 - j2 + j3, j1 + j2 - j3
    den = mp.mpf(j2 * (j2 + 1) * j3 * (j3 + 1))
    if J % 2 == 0:
        return (mp.sqrt(mp.mpf((j2 + 1) * (j3 + 1)) / (j2 * j3)) * _mp000(j1, j2, j3)
                + mp.sqrt(mp.mpf((J + 2) * (J + 3) * (Jm + 1) * (Jm + 2)) / den) / 2 * _mp000(j1, j2 + 1, j3 + 1))
    return -mp.sqrt(mp.mpf((J + 2) * (Jm + 1) * (Jp + 1) * Jq) / den) / 2 * _mp000(j1, j2, j3 + 1)


def test_oracle_m11_vs_racah_all_small():
    # the (0,-1,1) configuration of the lensing / aberration weights
    worst = 0.0
    for j2 in range(1, 21):
        for j3 in range(1, 21):
            jmin, col = oracle.threej_column(j2, j3, 0, -1, 1)
            for k, j1 in enumerate(range(jmin, j2 + j3 + 1)):
                worst = max(worst, abs(col[k] - racah.threej_float(j1, j2, j3, 0, -1, 1)))
    assert worst < 1e-14


def test_paper_m11_helper_matches_racah():
    mp.mp.dps = 40
    for (j1, j2, j3) in [(0, 1, 1), (1, 1, 1), (2, 1, 1), (3, 2, 4), (4, 2, 4), (5, 7, 3), (9, 6, 8), (12, 10, 5)]:
        assert abs(float(_paper_011(j1, j2, j3)) - racah.threej_float(j1, j2, j3, 0, -1, 1)) < 1e-15


def test_oracle_m11_large_l_vs_paper_appendix_b():
    mp.mp.dps = 40
    rnd = random.Random(23)
    worst = 0.0
    for _ in range(8):
        j2, j3 = rnd.randint(300, 3000), rnd.randint(300, 3000)
        jmin, col = oracle.threej_column(j2, j3, 0, -1, 1)
        for j1 in rnd.sample(range(jmin, j2 + j3 + 1), 4):
            ref = _paper_011(j1, j2, j3)
            scale = float(mp.sqrt(1 / mp.mpf(2 * max(j2, j3) + 1)))
            worst = max(worst, abs(col[j1 - jmin] - float(ref)) / scale)
    assert worst < 1e-12


# ---------------------------------------------------------------- matrices
def _dense(lmax, W, spectra, lmin=2, **kw):
    return oracle.coupling_dense(lmax, W, W, W, spectra, lmin=lmin, **kw)


def test_full_sky_is_identity():
    lmax = 40
    W = windows.full_sky(lmax)
    M, _ = _dense(lmax, W, oracle.TT | oracle.TE | oracle.EE | oracle.EEBB | oracle.EB)
    I = np.eye(lmax - 1)
    for s, want in zip(range(5), (I, I, I, 0 * I, I)):
        assert np.max(np.abs(M[0, s] - want)) < 1e-13


def test_constant_window_row_values():
    lmax = 48
    W = windows.constant(lmax)
    M, _ = _dense(lmax, W, oracle.TT | oracle.EE | oracle.EEBB)
    l2 = np.arange(2, lmax + 1)
    assert np.max(np.abs(M[0, 0] / (2 * l2 + 1)[None, :] - 1.0)) < 1e-12
    assert np.max(np.abs((M[0, 1] + M[0, 2]) / (2 * l2 + 1)[None, :] - 1.0)) < 1e-12


def test_column_sum_identity():
    # sum_l2 M[l1][l2] = (1/4pi) sum_l3 (2 l3 + 1) W_l3 for band-limited W
    lmax, Lw = 64, 16
    W = windows.random_positive(lmax, seed=9, band=Lw)
    target = np.sum((2 * np.arange(W.size) + 1) * W) / (4 * math.pi)
    M, _ = _dense(lmax, W, oracle.TT, lmin=0)
    rows = M[0, 0].sum(axis=1)
    assert np.max(np.abs(rows[: lmax - Lw + 1] / target - 1.0)) < 1e-12
    P, _ = _dense(lmax, W, oracle.EE | oracle.EEBB, lmin=2)
    prow = (P[0, 0] + P[0, 1]).sum(axis=1)
    assert np.max(np.abs(prow[: lmax - Lw - 1] / target - 1.0)) < 1e-12


def test_linearity_in_window():
    lmax = 30
    W1 = windows.random_positive(lmax, seed=1)
    W2 = windows.random_positive(lmax, seed=2)
    sp = oracle.TT | oracle.TE | oracle.EE | oracle.EEBB | oracle.EB
    a, b = 0.7, -1.3
    M1, _ = _dense(lmax, W1, sp)
    M2, _ = _dense(lmax, W2, sp)
    M12, S = _dense(lmax, a * W1 + b * W2, sp)
    assert np.max(np.abs(M12 - (a * M1 + b * M2)) / (S + 1e-300)) < 1e-13


def test_band_limit_is_exact():
    lmax, Lw = 60, 12
    W = windows.random_positive(lmax, seed=4, band=Lw)
    sp = oracle.TT | oracle.TE | oracle.EE | oracle.EEBB
    M0, _ = _dense(lmax, W, sp)
    M1, _ = _dense(lmax, W, sp, band_limit=[Lw])
    assert np.array_equal(M0, M1)


def test_eb_is_ee_minus_eebb():
    lmax = 30
    W = windows.random_positive(lmax, seed=8)
    M, _ = _dense(lmax, W, oracle.EE | oracle.EEBB | oracle.EB)
    assert np.max(np.abs(M[0, 2] - (M[0, 0] - M[0, 1]))) < 1e-15


def test_binning_definition():
    rng = np.random.default_rng(0)
    M = rng.normal(size=(2, 17, 17))
    e1 = oracle.bin_edges(2, 18, 1)
    assert np.allclose(oracle.bin_matrix(M, 2, e1), M)
    e = oracle.bin_edges(2, 18, 5)
    B = oracle.bin_matrix(M, 2, e)
    sizes = np.diff(e)
    # sum_b |b| M_bb' summed over b' equals the full sum of M
    assert np.allclose((B * sizes[:, None]).sum(axis=(-1, -2)), M.sum(axis=(-1, -2)))
    assert B.shape[-1] == 4 and sizes[-1] == 2


# ---------------------------------------------------------------- planted mistakes
# Each mistake is planted in a copy of the oracle's source (one expression
# replaced), compiled on its own; the oracle itself carries no switches.
MISTAKES = {
    # drop the (2 l3 + 1) weight of the l3 sum
    "drop_2l3p1": [("const double wt = 2.0 * l3 + 1.0;", "const double wt = 1.0;")],
    # 2j instead of 2j + 1 in B(j) of the recursion
    "b_weight": [("double w = 2.0 * j + 1.0;", "double w = 2.0 * j;")],
    # (2 l1 + 1) instead of (2 l2 + 1) as the prefactor
    "prefactor_l1": [("const double pref = 2.0 * l2 + 1.0;", "const double pref = 2.0 * l1 + 1.0;")],
    # the parity projectors swapped: EE takes odd L, EE->BB even L
    "swap_parity": [("(bit == ORC_EE)   s = even ? p * p : 0.0;", "(bit == ORC_EE)   s = !even ? p * p : 0.0;"),
                    ("(bit == ORC_EEBB) s = !even ? p * p : 0.0;", "(bit == ORC_EEBB) s = even ? p * p : 0.0;"),
                    ("s = even ? p * p : -p * p;", "s = !even ? p * p : -p * p;")],
    # the orthogonality normalisation skipped
    "no_normalise": [("double c = 1.0 / sqrt(norm);", "double c = 1e-3;")],
}


@pytest.fixture(scope="module")
def mutant_dir(tmp_path_factory):
    return str(tmp_path_factory.mktemp("oracle_mutants"))


def _mutant(name, where):
    src = open(oracle.SOURCE).read()
    for old, new in MISTAKES[name]:
        assert src.count(old) == 1, (name, old)    # the planted site exists exactly once
        src = src.replace(old, new)
    path = os.path.join(where, name + ".c")
    with open(path, "w") as f:
        f.write(src)
    return oracle.load_library(oracle.compile_source(path, os.path.join(where, "lib" + name + ".so")))


def _pins_pass(library=None):
    lmax = 32
    sp = oracle.TT | oracle.TE | oracle.EE | oracle.EEBB | oracle.EB
    ok = True
    M, _ = oracle.coupling_dense(lmax, *([windows.full_sky(lmax)] * 3), spectra=sp, library=library)
    I = np.eye(lmax - 1)
    ok &= all(np.max(np.abs(M[0, s] - w)) < 1e-12 for s, w in zip(range(5), (I, I, I, 0 * I, I)))
    M, _ = oracle.coupling_dense(lmax, *([windows.constant(lmax)] * 3), spectra=oracle.TT | oracle.EE | oracle.EEBB,
                                 library=library)
    l2 = np.arange(2, lmax + 1)
    ok &= np.max(np.abs(M[0, 0] / (2 * l2 + 1) - 1)) < 1e-12
    ok &= np.max(np.abs((M[0, 1] + M[0, 2]) / (2 * l2 + 1) - 1)) < 1e-12
    # a few direct symbol checks against Racah through the matrix: TE, EE at one pair
    W = windows.random_positive(lmax, seed=3)
    M, _ = oracle.coupling_pairs([5], [9], W, W, W, oracle.TE | oracle.EE, library=library)
    ref_te = sum((2 * l3 + 1) * W[l3] * racah.threej_float(5, 9, l3, 0, 0, 0) *
                 racah.threej_float(5, 9, l3, -2, 2, 0) for l3 in range(4, 15) if (14 + l3) % 2 == 0)
    ref_ee = sum((2 * l3 + 1) * W[l3] * racah.threej_float(5, 9, l3, -2, 2, 0) ** 2
                 for l3 in range(4, 15) if (14 + l3) % 2 == 0)
    ok &= abs(M[0, 0, 0] - 19 * ref_te / (4 * math.pi)) < 1e-13
    ok &= abs(M[0, 1, 0] - 19 * ref_ee / (4 * math.pi)) < 1e-13
    return bool(ok)


def test_pins_pass_on_the_oracle():
    assert _pins_pass()


@pytest.mark.parametrize("name", sorted(MISTAKES))
def test_planted_mistake_is_caught(name, mutant_dir):
    assert not _pins_pass(_mutant(name, mutant_dir))
