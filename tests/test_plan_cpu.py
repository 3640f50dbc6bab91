"""The plain path's work decomposition on the host (cpl_plan_info_fp64, no GPU).

The tile cover, the parity-selected l3 term counts, the algorithmic FLOP
behind the plain path's roofline (2 per term and separable contraction) and
the operand-table sizes are checked against direct enumeration:
- tiles: every 32 x 32 block of (i, j) = ((d - pi)/2, (s - pi)/2) that holds a
  pair lmin <= l1 <= l2 <= lmax, counted by brute force;
- terms: for every pair, the l3 of App. A's sums, l3 in [|l1 - l2|, l1 + l2]
  up to the window's band, split by the parity of l1 + l2 + l3;
- FLOP: 1, 3 or 6 contractions per even term (TT; TE; EE or anything that
  needs the polarisation expansion) and 3 per odd term, per window-role group.
"""
import numpy as np
import pytest

from paper_2602_15605_gb300 import coupling

T = 32


def tiles_brute(lmax, lmin):
    n = 0
    for pi in (0, 1):
        seen = set()
        for l1 in range(lmin, lmax + 1):
            for l2 in range(l1, lmax + 1):
                d, s = l2 - l1, l1 + l2
                if d % 2 != pi:
                    continue
                seen.add(((d - pi) // 2 // T, (s - pi) // 2 // T))
        n += len(seen)
    return n


def terms_brute(lmax, lmin, cap):
    even = odd = 0
    for l1 in range(lmin, lmax + 1):
        for l2 in range(l1, lmax + 1):
            for l3 in range(l2 - l1, min(l1 + l2, cap) + 1):
                if (l1 + l2 + l3) % 2:
                    odd += 1
                else:
                    even += 1
    return even, odd


def terms_numpy(lmax, lmin, cap):
    # the same counts in closed form per pair (for large l_max)
    l1, l2 = np.triu_indices(lmax + 1 - lmin)
    l1, l2 = l1 + lmin, l2 + lmin
    d, s = l2 - l1, l1 + l2
    hi = np.minimum(s, cap)
    ev = np.where(hi >= d, (hi - d) // 2 + 1, 0)            # l3 = d, d + 2, ... <= hi
    hio = np.minimum(s - 1, cap)
    od = np.where(hio >= d + 1, (hio - d - 1) // 2 + 1, 0)  # l3 = d + 1, d + 3, ... <= hio
    return int(ev.sum()), int(od.sum())


@pytest.mark.parametrize("lmax,lmin", [(2, 2), (5, 2), (31, 2), (40, 2), (64, 0), (97, 3), (130, 2)])
def test_tile_cover_and_terms(lmax, lmin):
    spectra = coupling.TT if lmin < 2 else coupling.ALL
    info = coupling.plan_info(lmax, 1, spectra, lmin=lmin)
    assert info["n_tiles"] == tiles_brute(lmax, lmin)
    e, o = terms_brute(lmax, lmin, 2 * lmax)
    assert (info["terms_even"], info["terms_odd"]) == (e, o)


def test_flop_per_sweep_structure():
    lmax = 57
    e, o = terms_brute(lmax, 2, 2 * lmax)
    cases = [
        (coupling.ALL, False, 1 + 3 + 6, 3, 3),    # separate W^TT, W^TP, W^PP: three sweeps
        (coupling.ALL, True, 6, 3, 1),             # one shared window: one sweep
        (coupling.TT, False, 1, 0, 1),
        (coupling.TE, False, 3, 0, 1),
        (coupling.EE, False, 6, 0, 1),
        (coupling.EEBB, False, 0, 3, 1),
        (coupling.EB, False, 6, 3, 1),
        (coupling.TT | coupling.EEBB, False, 1, 3, 2),
    ]
    for spectra, shared, ne, no, nl in cases:
        info = coupling.plan_info(lmax, 2, spectra, shared=shared)
        assert info["flop"] == 2 * 2 * (ne * e + no * o), (spectra, shared)
        assert info["n_launches"] == nl, (spectra, shared)
        assert info["terms_even"] == 2 * e and info["terms_odd"] == 2 * o


def test_band_limits_and_short_windows():
    lmax = 90
    caps = [7, 64, 2 * lmax]
    info = coupling.plan_info(lmax, 3, coupling.ALL, band_limit=caps, shared=True)
    e = o = 0
    for c in caps:
        ce, co = terms_brute(lmax, 2, c)
        e, o = e + ce, o + co
    assert (info["terms_even"], info["terms_odd"]) == (e, o)
    assert info["flop"] == 2 * (6 * e + 3 * o)
    # items: a tile whose smallest l3 (= its smallest d = 2 i0 + pi) exceeds the band is dropped
    items = 0
    for c in caps:
        for pi in (0, 1):
            seen = set()
            for l1 in range(2, lmax + 1):
                for l2 in range(l1, lmax + 1):
                    d, s = l2 - l1, l1 + l2
                    if d % 2 == pi:
                        seen.add(((d - pi) // 2 // T, (s - pi) // 2 // T))
            items += sum(1 for (ib, _) in seen if 2 * T * ib + pi <= c)
    assert info["n_items"] == items
    # a window that ends at its band limit (w_len = L_w + 1)
    short = coupling.plan_info(lmax, 1, coupling.TT, w_len=51, band_limit=[50])
    assert (short["terms_even"], short["terms_odd"]) == terms_brute(lmax, 2, 50)


def test_full_size_counts():
    # the bench's workload (l_max = 3000) and the largest l_max, in closed form
    for lmax in (3000, 10000):
        info = coupling.plan_info(lmax, 1, coupling.ALL)
        e, o = terms_numpy(lmax, 2, 2 * lmax)
        assert (info["terms_even"], info["terms_odd"]) == (e, o)
        assert info["flop"] == 2 * (10 * e + 3 * o)
    assert terms_numpy(40, 2, 80) == terms_brute(40, 2, 80)


def test_table_bytes():
    def a_blocks(lmax, lmin, cap):
        n = 0
        for pi in (0, 1):
            if lmax - lmin - pi < 0:
                continue
            imax = (lmax - lmin - pi) // 2
            for ib in range((lmax - lmin) // 2 // T + 1):
                if T * ib > imax:
                    continue
                cend = min((lmax - pi - T * ib + T - 1) // 16, (cap // 2) // 16) + 1
                n += max(0, cend - 2 * ib)
        return n
    for lmax in (40, 300, 3000):
        njb = lmax // T + 1
        info = coupling.plan_info(lmax, 1, coupling.ALL)
        assert info["table_bytes_b"] == 2 * njb * (njb + 1) * 6 * 4096
        # A rows per sweep: TT 1, TE 2, polarisation 4 (a0, a0 v, a0 v^2, a1 v)
        assert info["table_bytes_a"] == a_blocks(lmax, 2, 2 * lmax) * (1 + 2 + 4) * 4096
    df = coupling.plan_info(300, 1, coupling.ALL, precision=coupling.DF32)
    assert df["table_bytes_a"] == 0 and df["table_bytes_b"] == 0 and df["flop"] > 0
    with pytest.raises(coupling.CouplingError):
        coupling.plan_info(300, 1, coupling.ALL, precision=coupling.MIXED_BF16)


def test_documented_table_sizes():
    # the header's figures for the FP64 operand tables: about 48 lmax^2 bytes
    # shared (0.43 GB at l_max 3000, 4.7 GB at 10000) and about 28 lmax^2
    # bytes per window with all spectra and separate windows
    for lmax, b_doc in ((3000, 0.43e9), (10000, 4.7e9)):
        info = coupling.plan_info(lmax, 1, coupling.ALL)
        assert abs(info["table_bytes_b"] / (48.0 * lmax ** 2) - 1.0) < 0.05
        assert abs(info["table_bytes_b"] / b_doc - 1.0) < 0.05
        assert abs(info["table_bytes_a"] / (28.0 * lmax ** 2) - 1.0) < 0.1
    # a band limit shrinks the per-window blocks
    full = coupling.plan_info(8000, 1, coupling.ALL)["table_bytes_a"]
    band = coupling.plan_info(8000, 1, coupling.ALL, band_limit=[512])["table_bytes_a"]
    assert band < full / 20


def test_errors():
    def status(fn):
        with pytest.raises(coupling.CouplingError) as e:
            fn()
        return e.value.status
    assert status(lambda: coupling.plan_info(1, 1, coupling.TT)) == 1                       # CPL_ERR_ARG
    assert status(lambda: coupling.plan_info(10, 1, coupling.EE, lmin=1)) == 1
    assert status(lambda: coupling.plan_info(40000, 1, coupling.TT)) == 2                   # CPL_ERR_RANGE
    assert status(lambda: coupling.plan_info(10, 1, coupling.TT, precision=coupling.MIXED_BF16)) == 6
