"""CPU-side checks of the C ABI: the library builds, loads and exports every
symbol include/coupling.h declares; host-only entry points (argument
validation, the g table) behave as documented.  No GPU work."""
import math
import os
import re
from fractions import Fraction
from math import comb

import numpy as np
import pytest

from paper_2602_15605_gb300 import build_ext, coupling

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "coupling.h")


@pytest.fixture(scope="module")
def lib():
    build_ext.build()
    return coupling.load()


def declared_symbols():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cpl_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_binding_exports():
    assert declared_symbols() == sorted(coupling.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_version(lib):
    assert "sm_103a" in coupling.version()


def test_g_table_matches_exact_rationals(lib):
    # Eq. gdef: g(p) = C(2p, p) / 4^p; each entry must be the correctly
    # rounded double of the exact value.
    pmax = 20002
    g = coupling.g_table(pmax)
    assert g[0] == 1.0 and g[1] == 0.5 and g[2] == 0.375
    ps = list(range(0, 600)) + list(range(600, pmax + 1, 97)) + [pmax]
    for p in ps:
        assert g[p] == float(Fraction(comb(2 * p, p), 4 ** p)), p


def _round_ratio(n, d):
    """The correctly rounded double (nearest, ties to even) of n / d for
    positive integers whose ratio lies in the normal range: an integer
    quotient of 66-67 bits with a sticky bit for the remainder, converted
    (Python rounds int -> float correctly) and scaled by a power of two."""
    k = 66 - (n.bit_length() - d.bit_length())
    q, r = divmod(n << k, d) if k >= 0 else divmod(n, d << -k)
    return math.ldexp(float((q << 1) | (1 if r else 0)), -k - 1)


def _exact_g_h(p, c):
    """g(p) = C(2p, p) / 4^p (Eq. gdef) and h(p) = 1 / ((2p + 1) g(p)),
    correctly rounded, from the exact c = C(2p, p)."""
    return _round_ratio(c, 1 << (2 * p)), _round_ratio(1 << (2 * p), (2 * p + 1) * c)


# The plain and mixed paths read g and h up to p = 2 l_max + 144 (l_max <=
# 32000: p <= 64144); cpl_threej_m11 builds them to 2 (j2 + j3 + 1) + 144
# (j2 + j3 <= 200000: p <= 400146).
P_BUILD_MAX = 64144
P_THREEJ_MAX = 400146


def test_g_h_tables_exact_over_the_build_range(lib):
    # every entry up to 2^16 (beyond the 64144 that l_max = 32000 reads),
    # from C(2p+2, p+1) = C(2p, p) * 2(2p+1) / (p+1) in exact integers
    pmax = 1 << 16
    assert pmax >= P_BUILD_MAX
    g, h = coupling.g_table(pmax), coupling.h_table(pmax)
    c = 1
    bad_g, bad_h = [], []
    for p in range(pmax + 1):
        if p:
            c = c * (2 * (2 * p - 1)) // p
        eg, eh = _exact_g_h(p, c)
        if g[p] != eg:
            bad_g.append(p)
        if h[p] != eh:
            bad_h.append(p)
    assert not bad_g, bad_g[:10]
    assert not bad_h, bad_h[:10]
    assert h[0] == 1.0 and h[1] == float(Fraction(2, 3)) and h[2] == float(Fraction(8, 15))


def test_g_h_tables_exact_at_the_threej_range(lib):
    # sampled entries up to the largest table the symbol generator builds
    ps = [100003, 131072, 200000, P_THREEJ_MAX]
    g, h = coupling.g_table(P_THREEJ_MAX), coupling.h_table(P_THREEJ_MAX)
    for p in ps:
        eg, eh = _exact_g_h(p, comb(2 * p, p))
        assert g[p] == eg, p
        assert h[p] == eh, p


def test_round_ratio_is_correct_rounding():
    # the rounding helper itself: halfway cases go to even, a remainder
    # beyond the half rounds up, exact values stay exact
    one = 1 << 52
    assert _round_ratio(2 * one + 1, 2) == float(one)              # 2^52 + 1/2 -> even 2^52
    assert _round_ratio(2 * one + 3, 2) == float(one + 2)          # 2^52 + 3/2 -> even 2^52 + 2
    assert _round_ratio(4 * one + 3, 4) == float(one + 1)          # 2^52 + 3/4 -> up
    assert _round_ratio(1, 3) == 1.0 / 3.0
    assert _round_ratio(2, 3) == 2.0 / 3.0
    assert _round_ratio(10, 4) == 2.5
    for n, d in ((1, 7), (22, 7), (355, 113), (10 ** 30 + 7, 3 ** 60)):
        assert _round_ratio(n, d) == float(Fraction(n, d))


def test_g_table_asymptote(lib):
    g = coupling.g_table(10000)
    p = np.arange(1000, 10001)
    rel = g[p] * np.sqrt(np.pi * p) - 1.0
    assert np.all(np.abs(rel + 1.0 / (8 * p)) < 2e-7)


def _status(fn):
    with pytest.raises(coupling.CouplingError) as e:
        fn()
    return e.value.status


def test_output_size_and_validation(lib):
    assert coupling.output_size(10, 1, coupling.TT) == 9 * 9
    assert coupling.output_size(10, 2, coupling.TT | coupling.EE, lmin=2) == 2 * 2 * 81
    assert coupling.output_size(10, 1, coupling.TT, lmin=0) == 121
    assert coupling.output_size(20, 3, coupling.ALL, bin_edges=[2, 7, 12, 21]) == 3 * 5 * 9
    assert _status(lambda: coupling.output_size(1, 1, coupling.TT)) == 1
    assert _status(lambda: coupling.output_size(10, 1, coupling.EE, lmin=1)) == 1
    assert _status(lambda: coupling.output_size(10, 1, 0)) == 1
    assert _status(lambda: coupling.output_size(10, 1, 64)) == 1
    assert _status(lambda: coupling.output_size(10, 0, coupling.TT)) == 1
    assert _status(lambda: coupling.output_size(10, 1, coupling.TT, w_len=15)) == 1
    assert coupling.output_size(10, 1, coupling.TT, w_len=15, band_limit=[14]) == 81
    assert _status(lambda: coupling.output_size(10, 1, coupling.TT, w_len=15, band_limit=[15])) == 1
    assert _status(lambda: coupling.output_size(10, 1, coupling.TT, bin_edges=[2, 2, 5])) == 1
    assert _status(lambda: coupling.output_size(10, 1, coupling.TT, bin_edges=[1, 5])) == 1
    assert _status(lambda: coupling.output_size(10, 1, coupling.TT, bin_edges=[2, 12])) == 1
    assert _status(lambda: coupling.output_size(40000, 1, coupling.TT)) == 2
    # mixed precision: 4..6 limbs (0 = default 6)
    for sl in (0, 4, 5, 6):
        assert coupling.output_size(10, 1, coupling.TT, precision=coupling.MIXED_BF16, slices=sl) == 81
    for sl in (3, 7, -1):
        assert _status(lambda: coupling.output_size(10, 1, coupling.TT, precision=coupling.MIXED_BF16, slices=sl)) == 1
    assert _status(lambda: coupling.output_size(10, 1, coupling.TT, precision=3)) == 1
    assert coupling.output_size(20, 1, coupling.TT, bin_edges=[2, 7, 21], bin_weight=1) == 4
    assert _status(lambda: coupling.output_size(20, 1, coupling.TT, bin_weight=1)) == 1
    assert _status(lambda: coupling.output_size(20, 1, coupling.TT, lmin=0, bin_edges=[0, 7, 21], bin_weight=1)) == 1
    assert _status(lambda: coupling.output_size(20, 1, coupling.TT, bin_edges=[2, 7, 21], bin_weight=2)) == 1
    assert coupling.output_size(10, 1, coupling.TT, precision=coupling.DF32) == 81
    assert _status(lambda: coupling.output_size(10001, 1, coupling.TT, precision=coupling.DF32)) == 2


def test_probe_argument_errors(lib):
    import ctypes
    flop = ctypes.c_double(0.0)
    sink = ctypes.c_double(0.0)
    L = coupling.load()
    assert L.cpl_probe_fp64(0, 10, ctypes.byref(sink), ctypes.byref(flop), None) == 1
    assert L.cpl_probe_fp64(10, 0, ctypes.byref(sink), ctypes.byref(flop), None) == 1
    assert L.cpl_probe_fp64(10, 10, None, ctypes.byref(flop), None) == 1
    assert L.cpl_probe_fp64(10, 10, ctypes.byref(sink), None, None) == 1
    assert L.cpl_probe_fp64(1 << 21, 10, ctypes.byref(sink), ctypes.byref(flop), None) == 2
    assert flop.value == 0.0


def test_ctx_create_without_gpu_fails_cleanly(lib):
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    with pytest.raises(coupling.CouplingError) as e:
        coupling.Context(0)
    assert e.value.status in (1, 4, 6)
