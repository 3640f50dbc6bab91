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
