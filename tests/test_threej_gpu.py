"""(j1 j2 j3; 0 -1 1) columns from the g table (cpl_threej_m11, GPU) against
the oracle's Schulten-Gordon recursion, itself pinned to Racah and to the
paper's App. B formulas (test_oracle_pins.py)."""
import numpy as np
import pytest

import oracle
from paper_2602_15605_gb300 import coupling

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2602_15605_gb300 import build_ext
    build_ext.build()
    c = coupling.Context(0)
    yield c
    c.close()


def _check(rows, j2s, j3s, stride, tol):
    worst = 0.0
    for q, (a, b) in enumerate(zip(j2s, j3s)):
        jmin, col = oracle.threej_column(int(a), int(b), 0, -1, 1)
        assert jmin == abs(a - b)
        n = col.size
        got = rows[q]
        assert np.all(got[n:] == 0.0)                  # zero padding of the row
        scale = 1.0 / np.sqrt(2.0 * max(a, b) + 1.0)   # |symbol| <~ this
        worst = max(worst, float(np.max(np.abs(got[:n] - col))) / scale)
    assert worst <= tol, worst
    return worst


def test_all_small_pairs(ctx):
    j2, j3 = np.meshgrid(np.arange(1, 41), np.arange(1, 41), indexing="ij")
    j2, j3 = j2.ravel(), j3.ravel()
    rows = ctx.threej_m11(j2, j3, stride=90).cpu().numpy()
    _check(rows, j2, j3, 90, 1e-13)


def test_large_and_unbalanced_pairs(ctx):
    rng = np.random.default_rng(5)
    j2 = np.concatenate([rng.integers(1000, 9000, size=12), [1, 1, 2, 5000, 20000], [30000]])
    j3 = np.concatenate([rng.integers(1000, 9000, size=12), [1, 20000, 7, 5001, 3], [29999]])
    rows = ctx.threej_m11(j2, j3).cpu().numpy()
    w = _check(rows, j2, j3, rows.shape[1], 1e-12)
    print("max scaled error", w)


def test_orthogonality_of_the_column(ctx):
    # sum over j1 of (2 j1 + 1) (j1 j2 j3; 0 -1 1)^2 = 1
    j2 = np.array([3, 50, 777, 4000])
    j3 = np.array([5, 61, 700, 3999])
    rows = ctx.threej_m11(j2, j3).cpu().numpy()
    for q, (a, b) in enumerate(zip(j2, j3)):
        j1 = np.arange(abs(a - b), a + b + 1)
        s = np.sum((2 * j1 + 1) * rows[q, :j1.size] ** 2)
        assert abs(s - 1.0) < 1e-12


def test_argument_errors(ctx):
    with pytest.raises(coupling.CouplingError) as e:
        ctx.threej_m11([0], [3], stride=8)
    assert e.value.status == 1
    with pytest.raises(coupling.CouplingError) as e:
        ctx.threej_m11([5], [3], stride=6)   # needs 2 * 3 + 1 = 7
    assert e.value.status == 1
    with pytest.raises(coupling.CouplingError) as e:
        ctx.threej_m11([150000], [60000], stride=120001)
    assert e.value.status == 2
