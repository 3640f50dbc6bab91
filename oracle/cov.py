"""CPU FP64 oracle for the approximate Gaussian pseudo-C_l covariance built
from coupling-type kernels (Sec. 2 and Sec. 4.3 "band-limited covariance
matrices" of arXiv 2602.15605).

TEST INFRASTRUCTURE ONLY (same rule as the rest of ``oracle/``).

When the spectra vary little across the band limit of the masks, the
covariance of pseudo-spectra reduces to the kernels

    Xi_X(l1, l2; W~) = (1/4pi) sum_l3 (2 l3 + 1) W~_l3 S_X(l1, l2, l3)

of App. A (the coupling matrices without their (2 l2 + 1) factor) evaluated
on W~, the power spectrum of the product of the squared masks, with the l3
sum truncated at the band limit (Sec. 4.3).  The covariance is a sum of
terms, one per Wick pairing of the four fields:

    Cov_{l1 l2} = sum_t Xi_{X_t}(l1, l2; W~_t) (A^t_l1 B^t_l2 + A^t_l2 B^t_l1) / 2

(e.g. for the TT auto-spectrum one term with A = C^TT, B = 2 C^TT).  The
binned covariance of flat band powers is
Cov_bb' = (1/|b||b'|) sum_{l1 in b} sum_{l2 in b'} Cov_{l1 l2}.

Xi comes from the S-G oracle (``coupling_dense``) divided by (2 l2 + 1),
taken from the upper triangle l1 <= l2 for both orders.
"""
import numpy as np

from . import coupling_dense


def kernel(lmax, W, spectrum, lmin=2, band_limit=None):
    """Xi_X(l1, l2; W) for l1, l2 = lmin .. lmax (dense, symmetric)."""
    M, _ = coupling_dense(lmax, W, W, W, spectrum, lmin=lmin,
                          band_limit=None if band_limit is None else [band_limit])
    l = np.arange(lmin, lmax + 1, dtype=np.float64)
    Xi = M[0, 0] / (2.0 * l + 1.0)[None, :]
    up = np.triu(Xi)
    return up + np.triu(Xi, 1).T


def gaussian(lmax, terms, lmin=2, bin_edges=None):
    """Cov for terms = [(spectrum, W, band_limit or None, A, B)] with A, B
    indexed by l (length >= lmax + 1)."""
    l = np.arange(lmin, lmax + 1)
    cov = np.zeros((l.size, l.size))
    for spectrum, W, band, A, B in terms:
        Xi = kernel(lmax, W, spectrum, lmin=lmin, band_limit=band)
        a = np.asarray(A, dtype=np.float64)[l]
        b = np.asarray(B, dtype=np.float64)[l]
        cov += Xi * 0.5 * (np.outer(a, b) + np.outer(b, a))
    if bin_edges is None:
        return cov
    return bin_cov(cov, lmin, bin_edges)


def bin_cov(cov, lmin, edges):
    """Cov_bb' = (1/|b||b'|) sum_{l1 in b} sum_{l2 in b'} Cov_{l1 l2}."""
    nb = len(edges) - 1
    out = np.zeros((nb, nb))
    for b in range(nb):
        r0, r1 = edges[b] - lmin, edges[b + 1] - lmin
        for c in range(nb):
            c0, c1 = edges[c] - lmin, edges[c + 1] - lmin
            out[b, c] = cov[r0:r1, c0:c1].sum() / ((r1 - r0) * (c1 - c0))
    return out
