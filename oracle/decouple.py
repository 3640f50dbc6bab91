"""CPU FP64 oracle for mode decoupling: solving Eq. pseudo_cl for the
underlying spectra (Sec. 2 of arXiv 2602.15605, with the kernels of App. A).

TEST INFRASTRUCTURE ONLY (same rule as the rest of ``oracle/``).

Eq. pseudo_cl relates the expected pseudo-spectra of masked maps to the
underlying spectra through the coupling matrices, row index l1 the
pseudo-spectrum multipole and column index l2 the underlying one:

    <C~^TT> = K^TT C^TT
    <C~^TE> = K^TE C^TE                      (TB alike, App. A)
    <C~^EE> = K^EE C^EE + K^EEBB C^BB
    <C~^BB> = K^EEBB C^EE + K^EE C^BB        (App. A: BB has the EE structure)
    <C~^EB> = K^EB C^EB,  K^EB = K^EE - K^EEBB

K^EEBB is the paper's odd-parity "EB" kernel (CPL_EEBB of the library); the
last line is the MASTER convention for the EB cross spectrum.  Binned systems
use the same equations with the binned matrices M_bb' = (1/|b|) sum_{l1 in b}
sum_{l2 in b'} M_{l1 l2} and binned pseudo-spectra pcl_b = (1/|b|) sum_{l in
b} pcl_l, which is exact when C is constant inside each bin.

Data layouts follow the library's:
    M    [n_windows][nspec][n][n], spectra in increasing bit order;
    pcl  [n_windows][n_rhs][n_fields][n], fields TT, TE, EE, BB, EB restricted
         to the requested set (EE and BB both present when EE is).
Each system is assembled in full (the EE/BB system as one 2n x 2n block
matrix) and solved with numpy.linalg.solve (LAPACK LU with partial pivoting).
"""
import numpy as np

TT, TE, EE, EEBB, EB = 1, 2, 4, 8, 16
_BITS = (TT, TE, EE, EEBB, EB)


def _slot(spectra, bit):
    if not spectra & bit:
        return -1
    return sum(1 for b in _BITS if b < bit and spectra & b)


def fields(spectra):
    """Names of the pseudo-spectrum fields of a spectrum set, in layout order.
    Raises ValueError when the set cannot be decoupled (EE without EE->BB,
    or EE->BB without EE)."""
    if bool(spectra & EE) != bool(spectra & EEBB):
        raise ValueError("the EE/BB system needs both the EE and the EE->BB kernels")
    f = []
    if spectra & TT:
        f.append("TT")
    if spectra & TE:
        f.append("TE")
    if spectra & EE:
        f += ["EE", "BB"]
    if spectra & EB:
        f.append("EB")
    if not f:
        raise ValueError("no spectrum to decouple")
    return f


def forward(M, C, spectra):
    """Expected pseudo-spectra from underlying spectra C (layout of pcl), by
    the matrix-vector products of Eq. pseudo_cl."""
    M = np.asarray(M, dtype=np.float64)
    C = np.asarray(C, dtype=np.float64)
    f = fields(spectra)
    out = np.zeros_like(C)
    for w in range(M.shape[0]):
        for r in range(C.shape[1]):
            x = dict(zip(f, C[w, r]))
            y = {}
            if spectra & TT:
                y["TT"] = M[w, _slot(spectra, TT)] @ x["TT"]
            if spectra & TE:
                y["TE"] = M[w, _slot(spectra, TE)] @ x["TE"]
            if spectra & EE:
                Kee, Keb = M[w, _slot(spectra, EE)], M[w, _slot(spectra, EEBB)]
                y["EE"] = Kee @ x["EE"] + Keb @ x["BB"]
                y["BB"] = Keb @ x["EE"] + Kee @ x["BB"]
            if spectra & EB:
                y["EB"] = M[w, _slot(spectra, EB)] @ x["EB"]
            out[w, r] = np.stack([y[k] for k in f])
    return out


def decouple(M, pcl, spectra):
    """Underlying spectra solving Eq. pseudo_cl for every window and every
    right-hand side (layout of pcl)."""
    M = np.asarray(M, dtype=np.float64)
    pcl = np.asarray(pcl, dtype=np.float64)
    f = fields(spectra)
    n = M.shape[-1]
    out = np.zeros_like(pcl)
    idx = {k: i for i, k in enumerate(f)}
    for w in range(M.shape[0]):
        rhs = pcl[w]                                    # [n_rhs][n_fields][n]
        if spectra & TT:
            out[w, :, idx["TT"]] = np.linalg.solve(M[w, _slot(spectra, TT)], rhs[:, idx["TT"]].T).T
        if spectra & TE:
            out[w, :, idx["TE"]] = np.linalg.solve(M[w, _slot(spectra, TE)], rhs[:, idx["TE"]].T).T
        if spectra & EE:
            Kee, Keb = M[w, _slot(spectra, EE)], M[w, _slot(spectra, EEBB)]
            big = np.block([[Kee, Keb], [Keb, Kee]])
            b = np.concatenate([rhs[:, idx["EE"]], rhs[:, idx["BB"]]], axis=1).T   # [2n][n_rhs]
            x = np.linalg.solve(big, b).T
            out[w, :, idx["EE"]] = x[:, :n]
            out[w, :, idx["BB"]] = x[:, n:]
        if spectra & EB:
            out[w, :, idx["EB"]] = np.linalg.solve(M[w, _slot(spectra, EB)], rhs[:, idx["EB"]].T).T
    return out


def bin_vector(v, lmin, edges, weight=0):
    """pcl_b = (1/|b|) sum_{l in b} pcl_l over the last axis (indexed from lmin);
    weight=1: each term times l(l+1)/2pi (band powers of D_l)."""
    v = np.asarray(v, dtype=np.float64)
    if weight:
        l = np.arange(lmin, lmin + v.shape[-1], dtype=np.float64)
        v = v * (l * (l + 1.0) / (2.0 * np.pi))
    nb = len(edges) - 1
    out = np.zeros(v.shape[:-1] + (nb,), dtype=np.float64)
    for b in range(nb):
        r0, r1 = edges[b] - lmin, edges[b + 1] - lmin
        out[..., b] = v[..., r0:r1].sum(axis=-1) / (r1 - r0)
    return out
