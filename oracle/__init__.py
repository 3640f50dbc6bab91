"""CPU FP64 oracle for the mode-coupling matrices (arXiv 2602.15605).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The library in
``paper_2602_15605_gb300`` never imports it and shares no code with it.

``coupling_oracle.c`` (compiled here with gcc + OpenMP and loaded through
ctypes) evaluates every Wigner-3j value by the Schulten-Gordon recursion and
forms the l3 sums of Appendix A directly.  ``racah.py`` holds the exact
rational second oracle.  ``bin_matrix`` is the flat band-power average
M_bb' = (1/|b|) sum_{l1 in b} sum_{l2 in b'} M_{l1 l2}.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "coupling_oracle.c")
SOURCE = _SRC
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liborcl.so")
_lock = threading.Lock()
_lib = None

TT, TE, EE, EEBB, EB = 1, 2, 4, 8, 16
SPEC_BITS = (TT, TE, EE, EEBB, EB)

def build(force=False):
    """Compile the C oracle into oracle/_build/liborcl.so (gcc, -O2, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    return compile_source(_SRC, _SO)


def compile_source(src, so):
    """gcc -O2 + OpenMP of one C source into a shared library."""
    tmp = so + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c99", "-D_DEFAULT_SOURCE", "-fopenmp", "-fPIC",
           "-shared", src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, so)
    return so


def load_library(path):
    """ctypes handle of a compiled oracle with its argument types set."""
    L = ctypes.CDLL(path)
    ip = ctypes.POINTER(ctypes.c_int)
    dp = ctypes.POINTER(ctypes.c_double)
    L.orc_threej_j1.argtypes = [ctypes.c_int] * 5 + [dp, ctypes.c_int]
    L.orc_threej_j1.restype = ctypes.c_int
    L.orc_coupling_pairs.argtypes = [ctypes.c_int, ip, ip, ctypes.c_int, dp, dp, dp,
                                     ctypes.c_int, ip, ctypes.c_uint, dp, dp, ctypes.c_int]
    L.orc_coupling_pairs.restype = ctypes.c_int
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = load_library(_SO)
    return _lib


def _dp(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def threej_column(j2, j3, m1, m2, m3):
    """(j j2 j3; m1 m2 m3) for j = jmin..j2+j3.  Returns (jmin, values)."""
    jmin = max(abs(j2 - j3), abs(m1))
    n = max(j2 + j3 - jmin + 1, 1)
    out = np.zeros(n, dtype=np.float64)
    got = lib().orc_threej_j1(j2, j3, m1, m2, m3, _dp(out), n)
    if got < 0:
        raise ValueError("bad 3j arguments")
    return jmin, out[:got]


def nspec(spectra):
    return sum(1 for b in SPEC_BITS if spectra & b)


def _win(W, n_win, w_len):
    if W is None:
        return None
    W = np.ascontiguousarray(np.asarray(W, dtype=np.float64).reshape(n_win, w_len))
    return W


def coupling_pairs(l1s, l2s, W_tt=None, W_tp=None, W_pp=None, spectra=TT,
                   band_limit=None, threads=0, library=None):
    """M and S_abs for the listed (l1, l2) pairs.

    W_* are [n_win, w_len] (or 1-D for one window).  Returns two arrays of
    shape [n_win, nspec, npairs].  `library` (default: this oracle) is a
    handle from load_library with the same entry points -- the pin tests pass
    copies of the oracle with a planted mistake."""
    ref = next(W for W in (W_tt, W_tp, W_pp) if W is not None)
    ref = np.asarray(ref)
    if ref.ndim == 1:
        ref = ref[None, :]
    n_win, w_len = ref.shape
    Wt, Wc, Wp = (_win(W, n_win, w_len) for W in (W_tt, W_tp, W_pp))
    l1s = np.ascontiguousarray(np.asarray(l1s, dtype=np.int32))
    l2s = np.ascontiguousarray(np.asarray(l2s, dtype=np.int32))
    bl = None if band_limit is None else np.ascontiguousarray(np.asarray(band_limit, dtype=np.int32))
    ns = nspec(spectra)
    out = np.zeros((n_win, ns, l1s.size), dtype=np.float64)
    sab = np.zeros_like(out)
    rc = (library or lib()).orc_coupling_pairs(int(l1s.size), _ip(l1s), _ip(l2s), n_win, _dp(Wt), _dp(Wc),
                                  _dp(Wp), w_len, _ip(bl), spectra, _dp(out), _dp(sab),
                                  int(threads))
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    return out, sab


def coupling_dense(lmax, W_tt=None, W_tp=None, W_pp=None, spectra=TT, lmin=2,
                   band_limit=None, threads=0, library=None):
    """Dense M[w][spec][l1-lmin][l2-lmin] and S_abs over lmin..lmax."""
    ls = np.arange(lmin, lmax + 1, dtype=np.int32)
    L1, L2 = np.meshgrid(ls, ls, indexing="ij")
    out, sab = coupling_pairs(L1.ravel(), L2.ravel(), W_tt, W_tp, W_pp, spectra,
                              band_limit, threads, library)
    n = ls.size
    return out.reshape(out.shape[0], out.shape[1], n, n), sab.reshape(out.shape[0], out.shape[1], n, n)


def bin_edges(lmin, lmax, delta):
    """Flat bins [lmin + k*delta, lmin + (k+1)*delta), last one cut at lmax."""
    edges = list(range(lmin, lmax + 1, delta))
    edges.append(lmax + 1)
    return np.asarray(edges, dtype=np.int32)


def bin_matrix(M, lmin, edges, weight=0):
    """M_bb' = (1/|b|) sum_{l1 in b} sum_{l2 in b'} M[l1][l2] over the last two
    axes (rows and columns indexed from lmin).  weight=1: band powers of
    D_l = l(l+1) C_l / 2pi, each term times l1(l1+1) / (l2(l2+1))."""
    M = np.asarray(M, dtype=np.float64)
    if weight:
        l = np.arange(lmin, lmin + M.shape[-1], dtype=np.float64)
        lw = l * (l + 1.0)
        M = M * lw[:, None] / lw[None, :]
    nb = len(edges) - 1
    out = np.zeros(M.shape[:-2] + (nb, nb), dtype=np.float64)
    for b in range(nb):
        r0, r1 = edges[b] - lmin, edges[b + 1] - lmin
        rows = M[..., r0:r1, :].sum(axis=-2)
        for c in range(nb):
            c0, c1 = edges[c] - lmin, edges[c + 1] - lmin
            out[..., b, c] = rows[..., c0:c1].sum(axis=-1) / (r1 - r0)
    return out
