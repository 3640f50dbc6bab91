"""Thin ctypes binding of the C ABI in include/coupling.h.

Argument marshalling only: every step of the computation runs in the CUDA
library ``_build/libcoupling.so``.  There is no CPU fallback -- if the
library has not been built (``paper_2602_15605_gb300.build_ext.build()``),
or no sm_103 GPU is present, the calls raise.

PyTorch supplies device memory and the current CUDA stream; the functions
take and return ``torch.Tensor`` objects (float64, on the context's device).
"""
import ctypes
import os
import threading

import numpy as np

from . import build_ext

TT, TE, EE, EEBB, EB = 1, 2, 4, 8, 16
SPEC_BITS = (TT, TE, EE, EEBB, EB)
SPEC_NAMES = {TT: "TT", TE: "TE", EE: "EE", EEBB: "EEBB", EB: "EB"}
ALL = TT | TE | EE | EEBB | EB
FP64, MIXED_BF16, DF32 = 0, 1, 2
TUNE_OFF, TUNE_MEASURE = 0, 1

STATUS = {0: "CPL_OK", 1: "CPL_ERR_ARG", 2: "CPL_ERR_RANGE", 3: "CPL_ERR_OOM", 4: "CPL_ERR_CUDA",
          5: "CPL_ERR_TIMEOUT", 6: "CPL_ERR_UNSUPPORTED"}


class CouplingError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class Request(ctypes.Structure):
    _fields_ = [("lmax", ctypes.c_int), ("lmin", ctypes.c_int), ("n_windows", ctypes.c_int),
                ("W_tt", ctypes.c_void_p), ("W_tp", ctypes.c_void_p), ("W_pp", ctypes.c_void_p),
                ("w_len", ctypes.c_int), ("band_limit", ctypes.POINTER(ctypes.c_int)),
                ("spectra", ctypes.c_uint), ("precision", ctypes.c_int), ("mixed_slices", ctypes.c_int),
                ("bin_edges", ctypes.POINTER(ctypes.c_int)), ("n_bins", ctypes.c_int),
                ("bin_weight", ctypes.c_int)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("n_tiles", ctypes.c_longlong), ("n_items", ctypes.c_longlong), ("n_launches", ctypes.c_int),
                ("terms_even", ctypes.c_double), ("terms_odd", ctypes.c_double), ("flop", ctypes.c_double),
                ("table_bytes_b", ctypes.c_ulonglong), ("table_bytes_a", ctypes.c_ulonglong)]


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 40), ("launches", ctypes.c_longlong), ("ms", ctypes.c_double),
                ("flop", ctypes.c_double), ("bytes", ctypes.c_double), ("issued_flop", ctypes.c_double)]


class CovTerm(ctypes.Structure):
    _fields_ = [("spectrum", ctypes.c_uint), ("W", ctypes.c_void_p), ("band_limit", ctypes.c_int),
                ("A", ctypes.c_void_p), ("B", ctypes.c_void_p)]


def decouple_fields(spectra):
    """Pseudo-spectrum fields per right-hand side of cpl_decouple: TT, TE, EE, BB, EB."""
    return (bool(spectra & TT) + bool(spectra & TE) + 2 * bool(spectra & EE) + bool(spectra & EB))


def decouple_systems(spectra):
    """Linear systems per window of cpl_decouple: TT, TE, EE+EEBB, EE-EEBB, EB."""
    return (bool(spectra & TT) + bool(spectra & TE) + 2 * bool(spectra & EE) + bool(spectra & EB))


# Every symbol include/coupling.h declares.
EXPORTS = ("cpl_version", "cpl_last_error", "cpl_ctx_create", "cpl_ctx_destroy", "cpl_ctx_sync",
           "cpl_output_size", "cpl_build", "cpl_build_host", "cpl_build_batch", "cpl_build_noalloc",
           "cpl_ctx_profile", "cpl_ctx_stats", "cpl_ctx_tune", "cpl_ctx_validate",
           "cpl_ctx_inject_alloc_failure", "cpl_threej_m11",
           "cpl_decouple", "cpl_cov_gaussian", "cpl_g_table", "cpl_h_table", "cpl_plan_info_fp64",
           "cpl_probe_fp64")

_lock = threading.Lock()
_lib = None


def library_path():
    return build_ext.LIB


def load():
    """Load libcoupling.so (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = build_ext.LIB
        if not os.path.exists(path):
            raise RuntimeError("CUDA library %s is missing: run paper_2602_15605_gb300.build_ext.build() "
                               "(there is no CPU fallback)" % path)
        L = ctypes.CDLL(path)
        vp, ip, dp = ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double)
        L.cpl_version.restype = ctypes.c_char_p
        L.cpl_last_error.restype = ctypes.c_char_p
        L.cpl_ctx_create.argtypes = [ctypes.POINTER(vp), ip]
        L.cpl_ctx_destroy.argtypes = [vp]
        L.cpl_ctx_sync.argtypes = [vp]
        L.cpl_output_size.argtypes = [ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_size_t)]
        L.cpl_plan_info_fp64.argtypes = [ctypes.POINTER(Request), ctypes.POINTER(PlanInfo)]
        L.cpl_build.argtypes = [vp, ctypes.POINTER(Request), vp, vp]
        L.cpl_build_host.argtypes = [vp, ctypes.POINTER(Request), vp]
        L.cpl_build_batch.argtypes = [vp, ctypes.POINTER(Request), ip, ctypes.POINTER(vp), vp]
        L.cpl_g_table.argtypes = [ip, dp]
        L.cpl_h_table.argtypes = [ip, dp]
        L.cpl_probe_fp64.argtypes = [ip, ip, vp, dp, vp]
        L.cpl_ctx_profile.argtypes = [vp, ip]
        L.cpl_ctx_validate.argtypes = [vp, ip]
        L.cpl_ctx_tune.argtypes = [vp, ip, ctypes.c_char_p]
        L.cpl_ctx_inject_alloc_failure.argtypes = [vp, ip]
        L.cpl_threej_m11.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), ip, vp,
                                     ctypes.c_longlong, vp]
        L.cpl_decouple.argtypes = [vp, ip, ip, ctypes.c_uint, vp, vp, ip, vp, vp, vp]
        L.cpl_cov_gaussian.argtypes = [vp, ip, ip, ctypes.POINTER(CovTerm), ip, ip, ip,
                                       ctypes.POINTER(ctypes.c_int), ip, vp, vp]
        L.cpl_ctx_stats.argtypes = [vp, ctypes.POINTER(KernelStat), ip, ctypes.POINTER(ctypes.c_int), ip]
        for name in EXPORTS:
            if name not in ("cpl_version", "cpl_last_error"):
                getattr(L, name).restype = ctypes.c_int
        _lib = L
        return L


def _check(status):
    if status != 0:
        raise CouplingError(status, load().cpl_last_error().decode())


def version():
    return load().cpl_version().decode()


def g_table(pmax):
    """The library's g(p) table (Eq. gdef), host-side, p = 0..pmax."""
    out = np.zeros(pmax + 1, dtype=np.float64)
    _check(load().cpl_g_table(int(pmax), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return out


def probe_fp64(n_blocks, iters, sink, stream=None):
    """cpl_probe_fp64: launch the FP64 FMA throughput probe on torch's current
    stream (or `stream`); `sink` is a device float64 tensor.  Returns the
    launch's FLOP count; time it with CUDA events on the same stream."""
    import torch
    st = torch.cuda.current_stream(sink.device).cuda_stream if stream is None else stream
    flop = ctypes.c_double(0.0)
    _check(load().cpl_probe_fp64(int(n_blocks), int(iters), ctypes.c_void_p(sink.data_ptr()), ctypes.byref(flop),
                                 ctypes.c_void_p(st)))
    return flop.value


def h_table(pmax):
    """The library's h(p) = 1 / ((2p + 1) g(p)) table, host-side, p = 0..pmax."""
    out = np.zeros(pmax + 1, dtype=np.float64)
    _check(load().cpl_h_table(int(pmax), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return out


def nspec(spectra):
    return sum(1 for b in SPEC_BITS if spectra & b)


class _Keep:
    """Holds the ctypes arrays a Request points into."""

    def __init__(self):
        self.refs = []


def _make_request(lmax, W_tt, W_tp, W_pp, spectra, lmin, band_limit, bin_edges, precision, slices,
                  ptr_of, n_windows, w_len, keep, bin_weight=0):
    r = Request()
    r.lmax, r.lmin, r.n_windows, r.w_len = int(lmax), int(lmin), int(n_windows), int(w_len)
    r.W_tt, r.W_tp, r.W_pp = ptr_of(W_tt), ptr_of(W_tp), ptr_of(W_pp)
    r.spectra, r.precision, r.mixed_slices = int(spectra), int(precision), int(slices)
    if band_limit is not None:
        bl = np.ascontiguousarray(np.asarray(band_limit, dtype=np.int32).reshape(-1))
        keep.refs.append(bl)
        r.band_limit = bl.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    if bin_edges is not None:
        be = np.ascontiguousarray(np.asarray(bin_edges, dtype=np.int32).reshape(-1))
        keep.refs.append(be)
        r.bin_edges = be.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        r.n_bins = be.size - 1
    r.bin_weight = int(bin_weight)
    return r


class Context:
    """An owned cpl_ctx on one CUDA device."""

    def __init__(self, device=0):
        L = load()
        h = ctypes.c_void_p()
        _check(L.cpl_ctx_create(ctypes.byref(h), int(device)))
        self.handle = h
        self.device = int(device)

    def close(self):
        if self.handle:
            load().cpl_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sync(self):
        _check(load().cpl_ctx_sync(self.handle))

    def validate(self, enable=True):
        """Check the windows of every build for NaN / Inf first (cpl_ctx_validate)."""
        _check(load().cpl_ctx_validate(self.handle, 1 if enable else 0))

    def profile(self, enable=True):
        """Turn per-launch event timing on or off (cpl_ctx_profile)."""
        _check(load().cpl_ctx_profile(self.handle, 1 if enable else 0))

    def tune(self, mode=True, cache_path=None):
        """Mixed-path tile-shape autotuner (cpl_ctx_tune): True / TUNE_MEASURE
        measures candidates on the first request of each shape, False / TUNE_OFF
        uses the built-in choice; cache_path persists the choices."""
        m = TUNE_MEASURE if mode is True else TUNE_OFF if mode is False else int(mode)
        path = None if cache_path is None else os.fsencode(str(cache_path))
        _check(load().cpl_ctx_tune(self.handle, m, path))

    def threej_m11(self, j2, j3, out=None, stride=None):
        """cpl_threej_m11: rows of (j1 j2 j3; 0 -1 1) for j1 = |j2 - j3| .. j2 + j3
        (zero-padded to `stride`), one row per (j2, j3) pair; a float64 CUDA
        tensor [n, stride] on torch's current stream."""
        import torch
        a = np.ascontiguousarray(np.asarray(j2, dtype=np.int32).reshape(-1))
        b = np.ascontiguousarray(np.asarray(j3, dtype=np.int32).reshape(-1))
        if a.size != b.size:
            raise ValueError("j2 and j3 must have the same length")
        if stride is None:
            stride = int(2 * np.minimum(a, b).max() + 1) if a.size else 1
        if out is None:
            out = torch.empty((a.size, stride), dtype=torch.float64, device="cuda:%d" % self.device)
        elif tuple(out.shape) != (a.size, stride) or out.dtype != torch.float64 or not out.is_contiguous():
            raise ValueError("out must be a contiguous float64 tensor of shape %s" % ((a.size, stride),))
        st = torch.cuda.current_stream(self.device).cuda_stream
        ip = ctypes.POINTER(ctypes.c_int)
        _check(load().cpl_threej_m11(self.handle, a.ctypes.data_as(ip), b.ctypes.data_as(ip), int(a.size),
                                     ctypes.c_void_p(out.data_ptr()), int(stride), ctypes.c_void_p(st)))
        return out

    def decouple(self, M, pcl, spectra, info=None, out=None):
        """cpl_decouple: underlying spectra from pseudo-spectra (Eq. pseudo_cl).
        M: float64 CUDA tensor [n_windows, nspec, n, n] (cpl_build layout);
        pcl: [n_windows, n_rhs, n_fields, n] with fields TT, TE, EE, BB, EB of
        `spectra`; info: optional int32 CUDA tensor [n_windows, n_systems].
        Returns `out` (layout of pcl) on torch's current stream."""
        import torch
        if M.dim() != 4 or M.shape[-1] != M.shape[-2] or M.dtype != torch.float64 or not M.is_contiguous():
            raise ValueError("M must be a contiguous float64 tensor [n_windows, nspec, n, n]")
        if pcl.dim() != 4 or pcl.dtype != torch.float64 or not pcl.is_contiguous():
            raise ValueError("pcl must be a contiguous float64 tensor [n_windows, n_rhs, n_fields, n]")
        nw, _, n, _ = M.shape
        if pcl.shape[0] != nw or pcl.shape[-1] != n or pcl.shape[2] != decouple_fields(spectra):
            raise ValueError("pcl shape %s does not match M %s and the spectrum set" % (tuple(pcl.shape), tuple(M.shape)))
        if out is None:
            out = torch.empty_like(pcl)
        elif out.shape != pcl.shape or out.dtype != torch.float64 or not out.is_contiguous():
            raise ValueError("out must be a contiguous float64 tensor shaped like pcl")
        ip_ = 0
        if info is not None:
            if info.dtype != torch.int32 or not info.is_contiguous() or info.numel() != nw * decouple_systems(spectra):
                raise ValueError("info must be a contiguous int32 tensor [n_windows, n_systems]")
            ip_ = info.data_ptr()
        st = torch.cuda.current_stream(self.device).cuda_stream
        _check(load().cpl_decouple(self.handle, int(n), int(nw), int(spectra), ctypes.c_void_p(M.data_ptr()),
                                   ctypes.c_void_p(pcl.data_ptr()), int(pcl.shape[1]), ctypes.c_void_p(out.data_ptr()),
                                   ctypes.c_void_p(ip_), ctypes.c_void_p(st)))
        return out

    def cov_gaussian(self, lmax, terms, lmin=2, precision=FP64, bin_edges=None, out=None):
        """cpl_cov_gaussian: sum over terms (spectrum, W~, band_limit or None, A, B)
        of Xi_spectrum(l1, l2; W~) (A_l1 B_l2 + A_l2 B_l1) / 2; W~, A, B float64
        CUDA tensors (A, B indexed by l, length >= lmax + 1).  Returns the dense
        [n, n] or binned [n_bins, n_bins] covariance on torch's current stream."""
        import torch
        if not terms:
            raise ValueError("at least one term")
        keep = []
        arr = (CovTerm * len(terms))()
        w_len = None
        for q, (sp, W, band, A, B) in enumerate(terms):
            for t in (W, A, B):
                if t.dtype != torch.float64 or not t.is_contiguous() or not t.is_cuda:
                    raise ValueError("W, A and B must be contiguous float64 CUDA tensors")
            if A.numel() < lmax + 1 or B.numel() < lmax + 1:
                raise ValueError("A and B need lmax + 1 entries")
            if w_len is not None and W.numel() != w_len:
                raise ValueError("every W must have the same length")
            w_len = W.numel()
            arr[q] = CovTerm(int(sp), W.data_ptr(), -1 if band is None else int(band), A.data_ptr(), B.data_ptr())
            keep += [W, A, B]
        if bin_edges is not None:
            e = np.ascontiguousarray(np.asarray(bin_edges, dtype=np.int32))
            ep, nb = e.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), int(e.size - 1)
            shape = (nb, nb)
        else:
            e, ep, nb = None, None, 0
            shape = (lmax - lmin + 1, lmax - lmin + 1)
        if out is None:
            out = torch.empty(shape, dtype=torch.float64, device="cuda:%d" % self.device)
        elif tuple(out.shape) != shape or out.dtype != torch.float64 or not out.is_contiguous():
            raise ValueError("out must be a contiguous float64 tensor of shape %s" % (shape,))
        st = torch.cuda.current_stream(self.device).cuda_stream
        _check(load().cpl_cov_gaussian(self.handle, int(lmax), int(lmin), arr, len(terms), int(w_len), int(precision),
                                       ep, nb, ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(st)))
        return out

    def inject_alloc_failure(self, n):
        """Test hook: the n-th device allocation from now on fails (0 disables)."""
        _check(load().cpl_ctx_inject_alloc_failure(self.handle, int(n)))

    def stats(self, reset=False):
        """{kernel family: dict(launches, ms, flop, bytes)} (cpl_ctx_stats)."""
        buf = (KernelStat * 64)()
        n = ctypes.c_int()
        _check(load().cpl_ctx_stats(self.handle, buf, 64, ctypes.byref(n), 1 if reset else 0))
        out = {}
        for q in range(min(n.value, 64)):
            k = buf[q]
            out[k.name.decode()] = dict(launches=k.launches, ms=k.ms, flop=k.flop, bytes=k.bytes,
                                        issued_flop=k.issued_flop)
        return out

    # ------------------------------------------------------------------ device
    def request(self, lmax, W_tt=None, W_tp=None, W_pp=None, spectra=TT, lmin=2, band_limit=None,
                bin_edges=None, precision=FP64, slices=0, bin_weight=0):
        """(Request, keepalive, shape) for torch device windows [n_win, w_len]."""
        import torch
        ws = [W for W in (W_tt, W_tp, W_pp) if W is not None]
        if not ws:
            raise ValueError("no window given")
        ref = ws[0]
        n_windows, w_len = (1, ref.shape[0]) if ref.dim() == 1 else tuple(ref.shape)
        for W in ws:
            if W.dtype != torch.float64 or not W.is_cuda or not W.is_contiguous():
                raise ValueError("windows must be contiguous float64 CUDA tensors")
            if W.numel() != n_windows * w_len:
                raise ValueError("all windows must have the same shape")
        keep = _Keep()
        r = _make_request(lmax, W_tt, W_tp, W_pp, spectra, lmin, band_limit, bin_edges, precision, slices,
                          lambda W: None if W is None else W.data_ptr(), n_windows, w_len, keep, bin_weight)
        ns = nspec(spectra)
        if bin_edges is not None:
            nb = len(bin_edges) - 1
            shape = (n_windows, ns, nb, nb)
        else:
            n = lmax - lmin + 1
            shape = (n_windows, ns, n, n)
        return r, keep, shape

    def build(self, lmax, W_tt=None, W_tp=None, W_pp=None, spectra=TT, lmin=2, band_limit=None,
              bin_edges=None, precision=FP64, slices=0, out=None, stream=None, bin_weight=0):
        """cpl_build on torch's current stream; returns out [n_win, nspec, n, n] (float64, device)."""
        import torch
        r, keep, shape = self.request(lmax, W_tt, W_tp, W_pp, spectra, lmin, band_limit, bin_edges,
                                      precision, slices, bin_weight)
        if out is None:
            out = torch.empty(shape, dtype=torch.float64, device="cuda:%d" % self.device)
        elif tuple(out.shape) != shape or out.dtype != torch.float64 or not out.is_contiguous():
            raise ValueError("out must be a contiguous float64 tensor of shape %s" % (shape,))
        st = torch.cuda.current_stream(self.device).cuda_stream if stream is None else stream
        _check(load().cpl_build(self.handle, ctypes.byref(r), ctypes.c_void_p(out.data_ptr()),
                                ctypes.c_void_p(st)))
        del keep
        return out

    def build_batch(self, jobs, outs=None, stream=None):
        """cpl_build_batch.  jobs: list of dicts with the keyword arguments of build()."""
        import torch
        reqs, keeps, shapes = [], [], []
        for j in jobs:
            r, keep, shape = self.request(**j)
            reqs.append(r)
            keeps.append(keep)
            shapes.append(shape)
        if outs is None:
            outs = [torch.empty(s, dtype=torch.float64, device="cuda:%d" % self.device) for s in shapes]
        arr = (Request * len(reqs))(*reqs)
        ptrs = (ctypes.c_void_p * len(outs))(*[o.data_ptr() for o in outs])
        st = torch.cuda.current_stream(self.device).cuda_stream if stream is None else stream
        _check(load().cpl_build_batch(self.handle, arr, len(reqs), ptrs, ctypes.c_void_p(st)))
        del keeps
        return outs

    # ------------------------------------------------------------------ host
    def build_host(self, lmax, W_tt=None, W_tp=None, W_pp=None, spectra=TT, lmin=2, band_limit=None,
                   bin_edges=None, precision=FP64, slices=0, out=None, bin_weight=0):
        """cpl_build_host: numpy windows in, numpy matrix out (copies inside the call)."""
        ws = [np.asarray(W) for W in (W_tt, W_tp, W_pp) if W is not None]
        ref = ws[0]
        n_windows, w_len = (1, ref.shape[0]) if ref.ndim == 1 else ref.shape
        keep = _Keep()

        def ptr(W):
            if W is None:
                return None
            a = np.ascontiguousarray(W, dtype=np.float64)
            keep.refs.append(a)
            return a.ctypes.data

        # the same array object for several roles keeps one shared pointer
        cache = {}

        def ptr_shared(W):
            if W is None:
                return None
            if id(W) not in cache:
                cache[id(W)] = ptr(W)
            return cache[id(W)]

        r = _make_request(lmax, W_tt, W_tp, W_pp, spectra, lmin, band_limit, bin_edges, precision, slices,
                          ptr_shared, n_windows, w_len, keep, bin_weight)
        ns = nspec(spectra)
        if bin_edges is not None:
            nb = len(bin_edges) - 1
            shape = (n_windows, ns, nb, nb)
        else:
            n = lmax - lmin + 1
            shape = (n_windows, ns, n, n)
        if out is None:
            out = np.empty(shape, dtype=np.float64)
        _check(load().cpl_build_host(self.handle, ctypes.byref(r), ctypes.c_void_p(out.ctypes.data)))
        del keep
        return out


def build_noalloc(lmax, W_tt=None, W_tp=None, W_pp=None, spectra=TT, lmin=2, band_limit=None, out=None,
                  stream=None):
    """cpl_build_noalloc on the current CUDA device and torch's current stream.

    For callers that cannot allocate device memory: the library's fixed
    1 MiB scratch array replaces the context's buffers (lmax <= 4096, at most
    4 windows, plain FP64, dense output).  `out` must be supplied by the
    caller in that setting; here it is allocated with torch when omitted."""
    import torch
    L = load()
    L.cpl_build_noalloc.argtypes = [ctypes.POINTER(Request), ctypes.c_void_p, ctypes.c_void_p]
    ws = [W for W in (W_tt, W_tp, W_pp) if W is not None]
    ref = ws[0]
    n_windows, w_len = (1, ref.shape[0]) if ref.dim() == 1 else tuple(ref.shape)
    keep = _Keep()
    r = _make_request(lmax, W_tt, W_tp, W_pp, spectra, lmin, band_limit, None, FP64, 0,
                      lambda W: None if W is None else W.data_ptr(), n_windows, w_len, keep)
    n = lmax - lmin + 1
    shape = (n_windows, nspec(spectra), n, n)
    if out is None:
        out = torch.empty(shape, dtype=torch.float64, device=ref.device)
    st = torch.cuda.current_stream(ref.device).cuda_stream if stream is None else stream
    _check(L.cpl_build_noalloc(ctypes.byref(r), ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(st)))
    del keep
    return out


def plan_info(lmax, n_windows, spectra, lmin=2, w_len=None, band_limit=None, precision=FP64, shared=False):
    """cpl_plan_info_fp64: host-only dry run of a plain-path build (needs no
    GPU).  shared=True: one window pointer serves every role (one sweep);
    False: separate W^TT, W^TP, W^PP.  Returns a dict of the PlanInfo fields."""
    keep = _Keep()
    w_len = 2 * lmax + 1 if w_len is None else w_len
    # distinct non-NULL addresses per role (never dereferenced)
    fakes = (0x1000, 0x1000, 0x1000) if shared else (0x1000, 0x2000, 0x3000)
    r = _make_request(lmax, fakes[0] if spectra & TT else None, fakes[1] if spectra & TE else None,
                      fakes[2] if spectra & (EE | EEBB | EB) else None, spectra, lmin, band_limit, None,
                      precision, 0, lambda W: W, n_windows, w_len, keep, 0)
    info = PlanInfo()
    _check(load().cpl_plan_info_fp64(ctypes.byref(r), ctypes.byref(info)))
    return {name: getattr(info, name) for name, _ in PlanInfo._fields_}


def output_size(lmax, n_windows, spectra, lmin=2, w_len=None, band_limit=None, bin_edges=None,
                precision=FP64, slices=0, bin_weight=0):
    """cpl_output_size for a request (validates it; needs no GPU)."""
    keep = _Keep()
    w_len = 2 * lmax + 1 if w_len is None else w_len
    fake = 0x1000  # any non-NULL address: output_size never dereferences the windows
    r = _make_request(lmax, fake if spectra & TT else None, fake if spectra & TE else None,
                      fake if spectra & (EE | EEBB | EB) else None, spectra, lmin, band_limit, bin_edges,
                      precision, slices, lambda W: W, n_windows, w_len, keep, bin_weight)
    n = ctypes.c_size_t()
    _check(load().cpl_output_size(ctypes.byref(r), ctypes.byref(n)))
    return n.value
