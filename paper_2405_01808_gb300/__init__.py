"""GB300 GRAND decoder: Python binding of the C ABI in include/grand.h.

This module only marshals arguments: every step of the decoding path runs in
the library's CUDA kernels (libgrand.so, built in-tree for sm_103a). PyTorch
supplies device memory and streams. If the library is missing the calls raise:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

__all__ = [
    "GrandError", "GrandArgumentError", "lib", "build", "polar_H", "Code", "Params", "demod", "decode_batch",
    "decode_symbols", "decode_symbols_host", "decode_mixed", "decode_mixed_host", "frame_desc", "ORDER_HAMMING", "ORDER_QAM_NNE",
    "ORDER_QAM_NEARER", "ORDER_QAM_NNE5", "MEMBERSHIP_AUTO", "MEMBERSHIP_DELTA", "MEMBERSHIP_ROW_PARITY", "MEMBERSHIP_HASH", "MEMBERSHIP_FASTEST", "MEMBERSHIP_SOLVE", "E_UNSUPPORTED",
    "LIK_THRESHOLD", "LIK_LITERAL", "stream_status", "E_TIMEOUT", "ABANDON_DEADLINE", "ABANDON_SUSPENDED",
    "CURSOR_BYTES", "decode_symbols_resumable", "decode_resume",
]

ORDER_HAMMING = 0
ORDER_QAM_NNE = 1
ORDER_QAM_NEARER = 2
ORDER_QAM_NNE5 = 3
MEMBERSHIP_AUTO = 0
MEMBERSHIP_DELTA = 1
MEMBERSHIP_ROW_PARITY = 2
MEMBERSHIP_HASH = 3
MEMBERSHIP_FASTEST = 4  # autotuner only: choose between the split search and the hash join
MEMBERSHIP_SOLVE = 5  # the first hit by Gaussian elimination over the frame's TEP coordinates
LIK_THRESHOLD = 0
LIK_LITERAL = 1
E_TIMEOUT = -5         # grand_status GRAND_E_TIMEOUT
E_UNSUPPORTED = -7     # grand_status GRAND_E_UNSUPPORTED
ABANDON_DEADLINE = 5   # abandon flag of a frame cut at grand_params.deadline_ns
ABANDON_SUSPENDED = 6  # abandon flag of a frame whose resumable search is suspended (GRAND_ABANDON_SUSPENDED)
CURSOR_BYTES = 144     # GRAND_CURSOR_BYTES: the search state of one suspended frame

_lock = threading.Lock()
_lib = None


class GrandError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = lib().grand_status_string(status).decode() if _lib is not None else str(status)
        super().__init__(f"{where}: {msg} ({status})")
        self.status = status


class GrandArgumentError(GrandError, ValueError):
    """An argument the binding rejects before it calls the library (a tensor
    of the wrong type, size or device): status GRAND_E_INVALID."""

    def __init__(self, msg: str):
        RuntimeError.__init__(self, msg)
        self.status = -1


class Params(ctypes.Structure):
    _fields_ = [
        ("order", ctypes.c_int32), ("M", ctypes.c_int32), ("S", ctypes.c_int32),
        ("max_weight", ctypes.c_int32), ("query_cap", ctypes.c_int64), ("lik_variant", ctypes.c_int32),
        ("tiles", ctypes.c_int32 * 4), ("membership", ctypes.c_int32), ("deadline_ns", ctypes.c_int64),
    ]

    @classmethod
    def make(cls, order=ORDER_QAM_NNE, M=16, S=10, max_weight=3, query_cap=1 << 20, lik_variant=LIK_THRESHOLD,
             tiles=(0, 0, 0, 0), membership=MEMBERSHIP_AUTO, deadline_ns=0):
        p = cls()
        p.membership = int(membership)
        p.deadline_ns = int(deadline_ns)
        p.order, p.M, p.S, p.max_weight = int(order), int(M), int(S), int(max_weight)
        p.query_cap, p.lik_variant = int(query_cap), int(lik_variant)
        for i, t in enumerate(tiles):
            p.tiles[i] = int(t)
        return p


class Stats(ctypes.Structure):
    _fields_ = [("evaluated_checks", ctypes.c_uint64), ("hard_frames", ctypes.c_uint64),
                ("search_useful", ctypes.c_uint64), ("prep_ms", ctypes.c_float), ("search_ms", ctypes.c_float)]


FRAME_DESC_DTYPE = np.dtype([("code", "<i4"), ("M", "<i4"), ("sym_offset", "<i8"), ("cw_offset", "<i8")])


def build(force: bool = False, verbose: bool = False) -> str:
    return _build.build(force=force, verbose=verbose)


def lib() -> ctypes.CDLL:
    """Load libgrand.so (building it first if the sources are newer)."""
    global _lib
    with _lock:
        if _lib is None:
            if not _build.up_to_date():
                _build.build()
            if not os.path.exists(_build.LIB):
                raise RuntimeError("libgrand.so is missing and could not be built")
            L = ctypes.CDLL(_build.LIB)
            P, i32, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
            L.grand_version.restype = i32
            L.grand_status_string.argtypes = [i32]
            L.grand_status_string.restype = ctypes.c_char_p
            L.grand_polar_H.argtypes = [i32, i32, ctypes.c_double, P, P]
            L.grand_code_create.argtypes = [P, i32, i32, ctypes.POINTER(P)]
            L.grand_code_destroy.argtypes = [P]
            L.grand_code_info.argtypes = [P, P, P]
            L.grand_stream_status.argtypes = [P, P]
            L.grand_demod.argtypes = [P, i64, i32, i32, ctypes.c_float, i32, P, P, P, P, P, i32, P]
            L.grand_decode_batch.argtypes = [P, P, P, P, P, P, i64, P, P, P, P, P]
            L.grand_decode_symbols.argtypes = [P, P, P, i64, ctypes.c_float, P, P, P, P, P]
            L.grand_decode_mixed.argtypes = [P, i32, P, P, i64, P, i64, ctypes.c_float, P, i64, P, P, P, P]
            L.grand_decode_symbols_noalloc.argtypes = [P, P, P, i64, ctypes.c_float, P, P, P, P]
            L.grand_decode_symbols_resumable.argtypes = [P, P, P, i64, ctypes.c_float, i32, P, P, P, P, P]
            L.grand_decode_resume.argtypes = [P, P, P, i64, i32, P, i64, P, P, P]
            L.grand_decode_symbols_host.argtypes = [P, P, P, i64, ctypes.c_float, P, P, P, i64, P]
            L.grand_decode_mixed_host.argtypes = [P, i32, P, P, i64, P, i64, ctypes.c_float, P, i64, P, P, i64, P]
            L.grand_plan_symbols.argtypes = [P, P, P, i64, ctypes.c_float, P, P, P, ctypes.POINTER(P)]
            L.grand_plan_mixed.argtypes = [P, i32, P, P, i64, P, i64, ctypes.c_float, P, i64, P, P, ctypes.POINTER(P)]
            L.grand_plan_launch.argtypes = [P, P]
            L.grand_plan_destroy.argtypes = [P]
            L.grand_autotune.argtypes = [P, P, P, i64, ctypes.c_float, ctypes.c_char_p, P, P]
            L.grand_autotune_mixed.argtypes = [P, i32, P, P, i64, P, i64, ctypes.c_float, i64, ctypes.c_char_p, P, P]
            L.grand_clock_ns.restype = i64
            L.grand_server_create.argtypes = [P, ctypes.POINTER(P)]
            L.grand_server_submit.argtypes = [P, P, i32, P]
            L.grand_server_poll.argtypes = [P, P, i32, P]
            L.grand_server_drain.argtypes = [P, i64]
            L.grand_server_get_stats.argtypes = [P, P]
            L.grand_server_destroy.argtypes = [P]
            for name in ("grand_polar_H", "grand_code_create", "grand_code_destroy", "grand_code_info",
                         "grand_stream_status",
                         "grand_demod", "grand_decode_batch", "grand_decode_symbols", "grand_decode_mixed",
                         "grand_decode_symbols_noalloc", "grand_decode_symbols_host", "grand_decode_mixed_host",
                         "grand_plan_symbols", "grand_plan_mixed",
                         "grand_plan_launch", "grand_plan_destroy", "grand_autotune", "grand_autotune_mixed",
                         "grand_server_create", "grand_server_submit", "grand_server_poll", "grand_server_drain",
                         "grand_server_get_stats", "grand_server_destroy"):
                getattr(L, name).restype = i32
            _lib = L
    return _lib


def _check(rc: int, where: str):
    if rc != 0:
        raise GrandError(rc, where)


def polar_H(N: int, K: int, design_snr_db: float = 0.0):
    """Parity-check matrix (N-K, N/32) uint32 and frozen set of the polar code."""
    H = np.zeros((N - K, N // 32), dtype=np.uint32)
    frozen = np.zeros(N - K, dtype=np.int32)
    _check(lib().grand_polar_H(N, K, float(design_snr_db), H.ctypes.data, frozen.ctypes.data), "grand_polar_H")
    return H, frozen


def H_from_dense(H: np.ndarray) -> np.ndarray:
    """(R, N) 0/1 matrix -> (R, N/32) packed rows."""
    H = np.asarray(H, dtype=np.uint64)
    R, N = H.shape
    sh = np.arange(32, dtype=np.uint64)
    return (H.reshape(R, N // 32, 32) << sh).sum(axis=2).astype(np.uint32)


class Code:
    """A code object (column-packed H on the current CUDA device)."""

    def __init__(self, H_packed: np.ndarray, N: int, K: int):
        H_packed = np.ascontiguousarray(H_packed, dtype=np.uint32)
        if H_packed.shape != (N - K, N // 32):
            raise ValueError("H must be (N-K, N/32) packed rows")
        h = ctypes.c_void_p()
        _check(lib().grand_code_create(H_packed.ctypes.data, N, K, ctypes.byref(h)), "grand_code_create")
        self._h = h
        self.N, self.K = N, K

    @classmethod
    def polar(cls, N: int, K: int, design_snr_db: float = 0.0) -> "Code":
        H, _ = polar_H(N, K, design_snr_db)
        return cls(H, N, K)

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("code was closed")
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None:
            lib().grand_code_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def stream_status(code: Code, stream=None) -> int:
    """grand_stream_status: synchronise the stream, then take and clear the
    code's deadline flag. Returns 0, or E_TIMEOUT when a frame of a decode on
    this code was cut at its deadline since the last call; raises on other
    errors."""
    rc = lib().grand_stream_status(code.handle, _stream(stream))
    if rc not in (0, E_TIMEOUT):
        _check(rc, "grand_stream_status")
    return rc


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _require_cuda(*ts):
    for t in ts:
        if t is not None and not t.is_cuda:
            raise GrandArgumentError("tensors must live on the CUDA device")
        if t is not None and not t.is_contiguous():
            raise GrandArgumentError("tensors must be contiguous")


# The library receives bare device pointers and trusts their sizes, so the
# binding checks every tensor's element type and element count against what
# the call will read or write (before any library call).
def _symbols_per_frame(N: int, M: int) -> int:
    if M == 2:
        return N
    m = (int(M).bit_length() - 1) >> 1
    if M < 4 or (1 << (2 * m)) != M:
        raise GrandArgumentError(f"M = {M} is not a square constellation 4^m (or 2 for BPSK)")
    return -(-N // (2 * m))


def _dtypes(*names):
    import torch

    return tuple(getattr(torch, n) for n in names if hasattr(torch, n))


def _need(t, name, dtypes, numel, exact=False):
    if t is None:
        return
    if t.dtype not in dtypes:
        raise GrandArgumentError(f"{name}: dtype {t.dtype}; expected {', '.join(str(d) for d in dtypes)}")
    if (t.numel() != numel) if exact else (t.numel() < numel):
        raise GrandArgumentError(f"{name}: {t.numel()} elements; {'exactly' if exact else 'at least'} {numel} expected")


def _check_symbols(symbols, M: int, L: int):
    """Received symbols of F frames: complex64 [F][L] (or float32 [F][L][2]);
    BPSK float32 [F][N]. Returns F."""
    F = symbols.shape[0] if symbols.dim() > 0 else 0
    if M == 2:
        _need(symbols, "symbols", _dtypes("float32"), F * L, exact=True)
    elif symbols.is_complex():
        _need(symbols, "symbols", _dtypes("complex64"), F * L, exact=True)
    else:
        _need(symbols, "symbols", _dtypes("float32", "complex64"), 2 * F * L, exact=True)
    return F


def _check_outputs(F, N, cw, queries, abandon):
    _need(cw, "cw", _dtypes("int32", "uint32"), F * (N // 32))
    _need(queries, "queries", _dtypes("int32", "uint32"), F)
    _need(abandon, "abandon", _dtypes("uint8"), F)


def _params_M(params) -> int:
    return 2 if params.order == ORDER_HAMMING else int(params.M)


def demod(symbols, M: int, N: int, N0: float = 1.0, lik_variant: int = LIK_THRESHOLD, outputs=None, stream=None):
    """grand_demod. symbols: complex64 (F, L) for QAM, float32 (F, N) for BPSK."""
    import torch

    L = _symbols_per_frame(N, M)
    F = _check_symbols(symbols, M, L)
    _require_cuda(symbols)
    sym = torch.view_as_real(symbols) if symbols.is_complex() else symbols
    dev = symbols.device
    if outputs is None:
        outputs = {"y": torch.empty((F, N // 32), dtype=torch.int32, device=dev)}
        if M == 2:
            outputs["nmask"] = torch.empty((F, N), dtype=torch.uint8, device=dev)
        else:
            outputs.update({
                "hard_idx": torch.empty((F, L), dtype=torch.int16, device=dev),
                "key": torch.empty((F, L), dtype=torch.int32, device=dev),
                "nmask": torch.empty((F, L), dtype=torch.uint8, device=dev),
                "rel": torch.empty((F, L), dtype=torch.float32, device=dev),
            })
    o = outputs
    _require_cuda(*o.values())
    _need(o.get("y"), "y", _dtypes("int32", "uint32"), F * (N // 32))
    n_per = F * (N if M == 2 else L)
    _need(o.get("nmask"), "nmask", _dtypes("uint8"), n_per)
    _need(o.get("hard_idx"), "hard_idx", _dtypes("int16", "uint16"), F * L)
    _need(o.get("key"), "key", _dtypes("int32", "uint32"), F * L)
    _need(o.get("rel"), "rel", _dtypes("float32"), F * L)
    rc = lib().grand_demod(_ptr(sym), F, L, M, float(N0), int(lik_variant), _ptr(o.get("hard_idx")), _ptr(o.get("key")),
                           _ptr(o.get("nmask")), _ptr(o.get("rel")), _ptr(o.get("y")), N, _stream(stream))
    _check(rc, "grand_demod")
    return o


def _outputs(F, N, dev, cw=None, queries=None, abandon=None):
    import torch

    if cw is None:
        cw = torch.empty((F, N // 32), dtype=torch.int32, device=dev)
    if queries is None:
        queries = torch.empty(F, dtype=torch.int32, device=dev)
    if abandon is None:
        abandon = torch.empty(F, dtype=torch.uint8, device=dev)
    return cw, queries, abandon


def _result(cw, queries, abandon, st, want_stats):
    r = {"cw": cw, "queries": queries, "abandon": abandon}
    if want_stats:
        r["evaluated_checks"] = int(st.evaluated_checks)
        r["hard_frames"] = int(st.hard_frames)
        r["search_useful"] = int(st.search_useful)
        r["prep_ms"] = float(st.prep_ms)
        r["search_ms"] = float(st.search_ms)
    return r


def decode_batch(code: Code, params: Params, y, hard_idx=None, key=None, nmask=None, cw=None, queries=None,
                 abandon=None, stats: bool = False, stream=None):
    """grand_decode_batch on demodulated frames (outputs of `demod`)."""
    F = y.shape[0]
    M = _params_M(params)
    L = _symbols_per_frame(code.N, M)
    _need(y, "y", _dtypes("int32", "uint32"), F * (code.N // 32), exact=True)
    if M == 2:
        _need(nmask, "nmask", _dtypes("uint8"), F * code.N)
    else:
        for t, name in ((hard_idx, "hard_idx"), (key, "key"), (nmask, "nmask")):
            if t is None:
                raise GrandArgumentError(f"{name} is required for the symbol-level orders")
        _need(hard_idx, "hard_idx", _dtypes("int16", "uint16"), F * L)
        _need(key, "key", _dtypes("int32", "uint32"), F * L)
        _need(nmask, "nmask", _dtypes("uint8"), F * L)
    _check_outputs(F, code.N, cw, queries, abandon)
    _require_cuda(y, hard_idx, key, nmask, cw, queries, abandon)
    cw, queries, abandon = _outputs(F, code.N, y.device, cw, queries, abandon)
    st = Stats()
    rc = lib().grand_decode_batch(code.handle, ctypes.byref(params), _ptr(hard_idx), _ptr(key), _ptr(nmask), _ptr(y), F,
                                  _ptr(cw), _ptr(queries), _ptr(abandon), ctypes.byref(st) if stats else None,
                                  _stream(stream))
    _check(rc, "grand_decode_batch")
    return _result(cw, queries, abandon, st, stats)


def decode_symbols(code: Code, params: Params, symbols, N0: float = 1.0, cw=None, queries=None, abandon=None,
                   stats: bool = False, stream=None):
    """grand_decode_symbols: demodulate and decode in one pass."""
    import torch

    F = _check_symbols(symbols, _params_M(params), _symbols_per_frame(code.N, _params_M(params)))
    _check_outputs(F, code.N, cw, queries, abandon)
    _require_cuda(symbols, cw, queries, abandon)
    sym = torch.view_as_real(symbols) if symbols.is_complex() else symbols
    cw, queries, abandon = _outputs(F, code.N, symbols.device, cw, queries, abandon)
    st = Stats()
    rc = lib().grand_decode_symbols(code.handle, ctypes.byref(params), _ptr(sym), F, float(N0), _ptr(cw),
                                    _ptr(queries), _ptr(abandon), ctypes.byref(st) if stats else None, _stream(stream))
    _check(rc, "grand_decode_symbols")
    return _result(cw, queries, abandon, st, stats)


def decode_symbols_resumable(code: Code, params: Params, symbols, weight_step: int, cursors=None, N0: float = 1.0,
                             cw=None, queries=None, abandon=None, stream=None):
    """grand_decode_symbols_resumable: the decode of `decode_symbols` with each
    frame's search limited to `weight_step` TEP weights beyond the
    preparation's. Frames left without a codeword and below the cap come back
    with abandon ABANDON_SUSPENDED and their cursor in `cursors` (uint8 device
    tensor of F * CURSOR_BYTES bytes; allocated when None). Returns the outputs
    and the cursors."""
    import torch

    F = _check_symbols(symbols, _params_M(params), _symbols_per_frame(code.N, _params_M(params)))
    _check_outputs(F, code.N, cw, queries, abandon)
    if cursors is None:
        cursors = torch.empty(max(1, F) * CURSOR_BYTES, dtype=torch.uint8, device=symbols.device)
    _need(cursors, "cursors", _dtypes("uint8"), F * CURSOR_BYTES)
    _require_cuda(symbols, cw, queries, abandon, cursors)
    sym = torch.view_as_real(symbols) if symbols.is_complex() else symbols
    cw, queries, abandon = _outputs(F, code.N, symbols.device, cw, queries, abandon)
    rc = lib().grand_decode_symbols_resumable(code.handle, ctypes.byref(params), _ptr(sym), F, float(N0),
                                              int(weight_step), _ptr(cursors), _ptr(cw), _ptr(queries),
                                              _ptr(abandon), _stream(stream))
    _check(rc, "grand_decode_symbols_resumable")
    return {"cw": cw, "queries": queries, "abandon": abandon, "cursors": cursors}


def decode_resume(code: Code, params: Params, cursors, cw, queries, abandon, weight_step: int = 0, stream=None):
    """grand_decode_resume: the next `weight_step` TEP weights (0: all left) of
    every frame whose abandon flag is ABANDON_SUSPENDED, on the arrays of a
    decode_symbols_resumable call (cw of shape (F, N/32))."""
    F = queries.numel()
    _check_outputs(F, code.N, cw, queries, abandon)
    _need(cursors, "cursors", _dtypes("uint8"), F * CURSOR_BYTES)
    _require_cuda(cursors, cw, queries, abandon)
    rc = lib().grand_decode_resume(code.handle, ctypes.byref(params), _ptr(cursors), F, int(weight_step), _ptr(cw),
                                   code.N // 32, _ptr(queries), _ptr(abandon), _stream(stream))
    _check(rc, "grand_decode_resume")
    return {"cw": cw, "queries": queries, "abandon": abandon, "cursors": cursors}


def frame_desc(code_idx, M, sym_offset, cw_offset) -> np.ndarray:
    d = np.zeros(len(code_idx), dtype=FRAME_DESC_DTYPE)
    d["code"], d["M"], d["sym_offset"], d["cw_offset"] = code_idx, M, sym_offset, cw_offset
    return d


def _check_mixed(desc, symbols):
    """Descriptor bytes (a whole number of FRAME_DESC_DTYPE records) and flat
    complex64 symbols (or float32 pairs); returns (frames, symbols)."""
    _need(desc, "desc", _dtypes("uint8"), desc.numel())
    if desc.numel() % FRAME_DESC_DTYPE.itemsize:
        raise GrandArgumentError(f"desc: {desc.numel()} bytes is not a whole number of "
                                 f"{FRAME_DESC_DTYPE.itemsize}-byte records")
    if symbols.is_complex():
        _need(symbols, "symbols", _dtypes("complex64"), 0)
        n_sym = symbols.numel()
    else:
        _need(symbols, "symbols", _dtypes("float32"), 0)
        if symbols.numel() % 2:
            raise GrandArgumentError("symbols: float32 pairs expected (an even number of elements)")
        n_sym = symbols.numel() // 2
    return desc.numel() // FRAME_DESC_DTYPE.itemsize, n_sym


def decode_mixed(codes, params: Params, desc, symbols, n_cw_words: int, N0: float = 1.0, cw=None, queries=None,
                 abandon=None, stats: bool = False, stream=None):
    """grand_decode_mixed. desc: device uint8 tensor holding FRAME_DESC_DTYPE records."""
    import torch

    F, n_sym = _check_mixed(desc, symbols)
    _need(cw, "cw", _dtypes("int32", "uint32"), n_cw_words)
    _need(queries, "queries", _dtypes("int32", "uint32"), F)
    _need(abandon, "abandon", _dtypes("uint8"), F)
    _require_cuda(desc, symbols, cw, queries, abandon)
    sym = torch.view_as_real(symbols) if symbols.is_complex() else symbols
    dev = symbols.device
    if cw is None:
        cw = torch.empty(n_cw_words, dtype=torch.int32, device=dev)
    if queries is None:
        queries = torch.empty(F, dtype=torch.int32, device=dev)
    if abandon is None:
        abandon = torch.empty(F, dtype=torch.uint8, device=dev)
    arr = (ctypes.c_void_p * len(codes))(*[c.handle.value for c in codes])
    st = Stats()
    rc = lib().grand_decode_mixed(arr, len(codes), ctypes.byref(params), _ptr(desc), F, _ptr(sym), n_sym, float(N0),
                                  _ptr(cw), n_cw_words, _ptr(queries), _ptr(abandon),
                                  ctypes.byref(st) if stats else None, _stream(stream))
    _check(rc, "grand_decode_mixed")
    return _result(cw, queries, abandon, st, stats)


def decode_mixed_host(codes, params: Params, desc, symbols, n_cw_words: int, N0: float = 1.0, cw=None, queries=None,
                      abandon=None, chunk_frames: int = 0, stream=None):
    """grand_decode_mixed_host: an uneven batch in host memory. desc: a
    FRAME_DESC_DTYPE numpy array (or its bytes as a CPU uint8 tensor);
    symbols: CPU complex64 tensor (best page-locked); returns host tensors."""
    import torch

    if isinstance(desc, np.ndarray):
        desc = torch.from_numpy(np.ascontiguousarray(desc).view(np.uint8))
    F, n_sym = _check_mixed(desc, symbols)
    _need(cw, "cw", _dtypes("int32", "uint32"), n_cw_words)
    _need(queries, "queries", _dtypes("int32", "uint32"), F)
    _need(abandon, "abandon", _dtypes("uint8"), F)
    for t in (desc, symbols, cw, queries, abandon):
        if t is not None and (t.is_cuda or not t.is_contiguous()):
            raise GrandArgumentError("host tensors (contiguous, on the CPU) expected")
    pin = torch.cuda.is_available()
    if cw is None:
        cw = torch.zeros(n_cw_words, dtype=torch.int32, pin_memory=pin)
    if queries is None:
        queries = torch.empty(F, dtype=torch.int32, pin_memory=pin)
    if abandon is None:
        abandon = torch.empty(F, dtype=torch.uint8, pin_memory=pin)
    sym = torch.view_as_real(symbols) if symbols.is_complex() else symbols
    arr = (ctypes.c_void_p * len(codes))(*[c.handle.value for c in codes])
    rc = lib().grand_decode_mixed_host(arr, len(codes), ctypes.byref(params), _ptr(desc), F, _ptr(sym), n_sym,
                                       float(N0), _ptr(cw), n_cw_words, _ptr(queries), _ptr(abandon),
                                       int(chunk_frames), _stream(stream))
    _check(rc, "grand_decode_mixed_host")
    return {"cw": cw, "queries": queries, "abandon": abandon}


NOALLOC_MAX_FRAMES = 16384


def decode_symbols_host(code: Code, params: Params, symbols, N0: float = 1.0, cw=None, queries=None, abandon=None,
                        chunk_frames: int = 0, stream=None):
    """grand_decode_symbols_host: frames in host memory (a CPU tensor, best
    page-locked) decoded with the copies overlapped; returns host tensors
    (page-locked when the call allocates them)."""
    import torch

    M = _params_M(params)
    F = _check_symbols(symbols, M, _symbols_per_frame(code.N, M))
    _check_outputs(F, code.N, cw, queries, abandon)
    for t in (symbols, cw, queries, abandon):
        if t is not None and (t.is_cuda or not t.is_contiguous()):
            raise GrandArgumentError("host tensors (contiguous, on the CPU) expected")
    pin = torch.cuda.is_available()
    if cw is None:
        cw = torch.empty((F, code.N // 32), dtype=torch.int32, pin_memory=pin)
    if queries is None:
        queries = torch.empty(F, dtype=torch.int32, pin_memory=pin)
    if abandon is None:
        abandon = torch.empty(F, dtype=torch.uint8, pin_memory=pin)
    sym = torch.view_as_real(symbols) if symbols.is_complex() else symbols
    rc = lib().grand_decode_symbols_host(code.handle, ctypes.byref(params), _ptr(sym), F, float(N0), _ptr(cw),
                                         _ptr(queries), _ptr(abandon), int(chunk_frames), _stream(stream))
    _check(rc, "grand_decode_symbols_host")
    return {"cw": cw, "queries": queries, "abandon": abandon}


def decode_symbols_noalloc(code: Code, params: Params, symbols, cw, queries, abandon, N0: float = 1.0, stream=None):
    """grand_decode_symbols_noalloc: the decode of `decode_symbols` for callers
    that may not allocate device memory while running. The caller passes every
    output buffer; at most NOALLOC_MAX_FRAMES frames per call; calls on one
    device must not overlap in time (they share one fixed scratch array)."""
    import torch

    F = _check_symbols(symbols, _params_M(params), _symbols_per_frame(code.N, _params_M(params)))
    for t, name in ((cw, "cw"), (queries, "queries"), (abandon, "abandon")):
        if t is None:
            raise GrandArgumentError(f"{name} is required")
    _check_outputs(F, code.N, cw, queries, abandon)
    _require_cuda(symbols, cw, queries, abandon)
    sym = torch.view_as_real(symbols) if symbols.is_complex() else symbols
    rc = lib().grand_decode_symbols_noalloc(code.handle, ctypes.byref(params), _ptr(sym), F, float(N0), _ptr(cw),
                                            _ptr(queries), _ptr(abandon), _stream(stream))
    _check(rc, "grand_decode_symbols_noalloc")
    return {"cw": cw, "queries": queries, "abandon": abandon}


class Plan:
    """A decode call captured into a CUDA graph (grand_plan_*): launch() replays
    it on the buffers given at creation. Keep those tensors alive."""

    def __init__(self, handle, keep):
        self._h = handle
        self._keep = keep

    def launch(self, stream=None):
        _check(lib().grand_plan_launch(self._h, _stream(stream)), "grand_plan_launch")

    def close(self):
        if getattr(self, "_h", None) is not None:
            lib().grand_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def plan_symbols(code: Code, params: Params, symbols, cw, queries, abandon, N0: float = 1.0) -> Plan:
    import torch

    F = _check_symbols(symbols, _params_M(params), _symbols_per_frame(code.N, _params_M(params)))
    for t, name in ((cw, "cw"), (queries, "queries"), (abandon, "abandon")):
        if t is None:
            raise GrandArgumentError(f"{name} is required")
    _check_outputs(F, code.N, cw, queries, abandon)
    _require_cuda(symbols, cw, queries, abandon)
    sym = torch.view_as_real(symbols) if symbols.is_complex() else symbols
    h = ctypes.c_void_p()
    rc = lib().grand_plan_symbols(code.handle, ctypes.byref(params), _ptr(sym), symbols.shape[0], float(N0), _ptr(cw),
                                  _ptr(queries), _ptr(abandon), ctypes.byref(h))
    _check(rc, "grand_plan_symbols")
    return Plan(h, (code, params, symbols, cw, queries, abandon))


def plan_mixed(codes, params: Params, desc, symbols, cw, queries, abandon, N0: float = 1.0) -> Plan:
    import torch

    F, n_sym = _check_mixed(desc, symbols)
    _need(cw, "cw", _dtypes("int32", "uint32"), 0)
    _need(queries, "queries", _dtypes("int32", "uint32"), F)
    _need(abandon, "abandon", _dtypes("uint8"), F)
    _require_cuda(desc, symbols, cw, queries, abandon)
    sym = torch.view_as_real(symbols) if symbols.is_complex() else symbols
    arr = (ctypes.c_void_p * len(codes))(*[c.handle.value for c in codes])
    h = ctypes.c_void_p()
    rc = lib().grand_plan_mixed(arr, len(codes), ctypes.byref(params), _ptr(desc), F, _ptr(sym), n_sym, float(N0),
                                _ptr(cw), cw.numel(), _ptr(queries), _ptr(abandon), ctypes.byref(h))
    _check(rc, "grand_plan_mixed")
    return Plan(h, (codes, params, desc, symbols, cw, queries, abandon))


class TuneResult(ctypes.Structure):
    _fields_ = [("best_ms", ctypes.c_float), ("candidates", ctypes.c_int32), ("from_cache", ctypes.c_int32),
                ("membership", ctypes.c_int32)]


def _tune_dict(p, r):
    return {"tiles": tuple(p.tiles), "best_ms": float(r.best_ms), "candidates": int(r.candidates),
            "from_cache": bool(r.from_cache), "membership": int(p.membership)}


def autotune(code: Code, params: Params, symbols, N0: float = 1.0, cache_path: str | None = None, stream=None):
    """grand_autotune: picks params.tiles on a sample batch (in place)."""
    import torch

    _check_symbols(symbols, _params_M(params), _symbols_per_frame(code.N, _params_M(params)))
    _require_cuda(symbols)
    sym = torch.view_as_real(symbols) if symbols.is_complex() else symbols
    r = TuneResult()
    rc = lib().grand_autotune(code.handle, ctypes.byref(params), _ptr(sym), symbols.shape[0], float(N0),
                              cache_path.encode() if cache_path else None, _stream(stream), ctypes.byref(r))
    _check(rc, "grand_autotune")
    return _tune_dict(params, r)


def autotune_mixed(codes, params: Params, desc, symbols, n_cw_words: int, N0: float = 1.0,
                   cache_path: str | None = None, stream=None):
    import torch

    F, n_sym = _check_mixed(desc, symbols)
    _require_cuda(desc, symbols)
    sym = torch.view_as_real(symbols) if symbols.is_complex() else symbols
    arr = (ctypes.c_void_p * len(codes))(*[c.handle.value for c in codes])
    r = TuneResult()
    rc = lib().grand_autotune_mixed(arr, len(codes), ctypes.byref(params), _ptr(desc), F, _ptr(sym), n_sym, float(N0),
                                    n_cw_words, cache_path.encode() if cache_path else None, _stream(stream),
                                    ctypes.byref(r))
    _check(rc, "grand_autotune_mixed")
    return _tune_dict(params, r)


# --------------------------------------------------------------------------
# serving loop
# --------------------------------------------------------------------------
REQUEST_DTYPE = np.dtype([("code", "<i4"), ("M", "<i4"), ("symbols", "<u8"), ("tag", "<u8"), ("arrival_ns", "<i8")])
RESULT_DTYPE = np.dtype([("tag", "<u8"), ("arrival_ns", "<i8"), ("done_ns", "<i8"), ("queries", "<u4"),
                         ("abandon", "u1"), ("continued", "u1"), ("pad", "u1", (2,)), ("cw", "<u4", (32,))])


class ServerCfg(ctypes.Structure):
    _fields_ = [("codes", ctypes.c_void_p), ("n_codes", ctypes.c_int32), ("params", Params), ("N0", ctypes.c_float),
                ("max_slots", ctypes.c_int32), ("max_device_bytes", ctypes.c_int64), ("max_batch", ctypes.c_int32),
                ("n_streams", ctypes.c_int32), ("resume_weight_step", ctypes.c_int32)]


class ServerStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("admitted", "rejected", "completed", "batches", "batched_frames",
                                              "max_inflight_batches", "errors", "live_slots", "live_bytes",
                                              "pending", "inflight_batches", "batch_service_ns",
                                              "max_batch_service_ns", "launch_ns", "max_launch_ns",
                                              "long_frames", "resume_launches", "long_live")]


def clock_ns() -> int:
    return int(lib().grand_clock_ns())


class Server:
    """grand_server_*: continuous-batching decode server on the current device."""

    def __init__(self, codes, params: Params, max_slots=65536, max_device_bytes=256 << 20, max_batch=0,
                 n_streams=4, N0=1.0, resume_weight_step=0):
        self._codes = list(codes)
        self._arr = (ctypes.c_void_p * len(codes))(*[c.handle.value for c in codes])
        cfg = ServerCfg()
        cfg.codes = ctypes.cast(self._arr, ctypes.c_void_p)
        cfg.n_codes = len(codes)
        cfg.params = params
        cfg.N0 = float(N0)
        cfg.max_slots, cfg.max_device_bytes = int(max_slots), int(max_device_bytes)
        cfg.max_batch, cfg.n_streams = int(max_batch), int(n_streams)
        cfg.resume_weight_step = int(resume_weight_step)
        h = ctypes.c_void_p()
        _check(lib().grand_server_create(ctypes.byref(cfg), ctypes.byref(h)), "grand_server_create")
        self._h = h
        self._poll_lock = threading.Lock()  # the result buffer below is shared by pollers

    def submit(self, reqs: np.ndarray) -> int:
        """Submit a REQUEST_DTYPE array (symbols = host addresses); returns how
        many (a prefix) were admitted; 0 when the server is full."""
        reqs = np.ascontiguousarray(reqs, dtype=REQUEST_DTYPE)
        n = ctypes.c_int(0)
        rc = lib().grand_server_submit(self._h, reqs.ctypes.data, len(reqs), ctypes.byref(n))
        if rc not in (0, -6):
            _check(rc, "grand_server_submit")
        return n.value

    def poll(self, max_results: int = 65536) -> np.ndarray:
        """Completed results (RESULT_DTYPE), at most max_results per call.
        Thread-safe: concurrent pollers take disjoint results."""
        with self._poll_lock:
            buf = getattr(self, "_buf", None)
            if buf is None or len(buf) < max_results:
                buf = self._buf = np.zeros(max_results, dtype=RESULT_DTYPE)
            n = ctypes.c_int(0)
            _check(lib().grand_server_poll(self._h, buf.ctypes.data, max_results, ctypes.byref(n)),
                   "grand_server_poll")
            return buf[: n.value].copy()

    def drain(self, timeout_s: float = 10.0):
        _check(lib().grand_server_drain(self._h, int(timeout_s * 1e9)), "grand_server_drain")

    def stats(self) -> dict:
        st = ServerStats()
        _check(lib().grand_server_get_stats(self._h, ctypes.byref(st)), "grand_server_get_stats")
        return {n: int(getattr(st, n)) for n, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None) is not None:
            lib().grand_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
