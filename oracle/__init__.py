"""CPU oracle for GRAND with the M-QAM likelihood order (arXiv 2405.01808).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg are the only callers. The decoding library never imports this
package and shares no code with it. The arithmetic lives in plain C
(`grand_oracle.c`); this module builds it with gcc and marshals numpy arrays.

Functions and the passages they follow:
  frozen_set / parity_H / generator_G / bhattacharyya  -- Def. II.1, Sec. II
  qam_d / qscale                                      -- Def. II.2, Eq. 2
  demod                                               -- Def. III.1, III.2, Alg. 2 Step 1
  tep_order / select                                  -- Alg. 2 Steps 2-4, Cor. III.1
  decode_qam                                          -- Alg. 2 (Steps 0-5, Return); order
                                                         variants: nearer axis first,
                                                         five-point NNE (Sec. II)
  decode_ab                                           -- GRAND-AB, Sec. I
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "grand_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction: the fp32 quantisation
    must be a plain rounded multiply)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-pthread", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def _setup(lib):
    P = ctypes.c_void_p
    i32, i64, dbl, flt = ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_float
    lib.oracle_polar_G.argtypes = [i32, P]
    lib.oracle_bhattacharyya.argtypes = [i32, dbl, dbl, P]
    lib.oracle_frozen_set.argtypes = [i32, i32, dbl, P]
    lib.oracle_frozen_set.restype = i32
    lib.oracle_parity_H.argtypes = [i32, i32, P, P]
    lib.oracle_qam_d.argtypes = [i32]
    lib.oracle_qam_d.restype = dbl
    lib.oracle_qam_qscale.argtypes = [i32]
    lib.oracle_qam_qscale.restype = flt
    lib.oracle_demod.argtypes = [P, i64, i32, i32, i32, i32, P, P, P, P, P]
    lib.oracle_decode_qam.argtypes = [P, i32, i32, P, i64, i32, i32, i32, i64, i32, i32, P, P, P]
    lib.oracle_decode_qam.restype = i32
    lib.oracle_decode_qam_order.argtypes = [P, i32, i32, P, i64, i32, i32, i32, i64, i32, i32, i32, P, P, P]
    lib.oracle_decode_qam_order.restype = i32
    lib.oracle_decode_ab.argtypes = [P, i32, i32, P, i64, i32, i64, i32, P, P, P]
    lib.oracle_decode_ab.restype = i32
    lib.oracle_tep_order.argtypes = [i32, P, P, i64]
    lib.oracle_tep_order.restype = i64
    lib.oracle_tep_order_n.argtypes = [i32, i32, P, P, i64]
    lib.oracle_tep_order_n.restype = i64
    lib.oracle_select.argtypes = [P, i32, i32, P]
    lib.oracle_select.restype = i32
    return lib


def build_variant(source_text: str, so_path: str) -> str:
    """Compile a modified copy of the oracle source (used by the tests that
    check that the pins catch planted mistakes)."""
    src = so_path + ".c"
    with open(src, "w") as fh:
        fh.write(source_text)
    subprocess.run(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-ffp-contract=off",
                    "-fno-fast-math", "-pthread", src, "-o", so_path, "-lm"], check=True)
    return so_path


def source_text() -> str:
    with open(_SRC) as fh:
        return fh.read()


def use_library(so_path: str | None):
    """Route every call to the library at so_path (None: the built oracle)."""
    global _lib
    with _lock:
        _lib = None if so_path is None else _setup(ctypes.CDLL(so_path))


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = _setup(ctypes.CDLL(_SO))
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def generator_G(N: int) -> np.ndarray:
    G = np.zeros((N, N), dtype=np.uint8)
    _load().oracle_polar_G(N, _ptr(G))
    return G


def bhattacharyya(N: int, rate: float, design_snr_db: float = 0.0) -> np.ndarray:
    z = np.zeros(N, dtype=np.float64)
    _load().oracle_bhattacharyya(N, float(rate), float(design_snr_db), _ptr(z))
    return z


def frozen_set(N: int, K: int, design_snr_db: float = 0.0) -> np.ndarray:
    f = np.zeros(N - K, dtype=np.int32)
    if _load().oracle_frozen_set(N, K, float(design_snr_db), _ptr(f)) != 0:
        raise ValueError("invalid (N, K)")
    return f


def info_set(N: int, K: int, design_snr_db: float = 0.0) -> np.ndarray:
    f = set(frozen_set(N, K, design_snr_db).tolist())
    return np.array([i for i in range(N) if i not in f], dtype=np.int64)


def parity_H(N: int, K: int, design_snr_db: float = 0.0) -> np.ndarray:
    """(N-K) x N uint8 matrix: row r is column frozen[r] of G_N."""
    f = frozen_set(N, K, design_snr_db)
    H = np.zeros((N - K, N), dtype=np.uint8)
    _load().oracle_parity_H(N, K, _ptr(f), _ptr(H))
    return H


def qam_d(M: int) -> float:
    return float(_load().oracle_qam_d(M))


def qscale(M: int) -> np.float32:
    return np.float32(_load().oracle_qam_qscale(M))


def demod(symbols: np.ndarray, M: int, N: int, literal: bool = False) -> dict:
    """Per-symbol hard index, Q16.16 key, neighbour mask, FP64 likelihood and
    the packed hard word, for complex64 symbols of shape (F, L)."""
    s = np.ascontiguousarray(symbols, dtype=np.complex64)
    F, L = s.shape
    out = {
        "hard_idx": np.zeros((F, L), np.uint16),
        "key": np.zeros((F, L), np.uint32),
        "nmask": np.zeros((F, L), np.uint8),
        "rel": np.zeros((F, L), np.float64),
        "y": np.zeros((F, N // 32), np.uint32),
    }
    _load().oracle_demod(_ptr(s), F, L, M, N, int(literal), _ptr(out["hard_idx"]), _ptr(out["key"]),
                         _ptr(out["nmask"]), _ptr(out["rel"]), _ptr(out["y"]))
    return out


ORDER_NNE, ORDER_NNE_DSORT, ORDER_NNE5 = 1, 2, 3


def decode_qam(H: np.ndarray, symbols: np.ndarray, M: int, S: int, cap: int, literal: bool = False,
               threads: int = 1, order: int = ORDER_NNE) -> dict:
    H = np.ascontiguousarray(H, dtype=np.uint8)
    R, N = H.shape
    s = np.ascontiguousarray(symbols, dtype=np.complex64)
    F, L = s.shape
    cw = np.zeros((F, N // 32), np.uint32)
    q = np.zeros(F, np.int64)
    ab = np.zeros(F, np.uint8)
    rc = _load().oracle_decode_qam_order(_ptr(H), N, N - R, _ptr(s), F, L, M, S, int(cap), int(literal),
                                         int(order), int(threads), _ptr(cw), _ptr(q), _ptr(ab))
    if rc != 0:
        raise ValueError("oracle_decode_qam: invalid arguments")
    return {"cw": cw, "queries": q, "abandon": ab}


def decode_ab(H: np.ndarray, r: np.ndarray, max_weight: int, cap: int, threads: int = 1) -> dict:
    H = np.ascontiguousarray(H, dtype=np.uint8)
    R, N = H.shape
    r = np.ascontiguousarray(r, dtype=np.float32)
    F = r.shape[0]
    cw = np.zeros((F, N // 32), np.uint32)
    q = np.zeros(F, np.int64)
    ab = np.zeros(F, np.uint8)
    rc = _load().oracle_decode_ab(_ptr(H), N, N - R, _ptr(r), F, int(max_weight), int(cap), int(threads),
                                  _ptr(cw), _ptr(q), _ptr(ab))
    if rc != 0:
        raise ValueError("oracle_decode_ab: invalid arguments")
    return {"cw": cw, "queries": q, "abandon": ab}


def tep_order(exists: np.ndarray, max_out: int = 1 << 20) -> tuple[np.ndarray, int]:
    """Canonical order of the valid TEPs for per-rank allowed-alternative masks
    (bit0 h, bit1 v, bit2 diag). Returns (codes[:min(total, max_out)], total)."""
    e = np.ascontiguousarray(exists, dtype=np.uint8)
    out = np.zeros(max_out, dtype=np.uint32)
    total = int(_load().oracle_tep_order(int(e.size), _ptr(e), _ptr(out), int(max_out)))
    return out[: min(total, max_out)].copy(), total


def tep_order_n(exists: np.ndarray, n_alt: int, max_out: int = 1 << 20) -> tuple[np.ndarray, int]:
    """As tep_order for n_alt alternatives per rank (bit c-1 of exists[r]:
    alternative c allowed), codes packed with 3 bits per rank."""
    e = np.ascontiguousarray(exists, dtype=np.uint8)
    out = np.zeros(max_out, dtype=np.uint32)
    total = int(_load().oracle_tep_order_n(int(e.size), int(n_alt), _ptr(e), _ptr(out), int(max_out)))
    if total < 0:
        raise ValueError("tep_order_n: invalid arguments")
    return out[: min(total, max_out)].copy(), total


def select(key: np.ndarray, S: int) -> np.ndarray:
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(max(1, min(S, k.size)), dtype=np.int32)
    n = _load().oracle_select(_ptr(k), int(k.size), int(S), _ptr(out))
    return out[:n].copy()
