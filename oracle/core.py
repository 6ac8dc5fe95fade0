"""ctypes front end of the plain C oracle (test infrastructure only).

The C source ``ldpc_oracle.c`` is compiled with gcc into ``oracle/_build``
on first use (or by ``__graft_entry__.build()``).  All functions take and
return numpy arrays; bit vectors here are unpacked (one 0/1 byte per bit).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ldpc_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

MSG_MAX = 127   # Algorithm 1 cap for 8-bit messages (reading: the full int8 range)
E_MAX = 127     # Algorithm 2 saturation magnitude for 8-bit messages
LLR_SCALE = 8.0  # LSB per nat (reading: the paper gives no quantisation step)

FOLD_FORWARD_BACKWARD = 0  # normative reading of Eq. 7
FOLD_LITERAL_EQ7 = 1       # per-edge right-nested fold, diagnostic
FOLD_MIN = 2               # tau := min (textbook min-sum), for pinning


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable C, no target-specific flags)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-pthread", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            P = ctypes.c_void_p
            I = ctypes.c_int
            L.orc_tau.argtypes = [I, I, I]
            L.orc_tau.restype = I
            L.orc_vn_update.argtypes = [I, I, I]
            L.orc_vn_update.restype = I
            L.orc_edge_count.argtypes = [P, I, I, I]
            L.orc_edge_count.restype = ctypes.c_int64
            L.orc_expand.argtypes = [P, I, I, I, P, P]
            L.orc_syndrome.argtypes = [P, I, I, I, P, I, P]
            L.orc_llr_magnitude.argtypes = [ctypes.c_double, ctypes.c_double]
            L.orc_llr_magnitude.restype = I
            L.orc_llr_frame.argtypes = [P, P, P, ctypes.c_double, ctypes.c_double, I, P]
            L.orc_llr_frame.restype = None
            L.orc_cn_magnitudes.argtypes = [P, I, I, I, P]
            L.orc_cn_magnitudes.restype = None
            L.orc_decode_batch.argtypes = [P, I, I, I, P, P, I, I, I, I, P, P, I, P, P, P, I]
            L.orc_num_cores.restype = I
            _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def tau(p: int, q: int, msg_max: int = MSG_MAX) -> int:
    return lib().orc_tau(int(p), int(q), int(msg_max))


def tau_table(msg_max: int = MSG_MAX, size: int = 128) -> np.ndarray:
    t = np.empty((size, size), dtype=np.int32)
    for p in range(size):
        for q in range(size):
            t[p, q] = lib().orc_tau(p, q, msg_max)
    return t


def vn_update(e_old: int, l_ji: int, l_ij_new: int) -> int:
    return lib().orc_vn_update(int(e_old), int(l_ji), int(l_ij_new))


def cn_magnitudes(a, msg_max: int = MSG_MAX, fold_mode: int = FOLD_FORWARD_BACKWARD) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.intc)
    m = np.zeros_like(a)
    lib().orc_cn_magnitudes(_ptr(a), len(a), msg_max, fold_mode, _ptr(m))
    return m


def _base(base):
    base = np.ascontiguousarray(base, dtype=np.int32)
    return base, base.shape[0], base.shape[1]


def expand(base, Z: int):
    """Row lists of H: (row_ptr[m+1], vn[edges]) in layer-major row order."""
    base, Mb, Nb = _base(base)
    e = lib().orc_edge_count(_ptr(base), Mb, Nb, Z)
    row_ptr = np.zeros(Mb * Z + 1, dtype=np.int32)
    vn = np.zeros(max(e, 1), dtype=np.int32)
    lib().orc_expand(_ptr(base), Mb, Nb, Z, _ptr(row_ptr), _ptr(vn))
    return row_ptr, vn[:e]


def syndrome(base, Z: int, bits: np.ndarray) -> np.ndarray:
    """H x mod 2 for unpacked bits [batch][n] -> [batch][m] (0/1)."""
    base, Mb, Nb = _base(base)
    bits = np.ascontiguousarray(np.atleast_2d(bits), dtype=np.uint8)
    syn = np.zeros((bits.shape[0], Mb * Z), dtype=np.uint8)
    lib().orc_syndrome(_ptr(base), Mb, Nb, Z, _ptr(bits), bits.shape[0], _ptr(syn))
    return syn


def llr_magnitude(p: float, scale: float = LLR_SCALE) -> int:
    return lib().orc_llr_magnitude(float(p), float(scale))


def llr_frames(y: np.ndarray, qber, state=None, known=None, scale: float = LLR_SCALE) -> np.ndarray:
    """Channel LLRs int8 [batch][n] from Bob's unpacked bits.

    ``state[f][j]``: 0 key bit, 1 punctured (LLR 0), 2 shortened (LLR +-127
    from ``known[f][j]``)."""
    y = np.ascontiguousarray(np.atleast_2d(y), dtype=np.uint8)
    B, n = y.shape
    q = np.broadcast_to(np.asarray(qber, dtype=np.float64), (B,))
    out = np.empty((B, n), dtype=np.int8)
    for f in range(B):
        st = None if state is None else np.ascontiguousarray(state[f], dtype=np.uint8)
        kn = None if known is None else np.ascontiguousarray(known[f], dtype=np.uint8)
        row = np.empty(n, dtype=np.int8)
        lib().orc_llr_frame(_ptr(y[f]), _ptr(st), _ptr(kn), float(q[f]), float(scale), n, _ptr(row))
        out[f] = row
    return out


def decode(base, Z: int, llr: np.ndarray, syn: np.ndarray, max_iter: int, *, msg_max: int = MSG_MAX,
           fold_mode: int = FOLD_FORWARD_BACKWARD, scale_q4=None, offset_q=None, stall_window: int = 0,
           threads: int = 0):
    """Decode a batch.  llr int8 [batch][n], syn unpacked [batch][m].

    ``stall_window`` K > 0 also stops a frame, as a failure, once its count
    of unsatisfied checks has set no new minimum for K iterations (the
    minimum tracked from iteration 1, with the first iteration reaching it);
    not part of the paper's decoder, which is K = 0.

    Returns (bits unpacked [batch][n], iters int32 [batch], ok uint8 [batch],
    threads used)."""
    base, Mb, Nb = _base(base)
    llr = np.ascontiguousarray(np.atleast_2d(llr), dtype=np.int8)
    syn = np.ascontiguousarray(np.atleast_2d(syn), dtype=np.uint8)
    B, n = llr.shape
    assert n == Nb * Z and syn.shape == (B, Mb * Z)
    sq = None if scale_q4 is None else np.ascontiguousarray(scale_q4, dtype=np.uint8)
    oq = None if offset_q is None else np.ascontiguousarray(offset_q, dtype=np.int8)
    for t in (sq, oq):
        if t is not None:
            assert t.shape == (max_iter, Mb)
    bits = np.zeros((B, n), dtype=np.uint8)
    iters = np.zeros(B, dtype=np.int32)
    ok = np.zeros(B, dtype=np.uint8)
    used = lib().orc_decode_batch(_ptr(base), Mb, Nb, Z, _ptr(llr), _ptr(syn), B, int(max_iter), int(msg_max),
                                  int(fold_mode), _ptr(sq), _ptr(oq), int(stall_window), _ptr(bits),
                                  _ptr(iters), _ptr(ok), int(threads))
    if used < 0:
        raise ValueError(f"oracle decode failed ({used})")
    return bits, iters, ok, used


def num_cores() -> int:
    return lib().orc_num_cores()
