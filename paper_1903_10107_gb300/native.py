"""ctypes binding of the C ABI declared in ``include/ldpc_gb300.h``.

Argument marshalling only: every function here forwards to the entry point
of the same name in ``libldpc_gb300.so``; all work runs in the library's CUDA
kernels.  Pointers are passed as integers (``tensor.data_ptr()``), streams as
``cudaStream_t`` integers.  There is no CPU fallback: if the library cannot
be built or loaded this module raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

LDPC_OK = 0
LDPC_EINVAL = -1
LDPC_ENOMEM = -2
LDPC_ECUDA = -3
LDPC_EUNSUPPORTED = -4
LDPC_EKERNEL = -5

_P = ctypes.c_void_p
_I = ctypes.c_int
_I64 = ctypes.c_int64
_D = ctypes.c_double

# name -> (restype, argtypes); kept in the order of the header
SIGNATURES = {
    "ldpc_code_create": (_I, [_P, _I, _I, _I, ctypes.POINTER(_P)]),
    "ldpc_code_destroy": (None, [_P]),
    "ldpc_code_info": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I64), ctypes.POINTER(_I)]),
    "ldpc_code_reserve": (_I, [_P, _I]),
    "ldpc_llr_magnitudes": (_I, [_P, _I, _D, _P]),
    "ldpc_llr_from_bsc": (_I, [_P, _P, _P, _P, _P, _P, _P, _I, _P, _P]),
    "ldpc_syndrome": (_I, [_P, _P, _I, _P, _P]),
    "ldpc_decode_batch": (_I, [_P, _P, _P, _I, _I, _P, _P, _P, _P]),
    "ldpc_decode_batch_ex": (_I, [_P, _P, _P, _I, _I, _P, _P, _P, _P, _P, _P]),
    "ldpc_decode_batch_words": (_I, [_P, _P, _P, _I, _I, _I, _P, _P, _P, _P]),
    "ldpc_reconcile_persistent": (_I, [_P, _P, _P, _P, _P, _P, _P, _P, _I, _P, _I, _I, _I, _I, _I, _I, _P, _P, _P,
                                       _P]),
    "ldpc_reconcile_interactive": (_I, [_P, _P, _P, _P, _P, _P, _P, _P, _I, _P, _I, _I, _I, _P, _I, _I, _I, _I, _P,
                                        _P, _P, _P, _P]),
    "ldpc_reconcile_interactive_host": (_I, [_P, _P, _P, _P, _P, _P, _P, _P, _I, _P, _I, _I, _I, _P, _I, _I, _I,
                                             _I, _P, _P, _P, _P, _P, _P, _P]),
    "ldpc_epoch_state_bytes": (_I, [_P, _I, _I, _I, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(_I)]),
    "ldpc_reconcile_epoch": (_I, [_P, _P, _P, _P, _P, _P, _P, _P, _I, _P, _I, _I, _I, _I, _I, _P, ctypes.c_size_t,
                                  _I, _I, _I, _P, _P, _P, _P, _P]),
    "ldpc_code_reserve_persistent": (_I, [_P, _I, _I, _I, _I]),
    "ldpc_relaxed_forward": (_I, [_P, _P, _P, _P, _I, _I, _P, _P, _P, _I, ctypes.c_float, _P, _P, _P, _P]),
    "ldpc_relaxed_backward": (_I, [_P, _P, _P, _I, _I, _P, _P, _P, _I, ctypes.c_float, _P, _P, _P, _P, _P, _P, _P,
                                   _P]),
    "ldpc_decode_batch_noalloc": (_I, [_P, _P, _P, _I, _I, _P, _P, _P, _P]),
    "ldpc_debug_tau_table": (_I, [_P, _P]),
    "ldpc_launch_count": (_I64, []),
    "ldpc_strerror": (ctypes.c_char_p, [_I]),
    "ldpc_last_error": (ctypes.c_char_p, []),
}


class LdpcError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str):
        super().__init__(f"{where} failed: {detail} (code {code})")
        self.code = code


def library_path() -> str:
    return _build.LIB_PATH


def load():
    """Load the library, building it first with nvcc if it is missing or stale."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            if not os.path.exists(path):
                raise ImportError(f"CUDA library {path} is missing")
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def check(rc: int, where: str) -> None:
    if rc != LDPC_OK:
        L = load()
        detail = (L.ldpc_last_error() or b"").decode() or L.ldpc_strerror(rc).decode()
        raise LdpcError(rc, where, detail)


def _call(name, *args):
    rc = getattr(load(), name)(*args)
    check(rc, name)
    return rc


def ldpc_code_create(base_ptr: int, Mb: int, Nb: int, Z: int) -> int:
    h = _P()
    _call("ldpc_code_create", base_ptr, Mb, Nb, Z, ctypes.byref(h))
    return h.value


def ldpc_code_destroy(code: int) -> None:
    load().ldpc_code_destroy(code)


def ldpc_code_info(code: int):
    n, m, mx = _I(), _I(), _I()
    e = _I64()
    _call("ldpc_code_info", code, ctypes.byref(n), ctypes.byref(m), ctypes.byref(e), ctypes.byref(mx))
    return n.value, m.value, e.value, mx.value


def ldpc_code_reserve(code: int, batch: int) -> None:
    _call("ldpc_code_reserve", code, batch)


def ldpc_llr_magnitudes(qber, batch, scale, mag_out):
    _call("ldpc_llr_magnitudes", qber, batch, scale, mag_out)


def ldpc_llr_from_bsc(code, bob_bits, llr_mag, rank, n_short, n_punct, known, batch, llr_out, stream):
    _call("ldpc_llr_from_bsc", code, bob_bits, llr_mag, rank, n_short, n_punct, known, batch, llr_out, stream)


def ldpc_syndrome(code, bits, batch, syn_out, stream):
    _call("ldpc_syndrome", code, bits, batch, syn_out, stream)


def ldpc_decode_batch(code, llr_in, target_syndrome, batch, max_iter, out_bits, out_iters, out_ok, stream):
    _call("ldpc_decode_batch", code, llr_in, target_syndrome, batch, max_iter, out_bits, out_iters, out_ok, stream)


def ldpc_decode_batch_ex(code, llr_in, target_syndrome, batch, max_iter, scale_q4, offset_q, out_bits, out_iters,
                         out_ok, stream):
    _call("ldpc_decode_batch_ex", code, llr_in, target_syndrome, batch, max_iter, scale_q4, offset_q, out_bits,
          out_iters, out_ok, stream)


def ldpc_decode_batch_words(code, llr_in, target_syndrome, batch, max_iter, words, out_bits, out_iters, out_ok,
                            stream):
    _call("ldpc_decode_batch_words", code, llr_in, target_syndrome, batch, max_iter, words, out_bits, out_iters,
          out_ok, stream)


def ldpc_reconcile_persistent(code, bob_bits, llr_mag, rank, n_short, n_punct, known, target_syndrome, batch,
                              frame_list, list_len, max_iter, stall_window, words, ctas_per_sm, threads, out_bits,
                              out_iters, out_ok, stream):
    _call("ldpc_reconcile_persistent", code, bob_bits, llr_mag, rank, n_short, n_punct, known, target_syndrome,
          batch, frame_list, list_len, max_iter, stall_window, words, ctas_per_sm, threads, out_bits, out_iters,
          out_ok, stream)


def ldpc_reconcile_interactive(code, bob_bits, llr_mag, rank, n_short, n_punct, known, target_syndrome, batch,
                               frame_list, list_len, max_iter, stall_window, reveal, max_rounds, words, ctas_per_sm,
                               threads, out_bits, out_iters, out_ok, out_rounds, stream):
    _call("ldpc_reconcile_interactive", code, bob_bits, llr_mag, rank, n_short, n_punct, known, target_syndrome,
          batch, frame_list, list_len, max_iter, stall_window, reveal, max_rounds, words, ctas_per_sm, threads,
          out_bits, out_iters, out_ok, out_rounds, stream)


def ldpc_reconcile_interactive_host(code, bob_bits, llr_mag, rank, n_short, n_punct, known, target_syndrome, batch,
                                    frame_list, list_len, max_iter, stall_window, reveal, max_rounds, words,
                                    ctas_per_sm, threads, out_bits, out_iters, out_ok, out_rounds, h2d_bytes,
                                    d2h_bytes, stream):
    _call("ldpc_reconcile_interactive_host", code, bob_bits, llr_mag, rank, n_short, n_punct, known,
          target_syndrome, batch, frame_list, list_len, max_iter, stall_window, reveal, max_rounds, words,
          ctas_per_sm, threads, out_bits, out_iters, out_ok, out_rounds, h2d_bytes, d2h_bytes, stream)


def ldpc_epoch_state_bytes(code, words, ctas_per_sm, threads):
    b, g = ctypes.c_size_t(), _I()
    _call("ldpc_epoch_state_bytes", code, words, ctas_per_sm, threads, ctypes.byref(b), ctypes.byref(g))
    return b.value, g.value


def ldpc_reconcile_epoch(code, bob_bits, llr_mag, rank, n_short, n_punct, known, target_syndrome, batch, frame_list,
                         list_len, max_iter, stall_window, epoch_iters, resume, lane_state, lane_state_bytes, words,
                         ctas_per_sm, threads, out_bits, out_iters, out_ok, out_claimed, stream):
    _call("ldpc_reconcile_epoch", code, bob_bits, llr_mag, rank, n_short, n_punct, known, target_syndrome, batch,
          frame_list, list_len, max_iter, stall_window, epoch_iters, resume, lane_state, lane_state_bytes, words,
          ctas_per_sm, threads, out_bits, out_iters, out_ok, out_claimed, stream)


def ldpc_code_reserve_persistent(code, list_len, words, ctas_per_sm, threads=0):
    _call("ldpc_code_reserve_persistent", code, list_len, words, ctas_per_sm, threads)


def ldpc_relaxed_forward(code, llr, syn, bits, batch, iters, alpha, gamma, layer_class, n_classes, kappa, ckE, ckL,
                         loss, stream):
    _call("ldpc_relaxed_forward", code, llr, syn, bits, batch, iters, alpha, gamma, layer_class, n_classes, kappa, ckE,
          ckL, loss, stream)


def ldpc_relaxed_backward(code, syn, bits, batch, iters, alpha, gamma, layer_class, n_classes, kappa, ckE, ckL, V, gL,
                          grad_alpha, grad_gamma, grad_llr, stream):
    _call("ldpc_relaxed_backward", code, syn, bits, batch, iters, alpha, gamma, layer_class, n_classes, kappa, ckE,
          ckL, V, gL, grad_alpha, grad_gamma, grad_llr, stream)


def ldpc_decode_batch_noalloc(code, llr_in, target_syndrome, batch, max_iter, out_bits, out_iters, out_ok, stream):
    _call("ldpc_decode_batch_noalloc", code, llr_in, target_syndrome, batch, max_iter, out_bits, out_iters, out_ok,
          stream)


def ldpc_debug_tau_table(out, stream):
    _call("ldpc_debug_tau_table", out, stream)


def ldpc_launch_count() -> int:
    return int(load().ldpc_launch_count())
