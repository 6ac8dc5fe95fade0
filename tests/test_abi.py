"""The C-ABI library builds for sm_103a, loads without a GPU and exports
every entry point that ``include/ldpc_gb300.h`` declares; host-side argument
checks fail cleanly without touching a device."""
import ctypes
import os
import re

import numpy as np

from paper_1903_10107_gb300 import native, rate
from paper_1903_10107_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(ldpc_\w+)\s*\(", src))
    return names


def test_header_declares_entry_points():
    d = _declared()
    for name in ("ldpc_code_create", "ldpc_decode_batch", "ldpc_syndrome", "ldpc_llr_from_bsc", "ldpc_strerror"):
        assert name in d


def test_library_exports_every_declared_symbol():
    lib = native.load()
    for name in sorted(_declared()):
        assert hasattr(lib, name), name
    assert set(native.SIGNATURES) >= _declared()


def test_binding_wraps_every_entry_point():
    """native.py has a function of the same name for every entry point (the
    error-string getters are read through the loaded library)."""
    missing = [k for k in native.SIGNATURES if not callable(getattr(native, k, None))]
    assert sorted(missing) == ["ldpc_last_error", "ldpc_strerror"]


def test_error_paths_without_gpu():
    lib = native.load()
    assert lib.ldpc_strerror(native.LDPC_EINVAL) == b"invalid argument"
    out = ctypes.c_void_p()
    assert lib.ldpc_code_create(None, 2, 2, 4, ctypes.byref(out)) == native.LDPC_EINVAL
    bad = np.array([[0, 5]], dtype=np.int32)  # shift 5 >= Z = 4
    assert lib.ldpc_code_create(bad.ctypes.data, 1, 2, 4, ctypes.byref(out)) == native.LDPC_EINVAL
    assert b"shift" in lib.ldpc_last_error()
    assert lib.ldpc_code_info(None, None, None, None, None) == native.LDPC_EINVAL
    assert lib.ldpc_decode_batch(None, None, None, 1, 5, None, None, None, None) == native.LDPC_EINVAL
    assert lib.ldpc_debug_tau_table(None, None) == native.LDPC_EINVAL
    # the host-buffer interactive entry checks its arguments before any copy
    args = [None] * 8 + [1, None, 1, 5, 0, None, 0, 1, 1, 0] + [None] * 7
    assert lib.ldpc_reconcile_interactive_host(*args) == native.LDPC_EINVAL
    assert b"NULL code" in lib.ldpc_last_error()


def test_product_rate_plan_matches_closed_form():
    n, m = 49152, 12288
    q = np.array([0.01, 0.02, 0.035, 0.05, 0.08])
    p, s = rate.plan(n, m, q, 1.1)
    f = rate.efficiency(n, m, p, s, q)
    assert np.all(np.abs(f - 1.1) < 1e-3)
    assert np.all((p == 0) | (s == 0))


def test_product_rank_orders_low_weight_first():
    base = inputs.qc_base_matrix(6, 12, 4, inputs.mixed_column_degrees(12, 0.3, 3, 6, 1), 1)
    rk = rate.puncture_rank(base, 4, inputs.tiebreak_permutation(48, 3))
    assert sorted(rk.tolist()) == list(range(48))
    w = np.repeat((base >= 0).sum(axis=0), 4)
    assert (np.diff(w[np.argsort(rk)]) >= 0).all()
