import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the sm_103a kernels)")
    config.addinivalue_line("markers", "slow: long-running")


def golden(name):
    """Rows of a whitespace-separated fixture under tests/golden, comments skipped."""
    rows = []
    with open(os.path.join(ROOT, "tests", "golden", name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append(line.split())
    return rows


def device_mags(q, scale=8.0):
    """Per-frame int8 LLR magnitudes of host QBERs (the library's host
    function), as a CUDA tensor: the decoders' per-frame input."""
    import numpy as np
    import torch
    from paper_1903_10107_gb300.decoder import llr_magnitudes
    return torch.from_numpy(llr_magnitudes(np.asarray(q, dtype=np.float64), scale)).cuda()
