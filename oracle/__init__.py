"""CPU oracle for the quantised layered LDPC decoder.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the library and
its CUDA path never do, and this package never imports them.

* :mod:`oracle.core`     -- ctypes front end of the plain C oracle
  (``ldpc_oracle.c``): tau of Algorithm 1, the saturation-oriented VN rule of
  Algorithm 2, the layered decoder, syndromes and channel LLRs.
* :mod:`oracle.rate`     -- rate adaptation by puncturing/shortening and the
  efficiency f = (1 - R) / h(QBER) (section 4.1).
* :mod:`oracle.tiny`     -- pure-Python decoder and maximum-likelihood
  enumeration for codes with n <= 20, brute-force check-node outputs.
* :mod:`oracle.relaxed64` -- FP64 reference of the differentiable FP32
  relaxation (box-plus of Eq. 6 with per-iteration scale/offset).
"""
