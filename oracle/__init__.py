"""CPU oracle for FNT-based Reed-Solomon erasure codes over F_65537.

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg may import this package; the product
library never does.  It shares no code with the CUDA path.

Two layers:

* ``fnt_rs_oracle.c`` (plain C, 64-bit products, ``%`` reduction) built into
  ``liboracle.so`` by :func:`build` and wrapped by :mod:`oracle.core`;
* :mod:`oracle.small` -- pure-Python restatements for tiny cases
  (DFT by definition, Gaussian elimination on the Vandermonde system,
  the paper's chirp step 3, the power-series step 5) used to pin the C code.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, invariants or brute force (see each test's docstring).
"""
from .core import (build, lib_path, root, encode, encode_rows, decode, pattern, dft,  # noqa: F401
                   max_threads, P, interpolate, encode_sys, decode_sys)
