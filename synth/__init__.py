"""Seeded synthetic workloads shared by the tests, the smoke check and the benchmark.

This package holds only random-number plumbing: it contains none of the
method's arithmetic, so both the CPU oracle and the GPU library can consume
its outputs without sharing code.  All draws use numpy ``Generator(PCG64)``.

The paper measures on synthetic data too (random source symbols, coderate
1/2, Sec. IV); these generators follow the shapes of that setting:

* source symbols: uniform 16-bit words, ``[k][W]`` (row i = packet i, column
  c = codeword c; the interleaved packet layout of Sec. II.B);
* erasure patterns: ``n - k`` erased positions drawn uniformly without
  replacement, or one contiguous burst; the decoder receives the remaining
  ``k`` positions in ascending order;
* received words for interpolation-only checks: uniform values in
  ``[0, 65536]`` (any vector of k values has a unique interpolant);
* ragged batches and serving streams: see :mod:`synth.workloads`.
"""
from .workloads import (  # noqa: F401
    CONFIGS,
    Config,
    source,
    received_uniform,
    erased_uniform,
    erased_burst,
    received_positions,
    ragged_groups,
    serving_requests,
)
