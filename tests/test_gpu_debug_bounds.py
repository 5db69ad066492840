"""The debug build: device index checks on, results unchanged.

The library built with -DFNTRS_DEBUG_BOUNDS=1 checks every shared-memory index
of the transform passes and every global index of the loaders, storers and
staged tiles on the device; a failed check would skip the access and raise
FNT_RS_E_BOUNDS in the plan's status word.  The small parity cases run here
in a child process that loads that library: they must stay bit-exact against
the oracle with a clean status word, so no check fires on correct inputs.
"""
import os
import subprocess
import sys

import pytest
import torch

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = [
    "tests/test_gpu_parity.py::test_encode_matches_oracle",
    "tests/test_gpu_parity.py::test_fnt_matches_dft_definition",
    "tests/test_gpu_parity.py::test_decode_random_received_matches_oracle",
    "tests/test_gpu_parity.py::test_decode_full_and_half_width_tiles",
    "tests/test_gpu_parity.py::test_encode_tma_and_fallback_paths",
    "tests/test_gpu_parity.py::test_decode_split_sizes_sampled",
    "tests/test_gpu_parity.py::test_lossless_fast_path",
    "tests/test_gpu_ragged.py::test_ragged_persistent_kernel_groups",
    "tests/test_gpu_ragged.py::test_ragged_long_codes_in_one_persistent_launch",
]


def test_parity_cases_under_device_index_checks():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_0907_1788_gb300 import build

    lib = build.build(debug_bounds=True)
    env = dict(os.environ, FNTRS_LIB=lib)
    probe = subprocess.run(
        [sys.executable, "-c",
         "import paper_0907_1788_gb300 as p; print(p.fnt_rs_debug_bounds(), p._lib.LIB_PATH)"],
        cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert probe.returncode == 0, probe.stderr
    flag, path = probe.stdout.split()
    assert flag == "1" and os.path.samefile(path, lib)
    res = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-m", "gpu", *CASES],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=3000)
    assert res.returncode == 0, res.stdout[-4000:] + res.stderr[-2000:]
