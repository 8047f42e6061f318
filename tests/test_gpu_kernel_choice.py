"""The parity suite with every GEMM sector forced onto one kernel.

The split-BF16 path picks, per sector, the tcgen05 tensor-core GEMM or the
exact-FP32 CUDA-core GEMM (SYM_TC_MIN_MN / SYM_TC_MIN_K / SYM_TC_MAX_K
thresholds).  Running the parity tests with all sectors on the tensor cores,
and with all on the CUDA cores, covers both kernels on every case; with
SYM_DIRECT_MAX=0 the sectors the direct kernel takes (B's matrix at most
4 x 4) go through the matrix form and the GEMM kernels instead; SYM_TUNE
sets the schedule parameters (include/symtensor.h, sym_tune) to extremes."""
import os
import subprocess
import sys

import pytest

from tests.conftest import ROOT

pytestmark = pytest.mark.gpu

FORCED = {
    "all_tensor_cores": {"SYM_TUNE": "tc_all=1,direct_max=0", "SYM_TC_MAX_K": "100000000"},
    "all_cuda_cores": {"SYM_TC_MIN_MN": "1000000000"},
    "no_direct_sectors": {"SYM_DIRECT_MAX": "0"},
    # the schedule parameters at their extremes: one-run rows tiles, 32-position
    # direct items, maximal split-K, 256-long thin slices, tiles in sector order
    "schedule_extremes": {"SYM_TUNE": "direct_chunk=32,rows_spans=1,splitk_ctas=64,thin_slice=256,tc_order=1,"
                                      "tc_min_mn=16,tc_min_k=16,tc_group=3"},
}


@pytest.mark.parametrize("mode", sorted(FORCED))
def test_parity_suite_with_forced_kernel(mode):
    env = dict(os.environ, PYTHONPATH=ROOT, **FORCED[mode])
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        "tests/test_gpu_parity.py", "-k", "float32"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
