"""bench.py's algorithmic FLOP counts equal the oracle's operation counter (no GPU)."""
import numpy as np

import bench


def test_flop_constants_match_oracle_count(orc):
    y = np.array([0.02, 0.1, 0.05, 0.2, -0.1, 0.1, 0.15, 0.0, 0.6, 0.8])
    rhs, step = orc.count_ops(y, 0.5, 0.5)
    add, mul, div, sqrt, cbrt, log, pw = rhs
    assert add + mul + div == bench.FLOPS_RHS and cbrt == 1 and log == 1 and sqrt == 0
    add, mul, div, sqrt, cbrt, log, pw = step
    assert add + mul + div == bench.FLOPS_STEP and sqrt == 1 and pw == 1 and cbrt == 0 and log == 0
    assert bench.FLOPS_ATTEMPT == 6 * bench.FLOPS_RHS + bench.FLOPS_STEP


def test_kernel_sha_is_stable():
    assert bench.kernel_sha() == bench.kernel_sha() and len(bench.kernel_sha()) == 16
