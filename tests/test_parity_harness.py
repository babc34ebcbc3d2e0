"""The parity checks themselves catch planted mistakes (CPU only): the oracle's outputs compared with
themselves pass, and the same outputs with one value corrupted fail."""
import numpy as np
import pytest

import workloads
from gpu_util import FP64_TOL, assert_fp64_parity, per_binary_errors


@pytest.fixture(scope="module")
def ref(orc):
    return orc.integrate(workloads.config("C0", n=64, seed=5))


def corrupted(o, key, idx, fn):
    g = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in o.items()}
    g[key][idx] = fn(g[key][idx])
    return g


def test_identical_outputs_pass(ref):
    e = assert_fp64_parity(ref, ref)
    assert all(v == 0.0 for v in e.values())


@pytest.mark.parametrize("key,idx,fn", [
    ("S1", (1, 7), lambda x: x * (1 + 5 * FP64_TOL)),
    ("Lhat", (2, 3), lambda x: x + 3 * FP64_TOL),
    ("t", 11, lambda x: x * (1 - 2 * FP64_TOL)),
    ("dot_s1s2", 0, lambda x: x + 2 * FP64_TOL),
    ("omega", 63, lambda x: x * (1 + 2 * FP64_TOL)),
])
def test_a_value_beyond_the_tolerance_fails(ref, key, idx, fn):
    with pytest.raises(AssertionError, match="parity exceeded"):
        assert_fp64_parity(corrupted(ref, key, idx, fn), ref)


def test_a_value_within_the_tolerance_passes(ref):
    assert_fp64_parity(corrupted(ref, "S2", (0, 5), lambda x: x * (1 + 0.2 * FP64_TOL)), ref)


def test_a_status_or_decision_change_fails(ref):
    with pytest.raises(AssertionError, match="status"):
        assert_fp64_parity(corrupted(ref, "status", 9, lambda x: 1), ref)
    g = corrupted(ref, "n_rej", 4, lambda x: x + 1)
    assert_fp64_parity(g, ref, max_divergent=1)  # one divergent binary allowed, and left out
    with pytest.raises(AssertionError, match="different step decisions"):
        assert_fp64_parity(corrupted(g, "n_acc", 8, lambda x: x + 1), ref, max_divergent=1)


def test_a_nan_where_the_oracle_is_finite_fails(ref):
    with pytest.raises(AssertionError):
        assert_fp64_parity(corrupted(ref, "dot_ls1", 2, lambda x: np.nan), ref)


def test_per_binary_errors_locate_the_corrupted_binary(ref):
    g = corrupted(ref, "S1", (0, 17), lambda x: x * (1 + 1e-6))
    e = per_binary_errors(g, ref)
    assert int(np.argmax(e["S1"])) == 17 and np.count_nonzero(e["S1"]) == 1
