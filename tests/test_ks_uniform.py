"""pn_ks_uniform, the library's host-only KS test from binned counts, against scipy's exact
one-sample KS test on the unbinned values (CPU only)."""
import numpy as np
import pytest
from scipy import stats


@pytest.fixture(scope="module")
def pn():
    import paper_0908_3889_b300 as pn
    from paper_0908_3889_b300.build import build
    build()
    return pn


@pytest.mark.parametrize("n,bins,shape", [(20_000, 4096, "uniform"), (200_000, 65536, "uniform"),
                                          (50_000, 8192, "skewed"), (1000, 100, "uniform")])
def test_bounds_bracket_the_exact_statistic(pn, n, bins, shape):
    rng = np.random.default_rng(n + bins)
    x = rng.uniform(-1, 1, n) if shape == "uniform" else 2 * rng.beta(1.2, 1.0, n) - 1
    counts, _ = np.histogram(x, bins=bins, range=(-1, 1))
    r = pn.pn_ks_uniform(counts, -1.0, 1.0)
    exact = stats.kstest(x, stats.uniform(loc=-1, scale=2).cdf)
    assert r["n"] == n
    assert r["d_lo"] <= exact.statistic <= r["d_hi"]
    assert r["d_hi"] - r["d_lo"] <= counts.max() / n + 1.0 / bins
    # the asymptotic p-value at the exact D sits between the two reported p-values
    assert r["p_at_d_hi"] <= r["p_at_d_lo"]
    if n >= 20_000:
        p_exact = stats.kstwobign.sf((np.sqrt(n) + 0.12 + 0.11 / np.sqrt(n)) * exact.statistic)
        assert r["p_at_d_hi"] - 1e-12 <= p_exact <= r["p_at_d_lo"] + 1e-12
        assert abs(exact.pvalue - p_exact) < 0.02 + 0.1 * p_exact


def test_kolmogorov_tail_matches_scipy(pn):
    """One bin holding every value: D = 1 - 1/bins exactly at the first edge; p from the series."""
    for bins in (2, 10, 1000):
        counts = np.zeros(bins, dtype=np.int64)
        counts[0] = 500
        r = pn.pn_ks_uniform(counts)
        assert r["d_lo"] == pytest.approx(1 - 1 / bins) and r["d_hi"] == pytest.approx(1.0)
    counts = np.full(64, 1000, dtype=np.int64)
    counts[:32] += 20  # a small excess in the lower half
    r = pn.pn_ks_uniform(counts)
    t = (np.sqrt(r["n"]) + 0.12 + 0.11 / np.sqrt(r["n"])) * r["d_lo"]
    assert r["p_at_d_lo"] == pytest.approx(stats.kstwobign.sf(t), rel=1e-9, abs=1e-15)


def test_argument_errors(pn):
    with pytest.raises(pn.PNError):
        pn.pn_ks_uniform(np.zeros(0, dtype=np.int64))
    with pytest.raises(pn.PNError):
        pn.pn_ks_uniform(np.array([1, -1]))
    with pytest.raises(pn.PNError):
        pn.pn_ks_uniform(np.array([1, 2]), 1.0, 1.0)
