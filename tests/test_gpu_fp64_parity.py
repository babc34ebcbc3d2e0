"""CUDA path vs the CPU oracle on identical seeded inputs (needs a B300)."""
import numpy as np
import pytest

import workloads
from gpu_util import (FP64_TOL, assert_fp64_parity, assert_fp64_parity_conditioned, decided_alike, parity_errors,
                      per_binary_errors, ulp_response)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pn():
    import torch
    import paper_0908_3889_b300 as pn
    from paper_0908_3889_b300.build import build
    assert torch.cuda.is_available()
    build()
    return pn


def run_gpu(pn, ens, **kw):
    import torch
    inp = pn.to_device(ens)
    out = pn.integrate(inp, **kw)
    torch.cuda.synchronize()
    return pn.to_numpy(out)


def oracle_params(orc, **kw):
    return orc.params(**kw)


@pytest.mark.parametrize("schedule", [1, 2])
def test_c0_all_binaries_fp64(pn, orc, schedule):
    """1,024 equal-mass maximal-spin binaries, omega 0.025 -> 0.05: every binary within 1e-10."""
    ens = workloads.config("C0")
    o = orc.integrate(ens)
    g = run_gpu(pn, ens, schedule=schedule)
    assert np.all(o["status"] == 0)
    assert_fp64_parity(g, o)


def test_schedules_and_blocks_bit_identical(pn):
    ens = workloads.config("C2", n=3000)
    ref = run_gpu(pn, ens, schedule=1, block=128)
    for sched, block, bpt in ((2, 64, 0), (2, 256, 0), (1, 64, 1), (2, 128, 0), (1, 128, 2), (1, 64, 2)):
        g = run_gpu(pn, ens, schedule=sched, block=block, bpt=bpt)
        for k in ref:
            assert np.array_equal(ref[k], g[k], equal_nan=True), (sched, block, bpt, k)


def test_c2_full_size_uneven_lengths_subsample(pn, orc):
    """4,194,304 binaries of uneven length (the largest ensemble), persistent schedule; 2,048 checked.

    With q up to 10 and chi2 down to 0, S2 can sit far below the absolute tolerance, where the error
    control does not constrain it: its direction then responds to a one-ulp change of an input (or of
    h0) by up to ~4e-10 in the oracle itself.  Each binary is held to max(1e-10, 10x that response),
    and all but a handful must meet 1e-10 outright."""
    import torch
    ens = workloads.config("C2")
    n = ens["m1"].shape[0]
    inp = pn.to_device(ens)
    with pn.Batch(n, pn.params(schedule=2)) as b:
        out = b.integrate(inp)
        torch.cuda.synchronize()
        st = b.stats(inp, out)
    assert st["count_by_status"][0] == n and st["attempts_max"] > 3 * st["attempts_min"]
    idx = workloads.subsample(n, 2048, seed=workloads.SEED_BASE + 102)
    g = {k: v[..., idx] for k, v in pn.to_numpy(out).items()}
    o, resp = ulp_response(orc, workloads.take(ens, idx))
    assert_fp64_parity_conditioned(g, o, resp, max_relaxed=8)


def test_c1_full_size_subsample_fp64(pn, orc):
    """1,048,576 binaries in the bench launch shape; a seeded 4,096 subsample checked against the oracle."""
    import torch
    ens = workloads.config("C1")
    n = ens["m1"].shape[0]
    inp = pn.to_device(ens)
    with pn.Batch(n, pn.params()) as b:
        out = b.integrate(inp)
        torch.cuda.synchronize()
        st = b.stats(inp, out)
    idx = workloads.subsample(n, 4096, seed=workloads.SEED_BASE + 101)
    g = {k: v[..., idx] for k, v in pn.to_numpy(out).items()}
    o = orc.integrate(workloads.take(ens, idx))
    assert_fp64_parity(g, o, max_divergent=1)
    assert st["count_by_status"][0] == n


@pytest.mark.parametrize("n", [1, 31, 33, 257, 1000])
def test_ragged_sizes(pn, orc, n):
    ens = workloads.config("C2", n=n, seed=1234 + n)
    o = orc.integrate(ens)
    for sched in (1, 2):
        assert_fp64_parity(run_gpu(pn, ens, schedule=sched), o)


def test_empty_batch_is_a_no_op(pn):
    import torch
    ens = workloads.config("C0", n=4)
    inp = pn.to_device(ens)
    out = pn.alloc_outputs(4)
    out["_block"].fill_(7.0)
    with pn.Batch(4) as b:
        pn.pn_batch_integrate(b.handle, 0, inp, out)
        torch.cuda.synchronize()
    assert torch.all(out["_block"] == 7.0)


def test_bad_inputs_and_limits(pn, orc):
    ens = workloads.config("C0", n=8)
    ens["chi1"][0] = 1.5
    ens["omega0"][1] = 0.06
    ens["m1"][2] = np.nan
    ens["m1"][3] = 0.7
    ens["lhat"][:, 4] = [0.0, 0.6, 0.6]
    ens["chi1"][5] = 0.0
    ens["chi2"][5] = 0.0
    o = orc.integrate(ens)
    g = run_gpu(pn, ens)
    assert list(g["status"][:5]) == [4] * 5 and list(g["status"][5:]) == [0] * 3
    assert np.all(np.isnan(g["t"][:5])) and np.all(g["n_acc"][:5] == 0)
    assert np.all(np.isnan(g["dot_s1s2"][5:6]))
    ok = np.arange(8) >= 5
    e = parity_errors(g, o, ok)
    assert max(e.values()) <= FP64_TOL
    for ms in (1, 2, 3, 17):
        o = orc.integrate(workloads.config("C0", n=16), orc.params(max_steps=ms))
        g = run_gpu(pn, workloads.config("C0", n=16), max_steps=ms)
        assert np.array_equal(g["status"], o["status"]) and np.array_equal(g["n_acc"], o["n_acc"])
        assert np.allclose(g["omega"], o["omega"], rtol=1e-12)


def test_first_cross_mode_within_its_conditioning(pn, orc):
    """Stopping at the first crossing returns the overshooting state, which depends directly on the last
    step size; the error controller fixes step sizes only to ~1e-9 under roundoff (the oracle itself moves
    that much when h0 or an input changes by one ulp).  The GPU must agree within 10x the largest of the
    oracle's own responses to one-ulp perturbations."""
    ens = workloads.config("C4", n=300)
    o = orc.integrate(ens, orc.params(stop_mode=1))
    sens = {}
    variants = []
    for kw in (dict(h0=10.0 * (1 + 2.0**-52)), dict(h0=10.0 * (1 - 2.0**-53))):
        variants.append((ens, kw))
    for key in ("omega0", "s1hat", "m1"):
        e2 = {k: v.copy() for k, v in ens.items()}
        e2[key] = e2[key] * (1 + 2.0**-52)
        if key == "m1":
            e2["m2"] = 1 - e2["m1"]
        variants.append((e2, {}))
    for e2, kw in variants:  # the oracle's own response to one-ulp perturbations
        e_ulp = parity_errors(orc.integrate(e2, orc.params(stop_mode=1, **kw)), o)
        sens = {k: max(sens.get(k, 0.0), v) for k, v in e_ulp.items()}
    g = run_gpu(pn, ens, stop_mode=1)
    assert np.array_equal(g["status"], o["status"]) and np.all(decided_alike(g, o))
    e = parity_errors(g, o)
    for k, v in e.items():
        assert v <= max(FP64_TOL, 10 * sens[k]), (k, v, sens[k])


@pytest.mark.parametrize("kw", [dict(theta_mode=1), dict(fixed_step=1, h0=20.0),
                                dict(term_mask=0x100), dict(term_mask=0x0FF), dict(rtol=1e-9, atol=1e-9),
                                dict(land_max_iter=1), dict(land_tol=1e-12)])
def test_modes_match_oracle(pn, orc, kw):
    ens = workloads.config("C4", n=300)
    o = orc.integrate(ens, orc.params(**kw))
    g = run_gpu(pn, ens, **kw)
    assert_fp64_parity(g, o)


def test_land_exactly_on_omega_f(pn):
    g = run_gpu(pn, workloads.config("C2", n=2000))
    assert np.all(g["status"] == 0)
    assert np.max(np.abs(g["omega"] / 0.05 - 1)) < 1e-15


@pytest.mark.parametrize("n,precision,pinned", [(5000, 0, True), (300_000, 0, True), (300_000, 2, True),
                                                (300_000, 1, False), (1_048_576, 0, True)])
def test_host_buffer_entry_point_matches_device(pn, n, precision, pinned):
    """The host-buffer entry point against the device-buffer one: bit-identical outputs in every
    precision, from pinned or pageable host memory, up to the bench's 1,048,576 binaries."""
    ens = workloads.config("C1", n=n)
    dev = run_gpu(pn, ens, precision=precision)
    hin = pn.to_device(ens, device="cpu", pin_memory=pinned)
    hout = pn.alloc_outputs(n, device="cpu", pin_memory=pinned)
    with pn.Batch(n, pn.params(precision=precision)) as b:
        pn.pn_batch_integrate_host(b.handle, n, hin, hout)
        h1 = pn.to_numpy(hout)
        pn.pn_batch_integrate_host(b.handle, n - 1000, hin, hout)   # a second, shorter call on the same batch
        h2 = pn.to_numpy(hout)
    for k in dev:
        assert np.array_equal(dev[k], h1[k], equal_nan=True), k
        assert np.array_equal(dev[k][..., :n - 1000], h2[k][..., :n - 1000], equal_nan=True), k


def test_host_async_calls_pipeline_and_match_device(pn):
    """Three asynchronous host-buffer calls in a row (the two staging sets in turn, copies overlapping
    the neighbouring integrations), each into its own output buffers, then one wait: every call's
    outputs are bit-identical to the device-buffer entry point's for its own inputs."""
    import torch
    n = 40_000
    ensa, ensb = workloads.config("C1", n=n), workloads.config("C2", n=n)
    deva, devb = run_gpu(pn, ensa), run_gpu(pn, ensb)
    hina = pn.to_device(ensa, device="cpu", pin_memory=True)
    hinb = pn.to_device(ensb, device="cpu", pin_memory=True)
    outs = [pn.alloc_outputs(n, pin_memory=True) for _ in range(3)]
    with pn.Batch(n) as b:
        pn.pn_batch_integrate_host_async(b.handle, n, hina, outs[0])
        pn.pn_batch_integrate_host_async(b.handle, n, hinb, outs[1])
        pn.pn_batch_integrate_host_async(b.handle, n - 5, hina, outs[2])
        pn.pn_batch_host_wait(b.handle)
    h = [pn.to_numpy(o) for o in outs]
    for k in deva:
        assert np.array_equal(deva[k], h[0][k], equal_nan=True), k
        assert np.array_equal(devb[k], h[1][k], equal_nan=True), k
        assert np.array_equal(deva[k][..., :n - 5], h[2][k][..., :n - 5], equal_nan=True), k


def test_repeat_calls_reuse_graph_and_agree(pn):
    import torch
    ens = workloads.config("C2", n=20000)
    inp = pn.to_device(ens)
    with pn.Batch(20000, pn.params(schedule=2)) as b:
        o1 = pn.to_numpy(b.integrate(inp))
        o2 = pn.to_numpy(b.integrate(inp))
        o3 = pn.to_numpy(b.integrate(inp, n=7000))
        torch.cuda.synchronize()
    for k in o1:
        assert np.array_equal(o1[k], o2[k], equal_nan=True)
        assert np.array_equal(o1[k][..., :7000], o3[k][..., :7000], equal_nan=True)


@pytest.mark.parametrize("schedule", [1, 2])
def test_kernel_timing_events(pn, schedule):
    """pn_batch_timing: the integration kernel's own time (events around it, inside the graph on the
    persistent schedule) is positive, below the whole call's, and most of it on a large batch; the
    times follow the last call (a bounded call included); no call yet is an argument error."""
    import torch
    ens = workloads.config("C1", n=200_000)
    inp = pn.to_device(ens)
    with pn.Batch(200_000, pn.params(schedule=schedule)) as b:
        with pytest.raises(pn.PNError):
            b.timing()
        out0 = pn.alloc_outputs(8)
        pn.pn_batch_integrate(b.handle, 0, inp, out0)  # n = 0: no kernel, so no kernel time yet
        assert np.isnan(b.timing()[1])
        for _ in range(2):  # the second persistent call replays the captured graph
            b.integrate(inp)
            call, kern = b.timing()
            assert 0.0 < kern < call and kern > 0.9 * call, (call, kern)
        out = b.integrate_budget(inp, budget=5)
        call5, kern5 = b.timing()
        assert 0.0 < kern5 < call5 and kern5 < 0.5 * kern, (kern5, kern)
        b.resume(inp, out)
        torch.cuda.synchronize()
        assert b.timing()[1] > 0.0


def test_autotune_choice_gives_same_results(pn):
    import torch
    ens = workloads.config("C2", n=40000)
    inp = pn.to_device(ens)
    ref = run_gpu(pn, ens, schedule=1, block=128)
    with pn.Batch(40000) as b:
        r = b.autotune(inp)
        assert r["n_candidates"] == 9 and r["schedule"] in (1, 2) and r["block"] in (64, 128, 256)
        assert r["bpt"] in (1, 2)
        g = pn.to_numpy(b.integrate(inp))
        torch.cuda.synchronize()
    for k in ref:
        assert np.array_equal(ref[k], g[k], equal_nan=True)


def test_autotune_cache_keys_on_workload_and_parameters(pn):
    """The process's tuning cache: the same inputs and parameters on a new batch reuse the shape
    without timing anything; other inputs (one value changed) or another tolerance tune afresh."""
    ens = workloads.config("C2", n=30000, seed=77)
    inp = pn.to_device(ens)
    with pn.Batch(30000) as b:
        r1 = b.autotune(inp)
    assert r1["n_candidates"] == 9
    with pn.Batch(30000) as b:
        r2 = b.autotune(inp)
        assert b.integrate(inp)["status"].eq(0).all()
    assert r2["n_candidates"] == 0
    assert (r2["schedule"], r2["block"], r2["bpt"], r2["best_ms"]) == (r1["schedule"], r1["block"], r1["bpt"],
                                                                        r1["best_ms"])
    changed = pn.to_device(ens)
    changed["omega0"][12345] = 0.0101
    with pn.Batch(30000) as b:
        assert b.autotune(changed)["n_candidates"] == 9
    with pn.Batch(30000, pn.params(rtol=4e-7)) as b:
        assert b.autotune(inp)["n_candidates"] == 9
    with pn.Batch(30000, pn.params(precision=2)) as b:
        assert b.autotune(inp)["n_candidates"] == 9



def test_sampler_bit_exact_against_oracle(pn, orc):
    import torch
    for d, od in (
        (pn.dist(chi=(0.0, 1.0), chi_mode=1, omega0=(0.01, 0.01)),
         orc.Dist(chi_mode=1, chi_lo=0.0, chi_hi=1.0)),
        (pn.dist(q=(1.0, 4.0), q_mode=1, omega0=(0.005, 0.02)),
         orc.Dist(q_mode=1, q_lo=1.0, q_hi=4.0, omega0_lo=0.005, omega0_hi=0.02)),
    ):
        with pn.Batch(100_000) as b:
            g = b.sample(4242, d, 100_000)
            torch.cuda.synchronize()
            g = {k: g[k].cpu().numpy() for k in pn.api.INPUT_KEYS}
        o = orc.sample(4242, od, 100_000)
        for k in g:
            assert np.array_equal(g[k], o[k]), k
    # log-uniform q uses exp/log, which agree to a few ulp between libraries
    with pn.Batch(50_000) as b:
        g = b.sample(7, pn.dist(q=(1.0, 10.0), q_mode=2), 50_000)
        torch.cuda.synchronize()
        g = {k: g[k].cpu().numpy() for k in pn.api.INPUT_KEYS}
    o = orc.sample(7, orc.Dist(q_mode=2, q_lo=1.0, q_hi=10.0), 50_000)
    assert np.allclose(g["m1"], o["m1"], rtol=4e-16, atol=0)
    for k in ("s1hat", "s2hat", "chi1", "omega0"):
        assert np.array_equal(g[k], o[k])


def test_stats_match_numpy(pn):
    import torch
    ens = workloads.config("SCIENCE", n=20000)
    inp = pn.to_device(ens)
    with pn.Batch(20000) as b:
        out = b.integrate(inp)
        st = b.stats(inp, out)
    g = pn.to_numpy(out)
    x0 = (ens["s1hat"] * ens["s2hat"]).sum(0)
    assert st["count_by_status"][0] == 20000
    assert st["acc_total"] == g["n_acc"].sum() and st["acc_max"] == g["n_acc"].max()
    assert abs(st["pearson_s1s2"] - np.corrcoef(x0, g["dot_s1s2"])[0, 1]) < 1e-10
    assert abs(st["pearson_s1s2"] - 0.99) < 0.01  # Sec. V A prints r = 0.99
    assert st["ms_last_integrate"] > 0


def test_degenerate_configurations(pn, orc):
    """The method's special cases, FP64 against the oracle, and the properties that hold exactly (also in
    both mixed precisions): zero spins (L-hat stays z, dots NaN), spins along L-hat (aligned or
    anti-aligned: nothing precesses), one spin zero, q = 10, omega_f barely above omega0 (the first step
    already crosses), and a tiny spin (1e-12)."""
    n = 6 * 32
    ens = workloads.config("C2", n=n, seed=4711)
    blocks = np.arange(n) // 32
    z = np.array([0.0, 0.0, 1.0])
    zero = blocks == 0
    ens["chi1"][zero] = 0.0
    ens["chi2"][zero] = 0.0
    aligned = blocks == 1
    sign = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    ens["s1hat"][:, aligned] = z[:, None] * sign[aligned]
    ens["s2hat"][:, aligned] = -z[:, None] * sign[aligned]
    one_zero = blocks == 2
    ens["chi2"][one_zero] = 0.0
    q10 = blocks == 3
    ens["m1"][q10], ens["m2"][q10] = 10.0 / 11.0, 1.0 / 11.0
    short = blocks == 4
    ens["omega_f"][short] = ens["omega0"][short] * (1 + 1e-5)
    tiny = blocks == 5
    ens["chi1"][tiny] = 1e-12
    o = orc.integrate(ens)
    g = run_gpu(pn, ens)
    assert np.all(o["status"] == 0)
    assert_fp64_parity(g, o)
    # exact properties on the GPU side
    assert np.all(g["Lhat"][:, zero] == z[:, None]) and np.all(g["S1"][:, zero] == 0.0)
    assert np.all(np.isnan(g["dot_s1s2"][zero])) and np.all(np.isnan(g["dot_ls1"][one_zero | zero]) == zero[one_zero | zero])
    assert np.all(np.isnan(g["dot_ls2"][one_zero]))
    assert np.all(g["Lhat"][:, aligned] == z[:, None])
    assert np.allclose(g["dot_s1s2"][aligned], -1.0, rtol=0, atol=1e-15)
    assert np.all(g["n_acc"][short] == 1) and np.allclose(g["omega"][short], ens["omega_f"][short], rtol=1e-12)
    assert np.all(np.isfinite(g["dot_s1s2"][tiny]))
    for precision in (1, 2):
        m = run_gpu(pn, ens, precision=precision)
        assert np.all(m["status"] == 0)
        assert np.all(m["Lhat"][:, zero | aligned] == z[:, None]) and np.all(m["S1"][:, zero] == 0.0)
        assert np.all(m["n_acc"][short] == 1)


def test_largest_single_batch_64bit_indexing(pn, orc):
    """2^26 binaries in one call (about 37 GB of device buffers: inputs, outputs and the set-up table
    with 37 x 2^26 doubles), drawn on the device by pn_batch_sample; a subsample spread over the whole
    index range, the last 32 binaries included, against the oracle fed by its own sampler."""
    import torch
    n = 1 << 26
    seed = 0x0908_3889_64
    with pn.Batch(n) as b:
        inp = b.sample(seed, pn.dist(q=(1.0, 1.0), chi=(0.0, 1.0), chi_mode=1, omega0=(0.01, 0.01)), n)
        out = b.integrate(inp)
        torch.cuda.synchronize()
        st = b.stats(inp, out)
        idx = np.union1d(workloads.subsample(n, 2048, seed=workloads.SEED_BASE + 107), np.arange(n - 32, n))
        it = torch.from_numpy(idx).cuda()
        g = {k: v.index_select(-1, it).cpu().numpy() for k, v in out.items() if not k.startswith("_")}
    assert st["count_by_status"][0] == n
    ens = orc.sample(seed, orc.Dist(q_mode=0, q_lo=1.0, q_hi=1.0, chi_mode=1, chi_lo=0.0, chi_hi=1.0,
                                    omega0_lo=0.01, omega0_hi=0.01, omega_f=0.05), 0, idx=idx)
    o = orc.integrate(ens)
    assert_fp64_parity(g, o, max_divergent=1)
