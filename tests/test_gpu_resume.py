"""Bounded integration with resume (pn_batch_integrate_budget / pn_batch_resume) against one
uninterrupted pn_batch_integrate call: bit-identical results (needs a B300)."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

RUNNING = 6


@pytest.fixture(scope="module")
def pn():
    import torch
    import paper_0908_3889_b300 as pn
    from paper_0908_3889_b300.build import build
    assert torch.cuda.is_available()
    build()
    return pn


def bounded_run(pn, b, inp, first, step):
    import torch
    out = b.integrate_budget(inp, budget=first)
    torch.cuda.synchronize()
    calls, running = 1, []
    while True:
        st = pn.to_numpy(out)["status"]
        running.append(int((st == RUNNING).sum()))
        if running[-1] == 0:
            break
        b.resume(inp, out, budget=step)
        calls += 1
        assert calls < 10_000
    torch.cuda.synchronize()
    return pn.to_numpy(out), calls, running


@pytest.mark.parametrize("precision", [0, 1, 2])
@pytest.mark.parametrize("schedule", [1, 2])
def test_bounded_run_is_bit_identical(pn, precision, schedule):
    import torch
    ens = workloads.config("C2", n=3000, seed=8080)  # lengths from ~10 to ~260 accepted steps
    inp = pn.to_device(ens)
    with pn.Batch(3000, pn.params(precision=precision, schedule=schedule, block=128)) as b:
        ref = pn.to_numpy(b.integrate(inp))
        torch.cuda.synchronize()
        got, calls, running = bounded_run(pn, b, inp, first=7, step=13)
    assert calls > 10 and running[0] > 2900 and running == sorted(running, reverse=True)
    for k in ref:
        assert np.array_equal(ref[k], got[k], equal_nan=True), k


def test_running_binaries_report_their_current_state(pn):
    import torch
    ens = workloads.config("C1", n=512, seed=99)
    inp = pn.to_device(ens)
    with pn.Batch(512) as b:
        full = pn.to_numpy(b.integrate(inp))
        torch.cuda.synchronize()
        out = b.integrate_budget(inp, budget=10)
        st = b.stats(inp, out)
        part = pn.to_numpy(out)
        assert st["count_by_status"][RUNNING] == 512
        assert np.all(part["t"] < full["t"]) and np.all(part["omega"] < full["omega"])
        assert np.all(part["n_acc"] + part["n_rej"] <= 10)
        b.resume(inp, out)  # budget 0: to the end in one call
        torch.cuda.synchronize()
        done = pn.to_numpy(out)
    for k in full:
        assert np.array_equal(full[k], done[k], equal_nan=True), k


def test_budget_with_max_steps_and_bad_inputs(pn):
    import torch
    ens = workloads.config("C2", n=400, seed=77)
    ens["chi1"][[3, 50]] = 1.5  # BAD_INPUT
    inp = pn.to_device(ens)
    with pn.Batch(400, pn.params(max_steps=60)) as b:
        ref = pn.to_numpy(b.integrate(inp))
        torch.cuda.synchronize()
        got, _, _ = bounded_run(pn, b, inp, first=5, step=9)
    assert np.sum(ref["status"] == 1) > 0 and np.all(ref["status"][[3, 50]] == 4)
    for k in ref:
        assert np.array_equal(ref[k], got[k], equal_nan=True), k


def test_bounded_call_argument_errors(pn):
    ens = workloads.config("C0", n=8)
    inp = pn.to_device(ens)
    out = pn.alloc_outputs(8, inp["m1"].device)
    with pn.Batch(8) as b:
        with pytest.raises(pn.PNError, match="budget"):
            b.integrate_budget(inp, out, budget=0)
        with pytest.raises(pn.PNError, match="resume"):
            b.resume(inp, out)
        with pytest.raises(pn.PNError, match="budget"):
            pn.pn_batch_resume(b.handle, 8, inp, out, -1)


def test_resume_refuses_a_changed_precision(pn):
    """The saved states are kept as the run's precision carries them, so a resume under another
    precision is an argument error, and the run then still continues under its own."""
    import torch
    ens = workloads.config("C1", n=256, seed=7)
    inp = pn.to_device(ens)
    with pn.Batch(256, pn.params(precision=2)) as b:
        ref = pn.to_numpy(b.integrate(inp))
        out = b.integrate_budget(inp, budget=10)
        b.set_params(pn.params(precision=0))
        with pytest.raises(pn.PNError, match="precision"):
            b.resume(inp, out)
        b.set_params(pn.params(precision=2))
        b.resume(inp, out)
        torch.cuda.synchronize()
        done = pn.to_numpy(out)
    for k in ref:
        assert np.array_equal(ref[k], done[k], equal_nan=True), k
