"""Hand-written adjoint (pn_batch_adjoint) against the oracle's forward-mode gradient and against
central finite differences of the replayed map (needs a B300)."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-9  # relative, vs the oracle's dual-number gradient of the same discrete map


@pytest.fixture(scope="module")
def pn():
    import torch
    import paper_0908_3889_b300 as pn
    from paper_0908_3889_b300.build import build
    assert torch.cuda.is_available()
    build()
    return pn


OUT = ("dot_s1s2", "dot_ls1", "dot_ls2", "Lx", "Ly", "Lz", "S1x", "S1y", "S1z", "S2x", "S2y", "S2z", "t")
PAR = ("s1x", "s1y", "s1z", "s2x", "s2y", "s2z", "q")


def cotangents(n, seed):
    rng = np.random.default_rng(seed)
    g = rng.normal(size=(13, n))
    g[12] *= 1e-4  # t is O(1e4): keep its term comparable
    return g


def run_adjoint(pn, ens, g, **kw):
    import torch
    inp = pn.to_device(ens)
    cot = {k: torch.from_numpy(np.ascontiguousarray(g[j])).cuda() for j, k in enumerate(OUT)}
    grads = pn.adjoint(inp, cot, **kw)
    return np.stack([grads[p].cpu().numpy() for p in PAR])


def oracle_grads(orc, ens, g):
    n = ens["m1"].shape[0]
    res = np.empty((7, n))
    for i in range(n):
        _, jac, _ = orc.grad(ens, i)
        res[:, i] = g[:, i] @ jac
    return res


def rel_err(a, b):
    """Relative error per gradient component, with components below 1e-3 of their binary's largest
    gradient measured against that 1e-3 floor: such a component is a sum g . J with cancellation,
    whose rounding error scales with the largest terms, not with the component."""
    scale = np.maximum(np.abs(b), np.max(np.abs(b), axis=0, keepdims=True) * 1e-3)
    return np.max(np.abs(a - b) / scale)


@pytest.mark.parametrize("name", ["C4", "C1", "C0"])
def test_adjoint_matches_oracle_forward_mode(pn, orc, name):
    ens = workloads.config(name, n=128, seed=900 + len(name))
    g = cotangents(128, 7)
    got = run_adjoint(pn, ens, g)
    ref = oracle_grads(orc, ens, g)
    assert np.all(np.isfinite(got))
    assert rel_err(got, ref) < GRAD_TOL, rel_err(got, ref)


def test_adjoint_full_size_subsample(pn, orc):
    """65,536 binaries (q ~ U[1,4], chi = 1, omega 0.01 -> 0.05), checkpoint every 64 steps; a 256 subsample
    against the oracle."""
    ens = workloads.config("C4")
    n = ens["m1"].shape[0]
    g = cotangents(n, 11)
    got = run_adjoint(pn, ens, g)
    idx = workloads.subsample(n, 256, seed=workloads.SEED_BASE + 105)
    ref = oracle_grads(orc, workloads.take(ens, idx), g[:, idx])
    assert np.all(np.isfinite(got))
    assert rel_err(got[:, idx], ref) < GRAD_TOL


@pytest.mark.parametrize("precision", [0, 2])
def test_recording_pass_outputs_equal_plain_integration(pn, precision):
    """The adjoint's recording forward pass (its own kernel, in the sweep's precision) integrates exactly
    as pn_batch_integrate in that precision: its outputs are bit-identical, landing moves and output dot
    products included."""
    import torch
    ens = workloads.config("C4", n=3000, seed=905)
    inp = pn.to_device(ens)
    plain = pn.to_numpy(pn.integrate(inp, precision=precision))
    cot = {"dot_s1s2": torch.ones(3000, dtype=torch.float64, device="cuda")}
    grads = {f: torch.empty(3000, dtype=torch.float64, device="cuda") for f in pn.native.GRAD_FIELDS}
    out = pn.alloc_outputs(3000)
    with pn.Batch(3000, pn.params(precision=precision)) as b:
        pn.pn_batch_adjoint(b.handle, 3000, inp, cot, grads, outputs=out)
        torch.cuda.synchronize()
    rec = pn.to_numpy(out)
    for k in plain:
        assert np.array_equal(plain[k], rec[k], equal_nan=True), k


def test_precision_switch_on_one_batch(pn):
    """One batch running the double-single adjoint, then FP64, then double-single again (its per-lane
    segment buffer holds 60 words per step for the double-single sweep and 306 for the FP64 one, and
    grows between them): each call's gradients bit-identical to a fresh batch's in that precision."""
    import torch
    n = 2000
    ens = workloads.config("C4", n=n, seed=907)
    inp = pn.to_device(ens)
    cot = {"dot_s1s2": torch.ones(n, dtype=torch.float64, device="cuda"),
           "Lz": torch.full((n,), 0.25, dtype=torch.float64, device="cuda")}

    def grads_of(b):
        g = {f: torch.empty(n, dtype=torch.float64, device="cuda") for f in pn.native.GRAD_FIELDS}
        pn.pn_batch_adjoint(b.handle, n, inp, cot, g)
        torch.cuda.synchronize()
        return {k: v.cpu().numpy() for k, v in g.items()}

    fresh = {}
    for prec in (0, 2):
        with pn.Batch(n, pn.params(precision=prec)) as b:
            fresh[prec] = grads_of(b)
    with pn.Batch(n, pn.params(precision=2)) as b:
        seq = []
        for prec in (2, 0, 2):
            b.set_params(pn.params(precision=prec))
            seq.append((prec, grads_of(b)))
    for prec, g in seq:
        for k in g:
            assert np.array_equal(g[k], fresh[prec][k], equal_nan=True), (prec, k)


def test_checkpoint_stride_does_not_change_gradients(pn):
    ens = workloads.config("C2", n=500, seed=77)
    g = cotangents(500, 3)
    base = run_adjoint(pn, ens, g, ckpt_every=64)
    for k in (1, 7, 200):
        other = run_adjoint(pn, ens, g, ckpt_every=k)
        assert np.array_equal(base, other), k


def test_adjoint_matches_central_differences(pn, orc):
    """FD (h = 1e-6, central) of the replayed map: same accepted steps, re-landed exactly on omega_f."""
    ens = workloads.config("C4", n=12, seed=31)
    g = cotangents(12, 5)
    got = run_adjoint(pn, ens, g)
    d = 1e-6
    for i in range(12):
        rows, hs = orc.trace(ens, i)
        fd = np.empty(7)
        for k in range(7):
            vals = []
            for sgn in (1, -1):
                p = workloads.take(ens, np.array([i]))
                if k < 3:
                    p["s1hat"][k, 0] += sgn * d
                elif k < 6:
                    p["s2hat"][k - 3, 0] += sgn * d
                else:
                    q = p["m1"][0] / p["m2"][0] + sgn * d
                    p["m1"][0], p["m2"][0] = q / (1 + q), 1 / (1 + q)
                y, t = orc.replay(p, 0, hs)
                S1, S2, L = y[1:4], y[4:7], y[7:10]
                n1, n2, nl = np.linalg.norm(S1), np.linalg.norm(S2), np.linalg.norm(L)
                out = np.concatenate([[S1 @ S2 / (n1 * n2), L @ S1 / (nl * n1), L @ S2 / (nl * n2)], L, S1, S2, [t]])
                vals.append(g[:, i] @ out)
            fd[k] = (vals[0] - vals[1]) / (2 * d)
        assert np.max(np.abs(got[:, i] - fd)) <= 2e-6 * max(1.0, np.max(np.abs(fd))), (i, got[:, i], fd)
    # Fully adaptive central differences (step sequence free to change) differ from the frozen-step
    # gradient by the step control's own sensitivity: reported, not gated.
    adaptive = []
    for i in range(4):
        fd = np.empty(7)
        for k in range(7):
            vals = []
            for sgn in (1, -1):
                p = workloads.take(ens, np.array([i]))
                if k < 3:
                    p["s1hat"][k, 0] += sgn * d
                elif k < 6:
                    p["s2hat"][k - 3, 0] += sgn * d
                else:
                    q = p["m1"][0] / p["m2"][0] + sgn * d
                    p["m1"][0], p["m2"][0] = q / (1 + q), 1 / (1 + q)
                o = orc.integrate(p)
                out = np.concatenate([[o["dot_s1s2"][0], o["dot_ls1"][0], o["dot_ls2"][0]], o["Lhat"][:, 0],
                                      o["S1"][:, 0], o["S2"][:, 0], [o["t"][0]]])
                vals.append(g[:, i] @ out)
            fd[k] = (vals[0] - vals[1]) / (2 * d)
        adaptive.append(np.max(np.abs(got[:, i] - fd)) / max(1.0, np.max(np.abs(fd))))
    print("adaptive-FD vs frozen-step adjoint, max scaled difference per binary:", adaptive)
    assert np.all(np.isfinite(adaptive))


def test_autograd_function_backward(pn):
    import torch
    ens = workloads.config("C4", n=64, seed=41)
    dev = "cuda"
    T = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)
    s1 = T(ens["s1hat"]).requires_grad_(True)
    s2 = T(ens["s2hat"]).requires_grad_(True)
    q = T(ens["m1"] / ens["m2"]).requires_grad_(True)
    outs = pn.PNAdjointFn.apply(s1, s2, q, T(ens["chi1"]), T(ens["chi2"]), T(ens["omega0"]), T(ens["omega_f"]),
                                T(ens["lhat"]))
    loss = outs[0].sum() + 0.5 * outs[3][2].sum()
    loss.backward()
    g = np.zeros((13, 64))
    g[0] = 1.0
    g[5] = 0.5
    ref = run_adjoint(pn, ens, g)
    got = np.concatenate([s1.grad.cpu().numpy(), s2.grad.cpu().numpy(), q.grad.cpu().numpy()[None]])
    assert np.allclose(got, ref, rtol=1e-9, atol=1e-12)  # m1, m2 round-trip through q = m1/m2


def test_masses_from_mass_ratio_on_the_device(pn):
    """pn_batch_masses: m1 = q/(1+q), m2 = 1/(1+q), bit for bit the IEEE divisions of the rounded 1 + q,
    over the ratios the workloads use and the extremes of the sampler's range; a ragged n leaves the
    elements beyond n untouched."""
    import torch
    rng = np.random.default_rng(7)
    q = np.concatenate([np.exp(rng.uniform(0.0, np.log(10.0), 1000)), rng.uniform(1.0, 4.0, 1000),
                        [1.0, 10.0, 0.4 / 0.6, 1e-300, 1e300]])
    n = q.shape[0]
    qd = torch.tensor(q, dtype=torch.float64, device="cuda")
    m = torch.full((2, n + 3), -7.0, dtype=torch.float64, device="cuda")
    with pn.Batch(n + 3) as b:
        pn.pn_batch_masses(b.handle, n, qd, m[0], m[1])
        torch.cuda.synchronize()
    got = m.cpu().numpy()
    one_q = 1.0 + q
    assert np.array_equal(got[0, :n], q / one_q) and np.array_equal(got[1, :n], 1.0 / one_q)
    assert np.all(got[:, n:] == -7.0)


DS_GRAD_TOL = 1e-8  # double-single sweep: ~48-bit arithmetic through a few hundred steps


@pytest.mark.parametrize("name", ["C4", "C2"])
def test_double_single_sweep_matches_oracle(pn, orc, name):
    """The reverse sweep in double-single arithmetic (precision PN_MIXED_DS) against the oracle's
    forward-mode gradient of the FP64 map and against the FP64 sweep."""
    ens = workloads.config(name, n=160, seed=300 + len(name))
    g = cotangents(160, 17)
    got = run_adjoint(pn, ens, g, precision=2)
    ref = oracle_grads(orc, ens, g)
    assert np.all(np.isfinite(got))
    assert rel_err(got, ref) < DS_GRAD_TOL, rel_err(got, ref)
    fp64 = run_adjoint(pn, ens, g)
    assert rel_err(got, fp64) < DS_GRAD_TOL


def test_double_single_sweep_full_size_subsample(pn, orc):
    ens = workloads.config("C4")
    n = ens["m1"].shape[0]
    g = cotangents(n, 13)
    got = run_adjoint(pn, ens, g, precision=2)
    idx = workloads.subsample(n, 256, seed=workloads.SEED_BASE + 106)
    ref = oracle_grads(orc, workloads.take(ens, idx), g[:, idx])
    assert np.all(np.isfinite(got))
    assert rel_err(got[:, idx], ref) < DS_GRAD_TOL


def test_adjoint_refuses_other_modes(pn):
    import torch
    ens = workloads.config("C4", n=8)
    inp = pn.to_device(ens)
    grads = {f: torch.empty(8, dtype=torch.float64, device="cuda") for f in pn.native.GRAD_FIELDS}
    for kw in (dict(precision=1), dict(stop_mode=1)):
        with pn.Batch(8, pn.params(**kw)) as b:
            with pytest.raises(pn.PNError, match="UNIMPLEMENTED"):
                pn.pn_batch_adjoint(b.handle, 8, inp, {}, grads)


def test_adjoint_uneven_lengths_bad_inputs_and_record_growth(pn, orc):
    """Binaries of very different lengths (the ordering by step count puts several lengths in one warp),
    a few invalid inputs (their gradients are NaN, the rest unaffected), and one binary longer than the
    default 256-step record, which makes the library grow the record and rerun the recording pass."""
    n = 70
    ens = workloads.config("C2", n=n, seed=4242)
    ens["omega0"][0] = 0.0025  # ~300 accepted steps
    bad = np.array([5, 17, 40])
    ens["m2"][bad] = ens["m1"][bad]  # m1 + m2 != 1: BAD_INPUT
    g = cotangents(n, 19)
    got = run_adjoint(pn, ens, g)
    assert np.all(np.isnan(got[:, bad]))
    good = np.setdiff1d(np.arange(n), bad)
    o = orc.integrate(ens)
    assert o["n_acc"][0] > 256 and np.all(o["status"][bad] == 4)
    ref = oracle_grads(orc, workloads.take(ens, good), g[:, good])
    assert np.all(np.isfinite(got[:, good]))
    assert rel_err(got[:, good], ref) < GRAD_TOL


@pytest.mark.parametrize("n", [1, 33])
def test_adjoint_small_ragged_batches(pn, orc, n):
    ens = workloads.config("C4", n=n, seed=600 + n)
    g = cotangents(n, n)
    got = run_adjoint(pn, ens, g)
    ref = oracle_grads(orc, ens, g)
    assert rel_err(got, ref) < GRAD_TOL


def test_tangent_projected_spin_gradients(pn):
    """The optional *_tan outputs are g - (g . s) s / |s|^2: orthogonal to s, equal to the projection."""
    import torch
    ens = workloads.config("C4", n=96, seed=73)
    g = cotangents(96, 23)
    inp = pn.to_device(ens)
    cot = {k: torch.from_numpy(np.ascontiguousarray(g[j])).cuda() for j, k in enumerate(OUT)}
    grads = {k: v.cpu().numpy() for k, v in pn.adjoint(inp, cot, tangent=True).items()}
    for sp, key in (("s1", "s1hat"), ("s2", "s2hat")):
        full = np.stack([grads[sp + a] for a in "xyz"])
        tan = np.stack([grads[sp + a + "_tan"] for a in "xyz"])
        s = ens[key]
        proj = full - (np.sum(full * s, axis=0) / np.sum(s * s, axis=0)) * s
        assert np.allclose(tan, proj, rtol=1e-12, atol=1e-14 * np.max(np.abs(full)))
        assert np.max(np.abs(np.sum(tan * s, axis=0))) <= 1e-12 * np.max(np.abs(full))


def _angles(s):
    return np.arccos(np.clip(s[2] / np.linalg.norm(s, axis=0), -1, 1)), np.arctan2(s[1], s[0])


def _direction(theta, phi, norm):
    return norm * np.stack([np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi), np.cos(theta)])


def test_angle_gradients_chain_rule_and_replayed_fd(pn, orc):
    """d/dtheta, d/dphi of each initial spin direction: equal to the chain rule applied to the component
    gradients, and to central differences (h = 1e-6) of the replayed map in the angles."""
    import torch
    n = 10
    ens = workloads.config("C4", n=n, seed=91)
    g = cotangents(n, 29)
    inp = pn.to_device(ens)
    cot = {k: torch.from_numpy(np.ascontiguousarray(g[j])).cuda() for j, k in enumerate(OUT)}
    gr = {k: v.cpu().numpy() for k, v in pn.adjoint(inp, cot, angles=True).items()}
    for sp, key in (("s1", "s1hat"), ("s2", "s2hat")):
        s = ens[key]
        th, ph = _angles(s)
        full = np.stack([gr[sp + a] for a in "xyz"])
        d_th = np.stack([np.cos(th) * np.cos(ph), np.cos(th) * np.sin(ph), -np.sin(th)])
        d_ph = np.stack([-np.sin(th) * np.sin(ph), np.sin(th) * np.cos(ph), np.zeros(n)])
        scale = np.max(np.abs(full))
        assert np.allclose(gr[sp + "_dtheta"], np.sum(full * d_th, axis=0), rtol=1e-10, atol=1e-12 * scale)
        assert np.allclose(gr[sp + "_dphi"], np.sum(full * d_ph, axis=0), rtol=1e-10, atol=1e-12 * scale)
    d = 1e-6
    for i in range(4):
        rows, hs = orc.trace(ens, i)
        for sp, key in (("s1", "s1hat"), ("s2", "s2hat")):
            for which in ("theta", "phi"):
                vals = []
                for sgn in (1, -1):
                    p = workloads.take(ens, np.array([i]))
                    th, ph = _angles(p[key])
                    if which == "theta":
                        th = th + sgn * d
                    else:
                        ph = ph + sgn * d
                    p[key] = _direction(th, ph, np.linalg.norm(p[key], axis=0))
                    y, t = orc.replay(p, 0, hs)
                    S1, S2, L = y[1:4], y[4:7], y[7:10]
                    n1, n2, nl = np.linalg.norm(S1), np.linalg.norm(S2), np.linalg.norm(L)
                    out = np.concatenate([[S1 @ S2 / (n1 * n2), L @ S1 / (nl * n1), L @ S2 / (nl * n2)], L, S1, S2,
                                          [t]])
                    vals.append(g[:, i] @ out)
                fd = (vals[0] - vals[1]) / (2 * d)
                got = gr[f"{sp}_d{which}"][i]
                assert abs(got - fd) <= 2e-6 * max(1.0, abs(fd)), (i, sp, which, got, fd)


def test_gradient_step_on_angles_moves_the_final_alignment(pn):
    """Sensitivity exploration with the adjoint: one gradient-ascent step on the four initial spin angles
    of each binary raises its final S1-hat.S2-hat by the first-order amount eps |grad|^2."""
    import torch
    n = 512
    ens = workloads.config("C4", n=n, seed=57)
    inp = pn.to_device(ens)
    cot = {"dot_s1s2": torch.ones(n, dtype=torch.float64, device="cuda")}
    gr = {k: v.cpu().numpy() for k, v in pn.adjoint(inp, cot, angles=True).items()}
    grad = np.stack([gr["s1_dtheta"], gr["s1_dphi"], gr["s2_dtheta"], gr["s2_dphi"]])
    base = pn.to_numpy(pn.integrate(inp))["dot_s1s2"]
    eps = 1e-4 / np.maximum(np.linalg.norm(grad, axis=0), 1e-3)  # angle step of 1e-4 rad along the gradient
    moved = {k: v.copy() for k, v in ens.items()}
    for k, key in ((0, "s1hat"), (2, "s2hat")):
        th, ph = _angles(ens[key])
        moved[key] = _direction(th + eps * grad[k], ph + eps * grad[k + 1], np.linalg.norm(ens[key], axis=0))
    after = pn.to_numpy(pn.integrate(pn.to_device(moved)))["dot_s1s2"]
    gain = after - base
    predicted = eps * np.sum(grad * grad, axis=0)
    big = predicted > 1e-5  # well above the step-control noise of the adaptive re-integration
    assert big.sum() > n // 2
    ratio = gain[big] / predicted[big]
    assert np.mean(gain[big] > 0) >= 0.98
    assert abs(np.median(ratio) - 1.0) < 0.05, np.median(ratio)
