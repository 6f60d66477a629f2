"""GPU adjoint: 2F and d2F/d(f, f1dot, alpha, delta) at off-grid parameters.

Checked against the oracle's analytic-plus-numeric gradient, against
central finite differences of the GPU's own 2F (step 1e-3 of the grid
spacing), through torch.autograd, and by gradient-ascent refinement
recovering injected signals.
"""

import numpy as np
import pytest
import torch

import paper_2201_00451_gb300 as pkg
from oracle import grad as og
from oracle import synth
from paper_2201_00451_gb300 import refine as rf
from workloads import small_target

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2201_00451_gb300 import build as fbuild

    fbuild.build()
    pkg.load()


def _setup(seed, noise=True, n=20000, rho2=150.0):
    t = small_target(n_samples=n, dt=1.0, n_fft=1 << 15, n_det=2, n_inj=1, rho2_range=(rho2, rho2),
                     seed=seed, f1dots=(-1e-9,), f2dots=(0.0,), dtype="c64")
    x = synth.make_data(t, noise=noise)
    plan = pkg.FstatPlan.from_target(t)
    for X in range(2):
        plan.set_data(X, x[X], t.sigmas[X])
    return t, x, plan


def _cands(rows, f2dot=0.0):
    c = np.empty(len(rows), dtype=pkg.CANDIDATE_DTYPE)
    rows = np.asarray(rows, dtype=np.float64)
    c["f"], c["f1dot"], c["alpha"], c["delta"] = rows.T
    c["f2dot"] = f2dot
    return c


def _scales(t):
    return np.array([1.0 / t.t_span, 1.0 / t.t_span ** 2, 1e-3, 1e-3])


def test_twoF_and_gradient_match_oracle():
    t, x, plan = _setup(41)
    inj = t.injections[0]
    rng = np.random.default_rng(1)
    base = np.array([inj.f0, inj.f1dot, inj.alpha, inj.delta])
    rows = [base + rng.uniform(-0.5, 0.5, 4) * _scales(t) for _ in range(4)]
    two_f, g = plan.grad(_cands(rows))
    two_f, g = two_f.cpu().numpy(), g.cpu().numpy()
    s = _scales(t)
    for i, th in enumerate(rows):
        v, gr = og.grad(t, x, th)
        assert abs(two_f[i] - v) <= 1e-4 * abs(v) + 1e-3
        # compare gradient components on the natural scales
        assert np.all(np.abs((g[i] - gr) * s) <= 2e-3 * abs(v) + 2e-3), (g[i] * s, gr * s)
    plan.close()


def test_gradient_matches_central_differences_of_gpu_2F():
    t, x, plan = _setup(42)
    inj = t.injections[0]
    s = _scales(t)
    base = np.array([inj.f0, inj.f1dot, inj.alpha, inj.delta]) + np.array([0.3, -0.2, 0.4, -0.3]) * s
    two_f, g = plan.grad(_cands([base]))
    g = g.cpu().numpy()[0]
    for i in range(4):
        h = 1e-3 * s[i]
        tp, tm = base.copy(), base.copy()
        tp[i] += h
        tm[i] -= h
        vp, _ = plan.grad(_cands([tp]))
        vm, _ = plan.grad(_cands([tm]))
        fd = (float(vp[0]) - float(vm[0])) / (2 * h)
        assert abs(g[i] - fd) * s[i] <= 0.02 * abs(g[i]) * s[i] + 2e-3 * float(two_f[0]) + 0.02, (i, g[i], fd)
    plan.close()


def test_autograd_function_returns_adjoint_gradient():
    t, x, plan = _setup(43)
    inj = t.injections[0]
    theta = torch.tensor([[inj.f0, inj.f1dot, inj.alpha, inj.delta]], dtype=torch.float64,
                         requires_grad=True)
    out = rf.twoF(theta, plan)
    (2.0 * out.sum()).backward()
    _, g = plan.grad(_cands(theta.detach().numpy()))
    assert torch.allclose(theta.grad, 2.0 * g.double().cpu(), rtol=1e-6, atol=0)
    plan.close()


def test_refinement_recovers_noise_free_injection():
    t, x, plan = _setup(44, noise=False, rho2=200.0)
    inj = t.injections[0]
    s = _scales(t)
    rng = np.random.default_rng(4)
    truth = np.array([inj.f0, inj.f1dot, inj.alpha, inj.delta])
    start = np.array([truth + rng.uniform(-0.5, 0.5, 4) * s * np.array([1, 1, 0, 0]) for _ in range(8)])
    theta, hist = rf.refine(plan, start, s, steps=20)
    hist = hist.numpy()
    assert np.all(hist[-1] >= hist[0])
    assert np.all(hist[-1] > 0.95 * inj.rho2)
    plan.close()


def _host_ascent(plan, theta, s, steps, step0=0.25):
    # The ascent rule written out on the host over fstat_grad, each double
    # operation rounded on its own in the order the rule states it.
    theta = np.array(theta, dtype=np.float64)
    eta = np.full(len(theta), step0)
    cur, g = plan.grad(_cands(theta))
    cur, g = cur.cpu().numpy(), g.cpu().numpy().astype(np.float64)
    hist = [cur.copy()]
    for _ in range(steps):
        sg = g * s
        sq = sg * sg
        nrm = np.sqrt(((sq[:, 0] + sq[:, 1]) + sq[:, 2]) + sq[:, 3])
        step = eta / np.maximum(nrm, 1e-300)
        trial = theta + (step[:, None] * sg) * s
        val, gt = plan.grad(_cands(trial))
        val, gt = val.cpu().numpy(), gt.cpu().numpy().astype(np.float64)
        ok = val > cur
        theta = np.where(ok[:, None], trial, theta)
        cur = np.where(ok, val, cur)
        g = np.where(ok[:, None], gt, g)
        eta = np.where(ok, eta * 1.25, eta * 0.5)
        hist.append(cur.copy())
    return theta, np.array(hist)


def test_device_ascent_equals_the_host_rule():
    # fstat_refine (the loop on the device) against the same rule on the
    # host over fstat_grad: identical candidates and 2F history, bit for bit
    t, x, plan = _setup(45, rho2=180.0)
    inj = t.injections[0]
    s = _scales(t)
    rng = np.random.default_rng(6)
    truth = np.array([inj.f0, inj.f1dot, inj.alpha, inj.delta])
    start = truth + rng.uniform(-0.6, 0.6, (37, 4)) * s
    th_h, hist_h = _host_ascent(plan, start, s, 12)
    out, hist_d = plan.refine(_cands(start), s, steps=12)
    th_d = np.stack([out["f"], out["f1dot"], out["alpha"], out["delta"]], axis=1)
    assert np.array_equal(hist_d, hist_h.astype(np.float32))
    assert np.array_equal(th_d, th_h)
    assert np.all(out["f2dot"] == 0.0)
    # zero steps: the start and its 2F; bad arguments are refused
    out0, h0 = plan.refine(_cands(start[:3]), s, steps=0)
    assert np.array_equal(np.stack([out0["f"], out0["f1dot"], out0["alpha"], out0["delta"]], 1), start[:3])
    assert np.array_equal(h0[0], hist_h[0][:3].astype(np.float32))
    for bad_s, bad_steps, bad_eta in ((s * np.array([1, 0, 1, 1]), 3, 0.25), (s, -1, 0.25), (s, 3, 0.0)):
        with pytest.raises(pkg.FstatError) as e:
            plan.refine(_cands(start[:3]), bad_s, steps=bad_steps, step0=bad_eta)
        assert e.value.code == -1
    plan.close()


def test_full_size_refinement_recovers_injections():
    # The 10-day two-detector data (10 injections), 4096 candidates seeded
    # +-0.5 grid step off the injections in (f, f1dot, alpha, delta), 20 ascent
    # steps; the refined 2F is compared with the oracle's 2F at the truth.
    from workloads import config2

    t = config2()
    x = synth.make_data(t)
    plan = pkg.FstatPlan.from_target(t)
    for X in range(2):
        plan.set_data(X, x[X], t.sigmas[X])
    scales = np.array([1.0 / t.t_span, 1.0 / t.t_span ** 2, np.radians(1 / 60), np.radians(1 / 60)])
    rng = np.random.default_rng(9)
    truth = np.array([[i.f0, i.f1dot, i.alpha, i.delta] for i in t.injections])
    owner = np.arange(4096) % len(truth)
    start = truth[owner] + rng.uniform(-0.5, 0.5, (4096, 4)) * scales
    theta, hist = rf.refine(plan, start, scales, steps=20)
    hist = hist.numpy()
    plan.close()
    assert np.all(hist[-1] >= hist[0])
    ref = np.array([og.twoF_at(t, x, th) for th in truth])
    got = np.array([hist[-1][owner == k].max() for k in range(len(truth))])
    med = np.array([np.median(hist[-1][owner == k]) for k in range(len(truth))])
    assert np.all(got >= 0.97 * ref), (got, ref)
    assert np.all(med >= 0.85 * ref), (med, ref)
