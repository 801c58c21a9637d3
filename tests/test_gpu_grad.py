"""Gradient of the log-likelihood (ppm_loglike_grad, hand-written adjoints)
against the FP64 oracle's forward-mode derivative and against central finite
differences of the oracle (step 1e-5 relative); tolerance 1e-3 relative per
component (plus a floor of 1e-5 of the largest scale-weighted component for
components near zero).

The model is piecewise smooth (template visibility, interpolation intervals);
where a difference step could straddle a branch change, the reference is
first checked against a second step size and only components whose two
references agree are compared.
"""
import math

import numpy as np
import pytest

from gpu_helpers import context
from grad_helpers import (NAMES, grad_tol, n_params, oracle_fd, oracle_ll, single)

pytestmark = pytest.mark.gpu

DEG = math.pi / 180.0


def gpu_grad(w, counts=None):
    import torch
    import paper_2510_07764_gb300 as ppm
    ctx = context(w)
    dp = ppm.DeviceParams(w.inst)
    cnt = torch.from_numpy(np.ascontiguousarray(w.counts if counts is None else counts)).cuda()
    ll, g = ctx.loglike_grad(dp, cnt, w.tau)
    ctx.sync()
    return ll.cpu().numpy(), g.cpu().numpy(), ctx.last_status.cpu().numpy()


def visible_two_cap(synth, atm, lens, **kw):
    """Two caps that stay on the visible hemisphere at every phase, with
    temperatures between table nodes."""
    w = synth.atm_two_spot(atm=atm, lens=lens, **kw)
    i = w.inst
    i.incl_rad[0] = 30 * DEG
    i.colat[0] = [25 * DEG, 55 * DEG]
    i.azim[0] = [0.3, math.pi]
    i.zeta[0] = [0.2, 0.15]
    i.logT[0] = [6.112, 6.023]
    i.mask_zeta[0] = [0.0, 0.0]
    return w


def counts_from_model(orc, w, seed=7):
    """Poisson counts drawn from the oracle's model of w on its own energy
    grid and response (bins without model flux get no counts, so logL stays
    finite where a generic count map would meet a zero or underflowing
    model)."""
    C = orc.counts_model(orc.profile(w), w.R, w.sigma_ism, float(w.inst.nh_1e20[0]))
    rng = np.random.default_rng(seed)
    return rng.poisson(np.maximum(w.tau * C, 0.0)).astype(np.int32)


def _check(g, ref, mask=None):
    assert np.isfinite(g).all() and np.isfinite(ref).all(), (g, ref)
    tol = grad_tol(ref)
    bad = np.abs(g - ref) > tol
    if mask is not None:
        bad &= mask
    assert not bad.any(), "\n".join(
        "%-10s gpu %.9e ref %.9e rel %.2e" % (NAMES[j], g[j], ref[j], abs(g[j] / ref[j] - 1))
        for j in np.nonzero(bad)[0])


def test_grad_two_caps_visible(orc, synth, atm, small_lens):
    w = visible_two_cap(synth, atm, small_lens, n_theta=16, n_phi=24, n_phase=32, n_E=64,
                        n_chan=40)
    ll, g, st = gpu_grad(w)
    assert st[0] == 0
    assert abs(ll[0] - oracle_ll(orc, w)) < 1e-3 * abs(ll[0])
    _check(g[0, :13], orc.grad_tangent(w))
    _check(g[0, :13], oracle_fd(orc, w, rel=1e-5))


def test_grad_cap_and_ring_with_limb(orc, synth, atm, small_lens):
    """The two-spot workload (a cap and a masked ring crossing the limb, 60 deg
    inclination), temperatures moved off the table nodes."""
    w = synth.atm_two_spot(n_theta=16, n_phi=24, n_phase=32, n_E=64, n_chan=40, atm=atm,
                           lens=small_lens)
    w.inst.logT[0] = [6.112, 6.023]
    ll, g, st = gpu_grad(w)
    assert st[0] == 0
    _check(g[0, :13], orc.grad_tangent(w))
    ref = oracle_fd(orc, w, rel=1e-5)
    ref2 = oracle_fd(orc, w, rel=5e-6)
    smooth = np.abs(ref - ref2) <= 1e-4 * np.abs(ref) + 1e-7 * np.max(np.abs(ref))
    assert smooth.sum() >= 10, "finite differences straddle branch changes in %d components" % (
        13 - smooth.sum())
    _check(g[0, :13], ref, mask=smooth)


def test_grad_one_spot_blackbody(orc, synth, small_lens):
    """Analytic blackbody emission (the logT derivative through kT), one cap."""
    w = synth.bb_small(n_theta=16, n_phi=20, n_phase=32, n_E=32, lens=small_lens)
    w = synth._with_response(w, 24, tau=1.0e3)
    w.inst.logT[0, 0] = 6.1
    ll, g, st = gpu_grad(w)
    assert st[0] == 0
    assert n_params(w.inst) == 9
    _check(g[0, :9], orc.grad_tangent(w))
    _check(g[0, :9], oracle_fd(orc, w, rel=1e-5))
    assert np.all(g[0, 9:] == 0.0)


def test_grad_batch_matches_single_and_flags_out_of_range(synth, atm, small_lens):
    w = visible_two_cap(synth, atm, small_lens, n_theta=12, n_phi=16, n_phase=32, n_E=48,
                        n_chan=30)
    inst = w.inst.select([0, 0, 0])
    inst.n_theta[:] = [12, 20, 12]
    inst.n_phi[:] = [16, 28, 16]
    inst.mass_msun[2] = 2.2      # u = 0.54, beyond the lens grid
    inst.incl_rad[1] = 40 * DEG
    w3 = synth.Workload("b", inst, small_lens, w.E_keV, atm=atm, R=w.R, sigma_ism=w.sigma_ism,
                        counts=np.concatenate([w.counts] * 3), tau=w.tau)
    ll, g, st = gpu_grad(w3)
    assert list(st) == [0, 0, 2]
    assert np.all(np.isnan(g[2])) and ll[2] == -np.inf
    for b in range(2):
        llb, gb, _ = gpu_grad(single(w3, b))
        assert abs(ll[b] - llb[0]) <= 1e-6 * abs(llb[0])
        assert np.all(np.abs(g[b] - gb[0]) <= grad_tol(gb[0], rtol=1e-5, floor=1e-7))


def test_autograd_function(synth, atm, small_lens):
    import torch
    import paper_2510_07764_gb300 as ppm
    w = visible_two_cap(synth, atm, small_lens, n_theta=8, n_phi=12, n_phase=32, n_E=48,
                        n_chan=30)
    inst = w.inst.select([0, 0])
    inst.incl_rad[1] = 35 * DEG
    w2 = synth.Workload("b", inst, small_lens, w.E_keV, atm=atm, R=w.R, sigma_ism=w.sigma_ism,
                        counts=np.concatenate([w.counts] * 2), tau=w.tau)
    ctx = context(w2)
    dp = ppm.DeviceParams(w2.inst)
    cnt = torch.from_numpy(w2.counts).cuda()
    theta = dp.theta().clone().requires_grad_(True)
    ll = ppm.LogLikelihood(theta, ctx, dp, cnt, w2.tau)
    (gt,) = torch.autograd.grad((ll * torch.tensor([1.0, -2.0], device="cuda",
                                                   dtype=torch.float64)).sum(), theta)
    _, g = ctx.loglike_grad(dp, cnt, w2.tau)
    # two calls: the backward adds in a fixed order, so they agree bit for bit
    assert torch.equal(gt[0], g[0])
    assert torch.equal(gt[1], -2.0 * g[1])


def test_grad_full_size_directional(synth, atm):
    """The differentiated workload's resolution (two caps, 128 x 128 elements,
    128 phases, 256 energies, 300 channels, default lens grid): the gradient
    against central differences of the GPU logL along three directions (the
    forward is FP32, so the step is 1e-4 relative and the tolerance 1e-2)."""
    import torch
    import paper_2510_07764_gb300 as ppm
    w = visible_two_cap(synth, atm, None)
    ctx = context(w)
    dp = ppm.DeviceParams(w.inst)
    cnt = torch.from_numpy(w.counts).cuda()
    _, g = ctx.loglike_grad(dp, cnt, w.tau)
    g = g[0].cpu().numpy()
    th0 = dp.theta()
    sc = torch.tensor([1.0, 10.0, 1.0, 0.3, 1.0, 1.0, 1.0, 0.2, 6.0, 1.0, 1.0, 0.2, 6.0],
                      dtype=torch.float64, device="cuda")
    rng = np.random.default_rng(7)
    for _ in range(3):
        v = torch.from_numpy(rng.standard_normal(13)).cuda() * sc
        h = 1e-4
        lls = []
        for sgn in (1.0, -1.0):
            dp.set_theta(th0 + sgn * h * v)
            lls.append(float(ctx.loglike(dp, cnt, w.tau)[0]))
        dp.set_theta(th0)
        fd = (lls[0] - lls[1]) / (2 * h)
        gv = float(np.dot(g, v.cpu().numpy()))
        assert abs(gv - fd) <= 1e-2 * abs(fd) + 1e-3 * float(np.sum(np.abs(g * v.cpu().numpy())))


def test_grad_with_phase_sub_samples(orc, synth, atm, small_lens):
    w = visible_two_cap(synth, atm, small_lens, n_theta=10, n_phi=12, n_phase=16, n_E=40,
                        n_chan=20)
    w.inst.phase_sub = 4
    ll, g, st = gpu_grad(w)
    assert st[0] == 0
    _check(g[0, :13], orc.grad_tangent(w))


@pytest.mark.parametrize("strategy", ["d", "a"])
def test_grad_energies_past_the_table_edges(orc, synth, atm, small_lens, strategy):
    """Energies from 0.06 to 9.5 keV put redshifted queries beyond both ends of
    the table's energy axis (clamped) and on its edge intervals (linear for the
    method's scheme, one-sided cubic for strategy a): the backward pass's
    general path."""
    w = visible_two_cap(synth, atm, small_lens, n_theta=8, n_phi=12, n_phase=16, n_E=40,
                        n_chan=20)
    w.E_keV = synth.logspace(0.06, 9.5, 40)
    w.R = synth.response(w.E_keV, 20)
    w.sigma_ism = synth.sigma_ism(w.E_keV)
    w.interp = strategy
    # the workload's generic count map puts counts near 9.5 keV, where the
    # model flux (~e^-80) underflows FP32 (logL -inf on the GPU, finite only
    # in FP64)
    w.counts = counts_from_model(orc, w)
    ll, g, st = gpu_grad(w)
    assert st[0] == 0
    _check(g[0, :13], orc.grad_tangent(w))


def test_grad_background_and_shared_counts(orc, synth, atm, small_lens):
    """lambda = tau C + bkg and one block of counts shared by two instances."""
    import torch
    import paper_2510_07764_gb300 as ppm
    from gpu_helpers import context
    w = visible_two_cap(synth, atm, small_lens, n_theta=8, n_phi=12, n_phase=16, n_E=40,
                        n_chan=20)
    inst = w.inst.select([0, 0])
    inst.incl_rad[1] = 0.7
    w2 = synth.Workload("b", inst, small_lens, w.E_keV, atm=atm, R=w.R, sigma_ism=w.sigma_ism,
                        counts=w.counts, tau=w.tau)
    bkg = np.full(w.counts.shape, 3.0, np.float32)
    ctx = context(w2)
    dp = ppm.DeviceParams(w2.inst)
    cnt = torch.from_numpy(w.counts).cuda()
    ll, g = ctx.loglike_grad(dp, cnt, w.tau, bkg=torch.from_numpy(bkg).cuda(), counts_shared=True)
    g = g.cpu().numpy()
    for b in range(2):
        # reference: central differences of the oracle with the background
        from grad_helpers import NAMES, SCALE, get_param, set_param
        single = synth.Workload("s", inst.select([b]), small_lens, w.E_keV, atm=atm, R=w.R,
                                sigma_ism=w.sigma_ism, counts=w.counts, tau=w.tau)

        def f(x, j):
            i2 = single.inst.copy()
            set_param(i2, j, x)
            s2 = synth.Workload("s", i2, small_lens, w.E_keV, atm=atm, R=w.R,
                                sigma_ism=w.sigma_ism, counts=w.counts, tau=w.tau)
            C = orc.counts_model(orc.profile(s2), w.R, w.sigma_ism, float(i2.nh_1e20[0]))
            return orc.loglike(C, w.counts, w.tau, bkg)
        ref = np.zeros(13)
        for j in range(13):
            th = get_param(single.inst, j)
            h = 1e-5 * max(abs(th), SCALE[j] / 10.0)
            ref[j] = (f(th + h, j) - f(th - h, j)) / (2 * h)
        _check(g[b], ref)


def test_grad_of_an_invisible_instance_is_nan(synth, atm, small_lens):
    """A star whose spots never face the observer has lambda = 0 with counts
    > 0: logL = -inf and the gradient is not defined (NaN)."""
    w = visible_two_cap(synth, atm, small_lens, n_theta=8, n_phi=12, n_phase=16, n_E=40,
                        n_chan=20)
    w.inst.incl_rad[0] = 0.0
    w.inst.colat[0] = [np.pi - 0.05, np.pi - 0.08]
    w.inst.zeta[0] = [0.03, 0.02]
    ll, g, st = gpu_grad(w)
    assert ll[0] == -np.inf and np.all(np.isnan(g[0]))


def test_gradient_is_bitwise_reproducible(synth, atm):
    """The full-resolution two-spot workload: repeated gradient calls agree
    bit for bit (per-warp adjoint copies summed in a fixed order)."""
    import torch
    import paper_2510_07764_gb300 as ppm
    w = synth.atm_two_spot(atm=atm)
    ctx = context(w)
    dp = ppm.DeviceParams(w.inst)
    cnt = torch.from_numpy(w.counts).cuda()
    ll1, g1 = ctx.loglike_grad(dp, cnt, w.tau)
    for _ in range(3):
        ll2, g2 = ctx.loglike_grad(dp, cnt, w.tau)
        assert torch.equal(g1, g2) and torch.equal(ll1, ll2)


def test_gradient_ascent_recovers_parameters(synth, atm, small_lens):
    """The autograd wrapper inside an optimiser: counts drawn from a known
    parameter vector, ascent from a perturbed start raises logL and moves the
    inclination and the spot colatitude back toward the truth."""
    import torch
    import paper_2510_07764_gb300 as ppm
    w = visible_two_cap(synth, atm, small_lens, n_theta=10, n_phi=14, n_phase=32, n_E=48,
                        n_chan=30)
    ctx = context(w)
    dp = ppm.DeviceParams(w.inst)
    truth = dp.theta().clone()
    tau = w.tau * 1e3   # a long exposure: ~1e4 counts per bin
    mc = torch.empty((dp.rows, w.nc), dtype=torch.float32, device="cuda")
    ctx.loglike(dp, torch.zeros((dp.rows, w.nc), dtype=torch.int32, device="cuda"), tau,
                model_counts=mc)
    g = torch.Generator(device="cuda").manual_seed(5)
    counts = torch.poisson(mc.double(), generator=g).to(torch.int32)
    start = truth.clone()
    start[0, 2] += 0.06     # inclination
    start[0, 5] -= 0.05     # colatitude of spot 1
    theta = start.clone().requires_grad_(True)
    free = torch.zeros_like(theta)
    free[0, 2] = free[0, 5] = 1.0
    opt = torch.optim.Adam([theta], lr=4e-3)
    ll0 = None
    for _ in range(60):
        opt.zero_grad()
        ll = ppm.LogLikelihood(theta, ctx, dp, counts, tau)
        if ll0 is None:
            ll0 = float(ll.detach())
        (-ll.sum()).backward()
        theta.grad *= free
        opt.step()
    ll1 = float(ppm.LogLikelihood(theta.detach(), ctx, dp, counts, tau))
    assert ll1 > ll0 + 10.0
    err0 = torch.abs(start - truth)[0, [2, 5]]
    err1 = torch.abs(theta.detach() - truth)[0, [2, 5]]
    assert torch.all(err1 < 0.3 * err0), (err0, err1)


def test_grad_full_size_against_the_oracle():
    """The differentiated workload as the benchmark times it (1024 two-cap
    instances at 128 x 128 elements, 128 phases, 256 energies, 300 channels,
    default lens grid, one ppm_loglike_grad call over the batch) against the
    FP64 oracle's forward-mode derivatives of the same instances, written by
    tests/golden/make_grad_golden.py: every gradient component at 1e-3
    relative (floor 1e-5 of the largest scale-weighted component) and three
    seeded directional derivatives at 1e-3 relative."""
    import json
    import os
    import torch
    import paper_2510_07764_gb300 as ppm
    from paper_2510_07764_gb300 import synth
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                       "grad_batch_full.json")))
    w = synth.grad_batch()
    ctx = context(w)
    dp = ppm.DeviceParams(w.inst)
    cnt = torch.from_numpy(w.counts).cuda()
    ll, g = ctx.loglike_grad(dp, cnt, w.tau)
    ctx.sync()
    ll, g = ll.cpu().numpy(), g.cpu().numpy()
    st = ctx.last_status.cpu().numpy()
    assert len(gold["instances"]) >= 3
    for rec in gold["instances"]:
        b = rec["b"]
        ref = np.asarray(rec["grad"])
        assert st[b] == 0 and np.isfinite(rec["logL"])
        d = w.counts[b * 128:(b + 1) * 128]             # 128 phases per instance
        assert abs(ll[b] - rec["logL"]) <= 1e-3 * float(np.sum(np.abs(d))) + 1e-6 * abs(rec["logL"])
        assert np.all(np.abs(g[b] - ref) <= grad_tol(ref)), \
            (b, np.abs(g[b] - ref) / np.abs(ref))
        for v, dv in zip(rec["directions"], rec["directional"]):
            v = np.asarray(v)
            gv = float(g[b] @ v)
            assert abs(gv - dv) <= 1e-3 * abs(dv) + 1e-5 * float(np.sum(np.abs(ref * v))), \
                (b, gv, dv)
