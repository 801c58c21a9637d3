"""The walks of the atmosphere shift-and-add against the FP64 oracle and
against the energy walk (ppm_tiles.walk = 1) on the same inputs: the
node-major walk (walk = 2; observed energies uniform in ln E with a step of
0.34-0.498 table nodes, every table interval holds two or three of them) and
the moment walk (the default, walk = 0) evaluate the same interpolants and
sum them in a different order."""
import math

import numpy as np
import pytest

from gpu_helpers import context, max_rel

pytestmark = pytest.mark.gpu

TOL_ATM = 1e-3
TOL_WALKS = 1e-4   # FP32 sums in another order, positions accumulated by the walk


def _workload(synth, atm, small_lens, n_E, lo, hi, interp="d", **kw):
    w = synth.atm_two_spot(n_theta=kw.get("n_theta", 14), n_phi=kw.get("n_phi", 40),
                           n_phase=kw.get("n_phase", 24), n_E=n_E, n_chan=8, atm=atm,
                           lens=small_lens)
    w.E_keV = synth.logspace(lo, hi, n_E)
    w.interp = interp
    return w


def _step(w, atm):
    """Observed-energy step in table nodes."""
    dln = (atm.lnE[-1] - atm.lnE[0]) / (len(atm.lnE) - 1)
    return math.log(w.E_keV[-1] / w.E_keV[0]) / (len(w.E_keV) - 1) / dln


def _walks(w, walks=(0, 1)):
    import paper_2510_07764_gb300 as ppm
    ctx = context(w)
    dp = ppm.DeviceParams(w.inst)
    out = []
    try:
        for walk in walks:
            ctx.set_tiles(walk=walk)
            Ft = ctx.profile(dp)
            ctx.sync()
            out.append(Ft.cpu().numpy().astype(np.float64))
    finally:
        ctx.set_tiles()
    return out


def _both_walks(w):
    """(node-major walk, energy walk)"""
    return _walks(w, (2, 1))


@pytest.mark.parametrize("interp", ["d", "a", "b", "c"])
def test_node_walk_matches_oracle_and_energy_walk(orc, synth, atm, small_lens, interp):
    w = _workload(synth, atm, small_lens, 96, 0.6, 2.6, interp)
    assert 0.34 <= _step(w, atm) <= 0.498
    node, energy = _both_walks(w)
    assert not np.array_equal(node, energy)       # the node-major walk ran
    assert max_rel(node, energy) < TOL_WALKS
    assert max_rel(node, orc.profile(w)) < TOL_ATM


@pytest.mark.parametrize("n_E,lo,hi", [
    (159, 0.5, 6.0),     # step 0.49, near the upper bound
    (230, 0.5, 6.6),     # step 0.349, near the lower bound: three energies per interval
    (300, 0.1, 5.215),   # the crescent workload's grid, step 0.41
])
def test_node_walk_steps(orc, synth, atm, small_lens, n_E, lo, hi):
    w = _workload(synth, atm, small_lens, n_E, lo, hi, n_phase=16)
    assert 0.34 <= _step(w, atm) <= 0.498
    node, energy = _both_walks(w)
    assert not np.array_equal(node, energy)
    assert max_rel(node, energy) < TOL_WALKS
    assert max_rel(node, orc.profile(w)) < TOL_ATM


@pytest.mark.parametrize("lo,hi", [(0.052, 0.32), (3.5, 7.8)])
def test_node_walk_with_table_edges(orc, synth, atm, small_lens, lo, hi):
    """Redshifted energies leave the table interior at its low or high end:
    elements of the same warp split between the walk and the general path."""
    n_E = int(round(math.log(hi / lo) / (0.45 * 0.0321))) + 1
    w = _workload(synth, atm, small_lens, n_E, lo, hi, n_phase=20)
    assert 0.34 <= _step(w, atm) <= 0.498
    node, energy = _both_walks(w)
    assert max_rel(node, energy) < TOL_WALKS
    assert max_rel(node, orc.profile(w)) < TOL_ATM


def test_walk_setting_is_inert_off_its_grids(synth, atm, small_lens):
    """A step above 1/2 node (and a grid not uniform in ln E) keeps the energy
    walk whatever the setting: both runs are bit-identical."""
    w = _workload(synth, atm, small_lens, 64, 0.6, 2.6)
    assert 0.5 < _step(w, atm) < 0.999
    node, energy = _both_walks(w)
    assert np.array_equal(node, energy)
    w = _workload(synth, atm, small_lens, 96, 0.6, 2.6)
    w.E_keV = w.E_keV * (1.0 + 0.01 * np.sin(np.arange(96)))
    node, energy = _both_walks(w)
    assert np.array_equal(node, energy)


def test_node_walk_persistent_schedule_is_bitwise_identical(synth, atm, small_lens):
    import paper_2510_07764_gb300 as ppm
    w = _workload(synth, atm, small_lens, 120, 0.4, 2.6, n_theta=20, n_phi=72, n_phase=40)
    inst = w.inst.select(np.zeros(5, dtype=int))
    inst.incl_rad[:] = np.linspace(0.3, 1.4, 5)
    w.inst = inst
    ctx = context(w)
    dp = ppm.DeviceParams(w.inst)
    res = []
    try:
        for pers in (False, True):
            ctx.set_tiles(16, 16, pers, walk=2)
            Ft = ctx.profile(dp)
            ctx.sync()
            res.append(Ft.cpu().numpy())
    finally:
        ctx.set_tiles()
    assert np.array_equal(res[0], res[1])


# ---- the backward shift-and-add on the node-major walk --------------------
def _grad_both_walks(w):
    import torch
    import paper_2510_07764_gb300 as ppm
    ctx = context(w)
    dp = ppm.DeviceParams(w.inst)
    cnt = torch.from_numpy(np.ascontiguousarray(w.counts)).cuda()
    out = []
    try:
        for walk in (2, 1):
            ctx.set_tiles(walk=walk)
            ll, g = ctx.loglike_grad(dp, cnt, w.tau)
            ctx.sync()
            out.append((ll.cpu().numpy(), g.cpu().numpy()))
    finally:
        ctx.set_tiles()
    return out


@pytest.mark.parametrize("interp", ["d", "b"])
def test_node_walk_gradient_matches_oracle_tangent(orc, synth, atm, small_lens, interp):
    """Two visible caps on a 96-energy grid of 0.48 table node per step: the
    gradient through the node-major backward against the oracle's forward
    mode (1e-3 relative per component) and against the energy walk.  The
    grid (0.3-1.3 keV) keeps strategy B's clipped flux positive in every
    bin (above ~1.5 keV its one-sided cubics clip whole bins to zero and
    logL is -inf, where the gradient is NaN by definition)."""
    import test_gpu_grad as tg
    from grad_helpers import grad_tol
    w = tg.visible_two_cap(synth, atm, small_lens, n_theta=12, n_phi=20, n_phase=24, n_E=96,
                           n_chan=30)
    w.E_keV = synth.logspace(0.3, 1.3, 96)
    w.R = synth.response(w.E_keV, 30)
    w.sigma_ism = synth.sigma_ism(w.E_keV)
    w.interp = interp
    assert 0.34 <= _step(w, atm) <= 0.498
    (ll0, g0), (ll1, g1) = _grad_both_walks(w)
    assert not np.array_equal(g0, g1)             # the node-major backward ran
    tg._check(g0[0, :13], orc.grad_tangent(w))
    # the walks agree to FP32 rounding, except where strategy B's clip
    # decision (I > 0) flips between them
    ref = g1[0, :13]
    assert np.all(np.abs(g0[0, :13] - ref) <= (1.0 if interp == "b" else 0.1) * grad_tol(ref))
    assert abs(ll0[0] - ll1[0]) <= 1e-6 * abs(ll1[0])


def test_node_walk_gradient_with_table_edges(orc, synth, atm, small_lens):
    """Energies whose redshifted images leave the table interior: warps with
    such elements take the general path, the others the walk."""
    import test_gpu_grad as tg
    w = tg.visible_two_cap(synth, atm, small_lens, n_theta=10, n_phi=16, n_phase=16, n_E=56,
                           n_chan=20)
    w.E_keV = synth.logspace(3.5, 7.8, 56)
    w.R = synth.response(w.E_keV, 20)
    w.sigma_ism = synth.sigma_ism(w.E_keV)
    assert 0.34 <= _step(w, atm) <= 0.498
    (ll0, g0), (ll1, g1) = _grad_both_walks(w)
    ref = orc.grad_tangent(w)
    tg._check(g0[0, :13], ref)
    tg._check(g1[0, :13], ref)


@pytest.mark.parametrize("walk", [2, 0])
def test_node_walk_cuda_graph_replay(synth, atm, small_lens, walk):
    """ppm_loglike_grad on the node-major walks (walk 2; the default walk 0
    takes the moment walk forward) captured once in a CUDA graph and replayed
    after in-place parameter updates equals the direct call bit for bit."""
    import torch
    import paper_2510_07764_gb300 as ppm
    w = _workload(synth, atm, small_lens, 96, 0.6, 2.6, n_theta=10, n_phi=24, n_phase=20)
    w.R = synth.response(w.E_keV, 8)
    w.sigma_ism = synth.sigma_ism(w.E_keV)
    ctx = context(w)
    ctx.set_tiles(walk=walk)
    try:
        dp = ppm.DeviceParams(w.inst)
        cnt = torch.from_numpy(w.counts).cuda()
        out = torch.empty(dp.B, dtype=torch.float64, device="cuda")
        grad = torch.empty((dp.B, ppm.N_GRAD), dtype=torch.float64, device="cuda")
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            for _ in range(2):
                ctx.loglike_grad(dp, cnt, w.tau, out=out, grad=grad, stream=s)
        s.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            ctx.loglike_grad(dp, cnt, w.tau, out=out, grad=grad, stream=s)
        th0 = dp.theta()
        for k in range(2):
            th = th0.clone()
            th[:, 2] += 0.04 * (k + 1)
            dp.set_theta(th)
            g.replay()
            torch.cuda.synchronize()
            got_ll, got_g = out.clone(), grad.clone()
            ref_ll, ref_g = ctx.loglike_grad(dp, cnt, w.tau)
            torch.cuda.synchronize()
            assert torch.equal(got_ll, ref_ll)
            assert torch.equal(torch.nan_to_num(got_g), torch.nan_to_num(ref_g))
    finally:
        ctx.set_tiles()


def test_node_walk_temperature_map(orc, synth, atm, small_lens):
    """A HEALPix temperature map (N_side 12) on a 96-energy grid of 0.48 node
    per step: the map kernel's node-major walk (two slabs per logT cell,
    each element's own cell weight) against the oracle and the energy walk."""
    w = synth.healpix_map(n_side=12, n_phase=24, n_E=96, n_chan=8, atm=atm, lens=small_lens)
    w.E_keV = synth.logspace(0.6, 2.6, 96)
    w.R = synth.response(w.E_keV, 8)
    w.sigma_ism = synth.sigma_ism(w.E_keV)
    assert 0.34 <= _step(w, atm) <= 0.498
    node, energy = _both_walks(w)
    assert not np.array_equal(node, energy)
    assert max_rel(node, energy) < TOL_WALKS
    assert max_rel(node, orc.profile(w)) < TOL_ATM


# ---- the moment walk (the default, ppm_tiles.walk = 0) --------------------
# Per group of 64 elements the walk sums the moments sum_p eps_p^j u_p of the
# contracted node values and evaluates one combined cubic per energy, plus
# the exact difference terms of elements whose own position crossed a node.
# It applies to every grid whose steps stay below one table node (not only
# the uniform ones of the node-major walk) and to every strategy but B.

@pytest.mark.parametrize("interp", ["d", "a", "c"])
def test_moment_walk_matches_oracle_and_other_walks(orc, synth, atm, small_lens, interp):
    w = _workload(synth, atm, small_lens, 96, 0.6, 2.6, interp)
    mom, node, energy = _walks(w, (0, 2, 1))
    assert not np.array_equal(mom, node)          # the moment walk ran
    assert max_rel(mom, energy) < TOL_WALKS
    assert max_rel(mom, orc.profile(w)) < TOL_ATM


def test_moment_walk_leaves_strategy_b_on_the_node_walk(synth, atm, small_lens):
    """The clipped interpolant is not linear in the table values: the
    setting keeps strategy B on the node-major walk, bit for bit."""
    w = _workload(synth, atm, small_lens, 96, 0.6, 2.6, "b")
    mom, node = _walks(w, (0, 2))
    assert np.array_equal(mom, node)


@pytest.mark.parametrize("n_E,lo,hi,wiggle", [
    (159, 0.5, 6.0, 0.0),     # step 0.49
    (230, 0.5, 6.6, 0.0),     # step 0.349
    (300, 0.1, 5.215, 0.0),   # the crescent workload's grid, step 0.41
    (64, 0.6, 2.6, 0.0),      # step 0.73: beyond the node-major walk
    (96, 0.6, 2.6, 0.01),     # not uniform in ln E
    (17, 0.6, 0.9, 0.0),      # one chunk of nodes
])
def test_moment_walk_grids(orc, synth, atm, small_lens, n_E, lo, hi, wiggle):
    w = _workload(synth, atm, small_lens, n_E, lo, hi, n_phase=16)
    w.E_keV = w.E_keV * (1.0 + wiggle * np.sin(np.arange(n_E)))
    mom, energy = _walks(w, (0, 1))
    assert not np.array_equal(mom, energy)
    assert max_rel(mom, energy) < TOL_WALKS
    assert max_rel(mom, orc.profile(w)) < TOL_ATM


@pytest.mark.parametrize("lo,hi", [(0.052, 0.32), (3.5, 7.8)])
def test_moment_walk_with_table_edges(orc, synth, atm, small_lens, lo, hi):
    """Elements of a group split between the walk and the general path."""
    n_E = int(round(math.log(hi / lo) / (0.45 * 0.0321))) + 1
    w = _workload(synth, atm, small_lens, n_E, lo, hi, n_phase=20)
    mom, energy = _walks(w, (0, 1))
    assert max_rel(mom, energy) < TOL_WALKS
    assert max_rel(mom, orc.profile(w)) < TOL_ATM


@pytest.mark.parametrize("wiggle", [0.0, 0.01])
def test_moment_walk_wide_groups(orc, synth, atm, small_lens, wiggle):
    """Large spots at 600 Hz: most groups spread over more than one table
    node in ln z and leave the moment walk for the node-major walk (uniform
    grid) or the energy walk (a grid not uniform in ln E), the others take
    it, in the same call."""
    w = _workload(synth, atm, small_lens, 96, 0.6, 2.6, n_phase=24)
    w.E_keV = w.E_keV * (1.0 + wiggle * np.sin(np.arange(96)))
    w.inst.spin_hz[:] = 600.0
    w.inst.zeta[0] = [0.6, 0.7]
    mom, energy = _walks(w, (0, 1))
    assert max_rel(mom, energy) < TOL_WALKS
    assert max_rel(mom, orc.profile(w)) < TOL_ATM


def test_moment_walk_fine_grid(orc, synth, atm, small_lens):
    """900 energies at 0.05 table node per step: groups list more candidate
    energies (energies within their spread of a node) than the per-group
    list holds, and the rest of a pass takes them one at a time; groups
    too wide for the moment walk take the energy walk (the step is below
    the node-major walk's)."""
    w = _workload(synth, atm, small_lens, 900, 0.6, 2.6, n_phase=12)
    assert _step(w, atm) < 0.06
    mom, energy = _walks(w, (0, 1))
    assert not np.array_equal(mom, energy)
    assert max_rel(mom, energy) < TOL_WALKS
    assert max_rel(mom, orc.profile(w)) < TOL_ATM


def test_moment_walk_crescent(orc, synth, atm):
    """The crescent geometry (narrow groups: difference terms at a few per
    cent of the energies) on its 300-energy grid."""
    w = synth.crescent_extreme(n_theta=24, n_phi=96, n_phase=32, n_E=300, n_chan=8, atm=atm)
    mom, energy = _walks(w, (0, 1))
    assert not np.array_equal(mom, energy)
    assert max_rel(mom, energy) < TOL_WALKS
    assert max_rel(mom, orc.profile(w)) < TOL_ATM


def test_moment_walk_persistent_schedule_is_bitwise_identical(synth, atm, small_lens):
    import paper_2510_07764_gb300 as ppm
    w = _workload(synth, atm, small_lens, 120, 0.4, 2.6, n_theta=20, n_phi=72, n_phase=40)
    inst = w.inst.select(np.zeros(5, dtype=int))
    inst.incl_rad[:] = np.linspace(0.3, 1.4, 5)
    w.inst = inst
    ctx = context(w)
    dp = ppm.DeviceParams(w.inst)
    res = []
    try:
        for pers in (False, True):
            ctx.set_tiles(16, 16, pers)
            Ft = ctx.profile(dp)
            ctx.sync()
            res.append(Ft.cpu().numpy())
    finally:
        ctx.set_tiles()
    assert np.array_equal(res[0], res[1])


def test_moment_walk_likelihood_and_gradient(synth, atm, small_lens):
    """ppm_loglike_grad with the moment walk in its forward pass equals the
    node-major run to FP32 rounding."""
    import torch
    import paper_2510_07764_gb300 as ppm
    from grad_helpers import grad_tol
    w = _workload(synth, atm, small_lens, 96, 0.6, 2.6, n_theta=10, n_phi=24, n_phase=20)
    w.R = synth.response(w.E_keV, 8)
    w.sigma_ism = synth.sigma_ism(w.E_keV)
    ctx = context(w)
    dp = ppm.DeviceParams(w.inst)
    cnt = torch.from_numpy(w.counts).cuda()
    out = []
    try:
        for walk in (0, 2):
            ctx.set_tiles(walk=walk)
            ll, g = ctx.loglike_grad(dp, cnt, w.tau)
            ctx.sync()
            out.append((ll.cpu().numpy(), g.cpu().numpy()))
    finally:
        ctx.set_tiles()
    (ll2, g2), (ll0, g0) = out
    assert abs(ll2[0] - ll0[0]) <= 1e-6 * abs(ll0[0])
    ref = g0[0, :13]
    assert np.all(np.abs(g2[0, :13] - ref) <= 0.1 * grad_tol(ref))
