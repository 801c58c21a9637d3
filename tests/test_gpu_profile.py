"""Parity of the CUDA forward profile (ppm_profile) with the FP64 oracle.

Tolerances (per phase-energy bin where the oracle flux is >= 1e-6 of its
maximum, the paper's "non-negligible flux" criterion):
  analytic blackbody workload ............. 1e-4 relative
  atmosphere-table workloads .............. 1e-3 relative
Full-size workloads are checked on sampled bins the oracle computes one by one.
"""
import math

import numpy as np
import pytest

from gpu_helpers import gpu_profile, max_rel, rows_of

pytestmark = pytest.mark.gpu

TOL_BB = 1e-4
TOL_ATM = 1e-3


def test_bb_small_full_size(orc, synth):
    w = synth.bb_small()
    got, st = gpu_profile(w)
    assert st[0] == 0
    ref = orc.profile(w)
    assert max_rel(got, ref) < TOL_BB


def test_bb_ragged_sizes(orc, synth, small_lens):
    # 37 rings x 45 elements (ragged vs 32 lanes), 70 phases (ragged vs 32), 41 energies
    w = synth.bb_small(n_theta=37, n_phi=45, n_phase=70, n_E=41, lens=small_lens)
    got, _ = gpu_profile(w)
    assert max_rel(got, orc.profile(w)) < TOL_BB


def test_atm_two_spot_reduced(orc, synth, atm, small_lens):
    w = synth.atm_two_spot(n_theta=24, n_phi=40, n_phase=40, n_E=72, n_chan=24, atm=atm,
                           lens=small_lens)
    got, st = gpu_profile(w)
    assert st[0] == 0
    assert max_rel(got, orc.profile(w)) < TOL_ATM


def test_atm_two_spot_full_size_sampled(orc, synth, atm):
    w = synth.atm_two_spot(atm=atm)
    got, _ = gpu_profile(w)
    rng = np.random.default_rng(3)
    js = np.sort(rng.choice(128, 6, replace=False))
    ks = np.sort(rng.choice(256, 10, replace=False))
    ref = orc.profile(w, jsel=js, ksel=ks)
    assert max_rel(got[np.ix_(js, ks)], ref) < TOL_ATM
    # every output is finite and the total is positive
    assert np.isfinite(got).all() and got.sum() > 0


def test_crescent_reduced(orc, synth, atm):
    w = synth.crescent_extreme(n_theta=48, n_phi=64, n_phase=64, n_E=100, n_chan=24, atm=atm)
    got, st = gpu_profile(w)
    assert st[0] == 0
    assert max_rel(got, orc.profile(w)) < TOL_ATM


def test_crescent_full_size_sampled(orc, synth, atm):
    w = synth.crescent_extreme(atm=atm)
    got, _ = gpu_profile(w)
    js = np.array([0, 63, 127, 128, 200, 255])
    ks = np.array([0, 37, 150, 299])
    ref = orc.profile(w, jsel=js, ksel=ks)
    assert max_rel(got[np.ix_(js, ks)], ref) < TOL_ATM


def test_batch_mixed_instances(orc, synth, atm):
    inst = synth.random_instances(7, seed=11, res_theta=(20, 33), res_phase=(32, 45), mask=True)
    w = synth.Workload("batch", inst, synth.LensSpec(), synth.logspace(0.1, 5.215, 64), atm=atm)
    got, st = gpu_profile(w)
    for b in range(inst.B):
        wb = synth.Workload("one", inst.select(b), w.lens, w.E_keV, atm=atm)
        try:
            ref = orc.profile(wb)
        except orc.OracleRangeError:
            assert st[b] == 2
            assert not got[rows_of(w, b)].any()
            continue
        assert st[b] == 0
        assert max_rel(got[rows_of(w, b)], ref) < TOL_ATM, b


def test_out_of_range_instance_is_isolated(orc, synth, atm, small_lens):
    w = synth.atm_two_spot(n_theta=12, n_phi=16, n_phase=32, n_E=40, n_chan=8, atm=atm,
                           lens=small_lens)
    inst = w.inst
    two = inst.select([0, 0, 0])
    two.radius_km[1] = 9.0          # u = 0.46: outside the lens grid [0.30, 0.40]
    two.logT[2, 0] = 7.5            # outside the atmosphere table
    w2 = synth.Workload("x", two, small_lens, w.E_keV, atm=atm)
    got, st = gpu_profile(w2)
    assert list(st) == [0, 2, 2]
    assert not got[32:].any()
    assert max_rel(got[:32], orc.profile(w)) < TOL_ATM


def test_invisible_and_empty_spots(orc, synth, atm, small_lens):
    w = synth.atm_two_spot(n_theta=10, n_phi=16, n_phase=32, n_E=40, n_chan=8, atm=atm,
                           lens=small_lens)
    # spot 0 hidden behind the star (observer at the north pole, spot at the
    # south pole), spot 1 fully masked (mask larger than the emitter)
    inst = w.inst.replace(incl_rad=0.0)
    inst.colat[0, 0] = math.pi - 0.05
    inst.zeta[0, 0] = 0.04
    inst.mask_zeta[0, 1] = 0.5
    w.inst = inst
    got, st = gpu_profile(w)
    assert st[0] == 0
    assert not got.any()
    assert not orc.profile(w).any()


def test_single_phase_single_energy(orc, synth, atm, small_lens):
    w = synth.atm_two_spot(n_theta=9, n_phi=7, n_phase=1, n_E=1, n_chan=3, atm=atm,
                           lens=small_lens)
    got, _ = gpu_profile(w)
    assert max_rel(got, orc.profile(w)) < TOL_ATM


def test_zero_inclination_is_phase_constant(synth, atm):
    # holds at any size: no rotational modulation is visible from the pole
    w = synth.atm_two_spot(atm=atm)
    w.inst = w.inst.replace(incl_rad=0.0)
    got, _ = gpu_profile(w)
    assert got.max() > 0
    assert np.max(np.abs(got - got[0:1])) / got.max() < 2e-5


def test_bad_resolution_is_rejected(synth, small_lens):
    import paper_2510_07764_gb300 as ppm
    from gpu_helpers import context
    w = synth.bb_small(lens=small_lens)
    ctx = context(w)
    for field, val in [("n_theta", 0), ("n_phi", 5000), ("n_phase", -1)]:
        inst = w.inst.replace(**{field: val})
        dp = ppm.DeviceParams(inst)
        with pytest.raises(ppm.PPMError) as e:
            ctx.profile(dp)
        assert e.value.status == ppm.PPM_EINVAL


def test_invalid_arguments_are_rejected_and_the_context_recovers(orc, synth, atm, small_lens):
    """Each documented argument rule of ppm_params / ppm_res returns
    PPM_EINVAL with its message before anything is enqueued, and the context
    stays usable: the next valid call matches the oracle."""
    import paper_2510_07764_gb300 as ppm
    from gpu_helpers import context
    w = synth.atm_two_spot(n_theta=8, n_phi=12, n_phase=16, n_E=24, n_chan=8, atm=atm,
                           lens=small_lens)
    ctx = context(w)
    one = dict(n_spots=1)  # the second spot's values stay in the arrays, unread
    n_side = 4
    tmap = np.full((1, 12 * n_side * n_side), 6.0)
    cases = [
        (dict(n_spots=3), "n_spots"),
        (dict(oblate=2), "oblate"),
        (dict(emission=2), "emission"),
        (dict(n_fp=4), "n_fp"),
        (dict(grid=2), "grid must be"),
        (dict(phase_sub=3), "phase_sub"),
        (dict(logT_map=tmap, **one), "needs grid"),
        (dict(logT_map=tmap, grid=1, n_theta=n_side), "needs n_spots = 1"),
        (dict(grid=1, n_theta=2000), "N_side"),
    ]
    for kw, msg in cases:
        inst = w.inst.replace(**kw)
        with pytest.raises(ppm.PPMError, match=msg) as e:
            ctx.profile(ppm.DeviceParams(inst))
        assert e.value.status == ppm.PPM_EINVAL, kw
    # a temperature map with a non-default interpolation strategy
    ctx.set_interpolation("b")
    try:
        inst = w.inst.replace(logT_map=tmap, grid=1, n_theta=n_side, **one)
        with pytest.raises(ppm.PPMError, match="default interpolation") as e:
            ctx.profile(ppm.DeviceParams(inst))
        assert e.value.status == ppm.PPM_EINVAL
    finally:
        ctx.set_interpolation("d")
    Ft, st = gpu_profile(w)
    assert st[0] == 0
    assert max_rel(Ft, orc.profile(w)) < TOL_ATM


def test_sync_times_out_on_a_busy_stream_and_recovers(synth, atm):
    """ppm_sync is a bounded wait: with about 36 ms of shift-and-add work still
    queued on the stream it returns PPM_ETIMEOUT after 0.1 ms instead of
    blocking; a later sync with a long limit returns PPM_OK, and the results
    are those of a single call."""
    import torch
    import paper_2510_07764_gb300 as ppm
    from gpu_helpers import context
    w = synth.atm_two_spot(atm=atm)
    ctx = context(w)
    dp = ppm.DeviceParams(w.inst)
    s = torch.cuda.Stream()
    first = ctx.profile(dp, stream=s)   # plan and workspace settle here
    ctx.sync(stream=s, timeout=60.0)
    ref = first.clone()
    # outputs allocated up front: nothing in the loop may synchronise the device
    outs = [torch.empty_like(ref) for _ in range(40)]
    sts = [torch.empty(1, dtype=torch.int32, device=ref.device) for _ in range(40)]
    torch.cuda.synchronize()
    for o, st in zip(outs, sts):
        ctx.profile(dp, out=o, status=st, stream=s)
    with pytest.raises(ppm.PPMError) as e:
        ctx.sync(stream=s, timeout=1e-4)
    assert e.value.status == ppm.PPM_ETIMEOUT
    ctx.sync(stream=s, timeout=60.0)
    assert all(torch.equal(o, ref) for o in outs)
    assert all(int(st[0]) == 0 for st in sts)


def test_energies_past_table_edges(orc, synth, atm, small_lens):
    """Redshifted energies leave the table (E' up to ~12 keV > 10 keV, down to
    0.07 keV near the 0.05 keV edge): linear edge intervals and clamping."""
    w = synth.atm_two_spot(n_theta=14, n_phi=20, n_phase=32, n_E=200, n_chan=8, atm=atm,
                           lens=small_lens)
    w.E_keV = synth.logspace(0.06, 9.5, 200)   # fine grid: sliding and edge lanes mix
    got, _ = gpu_profile(w)
    assert max_rel(got, orc.profile(w)) < TOL_ATM


def test_coarse_energy_grid_general_path(orc, synth, atm, small_lens):
    """Eight energies 0.1-5 keV step ~17 table nodes: the sliding window cannot
    be used and every energy takes the general interpolation path."""
    w = synth.atm_two_spot(n_theta=14, n_phi=36, n_phase=33, n_E=8, n_chan=8, atm=atm,
                           lens=small_lens)
    got, _ = gpu_profile(w)
    assert max_rel(got, orc.profile(w)) < TOL_ATM


@pytest.mark.parametrize("S", [2, 4, 16])
def test_phase_sub_samples_match_oracle(orc, synth, atm, small_lens, S):
    """Output phase bins averaged over S point samples (ppm_res.phase_sub)."""
    w = synth.atm_two_spot(n_theta=12, n_phi=16, n_phase=24, n_E=40, n_chan=8, atm=atm,
                           lens=small_lens)
    w.inst.phase_sub = S
    Ft, st = gpu_profile(w)
    assert st[0] == 0
    assert max_rel(Ft, orc.profile(w)) < 1e-3


@pytest.mark.parametrize("n_fp", [8, 1024])
def test_template_resolution_limits(orc, synth, atm, small_lens, n_fp):
    """The smallest and the largest template resolution the library accepts
    (8 and 1024 fine phases per ring; the paper uses 192) against the oracle,
    and the first values outside the range are rejected."""
    import paper_2510_07764_gb300 as ppm
    from gpu_helpers import context
    w = synth.atm_two_spot(n_theta=10, n_phi=20, n_phase=24, n_E=40, n_chan=8, atm=atm,
                           lens=small_lens)
    w.inst.n_fp = n_fp
    got, st = gpu_profile(w)
    assert st[0] == 0
    assert max_rel(got, orc.profile(w)) < TOL_ATM
    ctx = context(w)
    bad = w.inst.replace()
    bad.n_fp = 7 if n_fp == 8 else 1025
    with pytest.raises(ppm.PPMError) as e:
        ctx.profile(ppm.DeviceParams(bad))
    assert e.value.status == ppm.PPM_EINVAL
