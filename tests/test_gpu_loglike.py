"""Parity of ppm_loglike (ISM, response contraction, Poisson logL) with the oracle.

Model counts per (phase, channel) bin: 1e-3 relative where non-negligible.
logL: a relative error eps per bin moves logL by at most eps * sum|d - lambda|
(first order in lambda), so the test allows 1e-3 * sum|d - lambda| plus rounding.
"""
import numpy as np
import pytest

from gpu_helpers import gpu_loglike, gpu_profile, max_rel, rows_of

pytestmark = pytest.mark.gpu


def _oracle_ll(orc, w, b=0, counts=None, bkg=None):
    Ft = orc.profile(w, b=b)
    C = orc.counts_model(Ft, w.R, w.sigma_ism, float(w.inst.nh_1e20[b]))
    d = w.counts[rows_of(w, b)] if counts is None else counts
    return orc.loglike(C, d, w.tau, bkg), C


def _ll_tol(w, C, d):
    return 1e-3 * np.sum(np.abs(d - w.tau * C)) + 1e-9 * np.sum(d)


def test_loglike_two_spot_reduced(orc, synth, atm, small_lens):
    w = synth.atm_two_spot(n_theta=20, n_phi=36, n_phase=48, n_E=80, n_chan=70, atm=atm,
                           lens=small_lens)
    ll, mc, st = gpu_loglike(w)
    llr, C = _oracle_ll(orc, w)
    assert st[0] == 0
    assert max_rel(mc, w.tau * C) < 1e-3
    assert abs(ll[0] - llr) <= _ll_tol(w, C, w.counts)


def test_loglike_full_size(orc, synth, atm):
    """The benchmark workload: 2 x 128^2 elements, 128 phases, 256 energies,
    300 channels, 1e6 counts.  Oracle on sampled phases (all energies)."""
    w = synth.atm_two_spot(atm=atm)
    ll, mc, st = gpu_loglike(w)
    js = np.array([0, 31, 64, 100, 127])
    Ft = orc.profile(w, jsel=js)
    C = orc.counts_model(Ft, w.R, w.sigma_ism, float(w.inst.nh_1e20[0]))
    assert max_rel(mc[js], w.tau * C) < 1e-3
    assert np.isfinite(ll[0])


def test_loglike_background_and_batch(orc, synth, atm, small_lens):
    w = synth.atm_two_spot(n_theta=12, n_phi=20, n_phase=32, n_E=48, n_chan=30, atm=atm,
                           lens=small_lens)
    inst = w.inst.select([0, 0])
    inst.incl_rad[1] = 1.3
    inst.logT[1, 1] = 5.95
    w2 = synth.Workload("b", inst, small_lens, w.E_keV, atm=atm, R=w.R, sigma_ism=w.sigma_ism,
                        counts=np.concatenate([w.counts, w.counts[::-1]]), tau=w.tau)
    bkg = np.full(w2.counts.shape, 0.7, np.float32)
    ll, mc, st = gpu_loglike(w2, bkg=bkg)
    for b in range(2):
        d = w2.counts[rows_of(w2, b)]
        llr, C = _oracle_ll(orc, w2, b, counts=d, bkg=bkg[rows_of(w2, b)])
        assert abs(ll[b] - llr) <= _ll_tol(w2, C, d)
    # shared counts: one block of counts for every instance
    ll2, _, _ = gpu_loglike(w2, counts=w.counts, counts_shared=True)
    for b in range(2):
        llr, C = _oracle_ll(orc, w2, b, counts=w.counts)
        assert abs(ll2[b] - llr) <= _ll_tol(w2, C, w.counts)


def test_loglike_out_of_range_is_minus_inf(synth, atm, small_lens):
    w = synth.atm_two_spot(n_theta=8, n_phi=8, n_phase=32, n_E=32, n_chan=8, atm=atm,
                           lens=small_lens)
    inst = w.inst.select([0, 0])
    inst.mass_msun[1] = 2.2   # u = 0.54, beyond the lens grid
    w2 = synth.Workload("b", inst, small_lens, w.E_keV, atm=atm, R=w.R, sigma_ism=w.sigma_ism,
                        counts=np.concatenate([w.counts, w.counts]), tau=w.tau)
    ll, _, st = gpu_loglike(w2)
    assert st[0] == 0 and st[1] == 2
    assert np.isfinite(ll[0]) and ll[1] == -np.inf


def test_zero_model_with_counts_is_minus_inf(synth, atm, small_lens):
    w = synth.atm_two_spot(n_theta=8, n_phi=8, n_phase=32, n_E=32, n_chan=8, atm=atm,
                           lens=small_lens)
    w.inst = w.inst.replace(incl_rad=0.0)
    w.inst.colat[0] = [np.pi - 0.05, np.pi - 0.05]   # hidden spots: lambda = 0
    w.inst.zeta[0] = [0.04, 0.04]
    w.inst.mask_zeta[0] = [0.0, 0.0]
    ll, _, _ = gpu_loglike(w)
    assert ll[0] == -np.inf
    ll0, _, _ = gpu_loglike(w, counts=np.zeros_like(w.counts))
    assert ll0[0] == 0.0


def _with_env(key, val, fn):
    import os
    old = os.environ.get(key)
    os.environ[key] = val
    try:
        return fn()
    finally:
        if old is None:
            del os.environ[key]
        else:
            os.environ[key] = old


def test_tensor_core_response_matches_oracle(orc, synth, atm, small_lens):
    """The tcgen05 response contraction (BF16 hi/lo split, FP32 accumulation)
    against the oracle, on a ragged shape (100 rows, 300 channels, 200 energies)."""
    w = synth.atm_two_spot(n_theta=12, n_phi=24, n_phase=100, n_E=200, n_chan=300, atm=atm,
                           lens=small_lens)
    ll, mc, st = _with_env("PPM_RESP_TC", "1", lambda: gpu_loglike(w))
    llr, C = _oracle_ll(orc, w)
    assert st[0] == 0
    assert max_rel(mc, w.tau * C) < 1e-3
    assert abs(ll[0] - llr) <= _ll_tol(w, C, w.counts)


def test_tensor_core_and_fp32_paths_agree_on_a_batch(synth, atm, small_lens):
    """A batch of 24 instances x 32 phases (768 rows: the tensor-core path by
    default) against the FP32 tile path on the same profile."""
    w = synth.atm_two_spot(n_theta=10, n_phi=16, n_phase=32, n_E=64, n_chan=300, atm=atm,
                           lens=small_lens)
    inst = w.inst.select(np.zeros(24, dtype=int))
    inst.incl_rad[:] = np.linspace(0.3, 1.5, 24)
    w2 = synth.Workload("b", inst, small_lens, w.E_keV, atm=atm, R=w.R, sigma_ism=w.sigma_ism,
                        counts=np.concatenate([w.counts] * 24), tau=w.tau)
    ll_tc, mc_tc, _ = _with_env("PPM_RESP_TC", "1", lambda: gpu_loglike(w2))
    ll_32, mc_32, _ = _with_env("PPM_RESP_TC", "0", lambda: gpu_loglike(w2))
    assert max_rel(mc_tc, mc_32) < 1e-4
    for b in range(24):
        d = w2.counts[rows_of(w2, b)]
        assert abs(ll_tc[b] - ll_32[b]) <= 1e-4 * np.sum(np.abs(d - mc_32[rows_of(w2, b)])) + 1e-6


def test_fine_grid_response_through_downsampling(orc, synth, atm, small_lens):
    """ppm_set_response_fine (the library's FP64 DS x Rf) against the oracle's
    down-sampling matrix applied to the same fine response: same model counts
    and logL as installing the oracle's product with ppm_set_response."""
    import torch
    import paper_2510_07764_gb300 as ppm
    from gpu_helpers import context
    w = synth.atm_two_spot(n_theta=10, n_phi=16, n_phase=32, n_E=48, n_chan=40, atm=atm,
                           lens=small_lens)
    rng = np.random.default_rng(9)
    edges = np.linspace(0.08, 5.6, 301)          # 300 detector bins, past both grid ends
    lo, hi = edges[:-1], edges[1:]
    mid = 0.5 * (lo + hi)
    Rf = (np.exp(-0.5 * ((mid[:, None] - np.linspace(0.1, 5.5, 40)[None, :]) / 0.08) ** 2)
          * (1000.0 + 200.0 * rng.standard_normal(1)[0])).astype(np.float32)
    ctx = context(w)
    dp = ppm.DeviceParams(w.inst)
    cnt = torch.from_numpy(w.counts).cuda()
    mc1 = torch.empty((dp.rows, 40), dtype=torch.float32, device="cuda")
    mc2 = torch.empty_like(mc1)
    ctx.set_response_fine(lo, hi, Rf, w.sigma_ism)
    ll1 = ctx.loglike(dp, cnt, w.tau, model_counts=mc1).cpu().numpy()
    R = (orc.downsample_matrix(w.E_keV, lo, hi) @ Rf.astype(np.float64)).astype(np.float32)
    ctx.set_response(R, w.sigma_ism)
    ll2 = ctx.loglike(dp, cnt, w.tau, model_counts=mc2).cpu().numpy()
    ctx.set_response(w.R, w.sigma_ism)
    assert max_rel(mc1.cpu().numpy(), mc2.cpu().numpy()) < 1e-6
    assert abs(ll1[0] - ll2[0]) <= 1e-6 * abs(ll2[0])


def test_non_finite_parameters_flag_their_instance(orc, synth, atm, small_lens):
    """A NaN or infinite value in a parameter that no range comparison
    reaches (spot azimuth, N_H, mask geometry) flags its own instance
    (PPM_ERANGE, logL = -inf, zero profile rows) and leaves the others equal
    to a clean run; so does an infinite mass.  mask_zeta = -inf is no mask."""
    w = synth.atm_two_spot(n_theta=8, n_phi=8, n_phase=16, n_E=32, n_chan=8, atm=atm,
                           lens=small_lens)
    inst = w.inst.select([0] * 7)
    inst.azim[1, 0] = np.nan
    inst.nh_1e20[2] = np.nan
    inst.mask_zeta[3, 1] = np.inf
    inst.mask_colat[4, 1] = np.nan
    inst.mask_azim[5, 1] = np.inf
    inst.mass_msun[6] = np.inf
    w2 = synth.Workload("b", inst, small_lens, w.E_keV, atm=atm, R=w.R, sigma_ism=w.sigma_ism,
                        counts=np.concatenate([w.counts] * 7), tau=w.tau)
    ll, _, st = gpu_loglike(w2)
    assert list(st) == [0, 2, 2, 2, 2, 2, 2]
    assert np.isfinite(ll[0]) and np.all(ll[1:] == -np.inf)
    ref, _, _ = gpu_loglike(w)
    assert abs(ll[0] - ref[0]) <= 1e-6 * abs(ref[0])
    Ft, st2 = gpu_profile(w2)
    assert list(st2) == list(st)
    assert np.isfinite(Ft).all() and not Ft[rows_of(w2, 1).start:].any()
    # a spot without a mask may say so with -inf
    w3 = synth.Workload("c", w.inst.copy(), small_lens, w.E_keV, atm=atm, R=w.R,
                        sigma_ism=w.sigma_ism, counts=w.counts, tau=w.tau)
    w3.inst.mask_zeta[0, 0] = -np.inf
    ll3, _, st3 = gpu_loglike(w3)
    assert st3[0] == 0 and abs(ll3[0] - ref[0]) <= 1e-6 * abs(ref[0])


def test_non_finite_blackbody_temperature_flags_its_instance(synth, small_lens):
    w = synth.bb_small(n_theta=8, n_phi=8, n_phase=16, n_E=16, lens=small_lens)
    inst = w.inst.select([0, 0])
    inst.logT[1, 0] = np.nan
    w2 = synth.Workload("b", inst, small_lens, w.E_keV)
    Ft, st = gpu_profile(w2)
    assert list(st) == [0, 2]
    assert np.isfinite(Ft).all() and Ft[:16].any() and not Ft[16:].any()
