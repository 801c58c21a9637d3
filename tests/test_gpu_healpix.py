"""The HEALPix whole-surface mesh (Sect. 2.6) on the GPU against the oracle."""
import math

import numpy as np
import pytest

from gpu_helpers import context, gpu_loglike, gpu_profile, max_rel

pytestmark = pytest.mark.gpu


def on_mesh(w, N):
    w.inst.grid = 1
    w.inst.n_theta[:] = N
    w.inst.n_phi[:] = 4 * N
    return w


def test_two_spot_on_the_mesh(orc, synth, atm, small_lens):
    w = on_mesh(synth.atm_two_spot(n_phase=32, n_E=64, n_chan=30, atm=atm, lens=small_lens), 48)
    Ft, st = gpu_profile(w)
    assert st[0] == 0
    assert max_rel(Ft, orc.profile(w)) < 1e-3


def test_blackbody_cap_on_the_mesh(orc, synth, small_lens):
    w = on_mesh(synth.bb_small(n_phase=32, n_E=24, lens=small_lens), 40)
    Ft, st = gpu_profile(w)
    assert st[0] == 0
    assert max_rel(Ft, orc.profile(w)) < 1e-4


def test_mesh_likelihood_and_gradient_rejected(orc, synth, atm, small_lens):
    import torch
    import paper_2510_07764_gb300 as ppm
    w = on_mesh(synth.atm_two_spot(n_phase=32, n_E=48, n_chan=30, atm=atm, lens=small_lens), 24)
    ll, mc, st = gpu_loglike(w)
    C = orc.counts_model(orc.profile(w), w.R, w.sigma_ism, 1.0)
    assert max_rel(mc, w.tau * C) < 1e-3
    ctx = context(w)
    dp = ppm.DeviceParams(w.inst)
    with pytest.raises(ppm.PPMError, match="spot grid"):
        ctx.loglike_grad(dp, torch.from_numpy(w.counts).cuda(), w.tau)


def test_mesh_noalloc_matches_profile(synth, atm, small_lens):
    import ctypes as C
    import torch
    import paper_2510_07764_gb300 as ppm
    from paper_2510_07764_gb300 import _abi
    w = on_mesh(synth.atm_two_spot(n_phase=32, n_E=48, n_chan=8, atm=atm, lens=small_lens), 32)
    ctx = context(w)
    dp = ppm.DeviceParams(w.inst)
    a = ctx.profile(dp)
    b = torch.empty_like(a)
    st = _abi.ppm_profile_noalloc(ctx.h, dp.struct(), dp.res, C.c_void_p(b.data_ptr()), None,
                                  C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    torch.cuda.synchronize()
    assert torch.equal(a, b)


# ---- full-surface temperature maps ----------------------------------------
def _smooth_map(orc, w, north_only=True):
    from test_oracle_healpix import pixel_centres
    th, ph = pixel_centres(orc, w)
    lt = 6.0 + 0.2 * np.cos(th) + 0.05 * np.sin(2 * ph)
    if north_only:
        lt = np.where(th < 1.2, lt, 0.0)
    return lt[None, :]


def test_temperature_map_atmosphere(orc, synth, atm, small_lens):
    w = on_mesh(synth.atm_two_spot(n_phase=32, n_E=64, n_chan=8, atm=atm, lens=small_lens), 24)
    w.inst = w.inst.select([0])
    w.inst.n_spots = 1
    for f in ("colat", "azim", "zeta", "logT", "mask_colat", "mask_azim", "mask_zeta"):
        setattr(w.inst, f, np.ascontiguousarray(getattr(w.inst, f)[:, :1]))
    w.inst.logT_map = _smooth_map(orc, w)
    Ft, st = gpu_profile(w)
    assert st[0] == 0
    assert max_rel(Ft, orc.profile(w)) < 1e-3


def test_temperature_map_blackbody(orc, synth, small_lens):
    w = on_mesh(synth.bb_small(n_phase=32, n_E=24, lens=small_lens), 20)
    w.inst.logT_map = _smooth_map(orc, w, north_only=False)
    Ft, st = gpu_profile(w)
    assert st[0] == 0
    assert max_rel(Ft, orc.profile(w)) < 1e-4


def test_map_of_a_uniform_cap_equals_the_cap_on_gpu(orc, synth, small_lens):
    from test_oracle_healpix import pixel_centres
    import math
    w = on_mesh(synth.bb_small(n_phase=32, n_E=24, lens=small_lens), 24)
    w.inst.colat[:] = 1.0
    w.inst.zeta[:] = 0.35
    cap, _ = gpu_profile(w)
    th, ph = pixel_centres(orc, w)
    cd = np.cos(th) * math.cos(1.0) + np.sin(th) * math.sin(1.0) * np.cos(ph - w.inst.azim[0, 0])
    w.inst.logT_map = np.where(cd >= math.cos(0.35), float(w.inst.logT[0, 0]), 0.0)[None, :]
    mp, st = gpu_profile(w)
    assert st[0] == 0
    assert max_rel(mp, cap) < 1e-6


def test_full_size_map_workload_sampled(orc, synth, atm):
    """The HEALPix temperature-map workload at full size (N_side 52, 32,448
    pixels, 128 phases, 256 energies): sampled bins against the oracle at
    1e-3 relative."""
    from gpu_helpers import gpu_profile, max_rel
    w = synth.healpix_map(atm=atm)
    got, st = gpu_profile(w)
    assert st[0] == 0
    rng = np.random.default_rng(5)
    js = np.sort(rng.choice(128, 4, replace=False))
    ks = np.sort(rng.choice(256, 8, replace=False))
    ref = orc.profile(w, jsel=js, ksel=ks)
    assert max_rel(got[np.ix_(js, ks)], ref) < 1e-3
    assert np.isfinite(got).all() and got.sum() > 0
