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
