"""ppm_profile_noalloc: the forward profile for callers that cannot allocate
GPU memory while evaluating (a sampler whose pool owns the rest of the device,
or one that cannot tolerate the synchronisation cudaMalloc implies).

The entry point is called through the C ABI twice in a row and compared with
ppm_profile on the same inputs, within the tolerance of the other profile
tests (1e-3 relative per non-negligible bin; the two run the same kernels, so
the results are expected to agree to rounding).  This file is collected last
so that a run stopping at the first failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-3


def _call_noalloc(ctx, dp, rows, nE):
    import torch
    from paper_2510_07764_gb300 import _abi
    out = torch.full((rows, nE), float("nan"), dtype=torch.float32, device="cuda")
    st = torch.full((dp.B,), -1, dtype=torch.int32, device="cuda")
    rc = _abi.ppm_profile_noalloc(ctx.h, dp.struct(), dp.res, C.c_void_p(out.data_ptr()),
                                  C.c_void_p(st.data_ptr()),
                                  C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == _abi.PPM_OK, _abi.ppm_last_error(ctx.h)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64), st.cpu().numpy()


def _max_rel(a, b):
    m = np.abs(b) >= 1e-6 * np.abs(b).max()
    return float(np.max(np.abs(a[m] - b[m]) / np.abs(b[m])))


def test_noalloc_matches_profile_twice():
    import paper_2510_07764_gb300 as ppm
    from paper_2510_07764_gb300 import synth
    w = synth.atm_two_spot()                       # 2 x 128^2, 128 phases, 256 energies
    ctx = ppm.Context(0)
    ctx.setup(w)
    dp = ppm.DeviceParams(w.inst)
    ref = ctx.profile(dp).cpu().numpy().astype(np.float64)
    for _ in range(2):
        got, st = _call_noalloc(ctx, dp, dp.rows, len(w.E_keV))
        assert list(st) == [0]
        assert np.isfinite(got).all()
        assert _max_rel(got, ref) < TOL
    ctx.close()


def test_noalloc_batch_and_status_twice():
    import paper_2510_07764_gb300 as ppm
    from paper_2510_07764_gb300 import synth
    lens = synth.LensSpec(u_min=0.30, u_max=0.40, n_u=129, n_cpsi=512, n_calpha=256)
    w = synth.atm_two_spot(n_theta=20, n_phi=40, n_phase=40, n_E=64, n_chan=8, lens=lens)
    inst = w.inst.select([0, 0, 0])
    inst.incl_rad[1] = 1.2
    inst.radius_km[2] = 9.0                        # compactness outside the lens grid
    ctx = ppm.Context(0)
    ctx.setup(w)
    dp = ppm.DeviceParams(inst)
    ref = ctx.profile(dp).cpu().numpy().astype(np.float64)
    ref_st = ctx.last_status.cpu().numpy()
    for _ in range(2):
        got, st = _call_noalloc(ctx, dp, dp.rows, len(w.E_keV))
        assert list(st) == list(ref_st) == [0, 0, 2]
        assert not got[80:].any()
        assert _max_rel(got[:80], ref[:80]) < TOL
    ctx.close()


def test_noalloc_rejects_problems_beyond_its_scratch():
    import paper_2510_07764_gb300 as ppm
    from paper_2510_07764_gb300 import _abi, synth
    w = synth.atm_two_spot(n_theta=8, n_phi=8, n_phase=32, n_E=32, n_chan=8)
    ctx = ppm.Context(0)
    ctx.setup(w)
    big = w.inst.replace(n_theta=4096, n_phi=4096, n_phase=4096)
    dp = ppm.DeviceParams(big)
    rc = _abi.ppm_profile_noalloc(ctx.h, dp.struct(), dp.res, C.c_void_p(1), None, None)
    assert rc == _abi.PPM_EINVAL
    assert "limited to" in _abi.ppm_last_error(ctx.h)
    ctx.close()
