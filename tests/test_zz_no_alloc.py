"""ppm_profile_noalloc: the forward profile for callers that cannot allocate
GPU memory while evaluating (a sampler whose memory pool already owns the
rest of the device, or one that cannot tolerate the device-wide
synchronisation cudaMalloc and cudaFree imply while other work is in flight).

The entry point is called through the C ABI, twice in a row on the same
inputs:
* against ppm_profile: its plan follows ppm_profile's rules, so the two give
  the same floats bit for bit (the same items summed in the same order);
* against the FP64 oracle on a reduced two-spot case, at the 1e-3 relative
  tolerance of the other profile tests;
* with the free device memory read before and after, on a context that has
  never run ppm_profile: the calls allocate nothing.
This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-3


def _noalloc(ctx, dp, out, st, stream=None):
    import torch
    from paper_2510_07764_gb300 import _abi
    s = stream if stream is not None else torch.cuda.current_stream()
    return _abi.ppm_profile_noalloc(ctx.h, dp.struct(), dp.res, C.c_void_p(out.data_ptr()),
                                    C.c_void_p(st.data_ptr()), C.c_void_p(s.cuda_stream))


def _call_noalloc(ctx, dp, rows, nE):
    import torch
    from paper_2510_07764_gb300 import _abi
    out = torch.full((rows, nE), float("nan"), dtype=torch.float32, device="cuda")
    st = torch.full((dp.B,), -1, dtype=torch.int32, device="cuda")
    rc = _noalloc(ctx, dp, out, st)
    assert rc == _abi.PPM_OK, _abi.ppm_last_error(ctx.h)
    torch.cuda.synchronize()
    return out.cpu().numpy(), st.cpu().numpy()


def _max_rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    m = np.abs(b) >= 1e-6 * np.abs(b).max()
    return float(np.max(np.abs(a[m] - b[m]) / np.abs(b[m])))


def test_noalloc_equals_profile_bitwise_twice():
    import paper_2510_07764_gb300 as ppm
    from paper_2510_07764_gb300 import synth
    w = synth.atm_two_spot()                       # 2 x 128^2, 128 phases, 256 energies
    ctx = ppm.Context(0)
    ctx.setup(w)
    dp = ppm.DeviceParams(w.inst)
    ref = ctx.profile(dp).cpu().numpy()
    for _ in range(2):
        got, st = _call_noalloc(ctx, dp, dp.rows, len(w.E_keV))
        assert list(st) == [0]
        assert np.isfinite(got).all()
        assert np.array_equal(got, ref)
    ctx.close()


def test_noalloc_matches_the_oracle_twice(orc):
    import paper_2510_07764_gb300 as ppm
    from paper_2510_07764_gb300 import synth
    lens = synth.LensSpec(u_min=0.30, u_max=0.40, n_u=129, n_cpsi=512)
    w = synth.atm_two_spot(n_theta=24, n_phi=40, n_phase=40, n_E=72, n_chan=24, lens=lens)
    ctx = ppm.Context(0)
    ctx.setup(w)
    dp = ppm.DeviceParams(w.inst)
    ref = orc.profile(w)
    for _ in range(2):
        got, st = _call_noalloc(ctx, dp, dp.rows, len(w.E_keV))
        assert list(st) == [0]
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
    ref = ctx.profile(dp).cpu().numpy()
    ref_st = ctx.last_status.cpu().numpy()
    for _ in range(2):
        got, st = _call_noalloc(ctx, dp, dp.rows, len(w.E_keV))
        assert list(st) == list(ref_st) == [0, 0, 2]
        assert not got[80:].any()
        assert np.array_equal(got, ref)
    ctx.close()


def test_noalloc_allocates_no_device_memory():
    """A fresh context that has never run ppm_profile: after one warm-up call
    (the array's address is looked up on the first call), two more calls
    leave the device's free memory unchanged and give the same result."""
    import torch
    import paper_2510_07764_gb300 as ppm
    from paper_2510_07764_gb300 import _abi, synth
    lens = synth.LensSpec(u_min=0.30, u_max=0.40, n_u=129, n_cpsi=512)
    w = synth.atm_two_spot(n_theta=32, n_phi=48, n_phase=64, n_E=96, n_chan=8, lens=lens)
    ctx = ppm.Context(0)
    ctx.setup(w)
    dp = ppm.DeviceParams(w.inst)
    out = torch.empty((dp.rows, len(w.E_keV)), dtype=torch.float32, device="cuda")
    st = torch.empty((dp.B,), dtype=torch.int32, device="cuda")
    outs = [torch.full_like(out, float("nan")) for _ in range(2)]
    assert _noalloc(ctx, dp, out, st) == _abi.PPM_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for o in outs:
        assert _noalloc(ctx, dp, o, st) == _abi.PPM_OK, _abi.ppm_last_error(ctx.h)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
    for o in outs:
        assert torch.equal(o, out)
    ctx.close()


def test_noalloc_refuses_a_capturing_stream():
    """The plan comes from a static host buffer that the next call rewrites,
    so a stream in capture is refused before anything is enqueued; the
    capture itself stays usable."""
    import torch
    import paper_2510_07764_gb300 as ppm
    from paper_2510_07764_gb300 import _abi, synth
    lens = synth.LensSpec(u_min=0.30, u_max=0.40, n_u=129, n_cpsi=512)
    w = synth.atm_two_spot(n_theta=8, n_phi=12, n_phase=16, n_E=32, n_chan=8, lens=lens)
    ctx = ppm.Context(0)
    ctx.setup(w)
    dp = ppm.DeviceParams(w.inst)
    out = torch.zeros((dp.rows, len(w.E_keV)), dtype=torch.float32, device="cuda")
    st = torch.zeros((dp.B,), dtype=torch.int32, device="cuda")
    x = torch.zeros(4, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        rc = _noalloc(ctx, dp, out, st, stream=s)
        x.add_(1.0)
    assert rc == _abi.PPM_EINVAL
    assert "captured" in _abi.ppm_last_error(ctx.h)
    g.replay()
    torch.cuda.synchronize()
    assert float(x.sum()) == 4.0 and not out.any()
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
