"""Helpers shared by the GPU parity tests (CUDA path through the C ABI)."""
import numpy as np

_ctx_cache = {}


def context(w, key=None):
    """A library context with the tables of workload w (lens built once per spec)."""
    import paper_2510_07764_gb300 as ppm
    k = key or ("lens", tuple(sorted(vars(w.lens).items())))
    if k not in _ctx_cache:
        ctx = ppm.Context(0)
        ctx.build_lens(w.lens)
        _ctx_cache[k] = ctx
    ctx = _ctx_cache[k]
    if w.atm is not None:
        ctx.set_atmosphere(w.atm)
    ctx.set_interpolation(getattr(w, "interp", "d"))
    ctx.set_energies(w.E_keV)
    if w.R is not None:
        ctx.set_response(w.R, w.sigma_ism)
    return ctx


def gpu_profile(w):
    """(F_t float64 numpy [rows, nE], status numpy [B]) from ppm_profile."""
    import paper_2510_07764_gb300 as ppm
    ctx = context(w)
    dp = ppm.DeviceParams(w.inst)
    Ft = ctx.profile(dp)
    ctx.sync()
    return Ft.cpu().numpy().astype(np.float64), ctx.last_status.cpu().numpy()


def gpu_loglike(w, counts=None, counts_shared=False, bkg=None):
    import torch
    import paper_2510_07764_gb300 as ppm
    ctx = context(w)
    dp = ppm.DeviceParams(w.inst)
    cnt = torch.from_numpy(np.ascontiguousarray(w.counts if counts is None else counts)).cuda()
    bk = None if bkg is None else torch.from_numpy(np.ascontiguousarray(bkg, np.float32)).cuda()
    mc = torch.empty((dp.rows, w.nc), dtype=torch.float32, device="cuda")
    ll = ctx.loglike(dp, cnt, w.tau, bkg=bk, counts_shared=counts_shared, model_counts=mc)
    ctx.sync()
    return ll.cpu().numpy(), mc.cpu().numpy().astype(np.float64), ctx.last_status.cpu().numpy()


def rows_of(w, b):
    r0 = int(np.sum(w.inst.n_phase[:b]))
    return slice(r0, r0 + int(w.inst.n_phase[b]))


def max_rel(got, ref, floor_frac=1e-6):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    m = np.abs(ref) >= floor_frac * np.max(np.abs(ref))
    return float(np.max(np.abs(got[m] - ref[m]) / np.abs(ref[m]))) if m.any() else 0.0
