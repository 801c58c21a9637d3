"""GB300-native pulse-profile likelihood (arXiv 2510.07764).

Python front end of libppm.so.  PyTorch provides device memory and streams;
every step of the forward model and the likelihood runs in the library's CUDA
kernels.  ``Context`` wraps one library context; ``DeviceParams`` holds the
structure-of-arrays parameter vectors as CUDA tensors.
"""
from __future__ import annotations

import ctypes as C
from typing import Optional

import numpy as np

from . import _abi
from ._abi import (PPM_EINVAL, PPM_ENOMEM, PPM_ENOTREADY, PPM_ERANGE, PPM_ETIMEOUT, PPM_OK,
                   LibraryMissing)

__all__ = ["Context", "DeviceParams", "InstanceView", "PPMError", "LibraryMissing", "LogLikelihood",
           "GRAD_NAMES", "N_GRAD", "PPM_OK", "PPM_ERANGE", "PPM_EINVAL", "PPM_ENOMEM", "PPM_ETIMEOUT",
           "PPM_ENOTREADY"]

# order of the gradient columns of ppm_loglike_grad
GRAD_NAMES = ("mass_msun", "radius_km", "incl_rad", "dist_kpc", "nh_1e20",
              "colat_1", "azim_1", "zeta_1", "logT_1", "colat_2", "azim_2", "zeta_2", "logT_2")
N_GRAD = len(GRAD_NAMES)


class PPMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (_abi.STATUS_NAMES[status] if 0 <= status < 7 else status, msg))
        self.status = status


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


class DeviceParams:
    """SoA parameter vectors on the GPU (float64 CUDA tensors)."""

    def __init__(self, inst, device="cuda"):
        import torch
        self.inst = inst
        self.B = inst.B
        self.n_spots = inst.n_spots
        self.oblate = int(inst.oblate)
        self.emission = int(inst.emission)
        self.t = {f: torch.empty(getattr(inst, f).size, dtype=torch.float64, device=device)
                  for f in _abi.PARAM_FIELDS}
        tmap = getattr(inst, "logT_map", None)
        # full-surface temperature map (HEALPix ring order, instances concatenated)
        self.t_map = None if tmap is None else torch.from_numpy(
            np.ascontiguousarray(np.concatenate([np.asarray(tmap[b], dtype=np.float64).ravel()
                                                 for b in range(inst.B)]))).to(device)
        self.upload(inst)
        self._res_arrays(inst)

    def _res_arrays(self, inst):
        self.n_theta = np.ascontiguousarray(inst.n_theta, dtype=np.int32)
        self.n_phi = np.ascontiguousarray(inst.n_phi, dtype=np.int32)
        self.n_phase = np.ascontiguousarray(inst.n_phase, dtype=np.int32)
        self.n_fp = int(inst.n_fp)
        ip = C.POINTER(C.c_int)
        self.grid = int(getattr(inst, "grid", 0))
        self.phase_sub = int(getattr(inst, "phase_sub", 1))
        self.res = _abi.ppm_res(self.n_theta.ctypes.data_as(ip), self.n_phi.ctypes.data_as(ip),
                                self.n_phase.ctypes.data_as(ip), self.n_fp, self.grid,
                                self.phase_sub)
        self.rows = int(self.n_phase.sum())

    def upload(self, inst, non_blocking: bool = False):
        """Copy parameter values (host numpy or pinned tensors) into the device arrays."""
        import torch
        for f in _abi.PARAM_FIELDS:
            src = getattr(inst, f)
            if isinstance(src, torch.Tensor):
                self.t[f].copy_(src.reshape(-1), non_blocking=non_blocking)
            else:
                self.t[f].copy_(torch.from_numpy(np.ascontiguousarray(src, dtype=np.float64).reshape(-1)),
                                non_blocking=non_blocking)

    def set_theta(self, theta):
        """Write a [B, 13] float64 CUDA tensor of differentiated parameters
        (columns in ``GRAD_NAMES`` order) into the device arrays."""
        B, ns = self.B, self.n_spots
        for j, f in enumerate(("mass_msun", "radius_km", "incl_rad", "dist_kpc", "nh_1e20")):
            self.t[f].copy_(theta[:, j])
        for s in range(ns):
            for q, f in enumerate(("colat", "azim", "zeta", "logT")):
                self.t[f].view(B, ns)[:, s].copy_(theta[:, 5 + 4 * s + q])

    def theta(self):
        """The differentiated parameters as a [B, 13] float64 CUDA tensor."""
        import torch
        B, ns = self.B, self.n_spots
        th = torch.zeros((B, N_GRAD), dtype=torch.float64, device=self.t["mass_msun"].device)
        for j, f in enumerate(("mass_msun", "radius_km", "incl_rad", "dist_kpc", "nh_1e20")):
            th[:, j] = self.t[f]
        for s in range(ns):
            for q, f in enumerate(("colat", "azim", "zeta", "logT")):
                th[:, 5 + 4 * s + q] = self.t[f].view(B, ns)[:, s]
        return th

    def struct(self) -> _abi.ppm_params:
        p = _abi.ppm_params()
        p.B, p.n_spots, p.oblate, p.emission = self.B, self.n_spots, self.oblate, self.emission
        for f in _abi.PARAM_FIELDS:
            setattr(p, f, self.t[f].data_ptr())
        p.logT_map = None if self.t_map is None else self.t_map.data_ptr()
        return p

    def instance(self, b: int) -> "InstanceView":
        """Instance b alone, as a one-instance argument of the same calls; it
        points into these device arrays (no copy)."""
        return InstanceView(self, b)


# per-spot parameter arrays ([B, n_spots]); the others have one value per instance
_SPOT_FIELDS = ("colat", "azim", "zeta", "logT", "mask_colat", "mask_azim", "mask_zeta")


class InstanceView:
    """One instance of a DeviceParams (B = 1) sharing its device arrays: the
    pointers of its ppm_params and ppm_res are offset to instance b."""

    def __init__(self, dp: DeviceParams, b: int):
        if not 0 <= b < dp.B:
            raise IndexError("instance %d of %d" % (b, dp.B))
        self.parent, self.b = dp, b
        self.B, self.n_spots, self.oblate, self.emission = 1, dp.n_spots, dp.oblate, dp.emission
        self.rows = int(dp.n_phase[b])
        self.row0 = int(dp.n_phase[:b].sum())
        ip = C.POINTER(C.c_int)
        at = lambda a: C.cast(a.ctypes.data + 4 * b, ip)
        self.res = _abi.ppm_res(at(dp.n_theta), at(dp.n_phi), at(dp.n_phase), dp.n_fp, dp.grid,
                                dp.phase_sub)
        self._pix0 = int(sum(12 * int(n) ** 2 for n in dp.n_theta[:b])) if dp.grid == 1 else 0

    def struct(self) -> _abi.ppm_params:
        dp = self.parent
        p = _abi.ppm_params()
        p.B, p.n_spots, p.oblate, p.emission = 1, self.n_spots, self.oblate, self.emission
        for f in _abi.PARAM_FIELDS:
            per = self.n_spots if f in _SPOT_FIELDS else 1
            setattr(p, f, dp.t[f].data_ptr() + 8 * per * self.b)
        p.logT_map = None if dp.t_map is None else dp.t_map.data_ptr() + 8 * self._pix0
        return p


class Context:
    """One libppm context (tables + workspace) on a CUDA device."""

    def __init__(self, device: int = 0):
        st, h = _abi.ppm_create(device)
        if st != PPM_OK:
            raise PPMError(st, "ppm_create failed on device %d" % device)
        self.h = h
        self.device = device
        self.nE = 0
        self.nc = 0

    def close(self):
        if getattr(self, "h", None):
            _abi.ppm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int):
        if st != PPM_OK:
            raise PPMError(st, _abi.ppm_last_error(self.h))

    # ---- tables -------------------------------------------------------------
    def build_lens(self, spec, stream=None):
        s = _abi.ppm_lens_spec(spec.u_min, spec.u_max, spec.n_u, spec.cpsi_min, spec.cpsi_max,
                               spec.n_cpsi, spec.calpha_min, spec.calpha_max, spec.n_calpha,
                               spec.dalpha)
        self._check(_abi.ppm_build_lens(self.h, s, _stream_handle(stream)))
        self.lens_spec = spec

    def get_lens(self):
        s = self.lens_spec
        Ca = np.empty((s.n_u, s.n_cpsi))
        LF = np.empty((s.n_u, s.n_cpsi))
        TD = np.empty((s.n_u, s.n_calpha))
        self._check(_abi.ppm_get_lens(self.h, _dp(Ca), _dp(LF), _dp(TD)))
        return Ca, LF, TD

    def set_atmosphere(self, t):
        arrs = [np.ascontiguousarray(t.I, dtype=np.float32)] + \
               [np.ascontiguousarray(a, dtype=np.float64) for a in (t.logT, t.logg, t.mu, t.lnE)]
        I, lT, lg, mu, lnE = arrs
        self._check(_abi.ppm_set_atmosphere(self.h, _dp(I), _dp(lT), len(lT), _dp(lg), len(lg),
                                            _dp(mu), len(mu), _dp(lnE), len(lnE),
                                            int(t.n_protect)))

    def set_interpolation(self, strategy: str = "d"):
        """Atmosphere interpolation strategy of Sect. 4: "d" (the method's mixed
        scheme, default), "a" (cubic everywhere), "b" (a, clipped at zero),
        "c" (cubic everywhere with linear edges)."""
        self._check(_abi.ppm_set_interpolation(self.h, _abi.INTERP[strategy]))

    def set_energies(self, E_keV):
        E = np.ascontiguousarray(E_keV, dtype=np.float64)
        self._check(_abi.ppm_set_energies(self.h, _dp(E), len(E)))
        self.nE = len(E)

    def set_response(self, R, sigma):
        R = np.ascontiguousarray(R, dtype=np.float32)
        sg = np.ascontiguousarray(sigma, dtype=np.float32)
        self._check(_abi.ppm_set_response(self.h, _dp(R), R.shape[0], R.shape[1], _dp(sg)))
        self.nc = R.shape[1]

    def set_response_fine(self, E_lo, E_hi, Rf, sigma):
        """Response from a fine detector grid through the down-sampling matrix
        (see ppm_set_response_fine); Rf is [Ne, nc]."""
        lo = np.ascontiguousarray(E_lo, dtype=np.float64)
        hi = np.ascontiguousarray(E_hi, dtype=np.float64)
        Rf = np.ascontiguousarray(Rf, dtype=np.float32)
        sg = np.ascontiguousarray(sigma, dtype=np.float32)
        self._check(_abi.ppm_set_response_fine(self.h, _dp(lo), _dp(hi), len(lo), _dp(Rf),
                                               Rf.shape[1], _dp(sg)))
        self.nc = Rf.shape[1]

    def setup(self, w, build_lens: bool = True):
        """Load every table of a synthetic workload (``synth.Workload``)."""
        if build_lens:
            self.build_lens(w.lens)
        if w.atm is not None:
            self.set_atmosphere(w.atm)
        self.set_interpolation(getattr(w, "interp", "d"))
        self.set_energies(w.E_keV)
        if w.R is not None:
            self.set_response(w.R, w.sigma_ism)

    # ---- compute ------------------------------------------------------------
    def profile(self, dp: DeviceParams, out=None, status=None, stream=None):
        """F_t [sum_b n_phase_b, nE] float32 (CUDA tensor)."""
        import torch
        if out is None:
            out = torch.empty((max(dp.rows, 0), self.nE), dtype=torch.float32,
                              device="cuda:%d" % self.device)
        if status is None:
            status = torch.empty(dp.B, dtype=torch.int32, device=out.device)
        self._check(_abi.ppm_profile(self.h, dp.struct(), dp.res, C.c_void_p(out.data_ptr()),
                                     C.c_void_p(status.data_ptr()), _stream_handle(stream)))
        self.last_status = status
        return out

    def loglike(self, dp: DeviceParams, counts, tau: float, bkg=None, counts_shared=False,
                out=None, model_counts=None, status=None, stream=None):
        """Poisson log-likelihood per instance, float64 CUDA tensor [B]."""
        import torch
        dev = counts.device
        if out is None:
            out = torch.empty(dp.B, dtype=torch.float64, device=dev)
        if status is None:
            status = torch.empty(dp.B, dtype=torch.int32, device=dev)
        ptr = lambda t: C.c_void_p(t.data_ptr()) if t is not None else None
        self._check(_abi.ppm_loglike(self.h, dp.struct(), dp.res, ptr(counts), int(counts_shared),
                                     ptr(bkg), float(tau), ptr(out), ptr(model_counts),
                                     ptr(status), _stream_handle(stream)))
        self.last_status = status
        return out

    def loglike_grad(self, dp: DeviceParams, counts, tau: float, bkg=None, counts_shared=False,
                     out=None, grad=None, status=None, stream=None):
        """Log-likelihood [B] and its gradient [B, 13] (float64 CUDA tensors);
        gradient columns in ``GRAD_NAMES`` order."""
        import torch
        dev = counts.device
        if out is None:
            out = torch.empty(dp.B, dtype=torch.float64, device=dev)
        if grad is None:
            grad = torch.empty((dp.B, N_GRAD), dtype=torch.float64, device=dev)
        if status is None:
            status = torch.empty(dp.B, dtype=torch.int32, device=dev)
        ptr = lambda t: C.c_void_p(t.data_ptr()) if t is not None else None
        self._check(_abi.ppm_loglike_grad(self.h, dp.struct(), dp.res, ptr(counts),
                                          int(counts_shared), ptr(bkg), float(tau), ptr(out),
                                          ptr(grad), ptr(status), _stream_handle(stream)))
        self.last_status = status
        return out, grad

    def set_tiles(self, phase_tile: int = 0, waves: int = 16, persistent: bool = False,
                  walk: int = 0):
        """Work decomposition of the shift-and-add (see ppm_set_tiles)."""
        self._check(_abi.ppm_set_tiles(self.h, _abi.ppm_tiles(phase_tile, waves,
                                                               int(persistent), int(walk), 0.0)))

    def get_tiles(self) -> dict:
        t = _abi.ppm_tiles()
        self._check(_abi.ppm_get_tiles(self.h, t))
        return {"phase_tile": t.phase_tile, "waves": t.waves, "persistent": bool(t.persistent),
                "walk": t.walk}

    def autotune(self, dp: DeviceParams, stream=None) -> dict:
        """Time the tile candidates on dp's problem, keep the fastest, return it."""
        t = _abi.ppm_tiles()
        self._check(_abi.ppm_autotune(self.h, dp.struct(), dp.res, _stream_handle(stream), t))
        return {"phase_tile": t.phase_tile, "waves": t.waves, "persistent": bool(t.persistent),
                "walk": t.walk, "ms": t.ms}

    def set_timing(self, enable: bool = True):
        self._check(_abi.ppm_set_timing(self.h, int(enable)))

    def get_timing(self) -> dict:
        t = _abi.ppm_timing()
        self._check(_abi.ppm_get_timing(self.h, t))
        return {f: getattr(t, f) for f, _ in t._fields_}

    def sync(self, stream=None, timeout: float = 30.0):
        self._check(_abi.ppm_sync(self.h, _stream_handle(stream), timeout))


def _loglike_function():
    import torch

    class _LogLike(torch.autograd.Function):
        @staticmethod
        def forward(fctx, theta, ctx, dp, counts, tau, bkg, counts_shared):
            dp.set_theta(theta.detach())
            ll, g = ctx.loglike_grad(dp, counts, tau, bkg=bkg, counts_shared=counts_shared)
            fctx.save_for_backward(g)
            return ll

        @staticmethod
        def backward(fctx, gout):
            (g,) = fctx.saved_tensors
            return gout[:, None] * g, None, None, None, None, None, None

    return _LogLike


_LOGLIKE_FN = None


def LogLikelihood(theta, ctx: "Context", dp: DeviceParams, counts, tau: float, bkg=None,
                  counts_shared: bool = False):
    """logL[b](theta[b]) as a differentiable torch function.

    theta: [B, 13] float64 CUDA tensor (``GRAD_NAMES`` order, requires_grad as
    needed); the other parameters (spin, masks, resolutions) come from ``dp``.
    When autograd needs the gradient (grad mode on and theta requiring it) the
    forward call computes logL and its gradient together through
    ppm_loglike_grad and backward scales the stored gradient; otherwise it
    runs the forward likelihood alone (ppm_loglike)."""
    import torch
    if not (torch.is_grad_enabled() and theta.requires_grad):
        dp.set_theta(theta.detach())
        return ctx.loglike(dp, counts, tau, bkg=bkg, counts_shared=counts_shared)
    global _LOGLIKE_FN
    if _LOGLIKE_FN is None:
        _LOGLIKE_FN = _loglike_function()
    return _LOGLIKE_FN.apply(theta, ctx, dp, counts, tau, bkg, counts_shared)
