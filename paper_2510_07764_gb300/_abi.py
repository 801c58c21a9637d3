"""ctypes declarations of the C ABI in include/ppm.h (argument marshalling only).

The functions here carry the C names (``ppm_build_lens``, ``ppm_profile``,
``ppm_loglike`` ...).  Every computation happens in libppm.so; if the library
is missing this module raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# the bounds-checked build (libppm_check.so) is selected with PPM_LIB_PATH
LIB_PATH = os.environ.get("PPM_LIB_PATH") or os.path.join(HERE, "libppm.so")

PPM_OK, PPM_EINVAL, PPM_ERANGE, PPM_ENOMEM, PPM_ECUDA, PPM_ETIMEOUT, PPM_ENOTREADY = range(7)
STATUS_NAMES = ["PPM_OK", "PPM_EINVAL", "PPM_ERANGE", "PPM_ENOMEM", "PPM_ECUDA", "PPM_ETIMEOUT",
                "PPM_ENOTREADY"]

# every entry point declared in include/ppm.h
EXPORTS = ["ppm_create", "ppm_destroy", "ppm_last_error", "ppm_build_lens", "ppm_get_lens",
           "ppm_set_atmosphere", "ppm_set_energies", "ppm_set_response", "ppm_profile",
           "ppm_loglike", "ppm_sync", "ppm_set_timing", "ppm_get_timing",
           "ppm_profile_noalloc", "ppm_loglike_grad", "ppm_set_interpolation",
           "ppm_set_tiles", "ppm_get_tiles", "ppm_autotune", "ppm_set_response_fine",
           "ppm_fp32_peak"]

# interpolation strategies of Sect. 4 (PPM_INTERP_* in ppm.h), keyed by the
# paper's panel letters
INTERP = {"d": 0, "a": 1, "b": 2, "c": 3}


class ppm_lens_spec(C.Structure):
    _fields_ = [("u_min", C.c_double), ("u_max", C.c_double), ("n_u", C.c_int),
                ("cpsi_min", C.c_double), ("cpsi_max", C.c_double), ("n_cpsi", C.c_int),
                ("calpha_min", C.c_double), ("calpha_max", C.c_double), ("n_calpha", C.c_int),
                ("dalpha", C.c_double)]


PARAM_FIELDS = ["mass_msun", "radius_km", "spin_hz", "incl_rad", "dist_kpc", "nh_1e20",
                "colat", "azim", "zeta", "logT", "mask_colat", "mask_azim", "mask_zeta"]


class ppm_params(C.Structure):
    _fields_ = [("B", C.c_int), ("n_spots", C.c_int), ("oblate", C.c_int),
                ("emission", C.c_int)] + [(f, C.c_void_p) for f in PARAM_FIELDS] + \
               [("logT_map", C.c_void_p)]


class ppm_tiles(C.Structure):
    _fields_ = [("phase_tile", C.c_int), ("waves", C.c_int), ("persistent", C.c_int),
                ("walk", C.c_int), ("ms", C.c_double)]


class ppm_timing(C.Structure):
    _fields_ = [("ms_ring", C.c_double), ("ms_shift_add", C.c_double),
                ("ms_reduce", C.c_double), ("ms_loglike", C.c_double),
                ("ms_grad_resp", C.c_double), ("ms_shift_add_bwd", C.c_double),
                ("ms_template_bwd", C.c_double),
                ("calls", C.c_longlong), ("launches", C.c_longlong), ("triples", C.c_double)]


class ppm_res(C.Structure):
    _fields_ = [("n_theta", C.POINTER(C.c_int)), ("n_phi", C.POINTER(C.c_int)),
                ("n_phase", C.POINTER(C.c_int)), ("n_fp", C.c_int), ("grid", C.c_int),
                ("phase_sub", C.c_int)]


_lib = None


class LibraryMissing(RuntimeError):
    pass


def lib() -> C.CDLL:
    """Load libppm.so (built by ``paper_2510_07764_gb300.build.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise LibraryMissing("libppm.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
    L = C.CDLL(LIB_PATH)
    vp, i, d = C.c_void_p, C.c_int, C.c_double
    sig = {
        "ppm_create": (i, [C.POINTER(vp), i]),
        "ppm_destroy": (None, [vp]),
        "ppm_last_error": (C.c_char_p, [vp]),
        "ppm_build_lens": (i, [vp, C.POINTER(ppm_lens_spec), vp]),
        "ppm_get_lens": (i, [vp, vp, vp, vp]),
        "ppm_set_atmosphere": (i, [vp, vp, vp, i, vp, i, vp, i, vp, i, i]),
        "ppm_set_energies": (i, [vp, vp, i]),
        "ppm_set_interpolation": (i, [vp, i]),
        "ppm_set_response": (i, [vp, vp, i, i, vp]),
        "ppm_set_response_fine": (i, [vp, vp, vp, i, vp, i, vp]),
        "ppm_profile": (i, [vp, C.POINTER(ppm_params), C.POINTER(ppm_res), vp, vp, vp]),
        "ppm_profile_noalloc": (i, [vp, C.POINTER(ppm_params), C.POINTER(ppm_res), vp, vp, vp]),
        "ppm_loglike": (i, [vp, C.POINTER(ppm_params), C.POINTER(ppm_res), vp, i, vp, d, vp, vp,
                            vp, vp]),
        "ppm_loglike_grad": (i, [vp, C.POINTER(ppm_params), C.POINTER(ppm_res), vp, i, vp, d,
                                 vp, vp, vp, vp]),
        "ppm_sync": (i, [vp, vp, d]),
        "ppm_fp32_peak": (i, [i, i, vp, C.POINTER(d)]),
        "ppm_set_tiles": (i, [vp, C.POINTER(ppm_tiles)]),
        "ppm_get_tiles": (i, [vp, C.POINTER(ppm_tiles)]),
        "ppm_autotune": (i, [vp, C.POINTER(ppm_params), C.POINTER(ppm_res), vp,
                             C.POINTER(ppm_tiles)]),
        "ppm_set_timing": (i, [vp, i]),
        "ppm_get_timing": (i, [vp, C.POINTER(ppm_timing)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


# thin wrappers with the C names -------------------------------------------
def ppm_create(device: int = 0):
    h = C.c_void_p()
    st = lib().ppm_create(C.byref(h), device)
    return st, h


def ppm_destroy(ctx) -> None:
    lib().ppm_destroy(ctx)


def ppm_last_error(ctx) -> str:
    return lib().ppm_last_error(ctx).decode()


def ppm_build_lens(ctx, spec: ppm_lens_spec, stream=None) -> int:
    return lib().ppm_build_lens(ctx, C.byref(spec), stream)


def ppm_get_lens(ctx, Ca, LF, TD) -> int:
    return lib().ppm_get_lens(ctx, Ca, LF, TD)


def ppm_set_atmosphere(ctx, I, logT, nT, logg, ng, mu, nmu, lnE, nE, n_protect) -> int:
    return lib().ppm_set_atmosphere(ctx, I, logT, nT, logg, ng, mu, nmu, lnE, nE, n_protect)


def ppm_set_interpolation(ctx, strategy: int) -> int:
    return lib().ppm_set_interpolation(ctx, strategy)


def ppm_set_energies(ctx, E, nE) -> int:
    return lib().ppm_set_energies(ctx, E, nE)


def ppm_set_response(ctx, R, nE, nc, sigma) -> int:
    return lib().ppm_set_response(ctx, R, nE, nc, sigma)


def ppm_set_response_fine(ctx, E_lo, E_hi, Ne, Rf, nc, sigma) -> int:
    return lib().ppm_set_response_fine(ctx, E_lo, E_hi, Ne, Rf, nc, sigma)


def ppm_profile(ctx, params: ppm_params, res: ppm_res, Ft, inst_status, stream) -> int:
    return lib().ppm_profile(ctx, C.byref(params), C.byref(res), Ft, inst_status, stream)


def ppm_profile_noalloc(ctx, params: ppm_params, res: ppm_res, Ft, inst_status, stream) -> int:
    return lib().ppm_profile_noalloc(ctx, C.byref(params), C.byref(res), Ft, inst_status, stream)


def ppm_loglike(ctx, params: ppm_params, res: ppm_res, counts, counts_shared, bkg, tau, logL,
                model_counts, inst_status, stream) -> int:
    return lib().ppm_loglike(ctx, C.byref(params), C.byref(res), counts, counts_shared, bkg,
                             tau, logL, model_counts, inst_status, stream)


def ppm_loglike_grad(ctx, params: ppm_params, res: ppm_res, counts, counts_shared, bkg, tau,
                     logL, grad, inst_status, stream) -> int:
    return lib().ppm_loglike_grad(ctx, C.byref(params), C.byref(res), counts, counts_shared,
                                  bkg, tau, logL, grad, inst_status, stream)


def ppm_set_tiles(ctx, t: ppm_tiles) -> int:
    return lib().ppm_set_tiles(ctx, C.byref(t))


def ppm_get_tiles(ctx, t: ppm_tiles) -> int:
    return lib().ppm_get_tiles(ctx, C.byref(t))


def ppm_autotune(ctx, params: ppm_params, res: ppm_res, stream, best: ppm_tiles) -> int:
    return lib().ppm_autotune(ctx, C.byref(params), C.byref(res), stream, C.byref(best))


def ppm_fp32_peak(device: int, paired: int, stream):
    v = C.c_double()
    st = lib().ppm_fp32_peak(device, paired, stream, C.byref(v))
    return st, v.value


def ppm_sync(ctx, stream, timeout_s: float) -> int:
    return lib().ppm_sync(ctx, stream, timeout_s)


def ppm_set_timing(ctx, enable: int) -> int:
    return lib().ppm_set_timing(ctx, enable)


def ppm_get_timing(ctx, out: ppm_timing) -> int:
    return lib().ppm_get_timing(ctx, C.byref(out))
