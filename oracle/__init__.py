"""FP64 CPU oracle of the pulse-profile likelihood (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``.  The library's product path never
imports it.  The C source (``ppm_oracle.c``) shares nothing with the CUDA path.

Parity pins live in ``tests/test_oracle_*.py``.  Functions whose only check is
self-consistency say so in their docstring ("parity unpinned").
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ppm_oracle.c")
_LIB = os.path.join(_HERE, "libppm_oracle.so")
_SRC_T = os.path.join(_HERE, "ppm_oracle_tangent.c")
_LIB_T = os.path.join(_HERE, "libppm_oracle_tangent.so")
_lib = None
_lib_t = None

PI = math.pi


def _compile(src, lib, std, force):
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(src))
    if force or not os.path.exists(lib) or os.path.getmtime(lib) < newest:
        tmp = lib + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=" + std, "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, src, "-lm"])
        os.replace(tmp, lib)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (double precision, no FMA contraction), and
    its forward-mode (complex-step) build."""
    _compile(_SRC, _LIB, "c99", force)
    _compile(_SRC_T, _LIB_T, "c11", force)
    return _LIB


class LensSpecC(C.Structure):
    _fields_ = [("u_min", C.c_double), ("u_max", C.c_double), ("n_u", C.c_int),
                ("cpsi_min", C.c_double), ("cpsi_max", C.c_double), ("n_cpsi", C.c_int),
                ("calpha_min", C.c_double), ("calpha_max", C.c_double), ("n_calpha", C.c_int),
                ("dalpha", C.c_double)]


class LensC(C.Structure):
    _fields_ = [("spec", LensSpecC), ("Ca", C.POINTER(C.c_double)),
                ("LF", C.POINTER(C.c_double)), ("TD", C.POINTER(C.c_double))]


class AtmC(C.Structure):
    _fields_ = [("nT", C.c_int), ("ng", C.c_int), ("nmu", C.c_int), ("nE", C.c_int),
                ("n_protect", C.c_int),
                ("logT", C.POINTER(C.c_double)), ("logg", C.POINTER(C.c_double)),
                ("mu", C.POINTER(C.c_double)), ("lnE", C.POINTER(C.c_double)),
                ("I", C.POINTER(C.c_float)), ("strategy", C.c_int)]


# interpolation strategies of Sect. 4 (ORC_INTERP_* in ppm_oracle.c)
INTERP = {"d": 0, "a": 1, "b": 2, "c": 3}


class InstC(C.Structure):
    _fields_ = [("mass_msun", C.c_double), ("radius_km", C.c_double), ("spin_hz", C.c_double),
                ("incl_rad", C.c_double), ("dist_kpc", C.c_double), ("nh_1e20", C.c_double),
                ("colat", C.c_double * 2), ("azim", C.c_double * 2), ("zeta", C.c_double * 2),
                ("logT", C.c_double * 2), ("mask_colat", C.c_double * 2),
                ("mask_azim", C.c_double * 2), ("mask_zeta", C.c_double * 2),
                ("n_spots", C.c_int), ("oblate", C.c_int), ("emission", C.c_int),
                ("n_theta", C.c_int), ("n_phi", C.c_int), ("n_phase", C.c_int), ("n_fp", C.c_int),
                ("grid", C.c_int), ("phase_sub", C.c_int),
                ("logT_map", C.POINTER(C.c_double))]


def declare(L):
    """Set the ctypes signatures of an ordinary oracle build ``L`` (a CDLL);
    the tests use it on mutated copies of the oracle that check its pins."""
    d = C.c_double
    for name in ("orc_psi_out", "orc_td_out", "orc_rho", "orc_psi", "orc_td"):
        f = getattr(L, name)
        f.restype = d
        f.argtypes = [d, d]
    L.orc_lens_build.restype = C.c_int
    L.orc_lens_build.argtypes = [C.POINTER(LensSpecC), C.c_void_p, C.c_void_p, C.c_void_p]
    L.orc_lens_lookup.restype = C.c_int
    L.orc_lens_lookup.argtypes = [C.POINTER(LensC), d, d, C.POINTER(d), C.POINTER(d)]
    L.orc_td_lookup.restype = d
    L.orc_td_lookup.argtypes = [C.POINTER(LensC), d, d]
    L.orc_atm_interp.restype = d
    L.orc_atm_interp.argtypes = [C.POINTER(AtmC), d, d, d, d]
    L.orc_bb_intensity.restype = d
    L.orc_bb_intensity.argtypes = [d, d]
    L.orc_profile.restype = C.c_int
    L.orc_profile.argtypes = [C.POINTER(InstC), C.POINTER(LensC), C.POINTER(AtmC),
                              C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p,
                              C.c_int, C.c_int, C.c_void_p]
    L.orc_ring_template.restype = C.c_int
    L.orc_ring_template.argtypes = [C.POINTER(InstC), C.POINTER(LensC), C.c_int, C.c_int,
                                    C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    L.orc_counts.restype = None
    L.orc_counts.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_void_p,
                             d, C.c_void_p]
    L.orc_loglike.restype = d
    L.orc_loglike.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, d]
    return L


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = declare(C.CDLL(_LIB))
    return _lib


class _CD(C.Structure):
    """C99 double complex (real part, imaginary part)."""
    _fields_ = [("re", C.c_double), ("im", C.c_double)]


class InstT(C.Structure):
    """orc_inst of the tangent build: every real field is a complex pair."""
    _fields_ = [(n, (_CD * t._length_) if hasattr(t, "_length_") else _CD)
                if t is C.c_double or (hasattr(t, "_length_") and t._type_ is C.c_double)
                else (n, t) for n, t in InstC._fields_]


def lib_tangent():
    global _lib_t
    if _lib_t is None:
        build()
        L = C.CDLL(_LIB_T)
        L.orc_loglike_full.restype = C.c_int
        L.orc_loglike_full.argtypes = [C.POINTER(InstT), C.POINTER(LensC), C.POINTER(AtmC),
                                       C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p,
                                       C.c_void_p, C.c_void_p, C.c_double, C.c_void_p]
        _lib_t = L
    return _lib_t


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


# ---------------------------------------------------------------------------
# light bending (Sect. 2.3)
# ---------------------------------------------------------------------------
def psi(u: float, alpha: float) -> float:
    """Bending angle psi(u, alpha); inward rays via the periastron (Eq. rho)."""
    return lib().orc_psi(u, alpha)


def psi_out(u: float, alpha: float) -> float:
    """Eq. salmi_lf (outgoing rays)."""
    return lib().orc_psi_out(u, alpha)


def td(u: float, alpha: float) -> float:
    """c Delta t / R for any alpha (Eq. salmi_td; inward composition of Eq. tot_time_delay)."""
    return lib().orc_td(u, alpha)


def td_out(u: float, alpha: float) -> float:
    """c Delta t / R of an outgoing ray (Eq. salmi_td)."""
    return lib().orc_td_out(u, alpha)


def rho(u: float, alpha: float) -> float:
    """Periastron ratio R_p / R of Eq. rho (NaN when captured)."""
    return lib().orc_rho(u, alpha)


class Lens:
    """Lens tables built by the oracle (Sect. 2.8.2)."""

    def __init__(self, spec):
        self.spec = spec
        s = LensSpecC(spec.u_min, spec.u_max, spec.n_u, spec.cpsi_min, spec.cpsi_max,
                      spec.n_cpsi, spec.calpha_min, spec.calpha_max, spec.n_calpha, spec.dalpha)
        self.Ca = np.zeros((spec.n_u, spec.n_cpsi))
        self.LF = np.zeros((spec.n_u, spec.n_cpsi))
        self.TD = np.zeros((spec.n_u, spec.n_calpha))
        n = lib().orc_lens_build(C.byref(s), _ptr(self.Ca), _ptr(self.LF), _ptr(self.TD))
        if n < 0:
            raise ValueError("bad lens spec")
        self.march_len = n
        self.c = LensC(s, self.Ca.ctypes.data_as(C.POINTER(C.c_double)),
                       self.LF.ctypes.data_as(C.POINTER(C.c_double)),
                       self.TD.ctypes.data_as(C.POINTER(C.c_double)))

    def lookup(self, u, cpsi):
        ca, lf = C.c_double(), C.c_double()
        ok = lib().orc_lens_lookup(C.byref(self.c), u, cpsi, C.byref(ca), C.byref(lf))
        return (ca.value, lf.value) if ok else (math.nan, math.nan)

    def td_lookup(self, u, calpha):
        return lib().orc_td_lookup(C.byref(self.c), u, calpha)


_lens_cache = {}


def lens(spec) -> Lens:
    """The lens tables C_alpha, LF and TD of Sect. 2.8.2 (alpha march,
    numerical differentiation, resampling), cached per grid."""
    key = tuple(getattr(spec, f) for f in ("u_min", "u_max", "n_u", "cpsi_min", "cpsi_max",
                                           "n_cpsi", "calpha_min", "calpha_max", "n_calpha",
                                           "dalpha"))
    if key not in _lens_cache:
        _lens_cache[key] = Lens(spec)
    return _lens_cache[key]


# ---------------------------------------------------------------------------
# atmosphere (Sect. 4)
# ---------------------------------------------------------------------------
class Atm:
    def __init__(self, table, strategy: str = "d"):
        self.t = table
        self._arr = [np.ascontiguousarray(table.logT, dtype=np.float64),
                     np.ascontiguousarray(table.logg, dtype=np.float64),
                     np.ascontiguousarray(table.mu, dtype=np.float64),
                     np.ascontiguousarray(table.lnE, dtype=np.float64),
                     np.ascontiguousarray(table.I, dtype=np.float32)]
        a = self._arr
        dp = lambda x: x.ctypes.data_as(C.POINTER(C.c_double))
        self.c = AtmC(len(a[0]), len(a[1]), len(a[2]), len(a[3]), int(table.n_protect),
                      dp(a[0]), dp(a[1]), dp(a[2]), dp(a[3]),
                      a[4].ctypes.data_as(C.POINTER(C.c_float)), INTERP[strategy])

    def interp(self, logT, logg, mu, E_keV):
        return lib().orc_atm_interp(C.byref(self.c), logT, logg, mu, E_keV)


def bb_intensity(E_keV: float, kT_keV: float) -> float:
    """Blackbody specific intensity 2 E^3 / (h^3 c^2) / (e^{E/kT} - 1) (App. C)."""
    return lib().orc_bb_intensity(E_keV, kT_keV)


# ---------------------------------------------------------------------------
# forward model and likelihood
# ---------------------------------------------------------------------------
def inst_c(inst, b: int = 0) -> InstC:
    c = InstC()
    c.mass_msun = float(inst.mass_msun[b]); c.radius_km = float(inst.radius_km[b])
    c.spin_hz = float(inst.spin_hz[b]); c.incl_rad = float(inst.incl_rad[b])
    c.dist_kpc = float(inst.dist_kpc[b]); c.nh_1e20 = float(inst.nh_1e20[b])
    for name in ("colat", "azim", "zeta", "logT", "mask_colat", "mask_azim", "mask_zeta"):
        arr = getattr(c, name)
        v = getattr(inst, name)[b]
        for s in range(inst.n_spots):
            arr[s] = float(v[s])
    c.n_spots = inst.n_spots; c.oblate = inst.oblate; c.emission = inst.emission
    c.n_theta = int(inst.n_theta[b]); c.n_phi = int(inst.n_phi[b])
    c.n_phase = int(inst.n_phase[b]); c.n_fp = int(inst.n_fp)
    c.grid = int(getattr(inst, "grid", 0))
    c.phase_sub = int(getattr(inst, "phase_sub", 1))
    tmap = getattr(inst, "logT_map", None)
    if tmap is not None:
        arr = np.ascontiguousarray(tmap[b], dtype=np.float64)
        c._keep = arr   # the struct points into it
        c.logT_map = arr.ctypes.data_as(C.POINTER(C.c_double))
    return c


class OracleRangeError(RuntimeError):
    pass


def profile(w, b: int = 0, jsel: Optional[Sequence[int]] = None,
            ksel: Optional[Sequence[int]] = None, ring_stride: int = 1,
            lens_obj: Optional[Lens] = None, atm_obj: Optional[Atm] = None) -> np.ndarray:
    """F_t[j, k] (photons cm^-2 s^-1 keV^-1) of instance b of workload w:
    the shift-and-add of Sect. 2.8.3 (Eq. add_Ft) over the ring templates,
    with the flux of Sect. 2.5 / App. C and the atmosphere interpolation of
    Sect. 4.

    ``jsel``/``ksel`` restrict the output to selected phase/energy indices.
    """
    inst = w.inst
    L = lens_obj or lens(w.lens)
    A = atm_obj or (Atm(w.atm, getattr(w, "interp", "d")) if (inst.emission == 1) else None)
    E = np.ascontiguousarray(w.E_keV, dtype=np.float64)
    js = None if jsel is None else np.ascontiguousarray(jsel, dtype=np.int32)
    ks = None if ksel is None else np.ascontiguousarray(ksel, dtype=np.int32)
    nj = int(inst.n_phase[b]) if js is None else len(js)
    nk = len(E) if ks is None else len(ks)
    out = np.zeros((nj, nk))
    ic = inst_c(inst, b)
    st = lib().orc_profile(C.byref(ic), C.byref(L.c), C.byref(A.c) if A else None,
                           _ptr(E), len(E), _ptr(js), 0 if js is None else len(js),
                           _ptr(ks), 0 if ks is None else len(ks), ring_stride, _ptr(out))
    if st == 2:
        raise OracleRangeError("parameters outside the lens or atmosphere tables")
    if st != 0:
        raise ValueError("oracle rejected the instance (status %d)" % st)
    return out


def ring_template(w, spot: int, r: int, b: int = 0, lens_obj: Optional[Lens] = None):
    """Ring record and template arrays (F, z, phi_o, mu) of one ring: the
    star model of Sect. 2.1-2.2 and 2.4, the five template steps of Sect.
    2.8.3 and its invisible-segment fill."""
    inst = w.inst
    L = lens_obj or lens(w.lens)
    n = inst.n_fp + 1
    info = np.zeros(15)
    F, z, ph, mu = (np.zeros(n) for _ in range(4))
    ic = inst_c(inst, b)
    st = lib().orc_ring_template(C.byref(ic), C.byref(L.c), spot, r, _ptr(info),
                                 _ptr(F), _ptr(z), _ptr(ph), _ptr(mu))
    keys = ["theta", "dcos", "half", "R", "u", "f", "cos_eta", "sin_eta", "logg", "beta",
            "gamma", "dphi", "n_active", "status", "dt_obl"]
    return dict(zip(keys, info)), F, z, ph, mu


def counts_model(Ft: np.ndarray, R: np.ndarray, sigma: np.ndarray, nh_1e20: float) -> np.ndarray:
    """C = F_t diag(exp(-N_H sigma)) R, the count rate per phase and channel
    (ISM attenuation of Sect. 2.7, response of Sect. 2.8.4)."""
    Ft = np.ascontiguousarray(Ft, dtype=np.float64)
    R = np.ascontiguousarray(R, dtype=np.float32)
    sg = np.ascontiguousarray(sigma, dtype=np.float32)
    nP, nE = Ft.shape
    nc = R.shape[1]
    out = np.zeros((nP, nc))
    lib().orc_counts(_ptr(Ft), nP, nE, _ptr(R), nc, _ptr(sg), float(nh_1e20), _ptr(out))
    return out


def loglike(Cm: np.ndarray, d: np.ndarray, tau: float, bkg: Optional[np.ndarray] = None) -> float:
    """Poisson log-likelihood sum d ln(lam) - lam - lnGamma(d+1), lam = tau C + b
    (the likelihood whose chi^2 limit Sect. 5 uses and that Sect. 6
    accumulates on the GPU)."""
    Cm = np.ascontiguousarray(Cm, dtype=np.float64)
    d = np.ascontiguousarray(d, dtype=np.int32)
    bg = None if bkg is None else np.ascontiguousarray(bkg, dtype=np.float32)
    return lib().orc_loglike(_ptr(Cm), Cm.size, _ptr(d), _ptr(bg), float(tau))


# ---------------------------------------------------------------------------
# forward-mode derivatives (tangent build)
# ---------------------------------------------------------------------------
# differentiable parameters in the order of the GPU gradient
GRAD_PARAMS = (("mass_msun", None), ("radius_km", None), ("incl_rad", None),
               ("dist_kpc", None), ("nh_1e20", None),
               ("colat", 0), ("azim", 0), ("zeta", 0), ("logT", 0),
               ("colat", 1), ("azim", 1), ("zeta", 1), ("logT", 1))


def loglike_tangent(w, v, b: int = 0, h: float = 1e-20):
    """(logL, dlogL/dtheta . v) of instance b of w through the forward-mode
    build of the oracle; v has one entry per GRAD_PARAMS entry (13; the last
    four are ignored for one spot)."""
    inst = w.inst
    ic = InstT()
    base = inst_c(inst, b)
    for name, t in InstC._fields_:
        val = getattr(base, name)
        if t is C.c_double:
            getattr(ic, name).re = val
        elif hasattr(t, "_length_") and t._type_ is C.c_double:
            arr = getattr(ic, name)
            for s in range(len(arr)):
                arr[s].re = val[s]
        else:
            setattr(ic, name, val)
    for (name, s), vj in zip(GRAD_PARAMS, v):
        if s is None:
            getattr(ic, name).im = h * float(vj)
        elif s < inst.n_spots:
            getattr(ic, name)[s].im = h * float(vj)
    L = lens(w.lens)
    A = Atm(w.atm, getattr(w, "interp", "d")) if inst.emission == 1 else None
    E = np.ascontiguousarray(w.E_keV, dtype=np.float64)
    R = np.ascontiguousarray(w.R, dtype=np.float32)
    sg = np.ascontiguousarray(w.sigma_ism, dtype=np.float32)
    r0 = int(np.sum(inst.n_phase[:b]))
    d = np.ascontiguousarray(w.counts[r0:r0 + int(inst.n_phase[b])], dtype=np.int32)
    out = np.zeros(2)
    st = lib_tangent().orc_loglike_full(C.byref(ic), C.byref(L.c), C.byref(A.c) if A else None,
                                        _ptr(E), len(E), _ptr(R), R.shape[1], _ptr(sg),
                                        _ptr(d), None, float(w.tau), _ptr(out))
    if st == 2:
        raise OracleRangeError("parameters outside the lens or atmosphere tables")
    if st != 0:
        raise ValueError("oracle rejected the instance (status %d)" % st)
    return out[0], out[1] / h


def grad_tangent(w, b: int = 0):
    """Gradient of logL (GRAD_PARAMS order) by forward mode, one direction per
    parameter (the paper gives no derivative; this differentiates the same
    piecewise-smooth recipe, branches held fixed)."""
    n = 5 + 4 * w.inst.n_spots
    g = np.zeros(n)
    for j in range(n):
        e = np.zeros(13)
        e[j] = 1.0
        g[j] = loglike_tangent(w, e, b)[1]
    return g


# ---------------------------------------------------------------------------
# response down-sampling (Sect. 2.7, matrix DS)
# ---------------------------------------------------------------------------
def downsample_matrix(E_model, E_lo, E_hi) -> np.ndarray:
    """Down-sampling matrix DS of Sect. 2.7 (Eq. RSP).
    DS[i, e] = integral over detector bin e of the linear interpolant on
    E_model that is 1 at node i and 0 at the others (np.interp: constant
    beyond the ends).  Written from the definition: the bin is cut at every
    model node inside it, where the integrand is linear, and each piece is
    integrated exactly by its midpoint value."""
    Eo = np.asarray(E_model, dtype=np.float64)
    n = len(Eo)
    eye = np.eye(n)
    DS = np.zeros((n, len(E_lo)))
    for e, (a, b) in enumerate(zip(E_lo, E_hi)):
        cuts = np.unique(np.concatenate([[a, b], Eo[(Eo > a) & (Eo < b)]]))
        for x0, x1 in zip(cuts[:-1], cuts[1:]):
            mid = 0.5 * (x0 + x1)
            DS[:, e] += (x1 - x0) * np.array([np.interp(mid, Eo, eye[i]) for i in range(n)])
    return DS
