"""Seeded synthetic inputs for the pulse-profile likelihood.

This module only *generates data*: parameter vectors, grids, a synthetic
atmosphere table, a response matrix, ISM cross-sections and Poisson counts.
It holds none of the forward model's arithmetic (no light bending, no
template, no interpolation, no shift-and-add, no likelihood).  Both the
CUDA path and the FP64 CPU oracle consume exactly these arrays.

Workloads (sizes follow the paper's tiers, Table "tab:tiers", and its grid
ranges, Sect. 2.5 / 2.8):

* ``bb_small``          one circular spot, analytic isotropic blackbody,
                        S+D, 32x32 elements, 64 phases, 32 energies 0.2-3 keV.
* ``atm_two_spot``      a cap and a ring spot, synthetic 4-D atmosphere table,
                        OS, 128x128 elements per spot, 128 phases,
                        256 energies, ISM, 256x300 response, 1e6 counts.
* ``crescent_extreme``  crescent spot near the limb, u = 0.537, 512x512,
                        256 phases, 300 energies.
* ``batch``             B parameter vectors with mixed resolutions.
* ``grad_batch``        B two-cap vectors at 128x128, 128 phases.
* ``healpix_map``       whole-surface HEALPix mesh, N_side 52, with a
                        temperature map; the two-spot star and grids.

Every function takes explicit sizes so tests can build reduced versions of
the same workloads (several tiles plus a ragged tail).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

SEED = 2510

# Physical constants used only to fill the synthetic atmosphere table and to
# apply the compactness cut when drawing random stars (CODATA 2018, IAU 2015).
_H_KEV_S = 4.135667696e-18
_KB_KEV_K = 8.617333262e-8
_C_CM_S = 2.99792458e10
_GM_SUN = 1.32712440018e20
_C_M_S = 299792458.0

DEG = math.pi / 180.0


# --------------------------------------------------------------------------
# containers
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Instances:
    """Structure-of-arrays parameter vectors (length B; spots: [B, n_spots]).

    Units: mass in solar masses, equatorial radius in km, spin in Hz,
    inclination/colatitude/azimuth/angular radius in radians, distance in
    kpc, hydrogen column in 1e20 cm^-2, logT = log10(T_eff / K).
    ``mask_zeta <= 0`` means the spot has no masking cap.
    """
    mass_msun: np.ndarray
    radius_km: np.ndarray
    spin_hz: np.ndarray
    incl_rad: np.ndarray
    dist_kpc: np.ndarray
    nh_1e20: np.ndarray
    colat: np.ndarray
    azim: np.ndarray
    zeta: np.ndarray
    logT: np.ndarray
    mask_colat: np.ndarray
    mask_azim: np.ndarray
    mask_zeta: np.ndarray
    n_theta: np.ndarray
    n_phi: np.ndarray
    n_phase: np.ndarray
    n_spots: int
    oblate: int          # 0 = Schwarzschild+Doppler sphere, 1 = oblate Schwarzschild
    emission: int        # 0 = analytic isotropic blackbody, 1 = atmosphere table
    n_fp: int = 192
    grid: int = 0        # 0 = spot-bounding grid; 1 = HEALPix mesh with N_side = n_theta
    phase_sub: int = 1   # point samples per output phase bin (1, 2, 4, 8 or 16)
    logT_map: Optional[np.ndarray] = None  # [B, 12 N_side^2] log10 T per HEALPix pixel (grid 1)

    @property
    def B(self) -> int:
        return int(self.mass_msun.shape[0])

    def select(self, idx) -> "Instances":
        idx = np.atleast_1d(np.asarray(idx))
        kw = {}
        for f in dataclasses.fields(self):
            v = getattr(self, f.name)
            if isinstance(v, np.ndarray):
                kw[f.name] = np.ascontiguousarray(v[idx])
            else:
                kw[f.name] = v
        return Instances(**kw)

    def replace(self, **kw) -> "Instances":
        d = {f.name: getattr(self, f.name) for f in dataclasses.fields(self)}
        for k, v in kw.items():
            if isinstance(d[k], np.ndarray):
                v = np.array(np.broadcast_to(np.asarray(v, dtype=d[k].dtype), d[k].shape))
            d[k] = v
        return Instances(**d)

    def copy(self) -> "Instances":
        """Independent copy (arrays duplicated)."""
        d = {f.name: getattr(self, f.name) for f in dataclasses.fields(self)}
        return Instances(**{k: (np.array(v) if isinstance(v, np.ndarray) else v)
                            for k, v in d.items()})


@dataclasses.dataclass
class AtmTable:
    """4-D specific-intensity table I[logT][logg][mu][E] (float32, linear I).

    Axes: logT (uniform), logg (uniform), mu (clustered at both ends),
    lnE (uniform in ln E, E in keV).  ``n_protect`` small-mu nodes are the
    protected zone of the mixed-order interpolator (Sect. 4).
    """
    logT: np.ndarray
    logg: np.ndarray
    mu: np.ndarray
    lnE: np.ndarray
    I: np.ndarray
    n_protect: int = 4


@dataclasses.dataclass
class LensSpec:
    """Grids of the light-bending tables (Sect. 2.8.2, Eq. grids_def)."""
    u_min: float = 0.15
    u_max: float = 0.60
    n_u: int = 577
    cpsi_min: float = -0.995
    cpsi_max: float = 1.0
    n_cpsi: int = 1024
    calpha_min: float = -0.2
    calpha_max: float = 1.0
    n_calpha: int = 512
    dalpha: float = math.pi / 2048.0


@dataclasses.dataclass
class Workload:
    name: str
    inst: Instances
    lens: LensSpec
    E_keV: np.ndarray                      # model energy grid (float64)
    atm: Optional[AtmTable] = None
    R: Optional[np.ndarray] = None          # [nE, nc] float32 response (cm^2 keV)
    sigma_ism: Optional[np.ndarray] = None  # [nE] float32, cm^2
    counts: Optional[np.ndarray] = None     # [sum_b n_phase_b, nc] int32
    tau: float = 1.0                        # exposure scale: lambda = tau * C
    interp: str = "d"                       # atmosphere interpolation strategy (Sect. 4): d, a, b, c

    @property
    def nc(self) -> int:
        return 0 if self.R is None else int(self.R.shape[1])

    def rows(self) -> int:
        return int(np.sum(self.inst.n_phase))


# --------------------------------------------------------------------------
# grids
# --------------------------------------------------------------------------
def logspace(lo: float, hi: float, n: int) -> np.ndarray:
    """Logspace(lo, hi, n) of Sect. 2.8.4 (float64)."""
    i = np.arange(n, dtype=np.float64)
    if n == 1:
        return np.array([lo], dtype=np.float64)
    return np.exp(math.log(lo) + (math.log(hi) - math.log(lo)) * i / (n - 1))


def mu_nodes(n: int = 67, mu_min: float = 1e-6) -> np.ndarray:
    """mu nodes clustered at both ends: mu_m = mu_min + (1-mu_min)(1-cos(pi m/(n-1)))/2."""
    m = np.arange(n, dtype=np.float64)
    return mu_min + (1.0 - mu_min) * (1.0 - np.cos(math.pi * m / (n - 1))) / 2.0


# --------------------------------------------------------------------------
# atmosphere table
# --------------------------------------------------------------------------
def atm_table(n_T: int = 35, n_g: int = 11, n_mu: int = 67, n_E: int = 166,
              seed: int = SEED, steep_limb_mu0: float = 0.0) -> AtmTable:
    """Synthetic NSX-shaped table: blackbody x limb darkening x smooth +-5 %.

    I = B_E(E, T) (1 + a mu + b mu^2) (1 + 0.05 p), with
    a = 0.6 - 0.2 (logT - 6) + 0.1 (logg - 14.2), b = -0.25 + 0.05 (logT - 6),
    p a seeded sum of 8 separable low-frequency cosines scaled to max|p| = 1.
    Values below the float32 normal range are flushed to zero.

    steep_limb_mu0 > 0 multiplies I by (1 - exp(-mu / mu0)): a limb drop over
    the first few mu nodes, the kind of small-mu curvature that makes cubic
    stencils overshoot (a variant for the interpolation tests of Sect. 4; the
    default table has none).
    """
    logT = np.linspace(5.1, 6.8, n_T)
    logg = np.linspace(13.7, 14.7, n_g)
    mu = mu_nodes(n_mu)
    lnE = np.linspace(math.log(0.05), math.log(10.0), n_E)
    E = np.exp(lnE)

    T4, G4, M4, E4 = np.meshgrid(logT, logg, mu, E, indexing="ij")
    kT = _KB_KEV_K * 10.0 ** T4
    x = E4 / kT
    with np.errstate(over="ignore"):
        bb = 2.0 * E4 ** 3 / (_H_KEV_S ** 3 * _C_CM_S ** 2) / np.expm1(x)
    a = 0.6 - 0.2 * (T4 - 6.0) + 0.1 * (G4 - 14.2)
    b = -0.25 + 0.05 * (T4 - 6.0)
    limb = 1.0 + a * M4 + b * M4 ** 2

    rng = np.random.Generator(np.random.PCG64(seed))
    # normalised coordinates in [0, 1]
    xs = [(T4 - logT[0]) / (logT[-1] - logT[0]),
          (G4 - logg[0]) / (logg[-1] - logg[0]),
          M4,
          (np.log(E4) - lnE[0]) / (lnE[-1] - lnE[0])]
    p = np.zeros_like(T4)
    for _ in range(8):
        term = rng.uniform(-1.0, 1.0)
        for ax in range(4):
            k = rng.uniform(0.3, 2.0) * math.pi
            ph = rng.uniform(0.0, 2.0 * math.pi)
            term = term * np.cos(k * xs[ax] + ph)
        p = p + term
    p = p / np.max(np.abs(p))

    I = bb * limb * (1.0 + 0.05 * p)
    if steep_limb_mu0 > 0.0:
        I = I * -np.expm1(-M4 / steep_limb_mu0)
    I = np.where(np.isfinite(I), I, 0.0)
    I32 = I.astype(np.float32)
    I32[np.abs(I32) < np.finfo(np.float32).tiny] = 0.0
    return AtmTable(logT=logT, logg=logg, mu=mu, lnE=lnE,
                    I=np.ascontiguousarray(I32), n_protect=4)


# --------------------------------------------------------------------------
# ISM cross-section, response, counts
# --------------------------------------------------------------------------
def sigma_ism(E_keV: np.ndarray, sigma0: float = 2.0e-22) -> np.ndarray:
    """Synthetic photo-absorption cross-section sigma0 (E / 1 keV)^-2.5 (cm^2)."""
    return (sigma0 * (np.asarray(E_keV, dtype=np.float64) ** -2.5)).astype(np.float32)


def response(E_keV: np.ndarray, n_chan: int, fwhm_keV: float = 0.1) -> np.ndarray:
    """Dense response R[k, c] (cm^2 keV) on the model energy grid.

    R[k, c] = A(E_k) * w_k * P(c | E_k): a Gaussian redistribution of FWHM
    ``fwhm_keV`` integrated over ``n_chan`` uniform channels spanning the
    grid, a smooth effective area A(E) = 1500 cm^2 exp(-ln(E/1.5)^2 / 0.98)
    and the trapezoid width w_k of model energy k (so C = F_t diag(ATT) R is
    a count rate).
    """
    from scipy.special import erf
    E = np.asarray(E_keV, dtype=np.float64)
    n = E.shape[0]
    edges = np.linspace(E[0], E[-1], n_chan + 1)
    s = fwhm_keV / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    cdf = 0.5 * (1.0 + erf((edges[None, :] - E[:, None]) / (math.sqrt(2.0) * s)))
    P = np.diff(cdf, axis=1)
    A = 1500.0 * np.exp(-(np.log(E / 1.5)) ** 2 / (2.0 * 0.7 ** 2))
    w = np.empty(n)
    if n == 1:
        w[:] = 1.0
    else:
        w[0] = 0.5 * (E[1] - E[0])
        w[-1] = 0.5 * (E[-1] - E[-2])
        w[1:-1] = 0.5 * (E[2:] - E[:-2])
    return np.ascontiguousarray((A[:, None] * w[:, None] * P).astype(np.float32))


def counts(n_phase: np.ndarray, n_chan: int, total: float = 1.0e6,
           seed: int = SEED) -> np.ndarray:
    """Poisson counts for every instance: [sum_b n_phase_b, n_chan] int32.

    Each instance's mean map is a smooth pulsed shape (a fundamental plus a
    harmonic in phase times a broad bump in channel) scaled to ``total``
    expected counts, drawn with PCG64(seed).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    c = np.arange(n_chan) / max(n_chan - 1, 1)
    spec = np.exp(-0.5 * ((c - 0.25) / 0.15) ** 2) + 0.05
    for npb in np.asarray(n_phase):
        j = np.arange(int(npb)) / int(npb)
        pulse = 1.0 + 0.4 * np.cos(2 * math.pi * (j - 0.1)) + 0.1 * np.cos(4 * math.pi * (j - 0.3))
        lam = pulse[:, None] * spec[None, :]
        lam = lam * (total / lam.sum())
        out.append(rng.poisson(lam).astype(np.int32))
    return np.ascontiguousarray(np.concatenate(out, axis=0))


# --------------------------------------------------------------------------
# parameter vectors
# --------------------------------------------------------------------------
def _instances(B: int, n_spots: int, **kw) -> Instances:
    z = lambda: np.zeros(B, dtype=np.float64)
    zs = lambda: np.zeros((B, n_spots), dtype=np.float64)
    d = dict(mass_msun=z(), radius_km=z(), spin_hz=z(), incl_rad=z(),
             dist_kpc=z(), nh_1e20=z(), colat=zs(), azim=zs(), zeta=zs(),
             logT=zs(), mask_colat=zs(), mask_azim=zs(), mask_zeta=zs(),
             n_theta=np.zeros(B, dtype=np.int32), n_phi=np.zeros(B, dtype=np.int32),
             n_phase=np.zeros(B, dtype=np.int32), n_spots=n_spots, oblate=1,
             emission=1, n_fp=192)
    inst = Instances(**d)
    return inst.replace(**kw) if kw else inst


def bb_small(n_theta: int = 32, n_phi: int = 32, n_phase: int = 64, n_E: int = 32,
             lens: Optional[LensSpec] = None) -> Workload:
    """Plain method, small: one cap, analytic blackbody, S+D."""
    inst = _instances(1, 1, mass_msun=1.4, radius_km=12.0, spin_hz=205.0,
                      incl_rad=60 * DEG, dist_kpc=0.3, nh_1e20=1.0,
                      colat=45 * DEG, azim=0.0, zeta=0.2, logT=6.1,
                      mask_zeta=0.0, n_theta=n_theta, n_phi=n_phi, n_phase=n_phase)
    inst.oblate = 0
    inst.emission = 0
    return Workload("bb_small", inst, lens or LensSpec(), logspace(0.2, 3.0, n_E))


def _with_response(w: Workload, n_chan: int, total: float = 1.0e6, tau: float = 1.0) -> Workload:
    w.R = response(w.E_keV, n_chan)
    w.sigma_ism = sigma_ism(w.E_keV)
    w.counts = counts(w.inst.n_phase, n_chan, total=total)
    w.tau = tau
    return w


# Exposure scale for the two-spot workload: with this tau the truth
# parameters give ~1e6 expected counts (set from a one-off oracle run).
TAU_TWO_SPOT = 1.0e3


def atm_two_spot(n_theta: int = 128, n_phi: int = 128, n_phase: int = 128,
                 n_E: int = 256, n_chan: int = 300, atm: Optional[AtmTable] = None,
                 lens: Optional[LensSpec] = None) -> Workload:
    """Two hotspots (a cap and a concentric ring) with the atmosphere table, OS."""
    inst = _instances(1, 2, mass_msun=1.4, radius_km=12.0, spin_hz=205.0,
                      incl_rad=60 * DEG, dist_kpc=0.3, nh_1e20=1.0,
                      n_theta=n_theta, n_phi=n_phi, n_phase=n_phase)
    inst.colat[0] = [45 * DEG, 120 * DEG]
    inst.azim[0] = [0.0, math.pi]
    inst.zeta[0] = [0.2, 0.25]
    inst.logT[0] = [6.1, 6.0]
    inst.mask_colat[0] = [0.0, 120 * DEG]
    inst.mask_azim[0] = [0.0, math.pi]
    inst.mask_zeta[0] = [0.0, 0.12]
    w = Workload("atm_two_spot", inst, lens or LensSpec(), logspace(0.1, 5.215, n_E),
                 atm=atm if atm is not None else atm_table())
    return _with_response(w, n_chan, tau=TAU_TWO_SPOT)


# Spot-centre colatitude for the crescent workload: the far side of the
# spot passes 5 degrees inside the visible limb psi_limb(u = 0.537) = 165.5 deg
# seen at i = 85 deg, i.e. 165.5 - 5 - 85 = 75.5 deg.
CRESCENT_COLAT = 75.5 * DEG


def crescent_extreme(n_theta: int = 512, n_phi: int = 512, n_phase: int = 256,
                     n_E: int = 300, n_chan: int = 300, atm: Optional[AtmTable] = None,
                     lens: Optional[LensSpec] = None) -> Workload:
    """Crescent (emitter 0.05 rad minus a 0.035 rad mask offset 0.02 rad poleward)."""
    inst = _instances(1, 1, mass_msun=2.0, radius_km=11.0, spin_hz=346.0,
                      incl_rad=85 * DEG, dist_kpc=0.3, nh_1e20=1.0,
                      colat=CRESCENT_COLAT, azim=0.0, zeta=0.05, logT=6.78,
                      mask_colat=CRESCENT_COLAT - 0.02, mask_azim=0.0, mask_zeta=0.035,
                      n_theta=n_theta, n_phi=n_phi, n_phase=n_phase)
    w = Workload("crescent_extreme", inst, lens or LensSpec(), logspace(0.1, 5.215, n_E),
                 atm=atm if atm is not None else atm_table())
    return _with_response(w, n_chan, tau=TAU_TWO_SPOT)


def interp_test(case: int = 1, n: int = 32, n_phase: int = 64, n_E: int = 128,
                atm: Optional[AtmTable] = None, lens: Optional[LensSpec] = None,
                strategy: str = "d") -> Workload:
    """The two atmosphere-interpolation tests of Sect. 4 (table tab:interp):
    one point-like spot (zeta = 0.01) seen close to the limb so that many rays
    have mu -> 0.  Test 1: spot colatitude 1.983, inclination 0.01; test 2:
    spot at pi - 0.01, inclination 0.964.  M = 1.4, R_e = 12 km, 600 Hz,
    T = 1e6 K, D = 150 pc."""
    th, inc = (1.983, 0.01) if case == 1 else (math.pi - 0.01, 0.964)
    inst = _instances(1, 1, mass_msun=1.4, radius_km=12.0, spin_hz=600.0, incl_rad=inc,
                      dist_kpc=0.15, nh_1e20=1.0, colat=th, azim=0.0, zeta=0.01, logT=6.0,
                      mask_zeta=0.0, n_theta=n, n_phi=n, n_phase=n_phase)
    return Workload("interp_test_%d" % case, inst, lens or LensSpec(),
                    logspace(0.1, 5.215, n_E), atm=atm if atm is not None else atm_table(),
                    interp=strategy)


def _compactness(mass_msun, radius_km):
    return 2.0 * _GM_SUN * np.asarray(mass_msun) / _C_M_S ** 2 / (np.asarray(radius_km) * 1e3)


def random_instances(B: int, seed: int = SEED, res_theta=(64, 128, 256),
                     res_phase=(32, 64, 128), u_max: float = 0.55,
                     mask: bool = False) -> Instances:
    """B two-cap stars drawn uniformly (M 1-2.5, R 9-15 km, rejection to u <= u_max,
    i 5-90 deg, colatitudes 0-180 deg, radii 0.01-1 rad, logT 5.8-6.6),
    spin 300 Hz, D = 0.2 kpc, N_H = 1e20, OS, atmosphere table; per-instance
    element grid (n x n with n from ``res_theta``) and phase count from ``res_phase``.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    M = np.empty(B)
    R = np.empty(B)
    k = 0
    while k < B:
        m = rng.uniform(1.0, 2.5)
        r = rng.uniform(9.0, 15.0)
        if _compactness(m, r) <= u_max:
            M[k], R[k] = m, r
            k += 1
    inst = _instances(B, 2, mass_msun=M, radius_km=R, spin_hz=300.0,
                      dist_kpc=0.2, nh_1e20=1.0)
    inst.incl_rad[:] = rng.uniform(5 * DEG, 90 * DEG, B)
    inst.colat[:] = rng.uniform(0.0, math.pi, (B, 2))
    inst.azim[:, 0] = 0.0
    inst.azim[:, 1] = rng.uniform(0.0, 2 * math.pi, B)
    inst.zeta[:] = rng.uniform(0.01, 1.0, (B, 2))
    inst.logT[:] = rng.uniform(5.8, 6.6, (B, 2))
    if mask:
        inst.mask_colat[:] = inst.colat
        inst.mask_azim[:] = inst.azim
        inst.mask_zeta[:] = 0.5 * inst.zeta
    n = rng.choice(np.asarray(res_theta), B)
    inst.n_theta[:] = n
    inst.n_phi[:] = n
    inst.n_phase[:] = rng.choice(np.asarray(res_phase), B)
    return inst


def batch(B: int = 4096, n_E: int = 256, n_chan: int = 300, seed: int = SEED,
          atm: Optional[AtmTable] = None, lens: Optional[LensSpec] = None,
          **kw) -> Workload:
    """Batched workload: B random two-cap vectors with mixed resolutions."""
    inst = random_instances(B, seed=seed, **kw)
    w = Workload("batch", inst, lens or LensSpec(), logspace(0.1, 5.215, n_E),
                 atm=atm if atm is not None else atm_table())
    return _with_response(w, n_chan, tau=TAU_TWO_SPOT)


def grad_batch(B: int = 1024, n_res: int = 128, n_phase: int = 128, n_E: int = 256,
               n_chan: int = 300, seed: int = SEED + 1,
               atm: Optional[AtmTable] = None, lens: Optional[LensSpec] = None) -> Workload:
    """Differentiated workload: B two-cap vectors at n_res x n_res, fixed phases."""
    inst = random_instances(B, seed=seed, res_theta=(n_res,), res_phase=(n_phase,))
    w = Workload("grad_batch", inst, lens or LensSpec(), logspace(0.1, 5.215, n_E),
                 atm=atm if atm is not None else atm_table())
    return _with_response(w, n_chan, tau=TAU_TWO_SPOT)


def healpix_map(n_side: int = 52, n_phase: int = 128, n_E: int = 256, n_chan: int = 300,
                atm: Optional[AtmTable] = None, lens: Optional[LensSpec] = None,
                seed: int = SEED) -> Workload:
    """Whole-surface HEALPix mesh (Sect. 2.6) with a temperature map: N_side
    = 52 gives 12 N^2 = 32,448 pixels, about the two-spot workload's 32,768
    elements.  The map (ring order) is warm, log T 5.95-6.2 with a seeded
    ripple, on two pixel ranges (15 % and 10 % of the surface) and dark
    elsewhere (log T -1: no emission).  The two-spot star, atmosphere table,
    phases, energies and response."""
    inst = _instances(1, 1, mass_msun=1.4, radius_km=12.0, spin_hz=205.0,
                      incl_rad=60 * DEG, dist_kpc=0.3, nh_1e20=1.0,
                      colat=0.0, azim=0.0, zeta=math.pi, logT=6.0, mask_zeta=0.0,
                      n_theta=n_side, n_phi=4 * n_side, n_phase=n_phase)
    inst.grid = 1
    npix = 12 * n_side * n_side
    rng = np.random.Generator(np.random.PCG64(seed))
    k = np.arange(npix)
    lt = 6.075 + 0.125 * np.sin(2 * math.pi * 7.0 * k / npix + rng.uniform(0, 2 * math.pi))
    warm = ((k >= int(0.20 * npix)) & (k < int(0.35 * npix))) | \
           ((k >= int(0.60 * npix)) & (k < int(0.70 * npix)))
    inst.logT_map = np.where(warm, lt, -1.0)[None, :]
    w = Workload("healpix_map", inst, lens or LensSpec(), logspace(0.1, 5.215, n_E),
                 atm=atm if atm is not None else atm_table())
    return _with_response(w, n_chan, tau=TAU_TWO_SPOT)


WORKLOADS = {
    "bb_small": bb_small,
    "atm_two_spot": atm_two_spot,
    "crescent_extreme": crescent_extreme,
    "batch": batch,
    "grad_batch": grad_batch,
    "healpix_map": healpix_map,
}
