"""Pins of the oracle's forward model against what the physics fixes.

* closed form: a uniformly emitting non-rotating blackbody star gives
  F(E) = pi (R_inf/D)^2 I_{T_inf}(E) / E with R_inf = R/sqrt(1-u),
  T_inf = T sqrt(1-u) (App. C flux formula integrated over the visible
  sphere, int cos(alpha) dcos(alpha) dlambda = pi), for the analytic
  blackbody and for a tabulated isotropic blackbody;
* exact symmetries: i = 0 gives a phase-constant profile; the mirror
  (theta_c, i) -> (pi - theta_c, pi - i); the antipodal spot rolls the profile
  by half a cycle; an azimuth shift of 2 pi k / N rolls it by -k bins
  (a spot at larger longitude crosses the observer's meridian earlier);
  F scales as D^-2;
* flat space (u -> 0): the per-ring template against photon counting with
  explicit Lorentz boosts, and a single small spot's light curve against a
  direct time-domain simulation.
"""
import math

import numpy as np
import pytest

GM_SUN = 1.32712440018e20
C_MS = 299792458.0
KPC = 3.0856775814913673e19
KB = 8.617333262e-8
H = 4.135667696e-18
C_CMS = 29979245800.0


def planck_photon(E, kT):
    """B_E / E written out here (photons cm^-2 s^-1 keV^-1 sr^-1)."""
    return 2.0 * E ** 2 / (H ** 3 * C_CMS ** 2) / np.expm1(E / kT)


def whole_star(synth, N, n_fp, n_cpsi, emission=0, atm=None):
    lens = synth.LensSpec(u_min=0.34, u_max=0.35, n_u=3, n_cpsi=n_cpsi)
    w = synth.bb_small(n_theta=N, n_phi=N, n_phase=4, n_E=6, lens=lens)
    w.inst.colat[:] = 0.0
    w.inst.zeta[:] = math.pi
    w.inst.spin_hz[:] = 0.0
    w.inst.n_fp = n_fp
    w.inst.emission = emission
    w.atm = atm
    return w


def closed_form(w):
    M, R = w.inst.mass_msun[0], w.inst.radius_km[0] * 1e3
    u = 2 * GM_SUN * M / C_MS ** 2 / R
    D = w.inst.dist_kpc[0] * KPC
    kT_inf = KB * 10 ** w.inst.logT[0, 0] * math.sqrt(1 - u)
    return math.pi * (R / math.sqrt(1 - u) / D) ** 2 * planck_photon(w.E_keV, kT_inf)


def test_closed_form_blackbody_star(orc, synth):
    errs = []
    for N, nfp, ncp in [(64, 192, 512), (256, 384, 2048)]:
        w = whole_star(synth, N, nfp, ncp)
        F = orc.profile(w)
        ref = closed_form(w)[None, :]
        errs.append(np.max(np.abs(F / ref - 1)))
        # phase independent
        assert np.allclose(F, F[0:1], rtol=1e-12)
    assert errs[1] < 2e-6
    assert errs[1] < errs[0] / 4   # second-order convergence in the surface grid


def test_closed_form_tabulated_isotropic_blackbody(orc, synth):
    """Same closed form through the atmosphere-table path (isotropic blackbody
    table on the NSX-shaped axes; logT = 6.1 is a node)."""
    t = synth.atm_table(n_T=35, n_g=11, n_mu=67, n_E=166)
    E = np.exp(t.lnE)
    kT = KB * 10 ** t.logT
    with np.errstate(over="ignore"):
        bb = 2.0 * E[None, :] ** 3 / (H ** 3 * C_CMS ** 2) / np.expm1(E[None, :] / kT[:, None])
    I = np.broadcast_to(bb[:, None, None, :], t.I.shape).astype(np.float32)
    t.I = np.ascontiguousarray(I)
    w = whole_star(synth, 256, 384, 2048, emission=1, atm=t)
    F = orc.profile(w)
    ref = closed_form(w)[None, :]
    # cubic interpolation of linear intensity: the Wien tail (flux < 1e-3 of the
    # peak) carries the method's own interpolation error, excluded as in Sect. 5
    keep = ref[0] >= 1e-3 * ref.max()
    assert keep.sum() >= 3
    assert np.max(np.abs(F[:, keep] / ref[:, keep] - 1)) < 5e-5


def _two_spot(synth, atm, lens, **kw):
    w = synth.atm_two_spot(n_theta=12, n_phi=16, n_phase=32, n_E=12, n_chan=8, atm=atm,
                           lens=lens)
    w.inst = w.inst.replace(**kw)
    return w


def test_phase_constant_at_zero_inclination(orc, synth, atm, small_lens):
    w = _two_spot(synth, atm, small_lens, incl_rad=0.0)
    F = orc.profile(w)
    assert F.max() > 0
    assert np.max(np.abs(F - F[0:1]) / F.max()) < 1e-12


def test_mirror_symmetry(orc, synth, atm, small_lens):
    w = _two_spot(synth, atm, small_lens, incl_rad=1.1)
    F = orc.profile(w)
    m = w.inst.copy()
    m.colat[:] = math.pi - m.colat
    m.mask_colat[:] = math.pi - m.mask_colat
    m.incl_rad[:] = math.pi - m.incl_rad
    w2 = _two_spot(synth, atm, small_lens)
    w2.inst = m
    F2 = orc.profile(w2)
    assert np.max(np.abs(F2 - F)) / F.max() < 1e-11


def test_antipodal_spot_rolls_half_cycle(orc, synth, atm, small_lens):
    w = _two_spot(synth, atm, small_lens, incl_rad=1.1)
    F = orc.profile(w)
    a = w.inst.copy()
    a.colat[:] = math.pi - a.colat
    a.mask_colat[:] = math.pi - a.mask_colat
    a.azim[:] = a.azim + math.pi
    a.mask_azim[:] = a.mask_azim + math.pi
    a.incl_rad[:] = math.pi - a.incl_rad
    w2 = _two_spot(synth, atm, small_lens)
    w2.inst = a
    F2 = orc.profile(w2)
    n = F.shape[0]
    assert np.max(np.abs(np.roll(F, n // 2, axis=0) - F2)) / F.max() < 1e-11


def test_azimuth_shift_rolls_profile(orc, synth, atm, small_lens):
    w = _two_spot(synth, atm, small_lens, incl_rad=1.1)
    F = orc.profile(w)
    n = F.shape[0]
    k = 3
    a = w.inst.copy()
    a.azim[:] = a.azim + 2 * math.pi * k / n
    a.mask_azim[:] = a.mask_azim + 2 * math.pi * k / n
    w2 = _two_spot(synth, atm, small_lens)
    w2.inst = a
    F2 = orc.profile(w2)
    assert np.max(np.abs(np.roll(F, -k, axis=0) - F2)) / F.max() < 1e-11
    assert np.max(np.abs(np.roll(F, k, axis=0) - F2)) / F.max() > 1e-3


def test_distance_scaling(orc, synth, atm, small_lens):
    w = _two_spot(synth, atm, small_lens, incl_rad=1.1)
    F = orc.profile(w)
    w.inst.dist_kpc[:] = 2.5 * w.inst.dist_kpc
    F2 = orc.profile(w)
    assert np.allclose(F2 * 2.5 ** 2, F, rtol=1e-13, atol=0)


# ---------------------------------------------------------------------------
# flat space: independent special-relativistic photon counting
# ---------------------------------------------------------------------------
def _flat_workload(synth, nu=600.0, incl=1.2, colat=1.0, n_fp=192):
    u = 1e-7
    R = 12.0
    M = u * R * 1e3 * C_MS ** 2 / (2 * GM_SUN)
    lens = synth.LensSpec(u_min=0.0, u_max=2e-7, n_u=2, n_cpsi=4096)
    w = synth.bb_small(n_theta=4, n_phi=4, n_phase=64, n_E=8, lens=lens)
    w.inst = w.inst.replace(mass_msun=M, spin_hz=nu, incl_rad=incl, colat=colat, zeta=0.05)
    w.inst.n_fp = n_fp
    return w


def _boosted(theta, phi, incl, beta):
    """Photon toward the observer, lab direction k = (sin i, 0, cos i); surface
    velocity beta along phi-hat.  Returns (cos psi, delta, cos sigma')."""
    r = np.array([math.sin(theta) * math.cos(phi), math.sin(theta) * math.sin(phi), math.cos(theta)])
    k = np.array([math.sin(incl), 0.0, math.cos(incl)])
    v = beta * np.array([-math.sin(phi), math.cos(phi), 0.0])
    g = 1.0 / math.sqrt(1.0 - beta * beta)
    # boost of the photon 4-momentum (1, k): comoving energy and normal component
    E_co = g * (1.0 - v @ k)
    kn_co = k @ r                 # the normal r is perpendicular to the boost
    return k @ r, 1.0 / E_co, kn_co / E_co


def test_flat_space_template_matches_lorentz_boost(orc, synth):
    """Per element: N = delta^3 cos(sigma') dS_co I'/E / D^2 photons per unit
    observer time (dN = dN', dOmega' = delta^2 dOmega, dE' = dE/delta,
    proper time = delta x arrival time), comoving area dS_co = gamma dS_lab."""
    w = _flat_workload(synth)
    inst = w.inst
    R = inst.radius_km[0] * 1e3
    D = inst.dist_kpc[0] * KPC
    info, F, z, ph, mu = orc.ring_template(w, 0, 1)
    theta, dcos, dphi = info["theta"], info["dcos"], info["dphi"]
    beta = 2 * math.pi * inst.spin_hz[0] * R * math.sin(theta) / C_MS
    g = 1 / math.sqrt(1 - beta ** 2)
    n_fp = inst.n_fp
    nvis = 0
    for i in range(n_fp):
        phi = 2 * math.pi * i / n_fp
        cpsi, delta, cs_co = _boosted(theta, phi, inst.incl_rad[0], beta)
        if cpsi <= 1e-3:
            continue
        nvis += 1
        F_unit = delta ** 3 * g * R * R * dcos * dphi / D ** 2
        F_ref = F_unit * cs_co
        # residual bending at u = 1e-7 moves cos(alpha) by ~1e-7 near the limb
        assert F[i] == pytest.approx(F_ref, rel=2e-6, abs=3e-7 * F_unit)
        assert z[i] == pytest.approx(1 / delta, rel=2e-7)   # u = 1e-7 redshift
        assert mu[i] == pytest.approx(cs_co, rel=2e-6, abs=3e-7)
        # arrival delay relative to the sub-observer point: R (1 - cos psi) / c
        assert ph[i] == pytest.approx(i / n_fp + inst.spin_hz[0] * R * (1 - cpsi) / C_MS, abs=1e-9)
    assert nvis > 20


def test_flat_space_light_curve_time_domain(orc, synth):
    """A single element's light curve (one ring, one element) against a direct
    time-domain simulation: step the rotation finely, place each emission at its
    arrival phase, interpolate onto the output phases."""
    w = _flat_workload(synth, nu=500.0, incl=1.3, colat=1.2, n_fp=2048)
    w.inst = w.inst.replace(n_theta=1, n_phi=1, zeta=1e-3)
    inst = w.inst
    F = orc.profile(w)
    info, *_ = orc.ring_template(w, 0, 0)
    R = inst.radius_km[0] * 1e3
    D = inst.dist_kpc[0] * KPC
    nu = inst.spin_hz[0]
    theta, dcos, dphi = info["theta"], info["dcos"], info["dphi"]
    beta = 2 * math.pi * nu * R * math.sin(theta) / C_MS
    g = 1 / math.sqrt(1 - beta ** 2)
    kT = KB * 10 ** inst.logT[0, 0]
    Phi = np.linspace(0.0, 1.0, 20001)
    arr, flux = [], []
    for P in Phi:
        phi = inst.azim[0, 0] + 2 * math.pi * P     # rotation increases the azimuth
        cpsi, delta, cs_co = _boosted(theta, phi, inst.incl_rad[0], beta)
        arr.append(P + nu * R * (1 - cpsi) / C_MS)
        Ep = w.E_keV / delta
        flux.append(max(cs_co, 0.0) * delta ** 3 * g * R * R * dcos * dphi / D ** 2 *
                    2 * Ep ** 3 / (H ** 3 * C_CMS ** 2) / np.expm1(Ep / kT) / w.E_keV)
    arr = np.array(arr)
    flux = np.array(flux)
    out = np.arange(F.shape[0]) / F.shape[0]
    ref = np.empty_like(F)
    for k in range(F.shape[1]):
        ext_a = np.concatenate([arr - 1, arr, arr + 1])
        ext_f = np.concatenate([flux[:, k]] * 3)
        ref[:, k] = np.interp(out, ext_a, ext_f)
    scale = ref.max(axis=0)
    assert np.max(np.abs(F - ref) / scale) < 1e-5


@pytest.mark.parametrize("S", [2, 4])
def test_phase_sub_samples_are_azimuth_shifted_point_samples(orc, synth, atm, small_lens, S):
    """A phase bin with S sub-samples at offsets ((q + 1/2)/S - 1/2)/N is the
    mean of S point-sample profiles whose spots (and masks) are turned by
    2 pi times those offsets: the element grid moves with the azimuth."""
    w = synth.atm_two_spot(n_theta=8, n_phi=12, n_phase=16, n_E=10, n_chan=4, atm=atm,
                           lens=small_lens)
    w.inst.phase_sub = S
    F = orc.profile(w)
    N = int(w.inst.n_phase[0])
    acc = np.zeros_like(F)
    for q in range(S):
        d = 2 * math.pi * ((q + 0.5) / S - 0.5) / N
        v = _two_spot(synth, atm, small_lens)
        v.inst.n_phi[:] = 12
        v.inst.n_theta[:] = 8
        v.inst.n_phase[:] = 16
        v.E_keV = w.E_keV
        v.inst.azim[:] = w.inst.azim + d
        v.inst.mask_azim[:] = w.inst.mask_azim + d
        acc += orc.profile(v)
    np.testing.assert_allclose(F, acc / S, rtol=1e-9, atol=1e-12 * np.abs(F).max())
