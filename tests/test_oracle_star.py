"""Pins of the oracle's star model (Sect. 2.1-2.2, 2.4: Eqs. Rtheta, def_f,
Omega_c_def and the g(theta) fit) by invariants that do not restate its
coefficients: equatorial symmetry, flattening toward the poles, the slope f
against a numerical derivative of the oracle's own R(theta), gravity larger
at the pole than at the equator, the spherical, non-rotating limits, and
the oblate delay (Eq. delta_t_oblate) as the coordinate time of a radial
photon (Schwarzschild) from R(theta) out to R_e."""
import math

import numpy as np
import pytest


def _star(synth, spin_hz, oblate=1, colat=math.pi / 2, zeta=math.pi / 2, n_theta=64):
    inst = synth._instances(1, 1, mass_msun=1.4, radius_km=12.0, spin_hz=spin_hz,
                            incl_rad=1.0, dist_kpc=0.3, nh_1e20=1.0, colat=colat, azim=0.0,
                            zeta=zeta, logT=6.1, mask_zeta=0.0, n_theta=n_theta, n_phi=8,
                            n_phase=8)
    inst.oblate = oblate
    inst.emission = 0
    return inst


def _rings(orc, synth, inst, lens):
    w = synth.Workload("star", inst, lens, synth.logspace(0.5, 2.0, 4))
    recs = [orc.ring_template(w, 0, r)[0] for r in range(int(inst.n_theta[0]))]
    return {k: np.array([rec[k] for rec in recs]) for k in ("theta", "R", "u", "f", "logg",
                                                           "beta", "dt_obl")}


@pytest.fixture(scope="module")
def wide_lens(synth):
    return synth.LensSpec(u_min=0.25, u_max=0.45, n_u=65, n_cpsi=256, n_calpha=128)


def test_oblate_star_is_symmetric_about_the_equator(orc, synth, wide_lens):
    g = _rings(orc, synth, _star(synth, 600.0), wide_lens)
    # rings r and n-1-r lie at theta and pi - theta
    assert np.allclose(g["theta"] + g["theta"][::-1], math.pi, atol=1e-12)
    assert np.allclose(g["R"], g["R"][::-1], rtol=1e-12)
    assert np.allclose(g["logg"], g["logg"][::-1], rtol=1e-12)
    assert np.allclose(g["f"], -g["f"][::-1], atol=1e-12)
    assert np.allclose(g["beta"], g["beta"][::-1], rtol=1e-10)


def test_spinning_star_is_flattened_at_the_poles(orc, synth, wide_lens):
    g = _rings(orc, synth, _star(synth, 600.0), wide_lens)
    eq = np.argmin(np.abs(g["theta"] - math.pi / 2))
    # the equatorial radius is the largest; R decreases toward either pole
    assert np.argmax(g["R"]) in (eq - 1, eq, eq + 1)
    assert g["R"][0] < g["R"][eq] and g["R"][-1] < g["R"][eq]
    half = g["R"][: len(g["R"]) // 2]
    assert np.all(np.diff(half) > 0)
    # the equator lies at R_e (12 km) to second order in the ring offset
    assert abs(g["R"][eq] - 12.0e3) / 12.0e3 < 1e-3
    # the surface normal tilts poleward: f > 0 in the north, < 0 in the south
    assert np.all(g["f"][: eq - 1] > 0) and np.all(g["f"][eq + 2:] < 0)


@pytest.mark.parametrize("theta0", [0.4, 1.0, 2.3])
def test_slope_is_the_derivative_of_the_shape(orc, synth, wide_lens, theta0):
    """Eq. def_f: f = (dR/dtheta) / (R sqrt(1 - u)); dR/dtheta by central
    differences of the oracle's R on 201 rings 1e-4 rad apart."""
    n = 201
    g = _rings(orc, synth, _star(synth, 600.0, colat=theta0, zeta=0.01, n_theta=n), wide_lens)
    th, R, u, f = g["theta"], g["R"], g["u"], g["f"]
    dR = (R[2:] - R[:-2]) / (th[2:] - th[:-2])
    slope = f[1:-1] * R[1:-1] * np.sqrt(1.0 - u[1:-1])
    assert np.max(np.abs(dR - slope)) < 1e-5 * np.max(np.abs(slope))


def test_gravity_is_largest_at_the_pole(orc, synth, wide_lens):
    g = _rings(orc, synth, _star(synth, 600.0), wide_lens)
    eq = np.argmin(np.abs(g["theta"] - math.pi / 2))
    assert g["logg"][0] > g["logg"][eq] and g["logg"][-1] > g["logg"][eq]


@pytest.mark.parametrize("spin,oblate", [(0.0, 1), (600.0, 0)])
def test_non_rotating_or_spherical_star_is_uniform(orc, synth, wide_lens, spin, oblate):
    g = _rings(orc, synth, _star(synth, spin, oblate=oblate), wide_lens)
    assert np.allclose(g["R"], 12.0e3, rtol=1e-14)
    assert np.allclose(g["f"], 0.0, atol=1e-15)
    assert np.allclose(g["logg"], g["logg"][0], rtol=1e-14)
    # surface speed: zero without spin, vanishing toward the poles with it
    if spin == 0.0:
        assert np.all(g["beta"] == 0.0)
    else:
        assert g["beta"][0] < g["beta"][len(g["beta"]) // 2]


def test_oblate_delay_is_radial_photon_coordinate_time(orc, synth, wide_lens):
    """Eq. delta_t_oblate against the radial null geodesic: a photon from
    r = R(theta) to r = R_e takes coordinate time int dr / (c (1 - R_s / r))."""
    from scipy.integrate import quad
    c = 299792458.0
    g = _rings(orc, synth, _star(synth, 600.0, n_theta=16), wide_lens)
    Re = 12.0e3
    for R, u, dt in zip(g["R"], g["u"], g["dt_obl"]):
        Rs = u * R
        ref = quad(lambda r: 1.0 / (1.0 - Rs / r), R, Re, epsabs=0.0, epsrel=1e-13)[0] / c
        assert dt == pytest.approx(ref, rel=1e-9, abs=1e-18)
    assert np.all(g["dt_obl"] > 0.0)      # every ring below the equator's radius
