"""Pins of the oracle's forward-mode derivative (the complex-step build of
ppm_oracle.c) against what does not depend on it: the oracle's own value,
central differences of the ordinary build, closed forms for the distance and
the absorption column, and linearity in the seed direction."""
import math

import numpy as np
import pytest

from grad_helpers import SCALE, oracle_fd, oracle_ll

DEG = math.pi / 180.0


@pytest.fixture(scope="module")
def small_two_cap(synth, atm, small_lens):
    w = synth.atm_two_spot(n_theta=8, n_phi=12, n_phase=16, n_E=24, n_chan=12, atm=atm,
                           lens=small_lens)
    i = w.inst
    i.incl_rad[0] = 30 * DEG
    i.colat[0] = [25 * DEG, 55 * DEG]
    i.azim[0] = [0.3, math.pi]
    i.zeta[0] = [0.2, 0.15]
    i.logT[0] = [6.112, 6.023]
    i.mask_zeta[0] = [0.0, 0.0]
    return w


def test_tangent_value_is_the_oracle_value(orc, small_two_cap):
    v = np.arange(13, dtype=float) - 6.0
    ll, _ = orc.loglike_tangent(small_two_cap, v)
    assert ll == pytest.approx(oracle_ll(orc, small_two_cap), rel=1e-14)


def test_tangent_matches_central_differences(orc, small_two_cap):
    """Forward mode against 2-point central differences (step 1e-5 relative)
    of the ordinary build: 1e-5 relative per component, plus 1e-7 of the
    largest scale-weighted component (difference rounding and O(h^2))."""
    g = orc.grad_tangent(small_two_cap)
    fd = oracle_fd(orc, small_two_cap, rel=1e-5)
    sc = np.asarray(SCALE)
    tol = 1e-5 * np.abs(fd) + 1e-7 * np.max(np.abs(fd) * sc) / sc
    assert np.all(np.abs(g - fd) <= tol), np.abs(g / fd - 1)


def test_tangent_blackbody_logT_through_kT(orc, synth, small_lens):
    w = synth.bb_small(n_theta=8, n_phi=10, n_phase=16, n_E=16, lens=small_lens)
    w = synth._with_response(w, 12, tau=1.0e3)
    g = orc.grad_tangent(w)
    fd = oracle_fd(orc, w, rel=1e-5)
    assert len(g) == 9
    sc = np.asarray(SCALE[:9])
    tol = 1e-5 * np.abs(fd) + 1e-7 * np.max(np.abs(fd) * sc) / sc
    assert np.all(np.abs(g - fd) <= tol), np.abs(g / fd - 1)


def test_tangent_distance_and_column_closed_forms(orc, small_two_cap):
    """F_t scales as D^-2 and the attenuation is exp(-N_H sigma), so with
    H = tau (d / lambda - 1):
      dlogL/dD   = -2/D sum H C
      dlogL/dN_H = -1e20 sum_{j,c} H[j,c] sum_k F_t[j,k] sigma_k ATT_k R[k,c]."""
    w = small_two_cap
    Ft = orc.profile(w)
    nh = float(w.inst.nh_1e20[0])
    C = orc.counts_model(Ft, w.R, w.sigma_ism, nh)
    d = w.counts[:w.inst.n_phase[0]].astype(np.float64)
    H = w.tau * (d / (w.tau * C) - 1.0)
    D = float(w.inst.dist_kpc[0])
    sg = w.sigma_ism.astype(np.float64)
    att = np.exp(-nh * 1e20 * sg)
    dC = -1e20 * (Ft * sg * att) @ w.R.astype(np.float64)
    e = np.eye(13)
    gD = orc.loglike_tangent(w, e[3])[1]
    gN = orc.loglike_tangent(w, e[4])[1]
    assert gD == pytest.approx(-2.0 / D * np.sum(H * C), rel=1e-10)
    assert gN == pytest.approx(np.sum(H * dC), rel=1e-10)


def test_tangent_is_linear_in_the_direction(orc, small_two_cap):
    g = orc.grad_tangent(small_two_cap)
    v = np.linspace(-1.0, 1.0, 13) * np.asarray(SCALE)
    assert orc.loglike_tangent(small_two_cap, v)[1] == pytest.approx(float(g @ v), rel=1e-11)


def test_tangent_with_caps_over_the_poles(orc, synth, atm, small_lens):
    """Caps that contain a pole: the rings that encircle it have the clamped
    half-width pi, a constant with no derivative (the same branch-fixed
    function the ordinary build evaluates).  Forward mode against central
    differences, as above."""
    w = synth.atm_two_spot(n_theta=8, n_phi=12, n_phase=16, n_E=24, n_chan=12, atm=atm,
                           lens=small_lens)
    i = w.inst
    i.incl_rad[0] = 40 * DEG
    i.colat[0] = [0.3, math.pi - 0.25]
    i.azim[0] = [0.3, 2.0]
    i.zeta[0] = [0.5, 0.4]
    i.logT[0] = [6.112, 6.023]
    i.mask_zeta[0] = [0.0, 0.0]
    g = orc.grad_tangent(w)
    assert np.all(np.isfinite(g))
    fd = oracle_fd(orc, w, rel=1e-5)
    sc = np.asarray(SCALE)
    tol = 1e-5 * np.abs(fd) + 1e-7 * np.max(np.abs(fd) * sc) / sc
    assert np.all(np.abs(g - fd) <= tol), np.abs(g / fd - 1)
