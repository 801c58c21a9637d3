"""The oracle's reading for non-finite inputs (the paper is silent): a NaN or
infinite parameter that the instance uses is a range error; an infinite
distance is the zero-flux limit; a mask radius of -inf is no mask; a
temperature map makes the spot parameters unused.  The CUDA path takes the
same reading (tests/test_gpu_loglike.py)."""
import math

import numpy as np
import pytest


@pytest.fixture(scope="module")
def w(synth, atm, small_lens):
    return synth.atm_two_spot(n_theta=6, n_phi=8, n_phase=8, n_E=12, n_chan=4, atm=atm,
                              lens=small_lens)


CASES = [
    ("mass_msun", None, math.nan), ("mass_msun", None, math.inf),
    ("radius_km", None, math.inf), ("spin_hz", None, math.nan),
    ("incl_rad", None, -math.inf), ("nh_1e20", None, math.nan),
    ("dist_kpc", None, math.nan),
    ("colat", 0, math.nan), ("azim", 0, math.nan), ("azim", 1, math.inf),
    ("zeta", 1, math.inf), ("logT", 0, math.nan),
    ("mask_zeta", 1, math.nan), ("mask_zeta", 1, math.inf),
    ("mask_colat", 1, math.nan), ("mask_azim", 1, -math.inf),
]


@pytest.mark.parametrize("field,spot,value", CASES)
def test_non_finite_parameter_is_a_range_error(orc, w, field, spot, value):
    inst = w.inst.copy()
    arr = getattr(inst, field)
    if spot is None:
        arr[0] = value
    else:
        arr[0, spot] = value
    w2 = type(w)(w.name, inst, w.lens, w.E_keV, atm=w.atm, R=w.R, sigma_ism=w.sigma_ism,
                 counts=w.counts, tau=w.tau)
    with pytest.raises(orc.OracleRangeError):
        orc.profile(w2)


def test_infinite_distance_is_zero_flux(orc, w):
    inst = w.inst.copy()
    inst.dist_kpc[0] = math.inf
    w2 = type(w)(w.name, inst, w.lens, w.E_keV, atm=w.atm)
    Ft = orc.profile(w2)
    assert np.all(Ft == 0.0)


def test_minus_infinite_mask_radius_is_no_mask(orc, w):
    inst = w.inst.copy()
    inst.mask_zeta[0, 1] = 0.0
    ref = orc.profile(type(w)(w.name, inst, w.lens, w.E_keV, atm=w.atm))
    inst2 = w.inst.copy()
    inst2.mask_zeta[0, 1] = -math.inf
    inst2.mask_colat[0, 1] = math.nan     # unused without a mask
    got = orc.profile(type(w)(w.name, inst2, w.lens, w.E_keV, atm=w.atm))
    assert np.array_equal(got, ref)
    # and the mask did matter: the original ring differs
    assert not np.array_equal(orc.profile(w), ref)


def test_map_ignores_the_spot_parameters(orc, synth, small_lens):
    n_side = 4
    w = synth.bb_small(n_theta=n_side, n_phi=4, n_phase=8, n_E=8, lens=small_lens)
    inst = w.inst.replace(grid=1, logT_map=np.full((1, 12 * n_side * n_side), 6.3))
    ref = orc.profile(type(w)(w.name, inst, w.lens, w.E_keV))
    inst2 = inst.copy()
    inst2.azim[0, 0] = math.nan
    inst2.logT[0, 0] = math.inf
    inst2.mask_zeta[0, 0] = math.nan
    got = orc.profile(type(w)(w.name, inst2, w.lens, w.E_keV))
    assert np.array_equal(got, ref) and ref.max() > 0
