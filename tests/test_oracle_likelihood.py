"""Pins of the oracle's ISM, response contraction and Poisson likelihood
(Sect. 2.7, 2.8.4; the likelihood reading of Sect. 5 and 6)."""
import math

import numpy as np
import pytest
from scipy.stats import poisson


def test_counts_model_is_attenuated_matrix_product(orc):
    rng = np.random.default_rng(0)
    Ft = rng.uniform(0, 1, (7, 11))
    R = rng.uniform(0, 1, (11, 5)).astype(np.float32)
    sig = rng.uniform(1e-22, 1e-21, 11).astype(np.float32)
    nh = 3.0
    ref = Ft @ np.diag(np.exp(-nh * 1e20 * sig.astype(np.float64))) @ R.astype(np.float64)
    assert np.allclose(orc.counts_model(Ft, R, sig, nh), ref, rtol=1e-13)
    # N_H = 0: no attenuation; a permutation response moves columns exactly
    P = np.zeros((11, 11), np.float32)
    P[np.arange(11), (np.arange(11) + 4) % 11] = 1.0
    out = orc.counts_model(Ft, P, sig, 0.0)
    assert np.array_equal(out[:, (np.arange(11) + 4) % 11], Ft)


def test_loglike_matches_poisson_pmf(orc):
    rng = np.random.default_rng(1)
    lam = rng.uniform(0.1, 40.0, 500)
    d = rng.poisson(lam).astype(np.int32)
    tau = 2.5
    C = lam / tau
    assert orc.loglike(C, d, tau) == pytest.approx(poisson.logpmf(d, lam).sum(), rel=1e-12)
    bkg = rng.uniform(0, 2, 500).astype(np.float32)
    ref = poisson.logpmf(d, lam + bkg.astype(np.float64)).sum()
    assert orc.loglike(C, d, tau, bkg) == pytest.approx(ref, rel=1e-12)


def test_loglike_zero_rate_cases(orc):
    C = np.array([0.0, 1.0])
    assert orc.loglike(C, np.array([0, 2], np.int32), 1.0) == pytest.approx(
        poisson.logpmf(2, 1.0), rel=1e-13)
    assert orc.loglike(C, np.array([1, 2], np.int32), 1.0) == -math.inf


def test_loglike_stationary_at_data(orc):
    # d ln L / d lambda = d / lambda - 1 vanishes at lambda = d
    d = np.array([3, 17, 250], np.int32)
    h = 1e-4
    for i in range(3):
        C = d.astype(np.float64).copy()
        Cp, Cm = C.copy(), C.copy()
        Cp[i] += h
        Cm[i] -= h
        g = (orc.loglike(Cp, d, 1.0) - orc.loglike(Cm, d, 1.0)) / (2 * h)
        assert abs(g) < 1e-6


def test_chi2_approximates_minus_two_delta_loglike(orc):
    """Large counts: -2 Delta ln L ~ chi^2 of Eq. chi2_def (K = 1 at 1e6 counts)."""
    rng = np.random.default_rng(2)
    m = rng.uniform(0.5, 1.5, 2000)
    m *= 1e6 / m.sum()
    d_model = m * (1 + 1e-3 * rng.standard_normal(m.size))
    # both models evaluated on the same counts drawn from m
    d = np.round(m).astype(np.int32)
    chi2 = np.sum((m - d_model) ** 2 / m)
    dlnL = orc.loglike(d_model, d, 1.0) - orc.loglike(m, d, 1.0)
    # the difference of the two chi^2 w.r.t. the data equals -2 dlnL to leading order
    chi2_d = np.sum((d - d_model) ** 2 / d_model) - np.sum((d - m) ** 2 / m)
    assert -2 * dlnL == pytest.approx(chi2_d, rel=0.02)
    assert chi2 > 0
