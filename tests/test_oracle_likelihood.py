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


def _fine_grid(E, n=150, seed=4):
    rng = np.random.default_rng(seed)
    edges = np.sort(rng.uniform(E[0] * 0.8, E[-1] * 1.1, n + 1))
    return edges[:-1], edges[1:]


def test_downsample_partition_of_unity(orc):
    """The basis functions sum to one everywhere, so each detector bin's
    column of DS sums to the bin width (bins inside and beyond the grid)."""
    E = np.geomspace(0.2, 5.0, 40)
    lo, hi = _fine_grid(E)
    DS = orc.downsample_matrix(E, lo, hi)
    np.testing.assert_allclose(DS.sum(axis=0), hi - lo, rtol=1e-12)
    assert np.all(DS >= 0.0)


def test_downsample_integrates_linear_functions_exactly(orc):
    """Inside the grid the interpolant of a linear function is the function,
    so sum_i f(E_i) DS[i, e] is its exact integral over the bin."""
    E = np.geomspace(0.2, 5.0, 40)
    lo, hi = _fine_grid(E, seed=7)
    keep = (lo > E[0]) & (hi < E[-1])
    DS = orc.downsample_matrix(E, lo[keep], hi[keep])
    f = lambda x: 3.0 - 0.7 * x
    exact = 3.0 * (hi - lo)[keep] - 0.35 * (hi[keep] ** 2 - lo[keep] ** 2)
    np.testing.assert_allclose(f(E) @ DS, exact, rtol=1e-12, atol=1e-14)


def test_downsample_matches_quadrature(orc):
    """Against scipy's adaptive quadrature of np.interp of the unit vectors."""
    from scipy.integrate import quad
    E = np.geomspace(0.2, 5.0, 12)
    lo, hi = np.array([0.1, 0.33, 1.0, 4.7]), np.array([0.25, 0.61, 1.02, 6.0])
    DS = orc.downsample_matrix(E, lo, hi)
    eye = np.eye(len(E))
    for i in range(len(E)):
        for e in range(len(lo)):
            pts = E[(E > lo[e]) & (E < hi[e])]
            q, _ = quad(lambda x: np.interp(x, E, eye[i]), lo[e], hi[e],
                        points=pts if len(pts) else None, epsabs=1e-13)
            assert DS[i, e] == pytest.approx(q, abs=1e-12)
