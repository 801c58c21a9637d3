"""The seeded synthetic inputs match the input recipe and the benchmark
configurations: table axes and value model, cross-section, response,
counts, and the parameters and sizes of every workload.  (Generator checks:
no forward-model arithmetic is involved.)"""
import math

import numpy as np
import pytest

DEG = math.pi / 180.0


@pytest.fixture(scope="module")
def table(synth):
    return synth.atm_table()


def test_atmosphere_axes(table):
    assert table.I.shape == (35, 11, 67, 166) and table.I.dtype == np.float32
    assert table.logT[0] == 5.1 and table.logT[-1] == pytest.approx(6.8)
    assert table.logg[0] == 13.7 and table.logg[-1] == pytest.approx(14.7)
    assert np.allclose(np.diff(table.logT), np.diff(table.logT)[0])
    E = np.exp(table.lnE)
    assert E[0] == pytest.approx(0.05) and E[-1] == pytest.approx(10.0)
    assert np.allclose(np.diff(table.lnE), np.diff(table.lnE)[0])
    mu = table.mu
    assert mu[0] == pytest.approx(1e-6) and mu[-1] == pytest.approx(1.0)
    assert np.all(np.diff(mu) > 0)
    # clustered at both ends, symmetric about 1/2
    assert np.allclose(mu + mu[::-1], 1.0 + 1e-6)
    d = np.diff(mu)
    assert d[0] < d[33] / 10 and d[-1] < d[33] / 10
    assert table.n_protect == 4


def test_atmosphere_values_are_a_perturbed_limb_darkened_blackbody(table):
    I = table.I.astype(np.float64)
    assert np.all(np.isfinite(I)) and np.all(I >= 0.0)
    T4, G4, M4, E4 = np.meshgrid(table.logT, table.logg, table.mu, np.exp(table.lnE),
                                 indexing="ij")
    kT = 8.617333262e-8 * 10.0 ** T4
    with np.errstate(over="ignore"):
        bb = 2.0 * E4 ** 3 / (4.135667696e-18 ** 3 * 2.99792458e10 ** 2) / np.expm1(E4 / kT)
    limb = 1.0 + (0.6 - 0.2 * (T4 - 6.0) + 0.1 * (G4 - 14.2)) * M4 + \
        (-0.25 + 0.05 * (T4 - 6.0)) * M4 ** 2
    ok = I > 1e-30
    ratio = I[ok] / (bb[ok] * limb[ok])
    assert ratio.min() >= 0.95 * (1 - 1e-6) and ratio.max() <= 1.05 * (1 + 1e-6)
    assert ratio.max() - ratio.min() > 0.05      # the perturbation is there


def test_table_is_seeded(synth, table):
    again = synth.atm_table()
    assert np.array_equal(again.I, table.I)
    other = synth.atm_table(seed=7)
    assert not np.array_equal(other.I, table.I)


def test_ism_cross_section(synth):
    E = np.array([0.5, 1.0, 2.0, 4.0])
    s = synth.sigma_ism(E).astype(np.float64)
    assert s[1] == pytest.approx(2e-22, rel=1e-6)
    assert np.allclose(np.diff(np.log(s)) / np.diff(np.log(E)), -2.5, atol=1e-5)


def test_response_width_and_area(synth):
    E = synth.logspace(0.1, 5.215, 256)
    R = synth.response(E, 300).astype(np.float64)
    assert R.shape == (256, 300) and np.all(R >= 0)
    edges = np.linspace(E[0], E[-1], 301)
    centres = 0.5 * (edges[1:] + edges[:-1])
    w = np.empty_like(E)
    w[0], w[-1] = 0.5 * (E[1] - E[0]), 0.5 * (E[-1] - E[-2])
    w[1:-1] = 0.5 * (E[2:] - E[:-2])
    A = R.sum(axis=1) / w
    for k in (80, 128, 200):    # energies well inside the channel span
        p = R[k] / R[k].sum()
        mean = np.sum(p * centres)
        sd = math.sqrt(np.sum(p * (centres - mean) ** 2))
        assert mean == pytest.approx(E[k], abs=2e-3)
        # FWHM 0.1 keV, broadened by the channel width (variance + width^2 / 12)
        width = edges[1] - edges[0]
        assert sd == pytest.approx(math.sqrt((0.1 / 2.3548200450309493) ** 2 + width ** 2 / 12),
                                   rel=0.02)
    # the effective area peaks near 1.5 keV at 1500 cm^2
    k = np.argmax(A[20:-20]) + 20
    assert E[k] == pytest.approx(1.5, rel=0.03) and A[k] == pytest.approx(1500.0, rel=0.01)


def test_counts_total_and_seed(synth):
    c = synth.counts(np.array([128]), 300)
    assert c.shape == (128, 300) and c.dtype == np.int32
    assert abs(int(c.sum()) - 1_000_000) < 5 * 1000
    assert np.array_equal(c, synth.counts(np.array([128]), 300))


def test_small_blackbody_workload(synth):
    w = synth.bb_small()
    i = w.inst
    assert (i.B, i.n_spots, i.oblate, i.emission) == (1, 1, 0, 0)
    assert (int(i.n_theta[0]), int(i.n_phi[0]), int(i.n_phase[0])) == (32, 32, 64)
    assert len(w.E_keV) == 32 and w.E_keV[0] == pytest.approx(0.2) and \
        w.E_keV[-1] == pytest.approx(3.0)
    assert (i.mass_msun[0], i.radius_km[0], i.spin_hz[0], i.dist_kpc[0]) == (1.4, 12.0, 205.0, 0.3)
    assert i.incl_rad[0] == pytest.approx(60 * DEG) and i.colat[0, 0] == pytest.approx(45 * DEG)
    assert (i.zeta[0, 0], i.logT[0, 0]) == (0.2, 6.1)


def test_two_spot_workload(synth, table):
    w = synth.atm_two_spot(atm=table)
    i = w.inst
    assert (i.n_spots, i.oblate, i.emission) == (2, 1, 1)
    assert (int(i.n_theta[0]), int(i.n_phi[0]), int(i.n_phase[0])) == (128, 128, 128)
    assert len(w.E_keV) == 256 and w.R.shape == (256, 300)
    assert i.nh_1e20[0] == 1.0                       # N_H = 1e20 cm^-2
    assert i.mask_zeta[0, 0] <= 0 < i.mask_zeta[0, 1] < i.zeta[0, 1]   # a cap and a ring
    assert abs(int(w.counts.sum()) - 1_000_000) < 5 * 1000


def test_crescent_workload(synth, table):
    w = synth.crescent_extreme(atm=table)
    i = w.inst
    u = 2 * 1.32712440018e20 * 2.0 / 299792458.0 ** 2 / 11.0e3
    assert u == pytest.approx(0.537, abs=1e-3)
    assert (i.mass_msun[0], i.radius_km[0], i.spin_hz[0]) == (2.0, 11.0, 346.0)
    assert i.incl_rad[0] == pytest.approx(85 * DEG)
    assert (int(i.n_theta[0]), int(i.n_phi[0]), int(i.n_phase[0]), len(w.E_keV)) == \
        (512, 512, 256, 300)
    # emitter 0.05 rad, mask 0.035 rad offset 0.02 rad toward the pole: a crescent
    assert i.zeta[0, 0] == 0.05 and i.mask_zeta[0, 0] == 0.035
    assert i.colat[0, 0] - i.mask_colat[0, 0] == pytest.approx(0.02)
    # the last logT interval of the table
    assert table.logT[-2] < i.logT[0, 0] < table.logT[-1]


def test_batched_workloads(synth, table):
    w = synth.batch(B=512, atm=table)
    i = w.inst
    u = 2 * 1.32712440018e20 * i.mass_msun / 299792458.0 ** 2 / (i.radius_km * 1e3)
    assert np.all(u <= 0.55) and u.max() > 0.5
    assert np.all((1.0 <= i.mass_msun) & (i.mass_msun <= 2.5))
    assert np.all((9.0 <= i.radius_km) & (i.radius_km <= 15.0))
    assert np.all((5 * DEG <= i.incl_rad) & (i.incl_rad <= 90 * DEG))
    assert np.all((0.01 <= i.zeta) & (i.zeta <= 1.0))
    assert np.all((5.8 <= i.logT) & (i.logT <= 6.6))
    assert set(np.unique(i.n_theta)) == {64, 128, 256} and np.array_equal(i.n_theta, i.n_phi)
    assert set(np.unique(i.n_phase)) == {32, 64, 128}
    assert len(w.E_keV) == 256 and w.R.shape == (256, 300)
    g = synth.grad_batch(B=64, atm=table)
    assert np.all(g.inst.n_theta == 128) and np.all(g.inst.n_phase == 128)
    assert not np.array_equal(g.inst.mass_msun, w.inst.mass_msun[:64])


def test_healpix_map_workload(synth, table):
    w = synth.healpix_map(atm=table)
    i = w.inst
    m = i.logT_map[0]
    assert i.grid == 1 and int(i.n_theta[0]) == 52 and m.size == 12 * 52 * 52 == 32448
    warm = m > 0
    assert warm.mean() == pytest.approx(0.25, abs=1e-3)
    assert m[warm].min() >= 5.95 - 1e-12 and m[warm].max() <= 6.2 + 1e-12
    assert np.all(m[~warm] == -1.0)
