"""Pins of the oracle's HEALPix whole-surface mesh (Sect. 2.6; Gorski et al.
2005): pixel count and solid angle of the whole sphere, north-south
symmetry, equal-area latitude distribution, cap selection by area, and the
closed-form flux of a uniform non-rotating blackbody star on the mesh."""
import math

import numpy as np
import pytest

from test_oracle_physics import closed_form, whole_star


def mesh(synth, N, colat=0.0, zeta=math.pi):
    w = whole_star(synth, N, 64, 256)
    w.inst.grid = 1
    w.inst.colat[:] = colat
    w.inst.zeta[:] = zeta
    return w


def rings(orc, w):
    out = []
    for r in range(4 * int(w.inst.n_theta[0]) - 1):
        info = orc.ring_template(w, 0, r)[0]
        out.append((info["theta"], info["dcos"], info["dphi"], int(info["n_active"])))
    return np.array(out)


@pytest.mark.parametrize("N", [1, 2, 8, 16])
def test_whole_sphere_count_and_area(orc, synth, N):
    R = rings(orc, mesh(synth, N))
    assert len(R) == 4 * N - 1
    assert int(R[:, 3].sum()) == 12 * N * N
    # every pixel has the same solid angle, and they tile the sphere
    omega = R[:, 1] * R[:, 2]
    np.testing.assert_allclose(omega, math.pi / (3 * N * N), rtol=1e-13)
    assert float((omega * R[:, 3]).sum()) == pytest.approx(4 * math.pi, rel=1e-13)


def test_north_south_symmetry_and_equal_area_latitudes(orc, synth):
    N = 16
    R = rings(orc, mesh(synth, N))
    z = np.cos(R[:, 0])
    np.testing.assert_allclose(z, -z[::-1], atol=1e-14)
    np.testing.assert_array_equal(R[:, 3], R[::-1, 3])
    # equal area: the fraction of pixels with z above z0 tracks (1 - z0) / 2
    zz = np.repeat(z, R[:, 3].astype(int))
    for z0 in np.linspace(-0.9, 0.9, 13):
        frac = np.mean(zz > z0)
        assert abs(frac - (1 - z0) / 2) < 1.5 / (4 * N)


def test_cap_selection_by_area(orc, synth):
    """A cap selects about 12 N^2 (1 - cos zeta) / 2 pixels (error O(N zeta))."""
    N = 32
    for colat, zeta in [(0.7, 0.3), (2.0, 0.5), (math.pi / 2, 0.2)]:
        R = rings(orc, mesh(synth, N, colat, zeta))
        n = R[:, 3].sum()
        expect = 12 * N * N * (1 - math.cos(zeta)) / 2
        assert abs(n - expect) < 4 * (2 * math.pi * zeta) * N / math.sqrt(12) + 4


def test_closed_form_blackbody_star_on_the_mesh(orc, synth):
    """The mesh integrates the whole visible sphere: the closed-form flux
    pi (R_inf/D)^2 I(T_inf)/E is approached as N_side grows."""
    errs = []
    for N in (8, 32):
        w = mesh(synth, N)
        w.inst.n_fp = 384
        F = orc.profile(w)
        errs.append(np.max(np.abs(F / closed_form(w)[None, :] - 1)))
    assert errs[1] < 1e-5          # 1.9e-4 at N_side 8, 2.5e-6 at 32
    assert errs[1] < errs[0] / 10
