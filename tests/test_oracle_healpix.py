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


# ---- full-surface temperature maps (Sect. 2.6) ---------------------------
def pixel_centres(orc, w):
    """(theta, phi) of every mesh pixel in ring order, from the oracle's ring
    records (whole-sphere selection)."""
    v = mesh_like(w)
    th, ph = [], []
    N = int(w.inst.n_theta[0])
    for r in range(4 * N - 1):
        info = orc.ring_template(v, 0, r)[0]
        n = int(info["n_active"])
        i = r + 1
        if i < N or i > 3 * N:
            ip = i if i < N else 4 * N - i
            phi = (np.arange(n) + 0.5) * (math.pi / 2) / ip
        else:
            s = (i - N + 1) % 2
            phi = (np.arange(n) + 1 - s / 2) * math.pi / (2 * N)
        th.append(np.full(n, info["theta"]))
        ph.append(phi)
    return np.concatenate(th), np.concatenate(ph)


def mesh_like(w):
    v = copy_w(w)
    v.inst.colat[:] = 0.0
    v.inst.zeta[:] = math.pi
    v.inst.mask_zeta[:] = 0.0
    v.inst.logT_map = None
    return v


def copy_w(w):
    import copy
    v = copy.copy(w)
    v.inst = w.inst.copy()
    return v


def test_map_of_a_uniform_cap_is_the_cap(orc, synth):
    """A map that is T inside a cap and dark outside gives the cap's profile."""
    N = 16
    w = mesh(synth, N, colat=1.1, zeta=0.4)
    w.inst.azim[:] = 0.3
    w.inst.spin_hz[:] = 300.0
    ref = orc.profile(w)
    th, ph = pixel_centres(orc, w)
    tc, ac, z = 1.1, 0.3, 0.4
    cd = np.cos(th) * math.cos(tc) + np.sin(th) * math.sin(tc) * np.cos(ph - ac)
    m = np.where(cd >= math.cos(z), float(w.inst.logT[0, 0]), 0.0)
    v = copy_w(w)
    v.inst.logT_map = m[None, :]
    np.testing.assert_allclose(orc.profile(v), ref, rtol=1e-13, atol=0)


def test_map_profiles_add_over_disjoint_regions(orc, synth):
    N = 12
    w = mesh(synth, N)
    w.inst.spin_hz[:] = 300.0
    w.inst.incl_rad[:] = 1.0
    th, ph = pixel_centres(orc, w)
    lt = 6.0 + 0.2 * np.cos(th) + 0.05 * np.sin(2 * ph)
    north = th < 1.2
    maps = [np.where(north, lt, 0.0), np.where(~north, lt, 0.0), lt]
    F = []
    for m in maps:
        v = copy_w(w)
        v.inst.logT_map = m[None, :]
        F.append(orc.profile(v))
    np.testing.assert_allclose(F[0] + F[1], F[2], rtol=1e-12, atol=1e-30)


def test_uniform_whole_star_map_closed_form(orc, synth):
    N = 32
    w = mesh(synth, N)
    w.inst.n_fp = 384
    v = copy_w(w)
    v.inst.logT_map = np.full((1, 12 * N * N), float(w.inst.logT[0, 0]))
    F = orc.profile(v)
    assert np.max(np.abs(F / closed_form(w)[None, :] - 1)) < 1e-5
