"""Pins of the oracle's spot geometry and star model.

Element grid (the spot-bounding grid: n_theta rings uniform in theta over
the cap's colatitude range, each with n_phi elements spread over the cap's
azimuthal width at the ring centre, an element active unless its centre lies
inside the spot's mask cap; spots as emitter and mask caps, Sect. 2.6 and the
surface discretisation of Sect. 2.8.1).  What the geometry fixes:

* the summed element solid angle converges to the cap's 2 pi (1 - cos zeta),
  for caps away from the poles and caps that contain or touch a pole;
* a ring spot (concentric mask) gives 2 pi (cos zeta_mask - cos zeta);
* a crescent (offset mask) gives the cap minus the lens where the two caps
  overlap; the lens area is the closed form for two intersecting spherical
  caps (Gauss-Bonnet), itself checked here by a seeded Monte Carlo over the
  emitter cap that uses none of the oracle's code;
* every ring's outermost element edges phi_c +- Delta_i lie at great-circle
  distance zeta from the spot centre, and a ring whose half-width is pi lies
  inside the cap;
* each element's active flag equals an independent point-in-cap test on its
  3-D unit vector.

Star model (Sect. 2.2): the oracle's R(theta) and g(theta) are regressed onto
the monomials of Eq. Rtheta and of the g(theta)/g_0 fit over stars of varied
Omega_bar and x; the recovered coefficients must equal the printed ones
(`tests/golden/star_model_coefficients.json`).

Each pin is also run on mutated copies of the oracle (one plausible slip
planted per copy, compiled here on the CPU) and must fail there.
"""
import ctypes as C
import json
import math
import os
import subprocess

import numpy as np
import pytest

GM_SUN = 1.32712440018e20
C_MS = 299792458.0

HERE = os.path.dirname(os.path.abspath(__file__))
DEG = math.pi / 180.0


def lens_area(a, b, d):
    """Solid angle of the intersection of two caps of angular radii a, b whose
    centres are d apart (unit sphere).  By Gauss-Bonnet on the lens bounded by
    two small-circle arcs: 2 pi minus the two exterior vertex angles minus the
    arcs' geodesic curvature (cos r times the half-angle subtended at the
    circle's centre, for each circle)."""
    if d >= a + b:
        return 0.0
    if d <= abs(a - b):
        return 2.0 * math.pi * (1.0 - math.cos(min(a, b)))
    t0 = math.acos((math.cos(d) - math.cos(a) * math.cos(b)) / (math.sin(a) * math.sin(b)))
    ta = math.acos((math.cos(b) - math.cos(d) * math.cos(a)) / (math.sin(d) * math.sin(a)))
    tb = math.acos((math.cos(a) - math.cos(d) * math.cos(b)) / (math.sin(d) * math.sin(b)))
    return 2.0 * math.pi - 2.0 * t0 - 2.0 * math.cos(a) * ta - 2.0 * math.cos(b) * tb


def cap_area(z):
    return 2.0 * math.pi * (1.0 - math.cos(z))


def unit(theta, phi):
    theta = np.asarray(theta, dtype=np.float64)
    phi = np.asarray(phi, dtype=np.float64)
    return np.stack([np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi),
                     np.cos(theta)], axis=-1)


# ---------------------------------------------------------------------------
# helpers that read the oracle's element grid through orc_ring_template
# ---------------------------------------------------------------------------
def spot_workload(synth, colat, zeta, azim=0.0, mask=None, n=64, n_phi=None):
    lens = synth.LensSpec(u_min=0.30, u_max=0.40, n_u=3, n_cpsi=64, n_calpha=16)
    w = synth.bb_small(n_theta=n, n_phi=n_phi or n, n_phase=4, n_E=2, lens=lens)
    w.inst.colat[:] = colat
    w.inst.azim[:] = azim
    w.inst.zeta[:] = zeta
    if mask is not None:
        w.inst.mask_colat[:], w.inst.mask_azim[:], w.inst.mask_zeta[:] = mask
    w.inst.n_fp = 4
    return w


def rings(orc, w):
    return [orc.ring_template(w, 0, r)[0] for r in range(int(w.inst.n_theta[0]))]


def grid_area(orc, w):
    return sum(i["n_active"] * i["dcos"] * i["dphi"] for i in rings(orc, w))


# ---------------------------------------------------------------------------
# pin checks (plain functions so that the mutation tests can run them too)
# ---------------------------------------------------------------------------
CAPS = [(45 * DEG, 0.2),          # away from both poles
        (0.1, 0.3),               # contains the north pole
        (math.pi - 0.05, 0.2),    # contains the south pole
        (0.2, 0.2),               # touches the north pole
        (math.pi / 2, 1.0)]       # large, on the equator


def check_cap_areas(orc, synth, n=512, tol=5e-5):
    for colat, z in CAPS:
        a = grid_area(orc, spot_workload(synth, colat, z, n=n))
        assert abs(a / cap_area(z) - 1) < tol, (colat, z, a / cap_area(z) - 1)


def check_ring_spot_area(orc, synth, n=512, tol=2e-4):
    c = 120 * DEG
    w = spot_workload(synth, c, 0.25, azim=math.pi, mask=(c, math.pi, 0.12), n=n)
    exact = 2.0 * math.pi * (math.cos(0.12) - math.cos(0.25))
    a = grid_area(orc, w)
    assert abs(a / exact - 1) < tol, a / exact - 1


CRESCENTS = [
    # (emitter colat, azim, zeta), (mask colat, azim, zeta): the benchmark
    # crescent (mask 0.02 rad poleward), a large one, and one whose mask is
    # offset in azimuth as well
    ((75.5 * DEG, 0.0, 0.05), (75.5 * DEG - 0.02, 0.0, 0.035)),
    ((1.0, 0.0, 0.6), (0.7, 0.0, 0.4)),
    ((1.2, 0.5, 0.5), (1.1, 0.9, 0.35)),
]


def centre_distance(m, e):
    return math.acos(np.clip(unit(m[0], m[1]) @ unit(e[0], e[1]), -1.0, 1.0))


def check_crescent_areas(orc, synth, n=512, tol=2e-4):
    for e, m in CRESCENTS:
        d = centre_distance(m, e)
        exact = cap_area(e[2]) - lens_area(e[2], m[2], d)
        w = spot_workload(synth, e[0], e[2], azim=e[1], mask=m, n=n)
        a = grid_area(orc, w)
        assert abs(a / exact - 1) < tol, (e, m, a / exact - 1)


def check_edges_on_cap_boundary(orc, synth, n=48):
    cases = CAPS + [(e[0], e[2]) for e, _ in CRESCENTS]
    for colat, z in cases:
        for phc in (0.0, 2.0):
            w = spot_workload(synth, colat, z, azim=phc, n=n)
            lo, hi = max(0.0, colat - z), min(math.pi, colat + z)
            info = rings(orc, w)
            # rings: uniform in theta over the cap's colatitude range, and
            # their cos(theta) widths tile it exactly
            th = np.array([i["theta"] for i in info])
            np.testing.assert_allclose(th, lo + (np.arange(n) + 0.5) * (hi - lo) / n,
                                       rtol=0, atol=1e-13)
            assert sum(i["dcos"] for i in info) == pytest.approx(
                math.cos(lo) - math.cos(hi), rel=1e-12, abs=1e-15)
            centre = unit(colat, phc)
            for i in info:
                half = i["half"]
                assert i["dphi"] == pytest.approx(2 * half / n, rel=1e-13)
                if half < math.pi - 1e-12:
                    for s in (-1.0, 1.0):
                        edge = unit(i["theta"], phc + s * half)
                        assert edge @ centre == pytest.approx(math.cos(z), abs=1e-12)
                else:
                    # the whole parallel is inside the cap
                    far = unit(i["theta"], phc + math.pi)
                    assert far @ centre >= math.cos(z) - 1e-12


def check_active_flags(orc, synth, n=40):
    for e, m in CRESCENTS + [((120 * DEG, math.pi, 0.25), (120 * DEG, math.pi, 0.12))]:
        w = spot_workload(synth, e[0], e[2], azim=e[1], mask=m, n=n)
        mc = unit(m[0], m[1])
        for i in rings(orc, w):
            phi = e[1] - i["half"] + (np.arange(n) + 0.5) * i["dphi"]
            inside = unit(np.full(n, i["theta"]), phi) @ mc > math.cos(m[2])
            assert int(i["n_active"]) == int(np.sum(~inside)), (e, m, i["theta"])


STARS = [  # (M_sun, R_e km, spin Hz): Omega_bar 0.05-1.0, x 0.07-0.27
    (1.0, 15.0, 700.0), (1.4, 12.0, 205.0), (2.0, 11.0, 346.0), (2.5, 9.0, 600.0),
    (1.2, 14.0, 900.0), (1.8, 10.0, 1000.0), (1.0, 9.5, 450.0), (2.2, 13.0, 800.0),
    (1.6, 11.5, 120.0)]


def _star_samples(orc, synth):
    """(Omega_bar, x, theta, R/R_e, g/g_0) from the oracle's ring geometry."""
    rows = []
    for M, R, nu in STARS:
        lens = synth.LensSpec(u_min=0.30, u_max=0.40, n_u=3, n_cpsi=64, n_calpha=16)
        w = synth.bb_small(n_theta=23, n_phi=4, n_phase=4, n_E=2, lens=lens)
        w.inst = w.inst.replace(mass_msun=M, radius_km=R, spin_hz=nu)
        w.inst.oblate = 1
        w.inst.colat[:] = math.pi / 2
        w.inst.zeta[:] = math.pi / 2
        w.inst.n_fp = 4
        GM = GM_SUN * M
        Re = R * 1e3
        Ob = 2 * math.pi * nu * math.sqrt(Re ** 3 / GM)
        x = GM / (C_MS ** 2 * Re)
        g0 = GM / Re ** 2 / math.sqrt(1 - 2 * x)
        for r in range(23):
            i = orc.ring_template(w, 0, r)[0]
            rows.append((Ob, x, i["theta"], i["R"] / Re, 10 ** i["logg"] / 100.0 / g0))
    return np.array(rows)


def _golden():
    with open(os.path.join(HERE, "golden", "star_model_coefficients.json")) as f:
        return json.load(f)


ANG = {"sin2": lambda t: np.sin(t) ** 2, "cos2": lambda t: np.cos(t) ** 2,
       "abscos": lambda t: np.abs(np.cos(t))}


def check_star_model(orc, synth):
    S = _star_samples(orc, synth)
    Ob, x, th, Rr, gr = S.T
    gold = _golden()
    # g(theta)/g_0 - 1 on the monomials the printed fit uses
    expect = {}
    for ang, p, q, c in gold["g_ratio_terms"]:
        expect[(ang, p, q)] = expect.get((ang, p, q), 0.0) + c
    keys = sorted(expect)
    A = np.stack([ANG[a](th) * Ob ** p * x ** q for a, p, q in keys], axis=1)
    coef, *_ = np.linalg.lstsq(A, gr - 1.0, rcond=None)
    assert np.max(np.abs(A @ coef - (gr - 1.0))) < 1e-10       # the family is exact
    for k, c in zip(keys, coef):
        assert c == pytest.approx(expect[k], abs=1e-6), k
    # R / R_e - 1 = o_2 cos^2(theta) (Eq. Rtheta)
    B = np.stack([np.cos(th) ** 2 * Ob ** p * x ** q for p, q, _ in gold["o2_terms"]], axis=1)
    coef, *_ = np.linalg.lstsq(B, Rr - 1.0, rcond=None)
    assert np.max(np.abs(B @ coef - (Rr - 1.0))) < 1e-12
    for (p, q, c), got in zip(gold["o2_terms"], coef):
        assert got == pytest.approx(c, abs=1e-9), (p, q)


# ---------------------------------------------------------------------------
# the pins on the oracle as it stands
# ---------------------------------------------------------------------------
def test_cap_solid_angle(orc, synth):
    check_cap_areas(orc, synth)


def test_cap_area_converges(orc, synth):
    """The sum is a midpoint rule in theta with an exact cos(theta) width:
    its error shrinks as the grid is refined (sqrt end behaviour of the
    half-width at the cap's top and bottom: about h^1.5)."""
    for colat, z in CAPS[:2] + CAPS[3:]:
        errs = [abs(grid_area(orc, spot_workload(synth, colat, z, n=n)) / cap_area(z) - 1)
                for n in (32, 128, 512)]
        assert errs[2] < errs[1] < errs[0], (colat, z, errs)


def test_ring_spot_solid_angle(orc, synth):
    check_ring_spot_area(orc, synth)


def test_crescent_solid_angle(orc, synth):
    check_crescent_areas(orc, synth)


def test_lens_area_closed_form_against_monte_carlo():
    """The closed form used above, against uniform samples on the emitter cap
    (uniform in cos of the distance to its centre and in the angle around it),
    counted inside the mask: 4e6 samples per case, seeded."""
    rng = np.random.Generator(np.random.PCG64(2510))
    for a, b, d in [(0.05, 0.035, 0.02), (0.6, 0.4, 0.3), (1.0, 0.8, 1.2), (0.2, 0.2, 0.1),
                    (0.5, 0.35, 0.4)]:
        N = 4_000_000
        cz = 1.0 - rng.random(N) * (1.0 - math.cos(a))
        ph = rng.random(N) * 2 * math.pi
        sz = np.sqrt(1.0 - cz * cz)
        v = np.stack([sz * np.cos(ph), sz * np.sin(ph), cz], axis=1)
        frac = np.mean(v @ np.array([math.sin(d), 0.0, math.cos(d)]) > math.cos(b))
        mc = frac * cap_area(a)
        sd = math.sqrt(frac * (1 - frac) / N) * cap_area(a)
        assert abs(lens_area(a, b, d) - mc) < 4 * sd, (a, b, d)
    assert lens_area(0.3, 0.1, 0.5) == 0.0
    assert lens_area(0.3, 0.1, 0.1) == pytest.approx(cap_area(0.1), rel=1e-14)


def test_element_edges_on_cap_boundary(orc, synth):
    check_edges_on_cap_boundary(orc, synth)


def test_element_active_flags(orc, synth):
    check_active_flags(orc, synth)


def test_star_model_coefficients(orc, synth):
    check_star_model(orc, synth)


# ---------------------------------------------------------------------------
# planted slips: each pin must fail on a copy of the oracle carrying one
# ---------------------------------------------------------------------------
MUTANTS = {
    "mask comparison inverted": (
        "return !(cd > cos(mz));", "return (cd > cos(mz));",
        [check_crescent_areas, check_ring_spot_area, check_active_flags]),
    "half-width without the sin(theta) sin(theta_c) denominator": (
        "real a = num / den;", "real a = num;",
        [check_cap_areas, check_edges_on_cap_boundary]),
    "wrong arccos argument in the half-width": (
        "real num = r_cos(z) - r_cos(*theta) * r_cos(tc);",
        "real num = r_cos(z) - r_sin(*theta) * r_sin(tc);",
        [check_cap_areas, check_edges_on_cap_boundary]),
    "colatitude range not clamped at the south pole": (
        "real hi = RE(tc + z) < ORC_PI ? tc + z : ORC_PI;", "real hi = tc + z;",
        [check_cap_areas, check_edges_on_cap_boundary]),
    "colatitude range not clamped at the north pole": (
        "real lo = RE(tc - z) > 0.0 ? tc - z : 0.0;", "real lo = tc - z;",
        [check_cap_areas, check_edges_on_cap_boundary]),
    "mask azimuth with the wrong sign": (
        "cos(phi - RE(in->mask_azim[spot]))", "cos(phi + RE(in->mask_azim[spot]))",
        [check_crescent_areas, check_active_flags]),
    "gravity fit coefficient typo": (
        "(-0.791 + 0.776 * x)", "(-0.791 + 0.767 * x)", [check_star_model]),
    "gravity fit without |cos(theta)|": (
        "+ r_fabs(ct) * O4", "+ ct * O4", [check_star_model]),
    "shape coefficient typo": (
        "(-0.788 + 1.030 * s->x)", "(-0.788 + 1.300 * s->x)", [check_star_model]),
}


@pytest.fixture(scope="module")
def mutant_dir(tmp_path_factory):
    return tmp_path_factory.mktemp("oracle_mutants")


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_slip(orc, synth, monkeypatch, mutant_dir, name):
    old, new, checks = MUTANTS[name]
    src = open(os.path.join(os.path.dirname(HERE), "oracle", "ppm_oracle.c")).read()
    assert src.count(old) == 1, "mutation site not found exactly once: %r" % old
    tag = "m%d" % sorted(MUTANTS).index(name)
    c_path = os.path.join(str(mutant_dir), tag + ".c")
    so_path = os.path.join(str(mutant_dir), tag + ".so")
    with open(c_path, "w") as f:
        f.write(src.replace(old, new))
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math",
                           "-fPIC", "-shared", "-o", so_path, c_path, "-lm"])
    monkeypatch.setattr(orc, "_lib", orc.declare(C.CDLL(so_path)))
    monkeypatch.setattr(orc, "_lens_cache", {})
    for check in checks:
        with pytest.raises(AssertionError):
            check(orc, synth)
