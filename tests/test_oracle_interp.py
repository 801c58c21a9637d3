"""Pins of the oracle's mixed-order atmosphere interpolation (Sect. 4).

Reading: linear in logT and logg; cubic Lagrange (actual node positions) in mu
and ln E; linear on the intervals among the 4 protected small-mu nodes and
wherever the 4-node stencil would leave the grid; clamp outside the grid.
A cubic stencil reproduces cubics exactly, a linear one reproduces lines:
polynomial tables of degree (1, 1, 3, 3) and (1, 1, 1, 1) pin the weights,
the index bookkeeping and the zone rules independently of the implementation.
"""
import math

import numpy as np
import pytest


def poly_table(t, deg_mu=3, deg_E=3, seed=0):
    rng = np.random.default_rng(seed)
    cT, cg = rng.uniform(-1, 1, 2)
    cm = rng.uniform(-1, 1, deg_mu + 1)
    ce = rng.uniform(-1, 1, deg_E + 1)

    def P(lt, lg, mu, lnE):
        x = (lnE - t.lnE[0]) / (t.lnE[-1] - t.lnE[0])
        pm = sum(c * mu ** i for i, c in enumerate(cm))
        pe = sum(c * x ** i for i, c in enumerate(ce))
        return 5.0 + cT * (lt - 6.0) + cg * (lg - 14.2) + pm * pe
    T4, G4, M4, E4 = np.meshgrid(t.logT, t.logg, t.mu, t.lnE, indexing="ij")
    t.I = np.ascontiguousarray(P(T4, G4, M4, E4).astype(np.float32))
    return P


@pytest.fixture(scope="module")
def table(synth):
    return synth.atm_table(n_T=6, n_g=4, n_mu=12, n_E=14)


def test_cubic_zone_reproduces_cubics(orc, table):
    P = poly_table(table, 3, 3)
    A = orc.Atm(table)
    rng = np.random.default_rng(5)
    mu, lnE = table.mu, table.lnE
    for _ in range(300):
        lt = rng.uniform(table.logT[0], table.logT[-1])
        lg = rng.uniform(table.logg[0], table.logg[-1])
        m = rng.uniform(mu[3], mu[-2])          # intervals 3 .. n-3: cubic in mu
        le = rng.uniform(lnE[1], lnE[-2])       # intervals 1 .. n-3: cubic in E
        got = A.interp(lt, lg, m, math.exp(le))
        assert got == pytest.approx(P(lt, lg, m, le), abs=3e-6 * 10)


def test_linear_tables_exact_everywhere(orc, table):
    P = poly_table(table, 1, 1, seed=3)
    A = orc.Atm(table)
    rng = np.random.default_rng(6)
    for _ in range(300):
        lt = rng.uniform(table.logT[0], table.logT[-1])
        lg = rng.uniform(table.logg[0], table.logg[-1])
        m = rng.uniform(table.mu[0], table.mu[-1])
        le = rng.uniform(table.lnE[0], table.lnE[-1])
        assert A.interp(lt, lg, m, math.exp(le)) == pytest.approx(P(lt, lg, m, le), abs=3e-5)


def test_protected_zone_is_linear(orc, table):
    """With a table cubic in mu, queries among the 4 smallest mu nodes must be the
    straight line between the bracketing nodes (a cubic would differ)."""
    mu = table.mu
    s = mu[3]
    P = lambda m: 10.0 * (m / s) ** 3 - 4.0 * (m / s) ** 2 + 1.0
    I = np.broadcast_to(P(mu)[None, None, :, None], table.I.shape)
    table.I = np.ascontiguousarray(I.astype(np.float32))
    A = orc.Atm(table)
    lt, lg, E = table.logT[2], table.logg[1], math.exp(table.lnE[5])
    nodes = P(mu[:4])
    cubic_differs = 0
    for m in np.linspace(mu[0], mu[3], 41)[1:-1]:
        lin = np.interp(m, mu[:4], nodes)
        got = A.interp(lt, lg, m, E)
        assert got == pytest.approx(lin, abs=3e-5)
        cubic_differs += abs(P(m) - lin) > 1e-2
    assert cubic_differs > 5
    # first cubic interval (mu_3 .. mu_4) uses the stencil 2..5: exact on cubics
    m = 0.5 * (mu[3] + mu[4])
    assert A.interp(lt, lg, m, E) == pytest.approx(P(m), rel=1e-5)


def test_energy_edges_are_linear(orc, table):
    P = poly_table(table, 1, 3, seed=9)
    A = orc.Atm(table)
    lt, lg, m = table.logT[1], table.logg[2], table.mu[6]
    for lo, hi in [(0, 1), (len(table.lnE) - 2, len(table.lnE) - 1)]:
        le = 0.3 * table.lnE[lo] + 0.7 * table.lnE[hi]
        lin = 0.3 * P(lt, lg, m, table.lnE[lo]) + 0.7 * P(lt, lg, m, table.lnE[hi])
        assert A.interp(lt, lg, m, math.exp(le)) == pytest.approx(lin, abs=3e-5)


def test_nodes_and_clamping(orc, table):
    poly_table(table, 3, 3, seed=11)
    A = orc.Atm(table)
    I = table.I
    for (a, b, c, d) in [(0, 0, 0, 0), (5, 3, 11, 13), (2, 1, 6, 7), (3, 2, 2, 0)]:
        got = A.interp(table.logT[a], table.logg[b], table.mu[c], math.exp(table.lnE[d]))
        assert got == pytest.approx(float(I[a, b, c, d]), rel=1e-6)
    # below the smallest mu / above the largest energy: the edge node value
    got = A.interp(table.logT[1], table.logg[1], 0.0, 1e3)
    assert got == pytest.approx(float(I[1, 1, 0, -1]), rel=1e-6)


def test_negative_overshoot_is_kept(orc, table):
    """A kink in mu makes a cubic stencil overshoot below zero; the mixed scheme
    keeps negative interpolants (clipping is a different strategy)."""
    t = table
    I = np.zeros_like(t.I)
    I[:, :, 7:, :] = 1.0                      # step between mu_6 and mu_7
    t.I = I
    A = orc.Atm(t)
    m = t.mu[5] + 0.5 * (t.mu[6] - t.mu[5])   # interval 5: stencil 4..7 sees the step
    assert A.interp(t.logT[1], t.logg[1], m, math.exp(t.lnE[4])) < 0.0
