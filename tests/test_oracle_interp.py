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


# ---- the other strategies of Sect. 4 (a: cubic everywhere, one-sided at the
# edges; b: a with negatives clipped; c: cubic everywhere with the linear edge
# and protected-zone rules of the method)
def poly4(t, seed):
    """A table that is a cubic in each of (logT, logg, mu, ln E)."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(-1, 1, (4, 4))

    def P(lt, lg, mu, lnE):
        x = [(lt - 6.0) / 0.8, (lg - 14.2) / 0.5, mu,
             (lnE - t.lnE[0]) / (t.lnE[-1] - t.lnE[0])]
        v = 1.0
        for a in range(4):
            v = v * sum(c[a, i] * x[a] ** i for i in range(4))
        return 3.0 + v
    T4, G4, M4, E4 = np.meshgrid(t.logT, t.logg, t.mu, t.lnE, indexing="ij")
    t.I = np.ascontiguousarray(P(T4, G4, M4, E4).astype(np.float32))
    return P


def test_strategy_a_reproduces_cubics_everywhere(orc, synth):
    """One-sided four-node stencils are exact for cubics up to the table edges,
    including the small-mu intervals the method protects."""
    t = synth.atm_table(n_T=6, n_g=5, n_mu=12, n_E=14)
    P = poly4(t, 11)
    A = orc.Atm(t, "a")
    rng = np.random.default_rng(12)
    for _ in range(300):
        q = [rng.uniform(ax[0], ax[-1]) for ax in (t.logT, t.logg, t.mu, t.lnE)]
        assert A.interp(q[0], q[1], q[2], math.exp(q[3])) == pytest.approx(P(*q), abs=2e-5)


def test_strategy_c_cubic_inside_linear_at_edges(orc, synth):
    t = synth.atm_table(n_T=6, n_g=5, n_mu=12, n_E=14)
    P = poly4(t, 13)
    A = orc.Atm(t, "c")
    D = orc.Atm(t, "d")
    rng = np.random.default_rng(14)
    for _ in range(300):
        q = [rng.uniform(ax[1], ax[-2]) for ax in (t.logT, t.logg, t.lnE)]
        m = rng.uniform(t.mu[3], t.mu[-2])
        assert A.interp(q[0], q[1], m, math.exp(q[2])) == pytest.approx(P(q[0], q[1], m, q[2]),
                                                                       abs=2e-5)
    # protected small-mu zone and the ln E edges: the method's linear rules,
    # so with logT and logg on nodes (where cubic and linear agree) c equals d
    for _ in range(100):
        lt, lg = t.logT[2], t.logg[3]
        m = rng.uniform(t.mu[0], t.mu[3])
        le = rng.uniform(t.lnE[0], t.lnE[1])
        assert A.interp(lt, lg, m, math.exp(le)) == pytest.approx(
            D.interp(lt, lg, m, math.exp(le)), rel=1e-12, abs=1e-12)


def test_strategy_b_clips_what_a_overshoots(orc, synth):
    """A table with a sharp drop toward mu -> 0 (steep limb darkening): the
    one-sided cubic undershoots below zero between the first nodes, the clipped
    variant returns max(a, 0), and the method's protected linear zone stays
    between the node values."""
    t = synth.atm_table(n_T=5, n_g=4, n_mu=12, n_E=10)
    mu = t.mu
    prof = np.where(mu < mu[2], 0.0, 1.0) + 0.0 * mu
    prof[2] = 0.02
    t.I = np.ascontiguousarray(np.broadcast_to(prof[None, None, :, None], t.I.shape)
                               .astype(np.float32))
    Aa, Ab, Ad = orc.Atm(t, "a"), orc.Atm(t, "b"), orc.Atm(t, "d")
    lt, lg, E = t.logT[1], t.logg[1], math.exp(t.lnE[4])
    ms = np.linspace(mu[0], mu[4], 200)
    va = np.array([Aa.interp(lt, lg, m, E) for m in ms])
    vb = np.array([Ab.interp(lt, lg, m, E) for m in ms])
    vd = np.array([Ad.interp(lt, lg, m, E) for m in ms])
    assert va.min() < -1e-3
    assert np.array_equal(vb, np.maximum(va, 0.0))
    prot = ms <= mu[3]
    assert vd[prot].min() >= 0.0 and vd[prot].max() <= 1.0 + 1e-6


@pytest.mark.parametrize("strategy", ["a", "b", "c", "d"])
def test_every_strategy_returns_node_values(orc, synth, strategy):
    t = synth.atm_table(n_T=5, n_g=4, n_mu=10, n_E=12)
    rng = np.random.default_rng(21)
    t.I = np.ascontiguousarray(rng.uniform(-1.0, 2.0, t.I.shape).astype(np.float32))
    A = orc.Atm(t, strategy)
    for _ in range(60):
        i = [rng.integers(0, len(ax)) for ax in (t.logT, t.logg, t.mu, t.lnE)]
        v = float(t.I[i[0], i[1], i[2], i[3]])
        got = A.interp(t.logT[i[0]], t.logg[i[1]], t.mu[i[2]], math.exp(t.lnE[i[3]]))
        assert got == pytest.approx(max(v, 0.0) if strategy == "b" else v, abs=1e-12)
