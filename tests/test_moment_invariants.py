"""The moment walk of the shift-and-add, replayed on the CPU (no GPU, no
oracle): the kernel's float32 position arithmetic and its index rules for one
group of element slots, against direct evaluation of every slot's cubic in
ln E at every observed energy.

Per group the kernel
  * takes ref = (max X_p + min X_p) / 2 of the slots inside the window
    (X_p = pk_0 + ln z_p / dlnE), N0 = floor(ref), eps_p = X_p - ref (a
    group spread below 0.45 node keeps |eps_p| < 1/2);
  * sums the column weights Omega_j[c] = sum_p eps_p^j w_p[c - s_p] and the
    moments M_j[m] = sum_c Omega_j[c] S[N0 + m][c] of relative nodes
    m = -2 .. rmax + 3, rmax = floor(dref + pk_last - pk_0);
  * replaces, in place and 64 intervals per pass, the moments at index
    r + 1 by the combined cubic of reference interval r;
  * evaluates each energy's cubic at its reference position, and adds the
    fourth-difference terms of the slots on the other side of a node for
    the candidates (energies with tau + emax >= 1 or tau + emin < 0).

The walk is correct only if every slab row it reads lies within the two
zero rows below the table and the three above it, the in-place pass never
overwrites a moment a later interval reads, and the sum equals the direct
evaluation.
"""
import numpy as np
import pytest

f32 = np.float32
LEAD, MARGIN = 2, 3
SPREAD = 0.45


def lagrange(x):
    """4-point Lagrange basis on the nodes -1, 0, 1, 2 at x."""
    return np.array([-x * (x - 1) * (x - 2) / 6, (x + 1) * (x - 1) * (x - 2) / 2,
                     -(x + 1) * x * (x - 2) / 2, (x + 1) * x * (x - 1) / 6])


def coefs(y0, y1, y2, y3):
    c2 = 0.5 * (y0 + y2) - y1
    c3 = (y3 - y0) / 6 + 0.5 * (y1 - y2)
    return np.array([y1, 0.5 * (y2 - y0) - c3, c2, c3])


def moment_walk(S, W, s0, X, pk, terms=True):
    """The kernel's steps for one group; returns the summed spectrum and
    the rows it read (terms=False leaves out the difference terms)."""
    nEt, ncols = S.shape
    pad = np.zeros((nEt + LEAD + MARGIN, ncols))
    pad[LEAD:LEAD + nEt] = S
    rows = []

    def srow(n, c):
        rows.append(n)
        return pad[n + LEAD, c]

    pk0, pkl = pk[0], pk[-1]
    xmax, xmin = X.max(), X.min()
    ref = f32(f32(0.5) * f32(xmax + xmin))
    nf = np.floor(ref)
    dref = f32(ref - nf)
    N0 = int(nf)
    eps = (X - ref).astype(np.float64)
    emax, emin = float(f32(xmax - ref)), float(f32(xmin - ref))
    cmin = int(s0.min())
    ncol = int(s0.max()) - cmin + 4
    rmax = int(np.floor(f32(dref + f32(pkl - pk0))))
    nmom = int(np.ceil(float(pkl) - float(pk0))) + 8
    assert rmax + 6 <= nmom
    cell0 = s0 - cmin
    Om = np.zeros((ncol, 4))
    for c in range(ncol):
        for p in range(len(X)):
            d = c - cell0[p]
            if 0 <= d < 4:
                Om[c] += W[p, d] * eps[p] ** np.arange(4)
    Mv = np.full((nmom, 4), np.nan)
    for m in range(-2, rmax + 4):
        Mv[m + 2] = sum(Om[c] * srow(N0 + m, cmin + c) for c in range(ncol))
    for r0 in range(0, rmax + 1, 64):
        new = {}
        for r in range(r0, min(r0 + 64, rmax + 1)):
            m = Mv[r + 1:r + 5]
            assert not np.isnan(m).any()           # not yet overwritten
            a, b, c2, c3 = (coefs(*m[:, j]) for j in range(4))
            new[r] = [a[0] + b[1] + c2[2] + c3[3], a[1] + 2 * b[2] + 3 * c2[3],
                      a[2] + 3 * b[3], a[3]]
        for r, v in new.items():
            Mv[r + 1] = v
    F = np.zeros(len(pk))
    for k in range(len(pk)):
        y = f32(dref + f32(pk[k] - pk0))
        rf = np.floor(y)
        r, tau = int(rf), float(f32(y - rf))
        assert 0 <= r <= rmax
        P = Mv[r + 1]
        F[k] = P[0] + tau * (P[1] + tau * (P[2] + tau * P[3]))
        if terms and (tau + emax >= 1 or tau + emin < 0):
            up = tau + emax >= 1
            base = r - (1 if up else 2)
            D = np.array([sum(w * srow(N0 + base + j, cmin + c)
                              for j, w in enumerate((1, -4, 6, -4, 1))) for c in range(ncol)])
            for p in range(len(X)):
                t = tau + eps[p]
                if up and t >= 1:
                    g = t * (t - 1) * (t - 2)
                elif not up and t < 0:
                    g = -(t + 1) * t * (t - 1)
                else:
                    assert 0 <= t < 1                # crossings only on the candidate's side
                    g = 0.0
                F[k] += g / 6 * (W[p] @ D[cell0[p]:cell0[p] + 4])
    return F, rows


def direct(S, W, s0, X, pk):
    F = np.zeros(len(pk))
    for p in range(len(X)):
        for k in range(len(pk)):
            x = float(X[p]) + float(pk[k] - pk[0])
            n = int(np.floor(x))
            F[k] += lagrange(x - n) @ (S[n - 1:n + 3, s0[p]:s0[p] + 4] @ W[p])
    return F


def cases(seed, n):
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        nEt, nmu = 60, 20
        K = int(rng.integers(1, 120))
        d = rng.uniform(0.03, 0.99)
        pk = (1.0 + d * np.arange(K) + rng.uniform(0, 0.01, K).cumsum()).astype(f32)
        if not np.all(np.diff(pk) < 0.999):
            continue
        span = float(pk[-1] - pk[0])
        spread = rng.choice([0.0, 0.005, 0.05, 0.2, 0.44])
        hi = nEt - 2 - span - spread - 1e-3
        if hi <= 1.0:
            continue
        X = (rng.uniform(1.0, hi) + rng.uniform(0, spread, 64)).astype(f32)
        X = X[(X >= 1) & (f32(pk[-1]) + f32(X - pk[0]) < nEt - 2)]
        if len(X) == 0 or X.max() - X.min() >= SPREAD:
            continue
        s0 = rng.integers(2, 2 + int(rng.integers(1, 8)), len(X))
        out.append((pk, X, s0, int(rng.integers(1 << 30))))
    return out


@pytest.mark.parametrize("pk,X,s0,seed", cases(21, 40))
def test_moment_walk_equals_direct_and_stays_in_bounds(pk, X, s0, seed):
    rng = np.random.default_rng(seed)
    S = rng.standard_normal((60, 20))
    W = rng.standard_normal((len(X), 4))
    F, rows = moment_walk(S, W, s0, X, pk)
    assert min(rows) >= -LEAD and max(rows) < 60 + MARGIN
    ref = direct(S, W, s0, X.astype(np.float64), pk.astype(np.float64))
    # float32 positions: the reference position and the slots' offsets are
    # rounded differently from X_p + (pk_k - pk_0)
    assert np.max(np.abs(F - ref)) <= 1e-4 * np.max(np.abs(ref))


def test_catches_a_missing_difference_term():
    """Without the fourth-difference terms a group that straddles nodes is
    wrong: the comparison with direct evaluation has the power to see it."""
    rng = np.random.default_rng(5)
    pk = (1.0 + 0.4 * np.arange(80)).astype(f32)
    X = (10.0 + rng.uniform(0, 0.4, 64)).astype(f32)
    s0 = np.full(64, 3)
    S = rng.standard_normal((60, 20))
    W = rng.standard_normal((64, 4))
    ref = direct(S, W, s0, X.astype(np.float64), pk.astype(np.float64))
    F, _ = moment_walk(S, W, s0, X, pk)
    assert np.max(np.abs(F - ref)) <= 1e-4 * np.max(np.abs(ref))
    F0, _ = moment_walk(S, W, s0, X, pk, terms=False)
    assert np.max(np.abs(F0 - ref)) > 1e-3 * np.max(np.abs(ref))
