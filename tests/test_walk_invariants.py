"""Index invariants of the node-major walks of the shift-and-add (forward
and backward), checked on the CPU by replaying the kernels' float32 index
arithmetic for a warp of slots (no GPU, no oracle).

The forward walk moves every slot one table interval per iteration and
stores the values of the two or three energies inside it in a 16-row ring
(row = energy mod 16); every second interval a vote checks whether all
slots have passed the next block of 8 energies and the warp then sums it.
The walk is correct only if

  * every real energy (0 <= k < nE) is written exactly once per slot before
    its block is summed,
  * no write lands on a row that still holds an unsummed real energy,
  * the table rows read stay within the slab plus three margin rows.

The backward walk reads zero-padded adjoints; its indices must stay inside
the padded row (two leading, sixteen trailing entries).
"""
import numpy as np
import pytest

f32 = np.float32
N_T = 166            # table energy nodes of the synthetic atmosphere
LEAD, TAIL, MARGIN = 2, 16, 3


def start(pk0, lz, d):
    """Per-slot start of the walk as the kernels compute it: first interval
    n0, position t in [0, d) of the first (possibly virtual) energy, and its
    index -mv."""
    x0 = f32(pk0 + lz)
    n0 = np.floor(x0)
    f = f32(x0 - n0)
    mv = int(f * f32(f32(1) / d))
    t = f32(f32(-f32(mv) * d) + f)
    if t >= d:
        t = f32(t - d)
        mv += 1
    if t < 0:
        t = f32(t + d)
        mv -= 1
    return int(n0), t, -mv


def forward_walk(nE, d, pk0, lzs, sum_every=2):
    d = f32(d)
    pkl = f32(pk0 + f32((nE - 1) * d))
    S = len(lzs)
    st = [start(pk0, lz, d) for lz in lzs]
    t = np.array([s[1] for s in st], f32)
    k = np.array([s[2] for s in st])
    row = np.array([s[0] + 2 for s in st])          # highest stencil node
    nit = max(int(np.floor(f32(pkl + f32(lz)))) - s[0] + 1 for lz, s in zip(lzs, st)) + 1
    holds = np.full((16, S), -10**9)                # energy each ring row holds
    written = np.zeros((nE, S), int)
    r0 = 0

    def put(e, kk):
        r = kk % 16
        old = holds[r, e]
        assert not (0 <= old < nE and old >= r0 and old != kk), "unsummed row overwritten"
        holds[r, e] = kk
        if 0 <= kk < nE:
            written[kk, e] += 1

    def flush():
        for q in range(r0, min(r0 + 8, nE)):
            assert np.all(holds[q % 16] == q), "block summed before every slot wrote it"

    for it in range(nit):
        t2 = (t + d).astype(f32)
        t3 = (t2 + d).astype(f32)
        third = t3 < f32(1)
        for e in range(S):
            put(e, k[e])
            put(e, k[e] + 1)
            if third[e]:
                put(e, k[e] + 2)
        k = k + np.where(third, 3, 2)
        t = (np.where(third, (t3 + d).astype(f32), t3) - f32(1)).astype(f32)
        row = row + 1
        assert row.max() <= N_T - 1 + MARGIN, "read past the margin rows"
        if it % sum_every == sum_every - 1 and np.all(k >= r0 + 8):
            flush()
            r0 += 8
    while r0 < nE:
        flush()
        r0 += 8
    assert np.all(written == 1), "an energy was missed or written twice"


def backward_walk(nE, d, pk0, lzs):
    d = f32(d)
    pkl = f32(pk0 + f32((nE - 1) * d))
    st = [start(pk0, lz, d) for lz in lzs]
    nit = max(int(np.floor(f32(pkl + f32(lz)))) - s[0] + 1 for lz, s in zip(lzs, st)) + 1
    last = N_T - 1 + MARGIN
    for lz, (n0, t, k0) in zip(lzs, st):
        kidx, seen = LEAD + k0, []
        for i in range(nit):
            t2 = f32(t + d)
            t3 = f32(t2 + d)
            third = t3 < f32(1)
            assert 0 <= kidx and kidx + 2 < nE + LEAD + TAIL, "adjoint index out of the padded row"
            seen += [kidx - LEAD, kidx + 1 - LEAD] + ([kidx + 2 - LEAD] if third else [])
            kidx += 3 if third else 2
            t = f32((f32(t3 + d) if third else t3) - f32(1))
            # interval i retires node n0 - 1 + i (deferred contraction); the
            # cubic form (strategy B) loads node n0 + 3 + i
            assert n0 - 1 + i >= 0 and n0 + 3 + i <= last, "read past the margin rows"
        # after the walk the last three nodes of the window retire
        assert n0 - 1 + nit + 2 <= last, "read past the margin rows"
        real = sorted(q for q in seen if 0 <= q < nE)
        assert real == list(range(nE)), "an energy was missed or repeated"


def cases(seed, n):
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        nE = int(rng.choice([2, 5, 13, 14, 17, 64, 96, 256, 300]))
        d = rng.uniform(0.34, 0.498)
        pk0 = rng.uniform(-40.0, 10.0)
        lo = 1.0 - pk0
        hi = N_T - 2 - pk0 - (nE - 1) * d
        if hi - lo < 1e-2:
            continue
        lzs = rng.uniform(lo, hi - 1e-3, 64)
        # starts on and just below table nodes, and the lz used by idle lanes
        lzs[:6] = np.floor(lzs[:6]) + np.array([0.0, 1e-7, 0.9999999, 0.5, 0.25, 0.75])
        lzs[6] = 1.25 - pk0
        lzs = np.clip(lzs, lo, hi - 1e-3).astype(f32)
        out.append((nE, f32(d), f32(pk0), lzs))
    return out


@pytest.mark.parametrize("nE,d,pk0,lzs", cases(11, 60))
def test_forward_ring_invariants(nE, d, pk0, lzs):
    forward_walk(nE, d, pk0, lzs)


@pytest.mark.parametrize("nE,d,pk0,lzs", cases(12, 40))
def test_backward_padding_invariants(nE, d, pk0, lzs):
    backward_walk(nE, d, pk0, lzs[:32])


def test_catches_a_ring_overrun():
    """The check has teeth: summing blocks only every fourth interval
    overruns the 16-row ring on some grids."""
    hit = 0
    for nE, d, pk0, lzs in cases(13, 40):
        try:
            forward_walk(nE, d, pk0, lzs, sum_every=4)
        except AssertionError:
            hit += 1
    assert hit > 0
