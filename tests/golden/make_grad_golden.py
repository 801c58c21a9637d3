"""Write tests/golden/grad_batch_full.json: the FP64 oracle's log-likelihood
and its derivatives for instances of the differentiated workload at full
resolution (1024 two-cap instances, 128 x 128 elements per spot, 128 phases,
256 energies, 300 channels, default lens grid; seed as in synth.grad_batch).

For each stored instance: logL, the 13-component gradient by forward mode
(one complex-step run of the oracle per parameter: M, R_e, i, D, N_H, then
colatitude, azimuth, zeta and logT of each spot), and three directional
derivatives along seeded directions, each from its own forward-mode run.

Calls only oracle/ (and the seeded input generators).  One run takes three
to six minutes of one core; the runs are spread over a process pool (spawn).
Records of INSTANCES already in the output file are kept (--fresh recomputes
them all).
Usage: python tests/golden/make_grad_golden.py [n_workers] [--fresh]
"""
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "grad_batch_full.json")
# instances whose logL is finite (instances 1 and 3 have bins with counts and
# no model flux, logL = -inf, and no gradient)
INSTANCES = (0, 2, 4)
N_DIR = 3
SEED_DIR = 2510
# typical scale of each parameter (the same weights the gradient tests use)
SCALE = np.array([1.0, 10.0, 1.0, 0.3, 1.0, 1.0, 1.0, 0.2, 6.0, 1.0, 1.0, 0.2, 6.0])


def directions():
    rng = np.random.Generator(np.random.PCG64(SEED_DIR))
    return [rng.standard_normal(13) * SCALE for _ in range(N_DIR)]


def _job(args):
    b, v = args
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2510_07764_gb300 import synth
    w = synth.grad_batch()
    t = time.time()
    ll, dv = oracle.loglike_tangent(w, v, b=b)
    return b, list(v), float(ll), float(dv), time.time() - t


def main(n_workers, fresh=False):
    sys.path.insert(0, ROOT)
    import oracle
    oracle.build()
    have = {}
    if not fresh and os.path.exists(OUT):
        old = json.load(open(OUT))
        have = {r["b"]: r for r in old["instances"] if r["b"] in INSTANCES}
        cpu_old = old.get("cpu_seconds", 0.0) * len(have) / max(len(old["instances"]), 1)
    else:
        cpu_old = 0.0
    todo = [b for b in INSTANCES if b not in have]
    jobs = []
    for b in todo:
        for j in range(13):
            jobs.append((b, np.eye(13)[j]))
        for v in directions():
            jobs.append((b, v))
    ctx = mp.get_context("spawn")
    with ctx.Pool(n_workers) as pool:
        res = pool.map(_job, jobs, chunksize=1)
    out = {"workload": "grad_batch: 1024 two-cap instances, 128x128 elements per spot, "
                       "128 phases, 256 energies, 300 channels, default lens grid",
           "written_by": "tests/golden/make_grad_golden.py (oracle forward mode only)",
           "parameters": ["M", "R_e", "i", "D", "N_H", "colat_1", "azim_1", "zeta_1",
                          "logT_1", "colat_2", "azim_2", "zeta_2", "logT_2"],
           "cpu_seconds": cpu_old + float(sum(r[4] for r in res)),
           "instances": []}
    for b in INSTANCES:
        if b in have:
            out["instances"].append(have[b])
            continue
        rs = [r for r in res if r[0] == b]
        g = [r[3] for r in rs[:13]]
        lls = [r[2] for r in rs]
        out["instances"].append({
            "b": b, "logL": lls[0], "grad": g,
            "directions": [r[1] for r in rs[13:]],
            "directional": [r[3] for r in rs[13:]]})
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", OUT)


if __name__ == "__main__":
    nums = [a for a in sys.argv[1:] if a.isdigit()]
    main(int(nums[0]) if nums else max(1, os.cpu_count() - 1), fresh="--fresh" in sys.argv)
