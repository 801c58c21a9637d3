"""The bounds-checked build (libppm_check.so, -DPPM_BOUNDS_CHECK) runs the
forward, likelihood and gradient paths on workloads that reach the table
edges, the node-major and moment walks (with and without elements leaving
the table), the HEALPix mesh and a temperature map, and reports no failed
index check through ppm_sync; its results equal the ordinary build's."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import sys, numpy as np, torch
sys.path.insert(0, %(root)r); sys.path.insert(0, %(tests)r)
import paper_2510_07764_gb300 as ppm
from paper_2510_07764_gb300 import synth
from gpu_helpers import context
atm = synth.atm_table()
lens = synth.LensSpec(u_min=0.30, u_max=0.40, n_u=129, n_cpsi=512)
out = {}
w = synth.atm_two_spot(n_theta=12, n_phi=16, n_phase=32, n_E=40, n_chan=20, atm=atm, lens=lens)
w.E_keV = synth.logspace(0.06, 9.5, 40)
w.R = synth.response(w.E_keV, 20)
w.sigma_ism = synth.sigma_ism(w.E_keV)
for s in "dab":
    w.interp = s
    ctx = context(w)
    dp = ppm.DeviceParams(w.inst)
    cnt = torch.from_numpy(w.counts).cuda()
    ll, g = ctx.loglike_grad(dp, cnt, w.tau)
    ctx.sync()
    out["grad_" + s] = g.cpu().numpy()
    out["Ft_" + s] = ctx.profile(dp).cpu().numpy()
    ctx.sync()
# uniform ln E grids of 0.49 and 0.45 table node per step: the node-major walks
# (walk 2) of the forward and backward, the second with elements leaving the table top
for name, (lo, hi, n) in {"nw": (0.5, 6.0, 159), "nwedge": (3.5, 7.8, 56)}.items():
    v = synth.atm_two_spot(n_theta=12, n_phi=40, n_phase=24, n_E=n, n_chan=20, atm=atm, lens=lens)
    v.E_keV = synth.logspace(lo, hi, n)
    v.R = synth.response(v.E_keV, 20)
    v.sigma_ism = synth.sigma_ism(v.E_keV)
    for s in "db":
        v.interp = s
        ctx = context(v)
        ctx.set_tiles(walk=2)
        dp = ppm.DeviceParams(v.inst)
        cnt = torch.from_numpy(v.counts).cuda()
        ll, g = ctx.loglike_grad(dp, cnt, v.tau)
        ctx.sync()
        out[name + "_grad_" + s] = g.cpu().numpy()
        out[name + "_Ft_" + s] = ctx.profile(dp).cpu().numpy()
        ctx.sync()
        ctx.set_tiles()
c = synth.crescent_extreme(n_theta=24, n_phi=24, n_phase=32, n_E=48, n_chan=8, atm=atm)
ctx = context(c)
out["crescent"] = ctx.profile(ppm.DeviceParams(c.inst)).cpu().numpy()
ctx.sync()
# the moment walk (the default): both table edges, groups wider than a node, the crescent
for name, (lo, hi, n, spin, zeta) in {"mw": (0.5, 6.0, 159, 205.0, None),
                                      "mwlow": (0.052, 0.32, 58, 205.0, None),
                                      "mwedge": (3.5, 7.8, 56, 205.0, None),
                                      "mwwide": (0.6, 2.6, 96, 600.0, [0.6, 0.7]),
                                      "mwfine": (0.6, 2.6, 900, 205.0, None)}.items():
    v = synth.atm_two_spot(n_theta=12, n_phi=40, n_phase=24, n_E=n, n_chan=20, atm=atm, lens=lens)
    v.E_keV = synth.logspace(lo, hi, n)
    v.inst.spin_hz[:] = spin
    if zeta is not None:
        v.inst.zeta[0] = zeta
    for s in "da":
        v.interp = s
        ctx = context(v)
        out[name + "_Ft_" + s] = ctx.profile(ppm.DeviceParams(v.inst)).cpu().numpy()
        ctx.sync()
c = synth.crescent_extreme(n_theta=24, n_phi=96, n_phase=32, n_E=300, n_chan=8, atm=atm)
ctx = context(c)
out["crescent_mw"] = ctx.profile(ppm.DeviceParams(c.inst)).cpu().numpy()
ctx.sync()
hm = synth.healpix_map(n_side=8, n_phase=16, n_E=96, n_chan=8, atm=atm, lens=lens)
hm.E_keV = synth.logspace(0.6, 2.6, 96)
hm.R = synth.response(hm.E_keV, 8)
hm.sigma_ism = synth.sigma_ism(hm.E_keV)
ctx = context(hm)
out["atm_map_nodes"] = ctx.profile(ppm.DeviceParams(hm.inst)).cpu().numpy()
ctx.sync()
m = synth.bb_small(n_phase=16, n_E=16, lens=lens)
m.inst.grid = 1; m.inst.n_theta[:] = 12; m.inst.n_phi[:] = 48
m.inst.logT_map = np.full((1, 12 * 144), 6.05)
ctx = context(m)
out["map"] = ctx.profile(ppm.DeviceParams(m.inst)).cpu().numpy()
ctx.sync()
np.savez(sys.argv[1], **out)
print("ok")
'''


def _run(tmp_path, lib):
    script = tmp_path / "run.py"
    script.write_text(SCRIPT % {"root": ROOT, "tests": os.path.join(ROOT, "tests")})
    out = tmp_path / ("%s.npz" % os.path.basename(lib))
    env = dict(os.environ, PPM_LIB_PATH=lib)
    r = subprocess.run([sys.executable, str(script), str(out)], env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0 and "ok" in r.stdout, r.stdout + r.stderr
    import numpy as np
    return dict(np.load(out))


def test_bounds_checked_build_reports_no_violation(tmp_path):
    from paper_2510_07764_gb300 import build
    checked = build.build(check=True)
    a = _run(tmp_path, checked)             # ppm_sync raises on a failed check
    b = _run(tmp_path, build.build())
    import numpy as np
    for k in a:
        assert np.allclose(a[k], b[k], rtol=1e-6, atol=0, equal_nan=True), k
