"""Finite-difference gradients of the FP64 oracle's log-likelihood.

The parameter order is that of ppm_loglike_grad: M, R_e, inclination, D,
N_H, then (colatitude, azimuth, zeta, logT) of spot 1 and of spot 2.
"""
import copy

import numpy as np

NAMES = ("mass_msun", "radius_km", "incl_rad", "dist_kpc", "nh_1e20",
         "colat_1", "azim_1", "zeta_1", "logT_1", "colat_2", "azim_2", "zeta_2", "logT_2")
# typical scale of each parameter (relative steps and tolerance floors)
SCALE = (1.0, 10.0, 1.0, 0.3, 1.0, 1.0, 1.0, 0.2, 6.0, 1.0, 1.0, 0.2, 6.0)


def n_params(inst):
    return 5 + 4 * inst.n_spots


def get_param(inst, j, b=0):
    if j < 5:
        return float(getattr(inst, NAMES[j])[b])
    s, q = divmod(j - 5, 4)
    return float(getattr(inst, ("colat", "azim", "zeta", "logT")[q])[b, s])


def set_param(inst, j, val, b=0):
    if j < 5:
        getattr(inst, NAMES[j])[b] = val
    else:
        s, q = divmod(j - 5, 4)
        getattr(inst, ("colat", "azim", "zeta", "logT")[q])[b, s] = val


def single(w, b):
    """Workload holding instance b of w alone (counts rows of b)."""
    w2 = copy.copy(w)
    w2.inst = w.inst.select([b])
    r0 = int(np.sum(w.inst.n_phase[:b]))
    w2.counts = w.counts[r0:r0 + int(w.inst.n_phase[b])]
    return w2


def oracle_ll(orc, w, inst=None):
    """FP64 oracle logL of instance 0 of w (optionally with replaced params)."""
    w2 = copy.copy(w)
    if inst is not None:
        w2.inst = inst
    Ft = orc.profile(w2, b=0)
    C = orc.counts_model(Ft, w.R, w.sigma_ism, float(w2.inst.nh_1e20[0]))
    return orc.loglike(C, w.counts[:w2.inst.n_phase[0]], w.tau)


def oracle_fd(orc, w, rel=1e-5, stencil=2):
    """Central differences (2-point, or 4-point with stencil=4) of the oracle
    logL of instance 0; step rel x max(|theta_j|, SCALE_j / 10)."""
    g = np.zeros(n_params(w.inst))
    for j in range(len(g)):
        th = get_param(w.inst, j)
        h = rel * max(abs(th), SCALE[j] / 10.0)

        def f(x):
            inst = w.inst.copy()
            set_param(inst, j, x)
            return oracle_ll(orc, w, inst)

        if stencil == 2:
            g[j] = (f(th + h) - f(th - h)) / (2.0 * h)
        else:
            g[j] = (8.0 * (f(th + h) - f(th - h)) - (f(th + 2 * h) - f(th - 2 * h))) / (12.0 * h)
    return g


def grad_tol(ref, rtol=1e-3, floor=1e-5):
    """Per-component tolerance: rtol relative, plus a floor of `floor` times the
    largest scale-weighted component (for components near zero)."""
    ref = np.asarray(ref)
    sc = np.asarray(SCALE[:len(ref)])
    big = np.max(np.abs(ref) * sc)
    return rtol * np.abs(ref) + floor * big / sc
