"""GPU lens tables (FP64, built by ppm_build_lens) against the oracle's tables."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _compare(orc, synth, spec):
    import paper_2510_07764_gb300 as ppm
    ctx = ppm.Context(0)
    ctx.build_lens(spec)
    Ca, LF, TD = ctx.get_lens()
    ctx.close()
    L = orc.lens(spec)
    for got, ref in [(Ca, L.Ca), (LF, L.LF), (TD, L.TD)]:
        assert np.array_equal(np.isnan(got), np.isnan(ref))
    m = ~np.isnan(L.Ca)
    assert np.max(np.abs(Ca[m] - L.Ca[m])) < 1e-10
    assert np.max(np.abs(LF[m] - L.LF[m]) / np.abs(L.LF[m])) < 1e-7
    m = ~np.isnan(L.TD)
    assert np.max(np.abs(TD[m] - L.TD[m])) < 2e-11


def test_lens_tables_small_grid(orc, synth, small_lens):
    _compare(orc, synth, small_lens)


def test_lens_tables_default_grid(orc, synth):
    # the grid used by the benchmark: u in [0.15, 0.60], 577 x 1024 and 577 x 512
    _compare(orc, synth, synth.LensSpec())


def test_lens_ragged_and_coarse_march(orc, synth):
    spec = synth.LensSpec(u_min=0.2, u_max=0.55, n_u=37, n_cpsi=129, n_calpha=67,
                          dalpha=np.pi / 700)
    _compare(orc, synth, spec)


def test_lens_rejects_bad_specs(synth):
    import paper_2510_07764_gb300 as ppm
    ctx = ppm.Context(0)
    for bad in [dict(u_max=0.7), dict(n_u=1), dict(cpsi_max=0.9), dict(dalpha=0.5),
                dict(u_min=0.5, u_max=0.4)]:
        spec = synth.LensSpec(**{**vars(synth.LensSpec()), **bad})
        with pytest.raises(ppm.PPMError) as e:
            ctx.build_lens(spec)
        assert e.value.status == ppm.PPM_EINVAL
    ctx.close()
