"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/ppm.h (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ppm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ppm_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libppm():
    from paper_2510_07764_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_hot_path(libppm):
    names = declared_functions()
    for required in ["ppm_build_lens", "ppm_profile", "ppm_loglike", "ppm_loglike_grad"]:
        assert required in names


def test_every_declared_symbol_is_exported(libppm):
    from paper_2510_07764_gb300 import _abi
    names = declared_functions()
    for n in names:
        assert hasattr(libppm, n), n
    assert sorted(_abi.EXPORTS) == names


def test_create_without_device_is_an_error(libppm):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2510_07764_gb300 import _abi
    st, h = _abi.ppm_create(0)
    assert st == _abi.PPM_EINVAL and not h.value


def test_null_context_calls_fail_cleanly(libppm):
    from paper_2510_07764_gb300 import _abi
    spec = _abi.ppm_lens_spec(0.3, 0.4, 8, -0.9, 1.0, 8, -0.2, 1.0, 8, 0.01)
    assert _abi.ppm_build_lens(None, spec, None) == _abi.PPM_EINVAL
    assert _abi.ppm_sync(None, None, 1.0) == _abi.PPM_EINVAL
    assert _abi.ppm_last_error(None) == "null context"


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without libppm.so every entry point raises LibraryMissing: there is no
    CPU fallback behind the binding."""
    import paper_2510_07764_gb300 as ppm
    from paper_2510_07764_gb300 import _abi
    monkeypatch.setattr(_abi, "LIB_PATH", str(tmp_path / "libppm.so"))
    monkeypatch.setattr(_abi, "_lib", None)
    with pytest.raises(ppm.LibraryMissing):
        ppm.Context(0)
    with pytest.raises(ppm.LibraryMissing):
        _abi.ppm_sync(None, None, 1.0)


def test_product_path_does_not_import_the_oracle():
    """The package and the benchmark's GPU arm load no module of oracle/."""
    import subprocess
    import sys
    code = ("import sys; sys.path.insert(0, %r); import paper_2510_07764_gb300, "
            "paper_2510_07764_gb300.synth, paper_2510_07764_gb300._abi; "
            "print(any(m == 'oracle' or m.startswith('oracle.') for m in sys.modules))" % ROOT)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                         timeout=300, check=True)
    assert out.stdout.strip() == "False"
