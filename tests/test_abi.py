"""The C-ABI library builds for sm_103a and exports every entry point that
include/rt.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    with open(os.path.join(ROOT, "include", "rt.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rt_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for required in ("rt_create", "rt_init_mesh", "rt_set_sources", "rt_step", "rt_get_fields", "rt_destroy",
                     "rt_set_gas", "rt_set_radiation", "rt_sync", "rt_last_error"):
        assert required in syms


def test_library_exports_every_declared_symbol():
    from paper_2404_17630_gb300 import _build
    path = _build.build()
    lib = ctypes.CDLL(path)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing
    # the build targets sm_103a only
    assert "arch=compute_103a,code=sm_103a" in " ".join(_build.NVCC_FLAGS)


def test_binding_has_the_c_names():
    import paper_2404_17630_gb300.rt as rt
    for s in declared_symbols():
        assert hasattr(rt, s), s


def test_no_gpu_fails_loudly():
    """Without a CUDA device the library refuses with a status code and a
    message (no host fallback computes anything in its place)."""
    import pytest
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2404_17630_gb300 import RT, make_config
    from paper_2404_17630_gb300 import rt as rtb
    with pytest.raises(rtb.RTError) as e:
        RT(make_config(n_bins=3))
    assert "RT_CUDA" in str(e.value)
