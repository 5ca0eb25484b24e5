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


BAD_CONFIGS = [
    (dict(n_bins=0), "n_bins"), (dict(n_bins=4), "n_bins"), (dict(precision=7), "precision"),
    (dict(c_red=0.0), "c_red"), (dict(c_red=float("nan")), "c_red"), (dict(unit_length_cm=-1.0), "unit_length_cm"),
    (dict(cfl=0.0), "cfl"), (dict(box=-1.0), "box"), (dict(chem_mode=3), "chem_mode"), (dict(order=3), "order"),
    (dict(f_s=0.0), "substep"), (dict(f_max=float("nan")), "substep"), (dict(max_substeps=0), "substep"),
    (dict(x_floor=-1e-4), "substep"), (dict(y_he=-0.1), "y_he"), (dict(lim_eps=-1.0), "lim_eps"),
    (dict(gather_sum=2), "gather_sum"), (dict(splitting=2), "splitting"), (dict(time_order=3), "time_order"),
]


def _valid_or_no_device(cfg):
    """rt_create either succeeds (a GPU is present) or stops at the device
    query (none is): in both cases the configuration passed its checks."""
    from paper_2404_17630_gb300 import rt as rtb
    try:
        ctx = rtb.rt_create(cfg)
    except rtb.RTError as e:
        assert e.status == rtb.RT_CUDA, str(e)
        return
    rtb.rt_destroy(ctx)


def test_config_checked_before_any_device_call():
    """Every out-of-range configuration field is refused by rt_create with
    RT_INVALID_ARG and a message naming it, before any CUDA call (so also on
    a host without a GPU); the substep parameters are only checked where the
    chemistry runs."""
    import pytest
    from paper_2404_17630_gb300 import make_config
    from paper_2404_17630_gb300 import rt as rtb
    for kw, word in BAD_CONFIGS:
        with pytest.raises(rtb.RTError) as e:
            rtb.rt_create(make_config(**kw))
        assert e.value.status == rtb.RT_INVALID_ARG, kw
        assert word in str(e.value), (kw, str(e.value))
    _valid_or_no_device(make_config())
    _valid_or_no_device(make_config(chem_mode=0, f_s=0.0, max_substeps=0))
    _valid_or_no_device(make_config(n_bins=1, precision="mixed", order=1, splitting=1, time_order=2))
