"""Host-side checks of the C-ABI library (no GPU needed): it builds for sm_103a, loads, exports
every entry point include/lbm.h declares, agrees with the binding on the config layout, and
rejects bad configurations before touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1311_7239_gb300 import build, lbm

    build.build()
    return lbm.lib()


def _declared():
    txt = open(os.path.join(ROOT, "include", "lbm.h")).read()
    return re.findall(r"^LBM_API\s+[\w\s\*]+?\b(lbm_\w+)\s*\(", txt, flags=re.M)


def test_every_declared_symbol_is_exported_and_bound(L):
    from paper_1311_7239_gb300 import lbm

    names = _declared()
    assert len(names) >= 18
    for n in names:
        assert hasattr(L, n), n
        assert n in lbm.SIGNATURES, n
    assert set(lbm.SIGNATURES) == set(names)


def test_config_layout_matches(L):
    from paper_1311_7239_gb300 import lbm

    assert L.lbm_config_size() == ctypes.sizeof(lbm.Config)
    cfg = lbm.default_config()
    assert cfg.abi_version == lbm.ABI_VERSION
    assert (cfg.s_e, cfg.s_q, cfg.J, cfg.rho0) == (1.1, 1.2, 1.0, 1.0)
    assert all(t != t for t in cfg.T_wall)  # NaN = adiabatic


@pytest.mark.parametrize(
    "field,value,code",
    [
        ("abi_version", 99, -6),
        ("nx", 1, -1),
        ("precision", 7, -1),
        ("bc_y", 2, -1),
        ("nu", -0.1, -1),
        ("s_q", 2.5, -1),
        ("phi", 1.5, -1),
        ("dev_scale_log2", 99, -1),
        ("streaming", 2, -1),
        ("options", 2, -1),
    ],
)
def test_create_rejects_bad_configs_without_a_device(L, field, value, code):
    from paper_1311_7239_gb300 import lbm

    cfg = lbm.default_config()
    setattr(cfg, field, value)
    h = ctypes.c_void_p()
    assert L.lbm_create(ctypes.byref(cfg), ctypes.byref(h)) == code
    assert not h.value
    assert L.lbm_last_error()


@pytest.mark.parametrize("bc_x,bc_y", [(2, 1), (3, 1), (1, 3), (0, 3)])
def test_inplace_batch_rejects_extrapolated_sides_without_a_device(L, bc_x, bc_y):
    """A single lattice takes pressure columns and wall nodes with in-place streaming (their states
    are computed before each step); an in-place batch takes periodic and halfway-wall sides only."""
    from paper_1311_7239_gb300 import lbm

    cfgs = (lbm.Config * 2)(lbm.default_config(streaming=lbm.STREAM_INPLACE),
                            lbm.default_config(bc_x=bc_x, bc_y=bc_y, streaming=lbm.STREAM_INPLACE))
    h = ctypes.c_void_p()
    assert L.lbm_batch_create(cfgs, 2, ctypes.byref(h)) == lbm.EINVAL
    assert not h.value and b"in-place" in L.lbm_last_error()


def test_batch_rejects_mixed_streaming_without_a_device(L):
    from paper_1311_7239_gb300 import lbm

    cfgs = (lbm.Config * 2)(lbm.default_config(), lbm.default_config(streaming=lbm.STREAM_INPLACE))
    h = ctypes.c_void_p()
    assert L.lbm_batch_create(cfgs, 2, ctypes.byref(h)) == lbm.EINVAL
    assert L.lbm_create_batch(cfgs, 2, ctypes.byref(h)) == lbm.EINVAL  # the same call under its other name
    assert not h.value and b"streaming" in L.lbm_last_error()


def test_strerror_names_every_code(L):
    for code in (0, -1, -2, -3, -4, -5, -6, -7):
        assert L.lbm_strerror(code) and L.lbm_strerror(code) != b"unknown error"
    assert L.lbm_strerror(-99) == b"unknown error"


def test_null_arguments_are_rejected(L):
    assert L.lbm_step(None, 1) == -1
    assert L.lbm_macros(None, None, None, None, None) == -1
    L.lbm_destroy(None)
