"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/mcx.h declares; argument checks that run before any device work behave as the
header documents.  No compute call is made here (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1711_03244_gb300 import build
    build.build()
    import paper_1711_03244_gb300 as m
    return m, m.load()


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "mcx.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mcx_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    m, L = lib
    names = _declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(L, n), n
    # and the binding covers them all with signatures
    assert set(names) == set(m.SIGNATURES)


def test_library_is_built_for_sm_103a_only():
    from paper_1711_03244_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_struct_layouts_match_binding(lib):
    m, L = lib
    cfg = m.McxRunCfg()
    L.mcx_run_cfg_default(ctypes.byref(cfg))
    assert cfg.struct_size == ctypes.sizeof(m.McxRunCfg)
    assert cfg.n_gates == 1 and abs(cfg.rr_threshold - 1e-4) < 1e-9 and cfg.rr_m == 10.0
    assert cfg.accum_mode == 2 and cfg.precision == 0
    assert ctypes.sizeof(m.McxExit) == 40
    assert L.mcx_abi_version() == 1


def test_status_strings(lib):
    m, L = lib
    for st in (0, -1, -2, -3, -4, -5, -6):
        assert L.mcx_status_string(st)


def test_argument_errors_before_device_work(lib):
    m, L = lib
    h = ctypes.c_void_p()
    lab = (ctypes.c_uint8 * 8)()
    assert L.mcx_create_volume(None, 2, 2, 2, 1.0, lab, 0) == m.MCX_E_ARG
    assert L.mcx_create_volume(ctypes.byref(h), 2, 2, 2, 1.0, None, 0) == m.MCX_E_ARG
    assert L.mcx_create_volume(ctypes.byref(h), 0, 2, 2, 1.0, lab, 0) == m.MCX_E_ARG
    assert L.mcx_create_volume(ctypes.byref(h), 2, 2, 2, -1.0, lab, 0) == m.MCX_E_ARG
    assert L.mcx_create_volume(ctypes.byref(h), 65536, 65536, 2, 1.0, lab, 0) == m.MCX_E_ARG
    assert b"2^32" in L.mcx_last_error(None)
    assert L.mcx_set_media(None, 1, None) == m.MCX_E_ARG
    assert L.mcx_run(None, None) == m.MCX_E_ARG
    assert L.mcx_debug_primitive(7, 1, None, None) == m.MCX_E_ARG
    L.mcx_destroy(None)


def test_missing_library_fails_loudly(tmp_path):
    import paper_1711_03244_gb300 as m
    saved = m._lib
    m._lib = None
    try:
        with pytest.raises(ImportError):
            m.load(str(tmp_path / "nope.so"))
    finally:
        m._lib = saved
