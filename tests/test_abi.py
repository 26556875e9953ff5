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
    assert L.mcx_abi_version() == 2


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
    # the bordered device copy must stay below 2^32 voxels: 4094^2 x 256 does not
    assert L.mcx_create_volume(ctypes.byref(h), 4094, 4094, 254, 1.0, lab, 0) == m.MCX_E_ARG
    r = ctypes.c_double()
    assert L.mcx_probe_rate(10, 0, ctypes.byref(r)) == m.MCX_E_ARG
    assert L.mcx_probe_rate(-1, 0, ctypes.byref(r)) == m.MCX_E_ARG
    assert L.mcx_probe_rate(0, 0, None) == m.MCX_E_ARG
    L.mcx_destroy(None)


def test_denoiser_and_batch_argument_errors(lib):
    """The denoiser's shape limits and every NULL handle are rejected with MCX_E_ARG
    before any device work, leaving the output handle NULL."""
    m, L = lib
    d = ctypes.c_void_p()
    assert L.mcx_denoiser_create(None, 64, 64, 64, 1, 0, 0) == m.MCX_E_ARG
    for nx, ny, nz, batch, n_aux in [(60, 64, 64, 1, 0), (256, 64, 64, 1, 0), (64, 6, 64, 1, 0),
                                     (64, 64, 2, 1, 0), (64, 64, 64, 0, 0), (64, 64, 64, 1, 8),
                                     (192, 252, 252, 64, 0)]:
        d.value = None
        assert L.mcx_denoiser_create(ctypes.byref(d), nx, ny, nz, batch, n_aux, 0) == m.MCX_E_ARG
        assert not d.value
    n = ctypes.c_uint64()
    assert L.mcx_denoiser_param_count(None, ctypes.byref(n)) == m.MCX_E_ARG
    assert L.mcx_denoiser_get_params(None, None, 0, 0) == m.MCX_E_ARG
    assert L.mcx_denoiser_set_params(None, None, 0) == m.MCX_E_ARG
    assert L.mcx_denoiser_set_encoding(None, 1e-8, -4.0, 2.0) == m.MCX_E_ARG
    assert L.mcx_denoiser_forward(None, None, None, None, 1, None) == m.MCX_E_ARG
    loss = ctypes.c_float()
    assert L.mcx_denoiser_train_step(None, None, None, None, 1, 1e-3, ctypes.byref(loss), None) == m.MCX_E_ARG
    assert L.mcx_denoiser_encode(None, None, None, 0, None) == m.MCX_E_ARG
    assert L.mcx_denoiser_decode(None, None, None, 0, None) == m.MCX_E_ARG
    assert L.mcx_denoiser_apply(None, None, None, None, 1, None) == m.MCX_E_ARG
    # the debug convolution: the direct input layer takes cin 1 with cout 16 only, and every
    # kind needs a width that is a multiple of 16 (checked before any device work)
    f = (ctypes.c_float * 64)()
    assert L.mcx_debug_conv3d(0, 1, 1, 1, 16, 1, 32, f, f, None, None, f) == m.MCX_E_ARG
    assert L.mcx_debug_conv3d(0, 1, 1, 1, 12, 1, 16, f, f, None, None, f) == m.MCX_E_ARG
    assert L.mcx_debug_conv3d(2, 1, 1, 1, 16, 16, 16, f, f, None, None, f) == m.MCX_E_ARG
    assert L.mcx_debug_conv3d(1, 1, 1, 1, 16, 16, 16, f, None, None, None, f) == m.MCX_E_ARG
    assert L.mcx_denoiser_sync(None) == m.MCX_E_ARG
    L.mcx_denoiser_destroy(None)
    assert L.mcx_batch_create(None) == m.MCX_E_ARG
    assert L.mcx_batch_run(None, None) == m.MCX_E_ARG
    assert L.mcx_batch_sync(None) == m.MCX_E_ARG
    ms = ctypes.c_float()
    assert L.mcx_batch_last_ms(None, ctypes.byref(ms)) == m.MCX_E_ARG
    assert L.mcx_batch_read_fluence(None, 0, None, 0, 0, 0) == m.MCX_E_ARG
    assert L.mcx_batch_read_tally(None, 0, None) == m.MCX_E_ARG
    assert L.mcx_batch_read_stats(None, None) == m.MCX_E_ARG
    assert L.mcx_batch_autotune(None, None, 0.1, ctypes.byref(ms)) == m.MCX_E_ARG
    assert L.mcx_batch_size(None) == 0
    L.mcx_batch_destroy(None)


def test_no_device_is_an_error_not_a_fallback(lib):
    """Without a usable CUDA device every constructor fails with MCX_E_CUDA and leaves its
    handle NULL: the library has no CPU path to fall back on."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    m, L = lib
    h = ctypes.c_void_p()
    lab = (ctypes.c_uint8 * 8)(*([1] * 8))
    assert L.mcx_create_volume(ctypes.byref(h), 2, 2, 2, 1.0, lab, 0) == m.MCX_E_CUDA
    assert not h.value and L.mcx_last_error(None)
    b = ctypes.c_void_p()
    assert L.mcx_batch_create(ctypes.byref(b)) == m.MCX_E_CUDA
    assert not b.value
    d = ctypes.c_void_p()
    assert L.mcx_denoiser_create(ctypes.byref(d), 64, 64, 64, 1, 0, 0) == m.MCX_E_CUDA
    assert not d.value


def test_missing_library_fails_loudly(tmp_path):
    import paper_1711_03244_gb300 as m
    saved = m._lib
    m._lib = None
    try:
        with pytest.raises(ImportError):
            m.load(str(tmp_path / "nope.so"))
    finally:
        m._lib = saved
