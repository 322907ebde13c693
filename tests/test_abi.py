"""Host-side checks of the C ABI (no GPU needed): the library builds for
sm_103a, loads, and exports every entry point include/rom.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "rom.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rom_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2009_11742_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ["rom_create", "rom_destroy", "rom_run_rank1", "rom_run_rank2",
                 "rom_spectral_radius", "rom_status_string"]:
        assert name in syms


def test_library_exports_every_declared_symbol(lib):
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_names_match_header():
    from paper_2009_11742_gb300 import rom
    assert sorted(rom.EXPORTED) == declared_symbols()
    for s in rom.EXPORTED:
        assert callable(getattr(rom, s, None)), s


def test_status_strings_without_gpu(lib):
    lib.rom_status_string.restype = ctypes.c_char_p
    assert lib.rom_status_string(0) == b"ROM_OK"
    assert b"UNSTABLE" in lib.rom_status_string(4)
    assert lib.rom_version() >= 100


def test_noconv_status_string(lib):
    lib.rom_status_string.restype = ctypes.c_char_p
    assert b"NOCONV" in lib.rom_status_string(8)


def test_noalloc_errors_without_gpu(lib):
    """The allocation-free entry point checks its sizes before any CUDA call,
    and a failing CUDA call is reported through rom_last_error like every
    other entry point's."""
    lib.rom_last_error.restype = ctypes.c_char_p
    rho = ctypes.c_double(0.0)
    fake = ctypes.c_void_p(16)
    assert lib.rom_spectral_radius_noalloc(fake, fake, 4097, 4, ctypes.byref(rho), None) == 1
    assert lib.rom_spectral_radius_noalloc(fake, fake, 0, 4, ctypes.byref(rho), None) == 1
    assert lib.rom_spectral_radius_noalloc(None, fake, 4, 4, ctypes.byref(rho), None) == 1
    import torch
    if torch.cuda.is_available():
        return
    rc = lib.rom_spectral_radius_noalloc(fake, fake, 4, 4, ctypes.byref(rho), None)
    assert rc in (2, 3)  # ROM_E_NOMEM / ROM_E_CUDA: no device to run on
    assert b"rom_spectral_radius_noalloc" in lib.rom_last_error()


def test_null_arguments_rejected_without_gpu(lib):
    """Argument checks happen before any CUDA call."""
    h = ctypes.c_void_p()
    rc = lib.rom_create(None, None, None, None, 4, 4, 0, ctypes.c_double(0.1), 0,
                        ctypes.byref(h), None)
    assert rc == 1  # ROM_E_INVAL
    rc = lib.rom_run_rank2(None, None, None, None, 1, 1, ctypes.c_long(0), 0, None, 1, None)
    assert rc == 1
    assert lib.rom_run_rank3(None, 2, None, None, None, 4, 10, 0, None, 1, None) == 1
    assert lib.rom_set_reference(None, None, None, 4, 0) == 1
    d = ctypes.c_double
    f = ctypes.c_void_p()
    for bad in [(1, 12), (8, 2), (70000, 12)]:  # Nr < 2, Ntheta < 3, Nr > 65535
        rc = lib.rom_fom_create(bad[0], bad[1], d(3480e3), d(6371e3), d(2500.0), d(5000.0),
                                d(0.05), ctypes.byref(f))
        assert rc == 1 and not f.value
    rc = lib.rom_fom_create(8, 12, d(3480e3), d(3000e3), d(2500.0), d(5000.0), d(0.05),
                            ctypes.byref(f))
    assert rc == 1  # r_earth below r_cmb
    assert lib.rom_fom_run(None, None, None, None, 1, 10, ctypes.c_long(0), -1, None, 1, None, 0,
                           0, None, 1, None) == 1
    assert lib.rom_fom_set_passes(None, 1) == 1
    assert lib.rom_fom_dims(None, None, None, None) == 1


def test_missing_library_fails_loudly(tmp_path):
    from paper_2009_11742_gb300 import rom
    with pytest.raises(RuntimeError, match="not found"):
        old = rom._lib
        rom._lib = None
        try:
            rom.load(str(tmp_path / "nope.so"))
        finally:
            rom._lib = old
