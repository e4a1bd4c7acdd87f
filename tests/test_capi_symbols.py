"""The C-ABI library builds, loads and exports every symbol include/heat.h declares.
CPU only: no compute call is made."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_]+\s*\*?\s*([a-z_0-9]+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1912_03744_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared("heat.h")
    assert "heat_create" in names and "heat_step" in names and len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n


def test_binding_symbol_list_matches_header():
    from paper_1912_03744_gb300.heat import SYMBOLS
    assert sorted(SYMBOLS) == _declared("heat.h")


def test_surrogate_symbols_exported_and_bound(lib):
    from paper_1912_03744_gb300.surrogate import SURR_SYMBOLS
    names = _declared("surrogate.h")
    assert sorted(SURR_SYMBOLS) == names and len(names) == 12
    for n in names:
        assert hasattr(lib, n), n


def test_surrogate_arguments_rejected_without_gpu():
    from paper_1912_03744_gb300 import surrogate as sg
    L = sg._lib()
    h = ctypes.c_void_p()
    assert L.surr_create(None, None, None, 0, 1.0, 1, 1, None, ctypes.byref(h)) == -1
    assert L.surr_forward(None, None, 1, None, 0) == -1
    assert L.surr_adam(None, 1e-3, 0.9, 0.999, 1e-8) == -1
    assert L.surr_n_params(None) == 0


def test_strerror_without_gpu(lib):
    lib.heat_strerror.restype = ctypes.c_char_p
    assert lib.heat_strerror(0) == b"ok"
    assert lib.heat_strerror(-1) == b"invalid argument"


def test_invalid_arguments_rejected_without_gpu(lib):
    """heat_create validates on the host before touching the device."""
    from paper_1912_03744_gb300 import heat as hb
    hb.load()
    L = hb._lib
    h = ctypes.c_void_p()
    assert L.heat_create(None, None, None, 1.0, None, ctypes.byref(h)) == -1
    assert L.heat_step(None, 1) == -1
    assert L.heat_sweep(None, 0) == -1


def test_batch_arguments_rejected_without_gpu():
    from paper_1912_03744_gb300 import heat as hb
    L = hb.load()
    h = ctypes.c_void_p()
    assert L.heat_batch_create(0, None, None, None, None, None, ctypes.byref(h)) == -1
    assert L.heat_batch_create(1, None, None, None, None, None, None) == -1
    assert L.heat_batch_step(None, 1) == -1
    assert L.heat_batch_tune(None, 1, None) == -1
    assert L.heat_batch_set_tuning(None, 8, 0, 0) == -1
    assert L.heat_batch_member(None, 0, ctypes.byref(h)) == -1
    assert L.heat_batch_launches_per_step(None) == -1
