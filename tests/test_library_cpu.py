"""Host-side checks of the C-ABI library that need no GPU: it builds, loads,
exports every entry point include/dgswe.h declares, and its argument checks
answer without touching a device."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2303_11767_gb300 import build as libbuild
from paper_2303_11767_gb300 import dgswe, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dgswe.h")


def header_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dg_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def L():
    libbuild.build()
    return dgswe.lib()


def test_header_declares_the_boundary():
    names = header_functions()
    for required in ("dg_create", "dg_destroy", "dg_set_state", "dg_get_state", "dg_rhs", "dg_step",
                     "dg_total_mass", "dg_max_dt", "dg_project_nodal", "dg_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(L):
    for name in header_functions():
        assert hasattr(L, name), name
    assert set(header_functions()) == set(dgswe.SIGNATURES), "binding and header disagree"


def test_argument_checks_without_a_device(L):
    h = ctypes.c_void_p()
    assert L.dg_create(0, 10, 1, 1.0, 1.0, 0.0, ctypes.byref(h)) == dgswe.DG_EINVAL
    assert not h.value
    assert b"nlon" in L.dg_last_error(None)
    assert L.dg_create(20, 10, 7, 1.0, 1.0, 0.0, ctypes.byref(h)) == dgswe.DG_EINVAL
    assert L.dg_create(20, 10, 1, -1.0, 1.0, 0.0, ctypes.byref(h)) == dgswe.DG_EINVAL
    assert L.dg_create(20, 10, 1, 1.0, 1.0, 0.0, None) == dgswe.DG_EINVAL
    assert L.dg_state_len(None) == 0
    assert L.dg_destroy(None) == dgswe.DG_OK
    assert L.dg_step(None, 1, 1.0) == dgswe.DG_EINVAL
    assert L.dg_set_option(None, 1, 0) == dgswe.DG_EINVAL


def test_binding_fails_loudly_without_the_library(tmp_path):
    saved = dgswe._lib
    try:
        dgswe._lib = None
        with pytest.raises(ImportError):
            dgswe.lib(str(tmp_path / "missing.so"))
    finally:
        dgswe._lib = saved


def test_synthetic_fields_are_seeded_and_in_range():
    a = synth.SmoothField(2)
    b = synth.SmoothField(2)
    lam = np.linspace(0, 2 * np.pi, 40)
    th = np.linspace(-np.pi / 2, np.pi / 2, 21)
    for x, y in zip(a.fields_grid(lam, th), b.fields_grid(lam, th)):
        np.testing.assert_array_equal(x, y)
    h, hu, hv = a.fields_grid(lam, th)
    assert abs(h - synth.H0).max() <= synth.H_AMP * (1 + 1e-12)
    speed = np.hypot(hu / h, hv / h)
    assert speed.max() <= synth.U_MAX * 1.01
    assert not np.allclose(synth.SmoothField(3).fields_grid(lam, th)[0], h)
