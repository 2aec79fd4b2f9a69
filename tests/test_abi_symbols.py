"""The C-ABI library loads and exports every entry point include/grmhd.h
declares (no compute: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if not f.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(grmhd_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2205_02484_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("grmhd_init_grid", "grmhd_set_metric", "grmhd_init_torus", "grmhd_step",
              "grmhd_con2prim", "grmhd_diagnostics", "grmhd_set_state", "grmhd_get_state",
              "grmhd_destroy", "grmhd_sync"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2205_02484_gb300 import grmhd
    assert _declared() <= set(grmhd.SIGNATURES)


def test_version_without_gpu(lib):
    from paper_2205_02484_gb300 import grmhd
    assert "sm_103a" in grmhd.version()


def test_init_grid_rejects_bad_parameters_without_gpu():
    from paper_2205_02484_gb300 import grmhd
    g = grmhd.default_grid(0, 8, 1)
    with pytest.raises(grmhd.GrmhdError) as e:
        grmhd.init_grid(g, grmhd.default_phys())
    assert e.value.code == -1
