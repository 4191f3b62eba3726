"""The C-ABI library builds for sm_103a, loads, and exports every entry point of include/dlra.h.

No compute call is made: these run on a machine without a GPU.
"""
import os
import re

import pytest

from paper_2508_04484_gb300 import build as B
from paper_2508_04484_gb300 import dlra as D
from paper_2508_04484_gb300 import workloads as WL

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return D.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "dlra.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dlra_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("dlra_init", "dlra_set_materials", "dlra_add_beam", "dlra_step", "dlra_dose"):
        assert required in names
    assert set(names) == set(D.SIGNATURES), "binding and header disagree"


def test_library_exports_every_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_library_is_sm103a():
    # the build targets sm_103a only
    assert "arch=compute_103a,code=sm_103a" in " ".join(B.ARCH)


def _init_status(**kw):
    cfg = WL.base_config(**kw)
    c, keep = D.make_config(cfg)
    h = D._P()
    return D.load().dlra_init(D.C.byref(c), D.C.byref(h)), h


@pytest.mark.parametrize("kw", [dict(nx=0), dict(N=0), dict(N=40), dict(rank_max=100), dict(rank=0),
                                dict(e_min=200.0), dict(collision=7), dict(precision=5), dict(rank_mode=9),
                                dict(dx=-0.1), dict(precision=0, rank_max=48, rank=5)])
def test_invalid_config_is_rejected_on_the_host(lib, kw):
    st, h = _init_status(**kw)
    assert st == 1   # DLRA_ERR_ARG, before any device call
    if h.value:
        lib.dlra_destroy(h)


def test_null_context_calls_fail_cleanly(lib):
    assert lib.dlra_step(None, 1) == 1
    assert lib.dlra_dose(None, None, 0, 0) == 1
    assert isinstance(lib.dlra_last_error(None), bytes)
    assert lib.dlra_kstep(None) == 1
    lib.dlra_destroy(None)
