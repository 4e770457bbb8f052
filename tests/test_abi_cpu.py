"""Host-side checks of the C ABI that need no GPU: the library loads, exports every entry point
declared in include/pic.h, and validates configurations without touching a device."""
import ctypes as C
import os
import re

import pytest

from paper_2606_28534_gb300 import build, pic
from paper_2606_28534_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return pic.lib()


def _declared():
    txt = open(os.path.join(ROOT, "include", "pic.h")).read()
    return sorted(set(re.findall(r"\b(pic_[a-z_0-9]+)\s*\(", txt)))


def test_header_declares_what_the_binding_knows():
    assert sorted(pic.SYMBOLS) == _declared()


def test_library_exports_every_declared_symbol(L):
    for name in _declared():
        assert hasattr(L, name), name


def test_strerror_names_every_status(L):
    for code in range(8):
        assert L.pic_strerror(code).decode()
    assert L.pic_strerror(99).decode() == "unknown status"


def test_workspace_size_validates_and_scales(L):
    small = pic.workspace_size(W.SMALL_C2)
    big = pic.workspace_size(W.variant(W.SMALL_C2, ppc=(530, 530)))
    assert 0 < small < big
    plain = pic.workspace_size(W.variant(W.SMALL_C2, precision=W.PRECISION_FP64_PLAIN))
    assert plain > 0
    for bad in (dict(ncells=1), dict(ppc=(0, 1)), dict(dt=0.0), dict(sort_interval=0),
                dict(capacity_factor=0.5), dict(field_mode=7), dict(precision=5),
                dict(load_profile=W.LOAD_EXP, profile_scale=0.0), dict(ncells=300000)):
        with pytest.raises(pic.PicError) as e:
            pic.workspace_size(W.variant(W.SMALL_C2, **bad))
        assert e.value.status == 1
    c = pic.make_config(W.SMALL_C2)
    c.abi_version = 2
    n = C.c_size_t(0)
    assert L.pic_workspace_size(C.byref(c), C.byref(n)) == 1


def test_init_rejects_bad_arguments_before_any_device_work(L):
    c = pic.make_config(W.variant(W.SMALL_C2, ncells=0))
    h = C.c_void_p(1)
    assert L.pic_init(C.byref(c), None, 0, None, C.byref(h)) == 1
    assert h.value is None
    assert L.pic_step(None, 1) == 1
    assert L.pic_diag(None, None) == 1
    assert L.pic_poisson(None, 8, 1.0, 0.0, 0.0, None, None, None) == 1
