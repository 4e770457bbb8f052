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
    c.abi_version = 1  # an older layout of pic_config
    n = C.c_size_t(0)
    assert L.pic_workspace_size(C.byref(c), C.byref(n)) == 1


def test_sheath_physics_validates_and_adds_its_buffers(L):
    base = pic.workspace_size(W.variant(W.SMALL_C6, neutrals=0, neutral_ppc=0, smooth_passes=0))
    assert pic.workspace_size(W.variant(W.SMALL_C6, neutrals=0, neutral_ppc=0)) == base  # smoothing: no memory
    with_nt = pic.workspace_size(W.SMALL_C6)
    more_nt = pic.workspace_size(W.variant(W.SMALL_C6, neutral_ppc=400))
    assert base < with_nt < more_nt
    for bad in (dict(precision=W.PRECISION_FP64_PLAIN),          # FP32 path only
                dict(charge=(-1.0, 1.5)),                         # integer charges (exact solve)
                dict(smooth_passes=5), dict(smooth_passes=-1),
                dict(recycle=1.5), dict(recycle=-0.1), dict(K_iz=-1.0), dict(T_rec=-1.0), dict(T_sec=-1.0),
                dict(neutral_capacity=0.5), dict(neutral_ppc=-3), dict(neutrals=2),
                dict(neutrals=0),                                 # initial neutrals need the species
                dict(reserved=1)):
        with pytest.raises(pic.PicError) as e:
            pic.workspace_size(W.variant(W.SMALL_C6, **bad))
        assert e.value.status == 1, bad
    assert pic.workspace_size(W.variant(W.SMALL_C6, smooth_passes=4, recycle=0.0, K_iz=0.0)) > 0


def test_init_rejects_bad_arguments_before_any_device_work(L):
    c = pic.make_config(W.variant(W.SMALL_C2, ncells=0))
    h = C.c_void_p(1)
    assert L.pic_init(C.byref(c), None, 0, None, C.byref(h)) == 1
    assert h.value is None
    assert L.pic_step(None, 1) == 1
    assert L.pic_diag(None, None) == 1
    assert L.pic_poisson(None, 8, 1.0, 0.0, 0.0, None, None, None) == 1


def test_no_alloc_entry_rejects_bad_arguments_before_any_device_work(L):
    # the C entry point checks its configuration before it looks up its scratch or launches
    R = C.c_void_p(16)
    E = C.c_void_p(16)
    for bad in (W.variant(W.SMALL_C2, ncells=65537, L=65537.0), W.variant(W.SMALL_C2, smooth_passes=5),
                W.variant(W.SMALL_C2, charge=(-1.0, 1.5)), W.variant(W.SMALL_C2, ncells=1, L=1.0)):
        c = pic.make_config(bad)
        assert L.pic_field_noalloc(C.byref(c), None, None, 0, None, None, 0, R, E, None) == 1
    c = pic.make_config(W.SMALL_C2)
    assert L.pic_field_noalloc(C.byref(c), None, None, 4, None, None, 0, R, E, None) == 1  # n without arrays
    assert L.pic_field_noalloc(C.byref(c), None, None, 0, None, None, 0, None, E, None) == 1


def test_no_alloc_binding_refuses_mismatched_tensors_before_the_call():
    # the binding hands raw pointers to a kernel that reads frac_s[i] for i < len(cell_s): a shorter
    # frac tensor, other dtypes, views that are not contiguous or tensors off the GPU never reach it
    import torch

    c = torch.zeros(8, dtype=torch.int32)
    f = torch.zeros(8, dtype=torch.float32)
    for args in ((c, f[:4], c, f), (c, f, c[:4], f), (c.long(), f, c, f), (c, f.double(), c, f),
                 (c.reshape(2, 4), f.reshape(2, 4), c, f), (c, f, c, f)):
        with pytest.raises(pic.PicError) as e:
            pic.field_noalloc(W.SMALL_C2, *args)
        assert e.value.status == 1


# ---- ensembles --------------------------------------------------------------------------------
def test_batch_shapes_are_listed(L):
    names = pic.batch_variants()
    assert len(names) >= 2 and all(re.fullmatch(r"tpb\d+_minb\d+_stages\d+", n) for n in names)
    assert L.pic_batch_variant_name(len(names)) is None
    assert L.pic_batch_variant_name(-1) is None


def test_batch_workspace_is_the_sum_of_its_parts(L):
    runs = W.small_ensemble()
    total = pic.batch_workspace_size(runs)
    assert total > 0
    # one more simulation needs more room
    assert pic.batch_workspace_size(runs + [runs[3]]) > total
    # the C4 ensemble: about 5.9e8 particles, two SoA buffers of 28 bytes a slot with headroom
    c4 = W.c4()
    n = sum(2 * p["ncells"] * p["ppc"][0] for p in c4)
    assert 5.0e8 < n < 6.5e8
    assert 2 * 28 * n < pic.batch_workspace_size(c4) < 2 * 28 * n * 1.5


@pytest.mark.parametrize("bad", [
    dict(dt=0.05),                       # time step shared by the batch
    dict(L=200.0),                       # cell size shared (L / ncells)
    dict(B=0.25),
    dict(B_angle_deg=10.0),
    dict(mass=(1.0, 1836.0)),
    dict(charge=(-1.0, 2.0)),
    dict(sort_interval=4),
    dict(field_mode=W.FIELD_ZERO),
    dict(frozen_mask=2),
    dict(precision=W.PRECISION_FP64_PLAIN),  # the batch is the FP32 path
    dict(source_mode=W.SOURCE_PAIRS, source_x1=4.0),
    dict(smooth_passes=1),  # the sheath physics runs in single simulations only
    dict(neutrals=1, recycle=1.0, T_rec=0.1, neutral_capacity=1.5),
])
def test_batch_rejects_configurations_that_cannot_share_a_launch(L, bad):
    runs = W.small_ensemble()
    runs[5] = W.variant(runs[5], **bad)
    with pytest.raises(pic.PicError) as e:
        pic.batch_workspace_size(runs)
    assert e.value.status == 1


def test_batch_accepts_per_run_physics(L):
    runs = W.small_ensemble()
    runs[5] = W.variant(runs[5], V_left=-4.0, V_right=0.5, n_gas=3.0, sigma_cx=0.05, Tg=0.2,
                        T=(2.0, 0.3), E_cap=40.0, capacity_factor=2.0, seed=5,
                        load_profile=W.LOAD_QUIET_SINE, profile_scale=0.2, profile_mode=3)
    assert pic.batch_workspace_size(runs) > 0


def test_batch_init_rejects_bad_arguments_before_any_device_work(L):
    runs = W.small_ensemble()
    arr = (pic.PicConfig * len(runs))(*[pic.make_config(p) for p in runs])
    h = C.c_void_p(1)
    assert L.pic_batch_init(arr, 0, None, 0, None, C.byref(h)) == 1
    assert h.value is None
    assert L.pic_batch_init(arr, pic.PIC_BATCH_MAX_SIMS + 1, None, 0, None, C.byref(h)) == 1
    assert L.pic_batch_init(None, 3, None, 0, None, C.byref(h)) == 1
    # a workspace that is not 256-byte aligned
    assert L.pic_batch_init(arr, len(runs), C.c_void_p(16), 1 << 30, None, C.byref(h)) == 1
    n = C.c_size_t(0)
    assert L.pic_batch_workspace_size(arr, len(runs), None) == 1
    assert L.pic_batch_workspace_size(arr, len(runs), C.byref(n)) == 0 and n.value > 0
    assert L.pic_batch_step(None, 1) == 1
    assert L.pic_batch_sync(None) == 1
    assert L.pic_batch_diag(None, None, 0) == 1
    assert L.pic_batch_snapshot(None, 0, None, 0, None) == 1
    assert L.pic_batch_restore(None, None, None) == 1
    assert L.pic_batch_reset(None) == 1
    assert L.pic_batch_set_tuning(None, None) == 1
    L.pic_batch_free(None)


def test_adjoint_rejects_the_sheath_physics(L):
    assert pic.adj_workspace_size(W.C5, 20, 5) > 0
    for bad in (dict(smooth_passes=2), dict(neutrals=1, recycle=1.0, neutral_capacity=1.5)):
        with pytest.raises(pic.PicError) as e:
            pic.adj_workspace_size(W.variant(W.C5, **bad), 20, 5)
        assert e.value.status == 1


def test_blob_checksum_is_zlibs_crc32():
    # the snapshot's closing checksum (pure host code: four interleaved registers per thread, the
    # threads' parts joined in GF(2)); lengths around the split thresholds and one of 70 MB that
    # the library spreads over several threads
    import zlib

    import numpy as np

    rng = np.random.default_rng(11)
    data = rng.integers(0, 256, size=(70 << 20) + 13, dtype=np.uint8).tobytes()
    for n in (0, 1, 7, 8, 9, 255, 16383, 16384, 16391, 131079, 1 << 20, (33 << 20) + 5, len(data)):
        assert pic.blob_crc32(data[:n]) == zlib.crc32(data[:n]), n
    assert pic.blob_crc32(bytearray(data[:1000])) == zlib.crc32(data[:1000])
