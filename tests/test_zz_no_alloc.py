"""pic_field_noalloc: the allocation-free variant of the deposit + field solve.

Some callers cannot allocate device memory (they live inside another framework's fixed memory
pool, or must not allocate after start-up); for them the library offers one entry point whose
scratch is a fixed device array inside the library.  This file checks, through the C ABI, that it
gives what the method fixes for the same particles -- the oracle's int64 deposit R exactly, and its
FP64 node field within the conditioning bound of the tridiagonal solve -- and what the ordinary
entry points give (pic_restore + pic_get_field on a handle with its own workspace), on consecutive
calls with different states and configurations (one with density smoothing), so that a call that
failed to clear what the previous call left in the shared scratch would show up; and that a grid
larger than the fixed scratch, or mismatched input tensors, are refused.  It lives in a file of its
own that pytest collects last, so that a run stopping at the first failure has already run
everything else.
"""
import math

import numpy as np
import pytest

import snapfmt
from oracle import oracle as O
from paper_2606_28534_gb300 import build, pic
from paper_2606_28534_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    import torch

    assert torch.cuda.is_available(), "GPU tests need CUDA"
    pic.lib()


def _state(params, steps):
    o = O.OracleSim(params)
    o.step(steps)
    return snapfmt.round_to_fp32(o.snapshot())


def _reference_fields(params, blob):
    g = pic.Simulation(params)
    assert g.restore(blob) == 0
    f = g.fields()
    g.close()
    return f["R"], f["E"]


def _oracle_fields(params, blob):
    o = O.OracleSim(params)
    assert o.restore(blob) == 0
    f = o.fields()
    o.close()
    return f["R"], f["E"], f["phi"]


def _cond_tol(N):
    return max(1e-13, 4 * N * N / math.pi**2 * 2.0**-52)


def _device_particles(blob):
    import torch

    sp = snapfmt.parse(blob)["species"]
    out = []
    for s in sp:
        out.append(torch.from_numpy(np.ascontiguousarray(s["cell"], np.int32)).cuda())
        out.append(torch.from_numpy(np.ascontiguousarray(s["frac"].astype(np.float32))).cuda())
    return out


def test_no_alloc_matches_the_oracle_and_the_workspace_path_on_consecutive_calls():
    p = W.variant(W.SMALL_C3, ncells=4096, L=4096.0, profile_scale=512.0, source_x1=256.0)
    ps = W.variant(W.SMALL_C2, smooth_passes=2, V_left=-2.0)  # smoothed density before the solve
    for q, steps in ((p, 2), (p, 7), (ps, 3), (p, 4)):  # consecutive calls, different states
        blob = _state(q, steps)
        R_o, E_o, phi_o = _oracle_fields(q, blob)
        R_ref, E_ref = _reference_fields(q, blob)
        c0, f0, c1, f1 = _device_particles(blob)
        R, E = pic.field_noalloc(q, c0, f0, c1, f1)
        R, E = R.cpu().numpy(), E.cpu().numpy()
        assert np.array_equal(R, R_o)  # integer deposit: exact, against the oracle
        assert np.array_equal(R, R_ref)  # and against the workspace path
        # the FP64 field against the oracle's Thomas solve and centred differences, at the
        # conditioning bound of tridiag(-1, 2, -1) (as the field solve's own parity)
        N, dx = q["ncells"], q["L"] / q["ncells"]
        scale = np.abs(phi_o).max()
        assert np.abs(E - E_o).max() <= _cond_tol(N) * scale / dx * 4, q
        # and what pic_get_field reports (FP32) for the same state
        assert np.abs(E.astype(np.float32) - E_ref).max() <= 2.0**-23 * np.abs(E_ref).max()


def test_no_alloc_refuses_mismatched_inputs():
    import torch

    p = W.SMALL_C2
    c = torch.zeros(8, dtype=torch.int32, device="cuda")
    f = torch.zeros(8, dtype=torch.float32, device="cuda")
    for args in ((c, f[:4], c, f), (c, f, c[:4], f), (c.long(), f, c, f), (c, f.double(), c, f),
                 (c[::2], f[::2], c, f)):
        with pytest.raises(pic.PicError) as e:
            pic.field_noalloc(p, *args)
        assert e.value.status == 1


def test_no_alloc_refuses_grids_beyond_its_scratch():
    import torch

    p = W.variant(W.SMALL_C2, ncells=65537, L=65537.0)
    z = torch.zeros(4, dtype=torch.int32, device="cuda")
    f = torch.zeros(4, dtype=torch.float32, device="cuda")
    with pytest.raises(pic.PicError) as e:
        pic.field_noalloc(p, z, f, z, f)
    assert e.value.status == 1
