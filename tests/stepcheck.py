"""One FP32 step of the GPU path against one FP64 step of the oracle from the same state.

Tolerances (see the header of test_gpu_parity.py): |dv| <= 1e-5 |v| + 1e-6 v_th and |dx| <= 2e-6
cells per particle matched by id, the null-collision countdown equal; every other disagreement is a
near-threshold collision draw,
counted by both codes; wall hits and candidate counts exact; the net deposit exactly 2^32 times
the net particle charge; the field and deposit within the FP32 position error.
"""
import math

import numpy as np

import snapfmt


def cond_tol(N):
    return max(1e-13, 4 * N * N / math.pi**2 * 2.0**-52)


def by_id(sp):
    o = np.argsort(sp["id"])
    return {k: (v[o] if k != "v" else v[o, :]) for k, v in sp.items()}


def assert_one_step(p, blob, do, so_blob, fo, dg, sg_blob, fg):
    """blob: the common state; (do, so_blob, fo): oracle diag/snapshot/fields after one step;
    (dg, sg_blob, fg): the same of the GPU."""
    so = snapfmt.parse(so_blob)["species"]
    sg = snapfmt.parse(sg_blob)["species"]
    d0 = snapfmt.parse(blob)
    base_near = int(d0["counters"][9] + d0["counters"][10])
    near = (sum(do["near_threshold"]) - base_near) + (sum(dg["near_threshold"]) - base_near)
    mismatched = 0
    for s in range(2):
        a, b = by_id(sg[s]), by_id(so[s])
        common, ia, ib = np.intersect1d(a["id"], b["id"], return_indices=True)
        only = len(a["id"]) + len(b["id"]) - 2 * len(common)
        xa = a["cell"][ia] + a["frac"][ia]
        xb = b["cell"][ib] + b["frac"][ib]
        vt = math.sqrt(p["T"][s] / p["mass"][s])
        dv = np.abs(a["v"][ia] - b["v"][ib]).max(axis=1) if len(common) else np.zeros(0)
        okv = dv <= 1e-5 * np.abs(b["v"][ib]).max(axis=1) + 1e-6 * vt if len(common) else np.zeros(0, bool)
        okx = np.abs(xa - xb) <= 2e-6
        okn = a["next"][ia] == b["next"][ib]
        bad = ~(okv & okx & okn)
        mismatched += int(bad.sum()) + only
    # every disagreement is a near-threshold collision draw (each can add a particle pair)
    assert mismatched <= 4 * near, (mismatched, near)
    for s in range(2):
        assert dg["wall_hits"][s] == do["wall_hits"][s]
    for k in range(4):
        assert abs(dg["coll"][k] - do["coll"][k]) <= near
    assert dg["coll"][4] == do["coll"][4]  # the candidate test uses identical values
    assert dg["net_charge_units"] == 2**32 * (dg["n"][1] - dg["n"][0])
    scale = max(np.abs(fo["phi"]).max(), 1e-3)
    assert np.abs(fo["phi"] - fg["phi"]).max() <= 1e-5 * scale + cond_tol(p["ncells"]) * scale
    # integer deposit: each particle's W_r differs by at most its FP32 position error 2^32 * 2e-6
    count = np.abs(fo["R"]).max() / 2**32 + 1
    assert np.abs(fo["R"] - fg["R"]).max() <= count * 2**32 * 2e-6 + 2**33 * mismatched
    return mismatched, near
