"""Ensembles (pic_batch_*) through the C ABI: every simulation of a batch computes what its own
configuration computes alone.

* Parity with the FP64 oracle, as for one simulation: a common state (oracle runs, rounded to
  FP32) is restored into every simulation of a heterogeneous batch, the batch takes one step, and
  each simulation is compared with one oracle step of its own configuration at the single-step
  tolerances (tests/stepcheck.py).
* Agreement with the single-simulation path: a batch and the same configurations run one at a time
  produce byte-identical snapshots, identical diagnostics and identical fields over many steps and
  several sorts, for every compiled shape of the batch step kernel, with and without CUDA graphs.
* The C4 ensemble at full size (256 runs, 5.7e8 particles): sampled initial particles against the
  oracle's loader, charge and particle accounting of every run after 20 steps, the node deposits of
  three runs against an exact integer sum over their stored particles, and one run against the same
  configuration run alone.
"""
import math

import numpy as np
import pytest

import snapfmt
import stepcheck
from oracle import oracle as O
from paper_2606_28534_gb300 import build, pic
from paper_2606_28534_gb300 import workloads as W

pytestmark = pytest.mark.gpu

NVARIANTS = 4  # compiled shapes of the batch step kernel (checked against the library below)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    import torch

    assert torch.cuda.is_available(), "GPU tests need CUDA"
    assert len(pic.batch_variants()) == NVARIANTS


def _oracle_blob_fp32(params, steps):
    o = O.OracleSim(params)
    if steps:
        o.step(steps)
    return snapfmt.round_to_fp32(o.snapshot())


def _strip(d):
    d = dict(d)
    d.pop("particle_steps")  # counted since init / restore
    return d


# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("steps", [3, 10])  # 10: the batch step is a sort step
def test_one_batch_step_matches_the_oracle_for_every_simulation(steps):
    runs = W.small_ensemble()
    blobs = [_oracle_blob_fp32(p, steps) for p in runs]
    b = pic.Batch(runs)
    assert b.restore(blobs) == 0
    b.step(1)
    diags = b.diag()
    assert all(d["step"] == steps + 1 for d in diags)
    for k, p in enumerate(runs):
        o = O.OracleSim(p)
        assert o.restore(blobs[k]) == 0
        o.step(1)
        stepcheck.assert_one_step(p, blobs[k], o.diag(), o.snapshot(), o.fields(), diags[k], b.snapshot(k),
                                  b.fields(k))
    b.close()


def test_batch_restore_deposits_exactly_what_the_oracle_deposits():
    runs = W.small_ensemble()
    blobs = [_oracle_blob_fp32(p, 4) for p in runs]
    b = pic.Batch(runs)
    assert b.restore(blobs) == 0
    for k, p in enumerate(runs):
        o = O.OracleSim(p)
        assert o.restore(blobs[k]) == 0
        fo, fg = o.fields(), b.fields(k)
        assert np.array_equal(fo["R"], fg["R"])
        scale = np.abs(fo["phi"]).max()
        assert np.abs(fo["phi"] - fg["phi"]).max() <= stepcheck.cond_tol(p["ncells"]) * scale
        # the restored state comes back exactly, except that the wall energies are kept in
        # 2^-24 fixed point (per particle weight w) on the device
        a, r = snapfmt.parse(b.snapshot(k)), snapfmt.parse(blobs[k])
        assert a["step"] == r["step"] and a["wall_charge"] == r["wall_charge"]
        assert np.array_equal(a["counters"], r["counters"])
        for s in range(2):
            w = (p["L"] / p["ncells"]) / p["ppc"][s]
            assert abs(a["wall_energy"][s] - r["wall_energy"][s]) <= 2.0**-24 * w
            for key in ("id", "cell", "frac", "v"):
                assert np.array_equal(a["species"][s][key], r["species"][s][key]), (k, s, key)
    b.close()


# ------------------------------------------------------------------------------------------------
def _single_runs(runs, steps):
    out = []
    for p in runs:
        g = pic.Simulation(p)
        g.step(steps)
        out.append((g.snapshot(), _strip(g.diag()), g.fields()))
        g.close()
    return out


@pytest.fixture(scope="module")
def sorted_often():
    runs = [W.variant(p, sort_interval=3) for p in W.small_ensemble()]
    return runs, _single_runs(runs, 13)


@pytest.mark.parametrize("graph", [False, True])
@pytest.mark.parametrize("variant", range(NVARIANTS))
def test_batch_equals_the_runs_one_at_a_time(sorted_often, variant, graph):
    runs, ref = sorted_often
    b = pic.Batch(runs)
    b.set_tuning(variant=variant, use_graph=graph)
    b.set_diag_interval(variant % 2)  # kinetic energy summed in the step, or by pic_batch_diag
    b.step(13)  # with graphs: two replays of 6 steps and one step launched directly
    b.sync()
    diags = b.diag()
    for k in range(len(runs)):
        snap, diag, fields = ref[k]
        assert b.snapshot(k) == snap, k
        assert _strip(diags[k]) == diag, k
        f = b.fields(k)
        for key in ("R", "E", "phi"):
            assert np.array_equal(f[key], fields[key]), (k, key)
    b.close()


def test_fewer_ctas_give_the_same_state(sorted_often):
    runs, ref = sorted_often
    b = pic.Batch(runs)
    b.set_tuning(variant=0, ctas_per_sm=1, use_graph=True)
    b.step(13)
    for k in range(len(runs)):
        assert b.snapshot(k) == ref[k][0], k
    b.close()


def test_batch_snapshot_restore_continuation_and_interchange():
    runs = [W.variant(p, sort_interval=4) for p in W.small_ensemble()]
    a = pic.Batch(runs)
    a.step(6)
    blobs = [a.snapshot(k) for k in range(len(runs))]
    a.step(9)
    b = pic.Batch(runs)
    assert b.restore(blobs) == 0
    b.step(9)
    for k in range(len(runs)):
        assert a.snapshot(k) == b.snapshot(k)
    # a batch snapshot restores into a single handle of the same configuration and continues alike
    k = 3
    g = pic.Simulation(runs[k])
    assert g.restore(blobs[k]) == 0
    g.step(9)
    assert g.snapshot() == a.snapshot(k)
    # reset returns to the initial state
    fresh = pic.Batch(runs)
    a.reset()
    for k in range(len(runs)):
        assert a.snapshot(k) == fresh.snapshot(k)
    a.step(5)
    fresh.step(5)
    for k in range(len(runs)):
        assert a.snapshot(k) == fresh.snapshot(k)
    for x in (a, b, fresh, g):
        x.close()


def test_batch_restore_checks_every_blob_before_changing_state():
    runs = W.small_ensemble()
    b = pic.Batch(runs)
    b.step(2)
    before = [b.snapshot(k) for k in range(len(runs))]
    good = [_oracle_blob_fp32(p, 3) for p in runs]
    bad = list(good)
    corrupt = bytearray(good[6])
    corrupt[200] ^= 0x01
    bad[6] = bytes(corrupt)
    assert b.restore(bad) == 5
    wrong_config = list(good)
    wrong_config[2] = good[3]
    assert b.restore(wrong_config) == 5
    other_step = list(good)
    other_step[1] = _oracle_blob_fp32(runs[1], 4)
    assert b.restore(other_step) == 1
    after = [b.snapshot(k) for k in range(len(runs))]
    assert before == after
    with pytest.raises(pic.PicError) as e:
        b.set_tuning(variant=NVARIANTS)
    assert e.value.status == 1
    b.close()


def test_batch_invariants_every_step():
    runs = W.small_ensemble()
    b = pic.Batch(runs)
    d0 = b.diag()
    for _ in range(24):
        b.step(1)
        for k, d in enumerate(b.diag()):
            n0 = d0[k]["n"]
            assert d["net_charge_units"] == 2**32 * (d["n"][1] - d["n"][0])
            assert (d["n"][1] - d["n"][0]) + d["wall_charge"] == n0[1] - n0[0]
            for s in range(2):
                lost = d["wall_hits"][s][0] + d["wall_hits"][s][1]
                assert d["n"][s] == n0[s] + d["births"][s] - lost
            if runs[k]["coll_mask"] == 0:
                assert d["coll"][4] == 0
    b.close()


# ------------------------------------------------------------------------------------------------
def test_c4_full_size():
    runs = W.c4()
    b = pic.Batch(runs)
    d0 = b.diag()
    sizes = [2 * p["ncells"] * p["ppc"][0] for p in runs]
    for k, p in enumerate(runs):
        assert d0[k]["n"] == [p["ncells"] * p["ppc"][0]] * 2
    # sampled initial particles of the smallest, a middle and the largest run, computed one by one
    # by the oracle's loader
    order = np.argsort(sizes)
    rng = np.random.default_rng(11)
    for k in (int(order[0]), int(order[len(order) // 2]), int(order[-1])):
        p = runs[k]
        sp = snapfmt.parse(b.snapshot(k))["species"]
        for s in range(2):
            n = p["ncells"] * p["ppc"][s]
            idx = rng.choice(n, min(n, 1000), replace=False)
            x, v, ids = O.load_particles(p, s, idx)
            pos = np.searchsorted(sp[s]["id"], ids)
            assert np.array_equal(sp[s]["id"][pos], ids)
            assert np.abs(sp[s]["cell"][pos] + sp[s]["frac"][pos] - x).max() <= 2.0**-23 * 2
            vt = math.sqrt(p["T"][s] / p["mass"][s])
            assert np.abs(sp[s]["v"][pos] - v).max() <= 8e-6 * vt
    b.step(20)
    b.sync()
    for k, d in enumerate(b.diag()):
        n0 = d0[k]["n"]
        assert d["dropped"] == 0
        assert d["net_charge_units"] == 2**32 * (d["n"][1] - d["n"][0])
        assert (d["n"][1] - d["n"][0]) + d["wall_charge"] == n0[1] - n0[0]
        for s in range(2):
            lost = d["wall_hits"][s][0] + d["wall_hits"][s][1]
            assert d["n"][s] == n0[s] + d["births"][s] - lost
        assert d["coll"][4] > 0
    # every particle deposited exactly once (at this size the ensemble's step claims its chunks in
    # segments from a counter of the batch): the node deposits of the smallest, a middle and the
    # largest run equal the CIC deposit of their stored particles, W_r = rint(f 2^32), summed here
    # exactly (integers below 2^53)
    for k in (int(order[0]), int(order[len(order) // 2]), int(order[-1])):
        N = runs[k]["ncells"]
        sp = snapfmt.parse(b.snapshot(k))["species"]
        R = b.fields(k)["R"]
        for s in range(2):
            cell, wr = sp[s]["cell"].astype(np.int64), np.rint(sp[s]["frac"] * 2.0**32)
            Rh = (np.bincount(cell, weights=2.0**32 - wr, minlength=N + 1)
                  + np.bincount(cell + 1, weights=wr, minlength=N + 1))
            assert np.array_equal(Rh.astype(np.int64), R[s]), (k, s)
    # one mid-size run against the same configuration alone (byte-identical state)
    k = int(order[len(order) // 2])
    g = pic.Simulation(runs[k])
    g.step(20)
    assert g.snapshot() == b.snapshot(k)
    g.close()
    b.close()
