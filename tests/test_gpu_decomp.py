"""A simulation decomposed by particles (pic_keep_subset, pic_local_deposit, pic_solve_deposit,
pic_step_begin / pic_step_end) against the same simulation in one handle.

The parts hold disjoint subsets of the particles over the whole grid and exchange only their int64
node deposits, whose sum is exact; so the union of the parts must equal the whole run particle for
particle and bit for bit (cells, fractions, velocities, ids, null-collision countdowns), the field
must be identical, and the parts' counters must add up to the whole run's -- through sorts, wall
losses and ionization births.  The exchange here is a sum of CUDA tensors in one process (what an
all-reduce computes); paper_2606_28534_gb300.decomp does the same over a process group.
"""
import numpy as np
import pytest

import snapfmt
from paper_2606_28534_gb300 import build, pic
from paper_2606_28534_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    import torch

    assert torch.cuda.is_available(), "GPU tests need CUDA"
    pic.lib()


def _union(blobs):
    out = []
    for s in range(2):
        parts = [snapfmt.parse(b)["species"][s] for b in blobs]
        cat = {k: np.concatenate([q[k] for q in parts]) for k in ("cell", "frac", "v", "id", "next")}
        o = np.argsort(cat["id"])
        out.append({k: v[o] for k, v in cat.items()})
    return out


def _check_equal(whole, parts):
    w = snapfmt.parse(whole.snapshot())["species"]
    u = _union([h.snapshot() for h in parts])
    for s in range(2):
        for k in ("id", "cell", "frac", "v", "next"):
            assert np.array_equal(u[s][k], w[s][k]), (s, k)
    fw = whole.fields()
    for h in parts:
        f = h.fields()
        for k in ("R", "rho", "phi", "E"):
            assert np.array_equal(f[k], fw[k]), k
    dw = whole.diag()
    dp = [h.diag() for h in parts]
    for k in ("n", "wall_hits", "coll", "births", "near_threshold", "nu_max_violations"):
        tot = np.sum([np.asarray(d[k], np.int64) for d in dp], axis=0)
        assert np.array_equal(tot, np.asarray(dw[k], np.int64)), k
    assert sum(d["wall_charge"] for d in dp) == dw["wall_charge"]
    for d in dp:  # grid quantities are the whole simulation's on every part
        assert d["net_charge_units"] == dw["net_charge_units"] and d["field_energy"] == dw["field_energy"]
    for s in range(2):
        assert abs(sum(d["ke"][s] for d in dp) - dw["ke"][s]) <= 1e-12 * abs(dw["ke"][s])


@pytest.mark.parametrize("name,nparts", [("SMALL_C2", 2), ("SMALL_COLL", 3), ("SMALL_C1", 2)])
def test_parts_reproduce_the_whole_run_bit_for_bit(name, nparts):
    import torch

    p = W.variant(getattr(W, name), sort_interval=3)
    whole = pic.Simulation(p)
    parts = [pic.Simulation(p) for _ in range(nparts)]
    for k, h in enumerate(parts):
        h.keep_subset(k, nparts)
    n1 = p["ncells"] + 1
    R = [torch.empty(2 * n1, dtype=torch.int64, device="cuda") for _ in parts]
    for h, r in zip(parts, R):
        h.local_deposit(r)
    tot = torch.stack(R).sum(0)
    for h in parts:
        h.solve_deposit(tot)
    assert sum(h.diag()["n"][0] for h in parts) == whole.diag()["n"][0]
    _check_equal(whole, parts)
    for _ in range(11):  # across sorts (every third step) and the steps that move the particles
        whole.step(1)
        for h, r in zip(parts, R):
            h.step_begin(r)
        tot = torch.stack(R).sum(0)
        for h in parts:
            h.step_end(tot)
    _check_equal(whole, parts)
    assert whole.diag()["coll"][4] > 0


def test_split_step_calls_are_refused_where_they_cannot_hold():
    import torch

    g = pic.Simulation(W.SMALL_C2)
    R = torch.zeros(2 * (W.SMALL_C2["ncells"] + 1), dtype=torch.int64, device="cuda")
    with pytest.raises(pic.PicError):
        g.step_end(R)  # no open step
    g.step_begin(R)
    with pytest.raises(pic.PicError):
        g.step(1)  # a step is open
    with pytest.raises(pic.PicError):
        g.step_begin(R)
    g.step_end(R)
    g.step(1)
    with pytest.raises(pic.PicError):
        g.keep_subset(2, 2)
    with pytest.raises(pic.PicError):
        g.local_deposit(R[:-1])
    g.close()
    for bad in (W.variant(W.SMALL_C2, precision=W.PRECISION_FP64_PLAIN), W.SMALL_C3, W.SMALL_C6):
        h = pic.Simulation(W.variant(bad, capacity_factor=2.0) if bad is W.SMALL_C6 else bad)
        with pytest.raises(pic.PicError):  # plain path, pair source, tracked neutrals
            h.keep_subset(0, 2)
        h.close()


def test_decomposed_over_a_process_group_of_one_is_the_whole_run():
    # the orchestration of paper_2606_28534_gb300.decomp with a single rank (no process group)
    from paper_2606_28534_gb300 import decomp

    p = W.variant(W.SMALL_COLL, sort_interval=4)
    d = decomp.Decomposed(p)
    whole = pic.Simulation(p)
    d.step(9)
    whole.step(9)
    assert d.sim.snapshot() == whole.snapshot()
    d.close()
