"""The arranger's own output: BIT1's "natural sorting" (Sec. 2; the arranger of Sec. 5.1), read
through pic_storage_order, against the oracle's stable counting sort of the same particles.

Two paths sort on the GPU:
* the full sort of pic_init / pic_restore (k_sort_scan + k_sort_scatter): afterwards the live
  slots come first, in non-decreasing cell order, followed by dead padding only; the sequence of
  cells, and the set of ids inside every cell's block, equal the oracle's after its stable counting
  sort of the same state (the order inside a cell follows atomic slot claims and is not unique);
* the deferred sort of a sort step (k_sort_scan turns the step's per-cell counts into cursors) and
  the step after it (k_step32 in scatter mode writes every particle to its slot): the slots
  [0, n) form one block per cell, with the block sizes of the counts, holding exactly the particles
  whose cell was that cell when the sort step ended, minus those absorbed in the step that moved
  them (dead slots, no stale particle); the step's births follow the blocks.
Both checks are exact: cells and ids are integers and both codes start from the same state.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2606_28534_gb300 import build, pic
from paper_2606_28534_gb300 import workloads as W

pytestmark = pytest.mark.gpu

DEAD = np.int32(-(2**31))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    import torch

    assert torch.cuda.is_available(), "GPU tests need CUDA"
    pic.lib()


def _oracle_sorted(p, blob):
    """Per species, the cells and ids in the oracle's storage order after its restore of blob (which
    ends with the stable counting sort)."""
    import os

    o = O.OracleSim(p, threads=len(os.sched_getaffinity(0)))
    assert o.restore(blob) == 0
    out = []
    for s in range(2):
        x, _v, ids = o.particles(s)
        out.append((np.floor(x).astype(np.int32), ids))
    o.close()
    return out


def _pairs(cells, ids):
    o = np.lexsort((ids, cells))
    return cells[o], ids[o]


def check_full_sort(cell, ids, ocell, oid):
    n = len(ocell)
    assert len(cell) == (n + 3) // 4 * 4  # extent: the live particles, padded to 4
    assert (cell[n:] == DEAD).all()
    live = cell[:n]
    assert (live != DEAD).all()  # compaction: no dead slot among the first n
    assert (np.diff(live) >= 0).all() if n > 1 else True  # non-decreasing cells
    assert np.array_equal(live, ocell)  # the same block of every cell
    a, b = _pairs(live, ids[:n]), _pairs(ocell, oid)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])  # the same ids in each block


def check_deferred_sort(cell, ids, ocell, oid, absorbed, born):
    """(cell, ids): storage after the step that applied the sort; (ocell, oid): the oracle's stable
    counting sort of the state the sort step ended with; absorbed / born: particles of the species
    absorbed / created in the step that moved them."""
    n = len(ocell)
    ext = (n + 3) // 4 * 4
    assert len(cell) >= ext
    blk = cell[:ext]
    assert (blk[n:] == DEAD).all()  # padding of the blocks
    dead = blk[:n] == DEAD
    assert int(dead.sum()) == absorbed  # a dead slot for each particle absorbed in that step, no more
    live_j = np.flatnonzero(~dead)
    # slot j belongs to the block of cell ocell[j] (the stable sort's order); the particle in it moved
    # at most two cells in the step
    assert (np.abs(blk[live_j].astype(np.int64) - ocell[live_j]) <= 2).all()
    # the (block cell, id) pairs equal the oracle's (cell, id) pairs minus the absorbed particles
    tail = cell[ext:]
    tail_ids = ids[ext:][tail != DEAD]
    assert len(tail_ids) == born
    live_ids = np.concatenate([ids[live_j], tail_ids])
    assert len(np.unique(live_ids)) == len(live_ids)
    kept = np.sort(ids[live_j])
    pos = np.minimum(np.searchsorted(kept, oid), max(len(kept) - 1, 0))
    gone = (kept[pos] != oid) if len(kept) else np.ones(len(oid), bool)
    assert int(gone.sum()) == absorbed
    a = _pairs(ocell[live_j], ids[live_j])
    b = _pairs(ocell[~gone], oid[~gone])
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    so = np.sort(oid)
    if len(so) and len(tail_ids):  # births carry new ids
        q = np.minimum(np.searchsorted(so, tail_ids), len(so) - 1)
        assert not (so[q] == tail_ids).any()


def _hits(d, s):
    return sum(d["wall_hits"][s])


@pytest.mark.parametrize("name", ["SMALL_C3", "SMALL_COLL", "C2"])
def test_single_run_sort_output_matches_the_oracle_sort(name):
    p = W.variant(getattr(W, name), sort_interval=4 if name != "C2" else 10)
    interval = p["sort_interval"]
    g = pic.Simulation(p)
    # the full sort of pic_init and of pic_restore
    blob0 = g.snapshot()
    ref0 = _oracle_sorted(p, blob0)
    for s in range(2):
        check_full_sort(*g.storage_order(s), *ref0[s])
    g2 = pic.Simulation(p)
    assert g2.restore(blob0) == 0
    for s in range(2):
        check_full_sort(*g2.storage_order(s), *ref0[s])
    g2.close()
    # two deferred sorts: the steps with index 0 and `interval` sort
    for k in range(2):
        g.step(1 if k == 0 else interval - 1)
        d0 = g.diag()
        assert (d0["step"] - 1) % interval == 0  # the last step was a sort step
        blob = g.snapshot()
        g.step(1)  # the step that moves the particles to their slots
        d1 = g.diag()
        born = [d1["births"][s] - d0["births"][s] + d1["source_pairs"] - d0["source_pairs"] for s in range(2)]
        ref = _oracle_sorted(p, blob)
        for s in range(2):
            ocell, oid = ref[s]
            check_deferred_sort(*g.storage_order(s), ocell, oid, _hits(d1, s) - _hits(d0, s), born[s])
    g.close()


def test_ensemble_sort_output_matches_the_oracle_sort():
    runs = [W.variant(q, sort_interval=3) for q in W.small_ensemble()]
    b = pic.Batch(runs)
    blobs = [b.snapshot(k) for k in range(len(runs))]
    for k, q in enumerate(runs):  # the load's full sort
        ref = _oracle_sorted(q, blobs[k])
        for s in range(2):
            check_full_sort(*b.storage_order(k, s), *ref[s])
    for rounds in range(2):
        b.step(1 if rounds == 0 else 2)  # the steps with index 0 and 3 sort
        d0 = b.diag()
        blobs = [b.snapshot(k) for k in range(len(runs))]
        b.step(1)
        d1 = b.diag()
        for k, q in enumerate(runs):
            assert (d0[k]["step"] - 1) % 3 == 0
            ref = _oracle_sorted(q, blobs[k])
            for s in range(2):
                ocell, oid = ref[s]
                born = d1[k]["births"][s] - d0[k]["births"][s]
                check_deferred_sort(*b.storage_order(k, s), ocell, oid, _hits(d1[k], s) - _hits(d0[k], s), born)
    b.close()


def test_storage_order_refuses_what_it_cannot_report():
    g = pic.Simulation(W.variant(W.SMALL_C1, precision=W.PRECISION_FP64_PLAIN))
    with pytest.raises(pic.PicError):
        g.storage_order(0)  # the plain path keeps no cell order
    g.close()
    h = pic.Simulation(W.SMALL_C1)
    with pytest.raises(pic.PicError):
        h.storage_order(2)
    h.close()
