"""GPU path of the D+/e/D sheath physics (recycling into tracked neutrals, their ionization, density
smoothing) through the C ABI, against the FP64 CPU oracle.

States come from the oracle (its load, or particles placed by the test and written with the snapshot
format), rounded to FP32, and are given to both codes; one step of each is compared particle by
particle (matched by id) for electrons, ions and neutrals, counter by counter, node by node.

Tolerances: those of the charged single step (|dv| <= 1e-5 |v| + 1e-6 v_th, |dx| <= 2e-6 cells), for
the neutrals too (v_th of the recycling temperature); the recycling decision is an exact integer
comparison (equal counts); a neutral's ionization is decided in FP32 on the GPU and FP64 in the oracle,
so a draw within 1e-5 P of P may go either way: both codes count such draws, and each can account for
three particles (the neutral, the ion it becomes, the electron born).  A neutral whose new position is
within 1e-5 cells of a wall may be lost in one code and not in the other.
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

ROOMY = dict(capacity_factor=2.0, neutral_capacity=2.0)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    import torch

    assert torch.cuda.is_available(), "GPU tests need CUDA"
    pic.lib()


def _records(sp):
    return {"x": sp["cell"] + sp["frac"], "v": sp["v"], "id": sp["id"]}


def _busy_blob(p, seed, step=0):
    """The oracle's load of p plus ions leaving through both walls and neutrals near both walls, at
    step `step` (0: a sort step, the neutral step compacts; else in place unless step % interval = 0)."""
    rng = np.random.default_rng(seed)
    N = p["ncells"]
    d = snapfmt.parse(O.OracleSim(p).snapshot())
    el, io, nt = _records(d["species"][0]), _records(d["species"][1]), _records(d["neutrals"])
    h = 300
    wx = np.concatenate([rng.uniform(0.0, 0.01, h), N - rng.uniform(1e-3, 0.01, h)])
    wv = np.zeros((2 * h, 3))
    wv[:h, 0], wv[h:, 0] = -0.5, 0.5
    wv[:, 1:] = rng.normal(size=(2 * h, 2))
    io = {"x": np.concatenate([io["x"], wx]), "v": np.concatenate([io["v"], wv]),
          "id": np.concatenate([io["id"], (np.uint64(1) << np.uint64(62)) + np.uint64(10**6) + np.arange(2 * h, dtype=np.uint64)])}
    xn = np.concatenate([nt["x"], rng.uniform(0, 0.02, 200), N - rng.uniform(1e-3, 0.02, 200)])
    vn = np.concatenate([nt["v"], rng.normal(size=(400, 3)) * 0.2])
    vn[-400:-200, 0] = -np.abs(vn[-400:-200, 0])
    vn[-200:, 0] = np.abs(vn[-200:, 0])
    nt = {"x": xn, "v": vn, "id": np.concatenate([nt["id"], (np.uint64(5) << np.uint64(60)) + np.arange(400, dtype=np.uint64)])}
    base = O.OracleSim(p).snapshot()
    return snapfmt.round_to_fp32(snapfmt.with_particles(base, [el, io], step=step, neutrals=nt))


def _both(p, blob):
    o = O.OracleSim(p)
    assert o.restore(blob) == 0
    g = pic.Simulation(p)
    assert g.restore(blob) == 0
    return o, g


def _match(a, b, vt):
    """Particles of a and b (parsed records) matched by id: (bad, only) counts."""
    a, b = stepcheck.by_id(a), stepcheck.by_id(b)
    common, ia, ib = np.intersect1d(a["id"], b["id"], return_indices=True)
    only = len(a["id"]) + len(b["id"]) - 2 * len(common)
    if not len(common):
        return 0, only
    xa, xb = a["cell"][ia] + a["frac"][ia], b["cell"][ib] + b["frac"][ib]
    dv = np.abs(a["v"][ia] - b["v"][ib]).max(axis=1)
    okv = dv <= 1e-5 * np.abs(b["v"][ib]).max(axis=1) + 1e-6 * vt
    okx = np.abs(xa - xb) <= 2e-6
    return int((~(okv & okx)).sum()), only


def _compare_one_step(p, blob, o, g):
    N = p["ncells"]
    d0 = snapfmt.parse(blob)
    so, sg = snapfmt.parse(o.snapshot()), snapfmt.parse(g.snapshot())
    do, dg = o.diag(), g.diag()
    no, ng = o.neutral_diag(), g.neutral_diag()
    base_near = int(d0["counters"][9] + d0["counters"][10])
    near = (sum(do["near_threshold"]) + sum(dg["near_threshold"]) - 2 * base_near +
            no["near_threshold"] + ng["near_threshold"] - 2 * int(d0["nt_counters"][5]))
    bad = only = 0
    for s in range(2):
        b_, o_ = _match(sg["species"][s], so["species"][s], math.sqrt(p["T"][s] / p["mass"][s]))
        bad, only = bad + b_, only + o_
    # neutrals near a wall after their move may be lost in one code only
    n0 = d0["neutrals"]
    x1 = n0["cell"] + n0["frac"] + n0["v"][:, 0] * p["dt"] / (p["L"] / N)
    edge = int(((np.abs(x1) < 1e-5) | (np.abs(x1 - N) < 1e-5)).sum())
    b_, o_ = _match(sg["neutrals"], so["neutrals"], math.sqrt(max(p["T_rec"], 1e-12) / p["mass"][1]))
    bad, only = bad + b_, only + o_
    assert bad + only <= 4 * near + edge, (bad, only, near, edge)
    for s in range(2):
        assert dg["wall_hits"][s] == do["wall_hits"][s]
    assert ng["recycled"] == no["recycled"]
    assert abs(sum(ng["lost"]) - sum(no["lost"])) <= edge
    assert abs(ng["ionized"] - no["ionized"]) <= near
    assert ng["n"] == len(sg["neutrals"]["id"]) and no["n"] == len(so["neutrals"]["id"])
    assert dg["coll"][4] == do["coll"][4]
    for k in range(4):
        assert abs(dg["coll"][k] - do["coll"][k]) <= near
    assert dg["net_charge_units"] == 2**32 * (dg["n"][1] - dg["n"][0])
    fo, fg = o.fields(), g.fields()
    scale = max(np.abs(fo["phi"]).max(), 1e-3)
    assert np.abs(fo["phi"] - fg["phi"]).max() <= 1e-5 * scale + stepcheck.cond_tol(N) * scale
    assert np.abs(fo["rho"] - fg["rho"]).max() <= 1e-5 * max(np.abs(fo["rho"]).max(), 1e-3) + 1e-9
    count = np.abs(fo["R"]).max() / 2**32 + 1
    assert np.abs(fo["R"] - fg["R"]).max() <= count * 2**32 * 2e-6 + 2**33 * (bad + only)
    return ng, no


# ------------------------------------------------------------------------------------------------
def test_initial_neutrals_match_the_oracle_load():
    p = W.variant(W.SMALL_C6, neutral_ppc=77, T_rec=0.3)
    g = pic.Simulation(p)
    sg, so = snapfmt.parse(g.snapshot()), snapfmt.parse(O.OracleSim(p).snapshot())
    a, b = stepcheck.by_id(sg["neutrals"]), stepcheck.by_id(so["neutrals"])
    assert np.array_equal(a["id"], b["id"]) and np.array_equal(a["cell"], b["cell"])
    assert np.array_equal(a["frac"], b["frac"])  # 24-bit fractions: exact in FP32
    assert np.abs(a["v"] - b["v"]).max() <= 1e-6 * np.abs(b["v"]).max()
    nd = g.neutral_diag()
    assert nd["n"] == 77 * p["ncells"] and nd["particle_steps"] == 0
    ke = 0.5 * p["mass"][1] * (b["v"] ** 2).sum() * (p["L"] / p["ncells"] / p["ppc"][1])
    assert abs(nd["ke"] - ke) <= 1e-6 * ke


@pytest.mark.parametrize("passes", [1, 2, 4])
def test_smoothed_field_matches_the_oracle(passes):
    p = W.variant(W.SMALL_C6, smooth_passes=passes, V_left=-2.0)
    blob = snapfmt.round_to_fp32(O.OracleSim(p).snapshot())
    o, g = _both(p, blob)
    fo, fg = o.fields(), g.fields()
    assert np.array_equal(fo["R"], fg["R"])  # identical FP32 positions: identical integer deposit
    s = np.abs(fo["rho"]).max()
    assert np.abs(fg["rho"] - fo["rho"]).max() <= 1e-13 * s
    sphi = max(np.abs(fo["phi"]).max(), 1.0)
    assert np.abs(fg["phi"] - fo["phi"]).max() <= stepcheck.cond_tol(p["ncells"]) * sphi
    # the FP32 node field the particles see comes from the integer solve of the smoothed charge
    sE = np.abs(fo["E"]).max()
    assert np.abs(fg["E"] - fo["E"]).max() <= 2.0**-23 * sE + stepcheck.cond_tol(p["ncells"]) * sE


@pytest.mark.parametrize("start", [0, 7], ids=["compacting", "in_place"])
@pytest.mark.parametrize("case", ["load", "busy", "partial", "no_ionization"])
def test_one_step_matches_the_oracle(case, start):
    p = W.variant(W.SMALL_C6, V_left=-2.0, **ROOMY)
    if case == "partial":
        p = W.variant(p, recycle=0.4)
    if case == "no_ionization":
        p = W.variant(p, K_iz=0.0)
    if case == "load":
        d = snapfmt.parse(O.OracleSim(p).snapshot())
        d["step"] = start
        blob = snapfmt.round_to_fp32(snapfmt.build(d))
    else:
        blob = _busy_blob(p, 11, step=start)
    o, g = _both(p, blob)
    o.step(1)
    g.step(1)
    ng, no = _compare_one_step(p, blob, o, g)
    if case != "load":
        assert sum(ng["recycled"]) > 0 and sum(ng["lost"]) > 0
    if case != "no_ionization":
        assert ng["ionized"] > 0


def test_steps_after_a_sort_and_a_scatter_match_the_oracle():
    # step 0 sorts (the scan), step 1 moves every particle to its sorted slot: births and the
    # neutral step's appends go past the new extent
    p = W.variant(W.SMALL_C6, V_left=-2.0, sort_interval=1, **ROOMY)
    blob = _busy_blob(p, 12)
    for k in range(3):
        o, g = _both(p, blob)
        o.step(1)
        g.step(1)
        _compare_one_step(p, blob, o, g)
        blob = snapfmt.round_to_fp32(o.snapshot())


def test_rerun_and_snapshot_continuation_are_bit_exact():
    p = W.variant(W.SMALL_C6, V_left=-2.0, sort_interval=3, **ROOMY)
    blob = _busy_blob(p, 13)
    a = pic.Simulation(p)
    assert a.restore(blob) == 0
    a.step(10)
    mid = a.snapshot()
    a.step(15)
    b = pic.Simulation(p)
    assert b.restore(blob) == 0
    b.step(25)
    c = pic.Simulation(p)
    assert c.restore(mid) == 0
    c.step(15)
    sa, sb, sc = a.snapshot(), b.snapshot(), c.snapshot()
    assert sa == sb == sc  # storage order differs between runs; the state does not
    assert a.neutral_diag() == b.neutral_diag()


def test_in_place_steps_then_a_compacting_step_match_the_oracle():
    # steps 7, 8, 9 update the neutral buffer in place (dead slots accumulate, recycled neutrals are
    # appended past the extent); step 10 compacts it
    p = W.variant(W.SMALL_C6, V_left=-2.0, **ROOMY)
    blob = _busy_blob(p, 15, step=7)
    for k in range(4):
        o, g = _both(p, blob)
        o.step(1)
        g.step(1)
        _compare_one_step(p, blob, o, g)
        blob = snapfmt.round_to_fp32(o.snapshot())


def test_neutrals_over_a_frozen_plasma_match_the_oracle_for_twelve_steps():
    # frozen charged species and no field: the neutrals' motion, wall losses and ionization (from a
    # fixed electron density) follow the same trajectories in both codes step after step, through
    # in-place steps (dead slots accumulate) and two compacting ones (steps 0 and 10)
    p = W.variant(W.SMALL_C6, frozen_mask=3, field_mode=W.FIELD_ZERO, coll_mask=0, K_iz=0.3,
                  source_mode=W.SOURCE_NONE, **ROOMY)
    N = p["ncells"]
    rng = np.random.default_rng(16)
    d = snapfmt.parse(O.OracleSim(p).snapshot())
    el, io = _records(d["species"][0]), _records(d["species"][1])
    n = 4000
    xn = np.concatenate([rng.uniform(0.0, N, n - 400), rng.uniform(0.0, 0.5, 200), N - rng.uniform(0.01, 0.5, 200)])
    vn = rng.normal(size=(n, 3)) * 0.3
    vn[-400:-200, 0] = -np.abs(vn[-400:-200, 0])
    vn[-200:, 0] = np.abs(vn[-200:, 0])
    ids = (np.uint64(5) << np.uint64(60)) + np.arange(n, dtype=np.uint64)
    blob = snapfmt.round_to_fp32(snapfmt.with_particles(O.OracleSim(p).snapshot(), [el, io],
                                                        neutrals={"x": xn, "v": vn, "id": ids}))
    o, g = _both(p, blob)
    steps = 12
    o.step(steps)
    g.step(steps)
    no, ng = o.neutral_diag(), g.neutral_diag()
    near = no["near_threshold"] + ng["near_threshold"]
    a, b = stepcheck.by_id(snapfmt.parse(g.snapshot())["neutrals"]), stepcheck.by_id(snapfmt.parse(o.snapshot())["neutrals"])
    common, ia, ib = np.intersect1d(a["id"], b["id"], return_indices=True)
    x1 = xn + steps * vn[:, 0] * p["dt"] / (p["L"] / N)
    edge = int(((np.abs(x1) < 1e-4) | (np.abs(x1 - N) < 1e-4)).sum())
    assert len(a["id"]) + len(b["id"]) - 2 * len(common) <= 2 * near + edge
    assert np.abs((a["cell"][ia] + a["frac"][ia]) - (b["cell"][ib] + b["frac"][ib])).max() <= steps * 2e-6
    assert np.array_equal(a["v"][ia], np.float32(b["v"][ib]).astype(np.float64))  # velocities never change
    assert abs(ng["ionized"] - no["ionized"]) <= near and ng["ionized"] > 0
    assert abs(sum(ng["lost"]) - sum(no["lost"])) <= edge and sum(ng["lost"]) > 0
    assert ng["particle_steps"] == no["particle_steps"] or near + edge > 0


def test_accounting_is_exact_over_many_steps():
    p = W.variant(W.SMALL_C6, V_left=-2.0, **ROOMY)
    g = pic.Simulation(p)
    assert g.restore(_busy_blob(p, 14)) == 0
    d0, n0 = g.diag(), g.neutral_diag()
    steps = 40
    for _ in range(steps):
        g.step(1)
    d, nd = g.diag(), g.neutral_diag()
    assert nd["n"] == n0["n"] + sum(nd["recycled"]) - sum(nd["lost"]) - nd["ionized"]
    assert nd["recycled"] == d["wall_hits"][1]
    for s in range(2):
        lost = sum(d["wall_hits"][s]) - sum(d0["wall_hits"][s])
        assert d["n"][s] == d0["n"][s] + d["births"][s] - d0["births"][s] + nd["ionized"] - lost
    assert d["net_charge_units"] == 2**32 * (d["n"][1] - d["n"][0])
    assert nd["ionized"] > 0 and sum(nd["recycled"]) > 0


def test_full_size_sheath_invariants():
    # the 150 M-particle sheath in the bench's launch configuration: properties that hold at any size
    p = W.C6
    g = pic.Simulation(p)
    d0, n0 = g.diag(), g.neutral_diag()
    assert n0["n"] == p["neutral_ppc"] * p["ncells"]
    prev_n = n0["n"]
    ps = 0
    for _ in range(12):  # one sort (step 10) and the scattering step after it
        g.step(1)
        ps += prev_n
        nd = g.neutral_diag()
        prev_n = nd["n"]
    d = g.diag()
    assert nd["particle_steps"] == ps
    assert nd["n"] == n0["n"] + sum(nd["recycled"]) - sum(nd["lost"]) - nd["ionized"]
    assert nd["recycled"] == [d["wall_hits"][1][k] - d0["wall_hits"][1][k] for k in range(2)]
    assert nd["ionized"] > 0
    for s in range(2):
        lost = sum(d["wall_hits"][s]) - sum(d0["wall_hits"][s])
        born = d["births"][s] - d0["births"][s] + nd["ionized"] + (d["source_pairs"] - d0["source_pairs"])
        assert d["n"][s] == d0["n"][s] + born - lost
    assert d["net_charge_units"] == 2**32 * (d["n"][1] - d["n"][0])
    # the ionization rate at n_e ~ 1 stays near K_iz dt per step
    rate = nd["ionized"] / ps
    assert 0.3 * p["K_iz"] * p["dt"] < rate < 3.0 * p["K_iz"] * p["dt"]



def test_full_size_sheath_long_run_keeps_every_invariant():
    # the 150 M-particle sheath over 400 steps (40 compacting sorts of the neutrals; the two kinds
    # of ionization grow each charged species by about a tenth, inside its capacity): the neutral
    # and charged accounting, the charge identity and the capacities hold at every check
    p = W.C6
    g = pic.Simulation(p)
    d0, n0 = g.diag(), g.neutral_diag()
    ncap = int(p["neutral_capacity"] * max(p["neutral_ppc"], p["ppc"][1]) * p["ncells"])
    for _ in range(4):
        g.step(100)
        d, nd = g.diag(), g.neutral_diag()
        assert d["dropped"] == 0
        assert nd["n"] == n0["n"] + sum(nd["recycled"]) - sum(nd["lost"]) - nd["ionized"]
        assert nd["recycled"] == [d["wall_hits"][1][k] - d0["wall_hits"][1][k] for k in range(2)]
        assert 0 < nd["n"] <= ncap
        for s in range(2):
            lost = sum(d["wall_hits"][s]) - sum(d0["wall_hits"][s])
            born = d["births"][s] - d0["births"][s] + nd["ionized"] + (d["source_pairs"] - d0["source_pairs"])
            assert d["n"][s] == d0["n"][s] + born - lost
            assert d["n"][s] <= int(p["capacity_factor"] * p["ppc"][s] * p["ncells"])
        assert d["net_charge_units"] == 2**32 * (d["n"][1] - d["n"][0])
        assert math.isfinite(nd["ke"]) and math.isfinite(d["field_energy"])
    assert d["step"] == 400


def test_batch_and_adjoint_refuse_the_sheath_physics():
    with pytest.raises(pic.PicError):
        pic.Batch([W.SMALL_C6])


def test_smallest_grid_with_four_smoothing_passes_matches_the_oracle():
    # N = 2: one interior node between the walls; the smoothing's wall rules act on every node
    p = W.variant(W.SMALL_C6, ncells=2, L=2.0, ppc=(7, 7), neutral_ppc=5, smooth_passes=4, V_left=-1.0, **ROOMY)
    blob = snapfmt.round_to_fp32(O.OracleSim(p).snapshot())
    o, g = _both(p, blob)
    fo, fg = o.fields(), g.fields()
    assert np.array_equal(fo["R"], fg["R"])
    assert np.abs(fg["rho"] - fo["rho"]).max() <= 1e-13 * np.abs(fo["rho"]).max()
    assert np.abs(fg["E"] - fo["E"]).max() <= 2.0**-23 * np.abs(fo["E"]).max() + 1e-12
    o.step(1)
    g.step(1)
    _compare_one_step(p, blob, o, g)


def test_largest_grid_smoothing_crosses_every_cluster_boundary():
    # 196607 cells: 24576 nodes per CTA of the field cluster; the stencil reads its neighbours across
    # the seven CTA boundaries in each of the three passes
    p = W.variant(W.SMALL_C6, ncells=196607, L=196607.0, ppc=(2, 2), neutral_ppc=1, smooth_passes=3,
                  V_left=-2.0, load_profile=W.LOAD_EXP, profile_scale=20000.0, **ROOMY)
    blob = snapfmt.round_to_fp32(O.OracleSim(p).snapshot())
    o, g = _both(p, blob)
    fo, fg = o.fields(), g.fields()
    assert np.array_equal(fo["R"], fg["R"])
    assert np.abs(fg["rho"] - fo["rho"]).max() <= 1e-13 * np.abs(fo["rho"]).max()
    s = max(np.abs(fo["phi"]).max(), 1.0)
    assert np.abs(fg["phi"] - fo["phi"]).max() <= stepcheck.cond_tol(p["ncells"]) * s
    sE = np.abs(fo["E"]).max()
    assert np.abs(fg["E"] - fo["E"]).max() <= 2.0**-23 * sE + stepcheck.cond_tol(p["ncells"]) * sE


def test_a_full_neutral_buffer_reports_an_overflow_and_drops_the_rest():
    # room for 6144 neutrals: 58 per cell at t = 0 and 400 more in the state leave 176 free slots;
    # 600 ions recycle in the first step
    p = W.variant(W.SMALL_C6, neutral_ppc=58, neutral_capacity=1.0, capacity_factor=2.0, K_iz=0.0)
    g = pic.Simulation(p)
    assert g.restore(_busy_blob(p, 17, step=3)) == 0  # an in-place step: recycled neutrals are appended
    g.step(1)
    with pytest.raises(pic.PicError) as e:
        g.sync()
    assert e.value.status == 4  # PIC_EOVERFLOW
    # the state can still be saved: the blob holds the neutrals that found a slot
    import zlib

    blob = g.snapshot()
    assert zlib.crc32(blob[:-4]) == int.from_bytes(blob[-4:], "little")
    nt = snapfmt.parse(blob)["neutrals"]
    assert 0 < len(nt["id"]) <= 6144 and len(np.unique(nt["id"])) == len(nt["id"])
    g.close()


def test_blobs_of_other_configurations_or_versions_are_refused():
    p = W.variant(W.SMALL_C6, **ROOMY)
    g = pic.Simulation(p)
    good = g.snapshot()
    assert snapfmt.parse(good)["version"] == 4
    assert g.restore(good[:-9] + good[-4:]) == 5                   # truncated: PIC_ECORRUPT
    other = pic.Simulation(W.variant(p, K_iz=0.25)).snapshot()     # other physics: other hash
    assert g.restore(other) == 5
    plain = pic.Simulation(W.variant(p, neutrals=0, neutral_ppc=0)).snapshot()
    assert snapfmt.parse(plain)["version"] == 3 and g.restore(plain) == 5
    assert g.restore(good) == 0
