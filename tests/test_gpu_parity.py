"""GPU path (through the C ABI) against the FP64 CPU oracle.

Every input of the oracle comes from the oracle itself or from seeded generators; the GPU is
given the same state (an oracle snapshot, rounded to FP32 where the FP32 path stores FP32) and
the two are compared particle by particle (matched by id), node by node, counter by counter.

Tolerances:
* Philox words, integer deposits of identical FP32 states, particle counts, ids: exact.
* FP32 single step: |dv| <= 1e-5 |v| + 1e-6 v_th and |dx| <= 2e-6 cells (FP32 fraction);
  collisions identical except near-threshold draws (bounded by both codes' counters).
* FP64 plain single step: 1e-11 relative.
* Field solve: the conditioning bound of tridiag(-1, 2, -1), 4 N^2/pi^2 * 2^-52, times max|phi|
  (plus the FP32 input rounding where the charge came from an FP32 step).
"""
import math
import struct

import numpy as np
import pytest

import snapfmt
import stepcheck
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


def _cond_tol(N):
    return max(1e-13, 4 * N * N / math.pi**2 * 2.0**-52)


def _by_id(sp):
    o = np.argsort(sp["id"])
    return {k: (v[o] if k != "v" else v[o, :]) for k, v in sp.items()}


def _oracle_blob_fp32(params, steps=0):
    o = O.OracleSim(params)
    if steps:
        o.step(steps)
    return snapfmt.round_to_fp32(o.snapshot())


# ------------------------------------------------------------------------------------------------
def test_philox_bit_exact_against_oracle():
    import torch

    rng = np.random.default_rng(1)
    n = 1 << 20
    ctr = rng.integers(0, 2**32, (n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2**32, (n, 2), dtype=np.uint64).astype(np.uint32)
    ctr[:3] = [[0, 0, 0, 0], [0xFFFFFFFF] * 4, [0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344]]
    key[:3] = [[0, 0], [0xFFFFFFFF] * 2, [0xA4093822, 0x299F31D0]]
    out = pic.philox(torch.from_numpy(ctr.view(np.int32)).cuda(),
                     torch.from_numpy(key.view(np.int32)).cuda()).cpu().numpy().view(np.uint32)
    ref = O.philox(ctr, key)
    assert np.array_equal(out, ref)
    assert out[0].tolist() == [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]


@pytest.mark.parametrize("N", [2, 3, 7, 100, 1023, 8191, 8192, 65536, 196607])
def test_poisson_matches_thomas(N):
    import torch

    rng = np.random.default_rng(N)
    dx = 0.5 + rng.random()
    rho = rng.standard_normal(N + 1) + 0.3
    VL, VR = -3.0 * rng.random(), rng.random()
    phi, E = pic.poisson(torch.from_numpy(rho).cuda(), dx, VL, VR)
    phi, E = phi.cpu().numpy(), E.cpu().numpy()
    ref = O.poisson_thomas(rho, dx, VL, VR)
    Eref = O.efield(ref, rho, dx)
    scale = np.abs(ref).max()
    assert phi[0] == VL and phi[N] == VR
    assert np.abs(phi - ref).max() <= _cond_tol(N) * scale
    assert np.abs(E - Eref).max() <= _cond_tol(N) * scale / dx * 4


def test_poisson_closed_form_on_gpu():
    import torch

    N, dx, r0 = 65536, 1.0, 0.25
    phi, E = pic.poisson(torch.full((N + 1,), r0, dtype=torch.float64, device="cuda"), dx, 0.0, 0.0)
    x = np.arange(N + 1) * dx
    exact = r0 * x * (N * dx - x) / 2
    assert np.abs(phi.cpu().numpy() - exact).max() <= _cond_tol(N) * exact.max()


# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("name", ["SMALL_C1", "SMALL_C3", "QUIET"])
def test_load_matches_oracle(name):
    p = W.variant(W.BASE, ncells=64, L=64.0, ppc=(37, 37), load_profile=W.LOAD_QUIET_SINE,
                  profile_scale=0.3, profile_mode=2) if name == "QUIET" else getattr(W, name)
    g = pic.Simulation(p)
    gs = snapfmt.parse(g.snapshot())["species"]
    os_ = snapfmt.parse(O.OracleSim(p).snapshot())["species"]
    for s in range(2):
        a, b = gs[s], os_[s]
        assert np.array_equal(a["id"], b["id"])
        xa, xb = a["cell"] + a["frac"], b["cell"] + b["frac"]
        assert np.abs(xa - xb).max() <= 2.0 ** -23  # FP32 rounding of the fraction
        vt = math.sqrt(p["T"][s] / p["mass"][s])
        assert np.abs(a["v"] - b["v"]).max() <= 1e-6 * vt * 8


def test_restore_deposit_is_bit_exact():
    # identical FP32-representable particle states deposit identical int64 charge on both sides
    for p in (W.SMALL_C2, W.SMALL_C3):
        blob = _oracle_blob_fp32(p)
        o = O.OracleSim(p)
        assert o.restore(blob) == 0
        g = pic.Simulation(p)
        assert g.restore(blob) == 0
        fo, fg = o.fields(), g.fields()
        assert np.array_equal(fo["R"], fg["R"])
        assert np.abs(fo["rho"] - fg["rho"]).max() <= 1e-15 * np.abs(fo["rho"]).max()
        scale = np.abs(fo["phi"]).max()
        assert np.abs(fo["phi"] - fg["phi"]).max() <= _cond_tol(p["ncells"]) * scale
        # the field the particles see (FP32), against the oracle's Thomas solve and centred
        # differences: FP32 rounding plus the conditioning bound of the solve
        escale = np.abs(fo["E"]).max()
        assert np.abs(fo["E"] - fg["E"]).max() <= 2.0**-23 * escale + _cond_tol(p["ncells"]) * scale
        # the snapshot round-trips byte for byte (format written independently on both sides)
        assert g.snapshot() == blob


def test_non_integer_charges_use_the_fp64_solve():
    # charges that are not small integers take the FP64 Green's function; same bar
    p = W.variant(W.SMALL_C2, charge=(-1.0, 1.5), ppc=(53, 35))
    blob = _oracle_blob_fp32(p)
    o = O.OracleSim(p)
    assert o.restore(blob) == 0
    g = pic.Simulation(p)
    assert g.restore(blob) == 0
    fo, fg = o.fields(), g.fields()
    assert np.array_equal(fo["R"], fg["R"])
    scale = np.abs(fo["phi"]).max()
    assert np.abs(fo["phi"] - fg["phi"]).max() <= _cond_tol(p["ncells"]) * scale
    escale = np.abs(fo["E"]).max()
    assert np.abs(fo["E"] - fg["E"]).max() <= 2.0**-23 * escale + _cond_tol(p["ncells"]) * scale
    o.step(2)
    g.step(2)
    assert o.diag()["n"] == g.diag()["n"]


@pytest.mark.parametrize("name", ["SMALL_C1", "SMALL_C2", "SMALL_C3", "SMALL_COLL"])
def test_single_step_fp32_matches_oracle(name):
    p = getattr(W, name)
    blob = _oracle_blob_fp32(p, steps=3)
    o = O.OracleSim(p)
    assert o.restore(blob) == 0
    g = pic.Simulation(p)
    assert g.restore(blob) == 0
    o.step(1)
    g.step(1)
    stepcheck.assert_one_step(p, blob, o.diag(), o.snapshot(), o.fields(), g.diag(), g.snapshot(), g.fields())


@pytest.mark.parametrize("name", ["SMALL_C1", "SMALL_C2", "SMALL_C3"])
def test_single_step_fp64_plain_matches_oracle(name):
    p = W.variant(getattr(W, name), precision=W.PRECISION_FP64_PLAIN)
    o = O.OracleSim(p)
    o.step(3)
    blob = o.snapshot()
    g = pic.Simulation(p)
    assert g.restore(blob) == 0
    o.step(2)
    g.step(2)
    so = snapfmt.parse(o.snapshot())["species"]
    sg = snapfmt.parse(g.snapshot())["species"]
    for s in range(2):
        a, b = _by_id(sg[s]), _by_id(so[s])
        assert np.array_equal(a["id"], b["id"])
        assert np.array_equal(a["cell"], b["cell"])
        assert np.abs(a["frac"] - b["frac"]).max() <= 1e-9
        assert np.abs(a["v"] - b["v"]).max() <= 1e-11 * max(1.0, np.abs(b["v"]).max())
    do, dg = o.diag(), g.diag()
    for k in ("n", "wall_hits", "coll", "births", "source_pairs", "wall_charge"):
        assert dg[k] == do[k], k
    assert abs(dg["ke"][0] - do["ke"][0]) <= 1e-6 * do["ke"][0]


def test_error_of_each_diagnostic_against_the_oracle():
    # one step from the same state (the GPU's FP32 values) in the oracle, the FP32 path and the plain
    # FP64 path: the energies within their arithmetic's rounding, the counts equal up to the
    # near-threshold draws both codes count
    p = W.variant(W.SMALL_C2, V_left=-2.0)
    g = pic.Simulation(p)
    g.step(20)
    blob = g.snapshot()
    o = O.OracleSim(p)
    assert o.restore(blob) == 0
    o.step(1)
    do = o.diag()
    # both GPU paths sum energies in 2^-24 fixed point per particle: up to n 2^-25 w of quantisation
    w = np.array([p["L"] / p["ncells"] / p["ppc"][s] for s in range(2)])
    quant = {"ke": np.array(do["n"]) * 2.0**-25 * w, "wall_energy": np.array(
        [sum(do["wall_hits"][s]) for s in range(2)]) * 2.0**-25 * w, "field_energy": 0.0}
    for prec, tol in ((W.PRECISION_FP32, {"ke": 1e-6, "wall_energy": 1e-6, "field_energy": 1e-3}),
                      (W.PRECISION_FP64_PLAIN, {"ke": 1e-12, "wall_energy": 1e-12, "field_energy": 1e-9})):
        h = pic.Simulation(W.variant(p, precision=prec))
        assert h.restore(blob) == 0
        h.step(1)
        d = h.diag()
        near = sum(d["near_threshold"]) + sum(do["near_threshold"]) - 2 * sum(snapfmt.parse(blob)["counters"][9:11])
        for k, t in tol.items():
            a, b = np.atleast_1d(d[k]), np.atleast_1d(do[k])
            assert np.all(np.abs(a - b) <= t * np.abs(b) + quant[k] + 1e-300), (prec, k, a, b)
        assert d["wall_hits"] == do["wall_hits"] and d["wall_charge"] == do["wall_charge"]
        assert all(abs(x - y) <= near for x, y in zip(d["coll"], do["coll"]))
        assert all(abs(x - y) <= 2 * near for x, y in zip(d["n"], do["n"]))
        h.close()


# ------------------------------------------------------------------------------------------------
def test_rerun_and_snapshot_continuation_are_bit_exact():
    p = W.variant(W.SMALL_COLL, sort_interval=3)
    a = pic.Simulation(p)
    a.step(7)
    blob7 = a.snapshot()
    a.step(6)
    b = pic.Simulation(p)
    assert b.restore(blob7) == 0
    b.step(6)
    c = pic.Simulation(p)
    c.step(13)
    sa, sb, sc = a.snapshot(), b.snapshot(), c.snapshot()
    assert sa == sb == sc
    da, db, dc = a.diag(), b.diag(), c.diag()
    for d in (da, db, dc):
        d.pop("particle_steps")  # counted since init / restore
    assert da == db == dc


def test_sort_interval_changes_nothing_but_the_order():
    # Sorting only reorders particles: every interval (1: a sort scan after every step and the
    # particles moved by the next step; 1000: never again after the initial sort) gives the same
    # particle set, byte-identical snapshots and identical diagnostics.
    base = W.variant(W.SMALL_COLL)
    ref = None
    for interval in (1, 2, 5, 1000):
        g = pic.Simulation(W.variant(base, sort_interval=interval))
        g.step(9)
        snap, d = g.snapshot(), g.diag()
        g.close()
        # the snapshot header carries the configuration hash (sort_interval is part of it)
        body = snap[24:-4]
        if ref is None:
            ref = (body, d)
        assert body == ref[0], interval
        assert d == ref[1], interval


def test_snapshot_while_the_sort_is_pending_continues_exactly():
    p = W.variant(W.SMALL_C3, sort_interval=4)
    a = pic.Simulation(p)
    a.step(1)  # step 0 sorted: the next step moves the particles to the other buffer
    blob = a.snapshot()
    a.step(6)
    b = pic.Simulation(p)
    assert b.restore(blob) == 0
    b.step(6)
    c = pic.Simulation(p)
    c.step(7)
    assert a.snapshot() == b.snapshot() == c.snapshot()


def test_step_kinetic_energy_is_the_exact_fixed_point_sum():
    # The FP32 step sums 0.5 m v^2 of every particle alive after the step (pushed, collided, born,
    # injected) in 2^-24 fixed point with each FP32 rounding spelled out; recomputing that sum
    # from the snapshot must give the same bits.
    for p, every in ((W.variant(W.SMALL_COLL), 1), (W.SMALL_C3, 1), (W.SMALL_C3, 0)):
        g = pic.Simulation(p)
        g.set_diag_interval(every)  # 1: summed in the step; 0: summed by pic_diag
        g.step(7)
        d = g.diag()
        sp = snapfmt.parse(g.snapshot())["species"]
        for s in range(2):
            v = sp[s]["v"].astype(np.float32)
            t = (v[:, 0] * v[:, 0] + v[:, 1] * v[:, 1]) + v[:, 2] * v[:, 2]
            e = (np.float32(0.5) * np.float32(p["mass"][s])) * t * np.float32(2.0**24)
            fx = int(np.rint(e.astype(np.float64)).astype(np.uint64).sum(dtype=np.uint64))
            w = (p["L"] / p["ncells"]) / p["ppc"][s]
            assert d["ke"][s] == float(fx) * (1.0 / 16777216.0) * w


def test_diag_interval_changes_no_bit_of_the_diagnostics():
    p = W.variant(W.SMALL_COLL, sort_interval=4)
    sims = [pic.Simulation(p) for _ in range(3)]
    for g, every in zip(sims, (0, 1, 3)):
        g.set_diag_interval(every)
    for _ in range(9):
        for g in sims:
            g.step(1)
        d = [g.diag() for g in sims]
        assert d[0] == d[1] == d[2]
    with pytest.raises(pic.PicError):
        sims[0].set_diag_interval(-1)
    for g in sims:
        g.close()


def test_asynchronous_diagnostics_equal_the_synchronous_ones():
    # pic_diag_async copies the control block as pic_diag would read it at that call; the host decodes
    # it after later steps were enqueued, and gets the diagnostics of the earlier state
    import torch

    p = W.variant(W.SMALL_C3, V_left=-2.0)
    a, b = pic.Simulation(p), pic.Simulation(p)
    a.set_diag_interval(1)  # also the path where the step sums the kinetic energy
    nb = pic.lib().pic_diag_bytes()
    bufs = [torch.empty(nb, dtype=torch.uint8, pin_memory=True) for _ in range(2)]
    evs = [torch.cuda.Event() for _ in range(2)]
    ref = []
    for k in range(12):
        b.step(1)
        ref.append(b.diag())
        a.step(1)
        a.diag_async(bufs[k % 2])
        evs[k % 2].record(a.stream)
        if k:
            evs[(k - 1) % 2].synchronize()
            assert a.diag_decode(bufs[(k - 1) % 2]) == ref[k - 1]
    evs[11 % 2].synchronize()
    assert a.diag_decode(bufs[11 % 2]) == ref[11] == a.diag()
    # counters only: no reduction runs; the energies and the net charge read 0, the rest is the same
    a.diag_async(bufs[0], counters_only=True)
    torch.cuda.synchronize()
    c = a.diag_decode(bufs[0])
    full = a.diag()
    assert c["ke"] == [0.0, 0.0] and c["field_energy"] == 0.0 and c["net_charge_units"] == 0
    for k in ("step", "n", "wall_hits", "coll", "births", "source_pairs", "particle_steps", "wall_energy"):
        assert c[k] == full[k], k
    with pytest.raises(ValueError):
        a.diag_async(torch.empty(8, dtype=torch.uint8, pin_memory=True))
    a.close()
    b.close()


def test_charge_and_accounting_invariants_every_step():
    p = W.variant(W.SMALL_C3, V_left=-2.0)
    g = pic.Simulation(p)
    d0 = g.diag()
    q0 = d0["n"][1] - d0["n"][0]
    for _ in range(25):
        g.step(1)
        d = g.diag()
        assert d["net_charge_units"] == 2**32 * (d["n"][1] - d["n"][0])
        assert (d["n"][1] - d["n"][0]) + d["wall_charge"] == q0
        assert d["source_pairs"] == d["wall_hits"][1][0] + d["wall_hits"][1][1]
        for s in range(2):
            lost = d["wall_hits"][s][0] + d["wall_hits"][s][1]
            assert d["n"][s] == d0["n"][s] + d["births"][s] - lost + d["source_pairs"]


def test_restore_error_codes():
    p = W.SMALL_C1
    g = pic.Simulation(p)
    blob = bytearray(g.snapshot())
    blob[250] ^= 0x10
    assert g.restore(bytes(blob)) == 5
    assert g.restore(g.snapshot()[:-5]) == 5
    other = pic.Simulation(W.variant(p, seed=p["seed"] + 7))
    assert g.restore(other.snapshot()) == 5
    # more particles than the capacity
    o = O.OracleSim(p)
    d = snapfmt.parse(o.snapshot())
    big = [{"x": np.random.default_rng(0).uniform(0, p["ncells"], 3 * len(s["id"])),
            "v": np.zeros((3 * len(s["id"]), 3)), "id": np.arange(3 * len(s["id"]))}
           for s in d["species"]]
    assert g.restore(snapfmt.with_particles(o.snapshot(), big)) == 4


def test_large_blob_restore_checks_on_the_device():
    # A blob of 16 MB or more (FP32 path) is checked on the device: the CRC of its 64 KB blocks,
    # joined on the host with the tail past the last full block, and every record's range.  Damage
    # anywhere -- inside a block, in the tail, in the stored CRC -- or a record out of range under a
    # valid CRC is PIC_ECORRUPT with the state untouched; the intact blob restores bit for bit.
    import zlib

    p = W.variant(W.SMALL_C3, ppc=(500, 500))
    g = pic.Simulation(p)
    g.step(4)
    blob = g.snapshot()
    g.close()
    assert len(blob) >= 16 << 20
    h = pic.Simulation(p)
    h.step(1)
    before = h.snapshot()
    n = len(blob) - 4
    for pos in (n // 2 + 12345, n - 100, n + 1):
        bad = bytearray(blob)
        bad[pos] ^= 0x04
        assert h.restore(bytes(bad)) == 5, pos
        assert h.snapshot() == before

    def with_crc(b):
        b[-4:] = (zlib.crc32(bytes(b[:-4])) & 0xFFFFFFFF).to_bytes(4, "little")
        return bytes(b)

    hdr = 208  # header bytes before species 0's cell words
    m0 = int.from_bytes(blob[32:40], "little")
    bad = bytearray(blob)
    w = int.from_bytes(bad[hdr + 4 * 7: hdr + 4 * 8], "little")
    bad[hdr + 4 * 7: hdr + 4 * 8] = ((w & ~0x3FFFF) | p["ncells"]).to_bytes(4, "little")  # cell N
    assert h.restore(with_crc(bad)) == 5
    bad = bytearray(blob)
    bad[hdr + 4 * m0 + 8 * 11: hdr + 4 * m0 + 8 * 12] = struct.pack("<d", 1.0)  # fraction 1
    assert h.restore(with_crc(bad)) == 5
    bad = bytearray(blob)
    w = int.from_bytes(bad[hdr + 4 * 3: hdr + 4 * 4], "little")
    bad[hdr + 4 * 3: hdr + 4 * 4] = ((w & 0x3FFFF) | (0x1000 << 18)).to_bytes(4, "little")  # countdown 0, flag 1
    assert h.restore(with_crc(bad)) == 5
    assert h.snapshot() == before
    assert h.restore(blob) == 0
    assert h.snapshot() == blob
    h.close()


@pytest.mark.parametrize("precision", [W.PRECISION_FP32, W.PRECISION_FP64_PLAIN])
def test_config1_long_run_moments_match_the_oracle_statistically(precision):
    # Config 1 (256 cells, 100 ppc per species, 1000 steps; R16: parity of long runs is statistical):
    # 24 moments (counts over time, wall losses, collisions, energies, T_e, the time-averaged
    # potential at 8 nodes) of 8 GPU seeds against 16 oracle seeds, each moment by a two-sided Welch
    # test at a family-wise level of 1e-3 (Bonferroni: every p-value >= 1e-3 / 24).  A correct code
    # fails this with probability <= 1e-3 (for moments close to normal).
    import multiprocessing as mp

    import longrun

    base = W.variant(W.C1, precision=precision)
    with mp.get_context("spawn").Pool(min(16, max(2, len(__import__("os").sched_getaffinity(0))))) as pool:
        ora = pool.map_async(longrun.oracle_moments, [(base, 5000 + k) for k in range(16)])
        gpu = []
        for k in range(8):
            g = pic.Simulation(W.variant(base, seed=7000 + k))
            gpu.append(longrun.run(g, base))
            g.close()
        ora = np.array(ora.get())
    gpu = np.array(gpu)
    pv = longrun.welch_pvalues(gpu, ora)
    bad = [(longrun.NAMES[k], gpu[:, k].mean(), ora[:, k].mean(), ora[:, k].std(ddof=1), pv[k])
           for k in range(len(pv)) if pv[k] < 1e-3 / len(pv)]
    assert not bad, bad


# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("name", ["C2", "C3"])
def test_full_size_sampled_load_and_invariants(name):
    p = getattr(W, name)
    g = pic.Simulation(p)
    d0 = g.diag()
    n0 = [p["ppc"][s] * p["ncells"] for s in range(2)]
    assert d0["n"] == n0
    # sampled particles of the initial load, computed one by one by the oracle (the 100M-particle
    # case is checked through its invariants only: its snapshot would be a 4.4 GB host blob)
    blob = g.snapshot() if name == "C2" else None
    sp = snapfmt.parse(blob)["species"] if blob else None
    if blob:
        # checksum of a large blob (threaded on both sides of the format) against zlib, and a
        # restore of it into a fresh handle writes the same bytes back
        import zlib

        assert zlib.crc32(blob[:-4]) & 0xFFFFFFFF == int.from_bytes(blob[-4:], "little")
        g2 = pic.Simulation(p)
        assert g2.restore(blob) == 0
        assert g2.snapshot() == blob
        g2.close()
    rng = np.random.default_rng(3)
    for s in range(2 if sp else 0):
        idx = rng.choice(n0[s], 2000, replace=False)
        x, v, ids = O.load_particles(p, s, idx)
        pos = np.searchsorted(sp[s]["id"], ids)
        assert np.array_equal(sp[s]["id"][pos], ids)
        xg = sp[s]["cell"][pos] + sp[s]["frac"][pos]
        assert np.abs(xg - x).max() <= 2.0 ** -23 * 2
        vt = math.sqrt(p["T"][s] / p["mass"][s])
        assert np.abs(sp[s]["v"][pos] - v).max() <= 8e-6 * vt
    g.step(12)
    d = g.diag()
    assert d["dropped"] == 0
    assert d["net_charge_units"] == 2**32 * (d["n"][1] - d["n"][0])
    assert (d["n"][1] - d["n"][0]) + d["wall_charge"] == n0[1] - n0[0]
    for s in range(2):
        lost = d["wall_hits"][s][0] + d["wall_hits"][s][1]
        assert d["n"][s] == n0[s] + d["births"][s] - lost + d["source_pairs"]
    assert d["coll"][4] > 0 and d["coll"][0] > 0




def _species_views(blob: bytes) -> list:
    """(cell, frac, v columns, id, countdown pair) of each charged species of a snapshot, as views
    into the blob (cell and pair split from the cell word)."""
    n = struct.unpack_from("<QQ", blob, 32)
    off, out = snapfmt.HDR, []
    for m in n:
        word = np.frombuffer(blob, np.uint32, m, off)
        frac = np.frombuffer(blob, np.float64, m, off + 4 * m)
        v = [np.frombuffer(blob, np.float64, m, off + 12 * m + 8 * m * k) for k in range(3)]
        ids = np.frombuffer(blob, np.uint64, m, off + 36 * m)
        out.append(((word & snapfmt.CELL_MASK).astype(np.int32), frac, v, ids, word >> snapfmt.CELL_BITS))
        off += 44 * m
    return out


def test_full_size_sampled_step_matches_the_oracle_one_by_one():
    # config 3 at full size (1e8 particles) in the bench's launch configuration: 2000 particles of
    # each species, stepped one by one by the oracle (orc_step_sample: mover, walls, null-collision
    # MC) under the GPU's own node field, against the GPU's step of the whole state; the tolerances
    # of the single-step parity, absorption exact away from the walls, near-threshold draws counted
    p = W.C3
    g = pic.Simulation(p)
    g.step(3)  # the step that follows is an ordinary one (sorts run at multiples of 10)
    step = g.diag()["step"]
    E = g.fields()["E"].astype(np.float64)
    before = _species_views(g.snapshot())
    g.step(1)
    after = _species_views(g.snapshot())
    rng = np.random.default_rng(17)
    N = p["ncells"]
    # every particle of the stepped state deposited exactly once (at this size the step claims its
    # chunks in segments from a grid-wide counter): the node deposits equal the CIC deposit of the
    # stored particles, W_r = rint(f 2^32) (ties to even), summed here exactly (integers below 2^53)
    R = g.fields()["R"]
    for s in range(2):
        cell1, frac1 = after[s][0], after[s][1]
        wr = np.rint(frac1 * 2.0**32)
        Rh = (np.bincount(cell1, weights=2.0**32 - wr, minlength=N + 1)
              + np.bincount(cell1 + 1, weights=wr, minlength=N + 1))
        assert np.array_equal(Rh.astype(np.int64), R[s]), s
    for s in range(2):
        cell, frac, v, ids, nk = before[s]
        # 2000 anywhere, and up to 300 in the wall cells, where particles leave
        edge = np.flatnonzero((cell == 0) | (cell == N - 1))
        idx = np.union1d(rng.choice(len(ids), 2000, replace=False),
                         rng.choice(edge, min(300, edge.size), replace=False))
        x0 = cell[idx] + frac[idx]
        v0 = np.stack([c[idx] for c in v], 1)
        xo, vo, nko, fl = O.step_sample(p, s, step, E, x0, v0, ids[idx], nk[idx])
        cell1, frac1, v1, ids1, nk1 = after[s]
        pos = np.minimum(np.searchsorted(ids1, ids[idx]), len(ids1) - 1)
        found = ids1[pos] == ids[idx]
        absorbed = (fl & 1) != 0
        near = (fl & 4) != 0
        at_wall = (np.abs(xo) < 1e-4) | (np.abs(xo - N) < 1e-4)
        assert np.array_equal(found | near | at_wall, ~absorbed | near | at_wall)
        ok = found & ~absorbed
        xg = cell1[pos[ok]] + frac1[pos[ok]]
        vg = np.stack([c[pos[ok]] for c in v1], 1)
        vt = math.sqrt(p["T"][s] / p["mass"][s])
        dv = np.abs(vg - vo[ok]).max(axis=1)
        bad = (dv > 1e-5 * np.abs(vo[ok]).max(axis=1) + 1e-6 * vt) | (np.abs(xg - xo[ok]) > 2e-6)
        bad |= nk1[pos[ok]] != nko[ok]  # the null-collision countdown: exact
        assert int((bad & ~near[ok]).sum()) == 0, (s, int(bad.sum()))
        if s == 0:  # electrons: some sampled ones leave, some are collision candidates (P_null 1 %)
            assert int(absorbed.sum()) > 0
            assert int(((fl & 2) != 0).sum()) > 0


def test_full_size_config2_step_matches_the_oracle_for_every_particle():
    # config 2 at full size (8,192,000 particles, 4096 cells) in the launch configuration the bench
    # uses: the oracle's state rounded to FP32 is restored on both sides and both take one step; every
    # particle is matched by id at the single-step tolerances and every node's int64 deposit R within
    # the FP32 position bound (stepcheck).  Then the same for the step that follows a sort step (the
    # GPU's k_step32 in scatter mode), from the state the GPU's sort step left.
    import os

    p = W.C2
    cores = len(os.sched_getaffinity(0))
    o = O.OracleSim(p, threads=cores)
    o.step(2)
    blob = snapfmt.round_to_fp32(o.snapshot())
    assert o.restore(blob) == 0
    g = pic.Simulation(p)
    assert g.restore(blob) == 0
    o.step(1)
    g.step(1)
    mism, near = stepcheck.assert_one_step(p, blob, o.diag(), o.snapshot(), o.fields(), g.diag(), g.snapshot(),
                                           g.fields())
    assert mism <= 4 * near
    o.close()
    # steps 3 .. 9 ordinary, step 10 sorts (cursors only); step 11 moves every particle to its slot
    g.step(8)
    assert g.diag()["step"] == 11
    blob2 = g.snapshot()
    o2 = O.OracleSim(p, threads=cores)
    assert o2.restore(blob2) == 0
    o2.step(1)
    g.step(1)
    stepcheck.assert_one_step(p, blob2, o2.diag(), o2.snapshot(), o2.fields(), g.diag(), g.snapshot(), g.fields())


def test_full_size_long_run_keeps_every_invariant():
    # the 100M-particle workload over 1000 steps, the bench's timed run (100 sorts, the pair source
    # balancing the ion losses, ionization births growing each species by about 8 %): charge,
    # particle accounting and capacity hold at every check, and nothing is dropped
    p = W.C3
    g = pic.Simulation(p)
    n0 = [p["ppc"][s] * p["ncells"] for s in range(2)]
    cap = [int(p["capacity_factor"] * n) for n in n0]
    for _ in range(4):
        g.step(250)
        d = g.diag()
        assert d["dropped"] == 0
        assert d["net_charge_units"] == 2**32 * (d["n"][1] - d["n"][0])
        assert (d["n"][1] - d["n"][0]) + d["wall_charge"] == n0[1] - n0[0]
        for s in range(2):
            lost = d["wall_hits"][s][0] + d["wall_hits"][s][1]
            assert d["n"][s] == n0[s] + d["births"][s] - lost + d["source_pairs"]
            assert d["n"][s] <= cap[s]
        assert all(math.isfinite(x) for x in d["ke"]) and math.isfinite(d["field_energy"])
    assert d["step"] == 1000
    # the source has replaced the ions lost at the walls, one pair each
    assert d["source_pairs"] == d["wall_hits"][1][0] + d["wall_hits"][1][1]


# ---- edge cases ---------------------------------------------------------------------------------
def test_largest_grid_steps_and_matches_the_oracle():
    # the largest grid the FP32 path takes (8 CTAs of the field cluster x 24576 nodes, minus one)
    N = 8 * 24576 - 1
    p = W.variant(W.SMALL_C2, ncells=N, L=float(N), ppc=(1, 1), sort_interval=2)
    blob = _oracle_blob_fp32(p, steps=2)
    o = O.OracleSim(p)
    assert o.restore(blob) == 0
    g = pic.Simulation(p)
    assert g.restore(blob) == 0
    o.step(1)
    g.step(1)
    stepcheck.assert_one_step(p, blob, o.diag(), o.snapshot(), o.fields(), g.diag(), g.snapshot(), g.fields())
    g.step(5)  # across a sort and the step that moves the particles
    d = g.diag()
    assert d["net_charge_units"] == 2**32 * (d["n"][1] - d["n"][0])
    with pytest.raises(pic.PicError):
        pic.Simulation(W.variant(p, ncells=N + 1, L=float(N + 1)))


def test_species_that_empty_out_keep_stepping():
    # two cells, hot particles (seed chosen so that every particle reaches a wall within five
    # steps): the run goes on with empty species (zero extents), through sorts, and agrees with the
    # oracle throughout
    p = W.variant(W.SMALL_C1, ncells=2, L=2.0, ppc=(3, 3), T=(1e4, 1e6), sort_interval=2, coll_mask=0,
                  seed=3)
    o = O.OracleSim(p)
    g = pic.Simulation(p)
    for _ in range(12):
        o.step(1)
        g.step(1)
        do, dg = o.diag(), g.diag()
        assert dg["n"] == do["n"] and dg["wall_hits"] == do["wall_hits"]
        assert dg["net_charge_units"] == 2**32 * (dg["n"][1] - dg["n"][0])
    assert dg["n"] == [0, 0]
    a, b = snapfmt.parse(g.snapshot()), snapfmt.parse(o.snapshot())
    assert np.array_equal(a["counters"], b["counters"]) and a["wall_charge"] == b["wall_charge"]
    assert all(len(sp["id"]) == 0 for sp in a["species"])


def test_a_device_wait_that_cannot_complete_reports_a_timeout_and_the_context_survives():
    # failure detection without a fault: the bounded wait used by the particle kernels gives up after
    # its limit (about a second), the host reads PIC_ETIMEOUT, and the GPU keeps working
    rc, sec = pic.selftest_timeout()
    assert rc == 6, rc  # PIC_ETIMEOUT
    assert 0.5 < sec < 5.0, sec
    g = pic.Simulation(W.SMALL_C2)
    g.step(3)
    g.sync()
    assert g.diag()["step"] == 3
    g.close()
