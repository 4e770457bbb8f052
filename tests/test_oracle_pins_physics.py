"""Simulation-level pins of the oracle against physics and mathematics it must reproduce.

Each test fixes its expectation from outside the oracle: exact integer invariants (charge,
particle accounting), closed forms (cold plasma frequency under leapfrog, uniform-background
field, Maxwellian moments, n sigma <v> collision rates, kinematic energy balances), and
properties of a permutation (sorting) and of a serialisation (snapshots).
"""
import math

import numpy as np
import pytest
from scipy import integrate, stats

import snapfmt
from oracle import oracle as O
from paper_2606_28534_gb300 import workloads as W


def _sim(p, threads=1):
    return O.OracleSim(p, threads=threads)


# ------------------------------------------------------------------------------------------------
def test_charge_and_particle_accounting_exact_every_step():
    p = W.variant(W.SMALL_COLL, V_left=-2.0)
    s = _sim(p)
    d0 = s.diag()
    q0 = d0["n"][1] - d0["n"][0]
    for _ in range(30):
        s.step(1)
        d = s.diag()
        # every particle deposits exactly 2^32 units in total
        assert d["net_charge_units"] == 2**32 * (d["n"][1] - d["n"][0])
        # charge that left through the walls plus charge inside is conserved (pairs are neutral)
        assert (d["n"][1] - d["n"][0]) + d["wall_charge"] == q0
        for sp in range(2):
            lost = d["wall_hits"][sp][0] + d["wall_hits"][sp][1]
            assert d["n"][sp] == d0["n"][sp] + d["births"][sp] - lost
    assert d["coll"][2] > 0 and d["births"][0] == d["births"][1] == d["coll"][2]


def test_source_replaces_each_absorbed_ion():
    p = W.variant(W.SMALL_C3, V_left=0.0)
    s = _sim(p)
    n0 = s.diag()["n"][1]
    s.step(40)
    d = s.diag()
    ion_lost = d["wall_hits"][1][0] + d["wall_hits"][1][1]
    assert d["source_pairs"] == ion_lost > 0
    assert d["n"][1] == n0 + d["births"][1]
    x, v, ids = s.particles(1)
    # source ids: top bit, injection step in bits 32..62, 2k+1 for the ion of pair k; children of
    # ionization carry random ids and match this pattern with probability ~ 40/2^31
    step_field = (ids >> np.uint64(32)) & np.uint64(0x7FFFFFFF)
    src = ((ids >> np.uint64(63)) == 1) & (step_field < 40) & ((ids & np.uint64(1)) == 1)
    assert src.sum() == d["source_pairs"]
    # ions move less than 0.5 dx in 40 steps at T_i = 0.1
    assert (x[src] < p["source_x1"] + 0.5).all()


def test_deposit_charge_and_centroid_moments():
    # CIC puts the whole particle on its two nodes (zeroth moment) and preserves its position
    # (first moment): sum_j R_j = 2^32 N and sum_j j R_j = 2^32 sum_p x_p up to rint rounding.
    p = W.variant(W.BASE, ncells=8, L=8.0, ppc=(8, 3), coll_mask=0, field_mode=W.FIELD_ZERO)
    s = _sim(p)
    rng = np.random.default_rng(11)
    xs = [rng.uniform(0, 8, 64), np.array([0.0, 3.0, 7.999999])]
    sp = [{"x": x, "v": np.zeros((len(x), 3)), "id": np.arange(len(x)) + 1000 * k}
          for k, x in enumerate(xs)]
    assert s.restore(snapfmt.with_particles(s.snapshot(), sp)) == 0
    R = s.fields()["R"]
    for k, x in enumerate(xs):
        assert R[k].sum() == 2**32 * len(x)
        first = (np.arange(9, dtype=object) * R[k].astype(object)).sum()
        exact = sum(int(round(xx * 2**32)) for xx in x)
        assert abs(first - exact) <= len(x)
    # a particle on a node deposits on that node only
    assert R[1][3] >= 2**32 and R[1][0] == 2**32


def test_uniform_background_field_and_push():
    # frozen uniform ions, grounded walls: rho = w*ppc/dx = 1 inside, so E(x) = x - L/2 and an
    # electron at rest gains dv_x = -E(x) dt in one step (B = 0).
    p = W.variant(W.BASE, ncells=64, L=64.0, ppc=(2000, 400), coll_mask=0, frozen_mask=2,
                  load_profile=W.LOAD_QUIET_SINE, profile_scale=0.0, T=(0.0, 0.0))
    s = _sim(p)
    blob = s.snapshot()
    d = snapfmt.parse(blob)
    ions = d["species"][1]
    xe = np.array([10.25, 31.7, 50.5])
    sp = [{"x": xe, "v": np.zeros((3, 3)), "id": np.arange(3)},
          {"x": ions["cell"] + ions["frac"], "v": ions["v"], "id": ions["id"]}]
    assert s.restore(snapfmt.with_particles(blob, sp)) == 0
    s.step(1)
    x, v, ids = s.particles(0)
    o = np.argsort(ids)
    expect = -(xe - 32.0) * 0.1
    assert np.allclose(v[o, 0], expect, rtol=2e-3, atol=1e-4)
    assert np.allclose(x[o], xe + expect * 0.1, rtol=0, atol=1e-4)


def test_cold_plasma_oscillation_frequency():
    # cold electrons displaced by A sin(2 pi x/L) over frozen ions oscillate at the leapfrog
    # plasma frequency w = (2/dt) asin(w_p dt/2) (finite-grid corrections ~ (k dx)^2 ~ 1e-4).
    p = W.variant(W.BASE, ncells=256, L=256.0, ppc=(64, 64), coll_mask=0, frozen_mask=2,
                  load_profile=W.LOAD_QUIET_SINE, profile_mode=1, profile_scale=0.02,
                  T=(0.0, 0.0))
    s = _sim(p)
    nsteps, j = 700, 64
    series = [s.fields()["E"][j]]
    for _ in range(nsteps):
        s.step(1)
        series.append(s.fields()["E"][j])
    e = np.array(series)
    z = np.where(np.sign(e[:-1]) != np.sign(e[1:]))[0]
    t = z + e[z] / (e[z] - e[z + 1])  # linear interpolation of the zero crossings (in steps)
    half_periods = np.diff(t)
    w = np.pi / (half_periods.mean() * p["dt"])
    expect = (2 / p["dt"]) * math.asin(p["dt"] / 2)
    assert abs(expect - 1.000417) < 1e-6
    assert abs(w - expect) / expect < 1e-3, (w, expect)


def test_collisionless_energy_bounded():
    # grounded walls, no collisions: kinetic + field + wall-absorbed energy stays constant to the
    # leapfrog/grid accuracy; a reversed force or a wrong weight would run away.
    p = W.variant(W.BASE, ncells=128, L=128.0, ppc=(100, 100), coll_mask=0)
    s = _sim(p)

    def total(d):
        return sum(d["ke"]) + d["field_energy"] + sum(d["wall_energy"])

    e0 = total(s.diag())
    s.step(200)
    d = s.diag()
    assert sum(d["wall_energy"]) > 0
    assert abs(total(d) - e0) / e0 < 0.02, (total(d), e0)


# ------------------------------------------------------------------------------------------------
def _maxwell_mean_speed(T, m):
    return math.sqrt(8 * T / (math.pi * m))


@pytest.mark.parametrize("sigma_el", [0.1, 2.0])
def test_elastic_rate_matches_n_sigma_mean_speed(sigma_el):
    # constant cross section: collisions per particle-step = P_null nu/nu_max; summed over a
    # Maxwellian this is (1 - e^{-a})/a * n sigma <|v|> dt, a = nu_max dt (the chance that a
    # Poisson process of rate nu_max has an event within dt is 1 - e^{-a}).  sigma_el = 2 makes
    # a ~ 1.6, where that chance is far from its first-order value a.
    p = W.variant(W.BASE, ncells=200, L=200.0, ppc=(500, 1), coll_mask=W.COLL_EL,
                  field_mode=W.FIELD_ZERO, sigma_el=sigma_el)
    s = _sim(p)
    n = s.count(0)
    steps = 4
    s.step(steps)
    d = s.diag()
    numax, _ = O.nu_max(p)
    a = float(numax[0]) * p["dt"]
    expect = n * steps * (1 - math.exp(-a)) / a * p["n_gas"] * p["sigma_el"] * \
        _maxwell_mean_speed(1.0, 1.0) * p["dt"]
    sig = math.sqrt(expect)
    assert abs(d["coll"][0] - expect) < 4 * sig, (d["coll"][0], expect)
    # all candidates of electrons are elastic or null; no other process fires
    assert d["coll"][1] == d["coll"][2] == d["coll"][3] == 0


def _rate_integral(sig_of_E, T=1.0, m=1.0):
    # <sigma(E) |v|> for a 3D Maxwellian, by quadrature over speed
    f = lambda v: 4 * np.pi * v**2 * (m / (2 * np.pi * T)) ** 1.5 * np.exp(-m * v * v / (2 * T))
    val, _ = integrate.quad(lambda v: f(v) * sig_of_E(0.5 * m * v * v) * v, 0, 12, limit=200)
    return val


def test_threshold_process_rates_match_maxwellian_integrals():
    p = W.variant(W.BASE, ncells=200, L=200.0, ppc=(600, 1), field_mode=W.FIELD_ZERO,
                  coll_mask=W.COLL_EL | W.COLL_EX | W.COLL_IZ, sigma_el=0.05, sigma_ex=0.05,
                  sigma_iz=0.05, E_ex=1.5, E_iz=2.5)
    s = _sim(p)
    n = s.count(0)
    s.step(1)
    d = s.diag()
    numax, _ = O.nu_max(p)
    a = float(numax[0]) * p["dt"]
    fac = n * (1 - math.exp(-a)) / a * p["dt"] * p["n_gas"]
    lin = lambda E, E0, s0: s0 * min(max(E - E0, 0) / E0, 1.0) if E > E0 else 0.0
    exp_el = fac * _rate_integral(lambda E: p["sigma_el"])
    exp_ex = fac * _rate_integral(lambda E: lin(E, p["E_ex"], p["sigma_ex"]))
    exp_iz = fac * _rate_integral(lambda E: lin(E, p["E_iz"], p["sigma_iz"]))
    for got, exp in ((d["coll"][0], exp_el), (d["coll"][1], exp_ex), (d["coll"][2], exp_iz)):
        assert abs(got - exp) < 4 * math.sqrt(exp) + 2, (got, exp)


def _beam_sim(p, E0, n=4000):
    s = _sim(p)
    blob = s.snapshot()
    rng = np.random.default_rng(5)
    sp0 = math.sqrt(2 * E0)
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    x = rng.uniform(20, 40, n)
    sp = [{"x": x, "v": sp0 * d, "id": np.arange(n)},
          {"x": np.array([30.0]), "v": np.zeros((1, 3)), "id": np.array([2**62])}]
    assert s.restore(snapfmt.with_particles(blob, sp)) == 0
    return s, sp0 * d


def test_elastic_kinematics_energy_loss_and_isotropy():
    # isotropic elastic scattering off a neutral of mass M: E'/E = 1 - (2m/M)(1 - cos chi),
    # whose average over directions is 1 - 2m/M; new directions are uniform on the sphere.
    M = 8.0
    p = W.variant(W.BASE, ncells=64, L=64.0, ppc=(1, 1), field_mode=W.FIELD_ZERO,
                  coll_mask=W.COLL_EL, n_gas=400.0, m_gas=M)
    s, v0 = _beam_sim(p, 4.0)
    s.step(1)
    x, v, ids = s.particles(0)
    v = v[np.argsort(ids)]
    hit = np.linalg.norm(v - v0, axis=1) > 1e-9
    assert hit.sum() > 1000
    ratio = (v[hit] ** 2).sum(1) / (v0[hit] ** 2).sum(1)
    cchi = (v[hit] * v0[hit]).sum(1) / np.linalg.norm(v[hit], axis=1) / np.linalg.norm(v0[hit], axis=1)
    assert np.allclose(ratio, 1 - 2 / M * (1 - cchi), atol=1e-12)
    assert abs(ratio.mean() - (1 - 2 / M)) < 4 * ratio.std() / math.sqrt(hit.sum())
    dirs = v[hit] / np.linalg.norm(v[hit], axis=1)[:, None]
    assert stats.kstest((dirs[:, 2] + 1) / 2, "uniform").pvalue > 1e-4
    assert stats.kstest((np.arctan2(dirs[:, 1], dirs[:, 0]) + np.pi) / (2 * np.pi),
                        "uniform").pvalue > 1e-4


def test_excitation_and_ionization_energy_balance():
    p = W.variant(W.BASE, ncells=64, L=64.0, ppc=(1, 1), field_mode=W.FIELD_ZERO,
                  coll_mask=W.COLL_EX | W.COLL_IZ, n_gas=40.0, sigma_ex=0.05, sigma_iz=0.05,
                  E_ex=1.0, E_iz=2.0, Tg=0.3)
    E0 = 6.0
    s, v0 = _beam_sim(p, E0)
    s.step(1)
    x, v, ids = s.particles(0)
    orig = ids < 4000
    vo = v[orig][np.argsort(ids[orig])]
    Eo = 0.5 * (vo**2).sum(1)
    changed = np.abs(Eo - E0) > 1e-9
    d = s.diag()
    assert d["coll"][1] > 100 and d["coll"][2] > 100
    # each changed electron lost exactly E_ex (excitation) or at least E_iz (ionization)
    ex = np.isclose(Eo[changed], E0 - 1.0, atol=1e-12)
    assert ex.sum() == d["coll"][1]
    assert (Eo[changed][~ex] <= E0 - 2.0 + 1e-12).all()
    # ionization: primary + secondary energies = E0 - E_iz, secondary share uniform in [0, 1]
    kid_e = ~orig
    assert kid_e.sum() == d["coll"][2] == d["births"][0]
    Es = 0.5 * (v[kid_e] ** 2).sum(1)
    # pair each child with its parent through the energy balance: sorted sums
    Ep = np.sort(Eo[changed][~ex])
    assert np.isclose(Ep.sum() + Es.sum(), d["coll"][2] * (E0 - 2.0), rtol=1e-12)
    assert stats.kstest(Es / (E0 - 2.0), "uniform").pvalue > 1e-4
    # new ions: Maxwellian at T_g
    xi, vi, idi = s.particles(1)
    newi = idi != 2**62
    assert newi.sum() == d["coll"][2]
    var = vi[newi].var(axis=0)
    assert np.allclose(var, 0.3 / 7344.0, rtol=0.2)


def test_charge_exchange_ions_thermalise_to_gas():
    p = W.variant(W.BASE, ncells=64, L=64.0, ppc=(1, 2000), field_mode=W.FIELD_ZERO,
                  coll_mask=W.COLL_CX, sigma_cx=2000.0, T=(1.0, 4.0), Tg=0.1)
    s = _sim(p)
    x0, v0, id0 = s.particles(1)
    s.step(1)
    d = s.diag()
    x, v, ids = s.particles(1)
    # ions that reached a wall in this step are gone; compare the survivors by id
    _, i0, i1 = np.intersect1d(id0, ids, return_indices=True)
    assert len(i1) == len(ids) and len(ids) + sum(d["wall_hits"][1]) == len(id0)
    vn = v[i1]
    changed = np.linalg.norm(vn - v0[i0], axis=1) > 1e-12
    assert changed.sum() == d["coll"][3] > 1000
    vt2 = 0.1 / 7344.0
    var = vn[changed].var(axis=0)
    assert np.allclose(var, vt2, rtol=0.1)
    assert stats.kstest(vn[changed][:, 0] / math.sqrt(vt2), "norm").pvalue > 1e-4


# ------------------------------------------------------------------------------------------------
def test_loader_uniform_maxwellian():
    p = W.variant(W.BASE, ncells=64, L=64.0, ppc=(500, 500))
    s = _sim(p)
    for sp in range(2):
        x, v, ids = s.particles(sp)
        assert len(x) == 64 * 500
        counts = np.bincount(np.floor(x).astype(int), minlength=64)
        assert (counts == 500).all()
        assert stats.kstest(x - np.floor(x), "uniform").pvalue > 1e-4
        vt = math.sqrt(p["T"][sp] / p["mass"][sp])
        for k in range(3):
            assert stats.kstest(v[:, k] / vt, "norm").pvalue > 1e-4
        assert len(np.unique(ids)) == len(ids)


@pytest.mark.parametrize("scale", [None, 256.0])
def test_loader_exponential_profile(scale):
    # the density is exp(-x / lambda) truncated to [0, L): with lambda = L/2 the truncation holds
    # back 13.5 % of an untruncated exponential's mass
    p = W.variant(W.SMALL_C3) if scale is None else W.variant(W.SMALL_C3, profile_scale=scale)
    s = _sim(p)
    x, v, ids = s.particles(0)
    lam, L = p["profile_scale"], p["ncells"]
    cdf = lambda t: (1 - np.exp(-t / lam)) / (1 - np.exp(-L / lam))
    assert stats.kstest(x, cdf).pvalue > 1e-4


def test_quiet_load_density_is_uniform_at_every_node():
    # evenly spaced particles (quiet load, no displacement) fill every cell symmetrically: each
    # interior node collects one cell's worth of charge over dx, each wall node half of it over the
    # half cell dx/2, so the node density is the same everywhere.  Ions of charge 2 against
    # electrons of charge -1 leave a net density of +1.
    p = W.variant(W.BASE, ncells=24, L=24.0, ppc=(40, 40), charge=(-1.0, 2.0),
                  load_profile=W.LOAD_QUIET_SINE, profile_scale=0.0, profile_mode=1)
    rho = _sim(p).fields()["rho"]
    assert np.abs(rho - 1.0).max() < 1e-9, rho


def test_sort_orders_cells_and_keeps_the_set():
    p = W.variant(W.SMALL_COLL, sort_interval=3)
    s = _sim(p)
    for k in range(7):
        s.step(1)
        for sp in range(2):
            x, v, ids = s.particles(sp)
            assert len(np.unique(ids)) == len(ids)
            if (k % 3) == 0:
                c = np.floor(x)
                assert (np.diff(c) >= 0).all()


def test_thread_count_does_not_change_the_state():
    p = W.variant(W.SMALL_COLL)
    a, b = _sim(p, threads=1), _sim(p, threads=4)
    O.set_threads(1)
    a.step(12)
    O.set_threads(4)
    b.step(12)
    O.set_threads(1)
    assert a.snapshot() == b.snapshot()


def test_snapshot_roundtrip_and_continuation():
    p = W.variant(W.SMALL_COLL)
    a = _sim(p)
    a.step(7)
    blob7 = a.snapshot()
    a.step(5)
    b = _sim(p)
    assert b.restore(blob7) == 0
    assert b.snapshot() == blob7
    b.step(5)
    assert a.snapshot() == b.snapshot()
    da, db = a.diag(), b.diag()
    # particle_steps counts since creation / restore; everything else must agree
    assert da.pop("particle_steps") > db.pop("particle_steps") > 0
    assert da == db


def test_restore_rejects_corrupt_or_foreign_blobs():
    p = W.variant(W.SMALL_C1)
    a = _sim(p)
    blob = bytearray(a.snapshot())
    blob[300] ^= 1
    assert a.restore(bytes(blob)) == 5
    b = _sim(W.variant(p, seed=p["seed"] + 1))
    assert b.restore(a.snapshot()) == 5
    assert a.restore(a.snapshot()[:-9]) == 5


def test_step_sample_is_the_step_one_particle_at_a_time():
    # orc_step_sample (the oracle step of given particles under a given field, for checks that
    # sample a large state) against the whole oracle step from the same state: survivors bit for
    # bit, the absorbed set, and the candidate, near-threshold and ionization counts
    p = W.variant(W.SMALL_COLL, B=0.5, B_angle_deg=30.0, V_left=-2.0)
    o = O.OracleSim(p)
    o.step(3)
    d0, E = o.diag(), o.fields()["E"]
    before = [o.particles(s) for s in range(2)]
    nk0 = [o.countdown(s) for s in range(2)]
    out = [O.step_sample(p, s, d0["step"], E, *before[s], nk0[s]) for s in range(2)]
    o.step(1)
    d1 = o.diag()
    for s in range(2):
        x0, v0, id0 = before[s]
        xs, vs, nks, fl = out[s]
        x1, v1, id1 = o.particles(s)
        nk1 = o.countdown(s)
        absorbed = (fl & 1) != 0
        assert int(absorbed.sum()) == sum(d1["wall_hits"][s]) - sum(d0["wall_hits"][s])
        # every survivor, matched by id (births carry new ids; a sort may reorder)
        keep = ~absorbed
        o1 = np.argsort(id1)
        pos = np.searchsorted(id1, id0[keep], sorter=o1)
        j = o1[np.minimum(pos, len(id1) - 1)]
        assert np.array_equal(id1[j], id0[keep])
        assert np.array_equal(x1[j], xs[keep])
        assert np.array_equal(v1[j], vs[keep])
        assert np.array_equal(nk1[j], nks[keep])
        assert not np.isin(id0[absorbed], id1).any()
    assert sum(int(((f & 2) != 0).sum()) for *_, f in out) == d1["coll"][4] - d0["coll"][4]
    assert sum(int(((f & 4) != 0).sum()) for *_, f in out) == sum(d1["near_threshold"]) - sum(d0["near_threshold"])
    assert int(((out[0][3] & 8) != 0).sum()) == d1["births"][0] - d0["births"][0] > 0


def test_step_sample_uniform_field_is_uniform_acceleration():
    # B = 0, external uniform E, no collisions: v' = v + (q/m) E dt and x' = x + v' dt / dx
    p = W.variant(W.SMALL_C1, field_mode=W.FIELD_EXTERNAL, E_ext=0.3, B=0.0, coll_mask=0)
    rng = np.random.default_rng(5)
    n = 200
    x = rng.uniform(5.0, p["ncells"] - 5.0, n)
    v = rng.normal(size=(n, 3)) * 0.1
    for s in range(2):
        xo, vo, nko, fl = O.step_sample(p, s, 0, np.zeros(p["ncells"] + 1), x, v, np.arange(n, dtype=np.uint64),
                                        np.zeros(n, np.uint32))
        assert np.all(nko == 0)  # no null-collision test: no countdown
        a = p["charge"][s] / p["mass"][s] * p["E_ext"] * p["dt"]
        dx = p["L"] / p["ncells"]
        assert np.all(fl == 0)
        assert np.allclose(vo[:, 0], v[:, 0] + a, rtol=0, atol=1e-14)
        assert np.array_equal(vo[:, 1:], v[:, 1:])
        assert np.allclose(xo, x + vo[:, 0] * p["dt"] / dx, rtol=0, atol=1e-12)


def _candidate_flags(p, s, n, steps):
    """Candidate flags (steps x n) of n nearly cold particles of species s under no field: their
    process frequencies vanish, so every candidate is a null collision and nothing else changes."""
    o = O.OracleSim(W.variant(p, ncells=64, L=64.0, ppc=(max(1, n // 64), max(1, n // 64))))
    x, _v, ids = o.particles(s)
    nk = o.countdown(s)
    x, ids, nk = x[:n], ids[:n], nk[:n]
    v = np.full((len(x), 3), 1e-9)
    E = np.zeros(p["ncells"] + 1)
    flags = np.empty((steps, len(x)), bool)
    for t in range(steps):
        x, v, nk, fl = O.step_sample(p, s, t, E, x, v, ids, nk)
        assert not (fl & 1).any()
        flags[t] = (fl & 2) != 0
    return flags


@pytest.mark.parametrize("p_target", [0.04, 6e-4])
def test_countdown_candidates_are_bernoulli_per_step(p_target):
    # R17 replaces the per-step Bernoulli(P_null) test by a geometric countdown; in law the candidate
    # process must be the same: i.i.d. Bernoulli(P_null) per particle and step.  Checked: the rate
    # (binomial, 5 sigma), the spread of the per-step counts (binomial dispersion), and the waiting
    # times to a particle's next candidate (geometric, chi-square over a fixed window; a wait longer
    # than the window counts in the last bin).  The small P_null also exercises the countdown cap
    # (K > 4095 waits 4095 steps and draws again): a bin isolates waits of exactly 4095 steps.
    base = W.variant(W.SMALL_C1, field_mode=W.FIELD_ZERO, coll_mask=W.COLL_EL, E_cap=0.5, n_gas=1.0)
    # nu_max dt = n_gas sigma_el v_cap dt with v_cap = 1 (E_cap = 0.5, m = 1): pick sigma_el
    p = W.variant(base, sigma_el=-np.log1p(-p_target) / base["dt"])
    pn = float(O.nu_max(p)[1][0])
    q = 1.0 - pn
    n, steps = (3000, 600) if p_target > 0.01 else (1500, 9000)
    f = _candidate_flags(p, 0, n, steps)
    tot, trials = int(f.sum()), f.size
    assert abs(tot - trials * pn) <= 5 * np.sqrt(trials * pn * (1 - pn)), (tot, trials * pn)
    per_step = f.sum(axis=1)
    disp = per_step.var(ddof=1) / (f.shape[1] * pn * (1 - pn))
    assert abs(disp - 1.0) <= 6 * np.sqrt(1.0 / (f.shape[1] * pn * steps) + 2.0 / (steps - 1)), disp
    # waits from each start (the beginning, or a candidate) early enough to see a full window
    L = steps // 2
    waits = []
    for j in range(f.shape[1]):
        t = np.flatnonzero(f[:, j])
        for t0 in np.concatenate([[-1], t]):
            if t0 + L >= steps:
                break
            nxt = t[t > t0]
            waits.append(nxt[0] - t0 if len(nxt) and nxt[0] - t0 <= L else L + 1)  # L + 1: longer than L
    waits = np.array(waits)
    sf = lambda k: q ** (k - 1)  # P(wait >= k)
    edges = np.unique(np.concatenate([[1], 1 + np.ceil(np.log(np.linspace(1, 0.03, 12)[1:]) / np.log(q)),
                                      [4095, 4096, 4097] if L > 4097 else [], [L + 1]]).astype(int))
    edges = edges[edges <= L + 1]
    obs = [((waits >= a) & (waits < b)).sum() for a, b in zip(edges[:-1], edges[1:])] + [(waits >= edges[-1]).sum()]
    exp = [len(waits) * (sf(a) - sf(b)) for a, b in zip(edges[:-1], edges[1:])] + [len(waits) * sf(edges[-1])]
    chi2 = sum((o_ - e_) ** 2 / max(e_, 1.0) for o_, e_ in zip(obs, exp))
    assert chi2 < 45, (chi2, list(zip(edges.tolist(), obs, np.round(exp, 1))))
