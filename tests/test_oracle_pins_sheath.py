"""Pins of the oracle's D+/e/D sheath physics: density smoothing, recycling of ions into tracked
neutrals at the walls, the neutrals' ballistic motion and their electron-impact ionization.

Each expectation comes from outside the oracle: eigenvectors of the smoothing stencil with their
closed-form eigenvalues, conservation of the total charge, the moments of the flux-weighted
half-Maxwellian and of a Maxwellian, binomial counts of a known probability, straight-line motion,
exact particle accounting, and snapshot and thread-count invariance.  States are built with the
snapshot format (input plumbing only) from positions and velocities chosen here.
"""
import math

import numpy as np
import pytest

import snapfmt
from oracle import oracle as O
from paper_2606_28534_gb300 import workloads as W

# charged species frozen or absent, no field, no background collisions: only the piece under test acts
QUIET = dict(field_mode=W.FIELD_ZERO, coll_mask=0, source_mode=W.SOURCE_NONE, smooth_passes=0, K_iz=0.0,
             neutral_ppc=0)


def _quiet(**kw):
    return W.variant(W.variant(W.SMALL_C6, **QUIET), **kw)


def _state(p, electrons, ions, neutrals, step=0):
    """A blob of configuration p holding the given particles ({"x", "v", "id"} each)."""
    base = O.OracleSim(p).snapshot()
    return snapfmt.with_particles(base, [electrons, ions], step=step, neutrals=neutrals)


def _sim_from(p, blob, threads=1):
    s = O.OracleSim(p, threads=threads)
    assert s.restore(blob) == 0
    return s


def _empty():
    return {"x": np.zeros(0), "v": np.zeros((0, 3)), "id": np.zeros(0, np.uint64)}


def _binomial_ok(k, n, p, sigmas=4.0):
    return abs(k - n * p) <= sigmas * math.sqrt(n * p * (1 - p)) + 1


# ------------------------------------------------------------------------------------------------
# density smoothing
@pytest.mark.parametrize("N", [2, 3, 8, 37, 256])
def test_cosine_modes_are_eigenvectors_of_the_smoothing(N):
    # cos(pi m j / N) is mapped to cos^2(pi m / 2N) times itself by the (1,2,1)/4 stencil inside and
    # by the (1,1)/2 average at either wall node, for every m
    j = np.arange(N + 1)
    for m in sorted({0, 1, 2, N // 2, N - 1, N}):
        rho = np.cos(np.pi * m * j / N)
        for k in (1, 2, 4):
            lam = np.cos(np.pi * m / (2 * N)) ** (2 * k)
            assert np.abs(O.smooth(rho, k) - lam * rho).max() <= 1e-13, (N, m, k)


def test_smoothing_keeps_the_total_charge_and_a_uniform_density():
    rng = np.random.default_rng(5)
    for N in (2, 3, 50):
        vol = np.ones(N + 1)
        vol[0] = vol[-1] = 0.5  # half-cell volume of the wall nodes
        rho = rng.normal(size=N + 1)
        for k in range(5):
            out = O.smooth(rho, k)
            assert abs((out * vol).sum() - (rho * vol).sum()) <= 1e-13 * np.abs(rho).sum()
        assert np.array_equal(O.smooth(np.full(N + 1, 0.625), 3), np.full(N + 1, 0.625))
    assert np.array_equal(O.smooth(rho, 0), rho)


def test_the_field_solve_uses_the_smoothed_density():
    # the particles at t = 0 do not depend on the smoothing: the same deposit, the density smoothed
    # twice, and the potential of the smoothed density (Thomas, pinned elsewhere)
    p2 = W.SMALL_C6
    p0 = W.variant(p2, smooth_passes=0)
    fa, fb = O.OracleSim(p0).fields(), O.OracleSim(p2).fields()
    assert np.array_equal(fa["R"], fb["R"])
    assert np.abs(fb["rho"] - O.smooth(fa["rho"], 2)).max() <= 1e-14 * np.abs(fa["rho"]).max()
    assert np.abs(fb["rho"] - fa["rho"]).max() > 1e-3 * np.abs(fa["rho"]).max()
    dx = p2["L"] / p2["ncells"]
    phi = O.poisson_thomas(fb["rho"], dx, p2["V_left"], p2["V_right"])
    assert np.abs(fb["phi"] - phi).max() <= 1e-12 * np.abs(phi).max()


# ------------------------------------------------------------------------------------------------
# recycling at the walls
def _wall_ions(N, n, rng):
    """n ions that leave through the walls in the next step: half just inside the left wall moving
    left, half just inside the right wall moving right (|v_x| dt / dx = 0.05 > their distance)."""
    h = n // 2
    x = np.concatenate([rng.uniform(0.0, 0.01, h), N - rng.uniform(1e-3, 0.01, n - h)])
    v = np.zeros((n, 3))
    v[:h, 0] = -0.5
    v[h:, 0] = 0.5
    v[:, 1:] = rng.normal(size=(n, 2))
    return {"x": x, "v": v, "id": (np.uint64(1) << np.uint64(62)) + np.arange(n, dtype=np.uint64)}, h


def _one_electron(N):
    return {"x": np.array([N / 2]), "v": np.zeros((1, 3)), "id": np.array([7], np.uint64)}


def test_every_absorbed_ion_returns_as_one_neutral_at_its_wall():
    p = _quiet(frozen_mask=1, recycle=1.0)
    N = p["ncells"]
    ions, h = _wall_ions(N, 40000, np.random.default_rng(1))
    s = _sim_from(p, _state(p, _one_electron(N), ions, _empty()))
    s.step(1)
    d, nd = s.diag(), s.neutral_diag()
    assert d["wall_hits"][1] == [h, 40000 - h]
    assert nd["recycled"] == [h, 40000 - h] and nd["n"] == 40000
    x, v, ids = s.particles(2)
    assert len(np.unique(ids)) == 40000 and not np.isin(ids, ions["id"]).any()
    left = v[:, 0] > 0
    assert left.sum() == h and (v[~left, 0] < 0).all()
    # born on the wall: x = 0, or the last representable FP32 fraction of the last cell
    assert (x[left] == 0.0).all() and (x[~left] == N - 2.0**-24).all()
    # flux-weighted half-Maxwellian at T_rec: E|v_x| = v_t sqrt(pi/2), E v_x^2 = 2 v_t^2;
    # v_y, v_z Maxwellian
    vt = math.sqrt(p["T_rec"] / p["mass"][1])
    a = np.abs(v[:, 0]) / vt
    n = len(a)
    assert abs(a.mean() - math.sqrt(math.pi / 2)) <= 4 * math.sqrt((4 - math.pi) / 2 / n)
    assert abs((a**2).mean() - 2.0) <= 4 * 2.0 / math.sqrt(n)
    for k in (1, 2):
        b = v[:, k] / vt
        assert abs(b.mean()) <= 4 / math.sqrt(n)
        assert abs((b**2).mean() - 1.0) <= 4 * math.sqrt(2.0 / n)


def test_a_fraction_of_the_ions_return_when_recycling_is_partial():
    p = _quiet(frozen_mask=1, recycle=0.3)
    N = p["ncells"]
    ions, h = _wall_ions(N, 20000, np.random.default_rng(2))
    s = _sim_from(p, _state(p, _one_electron(N), ions, _empty()))
    s.step(1)
    nd = s.neutral_diag()
    assert _binomial_ok(nd["recycled"][0], h, 0.3) and _binomial_ok(nd["recycled"][1], 20000 - h, 0.3)
    assert nd["n"] == sum(nd["recycled"])
    # no recycling at all without it
    q = W.variant(p, recycle=0.0)
    s = _sim_from(q, _state(q, _one_electron(N), ions, _empty()))
    s.step(1)
    assert s.neutral_diag()["n"] == 0 and s.diag()["wall_hits"][1] == [h, 20000 - h]


# ------------------------------------------------------------------------------------------------
# neutral motion
def test_neutrals_move_in_straight_lines_and_leave_at_the_walls():
    # dx = 2 (L = 2N): the move is v dt / dx cells per step; no field, B or collision acts on them
    p = _quiet(frozen_mask=3, L=2.0 * W.SMALL_C6["ncells"], B=3.0,
                  field_mode=W.FIELD_EXTERNAL, E_ext=5.0)
    N = p["ncells"]
    rng = np.random.default_rng(3)
    n = 5000
    x0 = rng.uniform(0.0, N, n)
    v = rng.normal(size=(n, 3)) * 4.0
    ids = (np.uint64(3) << np.uint64(61)) + np.arange(n, dtype=np.uint64)
    s = _sim_from(p, _state(p, _one_electron(N), _empty(), {"x": x0, "v": v, "id": ids}))
    k = 7
    s.step(k)
    xk = x0 + k * (v[:, 0] * p["dt"] / (p["L"] / N))
    clear = (np.abs(xk) > 1e-9) & (np.abs(xk - N) > 1e-9)
    inside = (xk >= 0) & (xk < N)
    x, vv, ii = s.particles(2)
    o = np.argsort(ii)
    x, vv, ii = x[o], vv[o], ii[o]
    assert np.array_equal(ii, ids[inside])
    assert np.abs(x - xk[inside]).max() <= 1e-10
    assert np.array_equal(vv, v[inside])
    nd = s.neutral_diag()
    assert nd["lost"][0] == ((xk < 0) & clear).sum() and nd["lost"][1] == ((xk >= N) & clear).sum()
    assert nd["particle_steps"] >= n


# ------------------------------------------------------------------------------------------------
# electron-impact ionization of the neutrals
def _quiet_plasma(p):
    """Electrons and ions of a quiet load: node electron density exactly 1 everywhere."""
    q = W.variant(p, load_profile=W.LOAD_QUIET_SINE, profile_scale=0.0, profile_mode=1)
    d = snapfmt.parse(O.OracleSim(q).snapshot())
    return q, [{"x": sp["cell"] + sp["frac"], "v": sp["v"], "id": sp["id"]} for sp in d["species"]]


def test_neutrals_ionize_at_the_rate_of_a_uniform_plasma_up_to_the_walls():
    p, (el, io) = _quiet_plasma(_quiet(frozen_mask=3, K_iz=0.5, T_sec=2.0))
    N = p["ncells"]
    rng = np.random.default_rng(4)
    # at rest: 60000 spread over the domain and 20000 within 0.05 cells of either wall node, where
    # the electron density is that of a half-volume wall node
    xs = np.concatenate([rng.uniform(0.0, N, 60000), rng.uniform(0.0, 0.05, 10000),
                         N - rng.uniform(1e-4, 0.05, 10000)])
    n = len(xs)
    ids = (np.uint64(3) << np.uint64(61)) + np.arange(n, dtype=np.uint64)
    v = np.zeros((n, 3))
    s = _sim_from(p, _state(p, el, io, {"x": xs, "v": v, "id": ids}))
    f = s.fields()
    ne = f["R"][0] / 2.0**32 * (p["L"] / N / p["ppc"][0]) / np.r_[0.5, np.ones(N - 1), 0.5] / (p["L"] / N)
    assert np.abs(ne - 1.0).max() < 1e-9
    n0 = s.diag()["n"]
    s.step(1)
    P = 1.0 - math.exp(-p["K_iz"] * 1.0 * p["dt"])
    x, vv, ii = s.particles(2)
    gone = ~np.isin(ids, ii)
    k = int(gone.sum())
    assert s.neutral_diag()["ionized"] == k and s.neutral_diag()["n"] == n - k
    assert _binomial_ok(k, n, P)
    assert _binomial_ok(int(gone[60000:].sum()), 20000, P)  # the wall regions ionize at the same rate
    # each ionized neutral is now an ion with its id, position and velocity; an electron was born
    # beside it, Maxwellian at T_sec
    d = s.diag()
    assert d["n"][0] == n0[0] + k and d["n"][1] == n0[1] + k
    assert d["net_charge_units"] == 2**32 * (d["n"][1] - d["n"][0])
    xi, vi, iid = s.particles(1)
    new_ions = np.isin(iid, ids[gone])
    assert new_ions.sum() == k
    o = np.argsort(iid[new_ions])
    assert np.array_equal(xi[new_ions][o], xs[gone]) and not vi[new_ions].any()
    xe, ve, ide = s.particles(0)
    born = ~np.isin(ide, el["id"])
    assert born.sum() == k and np.array_equal(np.sort(xe[born]), np.sort(xs[gone]))
    b = ve[born] / math.sqrt(p["T_sec"] / p["mass"][0])
    assert np.abs(b.mean(axis=0)).max() <= 4 / math.sqrt(k)
    assert np.abs((b**2).mean(axis=0) - 1.0).max() <= 4 * math.sqrt(2.0 / k)


def test_no_ionization_without_a_rate_coefficient():
    p, (el, io) = _quiet_plasma(_quiet(frozen_mask=3))
    N = p["ncells"]
    xs = np.linspace(0.0, N - 0.5, 3000)
    s = _sim_from(p, _state(p, el, io, {"x": xs, "v": np.zeros((3000, 3)),
                                          "id": np.arange(3000, dtype=np.uint64) + (np.uint64(3) << np.uint64(61))}))
    s.step(3)
    assert s.neutral_diag()["ionized"] == 0 and s.neutral_diag()["n"] == 3000


# ------------------------------------------------------------------------------------------------
# loads, accounting, snapshots
def test_initial_neutrals_fill_every_cell_evenly_at_the_recycling_temperature():
    p = W.variant(W.SMALL_C6, neutral_ppc=400, T_rec=0.4)
    s = O.OracleSim(p)
    x, v, ids = s.particles(2)
    N = p["ncells"]
    assert np.array_equal(np.bincount(np.floor(x).astype(int), minlength=N), np.full(N, 400))
    assert np.array_equal(np.sort(ids), (np.uint64(3) << np.uint64(61)) + np.arange(400 * N, dtype=np.uint64))
    b = v / math.sqrt(p["T_rec"] / p["mass"][1])
    n = len(b)
    assert np.abs(b.mean(axis=0)).max() <= 4 / math.sqrt(n)
    assert np.abs((b**2).mean(axis=0) - 1.0).max() <= 4 * math.sqrt(2.0 / n)
    assert O.OracleSim(W.variant(p, neutral_ppc=0)).count(2) == 0


def _busy_state(p, seed):
    """A state in which every process of the sheath model acts within a few steps: ions leaving
    through both walls, neutrals near and inside the walls, a plasma that ionizes them."""
    rng = np.random.default_rng(seed)
    N = p["ncells"]
    d = snapfmt.parse(O.OracleSim(p).snapshot())
    el = {"x": d["species"][0]["cell"] + d["species"][0]["frac"], "v": d["species"][0]["v"], "id": d["species"][0]["id"]}
    io = {"x": d["species"][1]["cell"] + d["species"][1]["frac"], "v": d["species"][1]["v"], "id": d["species"][1]["id"]}
    w, _ = _wall_ions(N, 600, rng)
    io = {k: np.concatenate([io[k], w[k]]) for k in io}
    nt = snapfmt.parse(O.OracleSim(p).snapshot())["neutrals"]
    xn = np.concatenate([nt["cell"] + nt["frac"], rng.uniform(0, 0.02, 200), N - rng.uniform(1e-3, 0.02, 200)])
    vn = np.concatenate([nt["v"], rng.normal(size=(400, 3)) * 0.2])
    vn[-400:-200, 0] = -np.abs(vn[-400:-200, 0])
    vn[-200:, 0] = np.abs(vn[-200:, 0])
    idn = np.concatenate([nt["id"], (np.uint64(5) << np.uint64(60)) + np.arange(400, dtype=np.uint64)])
    return _state(p, el, io, {"x": xn, "v": vn, "id": idn})


def test_particle_accounting_is_exact_every_step():
    p = W.variant(W.SMALL_C6, V_left=-2.0)
    s = _sim_from(p, _busy_state(p, 6))
    d0, n0 = s.diag(), s.neutral_diag()
    for _ in range(6):
        s.step(1)
        d, nd = s.diag(), s.neutral_diag()
        assert d["net_charge_units"] == 2**32 * (d["n"][1] - d["n"][0])
        assert nd["n"] == n0["n"] + sum(nd["recycled"]) - sum(nd["lost"]) - nd["ionized"]
        for sp in range(2):
            lost = sum(d["wall_hits"][sp]) - sum(d0["wall_hits"][sp])
            assert d["n"][sp] == d0["n"][sp] + d["births"][sp] - d0["births"][sp] + nd["ionized"] - lost
        assert nd["recycled"] == d["wall_hits"][1]  # recycle = 1: every absorbed ion returns
    assert nd["ionized"] > 0 and sum(nd["lost"]) > 0 and sum(nd["recycled"]) > 0


def test_snapshot_continuation_and_thread_count_give_the_same_bytes():
    p = W.variant(W.SMALL_C6, V_left=-2.0, sort_interval=3)
    blob = _busy_state(p, 7)
    a = _sim_from(p, blob, threads=1)
    O.set_threads(1)
    a.step(2)
    mid = a.snapshot()
    assert snapfmt.parse(mid)["version"] == 4
    b = _sim_from(p, mid)
    c = _sim_from(p, blob, threads=4)
    O.set_threads(1)
    a.step(4)
    b.step(4)
    O.set_threads(4)
    c.step(6)
    O.set_threads(1)
    assert a.snapshot() == b.snapshot() == c.snapshot()
    # the sheath fields are part of the configuration hash; a version-3 reader refuses the blob
    assert O.config_hash(p) != O.config_hash(W.variant(p, K_iz=0.25))
    assert O.config_hash(W.C3) == O.config_hash(W.variant(W.C3, recycle=0.5, T_rec=2.0))
    assert O.OracleSim(W.variant(p, neutrals=0, neutral_ppc=0)).restore(mid) != 0
