"""The GPU path against physics the method must reproduce, beside the oracle's own pins: the cold
plasma frequency under leapfrog, the Boris gyration, and the energy balance of a collisionless
plasma between grounded walls compared with the oracle's seed-to-seed spread."""
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


def test_cold_plasma_oscillation_frequency():
    # cold electrons displaced by A sin(2 pi x/L) over frozen ions oscillate at the leapfrog plasma
    # frequency w = (2/dt) asin(w_p dt/2) = 1.000417 (finite-grid corrections ~ (k dx)^2 ~ 1e-4)
    p = W.variant(W.BASE, ncells=256, L=256.0, ppc=(64, 64), coll_mask=0, frozen_mask=2,
                  load_profile=W.LOAD_QUIET_SINE, profile_mode=1, profile_scale=0.02, T=(0.0, 0.0),
                  precision=W.PRECISION_FP32)
    g = pic.Simulation(p)
    j = 64
    series = [g.fields()["E"][j]]
    for _ in range(700):
        g.step(1)
        series.append(g.fields()["E"][j])
    e = np.array(series, np.float64)
    z = np.where(np.sign(e[:-1]) != np.sign(e[1:]))[0]
    t = z + e[z] / (e[z] - e[z + 1])
    w = np.pi / (np.diff(t).mean() * p["dt"])
    expect = (2 / p["dt"]) * math.asin(p["dt"] / 2)
    assert abs(w - expect) / expect < 1e-3, (w, expect)


def test_boris_gyration_keeps_the_speed_and_turns_at_the_boris_phase():
    # no electric field, B = 0.5 at 30 degrees: each step rotates v about B by 2 atan(w_c dt / 2);
    # |v| and the component along B stay fixed (FP32 rounding over 1000 steps)
    p = W.variant(W.BASE, ncells=64, L=64.0, ppc=(4, 4), coll_mask=0, field_mode=W.FIELD_ZERO, frozen_mask=2,
                  B=0.5, B_angle_deg=30.0, precision=W.PRECISION_FP32, dt=0.1)
    g = pic.Simulation(p)
    d = snapfmt.parse(g.snapshot())
    rng = np.random.default_rng(3)
    n = 64
    v0 = rng.normal(size=(n, 3)) * 1e-3  # slow: they stay far from the walls for 1000 steps
    x0 = rng.uniform(24.0, 40.0, n)
    ions = d["species"][1]
    blob = snapfmt.round_to_fp32(snapfmt.with_particles(
        g.snapshot(), [{"x": x0, "v": v0, "id": np.arange(n, dtype=np.uint64)},
                       {"x": ions["cell"] + ions["frac"], "v": ions["v"], "id": ions["id"]}]))
    assert g.restore(blob) == 0
    v0 = snapfmt.parse(blob)["species"][0]["v"]
    steps = 1000
    g.step(steps)
    sp = snapfmt.parse(g.snapshot())["species"][0]
    v = sp["v"][np.argsort(sp["id"])]
    bh = np.array([math.cos(math.pi / 6), math.sin(math.pi / 6), 0.0])
    # the Boris phase per step; an electron (q < 0) turns its perpendicular velocity towards b x v
    theta = steps * 2 * math.atan(p["B"] * p["dt"] / 2)
    par = v0 @ bh
    perp0 = v0 - np.outer(par, bh)
    rot = perp0 * math.cos(theta) + np.cross(bh, perp0) * math.sin(theta)
    expect = rot + np.outer(par, bh)
    speed0 = np.linalg.norm(v0, axis=1)
    assert np.abs(np.linalg.norm(v, axis=1) - speed0).max() <= 1e-5 * speed0.max()
    assert np.abs(v @ bh - par).max() <= 1e-5 * speed0.max()
    assert np.abs(v - expect).max() <= 2e-4 * speed0.max(), np.abs(v - expect).max() / speed0.max()


def test_energy_balance_of_a_collisionless_plasma_matches_the_oracle_spread():
    # grounded walls, no collisions: kinetic + field + wall-absorbed energy drifts only by grid
    # heating; the GPU run's relative drift after 200 steps must sit within 4 sigma of 8 oracle seeds
    base = W.variant(W.BASE, ncells=128, L=128.0, ppc=(100, 100), coll_mask=0, precision=W.PRECISION_FP32)

    def total(d):
        return sum(d["ke"]) + d["field_energy"] + sum(d["wall_energy"])

    drifts = []
    for k in range(8):
        o = O.OracleSim(W.variant(base, seed=700 + k))
        e0 = total(o.diag())
        o.step(200)
        drifts.append((total(o.diag()) - e0) / e0)
    drifts = np.array(drifts)
    g = pic.Simulation(W.variant(base, seed=799))
    e0 = total(g.diag())
    g.step(200)
    d = g.diag()
    drift = (total(d) - e0) / e0
    assert sum(d["wall_energy"]) > 0
    assert abs(drift) < 0.02
    assert abs(drift - drifts.mean()) <= 4 * drifts.std(ddof=1) + 1e-4, (drift, drifts.mean(), drifts.std(ddof=1))


def test_exb_drift():
    # uniform E along x, B along y: electrons starting at rest drift at E x B / B^2 (Boris keeps the
    # drift exactly); the time average of v over 40 gyro-periods
    E, B, dt = 0.05, 0.8, 0.1
    p = W.variant(W.BASE, ncells=64, L=64.0, ppc=(4, 4), coll_mask=0, field_mode=W.FIELD_EXTERNAL, E_ext=E,
                  frozen_mask=2, B=B, B_angle_deg=90.0, dt=dt, precision=W.PRECISION_FP32)
    g = pic.Simulation(p)
    d = snapfmt.parse(g.snapshot())
    n = 16
    ions = d["species"][1]
    blob = snapfmt.round_to_fp32(snapfmt.with_particles(
        g.snapshot(), [{"x": np.linspace(28.0, 36.0, n), "v": np.zeros((n, 3)), "id": np.arange(n, dtype=np.uint64)},
                       {"x": ions["cell"] + ions["frac"], "v": ions["v"], "id": ions["id"]}]))
    assert g.restore(blob) == 0
    steps = int(round(40 * 2 * math.pi / (2 * math.atan(B * dt / 2))))
    acc = np.zeros(3)
    for _ in range(steps):
        g.step(1)
        acc += snapfmt.parse(g.snapshot())["species"][0]["v"].mean(axis=0)
    mean = acc / steps
    drift = np.cross([E, 0.0, 0.0], [0.0, B, 0.0]) / (B * B)
    assert abs(mean[2] - drift[2]) / abs(drift[2]) < 2e-2, (mean, drift)
    assert np.abs(mean - drift).max() < 2e-3 * np.linalg.norm(drift) + 1e-4 + 2e-2 * abs(drift[2])
