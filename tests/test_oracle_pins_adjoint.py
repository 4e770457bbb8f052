"""Pins of the oracle's adjoint (oracle/pic_adjoint.c) against what the mathematics fixes.

* The field transpose: <mu, G rho> = <G^T mu, rho> for random vectors, and G^T equals the matrix
  transpose of G built column by column.
* The gradient equals central finite differences of the same frozen-schedule forward (FP64, small h)
  for self-consistent fields with and without B, an external field, frozen ions and a biased right
  wall, for both observables and both parameters.
* Ballistic electrons (no field): J_flux and dJ_flux/dT_e from the closed form of straight-line
  motion, written here from the initial load alone; dJ_flux/dV_L = 0.
* A frozen plasma: J_fe and dJ_fe/dV_L from the static field (E = E_rho + V_L / (N dx)).
* The recording forward is the main oracle's collisionless step (same absorbed particles, same final
  field up to the fixed-point deposit rounding).
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2606_28534_gb300 import workloads as W

BASE = W.variant(W.C5, ncells=48, L=48.0, ppc=(30, 30), V_left=-1.5, seed=77)


def _fd(params, steps, absorb, h):
    def f(dV, dT):
        q = dict(params, V_left=params["V_left"] + dV, T=(params["T"][0] + dT, params["T"][1]))
        return O.adj_forward(q, steps, absorb)[0]
    return np.array([(f(h, 0) - f(-h, 0)) / (2 * h), (f(0, h) - f(0, -h)) / (2 * h)])  # [param, observable]


@pytest.mark.parametrize("N", [2, 3, 17, 256])
def test_field_transpose_dot_product_and_matrix(N):
    rng = np.random.default_rng(N)
    dx = 0.5 + rng.random()
    rho, mu = rng.standard_normal(N + 1), rng.standard_normal(N + 1)
    lhs = mu @ O.field_apply(rho, dx)
    rhs = O.field_adjoint(mu, dx) @ rho
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + np.abs(mu).sum() * np.abs(rho).sum() * 1e-3)
    if N <= 17:
        G = np.stack([O.field_apply(np.eye(N + 1)[k], dx) for k in range(N + 1)], axis=1)
        GT = np.stack([O.field_adjoint(np.eye(N + 1)[k], dx) for k in range(N + 1)], axis=1)
        assert np.abs(GT - G.T).max() <= 1e-12 * np.abs(G).max()


@pytest.mark.parametrize("case", ["self", "magnetised", "external", "frozen_ions", "biased_right", "half_cells"])
def test_gradient_equals_central_differences(case):
    p = {
        "self": BASE,
        "half_cells": W.variant(BASE, L=24.0),  # dx = 1/2: positions advance by v dt / dx
        "magnetised": W.variant(BASE, B=0.5, B_angle_deg=30.0),
        "external": W.variant(BASE, field_mode=W.FIELD_EXTERNAL, E_ext=0.02),
        "frozen_ions": W.variant(BASE, frozen_mask=2),
        "biased_right": W.variant(BASE, V_right=0.7, T=(1.3, 0.1)),
    }[case]
    steps = 50
    g_flux, J, absorb = O.adj_gradient(p, steps, (1.0, 0.0))
    g_fe, J2, absorb2 = O.adj_gradient(p, steps, (0.0, 1.0))
    assert np.array_equal(J, J2) and np.array_equal(absorb, absorb2)
    assert (absorb < O.ADJ_NEVER).sum() > 0  # the walls absorbed particles: the schedule matters
    # The forward is piecewise smooth: CIC weights have kinks at cell boundaries, so an interval
    # [theta - h, theta + h] that holds a particle's crossing of a cell boundary biases the central
    # difference by O(1) of that particle's share.  Such intervals shrink with h; the pin asks that
    # one of three step sizes gives an interval without a kink (then the difference is O(h^2)).
    fds = [_fd(p, steps, absorb, h) for h in (1e-6, 3e-7, 1e-7)]
    for k in range(2):
        for g, obs in ((g_flux, 0), (g_fe, 1)):
            err = min(abs(g[k] - fd[k, obs]) for fd in fds)
            scale = max(abs(fds[-1][k, obs]), 1e-3 * abs(J[obs]))
            assert err <= 2e-6 * scale, (case, k, obs, g[k], [fd[k, obs] for fd in fds])
    # a weighted observable is the weighted sum (one reverse sweep per vector-Jacobian product)
    g_mix, _, _ = O.adj_gradient(p, steps, (0.3, -2.0))
    assert np.allclose(g_mix, 0.3 * g_flux - 2.0 * g_fe, rtol=1e-12, atol=1e-15)
    if case == "external":
        assert abs(g_flux[0]) == 0.0  # the particles do not see the bias


def test_ballistic_flux_closed_form():
    p = W.variant(BASE, field_mode=W.FIELD_ZERO, ncells=40, L=40.0, ppc=(25, 25))
    steps = 70
    g, J, absorb = O.adj_gradient(p, steps, (1.0, 0.0))
    n = p["ncells"] * p["ppc"][0]
    x0, v0, _ = O.load_particles(p, 0, np.arange(n))
    dt, N, w, Te = p["dt"], p["ncells"], (p["L"] / p["ncells"]) / p["ppc"][0], p["T"][0]
    vx = v0[:, 0]
    k = np.arange(1, steps + 1)[:, None]          # position after step n is x0 + (n + 1) vx dt
    x = x0[None, :] + k * vx[None, :] * dt
    out = (x < 0) | (x >= N)
    first_out = np.where(out.any(0), out.argmax(0), steps)  # step index n of the absorption
    alive = np.arange(steps)[:, None] < first_out[None, :]
    d = x - (N - 1)
    S = np.where(np.abs(d) < 1, 1 - np.abs(d), 0.0)
    dS = np.where(np.abs(d) < 1, -np.sign(d), 0.0)
    J_ref = (dt * w * vx[None, :] * S * alive).sum()
    dJ_dvx = (dt * w * (S + vx[None, :] * dS * k * dt) * alive).sum(0)
    g_ref = (dJ_dvx * vx / (2 * Te)).sum()
    assert J[0] == pytest.approx(J_ref, rel=1e-12)
    assert g[1] == pytest.approx(g_ref, rel=1e-10)
    assert g[0] == 0.0
    assert np.array_equal(np.asarray(absorb[:n]), np.where(first_out < steps, first_out, O.ADJ_NEVER))


def test_frozen_plasma_field_energy_closed_form():
    p = W.variant(BASE, frozen_mask=3, V_left=-2.0, V_right=0.25)
    steps = 5
    g_fe, J, _ = O.adj_gradient(p, steps, (0.0, 1.0))
    g_fl, Jf, _ = O.adj_gradient(p, steps, (1.0, 0.0))
    o = O.OracleSim(p)  # same initial particles; its field is the static field here
    E = o.fields()["E"]
    N, dx = p["ncells"], p["L"] / p["ncells"]
    c = np.ones(N + 1)
    c[0] = c[-1] = 0.5
    assert J[1] == pytest.approx((c * 0.5 * E**2 * dx).sum(), rel=1e-9)
    assert g_fe[0] == pytest.approx((c * E).sum() / N, rel=1e-9)
    assert g_fe[1] == 0.0
    # the flux of frozen electrons: each step adds the same sum; its T_e derivative is that sum / 2T_e
    n = N * p["ppc"][0]
    x0, v0, _ = O.load_particles(p, 0, np.arange(n))
    w = dx / p["ppc"][0]
    d = x0 - (N - 1)
    S = np.where(np.abs(d) < 1, 1 - np.abs(d), 0.0)
    per_step = (p["dt"] * w * v0[:, 0] * S).sum()
    assert Jf[0] == pytest.approx(steps * per_step, rel=1e-12)
    assert g_fl[1] == pytest.approx(steps * per_step / (2 * p["T"][0]), rel=1e-12)
    assert g_fl[0] == 0.0


def test_recording_forward_is_the_collisionless_step():
    p = W.variant(BASE, V_left=-0.8)
    steps = 30
    J, absorb = O.adj_forward(p, steps)
    o = O.OracleSim(p)
    o.step(steps)
    d = o.diag()
    n0 = p["ncells"] * p["ppc"][0]
    ab = np.asarray(absorb)
    assert (ab[:n0] < O.ADJ_NEVER).sum() == sum(d["wall_hits"][0])
    assert (ab[n0:] < O.ADJ_NEVER).sum() == sum(d["wall_hits"][1])
    # the main oracle deposits in 2^-32 fixed point; the model here in FP64
    assert J[1] == pytest.approx(d["field_energy"], rel=1e-8)


def test_bias_is_a_uniform_field():
    N, dx = 32, 1.0
    rho = np.random.default_rng(2).standard_normal(N + 1)
    phi0 = np.zeros(N + 1)
    phi1 = np.zeros(N + 1)
    O.lib().orc_poisson_thomas(N, dx, O._ptr(rho, O.C.c_double), 0.0, 0.0, O._ptr(phi0, O.C.c_double))
    O.lib().orc_poisson_thomas(N, dx, O._ptr(rho, O.C.c_double), -3.0, 0.0, O._ptr(phi1, O.C.c_double))
    E0, E1 = np.zeros(N + 1), np.zeros(N + 1)
    O.lib().orc_efield(N, dx, O._ptr(phi0, O.C.c_double), O._ptr(rho, O.C.c_double), O._ptr(E0, O.C.c_double))
    O.lib().orc_efield(N, dx, O._ptr(phi1, O.C.c_double), O._ptr(rho, O.C.c_double), O._ptr(E1, O.C.c_double))
    assert np.allclose(E1 - E0, -3.0 / (N * dx), rtol=0, atol=1e-12)
    assert math.isclose(float((E1 - E0).mean()), -3.0 / N, rel_tol=1e-12)


def test_reverse_sweep_over_a_given_tape_is_the_oracles_own():
    # the entry that reverses a trajectory recorded elsewhere runs the same sweep: fed the oracle's
    # own recording forward it returns the oracle's gradient bit for bit, and a perturbed tape moves it
    p = W.variant(W.C5, ncells=24, L=24.0, ppc=(9, 7), V_left=-0.8, B=0.4, B_angle_deg=50.0)
    steps = 30
    X, V, EN, ab, J = O.adj_trajectory(p, steps)
    for w in ((1.0, 0.0), (0.0, 1.0), (0.7, -1.3)):
        g, J2, ab2 = O.adj_gradient(p, steps, w)
        assert np.array_equal(ab, ab2) and np.array_equal(J, J2)
        assert np.array_equal(O.adj_gradient_from_tape(p, steps, w, X, V, EN, ab), g)
    V2 = V.copy()
    V2[0] *= 1.01
    assert not np.array_equal(O.adj_gradient_from_tape(p, steps, (0.0, 1.0), X, V2, EN, ab),
                              O.adj_gradient(p, steps, (0.0, 1.0))[0])
