"""Pins of the oracle's numerical building blocks against values fixed outside the oracle.

* Philox4x32-10 against the published known-answer vectors (tests/golden) and uniformity.
* Poisson (Thomas) against closed forms of the second-order difference operator and a dense
  library solve; the wall field against Gauss's law.
* Boris rotation against the analytic gyration phase and the E x B drift velocity.
"""
import os

import numpy as np
import pytest

from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            w = [int(t, 16) for t in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def test_philox_known_answers():
    rows = _kat()
    assert len(rows) == 3
    ctr = np.array([r[0] for r in rows], np.uint32)
    key = np.array([r[1] for r in rows], np.uint32)
    out = O.philox(ctr, key)
    assert out.tolist() == [r[2] for r in rows]


def test_philox_uniform_and_independent_words():
    n = 200_000
    rng = np.random.default_rng(7)
    ctr = np.zeros((n, 4), np.uint32)
    ctr[:, 0] = np.arange(n, dtype=np.uint32)
    ctr[:, 2] = 2
    key = rng.integers(0, 2**32, (n, 2), dtype=np.uint64).astype(np.uint32)
    out = O.philox(ctr, key)
    u = (out >> 8).astype(np.float64) / 2**24
    for k in range(4):
        counts, _ = np.histogram(u[:, k], bins=64, range=(0, 1))
        chi2 = ((counts - n / 64) ** 2 / (n / 64)).sum()
        assert chi2 < 130, chi2  # 63 dof, p ~ 1e-6
    c = np.corrcoef(u.T)
    assert np.abs(c - np.eye(4)).max() < 0.01
    # a change of one counter bit changes about half of the output bits (avalanche)
    ctr2 = ctr.copy()
    ctr2[:, 3] ^= 1
    out2 = O.philox(ctr2, key)
    flips = np.unpackbits((out ^ out2).view(np.uint8)).mean()
    assert abs(flips - 0.5) < 0.01


# ------------------------------------------------------------------------------------------------
def _cond_tol(N):
    # forward error bound of a tridiagonal solve: cond(tridiag(-1, 2, -1)) ~ 4 N^2 / pi^2 times
    # the unit roundoff, floored at 1e-13 for the smallest systems
    return max(1e-13, 4 * N * N / np.pi**2 * 2.0**-52)


@pytest.mark.parametrize("N,dx", [(2, 1.0), (7, 0.5), (256, 1.0), (4096, 2.0)])
def test_poisson_uniform_rho_is_exact_parabola(N, dx):
    # -phi'' = rho with phi(0) = phi(L) = 0 has phi = rho x (L - x)/2; the three-point
    # difference operator is exact on quadratics, so the discrete solution equals it at nodes.
    rho0 = 0.37
    rho = np.full(N + 1, rho0)
    phi = O.poisson_thomas(rho, dx, 0.0, 0.0)
    x = np.arange(N + 1) * dx
    exact = rho0 * x * (N * dx - x) / 2
    assert np.abs(phi - exact).max() <= _cond_tol(N) * np.abs(exact).max() + 1e-15


@pytest.mark.parametrize("N,m", [(64, 1), (64, 5), (1000, 17)])
def test_poisson_sine_mode_discrete_eigenvalue(N, m):
    # rho_j = sin(k x_j), k = pi m / L: the eigenvalue of (-1, 2, -1)/dx^2 on this mode is
    # 4 sin^2(k dx/2)/dx^2, so phi_j = sin(k x_j) dx^2 / (4 sin^2(k dx / 2)).
    dx = 0.75
    L = N * dx
    k = np.pi * m / L
    x = np.arange(N + 1) * dx
    rho = np.sin(k * x)
    phi = O.poisson_thomas(rho, dx, 0.0, 0.0)
    exact = np.sin(k * x) * dx**2 / (4 * np.sin(k * dx / 2) ** 2)
    assert np.abs(phi - exact).max() <= _cond_tol(N) * np.abs(exact).max()


def test_poisson_vacuum_is_linear_between_wall_potentials():
    N = 100
    phi = O.poisson_thomas(np.zeros(N + 1), 1.0, -3.0, 2.0)
    exact = -3.0 + 5.0 * np.arange(N + 1) / N
    assert np.abs(phi - exact).max() < 1e-13


def test_poisson_matches_dense_library_solve():
    rng = np.random.default_rng(3)
    N, dx = 50, 0.3
    rho = rng.standard_normal(N + 1)
    VL, VR = 1.5, -0.25
    phi = O.poisson_thomas(rho, dx, VL, VR)
    A = 2 * np.eye(N - 1) - np.eye(N - 1, k=1) - np.eye(N - 1, k=-1)
    b = dx * dx * rho[1:N].copy()
    b[0] += VL
    b[-1] += VR
    ref = np.linalg.solve(A, b)
    assert phi[0] == VL and phi[N] == VR
    assert np.abs(phi[1:N] - ref).max() <= 1e-12 * np.abs(ref).max()


def test_efield_centered_and_wall_gauss():
    # uniform rho, grounded walls: E = -phi' = rho (x - L/2), exact at interior nodes for a
    # parabola; at the walls Gauss's law over the half cell gives the same linear value.
    N, dx, rho0 = 40, 0.5, 0.8
    rho = np.full(N + 1, rho0)
    phi = O.poisson_thomas(rho, dx, 0.0, 0.0)
    E = O.efield(phi, rho, dx)
    x = np.arange(N + 1) * dx
    assert np.abs(E - rho0 * (x - N * dx / 2)).max() < 1e-12
    # total charge (trapezoid, half cells at walls) equals the jump of E across the domain
    q = dx * (rho[1:N].sum() + 0.5 * rho[0] + 0.5 * rho[N])
    assert abs((E[N] - E[0]) - q) < 1e-12


# ------------------------------------------------------------------------------------------------
def test_boris_gyration_phase_and_speed():
    # E = 0: the Boris rotation keeps |v| and v_parallel and turns v_perp by 2 atan(w_c dt/2)
    # per step (the Boris phase error of the exact w_c dt).
    B = 0.5 * np.array([np.cos(np.pi / 6), np.sin(np.pi / 6), 0.0])
    qm, dt = -1.0, 0.1
    b = B / np.linalg.norm(B)
    v0 = np.array([0.3, -1.1, 0.7])
    vpar0 = v0 @ b
    v = v0.copy()
    nsteps = 1000
    for _ in range(nsteps):
        v = O.boris(qm, dt, np.zeros(3), B, v)
    assert abs(np.linalg.norm(v) - np.linalg.norm(v0)) < 1e-12
    assert abs(v @ b - vpar0) < 1e-12
    e1 = v0 - vpar0 * b
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(b, e1)
    vp = v - (v @ b) * b
    ang = np.arctan2(vp @ e2, vp @ e1)
    wc = abs(qm) * np.linalg.norm(B)
    phase = 2 * np.arctan(wc * dt / 2)
    # electron (q < 0) turns counter-clockwise about b
    expect = np.angle(np.exp(1j * nsteps * phase))
    assert abs(np.angle(np.exp(1j * (ang - expect)))) < 1e-9
    assert abs(phase - 0.049989585) < 1e-8


def test_boris_exb_drift():
    # E perpendicular to B: the gyro-averaged velocity is E x B / B^2 (exact for Boris).
    B = np.array([0.0, 0.8, 0.0])
    E = np.array([0.05, 0.0, 0.0])
    qm, dt = -1.0, 0.1
    v = np.array([0.0, 0.0, 0.0])
    wc = abs(qm) * 0.8
    phase = 2 * np.arctan(wc * dt / 2)
    period = 2 * np.pi / phase
    n = int(round(period * 40))
    acc = np.zeros(3)
    for k in range(n):
        v_new = O.boris(qm, dt, E, B, v)
        acc += v_new
        v = v_new
    mean = acc / n
    drift = np.cross(E, B) / (B @ B)
    assert np.abs(mean - drift).max() < 2e-3 * np.linalg.norm(drift) + 1e-4
    assert abs(mean[2] - drift[2]) / abs(drift[2]) < 2e-2


def test_boris_pure_electric_acceleration():
    v = O.boris(-1.0, 0.1, np.array([2.0, 0, 0]), np.zeros(3), np.array([0.5, 0.1, -0.2]))
    assert np.allclose(v, [0.5 - 0.2, 0.1, -0.2], atol=1e-15)
