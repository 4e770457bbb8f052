"""The adjoint of the collisionless step (pic_adj_*, torch.autograd) against the FP64 oracle.

What is compared, and why these tolerances:
* Recording forward: the absorption schedule equals the oracle's particle for particle, and
  J = (J_flux, J_fe) agrees to the FP32 trajectory error (measured ~1e-7 relative; bound 2e-5).
* Gradient: the GPU adjoint (FP32 trajectory, FP64 reverse sweep) and the oracle's FP64 adjoint
  differentiate the same map along trajectories that differ by FP32 rounding.  The flux gradients
  agree to ~3e-5 relative (bound 1e-3 of the gradient's norm); the final field energy depends on the
  fine structure of the last field and its gradients differ by up to ~3e-3 of the gradient's norm
  at config 5 (bound 1e-2 of the norm).
* Central finite differences (h = 1e-3) of the replaying (frozen-schedule) forward: the map has a
  kink wherever a particle crosses a cell boundary, so at h = 1e-3 the secant of a 4e5-particle
  run is not the derivative (the oracle's own FP64 secant shows the same departure; at h <= 1e-6
  it converges to the adjoint, see test_oracle_pins_adjoint.py).  The GPU secant is therefore held
  to the oracle's FP64 secant at the same h, within the FP32 forward error divided by h.
* Checkpoint interval: any interval gives the same gradient (the recomputed states are bit-identical;
  only the order of FP64 atomic sums differs): 1e-12 relative.
* The reverse sweep alone: the oracle's reverse sweep run over the GPU's own recorded trajectory
  (its FP32 states, FP64 node fields and schedule, read back with pic_adj_tape) must give the GPU's
  gradient to 1e-9 relative per component.  That separates an error of the reverse sweep from the
  FP32-vs-FP64 trajectory difference the comparisons above allow for.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2606_28534_gb300 import build, pic
from paper_2606_28534_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SMALL = W.variant(W.C5, ncells=96, L=96.0, ppc=(40, 40), V_left=-1.5)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    import torch

    assert torch.cuda.is_available(), "GPU tests need CUDA"
    pic.lib()


def _grads(a):
    return np.array([a.gradient(1.0, 0.0), a.gradient(0.0, 1.0)])  # [observable, parameter]


def _oracle_grads(p, steps):
    gf, J, ab = O.adj_gradient(p, steps, (1.0, 0.0))
    ge, _, _ = O.adj_gradient(p, steps, (0.0, 1.0))
    return np.array([gf, ge]), J, ab


def _check_against_oracle(p, steps, K):
    a = pic.Adjoint(p, steps, K)
    J = np.array(a.forward(p["V_left"], p["T"][0]))
    g = _grads(a)
    go, Jo, abo = _oracle_grads(p, steps)
    assert np.array_equal(a.schedule(), abo)
    assert (abo < O.ADJ_NEVER).sum() > 0
    assert np.all(np.abs(J - Jo) <= 2e-5 * np.abs(Jo)), (J, Jo)
    assert np.linalg.norm(g[0] - go[0]) <= 1e-3 * np.linalg.norm(go[0]), (g[0], go[0])
    assert np.linalg.norm(g[1] - go[1]) <= 1e-2 * np.linalg.norm(go[1]), (g[1], go[1])
    return a, J, Jo


@pytest.mark.parametrize("case", ["plain", "magnetised", "biased_right", "frozen_ions"])
def test_gradient_matches_the_oracle_adjoint(case):
    p = {"plain": SMALL, "magnetised": W.variant(SMALL, B=0.5, B_angle_deg=30.0),
         "biased_right": W.variant(SMALL, V_right=0.6, T=(1.4, 0.1)),
         "frozen_ions": W.variant(SMALL, frozen_mask=2)}[case]
    a, _, _ = _check_against_oracle(p, 80, 20)
    a.close()


def test_replay_at_the_recorded_point_repeats_it_and_keeps_the_tape():
    a = pic.Adjoint(SMALL, 60, 20)
    J = a.forward(SMALL["V_left"], SMALL["T"][0])
    g = _grads(a)
    assert a.forward(SMALL["V_left"], SMALL["T"][0], replay=True) == J
    a.forward(SMALL["V_left"] + 0.3, SMALL["T"][0] * 1.1, replay=True)  # a replay leaves the tape alone
    assert np.allclose(_grads(a), g, rtol=1e-12, atol=0)
    a.close()


def test_checkpoint_interval_does_not_change_the_gradient():
    ref = None
    for K in (1, 7, 20, 60):
        a = pic.Adjoint(SMALL, 60, K)
        a.forward(SMALL["V_left"], SMALL["T"][0])
        g = _grads(a)
        a.close()
        if ref is None:
            ref = g
        assert np.allclose(g, ref, rtol=1e-12, atol=1e-15), (K, g, ref)


def test_autograd_function_runs_the_reverse_sweep():
    import torch

    from paper_2606_28534_gb300 import adjoint

    a = pic.Adjoint(SMALL, 60, 20)
    theta = torch.tensor([SMALL["V_left"], SMALL["T"][0]], dtype=torch.float64, requires_grad=True)
    J = adjoint.observables(theta, a)
    (gflux,) = torch.autograd.grad(J[0], theta, retain_graph=True)
    (gfe,) = torch.autograd.grad(J[1], theta, retain_graph=True)
    ref = _grads(a)
    assert np.allclose(gflux.numpy(), ref[0], rtol=1e-12) and np.allclose(gfe.numpy(), ref[1], rtol=1e-12)
    # a combination: one reverse sweep for the vector-Jacobian product
    (gmix,) = torch.autograd.grad(0.5 * J[0] - 2.0 * J[1], theta, retain_graph=True)
    assert np.allclose(gmix.numpy(), 0.5 * ref[0] - 2.0 * ref[1], rtol=1e-11)
    # a newer recording forward invalidates the older graph
    J2 = adjoint.observables(theta.detach().clone().requires_grad_(True), a)
    with pytest.raises(RuntimeError):
        torch.autograd.grad(J[0], theta)
    del J2
    a.close()


def test_replay_requires_a_recording_and_bad_arguments_are_refused():
    a = pic.Adjoint(SMALL, 20, 5)
    with pytest.raises(pic.PicError):
        a.forward(-1.0, 1.0, replay=True)
    with pytest.raises(pic.PicError):
        a.gradient()
    with pytest.raises(pic.PicError):
        a.forward(-1.0, 0.0)  # T_e must be positive
    a.close()
    for bad in (dict(coll_mask=1), dict(source_mode=W.SOURCE_PAIRS, source_x1=4.0)):
        with pytest.raises(pic.PicError):
            pic.Adjoint(W.variant(SMALL, **bad), 20, 5)
    with pytest.raises(pic.PicError):
        pic.Adjoint(SMALL, 20, 21)  # checkpoint interval beyond the run


def test_config5_full_size_against_the_oracle_and_finite_differences():
    p = W.variant(W.C5, V_left=-1.0)
    steps, h = W.C5_STEPS, 1e-3
    a, J, Jo = _check_against_oracle(p, steps, 20)
    sched = a.schedule()
    VL, Te = p["V_left"], p["T"][0]

    def fd_gpu():
        f = lambda dV, dT: np.array(a.forward(VL + dV, Te + dT, replay=True))
        return np.stack([(f(h, 0) - f(-h, 0)) / (2 * h), (f(0, h) - f(0, -h)) / (2 * h)], axis=1)

    def fd_oracle():
        f = lambda dV, dT: O.adj_forward(dict(p, V_left=VL + dV, T=(Te + dT, p["T"][1])), steps, sched)[0]
        return np.stack([(f(h, 0) - f(-h, 0)) / (2 * h), (f(0, h) - f(0, -h)) / (2 * h)], axis=1)

    fg, fo = fd_gpu(), fd_oracle()  # [observable, parameter]
    # the same secant of the same map: equal within the FP32 forward error over h (x5 margin; the
    # error at the base point, at least 1e-7 of J, stands for the error at theta +- h)
    tol = 5 * np.maximum(np.abs(J - Jo), 1e-7 * np.abs(Jo))[:, None] / h
    assert np.all(np.abs(fg - fo) <= tol), (fg, fo, tol)
    a.close()


def _gpu_tape(a, p, steps):
    """The GPU's recorded forward in the oracle's tape layout.  The FP32 push gathers the node field
    rounded to FP32, so the fields of the pushes (E^0 .. E^{steps-1}) are given as the pushes used
    them; the final field E^steps enters J_fe in FP64."""
    n = a.n
    X = np.empty((steps + 1, n))
    V = np.empty((steps + 1, n, 3))
    EN = np.empty((steps + 1, p["ncells"] + 1))
    for k in range(steps + 1):
        cell, fr, v, E = a.tape(k)
        with np.errstate(invalid="ignore", over="ignore"):  # absorbed particles hold arbitrary states
            X[k] = cell + fr.astype(np.float64)
            V[k] = v
        EN[k] = E.astype(np.float32).astype(np.float64) if k < steps else E
    return X, V, EN


@pytest.mark.parametrize("case", ["config5", "magnetised", "biased_right", "frozen_ions"])
def test_reverse_sweep_equals_the_oracles_on_the_gpu_trajectory(case):
    p, steps, K = {"config5": (W.variant(W.C5, V_left=-1.0), W.C5_STEPS, 20),
                   "magnetised": (W.variant(SMALL, B=0.5, B_angle_deg=30.0), 80, 20),
                   "biased_right": (W.variant(SMALL, V_right=0.6, T=(1.4, 0.1)), 80, 20),
                   "frozen_ions": (W.variant(SMALL, frozen_mask=2), 80, 20)}[case]
    a = pic.Adjoint(p, steps, K)
    a.forward(p["V_left"], p["T"][0])
    absorb = a.schedule()
    X, V, EN = _gpu_tape(a, p, steps)
    # the tape is the recorded forward: its state at a checkpoint step is the checkpoint itself, and
    # the particles the schedule keeps stay inside the walls
    alive = absorb > steps - 1
    assert (X[steps][alive] >= 0).all() and (X[steps][alive] < p["ncells"]).all()
    for w in ((1.0, 0.0), (0.0, 1.0)):
        g = np.array(a.gradient(*w))
        go = O.adj_gradient_from_tape(p, steps, w, X, V, EN, absorb)
        assert np.all(np.abs(g - go) <= 1e-9 * np.abs(go) + 1e-14 * np.abs(go).max()), (case, w, g, go)
    a.close()
