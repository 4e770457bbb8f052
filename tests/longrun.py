"""Long-run moments of a run of config 1's physics (256 cells, 100 particles per cell per species,
1000 steps), for the statistical parity of the GPU paths against the FP64 oracle.

Over many steps the FP32 and FP64 trajectories part (the dynamics is chaotic), so parity there is a
statement about distributions: the moments of independent seeds of the GPU path and of the oracle
must be samples of the same distribution.  ``moments`` turns the diagnostics and fields a run
reports into one vector; the oracle's side runs one seed per process (``oracle_moments``, started
by a spawn pool).

Moments (24): live electrons and ions after 250, 500, 750 and 1000 steps; electrons and ions
absorbed at the walls; elastic collisions, ionizations and electron births; kinetic energy of both
species; the electron temperature (2/3) KE_e / (N_e w_e); the potential averaged over the samples
at steps 550, 600, ..., 1000 at the eight nodes j = (2k + 1) N / 16.
"""
from __future__ import annotations

import numpy as np

STEPS = 1000
CHECKPOINTS = (250, 500, 750, 1000)
PHI_FROM, PHI_EVERY = 550, 50
NAMES = ([f"n{s}@{t}" for t in CHECKPOINTS for s in (0, 1)] +
         ["hits_e", "hits_i", "coll_el", "coll_iz", "births_e", "ke_e", "ke_i", "T_e"] +
         [f"phi@{2 * k + 1}/16" for k in range(8)])


def phi_nodes(N: int) -> np.ndarray:
    return np.array([(2 * k + 1) * N // 16 for k in range(8)])


def run(sim, params: dict) -> np.ndarray:
    """Advance ``sim`` (any object with step / diag / fields of the GPU binding's or the oracle's
    shape) by STEPS steps from its start and return the moment vector."""
    N = int(params["ncells"])
    w_e = (params["L"] / N) / params["ppc"][0]
    nodes = phi_nodes(N)
    counts, phi_sum, nphi, t = [], np.zeros(8), 0, 0
    marks = sorted(set(CHECKPOINTS) | set(range(PHI_FROM, STEPS + 1, PHI_EVERY)))
    d = None
    for m in marks:
        sim.step(m - t)
        t = m
        d = sim.diag()
        if m in CHECKPOINTS:
            counts += [d["n"][0], d["n"][1]]
        if m >= PHI_FROM and (m - PHI_FROM) % PHI_EVERY == 0:
            phi_sum += sim.fields()["phi"][nodes]
            nphi += 1
    tail = [sum(d["wall_hits"][0]), sum(d["wall_hits"][1]), d["coll"][0], d["coll"][2], d["births"][0],
            d["ke"][0], d["ke"][1], (2.0 / 3.0) * d["ke"][0] / (d["n"][0] * w_e)]
    return np.array(counts + tail + list(phi_sum / nphi), np.float64)


def oracle_moments(args) -> np.ndarray:
    """One oracle seed (single-threaded; a pool worker)."""
    params, seed = args
    import os
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    from oracle import oracle as O
    from paper_2606_28534_gb300 import workloads as W

    o = O.OracleSim(W.variant(params, seed=seed), threads=1)
    return run(o, params)


def welch_pvalues(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Two-sided Welch t-test of equal means, per column of the sample matrices a and b; a column
    with no spread in either sample gets 1 if the means agree, else 0."""
    from scipy import stats

    out = np.ones(a.shape[1])
    for k in range(a.shape[1]):
        x, y = a[:, k], b[:, k]
        if x.std() == 0 and y.std() == 0:
            out[k] = 1.0 if x.mean() == y.mean() else 0.0
        else:
            out[k] = stats.ttest_ind(x, y, equal_var=False).pvalue
    return out
