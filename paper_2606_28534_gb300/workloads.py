"""Seeded synthetic workloads of the 1D3V PIC Monte Carlo step.

Plain parameter dictionaries (no arithmetic of the method).  They stand in for the paper's
high-density sheath decks (Table 3: bounded, magnetised plasma between absorbing walls), which
are not available; sizes follow the five benchmark configurations, scaled to one GPU.
Both the GPU binding and the test oracle read these dictionaries; each fills its own
configuration struct from them.

Units: lengths in Debye lengths (dx = L/ncells = 1 here), time in 1/omega_pe, masses in m_e,
temperatures in T_e.  Cross sections are given as n_gas * sigma with n_gas = 1, so that
``sigma_el`` is the electron elastic collision frequency at the thermal speed (v_th,e = 1).
"""
from __future__ import annotations

COLL_EL, COLL_EX, COLL_IZ, COLL_CX = 1, 2, 4, 8
FIELD_SELF, FIELD_EXTERNAL, FIELD_ZERO = 0, 1, 2
LOAD_UNIFORM, LOAD_EXP, LOAD_QUIET_SINE = 0, 1, 2
SOURCE_NONE, SOURCE_PAIRS = 0, 1
PRECISION_FP32, PRECISION_FP64_PLAIN = 0, 1

SEED0 = 20260101

#: electrons + He+ (mass ratio 7344), T_e = 1, T_i = T_g = 0.1, omega_p dt = 0.1, grounded walls,
#: elastic (nu/omega_p = 0.01 at v_th,e) + ionization (0.1 sigma_el above E_iz = 2.46 T_e).
BASE = dict(
    ncells=256, L=256.0, dt=0.1, ppc=(100, 100), mass=(1.0, 7344.0), charge=(-1.0, 1.0),
    T=(1.0, 0.1), Tg=0.1, m_gas=7344.0, B=0.0, B_angle_deg=0.0, V_left=0.0, V_right=0.0,
    n_gas=1.0, sigma_el=0.01, sigma_ex=0.002, E_ex=1.98, sigma_iz=0.001, E_iz=2.46,
    sigma_cx=0.02, E_cap=32.0, E_ext=0.0, coll_mask=COLL_EL | COLL_IZ, field_mode=FIELD_SELF,
    frozen_mask=0, load_profile=LOAD_UNIFORM, profile_mode=0, profile_scale=0.0,
    source_mode=SOURCE_NONE, source_x1=0.0, sort_interval=10, capacity_factor=1.25,
    precision=PRECISION_FP32, seed=SEED0 + 1,
)


def variant(base: dict, **kw) -> dict:
    d = dict(base)
    d.update(kw)
    return d


#: config 1: plain PIC MC, 256 cells, 100 ppc per species (51,200 particles), 1000 steps.
C1 = variant(BASE, precision=PRECISION_FP64_PLAIN, seed=SEED0 + 1)
C1_STEPS = 1000

#: config 2: uniform load, 4096 cells x 1000 ppc per species (8,192,000 particles),
#: B = 0.5 at 30 degrees to the wall normal, all four processes, left wall at -3 T_e.
C2 = variant(BASE, ncells=4096, L=4096.0, ppc=(1000, 1000), B=0.5, B_angle_deg=30.0,
             V_left=-3.0, coll_mask=COLL_EL | COLL_EX | COLL_IZ | COLL_CX, seed=SEED0 + 2)
C2_WARMUP, C2_STEPS = 100, 200

#: config 3: non-uniform load, 65536 cells, 763 ppc per species on average (100,007,936
#: particles), density ~ exp(-x/(L/8)), pair source in [0, L/16), config 2's physics.
C3 = variant(C2, ncells=65536, L=65536.0, ppc=(763, 763), load_profile=LOAD_EXP,
             profile_scale=8192.0, source_mode=SOURCE_PAIRS, source_x1=4096.0,
             capacity_factor=1.15, seed=SEED0 + 3)
C3_STEPS = 100

#: config 4: an ensemble of 256 independent runs of config 2's physics (B = 0.5 at 30 degrees, all
#: four processes), each with its own size and plasma: cells uniform in [128, 8192] (dx = 1),
#: particles per cell uniform in [50, 500] (both species), electron collisionality nu/omega_p =
#: n_gas * sigma_el log-uniform in [0.001, 0.1], left-wall bias uniform in [-5, 0] T_e (right wall
#: grounded), 500 steps; about 5.9e8 particles in all.
C4_SIMS, C4_STEPS = 256, 500


def ensemble(n: int = C4_SIMS, seed: int = SEED0 + 4, cells=(128, 8192), ppc=(50, 500),
             nu=(1e-3, 1e-1), bias=(-5.0, 0.0), base: dict | None = None, **kw) -> list:
    """Seeded draw of ``n`` run configurations (numpy PCG64, fixed seed); run k gets the run seed
    ``seed * 4096 + k``.  Extra keyword arguments override fields of every run."""
    import numpy as np

    base = C2 if base is None else base
    g = np.random.default_rng(seed)
    out = []
    for k in range(n):
        N = int(g.integers(cells[0], cells[1] + 1))
        m = int(g.integers(ppc[0], ppc[1] + 1))
        lnu = g.uniform(np.log(nu[0]), np.log(nu[1]))
        V = float(g.uniform(bias[0], bias[1]))
        out.append(variant(base, ncells=N, L=float(N), ppc=(m, m), n_gas=float(np.exp(lnu)) / base["sigma_el"],
                           V_left=V, V_right=0.0, seed=seed * 4096 + k, **kw))
    return out


def c4() -> list:
    return ensemble()


#: a small heterogeneous ensemble the oracle finishes in seconds: sizes from 2 cells up, few
#: particles per cell, collisionality up to strongly collisional
def small_ensemble(n: int = 9, seed: int = SEED0 + 40) -> list:
    runs = ensemble(n, seed=seed, cells=(24, 220), ppc=(5, 48), nu=(1e-3, 2.5e-1))
    special = [dict(ncells=2, L=2.0, ppc=(7, 7)),                    # the smallest grid
               dict(coll_mask=0),                                    # collisionless
               dict(coll_mask=COLL_CX, ppc=(9, 23)),                 # ions only collide; unequal ppc
               dict(n_gas=25.0),                                     # every process fires often
               dict(load_profile=LOAD_EXP, profile_scale=16.0)]
    for k, kw in enumerate(special[:n]):
        runs[k] = variant(runs[k], **kw)
    return runs


#: D+/e/D sheath (Table 3: D+ ions recycled into D neutrals at the walls; Sec. 2: density
#: smoothing), on config 3's grid, load and source: deuterium ions (m_D / m_e = 3670.483), every ion
#: absorbed at a wall returns as a tracked neutral (flux half-Maxwellian at T_rec = 0.1), a uniform
#: neutral background of 763 per cell at t = 0 (50 M neutrals), electron-impact ionization of the
#: neutrals with K_iz n_e dt = 2e-4 per step at n_e = 1, two smoothing passes; 150 M particles.
M_D = 3670.483
C6 = variant(C3, mass=(1.0, M_D), m_gas=M_D, smooth_passes=2, neutrals=1, neutral_ppc=763, recycle=1.0,
             T_rec=0.1, K_iz=0.002, T_sec=1.0, neutral_capacity=1.15, seed=SEED0 + 6)
C6_STEPS = 100

#: config 5: collisionless adjoint case, 1024 cells x 200 ppc, 200 steps.
C5 = variant(BASE, ncells=1024, L=1024.0, ppc=(200, 200), coll_mask=0, seed=SEED0 + 5)
C5_STEPS = 200

# ------------------------------------------------------------------------------------------------
# Small cases the oracle finishes in seconds: several 1024-particle tiles and ragged tails.
SMALL_C1 = variant(C1, ncells=64, L=64.0, ppc=(37, 37), precision=PRECISION_FP32)
SMALL_C2 = variant(C2, ncells=96, L=96.0, ppc=(53, 53))
SMALL_C3 = variant(C3, ncells=512, L=512.0, ppc=(41, 41), profile_scale=64.0, source_x1=32.0)
#: strongly collisional: every process fires often, to exercise the collision paths.
SMALL_COLL = variant(SMALL_C2, n_gas=25.0, ncells=48, L=48.0, ppc=(61, 61))

#: the D+/e/D sheath, small: uniform plasma and neutrals on 96 cells, walls biased, ionization of
#: the neutrals fast enough to fire every step
SMALL_C6 = variant(C6, ncells=96, L=96.0, ppc=(53, 53), neutral_ppc=31, load_profile=LOAD_UNIFORM,
                   source_mode=SOURCE_NONE, K_iz=0.5)

#: profiling case: config 3's physics and profile with 1/8 of the particles (12.5 M, 350 MB of
#: particle data: larger than L2, small enough for multi-pass counter captures)
C3_PROFILE = variant(C3, ppc=(96, 96))
#: config 3 with half of its particles (profiling case of the step's claimed chunk segments, which a
#: species takes from 48 chunks per warp on: 25 M particles per species)
C3_HALF = variant(C3, ppc=(384, 384))

#: the D+/e/D sheath with 1/8 of the particles (profiling case)
C6_PROFILE = variant(C6, ppc=(96, 96), neutral_ppc=96)

CONFIGS = {"c1": C1, "c2": C2, "c3": C3, "c5": C5, "c3p": C3_PROFILE, "c3h": C3_HALF, "c6": C6,
           "c6p": C6_PROFILE}
