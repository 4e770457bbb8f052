/*
 * pic_oracle.h -- plain FP64 CPU oracle of the 1D3V electrostatic PIC Monte Carlo step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU-baseline leg
 * of the benchmark may load this library.  The GPU library never includes, links or calls it,
 * and this file includes nothing from the GPU library: the two share no code.
 *
 * What it computes follows the PIC cycle of the paper (Sec. 2: particle mover, deposition
 * to the grid, field solver, force interpolation, plus Monte Carlo collisions) for the BIT1
 * model of a bounded plasma between two absorbing walls (Table 3), taken step by step in the
 * order below, in FP64, with plain loops.  The paper gives no formulas; every numerical choice
 * is one of the stated readings (R1..R16 in the design notes), restated at the point of use.
 *
 * Units: lengths in Debye lengths, time in 1/omega_pe, m_e = e = eps0 = n0 = T_e = 1.
 * Positions are absolute, in units of the cell size dx (x_hat = x/dx), in [0, ncells).
 */
#ifndef PIC_ORACLE_H
#define PIC_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2
#define ORC_ECORRUPT 5

/* collision processes (bit mask) */
#define ORC_COLL_EL 1u /* electron-neutral elastic */
#define ORC_COLL_EX 2u /* electron-neutral excitation */
#define ORC_COLL_IZ 4u /* electron-impact ionization */
#define ORC_COLL_CX 8u /* ion-neutral charge exchange */

/* field modes */
#define ORC_FIELD_SELF 0u     /* self-consistent Poisson field */
#define ORC_FIELD_EXTERNAL 1u /* uniform E_x = E_ext, no self field on particles */
#define ORC_FIELD_ZERO 2u     /* no electric field */

/* load profiles */
#define ORC_LOAD_UNIFORM 0    /* ppc per cell, random position inside the cell */
#define ORC_LOAD_EXP 1        /* density ~ exp(-x/lambda), lambda = profile_scale (dx units) */
#define ORC_LOAD_QUIET_SINE 2 /* evenly spaced; species 0 displaced by A sin(2 pi m x/L) */

/* sources */
#define ORC_SOURCE_NONE 0
#define ORC_SOURCE_PAIRS 1 /* inject one (e, ion) pair per ion absorbed in this step */

/* Philox counter word 2: the stream ("channel") of a draw */
#define ORC_CH_INIT 1u
#define ORC_CH_COLL 2u
#define ORC_CH_SCAT 3u
#define ORC_CH_CHILD 4u
#define ORC_CH_SOURCE 5u
#define ORC_CH_RECYCLE 6u /* recycling of an absorbed ion into a neutral */
#define ORC_CH_NIZ 7u     /* electron-impact ionization of a tracked neutral */

#define ORC_MAX_SMOOTH 4 /* passes of the density filter */

typedef struct {
  int32_t ncells;         /* number of cells N (>= 2); nodes 0..N */
  int32_t ppc[2];         /* mean particles per cell per species; weight w_s = dx/ppc_s */
  int32_t load_profile;   /* ORC_LOAD_* */
  int32_t profile_mode;   /* QUIET_SINE mode number m */
  int32_t source_mode;    /* ORC_SOURCE_* */
  int32_t sort_interval;  /* sort + compact when step % sort_interval == 0 (>= 1) */
  uint32_t coll_mask;     /* ORC_COLL_* */
  uint32_t field_mode;    /* ORC_FIELD_* */
  uint32_t frozen_mask;   /* bit s: species s is neither pushed nor collided */
  double L;               /* domain length (Debye lengths); dx = L/N */
  double dt;              /* time step (1/omega_pe) */
  double mass[2];         /* species masses (m_e units); species 0 = electrons */
  double charge[2];       /* species charges (e units) */
  double T[2];            /* initial temperatures (T_e units) */
  double Tg;              /* neutral gas temperature (ion birth / CX velocity) */
  double m_gas;           /* neutral mass (elastic energy transfer) */
  double B;               /* |B| (omega_ce/omega_pe for an electron) */
  double B_angle_deg;     /* angle of B to the wall normal x, in the x-y plane */
  double V_left, V_right; /* wall potentials (T_e/e) */
  double n_gas;           /* neutral density */
  double sigma_el;        /* constant elastic cross section */
  double sigma_ex, E_ex;  /* excitation: sigma_ex * min((E-E_ex)/E_ex, 1) above E_ex */
  double sigma_iz, E_iz;  /* ionization: sigma_iz * min((E-E_iz)/E_iz, 1) above E_iz */
  double sigma_cx;        /* constant charge-exchange cross section */
  double E_cap;           /* null-collision energy cap before the wall-bias term */
  double E_ext;           /* ORC_FIELD_EXTERNAL field */
  double profile_scale;   /* EXP: scale length (dx units); QUIET_SINE: amplitude (dx units) */
  double source_x1;       /* source region [0, source_x1) (dx units) */
  uint64_t seed;          /* run seed: part of every Philox key and counter */
  /* D+/e/D sheath physics (Table 3: ions recycled into neutrals at the walls; Sec. 2: density
   * smoothing).  Zero: none of it. */
  int32_t smooth_passes;  /* binomial passes over the charge density before the solve (0..4) */
  uint32_t neutrals;      /* 1: species 2, tracked neutrals of the ion mass, charge 0 */
  int32_t neutral_ppc;    /* initial neutrals per cell: uniform, Maxwellian at T_rec (0: none) */
  uint32_t reserved;      /* 0 */
  double recycle;         /* probability that an ion absorbed at a wall returns as a neutral */
  double T_rec;           /* temperature of the recycled neutrals (flux half-Maxwellian) */
  double K_iz;            /* rate coefficient of electron-impact ionization of a neutral */
  double T_sec;           /* temperature of the electron a neutral's ionization creates */
} orc_config;

typedef struct {
  uint64_t step;
  uint64_t n[2];                 /* live particles */
  uint64_t wall_hits[2][2];      /* [species][0 = left wall, 1 = right wall] */
  uint64_t coll[5];              /* e elastic, e excitation, e ionization, ion CX, candidates */
  uint64_t near_threshold[2];    /* candidate draws within 1e-5 of a process boundary */
  uint64_t nu_max_violations[2]; /* candidates with nu_total > nu_max */
  uint64_t births[2];            /* particles created by ionization */
  uint64_t source_pairs;         /* pairs injected by the source */
  uint64_t dropped;              /* particles lost to a full buffer (always 0 here) */
  int64_t net_charge_units;      /* sum_j sum_s sign(q_s) R_sj, units 2^-32 particle */
  int64_t wall_charge;           /* sum over absorbed particles of sign(q) */
  double ke[2];                  /* sum 0.5 m v^2 w (at the half step) */
  double field_energy;           /* sum_j 0.5 eps0 E_j^2 dx, half weight at the walls */
  double wall_energy[2];         /* sum over absorbed particles of 0.5 m v^2 w */
  uint64_t particle_steps;       /* sum over steps of the live particles at step start */
} orc_diag_t;

/* Tracked neutrals (species 2), cumulative since creation unless stated. */
typedef struct {
  uint64_t n;                 /* live neutrals */
  uint64_t recycled[2];       /* neutrals created by recycling at [0 = left, 1 = right] wall */
  uint64_t lost[2];           /* neutrals absorbed at [left, right] wall */
  uint64_t ionized;           /* neutrals ionized (each became an ion and created an electron) */
  uint64_t near_threshold;    /* ionization draws within 1e-5 relative of the probability */
  uint64_t particle_steps;    /* sum over steps of the live neutrals at step start */
  double ke;                  /* sum 0.5 m v^2 w over live neutrals */
} orc_ndiag_t;

typedef struct orc_sim orc_sim;

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), one block. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* n blocks: ctr is n x 4 words, key n x 2 words, out n x 4 words. */
void orc_philox_batch(size_t n, const uint32_t* ctr, const uint32_t* key, uint32_t* out);

/* Interior Poisson problem by the Thomas algorithm: -phi_{j-1} + 2 phi_j - phi_{j+1} =
 * dx^2 rho_j / eps0 for j = 1..N-1, phi_0 = V_L, phi_N = V_R.  rho, phi: N+1 nodes. */
int orc_poisson_thomas(int32_t N, double dx, const double* rho, double V_L, double V_R,
                       double* phi);
/* Node field from phi (centred differences) and Gauss's law over the half cell at a wall. */
void orc_efield(int32_t N, double dx, const double* phi, const double* rho, double* E);

/* One Boris step of a velocity: E and B are 3-vectors, qm = q/m. */
void orc_boris(double qm, double dt, const double E[3], const double B[3], double v[3]);

/* Null-collision bound per species (R8), already rounded to FP32. */
void orc_nu_max(const orc_config* cfg, float nu_max[2], float p_null[2]);

/* Initial state of particle i of species sp (x in dx units, v, id) as the load creates it;
 * sp = 2: initial neutral i. */
void orc_load_particle(const orc_config* cfg, int sp, uint64_t i, double* x, double v[3], uint64_t* id);

/* Simulation object. */
orc_sim* orc_create(const orc_config* cfg, int* err);
void orc_free(orc_sim* s);
int orc_step(orc_sim* s, int32_t nsteps);
/* One step of n given particles of species sp under the node field E (N + 1 values): mover, wall
 * test and null-collision MC exactly as orc_step, for parity checks that sample a large state.
 * x in cells, v as n (vx, vy, vz) triples, nk the null-collision countdown pairs (k | c << 12, as a
 * snapshot's cell word carries them in bits 18..30), nko the pairs after the step; flags: 1 absorbed,
 * 2 candidate, 4 near-threshold draw, 8 ionization.  Neutrals and the pair source are not included. */
int orc_step_sample(const orc_config* cfg, int sp, uint64_t step, const double* E, size_t n, const double* x,
                    const double* v, const uint64_t* id, const uint32_t* nk, double* xo, double* vo, uint32_t* nko,
                    int32_t* flags);
int orc_diag(orc_sim* s, orc_diag_t* out);
/* R: 2 x (N+1) int64 fixed-point deposits, rho/phi/E: N+1 nodes each; any may be NULL. */
int orc_fields(orc_sim* s, int64_t* R, double* rho, double* phi, double* E);
uint64_t orc_count(orc_sim* s, int species);
int orc_neutral_diag(orc_sim* s, orc_ndiag_t* out);
/* The density filter of smooth_passes passes, in place on a node density rho (N + 1 nodes). */
void orc_smooth(int32_t N, int32_t passes, double* rho);
/* Copies the live particles of a species (2: the neutrals) in storage order: x_hat (dx units),
 * v (n x 3), id. */
int orc_particles(orc_sim* s, int species, double* x, double* v, uint64_t* id);
/* The null-collision countdown pairs (k | c << 12, R17; 0 for a species without the test) of the
 * live particles of a species, in the storage order of orc_particles. */
int orc_countdown(orc_sim* s, int species, uint32_t* nk);
/* Snapshot blob (format shared by specification with the GPU library, written separately). */
int orc_snapshot(orc_sim* s, void* buf, size_t cap, size_t* needed);
int orc_restore(orc_sim* s, const void* buf, size_t len);
uint64_t orc_config_hash(const orc_config* cfg);
/* OpenMP threads used by orc_step (1 = serial); returns the count in effect. */
int orc_set_threads(int n);

/* ---- adjoint of the collisionless step (pic_adjoint.c) ----------------------------------------
 * Frozen absorption schedule, observables J = (J_flux, J_fe) and parameters (V_left, T[0]) as the
 * header comment of pic_adjoint.c states.  Configurations: coll_mask 0, no source, T[0] > 0. */
#define ORC_ADJ_NEVER INT32_MAX
/* Node field of a charge density without wall bias, E = G rho, and its transpose rho_bar = G^T mu
 * (N + 1 nodes each). */
void orc_field_apply(int32_t N, double dx, const double* rho, double* E);
void orc_field_adjoint(int32_t N, double dx, const double* mu, double* rho_bar);
/* Particles of the model: electrons then ions, in load order. */
size_t orc_adj_particles(const orc_config* cfg);
/* Forward of `steps` steps.  replay == 0: records absorb[p] (the step at which particle p left
 * [0, N), ORC_ADJ_NEVER if it did not); replay != 0: absorbs particle p at step absorb[p].
 * J[0] = J_flux, J[1] = J_fe. */
int orc_adj_forward(const orc_config* cfg, int32_t steps, int replay, int32_t* absorb, double J[2]);
/* Recording forward, then the discrete adjoint: grad = d(w[0] J_flux + w[1] J_fe) / d(V_left, T[0]).
 * Also returns J and the recorded schedule. */
int orc_adj_gradient(const orc_config* cfg, int32_t steps, const double w[2], double grad[2], double J[2],
                     int32_t* absorb);
/* The same reverse sweep over a trajectory given by the caller instead of this oracle's own forward
 * (to hold another implementation's reverse sweep to this one on that implementation's recorded
 * forward): X[(steps+1) np] positions in cell units, V[(steps+1) 3 np] velocities, EN[(steps+1)(N+1)]
 * node fields (E^n: the field the push of step n uses; E^steps: the final field), absorb[np] the
 * schedule; particles electrons then ions in load order. */
int orc_adj_gradient_from_tape(const orc_config* cfg, int32_t steps, const double w[2], const double* X,
                               const double* V, const double* EN, const int32_t* absorb, double grad[2]);
/* The recording forward with its trajectory kept, in the layout orc_adj_gradient_from_tape takes. */
int orc_adj_trajectory(const orc_config* cfg, int32_t steps, double* X, double* V, double* EN, int32_t* absorb,
                       double J[2]);

#ifdef __cplusplus
}
#endif
#endif
