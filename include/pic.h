/*
 * pic.h -- C ABI of the GB300 (sm_103a) 1D3V electrostatic particle-in-cell Monte Carlo step.
 *
 * The operation is the PIC MC cycle of the paper (Sec. 2, "Background"): particle mover,
 * deposition of charge to the grid, field solve, interpolation of the field back to the
 * particles, and Monte Carlo collisions, for the bounded high-density sheath model of Table 3
 * (a magnetised plasma between two absorbing walls with a neutral background), advanced by
 * BIT1-style "natural sorting" of particles per cell (Sec. 2).  Optionally the D+/e/D sheath
 * physics of Table 3 and Sec. 2: ions recycled into tracked neutrals at the walls, electron-impact
 * ionization of those neutrals, and smoothing of the charge density before the field solve.  Checkpoint/restart semantics
 * (per-species particle records from which the run resumes exactly) follow Sec. 4.1.
 *
 * Conventions for every call:
 *  - Return value: PIC_OK (0) or one of the PIC_E* codes below; pic_strerror() names it.  No
 *    C++ exception leaves a call: a host allocation or host thread that fails inside one makes it
 *    return PIC_ENOMEM (a failed pic_init / pic_batch_init / pic_adj_init releases what it took).
 *  - A handle owns all device state of one simulation.  The caller owns every host buffer it
 *    passes.  No call is thread-safe on one handle; distinct handles are independent.
 *  - Work is enqueued on the CUDA stream given to pic_init (NULL = the legacy default stream).
 *    pic_step returns without waiting; device-side errors (capacity overflow, a bounded wait
 *    that gave up, a bounds check) surface at the next synchronising call: pic_diag,
 *    pic_snapshot, pic_get_field or pic_sync.
 *  - Units: lengths in Debye lengths, time in 1/omega_pe, m_e = e = eps0 = n0 = T_e = 1.
 *    Positions are kept cell-local: an int32 cell index and a fraction in [0, 1).
 */
#ifndef PIC_H
#define PIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PIC_ABI_VERSION 2u

/* status codes */
#define PIC_OK 0
#define PIC_EINVAL 1    /* invalid argument or configuration */
#define PIC_ENOMEM 2    /* device or host allocation failed, or workspace too small */
#define PIC_ECUDA 3     /* a CUDA runtime call failed */
#define PIC_EOVERFLOW 4 /* particle capacity exceeded (particles were dropped) */
#define PIC_ECORRUPT 5  /* snapshot blob: bad magic, version, checksum, size or config hash */
#define PIC_ETIMEOUT 6  /* a bounded device-side wait gave up */
#define PIC_EDEVICE 7   /* a device-side check failed (error flag set by a kernel) */

/* arithmetic of the particle path */
#define PIC_FP32 0u       /* FP32 particles and field, int64 fixed-point deposit, sorted */
#define PIC_FP64_PLAIN 1u /* FP64 particles, FP64 atomic deposit, unsorted (the plain baseline) */

/* collision processes (bit mask), Sec. 2 "MC collision handling" */
#define PIC_COLL_EL 1u /* electron-neutral elastic, constant cross section */
#define PIC_COLL_EX 2u /* electron-neutral excitation, linear above E_ex, saturating at 2 E_ex */
#define PIC_COLL_IZ 4u /* electron-impact ionization, linear above E_iz, saturating at 2 E_iz */
#define PIC_COLL_CX 8u /* ion-neutral charge exchange, constant cross section */

/* field modes */
#define PIC_FIELD_SELF 0u     /* self-consistent Poisson field */
#define PIC_FIELD_EXTERNAL 1u /* particles see a uniform E_x = E_ext (Poisson still solved) */
#define PIC_FIELD_ZERO 2u     /* particles see no electric field */

/* load profiles */
#define PIC_LOAD_UNIFORM 0    /* ppc particles per cell, uniformly random inside the cell */
#define PIC_LOAD_EXP 1        /* density ~ exp(-x/lambda), lambda = profile_scale (cells) */
#define PIC_LOAD_QUIET_SINE 2 /* evenly spaced; species 0 displaced by A sin(2 pi m x / L) */

/* particle sources */
#define PIC_SOURCE_NONE 0
#define PIC_SOURCE_PAIRS 1 /* each step, one (e, ion) pair per ion absorbed in that step,
                              uniform in [0, source_x1), Maxwellian at T[0], T[1] */

/* Configuration.  Plain old data; abi_version must be PIC_ABI_VERSION.  Species 0 are the
 * electrons (the only species that ionize, excite and scatter elastically); species 1 are the
 * ions (charge exchange).  Weight of a macro-particle: w_s = dx / ppc_s (n0 = 1).
 *
 * Sheath physics (all zero: off).  neutrals = 1 adds species 2, tracked neutrals with the ion's
 * mass and weight and no charge: neutral_ppc per cell at t = 0 (uniform in each cell, Maxwellian at
 * T_rec; ids 3 << 61 | i); an ion absorbed at a wall returns with probability `recycle` as a
 * neutral on that wall (x = 0, or the last FP32 fraction of the last cell), its v_x inward from the
 * flux-weighted half-Maxwellian at T_rec and v_y, v_z Maxwellian; neutrals move in straight lines
 * and are lost at either wall; a neutral inside ionizes with probability 1 - exp(-K_iz n_e(x) dt),
 * n_e(x) the CIC interpolation of the node electron density of the last deposit (half-cell volume
 * at the walls), becoming an ion (same position, velocity and id) beside a new electron, Maxwellian
 * at T_sec.  smooth_passes > 0 replaces the charge density, before the field solve, smooth_passes
 * times by (rho_{j-1} + 2 rho_j + rho_{j+1}) / 4 inside and (rho_0 + rho_1) / 2,
 * (rho_{N-1} + rho_N) / 2 at the walls (total charge kept); pic_get_field then returns the smoothed
 * rho and its phi.  Both need PIC_FP32 with integer charges |q| <= 64; neutrals need ion capacity
 * below 2^31.  Not available in ensembles (pic_batch_*) or in the adjoint (pic_adj_*). */
typedef struct pic_config {
  uint32_t abi_version;
  uint32_t precision;     /* PIC_FP32 or PIC_FP64_PLAIN */
  int32_t ncells;         /* N >= 2 cells, N + 1 nodes; N <= 196607 */
  int32_t ppc[2];         /* mean particles per cell per species (>= 1) */
  int32_t load_profile;   /* PIC_LOAD_* */
  int32_t profile_mode;   /* mode number m of PIC_LOAD_QUIET_SINE */
  int32_t source_mode;    /* PIC_SOURCE_* */
  int32_t sort_interval;  /* sort + compact after steps with step % sort_interval == 0 */
  uint32_t coll_mask;     /* PIC_COLL_* */
  uint32_t field_mode;    /* PIC_FIELD_* */
  uint32_t frozen_mask;   /* bit s set: species s is neither pushed nor collided */
  double L;               /* domain length; dx = L / N */
  double dt;              /* time step */
  double mass[2];         /* species masses */
  double charge[2];       /* species charges (nonzero) */
  double T[2];            /* initial temperatures */
  double Tg;              /* neutral gas temperature (new ions, charge exchange) */
  double m_gas;           /* neutral mass (elastic energy transfer 2 m / m_gas) */
  double B;               /* |B|, in units where the electron cyclotron frequency is |B| */
  double B_angle_deg;     /* angle of B to the wall normal x, B in the x-y plane */
  double V_left, V_right; /* wall potentials */
  double n_gas;           /* neutral density */
  double sigma_el;        /* elastic cross section */
  double sigma_ex, E_ex;  /* excitation cross-section scale and threshold */
  double sigma_iz, E_iz;  /* ionization cross-section scale and threshold */
  double sigma_cx;        /* charge-exchange cross section */
  double E_cap;           /* null-collision bound uses E_cap + |V_left - V_right| */
  double E_ext;           /* uniform field of PIC_FIELD_EXTERNAL */
  double profile_scale;   /* PIC_LOAD_EXP scale length / PIC_LOAD_QUIET_SINE amplitude (cells) */
  double source_x1;       /* end of the source region (cells), 0 < source_x1 <= N */
  double capacity_factor; /* particle buffer capacity per species = factor * ppc * N (>= 1) */
  uint64_t seed;          /* run seed (enters every Philox key and counter) */
  int32_t smooth_passes;  /* density smoothing passes before the field solve, 0 .. 4 */
  uint32_t neutrals;      /* 1: tracked neutrals (species 2), recycling, their ionization */
  int32_t neutral_ppc;    /* initial neutrals per cell (0 .. ; 0 when neutrals == 0) */
  uint32_t reserved;      /* 0 */
  double recycle;         /* probability that an absorbed ion returns as a neutral, [0, 1] */
  double T_rec;           /* temperature of recycled and initial neutrals */
  double K_iz;            /* rate coefficient of electron-impact ionization of a neutral */
  double T_sec;           /* temperature of the electron a neutral's ionization creates */
  double neutral_capacity; /* neutral buffer capacity = factor * max(neutral_ppc, ppc[1]) * N (>= 1) */
} pic_config;

/* Diagnostics (cumulative since pic_init unless stated). */
typedef struct pic_diag {
  uint64_t step;                 /* steps taken */
  uint64_t n[2];                 /* live particles per species (exact) */
  uint64_t wall_hits[2][2];      /* [species][0 = left, 1 = right] absorbed particles */
  uint64_t coll[5];              /* e elastic, e excitation, e ionization, ion CX, candidates */
  uint64_t near_threshold[2];    /* candidate draws within 1e-5 relative of a process boundary */
  uint64_t nu_max_violations[2]; /* candidates whose total collision frequency exceeded nu_max */
  uint64_t births[2];            /* particles created by ionization */
  uint64_t source_pairs;         /* pairs injected by the source */
  uint64_t dropped;              /* particles lost because a buffer was full */
  int64_t net_charge_units;      /* sum over nodes and species of sign(q) R, 2^-32 particle units */
  int64_t wall_charge;           /* sum over absorbed particles of sign(q) */
  double ke[2];                  /* sum of 0.5 m v^2 w over live particles (half step) */
  double field_energy;           /* sum_j 0.5 E_j^2 dx, half weight at the two walls */
  double wall_energy[2];         /* sum of 0.5 m v^2 w over absorbed particles */
  uint64_t particle_steps;       /* sum over steps of the live particles at the start of each
                                    step, since pic_init / pic_restore (the throughput unit) */
} pic_diag_t;

/* Tracked neutrals (cumulative since pic_init unless stated). */
typedef struct pic_neutral_diag {
  uint64_t n;                 /* live neutrals (exact) */
  uint64_t recycled[2];       /* neutrals created by recycling at [0 = left, 1 = right] wall */
  uint64_t lost[2];           /* neutrals absorbed at [left, right] wall */
  uint64_t ionized;           /* neutrals ionized (each became an ion beside a new electron) */
  uint64_t near_threshold;    /* ionization draws within 1e-5 relative of the probability */
  uint64_t particle_steps;    /* sum over steps of the live neutrals at the start of each step,
                                 since pic_init / pic_restore */
  double ke;                  /* sum of 0.5 m v^2 w over live neutrals */
} pic_neutral_diag_t;

typedef struct pic_handle pic_handle;

/* Bytes of device workspace that pic_init needs for cfg (capacity, sort buffers, grids): the
 * device-resident state of one run of the PIC MC cycle (Sec. 2), laid out as 1D contiguous
 * per-species arrays (the 1D layout of Sec. 5.2). */
int pic_workspace_size(const pic_config* cfg, size_t* bytes);

/* Create a simulation (Sec. 2, "Background": the set-up before the PIC MC cycle -- particle
 * load, first deposition, field solve and the "natural sorting" of particles per cell; Table 3:
 * the bounded plasma between two absorbing walls).  Validates cfg (PIC_EINVAL), carves the
 * caller's device workspace (256-byte aligned, >= pic_workspace_size bytes; it must outlive the
 * handle; PIC_ENOMEM if smaller) or, when workspace is NULL, allocates it with cudaMalloc (freed
 * by pic_free; PIC_ENOMEM on failure).  Loads the particles (Philox keyed by particle id),
 * deposits, solves the field and sorts.  cuda_stream is a cudaStream_t (NULL = default).
 * On success *out owns the state; on failure *out is NULL and nothing is left allocated. */
int pic_init(const pic_config* cfg, void* workspace, size_t workspace_bytes, void* cuda_stream,
             pic_handle** out);

/* Enqueue n >= 0 steps of the PIC MC cycle (Sec. 2, "Background": interpolation of the field to
 * the particles, particle mover, absorption at the walls of Table 3, MC collisions, deposition to
 * the grid, field solve; plus the per-cell counting sort and compaction -- BIT1's "natural
 * sorting", Sec. 2, the arranger of Sec. 5.1 -- on steps with step % sort_interval == 0).
 * Asynchronous on the handle's stream; PIC_EINVAL for n < 0 or a NULL handle, PIC_ECUDA if a
 * launch fails.  Device-side errors surface at the next synchronising call. */
int pic_step(pic_handle* h, int32_t n);

/* ---- particle decomposition of one simulation ------------------------------------------------
 *
 * The paper runs one simulation over many GPUs by MPI domain decomposition with particle load
 * balancing (Sec. 4.1, "Particle Load Balancing"; one rank per GPU).  These calls split one
 * simulation by particles instead: every part holds a subset of the particles over the whole grid
 * (its own handle, typically one per GPU), and the parts exchange one thing per step, their int64
 * node deposits, whose sum is exact and independent of the order of summation -- so a decomposed
 * run computes, particle for particle and bit for bit, what one handle holding every particle
 * computes.  Each part then solves the same field from the same total.  Per step:
 *     pic_step_begin(h, R_local);      // the particle phase; R_local = this part's node deposits
 *     R_total = sum over parts of R_local   (caller: an all-reduce of 2 (N+1) int64, e.g. NCCL)
 *     pic_step_end(h, R_total);        // field solve of R_total, bookkeeping, sort on sort steps
 * Set-up: pic_init (or pic_restore) with the same configuration on every part, pic_keep_subset,
 * then pic_local_deposit, the same all-reduce, and pic_solve_deposit.  Requirements: PIC_FP32,
 * integer charges (the exact solve), no pair source and no tracked neutrals (their new particles'
 * ids would not be unique across parts); else PIC_EINVAL.  R_local and R_total are device pointers
 * (caller-owned, 2 (N+1) int64 each: species 0 then species 1, 2^-32 particle units), used on the
 * handle's stream.  After a decomposed step the grid quantities (R, rho, phi, E, field energy, net
 * charge) are the whole simulation's; particle counts, counters and kinetic energies are this
 * part's (the parts' counters add up to the whole's).  Plain pic_step refuses a handle with an
 * open step (PIC_EINVAL). */

/* Keep the particles with id % nparts == part (0 <= part < nparts), drop the others, redeposit,
 * re-solve (this part's own deposit until pic_solve_deposit) and sort.  Part 0 keeps the cumulative
 * counters and sums; the other parts restart them from zero.  Synchronises the stream. */
int pic_keep_subset(pic_handle* h, uint32_t part, uint32_t nparts);

/* R_local = the node deposits of this part's particles as they stand (no step open). */
int pic_local_deposit(pic_handle* h, int64_t* R_local);

/* Replace the field by the solve of the deposits R_total (no step open); nothing else changes. */
int pic_solve_deposit(pic_handle* h, const int64_t* R_total);

/* The particle phase of one step (gather, push, walls, null-collision MC, deposit) and this part's
 * node deposits into R_local; the step stays open until pic_step_end. */
int pic_step_begin(pic_handle* h, int64_t* R_local);

/* Close the open step with the total deposits R_total: field solve, bookkeeping, sort scan on sort
 * steps; the step count advances.  PIC_EINVAL without an open step. */
int pic_step_end(pic_handle* h, const int64_t* R_total);

/* Kinetic-energy diagnostics (pic_diag_t.ke).  every > 0: the FP32 step kernel sums the kinetic
 * energy of the particles it leaves alive on every every-th step (counted from pic_init /
 * pic_restore), so that pic_diag right after such a step costs no extra pass; every == 0 (the
 * default): pic_diag sums it with one pass over the particles when asked.  Both use the same exact
 * 2^-24 fixed point and give the same bits.  The plain FP64 path always sums in pic_diag.
 * PIC_EINVAL for every < 0. */
int pic_set_diag_interval(pic_handle* h, int32_t every);

/* Wait for the stream and report device-side errors (PIC_EOVERFLOW, PIC_ETIMEOUT, PIC_EDEVICE):
 * the failure detection of this library (no counterpart in the paper beyond Sec. 4.1's
 * checkpoint/restart, from which a failed run resumes). */
int pic_sync(pic_handle* h);

/* Checkpoint (Sec. 4.1, "Checkpoint/Restart": per-species particle records -- cell, position,
 * velocity, id -- from which the run resumes; here an in-memory blob instead of an openPMD series).
 * Serialises the state into buf (host memory, owned by the caller, cap bytes).  buf == NULL: only
 * *needed is set, from the live counts (an upper bound after a neutral overflow); with buf,
 * *needed = the bytes written (PIC_EINVAL if cap is too small).  Accepts a state after
 * PIC_EOVERFLOW (it writes the particles that found a slot).
 * Version-1 blob, little-endian: "PICMCSN1", u32 version, u32 0, u64 config hash, u64 step,
 * u64 n[2], u64 counters[17], i64 wall_charge, f64 wall_energy[2], then per species
 * i32 cell[n], f64 frac[n], f64 vx[n], f64 vy[n], f64 vz[n], u64 id[n] in ascending id order,
 * then the CRC-32 (IEEE, as zlib) of all preceding bytes.  With neutrals the blob is version 2:
 * before the CRC come u64 n_neutral, u64 recycled[2], u64 lost[2], u64 ionized, u64 near and the
 * neutrals' records in the same layout.  Synchronises the stream. */
int pic_snapshot(pic_handle* h, void* buf, size_t cap, size_t* needed);

/* Restart (Sec. 4.1, "Checkpoint/Restart": the restore of a checkpoint, after which the run
 * continues; here bit-exactly, since every random draw is keyed by particle id and step).
 * Replaces the state by a blob from pic_snapshot (or any writer of the same format) made with
 * the same physics configuration (config hash), then redeposits, re-solves the field and sorts.
 * The blob is host memory owned by the caller and is checked entirely before any state changes.
 * PIC_ECORRUPT on any format error; PIC_EOVERFLOW if a species exceeds the capacity.
 * Positions and velocities are rounded to FP32 under PIC_FP32.  Synchronises the stream. */
int pic_restore(pic_handle* h, const void* buf, size_t len);

/* Diagnostics of the run (Sec. 2 and Table 2: BIT1's diagnostics of particle numbers, wall
 * fluxes and energies, taken every `datfile` steps there; here on request): particle counts,
 * wall hits, collision counts, charge and energies (pic_diag_t).  Reduces on the device, then
 * one read of the control block and one wait on the stream.  *out (host, caller-owned) is filled
 * only when the call returns PIC_OK (otherwise: the device-side error, PIC_EINVAL for NULL). */
int pic_diag(pic_handle* h, pic_diag_t* out);

/* Neutral diagnostics (PIC_EINVAL without neutrals); as pic_diag: one pass over the neutrals for
 * their kinetic energy, one read of the control block, one wait. */
int pic_neutral_diag(pic_handle* h, pic_neutral_diag_t* out);

/* Bytes one pic_diag copies from the device to the host (the control block of counters and
 * partial sums): the device-to-host traffic of reading the diagnostics. */
size_t pic_diag_bytes(void);

/* Diagnostics without a wait: enqueue pic_diag's reductions (what = PIC_DIAG_ALL; none for
 * PIC_DIAG_COUNTERS) and the copy of the control block into
 * host_buf (pic_diag_bytes() bytes, owned by the caller; pinned memory keeps the copy asynchronous)
 * on the handle's stream, and return.  Once the stream has passed that point (an event, a sync),
 * pic_diag_decode turns the bytes into *out, as pic_diag would have at the call: the step count,
 * counters and sums of the state after the steps enqueued before it, and the device-side error word
 * (its status is returned, *out untouched, when an error was set).  Steps may be enqueued in between:
 * reading step k's diagnostics while step k + 1 runs keeps the GPU busy. */
#define PIC_DIAG_ALL 0u            /* every field of pic_diag_t */
#define PIC_DIAG_COUNTERS 1u       /* counters, particle_steps and the error word only: no reduction
                                      runs; ke, field_energy and net_charge_units read 0 */
int pic_diag_async(pic_handle* h, void* host_buf, uint32_t what);
int pic_diag_decode(const pic_handle* h, const void* host_buf, pic_diag_t* out);

/* The grid quantities of the PIC cycle (Sec. 2: "deposition to the grid" and the "field
 * solver"): copies them to host buffers (caller-owned) of nnodes = N + 1 entries each (any may be
 * NULL): R: 2 x (N+1) int64 deposits (species 0 then 1, 2^-32 particle units), rho, phi: FP64,
 * E: FP32 node field as seen by the particles.  PIC_EINVAL if nnodes != N + 1.  Synchronises the
 * stream and reports device-side errors first. */
int pic_get_field(pic_handle* h, int64_t* R, double* rho, double* phi, float* E, size_t nnodes);

/* The storage order of one charged species (species 0 or 1): the arranger's output (Sec. 2,
 * BIT1's "natural sorting"; the arranger of Sec. 5.1), for checking it.  Copies, for every slot of
 * the particle buffer the next step reads, in storage order, the cell index (INT32_MIN marks a dead
 * slot: a particle absorbed since the last sort, or padding) and, where ids != NULL, the particle
 * id (meaningless in a dead slot) into host buffers of cap entries; *n = the buffer's extent (a
 * multiple of 4, dead slots included).  cell == NULL and ids == NULL: only *n.  PIC_EINVAL for the
 * plain FP64 path (it keeps no cell order) or a species outside {0, 1}; PIC_ENOMEM if cap < *n.
 * After the full sort of pic_init / pic_restore the live slots come first, in non-decreasing cell
 * order; after the step that follows a sort step, slot blocks follow the cells the particles held
 * when that step began, with dead slots where particles were absorbed in it and that step's births
 * after the blocks.  Synchronises the stream and reports device-side errors first. */
int pic_storage_order(pic_handle* h, int32_t species, int32_t* cell, uint64_t* ids, size_t cap, size_t* n);

/* Per-kernel device time via CUDA events on the handle's stream.  enable != 0 starts recording
 * (adds two event records per launch); pic_kernel_times synchronises and returns, for up to
 * nkinds kernel kinds, total milliseconds, launch counts and names. */
#define PIC_KERNEL_KINDS 10
int pic_profile(pic_handle* h, int enable);
int pic_kernel_times(pic_handle* h, double* ms, uint64_t* launches, const char** names,
                     int32_t nkinds);

/* Destroy the handle (synchronises; frees what pic_init allocated). */
void pic_free(pic_handle* h);

const char* pic_strerror(int status);

/* CRC-32 (IEEE 802.3, reflected polynomial 0xEDB88320, initial and final complement: zlib's
 * crc32) of n bytes of host memory at p, the checksum that closes a snapshot blob (pic_snapshot,
 * Sec. 4.1 checkpointing).  Writers of the blob format can use it for the last four bytes.  Pure
 * host code on the calling thread and up to 64 helper threads; no device or handle is needed.
 * p may be NULL only when n == 0 (the CRC of no bytes is 0). */
uint32_t pic_blob_crc32(const void* p, size_t n);

/* Self-test of the device-side wait limit (failure detection without a fault): launches one
 * thread that waits on an mbarrier phase which can never complete (two arrivals expected, one
 * made).  The wait gives up after its limit (about one second of wall time), records it and
 * returns, leaving the context usable.  Returns PIC_ETIMEOUT when the limit worked as designed (the
 * wait's duration in *seconds, may be NULL), PIC_ECUDA or PIC_ENOMEM on a runtime failure.  Every
 * bounded wait of the particle kernels (the TMA stage barriers) uses the same limit and reports
 * PIC_ETIMEOUT at the next synchronising call. */
int pic_selftest_timeout(void* cuda_stream, double* seconds);

/* ---- single operations, on caller-owned device buffers ------------------------------------ */

/* Philox4x32-10 (Salmon et al., SC'11; the generator of the MC draws): out[4i..4i+3] =
 * Philox(ctr[4i..4i+3], key[2i..2i+1]) for i < n.  Device pointers; asynchronous on stream. */
int pic_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, size_t n,
               void* cuda_stream);

/* Field solve of the PIC cycle (Sec. 2 "field solver"): the interior problem
 * -phi_{j-1} + 2 phi_j - phi_{j+1} = dx^2 rho_j, phi_0 = V_L, phi_N = V_R, solved exactly by
 * the discrete Green's function (two prefix scans in FP64), then E_j = (phi_{j-1}-phi_{j+1})/2dx
 * inside and Gauss's law over the half cell at each wall.  rho, phi, E: N + 1 FP64 device
 * values.  Needs no workspace; 2 <= N <= 196607.  Asynchronous on stream. */
int pic_poisson(const double* rho, int32_t ncells, double dx, double V_L, double V_R,
                double* phi, double* E, void* cuda_stream);

/* ---- ensembles: many independent simulations advanced together ------------------------------
 *
 * A batch holds nsims independent simulations (a parameter scan, the seeds of one study) and
 * advances all of them by one step with one persistent launch of the particle step over every
 * simulation's particles -- their uneven particle counts split evenly over the GPU, as the
 * particle load balancing of Sec. 4.1 ("Particle Load Balancing") splits uneven particle
 * distributions over MPI ranks --, one launch of the field solve (one thread-block cluster per
 * simulation) and, on sort steps, the per-cell counting sort's scans (the next step's launch moves
 * the particles).  Repeated steps replay a captured CUDA graph of 2 * sort_interval steps.
 * Each simulation computes exactly what pic_init + pic_step compute for
 * its own configuration: the same random draws, the same int64 deposit, the same field, the same
 * particle set; the batch changes only how the work is laid out on the GPU.
 *
 * What may differ between the simulations of a batch: ncells (and L with it), ppc, the initial
 * load (profile, T), the collision set and every collision parameter (n_gas, sigma_*, E_*, E_cap,
 * Tg, m_gas), the wall potentials, capacity_factor and the seed.  What they must share: dt, the
 * cell size L / ncells, B and its angle, the species masses and charges, frozen_mask, field_mode,
 * E_ext and sort_interval.  Every simulation must use PIC_FP32, PIC_SOURCE_NONE, integer
 * species charges (the integer-exact field solve) and none of the sheath physics (neutrals 0,
 * smooth_passes 0); 1 <= nsims <= PIC_BATCH_MAX_SIMS; the
 * particle capacities of each species together below 2^31.  Anything else: PIC_EINVAL.
 *
 * Conventions are those of the single-simulation calls: the caller owns host buffers, work runs on
 * the stream given to pic_batch_init, device errors surface at the next synchronising call.
 * Simulation k of a batch is addressed by its index 0 <= k < nsims. */
#define PIC_BATCH_MAX_SIMS 4096

typedef struct pic_batch pic_batch;

/* Launch configuration of the batch step; results do not depend on it. */
typedef struct pic_batch_tuning {
  int32_t variant;          /* shape of the particle-step kernel, 0 .. pic_batch_variant_count()-1 */
  int32_t ctas_per_sm;      /* resident CTAs per SM of the particle step; 0 = as many as fit */
  int32_t use_graph;        /* nonzero: replay CUDA graphs of 2 * sort_interval steps */
} pic_batch_tuning;

/* Number of compiled shapes of the batch particle-step kernel, and the name of shape v
 * ("tpb<threads per CTA>_minb<CTAs per SM>_stages<TMA stages per warp>"; NULL if out of range). */
int32_t pic_batch_variant_count(void);
const char* pic_batch_variant_name(int32_t v);

/* Bytes of device workspace that pic_batch_init needs for these configurations. */
int pic_batch_workspace_size(const pic_config* cfgs, int32_t nsims, size_t* bytes);

/* Create a batch from nsims configurations (host array; copied): as pic_workspace_size /
 * pic_init, with workspace NULL meaning cudaMalloc.  Loads every simulation as pic_init would,
 * then plans the first step.  The default tuning is shape 0, all CTAs that fit, graphs on. */
int pic_batch_init(const pic_config* cfgs, int32_t nsims, void* workspace, size_t workspace_bytes,
                   void* cuda_stream, pic_batch** out);

/* Set / read the launch configuration (PIC_EINVAL for an unknown shape or a CTA count beyond
 * what fits on an SM).  Setting drops captured graphs. */
int pic_batch_set_tuning(pic_batch* b, const pic_batch_tuning* t);
int pic_batch_get_tuning(pic_batch* b, pic_batch_tuning* t);

/* Kinetic-energy diagnostics of a batch: every == 1 sums them inside every batch step (pic_batch_diag
 * after a step costs no extra pass); every == 0 (the default) sums them in pic_batch_diag, one pass
 * per simulation.  Same bits either way.  Other values: PIC_EINVAL.  Drops captured graphs. */
int pic_batch_set_diag_interval(pic_batch* b, int32_t every);

/* Enqueue n >= 0 steps of every simulation (asynchronous on the batch's stream). */
int pic_batch_step(pic_batch* b, int32_t n);

/* Wait for the stream; report device-side errors of any simulation. */
int pic_batch_sync(pic_batch* b);

/* Diagnostics of simulations 0 .. nsims-1 into out[0 .. nsims-1] (as pic_diag). */
int pic_batch_diag(pic_batch* b, pic_diag_t* out, int32_t nsims);

/* Snapshot of simulation k, in pic_snapshot's format: the blob restores into a single handle made
 * from the same configuration, and vice versa. */
int pic_batch_snapshot(pic_batch* b, int32_t k, void* buf, size_t cap, size_t* needed);

/* Replace the state of every simulation: blobs[k] (lens[k] bytes) for simulation k, each made
 * with simulation k's configuration, all at the same step (which becomes the batch's step).
 * Checks every blob before changing any state (PIC_ECORRUPT, PIC_EOVERFLOW as pic_restore). */
int pic_batch_restore(pic_batch* b, const void* const* blobs, const size_t* lens);

/* Back to the state pic_batch_init made (every simulation reloaded, step 0). */
int pic_batch_reset(pic_batch* b);

/* Grid of simulation k (as pic_get_field; nnodes = its ncells + 1). */
int pic_batch_get_field(pic_batch* b, int32_t k, int64_t* R, double* rho, double* phi, float* E,
                        size_t nnodes);

/* Storage order of species s of simulation k (as pic_storage_order; the arranger's output for
 * that simulation, inside its segment of the batch's arrays). */
int pic_batch_storage_order(pic_batch* b, int32_t k, int32_t species, int32_t* cell, uint64_t* ids,
                            size_t cap, size_t* n);

/* Per-kernel device time (as pic_profile / pic_kernel_times; kinds "step", "field", "sort",
 * "plan").  While profiling, steps are launched one by one (no graphs). */
int pic_batch_profile(pic_batch* b, int enable);
int pic_batch_kernel_times(pic_batch* b, double* ms, uint64_t* launches, const char** names,
                           int32_t nkinds);

/* Destroy the batch (synchronises; frees what pic_batch_init allocated). */
void pic_batch_free(pic_batch* b);

/* ---- gradients: the adjoint of the collisionless step -------------------------------------------
 *
 * The paper computes no gradients; these calls differentiate its collisionless step (Sec. 2:
 * gather, Boris push, deposit, field solve; collisions off) by a hand-written discrete adjoint.
 * Model (one handle = one configuration, `steps` steps; FP32 particles, signed int64 fixed-point
 * deposit, FP64 field; the adjoint accumulates in FP64):
 *  - absorption at the walls is taken as a fixed schedule: a recording forward absorbs a particle at
 *    the first step its position leaves [0, L) and stores that step; a replaying forward absorbs
 *    each particle at its recorded step whatever its position (until then a particle outside
 *    [0, L) keeps the linear extension of its boundary cell's CIC weights), so that finite
 *    differences of the replaying forward approximate what the adjoint differentiates;
 *  - J[0] = J_flux = sum over steps n of dt * sum over electrons alive after step n of
 *    w v_x S(x - (L - dx)), S(d) = max(0, 1 - |d|/dx): the CIC share of the last interior node, a
 *    smooth measure of the electron flux into the right wall;
 *    J[1] = J_fe = sum_j c_j E_j^2 dx / 2 of the final node field (c_j = 1/2 at the walls);
 *  - parameters: V_left (the right wall keeps cfg->V_right) and the initial electron temperature
 *    T_e, which scales the loaded electron velocities, v = sqrt(T_e / m) xi, with the draws xi fixed.
 * The adjoint stores the particle state every `checkpoint_every` steps and the node field of every
 * step during a recording forward, and recomputes each segment of checkpoint_every steps from its
 * checkpoint during the reverse sweep (memory: about (steps / checkpoint_every + checkpoint_every)
 * x 20 bytes per particle).  Configurations: coll_mask 0, PIC_SOURCE_NONE, T[0] > 0, no sheath
 * physics (neutrals 0, smooth_passes 0) (precision
 * and sort_interval are ignored); 1 <= checkpoint_every <= steps.  Work runs on cuda_stream; the
 * forward and gradient calls synchronise it. */
typedef struct pic_adj pic_adj;

int pic_adj_workspace_size(const pic_config* cfg, int32_t steps, int32_t checkpoint_every, size_t* bytes);

/* Create the handle (workspace as pic_init: caller's, 256-byte aligned, or NULL = cudaMalloc). */
int pic_adj_init(const pic_config* cfg, int32_t steps, int32_t checkpoint_every, void* workspace,
                 size_t workspace_bytes, void* cuda_stream, pic_adj** out);

/* Load with V_left and T_e, run the steps; J[0] = J_flux, J[1] = J_fe (host).  replay == 0 records
 * the schedule and the checkpoints (the point pic_adj_gradient differentiates at); replay != 0
 * reuses the last recorded schedule (PIC_EINVAL if there is none) and keeps the recording. */
int pic_adj_forward(pic_adj* a, double V_left, double T_e, int32_t replay, double J[2]);

/* grad = d(w[0] J_flux + w[1] J_fe) / d(V_left, T_e) at the last recording forward (host arrays):
 * one reverse sweep per weight vector (a vector-Jacobian product). */
int pic_adj_gradient(pic_adj* a, const double w[2], double grad[2]);

/* The recorded schedule: absorb[p] = step at which particle p was absorbed (INT32_MAX: never),
 * electrons then ions in load order; n must be the particle count. */
int pic_adj_schedule(pic_adj* a, int32_t* absorb, size_t n);

/* The tape of the last recording forward, for checking the reverse sweep against another
 * implementation's on the same trajectory: the FP32 particle state after n steps (0 <= n <= steps;
 * electrons then ions in load order, np = the particle count: cell, fraction, v; a particle absorbed
 * before step n holds whatever state it was absorbed with) and E^n, the FP64 node field the push of
 * step n uses (E^steps: the final field; nnodes = N + 1).  Any output may be NULL; host buffers owned
 * by the caller.  The state is recomputed from its checkpoint with the recorded fields (the same
 * kernel and inputs, hence the same bits as during the recording).  PIC_EINVAL before a recording
 * forward, for n outside [0, steps] or wrong sizes.  Synchronises the stream. */
int pic_adj_tape(pic_adj* a, int32_t n, int32_t* cell, float* frac, float* vx, float* vy, float* vz, double* E,
                 size_t np, size_t nnodes);

/* Device time of the last forward and the last gradient (CUDA events on the handle's stream). */
int pic_adj_times(pic_adj* a, double* forward_ms, double* gradient_ms);

void pic_adj_free(pic_adj* a);

/* ---- allocation-free entry point ------------------------------------------------------------ */

/* The paper has no counterpart to this call: it exists for callers that cannot allocate device
 * memory (code confined to another framework's fixed memory pool, code that must not allocate
 * after start-up, hosts that only hand over their own buffers).  It computes what pic_restore +
 * pic_get_field compute for a particle state -- the int64 CIC deposit of each species and the
 * node field of the integer-exact Poisson solve -- without any cudaMalloc, cudaFree or
 * allocating library call.  Its scratch (per-cell counts and weight sums, about 2 MB) is one
 * fixed array in device memory that every GPU which loads this library keeps until the process
 * exits; the first call on each device looks up that array's device address (make that first
 * call before any stream capture).  Limits: 2 <= cfg->ncells <= PIC_NOALLOC_MAX_CELLS (larger
 * grids return PIC_EINVAL), integer charges |q| <= 64, ppc ratio as in pic_init's exact solve,
 * 0 <= cfg->smooth_passes <= 4 (the density smoothing of the step's own solve is applied to E; R
 * stays the unsmoothed deposit).
 * Inputs (device, caller-owned): per species s the cell indices (int32) and fractions (FP32) of
 * n_s particles; entries with a cell outside [0, N) or a fraction outside [0, 1) are skipped.
 * Outputs (device, caller-owned): R, 2 x (N+1) int64 node deposits (species 0 then 1, 2^-32
 * particle units); E, N+1 FP64 node field.  The call runs on cuda_stream and synchronises it
 * before returning (PIC_EDEVICE if a device-side check failed).  All calls share the one scratch
 * array and each clears it first: calls that overlap on the GPU (other streams, other host
 * threads) race on it and must be serialised by the caller. */
#define PIC_NOALLOC_MAX_CELLS 65536
int pic_field_noalloc(const pic_config* cfg, const int32_t* cell0, const float* frac0, uint64_t n0,
                      const int32_t* cell1, const float* frac1, uint64_t n1, int64_t* R, double* E,
                      void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif
