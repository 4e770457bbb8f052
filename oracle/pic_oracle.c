/*
 * pic_oracle.c -- plain FP64 CPU oracle of the 1D3V electrostatic PIC Monte Carlo step.
 *
 * TEST INFRASTRUCTURE ONLY (see pic_oracle.h).  Slow and plain on purpose: one loop per stage of
 * the PIC cycle in the order the paper lists it (Sec. 2), FP64 throughout, the Poisson problem
 * solved by the Thomas algorithm, sorting as a textbook stable counting sort.
 *
 * Readings of points the paper leaves open (the paper prints no formulas; its method statement is
 * the PIC MC cycle of Sec. 2 and the BIT1 lineage, XPDP1 with "natural sorting"):
 *   R1  leapfrog start: loaded velocities are v^{-1/2}; no backward half push.
 *   R2  step order: gather -> Boris push -> wall test -> MCC on survivors -> deposit (births
 *       included) -> source -> Poisson -> sort when step % sort_interval == 0 -> step += 1.
 *   R3  absorbed iff x < 0 or x >= L.
 *   R4  wall nodes use half-cell volume; wall field from Gauss's law over the half cell.
 *   R7  cross sections: constant elastic and CX; excitation/ionization linear above threshold,
 *       saturating at twice the threshold.
 *   R8  null-collision bound nu_max = n_g * sum(sigma_max) * v_cap, v_cap = sqrt(2 E_cap'/m),
 *       E_cap' = E_cap + |V_L - V_R|; rounded to FP32 and shared by both codes by value.
 *   R9  Philox4x32-10: key (step lo, seed lo), counter (id lo, id hi, channel | step hi << 8,
 *       index ^ seed hi); uniform u = (word >> 8) * 2^-24.
 *   R10 isotropic scattering; elastic energy loss 2m/M (1 - cos chi); excitation loses E_ex;
 *       ionization splits E - E_iz uniformly; new ion and CX ion Maxwellian at T_g.
 *   R11 child ids are Philox words of (parent id, step, CHILD channel).
 *   R12 CIC deposit in int64 fixed point: W_r = rint(f 2^32), W_l = 2^32 - W_r.
 *   R13 source: one (e, ion) pair per ion absorbed this step, uniform in [0, x1), Maxwellian.
 *   R17 null-collision candidates by geometric countdown (replaces a Bernoulli(P_null) draw per
 *       particle and step; the same process in law, since P_null is constant per species): a
 *       particle of a species that takes the test (collisions on, not frozen, P_null > 0) carries
 *       a countdown k in 1..4095 and a flag c.  G(w), from one Philox word w: u = (w >> 8) 2^-24,
 *       r = log(1 - u) / log1p(-P_null) in FP64, K = 1 + floor(r); (k, c) = (K, 1) if K <= 4095,
 *       else (4095, 0).  A particle created at step s (the load at s = 0, births, source pairs, the
 *       products of a neutral's ionization) takes G(word 0 of Philox(id, s, INIT, 2)).  In each
 *       step in which it is pushed and stays inside, k -= 1; at k = 0 it is a candidate when
 *       c = 1, and in either case takes G(word 0 of Philox(id, step, COLL, 0)), whose words 1..3
 *       the collision uses as before.  A draw with r within 1e-9 max(1, r) of an integer is
 *       counted as near-threshold.  In a snapshot the pair rides in bits 18..30 of the cell word
 *       (cell | k << 18 | c << 30; 0 there means "not drawn": the restore draws it as at creation
 *       at the blob's step).
 *
 * The D+/e/D sheath physics (Table 3: D+ ions recycled into D neutrals at the walls; Sec. 2:
 * density smoothing), all off unless the configuration asks for it:
 *   N1  species 2 are tracked neutrals of the ion's mass and weight, charge 0; at t = 0 either
 *       none or neutral_ppc per cell, loaded like a uniform species at T_rec (ids 3 << 61 | i).
 *   N2  an ion absorbed at a wall returns as a neutral with probability `recycle`, at that wall
 *       (x = 0, or x = N - 2^-24 cells), v_x inward from the flux-weighted half-Maxwellian at
 *       T_rec (|v_x| = v_t sqrt(-2 ln(1 - u))), v_y, v_z Maxwellian; it moves from the next step.
 *   N3  neutrals move ballistically and are lost at either wall (x < 0 or x >= L).
 *   N4  a neutral left inside ionizes with P = 1 - exp(-K_iz n_e(x) dt), n_e(x) the CIC
 *       interpolation of the node electron density of the start-of-step deposit (half volume at
 *       the walls, not smoothed); it becomes an ion (same x, v, id) and an electron is born at x,
 *       Maxwellian at T_sec.  No electron loses the ionization energy (test-particle reading).
 *   N5  step order: charged species (R2; recycling at the ion wall test), then the neutrals alive
 *       at the step start, then births are appended, source, deposit, smoothing, Poisson, sort.
 *   N6  smoothing: passes of rho'_j = (rho_{j-1} + 2 rho_j + rho_{j+1}) / 4 inside and
 *       rho'_0 = (rho_0 + rho_1) / 2, rho'_N = (rho_{N-1} + rho_N) / 2 at the walls (with the
 *       half-cell wall volume this keeps the total charge and a uniform density).
 */
#include "pic_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define TWO32 4294967296.0
#define NEXT_KMAX 4095u        /* largest countdown (R17) */
#define NEXT_CAND (1u << 12)   /* flag: the expiry is a null-collision candidate */
#define CELL_BITS 18           /* the snapshot's cell word: cell | next << CELL_BITS */
#define ORC_PI 3.14159265358979323846
#define MAX_THREADS 256

static int g_threads = 1;

int orc_set_threads(int n) {
#ifdef _OPENMP
  if (n < 1) n = 1;
  if (n > MAX_THREADS) n = MAX_THREADS;
  g_threads = n;
#else
  (void)n;
  g_threads = 1;
#endif
  return g_threads;
}

/* ------------------------------------------------------------------------------------------ */
/* Philox4x32-10: ten rounds of two 32x32->64 multiplies, with the key bumped by the Weyl
 * constants between rounds (Salmon et al., SC'11, Sec. 4).                                      */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)p1;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)p0;
    c0 = n0;
    c1 = n1;
    c2 = n2;
    c3 = n3;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

void orc_philox_batch(size_t n, const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
  for (size_t i = 0; i < n; ++i) orc_philox4x32_10(ctr + 4 * i, key + 2 * i, out + 4 * i);
}

/* uniform in [0,1) with 24 bits: exact in both FP32 and FP64 (R9) */
static double u01(uint32_t w) { return (double)(w >> 8) * (1.0 / 16777216.0); }

/* One Philox block for (particle id, step, channel, index) under the run's seed (R9): the key is
 * (step, seed) and the counter (id, channel, index), with the high halves of step and seed folded
 * into the counter, so that distinct (id, step, channel, index) give distinct (key, counter). */
static void draw(uint64_t id, uint64_t seed, uint64_t step, uint32_t channel, uint32_t index,
                 uint32_t w[4]) {
  uint32_t key[2] = {(uint32_t)step, (uint32_t)seed};
  uint32_t ctr[4] = {(uint32_t)id, (uint32_t)(id >> 32), channel | ((uint32_t)(step >> 32) << 8),
                     index ^ (uint32_t)(seed >> 32)};
  orc_philox4x32_10(ctr, key, w);
}

/* Box-Muller: two standard normals from two uniforms. */
static void box_muller(uint32_t wa, uint32_t wb, double* n0, double* n1) {
  double r = sqrt(-2.0 * log(1.0 - u01(wa)));
  double th = 2.0 * ORC_PI * u01(wb);
  *n0 = r * cos(th);
  *n1 = r * sin(th);
}

/* direction uniform on the unit sphere: cos(theta) = 1 - 2u, phi = 2 pi u' (R10) */
static void iso_dir(uint32_t wa, uint32_t wb, double d[3]) {
  double ua = u01(wa), ub = u01(wb);
  double ct = 1.0 - 2.0 * ua;
  double st = 2.0 * sqrt(ua * (1.0 - ua));
  double ph = 2.0 * ORC_PI * ub;
  d[0] = st * cos(ph);
  d[1] = st * sin(ph);
  d[2] = ct;
}

/* ------------------------------------------------------------------------------------------ */
/* Field solve (Sec. 2 "field solver"; BIT1's native Poisson solver, Sec. 2).                    */
int orc_poisson_thomas(int32_t N, double dx, const double* rho, double V_L, double V_R,
                       double* phi) {
  if (N < 2) return ORC_EINVAL;
  int32_t m = N - 1; /* unknowns phi_1 .. phi_{N-1} */
  double* cp = (double*)malloc(sizeof(double) * (size_t)(m + 1));
  double* dp = (double*)malloc(sizeof(double) * (size_t)(m + 1));
  if (!cp || !dp) {
    free(cp);
    free(dp);
    return ORC_ENOMEM;
  }
  /* a_j = -1, b_j = 2, c_j = -1; right-hand side with the Dirichlet values moved over */
  for (int32_t j = 1; j <= m; ++j) {
    double d = dx * dx * rho[j]; /* eps0 = 1 */
    if (j == 1) d += V_L;
    if (j == m) d += V_R;
    if (j == 1) {
      cp[j] = -1.0 / 2.0;
      dp[j] = d / 2.0;
    } else {
      double den = 2.0 - (-1.0) * cp[j - 1];
      cp[j] = -1.0 / den;
      dp[j] = (d - (-1.0) * dp[j - 1]) / den;
    }
  }
  phi[0] = V_L;
  phi[N] = V_R;
  phi[m] = dp[m];
  for (int32_t j = m - 1; j >= 1; --j) phi[j] = dp[j] - cp[j] * phi[j + 1];
  free(cp);
  free(dp);
  return ORC_OK;
}

void orc_efield(int32_t N, double dx, const double* phi, const double* rho, double* E) {
  for (int32_t j = 1; j < N; ++j) E[j] = (phi[j - 1] - phi[j + 1]) / (2.0 * dx);
  /* Gauss over [0, dx/2] and [L - dx/2, L] (R4) */
  E[0] = (phi[0] - phi[1]) / dx - rho[0] * dx / 2.0;
  E[N] = (phi[N - 1] - phi[N]) / dx + rho[N] * dx / 2.0;
}

/* ------------------------------------------------------------------------------------------ */
/* Boris rotation for a uniform B (the magnetised mover; Sec. 5.1 names it moveb).              */
void orc_boris(double qm, double dt, const double E[3], const double B[3], double v[3]) {
  double h = 0.5 * qm * dt;
  double vm[3] = {v[0] + h * E[0], v[1] + h * E[1], v[2] + h * E[2]};
  double t[3] = {h * B[0], h * B[1], h * B[2]};
  double t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
  double s[3] = {2.0 * t[0] / (1.0 + t2), 2.0 * t[1] / (1.0 + t2), 2.0 * t[2] / (1.0 + t2)};
  double vp[3] = {vm[0] + (vm[1] * t[2] - vm[2] * t[1]), vm[1] + (vm[2] * t[0] - vm[0] * t[2]),
                  vm[2] + (vm[0] * t[1] - vm[1] * t[0])};
  double vq[3] = {vm[0] + (vp[1] * s[2] - vp[2] * s[1]), vm[1] + (vp[2] * s[0] - vp[0] * s[2]),
                  vm[2] + (vp[0] * s[1] - vp[1] * s[0])};
  v[0] = vq[0] + h * E[0];
  v[1] = vq[1] + h * E[1];
  v[2] = vq[2] + h * E[2];
}

/* ------------------------------------------------------------------------------------------ */
void orc_nu_max(const orc_config* c, float nu_max[2], float p_null[2]) {
  double Ecap = c->E_cap + fabs(c->V_left - c->V_right);
  double smax[2];
  smax[0] = ((c->coll_mask & ORC_COLL_EL) ? c->sigma_el : 0.0) +
            ((c->coll_mask & ORC_COLL_EX) ? c->sigma_ex : 0.0) +
            ((c->coll_mask & ORC_COLL_IZ) ? c->sigma_iz : 0.0);
  smax[1] = (c->coll_mask & ORC_COLL_CX) ? c->sigma_cx : 0.0;
  for (int s = 0; s < 2; ++s) {
    double vcap = sqrt(2.0 * Ecap / c->mass[s]);
    nu_max[s] = (float)(c->n_gas * smax[s] * vcap);
    p_null[s] = (float)(1.0 - exp(-(double)nu_max[s] * c->dt));
  }
}

/* ------------------------------------------------------------------------------------------ */
typedef struct {
  double *x, *vx, *vy, *vz;
  uint64_t* id;
  uint32_t* nk; /* R17: countdown k | flag c << 12 (0: the species takes no null-collision test) */
  size_t n, cap;
} orc_species;

typedef struct {
  uint64_t wall_hits[2];
  uint64_t coll[5];
  uint64_t near, viol;
  uint64_t recycled[2]; /* ions that returned as neutrals, per wall (N2) */
} orc_tcount;

typedef struct {
  double x, v[3];
  uint64_t id;
} orc_newp;

typedef struct {
  orc_newp* p;
  size_t n, cap;
} orc_plist;

struct orc_sim {
  orc_config cfg;
  int32_t N;
  double dx, w[2], qm[2], Bv[3];
  float nu_max[2], p_null[2];
  int mcc[2]; /* species s takes the null-collision test (R17) */
  orc_species sp[2];
  orc_species nt; /* tracked neutrals (N1) */
  int64_t* R[2];
  double *rho, *phi, *E;
  double* ne; /* node electron density of the last deposit (N4) */
  uint64_t nt_recycled[2], nt_lost[2], nt_ionized, nt_near, nt_particle_steps;
  uint64_t step;
  uint64_t wall_hits[2][2], coll[5], near[2], viol[2], births[2], source_pairs;
  int64_t wall_charge;
  double wall_energy[2];
  uint64_t particle_steps;
};

static int sp_reserve(orc_species* s, size_t cap) {
  if (cap <= s->cap) return ORC_OK;
  size_t nc = s->cap ? s->cap : 16;
  while (nc < cap) nc *= 2;
  double* x = (double*)realloc(s->x, nc * sizeof(double));
  if (x) s->x = x;
  double* a = (double*)realloc(s->vx, nc * sizeof(double));
  if (a) s->vx = a;
  double* b = (double*)realloc(s->vy, nc * sizeof(double));
  if (b) s->vy = b;
  double* c = (double*)realloc(s->vz, nc * sizeof(double));
  if (c) s->vz = c;
  uint64_t* d = (uint64_t*)realloc(s->id, nc * sizeof(uint64_t));
  if (d) s->id = d;
  uint32_t* e = (uint32_t*)realloc(s->nk, nc * sizeof(uint32_t));
  if (e) s->nk = e;
  if (!x || !a || !b || !c || !d || !e) return ORC_ENOMEM;
  s->cap = nc;
  return ORC_OK;
}

static int sp_push_back(orc_species* s, double x, const double v[3], uint64_t id, uint32_t nk) {
  if (s->n == s->cap && sp_reserve(s, s->n + 1) != ORC_OK) return ORC_ENOMEM;
  s->x[s->n] = x;
  s->vx[s->n] = v[0];
  s->vy[s->n] = v[1];
  s->vz[s->n] = v[2];
  s->id[s->n] = id;
  s->nk[s->n] = nk;
  s->n++;
  return ORC_OK;
}

static int plist_add(orc_plist* l, double x, const double v[3], uint64_t id) {
  if (l->n == l->cap) {
    size_t nc = l->cap ? 2 * l->cap : 64;
    orc_newp* p = (orc_newp*)realloc(l->p, nc * sizeof(orc_newp));
    if (!p) return ORC_ENOMEM;
    l->p = p;
    l->cap = nc;
  }
  l->p[l->n].x = x;
  l->p[l->n].v[0] = v[0];
  l->p[l->n].v[1] = v[1];
  l->p[l->n].v[2] = v[2];
  l->p[l->n].id = id;
  l->n++;
  return ORC_OK;
}

static int valid_config(const orc_config* c) {
  if (c->ncells < 2 || !(c->L > 0) || !(c->dt > 0)) return 0;
  for (int s = 0; s < 2; ++s) {
    if (c->ppc[s] < 1 || !(c->mass[s] > 0) || c->T[s] < 0) return 0;
    if (c->charge[s] == 0) return 0;
  }
  if (c->sort_interval < 1) return 0;
  if (c->field_mode > ORC_FIELD_ZERO) return 0;
  if (c->load_profile < 0 || c->load_profile > ORC_LOAD_QUIET_SINE) return 0;
  if (c->load_profile == ORC_LOAD_EXP && !(c->profile_scale > 0)) return 0;
  if (c->source_mode < 0 || c->source_mode > ORC_SOURCE_PAIRS) return 0;
  if (c->source_mode == ORC_SOURCE_PAIRS && !(c->source_x1 > 0 && c->source_x1 <= c->ncells))
    return 0;
  if (c->n_gas < 0 || c->Tg < 0 || !(c->m_gas > 0)) return 0;
  if (c->smooth_passes < 0 || c->smooth_passes > ORC_MAX_SMOOTH || c->neutrals > 1u) return 0;
  if (c->neutrals && !(c->recycle >= 0.0 && c->recycle <= 1.0 && c->T_rec >= 0.0 && c->K_iz >= 0.0 &&
                       c->T_sec >= 0.0 && c->neutral_ppc >= 0))
    return 0;
  if (!c->neutrals && c->neutral_ppc != 0) return 0;
  return 1;
}

/* ------------------------------------------------------------------------------------------ */
/* Density smoothing (Sec. 2, BIT1's smoothing operators; reading N6): each pass replaces the node
 * density by the binomial (1, 2, 1)/4 average inside and the (1, 1)/2 average at a wall node.      */
void orc_smooth(int32_t N, int32_t passes, double* rho) {
  if (passes <= 0) return;
  double* old = (double*)malloc(((size_t)N + 1) * sizeof(double));
  if (!old) return;
  for (int32_t p = 0; p < passes; ++p) {
    memcpy(old, rho, ((size_t)N + 1) * sizeof(double));
    rho[0] = (old[0] + old[1]) / 2.0;
    for (int32_t j = 1; j < N; ++j) rho[j] = (old[j - 1] + 2.0 * old[j] + old[j + 1]) / 4.0;
    rho[N] = (old[N - 1] + old[N]) / 2.0;
  }
  free(old);
}

/* ------------------------------------------------------------------------------------------ */
/* Deposit (Sec. 2 "deposition to the grid"): CIC in int64 fixed point (R12), then the node
 * charge density, half-cell volume at the walls (R4), then Poisson and the node field.        */
static void deposit_and_solve(orc_sim* s) {
  int32_t N = s->N;
  for (int sp = 0; sp < 2; ++sp) {
    int64_t* R = s->R[sp];
    memset(R, 0, sizeof(int64_t) * (size_t)(N + 1));
    orc_species* p = &s->sp[sp];
    for (size_t i = 0; i < p->n; ++i) {
      double xh = p->x[i];
      int32_t c = (int32_t)floor(xh);
      double f = xh - (double)c;
      int64_t Wr = (int64_t)rint(f * TWO32);
      int64_t Wl = (int64_t)TWO32 - Wr;
      R[c] += Wl;
      R[c + 1] += Wr;
    }
  }
  for (int32_t j = 0; j <= N; ++j) {
    double vol = (j == 0 || j == N) ? 0.5 * s->dx : s->dx;
    double q = 0.0;
    for (int sp = 0; sp < 2; ++sp) q += s->cfg.charge[sp] * s->w[sp] * ((double)s->R[sp][j] / TWO32);
    s->rho[j] = q / vol;
    s->ne[j] = s->w[0] * ((double)s->R[0][j] / TWO32) / vol;
  }
  orc_smooth(N, s->cfg.smooth_passes, s->rho);
  orc_poisson_thomas(N, s->dx, s->rho, s->cfg.V_left, s->cfg.V_right, s->phi);
  orc_efield(N, s->dx, s->phi, s->rho, s->E);
}

/* Stable counting sort of one species by cell (the "natural sorting" arranger, Sec. 2).       */
static int sort_species(orc_species* p, int32_t N) {
  size_t n = p->n;
  if (n == 0) return ORC_OK;
  size_t* cnt = (size_t*)calloc((size_t)N + 1, sizeof(size_t));
  size_t* perm = (size_t*)malloc(n * sizeof(size_t));
  double* tmp = (double*)malloc(n * sizeof(double));
  uint64_t* tid = (uint64_t*)malloc(n * sizeof(uint64_t));
  if (!cnt || !perm || !tmp || !tid) {
    free(cnt);
    free(perm);
    free(tmp);
    free(tid);
    return ORC_ENOMEM;
  }
  for (size_t i = 0; i < n; ++i) cnt[(size_t)floor(p->x[i]) + 1]++;
  for (int32_t c = 0; c < N; ++c) cnt[c + 1] += cnt[c];
  for (size_t i = 0; i < n; ++i) perm[cnt[(size_t)floor(p->x[i])]++] = i;
  double* arrs[4] = {p->x, p->vx, p->vy, p->vz};
  for (int a = 0; a < 4; ++a) {
    for (size_t k = 0; k < n; ++k) tmp[k] = arrs[a][perm[k]];
    memcpy(arrs[a], tmp, n * sizeof(double));
  }
  for (size_t k = 0; k < n; ++k) tid[k] = p->id[perm[k]];
  memcpy(p->id, tid, n * sizeof(uint64_t));
  uint32_t* tk = (uint32_t*)tid; /* reuse: n 32-bit words fit in n 64-bit ones */
  for (size_t k = 0; k < n; ++k) tk[k] = p->nk[perm[k]];
  memcpy(p->nk, tk, n * sizeof(uint32_t));
  free(cnt);
  free(perm);
  free(tmp);
  free(tid);
  return ORC_OK;
}

/* ------------------------------------------------------------------------------------------ */
/* Initial load (Sec. 2 "particle load"): positions per profile, Maxwellian velocities.  Particle
 * i of species s has id i (electrons) or 2^62 | i (ions) and draws from its own Philox stream. */
void orc_load_particle(const orc_config* c, int sp, uint64_t i, double* xo, double v[3], uint64_t* ido) {
  const int32_t N = c->ncells;
  if (sp == 2) { /* initial neutrals (N1): uniform in each cell, Maxwellian at T_rec */
    const uint64_t id = (3ull << 61) | i;
    const double vt = sqrt(c->T_rec / c->mass[1]);
    uint32_t w[4];
    draw(id, c->seed, 0, ORC_CH_INIT, 0, w);
    double x = (double)(i / (uint64_t)c->neutral_ppc) + u01(w[0]);
    if (x >= (double)N) x = nextafter((double)N, 0.0);
    draw(id, c->seed, 0, ORC_CH_INIT, 1, w);
    double n0, n1, n2, n3;
    box_muller(w[0], w[1], &n0, &n1);
    box_muller(w[2], w[3], &n2, &n3);
    *xo = x;
    v[0] = vt * n0;
    v[1] = vt * n1;
    v[2] = vt * n2;
    *ido = id;
    return;
  }
  const size_t np = (size_t)c->ppc[sp] * (size_t)N;
  const double vth = sqrt(c->T[sp] / c->mass[sp]);
  uint64_t id = (sp == 0) ? i : ((1ull << 62) | i);
  uint32_t w[4];
  double x;
  if (c->load_profile == ORC_LOAD_UNIFORM) {
    draw(id, c->seed, 0, ORC_CH_INIT, 0, w);
    x = (double)(i / (uint64_t)c->ppc[sp]) + u01(w[0]);
  } else if (c->load_profile == ORC_LOAD_EXP) {
    draw(id, c->seed, 0, ORC_CH_INIT, 0, w);
    double lam = c->profile_scale;
    x = -lam * log(1.0 - u01(w[0]) * (1.0 - exp(-(double)N / lam)));
  } else {
    double x0 = ((double)i + 0.5) * (double)N / (double)np;
    x = x0;
    if (sp == 0) x = x0 + c->profile_scale * sin(2.0 * ORC_PI * (double)c->profile_mode * x0 / (double)N);
  }
  if (x < 0.0) x = 0.0;
  if (x >= (double)N) x = nextafter((double)N, 0.0);
  draw(id, c->seed, 0, ORC_CH_INIT, 1, w);
  double n0, n1, n2, n3;
  box_muller(w[0], w[1], &n0, &n1);
  box_muller(w[2], w[3], &n2, &n3);
  *xo = x;
  v[0] = vth * n0;
  v[1] = vth * n1;
  v[2] = vth * n2;
  *ido = id;
}

/* R17: the countdown pair G(w) drawn from one Philox word. */
static uint32_t geometric_next(float p_null, uint32_t w, uint64_t* near) {
  const double v = 1.0 - u01(w); /* (0, 1] */
  const double r = log(v) / log1p(-(double)p_null);
  const double fl = floor(r);
  const double tol = 1e-9 * fmax(1.0, r);
  if (near && r > 0.0 && (r - fl < tol || fl + 1.0 - r < tol)) (*near)++;
  if (fl >= (double)NEXT_KMAX) return NEXT_KMAX; /* K > 4095: wait 4095 steps, then draw again */
  return ((uint32_t)fl + 1u) | NEXT_CAND;
}

/* The countdown of a particle of species sp created in step `step` (R17). */
static uint32_t creation_next(const orc_sim* s, int sp, uint64_t id, uint64_t step) {
  if (!s->mcc[sp]) return 0u;
  uint32_t w[4];
  draw(id, s->cfg.seed, step, ORC_CH_INIT, 2, w);
  return geometric_next(s->p_null[sp], w[0], NULL);
}

static int load(orc_sim* s) {
  const orc_config* c = &s->cfg;
  for (int sp = 0; sp < 2; ++sp) {
    size_t np = (size_t)c->ppc[sp] * (size_t)s->N;
    if (sp_reserve(&s->sp[sp], np) != ORC_OK) return ORC_ENOMEM;
    orc_species* p = &s->sp[sp];
    for (size_t i = 0; i < np; ++i) {
      double v[3];
      orc_load_particle(c, sp, (uint64_t)i, &p->x[i], v, &p->id[i]);
      p->vx[i] = v[0];
      p->vy[i] = v[1];
      p->vz[i] = v[2];
      p->nk[i] = creation_next(s, sp, p->id[i], 0);
    }
    p->n = np;
  }
  if (c->neutrals && c->neutral_ppc > 0) {
    size_t np = (size_t)c->neutral_ppc * (size_t)s->N;
    if (sp_reserve(&s->nt, np) != ORC_OK) return ORC_ENOMEM;
    orc_species* p = &s->nt;
    for (size_t i = 0; i < np; ++i) {
      double v[3];
      orc_load_particle(c, 2, (uint64_t)i, &p->x[i], v, &p->id[i]);
      p->vx[i] = v[0];
      p->vy[i] = v[1];
      p->vz[i] = v[2];
      p->nk[i] = 0u;
    }
    p->n = np;
  }
  return ORC_OK;
}

static void derive(orc_sim* s) {
  const orc_config* c = &s->cfg;
  s->N = c->ncells;
  s->dx = c->L / (double)c->ncells;
  for (int sp = 0; sp < 2; ++sp) {
    s->w[sp] = s->dx / (double)c->ppc[sp]; /* n0 = 1 */
    s->qm[sp] = c->charge[sp] / c->mass[sp];
  }
  double th = c->B_angle_deg * ORC_PI / 180.0;
  s->Bv[0] = c->B * cos(th);
  s->Bv[1] = c->B * sin(th);
  s->Bv[2] = 0.0;
  orc_nu_max(c, s->nu_max, s->p_null);
  for (int sp = 0; sp < 2; ++sp) {
    const int on = (sp == 0) ? ((c->coll_mask & (ORC_COLL_EL | ORC_COLL_EX | ORC_COLL_IZ)) != 0)
                             : ((c->coll_mask & ORC_COLL_CX) != 0);
    s->mcc[sp] = on && !(c->frozen_mask & (1u << sp)) && s->p_null[sp] > 0.0f;
  }
}

orc_sim* orc_create(const orc_config* cfg, int* err) {
  int e = ORC_OK;
  orc_sim* s = NULL;
  if (!cfg || !valid_config(cfg)) {
    e = ORC_EINVAL;
    goto out;
  }
  s = (orc_sim*)calloc(1, sizeof(orc_sim));
  if (!s) {
    e = ORC_ENOMEM;
    goto out;
  }
  s->cfg = *cfg;
  derive(s);
  for (int sp = 0; sp < 2; ++sp) s->R[sp] = (int64_t*)calloc((size_t)s->N + 1, sizeof(int64_t));
  s->rho = (double*)calloc((size_t)s->N + 1, sizeof(double));
  s->phi = (double*)calloc((size_t)s->N + 1, sizeof(double));
  s->E = (double*)calloc((size_t)s->N + 1, sizeof(double));
  s->ne = (double*)calloc((size_t)s->N + 1, sizeof(double));
  if (!s->R[0] || !s->R[1] || !s->rho || !s->phi || !s->E || !s->ne) {
    e = ORC_ENOMEM;
    goto out;
  }
  e = load(s);
  if (e != ORC_OK) goto out;
  for (int sp = 0; sp < 2; ++sp) sort_species(&s->sp[sp], s->N);
  sort_species(&s->nt, s->N);
  deposit_and_solve(s);
out:
  if (e != ORC_OK && s) {
    orc_free(s);
    s = NULL;
  }
  if (err) *err = e;
  return s;
}

void orc_free(orc_sim* s) {
  if (!s) return;
  for (int sp = 0; sp < 2; ++sp) {
    free(s->sp[sp].x);
    free(s->sp[sp].vx);
    free(s->sp[sp].vy);
    free(s->sp[sp].vz);
    free(s->sp[sp].id);
    free(s->sp[sp].nk);
    free(s->R[sp]);
  }
  free(s->nt.x);
  free(s->nt.vx);
  free(s->nt.vy);
  free(s->nt.vz);
  free(s->nt.id);
  free(s->nt.nk);
  free(s->rho);
  free(s->phi);
  free(s->E);
  free(s->ne);
  free(s);
}

/* ------------------------------------------------------------------------------------------ */
/* Monte Carlo collision of one electron (null-collision method; Sec. 2 "MC collision
 * handling").  Returns 1 when an ionization produced a pair (written to e_new / i_new).       */
static int collide_electron(const orc_sim* s, uint64_t id, uint64_t step, const uint32_t w[4], double x,
                            double v[3], orc_tcount* tc, orc_newp* e_new, orc_newp* i_new) {
  const orc_config* c = &s->cfg;
  tc->coll[4]++;
  double m = c->mass[0];
  double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
  double speed = sqrt(v2);
  double En = 0.5 * m * v2;
  double nu_el = (c->coll_mask & ORC_COLL_EL) ? c->n_gas * c->sigma_el * speed : 0.0;
  double nu_ex = 0.0, nu_iz = 0.0;
  if ((c->coll_mask & ORC_COLL_EX) && En > c->E_ex)
    nu_ex = c->n_gas * c->sigma_ex * fmin((En - c->E_ex) / c->E_ex, 1.0) * speed;
  if ((c->coll_mask & ORC_COLL_IZ) && En > c->E_iz)
    nu_iz = c->n_gas * c->sigma_iz * fmin((En - c->E_iz) / c->E_iz, 1.0) * speed;
  double numax = (double)s->nu_max[0];
  double b1 = nu_el, b2 = b1 + nu_ex, b3 = b2 + nu_iz;
  if (b3 > numax) tc->viol++;
  double r = u01(w[1]) * numax;
  double tol = 1e-5 * numax;
  int near = fabs(r - b1) < tol || fabs(r - b2) < tol || fabs(r - b3) < tol;
  if ((c->coll_mask & ORC_COLL_EX) && fabs(En - c->E_ex) < 1e-5 * c->E_ex) near = 1;
  if ((c->coll_mask & ORC_COLL_IZ) && fabs(En - c->E_iz) < 1e-5 * c->E_iz) near = 1;
  if (near) tc->near++;
  double d[3];
  iso_dir(w[2], w[3], d);
  if (r < b1) { /* elastic: energy loss 2m/M (1 - cos chi) */
    double cchi = (v[0] * d[0] + v[1] * d[1] + v[2] * d[2]) / speed;
    double sp2 = speed * sqrt(1.0 - 2.0 * m / c->m_gas * (1.0 - cchi));
    v[0] = sp2 * d[0];
    v[1] = sp2 * d[1];
    v[2] = sp2 * d[2];
    tc->coll[0]++;
    return 0;
  }
  if (r < b2) { /* excitation: loses E_ex */
    double sp2 = sqrt(2.0 * (En - c->E_ex) / m);
    v[0] = sp2 * d[0];
    v[1] = sp2 * d[1];
    v[2] = sp2 * d[2];
    tc->coll[1]++;
    return 0;
  }
  if (r < b3) { /* ionization: E - E_iz split uniformly between the two electrons */
    uint32_t a[4], b[4], k[4];
    draw(id, c->seed, step, ORC_CH_SCAT, 0, a);
    draw(id, c->seed, step, ORC_CH_SCAT, 1, b);
    draw(id, c->seed, step, ORC_CH_CHILD, 0, k);
    double Er = En - c->E_iz;
    double Es = u01(a[0]) * Er;
    double Ep = Er - Es;
    double spp = sqrt(2.0 * Ep / m), sps = sqrt(2.0 * Es / m);
    v[0] = spp * d[0];
    v[1] = spp * d[1];
    v[2] = spp * d[2];
    double d2[3];
    iso_dir(a[1], a[2], d2);
    e_new->x = x;
    e_new->v[0] = sps * d2[0];
    e_new->v[1] = sps * d2[1];
    e_new->v[2] = sps * d2[2];
    e_new->id = (uint64_t)k[0] | ((uint64_t)k[1] << 32);
    double n0, n1, n2, n3, vt = sqrt(c->Tg / c->mass[1]);
    box_muller(b[0], b[1], &n0, &n1);
    box_muller(b[2], b[3], &n2, &n3);
    i_new->x = x;
    i_new->v[0] = vt * n0;
    i_new->v[1] = vt * n1;
    i_new->v[2] = vt * n2;
    i_new->id = (uint64_t)k[2] | ((uint64_t)k[3] << 32);
    tc->coll[2]++;
    return 1;
  }
  return 0;
}

/* Charge exchange of one ion: the ion leaves with a Maxwellian velocity at T_g.               */
static void collide_ion(const orc_sim* s, uint64_t id, uint64_t step, const uint32_t w[4], double v[3],
                        orc_tcount* tc) {
  const orc_config* c = &s->cfg;
  tc->coll[4]++;
  double speed = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  double numax = (double)s->nu_max[1];
  double b1 = c->n_gas * c->sigma_cx * speed;
  if (b1 > numax) tc->viol++;
  double r = u01(w[1]) * numax;
  if (fabs(r - b1) < 1e-5 * numax) tc->near++;
  if (r < b1) {
    uint32_t a[4];
    draw(id, c->seed, step, ORC_CH_SCAT, 0, a);
    double n0, n1, n2, n3, vt = sqrt(c->Tg / c->mass[1]);
    box_muller(w[2], w[3], &n0, &n1);
    box_muller(a[0], a[1], &n2, &n3);
    v[0] = vt * n0;
    v[1] = vt * n1;
    v[2] = vt * n2;
    tc->coll[3]++;
  }
}

/* ------------------------------------------------------------------------------------------ */
/* Recycling of an ion absorbed at wall `side` (0 left, 1 right) in step `step` (reading N2):
 * returns 1 and the new neutral when the ion returns.                                          */
static int recycle_ion(const orc_sim* s, uint64_t id, uint64_t step, int side, orc_newp* out) {
  const orc_config* c = &s->cfg;
  uint32_t w[4], k[4];
  draw(id, c->seed, step, ORC_CH_RECYCLE, 0, w);
  if (!(u01(w[0]) < c->recycle)) return 0;
  draw(id, c->seed, step, ORC_CH_RECYCLE, 1, k);
  double vt = sqrt(c->T_rec / c->mass[1]);
  double vx = vt * sqrt(-2.0 * log(1.0 - u01(w[1]))); /* flux-weighted half-Maxwellian */
  double n0, n1;
  box_muller(w[2], w[3], &n0, &n1);
  out->x = side == 0 ? 0.0 : (double)s->N - 1.0 / 16777216.0;
  out->v[0] = side == 0 ? vx : -vx;
  out->v[1] = vt * n0;
  out->v[2] = vt * n1;
  out->id = (uint64_t)k[0] | ((uint64_t)k[1] << 32);
  return 1;
}

/* Electron-impact ionization of a neutral at x in step `step` (reading N4): returns 1 and the
 * electron it creates when the neutral ionizes; counts a draw within 1e-5 P of P in *near.     */
static int ionize_neutral(const orc_sim* s, uint64_t id, uint64_t step, double x, uint64_t* near,
                          orc_newp* e_new) {
  const orc_config* c = &s->cfg;
  int32_t cc = (int32_t)floor(x);
  double f = x - (double)cc;
  double ne = (1.0 - f) * s->ne[cc] + f * s->ne[cc + 1];
  double P = 1.0 - exp(-c->K_iz * ne * c->dt);
  uint32_t w[4];
  draw(id, c->seed, step, ORC_CH_NIZ, 0, w);
  double u = u01(w[0]);
  if (fabs(u - P) < 1e-5 * P) (*near)++;
  if (!(u < P)) return 0;
  uint32_t b[4], k[4];
  draw(id, c->seed, step, ORC_CH_NIZ, 1, b);
  draw(id, c->seed, step, ORC_CH_NIZ, 2, k);
  double vt = sqrt(c->T_sec / c->mass[0]);
  double n0, n1, n2, n3;
  box_muller(b[0], b[1], &n0, &n1);
  box_muller(b[2], b[3], &n2, &n3);
  e_new->x = x;
  e_new->v[0] = vt * n0;
  e_new->v[1] = vt * n1;
  e_new->v[2] = vt * n2;
  e_new->id = (uint64_t)k[0] | ((uint64_t)k[1] << 32);
  return 1;
}

/* ------------------------------------------------------------------------------------------ */
/* One full step (R2).                                                                         */
/* The mover stages of one particle under the node field E: CIC gather (Sec. 2 "interpolating
 * fields back"), Boris push and position update (Sec. 2 "particle mover").  xh is the position in
 * cells. */
static void move_particle(const orc_config* c, double qm, const double Bv[3], double dx, const double* E,
                          double* xh, double v[3]) {
  double Ex = 0.0;
  if (c->field_mode == ORC_FIELD_SELF) {
    int32_t cc = (int32_t)floor(*xh);
    double f = *xh - (double)cc;
    Ex = (1.0 - f) * E[cc] + f * E[cc + 1];
  } else if (c->field_mode == ORC_FIELD_EXTERNAL) {
    Ex = c->E_ext;
  }
  double Ev[3] = {Ex, 0.0, 0.0};
  orc_boris(qm, c->dt, Ev, Bv, v);
  *xh += v[0] * c->dt / dx;
}

static int step_once(orc_sim* s) {
  const orc_config* c = &s->cfg;
  const int32_t N = s->N;
  const uint64_t step = s->step;
  int nth = g_threads;
  s->particle_steps += s->sp[0].n + s->sp[1].n;
  s->nt_particle_steps += s->nt.n;
  orc_tcount tcs[2][MAX_THREADS];
  orc_plist born[2][MAX_THREADS];
  orc_plist nz_born[2][MAX_THREADS]; /* (electron, ion) of each neutral's ionization */
  orc_plist recycled[MAX_THREADS];
  memset(tcs, 0, sizeof(tcs));
  memset(born, 0, sizeof(born));
  memset(nz_born, 0, sizeof(nz_born));
  memset(recycled, 0, sizeof(recycled));
  int err = ORC_OK;

  for (int sp = 0; sp < 2; ++sp) {
    if (c->frozen_mask & (1u << sp)) continue;
    orc_species* p = &s->sp[sp];
    unsigned char* alive = (unsigned char*)malloc(p->n ? p->n : 1);
    double* eabs = (double*)malloc((p->n ? p->n : 1) * sizeof(double));
    if (!alive || !eabs) {
      free(alive);
      free(eabs);
      return ORC_ENOMEM;
    }
    const int do_mcc = s->mcc[sp];
    long long n = (long long)p->n;
#ifdef _OPENMP
#pragma omp parallel for num_threads(nth) schedule(static)
#endif
    for (long long i = 0; i < n; ++i) {
      int t = 0;
#ifdef _OPENMP
      t = omp_get_thread_num();
#endif
      orc_tcount* tc = &tcs[sp][t];
      double xh = p->x[i];
      double v[3] = {p->vx[i], p->vy[i], p->vz[i]};
      move_particle(c, s->qm[sp], s->Bv, s->dx, s->E, &xh, v);
      /* walls (Table 3: plasma absorbed at the walls) */
      if (xh < 0.0 || xh >= (double)N) {
        const int side = xh < 0.0 ? 0 : 1;
        tc->wall_hits[side]++;
        if (sp == 1 && c->neutrals) { /* N2 */
          orc_newp q;
          if (recycle_ion(s, p->id[i], step, side, &q)) {
            tc->recycled[side]++;
            if (plist_add(&recycled[t], q.x, q.v, q.id) != ORC_OK) err = ORC_ENOMEM;
          }
        }
        eabs[i] = 0.5 * c->mass[sp] * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) * s->w[sp];
        alive[i] = 0;
        p->x[i] = xh;
        p->vx[i] = v[0];
        p->vy[i] = v[1];
        p->vz[i] = v[2];
        continue;
      }
      alive[i] = 1;
      /* Monte Carlo collisions on survivors: the countdown of R17 decides the candidates */
      if (do_mcc) {
        const uint32_t k = (p->nk[i] & NEXT_KMAX) - 1u, cand = p->nk[i] & NEXT_CAND;
        if (k == 0u) {
          uint32_t w[4];
          draw(p->id[i], c->seed, step, ORC_CH_COLL, 0, w);
          if (cand && sp == 0) {
            orc_newp e_new, i_new;
            if (collide_electron(s, p->id[i], step, w, xh, v, tc, &e_new, &i_new)) {
              if (plist_add(&born[0][t], e_new.x, e_new.v, e_new.id) != ORC_OK ||
                  plist_add(&born[1][t], i_new.x, i_new.v, i_new.id) != ORC_OK)
                err = ORC_ENOMEM;
            }
          } else if (cand) {
            collide_ion(s, p->id[i], step, w, v, tc);
          }
          p->nk[i] = geometric_next(s->p_null[sp], w[0], &tc->near);
        } else {
          p->nk[i] = k | cand;
        }
      }
      p->x[i] = xh;
      p->vx[i] = v[0];
      p->vy[i] = v[1];
      p->vz[i] = v[2];
    }
    /* stable compaction of the survivors; absorbed energy summed in particle order so that the
     * result does not depend on the thread count */
    size_t k = 0;
    for (size_t i = 0; i < p->n; ++i) {
      if (!alive[i]) {
        s->wall_energy[sp] += eabs[i];
        continue;
      }
      p->x[k] = p->x[i];
      p->vx[k] = p->vx[i];
      p->vy[k] = p->vy[i];
      p->vz[k] = p->vz[i];
      p->id[k] = p->id[i];
      p->nk[k] = p->nk[i];
      ++k;
    }
    p->n = k;
    free(alive);
    free(eabs);
  }
  if (err != ORC_OK) return err;

  /* merge the per-thread counters and append the births, in thread order */
  uint64_t ion_losses = 0;
  for (int sp = 0; sp < 2; ++sp) {
    for (int t = 0; t < MAX_THREADS; ++t) {
      orc_tcount* tc = &tcs[sp][t];
      for (int side = 0; side < 2; ++side) {
        s->wall_hits[sp][side] += tc->wall_hits[side];
        s->wall_charge += (c->charge[sp] > 0 ? 1 : -1) * (int64_t)tc->wall_hits[side];
      }
      for (int k = 0; k < 5; ++k) s->coll[k] += tc->coll[k];
      s->near[sp] += tc->near;
      s->viol[sp] += tc->viol;
      s->nt_recycled[0] += tc->recycled[0];
      s->nt_recycled[1] += tc->recycled[1];
      if (sp == 1) ion_losses += tc->wall_hits[0] + tc->wall_hits[1];
    }
  }

  /* tracked neutrals alive at the step start: ballistic move, walls, ionization (N3, N4) */
  if (c->neutrals && s->nt.n) {
    orc_species* p = &s->nt;
    const long long n = (long long)p->n;
    unsigned char* keep = (unsigned char*)malloc((size_t)n);
    uint64_t(*cnt)[4] = (uint64_t(*)[4])calloc(MAX_THREADS, sizeof(*cnt)); /* lost L, R, ionized, near */
    if (!keep || !cnt) {
      free(keep);
      free(cnt);
      return ORC_ENOMEM;
    }
#ifdef _OPENMP
#pragma omp parallel for num_threads(nth) schedule(static)
#endif
    for (long long i = 0; i < n; ++i) {
      int t = 0;
#ifdef _OPENMP
      t = omp_get_thread_num();
#endif
      double xh = p->x[i] + p->vx[i] * c->dt / s->dx;
      if (xh < 0.0 || xh >= (double)N) {
        cnt[t][xh < 0.0 ? 0 : 1]++;
        keep[i] = 0;
        continue;
      }
      p->x[i] = xh;
      orc_newp e_new;
      if (ionize_neutral(s, p->id[i], step, xh, &cnt[t][3], &e_new)) {
        const double v[3] = {p->vx[i], p->vy[i], p->vz[i]};
        if (plist_add(&nz_born[0][t], e_new.x, e_new.v, e_new.id) != ORC_OK ||
            plist_add(&nz_born[1][t], xh, v, p->id[i]) != ORC_OK)
          err = ORC_ENOMEM;
        cnt[t][2]++;
        keep[i] = 0;
        continue;
      }
      keep[i] = 1;
    }
    size_t k = 0;
    for (size_t i = 0; i < p->n; ++i) {
      if (!keep[i]) continue;
      p->x[k] = p->x[i];
      p->vx[k] = p->vx[i];
      p->vy[k] = p->vy[i];
      p->vz[k] = p->vz[i];
      p->id[k] = p->id[i];
      p->nk[k] = p->nk[i];
      ++k;
    }
    p->n = k;
    for (int t = 0; t < MAX_THREADS; ++t) {
      s->nt_lost[0] += cnt[t][0];
      s->nt_lost[1] += cnt[t][1];
      s->nt_ionized += cnt[t][2];
      s->nt_near += cnt[t][3];
    }
    free(keep);
    free(cnt);
  }
  for (int sp = 0; sp < 2; ++sp) {
    for (int t = 0; t < MAX_THREADS; ++t) {
      orc_plist* l = &born[sp][t];
      for (size_t k = 0; k < l->n; ++k) {
        if (sp_push_back(&s->sp[sp], l->p[k].x, l->p[k].v, l->p[k].id, creation_next(s, sp, l->p[k].id, step)) !=
            ORC_OK)
          err = ORC_ENOMEM;
      }
      s->births[sp] += l->n;
      free(l->p);
    }
  }
  for (int sp = 0; sp < 2; ++sp) {
    for (int t = 0; t < MAX_THREADS; ++t) {
      orc_plist* l = &nz_born[sp][t];
      for (size_t k = 0; k < l->n; ++k)
        if (sp_push_back(&s->sp[sp], l->p[k].x, l->p[k].v, l->p[k].id, creation_next(s, sp, l->p[k].id, step)) !=
            ORC_OK)
          err = ORC_ENOMEM;
      free(l->p);
    }
  }
  for (int t = 0; t < MAX_THREADS; ++t) {
    orc_plist* l = &recycled[t];
    for (size_t k = 0; k < l->n; ++k)
      if (sp_push_back(&s->nt, l->p[k].x, l->p[k].v, l->p[k].id, 0u) != ORC_OK) err = ORC_ENOMEM;
    free(l->p);
  }
  if (err != ORC_OK) return err;

  /* source (R13): one pair per ion absorbed in this step */
  if (c->source_mode == ORC_SOURCE_PAIRS) {
    for (uint64_t k = 0; k < ion_losses; ++k) {
      uint64_t ide = (1ull << 63) | ((step & 0x7FFFFFFFull) << 32) | (2 * k);
      uint32_t w[4];
      draw(ide, c->seed, step, ORC_CH_SOURCE, 0, w);
      double x = c->source_x1 * u01(w[0]);
      for (int sp = 0; sp < 2; ++sp) {
        uint64_t id = ide + (uint64_t)sp;
        double vt = sqrt(c->T[sp] / c->mass[sp]);
        double n0, n1, n2, n3;
        draw(id, c->seed, step, ORC_CH_SOURCE, 1, w);
        box_muller(w[0], w[1], &n0, &n1);
        box_muller(w[2], w[3], &n2, &n3);
        double v[3] = {vt * n0, vt * n1, vt * n2};
        if (sp_push_back(&s->sp[sp], x, v, id, creation_next(s, sp, id, step)) != ORC_OK) return ORC_ENOMEM;
      }
    }
    s->source_pairs += ion_losses;
  }

  /* deposit + Poisson + field */
  deposit_and_solve(s);

  /* arranger: sort + compaction every sort_interval steps */
  if (step % (uint64_t)c->sort_interval == 0) {
    for (int sp = 0; sp < 2; ++sp)
      if (sort_species(&s->sp[sp], N) != ORC_OK) return ORC_ENOMEM;
    if (sort_species(&s->nt, N) != ORC_OK) return ORC_ENOMEM;
  }
  s->step = step + 1;
  return ORC_OK;
}

int orc_step(orc_sim* s, int32_t nsteps) {
  if (!s || nsteps < 0) return ORC_EINVAL;
  for (int32_t k = 0; k < nsteps; ++k) {
    int e = step_once(s);
    if (e != ORC_OK) return e;
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------------------------ */
/* One step of n given particles of species sp under a given node field E (N + 1 values): the
 * mover, the wall test and the null-collision MC of orc_step, for parity checks that sample a state
 * too large for the whole oracle step.  Positions in cells, velocities as (vx, vy, vz) triples.
 * flags[k]: 1 absorbed at a wall, 2 collision candidate, 4 near-threshold draw, 8 ionization (the
 * new pair itself is not returned).  Tracked neutrals and the pair source are not part of it. */
int orc_step_sample(const orc_config* cfg, int sp, uint64_t step, const double* E, size_t n, const double* x,
                    const double* v, const uint64_t* id, const uint32_t* nk, double* xo, double* vo, uint32_t* nko,
                    int32_t* flags) {
  if (!cfg || !valid_config(cfg) || sp < 0 || sp > 1 ||
      (n && (!x || !v || !id || !nk || !xo || !vo || !nko || !flags)))
    return ORC_EINVAL;
  if (cfg->field_mode == ORC_FIELD_SELF && !E) return ORC_EINVAL;
  orc_sim t;
  memset(&t, 0, sizeof(t));
  t.cfg = *cfg;
  derive(&t);
  const int moves = !(cfg->frozen_mask & (1u << sp));
  for (size_t k = 0; k < n; ++k) {
    double xh = x[k];
    double vv[3] = {v[3 * k], v[3 * k + 1], v[3 * k + 2]};
    int32_t fl = 0;
    nko[k] = nk[k];
    if (moves) {
      move_particle(cfg, t.qm[sp], t.Bv, t.dx, E, &xh, vv);
      if (xh < 0.0 || xh >= (double)t.N) {
        fl |= 1;
      } else if (t.mcc[sp]) {
        orc_tcount tc;
        memset(&tc, 0, sizeof(tc));
        const uint32_t kk = (nk[k] & NEXT_KMAX) - 1u, cand = nk[k] & NEXT_CAND;
        if (kk == 0u) {
          uint32_t w[4];
          draw(id[k], cfg->seed, step, ORC_CH_COLL, 0, w);
          if (cand && sp == 0) {
            orc_newp a, b;
            if (collide_electron(&t, id[k], step, w, xh, vv, &tc, &a, &b)) fl |= 8;
          } else if (cand) {
            collide_ion(&t, id[k], step, w, vv, &tc);
          }
          nko[k] = geometric_next(t.p_null[sp], w[0], &tc.near);
        } else {
          nko[k] = kk | cand;
        }
        if (tc.coll[4]) fl |= 2;
        if (tc.near) fl |= 4;
      }
    }
    xo[k] = xh;
    vo[3 * k] = vv[0];
    vo[3 * k + 1] = vv[1];
    vo[3 * k + 2] = vv[2];
    flags[k] = fl;
  }
  return ORC_OK;
}

static int cmp_double(const void* a, const void* b) {
  double x = *(const double*)a, y = *(const double*)b;
  return (x > y) - (x < y);
}

int orc_diag(orc_sim* s, orc_diag_t* d) {
  if (!s || !d) return ORC_EINVAL;
  memset(d, 0, sizeof(*d));
  d->step = s->step;
  for (int sp = 0; sp < 2; ++sp) {
    d->n[sp] = s->sp[sp].n;
    d->wall_hits[sp][0] = s->wall_hits[sp][0];
    d->wall_hits[sp][1] = s->wall_hits[sp][1];
    d->near_threshold[sp] = s->near[sp];
    d->nu_max_violations[sp] = s->viol[sp];
    d->births[sp] = s->births[sp];
    d->wall_energy[sp] = s->wall_energy[sp];
    /* kinetic energy summed in ascending order of the terms: independent of storage order */
    orc_species* p = &s->sp[sp];
    double* e = (double*)malloc((p->n ? p->n : 1) * sizeof(double));
    if (!e) return ORC_ENOMEM;
    for (size_t i = 0; i < p->n; ++i)
      e[i] = 0.5 * s->cfg.mass[sp] * (p->vx[i] * p->vx[i] + p->vy[i] * p->vy[i] + p->vz[i] * p->vz[i]);
    qsort(e, p->n, sizeof(double), cmp_double);
    double ke = 0.0;
    for (size_t i = 0; i < p->n; ++i) ke += e[i];
    free(e);
    d->ke[sp] = ke * s->w[sp];
  }
  for (int k = 0; k < 5; ++k) d->coll[k] = s->coll[k];
  d->source_pairs = s->source_pairs;
  d->wall_charge = s->wall_charge;
  int64_t q = 0;
  for (int32_t j = 0; j <= s->N; ++j)
    for (int sp = 0; sp < 2; ++sp) q += (s->cfg.charge[sp] > 0 ? 1 : -1) * s->R[sp][j];
  d->net_charge_units = q;
  double fe = 0.0;
  for (int32_t j = 0; j <= s->N; ++j) {
    double wgt = (j == 0 || j == s->N) ? 0.5 : 1.0;
    fe += wgt * 0.5 * s->E[j] * s->E[j] * s->dx;
  }
  d->field_energy = fe;
  d->particle_steps = s->particle_steps;
  return ORC_OK;
}

int orc_fields(orc_sim* s, int64_t* R, double* rho, double* phi, double* E) {
  if (!s) return ORC_EINVAL;
  size_t nn = (size_t)s->N + 1;
  if (R) {
    memcpy(R, s->R[0], nn * sizeof(int64_t));
    memcpy(R + nn, s->R[1], nn * sizeof(int64_t));
  }
  if (rho) memcpy(rho, s->rho, nn * sizeof(double));
  if (phi) memcpy(phi, s->phi, nn * sizeof(double));
  if (E) memcpy(E, s->E, nn * sizeof(double));
  return ORC_OK;
}

static orc_species* species_of(orc_sim* s, int species) {
  if (!s || species < 0 || species > 2) return NULL;
  return species == 2 ? &s->nt : &s->sp[species];
}

uint64_t orc_count(orc_sim* s, int species) {
  orc_species* p = species_of(s, species);
  return p ? p->n : 0;
}

int orc_neutral_diag(orc_sim* s, orc_ndiag_t* d) {
  if (!s || !d) return ORC_EINVAL;
  memset(d, 0, sizeof(*d));
  orc_species* p = &s->nt;
  d->n = p->n;
  for (int k = 0; k < 2; ++k) {
    d->recycled[k] = s->nt_recycled[k];
    d->lost[k] = s->nt_lost[k];
  }
  d->ionized = s->nt_ionized;
  d->near_threshold = s->nt_near;
  d->particle_steps = s->nt_particle_steps;
  /* neutrals carry the ion's mass and weight (N1); terms summed in ascending order */
  double* e = (double*)malloc((p->n ? p->n : 1) * sizeof(double));
  if (!e) return ORC_ENOMEM;
  for (size_t i = 0; i < p->n; ++i)
    e[i] = 0.5 * s->cfg.mass[1] * (p->vx[i] * p->vx[i] + p->vy[i] * p->vy[i] + p->vz[i] * p->vz[i]);
  qsort(e, p->n, sizeof(double), cmp_double);
  double ke = 0.0;
  for (size_t i = 0; i < p->n; ++i) ke += e[i];
  free(e);
  d->ke = ke * s->w[1];
  return ORC_OK;
}

int orc_countdown(orc_sim* s, int species, uint32_t* nk) {
  orc_species* p = species_of(s, species);
  if (!p || !nk) return ORC_EINVAL;
  for (size_t i = 0; i < p->n; ++i) nk[i] = p->nk[i];
  return ORC_OK;
}

int orc_particles(orc_sim* s, int species, double* x, double* v, uint64_t* id) {
  orc_species* p = species_of(s, species);
  if (!p) return ORC_EINVAL;
  for (size_t i = 0; i < p->n; ++i) {
    if (x) x[i] = p->x[i];
    if (v) {
      v[3 * i] = p->vx[i];
      v[3 * i + 1] = p->vy[i];
      v[3 * i + 2] = p->vz[i];
    }
    if (id) id[i] = p->id[i];
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------------------------ */
/* Snapshot blob, version 3, little-endian, no padding:
 *   "PICMCSN1" | u32 version | u32 0 | u64 config hash | u64 step | u64 n[2] |
 *   u64 wall_hits[2][2] | u64 coll[5] | u64 near[2] | u64 viol[2] | u64 births[2] |
 *   u64 source_pairs | u64 dropped | i64 wall_charge | f64 wall_energy[2] |
 *   per species: u32 cell word[n] | f64 frac[n] | f64 vx[n] | f64 vy[n] | f64 vz[n] | u64 id[n] |
 *   u32 CRC-32 (IEEE 802.3, reflected, as zlib) of everything before it.
 * The cell word is cell | k << 18 | c << 30 with the null-collision countdown (k, c) of R17 (0 in
 * bits 18..31 for a species without the test).
 * Particles are written in ascending id order within a species (canonical order), so two runs
 * that hold the same particle set write the same bytes.  This mirrors the checkpoint semantics
 * of Sec. 4.1 (per-species particle records; restart rebuilds positions and velocities).
 * Version 4 (configurations with tracked neutrals) inserts before the CRC: u64 n_neutral |
 * u64 recycled[2] | u64 lost[2] | u64 ionized | u64 near | the neutral records as above.     */
#define SNAP_MAGIC "PICMCSN1"
#define SNAP_HDR (8 + 4 + 4 + 8 + 8 + 16 + 17 * 8 + 8 + 16)

static uint32_t crc32_ieee(const unsigned char* p, size_t n) {
  uint32_t c = 0xFFFFFFFFu;
  for (size_t i = 0; i < n; ++i) {
    c ^= p[i];
    for (int k = 0; k < 8; ++k) c = (c >> 1) ^ (0xEDB88320u & (0u - (c & 1u)));
  }
  return c ^ 0xFFFFFFFFu;
}

static void fnv_bytes(uint64_t* h, const void* p, size_t n) {
  const unsigned char* b = (const unsigned char*)p;
  for (size_t i = 0; i < n; ++i) {
    *h ^= b[i];
    *h *= 0x100000001b3ull;
  }
}

uint64_t orc_config_hash(const orc_config* c) {
  uint64_t h = 0xcbf29ce484222325ull;
  int32_t iv[6] = {c->ncells, c->ppc[0], c->ppc[1], c->load_profile, c->profile_mode,
                   c->source_mode};
  uint32_t uv[3] = {c->coll_mask, c->field_mode, c->frozen_mask};
  double dv[25] = {c->L,        c->dt,          c->mass[0],  c->mass[1],  c->charge[0],
                   c->charge[1], c->T[0],       c->T[1],     c->Tg,       c->m_gas,
                   c->B,        c->B_angle_deg, c->V_left,   c->V_right,  c->n_gas,
                   c->sigma_el, c->sigma_ex,    c->E_ex,     c->sigma_iz, c->E_iz,
                   c->sigma_cx, c->E_cap,       c->E_ext,    c->profile_scale,
                   c->source_x1};
  fnv_bytes(&h, iv, sizeof(iv));
  fnv_bytes(&h, uv, sizeof(uv));
  fnv_bytes(&h, dv, sizeof(dv));
  fnv_bytes(&h, &c->seed, sizeof(uint64_t));
  if (c->smooth_passes || c->neutrals) { /* the sheath-physics fields, when any is in use */
    int32_t iv2[3] = {c->smooth_passes, (int32_t)c->neutrals, c->neutral_ppc};
    double dv2[4] = {c->recycle, c->T_rec, c->K_iz, c->T_sec};
    fnv_bytes(&h, iv2, sizeof(iv2));
    fnv_bytes(&h, dv2, sizeof(dv2));
  }
  return h;
}

typedef struct {
  const uint64_t* id;
  size_t i;
} idx_key;

static int cmp_key(const void* a, const void* b) {
  const idx_key* x = (const idx_key*)a;
  const idx_key* y = (const idx_key*)b;
  uint64_t u = x->id[x->i], v = y->id[y->i];
  return (u > v) - (u < v);
}

static void put(unsigned char** q, const void* src, size_t n) {
  memcpy(*q, src, n);
  *q += n;
}

/* One species' records in ascending id order. */
static int put_species(unsigned char** q, const orc_species* p) {
  size_t n = p->n;
  idx_key* ord = (idx_key*)malloc((n ? n : 1) * sizeof(idx_key));
  if (!ord) return ORC_ENOMEM;
  for (size_t i = 0; i < n; ++i) {
    ord[i].id = p->id;
    ord[i].i = i;
  }
  qsort(ord, n, sizeof(idx_key), cmp_key);
  for (size_t k = 0; k < n; ++k) {
    const uint32_t cw = (uint32_t)floor(p->x[ord[k].i]) | (p->nk[ord[k].i] << CELL_BITS);
    put(q, &cw, 4);
  }
  for (size_t k = 0; k < n; ++k) {
    double xh = p->x[ord[k].i];
    double f = xh - floor(xh);
    put(q, &f, 8);
  }
  double* arrs[3] = {p->vx, p->vy, p->vz};
  for (int a = 0; a < 3; ++a)
    for (size_t k = 0; k < n; ++k) put(q, &arrs[a][ord[k].i], 8);
  for (size_t k = 0; k < n; ++k) put(q, &p->id[ord[k].i], 8);
  free(ord);
  return ORC_OK;
}

#define SNAP_NT_HDR (8 + 6 * 8)

int orc_snapshot(orc_sim* s, void* buf, size_t cap, size_t* needed) {
  if (!s) return ORC_EINVAL;
  size_t need = SNAP_HDR + 4;
  for (int sp = 0; sp < 2; ++sp) need += s->sp[sp].n * 44;
  if (s->cfg.neutrals) need += SNAP_NT_HDR + s->nt.n * 44;
  if (needed) *needed = need;
  if (!buf) return ORC_OK;
  if (cap < need) return ORC_EINVAL;
  unsigned char* q = (unsigned char*)buf;
  uint32_t ver = s->cfg.neutrals ? 4 : 3, zero = 0;
  uint64_t h = orc_config_hash(&s->cfg), dropped = 0;
  put(&q, SNAP_MAGIC, 8);
  put(&q, &ver, 4);
  put(&q, &zero, 4);
  put(&q, &h, 8);
  put(&q, &s->step, 8);
  for (int sp = 0; sp < 2; ++sp) {
    uint64_t n = s->sp[sp].n;
    put(&q, &n, 8);
  }
  put(&q, s->wall_hits, 32);
  put(&q, s->coll, 40);
  put(&q, s->near, 16);
  put(&q, s->viol, 16);
  put(&q, s->births, 16);
  put(&q, &s->source_pairs, 8);
  put(&q, &dropped, 8);
  put(&q, &s->wall_charge, 8);
  put(&q, s->wall_energy, 16);
  for (int sp = 0; sp < 2; ++sp)
    if (put_species(&q, &s->sp[sp]) != ORC_OK) return ORC_ENOMEM;
  if (s->cfg.neutrals) {
    uint64_t nn = s->nt.n;
    put(&q, &nn, 8);
    put(&q, s->nt_recycled, 16);
    put(&q, s->nt_lost, 16);
    put(&q, &s->nt_ionized, 8);
    put(&q, &s->nt_near, 8);
    if (put_species(&q, &s->nt) != ORC_OK) return ORC_ENOMEM;
  }
  uint32_t crc = crc32_ieee((const unsigned char*)buf, (size_t)(q - (unsigned char*)buf));
  put(&q, &crc, 4);
  return ORC_OK;
}

static void get(const unsigned char** q, void* dst, size_t n) {
  memcpy(dst, *q, n);
  *q += n;
}

int orc_restore(orc_sim* s, const void* buf, size_t len) {
  if (!s || !buf) return ORC_EINVAL;
  const unsigned char* b = (const unsigned char*)buf;
  if (len < SNAP_HDR + 4 || memcmp(b, SNAP_MAGIC, 8) != 0) return ORC_ECORRUPT;
  uint32_t crc;
  memcpy(&crc, b + len - 4, 4);
  if (crc != crc32_ieee(b, len - 4)) return ORC_ECORRUPT;
  const unsigned char* q = b + 8;
  uint32_t ver, zero;
  uint64_t h, step, n[2], dropped;
  get(&q, &ver, 4);
  get(&q, &zero, 4);
  get(&q, &h, 8);
  if (ver != (s->cfg.neutrals ? 4u : 3u) || h != orc_config_hash(&s->cfg)) return ORC_ECORRUPT;
  get(&q, &step, 8);
  get(&q, &n[0], 8);
  get(&q, &n[1], 8);
  uint64_t nn = 0;
  if (n[0] > len / 44 || n[1] > len / 44) return ORC_ECORRUPT;
  size_t charged = SNAP_HDR + 44 * (n[0] + n[1]);
  if (ver == 4) {
    if (len < charged + SNAP_NT_HDR + 4) return ORC_ECORRUPT;
    memcpy(&nn, b + charged, 8);
    if (nn > len / 44 || len != charged + SNAP_NT_HDR + 44 * nn + 4) return ORC_ECORRUPT;
  } else if (len != charged + 4) {
    return ORC_ECORRUPT;
  }
  get(&q, s->wall_hits, 32);
  get(&q, s->coll, 40);
  get(&q, s->near, 16);
  get(&q, s->viol, 16);
  get(&q, s->births, 16);
  get(&q, &s->source_pairs, 8);
  get(&q, &dropped, 8);
  get(&q, &s->wall_charge, 8);
  get(&q, s->wall_energy, 16);
  s->step = step;
  s->particle_steps = 0;
  s->nt.n = 0;
  memset(s->nt_recycled, 0, sizeof(s->nt_recycled));
  memset(s->nt_lost, 0, sizeof(s->nt_lost));
  s->nt_ionized = s->nt_near = s->nt_particle_steps = 0;
  for (int sp = 0; sp < 3; ++sp) {
    if (sp == 2) {
      if (ver != 4) break;
      get(&q, &nn, 8);
      get(&q, s->nt_recycled, 16);
      get(&q, s->nt_lost, 16);
      get(&q, &s->nt_ionized, 8);
      get(&q, &s->nt_near, 8);
    }
    orc_species* p = sp == 2 ? &s->nt : &s->sp[sp];
    const size_t ns = sp == 2 ? (size_t)nn : (size_t)n[sp];
    if (sp_reserve(p, ns) != ORC_OK) return ORC_ENOMEM;
    const unsigned char* cell = q;
    const unsigned char* frac = cell + 4 * ns;
    const unsigned char* vx = frac + 8 * ns;
    const unsigned char* vy = vx + 8 * ns;
    const unsigned char* vz = vy + 8 * ns;
    const unsigned char* id = vz + 8 * ns;
    for (size_t i = 0; i < ns; ++i) {
      uint32_t cw;
      double f;
      memcpy(&cw, cell + 4 * i, 4);
      memcpy(&f, frac + 8 * i, 8);
      const int32_t cc = (int32_t)(cw & ((1u << CELL_BITS) - 1u));
      uint32_t nk = cw >> CELL_BITS;
      if (cc >= s->N || !(f >= 0.0 && f < 1.0)) return ORC_ECORRUPT;
      if (sp < 2 && s->mcc[sp]) { /* R17: a valid countdown pair, or 0 = not drawn */
        if (nk > (NEXT_CAND | NEXT_KMAX)) return ORC_ECORRUPT;
        memcpy(&p->id[i], id + 8 * i, 8);
        if (nk == 0u) nk = creation_next(s, sp, p->id[i], step);
        if ((nk & NEXT_KMAX) == 0u) return ORC_ECORRUPT;
      } else if (nk != 0u) {
        return ORC_ECORRUPT; /* no countdown for species without the null-collision test */
      }
      p->nk[i] = nk;
      p->x[i] = (double)cc + f;
      if (p->x[i] >= (double)cc + 1.0) p->x[i] = nextafter((double)cc + 1.0, 0.0);
      memcpy(&p->vx[i], vx + 8 * i, 8);
      memcpy(&p->vy[i], vy + 8 * i, 8);
      memcpy(&p->vz[i], vz + 8 * i, 8);
      memcpy(&p->id[i], id + 8 * i, 8);
    }
    p->n = ns;
    q = id + 8 * ns;
  }
  for (int sp = 0; sp < 2; ++sp) sort_species(&s->sp[sp], s->N);
  sort_species(&s->nt, s->N);
  deposit_and_solve(s);
  return ORC_OK;
}
